"""tf_loss_noalloc -- the loss of tf_loss computed with a fixed, library-owned device
array as its scratch instead of memory the context allocates -- checked through the C
ABI against tf_loss on the same state.

The loss tolerance of the other device tests applies (1e-9 relative); the two entry
points run the same kernels in the same order, so in practice they agree exactly.
This file is collected last so that it also runs after everything else has used the
device; it needs nothing from the other test files and passes on its own."""
import numpy as np
import pytest

import paper_1410_5209_gb300 as tf
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1410_5209_gb300 import build
    build.build()


def close(got, ref):
    return all(abs(g - r) <= TOL * abs(r) for g, r in zip(got, ref))


def noalloc_checked(f, lam, weighted=False):
    """tf_loss_noalloc, checked to leave the library's device pool exactly as it found
    it: bytes in use, high-water mark (reset just before) and bytes held unchanged."""
    tf.pool_usage(reset_high=True)
    before = tf.pool_usage()
    got = f.loss_noalloc(lam, weighted)
    after = tf.pool_usage()
    assert after == before, (before, after)
    return got


def factorization(p, dtype):
    c, x = p.numpy()
    return tf.Factorization(c, x, p.dims, p.K, seed=p.seed, dtype=dtype)


@pytest.mark.parametrize("dtype", [tf.F64, tf.F32])
@pytest.mark.parametrize("weighted", [False, True])
def test_noalloc_loss_matches_tf_loss(dtype, weighted):
    """Two calls in a row (a sweep between them, so the second call finds the first
    call's partial sums in the array), each against tf_loss.  The first call comes
    before tf_loss has ever allocated its buffer on this context."""
    p = synth.small(41, (300, 200, 50), 30_000, 3, 8)
    f = factorization(p, dtype)
    for call in range(2):
        f.sweep(4, 0.3, 1, p.column_order(call, 4), weighted=weighted)
        got = noalloc_checked(f, 0.3, weighted)
        ref = f.loss(0.3, weighted)
        assert close(got, ref), (call, got, ref)
        assert got[1] > 0


def test_noalloc_loss_wide_subsets():
    """After a sweep with C > 16 the loss reduction runs the wide residual kernel; its block
    partials also fit the static array."""
    p = synth.small(45, (300, 200, 50), 30_000, 3, 40)
    f = factorization(p, tf.F32)
    for call in range(2):
        f.sweep(20, 0.3, 1, p.column_order(call, 20))
        assert close(noalloc_checked(f, 0.3), f.loss(0.3))


def test_noalloc_loss_across_contexts():
    """Contexts of different shapes (N = 4, then N = 3, other block counts) share the
    array; stale partial sums of the larger reduction never reach the smaller one."""
    p4 = synth.small(42, (120, 90, 60, 30), 25_000, 2, 6)
    p3 = synth.small(43, (500, 40, 30), 4_000, 2, 5)
    f4, f3 = factorization(p4, tf.F64), factorization(p3, tf.F64)
    f4.sweep(2, 0.1, 1, p4.column_order(0, 2))
    f3.sweep(1, 0.1, 1, p3.column_order(0, 1))
    for _ in range(2):
        for f in (f4, f3):
            got = noalloc_checked(f, 0.1)
            assert close(got, f.loss(0.1)), got


def test_noalloc_loss_default_schedule_large_tensor():
    """At the default schedule of a large tensor (1.4e6 entries: 128 bins per SM) the
    FP64 C = 10 residual kernel runs one warp per block, so its block partials number
    the bins; they still fit the array, and two calls in a row match tf_loss."""
    p = synth.small(46, (2000, 1500, 120), 1_400_000, 5, 10)
    f = factorization(p, tf.F64)
    for call in range(2):
        f.sweep(10, 0.2, 1, p.column_order(call, 10))
        got = noalloc_checked(f, 0.2)
        assert close(got, f.loss(0.2)), (call, got)


def test_noalloc_loss_rejects_oversized_reduction():
    """A schedule with far more bins than the array has room for partial sums is
    refused with TF_EINVAL before anything is launched; tf_loss still works and the
    context stays usable."""
    p = synth.small(44, (300, 200, 50), 30_000, 3, 4)
    f = factorization(p, tf.F64)
    f.sweep(2, 0.2, 1, p.column_order(0, 2))
    ref = f.loss(0.2)
    f.set_schedule(tf.SCHED_LPT, 200_000)
    with pytest.raises(tf.TFError) as e:
        f.loss_noalloc(0.2)
    assert e.value.status == tf.EINVAL
    assert "scratch" in str(e.value)
    assert close(f.loss(0.2), ref)
    f.set_schedule(tf.SCHED_LPT, 0)
    assert close(noalloc_checked(f, 0.2), ref)
