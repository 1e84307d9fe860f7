"""Many small independent tensors factorised as one block-diagonal tensor.

Rows of a mode are independent given the other modes (Section 3.3), and no entry of a
block-diagonal concatenation couples two tensors, so one sweep over the concatenation
is the same computation as one sweep over each tensor (same column order): this is how
a batch of tensors runs in one set of launches."""
import numpy as np
import pytest

import oracle
import paper_1410_5209_gb300 as tf
import synth


def _problems():
    return [synth.small(100 + b, dims, nnz, 3, 8)
            for b, (dims, nnz) in enumerate([((40, 30, 20), 3_000), ((25, 60, 11), 2_500),
                                              ((70, 9, 33), 4_000)])]


def _split(A, row_off, b):
    return [np.array(A[n][row_off[b, n]:row_off[b + 1, n]], copy=True) for n in range(3)]


def test_block_diagonal_oracle_equals_independent_tensors():
    probs = _problems()
    p, row_off, ent_off = synth.concat_block_diagonal(probs, 8, seed=7)
    c, x = p.numpy()
    t = oracle.Tensor(c, x, p.dims)
    A = [a.numpy() for a in p.init_factors()]
    parts = [_split(A, row_off, b) for b in range(len(probs))]
    tb = [oracle.Tensor(*q.numpy(), q.dims) for q in probs]
    r = oracle.residual(t, A)
    rb = [oracle.residual(tb[b], parts[b]) for b in range(len(probs))]
    for s in range(2):
        order = p.column_order(s, 4)
        oracle.sals_sweep(t, A, r, 4, 0.3, 1, order)
        for b in range(len(probs)):
            oracle.sals_sweep(tb[b], parts[b], rb[b], 4, 0.3, 1, order)
    for b in range(len(probs)):
        for n in range(3):
            got = A[n][row_off[b, n]:row_off[b + 1, n]]
            assert np.max(np.abs(got - parts[b][n])) <= 1e-12 * max(1.0, np.max(np.abs(got)))
        assert np.allclose(r[ent_off[b]:ent_off[b + 1]], rb[b], rtol=0, atol=1e-12)


@pytest.mark.gpu
def test_block_diagonal_batch_on_device():
    from paper_1410_5209_gb300 import build
    build.build()
    probs = _problems()
    p, row_off, ent_off = synth.concat_block_diagonal(probs, 8, seed=7)
    c, x = p.numpy()
    A = [a.numpy() for a in p.init_factors()]
    f = tf.Factorization(c, x, p.dims, 8, dtype=tf.F64)
    for n in range(3):
        f.set_factors(n, A[n])
    parts = [_split(A, row_off, b) for b in range(len(probs))]
    tb = [oracle.Tensor(*q.numpy(), q.dims) for q in probs]
    rb = [oracle.residual(tb[b], parts[b]) for b in range(len(probs))]
    for s in range(2):
        order = p.column_order(s, 4)
        f.sweep(4, 0.3, 1, order)
        for b in range(len(probs)):
            oracle.sals_sweep(tb[b], parts[b], rb[b], 4, 0.3, 1, order)
    for n in range(3):
        got = f.factors(n)
        for b in range(len(probs)):
            seg = got[row_off[b, n]:row_off[b + 1, n]]
            assert np.linalg.norm(seg - parts[b][n]) <= 1e-9 * max(np.linalg.norm(parts[b][n]), 1e-300)
    res = f.residual()
    for b in range(len(probs)):
        assert np.linalg.norm(res[ent_off[b]:ent_off[b + 1]] - rb[b]) <= 1e-9 * np.linalg.norm(rb[b])
