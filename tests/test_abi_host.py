"""Host-side checks of the C-ABI library: it loads, exports every declared symbol, and
its host-only scheduling logic follows Algorithm 3 (hand-worked fixtures and the
oracle) and covers every entry exactly once.  No GPU is used."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1410_5209_gb300 as tf
from tests import golden


@pytest.fixture(scope="module")
def lib():
    try:
        return tf.load()
    except tf.LibraryMissing:
        from paper_1410_5209_gb300 import build
        build.build()
        return tf.load()


def test_library_exports_every_declared_symbol(lib):
    names = tf.declared_symbols()
    assert len(names) >= 19
    for n in names:
        assert hasattr(lib, n), n
        # and the binding declares its argument types (no default ctypes conversions)
        assert getattr(lib, n).argtypes is not None, n
    assert tf.version().startswith("sals-gb300")


def test_create_rejects_bad_arguments_without_gpu(lib):
    """Argument checks happen before any CUDA call."""
    out = ctypes.c_void_p()
    dims = np.array([3, 3], np.int64)
    c = np.zeros((1, 2), np.int32)
    v = np.zeros(1, np.float32)
    P = ctypes.c_void_p
    st = lib.tf_create(P(c.ctypes.data), P(v.ctypes.data), 0, P(dims.ctypes.data), 0, 1, 4,
                       ctypes.c_uint64(0), None, 0, ctypes.byref(out))
    assert st == tf.EINVAL and not out.value
    st = lib.tf_create(P(c.ctypes.data), P(v.ctypes.data), 0, P(dims.ctypes.data), 2, 1, 0,
                       ctypes.c_uint64(0), None, 0, ctypes.byref(out))
    assert st == tf.EINVAL
    bad = np.array([3, 0], np.int64)
    st = lib.tf_create(P(c.ctypes.data), P(v.ctypes.data), 0, P(bad.ctypes.data), 2, 1, 4,
                       ctypes.c_uint64(0), None, 0, ctypes.byref(out))
    assert st == tf.EINVAL
    assert b"mode lengths" in lib.tf_last_error(None)
    assert lib.tf_sals_sweep(None, 1, 0.1, 1) == tf.EINVAL
    assert lib.tf_loss(None, 0.1, 0, None, None) == tf.EINVAL


def test_greedy_policy_matches_algorithm3_hand_cases(lib):
    for case in golden.alg3_cases():
        dims = [len(m) for m in case["modes"]]
        got = tf.assign_rows(tf.SCHED_GREEDY, dims, case["modes"], case["M"])
        for g, e in zip(got, case["expect"]):
            assert list(g) == e, case["name"]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_greedy_policy_matches_oracle_algorithm3(lib, seed):
    rng = np.random.default_rng(seed)
    dims = [int(rng.integers(20, 300)) for _ in range(3)]
    nnz = 2000
    row_nnz = []
    for d in dims:
        w = rng.zipf(1.3, d).astype(np.float64)
        cnt = np.floor(w / w.sum() * nnz).astype(np.int64)
        cnt[0] += nnz - cnt.sum()
        row_nnz.append(cnt)
    M = int(rng.integers(2, 17))
    ours = tf.assign_rows(tf.SCHED_GREEDY, dims, row_nnz, M)
    ref = oracle.greedy_assign(dims, row_nnz, M)
    for a, b in zip(ours, ref):
        assert np.array_equal(a, b)


def test_seq_policy_is_contiguous_ranges(lib):
    # Section 5.5 footnote, 1-based: I(m-1)/M < i <= I m / M; for I = 10, M = 3 the
    # machines get rows {1,2,3}, {4,5,6}, {7,8,9,10}.
    a = tf.assign_rows(tf.SCHED_SEQ, [10], [np.ones(10, np.int64)], 3)[0]
    assert list(a) == [0, 0, 0, 1, 1, 1, 2, 2, 2, 2]


def _offsets(lengths):
    return np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)


@pytest.mark.parametrize("policy", [tf.SCHED_LPT, tf.SCHED_GREEDY, tf.SCHED_SEQ, tf.SCHED_RAN])
def test_plan_covers_every_entry_once(lib, policy):
    rng = np.random.default_rng(7)
    lengths = np.concatenate([rng.zipf(1.2, 500).clip(max=20000), np.zeros(7, np.int64)])
    rng.shuffle(lengths)
    off = _offsets(lengths)
    P = 37
    items, n_slots, bin_ptr = tf.plan_mode(off, P, 0, policy)
    cover = np.zeros(off[-1], np.int32)
    rows_seen = set()
    for it in items:
        cover[it["begin"]:it["begin"] + it["len"]] += 1
        r = it["row"]
        assert off[r] <= it["begin"] and it["begin"] + it["len"] <= off[r + 1]
        rows_seen.add(int(r))
    assert np.all(cover == 1)
    assert rows_seen == set(range(len(lengths)))        # empty rows are items too
    assert bin_ptr[0] == 0 and bin_ptr[-1] == len(items)
    for b in range(P):
        assert np.all(items["bin"][bin_ptr[b]:bin_ptr[b + 1]] == b)
    assert n_slots == len(items)
    assert sorted(items["slot"]) == list(range(len(items)))
    if policy != tf.SCHED_LPT:   # whole rows only
        assert len(items) == len(lengths)


def test_lpt_splits_heavy_rows_and_balances(lib):
    rng = np.random.default_rng(8)
    lengths = np.concatenate([rng.zipf(1.1, 3000).clip(max=10 ** 4), [400_000, 90_000]])
    off = _offsets(lengths)
    P = 64
    items, n_slots, bin_ptr = tf.plan_mode(off, P, 0, tf.SCHED_LPT)
    nnz = int(off[-1])
    cap = -(-nnz // P)
    assert items["len"].max() <= cap
    # chunks of a split row take consecutive slots in entry order
    rows, counts = np.unique(items["row"], return_counts=True)
    split = rows[counts > 1]
    assert len(split) > 0 and n_slots == len(items)
    chunks = items[np.isin(items["row"], split)]
    for r in split:
        c = np.sort(chunks[chunks["row"] == r], order="slot")
        assert np.all(np.diff(c["slot"]) == 1)
        assert np.all(c["begin"][1:] == c["begin"][:-1] + c["len"][:-1])
        assert c["begin"][0] == off[r] and c["begin"][-1] + c["len"][-1] == off[r + 1]
    loads = np.array([items["len"][bin_ptr[b]:bin_ptr[b + 1]].sum() for b in range(P)])
    # Graham's bound for longest-processing-time list scheduling
    assert loads.max() <= nnz / P + cap
    assert loads.max() <= 1.05 * nnz / P + 1


def test_plan_handles_empty_mode(lib):
    items, n_slots, bin_ptr = tf.plan_mode(np.zeros(4, np.int64), 8, 0, tf.SCHED_LPT)
    assert len(items) == 3 and np.all(items["len"] == 0) and n_slots == 3


def test_pool_trim_rejects_negative_without_gpu(lib):
    assert lib.tf_pool_trim(-1) == tf.EINVAL


def test_lpt_spreads_short_and_empty_rows(lib):
    """Many empty and one-entry rows beside a few long ones (a batch of small tensors):
    LPT balances the items per bin as well as the entries, so no warp is left with
    thousands of tiny items after the others finish."""
    rng = np.random.default_rng(5)
    cnt = np.concatenate([np.zeros(20_000, np.int64), np.ones(20_000, np.int64),
                          rng.integers(2, 200, 20_000), rng.integers(1_000, 50_000, 200)])
    rng.shuffle(cnt)
    off = np.zeros(len(cnt) + 1, np.int64)
    off[1:] = np.cumsum(cnt)
    P = 2048
    items, n_slots, bin_ptr = tf.plan_mode(off, P)
    per_bin = np.diff(bin_ptr)
    assert per_bin.max() <= 4 * per_bin.mean() + 8, (per_bin.max(), per_bin.mean())
    loads = np.zeros(P)
    np.add.at(loads, items["bin"], items["len"])
    assert loads.max() <= 1.1 * loads.mean() + 100
