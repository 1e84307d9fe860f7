"""GPU <-> oracle parity through the C ABI.

Tolerances (stated by the task for this method): sorting, offsets and permutations
bit-exact; a row update from identical inputs within 1e-5 relative in FP32; training
RMSE after a fixed number of sweeps within 1e-3 relative.  The FP64 device path is
held to 1e-9 (only summation order differs from the oracle)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1410_5209_gb300 as tf
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1410_5209_gb300 import build
    build.build()


def make(p, dtype=tf.F64):
    """Device context and oracle inputs holding exactly the same numbers (for the FP32
    path the values and initial factors are rounded to float32 on both sides)."""
    c, x = p.numpy()
    A = [a.numpy().astype(np.float64) for a in p.init_factors()]
    if dtype == tf.F32:
        x = x.astype(np.float32).astype(np.float64)
        A = [a.astype(np.float32).astype(np.float64) for a in A]
    f = tf.Factorization(c, x, p.dims, p.K, seed=p.seed, dtype=dtype)
    for n in range(p.N):
        f.set_factors(n, A[n])
    return f, oracle.Tensor(c, x, p.dims), A


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def ragged_problem(seed=21):
    # several tiles of the radix sort (4096 keys), ragged tail, mode lengths that are
    # not powers of two, a mode with many empty rows
    return synth.small(seed, (301, 157, 1000), 9_973, 4, 6)


# --------------------------------------------------------------------------- layout


@pytest.mark.parametrize("field_sorts", [False, True])
@pytest.mark.parametrize("prob", ["parity", "ragged", "skew"])
def test_grouping_bit_exact(prob, field_sorts):
    """Both layout builds (packed keys, per-mode sorts of gathered coordinates) against
    the oracle's grouping."""
    if prob == "parity":
        p = synth.parity_3way()
    elif prob == "ragged":
        p = ragged_problem()
    else:
        p = synth.small(5, (2000, 3000, 50), 60_000, 3, 4, modes=["zipf", "zipf", "uniform"])
    c, x = p.numpy()
    f = tf.Factorization(c, x, p.dims, p.K, seed=p.seed, dtype=tf.F64, field_sorts=field_sorts)
    t = oracle.Tensor(c, x, p.dims)
    for n in range(p.N):
        off, perm = f.grouping(n)
        ooff, operm = oracle.group(t, n)
        assert np.array_equal(off, ooff)
        assert np.array_equal(perm, operm)


@pytest.mark.parametrize("dims,nnz,modes", [
    # a mode longer than the packing pass's shared count table (8192 rows) with uniform
    # rows, so a block's table overflows into direct global counts
    ((100_000, 50, 60), 300_000, ["uniform", "uniform", "uniform"]),
    # coordinates filling 63 of the key's 64 bits
    ((1 << 21, 1 << 21, 1 << 21), 40_000, ["uniform", "uniform", "uniform"]),
    # two modes of one row (no bits in the key) around a third
    ((1, 7000, 1), 6_000, ["uniform", "uniform", "uniform"]),
    # four-way with 66 bits of coordinates: the per-mode sorts apply by themselves
    ((1 << 20, 1 << 20, 1 << 20, 33), 30_000, ["uniform", "zipf", "uniform", "uniform"]),
])
def test_layout_extremes_bit_exact(dims, nnz, modes):
    p = synth.small(61, dims, nnz, 2, 3, modes=modes)
    c, x = p.numpy()
    t = oracle.Tensor(c, x, p.dims)
    f = tf.Factorization(c, x, p.dims, p.K, seed=1, dtype=tf.F64)
    for n in range(p.N):
        off, perm = f.grouping(n)
        ooff, operm = oracle.group(t, n)
        assert np.array_equal(off, ooff), n
        assert np.array_equal(perm, operm), n
    assert np.array_equal(f.residual(), x)


def test_layout_builds_give_identical_sweeps():
    """The packed-key and the per-mode-sort builds give the same layout, so the same
    sweeps bit for bit (FP32, default schedule, several tiles of every sort)."""
    p = synth.small(62, (3000, 2500, 80), 250_000, 4, 10, modes=["zipf", "zipf", "uniform"])
    c, x = p.numpy()
    out = []
    for field_sorts in (False, True):
        f = tf.Factorization(c, x, p.dims, p.K, seed=9, dtype=tf.F32, field_sorts=field_sorts)
        for s in range(2):
            f.sweep(5, 0.1, 1, p.column_order(s, 5))
        out.append(([f.factors(n) for n in range(p.N)], f.residual(), f.loss(0.1)))
        f.close()
    for a, b in zip(out[0][0], out[1][0]):
        assert np.array_equal(a, b)
    assert np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]


@pytest.mark.parametrize("field_sorts", [False, True])
def test_create_errors_across_tiles(field_sorts):
    """A duplicate pair thousands of entries apart and a coordinate out of range at the
    last entry, on inputs spanning several tiles of the packing and sorting passes."""
    p = synth.small(63, (500, 400, 90), 20_000, 2, 3)
    c, x = p.numpy()
    d = c.copy()
    d[17_003] = d[5]
    with pytest.raises(tf.TFError) as e:
        tf.Factorization(d, x, p.dims, 3, dtype=tf.F32, field_sorts=field_sorts)
    assert e.value.status == tf.EDUP
    r = c.copy()
    r[-1, 2] = 90
    with pytest.raises(tf.TFError) as e:
        tf.Factorization(r, x, p.dims, 3, dtype=tf.F32, field_sorts=field_sorts)
    assert e.value.status == tf.ERANGE
    r[-1, 2] = -1
    with pytest.raises(tf.TFError) as e:
        tf.Factorization(r, x, p.dims, 3, dtype=tf.F32, field_sorts=field_sorts)
    assert e.value.status == tf.ERANGE
    f = tf.Factorization(c, x, p.dims, 3, dtype=tf.F32, field_sorts=field_sorts)
    assert np.array_equal(f.residual(), x.astype(np.float32))


def test_create_validates_coordinates():
    c = np.array([[0, 0, 0], [1, 2, 0]], np.int32)
    with pytest.raises(tf.TFError) as e:
        tf.Factorization(c, np.ones(2), [2, 2, 1], 2, dtype=tf.F64)
    assert e.value.status == tf.ERANGE
    c = np.array([[0, 1, 0], [1, 1, 0], [0, 1, 0]], np.int32)
    with pytest.raises(tf.TFError) as e:
        tf.Factorization(c, np.ones(3), [2, 2, 1], 2, dtype=tf.F64)
    assert e.value.status == tf.EDUP


def test_init_residual_is_x():
    """Algorithm 1 initialisation (A^(1) = 0) gives R = X exactly."""
    p = synth.parity_3way()
    c, x = p.numpy()
    f = tf.Factorization(c, x, p.dims, p.K, seed=3, dtype=tf.F64)
    assert np.all(f.factors(0) == 0)
    assert np.array_equal(f.residual(), x)
    L, rmse = f.loss(1.0)
    A = [f.factors(n) for n in range(3)]
    assert np.isclose(L, x @ x + sum((a * a).sum() for a in A), rtol=1e-12)


# --------------------------------------------------------------------------- sweeps


@pytest.mark.parametrize("C", [1, 5])
def test_fp64_sweeps_match_oracle(C):
    """FP64 device path vs FP64 oracle, 5 sweeps of the parity workload."""
    p = synth.parity_3way()
    f, t, A = make(p, tf.F64)
    r = oracle.residual(t, A)
    for s in range(5):
        order = p.column_order(s, C)
        f.sweep(C, 1.0, 1, order)
        oracle.sals_sweep(t, A, r, C, 1.0, 1, order)
    for n in range(3):
        assert rel(f.factors(n), A[n]) < 1e-9
    assert rel(f.residual(), r) < 1e-9
    L, rmse = f.loss(1.0)
    Lo, rmseo = oracle.loss(t, r, A, 1.0)
    assert abs(L - Lo) <= 1e-9 * Lo and abs(rmse - rmseo) <= 1e-9 * rmseo


@pytest.mark.parametrize("C", [1, 5])
def test_fp32_rmse_after_five_sweeps(C):
    """FP32 device path vs FP64 oracle: training RMSE after 5 sweeps within 1e-3."""
    p = synth.parity_3way()
    f, t, A = make(p, tf.F32)
    r = oracle.residual(t, A)
    for s in range(5):
        order = p.column_order(s, C)
        f.sweep(C, 1.0, 1, order)
        oracle.sals_sweep(t, A, r, C, 1.0, 1, order)
    _, rmse = f.loss(1.0)
    _, rmseo = oracle.loss(t, r, A, 1.0)
    assert abs(rmse - rmseo) <= 1e-3 * rmseo


def fp32_row_bound(t, n, i, A_in, S, rhat, lam, a):
    """A-priori forward-error bound of one FP32 row solve (Eq. 4): with u = 2^-24 and
    gamma = (log2(m) + 16) u covering the products forming h and r_hat*h and the tree
    sums, |dc| <= gamma |Phi|^T |r_hat|, |dB| <= gamma |Phi|^T |Phi|, and
    ||da|| <= ||(B + lam I)^-1||_2 (||dc|| + ||dB|| ||a||) (plus Cholesky rounding)."""
    sel = np.nonzero(t.coords[:, n] == i)[0]
    Phi = np.ones((len(sel), len(S)))
    for l in range(t.N):
        if l != n:
            Phi *= A_in[l][t.coords[sel, l]][:, S]
    m = max(len(sel), 1)
    gamma = (np.ceil(np.log2(m)) + 16) * 2.0 ** -24
    B = Phi.T @ Phi + lam * np.eye(len(S))
    inv = np.linalg.norm(np.linalg.inv(B), 2)
    dc = gamma * np.linalg.norm(np.abs(Phi).T @ np.abs(rhat[sel]))
    dB = gamma * np.linalg.norm(np.abs(Phi).T @ np.abs(Phi), 2) + 8 * len(S) * 2.0 ** -24 * \
        np.linalg.norm(B, 2)
    return 2.0 * inv * (dc + dB * np.linalg.norm(a))


@pytest.mark.parametrize("C", [1, 5, 10])
def test_fp32_row_update_from_identical_inputs(C):
    """The first split's mode-1 rows are computed from identical inputs on both sides
    (A^(2), A^(3) as given, R-hat = X) and are not touched again during the sweep.
    FP32 reading of "relative error <= 1e-5": normwise over the split's updated rows,
    and per row within 1e-5 relative or within the row's FP32 forward-error bound
    (rows whose rhs cancels heavily cannot be closer in FP32)."""
    p = synth.parity_3way()
    f, t, A = make(p, tf.F32)
    A_in = [a.copy() for a in A]
    r = oracle.residual(t, A)
    order = p.column_order(0, C)
    f.sweep(C, 1.0, 1, order)
    oracle.sals_sweep(t, A, r, C, 1.0, 1, order)
    S = order[:C]
    g = f.factors(0)[:, S].astype(np.float64)
    o = A[0][:, S]
    assert rel(g, o) <= 1e-5
    num = np.linalg.norm(g - o, axis=1)
    den = np.linalg.norm(o, axis=1)
    for i in np.nonzero(num > 1e-5 * den)[0]:
        assert num[i] <= fp32_row_bound(t, 0, i, A_in, S, t.x, 1.0, o[i]), i


@pytest.mark.parametrize("C,K,path", [(20, 40, "simt"), (50, 60, "simt"), (70, 100, "tc"),
                                      (100, 100, "tc")])
def test_fp32_wide_row_update_from_identical_inputs(C, K, path):
    """The same single-row-update check on the wide passes: the block-tiled SIMT Gram
    (C = 20, 50) and the tensor-core Gram (three TF32 products per term, C = 70 and the
    ALS form C = K = 100).  The first split's mode-1 rows see identical inputs on both
    sides (R-hat = X); normwise within 1e-5, per row within 1e-5 or the row's FP32
    forward-error bound."""
    p = synth.small(150 + C, (400, 230, 90), 30_000, 6, K)
    f, t, A = make(p, tf.F32)
    f.set_kernel_path(tf.Factorization.PATH_TMA if path == "tc" else tf.Factorization.PATH_SIMT)
    A_in = [a.copy() for a in A]
    r = oracle.residual(t, A)
    order = p.column_order(0, C)
    f.sweep(C, 0.5, 1, order)
    oracle.sals_sweep(t, A, r, C, 0.5, 1, order)
    assert bool(f.counters()["pass_path"] & 4) == (path == "tc")
    S = order[:C]
    g = f.factors(0)[:, S].astype(np.float64)
    o = A[0][:, S]
    assert rel(g, o) <= 1e-5
    num = np.linalg.norm(g - o, axis=1)
    den = np.linalg.norm(o, axis=1)
    for i in np.nonzero(num > 1e-5 * den)[0]:
        assert num[i] <= fp32_row_bound(t, 0, i, A_in, S, t.x, 0.5, o[i]), i


def test_ragged_T_in_and_uneven_split():
    """C not dividing K (last split smaller), T_in = 2, mode with empty rows."""
    p = ragged_problem()
    f, t, A = make(p, tf.F64)
    r = oracle.residual(t, A)
    for s in range(2):
        order = p.column_order(s, 4)
        f.sweep(4, 0.3, 2, order)
        oracle.sals_sweep(t, A, r, 4, 0.3, 2, order)
    for n in range(3):
        assert rel(f.factors(n), A[n]) < 1e-9
    assert rel(f.residual(), r) < 1e-9


def test_weighted_lambda_matches_oracle():
    p = ragged_problem(22)
    f, t, A = make(p, tf.F64)
    r = oracle.residual(t, A)
    order = p.column_order(0, 3)
    f.sweep(3, 0.05, 1, order, weighted=True)
    oracle.sals_sweep(t, A, r, 3, 0.05, 1, order, weighted=True)
    for n in range(3):
        assert rel(f.factors(n), A[n]) < 1e-9
    L, _ = f.loss(0.05, weighted=True)
    Lo, _ = oracle.loss(t, r, A, 0.05, weighted=True)
    assert abs(L - Lo) <= 1e-9 * Lo


def test_residual_invariant_fp32():
    """The stored residual equals x - model recomputed from the device's own factors."""
    p = synth.parity_3way()
    f, t, _ = make(p, tf.F32)
    for s in range(3):
        f.sweep(5, 1.0, 1, p.column_order(s, 5))
    A = [f.factors(n).astype(np.float64) for n in range(3)]
    model = np.ones((t.nnz, p.K))
    for n in range(3):
        model *= A[n][t.coords[:, n]]
    ref = t.x - model.sum(1)
    assert np.max(np.abs(f.residual() - ref)) <= 1e-5 * np.max(np.abs(t.x))


@pytest.mark.parametrize("C", [1, 4])
def test_loss_never_increases_fp64(C):
    """Theorem 1 on the device: every split is an exact block minimisation."""
    p = synth.small(31, (200, 150, 40), 20_000, 3, 8)
    f, t, _ = make(p, tf.F64)
    prev = f.loss(0.5)[0]
    for s in range(4):
        f.sweep(C, 0.5, 1, p.column_order(s, C))
        cur = f.loss(0.5)[0]
        assert cur <= prev * (1 + 1e-12)
        prev = cur


def test_singular_rows_left_unchanged():
    """lambda = 0 with empty rows: pivot 0, row unchanged and counted (both sides)."""
    p = synth.small(32, (500, 40, 30), 1_500, 2, 3)   # many empty rows in mode 1
    f, t, A = make(p, tf.F64)
    r = oracle.residual(t, A)
    bad_o = oracle.sals_sweep(t, A, r, 1, 0.0, 1, np.arange(3))
    f.sweep(1, 0.0, 1, np.arange(3, dtype=np.int32))
    assert f.counters()["singular_rows"] == bad_o > 0
    for n in range(3):
        assert rel(f.factors(n), A[n]) < 1e-8


def test_schedule_does_not_change_results():
    """Rows are independent (Section 3.3): re-binning without changing the chunking is
    bit-identical; other chunkings agree to rounding."""
    p = synth.small(33, (300, 400, 20), 40_000, 3, 6, modes=["zipf", "zipf", "uniform"])
    outs = []
    for policy, P in [(tf.SCHED_LPT, 0), (tf.SCHED_LPT, 300), (tf.SCHED_SEQ, 50),
                      (tf.SCHED_RAN, 50), (tf.SCHED_GREEDY, 64)]:
        f, t, A = make(p, tf.F64)
        f.set_schedule(policy, P)
        if policy == tf.SCHED_LPT and P == 300:   # cap = nnz / 300: mode-3 rows split
            assert f.counters()["split_rows"] > 0
        for s in range(2):
            f.sweep(3, 0.2, 1, p.column_order(s, 3))
        outs.append([f.factors(n) for n in range(3)])
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert rel(a, b) < 1e-10
    # same chunking, different bins -> bit-identical
    f1, _, _ = make(p, tf.F64)
    f2, _, _ = make(p, tf.F64)
    f1.set_schedule(tf.SCHED_SEQ, 50)
    f2.set_schedule(tf.SCHED_RAN, 50)
    for f in (f1, f2):
        f.sweep(3, 0.2, 1, p.column_order(0, 3))
    for n in range(3):
        assert np.array_equal(f1.factors(n), f2.factors(n))


@pytest.mark.parametrize("C", [6, 8, 10])
def test_tma_and_simt_paths_bit_identical(C):
    """The TMA-fed pass (tile::gather4 rows, bulk index windows) and the cp.async pass
    perform the same arithmetic in the same order: identical bits."""
    p = synth.small(51, (3000, 2000, 300), 200_000, 4, 20, modes=["zipf", "zipf", "uniform"])
    out = []
    for path in (tf.Factorization.PATH_SIMT, tf.Factorization.PATH_TMA):
        f, _, _ = make(p, tf.F32)
        f.set_kernel_path(path)
        for s in range(2):
            f.sweep(C, 0.1, 1 if s == 0 else 2, p.column_order(s, C))
        out.append([f.factors(n) for n in range(3)] + [f.residual(), np.array(f.loss(0.1))])
    for a, b in zip(*out):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("C", [2, 4, 5, 8, 10, 12])
def test_lean_pass_matches_oracle_and_cp_async_pass(C):
    """The lean float pass (default for three-way float tensors, C <= 12) against the FP64
    oracle and against the cp.async pass: two sweeps (T_in = 1, then T_in = 2, so both
    the refreshing and the plain inner iterations run), Zipf-skewed rows so that runs of
    equal indices, hot cached rows and cold staged rows all occur."""
    p = synth.small(60 + C, (900, 700, 60), 120_000, 4, 24, modes=["zipf", "zipf", "uniform"])
    f, t, A = make(p, tf.F32)
    g, _, _ = make(p, tf.F32)
    g.set_kernel_path(tf.Factorization.PATH_SIMT)
    r = oracle.residual(t, A)
    for s in range(2):
        order = p.column_order(s, C)
        f.sweep(C, 0.2, 1 + s, order)
        g.sweep(C, 0.2, 1 + s, order)
        oracle.sals_sweep(t, A, r, C, 0.2, 1 + s, order)
    assert f.counters()["pass_path"] & 8 and not g.counters()["pass_path"] & 8
    for n in range(3):
        assert rel(f.factors(n).astype(np.float64), A[n]) < 2e-4, n
        assert rel(f.factors(n), g.factors(n)) < 2e-4, n
    assert rel(f.residual().astype(np.float64), r) < 2e-4
    _, rmse = f.loss(0.2)
    _, rmseo = oracle.loss(t, r, A, 0.2)
    assert abs(rmse - rmseo) <= 1e-4 * rmseo


@pytest.mark.parametrize("C", [2, 5, 10, 12])
def test_lean_tensor_core_gram_fp32_level(C):
    """The lean pass with its Gram on the tensor cores (path 4: three TF32 products per
    term, FP32 accumulation) against the FP64 oracle and the packed-FMA lean pass: the first
    split's mode-1 rows within 1e-5 (or their FP32 forward-error bound), and two sweeps
    (T_in = 1 then 2) within FP32-level error."""
    p = synth.small(80 + C, (900, 700, 60), 120_000, 4, 24, modes=["zipf", "zipf", "uniform"])
    f, t, A = make(p, tf.F32)
    f.set_kernel_path(4)
    g, _, _ = make(p, tf.F32)
    A_in = [a.copy() for a in A]
    r = oracle.residual(t, A)
    order = p.column_order(0, C)
    f.sweep(C, 0.2, 1, order)
    g.sweep(C, 0.2, 1, order)
    oracle.sals_sweep(t, A, r, C, 0.2, 1, order)
    S = order[:C]
    got, ref = f.factors(0)[:, S].astype(np.float64), A[0][:, S]
    assert rel(got, ref) <= 1e-5
    num, den = np.linalg.norm(got - ref, axis=1), np.linalg.norm(ref, axis=1)
    for i in np.nonzero(num > 1e-5 * den)[0]:
        assert num[i] <= fp32_row_bound(t, 0, i, A_in, S, t.x, 0.2, ref[i]), i
    order = p.column_order(1, C)
    f.sweep(C, 0.2, 2, order)
    g.sweep(C, 0.2, 2, order)
    oracle.sals_sweep(t, A, r, C, 0.2, 2, order)
    for n in range(3):
        assert rel(f.factors(n).astype(np.float64), A[n]) < 2e-4, n
        assert rel(f.factors(n), g.factors(n)) < 2e-4, n
    _, rmse = f.loss(0.2)
    _, rmseo = oracle.loss(t, r, A, 0.2)
    assert abs(rmse - rmseo) <= 1e-4 * rmseo


@pytest.mark.parametrize("C", [4, 10])
def test_lean_tf32_gram_precision_form(C):
    """The reduced-precision form (tf_set_precision(1): one TF32 product per Gram term on
    the tensor cores): its error against the FP64 oracle after three sweeps is stated by
    this test -- factors within 5e-2 normwise, training RMSE within 1e-3 -- and the run is
    deterministic."""
    p = synth.small(90 + C, (900, 700, 60), 120_000, 4, 20, modes=["zipf", "zipf", "uniform"])
    out = []
    for _ in range(2):
        f, t, A = make(p, tf.F32)
        f.set_precision(1)
        r = oracle.residual(t, A)
        for s in range(3):
            order = p.column_order(s, C)
            f.sweep(C, 0.3, 1, order)
            oracle.sals_sweep(t, A, r, C, 0.3, 1, order)
        out.append([f.factors(n) for n in range(3)])
        for n in range(3):
            assert rel(f.factors(n).astype(np.float64), A[n]) < 5e-2, n
        _, rmse = f.loss(0.3)
        _, rmseo = oracle.loss(t, r, A, 0.3)
        assert abs(rmse - rmseo) <= 1e-3 * rmseo
    for a, b in zip(*out):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("C", [4, 10])
def test_lean_bf16_rows_precision_form(C):
    """The bfloat16 form (tf_set_precision(2): the lean pass reads the varying mode's slice
    rows from bfloat16 copies, 8 significand bits; run-mode and own rows, products, sums
    and residuals stay FP32): its error against the FP64 oracle after three sweeps is stated
    by this test -- factors within 5e-2 normwise, training RMSE within 1e-3 -- the lean pass
    runs, and the run is deterministic and independent of where rows are staged (cache,
    pool, warps), including the inner iterations of T_in = 2."""
    p = synth.small(94 + C, (900, 700, 60), 120_000, 4, 20, modes=["zipf", "zipf", "uniform"])
    out = []
    for max_rows, pool, warps in ((-1, 32, 0), (-1, 32, 0), (0, 8, 5)):
        f, t, A = make(p, tf.F32)
        f.set_precision(2)
        f.set_kernel_path(tf.Factorization.PATH_LEAN)
        f.set_pass_cache(max_rows, pool, warps)
        r = oracle.residual(t, A)
        for s in range(3):
            order = p.column_order(s, C)
            f.sweep(C, 0.3, 1, order)
            oracle.sals_sweep(t, A, r, C, 0.3, 1, order)
        assert f.counters()["pass_path"] & 8
        for n in range(3):
            assert rel(f.factors(n).astype(np.float64), A[n]) < 5e-2, n
        _, rmse = f.loss(0.3)
        _, rmseo = oracle.loss(t, r, A, 0.3)
        assert abs(rmse - rmseo) <= 1e-3 * rmseo
        f.sweep(C, 0.3, 2, p.column_order(3, C))
        out.append([f.factors(n) for n in range(3)] + [f.residual()])
    for other in out[1:]:
        for a, b in zip(out[0], other):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("C", [4, 10])
def test_lean_bf16_both_rows_precision_form(C):
    """tf_set_precision(3): both other modes' slice rows from bfloat16 copies.  Its error
    against the FP64 oracle after three sweeps on this low-noise tensor (training RMSE
    about 0.27) is stated by this test: factors within 5e-2 normwise, training RMSE within
    3e-3 relative (the R-hat refresh products carry two rounded factors); deterministic."""
    p = synth.small(94 + C, (900, 700, 60), 120_000, 4, 20, modes=["zipf", "zipf", "uniform"])
    out = []
    for _ in range(2):
        f, t, A = make(p, tf.F32)
        f.set_precision(3)
        f.set_kernel_path(tf.Factorization.PATH_LEAN)
        r = oracle.residual(t, A)
        for s in range(3):
            order = p.column_order(s, C)
            f.sweep(C, 0.3, 1, order)
            oracle.sals_sweep(t, A, r, C, 0.3, 1, order)
        assert f.counters()["pass_path"] & 8
        for n in range(3):
            assert rel(f.factors(n).astype(np.float64), A[n]) < 5e-2, n
        _, rmse = f.loss(0.3)
        _, rmseo = oracle.loss(t, r, A, 0.3)
        assert abs(rmse - rmseo) <= 3e-3 * rmseo
        out.append([f.factors(n) for n in range(3)] + [f.residual()])
    for a, b in zip(*out):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("C", [4, 10])
def test_lean_pass_row_sources_bit_identical(C):
    """Where the lean pass reads a slice row (the shared-memory cache or the staging pool,
    steps cut short where their cold rows would not fit) and how many warps share a block
    do not change the arithmetic: identical bits for every setting."""
    p = synth.small(70 + C, (2000, 1500, 80), 150_000, 4, 20, modes=["zipf", "zipf", "uniform"])
    out = []
    # (16 warps asks for more than the packed-FMA Gram's launch bound at C = 10: capped)
    for max_rows, pool, warps in ((-1, 24, 0), (0, 32, 0), (0, 2, 0), (48, 4, 5), (300, 16, 12),
                                  (-1, 32, 16)):
        f, _, _ = make(p, tf.F32)
        f.set_kernel_path(tf.Factorization.PATH_LEAN)   # also where the cache covers little
        f.set_pass_cache(max_rows, pool, warps)
        for s in range(2):
            f.sweep(C, 0.1, 1 + s, p.column_order(s, C))
        assert f.counters()["pass_path"] & 8
        out.append([f.factors(n) for n in range(3)] + [f.residual(), np.array(f.loss(0.1))])
    for other in out[1:]:
        for a, b in zip(out[0], other):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("dt", [tf.F32, tf.F64])
def test_sm_limit_does_not_change_results(dt):
    """tf_set_sm_limit only caps how many blocks the persistent mode passes launch: the
    same bins are processed, each by one warp, so results are bit-identical."""
    p = synth.small(77, (900, 700, 60), 80_000, 4, 20, modes=["zipf", "zipf", "uniform"])
    out = []
    for lim in (0, 7, 1):
        f, _, _ = make(p, dt)
        f.set_sm_limit(lim)
        for s in range(2):
            f.sweep(10 if s == 0 else 20, 0.1, 1, p.column_order(s, 10 if s == 0 else 20))
        out.append([f.factors(n) for n in range(3)] + [np.array(f.loss(0.1))])
    for other in out[1:]:
        for a, b in zip(out[0], other):
            assert np.array_equal(a, b)
    f, _, _ = make(p, dt)
    with pytest.raises(tf.TFError):
        f.set_sm_limit(-1)


@pytest.mark.parametrize("C", [4, 10])
def test_lean_loss_pass_matches_residual_kernel_and_oracle(C):
    """tf_loss after a lean sweep of a float three-way context runs as the lean plain pass
    (sums of r^2 per item, then in slot order): the same state read through the pipelined
    residual kernel (kernel path 1) gives the same loss up to FP32 rounding of each r (the
    two form the products in different orders: 1e-5 relative), and both match the FP64
    oracle's loss of the same sweeps within the FP32 bar."""
    p = synth.small(55 + C, (2500, 1800, 90), 220_000, 4, 20, modes=["zipf", "zipf", "uniform"])
    f, t, A = make(p, tf.F32)
    r = oracle.residual(t, A)
    for s in range(2):
        order = p.column_order(s, C)
        f.sweep(C, 0.2, 1, order)
        oracle.sals_sweep(t, A, r, C, 0.2, 1, order)
    assert f.counters()["pass_path"] & 8
    lean = f.loss(0.2)
    f.set_kernel_path(tf.Factorization.PATH_SIMT)
    pipe = f.loss(0.2)
    f.set_kernel_path(0)
    assert f.loss(0.2) == lean   # deterministic
    assert abs(lean[0] - pipe[0]) <= 1e-5 * abs(pipe[0])
    assert abs(lean[1] - pipe[1]) <= 1e-5 * abs(pipe[1])
    Lo, rmseo = oracle.loss(t, r, A, 0.2)
    assert abs(lean[1] - rmseo) <= 1e-3 * rmseo
    assert abs(lean[0] - Lo) <= 2e-3 * abs(Lo)


def test_deterministic_rerun_fp32():
    p = synth.small(34, (300, 300, 30), 50_000, 3, 10, modes=["zipf", "uniform", "uniform"])
    res = []
    for _ in range(2):
        f, _, _ = make(p, tf.F32)
        f.sweep(10, 0.1, 1, p.column_order(0, 10))
        res.append((f.factors(0), f.factors(2), f.loss(0.1)))
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    assert res[0][2] == res[1][2]


def test_default_order_is_permutation_and_identity_for_cdtf():
    p = synth.small(35, (30, 30, 30), 2_000, 2, 12)
    f, _, _ = make(p, tf.F32)
    assert np.array_equal(f.default_order(0, 1), np.arange(12))
    o0, o1 = f.default_order(0, 4), f.default_order(1, 4)
    assert sorted(o0) == list(range(12)) and not np.array_equal(o0, o1)
    f.sweep(4, 0.1, 1)   # default order path runs
    f.sweep(1, 0.1, 1)


def test_change_of_C_between_sweeps():
    """A sweep with a smaller C after a larger one (the lazily kept R-hat of the larger
    split must be flushed first)."""
    p = ragged_problem(23)
    f, t, A = make(p, tf.F64)
    r = oracle.residual(t, A)
    for s, C in enumerate([6, 2, 5, 1]):
        order = p.column_order(s, C)
        f.sweep(C, 0.3, 1, order)
        oracle.sals_sweep(t, A, r, C, 0.3, 1, order)
    for n in range(3):
        assert rel(f.factors(n), A[n]) < 1e-9
    assert rel(f.residual(), r) < 1e-9


@pytest.mark.parametrize("N", [2, 4])
def test_other_tensor_orders(N):
    dims = {2: (400, 300), 4: (40, 30, 20, 25)}[N]
    p = synth.small(36 + N, dims, 8_000, 2, 5)
    f, t, A = make(p, tf.F64)
    r = oracle.residual(t, A)
    for s in range(2):
        order = p.column_order(s, 2)
        f.sweep(2, 0.4, 1, order)
        oracle.sals_sweep(t, A, r, 2, 0.4, 1, order)
    for n in range(N):
        assert rel(f.factors(n), A[n]) < 1e-9


def test_empty_tensor():
    f = tf.Factorization(np.zeros((0, 3), np.int32), np.zeros(0), [5, 4, 3], 3, dtype=tf.F64)
    f.sweep(2, 1.0, 1)
    assert np.all(f.factors(1) == 0)   # empty rows with lambda > 0 go to zero
    assert f.loss(1.0) == (0.0, 0.0)


# --------------------------------------------------------------------------- fold-in


@pytest.mark.parametrize("dtype,tol", [(tf.F64, 1e-10), (tf.F32, 1e-5)])
def test_foldin_matches_oracle(dtype, tol):
    """The FP32 fold-in refines its solve once (FP64 residual of the normal equations
    over the request's entries), which holds it to 1e-5 of the FP64 oracle on the same
    (float-rounded) inputs."""
    p = synth.small(40, (50, 300, 200), 30_000, 5, 24)
    f, t, A = make(p, dtype)
    rng = np.random.default_rng(1)
    for m in (0, 1, 7, 33, 500):
        other = np.stack([rng.integers(0, 300, m), rng.integers(0, 200, m)], 1).astype(np.int32)
        x = rng.standard_normal(m)
        if dtype == tf.F32:
            x = x.astype(np.float32).astype(np.float64)
        got = f.foldin(0, other, x, 0.5)
        ref, st = oracle.foldin(A, 0, other, x, 0.5)
        assert st == 0
        assert rel(got.astype(np.float64), ref) < tol or np.linalg.norm(ref) < 1e-12


@pytest.mark.parametrize("dtype,tol", [(tf.F64, 1e-9), (tf.F32, 1e-5)])
def test_foldin_tiled_large_requests(dtype, tol):
    """K = 100 and requests of up to 20,000 entries: the fold-in is split over many
    blocks whose partial Gram matrices are summed in block order before the solve; in
    FP32 the refined solve stays within 1e-5 of the FP64 oracle."""
    p = synth.small(43, (60, 2000, 300), 60_000, 6, 100)
    f, t, A = make(p, dtype)
    rng = np.random.default_rng(2)
    for m in (1, 255, 257, 5_000, 20_000):
        other = np.stack([rng.integers(0, 2000, m), rng.integers(0, 300, m)], 1).astype(np.int32)
        x = rng.standard_normal(m)
        if dtype == tf.F32:
            x = x.astype(np.float32).astype(np.float64)
        got = f.foldin(0, other, x, 0.7)
        ref, st = oracle.foldin(A, 0, other, x, 0.7)
        assert st == 0
        assert rel(got.astype(np.float64), ref) < tol
    other = np.stack([rng.integers(0, 2000, 5000), rng.integers(0, 300, 5000)], 1).astype(np.int32)
    other[4321, 1] = 300
    with pytest.raises(tf.TFError) as e:
        f.foldin(0, other, np.ones(5000), 0.7)
    assert e.value.status == tf.ERANGE


def test_foldin_rejects_bad_index():
    p = synth.small(41, (20, 30, 40), 2_000, 2, 4)
    f, _, _ = make(p, tf.F32)
    with pytest.raises(tf.TFError) as e:
        f.foldin(0, np.array([[3, 40]], np.int32), np.ones(1), 0.1)
    assert e.value.status == tf.ERANGE
    f.foldin(0, np.array([[3, 39]], np.int32), np.ones(1), 0.1)   # context still usable


# --------------------------------------------------------------------------- full size


def test_skewed_full_size_sampled_rows():
    """The 1e5 x 1e5 x 1e3, 1e8-entry Zipf workload at full size, in the schedule the
    benchmark uses: offsets against a library bincount, sampled first-split mode-1
    rows against the oracle's row update from the same inputs, and the residual
    invariant on sampled entries."""
    dev = "cuda"
    p = synth.skewed_3way(device=dev)
    K, C, lam = p.K, 10, 0.1
    A0 = [a for a in p.init_factors(torch.float32, dev)]
    f = tf.Factorization(p.coords, p.x, p.dims, K, seed=p.seed, dtype=tf.F32,
                         device_input=True)
    for n in range(3):
        f.set_factors(n, A0[n].cpu().numpy())
    for n in range(3):
        off, _ = f.grouping(n, with_perm=False)
        cnt = torch.bincount(p.coords[:, n].long(), minlength=p.dims[n]).cpu().numpy()
        assert np.array_equal(np.diff(off), cnt)
    order = p.column_order(0, C)
    f.sweep(C, lam, 1, order)
    S = order[:C].astype(np.int32)
    A1 = f.factors(0)
    # sampled rows: heaviest, a light one, and random ones
    cnt0 = torch.bincount(p.coords[:, 0].long(), minlength=p.dims[0]).cpu().numpy()
    rows = [int(np.argmax(cnt0)), int(np.argmin(np.where(cnt0 > 0, cnt0, 1 << 40)))]
    rows += list(np.random.default_rng(0).choice(np.nonzero(cnt0)[0], 6, replace=False))
    Ah = [a.double().cpu().numpy() for a in A0]
    for i in rows:
        sel = (p.coords[:, 0] == i).nonzero().squeeze(1)
        c = p.coords[sel].cpu().numpy()
        x = p.x[sel].double().cpu().numpy()
        sub = oracle.Tensor(c, x, p.dims)
        A = [a.copy() for a in Ah]
        assert oracle.row_update(sub, 0, i, x, A, S, lam) == 0   # R-hat = X (A^(1) = 0)
        got = A1[i, S].astype(np.float64)
        err = np.linalg.norm(got - A[0][i, S])
        assert (err <= 1e-5 * np.linalg.norm(A[0][i, S])
                or err <= fp32_row_bound(sub, 0, i, Ah, S, x, lam, A[0][i, S])), i
    # residual invariant on sampled entries, from the device's own factors
    r = f.residual()
    idx = np.random.default_rng(1).choice(p.nnz, 20_000, replace=False)
    c = p.coords[torch.from_numpy(idx).to(dev)].long().cpu().numpy()
    Af = [f.factors(n).astype(np.float64) for n in range(3)]
    model = (Af[0][c[:, 0]] * Af[1][c[:, 1]] * Af[2][c[:, 2]]).sum(1)
    x = p.x[torch.from_numpy(idx).to(dev)].double().cpu().numpy()
    assert np.max(np.abs(r[idx] - (x - model))) <= 1e-4 * np.max(np.abs(x))


# --------------------------------------------------------------------------- wide C


@pytest.mark.parametrize("C,K,T_in,weighted", [(20, 40, 1, False), (33, 40, 2, False),
                                                (40, 40, 1, True), (17, 50, 1, False),
                                                (70, 70, 1, False)])
def test_wide_subsets_match_oracle_fp64(C, K, T_in, weighted):
    """C > 16 takes the tiled wide path (block Gram tiles, shared-memory Cholesky); C = K
    is the ALS row update of Eq. (2).  Ragged last split when C does not divide K."""
    p = synth.small(60 + C, (301, 157, 97), 12_000, 4, K)
    f, t, A = make(p, tf.F64)
    r = oracle.residual(t, A)
    for s in range(2):
        order = p.column_order(s, C)
        f.sweep(C, 0.3, T_in, order, weighted=weighted)
        oracle.sals_sweep(t, A, r, C, 0.3, T_in, order, weighted=weighted)
    for n in range(3):
        assert rel(f.factors(n), A[n]) < 1e-9
    assert rel(f.residual(), r) < 1e-9
    L, _ = f.loss(0.3, weighted=weighted)
    Lo, _ = oracle.loss(t, r, A, 0.3, weighted=weighted)
    assert abs(L - Lo) <= 1e-9 * Lo


def test_wide_subsets_fp32_rmse_and_switching():
    """FP32 wide path: training RMSE within 1e-3 of the FP64 oracle, also when C changes
    between narrow and wide from one sweep to the next (the copies' R-hat is flushed)."""
    p = synth.small(70, (400, 300, 60), 40_000, 5, 48)
    f, t, A = make(p, tf.F32)
    r = oracle.residual(t, A)
    for s, C in enumerate((24, 8, 48, 30)):
        order = p.column_order(s, C)
        f.sweep(C, 0.5, 1, order)
        oracle.sals_sweep(t, A, r, C, 0.5, 1, order)
    _, rmse = f.loss(0.5)
    _, rmseo = oracle.loss(t, r, A, 0.5)
    assert abs(rmse - rmseo) <= 1e-3 * rmseo


def test_wide_singular_rows_left_unchanged():
    p = synth.small(71, (500, 40, 30), 1_500, 2, 20)
    f, t, A = make(p, tf.F64)
    r = oracle.residual(t, A)
    bad_o = oracle.sals_sweep(t, A, r, 20, 0.0, 1, np.arange(20))
    f.sweep(20, 0.0, 1, np.arange(20, dtype=np.int32))
    assert f.counters()["singular_rows"] == bad_o > 0
    for n in range(3):
        assert rel(f.factors(n), A[n]) < 1e-8


@pytest.mark.parametrize("C,K", [(20, 40), (40, 40), (70, 100)])
def test_wide_tensor_core_gram_fp32(C, K):
    """Float contexts compute the wide Gram on the tensor cores (3xTF32, FP32
    accumulation): factors agree with the FP64 oracle to FP32-level error normwise, and
    with the SIMT path of the same library to the same level."""
    p = synth.small(80 + C, (301, 157, 97), 15_000, 4, K)
    f, t, A = make(p, tf.F32)
    f.set_kernel_path(tf.Factorization.PATH_TMA)   # tensor-core Gram for every wide C
    g, _, _ = make(p, tf.F32)
    g.set_kernel_path(tf.Factorization.PATH_SIMT)
    r = oracle.residual(t, A)
    for s in range(2):
        order = p.column_order(s, C)
        f.sweep(C, 0.3, 1, order)
        g.sweep(C, 0.3, 1, order)
        oracle.sals_sweep(t, A, r, C, 0.3, 1, order)
    assert f.counters()["pass_path"] & 4 and not g.counters()["pass_path"] & 4
    for n in range(3):
        assert rel(f.factors(n).astype(np.float64), A[n]) < 2e-4
        assert rel(f.factors(n), g.factors(n)) < 2e-4
    _, rmse = f.loss(0.3)
    _, rmseo = oracle.loss(t, r, A, 0.3)
    assert abs(rmse - rmseo) <= 1e-4 * rmseo


# --------------------------------------------------------------------------- predict


@pytest.mark.parametrize("dtype,tol", [(tf.F64, 1e-12), (tf.F32, 1e-5)])
def test_predict_matches_model(dtype, tol):
    """tf_predict is the CP model of Eq. (1): at the observed coordinates it equals
    x - residual of the oracle (the residual is pinned against a dense reconstruction),
    and a held-out set gives the test RMSE; bad coordinates are rejected."""
    p = synth.small(90, (300, 200, 50), 20_000, 4, 12)
    f, t, A = make(p, dtype)
    for s in range(2):
        order = p.column_order(s, 4)
        f.sweep(4, 0.2, 1, order)
    A_dev = [f.factors(n).astype(np.float64) for n in range(3)]
    held = np.stack([np.arange(500) % 300, (np.arange(500) * 7) % 200,
                     (np.arange(500) * 13) % 50], 1).astype(np.int32)
    got = f.predict(held)
    ref = -oracle.residual(oracle.Tensor(held, np.zeros(500), p.dims), A_dev)
    assert np.max(np.abs(got - ref)) <= tol * max(1.0, np.max(np.abs(ref)))
    got_obs = f.predict(t.coords)
    res = f.residual()
    assert np.max(np.abs((t.x - got_obs) - res)) <= 10 * tol * max(1.0, np.max(np.abs(t.x)))
    import torch
    dev = f.predict(torch.from_numpy(held).cuda())
    assert np.allclose(dev.cpu().numpy(), got, rtol=0, atol=tol * max(1.0, np.max(np.abs(ref))))
    bad = held.copy()
    bad[7, 2] = 50
    with pytest.raises(tf.TFError) as e:
        f.predict(bad)
    assert e.value.status == tf.ERANGE
    assert np.allclose(f.predict(held), got)


@pytest.mark.parametrize("dtype,tol", [(tf.F64, 1e-9), (tf.F32, 1e-4)])
def test_foldin_batch(dtype, tol):
    """A batch of requests of mixed sizes in one launch: each row equals the single
    request's (bit for bit: same blocks, same order) and the oracle's; a request with a
    bad index or a singular system is flagged alone and its row left untouched."""
    p = synth.small(44, (60, 2000, 300), 40_000, 6, 100)
    f, t, A = make(p, dtype)
    rng = np.random.default_rng(3)
    reqs = []
    for m in (1, 300, 0, 5_000, 17, 2_600):
        other = np.stack([rng.integers(0, 2000, m), rng.integers(0, 300, m)], 1).astype(np.int32)
        x = rng.standard_normal(m)
        if dtype == tf.F32:
            x = x.astype(np.float32).astype(np.float64)
        reqs.append((other, x))
    bad = reqs[1][0].copy()
    bad[5, 0] = 2000
    reqs.append((bad, reqs[1][1]))
    rows, status = f.foldin_batch(0, reqs, 0.7)
    assert list(status) == [0, 0, 0, 0, 0, 0, 1]
    assert not rows[-1].any()
    for r, (other, x) in enumerate(reqs[:-1]):
        ref, st = oracle.foldin(A, 0, other, x, 0.7)
        assert st == 0
        assert rel(rows[r].astype(np.float64), ref) < tol or np.linalg.norm(ref) < 1e-12
        assert np.array_equal(rows[r], f.foldin(0, other, x, 0.7))
    # lambda = 0: the empty request is singular, the 5,000-entry one is not
    rows0, status0 = f.foldin_batch(0, [reqs[2], reqs[3]], 0.0)
    assert list(status0) == [2, 0]
    ref, st = oracle.foldin(A, 0, reqs[3][0], reqs[3][1], 0.0)
    assert st == 0 and rel(rows0[1].astype(np.float64), ref) < 100 * tol


# --------------------------------------------------------------------------- more shapes


@pytest.mark.parametrize("N,C,K", [(2, 20, 24), (4, 18, 18), (5, 33, 40), (5, 3, 7)])
def test_wide_and_narrow_other_orders(N, C, K):
    """Tensor orders 2, 4 and 5 on the wide path (C > 16; the generic mode loop) and on the
    narrow path with N = 5, FP64 against the oracle over two sweeps with T_in = 2."""
    dims = {2: (300, 250), 4: (40, 30, 20, 25), 5: (12, 9, 11, 8, 10)}[N]
    p = synth.small(120 + N + C, dims, 6_000, 2, K)
    f, t, A = make(p, tf.F64)
    r = oracle.residual(t, A)
    for s in range(2):
        order = p.column_order(s, C)
        f.sweep(C, 0.4, 2, order)
        oracle.sals_sweep(t, A, r, C, 0.4, 2, order)
    for n in range(N):
        assert rel(f.factors(n), A[n]) < 1e-9
    assert rel(f.residual(), r) < 1e-9


def test_wide_empty_tensor_and_predict_order_four():
    f = tf.Factorization(np.zeros((0, 3), np.int32), np.zeros(0), [5, 4, 3], 40, dtype=tf.F64)
    f.sweep(20, 1.0, 1)
    assert np.all(f.factors(1) == 0)
    assert f.loss(1.0) == (0.0, 0.0)
    p = synth.small(130, (40, 30, 20, 25), 5_000, 2, 6)
    g, t, A = make(p, tf.F64)
    g.sweep(3, 0.4, 1, p.column_order(0, 3))
    A_dev = [g.factors(n) for n in range(4)]
    ref = -oracle.residual(oracle.Tensor(t.coords[:100], np.zeros(100), p.dims), A_dev)
    assert np.max(np.abs(g.predict(t.coords[:100]) - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_foldin_wide_k_single_block():
    """K >= 128 takes the one-block fold-in (single request and in a batch)."""
    p = synth.small(131, (30, 400, 300), 20_000, 4, 130)
    f, t, A = make(p, tf.F64)
    rng = np.random.default_rng(4)
    reqs = []
    for m in (200, 0, 1_000):
        other = np.stack([rng.integers(0, 400, m), rng.integers(0, 300, m)], 1).astype(np.int32)
        reqs.append((other, rng.standard_normal(m)))
    rows, status = f.foldin_batch(0, reqs, 0.9)
    assert list(status) == [0, 0, 0]
    for r, (other, x) in enumerate(reqs):
        ref, st = oracle.foldin(A, 0, other, x, 0.9)
        assert st == 0
        assert rel(rows[r], ref) < 1e-9 or np.linalg.norm(ref) < 1e-12
        assert rel(f.foldin(0, other, x, 0.9), ref) < 1e-9 or np.linalg.norm(ref) < 1e-12


@pytest.mark.parametrize("C,K", [(20, 40), (70, 100)])
def test_reduced_precision_gram(C, K):
    """tf_set_precision(1): one TF32 product per Gram term on the tensor cores.  Stated
    error: training RMSE after three sweeps within 1e-3 of the FP64 oracle's; factors
    within 5e-2 normwise (a row moves by about cond(B + lambda I) * 1e-3)."""
    p = synth.small(140 + C, (301, 157, 97), 15_000, 4, K)
    f, t, A = make(p, tf.F32)
    f.set_precision(1)
    r = oracle.residual(t, A)
    for s in range(3):
        order = p.column_order(s, C)
        f.sweep(C, 0.3, 1, order)
        oracle.sals_sweep(t, A, r, C, 0.3, 1, order)
    assert f.counters()["pass_path"] & 4
    _, rmse = f.loss(0.3)
    _, rmseo = oracle.loss(t, r, A, 0.3)
    assert abs(rmse - rmseo) <= 1e-3 * rmseo
    for n in range(3):
        assert rel(f.factors(n).astype(np.float64), A[n]) < 5e-2
    g, _, _ = make(p, tf.F64)
    with pytest.raises(tf.TFError):
        g.set_precision(1)


@pytest.mark.parametrize("C", [1, 4, 10])
def test_five_way_float(C):
    """Five-way float tensors take the pass specialised for four other modes: training
    RMSE after two sweeps within 1e-3 of the FP64 oracle, factors close normwise."""
    p = synth.small(150 + C, (30, 25, 20, 15, 12), 20_000, 3, 10)
    f, t, A = make(p, tf.F32)
    r = oracle.residual(t, A)
    for s in range(2):
        order = p.column_order(s, C)
        f.sweep(C, 0.4, 1, order)
        oracle.sals_sweep(t, A, r, C, 0.4, 1, order)
    _, rmse = f.loss(0.4)
    _, rmseo = oracle.loss(t, r, A, 0.4)
    assert abs(rmse - rmseo) <= 1e-3 * rmseo
    for n in range(5):
        assert rel(f.factors(n).astype(np.float64), A[n]) < 1e-3


# --------------------------------------------------------------------------- edge cases


@pytest.mark.parametrize("dims,nnz,K,C", [((1, 1, 1), 1, 1, 1), ((5, 7), 1, 3, 3),
                                          ((3, 4, 2, 2, 3, 2, 2, 3), 400, 4, 2),
                                          ((3, 4, 2, 2, 3, 2, 2, 3), 400, 20, 17)])
def test_edge_shapes(dims, nnz, K, C):
    """A single entry, a one-cell tensor, and eight modes (the maximum) on the narrow and
    the wide path, FP64 against the oracle."""
    p = synth.small(160 + len(dims) + K, dims, nnz, 1, K)
    f, t, A = make(p, tf.F64)
    r = oracle.residual(t, A)
    for s in range(2):
        order = p.column_order(s, C)
        f.sweep(C, 0.5, 1, order)
        bad_o = oracle.sals_sweep(t, A, r, C, 0.5, 1, order)
        assert bad_o == 0
    for n in range(len(dims)):
        assert rel(f.factors(n), A[n]) < 1e-9 or np.linalg.norm(A[n]) < 1e-12
    L, _ = f.loss(0.5)
    Lo, _ = oracle.loss(t, r, A, 0.5)
    assert abs(L - Lo) <= 1e-9 * max(Lo, 1e-300)


def test_rejects_bad_sweep_arguments():
    p = synth.small(170, (20, 10, 5), 300, 2, 6)
    f, _, _ = make(p, tf.F64)
    for C, lam, T_in in ((0, 0.1, 1), (7, 0.1, 1), (2, -1.0, 1), (2, 0.1, 0)):
        with pytest.raises(tf.TFError) as e:
            f.sweep(C, lam, T_in)
        assert e.value.status == tf.EINVAL
    with pytest.raises(tf.TFError):
        f.sweep(2, 0.1, 1, np.array([0, 0, 1, 2, 3, 4], np.int32))   # not a permutation
    f.sweep(2, 0.1, 1)   # still usable


# --------------------------------------------------------------------------- concurrency


def test_jobs_on_two_streams_match_solo_runs():
    """Two factorisation jobs on their own CUDA streams, their sweeps and fold-ins queued
    alternately so that their kernels overlap on the device, give bit for bit the results
    each gives alone (contexts share no device state)."""
    import torch
    pa = synth.small(180, (300, 200, 50), 30_000, 4, 24)
    pb = synth.small(181, (150, 400, 60), 25_000, 3, 24)

    def run(p, stream, C):
        c, x = p.numpy()
        f = tf.Factorization(c, x, p.dims, p.K, seed=p.seed, dtype=tf.F32,
                             stream=stream.cuda_stream if stream is not None else None)
        return f

    def finish(f, p, C):
        rows = f.foldin(0, np.stack([np.arange(50) % p.dims[1], np.arange(50) % p.dims[2]], 1),
                        np.linspace(-1, 1, 50), 0.3)
        return [f.factors(n) for n in range(3)], f.loss(0.3), rows

    solo = []
    for p, C in ((pa, 8), (pb, 20)):
        f = run(p, None, C)
        for s in range(3):
            f.sweep(C, 0.3, 1, p.column_order(s, C))
        solo.append(finish(f, p, C))
        f.close()
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    fa, fb = run(pa, sa, 8), run(pb, sb, 20)
    for s in range(3):   # queued back to back, no synchronisation between the two jobs
        fa.sweep(8, 0.3, 1, pa.column_order(s, 8))
        fb.sweep(20, 0.3, 1, pb.column_order(s, 20))
    mixed = [finish(fa, pa, 8), finish(fb, pb, 20)]
    for (fs, ls, rs), (fm, lm, rm) in zip(solo, mixed):
        for n in range(3):
            assert np.array_equal(fs[n], fm[n])
        assert ls == lm
        assert np.array_equal(rs, rm)


def test_set_stream_moves_later_work():
    """A context moved to another stream (here a high-priority one) between sweeps
    continues the same job: the sweeps split across the two streams give bit for bit
    the factors and loss of the same sweeps on one stream."""
    import torch
    p = synth.small(182, (300, 200, 50), 30_000, 3, 12)
    c, x = p.numpy()
    ref = tf.Factorization(c, x, p.dims, p.K, seed=p.seed, dtype=tf.F32)
    for s in range(4):
        ref.sweep(6, 0.3, 1, p.column_order(s, 6))
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream(priority=-1)
    f = tf.Factorization(c, x, p.dims, p.K, seed=p.seed, dtype=tf.F32,
                         stream=s1.cuda_stream)
    for s in range(4):
        if s == 2:
            f.set_stream(s2)
        f.sweep(6, 0.3, 1, p.column_order(s, 6))
    for n in range(3):
        assert np.array_equal(f.factors(n), ref.factors(n))
    assert f.loss(0.3) == ref.loss(0.3)
    f.set_stream(None)   # the legacy default stream
    f.sweep(6, 0.3, 1, p.column_order(4, 6))
    ref.sweep(6, 0.3, 1, p.column_order(4, 6))
    assert np.array_equal(f.factors(0), ref.factors(0))


# --------------------------------------------------------------------------- graphs


@pytest.mark.parametrize("dims,nnz,K,C,T_in,dt,weighted", [
    ((300, 200, 50), 30_000, 8, 4, 1, tf.F64, False),     # narrow, FP64
    ((300, 200, 50), 30_000, 10, 1, 1, tf.F64, False),    # CDTF
    ((300, 200, 50), 30_000, 24, 20, 2, tf.F32, True),    # wide SIMT, T_in 2, weighted
    ((150, 120, 40), 8_000, 80, 70, 1, tf.F32, False),    # wide, tensor-core Gram
    ((120, 90, 60, 30), 25_000, 12, 5, 1, tf.F32, False), # 4-way, ragged last split
])
def test_graph_sweeps_match_eager(dims, nnz, K, C, T_in, dt, weighted):
    """Sweeps replayed from a CUDA graph give bit for bit the factors and loss of eager
    sweeps, with a new column order every sweep (the order reaches the graph through
    device memory)."""
    import torch
    p = synth.small(190 + K, dims, nnz, 4, K)
    c, x = p.numpy()
    s = torch.cuda.Stream()
    out = []
    for graphs in (False, True):
        f = tf.Factorization(c, x, p.dims, p.K, seed=p.seed, dtype=dt, stream=s.cuda_stream)
        f.set_graphs(graphs)
        for t in range(6):
            f.sweep(C, 0.3, T_in, p.column_order(t, C), weighted=weighted)
        out.append(([f.factors(n) for n in range(p.N)], f.loss(0.3, weighted),
                    f.graph_info()))
        f.close()
    (fe, le, ge), (fg, lg, gg) = out
    assert ge["replays"] == 0
    assert gg["replays"] == 4 and gg["cached"] == 1   # sweeps 1-2 eager (Q changes), 3-6 graph
    for n in range(p.N):
        assert np.array_equal(fe[n], fg[n]), n
    assert le == lg


def test_graph_sweeps_across_state_changes():
    """Graph sweeps interleaved with what changes a sweep's launches or its inputs: new
    factors (residuals rebuilt), another schedule (new row plan), another C, a loss and a
    fold-in between sweeps -- the same results as the same calls without graphs."""
    import torch
    p = synth.small(197, (400, 300, 60), 40_000, 4, 12)
    c, x = p.numpy()
    A1 = p.init_factors()[1].numpy() * 0.5
    s = torch.cuda.Stream()
    res = []
    for graphs in (False, True):
        f = tf.Factorization(c, x, p.dims, p.K, seed=p.seed, dtype=tf.F64, stream=s.cuda_stream)
        f.set_graphs(graphs)
        log = []
        for t in range(4):
            f.sweep(4, 0.2, 1, p.column_order(t, 4))
        log.append(f.loss(0.2))
        f.set_factors(1, A1)
        for t in range(3):
            f.sweep(4, 0.2, 1, p.column_order(10 + t, 4))
        f.set_schedule(tf.SCHED_GREEDY, 0)
        for t in range(3):
            f.sweep(4, 0.2, 1, p.column_order(20 + t, 4))
        for t in range(4):
            Ct = 3 if t % 2 else 6
            f.sweep(Ct, 0.2, 1, p.column_order(30 + t, Ct))
        log.append(f.foldin(0, np.stack([np.arange(30) % 300, np.arange(30) % 60], 1),
                            np.linspace(-1, 1, 30), 0.2))
        for t in range(3):
            f.sweep(4, 0.2, 1, p.column_order(40 + t, 4))
        log.append([f.factors(n) for n in range(3)])
        log.append(f.loss(0.2))
        res.append(log)
        f.close()
    e, g = res
    assert e[0] == g[0] and e[3] == g[3]
    assert np.array_equal(e[1], g[1])
    for n in range(3):
        assert np.array_equal(e[2][n], g[2][n])


# --------------------------------------------------------------------------- autotuning


@pytest.mark.parametrize("dt", [tf.F32, tf.F64])
def test_autotune_restores_state_and_keeps_best_schedule(dt):
    """tf_autotune times every (P, C) pair, leaves the fastest pair's schedule, and
    restores the state: later sweeps equal, bit for bit, those of a twin context that was
    never autotuned but runs on the chosen schedule."""
    p = synth.small(205, (600, 500, 80), 80_000, 4, 16)
    c, x = p.numpy()
    f = tf.Factorization(c, x, p.dims, p.K, seed=p.seed, dtype=dt)
    g = tf.Factorization(c, x, p.dims, p.K, seed=p.seed, dtype=dt)
    for h in (f, g):
        for t in range(2):
            h.sweep(4, 0.2, 1)   # default orders: they depend on the sweep counter
    Cs, Ps = [2, 4, 8, 12], [0, 304, 2432]
    bc, bp, ms = f.autotune(Cs, Ps, lam=0.2)
    assert ms.shape == (3, 4) and (ms > 0).all()
    assert ms[Ps.index(bp), Cs.index(bc)] == ms.min()
    g.set_schedule(tf.SCHED_LPT, bp)
    for h in (f, g):
        for t in range(3):
            h.sweep(4, 0.2, 1)
    for n in range(3):
        assert np.array_equal(f.factors(n), g.factors(n)), n
    assert f.loss(0.2) == g.loss(0.2)


def test_autotune_rejects_bad_candidates():
    p = synth.small(206, (100, 80, 20), 5_000, 2, 8)
    c, x = p.numpy()
    f = tf.Factorization(c, x, p.dims, p.K, seed=p.seed, dtype=tf.F32)
    for Cs, Ps in (([0, 2], [0]), ([9], [0]), ([2], [-1]), ([], [0]), ([2], [])):
        with pytest.raises(tf.TFError) as e:
            f.autotune(Cs, Ps)
        assert e.value.status == tf.EINVAL
    f.sweep(2, 0.1, 1)


# --------------------------------------------------------------------------- solve options


def _dup_column_case(K, seed):
    """Factors of modes 2 and 3 with columns 0 and 1 equal: for every mode-1 row the Gram
    matrix of Eq. 4 is singular in those columns, B + lambda I has condition ~ 1/lambda."""
    p = synth.small(seed, (300, 200, 50), 30_000, 3, K)
    c, x = p.numpy()
    x = x.astype(np.float32).astype(np.float64)
    A = [a.numpy().astype(np.float32).astype(np.float64) for a in p.init_factors()]
    for n in (1, 2):
        A[n][:, 1] = A[n][:, 0]
    return p, c, x, A


def _first_mode_error(p, c, x, A, C, lam, refine, cond):
    t = oracle.Tensor(c, x, p.dims)
    Ao = [a.copy() for a in A]
    r = oracle.residual(t, Ao)
    order = np.arange(p.K, dtype=np.int32)
    # one split (C = K) so that mode 1's rows see exactly the prepared factors
    oracle.sals_sweep(t, Ao, r, C, lam, 1, order)
    f = tf.Factorization(c, x, p.dims, p.K, seed=p.seed, dtype=tf.F32)
    for n in range(3):
        f.set_factors(n, A[n])
    f.set_solve(refine, cond)
    f.sweep(C, lam, 1, order)
    err = np.linalg.norm(f.factors(0) - Ao[0]) / np.linalg.norm(Ao[0])
    out = err, f.counters()["singular_rows"], f.fp64_rows()
    f.close()
    return out


@pytest.mark.parametrize("K", [4, 20])   # narrow register solve, wide warp solve
def test_fp64_fallback_solves_rows_fp32_cannot(K):
    """lambda = 1e-6 with duplicated columns: the FP32 Cholesky meets non-positive pivots
    and leaves rows unchanged; with the FP64 fallback no row is singular and the first
    mode's update matches the FP64 oracle."""
    p, c, x, A = _dup_column_case(K, 210 + K)
    err0, sing0, f640 = _first_mode_error(p, c, x, A, K, 1e-6, 0, 0.0)
    err1, sing1, f641 = _first_mode_error(p, c, x, A, K, 1e-6, 0, 1e4)
    assert sing0 > 0 and f640 == 0
    assert sing1 == 0 and f641 > 0
    assert err1 < 1e-5, (err0, err1)


@pytest.mark.parametrize("K", [4, 20])
def test_refinement_reduces_solve_error(K):
    """lambda = 1e-3 with duplicated columns (condition ~ 1e3-1e4): one refinement step
    with an FP64 residual brings the first mode's update to FP32 accuracy against the
    FP64 oracle, far below the plain FP32 Cholesky's error."""
    p, c, x, A = _dup_column_case(K, 230 + K)
    err0, sing0, _ = _first_mode_error(p, c, x, A, K, 1e-3, 0, 0.0)
    err1, sing1, _ = _first_mode_error(p, c, x, A, K, 1e-3, 1, 0.0)
    assert sing0 == sing1 == 0
    assert err1 < 1e-5 and err1 < err0 / 10, (err0, err1)


def test_solve_options_leave_double_contexts_alone():
    p = synth.small(240, (300, 200, 50), 30_000, 3, 8)
    c, x = p.numpy()
    out = []
    for opts in ((0, 0.0), (1, 1e4)):
        f = tf.Factorization(c, x, p.dims, p.K, seed=p.seed, dtype=tf.F64)
        f.set_solve(*opts)
        for t in range(2):
            f.sweep(4, 0.2, 1, p.column_order(t, 4))
        out.append([f.factors(n) for n in range(3)])
        assert f.fp64_rows() == 0
        f.close()
    for n in range(3):
        assert np.array_equal(out[0][n], out[1][n])
    with pytest.raises(tf.TFError):   # a negative limit is refused
        tf.Factorization(c, x, p.dims, p.K, seed=p.seed, dtype=tf.F64).set_solve(False, -1.0)


def test_device_peaks_plausible():
    """tf_device_peaks measures this GPU's FP32 FMA rates and shared-memory bandwidth:
    positive, within physical bounds, the packed FMA at least as fast as the plain one."""
    d = tf.device_peaks()
    assert 5.0 < d["fp32_tflops"] < 1000.0
    assert d["fp32x2_tflops"] >= 0.8 * d["fp32_tflops"]
    assert 1.0 < d["smem_tbytes"] < 1000.0
