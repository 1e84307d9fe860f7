"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here re-calls the oracle to check itself: each test compares it with an
independent route -- a library least-squares solve, a numpy restatement of a different
algorithm that must coincide (ALS, Eq. (2); CDTF's scalar closed form, Section 3.1),
finite differences of the loss (Theorem 1), hand-worked fixtures (tests/golden), a
library sort, or an invariant of the residual tensor (Section 3.1).
The mutation test at the end plants typical mistakes in a copy of the oracle source
and checks that these pins catch every one.
"""
import os
import shutil
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from tests import golden

# --------------------------------------------------------------------------- helpers


def tiny_problem(seed, dims=(6, 5, 4), nnz=60, rank=2, K=4, noise=0.1):
    p = synth.small(seed, dims, nnz, rank, K, noise_std=noise)
    c, x = p.numpy()
    A = [a.numpy().copy() for a in p.init_factors()]
    return p, oracle.Tensor(c, x, p.dims), A


def model_np(coords, A):
    """sum_k prod_n A_n[i_n, k] evaluated with numpy fancy indexing."""
    prod = np.ones((coords.shape[0], A[0].shape[1]))
    for n, a in enumerate(A):
        prod = prod * a[coords[:, n]]
    return prod.sum(axis=1)


def loss_np(t, A, lam):
    r = t.x - model_np(t.coords, A)
    return float(r @ r + lam * sum((a * a).sum() for a in A))


def ridge_lstsq(Phi, y, lam):
    """argmin ||y - Phi a||^2 + lam ||a||^2 by an SVD least-squares solve of the stacked
    system [Phi; sqrt(lam) I] a = [y; 0] (no normal equations)."""
    C = Phi.shape[1]
    M = np.vstack([Phi, np.sqrt(lam) * np.eye(C)])
    rhs = np.concatenate([y, np.zeros(C)])
    return np.linalg.lstsq(M, rhs, rcond=None)[0]


def design_rows(t, n, i, A, S):
    """Phi[e, q] = prod_{l != n} A_l[i_l, S_q] for the entries of row i of mode n."""
    sel = np.nonzero(t.coords[:, n] == i)[0]
    Phi = np.ones((len(sel), len(S)))
    for l in range(t.N):
        if l != n:
            Phi *= A[l][t.coords[sel, l]][:, S]
    return sel, Phi


def als_np(t, A, lam):
    """Full ALS outer iteration, Eq. (2), with numpy: for each mode, each row solves
    (B + lam I_K) a = c with c built from the observed values x."""
    A = [a.copy() for a in A]
    K = A[0].shape[1]
    for n in range(t.N):
        for i in range(int(t.dims[n])):
            sel, Phi = design_rows(t, n, i, A, np.arange(K))
            B = Phi.T @ Phi + lam * np.eye(K)
            A[n][i] = np.linalg.solve(B, Phi.T @ t.x[sel])
    return A


def cdtf_np(t, A, r, lam, T_in, order):
    """CDTF (Section 3.1): columns one at a time in `order`; each entry of the column
    is the scalar minimiser sum(rhat*h) / (lam + sum h^2)."""
    A = [a.copy() for a in A]
    r = r.copy()
    for k in order:
        colprod = np.ones(t.nnz)
        for l in range(t.N):
            colprod *= A[l][t.coords[:, l], k]
        rhat = r + colprod
        for _ in range(T_in):
            for n in range(t.N):
                for i in range(int(t.dims[n])):
                    sel = np.nonzero(t.coords[:, n] == i)[0]
                    h = np.ones(len(sel))
                    for l in range(t.N):
                        if l != n:
                            h *= A[l][t.coords[sel, l], k]
                    A[n][i, k] = (rhat[sel] @ h) / (lam + h @ h)
        colprod = np.ones(t.nnz)
        for l in range(t.N):
            colprod *= A[l][t.coords[:, l], k]
        r = rhat - colprod
    return A, r


# --------------------------------------------------------------------------- pins
# Each pin takes the oracle library handle so the mutation test can re-run it.


def pin_group(lib):
    p, t, _ = tiny_problem(3, dims=(9, 7, 5), nnz=150)
    for n in range(t.N):
        off, perm = oracle.group(t, n, lib)
        keys = [t.coords[:, (n + s) % t.N] for s in range(t.N)]
        ref = np.lexsort(keys[::-1])          # numpy: last key is the primary one
        assert np.array_equal(perm, ref)
        cnt = np.bincount(t.coords[:, n], minlength=int(t.dims[n]))
        assert np.array_equal(off, np.concatenate([[0], np.cumsum(cnt)]))


def pin_residual(lib):
    p, t, A = tiny_problem(4)
    rng = np.random.default_rng(0)
    A[0] = rng.standard_normal(A[0].shape)
    r = oracle.residual(t, A, lib)
    assert np.allclose(r, t.x - model_np(t.coords, A), rtol=1e-13, atol=1e-13)


def pin_row_update_lstsq(lib, weighted=False):
    """Eq. (4) / Theorem 1: each row's C parameters are the ridge least-squares
    minimiser over Omega_i^(n), here for every row of every mode."""
    p, t, A = tiny_problem(5, dims=(5, 4, 3), nnz=40, K=5)
    rng = np.random.default_rng(1)
    A = [rng.standard_normal(a.shape) for a in A]
    rhat = rng.standard_normal(t.nnz)
    S = np.array([3, 0, 4], np.int32)
    lam = 0.7
    for n in range(t.N):
        for i in range(int(t.dims[n])):
            A2 = [a.copy() for a in A]
            st = oracle.row_update(t, n, i, rhat, A2, S, lam, weighted, lib)
            assert st == 0
            sel, Phi = design_rows(t, n, i, A, S)
            lam_i = lam * (len(sel) if weighted else 1)
            ref = ridge_lstsq(Phi, rhat[sel], lam_i)
            assert np.allclose(A2[n][i, S], ref, rtol=1e-10, atol=1e-12)
            untouched = np.setdiff1d(np.arange(A[0].shape[1]), S)
            assert np.array_equal(A2[n][i, untouched], A[n][i, untouched])


def pin_als(lib):
    """SALS with C = K and T_in = 1 is ALS (Section 3)."""
    p, t, A = tiny_problem(6, dims=(6, 5, 4), nnz=70, K=3)
    r = oracle.residual(t, A, lib)
    lam = 0.3
    order = np.array([2, 0, 1], np.int32)
    A_s = [a.copy() for a in A]
    oracle.sals_sweep(t, A_s, r, C=3, lam=lam, T_in=1, col_order=order, lib=lib)
    A_a = als_np(t, A, lam)
    for a, b in zip(A_s, A_a):
        assert np.allclose(a, b, rtol=1e-9, atol=1e-11)
    assert np.allclose(r, t.x - model_np(t.coords, A_a), rtol=1e-9, atol=1e-11)


def pin_cdtf(lib):
    """SALS with C = 1 is CDTF; compared against the scalar closed form, T_in = 2."""
    p, t, A = tiny_problem(7, dims=(5, 6, 3), nnz=50, K=3)
    rng = np.random.default_rng(2)
    A[0] = rng.standard_normal(A[0].shape) * 0.5
    r = oracle.residual(t, A, lib)
    order = np.array([1, 2, 0], np.int32)
    A_c, r_c = cdtf_np(t, A, r, 0.4, 2, order)
    oracle.sals_sweep(t, A, r, C=1, lam=0.4, T_in=2, col_order=order, lib=lib)
    for a, b in zip(A, A_c):
        assert np.allclose(a, b, rtol=1e-10, atol=1e-12)
    assert np.allclose(r, r_c, rtol=1e-10, atol=1e-12)


def pin_golden_cdtf(lib):
    d = golden.cdtf_tiny()
    coords = np.array([[int(v) for v in e[:3]] for e in d["entries"]], np.int32)
    x = np.array([float(e[3]) for e in d["entries"]])
    t = oracle.Tensor(coords, x, [int(v) for v in d["dims"]])
    A = [np.array([[float(v)] for v in d[f"init A{n}"]]) for n in (1, 2, 3)]
    r = oracle.residual(t, A, lib)
    oracle.sals_sweep(t, A, r, C=1, lam=float(d["lambda"][0]), T_in=1, lib=lib)
    for n in (1, 2, 3):
        exp = np.array([float(v) for v in d[f"final A{n}"]])
        assert np.allclose(A[n - 1][:, 0], exp, rtol=1e-14, atol=0)
    assert np.allclose(r, [float(v) for v in d["final r"]], rtol=1e-14, atol=0)


def pin_sals_general(lib):
    """C = 2 (not dividing K = 5), T_in = 2: every pass keeps the stored residual equal
    to the residual recomputed from the factors, and after the sweep the last mode's
    rows are stationary points of the loss in the last split's columns (Theorem 1)."""
    p, t, A = tiny_problem(8, dims=(5, 4, 6), nnz=60, K=5)
    A[0] = np.random.default_rng(7).standard_normal(A[0].shape) * 0.5  # R-hat != R
    r = oracle.residual(t, A, lib)
    lam = 0.5
    order = np.array([4, 1, 3, 0, 2], np.int32)
    oracle.sals_sweep(t, A, r, C=2, lam=lam, T_in=2, col_order=order, lib=lib)
    assert np.allclose(r, t.x - model_np(t.coords, A), rtol=1e-11, atol=1e-12)
    # last split is the single column order[4] = 2; with T_in = 2 its last pass is mode 3
    k = 2
    eps = 1e-5
    for i in range(int(t.dims[2])):
        def L(delta):
            B = [a.copy() for a in A]
            B[2][i, k] += delta
            return loss_np(t, B, lam)
        g = (L(eps) - L(-eps)) / (2 * eps)
        assert abs(g) < 1e-6 * max(1.0, L(0.0))
        assert L(1e-3) >= L(0.0) and L(-1e-3) >= L(0.0)


# --------------------------------------------------------------------------- tests


def test_group_matches_library_lexsort():
    pin_group(oracle.load())


def pin_validate(lib):
    t = oracle.Tensor(np.array([[0, 0], [1, 2]], np.int32), [1.0, 2.0], [2, 3])
    assert oracle.validate(t, lib) == oracle.OK
    t = oracle.Tensor(np.array([[0, 0], [1, 3]], np.int32), [1.0, 2.0], [2, 3])
    assert oracle.validate(t, lib) == oracle.ERANGE
    t = oracle.Tensor(np.array([[1, 2], [0, 0], [1, 2]], np.int32), [1.0, 2.0, 3.0], [2, 3])
    assert oracle.validate(t, lib) == oracle.EDUP


def test_validate_rejects_range_and_duplicates():
    pin_validate(oracle.load())


def test_residual_matches_dense_reconstruction():
    pin_residual(oracle.load())


def test_init_invariant_R_equals_X():
    """Algorithm 1 initialisation: A^(1) = 0 makes R = X exactly."""
    p, t, A = tiny_problem(9)
    assert np.all(A[0] == 0)
    assert np.array_equal(oracle.residual(t, A), t.x)


def pin_loss(lib):
    """Eq. (1) and the training RMSE, from the numpy model (not the oracle's residual)."""
    p, t, A = tiny_problem(10)
    rng = np.random.default_rng(3)
    A = [rng.standard_normal(a.shape) for a in A]
    r = t.x - model_np(t.coords, A)
    L, rmse = oracle.loss(t, r, A, 0.25, lib=lib)
    assert np.isclose(L, loss_np(t, A, 0.25), rtol=1e-13)
    assert np.isclose(rmse, np.sqrt(np.mean(r ** 2)), rtol=1e-13)


def pin_weighted_loss(lib):
    """The weighted regulariser (Section 5.1.3): row i of mode n counts |Omega_i^(n)| times."""
    p, t, A = tiny_problem(10)
    rng = np.random.default_rng(3)
    A = [rng.standard_normal(a.shape) for a in A]
    r = t.x - model_np(t.coords, A)
    L, _ = oracle.loss(t, r, A, 0.25, weighted=True, lib=lib)
    reg = sum((np.bincount(t.coords[:, n], minlength=int(t.dims[n])) * (A[n] ** 2).sum(1)).sum()
              for n in range(t.N))
    assert np.isclose(L, r @ r + 0.25 * reg, rtol=1e-13)


def test_loss_matches_definition():
    pin_loss(oracle.load())


def test_weighted_loss_definition():
    pin_weighted_loss(oracle.load())


def test_row_update_is_ridge_least_squares():
    pin_row_update_lstsq(oracle.load())


def test_row_update_weighted_lambda_is_ridge_least_squares():
    pin_row_update_lstsq(oracle.load(), weighted=True)


def test_sals_with_C_equal_K_is_als():
    pin_als(oracle.load())


def test_sals_with_C_one_is_cdtf_closed_form():
    pin_cdtf(oracle.load())


def test_cdtf_hand_worked_example():
    pin_golden_cdtf(oracle.load())


def test_residual_invariant_and_stationarity():
    pin_sals_general(oracle.load())


@pytest.mark.parametrize("C", [1, 2, 4])
def test_loss_never_increases(C):
    """Theorem 1: every row update is an exact block minimiser, so the loss is
    non-increasing over sweeps (checked with the numpy loss, not the oracle's)."""
    p, t, A = tiny_problem(11, dims=(8, 7, 6), nnz=150, K=4)
    r = oracle.residual(t, A)
    prev = loss_np(t, A, 0.2)
    for s in range(6):
        oracle.sals_sweep(t, A, r, C=C, lam=0.2, col_order=p.column_order(s, C))
        cur = loss_np(t, A, 0.2)
        assert cur <= prev * (1 + 1e-12)
        prev = cur


def test_row_relabel_invariance():
    """Rows are independent (Section 3.3): relabelling the rows of a mode permutes the
    result and changes nothing else (up to summation order)."""
    p, t, A = tiny_problem(12, dims=(7, 6, 5), nnz=90, K=3)
    perm = np.random.default_rng(4).permutation(7)
    c2 = t.coords.copy()
    c2[:, 0] = perm[t.coords[:, 0]]
    t2 = oracle.Tensor(c2, t.x, t.dims)
    A2 = [a.copy() for a in A]
    A2[0][perm] = A[0]
    r1, r2 = oracle.residual(t, A), oracle.residual(t2, A2)
    order = np.array([1, 0, 2], np.int32)
    oracle.sals_sweep(t, A, r1, 2, 0.3, col_order=order)
    oracle.sals_sweep(t2, A2, r2, 2, 0.3, col_order=order)
    assert np.allclose(A2[0][perm], A[0], rtol=1e-12, atol=1e-14)
    assert np.allclose(A2[1], A[1], rtol=1e-12, atol=1e-14)
    assert np.allclose(A2[2], A[2], rtol=1e-12, atol=1e-14)
    assert np.allclose(r1, r2, rtol=1e-12, atol=1e-14)


def pin_singular(lib):
    """Reading for lambda = 0: an empty row has B + lambda I = 0, a zero pivot; the row
    keeps its value and is counted (with lambda > 0 the empty row's solution is 0)."""
    coords = np.array([[0, 0, 0], [0, 1, 0], [2, 1, 0]], np.int32)  # row 1 of mode 1 empty
    t = oracle.Tensor(coords, [1.0, 2.0, 3.0], [3, 2, 1])
    A = [np.full((3, 1), 0.5), np.ones((2, 1)), np.ones((1, 1))]
    r = oracle.residual(t, A, lib)
    bad = oracle.sals_sweep(t, A, r, 1, 0.0, lib=lib)
    assert bad == 1 and A[0][1, 0] == 0.5
    A = [np.full((3, 1), 0.5), np.ones((2, 1)), np.ones((1, 1))]
    r = oracle.residual(t, A, lib)
    assert oracle.sals_sweep(t, A, r, 1, 0.1, lib=lib) == 0 and A[0][1, 0] == 0.0


def test_singular_row_left_unchanged():
    pin_singular(oracle.load())


def test_convergence_on_noiseless_low_rank():
    """Sanity (not a parity pin): on exact rank-2 data with K = 3, small lambda and many
    observations, the training RMSE falls by orders of magnitude."""
    p = synth.small(13, (20, 20, 20), 4000, 2, 3, noise_std=0.0)
    c, x = p.numpy()
    t = oracle.Tensor(c, x, p.dims)
    A = [a.numpy().copy() for a in p.init_factors()]
    r = oracle.residual(t, A)
    rmse0 = oracle.loss(t, r, A, 1e-4)[1]
    for s in range(40):
        oracle.sals_sweep(t, A, r, 3, 1e-4, col_order=p.column_order(s, 3))
    rmse = oracle.loss(t, r, A, 1e-4)[1]
    assert rmse < 1e-2 * rmse0


def pin_foldin(lib):
    """Eq. (2) for a new row against frozen factors: the ridge least-squares row."""
    p, t, A = tiny_problem(14, dims=(5, 30, 20), nnz=300, K=6)
    rng = np.random.default_rng(5)
    A = [rng.standard_normal(a.shape) for a in A]
    m = 40
    other = np.stack([rng.integers(0, 30, m), rng.integers(0, 20, m)], 1).astype(np.int32)
    x = rng.standard_normal(m)
    row, st = oracle.foldin(A, 0, other, x, 0.3, lib)
    Phi = A[1][other[:, 0]] * A[2][other[:, 1]]
    assert st == 0
    assert np.allclose(row, ridge_lstsq(Phi, x, 0.3), rtol=1e-10, atol=1e-12)


def test_foldin_is_ridge_least_squares():
    pin_foldin(oracle.load())


def pin_alg3(lib):
    for case in golden.alg3_cases():
        dims = [len(m) for m in case["modes"]]
        got = oracle.greedy_assign(dims, case["modes"], case["M"], lib)
        for g, e in zip(got, case["expect"]):
            assert list(g) == e, case["name"]


def test_greedy_assignment_hand_cases():
    pin_alg3(oracle.load())


def test_greedy_assignment_respects_cap_and_balances():
    rng = np.random.default_rng(6)
    nnz = rng.zipf(1.5, 200).clip(max=500)
    M = 7
    a = oracle.greedy_assign([200], [nnz], M)[0]
    rows = np.bincount(a, minlength=M)
    assert rows.max() <= -(-200 // M)
    load = np.bincount(a, weights=nnz, minlength=M)
    assert load.max() - load.min() <= nnz.max()


# --------------------------------------------------------------------------- mutations

MUTANTS = {
    "lambda dropped": ("B[q * C + q] += lam;", "B[q * C + q] += 0.0 * lam;"),
    "sign of Eq. (5)": ("r[e] = rhat[e] - model_part", "r[e] = rhat[e] + model_part"),
    "own mode in h": ("if (l != n) p *= A[l]", "p *= A[l]"),
    "R-hat not formed": ("rhat[e] = r[e] + model_part(N, coords + e * N, K, A, S, Cs);",
                         "rhat[e] = r[e];"),
    "transposed factor in back-substitution": ("s -= M[k * m + i] * a[k];",
                                               "s -= M[i * m + k] * a[k];"),
    "rhs squared h": ("c[q1] += rhat[e] * h[q1];", "c[q1] += rhat[e] * h[q1] * h[q1];"),
    "wrong column in h": ("* K + S[q]];\n            h[q] = p;", "* K + S[0]];\n            h[q] = p;"),
    "tie-break on rows reversed": ("rows_n[m] < rows_n[best]", "rows_n[m] > rows_n[best]"),
    "residual sign": ("r[e] = x[e] - s;", "r[e] = s - x[e];"),
    "weighted lambda ignored in the row update": (
        "if (flags & ORC_WEIGHTED) lam *= (double)(off[i + 1] - off[i]);",
        "if (flags & ORC_WEIGHTED) lam *= 1.0;"),
    "regulariser dropped from the loss": ("*loss = sr + lambda * reg;", "*loss = sr;"),
    "row weights ignored in the weighted loss": (
        "double w = (flags & ORC_WEIGHTED) ? (double)row_nnz[n][i] : 1.0;", "double w = 1.0;"),
    "RMSE not divided by the entry count": ("sqrt(sr / (double)nnz)", "sqrt(sr)"),
    "inner iterations run once": ("for (int t = 0; t < T_in; ++t)", "for (int t = 0; t < 1; ++t)"),
    "lambda dropped from the fold-in": ("for (int k = 0; k < K; ++k) B[k * K + k] += lambda;",
                                        "for (int k = 0; k < K; ++k) B[k * K + k] += 0.0 * lambda;"),
    "fold-in rhs not weighted by the values": ("c[k1] += x[j] * h[k1];", "c[k1] += h[k1];"),
    "cyclic order of the remaining modes reversed": ("int m = (g_mode + t) % g_N;",
                                                      "int m = (g_mode + g_N - t) % g_N;"),
    "Cholesky column update dropped": (
        "for (int k = 0; k < j; ++k) s -= M[i * m + k] * M[j * m + k];",
        "for (int k = 0; k < 0; ++k) s -= M[i * m + k] * M[j * m + k];"),
    "transposed factor in forward substitution": ("s -= M[i * m + k] * a[k];",
                                                  "s -= M[k * m + i] * a[k];"),
    "pivot not square-rooted": ("double ljj = sqrt(d);", "double ljj = d;"),
    "range check off by one": ("coords[e * N + n] >= dims[n]) return ORC_ERANGE;",
                               "coords[e * N + n] > dims[n]) return ORC_ERANGE;"),
    "duplicates accepted": ("if (same) st = ORC_EDUP;", "if (same) st = ORC_OK;"),
    "row cap of Algorithm 3 ignored": ("if (rows_n[m] >= cap) continue;",
                                       "if (rows_n[m] > In) continue;"),
    "Algorithm 3 rows in increasing length": (
        "return g_rownnz[a] > g_rownnz[b] ? -1 : 1;", "return g_rownnz[a] > g_rownnz[b] ? 1 : -1;"),
    "residuals not squared in the loss": ("sr += r[e] * r[e];", "sr += r[e];"),
    "zero pivot accepted": ("if (!(d > 0.0)) return 1;", "if (d < 0.0) return 1;"),
    "R-hat and Eq. (5) carry only the subset's first column": (
        "for (int q = 0; q < C; ++q) {\n        double p = 1.0;\n        for (int n = 0; n < N; ++n) p *= A[n][(int64_t)ce[n]",
        "for (int q = 0; q < 1; ++q) {\n        double p = 1.0;\n        for (int n = 0; n < N; ++n) p *= A[n][(int64_t)ce[n]"),
}

def pin_row_update_weighted(lib):
    pin_row_update_lstsq(lib, weighted=True)


PINS = [pin_group, pin_validate, pin_residual, pin_loss, pin_weighted_loss, pin_row_update_lstsq,
        pin_row_update_weighted, pin_als, pin_cdtf, pin_golden_cdtf, pin_sals_general, pin_foldin,
        pin_singular, pin_alg3]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name):
    """Plant one mistake in a copy of the oracle source (on the CPU) and check that at
    least one pin fails on it."""
    if shutil.which("gcc") is None:
        pytest.skip("gcc missing")
    old, new = MUTANTS[name]
    src = open(oracle._SRC).read()
    assert src.count(old) == 1, name
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "mut.c")
        with open(path, "w") as f:
            f.write(src.replace(old, new))
        so = oracle.build(path, os.path.join(d, "libmut.so"))
        lib = oracle.load(so)
        caught = []
        for pin in PINS:
            try:
                pin(lib)
            except AssertionError:
                caught.append(pin.__name__)
        assert caught, f"mutant '{name}' passed every pin"
