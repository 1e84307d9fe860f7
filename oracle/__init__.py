"""FP64 CPU oracle for SALS / CDTF (arXiv 1410.5209) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import this package.  The product library never loads it and the
two share no code.  The arithmetic lives in ``sals_oracle.c`` (plain serial C, FP64);
this module only compiles it with gcc and marshals numpy arrays through ctypes.

Citations (paper sections / equations / algorithms):
  * :func:`residual`, :func:`loss` -- Definition 1, Eq. (1); residual tensor R (Section 3.1)
  * :func:`group`                  -- Omega_i^(n) (table of symbols)
  * :func:`row_update`             -- Eq. (4) with the Cholesky solve of Section 3.1
  * :func:`sals_sweep`             -- Algorithm 1 (one outer iteration), Eq. (4), Eq. (5)
  * :func:`foldin`                 -- Eq. (2) row solve against frozen factors
  * :func:`greedy_assign`          -- Algorithm 3 with both tie-breaks

Pins: every function above is checked in ``tests/test_oracle_pins.py`` against
something other than itself (brute-force least squares, closed forms, independent
ALS/CDTF restatements, finite differences, hand-worked fixtures in tests/golden).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sals_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsals_oracle.so")

OK, EINVAL, ERANGE, EDUP, ENOMEM = 0, 1, 2, 3, 4
WEIGHTED = 1

_lib = None


_OMP_PATH = os.path.join(_BUILD, "libsals_oracle_omp.so")


def build(src: str = _SRC, out: str = _LIB_PATH, openmp: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math); openmp=True also builds the
    OpenMP variant used only as the benchmark's multi-core CPU baseline."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", out, src, "-lm"]
    subprocess.run(cmd, check=True)
    if openmp:
        subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o",
                        _OMP_PATH, src, "-lm"], check=True)
    return out


_omp_lib = None


def load_parallel():
    """The OpenMP build of the same source (rows of a mode in parallel, each row's
    arithmetic unchanged): for the multi-core CPU baseline only."""
    global _omp_lib
    if _omp_lib is None:
        if (not os.path.exists(_OMP_PATH)
                or os.path.getmtime(_OMP_PATH) < os.path.getmtime(_SRC)):
            build(openmp=True)
        _omp_lib = _bind(ctypes.CDLL(_OMP_PATH))
    return _omp_lib


def load(path: str | None = None):
    """Load (building if needed) the oracle shared library."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    if _lib is None:
        if (not os.path.exists(_LIB_PATH)
                or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
            build()
        _lib = _bind(ctypes.CDLL(_LIB_PATH))
    return _lib


def _bind(lib):
    P = ctypes.c_void_p
    i32, i64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_double
    lib.orc_group.argtypes = [i32, P, i64, P, i32, P, P]
    lib.orc_validate.argtypes = [i32, P, i64, P]
    lib.orc_residual.argtypes = [i32, i64, P, P, i32, P, P]
    lib.orc_loss.argtypes = [i32, P, i64, P, i32, P, f64, i32, P, P, P]
    lib.orc_row_update.argtypes = [i32, i32, i64, P, P, i32, P, P, i32, f64, i32, P, P]
    lib.orc_sals_sweep.argtypes = [i32, P, i64, P, i32, P, P, i32, f64, i32, i32, P, P, P, P]
    lib.orc_foldin.argtypes = [i32, i32, P, i32, i64, P, P, f64, P]
    lib.orc_greedy_assign.argtypes = [i32, P, P, i32, P]
    for f in (lib.orc_group, lib.orc_validate, lib.orc_residual, lib.orc_loss,
              lib.orc_row_update, lib.orc_sals_sweep, lib.orc_foldin, lib.orc_greedy_assign):
        f.restype = ctypes.c_int
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _ptrs(arrs):
    """Array of row pointers (double** / int64_t**), kept alive by the caller."""
    return (ctypes.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class Tensor:
    """Observed entries of an N-way tensor: coords [nnz, N] int32, x [nnz] float64."""

    def __init__(self, coords, x, dims):
        self.coords = _c(coords, np.int32).reshape(-1, len(dims))
        self.x = _c(x, np.float64)
        self.dims = _c(dims, np.int64)
        self.N = len(dims)
        self.nnz = self.coords.shape[0]
        self._groups = None

    def group_of(self, n, lib=None):
        """(off, perm) of mode n, computed once by :func:`group`."""
        if self._groups is None:
            self._groups = [None] * self.N
        if self._groups[n] is None:
            self._groups[n] = group(self, n, lib)
        return self._groups[n]

    def groups(self, lib=None):
        """(off[n], perm[n]) for every mode."""
        return [self.group_of(n, lib) for n in range(self.N)]

    def row_nnz(self, lib=None):
        return [np.diff(off) for off, _ in self.groups(lib)]


def validate(t: Tensor, lib=None) -> int:
    lib = lib or load()
    return lib.orc_validate(t.N, _p(t.dims), t.nnz, _p(t.coords))


def group(t: Tensor, n: int, lib=None):
    lib = lib or load()
    off = np.zeros(int(t.dims[n]) + 1, np.int64)
    perm = np.zeros(max(t.nnz, 1), np.int64)
    st = lib.orc_group(t.N, _p(t.dims), t.nnz, _p(t.coords), n, _p(off), _p(perm))
    assert st == OK, st
    return off, perm[: t.nnz]


def residual(t: Tensor, A, lib=None) -> np.ndarray:
    lib = lib or load()
    A = [_c(a, np.float64) for a in A]
    K = A[0].shape[1]
    r = np.zeros(max(t.nnz, 1), np.float64)
    pa = _ptrs(A)
    lib.orc_residual(t.N, t.nnz, _p(t.coords), _p(t.x), K, pa, _p(r))
    return r[: t.nnz]


def loss(t: Tensor, r, A, lam, weighted=False, lib=None):
    lib = lib or load()
    A = [_c(a, np.float64) for a in A]
    r = _c(r, np.float64)
    K = A[0].shape[1]
    rn = [_c(v, np.int64) for v in t.row_nnz(lib)]
    out_l, out_r = ctypes.c_double(), ctypes.c_double()
    pa, pr = _ptrs(A), _ptrs(rn)
    lib.orc_loss(t.N, _p(t.dims), t.nnz, _p(r), K, pa, float(lam),
                 WEIGHTED if weighted else 0, pr, ctypes.byref(out_l), ctypes.byref(out_r))
    return out_l.value, out_r.value


def row_update(t: Tensor, n, i, rhat, A, S, lam, weighted=False, lib=None):
    """Eq. (4) for one row; updates A[n] in place; returns the status (0 ok, 1 pivot)."""
    lib = lib or load()
    K = A[0].shape[1]
    S = _c(S, np.int32)
    rhat = _c(rhat, np.float64)
    off, perm = t.group_of(n, lib)
    pa = _ptrs(A)
    return lib.orc_row_update(t.N, n, int(i), _p(t.coords), _p(rhat), K, pa, _p(S), len(S),
                              float(lam), WEIGHTED if weighted else 0, _p(off), _p(perm))


def sals_sweep(t: Tensor, A, r, C, lam, T_in=1, col_order=None, weighted=False, lib=None):
    """Algorithm 1, one outer iteration.  A (list of float64 [I_n, K]) and r are updated
    in place.  Returns the number of rows left unchanged by a non-positive pivot."""
    lib = lib or load()
    for a in A:
        assert a.dtype == np.float64 and a.flags.c_contiguous
    assert r.dtype == np.float64 and r.flags.c_contiguous
    K = A[0].shape[1]
    order = np.arange(K, dtype=np.int32) if col_order is None else _c(col_order, np.int32)
    offs = [g[0] for g in t.groups(lib)]
    perms = [g[1] for g in t.groups(lib)]
    stats = np.zeros(1, np.int64)
    pa, po, pp = _ptrs(A), _ptrs(offs), _ptrs(perms)
    st = lib.orc_sals_sweep(t.N, _p(t.dims), t.nnz, _p(t.coords), K, pa, _p(r), int(C),
                            float(lam), int(T_in), WEIGHTED if weighted else 0, _p(order),
                            po, pp, _p(stats))
    assert st == OK, st
    return int(stats[0])


def foldin(A, mode, other, x, lam, lib=None):
    """Eq. (2) solve for a new row of `mode`; other is [m, N-1] int32 (other modes in
    increasing order).  Returns (row float64[K], status)."""
    lib = lib or load()
    A = [_c(a, np.float64) for a in A]
    N, K = len(A), A[0].shape[1]
    other = _c(other, np.int32).reshape(-1, N - 1)
    x = _c(x, np.float64)
    out = np.zeros(K, np.float64)
    pa = _ptrs(A)
    st = lib.orc_foldin(N, K, pa, int(mode), other.shape[0], _p(other), _p(x), float(lam),
                        _p(out))
    return out, st


def greedy_assign(dims, row_nnz, M, lib=None):
    """Algorithm 3: machine of every row of every mode."""
    lib = lib or load()
    dims = _c(dims, np.int64)
    rn = [_c(v, np.int64) for v in row_nnz]
    out = [np.zeros(max(int(d), 1), np.int32) for d in dims]
    pr, po = _ptrs(rn), _ptrs(out)
    st = lib.orc_greedy_assign(len(dims), _p(dims), pr, int(M), po)
    assert st == OK, st
    return [o[: int(d)] for o, d in zip(out, dims)]

