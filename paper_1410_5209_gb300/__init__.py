"""Python binding of the GB300 SALS / CDTF library (C ABI in include/tf_sals.h).

Argument marshalling only: every step of the method runs in the CUDA kernels of
``libtfsals.so``.  There is no CPU fallback; if the shared library is missing or was
built for another machine, importing works but the first call raises
:class:`LibraryMissing` (build it with ``python -m paper_1410_5209_gb300.build``).
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtfsals.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "tf_sals.h")
SERVER_HEADER = os.path.join(os.path.dirname(_HERE), "include", "tf_server.h")

OK, EINVAL, ERANGE, EDUP, ENOMEM, ECUDA, ETIMEOUT, EBUSY = range(8)
STATUS_NAMES = ["TF_OK", "TF_EINVAL", "TF_ERANGE", "TF_EDUP", "TF_ENOMEM", "TF_ECUDA",
                "TF_ETIMEOUT", "TF_EBUSY"]
F32, F64 = 0, 1
INPUT_DEVICE = 1
LAYOUT_FIELD_SORTS = 2   # tf_create: per-mode sorts of gathered coordinates
WEIGHTED_LAMBDA = 1
SCHED_LPT, SCHED_GREEDY, SCHED_SEQ, SCHED_RAN = 0, 1, 2, 3


class LibraryMissing(RuntimeError):
    pass


class TFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


class Item(ctypes.Structure):
    _fields_ = [("begin", ctypes.c_int64), ("len", ctypes.c_int32), ("row", ctypes.c_int32),
                ("slot", ctypes.c_int32), ("bin", ctypes.c_int32)]


ITEM_DTYPE = np.dtype([("begin", np.int64), ("len", np.int32), ("row", np.int32),
                       ("slot", np.int32), ("bin", np.int32)])

_lib = None


def load():
    """Load libtfsals.so (no automatic build: build() is explicit)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise LibraryMissing(f"{LIB_PATH} not built; run python -m paper_1410_5209_gb300.build")
    lib = ctypes.CDLL(LIB_PATH)
    P, i32, i64, u32, u64 = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint32,
                             ctypes.c_uint64)
    f64 = ctypes.c_double
    sig = {
        "tf_create": [P, P, i32, P, i32, i64, i32, u64, P, u32, P],
        "tf_destroy": [P],
        "tf_last_error": [P],
        "tf_sync": [P],
        "tf_set_factors": [P, i32, P],
        "tf_get_factors": [P, i32, P],
        "tf_sals_sweep": [P, i32, f64, i32],
        "tf_sals_sweep_order": [P, i32, f64, i32, P],
        "tf_sals_sweep_ex": [P, i32, f64, i32, P, u32],
        "tf_default_order": [P, i32, i32, P],
        "tf_loss": [P, f64, u32, P, P],
        "tf_loss_noalloc": [P, f64, u32, P, P],
        "tf_foldin": [P, i32, P, P, i64, f64, P],
        "tf_predict": [P, P, i64, P, u32],
        "tf_foldin_batch": [P, i32, i32, P, P, P, f64, P, P],
        "tf_get_grouping": [P, i32, P, P],
        "tf_get_residual": [P, P],
        "tf_get_counters": [P, P],
        "tf_set_schedule": [P, i32, i32],
        "tf_set_kernel_path": [P, i32],
        "tf_set_pass_cache": [P, i32, i32, i32],
        "tf_set_sm_limit": [P, i32],
        "tf_set_precision": [P, i32],
        "tf_device_peaks": [P, P, P],
        "tf_set_stream": [P, P],
        "tf_profile": [P, i32],
        "tf_get_profile": [P, P, P],
        "tf_get_launch_trace": [P, i64, P, P, P, P],
        "tf_assign_rows": [i32, i32, P, P, i32, u64, P],
        "tf_plan_mode": [P, i64, i32, i64, i32, u64, P, i64, P, P, P],
        "tf_version": [],
        "tf_get_shape": [P, P, P, P],
        "tf_set_graphs": [P, i32],
        "tf_set_solve": [P, i32, f64],
        "tf_solve_info": [P, P],
        "tf_autotune": [P, P, i32, P, i32, f64, i32, u32, P, P, P],
        "tf_graph_info": [P, P, P],
        "tf_get_stream": [P, P],
        "tf_estimate_bytes": [P, i32, i64, i32, i32, i32, u32, i32, P],
        "tf_pool_usage": [P, P, P, i32],
        "tf_pool_trim": [i64],
        "tf_server_create": [P, P, P],
        "tf_server_destroy": [P],
        "tf_server_last_error": [P],
        "tf_server_submit_job": [P, P, P],
        "tf_server_job_info": [P, i64, P],
        "tf_server_wait_job": [P, i64, f64, P],
        "tf_server_job_factors": [P, i64, i32, P],
        "tf_server_release_job": [P, i64],
        "tf_server_submit_foldin": [P, i32, P, P, i64, f64, P],
        "tf_server_wait_foldin": [P, i64, f64, P, P, P],
        "tf_server_get_stats": [P, P],
        "tf_server_plan_admission": [i32, P, P, i64, i64, i32, i32, P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.tf_destroy.restype = None
    lib.tf_last_error.restype = ctypes.c_char_p
    lib.tf_version.restype = ctypes.c_char_p
    lib.tf_server_destroy.restype = None
    lib.tf_server_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def declared_symbols(headers=(HEADER, SERVER_HEADER)):
    """Names of the functions declared in the public headers."""
    names = set()
    for h in ([headers] if isinstance(headers, str) else headers):
        txt = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names.update(re.findall(r"\b(tf_[a-z_0-9]+)\s*\(", txt))
    return sorted(names)


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _tensor_ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _is_cuda_tensor(x):
    return type(x).__module__.startswith("torch") and getattr(x, "is_cuda", False)


def _np_dtype(dtype):
    return np.float32 if dtype == F32 else np.float64


class Factorization:
    """A tensor resident on the GPU together with its factor matrices.

    coords [nnz, N] int32 and values [nnz] as numpy arrays (host) or, with
    device_input=True, as CUDA torch tensors.  dtype F32 or F64 selects the device
    arithmetic.  stream: a cudaStream_t handle as int (None = default stream).
    field_sorts=True builds the layout by per-mode sorts of gathered coordinates
    (TF_LAYOUT_FIELD_SORTS) instead of packed keys; the layout is the same."""

    def __init__(self, coords, values, dims, K, seed=0, dtype=F32, stream=None,
                 device_input=False, field_sorts=False):
        self._lib = load()
        self.dims = [int(d) for d in dims]
        self.N = len(self.dims)
        self.K = int(K)
        self.dtype = dtype
        self.npdt = _np_dtype(dtype)
        dims_a = np.asarray(self.dims, np.int64)
        ctx = ctypes.c_void_p()
        if device_input:
            import torch
            coords = coords.to(torch.int32).contiguous()
            values = values.to(torch.float32 if dtype == F32 else torch.float64).contiguous()
            nnz = int(coords.shape[0])
            cp, vp = _tensor_ptr(coords), _tensor_ptr(values)
            flags = INPUT_DEVICE
            keep = (coords, values)
        else:
            coords = np.ascontiguousarray(coords, np.int32).reshape(-1, self.N)
            values = np.ascontiguousarray(values, self.npdt)
            nnz = int(coords.shape[0])
            cp, vp = _ptr(coords), _ptr(values)
            flags = 0
            keep = (coords, values)
        self.nnz = nnz
        if field_sorts:
            flags |= LAYOUT_FIELD_SORTS
        st = self._lib.tf_create(cp, vp, int(dtype), _ptr(dims_a), self.N, nnz, self.K,
                                 ctypes.c_uint64(seed), ctypes.c_void_p(stream or 0), flags,
                                 ctypes.byref(ctx))
        del keep
        if st != OK:
            raise TFError(st, self._lib.tf_last_error(None).decode())
        self._ctx = ctx

    # -- plumbing
    def _check(self, st):
        if st != OK:
            raise TFError(st, self._lib.tf_last_error(self._ctx).decode())

    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.tf_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._ctx

    # -- the method
    def sweep(self, C, lam, T_in=1, order=None, weighted=False):
        o = None if order is None else np.ascontiguousarray(order, np.int32)
        self._check(self._lib.tf_sals_sweep_ex(self._ctx, int(C), float(lam), int(T_in),
                                               _ptr(o), WEIGHTED_LAMBDA if weighted else 0))

    def loss(self, lam, weighted=False):
        l, r = ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.tf_loss(self._ctx, float(lam), WEIGHTED_LAMBDA if weighted else 0,
                                      ctypes.byref(l), ctypes.byref(r)))
        return l.value, r.value

    def loss_noalloc(self, lam, weighted=False):
        """As loss(), through tf_loss_noalloc: no device allocation, fixed-size scratch."""
        l, r = ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.tf_loss_noalloc(self._ctx, float(lam),
                                              WEIGHTED_LAMBDA if weighted else 0,
                                              ctypes.byref(l), ctypes.byref(r)))
        return l.value, r.value

    def foldin_batch(self, mode, requests, lam):
        """Fold-in of many requests [(other [m][N-1], values [m])] in one batch: returns
        (rows [n][K], status [n]) with status 0 ok, 1 bad index, 2 bad pivot."""
        n = len(requests)
        offs = np.zeros(n + 1, np.int64)
        for r, (o, _) in enumerate(requests):
            offs[r + 1] = offs[r] + len(o)
        other = np.ascontiguousarray(np.concatenate([np.asarray(o, np.int32).reshape(-1, self.N - 1)
                                                     for o, _ in requests]) if n else
                                     np.zeros((0, self.N - 1), np.int32), np.int32)
        vals = np.ascontiguousarray(np.concatenate([np.asarray(v) for _, v in requests]) if n else
                                    np.zeros(0), self.npdt)
        out = np.zeros((n, self.K), self.npdt)
        status = np.zeros(n, np.int32)
        self._check(self._lib.tf_foldin_batch(self._ctx, int(mode), n, _ptr(offs), _ptr(other),
                                              _ptr(vals), float(lam), _ptr(out), _ptr(status)))
        return out, status

    def predict(self, coords):
        """Model values at coordinates [m][N] (host arrays, or torch CUDA tensors)."""
        if _is_cuda_tensor(coords):
            import torch
            c = coords.to(torch.int32).contiguous()
            out = torch.empty(c.shape[0], dtype=torch.float32 if self.dtype == F32 else torch.float64,
                              device=c.device)
            self._check(self._lib.tf_predict(self._ctx, _tensor_ptr(c), int(c.shape[0]),
                                             _tensor_ptr(out), INPUT_DEVICE))
            return out
        c = np.ascontiguousarray(coords, np.int32).reshape(-1, self.N)
        out = np.zeros(c.shape[0], self.npdt)
        self._check(self._lib.tf_predict(self._ctx, _ptr(c), int(c.shape[0]), _ptr(out), 0))
        return out

    def foldin(self, mode, other, values, lam):
        other = np.ascontiguousarray(other, np.int32).reshape(-1, self.N - 1)
        values = np.ascontiguousarray(values, self.npdt)
        out = np.zeros(self.K, self.npdt)
        self._check(self._lib.tf_foldin(self._ctx, int(mode), _ptr(other), _ptr(values),
                                        int(other.shape[0]), float(lam), _ptr(out)))
        return out

    # -- state
    def factors(self, n):
        out = np.empty((self.dims[n], self.K), self.npdt)
        self._check(self._lib.tf_get_factors(self._ctx, int(n), _ptr(out)))
        return out

    def set_factors(self, n, A):
        A = np.ascontiguousarray(A, self.npdt).reshape(self.dims[n], self.K)
        self._check(self._lib.tf_set_factors(self._ctx, int(n), _ptr(A)))

    def grouping(self, n, with_perm=True):
        off = np.empty(self.dims[n] + 1, np.int64)
        perm = np.empty(max(self.nnz, 1), np.int64) if with_perm else None
        self._check(self._lib.tf_get_grouping(self._ctx, int(n), _ptr(off), _ptr(perm)))
        return off, (perm[: self.nnz] if with_perm else None)

    def residual(self):
        out = np.empty(max(self.nnz, 1), self.npdt)
        self._check(self._lib.tf_get_residual(self._ctx, _ptr(out)))
        return out[: self.nnz]

    def counters(self):
        c = np.zeros(8, np.int64)
        self._check(self._lib.tf_get_counters(self._ctx, _ptr(c)))
        keys = ["singular_rows", "sweeps", "last_sweep_launches", "items", "split_rows", "bins",
                "loss_launches", "pass_path"]
        return {k: int(v) for k, v in zip(keys, c)}

    def default_order(self, sweep, C):
        out = np.empty(self.K, np.int32)
        self._check(self._lib.tf_default_order(self._ctx, int(sweep), int(C), _ptr(out)))
        return out

    PATH_AUTO, PATH_SIMT, PATH_TMA, PATH_LEAN = 0, 1, 2, 3

    def set_kernel_path(self, path):
        self._check(self._lib.tf_set_kernel_path(self._ctx, int(path)))

    def set_sm_limit(self, sms=0):
        """Blocks of the persistent mode passes (0: one per SM); leaves SMs to other streams."""
        self._check(self._lib.tf_set_sm_limit(self._ctx, int(sms)))

    def set_pass_cache(self, max_rows=-1, pool_rows=32, warps=0):
        """Lean pass: cached rows per other mode (< 0 as fit, 0 none), staged rows per
        step, warps per block (0 default)."""
        self._check(self._lib.tf_set_pass_cache(self._ctx, int(max_rows), int(pool_rows),
                                                int(warps)))

    def set_solve(self, refine=False, cond_limit=0.0):
        """Float row solves: one FP64-residual refinement step; FP64 re-solve of rows whose
        pivot ratio is below 1 / cond_limit (0: never)."""
        self._check(self._lib.tf_set_solve(self._ctx, 1 if refine else 0, float(cond_limit)))

    def fp64_rows(self):
        n = ctypes.c_int64()
        self._check(self._lib.tf_solve_info(self._ctx, ctypes.byref(n)))
        return n.value

    def set_graphs(self, enable=True):
        """Run sweeps as CUDA graphs (captured on a shape's second sweep, then replayed)."""
        self._check(self._lib.tf_set_graphs(self._ctx, 1 if enable else 0))

    def autotune(self, C_list, P_list=(0,), lam=0.1, T_in=1, weighted=False):
        """Fastest (C, P) by one timed sweep each; state restored, best P kept.
        Returns (best_C, best_P, ms [len(P_list)][len(C_list)])."""
        cl = np.ascontiguousarray(C_list, np.int32)
        pl = np.ascontiguousarray(P_list, np.int32)
        ms = np.zeros((len(pl), len(cl)), np.float32)
        bc, bp = ctypes.c_int32(), ctypes.c_int32()
        self._check(self._lib.tf_autotune(self._ctx, _ptr(cl), len(cl), _ptr(pl), len(pl),
                                          float(lam), int(T_in),
                                          WEIGHTED_LAMBDA if weighted else 0,
                                          ctypes.byref(bc), ctypes.byref(bp), _ptr(ms)))
        return bc.value, bp.value, ms

    def graph_info(self):
        r, c = ctypes.c_int64(), ctypes.c_int64()
        self._check(self._lib.tf_graph_info(self._ctx, ctypes.byref(r), ctypes.byref(c)))
        return {"replays": r.value, "cached": c.value}

    def set_stream(self, stream):
        """Queue later work on `stream` (a cudaStream_t handle as int, or a torch stream)."""
        handle = getattr(stream, "cuda_stream", stream)
        self._check(self._lib.tf_set_stream(self._ctx, ctypes.c_void_p(handle or 0)))

    def set_precision(self, mode):
        """0: FP32-level Gram; 1: single-TF32 tensor-core Gram (wide subsets, and narrow
        ones of three-way float tensors); 2: the lean pass reads the varying mode's slice
        rows from bfloat16 copies; 3: both other modes' rows (narrow subsets of three-way
        float tensors)."""
        self._check(self._lib.tf_set_precision(self._ctx, int(mode)))

    def set_schedule(self, policy=SCHED_LPT, P=0):
        self._check(self._lib.tf_set_schedule(self._ctx, int(policy), int(P)))

    KINDS = ["pack", "mode_pass", "combine", "loss", "other", "solve"]

    def profile(self, enable=True):
        self._check(self._lib.tf_profile(self._ctx, 1 if enable else 0))

    def get_profile(self):
        n = np.zeros(len(self.KINDS), np.int64)
        ms = np.zeros(len(self.KINDS), np.float64)
        self._check(self._lib.tf_get_profile(self._ctx, _ptr(n), _ptr(ms)))
        return {k: (int(a), float(b)) for k, a, b in zip(self.KINDS, n, ms)}

    def launch_trace(self):
        """[(kind, mode, ms)] of every timed launch since profile(True)."""
        n = ctypes.c_int64()
        self._check(self._lib.tf_get_launch_trace(self._ctx, 0, ctypes.byref(n), None, None,
                                                  None))
        k = np.zeros(max(n.value, 1), np.int32)
        m = np.zeros(max(n.value, 1), np.int32)
        ms = np.zeros(max(n.value, 1), np.float32)
        self._check(self._lib.tf_get_launch_trace(self._ctx, n.value, ctypes.byref(n), _ptr(k),
                                                  _ptr(m), _ptr(ms)))
        return [(self.KINDS[a], int(b), float(c)) for a, b, c in zip(k[:n.value], m[:n.value],
                                                                    ms[:n.value])]

    def sync(self):
        self._check(self._lib.tf_sync(self._ctx))


# ---------------------------------------------------------------- host-only calls

def assign_rows(policy, dims, row_nnz, M, seed=0):
    """Row -> bin of every mode (Algorithm 3 with SCHED_GREEDY).  No GPU needed."""
    lib = load()
    dims_a = np.asarray(dims, np.int64)
    rn = [np.ascontiguousarray(v, np.int64) for v in row_nnz]
    out = [np.zeros(max(int(d), 1), np.int32) for d in dims]
    prn = (ctypes.c_void_p * len(rn))(*[a.ctypes.data for a in rn])
    pout = (ctypes.c_void_p * len(out))(*[a.ctypes.data for a in out])
    st = lib.tf_assign_rows(int(policy), len(dims), _ptr(dims_a), prn, int(M),
                            ctypes.c_uint64(seed), pout)
    if st != OK:
        raise TFError(st, "tf_assign_rows failed")
    return [o[: int(d)] for o, d in zip(out, dims)]


def plan_mode(off, P, cap=0, policy=SCHED_LPT, seed=0):
    """Work items of one mode (numpy structured array), number of partial slots, bin_ptr."""
    lib = load()
    off = np.ascontiguousarray(off, np.int64)
    I = len(off) - 1
    n_items, n_slots = ctypes.c_int64(), ctypes.c_int64()
    bin_ptr = np.zeros(P + 1, np.int64)
    st = lib.tf_plan_mode(_ptr(off), I, int(P), int(cap), int(policy), ctypes.c_uint64(seed),
                          None, 0, ctypes.byref(n_items), ctypes.byref(n_slots), None)
    if st not in (OK, ENOMEM):
        raise TFError(st, "tf_plan_mode failed")
    items = np.zeros(max(n_items.value, 1), ITEM_DTYPE)
    st = lib.tf_plan_mode(_ptr(off), I, int(P), int(cap), int(policy), ctypes.c_uint64(seed),
                          _ptr(items), n_items.value, ctypes.byref(n_items),
                          ctypes.byref(n_slots), _ptr(bin_ptr))
    if st != OK:
        raise TFError(st, "tf_plan_mode failed")
    return items[: n_items.value], n_slots.value, bin_ptr


def version():
    return load().tf_version().decode()


def device_peaks():
    """Measured FP32 FMA rates (plain, packed two-wide; TFLOP/s) and shared-memory load
    bandwidth (TB/s) of the current device (tf_device_peaks)."""
    lib = load()
    v = [ctypes.c_double() for _ in range(3)]
    st = lib.tf_device_peaks(*[ctypes.byref(x) for x in v])
    if st != OK:
        raise TFError(st, "tf_device_peaks failed")
    return {"fp32_tflops": v[0].value, "fp32x2_tflops": v[1].value, "smem_tbytes": v[2].value}


def estimate_bytes(dims, nnz, K, C_max, dtype=F32, device_input=False, num_sms=0):
    """Upper bound of a context's device memory from tf_create through sweeps with
    C <= C_max (tf_estimate_bytes); num_sms > 0 needs no GPU."""
    lib = load()
    d = np.ascontiguousarray(dims, np.int64)
    out = ctypes.c_int64()
    st = lib.tf_estimate_bytes(_ptr(d), len(d), int(nnz), int(K), int(C_max), int(dtype),
                               INPUT_DEVICE if device_input else 0, int(num_sms),
                               ctypes.byref(out))
    if st != OK:
        raise TFError(st, "tf_estimate_bytes refused the shape")
    return out.value


def pool_usage(reset_high=False):
    """(bytes in use, high-water mark, bytes held) of the library's device memory pool."""
    used, high, held = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    st = load().tf_pool_usage(ctypes.byref(used), ctypes.byref(high), ctypes.byref(held),
                              1 if reset_high else 0)
    if st != OK:
        raise TFError(st, "tf_pool_usage failed")
    return used.value, high.value, held.value


def pool_trim(keep_bytes=0):
    """Return the pool's unused device memory, keeping at most keep_bytes."""
    st = load().tf_pool_trim(int(keep_bytes))
    if st != OK:
        raise TFError(st, "tf_pool_trim failed")


# ---------------------------------------------------------------- serving (tf_server.h)

class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_int64), ("hbm_reserve", ctypes.c_int64),
                ("max_running", ctypes.c_int), ("max_batch", ctypes.c_int),
                ("max_bypass", ctypes.c_int), ("reserve_sms", ctypes.c_int)]


class JobDesc(ctypes.Structure):
    _fields_ = [("coords", ctypes.c_void_p), ("values", ctypes.c_void_p),
                ("dims", ctypes.c_void_p), ("N", ctypes.c_int), ("nnz", ctypes.c_int64),
                ("K", ctypes.c_int), ("dtype", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("C", ctypes.c_int), ("lam", ctypes.c_double), ("T_in", ctypes.c_int),
                ("sweeps", ctypes.c_int), ("sweep_flags", ctypes.c_uint32),
                ("col_orders", ctypes.c_void_p)]


class JobInfo(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int), ("status", ctypes.c_int),
                ("sweeps_done", ctypes.c_int), ("loss", ctypes.c_double),
                ("rmse", ctypes.c_double), ("bytes", ctypes.c_int64),
                ("queued_s", ctypes.c_double), ("started_s", ctypes.c_double),
                ("finished_s", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in (
        "jobs_queued", "jobs_running", "jobs_done", "jobs_failed", "foldins_done",
        "foldin_batches", "foldin_max_batch", "bytes_admitted", "bytes_admitted_peak",
        "running_peak")]


JOB_QUEUED, JOB_RUNNING, JOB_DONE, JOB_FAILED = range(4)


def _struct_dict(s):
    return {k: getattr(s, k) for k, _ in s._fields_}


class Server:
    """Serving loop (include/tf_server.h): factorisation jobs admitted against free device
    memory, each on its own stream and host thread, and continuously batched fold-in
    requests against `model` (a Factorization, owned by the server until close())."""

    def __init__(self, model=None, hbm_budget=0, hbm_reserve=0, max_running=0, max_batch=0,
                 max_bypass=0, reserve_sms=0):
        self._lib = load()
        cfg = ServerConfig(int(hbm_budget), int(hbm_reserve), int(max_running),
                           int(max_batch), int(max_bypass), int(reserve_sms))
        self._srv = ctypes.c_void_p()
        self.model = model
        st = self._lib.tf_server_create(ctypes.byref(cfg), model._ctx if model else None,
                                        ctypes.byref(self._srv))
        if st != OK:
            raise TFError(st, self._lib.tf_server_last_error(None).decode())
        self._dtype = model.dtype if model else F32
        self._K = model.K if model else 0
        self._keep = {}

    def _check(self, st, what):
        if st != OK:
            raise TFError(st, f"{what}: {self._lib.tf_server_last_error(self._srv).decode()}")

    def close(self):
        if self._srv:
            self._lib.tf_server_destroy(self._srv)
            self._srv = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit_job(self, coords, values, dims, K, C, lam, sweeps, T_in=1, seed=0, dtype=F32,
                   orders=None, weighted=False):
        c = np.ascontiguousarray(coords, np.int32)
        x = np.ascontiguousarray(values, _np_dtype(dtype))
        d = np.ascontiguousarray(dims, np.int64)
        o = None if orders is None else np.ascontiguousarray(orders, np.int32)
        desc = JobDesc(c.ctypes.data, x.ctypes.data, d.ctypes.data, len(d), len(x), int(K),
                       int(dtype), ctypes.c_uint64(seed).value, int(C), float(lam), int(T_in),
                       int(sweeps), WEIGHTED_LAMBDA if weighted else 0,
                       o.ctypes.data if o is not None else None)
        jid = ctypes.c_int64()
        self._check(self._lib.tf_server_submit_job(self._srv, ctypes.byref(desc),
                                                   ctypes.byref(jid)), "submit_job")
        self._keep[jid.value] = (tuple(int(v) for v in d), int(K), dtype)
        return jid.value

    def job_info(self, jid):
        info = JobInfo()
        self._check(self._lib.tf_server_job_info(self._srv, int(jid), ctypes.byref(info)),
                    "job_info")
        return _struct_dict(info)

    def wait_job(self, jid, timeout=600.0):
        """Job info once done or failed; raises TFError(ETIMEOUT) if still running."""
        info = JobInfo()
        self._check(self._lib.tf_server_wait_job(self._srv, int(jid), float(timeout),
                                                 ctypes.byref(info)), "wait_job")
        return _struct_dict(info)

    def job_factors(self, jid, n):
        dims, K, dtype = self._keep[jid]
        out = np.empty((dims[n], K), _np_dtype(dtype))
        self._check(self._lib.tf_server_job_factors(self._srv, int(jid), int(n), _ptr(out)),
                    "job_factors")
        return out

    def release_job(self, jid):
        self._check(self._lib.tf_server_release_job(self._srv, int(jid)), "release_job")
        self._keep.pop(jid, None)

    def submit_foldin(self, mode, other, values, lam):
        o = np.ascontiguousarray(other, np.int32)
        v = np.ascontiguousarray(values, _np_dtype(self._dtype))
        rid = ctypes.c_int64()
        self._check(self._lib.tf_server_submit_foldin(self._srv, int(mode), _ptr(o), _ptr(v),
                                                      len(v), float(lam), ctypes.byref(rid)),
                    "submit_foldin")
        return rid.value

    def wait_foldin(self, rid, timeout=60.0):
        """(row [K], status, latency seconds)."""
        row = np.empty(self._K, _np_dtype(self._dtype))
        status, lat = ctypes.c_int32(), ctypes.c_double()
        self._check(self._lib.tf_server_wait_foldin(self._srv, int(rid), float(timeout),
                                                    _ptr(row), ctypes.byref(status),
                                                    ctypes.byref(lat)), "wait_foldin")
        return row, status.value, lat.value

    def stats(self):
        s = ServerStats()
        self._check(self._lib.tf_server_get_stats(self._srv, ctypes.byref(s)), "stats")
        return _struct_dict(s)


def plan_admission(need, bypassed, room, budget_left=-1, slots=1 << 30, max_bypass=8):
    """The scheduler's admission decision (host only): (admit flags, updated pass counts)."""
    need = np.ascontiguousarray(need, np.int64)
    byp = np.array(bypassed, np.int32, copy=True)
    admit = np.zeros(len(need), np.int32)
    load().tf_server_plan_admission(len(need), _ptr(need), _ptr(byp), int(room),
                                    int(budget_left), int(slots), int(max_bypass), _ptr(admit))
    return admit.astype(bool), byp
