"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the tests, the benchmark and both sides of every parity
check (the CUDA path and the CPU oracle).  It holds no arithmetic of the method
itself: only counter-based random numbers, coordinate sampling, de-duplication and
the evaluation of a ground-truth CP model that produces the observed values.

Randomness is counter based: splitmix64 (Steele, Lea and Flood, OOPSLA 2014) applied
to ``key(seed, stream) + (index + 1) * golden``.  Every array is a pure function of
its seed, independent of chunking, threads and device.  Integer outputs
(coordinates, permutations, column orders) are bit-identical on CPU and CUDA; the
floating-point values go through log/cos/sqrt and may differ in the last ulp
between devices, which never matters because both sides of a parity check always
receive the very same arrays.

Workload recipes.  The paper describes its synthetic tensors only by scale (Table 5,
generated as in the Hogwild "Jumbo" set) and evaluates on three rating datasets
(Table 4) that are not available here; these seeded tensors stand in for them:

* :func:`parity_3way`  1000 x 1000 x 100, 1e5 distinct uniform coordinates, rank-10 CP
  ground truth with factor entries N(0, 1/10), noise N(0, 0.1^2), float64.
* :func:`skewed_3way`  1e5 x 1e5 x 1e3, 1e8 distinct coordinates; modes 1-2 Zipf(1.1)
  (ranks mapped through a seeded permutation), mode 3 uniform; rank-50 ground truth
  (factor std 50^(-1/6), unit signal variance) + N(0, 0.1^2), float32.
"""
from __future__ import annotations

import math
import numpy as np
import torch

_MASK64 = (1 << 64) - 1


def _s64(u: int) -> int:
    """uint64 constant -> the int64 with the same bits."""
    u &= _MASK64
    return u - (1 << 64) if u >= (1 << 63) else u


_G = _s64(0x9E3779B97F4A7C15)
_M1 = _s64(0xBF58476D1CE4E5B9)
_M2 = _s64(0x94D049BB133111EB)


def _lsr(z: torch.Tensor, k: int) -> torch.Tensor:
    """Logical right shift of int64 bit patterns."""
    return (z >> k) & ((1 << (64 - k)) - 1)


def _mix(z: torch.Tensor) -> torch.Tensor:
    """splitmix64 finaliser on int64 tensors holding uint64 bit patterns (wrapping)."""
    z = z ^ _lsr(z, 30)
    z = z * _M1
    z = z ^ _lsr(z, 27)
    z = z * _M2
    return z ^ _lsr(z, 31)


def _mix_int(z: int) -> int:
    z &= _MASK64
    z ^= z >> 30
    z = (z * 0xBF58476D1CE4E5B9) & _MASK64
    z ^= z >> 27
    z = (z * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def _key(seed: int, stream: int) -> int:
    s = (seed * 0x9E3779B97F4A7C15 + stream * 0xD1B54A32D192ED03) & _MASK64
    return _s64(_mix_int(s + 0x9E3779B97F4A7C15))


def bits64(seed, stream, start, n, device="cpu") -> torch.Tensor:
    """int64 tensor holding the uint64 outputs for counters start..start+n-1."""
    i = torch.arange(start + 1, start + n + 1, dtype=torch.int64, device=device)
    return _mix(_key(seed, stream) + i * _G)


def bits64_reference(seed, stream, index) -> int:
    """Pure-Python value of one counter (for cross-checking the tensor version)."""
    k = _key(seed, stream) & _MASK64
    return _mix_int(k + (index + 1) * 0x9E3779B97F4A7C15)


def uniform01(seed, stream, start, n, device="cpu"):
    """float64 in [0, 1) from the top 53 bits."""
    return _lsr(bits64(seed, stream, start, n, device), 11).double() * (2.0 ** -53)


def normal(seed, stream, start, n, std=1.0, device="cpu"):
    """Box-Muller normals (cosine branch), one per counter, float64."""
    u1 = uniform01(seed, 2 * stream + 0x1000, start, n, device)
    u2 = uniform01(seed, 2 * stream + 0x1001, start, n, device)
    return std * torch.sqrt(-2.0 * torch.log1p(-u1)) * torch.cos(2.0 * math.pi * u2)


def uniform_int(seed, stream, start, n, high, device="cpu"):
    u = uniform01(seed, stream, start, n, device)
    return torch.clamp((u * high).long(), max=high - 1)


def permutation(seed, stream, n, device="cpu"):
    """Seeded permutation of range(n): stable argsort of random 63-bit keys."""
    k = _lsr(bits64(seed, stream, 0, n, device), 1)
    return torch.sort(k, stable=True).indices


class Zipf:
    """Zipf(s) over {0..I-1} by inverse CDF; rank r is mapped to row perm[r]."""

    def __init__(self, I, s, seed, stream, device="cpu"):
        w = np.arange(1, I + 1, dtype=np.float64) ** (-s)
        cdf = np.cumsum(w) / w.sum()   # numpy on the host: identical on every device
        cdf[-1] = 1.0
        self.cdf = torch.from_numpy(cdf).to(device)
        self.perm = permutation(seed, stream + 0x777, I, device)
        self.I = I

    def sample(self, u):
        r = torch.searchsorted(self.cdf, u, right=True)
        return self.perm[torch.clamp(r, max=self.I - 1)]


def distinct_coords(dims, nnz, seed, modes=None, zipf_s=1.1, stream=100, device="cpu"):
    """nnz distinct coordinates [nnz, N] int32, in draw order of first occurrence.

    modes[n] is "uniform" or "zipf".  Batches of draws are appended until nnz distinct
    tuples exist; a draw equal to an earlier one is dropped."""
    N = len(dims)
    modes = modes or ["uniform"] * N
    samplers = [Zipf(int(dims[n]), zipf_s, seed, stream + n, device)
                if modes[n] == "zipf" else None for n in range(N)]
    # modes grouped so that each group's packed index fits in 62 bits (one group unless
    # the tensor has more than 2^62 cells)
    groups, cur, prod = [], [], 1
    for n in range(N):
        if cur and prod * int(dims[n]) >= 2 ** 62:
            groups.append(cur)
            cur, prod = [], 1
        cur.append(n)
        prod *= int(dims[n])
    groups.append(cur)
    mult = [1] * N
    for g in groups:
        for k in range(len(g) - 2, -1, -1):
            mult[g[k]] = mult[g[k + 1]] * int(dims[g[k + 1]])

    def draw(start, n):
        cols = []
        for m in range(N):
            if samplers[m] is None:
                cols.append(uniform_int(seed, stream + 10 + m, start, n, int(dims[m]), device))
            else:
                cols.append(samplers[m].sample(uniform01(seed, stream + 10 + m, start, n,
                                                         device)))
        return torch.stack(cols, dim=1).to(torch.int32)

    def keys(c, g):
        k = torch.zeros(c.shape[0], dtype=torch.int64, device=device)
        for m in g:
            k += c[:, m].long() * mult[m]
        return k

    have = torch.zeros((0, N), dtype=torch.int32, device=device)
    start, need = 0, nnz
    while True:
        n_draw = int(need * 1.15) + 1024
        c = draw(start, n_draw)
        start += n_draw
        allc = torch.cat([have, c]) if have.shape[0] else c
        if len(groups) == 1:
            ks, idx = torch.sort(keys(allc, groups[0]), stable=True)
            first = torch.ones_like(ks, dtype=torch.bool)
            first[1:] = ks[1:] != ks[:-1]
        else:  # stable sorts from the least significant group; equal tuples stay in draw order
            idx = torch.arange(allc.shape[0], device=device)
            for g in reversed(groups):
                _, o = torch.sort(keys(allc, g)[idx], stable=True)
                idx = idx[o]
            first = torch.ones(idx.shape[0], dtype=torch.bool, device=device)
            same = torch.ones(idx.shape[0] - 1, dtype=torch.bool, device=device)
            for g in groups:
                kg = keys(allc, g)[idx]
                same &= kg[1:] == kg[:-1]
            first[1:] = ~same
            ks = None
        keep = torch.sort(idx[first]).values
        del ks, idx, first
        if keep.numel() >= nnz:
            return allc[keep[:nnz]].contiguous()
        rate = keep.numel() / allc.shape[0]
        have = allc[keep]
        need = int((nnz - keep.numel()) / max(rate, 0.05))


def cp_values(coords, factors, chunk=1 << 22):
    """x_e = sum_r prod_n U_n[i_n, r] for the ground-truth factors (no noise)."""
    nnz = coords.shape[0]
    out = torch.empty(nnz, dtype=factors[0].dtype, device=coords.device)
    for s in range(0, nnz, chunk):
        c = coords[s:s + chunk].long()
        p = factors[0][c[:, 0]].clone()
        for n in range(1, len(factors)):
            p *= factors[n][c[:, n]]
        out[s:s + chunk] = p.sum(dim=1)
    return out


class Problem:
    """One synthetic tensor, plus its initial factors and per-sweep column orders.

    ``coords`` [nnz, N] int32 and ``x`` [nnz] live on ``device``; :meth:`numpy` gives
    host copies (what the oracle and the host-buffer C-ABI calls take)."""

    def __init__(self, dims, coords, x, K, seed, truth=None):
        self.dims = [int(d) for d in dims]
        self.N = len(dims)
        self.coords = coords
        self.x = x
        self.K = K
        self.seed = seed
        self.truth = truth

    @property
    def nnz(self):
        return int(self.coords.shape[0])

    @property
    def device(self):
        return self.coords.device

    def numpy(self):
        return self.coords.cpu().numpy(), self.x.cpu().numpy()

    def init_factors(self, dtype=torch.float64, device=None):
        """Algorithm 1 initialisation: A^(1) = 0 and the other modes i.i.d. normal with
        std K^(-1/(2N)) (the paper says only "random values")."""
        device = device or self.device
        std = float(self.K) ** (-1.0 / (2 * self.N))
        A = [torch.zeros((self.dims[0], self.K), dtype=dtype, device=device)]
        for n in range(1, self.N):
            cnt = self.dims[n] * self.K
            A.append(normal(self.seed, 500 + n, 0, cnt, std, device).reshape(-1, self.K)
                     .to(dtype))
        return A

    def column_order(self, sweep, C):
        """Columns chosen without replacement (Algorithm 1): a seeded permutation per
        sweep for C > 1, the identity for CDTF (C = 1, Section 3.1).  Host int32."""
        if C == 1:
            return np.arange(self.K, dtype=np.int32)
        return permutation(self.seed, 900 + sweep, self.K).numpy().astype(np.int32)


def make_problem(dims, nnz, rank, K, seed, modes=None, factor_std=None, noise_std=0.1,
                 dtype=torch.float64, zipf_s=1.1, device="cpu"):
    dims = [int(d) for d in dims]
    N = len(dims)
    nnz = min(int(nnz), int(0.5 * float(np.prod(np.array(dims, dtype=np.float64)))))
    coords = distinct_coords(dims, nnz, seed, modes, zipf_s, device=device)
    std = factor_std if factor_std is not None else float(rank) ** (-1.0 / (2 * N))
    truth = [normal(seed, 300 + n, 0, dims[n] * rank, std, device)
             .reshape(dims[n], rank).to(dtype) for n in range(N)]
    x = cp_values(coords, truth)
    if noise_std:
        x += normal(seed, 400, 0, x.shape[0], noise_std, device).to(dtype)
    return Problem(dims, coords, x, K, seed, truth)


def parity_3way(seed=1, nnz=100_000, dims=(1000, 1000, 100), K=10, device="cpu"):
    """Parity workload: rank-10 CP + N(0, 0.1^2), factor entries N(0, 1/10), float64."""
    return make_problem(dims, nnz, 10, K, seed, factor_std=1.0 / math.sqrt(10.0),
                        noise_std=0.1, dtype=torch.float64, device=device)


def skewed_3way(seed=2, nnz=100_000_000, dims=(100_000, 100_000, 1_000), K=100,
                device="cpu"):
    """Skewed workload: Zipf(1.1) modes 1-2, uniform mode 3, rank-50 CP + noise, float32."""
    return make_problem(dims, nnz, 50, K, seed, modes=["zipf", "zipf", "uniform"],
                        noise_std=0.1, dtype=torch.float32, device=device)


def foldin_requests(p, count, seed, mode=0, m_min=10, m_max=10_000, noise_std=0.1,
                    zipf_s=1.1, modes=("zipf", "zipf", "uniform")):
    """Fold-in requests against a problem's ground truth: each a new slice of `mode`
    with m log-uniform in [m_min, m_max] distinct entries whose other-mode indices are
    drawn like the tensor's (Zipf / uniform per mode), values from a fresh ground-truth
    row of the same law plus noise.  Returns [(other [m][N-1] int32, x [m])] on the host."""
    N = p.N
    rank = p.truth[0].shape[1]
    std = float(rank) ** (-1.0 / (2 * N))
    others = [l for l in range(N) if l != mode]
    samplers = {l: Zipf(int(p.dims[l]), zipf_s, seed, 700 + l) for l in others
                if modes[l] == "zipf"}
    truth = [t.to("cpu", torch.float64) for t in p.truth]
    u = uniform01(seed, 710, 0, count)
    ms = torch.exp(math.log(m_min) + u * (math.log(m_max) - math.log(m_min))).long()
    out = []
    base = 0
    for q in range(count):
        m = int(ms[q])
        row = normal(seed, 720, q * rank, rank, std)
        cols = []
        for l in others:
            n_draw = 4 * m + 64
            if l in samplers:
                cols.append(samplers[l].sample(uniform01(seed, 730 + l, base, n_draw)))
            else:
                cols.append(uniform_int(seed, 730 + l, base, n_draw, int(p.dims[l])))
        base += 4 * m + 64
        c = torch.stack(cols, 1)
        key = c[:, 0].clone()
        for k in range(1, c.shape[1]):
            key = key * int(p.dims[others[k]]) + c[:, k]
        _, first = np.unique(key.numpy(), return_index=True)
        c = c[torch.from_numpy(np.sort(first))[:m]]
        val = row.clone().expand(c.shape[0], rank).clone()
        for k, l in enumerate(others):
            val *= truth[l][c[:, k]]
        x = val.sum(1) + normal(seed, 740, q * m_max, c.shape[0], noise_std)
        out.append((c.to(torch.int32).numpy(), x.numpy()))
    return out


def concat_block_diagonal(problems, K, seed):
    """Independent tensors (same N) as one block-diagonal tensor: tensor b's indices of
    mode n are shifted by the summed mode-n lengths of the tensors before it, so no
    entry couples two tensors.  Returns (Problem, row_offsets [count + 1][N],
    entry_offsets [count + 1])."""
    N = problems[0].N
    count = len(problems)
    row_off = np.zeros((count + 1, N), np.int64)
    ent_off = np.zeros(count + 1, np.int64)
    for b, q in enumerate(problems):
        row_off[b + 1] = row_off[b] + np.asarray(q.dims, np.int64)
        ent_off[b + 1] = ent_off[b] + q.nnz
    dev = problems[0].coords.device
    shift = torch.from_numpy(row_off[:-1].astype(np.int32)).to(dev)
    coords = torch.cat([q.coords + shift[b] for b, q in enumerate(problems)])
    x = torch.cat([q.x for q in problems])
    truth = None
    if all(q.truth is not None for q in problems) and \
            len({q.truth[0].shape[1] for q in problems}) == 1:
        truth = [torch.cat([q.truth[n] for q in problems]) for n in range(N)]
    p = Problem([int(d) for d in row_off[-1]], coords, x, K, seed, truth)
    return p, row_off, ent_off


def batched(count, seed=4, dims_range=(50, 5000), nnz_range=(1_000, 1_000_000), rank=16,
            K=16, dtype=torch.float32, device="cpu"):
    """Many small 3-way tensors: per tensor, mode lengths and entry counts log-uniform in
    the given ranges (entries capped at half the cells), rank-`rank` ground truth with
    unit signal variance plus N(0, 0.1^2) noise; concatenated block-diagonally."""
    u = uniform01(seed, 800, 0, 4 * count).reshape(count, 4)
    lo_d, hi_d = math.log(dims_range[0]), math.log(dims_range[1])
    lo_n, hi_n = math.log(nnz_range[0]), math.log(nnz_range[1])
    probs = []
    for b in range(count):
        dims = [int(math.exp(lo_d + float(u[b, n]) * (hi_d - lo_d))) for n in range(3)]
        nnz = int(math.exp(lo_n + float(u[b, 3]) * (hi_n - lo_n)))
        probs.append(make_problem(dims, nnz, rank, K, seed * 100_003 + b, dtype=dtype,
                                  device=device))
    return concat_block_diagonal(probs, K, seed)


def small(seed, dims, nnz, rank, K, noise_std=0.1, modes=None, dtype=torch.float64,
          device="cpu"):
    """Small tensors for tests (any shape)."""
    return make_problem(dims, nnz, rank, K, seed, modes=modes, noise_std=noise_std,
                        dtype=dtype, device=device)
