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


@pytest.mark.gpu
def test_many_tensors_fp32_graph_replayed():
    """64 small FP32 tensors of uneven shapes batched as one block-diagonal tensor, the
    sweeps captured into a CUDA graph and replayed (second sweep captured, third and
    fourth replayed), against 64 separate FP64 oracle runs from the same float-rounded
    inputs: each tensor's factors within FP32-level error and its training RMSE within
    1e-3 of the oracle's."""
    from paper_1410_5209_gb300 import build
    build.build()
    rng = np.random.default_rng(11)
    probs = []
    for b in range(64):
        dims = tuple(int(v) for v in rng.integers(8, 60, 3))
        nnz = int(min(rng.integers(200, 3_000), dims[0] * dims[1] * dims[2] // 2))
        probs.append(synth.small(300 + b, dims, nnz, 3, 16))
    K, C = 16, 4
    p, row_off, ent_off = synth.concat_block_diagonal(probs, K, seed=9)
    c, x = p.numpy()
    x = x.astype(np.float32).astype(np.float64)
    A = [a.numpy().astype(np.float32).astype(np.float64) for a in p.init_factors()]
    import torch
    stream = torch.cuda.Stream()   # graphs are captured on a stream of the caller's
    f = tf.Factorization(c, x, p.dims, K, dtype=tf.F32, stream=stream.cuda_stream)
    for n in range(3):
        f.set_factors(n, A[n])
    f.set_graphs(True)
    parts = [_split(A, row_off, b) for b in range(len(probs))]
    tb = []
    for b, q in enumerate(probs):
        tb.append(oracle.Tensor(q.numpy()[0], x[ent_off[b]:ent_off[b + 1]], q.dims))
    rb = [oracle.residual(tb[b], parts[b]) for b in range(len(probs))]
    for s in range(4):
        order = p.column_order(s, C)
        f.sweep(C, 0.3, 1, order)
        for b in range(len(probs)):
            oracle.sals_sweep(tb[b], parts[b], rb[b], C, 0.3, 1, order)
    gi = f.graph_info()
    assert gi["replays"] == 2 and gi["cached"] == 1   # sweeps 1-2 eager, 3 captured, 4 replayed
    got = [f.factors(n).astype(np.float64) for n in range(3)]
    res = f.residual().astype(np.float64)
    for b in range(len(probs)):
        for n in range(3):
            seg = got[n][row_off[b, n]:row_off[b + 1, n]]
            ref = parts[b][n]
            assert np.linalg.norm(seg - ref) <= 2e-4 * max(np.linalg.norm(ref), 1e-30), (b, n)
        rmse = np.sqrt(np.mean(res[ent_off[b]:ent_off[b + 1]] ** 2))
        rmse_o = np.sqrt(np.mean(rb[b] ** 2))
        assert abs(rmse - rmse_o) <= 1e-3 * rmse_o, (b, rmse, rmse_o)
