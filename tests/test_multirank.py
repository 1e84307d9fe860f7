"""The bench's N > 1 path on CPU: two gloo ranks (127.0.0.1) that each timed their own
replica agree on the whole-job figures -- the slowest rank's time and the units of all
ranks -- exactly as a GPU run over NCCL reduces them.  No GPU needed."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [120.0, 95.5][rank]          # the second rank was faster
    units = [1.0e10, 1.0e10][rank]    # each processed its own replica
    out[rank] = bench.job_rate(ms, units, world, device="cpu")
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_bench():
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        ms, units, value = res[r]
        assert ms == 120.0                      # max over ranks
        assert units == 2.0e10                  # all ranks' units
        assert value == pytest.approx(2.0e10 / 0.120)


def test_single_rank_is_a_no_op():
    import bench
    assert bench.job_rate(50.0, 1e9, 1) == (50.0, 1e9, 1e9 / 0.05)


# ------------------------------------------------------------------------------------
# The row-sharded form of a sweep (the multi-GPU design that a box with several GPUs
# would run): rows of every mode partitioned over the ranks by Algorithm 3's greedy
# assignment, each rank updating only its own rows (Eq. 4) from replicated factors and
# residuals, then an all-reduce of the updated columns S of A^(n) (each row is owned by
# exactly one rank, so a sum of the ranks' contributions is the all-gather).  Emulated
# with gloo ranks on the CPU, in FP64, against the single-process oracle.


def _sharded_sweep(rank, world, port, out, coords, x, dims, A0, C, lam, order):
    import numpy as np
    import paper_1410_5209_gb300 as tf
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    N, K = len(dims), A0[0].shape[1]
    A = [a.copy() for a in A0]
    row_nnz = [np.bincount(coords[:, n], minlength=dims[n]).astype(np.int64) for n in range(N)]
    owner = tf.assign_rows(tf.SCHED_GREEDY, dims, row_nnz, world)
    model = lambda cols: sum(np.prod([A[n][coords[:, n], k] for n in range(N)], axis=0)
                             for k in cols)
    r = x - model(range(K))
    for s0 in range(0, K, C):
        S = list(order[s0:s0 + C])
        rhat = r + model(S)                                   # Algorithm 1's R-hat
        for n in range(N):
            upd = np.zeros((dims[n], len(S)))
            mine = np.flatnonzero(owner[n] == rank)
            h_all = np.prod([A[l][coords[:, l]][:, S] for l in range(N) if l != n], axis=0)
            for i in mine:                                    # this rank's rows only
                e = np.flatnonzero(coords[:, n] == i)
                h = h_all[e]
                B = h.T @ h + lam * np.eye(len(S))
                upd[i] = np.linalg.solve(B, h.T @ rhat[e])
            t = torch.from_numpy(upd)
            dist.all_reduce(t, op=dist.ReduceOp.SUM)          # the exchange of the slice
            A[n][:, S] = t.numpy()
        r = rhat - model(S)                                   # Eq. 5
    out[rank] = [a.copy() for a in A]
    dist.barrier()
    dist.destroy_process_group()


def test_row_sharded_sweep_over_two_gloo_ranks_matches_the_oracle():
    import numpy as np
    import oracle
    import synth
    p = synth.small(250, (40, 30, 12), 2_500, 3, 6)
    c, x = p.numpy()
    A0 = [a.numpy() for a in p.init_factors()]
    order = p.column_order(0, 3)
    t = oracle.Tensor(c, x, p.dims)
    Ao = [a.copy() for a in A0]
    r = oracle.residual(t, Ao)
    oracle.sals_sweep(t, Ao, r, 3, 0.5, 1, order)
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_sharded_sweep, args=(2, port, out, c, x, list(p.dims), A0, 3, 0.5,
                                       np.asarray(order)), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        for n in range(3):
            err = np.linalg.norm(res[rank][n] - Ao[n]) / np.linalg.norm(Ao[n])
            assert err < 1e-10, (rank, n, err)
