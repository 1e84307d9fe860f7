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
    with mp.Manager() as m:
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
