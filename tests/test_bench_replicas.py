"""The multi-GPU path of bench.py is replicas only (independent frames per GPU, no collective
on the data path); its one exchange -- the slowest rank's time and the sum of rays -- runs
here on two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        t, r = bench.combine_replicas(10.0 + 5.0 * rank, 1000.0 * (rank + 1))
        out[rank] = (t, r)
    finally:
        dist.destroy_process_group()


def test_replicas_combine_max_time_and_sum_of_rays():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == (15.0, 3000.0)


def test_single_process_returns_local_figures():
    import bench
    assert bench.combine_replicas(3.5, 42.0) == (3.5, 42.0)
