"""The multi-process path of bench.py on CPU (gloo, world size 2): replicas with a
barrier and max-over-ranks timing, the whole-job rate from the slowest rank, and the
reference arm's rank filter.  No GPU is involved: the GPU work of each rank is the
single-GPU path, tested elsewhere."""
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


def _worker(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench._dist()
        assert (w, r, local) == (world, rank, rank)
        dist.barrier()
        slowest = bench.max_over_ranks(times[rank], dist, "cpu")
        out[rank] = (slowest, bench.job_rate(w, 5, slowest))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    world = 2
    times = [1200.0, 1500.0]  # ms of each rank's timed steps
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), times, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        slowest, rate = res[rank]
        assert slowest == 1500.0
        assert rate == pytest.approx(world * 5 / 1.5)


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_rate(1, 4, 2000.0) == pytest.approx(2.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        gpus, steps, warmup, ref_sample_steps = 2, 1, 3, 2

    assert bench.run_reference(Args()) is None
    assert capsys.readouterr().out == ""
