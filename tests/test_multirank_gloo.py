"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

On GPUs every rank evaluates its own independent shell (replicas, no
collective on the data path); the only communication is the barrier and the
max-over-ranks of the timed region, and the whole-job value is all ranks'
cell updates over the slowest rank's time.
"""
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


def _worker(rank, world, port, queue):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    d = bench.init_dist(world, "gloo")
    try:
        seconds = [0.5, 0.8][rank]          # rank 1 is the slowest
        bench.barrier(d)
        slowest = bench.max_over_ranks(d, seconds)
        units = 1000 * (rank + 1)
        all_units = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(all_units, torch.tensor([float(units)], dtype=torch.float64))
        value = bench.aggregate([float(u.item()) for u in all_units], [slowest])
        queue.put((rank, slowest, value))
    finally:
        dist.destroy_process_group()


def test_replicas_max_over_ranks_and_whole_job_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, slowest, value in out:
        assert slowest == 0.8                      # every rank sees the slowest time
        assert value == pytest.approx(3000 / 0.8)  # all units over the slowest time


def test_reference_arm_only_rank0_prints(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup = 1, 0
    bench.run_reference(A())
    assert capsys.readouterr().out == ""
