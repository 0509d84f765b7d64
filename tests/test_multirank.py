"""The multi-rank path of the benchmark on CPU (gloo, world size 2).

Each rank runs an independent replica of the lattice (the spinodal lattices
are independent problems; nothing is exchanged on the data path), so the only
cross-rank steps are the barriers around the timed region and the maximum over
ranks of its duration.  Two spawned ranks pass different durations: both must
end with the slower one, and the whole-job value counts every rank's cells.
The reference arm does its work on rank 0 only."""
import argparse
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench as b
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, l = b.dist_env()
    seconds = b.reduce_max(1.0 + 0.25 * rank)     # rank 1 is the slower one
    dist.barrier()
    q.put((rank, r, w, l, seconds, b.weak_value(w, 4096, 7, seconds)))
    dist.destroy_process_group()


def test_two_ranks_report_the_slowest_interval():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, r, w, l, seconds, value in out:
        assert (r, w, l) == (rank, 2, rank)
        assert seconds == 1.25
        assert value == pytest.approx(2 * 4096 * 7 / 1.25 / 1e6, rel=1e-15)


def test_one_process_needs_no_group():
    assert bench.reduce_max(3.5) == 3.5
    assert bench.weak_value(1, 100, 10, 2.0) == pytest.approx(5e-4)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    args = argparse.Namespace(steps=1, warmup=0, gpus=2)
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
