"""Host-side logic of bench.py: whole-job aggregation over ranks (max time,
summed units) on a world-size-2 gloo process group, and the reference arm's
rank handling under torchrun. No GPU."""

import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench as b
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        rmax, rsum = b.torch_reducers()
        # rank r: local time 2 + r ms for 1000 * (r + 1) units
        ms, units, value = b.aggregate(2.0 + rank, 1000.0 * (rank + 1), world, rmax, rsum)
        out.put((rank, ms, units, value))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_aggregate_single_rank():
    ms, units, value = bench.aggregate(2.0, 500.0, 1)
    assert (ms, units) == (2.0, 500.0)
    assert value == pytest.approx(500.0 / 2e-3)


def test_aggregate_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, units, value in res:
        assert ms == 3.0            # the slower rank's time
        assert units == 3000.0      # every rank's units
        assert value == pytest.approx(3000.0 / 3e-3)


def test_reference_arm_nonzero_rank_exits_without_work(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "1"])
    called = []
    monkeypatch.setattr(bench, "run_oracle_sample", lambda *a, **k: called.append(1))
    assert bench.main() == 0
    assert not called
