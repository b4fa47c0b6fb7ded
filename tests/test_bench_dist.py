"""Replica path of the benchmark on two CPU ranks (gloo): the whole-job figure
is all ranks' site updates over the slowest rank's time, and the reference
arm runs on rank 0 only."""
import os
import sys
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    d = bench.Dist(backend="gloo")
    units = 1000.0 * (rank + 1)          # ranks 0, 1 did 1000, 2000 site updates
    seconds = 0.5 + rank                 # in 0.5 s and 1.5 s
    value, tmax = bench.aggregate(d, units, seconds)
    d.barrier()
    ref = bench.main_reference(None, d) if rank != 0 else "skipped"
    out.put((rank, value, tmax, ref))
    d.close()


def test_aggregate_two_ranks_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, tmax, ref in got:
        assert tmax == pytest.approx(1.5)
        assert value == pytest.approx(3000.0 / 1.5)
        if rank != 0:
            assert ref is None                # the reference arm prints on rank 0 alone


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    d = bench.Dist()
    assert d.world == int(os.environ.get("WORLD_SIZE", "1"))
    if d.world == 1:
        assert bench.aggregate(d, 10.0, 2.0) == (5.0, 2.0)


def test_reference_arm_line_keeps_the_contract():
    """The reference arm (the CPU oracle) on rank 0: one JSON-ready line with
    the GPU arm's metric, unit and workload name, its cpu_baseline and a
    zero-copy e2e, from a short run."""
    import argparse
    import bench
    d = bench.Dist(backend=None)
    args = argparse.Namespace(steps=1, warmup=1, size=512)
    line = bench.main_reference(args, d)
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["higher_is_better"] is True and line["value"] > 0
    assert line["config"]["workload"] == bench.workload_name(512)
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT,
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
