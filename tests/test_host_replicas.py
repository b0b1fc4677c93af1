"""Host side of the multi-GPU replica runs, on CPU with two gloo ranks.

Each rank runs the whole workload on its own GPU; the only exchange is the
timing: a barrier around the timed region, the maximum of the per-rank
elapsed times and the sum of the per-rank cell-updates.  These tests run that
host logic (bench.Ranks) in two processes without a GPU, and check the JSON
contract of the benchmark's reference arm (the oracle on the host cores).
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    r = bench.Ranks(world, "gloo", "cpu")
    # per-rank measurements: elapsed ms and cell-updates
    ms = [120.0, 135.5][rank]
    cells = [3.0e9, 2.5e9][rank]
    r.barrier()
    ms_max = r.max(ms)
    total = r.sum(cells)
    value = total / (ms_max * 1e-3)
    # the reference arm: only rank 0 works, the others return nothing
    ref = bench.run_reference(None, rank, world) if rank != 0 else "rank0"
    q.put((rank, ms_max, total, value, ref))
    r.close()


def test_two_rank_timing_reduction():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(world):
        rank, ms_max, total, value, ref = q.get(timeout=120)
        out[rank] = (ms_max, total, value, ref)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in range(world):
        ms_max, total, value, ref = out[rank]
        assert ms_max == 135.5                     # slowest rank
        assert total == 5.5e9                      # all ranks' cell-updates
        assert value == pytest.approx(5.5e9 / 0.1355)
    assert out[1][3] is None                       # reference arm: rank 1 exits without work


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    r = bench.Ranks(1, "gloo", "cpu")
    assert r.dist is None
    assert r.max(3.0) == 3.0 and r.sum(4.0) == 4.0
    r.barrier()
    r.close()


def test_reference_arm_json_contract():
    """bench.py --impl reference: the oracle on the host cores, same metric and
    unit as the GPU arm, with the cpu_baseline and e2e objects (small case)."""
    import argparse
    sys.path.insert(0, ROOT)
    import bench
    args = argparse.Namespace(lmax=1, steps=1, warmup=1)
    res = bench.run_reference(args, 0, 1)
    assert res["impl"] == "reference" and res["metric"] == bench.METRIC and res["unit"] == bench.UNIT
    assert res["value"] > 0 and res["higher_is_better"] is True
    cb = res["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == res["value"] and cb["sample"]
    assert res["e2e"] == {"value": res["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_roofline_flop_accounting():
    """bench.py's FLOP count per face: all fields upwinded with WENO5 gives
    the Roe eigensystem, the six g projections, the tests, R g and five WENO5
    reconstructions; a field that splits adds its v projection, the split and
    a second reconstruction; linear faces replace WENO5 on fields 0, 1, 4."""
    sys.path.insert(0, ROOT)
    import bench
    base = bench.FLOP_ROE + bench.FLOP_PROJ_G + bench.FLOP_TESTS + bench.FLOP_RG
    pf, pc = bench.roofline_numbers(0.0)
    assert pf == base + 5 * bench.FLOP_WENO
    assert pc == 3 * (17 / 16 * pf + 22 / 16 * 25) + 50
    pf1, _ = bench.roofline_numbers(0.0, (1.0, 0.0, 0.0, 0.0, 0.0))
    assert pf1 - pf == bench.FLOP_V[0] + bench.FLOP_SPLIT + bench.FLOP_WENO
    pf2, _ = bench.roofline_numbers(0.0, (0.0, 0.0, 0.5, 0.0, 0.0))
    assert pf2 - pf == 0.5 * (bench.FLOP_V[2] + bench.FLOP_SPLIT + bench.FLOP_WENO)
    pl, _ = bench.roofline_numbers(1.0)
    assert pf - pl == 3 * (bench.FLOP_WENO - bench.FLOP_LIN)


def test_reference_arm_under_torchrun_prints_one_line():
    """The driver's launch of the reference arm at N = 2: rank 0 alone runs
    the oracle and prints one JSON line; rank 1 exits 0 without work."""
    import json
    import subprocess
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--lmax", "1"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, OMP_NUM_THREADS="2"))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    res = json.loads(lines[0])
    assert res["impl"] == "reference" and res["n_gpus"] == 2 and res["value"] > 0
