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
    args = argparse.Namespace(workload=bench.HEADLINE, lmax=1, steps=1, warmup=1)
    res = bench.run_reference(args, 0, 1)
    assert res["impl"] == "reference" and res["metric"] == bench.METRIC and res["unit"] == bench.UNIT
    assert res["value"] > 0 and res["higher_is_better"] is True
    cb = res["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == res["value"] and cb["sample"]
    assert res["e2e"] == {"value": res["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_roofline_flop_accounting():
    """bench.py's FLOP count, from the oracle's row counts: all fields
    upwinded gives the all-upwinded row; a split pattern adds its extra in
    proportion to its share of faces; linear reconstructions of fields 0, 1, 4
    save the difference of the two reconstructions' counts, once per
    reconstruction (two for a field that splits); per cell and stage three
    directions of row / 16 plus the flux differences and the update."""
    sys.path.insert(0, ROOT)
    import bench
    t = bench.flop_table()
    w = {k: v[0] for k, v in t["row"]["weno5"].items()}
    lin = {k: v[0] for k, v in t["row"]["linear5"].items()}
    pf, pc = bench.roofline_numbers(0.0)
    assert pf == w["all_upwind"] / 17
    assert pc == 3 * w["all_upwind"] / 16 + 30 + 20
    pf1, _ = bench.roofline_numbers(0.0, (0.0, 1.0, 1.0, 1.0, 0.0))
    assert pf1 == w["split_123"] / 17
    pf2, _ = bench.roofline_numbers(0.0, (0.5, 0.0, 0.0, 0.0, 0.0))
    assert pf2 == pytest.approx((w["all_upwind"] + 0.5 * (w["split_0"] - w["all_upwind"])) / 17)
    # all five fields linear in the oracle's own count = WENO5 row minus two
    # linear fields' worth (the shear fields keep WENO5 in the selector path)
    save = t["recon"]["weno5"][0] - t["recon"]["linear5"][0]
    pl, _ = bench.roofline_numbers(1.0)
    assert pl * 17 == w["all_upwind"] - 17 * 3 * save
    assert lin["all_upwind"] == w["all_upwind"] - 17 * 5 * save
    pls, _ = bench.roofline_numbers(1.0, (0.0, 1.0, 1.0, 1.0, 0.0))
    assert pls * 17 == w["split_123"] - 17 * 4 * save
    assert lin["split_123"] == w["split_123"] - 17 * 8 * save


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
