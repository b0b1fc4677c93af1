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


# ------------------------------------------------------------------ ensemble sharding
def _oracle_ensemble_sums(cfg, ic, steps):
    """Per-instance conserved totals after `steps` oracle steps of a batched
    run built by Alg. (Initialization) (ic(cfg, geo, keys))."""
    import numpy as np

    import oracle
    o = oracle.Oracle(cfg, n_threads=2)
    lmax = max(cfg.lmax_of(i) for i in range(cfg.n_instances))
    o.set_state(o.keys(), ic(cfg, o.geometry(), o.keys()))
    for m in range(1, lmax + 1):
        o.fill_halos()
        geo = o.geometry()
        o.remesh((geo[:, 0] == m - 1).astype(np.int8))
        o.set_state(o.keys(level=m), ic(cfg, o.geometry(level=m), o.keys(level=m)))
        if m > 1:
            o.fill_halos()
            t, _ = o.predict_and_tag(allow_refine=False)
            o.remesh(t)
    o.project()
    o.step(steps)
    return o.sums()


def _shard_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    from paper_2012_04385_gb300 import inputs as I
    from paper_2012_04385_gb300 import shard
    dist.init_process_group("gloo")
    cfg = I.ensemble_config(n=5, lmax=(1, 2, 1, 2, 1))
    mine = shard.instance_shards(cfg, world)[rank]
    sums = _oracle_ensemble_sums(shard.shard_config(cfg, mine), shard.shard_ic(I.ic_ensemble, mine), 1)
    gathered = [None] * world
    dist.all_gather_object(gathered, (mine, sums.tolist()))
    q.put((rank, gathered))
    dist.destroy_process_group()


def test_ensemble_sharded_by_instance_over_two_ranks():
    """The batched ensemble splits by instance with no exchange: two gloo
    ranks each run their instances (the oracle standing in for each rank's
    GPU), and the gathered per-instance conserved totals after one MR step
    equal those of one batched run of the whole ensemble bit for bit.  The
    partition covers every instance once and balances the effective cells."""
    import numpy as np

    sys.path.insert(0, ROOT)
    from paper_2012_04385_gb300 import inputs as I
    from paper_2012_04385_gb300 import shard
    cfg = I.ensemble_config(n=5, lmax=(1, 2, 1, 2, 1))
    parts = shard.instance_shards(cfg, 2)
    assert sorted(sum(parts, [])) == list(range(5))
    cost = [sum(shard.instance_cost(cfg, i) for i in p) for p in parts]
    assert max(cost) <= 1.25 * min(cost)
    assert shard.instance_shards(cfg, 1) == [list(range(5))]
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(world):
        rank, gathered = q.get(timeout=600)
        out[rank] = gathered
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0] == out[1]
    got = np.zeros((5, 5))
    for mine, sums in out[0]:
        got[mine] = np.array(sums)
    ref = _oracle_ensemble_sums(cfg, I.ic_ensemble, 1)
    assert np.array_equal(got, ref)
