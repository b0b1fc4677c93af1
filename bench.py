"""Benchmark: leaf cell-updates/s per RK stage of the block-based MR Euler hot path.

Workload (N = 1): the MR spherical explosion of the paper's workload family --
unit cube, base 2^3 blocks of 16^3 cells, levels 0..3 (effective 256^3), eps =
1e-3 at l_max, rho, p = 1, 1 inside r < 0.4 and 0.125, 0.1 outside, at rest --
with the tree built by Alg. (Initialization).  One step = the library's
mrb_step: CFL time step, three fused TVD-RK3 stages (halo fill, RHS + update,
jump correction, averaging), MR analysis and remesh.  value = sum over timed
steps of (leaf internal cells at the step) x 3 stages / device time.

The headline path is the FP32-bulk path (FP32 reconstruction and fluxes, FP64
state, update, conservation sums and time-step reduction); the all-FP64 path is
timed on the same workload and reported beside it, with the L1 density error
between them.  `--impl reference` times the CPU oracle on the same workload.

Multi-GPU (torchrun, one rank per GPU): independent replicas of the workload,
no data-path collective ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import os
import shutil
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "leaf cell-updates/s per RK stage, FP32+learned vs FP64 at L1 err ≤1e-4"
UNIT = "cell-updates/s"
WORKLOAD = "explosion_mr_256cubed_l3"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mrb", choices=["mrb", "reference"])
    ap.add_argument("--lmax", type=int, default=3)
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def workload_config(lmax: int, precision: int):
    from paper_2012_04385_gb300 import inputs as I
    return I.explosion_config(lmax=lmax, precision=precision)


def slots_for(cfg) -> int:
    # fully refined upper bound of the tree: sum_l 8^l * base blocks
    base = int(np.prod(cfg.base_blocks)) * cfg.n_instances
    return int(sum(base * 8 ** l for l in range(cfg.lmax_of(0) + 1)))


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        if not shutil.which("nvidia-smi"):
            return
        self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                      "-lms", "200", "-i", str(self.idx)], stdout=subprocess.PIPE,
                                     stderr=subprocess.DEVNULL, text=True)
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=5)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) >= 9:
                for n, v in zip(names, r[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ helpers
def build_tree(ctx, cfg):
    from paper_2012_04385_gb300 import inputs as I
    from paper_2012_04385_gb300 import mrb
    mrb.init_tree(ctx, lambda c, geo: I.ic_explosion(c, geo))


def oracle_init_tree(o, cfg, ic):
    """Alg. (Initialization) through the oracle's calls (same sequence as mrb.init_tree)."""
    o.set_state(o.keys(level=0), ic(cfg, o.geometry(level=0)))
    for m in range(1, cfg.lmax_of(0) + 1):
        o.fill_halos()
        geo = o.geometry()
        o.remesh((geo[:, 0] == m - 1).astype(np.int8))
        o.set_state(o.keys(level=m), ic(cfg, o.geometry(level=m)))
        if m > 1:
            o.fill_halos()
            t, _ = o.predict_and_tag(allow_refine=False)
            o.remesh(t)
    o.project()


def finest_density(keys, geo, rho, cfg):
    """Inject leaf densities onto the finest uniform grid (piecewise constant)."""
    L = cfg.lmax_of(0)
    n = [cfg.base_blocks[d] * 16 << L for d in range(3)]
    out = np.zeros((n[2], n[1], n[0]))
    for b in range(len(keys)):
        lvl, X, Y, Z = geo[b]
        f = 1 << (L - lvl)
        blk = np.repeat(np.repeat(np.repeat(rho[b], f, 0), f, 1), f, 2)
        out[Z * 16 * f:(Z + 1) * 16 * f, Y * 16 * f:(Y + 1) * 16 * f, X * 16 * f:(X + 1) * 16 * f] = blk
    return out


def roofline_numbers():
    """Algorithmic FLOPs of the fused stage kernel per leaf cell and stage, and
    the FP32 CUDA-core peak; see the accounting in this function's body."""
    # Per face (the oracle's face flux, WENO5 on every field, Roe upwinding on
    # every field, zero matrix entries skipped): Roe average and eigensystem 71,
    # characteristic projections 6 cells x 62, split tests 6, WENO5 5 x 66,
    # R g 33 -> 812.  Per cell and direction: primitive variables and physical
    # flux 25.  Per cell and stage: 3 x (17/16 faces x 812 + 22/16 x 25)
    # + divergence 30 + update 20 = 2747 + 103 + 50.
    per_face = 812
    per_cell = 3 * (17 / 16 * per_face + 22 / 16 * 25) + 30 + 20
    return per_face, per_cell


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path))
    except Exception:
        return {}


# ------------------------------------------------------------------ GPU arm
def run_gpu(args, rank, world):
    import torch

    from paper_2012_04385_gb300 import inputs as I
    from paper_2012_04385_gb300 import mrb

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    def max_over_ranks(x):
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def sum_over_ranks(x):
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return float(t.item())

    stream = torch.cuda.current_stream()
    cfg = workload_config(args.lmax, I.FP32_ACC64)
    ctx = mrb.Context(cfg, slots_for(cfg), stream=stream)
    build_tree(ctx, cfg)
    keys0 = ctx.keys()
    state0 = ctx.get_state(keys0).clone()
    for _ in range(args.warmup):
        ctx.step(1)
    barrier()
    # ---- timed region (device time, CUDA events on the launching stream)
    sampler = ClockSampler(dev)
    sampler.start()
    ctx.profile(True)
    cells = 0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        cells += ctx.n_leaves() * 4096 * 3
        ctx.step(1)
    ev1.record(stream)
    barrier()
    ms = ev0.elapsed_time(ev1)
    rhs_ms, rhs_n, n_kernels = ctx.profile_read()
    ctx.profile(False)
    clocks = sampler.stop()
    ms_max = max_over_ranks(ms)
    total_cells = sum_over_ranks(cells)
    value = total_cells / (ms_max * 1e-3)
    leaves_end = ctx.n_leaves()

    # ---- roofline of the fused stage kernel
    per_face, per_cell = roofline_numbers()
    pk = measured_peaks()
    clk = clocks["sm_mhz"] or pk.get("clocks_under_load", {}).get("sm_mhz_median") or 1447.0
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = nsm * 128 * 2 * clk * 1e6 / 1e12          # TFLOP/s at the sampled clock
    avg_launch_ms = rhs_ms / max(rhs_n, 1)
    achieved = (cells / 3 / args.steps) * per_cell / (avg_launch_ms * 1e-3) / 1e12   # per launch: one stage

    # ---- FP64 path on the same workload
    cfg64 = workload_config(args.lmax, I.FP64)
    ctx64 = mrb.Context(cfg64, slots_for(cfg64), stream=stream)
    build_tree(ctx64, cfg64)
    ctx64.step(1)
    barrier()
    cells64 = 0
    ctx64.profile(True)
    ev0.record(stream)
    for _ in range(args.fp64_steps):
        cells64 += ctx64.n_leaves() * 4096 * 3
        ctx64.step(1)
    ev1.record(stream)
    barrier()
    ms64 = ev0.elapsed_time(ev1)
    rhs64_ms, rhs64_n, _ = ctx64.profile_read()
    value64 = sum_over_ranks(cells64) / (max_over_ranks(ms64) * 1e-3)

    # ---- L1 density error FP32-bulk vs FP64, same initial tree, same steps
    ca = mrb.Context(cfg, slots_for(cfg), stream=stream)
    cb = mrb.Context(cfg64, slots_for(cfg64), stream=stream)
    build_tree(ca, cfg)
    build_tree(cb, cfg64)
    nerr = max(args.fp64_steps, 3)
    ca.step(nerr)
    cb.step(nerr)
    ka, ga = ca.list_blocks()
    kb, gb = cb.list_blocks()
    ra = finest_density(ka, ga, ca.get_state(ka).cpu().numpy()[:, 0], cfg)
    rb = finest_density(kb, gb, cb.get_state(kb).cpu().numpy()[:, 0], cfg)
    l1 = float(np.abs(ra - rb).sum() / np.abs(rb).sum())
    same_tree = bool(np.array_equal(ka, kb))
    del ca, cb, ctx64

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        # per step: H2D of the step's input state from pinned host memory,
        # mrb_set_cons + mrb_step + mrb_get_state, D2H of the result state and
        # the conservation sums
        cap = slots_for(cfg)
        host = [torch.empty((cap, 5, 16, 16, 16), dtype=torch.float64).pin_memory() for _ in range(2)]
        dev_buf = torch.empty((cap, 5, 16, 16, 16), dtype=torch.float64, device="cuda")
        sums = torch.empty((1, 5), dtype=torch.float64, device="cuda")
        host_sums = torch.empty((1, 5), dtype=torch.float64).pin_memory()
        keys = ctx.keys()
        n = len(keys)
        host[0][:n].copy_(ctx.get_state(keys))
        barrier()
        t0 = time.perf_counter()
        ecells, h2d, d2h = 0, 0, 0
        e_steps = max(3, args.steps // 2)
        for it in range(e_steps):
            src, dst = host[it % 2], host[(it + 1) % 2]
            dev_buf[:n].copy_(src[:n], non_blocking=True)
            h2d += n * 5 * 4096 * 8
            ctx.set_cons(keys, dev_buf[:n])
            ecells += n * 4096 * 3
            ctx.step(1)
            keys = ctx.keys()
            n = len(keys)
            ctx.get_state(keys, out=dev_buf[:n])
            dst[:n].copy_(dev_buf[:n], non_blocking=True)
            ctx.sums(sums)
            host_sums.copy_(sums, non_blocking=True)
            d2h += n * 5 * 4096 * 8 + 5 * 8
            stream.synchronize()
        barrier()
        el = time.perf_counter() - t0
        e2e_value = sum_over_ranks(ecells) / max_over_ranks(el)
        e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d // e_steps),
               "d2h_bytes_per_step": int(d2h // e_steps)}

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 bulk / f64 state+update", "data": "synthetic",
        "config": {"workload": WORKLOAD, "path": "FP32 bulk + FP64 accumulate, WENO5-JS",
                   "effective_resolution": "256^3", "lmax": args.lmax,
                   "leaf_blocks_start": int(len(keys0)), "leaf_blocks_end": int(leaves_end),
                   "l2": "inputs larger than L2 (block pool %.1f GB)" % (ctx.pool.numel() / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak, "traffic": None,
                     "kernel": "k_rhs_rk<float> (fused RHS + RK stage)",
                     "flops_per_cell_stage": per_cell, "avg_launch_ms": avg_launch_ms,
                     "peak_basis": f"FP32 CUDA cores {nsm} SMs x 128 lanes x 2 x {clk:.0f} MHz sampled"},
        "gpu_launches": int(n_kernels),
        "clocks": clocks,
        "fp64_path": {"value": value64, "unit": UNIT, "steps": args.fp64_steps, "ms_per_step": ms64 / args.fp64_steps,
                      "stage_kernel_ms": rhs64_ms / max(rhs64_n, 1)},
        "l1_density_err_fp32_vs_fp64": l1, "l1_steps": nerr, "l1_same_tree": same_tree,
    }
    if e2e:
        result["e2e"] = e2e
    if rank == 0 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(args)
    if dist is not None:
        dist.destroy_process_group()
    return result


# ------------------------------------------------------------------ oracle
def cpu_baseline(args, steps=1):
    """The CPU oracle as it stands, on the same workload's initial tree, for
    `steps` full steps (a bounded sample)."""
    import oracle
    from paper_2012_04385_gb300 import inputs as I
    cfg = workload_config(args.lmax, I.FP64)
    o = oracle.Oracle(cfg)
    oracle_init_tree(o, cfg, I.ic_explosion)
    cells = 0
    t0 = time.perf_counter()
    for _ in range(steps):
        cells += o.n_leaves() * 4096 * 3
        o.step(1)
    el = time.perf_counter() - t0
    return {"value": cells / el, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": f"{steps} full step(s) of {WORKLOAD} from its initial tree ({cells // 3 // 4096} leaf blocks), "
                      f"{el:.1f} s"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    import oracle
    from paper_2012_04385_gb300 import inputs as I
    cfg = workload_config(args.lmax, I.FP64)
    o = oracle.Oracle(cfg)
    oracle_init_tree(o, cfg, I.ic_explosion)
    for _ in range(args.warmup):
        o.step(1)
    cells = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cells += o.n_leaves() * 4096 * 3
        o.step(1)
    el = time.perf_counter() - t0
    v = cells / el
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "path": "CPU FP64 oracle", "lmax": args.lmax},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                             "sample": f"{args.steps} full oracle steps after {args.warmup} warm-up"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", args.gpus))
    if args.impl == "reference":
        res = run_reference(args, rank, world)
    else:
        res = run_gpu(args, rank, world)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
