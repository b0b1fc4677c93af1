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


# FP32-path variants timed beside the headline: (name, reconstruction, flux scheme)
VARIANTS = [("weno5_roe", 0, 0), ("linear5_roe", 2, 0), ("teno5_roe", 3, 0), ("wenoao53_roe", 4, 0),
            ("weno5_llf", 0, 1), ("teno5_llf", 3, 1), ("weno5_hllc", 0, 2), ("teno5_hllc", 3, 2),
            ("wenoao53_hllc", 4, 2)]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mrb", choices=["mrb", "reference"])
    ap.add_argument("--lmax", type=int, default=3)
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip timing the reconstruction/flux variants of the FP32 path")
    # wrap the headline path's timed steps in cudaProfilerStart/Stop (for
    # ncu --profile-from-start off)
    ap.add_argument("--profile-range", action="store_true")
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


# FLOPs of the face flux by part, as the oracle's face flux performs them
# (zero entries of the eigenvectors and loop-invariant constants skipped).
FLOP_ROE = 71                  # Roe average and eigensystem
FLOP_PROJ_G = 6 * 31           # g = L F(U) of the six cells: 9 per acoustic / entropy field, 2 per shear field
FLOP_TESTS = 6                 # eigenvalue sign tests
FLOP_RG = 33                   # F = R g_hat
FLOP_WENO, FLOP_LIN = 66, 21   # one WENO5-JS / linear 5th-order reconstruction
FLOP_V = (54, 54, 12, 12, 54)  # v = l_k U of the six cells, needed only by a split field k
FLOP_SPLIT = 34                # alpha (3), the split halves of the six cells (30), the sum (1)


def roofline_numbers(linear_fraction=0.0, split=None):
    """Algorithmic FP32 FLOPs of the fused stage kernel per face and per leaf
    cell and stage.  `linear_fraction`: share of faces whose fields 0, 1, 4
    take the linear scheme (averaged over the stages timed); `split[k]`: share
    of faces where characteristic field k takes the LLF split (the census of
    mrb_flux_census), which adds its v projection, the split and a second
    reconstruction.  Per cell and direction the primitive variables and the
    physical flux cost 25; per cell and stage: 3 x (17/16 x per_face + 22/16
    x 25) + divergence 30 + update 20.  The selector's MLP runs on the tensor
    cores and is not counted."""
    split = split if split is not None else (0.0,) * 5
    per_face = FLOP_ROE + FLOP_PROJ_G + FLOP_TESTS + FLOP_RG
    for k in range(5):
        rec = FLOP_WENO if k in (2, 3) else (1 - linear_fraction) * FLOP_WENO + linear_fraction * FLOP_LIN
        per_face += rec + split[k] * (FLOP_V[k] + FLOP_SPLIT + rec)
    per_cell = 3 * (17 / 16 * per_face + 22 / 16 * 25) + 30 + 20
    return per_face, per_cell


# DRAM bytes per leaf cell of one launch of the stage kernels, from the ncu
# capture summarised in profiles/stage_kernels_explosion_256.md (levels 0-2
# explosion; traffic grows in proportion to the leaf cells of a launch).
# Learned path: the mean over its stage-0 and stage-1/2 variants (1 + 2 launches).
TRAFFIC_BYTES_PER_CELL = {"learned": (148.2 + 155.0 + 155.1) / 3, "weno": (146.6 + 154.0 + 154.3) / 3}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path))
    except Exception:
        return {}


# ------------------------------------------------------------------ ranks
class Ranks:
    """Host side of the replica runs: one process per GPU, each running the
    whole workload; only the timing is combined (barrier, max of the elapsed
    times, sum of the cell-updates).  No data-path collective."""

    def __init__(self, world: int, backend: str = "nccl", device: str = "cuda"):
        import torch
        self.world, self.device, self.dist = world, device, None
        if world > 1:
            import torch.distributed as dist
            if not dist.is_initialized():
                dist.init_process_group(backend)
            self.dist = dist
        self._torch = torch

    def barrier(self):
        if self.device == "cuda":
            self._torch.cuda.synchronize()
        if self.dist is not None:
            self.dist.barrier()

    def _reduce(self, x, op):
        if self.dist is None:
            return x
        t = self._torch.tensor([float(x)], dtype=self._torch.float64, device=self.device)
        self.dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, x):
        return self._reduce(x, self.dist.ReduceOp.MAX) if self.dist is not None else x

    def sum(self, x):
        return self._reduce(x, self.dist.ReduceOp.SUM) if self.dist is not None else x

    def close(self):
        if self.dist is not None and self.dist.is_initialized():
            self.dist.destroy_process_group()


# ------------------------------------------------------------------ GPU arm
def census_fractions(ctx):
    """Shares of faces where each characteristic field takes the LLF split,
    on the current state (halos filled first; outside any timed region)."""
    ctx.fill_halos()
    c = ctx.flux_census().astype(np.float64)
    return c[:5] / max(c[5], 1.0)


def timed_path(args, cfg, stream, steps, warmup, mlp_params=None, profile=True, profiler_range=False, census=False):
    """Build the workload tree, warm up, time `steps` full steps with CUDA
    events on the launching stream; returns the context and measurements."""
    import torch

    from paper_2012_04385_gb300 import mrb
    ctx = mrb.Context(cfg, slots_for(cfg), stream=stream, mlp_params=mlp_params)
    build_tree(ctx, cfg)
    for _ in range(warmup):
        ctx.step(1)
    torch.cuda.synchronize()
    split0 = census_fractions(ctx) if census else None
    if profile:
        ctx.profile(True)
    ctx.learned_stats(reset=True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cells = 0
    if profiler_range:
        torch.cuda.profiler.start()
    ev0.record(stream)
    for _ in range(steps):
        cells += ctx.n_leaves() * 4096 * 3
        ctx.step(1)
    ev1.record(stream)
    torch.cuda.synchronize()
    if profiler_range:
        torch.cuda.profiler.stop()
    ms = ev0.elapsed_time(ev1)
    kms, kn, nk = ctx.profile_read() if profile else (0.0, 0, 0)
    lin, tot = ctx.learned_stats()
    # the census of the switch at the start and the end of the timed steps
    split = tuple(0.5 * (split0 + census_fractions(ctx))) if census else None
    return ctx, dict(ms=ms, cells=cells, stage_ms=kms / max(kn, 1), launches=nk,
                     linear_fraction=(lin / tot) if tot else 0.0, split=split)


def l1_after(cfg_a, cfg_b, stream, nsteps, params=None):
    """L1 density difference of two paths after nsteps from the same initial tree."""
    from paper_2012_04385_gb300 import mrb
    out = []
    for cfg in (cfg_a, cfg_b):
        ctx = mrb.Context(cfg, slots_for(cfg), stream=stream,
                          mlp_params=params if cfg.recon == 1 else None)
        build_tree(ctx, cfg)
        ctx.step(nsteps)
        k, g = ctx.list_blocks()
        out.append((k, finest_density(k, g, ctx.get_state(k).cpu().numpy()[:, 0], cfg)))
        ctx.close()
    (ka, ra), (kb, rb) = out
    return float(np.abs(ra - rb).sum() / np.abs(rb).sum()), bool(np.array_equal(ka, kb))


def run_gpu(args, rank, world):
    import torch

    from paper_2012_04385_gb300 import inputs as I
    from paper_2012_04385_gb300 import learned, mrb

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    ranks = Ranks(world, "nccl", "cuda")
    barrier, max_over_ranks, sum_over_ranks = ranks.barrier, ranks.max, ranks.sum

    stream = torch.cuda.current_stream()
    # ---- the learned selector, trained on the GPU by the library's own kernels
    t0 = time.perf_counter()
    data = learned.generate()
    params, tau, rep = learned.train(data, epochs=10)
    train_s = time.perf_counter() - t0
    cfg_l = workload_config(args.lmax, I.FP32_ACC64)
    cfg_l.recon, cfg_l.mlp_tau = I.RECON_LEARNED, tau
    cfg_w = workload_config(args.lmax, I.FP32_ACC64)
    cfg_64 = workload_config(args.lmax, I.FP64)

    # ---- headline: FP32 bulk + learned selector, timed region with clocks
    barrier()
    sampler = ClockSampler(dev)
    sampler.start()
    ctx, m = timed_path(args, cfg_l, stream, args.steps, args.warmup, mlp_params=params,
                        profiler_range=args.profile_range, census=True)
    clocks = sampler.stop()
    barrier()
    ms_max = max_over_ranks(m["ms"])
    value = sum_over_ranks(m["cells"]) / (ms_max * 1e-3)
    keys0 = ctx.keys()

    # ---- roofline of the fused stage kernel (FP32 CUDA cores)
    # stage 0 evaluates the selector with WENO5 fluxes; stages 1 and 2 use its decisions
    per_face, per_cell = roofline_numbers(m["linear_fraction"] * 2 / 3, m["split"])
    pk = measured_peaks()
    clk = clocks["sm_mhz"] or pk.get("clocks_under_load", {}).get("sm_mhz_median") or 1447.0
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = nsm * 128 * 2 * clk * 1e6 / 1e12
    cells_per_launch = m["cells"] / 3 / args.steps
    achieved = cells_per_launch * per_cell / (m["stage_ms"] * 1e-3) / 1e12

    # ---- the same workload on the FP32 WENO5 path and the all-FP64 path
    _, mw = timed_path(args, cfg_w, stream, args.steps, args.warmup, census=True)
    _, m64 = timed_path(args, cfg_64, stream, args.fp64_steps, 1)
    value_w = sum_over_ranks(mw["cells"]) / (max_over_ranks(mw["ms"]) * 1e-3)
    value_64 = sum_over_ranks(m64["cells"]) / (max_over_ranks(m64["ms"]) * 1e-3)
    _, pfw = roofline_numbers(0.0, mw["split"])
    achieved_w = (mw["cells"] / 3 / args.steps) * pfw / (mw["stage_ms"] * 1e-3) / 1e12

    # ---- reconstruction / flux variants of the FP32 path on the same workload
    variants = None
    if not args.no_variants:
        variants = {}
        vsteps = max(3, min(args.steps, 10))
        for name, rec, fl in VARIANTS:
            cfg_v = workload_config(args.lmax, I.FP32_ACC64)
            cfg_v.recon, cfg_v.flux = rec, fl
            _, mv = timed_path(args, cfg_v, stream, vsteps, 2)
            variants[name] = {"value": sum_over_ranks(mv["cells"]) / (max_over_ranks(mv["ms"]) * 1e-3),
                              "ms_per_step": mv["ms"] / vsteps, "stage_kernel_ms": mv["stage_ms"],
                              "steps": vsteps}

    # ---- L1 density errors against the FP64 GPU path (same initial tree, same steps)
    nerr = max(args.fp64_steps, 3)
    l1_l, same_l = l1_after(cfg_l, cfg_64, stream, nerr, params)
    l1_w, same_w = l1_after(cfg_w, cfg_64, stream, nerr)

    # ---- end to end through the C ABI with host buffers (headline path)
    e2e = None
    if not args.no_e2e:
        # per step: H2D of the step's input state from pinned host memory,
        # mrb_set_cons + mrb_step + mrb_get_state, D2H of the result state and
        # the conservation sums
        cap = slots_for(cfg_l)
        host = [torch.empty((cap, 5, 16, 16, 16), dtype=torch.float64).pin_memory() for _ in range(2)]
        dev_buf = torch.empty((cap, 5, 16, 16, 16), dtype=torch.float64, device="cuda")
        sums = torch.empty((1, 5), dtype=torch.float64, device="cuda")
        host_sums = torch.empty((1, 5), dtype=torch.float64).pin_memory()
        keys = ctx.keys()
        n = len(keys)
        host[0][:n].copy_(ctx.get_state(keys))
        barrier()
        t1 = time.perf_counter()
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
        el = time.perf_counter() - t1
        e2e = {"value": sum_over_ranks(ecells) / max_over_ranks(el), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d // e_steps), "d2h_bytes_per_step": int(d2h // e_steps)}

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 bulk (bf16 tensor-core selector) / f64 state+update", "data": "synthetic",
        "config": {"workload": WORKLOAD, "path": "FP32 bulk + FP64 accumulate, learned WENO5/linear selector",
                   "effective_resolution": "256^3", "lmax": args.lmax,
                   "leaf_blocks_start": int(len(keys0)),
                   "l2": "inputs larger than L2 (block pool %.1f GB)" % (ctx.pool.numel() / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak,
                     "traffic": (TRAFFIC_BYTES_PER_CELL["learned"] * cells_per_launch
                                 if TRAFFIC_BYTES_PER_CELL["learned"] else None),
                     "traffic_note": "ncu dram bytes per leaf cell of 2.1M-cell launches (stage 0, 1, 2 mean) x the launch's leaf cells",
                     "kernel": "k_stage_f32<1> (stage 0, selector evaluated) + k_stage_f32<3> (stages 1, 2): fused RHS + RK stage",
                     "flops_per_cell_stage": per_cell, "flops_per_face": per_face,
                     "llf_split_share_per_field": [round(x, 4) for x in m["split"]],
                     "avg_launch_ms": m["stage_ms"],
                     "peak_basis": f"FP32 CUDA cores {nsm} SMs x 128 lanes x 2 x {clk:.0f} MHz sampled"},
        "gpu_launches": int(m["launches"]),
        "clocks": clocks,
        "selector": {"linear_fraction": m["linear_fraction"], "tau": tau, "train_s": round(train_s, 1),
                     "train_samples": rep["samples"], "holdout_accuracy": rep["holdout_accuracy"],
                     "holdout_missed_positives": rep["holdout_missed_positives"]},
        "fp32_weno_path": {"value": value_w, "unit": UNIT, "ms_per_step": mw["ms"] / args.steps,
                           "stage_kernel_ms": mw["stage_ms"], "roofline_frac": achieved_w / fp32_peak},
        "fp64_path": {"value": value_64, "unit": UNIT, "steps": args.fp64_steps,
                      "ms_per_step": m64["ms"] / args.fp64_steps, "stage_kernel_ms": m64["stage_ms"]},
        "l1_density_err_vs_fp64": {"fp32_learned": l1_l, "fp32_weno": l1_w, "steps": nerr,
                                   "same_tree": same_l and same_w},
    }
    if variants:
        result["fp32_variants"] = variants
    if e2e:
        result["e2e"] = e2e
    # the host-core baseline is taken once, by the single rank of an N = 1 run
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(args)
    ranks.close()
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


REFERENCE_BUDGET_S = 90.0


def run_reference(args, rank, world):
    """The oracle as it stands on the host cores, on the same workload.  Each
    step is one full oracle step; the run is a bounded sample: one untimed
    warm-up step, then timed steps until `--steps` or REFERENCE_BUDGET_S of
    host time, whichever comes first."""
    if rank != 0:
        return None
    import oracle
    from paper_2012_04385_gb300 import inputs as I
    cfg = workload_config(args.lmax, I.FP64)
    o = oracle.Oracle(cfg)
    oracle_init_tree(o, cfg, I.ic_explosion)
    for _ in range(min(args.warmup, 1)):
        o.step(1)
    cells, done = 0, 0
    t0 = time.perf_counter()
    while done < args.steps and (done == 0 or time.perf_counter() - t0 < REFERENCE_BUDGET_S):
        cells += o.n_leaves() * 4096 * 3
        o.step(1)
        done += 1
    el = time.perf_counter() - t0
    v = cells / el
    sample = (f"{done} of {args.steps} full oracle steps of {WORKLOAD} after {min(args.warmup, 1)} warm-up "
              f"({el:.1f} s, bounded at {REFERENCE_BUDGET_S:.0f} s)")
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el * 1e3 / done, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "path": "CPU FP64 oracle", "lmax": args.lmax},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle", "sample": sample},
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
