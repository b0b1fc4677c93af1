"""Benchmark: leaf cell-updates/s per RK stage of the block-based MR Euler hot path.

Workload (N = 1): the shock-bubble interaction -- unit cube, base 2^3 blocks of
16^3 cells, levels 0..4 (effective 512^3), eps = 1e-3 at l_max, a planar Mach
1.22 shock at x = 0.27 moving +x into air at rest (rho 1, p 1, gamma 1.4) that
holds a light bubble (rho 0.14, radius 0.1 at (0.4, 0.5, 0.5), tanh edge two
finest cells wide), zero-gradient boundaries -- with the tree built by Alg.
(Initialization).  The learned WENO5/linear selector is trained on faces of the
Sod tube and of the spherical explosion only, never on this workload.  One step
= the library's mrb_step: CFL time step, three fused TVD-RK3 stages (halo fill,
RHS + update, jump correction, averaging), MR analysis and remesh.  value = sum
over the timed steps of (leaf internal cells at the step) x 3 stages / device
time of those steps.

The headline path is the FP32-bulk path with the learned selector (FP32
reconstruction and fluxes; FP64 state, update, conservation sums and time-step
reduction).  The FP32 WENO5 path and the all-FP64 path are timed on the same
workload and reported beside it, with the L1 density error of each FP32 path
against the FP64 path after the same steps from the same initial tree.  Side
lines: the MR spherical explosion (levels 0..3, effective 256^3) and the
memory-sized Rayleigh-Taylor layer (levels 0..5).  `--impl reference` times the
CPU oracle on the same workload.

Timing: CUDA events on the launching stream around every step (the bench line's
value is the K timed steps together; the median of the per-step rates is
reported beside it); the block pool is far larger than L2, so every step runs
from HBM.

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

# workload name -> (initial condition family, l_max, effective resolution)
WORKLOADS = {
    "shock_bubble_mr_512cubed_l4": ("shock_bubble", 4, "512^3"),
    "explosion_mr_256cubed_l3": ("explosion", 3, "256^3"),
    "rt_layer_mr_l5_memory_sized": ("rt", 5, "1024^2 x 2048"),
    # instances 0..15 of the 64-instance four-quadrant ensemble (levels 0..2+(i mod 3)),
    # one launch per RK stage for all sixteen (the 64 instances run as four such batches)
    "ensemble_quadrants_16_of_64": ("ensemble", None, "16 instances, 128^3 to 512^3"),
}
# pool blocks per four-quadrant instance by finest level, with room for the
# initialisation's transient refinement of the whole level below
QUAD_SLOTS = {2: 1200, 3: 6000, 4: 20000}
HEADLINE = "shock_bubble_mr_512cubed_l4"

# FP32-path variants timed beside the headline: (name, reconstruction, flux scheme)
VARIANTS = [("weno5_roe", 0, 0), ("linear5_roe", 2, 0), ("teno5_roe", 3, 0), ("wenoao53_roe", 4, 0),
            ("weno5_llf", 0, 1), ("teno5_llf", 3, 1), ("weno5_hllc", 0, 2), ("teno5_hllc", 3, 2),
            ("wenoao53_hllc", 4, 2)]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mrb", choices=["mrb", "reference"])
    ap.add_argument("--workload", default=HEADLINE, choices=sorted(WORKLOADS))
    ap.add_argument("--lmax", type=int, default=None, help="override the workload's finest level")
    ap.add_argument("--l1-steps", "--fp64-steps", dest="l1_steps", type=int, default=10,
                    help="steps of the FP64 path (timed after its first) and of the L1 comparison")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip timing the reconstruction/flux variants of the FP32 path")
    ap.add_argument("--no-side", action="store_true", help="skip the side-line workloads")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    # wrap the timed steps of one path (the headline, or the FP32 WENO5 path)
    # in cudaProfilerStart/Stop (for ncu --profile-from-start off)
    ap.add_argument("--profile-range", nargs="?", const="headline", default=None, choices=["headline", "weno"])
    ap.add_argument("--repeats", type=int, default=5,
                    help="timed regions of --steps steps on the headline path; value is their median")
    return ap.parse_args()


def workload_config(name: str, precision: int, lmax=None):
    """(run configuration, initial condition) of a named workload."""
    from paper_2012_04385_gb300 import inputs as I
    kind, lm, _ = WORKLOADS[name]
    lm = lm if lmax is None else lmax
    if kind == "shock_bubble":
        return I.shock_bubble_config(lmax=lm, precision=precision), I.ic_shock_bubble
    if kind == "explosion":
        return I.explosion_config(lmax=lm, precision=precision), I.ic_explosion
    if kind == "ensemble":
        return I.ensemble_config(n=16, precision=precision), I.ic_ensemble
    return I.rt_config(lmax=lm, precision=precision), I.ic_rt


def slots_for(cfg) -> int:
    if cfg.n_instances > 1:
        return int(sum(QUAD_SLOTS[cfg.lmax_of(i)] for i in range(cfg.n_instances)))
    # fully refined upper bound of the tree: sum_l 8^l * base blocks
    base = int(np.prod(cfg.base_blocks)) * cfg.n_instances
    return int(sum(base * 8 ** l for l in range(cfg.lmax_of(0) + 1)))


def memory_sized_slots(cfg, frac=0.75) -> int:
    """Pool blocks filling `frac` of the free device memory (the memory-sized
    workload), capped by the fully refined tree."""
    import torch

    from paper_2012_04385_gb300 import mrb
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    per = mrb.pool_bytes(cfg, 1000) / 1000
    return int(min(slots_for(cfg), frac * torch.cuda.mem_get_info()[0] / per))


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


def l1_density(a, b, cfg):
    """L1 density difference sum |rho_a - rho_b| / sum |rho_b| on the common
    finest uniform grid (leaf values injected piecewise constant).  On
    identical trees that is the leaf sum weighted by cell volume, computed
    without forming the grid.  a, b = (keys, geometry, rho[n, 16, 16, 16])."""
    (ka, ga, ra), (kb, gb, rb) = a, b
    if np.array_equal(ka, kb):
        w = np.ldexp(1.0, -3 * ga[:, 0].astype(np.int64))
        num = (w * np.abs(ra - rb).reshape(len(ka), -1).sum(axis=1)).sum()
        den = (w * np.abs(rb).reshape(len(kb), -1).sum(axis=1)).sum()
        return float(num / den), True
    fa, fb = finest_density(ka, ga, ra, cfg), finest_density(kb, gb, rb, cfg)
    return float(np.abs(fa - fb).sum() / np.abs(fb).sum()), False


def mirror_asymmetry(keys, geo, rho, cfg):
    """Largest |rho(x) - rho(mirror of x)| over the finest grid, for the mirror
    planes x = 1/2, y = 1/2, z = 1/2 of a symmetric problem, relative to max rho."""
    f = finest_density(keys, geo, rho, cfg)
    m = np.abs(f).max()
    return [float(np.abs(f - np.flip(f, axis=ax)).max() / m) for ax in (2, 1, 0)]


# Algorithmic FP32 FLOPs of the face flux, counted by running the oracle's own
# face-flux code on a counting number type (tests/golden/face_flops.json,
# written by oracle/count_flops.py; see that script for the rules).
FLOPS_FILE = os.path.join(ROOT, "tests", "golden", "face_flops.json")


def flop_table():
    try:
        return json.load(open(FLOPS_FILE))
    except Exception:
        return None


def roofline_numbers(linear_fraction=0.0, split=None, table=None):
    """Algorithmic FLOPs of the fused stage kernel per face and per leaf cell
    and stage.  `split[k]`: share of faces where characteristic field k takes
    the LLF split (the census of mrb_flux_census; fields 1-3 share the
    eigenvalue u and split together); `linear_fraction`: share of faces whose
    fields 0, 1, 4 take the linear scheme instead of WENO5 (averaged over the
    stages timed).  The counts are the oracle's own, measured on one block row
    of 16 cells and 17 faces (tests/golden/face_flops.json): the all-upwinded
    row plus the extra of each split pattern, and a linear reconstruction
    saving the difference of the two reconstructions' counts.  Per cell and
    stage: 3 directions x row / 16 + the flux differences + the update.  The
    selector's MLP runs on the tensor cores and is not counted."""
    t = table if table is not None else flop_table()
    if t is None:
        raise RuntimeError("tests/golden/face_flops.json missing: run python oracle/count_flops.py")
    s = split if split is not None else (0.0,) * 5
    w = {k: v[0] for k, v in t["row"]["weno5"].items()}
    s123, s0, s4 = s[1], s[0], s[4]
    per_row = (w["all_upwind"] + s123 * (w["split_123"] - w["all_upwind"]) + s0 * (w["split_0"] - w["all_upwind"])
               + s4 * (w["split_4"] - w["all_upwind"]))
    # reconstructions of fields 0, 1, 4 per face: one each, two where the field splits
    saving = t["recon"]["weno5"][0] - t["recon"]["linear5"][0]
    per_row -= linear_fraction * t["row"]["faces"] * saving * (3 + s123 + s0 + s4)
    per_face = per_row / t["row"]["faces"]
    per_cell = 3 * per_row / t["row"]["cells"] + t["cell"]["divergence"] + t["cell"]["update_rk3_mean"]
    return per_face, per_cell


# DRAM bytes (read + write) per leaf cell of one launch of the stage kernels
# on the shock-bubble workload (levels 0..4, 5,720 leaves), from the
# full-size ncu capture summarised in
# profiles/stage_kernels_shock_bubble_512.md: the mean over one step, for the
# learned path k_stage_f32<1> (250.8) and k_stage_f32<3> twice (222.6), for
# the WENO5 path k_stage_f32<0> (247.2 at stage 0, 222.2 at stages 1 and 2).
# Traffic grows in proportion to the leaf cells of a launch.
TRAFFIC_BYTES_PER_CELL = {"learned": 232.2, "weno": 230.6}


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


def release(*ctxs):
    import torch
    for c in ctxs:
        if c is not None:
            c.close()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def make_context(name, precision, lmax=None, recon=0, flux=0, tau=0.0, params=None, slots=None, stream=None, lts=0):
    from paper_2012_04385_gb300 import mrb
    cfg, ic = workload_config(name, precision, lmax)
    cfg.recon, cfg.flux, cfg.mlp_tau, cfg.lts = recon, flux, tau, lts
    ctx = mrb.Context(cfg, slots or slots_for(cfg), stream=stream, mlp_params=params if recon == 1 else None)
    t0 = time.perf_counter()
    if cfg.n_instances > 1:
        mrb.init_tree(ctx, ic, with_keys=True)
    else:
        mrb.init_tree(ctx, lambda c, geo: ic(c, geo))
    ctx.init_s = time.perf_counter() - t0
    return ctx


def timed_steps(ctx, stream, steps, warmup, profile=True, profiler_range=False, census=False):
    """Warm up, then time `steps` full steps with CUDA events on the launching
    stream (one pair around every step).  Returns the measurements."""
    import torch
    for _ in range(warmup):
        ctx.step(1)
    torch.cuda.synchronize()
    split0 = census_fractions(ctx) if census else None
    if profile:
        ctx.profile(True)
    ctx.learned_stats(reset=True)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    cells = []
    if profiler_range:
        torch.cuda.profiler.start()
    ev[0].record(stream)
    for s in range(steps):
        cells.append(ctx.n_leaves() * 4096 * 3)
        ctx.step(1)
        ev[s + 1].record(stream)
    torch.cuda.synchronize()
    if profiler_range:
        torch.cuda.profiler.stop()
    step_ms = [ev[s].elapsed_time(ev[s + 1]) for s in range(steps)]
    ms = ev[0].elapsed_time(ev[steps])
    kms, kn, nk = ctx.profile_read() if profile else (0.0, 0, 0)
    if profile:
        ctx.profile(False)
    lin, tot = ctx.learned_stats()
    # the census of the switch at the start and the end of the timed steps
    split = tuple(0.5 * (split0 + census_fractions(ctx))) if census else None
    rates = [c / (t * 1e-3) for c, t in zip(cells, step_ms)]
    return dict(ms=ms, cells=int(sum(cells)), step_ms=step_ms, median_rate=float(np.median(rates)),
                stage_ms=kms / max(kn, 1), stage_launches=kn, launches=nk,
                linear_fraction=(lin / tot) if tot else 0.0, split=split)


def leaf_density(ctx):
    k, g = ctx.list_blocks()
    return k, g, ctx.get_state(k).cpu().numpy()[:, 0]


def step_log(ctx, steps):
    """Per-step diagnostics of a run (outside any timed region): time step,
    leaves per level, compression C = 1 - cells / effective cells (Eq.
    Compression), conserved totals and the share of faces the selector sends
    to the linear scheme."""
    import torch
    cfg = ctx.cfg
    eff = cfg.effective_cells(0)
    out = []
    dt = torch.empty(cfg.n_instances, dtype=torch.float64, device="cuda")
    for s in range(steps):
        geo = ctx.geometry()
        lv = np.bincount(geo[:, 0], minlength=cfg.lmax_of(0) + 1)
        ctx.learned_stats(reset=True)
        ctx.step(1, dt_hist=dt)
        lin, tot = ctx.learned_stats()
        sums = ctx.sums().cpu().numpy()[0]
        out.append({"step": s, "dt": float(dt[0].item()), "leaves_per_level": [int(x) for x in lv],
                    "compression": 1.0 - len(geo) * 4096 / eff,
                    "totals": [float(x) for x in sums],
                    "linear_face_fraction": (lin / tot) if tot else None})
    return out


def fp64_run(name, stream, steps, lmax=None):
    """The all-FP64 GPU path on the workload: every step timed with CUDA
    events, the first one (graph capture) left out of the rate."""
    import torch

    from paper_2012_04385_gb300 import inputs as I
    ctx = make_context(name, I.FP64, lmax=lmax, stream=stream)
    ctx.profile(True)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    cells = []
    ev[0].record(stream)
    for s in range(steps):
        cells.append(ctx.n_leaves() * 4096 * 3)
        ctx.step(1)
        ev[s + 1].record(stream)
    torch.cuda.synchronize()
    kms, kn, _ = ctx.profile_read()
    ctx.profile(False)
    step_ms = [ev[s].elapsed_time(ev[s + 1]) for s in range(steps)]
    t = sum(step_ms[1:]) if steps > 1 else step_ms[0]
    c = sum(cells[1:]) if steps > 1 else cells[0]
    res = dict(value=c / (t * 1e-3), ms_per_step=t / max(steps - 1, 1), stage_ms=kms / max(kn, 1),
               timed_steps=max(steps - 1, 1), state=leaf_density(ctx), init_s=ctx.init_s)
    release(ctx)
    return res


def fp32_state_after(name, stream, steps, recon, tau=0.0, params=None, lmax=None, log=False):
    from paper_2012_04385_gb300 import inputs as I
    ctx = make_context(name, I.FP32_ACC64, lmax=lmax, recon=recon, tau=tau, params=params, stream=stream)
    lg = step_log(ctx, steps) if log else None
    if not log:
        ctx.step(steps)
    st = leaf_density(ctx)
    release(ctx)
    return st, lg


def run_gpu(args, rank, world):
    import torch

    from paper_2012_04385_gb300 import inputs as I
    from paper_2012_04385_gb300 import learned

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    ranks = Ranks(world, "nccl", "cuda")
    barrier, max_over_ranks, sum_over_ranks = ranks.barrier, ranks.max, ranks.sum
    name, lmax = args.workload, args.lmax
    stream = torch.cuda.current_stream()

    # ---- the learned selector, trained on the GPU by the library's own kernels
    t0 = time.perf_counter()
    data = learned.generate()
    params, tau, rep = learned.train(data, epochs=10)
    train_s = time.perf_counter() - t0

    # ---- headline: FP32 bulk + learned selector, timed region with clocks
    ctx = make_context(name, I.FP32_ACC64, lmax=lmax, recon=I.RECON_LEARNED, tau=tau, params=params, stream=stream)
    cfg = ctx.cfg
    # the project's autotuner picks the launch shapes on this tree (scheduling
    # only; the state is left as it was)
    tune = None if args.no_autotune else ctx.autotune(reps=3)
    keys0 = ctx.keys()
    pool_gb = ctx.pool.numel() / 1e9
    # `repeats` timed regions of exactly `steps` steps each, every one
    # bracketed by a barrier and a device synchronisation, max over ranks;
    # the first also takes the kernel profile and the census.  The headline
    # value is the median region's rate.
    barrier()
    sampler = ClockSampler(dev)
    sampler.start()
    m = timed_steps(ctx, stream, args.steps, args.warmup, profiler_range=args.profile_range == "headline",
                    census=True)
    barrier()
    regions = [(max_over_ranks(m["ms"]), sum_over_ranks(m["cells"]))]
    for _ in range(args.repeats - 1):
        barrier()
        r = timed_steps(ctx, stream, args.steps, 0, profile=False)
        barrier()
        regions.append((max_over_ranks(r["ms"]), sum_over_ranks(r["cells"])))
    clocks = sampler.stop()
    rates = [c / (t * 1e-3) for t, c in regions]
    med = int(np.argsort(rates)[len(rates) // 2])
    ms_max, value = regions[med][0], rates[med]

    # ---- end to end through the C ABI with host buffers (headline path)
    e2e = None
    if not args.no_e2e:
        # per step: H2D of the step's input state from pinned host memory,
        # mrb_set_cons + mrb_step + mrb_get_state, D2H of the result state and
        # the conservation sums
        keys = ctx.keys()
        n = len(keys)
        cap = min(ctx.n_slots, 2 * n)        # room for the tree to grow by refinement
        host = [torch.empty((cap, 5, 16, 16, 16), dtype=torch.float64).pin_memory() for _ in range(2)]
        dev_buf = torch.empty((cap, 5, 16, 16, 16), dtype=torch.float64, device="cuda")
        sums = torch.empty((1, 5), dtype=torch.float64, device="cuda")
        host_sums = torch.empty((1, 5), dtype=torch.float64).pin_memory()
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
            if n > cap:
                raise RuntimeError(f"tree grew past the end-to-end buffers ({n} > {cap} leaves)")
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
        del host, dev_buf
    release(ctx)
    ctx = None

    # ---- roofline of the fused stage kernel (FP32 CUDA cores)
    # stage 0 evaluates the selector with WENO5 fluxes; stages 1 and 2 use its decisions
    table = flop_table()
    per_face, per_cell = roofline_numbers(m["linear_fraction"] * 2 / 3, m["split"], table)
    pk = measured_peaks()
    clk = clocks["sm_mhz"] or pk.get("clocks_under_load", {}).get("sm_mhz_median") or 1447.0
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = nsm * 128 * 2 * clk * 1e6 / 1e12
    cells_per_launch = m["cells"] / 3 / args.steps
    achieved = cells_per_launch * per_cell / (m["stage_ms"] * 1e-3) / 1e12

    # ---- the same workload on the FP32 WENO5 path
    ctx = make_context(name, I.FP32_ACC64, lmax=lmax, stream=stream)
    tune_w = None if args.no_autotune else ctx.autotune(reps=3)
    mw = timed_steps(ctx, stream, args.steps, args.warmup, profiler_range=args.profile_range == "weno",
                     census=True)
    release(ctx)
    ctx = None
    value_w = sum_over_ranks(mw["cells"]) / (max_over_ranks(mw["ms"]) * 1e-3)
    _, pfw = roofline_numbers(0.0, mw["split"], table)
    achieved_w = (mw["cells"] / 3 / args.steps) * pfw / (mw["stage_ms"] * 1e-3) / 1e12

    # ---- the all-FP64 path, and the L1 density errors against it (same initial
    # tree, same steps)
    f64 = fp64_run(name, stream, args.l1_steps, lmax)
    st_l, log_l = fp32_state_after(name, stream, args.l1_steps, I.RECON_LEARNED, tau, params, lmax, log=True)
    st_w, _ = fp32_state_after(name, stream, args.l1_steps, I.RECON_WENO, lmax=lmax)
    l1_l, same_l = l1_density(st_l, f64["state"], cfg)
    l1_w, same_w = l1_density(st_w, f64["state"], cfg)
    del st_l, st_w

    # ---- reconstruction / flux variants of the FP32 path on the same workload
    variants = None
    if not args.no_variants:
        variants = {}
        vsteps = max(3, min(args.steps, 5))
        for vname, rec, fl in VARIANTS:
            ctx = make_context(name, I.FP32_ACC64, lmax=lmax, recon=rec, flux=fl, stream=stream)
            mv = timed_steps(ctx, stream, vsteps, 2)
            release(ctx)
            ctx = None
            variants[vname] = {"value": sum_over_ranks(mv["cells"]) / (max_over_ranks(mv["ms"]) * 1e-3),
                               "ms_per_step": mv["ms"] / vsteps, "stage_kernel_ms": mv["stage_ms"],
                               "steps": vsteps}

    # ---- local time stepping on the same workload (Eq. LtsTimestep): a macro
    # step advances every level by 2^lmax finest steps, level l in 2^l steps
    lts = None
    if not args.no_side:
        import torch as _t
        ctx = make_context(name, I.FP32_ACC64, lmax=lmax, recon=I.RECON_LEARNED, tau=tau, params=params,
                           stream=stream, lts=1)
        L = ctx.cfg.lmax_of(0)
        ctx.step(1)                                  # warm-up macro step
        nmac = 2
        dts = _t.empty((nmac, 1), dtype=_t.float64, device="cuda")
        ev0, ev1 = _t.cuda.Event(enable_timing=True), _t.cuda.Event(enable_timing=True)
        geo = ctx.geometry()
        lcells = sum(int((geo[:, 0] == l).sum()) * 4096 * 3 * (1 << l) for l in range(L + 1))
        _t.cuda.synchronize()
        ev0.record(stream)
        ctx.step(nmac, dt_hist=dts)
        ev1.record(stream)
        _t.cuda.synchronize()
        ms_l = ev0.elapsed_time(ev1)
        sim_t = float(dts.sum().item()) * (1 << L)
        lts = {"path": "FP32 bulk + learned selector, local time stepping", "macro_steps": nmac,
               "ms_per_macro_step": ms_l / nmac, "leaf_cell_updates_per_macro_step": lcells,
               "leaf_cell_updates_per_s": lcells * nmac / (ms_l * 1e-3),
               "simulated_time_per_s": sim_t / (ms_l * 1e-3),
               "global_stepping_simulated_time_per_s": (sum(log_l[i]["dt"] for i in range(len(log_l))) /
                                                         len(log_l)) / (m["ms"] / args.steps * 1e-3),
               "leaves_per_level": [int((geo[:, 0] == l).sum()) for l in range(L + 1)]}
        release(ctx)
        ctx = None

    # ---- side lines: the other single-GPU workloads of the family
    side = None
    if not args.no_side:
        side = {}
        for sname in WORKLOADS:
            if sname == name:
                continue
            kind = WORKLOADS[sname][0]
            slots = memory_sized_slots(workload_config(sname, I.FP32_ACC64)[0]) if kind == "rt" else None
            ctx = make_context(sname, I.FP32_ACC64, recon=I.RECON_LEARNED, tau=tau, params=params, slots=slots,
                               stream=stream)
            big = kind in ("rt", "ensemble")
            ssteps = 3 if big else max(3, min(args.steps, 10))
            ms_ = timed_steps(ctx, stream, ssteps, 1 if big else 2)
            entry = {"path": "FP32 bulk + learned selector", "value": ms_["cells"] / (ms_["ms"] * 1e-3),
                     "median_step_value": ms_["median_rate"], "ms_per_step": ms_["ms"] / ssteps,
                     "stage_kernel_ms": ms_["stage_ms"], "steps": ssteps, "leaf_blocks_end": ctx.n_leaves(),
                     "linear_fraction": ms_["linear_fraction"], "pool_gb": round(ctx.pool.numel() / 1e9, 1),
                     "init_s": round(ctx.init_s, 1)}
            if kind == "ensemble":
                inst = (ctx.keys() >> np.uint64(56)).astype(np.int64)
                entry["instances"] = int(ctx.cfg.n_instances)
                entry["leaf_blocks_per_instance"] = np.bincount(inst, minlength=ctx.cfg.n_instances).tolist()
            release(ctx)
            ctx = None
            if kind == "explosion":
                # the mirror symmetry of the symmetric explosion after a few steps,
                # FP64 and FP32 paths (the oracle's is checked by the tests)
                nsym = 5
                sym = {}
                f = fp64_run(sname, stream, nsym)
                sym["fp64"] = mirror_asymmetry(*f["state"], workload_config(sname, I.FP64)[0])
                for lab, rec in (("fp32_weno5", I.RECON_WENO), ("fp32_learned", I.RECON_LEARNED)):
                    s_, _ = fp32_state_after(sname, stream, nsym, rec, tau, params)
                    sym[lab] = mirror_asymmetry(*s_, workload_config(sname, I.FP64)[0])
                entry["mirror_asymmetry_xyz_after_5_steps"] = sym
            side[sname] = entry

    traffic_pc = TRAFFIC_BYTES_PER_CELL["learned"]
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 bulk (bf16 tensor-core selector) / f64 state+update", "data": "synthetic",
        "config": {"workload": name, "path": "FP32 bulk + FP64 accumulate, learned WENO5/linear selector",
                   "effective_resolution": WORKLOADS[name][2], "lmax": cfg.lmax_of(0),
                   "leaf_blocks_start": int(len(keys0)), "leaf_cells_start": int(len(keys0)) * 4096,
                   "l2": "inputs larger than L2 (block pool %.1f GB)" % pool_gb,
                   "selector_training": "Sod tube and MR spherical explosion faces only",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "median_step_value": m["median_rate"],
        "repeats": {"n": len(rates), "steps_each": args.steps, "values": rates,
                    "ms_per_step": [t / args.steps for t, _ in regions],
                    "note": "value is the median region; each region is timed like the contract's K steps"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak,
                     "traffic": (traffic_pc * cells_per_launch if traffic_pc else None),
                     "traffic_note": "ncu dram bytes per leaf cell of the stage kernels (profiles/) x the launch's leaf cells",
                     "kernel": "k_stage_f32<1> (stage 0, selector evaluated) + k_stage_f32<3> (stages 1, 2): fused RHS + RK stage",
                     "flops_per_cell_stage": per_cell, "flops_per_face": per_face,
                     "flops_source": "oracle op count (tests/golden/face_flops.json)",
                     "llf_split_share_per_field": [round(x, 4) for x in m["split"]],
                     "avg_launch_ms": m["stage_ms"], "launches": m["stage_launches"],
                     "peak_basis": f"FP32 CUDA cores {nsm} SMs x 128 lanes x 2 x {clk:.0f} MHz sampled"},
        "gpu_launches": int(m["launches"]),
        "autotune": {"learned_path": tune, "weno5_path": tune_w,
                     "params": "stage waves, item order (1 blocked), fill copy / predict CTAs per SM, "
                               "averaging CTAs per SM; times ms (default, tuned)"},
        "clocks": clocks,
        "selector": {"linear_fraction": m["linear_fraction"], "tau": tau, "train_s": round(train_s, 1),
                     "train_samples": rep["samples"], "holdout_accuracy": rep["holdout_accuracy"],
                     "holdout_missed_positives": rep["holdout_missed_positives"]},
        "fp32_weno_path": {"value": value_w, "unit": UNIT, "median_step_value": mw["median_rate"],
                           "ms_per_step": mw["ms"] / args.steps, "stage_kernel_ms": mw["stage_ms"],
                           "roofline_frac": achieved_w / fp32_peak, "flops_per_cell_stage": pfw,
                           "traffic": (TRAFFIC_BYTES_PER_CELL["weno"] * mw["cells"] / 3 / args.steps
                                       if TRAFFIC_BYTES_PER_CELL["weno"] else None)},
        "learned_vs_weno5_throughput": value / value_w,
        "fp64_path": {"value": f64["value"], "unit": UNIT, "timed_steps": f64["timed_steps"],
                      "ms_per_step": f64["ms_per_step"], "stage_kernel_ms": f64["stage_ms"]},
        "fp32_learned_vs_fp64_throughput": value / f64["value"],
        "l1_density_err_vs_fp64": {"fp32_learned": l1_l, "fp32_weno": l1_w, "steps": args.l1_steps,
                                   "same_tree": same_l and same_w, "bound": 1e-4},
        "step_log_fp32_learned": log_l,
    }
    if variants:
        result["fp32_variants"] = variants
    if side:
        result["side_lines"] = side
    if lts:
        result["local_time_stepping"] = lts
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
    cfg, ic = workload_config(args.workload, I.FP64, args.lmax)
    o = oracle.Oracle(cfg)
    oracle_init_tree(o, cfg, ic)
    cells = 0
    t0 = time.perf_counter()
    for _ in range(steps):
        cells += o.n_leaves() * 4096 * 3
        o.step(1)
    el = time.perf_counter() - t0
    return {"value": cells / el, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": f"{steps} full step(s) of {args.workload} from its initial tree "
                      f"({cells // 3 // 4096} leaf blocks), {el:.1f} s"}


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
    cfg, ic = workload_config(args.workload, I.FP64, args.lmax)
    o = oracle.Oracle(cfg)
    oracle_init_tree(o, cfg, ic)
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
    sample = (f"{done} of {args.steps} full oracle steps of {args.workload} after {min(args.warmup, 1)} warm-up "
              f"({el:.1f} s, bounded at {REFERENCE_BUDGET_S:.0f} s)")
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el * 1e3 / done, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "path": "CPU FP64 oracle", "lmax": cfg.lmax_of(0),
                       "effective_resolution": WORKLOADS[args.workload][2],
                       "parallelism": "single GPU" if world == 1 else "replicas"},
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
