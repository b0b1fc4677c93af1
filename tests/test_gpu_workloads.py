"""The paper-shaped workloads on the GPU against the oracle: the shock-bubble
interaction and the Rayleigh-Taylor layer (gravity source, symmetry walls) on
small trees, the MR explosion at its full size (levels 0..3, 256^3
effective) in the launch configuration the benchmark times, free-stream
preservation on every GPU path across resolution jumps, and the viscous
single-mode Rayleigh-Taylor growth rate against the linear theory.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2012_04385_gb300 import inputs as I
from rti_theory import growth_rate

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2012_04385_gb300 import learned, mrb  # noqa: E402


def oracle_init_tree(o, cfg, ic):
    """Alg. (Initialization) on the oracle (same sequence as mrb.init_tree)."""
    lmax = max(cfg.lmax_of(i) for i in range(cfg.n_instances))
    o.set_state(o.keys(), ic(cfg, o.geometry()))
    for m in range(1, lmax + 1):
        o.fill_halos()
        geo = o.geometry()
        o.remesh((geo[:, 0] == m - 1).astype(np.int8))
        o.set_state(o.keys(level=m), ic(cfg, o.geometry(level=m)))
        if m > 1:
            o.fill_halos()
            t, _ = o.predict_and_tag(allow_refine=False)
            o.remesh(t)
    o.project()


def slots(cfg):
    base = int(np.prod(cfg.base_blocks)) * cfg.n_instances
    return int(sum(base * 8 ** l for l in range(max(cfg.lmax_of(i) for i in range(cfg.n_instances)) + 1)))


def run_pair(cfg, ic, nsteps):
    o = oracle.Oracle(cfg)
    oracle_init_tree(o, cfg, ic)
    g = mrb.Context(cfg, slots(cfg))
    mrb.init_tree(g, ic)
    assert np.array_equal(o.keys(leaves_only=False), g.keys(leaves_only=False))
    dts_o = o.step(nsteps)
    dts_g = torch.empty((nsteps, cfg.n_instances), dtype=torch.float64, device="cuda")
    g.step(nsteps, dts_g)
    return o, g, dts_o, dts_g.cpu().numpy()


@pytest.mark.parametrize("name", ["shock_bubble", "rayleigh_taylor"])
def test_paper_workloads_fp64_bit_exact(name):
    if name == "shock_bubble":
        cfg, ic, n = I.shock_bubble_config(lmax=2), I.ic_shock_bubble, 3
    else:
        cfg, ic, n = I.rt_config(lmax=1), I.ic_rt, 3
    o, g, dts_o, dts_g = run_pair(cfg, ic, n)
    assert np.array_equal(dts_g, dts_o)
    assert np.array_equal(o.keys(leaves_only=False), g.keys(leaves_only=False))
    k = o.keys()
    ref, got = o.get_state(k), g.get_state(k).cpu().numpy()
    print(name, "leaves", len(k), "values not bit-identical:", np.count_nonzero(got != ref))
    assert np.array_equal(got, ref)


@pytest.mark.slow
def test_full_size_explosion_one_step_vs_oracle():
    """The benchmark's workload (levels 0..3, initial tree about 2500 leaves):
    one full step of the FP64 GPU path is bit-identical to the oracle's, and
    the FP32 bulk path is within 1e-5 L1 density of it."""
    cfg = I.explosion_config(lmax=3)
    o, g, dts_o, dts_g = run_pair(cfg, I.ic_explosion, 1)
    assert np.array_equal(dts_g, dts_o)
    assert np.array_equal(o.keys(leaves_only=False), g.keys(leaves_only=False))
    k = o.keys()
    ref = o.get_state(k)
    assert np.array_equal(g.get_state(k).cpu().numpy(), ref)
    g32 = mrb.Context(I.explosion_config(lmax=3, precision=I.FP32_ACC64), slots(cfg))
    mrb.init_tree(g32, I.ic_explosion)
    g32.step(1)
    assert np.array_equal(g32.keys(leaves_only=False), o.keys(leaves_only=False))
    got = g32.get_state(k).cpu().numpy()
    l1 = np.abs(got[:, 0] - ref[:, 0]).sum() / np.abs(ref[:, 0]).sum()
    print("full size, FP32 bulk L1 density vs oracle after one step:", l1)
    assert l1 < 1e-5


@pytest.fixture(scope="module")
def selector():
    data = learned.generate(sod_steps=6, explosion_steps=4, every=3, stride=9, explosion_lmax=2)
    params, tau, _ = learned.train(data, epochs=3, batch=8192)
    return params, tau


@pytest.mark.parametrize("path", ["fp64", "fp32_weno", "fp32_linear", "fp32_learned", "fp64_hllc", "fp32_hllc",
                                  "fp32_llf", "fp32_wenoao", "fp64_viscous", "fp32_viscous"])
def test_free_stream_preserved(path, selector):
    """A uniform state on a tree with resolution jumps: the RHS is bitwise
    zero (identical face fluxes cancel; prediction of a constant is exact), so
    after 4 steps every cell still holds one and the same value, within the
    rounding of the TVD-RK3 convex combinations (2 ulp per step) of the
    initial one."""
    kw = dict(precision=I.FP64) if path.startswith("fp64") else dict(precision=I.FP32_ACC64)
    if path.endswith("hllc"):
        kw["flux"] = I.FLUX_HLLC
    if path == "fp32_llf":
        kw["flux"] = I.FLUX_LLF
    if path == "fp32_wenoao":
        kw["recon"] = I.RECON_WENOAO
    if path.endswith("viscous"):
        kw["mu"] = 0.01
    if path == "fp32_linear":
        kw["recon"] = I.RECON_LINEAR
    if path == "fp32_learned":
        kw["recon"], kw["mlp_tau"] = I.RECON_LEARNED, selector[1]
    cfg = I.periodic_config(base=(2, 2, 2), lmax=2, **kw)
    g = mrb.Context(cfg, 8 * 73, mlp_params=selector[0] if path == "fp32_learned" else None)
    k, geo = g.list_blocks()
    g.set_state(k, I.ic_uniform(cfg, geo))
    g.fill_halos()
    mask = (geo[:, 1] == 0).astype(np.int8)           # refine half of the blocks: jumps
    g.remesh(mask)
    k, geo = g.list_blocks()
    g.set_state(k, I.ic_uniform(cfg, geo))
    g.mr_project()
    g.fill_halos()
    assert np.count_nonzero(g.compute_rhs().cpu().numpy()) == 0, path
    u0 = g.get_state(k).cpu().numpy()
    g.step(4)
    assert np.array_equal(g.keys(), k)
    u1 = g.get_state(k).cpu().numpy()
    for v in range(5):
        vals = np.unique(u1[:, v])
        assert vals.size == 1, (path, v)
        ref = u0[0, v, 0, 0, 0]
        assert abs(vals[0] - ref) <= 2 * 4 * np.spacing(abs(ref)) + 1e-300, (path, v)


def _centreline_interface(g, cfg, k, mid):
    """Height of the interface (the crossing of the mid density) on the
    vertical centreline x = lambda / 2, from the leaves that hold it (cell
    values weighted linearly around x = lambda / 2, averaged over y)."""
    lam = 2.0 * math.pi / k
    keys, geo = g.list_blocks()
    dxs = cfg.dx0 * 0.5 ** geo[:, 0]
    x0 = geo[:, 1] * 16 * dxs
    sel = (x0 <= lam / 2) & (x0 + 16 * dxs >= lam / 2)
    U = g.get_state(keys[sel]).cpu().numpy()
    zs, rs = [], []
    for b, (lvl, X, _, Z) in enumerate(geo[sel]):
        dx = cfg.dx0 * 0.5 ** lvl
        xc = (X * 16 + np.arange(16) + 0.5) * dx
        w = np.maximum(0.0, 1.0 - np.abs(xc - lam / 2) / dx)
        if w.sum() == 0:
            continue
        zs.append((Z * 16 + np.arange(16) + 0.5) * dx)
        rs.append(((U[b, 0] * w).sum(axis=2) / w.sum()).mean(axis=1))
    z, r = np.concatenate(zs), np.concatenate(rs)
    o = np.argsort(z, kind="stable")
    z, r = z[o], r[o]
    i = np.where((r[:-1] - mid) * (r[1:] - mid) <= 0)[0]
    j = i[np.argmin(np.abs(z[i] - 5.0 * lam))]
    return z[j] + (mid - r[j]) * (z[j + 1] - z[j]) / (r[j + 1] - r[j])


@pytest.mark.parametrize("k", [2.0, 5.0])
def test_viscous_rti_growth_rate_vs_linear_theory(k):
    """Sec. 5's viscous Rayleigh-Taylor growth-rate study (At = 0.5, mu = 0.1,
    g = 1, equal dynamic viscosities): a single mode of wavenumber k on a
    lambda x 10 lambda column (64 cells per wavelength at the finest level),
    FP32 bulk path with the viscous terms and gravity.  The interface
    displacement d(t) on the centreline grows as exp(n t); n is fitted on
    2 <= d / d(0) <= 6 (still linear: k d <= 0.3) and must match the root of
    Eq. (SinglePhaseGrowth) within 5%."""
    cfg = I.rti_growth_config(k, precision=I.FP32_ACC64)
    lam = 2.0 * math.pi / k
    rho_h, rho_l, _ = I.RTI_FLUIDS[0.5]
    mid = 0.5 * (rho_h + rho_l)
    g = mrb.Context(cfg, 6000)
    mrb.init_tree(g, lambda c, geo: I.ic_rti_single_mode(c, geo, k))
    d0 = 5.0 * lam - _centreline_interface(g, cfg, k, mid)
    assert abs(d0 - 0.05 / k) < 0.1 * 0.05 / k
    n_th = growth_rate(k, rho_h, rho_l, I.RTI_FLUIDS[0.5][2])
    dts = torch.empty((50, 1), dtype=torch.float64, device="cuda")
    t, ts, ds = 0.0, [0.0], [d0]
    while ds[-1] / d0 < 7.0 and t < 15.0 / n_th:
        g.step(50, dts)
        t += float(dts.sum())
        ts.append(t)
        ds.append(5.0 * lam - _centreline_interface(g, cfg, k, mid))
    assert g.status() == mrb.MRB_OK
    ts, ratio = np.array(ts), np.array(ds) / d0
    w = (ratio >= 2.0) & (ratio <= 6.0)
    assert w.sum() >= 5
    n_fit = np.polyfit(ts[w], np.log(ratio[w]), 1)[0]
    print(f"k = {k}: growth rate {n_fit:.4f}, linear theory {n_th:.4f}, relative {(n_fit - n_th) / n_th:+.3f}, "
          f"t = {t:.2f}, {g.n_leaves()} leaves")
    assert abs(n_fit - n_th) <= 0.05 * n_th
