"""GPU parity of local time stepping (Eq. LtsTimestep) against the oracle's
reading: per-level time steps inside a macro step, coarse levels first, every
node of a stepping level advanced, coarser levels interpolated in time for the
halo fills, levels averaged when their step ends and the integrated boundary-
face fluxes exchanged at the end of the macro step.

The FP64 path follows the oracle's operation order (no FMA contraction), so
trees must match bit for bit and states within 1e-11 per cell (reported: how
many values are not bit-identical); the FP32 path is checked for conservation
and against the FP64 path.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2012_04385_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2012_04385_gb300 import mrb  # noqa: E402

from test_gpu_parity import close, make_pair, wrap  # noqa: E402


def _lts(cfg):
    return dataclasses.replace(cfg, lts=1)


def test_lts_shock_bubble_macro_steps_bit_exact():
    """Shock-bubble tree on levels 1 and 2 (jumps where the shock and the
    bubble's edge are refined): two macro steps with the MR analysis and
    remeshing after each, FP64, against the oracle."""
    cfg = _lts(I.shock_bubble_config(lmax=2))
    g = mrb.Context(cfg, 600)
    mrb.init_tree(g, I.ic_shock_bubble)
    o = oracle.Oracle(cfg)
    o.set_state(o.keys(level=0), I.ic_shock_bubble(cfg, o.geometry(level=0)))
    for m in range(1, 3):
        o.fill_halos()
        geo = o.geometry()
        o.remesh((geo[:, 0] == m - 1).astype(np.int8))
        o.set_state(o.keys(level=m), I.ic_shock_bubble(cfg, o.geometry(level=m)))
        if m > 1:
            o.fill_halos()
            t, _ = o.predict_and_tag(allow_refine=False)
            o.remesh(t)
    o.project()
    assert np.array_equal(g.keys(), o.keys())
    assert len(set(o.geometry()[:, 0])) == 2
    for step in range(2):
        dt_o = o.step(1)
        dt_g = torch.empty(1, dtype=torch.float64, device="cuda")
        g.step(1, dt_hist=dt_g)
        assert g.status() == mrb.MRB_OK
        assert dt_o[0, 0] == dt_g.item()
        kg, ko = g.keys(), o.keys()
        assert np.array_equal(kg, ko), step
        n = close(g.get_state(kg).cpu().numpy(), o.get_state(ko), what=f"LTS macro step {step}")
        print("values not bit-identical:", n)


def test_lts_periodic_jumps_bit_exact_and_conservative():
    """Periodic domain with levels 1 to 3 (level-1 leaves facing level-3
    leaves across internal nodes of level 2): one macro step (eight micro
    steps, then the MR analysis) against the oracle, and the conserved
    totals to round-off."""
    cfg = _lts(I.periodic_config(base=(2, 2, 2), lmax=3))
    plans = [lambda g: np.ones(len(g), bool), lambda g: (g[:, 0] == 1) & (g[:, 1] == 1) & (g[:, 2] == 1),
             lambda g: (g[:, 0] == 2) & (g[:, 1] == 2)]
    o, g = make_pair(cfg, wrap(I.ic_random_smooth), plans, n_slots=2000)
    assert set(o.geometry()[:, 0]) == {1, 2, 3}
    s0 = g.sums().cpu().numpy()
    o.step(1)
    g.step(1)
    assert g.status() == mrb.MRB_OK
    kg, ko = g.keys(), o.keys()
    assert np.array_equal(kg, ko)
    U = g.get_state(kg).cpu().numpy()
    close(U, o.get_state(ko), what="LTS periodic macro step")
    s1 = g.sums().cpu().numpy()
    scale = np.abs(U).max(axis=(0, 2, 3, 4))
    assert (np.abs(s1 - s0) <= 1e-13 * np.maximum(np.abs(s0), scale)).all(), (s1 - s0)


def test_lts_fp32_path_conserves_and_follows_fp64():
    """The mixed-precision path under local time stepping: the same trees as
    the FP64 path over two macro steps of the shock-bubble case, L1 density
    within 1e-6 of it, and the totals conserved to the FP32 bound on a
    periodic tree with jumps."""
    res = {}
    for prec in (I.FP64, I.FP32_ACC64):
        cfg = _lts(I.shock_bubble_config(lmax=2, precision=prec))
        g = mrb.Context(cfg, 600)
        mrb.init_tree(g, I.ic_shock_bubble)
        g.step(2)
        assert g.status() == mrb.MRB_OK
        k, geo = g.list_blocks()
        res[prec] = (k, geo, g.get_state(k).cpu().numpy()[:, 0])
        g.close()
    (k64, geo, r64), (k32, _, r32) = res[I.FP64], res[I.FP32_ACC64]
    assert np.array_equal(k64, k32)
    w = np.ldexp(1.0, -3 * geo[:, 0].astype(np.int64))
    l1 = (w * np.abs(r32 - r64).reshape(len(k64), -1).sum(1)).sum() / (w * np.abs(r64).reshape(len(k64), -1).sum(1)).sum()
    print("LTS FP32 vs FP64 L1 density after 2 macro steps:", l1)
    assert l1 <= 1e-6
    cfg = _lts(I.periodic_config(base=(2, 2, 2), lmax=2, precision=I.FP32_ACC64, eps=1e-4))
    plans = [lambda g: np.ones(len(g), bool), lambda g: (g[:, 1] == 1) & (g[:, 2] == 2)]
    _, g = make_pair(cfg, wrap(I.ic_random_smooth), plans, n_slots=1000)
    s0 = g.sums().cpu().numpy()
    g.step(2)
    s1 = g.sums().cpu().numpy()
    assert np.abs(s1[0, 0] - s0[0, 0]) <= 2 * 3 * 8 * 2.0 ** -24 * abs(s0[0, 0])


@pytest.mark.parametrize("variant", ["rk2", "viscous", "hllc"])
def test_lts_variants_bit_exact(variant):
    """Local time stepping with the other schemes of the stage: TVD-RK2 (its
    stage times 0, 1 and flux weights 1/2, 1/2 in the time interpolation and
    the integrated fluxes), the viscous terms (their boundary-face fluxes
    enter the exchange) and the HLLC flux, FP64 on a periodic tree with
    levels 1 to 3, one macro step against the oracle, and the totals to
    round-off."""
    kw = {"rk2": dict(rk_stages=2), "viscous": dict(mu=0.02), "hllc": dict(flux=I.FLUX_HLLC)}[variant]
    cfg = _lts(I.periodic_config(base=(2, 2, 2), lmax=3, **kw))
    plans = [lambda g: np.ones(len(g), bool), lambda g: (g[:, 0] == 1) & (g[:, 1] == 1) & (g[:, 2] == 1),
             lambda g: (g[:, 0] == 2) & (g[:, 1] == 2)]
    o, g = make_pair(cfg, wrap(I.ic_random_smooth), plans, n_slots=2000)
    s0 = g.sums().cpu().numpy()
    o.step(1)
    g.step(1)
    assert g.status() == mrb.MRB_OK
    kg, ko = g.keys(), o.keys()
    assert np.array_equal(kg, ko)
    U = g.get_state(kg).cpu().numpy()
    n = close(U, o.get_state(ko), what=f"LTS {variant} macro step")
    print(variant, "values not bit-identical:", n)
    s1 = g.sums().cpu().numpy()
    scale = np.abs(U).max(axis=(0, 2, 3, 4))
    assert (np.abs(s1 - s0) <= 1e-13 * np.maximum(np.abs(s0), scale)).all(), (s1 - s0)
