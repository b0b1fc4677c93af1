"""Runtime properties of the GPU path: batched instances against the oracle,
checkpoint / resume, run-to-run determinism, and recovery from a reported
non-physical state.
"""
import numpy as np
import pytest

import oracle
from paper_2012_04385_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2012_04385_gb300 import mrb  # noqa: E402


def oracle_init_tree(o, cfg, ic):
    """Alg. (Initialization) on the oracle, ic(cfg, geo, keys)."""
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


def l1_density(a, b):
    return float(np.abs(a[:, 0] - b[:, 0]).sum() / np.abs(b[:, 0]).sum())


def test_batched_ensemble_vs_oracle():
    """Three four-quadrant instances with uneven trees (levels 0..1, 0..2,
    0..1) in one pool and one launch per stage: FP64 bit-identical to the
    oracle (trees, per-instance time steps, states) after 2 steps; the FP32
    bulk path on the same batch within 1e-5 L1 density per instance."""
    cfg = I.ensemble_config(n=3, lmax=(1, 2, 1))
    o = oracle.Oracle(cfg)
    oracle_init_tree(o, cfg, I.ic_ensemble)
    g = mrb.Context(cfg, 3 * 8 * 73)
    mrb.init_tree(g, I.ic_ensemble, with_keys=True)
    assert np.array_equal(o.keys(leaves_only=False), g.keys(leaves_only=False))
    inst = (o.keys() >> np.uint64(56)).astype(np.int64)
    assert set(inst.tolist()) == {0, 1, 2}
    dts_o = o.step(2)
    dts_g = torch.empty((2, 3), dtype=torch.float64, device="cuda")
    g.step(2, dts_g)
    assert np.array_equal(dts_g.cpu().numpy(), dts_o)
    assert len(set(dts_o[0].tolist())) == 3            # every instance has its own time step
    assert np.array_equal(o.keys(leaves_only=False), g.keys(leaves_only=False))
    k = o.keys()
    ref = o.get_state(k)
    got = g.get_state(k).cpu().numpy()
    print("ensemble FP64: values not bit-identical:", np.count_nonzero(got != ref))
    assert np.array_equal(got, ref)
    # FP32 bulk + FP64 accumulation on the same batch
    cfg32 = I.ensemble_config(n=3, lmax=(1, 2, 1), precision=I.FP32_ACC64)
    g32 = mrb.Context(cfg32, 3 * 8 * 73)
    mrb.init_tree(g32, I.ic_ensemble, with_keys=True)
    g32.step(2)
    if np.array_equal(g32.keys(leaves_only=False), o.keys(leaves_only=False)):
        got32 = g32.get_state(k).cpu().numpy()
        kinst = (k >> np.uint64(56)).astype(np.int64)
        for i in range(3):
            e = l1_density(got32[kinst == i], ref[kinst == i])
            print("instance", i, "FP32 L1 density vs FP64:", e)
            assert e < 1e-5
    else:
        pytest.fail("FP32 path changed the tree within 2 steps")


def test_restart_continuation_bit_exact():
    """Checkpoint (all node ids + conserved states) after 2 steps, restore in
    a fresh context, and continue 2 steps: identical to the uninterrupted run."""
    cfg = I.explosion_config(lmax=2)
    a = mrb.Context(cfg, 8 * 73)
    mrb.init_tree(a, lambda c, geo: I.ic_explosion(c, geo))
    a.step(2)
    nodes = a.keys(leaves_only=False)
    snap = a.get_state(nodes).clone()
    b = mrb.Context(cfg, 8 * 73)
    mrb.restore_tree(b, nodes)
    b.set_cons(nodes, snap)
    a.step(2)
    b.step(2)
    assert np.array_equal(a.keys(leaves_only=False), b.keys(leaves_only=False))
    k = a.keys()
    assert torch.equal(a.get_state(k), b.get_state(k))


@pytest.mark.parametrize("precision", [I.FP64, I.FP32_ACC64])
def test_runs_are_deterministic(precision):
    """The same run twice gives bit-identical states (no floating-point
    atomics; every reduction in a fixed order)."""
    cfg = I.explosion_config(lmax=2, precision=precision)
    out = []
    for _ in range(2):
        g = mrb.Context(cfg, 8 * 73)
        mrb.init_tree(g, lambda c, geo: I.ic_explosion(c, geo))
        dts = torch.empty((3, 1), dtype=torch.float64, device="cuda")
        g.step(3, dts)
        k = g.keys()
        out.append((k, g.get_state(k).cpu().numpy(), dts.cpu().numpy(), g.sums().cpu().numpy()))
        g.close()
    assert np.array_equal(out[0][0], out[1][0])
    for q in range(1, 4):
        assert np.array_equal(out[0][q], out[1][q])


def test_nonphysical_state_is_reported_and_cleared():
    cfg = I.sod_config()
    g = mrb.Context(cfg, 8)
    k, geo = g.list_blocks()
    bad = I.ic_sod(cfg, geo)
    bad[3, 0, 5, 6, 7] = -0.5                   # negative density in one cell
    g.set_state(k, bad)
    g.cfl_dt()
    assert g.status() == mrb.MRB_ENONPHYS
    with pytest.raises(mrb.MrbError) as e:
        g.sync()
    assert e.value.code == mrb.MRB_ENONPHYS
    # repair the state, clear the status: the context keeps working
    g.set_state(k, I.ic_sod(cfg, geo))
    g.clear_status()
    g.step(2)
    g.sync()
    assert g.status() == mrb.MRB_OK
    assert np.isfinite(g.get_state(k).cpu().numpy()).all()


@pytest.mark.parametrize("recon", [I.RECON_WENO, I.RECON_LEARNED])
def test_fp32_records_follow_the_fp64_state(recon):
    """The mixed-precision path keeps FP32 primitive records of every node's
    internal cells (leaves and internal nodes, both stage buffers in turn) and
    its stage kernel reads them instead of converting the FP64 state.  After
    initialisation, after single stages with resolution jumps (the leaves
    after the stage update and jump correction, every node after the
    averaging) and after full steps with remeshing, the kept records equal a
    fresh conversion of the FP64 state bit for bit."""
    cfg = I.shock_bubble_config(lmax=2, precision=I.FP32_ACC64, recon=recon)
    params = None
    if recon == I.RECON_LEARNED:
        from paper_2012_04385_gb300 import learned
        params = torch.from_numpy(learned.init_params(3)).cuda()
        cfg.mlp_tau = 0.0
    g = mrb.Context(cfg, 600, mlp_params=params)
    mrb.init_tree(g, I.ic_shock_bubble)

    def check(what, leaves_only=False):
        k = g.keys(leaves_only=leaves_only)
        kept = g.get_records(k).cpu().numpy()
        fresh = g.get_records(k, fresh=True).cpu().numpy()
        bad = np.argwhere(kept.view(np.uint32) != fresh.view(np.uint32))
        assert len(bad) == 0, (what, len(bad), bad[:5])

    check("initial tree")
    dt = g.cfl_dt()
    for s in range(3):
        g.fill_halos()
        g.rk_stage(s, dt)
        check(f"stage {s}", leaves_only=True)     # internal nodes are averaged next
        g.mr_project()
        check(f"stage {s} averaged")
    g.step(3)
    assert g.status() == mrb.MRB_OK
    check("after 3 steps")
    g.close()


@pytest.mark.parametrize("precision", [I.FP64, I.FP32_ACC64])
def test_launch_shapes_do_not_change_results(precision):
    """The autotuner's knobs only schedule work: stage waves, work-item order,
    fill and averaging grid shapes give bit-identical trees and states after
    two MR steps (remeshing included); mrb_autotune leaves the state as it
    found it and the run continues bit for bit like an untuned one."""
    shapes = [[1, 0, 8, 4, 8], [2, 1, 4, 2, 4], [4, 0, 16, 8, 16], [1, 1, 1, 1, 1]]
    ref = None
    for q in shapes:
        cfg = I.shock_bubble_config(lmax=2, precision=precision)
        g = mrb.Context(cfg, 600)
        mrb.init_tree(g, I.ic_shock_bubble)
        g.set_tune(q)
        assert g.get_tune() == q
        g.step(2)
        assert g.status() == mrb.MRB_OK
        k = g.keys()
        st = g.get_state(k).cpu().numpy()
        if ref is None:
            ref = (k, st)
        else:
            assert np.array_equal(k, ref[0]), q
            assert np.array_equal(st.view(np.uint64), ref[1].view(np.uint64)), q
        g.close()
    with pytest.raises(mrb.MrbError):
        g = mrb.Context(I.shock_bubble_config(lmax=2, precision=precision), 600)
        g.set_tune([0, 0, 8, 4, 8])
    g = mrb.Context(I.shock_bubble_config(lmax=2, precision=precision), 600)
    mrb.init_tree(g, I.ic_shock_bubble)
    k0 = g.keys(leaves_only=False)
    s0 = g.get_state(k0).cpu().numpy()
    rep = g.autotune(reps=2)
    print(rep)
    assert np.array_equal(g.get_state(k0).cpu().numpy().view(np.uint64), s0.view(np.uint64))
    q = rep["params"]
    assert 1 <= q[0] <= 8 and q[1] in (0, 1) and all(1 <= x <= 32 for x in q[2:])
    assert rep["stage_ms"][1] <= rep["stage_ms"][0]
    g.step(2)
    k = g.keys()
    assert np.array_equal(k, ref[0])
    assert np.array_equal(g.get_state(k).cpu().numpy().view(np.uint64), ref[1].view(np.uint64))
    g.close()
