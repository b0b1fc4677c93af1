"""The paper-shaped configurations at their full sizes on the GPU.

The oracle cannot run these within a test's time, so they are checked through
properties that hold at any size:

* the batched ensemble of 64 four-quadrant problems, instance i on levels
  0..2 + (i mod 3) (3 to 5 levels).  Its trees need about 265,000 blocks,
  which at 1.61 MB per FP32-path pool block is more than one GPU's memory, so the 64
  instances run as four batches of 16, one launch per RK stage each.  Inside a
  batch every instance evolves exactly as it does alone (bit-identical trees
  and states), and the FP32 bulk path stays within 1e-5 L1 density of the
  FP64 path per instance;
* the shock-bubble interaction on levels 0..4 (512^3 effective) with the
  learned selector trained on Sod and explosion faces only: the FP32 +
  learned path within 1e-4 L1 density of the FP64 path;
* the Rayleigh-Taylor layer on levels 0..5 (1024^2 x 2048 effective), FP32
  bulk with the learned selector, the block pool sized to three quarters of
  free HBM: total mass conserved over steps with remeshing (periodic sides,
  symmetry walls) up to the FP32 rounding of the per-cell increments.  Each
  cell's increment b dt/dx (sum of flux differences) is rounded twice in FP32
  before the FP64 accumulation, and per stage the increments' magnitudes sum
  to less than the total mass, so |dM| <= stages x 2 x 2^-24 x M.
"""
import dataclasses

import numpy as np
import pytest

from paper_2012_04385_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2012_04385_gb300 import learned, mrb  # noqa: E402

# pool blocks per four-quadrant instance by finest level, with room for the
# initialisation's transient refinement of the whole level below
QUAD_SLOTS = {2: 1200, 3: 6000, 4: 20000}
INST_MASK = np.uint64((1 << 56) - 1)


def free_bytes():
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return torch.cuda.mem_get_info()[0]


def release(*ctxs):
    for c in ctxs:
        c.close()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def quad_batch(first, n, precision):
    """Instances first .. first+n-1 of the 64-instance ensemble as one batch."""
    lm = tuple(2 + ((first + j) % 3) for j in range(n))
    cfg = dataclasses.replace(I.ensemble_config(n=n, precision=precision), lmax=lm)

    def ic(c, geo, keys):
        inst = (np.asarray(keys, np.uint64) >> np.uint64(56)).astype(np.int64)
        out = np.zeros((len(geo), 5, 16, 16, 16))
        for j in np.unique(inst):
            sel = inst == j
            out[sel] = I.ic_four_quadrant(c, geo[sel], inst=first + int(j))
        return out
    return cfg, ic, sum(QUAD_SLOTS[l] for l in lm)


def run(cfg, ic, slots, nsteps, **kw):
    assert mrb.pool_bytes(cfg, slots) < 0.92 * free_bytes(), "pool would not fit"
    g = mrb.Context(cfg, slots, **kw)
    mrb.init_tree(g, ic, with_keys=True)
    g.step(nsteps)
    assert g.status() == mrb.MRB_OK
    return g


def instance_state(g, inst):
    k = g.keys()
    sel = (k >> np.uint64(56)) == np.uint64(inst)
    return (k[sel] & INST_MASK), g.get_state(k[sel]).cpu().numpy()


def test_ensemble_64_full_size_batches():
    nsteps = 2
    for b in range(4):
        first = 16 * b
        cfg, ic, slots = quad_batch(first, 16, I.FP32_ACC64)
        g = run(cfg, ic, slots, nsteps)
        inst = (g.keys() >> np.uint64(56)).astype(np.int64)
        print(f"batch {b}: instances {first}..{first + 15}, {len(inst)} leaves, "
              f"per instance {np.bincount(inst).tolist()}")
        assert set(inst.tolist()) == set(range(16))
        # sampled instances (one per finest level) alone: FP32 bit-identical, FP64 within 1e-5 L1;
        # the batch's states are copied to the host and its pool released first
        sampled = {j: instance_state(g, j) for j in (b % 3, 3 + (b + 1) % 3, 6 + (b + 2) % 3)}
        release(g)
        del g
        for j, (kb, ub) in sampled.items():
            lm = 2 + ((first + j) % 3)
            for prec in (I.FP32_ACC64, I.FP64):
                c1 = dataclasses.replace(I.ensemble_config(n=1, precision=prec), lmax=(lm,))
                a = run(c1, lambda c, geo, keys, i=first + j: I.ic_four_quadrant(c, geo, inst=i), QUAD_SLOTS[lm],
                        nsteps)
                ka, ua = instance_state(a, 0)
                assert np.array_equal(ka, kb), (b, j, prec)
                if prec == I.FP32_ACC64:
                    assert np.array_equal(ua, ub), (b, j)
                else:
                    l1 = np.abs(ub[:, 0] - ua[:, 0]).sum() / np.abs(ua[:, 0]).sum()
                    print(f"  instance {first + j} (levels 0..{lm}, {len(ka)} leaves): FP32 batch vs FP64 alone L1 {l1:.2e}")
                    assert l1 < 1e-5
                release(a)
                del a


@pytest.fixture(scope="module")
def selector():
    data = learned.generate()
    params, tau, _ = learned.train(data, epochs=10)
    return params, tau


def test_shock_bubble_levels_0_4_learned_vs_fp64(selector):
    params, tau = selector
    nsteps = 10
    res = {}
    for name, kw in (("fp64", dict(precision=I.FP64)),
                     ("learned", dict(precision=I.FP32_ACC64, recon=I.RECON_LEARNED, mlp_tau=tau))):
        cfg = I.shock_bubble_config(lmax=4, **kw)
        g = mrb.Context(cfg, 16000, mlp_params=params if name == "learned" else None)
        mrb.init_tree(g, I.ic_shock_bubble)
        g.learned_stats(reset=True)
        g.step(nsteps)
        assert g.status() == mrb.MRB_OK
        k = g.keys()
        res[name] = (k, g.get_state(k).cpu().numpy()[:, 0])
        if name == "learned":
            lin, tot = g.learned_stats()
            print(f"shock-bubble levels 0..4: {len(k)} leaves, faces sent to linear {lin / tot:.3f}")
        release(g)
    (k64, r64), (kl, rl) = res["fp64"], res["learned"]
    common, i64, il = np.intersect1d(k64, kl, return_indices=True)
    print(f"leaves FP64 {len(k64)}, learned {len(kl)}, common {len(common)}")
    assert len(common) >= 0.99 * len(k64)
    l1 = np.abs(rl[il] - r64[i64]).sum() / np.abs(r64[i64]).sum()
    print(f"learned FP32 vs FP64 L1 density after {nsteps} steps: {l1:.2e}")
    assert l1 <= 1e-4


def test_rayleigh_taylor_levels_0_5_memory_sized(selector):
    params, tau = selector
    cfg = I.rt_config(lmax=5, precision=I.FP32_ACC64, recon=I.RECON_LEARNED, mlp_tau=tau)
    slots = int(0.75 * free_bytes() / (mrb.pool_bytes(cfg, 1000) / 1000))
    g = mrb.Context(cfg, slots, mlp_params=params)
    print(f"pool: {slots} blocks, {g.pool.numel() / 1e9:.1f} GB")
    mrb.init_tree(g, I.ic_rt)
    s0 = g.sums().cpu().numpy()
    n0 = g.n_leaves()
    nsteps = 4
    g.step(nsteps)
    assert g.status() == mrb.MRB_OK
    s1 = g.sums().cpu().numpy()
    dm = abs(s1[0, 0] - s0[0, 0]) / abs(s0[0, 0])
    print(f"leaves {n0} -> {g.n_leaves()}; mass {s0[0, 0]!r} -> {s1[0, 0]!r}, relative change {dm:.2e}")
    assert dm <= 3 * nsteps * 2 * 2.0 ** -24
    release(g)
