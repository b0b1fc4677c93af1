"""GPU checks of the learned reconstruction selector against the oracle.

Features and labels of sampled faces against the oracle's FP64 definition
(features within their FP32 bound, labels equal away from the decision
threshold), gradients of the training kernels against the FP64 reference
(same BF16 roundings), tensor-core logits against the reference forward, one
Adam step, training progress, and the learned path's accuracy against plain
WENO5 and against the FP64 oracle on an MR tree.
"""
import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from paper_2012_04385_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2012_04385_gb300 import learned, mrb  # noqa: E402


def _face_cells(U, li, fid_in_leaf):
    """Six lab-frame cells [6][5] of a face from a stored block array U [n][5][24][24][24]."""
    D, canon = fid_in_leaf // 4352, fid_in_leaf % 4352
    if D == 0:
        fx, y, z = canon % 17, (canon // 17) % 16, canon // 272
        cells = [(fx - 3 + m, y, z) for m in range(6)]
    elif D == 1:
        x, fy, z = canon % 16, (canon // 16) % 17, canon // 272
        cells = [(x, fy - 3 + m, z) for m in range(6)]
    else:
        x, y, fz = canon % 16, (canon // 16) % 16, canon // 256
        cells = [(x, y, fz - 3 + m) for m in range(6)]
    return D, np.array([U[li, :, k + 4, j + 4, i + 4] for (i, j, k) in cells])


EPS32 = 2.0 ** -23


def feature_bound(fo, S, k=64):
    """FP32 bound of each selector feature: the variation d = |dg| + alpha |dv|
    is a difference of FP32 values of size S (the field's largest |g| + alpha
    |v|), so its error is a few ulp of S; the compression sign(d) log10(1 +
    1e6 |d|) / 8 turns an error e of d into e 1e6 / (8 ln 10 (1 + 1e6 |d|)).
    k ulp of S, plus a few ulp of the feature itself."""
    d = (10.0 ** (8.0 * np.abs(fo)) - 1.0) / 1e6
    slope = 1e6 / (8.0 * np.log(10.0)) / (1.0 + 1e6 * d)
    return k * EPS32 * np.repeat(S, 5) * slope + 8 * EPS32


@pytest.mark.parametrize("ic_name", ["smooth", "rough"])
def test_features_and_labels_vs_oracle(ic_name):
    """Each sampled face's 15 features within their FP32 bound of the
    oracle's FP64 values, and its label equal to the oracle's wherever the
    oracle's decision margin |WENO5 - linear5| - threshold is larger than an
    FP32 budget (64 ulp of the values compared); faces inside the budget may
    go either way and must be rare."""
    cfg = I.periodic_config(base=(2, 1, 1), precision=I.FP32_ACC64)
    g = mrb.Context(cfg, 4)
    k, geo = g.list_blocks()
    prim = I.ic_random_smooth(cfg, geo) if ic_name == "smooth" else \
        I.random_states(len(k), seed=3, rho=(1.0, 1.5), p=(1.0, 1.5), vmax=0.3)
    g.set_state(k, prim)
    g.fill_halos()
    f, lab, where = g.face_samples(tau_lab=1e-3, stride=11, with_where=True)
    f, lab, where = f.cpu().numpy(), lab.cpu().numpy(), where.cpu().numpy()
    U = g.get_state(k, with_halo=True).cpu().numpy()
    n = len(where)
    worst, tight, near, mism = 0.0, 0, 0, []
    for s in range(n):
        li, fid = divmod(int(where[s]), 13056)
        D, U6 = _face_cells(U, li, fid)
        fo, lo, aux = oracle.face_features(U6, D, tau_lab=1e-3, with_aux=True)
        b = feature_bound(fo, aux[2:5])
        err = np.abs(f[s, :15] - fo)
        worst = max(worst, float((err / b).max()))
        tight += int((b < 1e-3).sum())
        budget = 64 * EPS32 * max(aux[1], aux[2:5].max())
        if abs(aux[0]) <= budget:
            near += 1
        elif lo != lab[s]:
            mism.append((s, lo, int(lab[s]), aux[0], budget))
    print(ic_name, "samples", n, "worst feature error / bound", worst, "features with bound < 1e-3",
          tight / (15 * n), "near-threshold faces", near / n, "positives", lab.mean())
    assert worst <= 1.0
    assert not mism, mism[:5]
    assert near <= 0.03 * n


def _rand_batch(n, seed):
    rng = np.random.default_rng(seed)
    X = np.zeros((n, 16), np.float32)
    X[:, :15] = rng.uniform(-1, 1, (n, 15))
    y = (rng.uniform(size=n) < 0.35).astype(np.uint8)
    return X, y


def test_training_gradient_vs_oracle():
    X, y = _rand_batch(3000, 1)
    p0 = learned.init_params(5) + np.random.default_rng(2).normal(0, 0.05, 1601).astype(np.float32)
    P = torch.from_numpy(p0.copy()).cuda()
    tr = mrb.MlpTrainer(P)
    grad = torch.zeros(1601, dtype=torch.float32, device="cuda")
    loss = tr.step(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), pos_weight=3.0, lr=0.0, grad=grad)
    gg = grad.cpu().numpy().astype(np.float64)
    lr_, gr = omlp.loss_and_grad(p0.astype(np.float64), X[:, :15].astype(np.float64), y, pos_weight=3.0, rounded=True)
    assert abs(float(loss.item()) - lr_) <= 1e-4 * abs(lr_)
    o = 0
    for name, shape in omlp.SIZES:
        m = int(np.prod(shape))
        a, b = gg[o:o + m], gr[o:o + m]
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        cos = float(a @ b / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30))
        print(name, "rel", rel, "cos", cos)
        assert rel <= 1e-2 and cos >= 0.999, name
        o += m
    # one Adam step matches the reference update given the same gradient
    P2 = torch.from_numpy(p0.copy()).cuda()
    tr2 = mrb.MlpTrainer(P2)
    tr2.step(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), pos_weight=3.0, lr=1e-2)
    ref, _, _ = omlp.adam(p0.astype(np.float64), gg, np.zeros(1601), np.zeros(1601), 1, lr=1e-2)
    assert np.abs(P2.cpu().numpy() - ref).max() < 1e-5


def test_tensor_core_logits_vs_oracle_forward():
    X, _ = _rand_batch(1000, 4)
    p0 = learned.init_params(7)
    z = mrb.mlp_logits(torch.from_numpy(p0).cuda(), torch.from_numpy(X).cuda()).cpu().numpy()
    zr, _ = omlp.forward(p0.astype(np.float64), X[:, :15].astype(np.float64), rounded=True)
    err = np.abs(z - zr)
    print("logit max abs err", err.max(), "scale", np.abs(zr).max())
    assert (err <= 2e-2 + 2e-2 * np.abs(zr)).all()


# Faces the selector stage evaluates per leaf and step: 17 x 16 x 16 x faces and
# as many y faces, and for each of the four 4-cell z slabs its 5 planes of 256
# z faces (the planes between slabs are evaluated by both).
SELECTOR_FACES_PER_LEAF_STEP = 2 * 17 * 16 * 16 + 4 * 5 * 256


@pytest.fixture(scope="module")
def small_selector():
    data = learned.generate(sod_steps=8, explosion_steps=6, every=3, stride=5, explosion_lmax=2)
    params, tau, rep = learned.train(data, epochs=6, batch=8192)
    return params, tau, rep


def test_training_lowers_loss_and_learned_path_accuracy(small_selector):
    params, tau, rep = small_selector
    print(rep)
    assert rep["losses"][-1] < rep["losses"][0]
    assert rep["holdout_missed_positives"] <= 0.01
    # learned FP32 path vs plain WENO5 FP32 path on the Sod tube
    res = {}
    for recon in (I.RECON_WENO, I.RECON_LEARNED):
        cfg = I.sod_config(precision=I.FP32_ACC64, recon=recon, mlp_tau=tau)
        g = mrb.Context(cfg, 8, mlp_params=params if recon == I.RECON_LEARNED else None)
        k, geo = g.list_blocks()
        g.set_state(k, I.ic_sod(cfg, geo))
        g.learned_stats(reset=True)
        g.step(20)
        res[recon] = g.get_state(k).cpu().numpy()
        if recon == I.RECON_LEARNED:
            lin, tot = g.learned_stats()
            print("faces sent to linear:", lin, "of", tot)
            assert tot == 20 * len(k) * SELECTOR_FACES_PER_LEAF_STEP   # the census is exact
            assert 0 < lin < tot
    a, b = res[I.RECON_LEARNED][:, 0], res[I.RECON_WENO][:, 0]
    l1 = np.abs(a - b).sum() / np.abs(b).sum()
    print("learned vs WENO L1 density difference:", l1)
    assert l1 <= 1e-4


def test_learned_path_vs_fp64_oracle_on_an_mr_tree(small_selector):
    """The headline accuracy bar checked against the oracle itself: the FP32 + learned
    path and the FP64 oracle (WENO5 everywhere) from the same initial MR tree
    (the explosion on levels 0..2, with resolution jumps) for 5 full steps,
    remeshing included: the same tree, and the L1 density difference on the
    finest grid (leaf cells weighted by volume) at most 1e-4."""
    params, tau, _ = small_selector
    cfg_g = I.explosion_config(lmax=2, precision=I.FP32_ACC64, recon=I.RECON_LEARNED, mlp_tau=tau)
    g = mrb.Context(cfg_g, 600, mlp_params=params)
    mrb.init_tree(g, I.ic_explosion)
    cfg_o = I.explosion_config(lmax=2)
    o = oracle.Oracle(cfg_o)
    o.set_state(o.keys(level=0), I.ic_explosion(cfg_o, o.geometry(level=0)))
    for m in range(1, 3):
        o.fill_halos()
        geo = o.geometry()
        o.remesh((geo[:, 0] == m - 1).astype(np.int8))
        o.set_state(o.keys(level=m), I.ic_explosion(cfg_o, o.geometry(level=m)))
        if m > 1:
            o.fill_halos()
            t, _ = o.predict_and_tag(allow_refine=False)
            o.remesh(t)
    o.project()
    assert np.array_equal(g.keys(), o.keys())
    g.learned_stats(reset=True)
    g.step(5)
    o.step(5)
    lin, tot = g.learned_stats()
    kg, geo = g.list_blocks()
    ko = o.keys()
    assert np.array_equal(kg, ko)
    rg = g.get_state(kg).cpu().numpy()[:, 0]
    ro = o.get_state(ko)[:, 0]
    w = np.ldexp(1.0, -3 * geo[:, 0].astype(np.int64))
    l1 = (w * np.abs(rg - ro).reshape(len(kg), -1).sum(1)).sum() / (w * np.abs(ro).reshape(len(ko), -1).sum(1)).sum()
    print(f"learned FP32 vs FP64 oracle after 5 steps: L1 density {l1:.2e}, faces sent to linear {lin / tot:.3f}")
    assert 0 < lin < tot
    assert l1 <= 1e-4


def test_threshold_is_the_quantile_of_the_label_1_logits():
    """mrb_mlp_threshold (radix selection on the device) against the linear-
    interpolation quantile of the label-1 logits: random logits with ties and
    both signs, a single label-1 sample, none, and the ends q = 0 and 1."""
    g = torch.Generator(device="cpu").manual_seed(7)
    cases = []
    for n, q, share in ((200_000, 1e-4, 0.3), (5_000, 0.5, 0.5), (777, 1.0, 0.2), (3_000, 0.0, 0.4),
                        (1_000, 0.37, 1.0)):
        z = (torch.randn(n, generator=g) * 3).float()
        z[: n // 10] = torch.round(z[: n // 10])             # ties
        y = (torch.rand(n, generator=g) < share).to(torch.uint8)
        cases.append((z, y, q))
    z1 = torch.randn(50, generator=g).float()
    y1 = torch.zeros(50, dtype=torch.uint8)
    y1[17] = 1
    cases.append((z1, y1, 0.25))
    for z, y, q in cases:
        want = float(torch.quantile(z[y == 1].double(), q).item())
        got = mrb.mlp_threshold(z.cuda(), y.cuda(), q)
        assert abs(got - want) <= 1e-6 * abs(want) + 1e-6, (q, got, want)
    none = mrb.mlp_threshold(z1.cuda(), torch.zeros(50, dtype=torch.uint8).cuda(), 0.5)
    assert none == 0.0
    with pytest.raises(mrb.MrbError):
        mrb.mlp_threshold(z1.cuda(), y1.cuda(), 1.5)
