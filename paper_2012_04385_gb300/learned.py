"""Training driver of the learned reconstruction selector (MRB_RECON_LEARNED).

The selector's data come from the method itself: faces of runs of the plain
Sod tube (2x2x2 blocks) and of the MR spherical explosion, sampled with
mrb_face_samples (features of the characteristic stencils, WENO-vs-linear
labels).  Training runs the library's own forward/backward kernels
(mrb_mlp_train_step, BF16 operands, FP32 accumulation, Adam) on the GPU.  The
logit threshold is then set on held-out faces so that at most `miss` of the
faces labelled "WENO needed" would be sent to the linear scheme.  Every call
here is argument marshalling around the C ABI; the arithmetic is in CUDA.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import inputs as I
from . import mrb

NPARAM = mrb.MLP_NPARAM


def init_params(seed: int = 0):
    """Seeded initial parameters: N(0, 1/fan_in) weights, zero biases."""
    rng = np.random.Generator(np.random.Philox(key=seed + 1000))
    w1 = rng.normal(0, 1 / np.sqrt(15), (32, 15))
    w2 = rng.normal(0, 1 / np.sqrt(32), (32, 32))
    w3 = rng.normal(0, 1 / np.sqrt(32), 32)
    return np.concatenate([w1.ravel(), np.zeros(32), w2.ravel(), np.zeros(32), w3, np.zeros(1)]).astype(np.float32)


@dataclasses.dataclass
class SelectorData:
    feats: object          # torch float32 [n, 16] (device)
    labels: object         # torch uint8 [n] (device)


def generate(tau_lab: float = 1e-5, sod_steps: int = 20, explosion_steps: int = 20, every: int = 4,
             stride: int = 7, explosion_lmax: int = 2) -> SelectorData:
    """Faces of the plain Sod tube and of the MR spherical explosion (FP32-bulk
    runs), sampled every `every` steps (every `stride`-th face)."""
    import torch
    feats, labels = [], []
    runs = [(I.sod_config(precision=I.FP32_ACC64), I.ic_sod, sod_steps),
            (I.explosion_config(lmax=explosion_lmax, precision=I.FP32_ACC64), I.ic_explosion, explosion_steps)]
    for cfg, ic, steps in runs:
        nslots = int(np.prod(cfg.base_blocks)) * sum(8 ** l for l in range(cfg.lmax_of(0) + 1))
        ctx = mrb.Context(cfg, nslots)
        mrb.init_tree(ctx, lambda c, geo: ic(c, geo))
        for s in range(steps + 1):
            if s % every == 0:
                ctx.fill_halos()
                f, l, _ = ctx.face_samples(tau_lab=tau_lab, stride=stride)
                feats.append(f.clone())
                labels.append(l.clone())
            if s < steps:
                ctx.step(1)
        ctx.close()
    return SelectorData(torch.cat(feats), torch.cat(labels))


def train(data: SelectorData, epochs: int = 20, batch: int = 16384, lr: float = 3e-3, pos_weight: float = 8.0,
          seed: int = 0, holdout: float = 0.1, miss: float = 1e-4, params=None):
    """Train on `data`; returns (params [1601] device float32, tau, report)."""
    import torch
    n = data.feats.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    perm = torch.randperm(n, generator=g).to(data.feats.device)
    nh = max(1, int(holdout * n))
    hold, tr = perm[:nh], perm[nh:]
    if params is None:
        params = torch.from_numpy(init_params(seed)).to(data.feats.device)
    trainer = mrb.MlpTrainer(params)
    losses = []
    for ep in range(epochs):
        order = tr[torch.randperm(tr.numel(), generator=g).to(tr.device)]
        for b0 in range(0, order.numel(), batch):
            idx = order[b0:b0 + batch]
            x = data.feats[idx].contiguous()
            y = data.labels[idx].contiguous()
            trainer.step(x, y, pos_weight=pos_weight, lr=lr)
        losses.append(float(trainer.loss.item()))
    # threshold on held-out faces: at most `miss` of the positives below tau
    z = mrb.mlp_logits(params, data.feats[hold].contiguous())
    y = data.labels[hold]
    tau = mrb.mlp_threshold(z, y.contiguous(), miss)
    lin = (z < tau)
    report = {"samples": int(n), "positives": float(data.labels.float().mean().item()), "losses": losses,
              "tau": tau, "holdout_linear_fraction": float(lin.float().mean().item()),
              "holdout_missed_positives": float((lin & (y == 1)).float().sum().item() / max(1, int((y == 1).sum()))),
              "holdout_accuracy": float(((z >= 0) == (y == 1)).float().mean().item())}
    return params, tau, report
