"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds run configurations and initial conditions only: none of the
method's arithmetic.  Both the CUDA library and the CPU oracle take their inputs
from here.  Random numbers come from splitmix64 (Steele, Lea & Flood, 2014)
evaluated on a counter (seed, instance, stream, index), so every draw is
reproducible on any machine.

Initial conditions are functions of block geometry rows (level, X, Y, Z) as
listed by either implementation, and return primitive states
prim[n, 5, 16, 16, 16] = (rho, u, v, w, p) of the internal cells (index order
[var][z][y][x]).  Discontinuous initial conditions are cell-centre point values;
the smooth convergence case uses exact cell averages.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Sequence

import numpy as np

NB = 16
BC_ZERO_GRADIENT, BC_PERIODIC, BC_SYMMETRY = 0, 1, 2
FP64, FP32_ACC64 = 0, 1
RECON_WENO, RECON_LEARNED, RECON_LINEAR, RECON_TENO, RECON_WENOAO = 0, 1, 2, 3, 4
FLUX_ROE, FLUX_LLF, FLUX_HLLC = 0, 1, 2


@dataclasses.dataclass
class RunConfig:
    n_instances: int = 1
    base_blocks: Sequence[int] = (2, 2, 2)
    lmax: Sequence[int] = (0,)
    domain_lo: Sequence[float] = (0.0, 0.0, 0.0)
    dx0: float = 1.0 / 32.0
    gamma: float = 1.4
    B: float = 0.0
    cfl: float = 0.6
    gravity: Sequence[float] = (0.0, 0.0, 0.0)
    bc: Sequence[int] = (BC_ZERO_GRADIENT,) * 6
    eps: float = 1e-3
    precision: int = FP64
    recon: int = RECON_WENO
    rk_stages: int = 3          # 3: TVD-RK3, 2: TVD-RK2
    flux: int = FLUX_ROE        # Roe with per-field LLF fallback, LLF, or HLLC
    mu: float = 0.0             # dynamic viscosity (Navier-Stokes terms); 0 = Euler
    lts: int = 0                # 1: local time stepping per level (Eq. LtsTimestep)
    mlp_tau: float = 0.0
    name: str = "custom"

    def lmax_of(self, inst: int) -> int:
        return int(self.lmax[inst] if len(self.lmax) > 1 else self.lmax[0])

    def effective_cells(self, inst: int = 0) -> int:
        l = self.lmax_of(inst)
        return int(np.prod(self.base_blocks)) * NB ** 3 * 8 ** l


# ------------------------------------------------------------------ configs
def sod_config(**kw) -> RunConfig:
    """Plain single-level Sod tube: 2x2x2 blocks of 16^3 (32^3 cells), FP64,
    zero-gradient in x, periodic in y and z, CFL 0.6, 20 steps."""
    c = RunConfig(name="sod_32cubed_l0", base_blocks=(2, 2, 2), lmax=(0,), dx0=1.0 / 32.0,
                  bc=(BC_ZERO_GRADIENT, BC_ZERO_GRADIENT, BC_PERIODIC, BC_PERIODIC, BC_PERIODIC, BC_PERIODIC))
    return dataclasses.replace(c, **kw)


def explosion_config(lmax: int = 3, **kw) -> RunConfig:
    """MR spherical explosion: unit cube, base 2^3 blocks of 16^3, levels 0..lmax
    (lmax = 3 gives an effective 256^3), eps = 1e-3 at lmax, zero-gradient."""
    c = RunConfig(name=f"explosion_l{lmax}", base_blocks=(2, 2, 2), lmax=(lmax,), dx0=1.0 / 32.0, eps=1e-3)
    return dataclasses.replace(c, **kw)


def ensemble_config(n: int = 64, **kw) -> RunConfig:
    """Batched ensemble: n unit-cube four-quadrant Riemann problems, instance i
    with lmax = 2 + (i mod 3) (3 to 5 levels), base 2^3 blocks, zero-gradient."""
    c = RunConfig(name=f"ensemble_{n}", n_instances=n, base_blocks=(2, 2, 2),
                  lmax=tuple(2 + (i % 3) for i in range(n)), dx0=1.0 / 32.0, eps=1e-3)
    return dataclasses.replace(c, **kw)


def shock_bubble_config(lmax: int = 4, **kw) -> RunConfig:
    """Shock-bubble interaction: unit cube, base 2^3, lmax 4 (effective 512^3)."""
    c = RunConfig(name=f"shock_bubble_l{lmax}", base_blocks=(2, 2, 2), lmax=(lmax,), dx0=1.0 / 32.0, eps=1e-3)
    return dataclasses.replace(c, **kw)


def rt_config(lmax: int = 5, **kw) -> RunConfig:
    """Density-stratified layer under gravity: [0,1]x[0,1]x[0,2], base 2x2x4,
    lmax 5 (effective 1024^2 x 2048), periodic x/y, symmetry z, g = (0,0,-1)."""
    c = RunConfig(name=f"rt_layer_l{lmax}", base_blocks=(2, 2, 4), lmax=(lmax,), dx0=1.0 / 32.0,
                  gravity=(0.0, 0.0, -1.0), eps=1e-3,
                  bc=(BC_PERIODIC, BC_PERIODIC, BC_PERIODIC, BC_PERIODIC, BC_SYMMETRY, BC_SYMMETRY))
    return dataclasses.replace(c, **kw)


# Fluid properties of the viscous single-mode Rayleigh-Taylor growth-rate study
# by Atwood number: rho_heavy, rho_light, mu (the table of the RTI section).
RTI_FLUIDS = {0.5: (1.5, 0.5, 0.1), 0.998: (99.9, 0.1, 0.5)}


def rti_growth_config(k: float, atwood: float = 0.5, lmax: int = 2, **kw) -> RunConfig:
    """Viscous single-mode Rayleigh-Taylor set-up of the growth-rate study:
    the short side (x) spans one wavelength 2 pi / k between symmetry walls,
    the long side (z, gravity -1) ten wavelengths between walls, one block in y
    (periodic, the flow is y-invariant); 16 cells per wavelength at level 0,
    so lmax = 2 gives 64 (the paper's lmax = 3 gives 128)."""
    lam = 2.0 * math.pi / k
    c = RunConfig(name=f"rti_k{k:g}_at{atwood:g}_l{lmax}", base_blocks=(1, 1, 10), lmax=(lmax,), dx0=lam / 16.0,
                  gravity=(0.0, 0.0, -1.0), mu=RTI_FLUIDS[atwood][2], eps=1e-3,
                  bc=(BC_SYMMETRY, BC_SYMMETRY, BC_PERIODIC, BC_PERIODIC, BC_SYMMETRY, BC_SYMMETRY))
    return dataclasses.replace(c, **kw)


def ic_rti_single_mode(cfg, geo, k: float, atwood: float = 0.5, p_interface: float | None = None):
    """Heavy over light fluid, interface z = 5 lambda + (0.05 / k) cos(k x)
    with a tanh edge two finest cells wide, at rest, hydrostatic pressure of
    the unperturbed layers (p at the interface chosen so that the top stays at
    p >= 10: low Mach number)."""
    rho_h, rho_l, _ = RTI_FLUIDS[atwood]
    lam = 2.0 * math.pi / k
    z0, g = 5.0 * lam, -cfg.gravity[2]
    if p_interface is None:
        p_interface = 10.0 + rho_h * g * 5.0 * lam
    X, _, Z, _ = cell_centres(cfg, geo)
    width = 2.0 * cfg.dx0 * 0.5 ** cfg.lmax_of(0)
    zi = z0 + (0.05 / k) * np.cos(k * X)
    s = 0.5 * (1.0 + np.tanh((Z - zi) / width))
    out = _prim(len(geo))
    out[:, 0] = rho_l + (rho_h - rho_l) * s
    out[:, 4] = np.where(Z < z0, p_interface + rho_l * g * (z0 - Z), p_interface - rho_h * g * (Z - z0))
    return out


def periodic_config(base=(2, 2, 2), lmax=0, **kw) -> RunConfig:
    c = RunConfig(name="periodic", base_blocks=tuple(base), lmax=(lmax,), dx0=1.0 / (16 * max(base)),
                  bc=(BC_PERIODIC,) * 6)
    return dataclasses.replace(c, **kw)


# ------------------------------------------------------------------ geometry
def cell_centres(cfg: RunConfig, geo: np.ndarray):
    """Cell-centre coordinates x, y, z of shape [n, 16, 16, 16] (index [z][y][x])."""
    geo = np.asarray(geo, dtype=np.int64)
    lvl = geo[:, 0].astype(np.float64)
    dx = cfg.dx0 * np.power(0.5, lvl)                        # [n]
    i = np.arange(NB, dtype=np.float64) + 0.5
    xs = cfg.domain_lo[0] + (geo[:, 1, None] * NB + i[None, :]) * dx[:, None]
    ys = cfg.domain_lo[1] + (geo[:, 2, None] * NB + i[None, :]) * dx[:, None]
    zs = cfg.domain_lo[2] + (geo[:, 3, None] * NB + i[None, :]) * dx[:, None]
    n = geo.shape[0]
    X = np.broadcast_to(xs[:, None, None, :], (n, NB, NB, NB))
    Y = np.broadcast_to(ys[:, None, :, None], (n, NB, NB, NB))
    Z = np.broadcast_to(zs[:, :, None, None], (n, NB, NB, NB))
    return X, Y, Z, dx


def _prim(n):
    return np.zeros((n, 5, NB, NB, NB), dtype=np.float64)


# ------------------------------------------------------------------ RNG
_M64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    x = (x + 0x9E3779B97F4A7C15) & _M64
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def uniform(seed: int, inst: int, stream: int, index: int) -> float:
    """U[0,1) from splitmix64 of the counter (seed, inst, stream, index)."""
    ctr = (((seed & 0xFFFF) << 48) | ((inst & 0xFFFF) << 32) | ((stream & 0xFFFF) << 16) | (index & 0xFFFF))
    return (splitmix64(ctr) >> 11) * (1.0 / (1 << 53))


def uniform_array(seed: int, stream: int, shape) -> np.ndarray:
    n = int(np.prod(shape))
    out = np.empty(n)
    for k in range(n):
        out[k] = uniform(seed, k >> 16, stream, k & 0xFFFF)
    return out.reshape(shape)


# ------------------------------------------------------------------ initial conditions
def ic_uniform(cfg, geo, rho=1.3, vel=(0.3, -0.2, 0.1), p=0.9):
    out = _prim(len(geo))
    out[:, 0], out[:, 1], out[:, 2], out[:, 3], out[:, 4] = rho, vel[0], vel[1], vel[2], p
    return out


def ic_sod(cfg, geo, x0=0.5, left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1)):
    """Sod tube along x: (rho, u, p) = left for x <= x0, right otherwise."""
    X, _, _, _ = cell_centres(cfg, geo)
    out = _prim(len(geo))
    L = X <= x0
    out[:, 0] = np.where(L, left[0], right[0])
    out[:, 1] = np.where(L, left[1], right[1])
    out[:, 4] = np.where(L, left[2], right[2])
    return out


def ic_explosion(cfg, geo, centre=(0.5, 0.5, 0.5), r0=0.4):
    """rho, p = 1, 1 for r < r0, else 0.125, 0.1; at rest."""
    X, Y, Z, _ = cell_centres(cfg, geo)
    r = np.sqrt((X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2)
    inside = r < r0
    out = _prim(len(geo))
    out[:, 0] = np.where(inside, 1.0, 0.125)
    out[:, 4] = np.where(inside, 1.0, 0.1)
    return out


def four_quadrant_states(seed: int, inst: int):
    """Per quadrant (q = qx + 2 qy): rho, p ~ U[0.1, 2]; velocity uniform in the unit ball."""
    st = np.zeros((4, 5))
    for q in range(4):
        rho = 0.1 + 1.9 * uniform(seed, inst, 1, q)
        p = 0.1 + 1.9 * uniform(seed, inst, 2, q)
        k = 0
        while True:  # rejection sampling in the unit ball, counter-indexed
            v = np.array([2.0 * uniform(seed, inst, 3 + d, 16 * q + k) - 1.0 for d in range(3)])
            k += 1
            if v @ v <= 1.0:
                break
        st[q] = (rho, v[0], v[1], v[2], p)
    return st


def ic_four_quadrant(cfg, geo, inst: int = 0, seed: int = 2012):
    """Four quadrants split at x = 0.5, y = 0.5, extruded in z; seeded states."""
    X, Y, _, _ = cell_centres(cfg, geo)
    st = four_quadrant_states(seed, inst)
    q = (X >= 0.5).astype(np.int64) + 2 * (Y >= 0.5).astype(np.int64)
    out = _prim(len(geo))
    for v in range(5):
        out[:, v] = st[q, v]
    return out


def ic_ensemble(cfg, geo, keys, seed: int = 2012):
    """Batched four-quadrant problems: block b belongs to instance keys[b] >> 56."""
    keys = np.asarray(keys, dtype=np.uint64)
    inst = (keys >> np.uint64(56)).astype(np.int64)
    out = _prim(len(geo))
    for i in np.unique(inst):
        sel = inst == i
        out[sel] = ic_four_quadrant(cfg, geo[sel], inst=int(i), seed=seed)
    return out


def post_shock_state(mach=1.22, gamma=1.4, rho1=1.0, p1=1.0):
    """Rankine-Hugoniot state behind a normal shock moving into rest."""
    g = gamma
    p2 = p1 * (1.0 + 2.0 * g / (g + 1.0) * (mach ** 2 - 1.0))
    rho2 = rho1 * (g + 1.0) * mach ** 2 / ((g - 1.0) * mach ** 2 + 2.0)
    S = mach * math.sqrt(g * p1 / rho1)
    u2 = S * (1.0 - rho1 / rho2)
    return rho2, u2, p2


def ic_shock_bubble(cfg, geo, centre=(0.4, 0.5, 0.5), radius=0.1, rho_b=0.14, x_shock=0.27, mach=1.22):
    """Planar Mach-1.22 shock at x = 0.27 moving +x into air at rest (rho 1, p 1)
    holding a light bubble (rho 0.14) with a tanh edge two finest cells wide."""
    X, Y, Z, _ = cell_centres(cfg, geo)
    width = 2.0 * cfg.dx0 * 0.5 ** cfg.lmax_of(0)
    r = np.sqrt((X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2)
    blend = 0.5 * (1.0 + np.tanh((r - radius) / width))   # 0 inside, 1 outside
    rho = rho_b + (1.0 - rho_b) * blend
    rho2, u2, p2 = post_shock_state(mach, cfg.gamma)
    post = X < x_shock
    out = _prim(len(geo))
    out[:, 0] = np.where(post, rho2, rho)
    out[:, 1] = np.where(post, u2, 0.0)
    out[:, 4] = np.where(post, p2, 1.0)
    return out


def rt_interface(seed: int, x: np.ndarray, y: np.ndarray, amp=1e-2, kmin=4, kmax=16):
    """z = 1 + sum over integer wavevectors kmin <= |k| <= kmax of cos(2 pi k.x + phi_k),
    normalised to a maximum amplitude amp (estimated on a 256^2 grid)."""
    ks = [(kx, ky) for kx in range(-kmax, kmax + 1) for ky in range(0, kmax + 1)
          if kmin ** 2 <= kx * kx + ky * ky <= kmax ** 2 and (ky > 0 or kx > 0)]
    ph = np.array([2.0 * math.pi * uniform(seed, 0, 7, n) for n in range(len(ks))])
    kk = np.array(ks, dtype=np.float64)

    def h(xx, yy):
        acc = np.zeros_like(xx)
        for n in range(len(ks)):
            acc += np.cos(2.0 * math.pi * (kk[n, 0] * xx + kk[n, 1] * yy) + ph[n])
        return acc

    g = (np.arange(256) + 0.5) / 256
    gx, gy = np.meshgrid(g, g, indexing="ij")
    scale = amp / np.abs(h(gx, gy)).max()
    return 1.0 + scale * h(x, y)


def ic_rt(cfg, geo, seed: int = 2012, rho_heavy=3.0, rho_light=1.0, p_interface=10.0):
    """Heavy fluid (rho 3) above light (rho 1) at z ~ 1 with a seeded multimode
    perturbation, tanh density edge two finest cells wide, hydrostatic pressure
    for g = (0, 0, -1) with p = 10 at z = 1."""
    X, Y, Z, _ = cell_centres(cfg, geo)
    width = 2.0 * cfg.dx0 * 0.5 ** cfg.lmax_of(0)
    # interface height per distinct (x, y) column (blocks stacked in z share columns)
    xy = np.stack([X[:, 0].ravel(), Y[:, 0].ravel()], axis=1)
    cols, inv = np.unique(xy, axis=0, return_inverse=True)
    zi = rt_interface(seed, cols[:, 0], cols[:, 1])[inv.ravel()].reshape(X[:, 0].shape)[:, None]
    s = 0.5 * (1.0 + np.tanh((Z - zi) / width))
    rho = rho_light + (rho_heavy - rho_light) * s
    g = -cfg.gravity[2]
    p = np.where(Z < 1.0, p_interface + rho_light * g * (1.0 - Z), p_interface - rho_heavy * g * (Z - 1.0))
    out = _prim(len(geo))
    out[:, 0] = rho
    out[:, 4] = p
    return out


def ic_density_wave(cfg, geo, axis=0, t=0.0, amp=0.2, speed=1.0):
    """rho = 1 + amp sin(2 pi (s - speed t)) along `axis`, velocity `speed` along
    it, p = 1; exact cell averages of rho (closed form), so that the conserved
    averages of rho, rho u and E are exact."""
    X, Y, Z, dx = cell_centres(cfg, geo)
    S = (X, Y, Z)[axis]
    h = dx[:, None, None, None]
    a, b = S - 0.5 * h - speed * t, S + 0.5 * h - speed * t
    avg = 1.0 + amp * (np.cos(2 * math.pi * a) - np.cos(2 * math.pi * b)) / (2 * math.pi * h)
    out = _prim(len(geo))
    out[:, 0] = avg
    out[:, 1 + axis] = speed
    out[:, 4] = 1.0
    return out


def ic_random_smooth(cfg, geo, seed: int = 7, modes: int = 3, amp=0.2):
    """Periodic piecewise-smooth random state (sum of a few seeded Fourier modes
    per variable plus a step in rho), for conservation tests on periodic domains."""
    X, Y, Z, _ = cell_centres(cfg, geo)
    L = [cfg.base_blocks[d] * NB * cfg.dx0 for d in range(3)]
    out = _prim(len(geo))
    base = [1.0, 0.1, -0.05, 0.05, 1.0]
    for v in range(5):
        f = np.full(X.shape, base[v])
        for m in range(modes):
            k = [1 + int(3 * uniform(seed, v, 10 + d, m)) for d in range(3)]
            ph = 2 * math.pi * uniform(seed, v, 20, m)
            f = f + amp / (m + 1) * np.sin(2 * math.pi * (k[0] * X / L[0] + k[1] * Y / L[1] + k[2] * Z / L[2]) + ph)
        out[:, v] = f
    step = (np.abs(X / L[0] - 0.5) < 0.2) & (np.abs(Y / L[1] - 0.5) < 0.25)
    out[:, 0] = np.where(step, out[:, 0] * 1.5, out[:, 0])
    return out


def random_states(n: int, seed: int = 1, rho=(0.2, 2.0), p=(0.2, 2.0), vmax=1.0):
    """Independent random primitive states per cell (for kernel parity on rough data)."""
    r = np.empty((n, 5, NB, NB, NB))
    shape = (n, NB, NB, NB)
    rng = np.random.Generator(np.random.Philox(key=seed))
    r[:, 0] = rng.uniform(rho[0], rho[1], shape)
    for d in range(3):
        r[:, 1 + d] = rng.uniform(-vmax, vmax, shape)
    r[:, 4] = rng.uniform(p[0], p[1], shape)
    return r
