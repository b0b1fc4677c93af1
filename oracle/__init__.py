"""CPU FP64 oracle of the block-based MR Euler method (arXiv:2012.04385).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg of ``bench.py`` may import this package; the product path
never does.  The numerical work lives in ``orc.cpp`` (plain scalar C++, see its
header for the pins and the evaluation order); this module only compiles it,
marshals numpy arrays through ctypes and adds the exact Riemann solver and the
MLP reference (``exact_riemann.py``, ``mlp.py``).

It shares no code with the CUDA library.  Run configurations are passed as any
object with the attributes of ``paper_2012_04385_gb300.inputs.RunConfig`` (duck
typed, so nothing here imports the product package).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "orc.cpp")
# ORC_LIB names an already built oracle library to load instead (the tests
# that plant mistakes in copies of orc.cpp use it); nothing is compiled then.
_LIB = os.environ.get("ORC_LIB") or os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

NB, HW, NS, NV = 16, 4, 24, 5
TAG_KEEP, TAG_REFINE, TAG_COARSEN = 0, 1, -1


def compile_to(src: str, out: str) -> None:
    """Compile an oracle source file into a shared library at `out`."""
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", src, "-o", out],
                   check=True)


def build(force: bool = False) -> str:
    """Compile orc.cpp into liborc.so (gcc, -ffp-contract=off, OpenMP)."""
    if os.environ.get("ORC_LIB"):
        return _LIB
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class OrcConfig(ctypes.Structure):
    _fields_ = [
        ("n_instances", ctypes.c_int32),
        ("base_blocks", ctypes.c_int32 * 3),
        ("lmax", ctypes.c_int32 * 256),
        ("bc", ctypes.c_int32 * 6),
        ("recon", ctypes.c_int32),
        ("n_threads", ctypes.c_int32),
        ("rk_stages", ctypes.c_int32),
        ("flux", ctypes.c_int32),
        ("domain_lo", ctypes.c_double * 3),
        ("dx0", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("B", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("gravity", ctypes.c_double * 3),
        ("eps", ctypes.c_double),
        ("mu", ctypes.c_double),
        ("lts", ctypes.c_int32),
    ]


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            vp, i32, i64, u64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
            sig = {
                "orc_create": (vp, [vp]),
                "orc_destroy": (None, [vp]),
                "orc_list": (i64, [vp, i32, i32, vp, i64]),
                "orc_list_geometry": (i64, [vp, i32, i32, vp, i64]),
                "orc_set_state": (ctypes.c_int, [vp, vp, i64, vp]),
                "orc_set_cons": (ctypes.c_int, [vp, vp, i64, vp]),
                "orc_get_state": (ctypes.c_int, [vp, vp, i64, vp, i32]),
                "orc_fill_halos": (None, [vp]),
                "orc_compute_rhs": (None, [vp, vp]),
                "orc_rk_stage": (None, [vp, i32, vp]),
                "orc_project": (None, [vp]),
                "orc_cfl_dt": (None, [vp, vp]),
                "orc_predict_and_tag": (None, [vp, i32, vp, vp]),
                "orc_remesh": (i64, [vp, vp]),
                "orc_sums": (None, [vp, vp]),
                "orc_flux_census": (None, [vp, vp]),
                "orc_step": (None, [vp, i32, vp]),
                "orc_neighbor": (i32, [vp, u64, i32, i32, i32, vp]),
                "orc_make_key": (u64, [i32, i32, i64, i64, i64]),
                "orc_key_level": (i32, [u64]),
                "orc_weno5": (dbl, [vp]),
                "orc_linear5": (dbl, [vp]),
                "orc_teno5": (dbl, [vp]),
                "orc_wenoao53": (dbl, [vp]),
                "orc_hllc": (None, [vp, vp, i32, dbl, dbl, vp]),
                "orc_flux": (None, [vp, i32, dbl, dbl, vp]),
                "orc_roe_eigen": (None, [vp, vp, i32, dbl, dbl, vp, vp, vp]),
                "orc_face_flux": (None, [vp, i32, dbl, dbl, i32, i32, vp]),
                "orc_predict_block": (None, [vp, i32, vp]),
                "orc_face_features": (None, [vp, i32, dbl, dbl, dbl, vp, vp, vp]),
                "orc_average_block": (None, [vp, vp]),
                "orc_threads": (i32, []),
                "orc_count_row_flops": (None, [vp, i32, dbl, dbl, i32, i32, vp]),
                "orc_lts_macro_step": (None, [vp, vp]),
                "orc_count_recon_flops": (None, [i32, vp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def make_config(cfg, n_threads: int = 0) -> OrcConfig:
    c = OrcConfig()
    c.n_instances = int(cfg.n_instances)
    for d in range(3):
        c.base_blocks[d] = int(cfg.base_blocks[d])
        c.domain_lo[d] = float(cfg.domain_lo[d])
        c.gravity[d] = float(cfg.gravity[d])
    lm = list(cfg.lmax)
    for i in range(c.n_instances):
        c.lmax[i] = int(lm[i] if len(lm) > 1 else lm[0])
    for s in range(6):
        c.bc[s] = int(cfg.bc[s])
    c.recon = int(cfg.recon)
    c.n_threads = int(n_threads)
    c.rk_stages = int(getattr(cfg, "rk_stages", 3))
    c.flux = int(getattr(cfg, "flux", 0))
    c.dx0 = float(cfg.dx0)
    c.gamma = float(cfg.gamma)
    c.B = float(cfg.B)
    c.cfl = float(cfg.cfl)
    c.eps = float(cfg.eps)
    c.mu = float(getattr(cfg, "mu", 0.0))
    c.lts = int(getattr(cfg, "lts", 0))
    return c


class Oracle:
    """One oracle context: a forest of block trees (one per instance)."""

    def __init__(self, cfg, n_threads: int = 0):
        self.cfg = cfg
        self._c = make_config(cfg, n_threads)
        self._h = lib().orc_create(ctypes.byref(self._c))

    def close(self):
        if self._h:
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- topology
    def keys(self, level: int = -1, leaves_only: bool = True) -> np.ndarray:
        n = lib().orc_list(self._h, level, int(leaves_only), None, 0)
        out = np.zeros(n, dtype=np.uint64)
        lib().orc_list(self._h, level, int(leaves_only), _p(out), n)
        return out

    def geometry(self, level: int = -1, leaves_only: bool = True) -> np.ndarray:
        n = lib().orc_list_geometry(self._h, level, int(leaves_only), None, 0)
        out = np.zeros((n, 4), dtype=np.int64)
        lib().orc_list_geometry(self._h, level, int(leaves_only), _p(out), n)
        return out

    def n_leaves(self) -> int:
        return int(lib().orc_list(self._h, -1, 1, None, 0))

    # ---- state
    def set_state(self, keys: np.ndarray, prim: np.ndarray):
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        prim = np.ascontiguousarray(prim, dtype=np.float64)
        assert prim.shape == (len(keys), NV, NB, NB, NB)
        if lib().orc_set_state(self._h, _p(keys), len(keys), _p(prim)) != 0:
            raise KeyError("unknown block key")

    def set_cons(self, keys: np.ndarray, cons: np.ndarray):
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        cons = np.ascontiguousarray(cons, dtype=np.float64)
        assert cons.shape == (len(keys), NV, NB, NB, NB)
        if lib().orc_set_cons(self._h, _p(keys), len(keys), _p(cons)) != 0:
            raise KeyError("unknown block key")

    def get_state(self, keys: np.ndarray | None = None, with_halo: bool = False) -> np.ndarray:
        if keys is None:
            keys = self.keys()
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        n = NS if with_halo else NB
        out = np.zeros((len(keys), NV, n, n, n))
        if lib().orc_get_state(self._h, _p(keys), len(keys), _p(out), int(with_halo)) != 0:
            raise KeyError("unknown block key")
        return out

    # ---- operations (each one the paper's step of the same name)
    def fill_halos(self):
        lib().orc_fill_halos(self._h)

    def compute_rhs(self) -> np.ndarray:
        out = np.zeros((self.n_leaves(), NV, NB, NB, NB))
        lib().orc_compute_rhs(self._h, _p(out))
        return out

    def rk_stage(self, s: int, dt: np.ndarray):
        dt = np.ascontiguousarray(dt, dtype=np.float64)
        lib().orc_rk_stage(self._h, s, _p(dt))

    def project(self):
        lib().orc_project(self._h)

    def cfl_dt(self) -> np.ndarray:
        out = np.zeros(self.cfg.n_instances)
        lib().orc_cfl_dt(self._h, _p(out))
        return out

    def predict_and_tag(self, allow_refine: bool = True):
        n = self.n_leaves()
        tags = np.zeros(n, dtype=np.int8)
        delta = np.zeros(n)
        lib().orc_predict_and_tag(self._h, int(allow_refine), _p(tags), _p(delta))
        return tags, delta

    def remesh(self, tags: np.ndarray) -> int:
        tags = np.ascontiguousarray(tags, dtype=np.int8)
        assert len(tags) == self.n_leaves()
        return int(lib().orc_remesh(self._h, _p(tags)))

    def sums(self) -> np.ndarray:
        out = np.zeros((self.cfg.n_instances, NV))
        lib().orc_sums(self._h, _p(out))
        return out

    def flux_census(self) -> np.ndarray:
        """Faces of all leaves where characteristic field k takes the LLF
        split ([0..4]) and the number of faces ([5]); halos must be filled."""
        out = np.zeros(6, dtype=np.uint64)
        lib().orc_flux_census(self._h, _p(out))
        return out

    def step(self, nsteps: int = 1) -> np.ndarray:
        dts = np.zeros((nsteps, self.cfg.n_instances))
        lib().orc_step(self._h, nsteps, _p(dts))
        return dts

    def lts_macro_step(self) -> np.ndarray:
        """One local-time-stepping macro step (no MR analysis); returns the
        finest level's time step per instance."""
        dt = np.zeros(self.cfg.n_instances)
        lib().orc_lts_macro_step(self._h, _p(dt))
        return dt

    def neighbor(self, key: int, sx: int, sy: int, sz: int):
        out = np.zeros(1, dtype=np.uint64)
        ok = lib().orc_neighbor(ctypes.byref(self._c), int(key), sx, sy, sz, _p(out))
        return int(out[0]) if ok else None


# ---- pure functions
def make_key(inst: int, level: int, x: int, y: int, z: int) -> int:
    return int(lib().orc_make_key(inst, level, x, y, z))


def key_level(key: int) -> int:
    return int(lib().orc_key_level(key))


def weno5(f) -> float:
    f = np.ascontiguousarray(f, dtype=np.float64)
    return float(lib().orc_weno5(_p(f)))


def linear5(f) -> float:
    f = np.ascontiguousarray(f, dtype=np.float64)
    return float(lib().orc_linear5(_p(f)))


def teno5(f) -> float:
    f = np.ascontiguousarray(f, dtype=np.float64)
    return float(lib().orc_teno5(_p(f)))


def wenoao53(f) -> float:
    f = np.ascontiguousarray(f, dtype=np.float64)
    return float(lib().orc_wenoao53(_p(f)))


def hllc(UL, UR, d: int, gamma: float = 1.4, B: float = 0.0) -> np.ndarray:
    """HLLC flux between two lab-frame conserved states along axis d."""
    UL = np.ascontiguousarray(UL, dtype=np.float64)
    UR = np.ascontiguousarray(UR, dtype=np.float64)
    F = np.zeros(5)
    lib().orc_hllc(_p(UL), _p(UR), d, gamma, B, _p(F))
    return F


def flux(U, d: int, gamma: float = 1.4, B: float = 0.0) -> np.ndarray:
    U = np.ascontiguousarray(U, dtype=np.float64)
    F = np.zeros(5)
    lib().orc_flux(_p(U), d, gamma, B, _p(F))
    return F


def roe_eigen(UL, UR, d: int = 0, gamma: float = 1.4, B: float = 0.0):
    UL = np.ascontiguousarray(UL, dtype=np.float64)
    UR = np.ascontiguousarray(UR, dtype=np.float64)
    Lm, Rm, lam = np.zeros((5, 5)), np.zeros((5, 5)), np.zeros(5)
    lib().orc_roe_eigen(_p(UL), _p(UR), d, gamma, B, _p(Lm), _p(Rm), _p(lam))
    return Lm, Rm, lam


def face_flux(U6, d: int, gamma: float = 1.4, B: float = 0.0, mode: int = 0, flux: int = 0) -> np.ndarray:
    U6 = np.ascontiguousarray(U6, dtype=np.float64)
    assert U6.shape == (6, 5)
    F = np.zeros(5)
    lib().orc_face_flux(_p(U6), d, gamma, B, mode, flux, _p(F))
    return F


def face_features(U6, d: int, gamma: float = 1.4, B: float = 0.0, tau_lab: float = 1e-3, with_aux: bool = False):
    """Selector features [15] and label of one face (U6: six lab-frame cells).
    With `with_aux` also the label's decision margin and scales (aux[5]: the
    largest |WENO5 - linear5| minus its threshold over the label's checks, the
    largest |input| of those checks, and per selected field the largest
    |g_m| + alpha |v_m|)."""
    U6 = np.ascontiguousarray(U6, dtype=np.float64)
    assert U6.shape == (6, 5)
    f = np.zeros(15)
    lab = np.zeros(1, dtype=np.int32)
    aux = np.zeros(5)
    lib().orc_face_features(_p(U6), d, gamma, B, tau_lab, _p(f), _p(lab), _p(aux))
    return (f, int(lab[0]), aux) if with_aux else (f, int(lab[0]))


def predict_block(parent: np.ndarray, child: int) -> np.ndarray:
    parent = np.ascontiguousarray(parent, dtype=np.float64)
    assert parent.shape == (NS, NS, NS)
    out = np.zeros((NS, NS, NS))
    lib().orc_predict_block(_p(parent), child, _p(out))
    return out


def average_block(children: np.ndarray) -> np.ndarray:
    children = np.ascontiguousarray(children, dtype=np.float64)
    assert children.shape == (8, NS, NS, NS)
    out = np.zeros((NB, NB, NB))
    lib().orc_average_block(_p(children), _p(out))
    return out


def threads() -> int:
    return int(lib().orc_threads())


def count_row_flops(urow: np.ndarray, d: int, gamma: float, B: float, mode: int, flux: int) -> np.ndarray:
    """Operation count of the 17 face fluxes of one block row along d
    (urow[22, 5]: conserved lab-frame states of cells -3..18), measured by
    running the oracle's face flux on its counting number type: [FLOPs,
    add/sub, mul, div, sqrt] (see the counting section of orc.cpp)."""
    urow = np.ascontiguousarray(urow, dtype=np.float64)
    assert urow.shape == (NB + 6, NV)
    out = np.zeros(5, dtype=np.int64)
    lib().orc_count_row_flops(_p(urow), int(d), float(gamma), float(B), int(mode), int(flux), _p(out))
    return out


def count_recon_flops(mode: int) -> np.ndarray:
    """Operation count of one reconstruction of the given mode (same layout)."""
    out = np.zeros(5, dtype=np.int64)
    lib().orc_count_recon_flops(int(mode), _p(out))
    return out

