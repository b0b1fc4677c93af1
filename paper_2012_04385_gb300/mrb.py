"""Thin Python binding of libmrb (include/mrb.h): argument marshalling only.

Every numerical step runs in the CUDA library; this module converts torch
tensors and numpy arrays to pointers and calls the C ABI functions of the same
names.  PyTorch supplies device memory (the block pool and all device
arguments) and the CUDA stream.  There is no CPU fallback: if the library
cannot be built or loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build
from .inputs import RunConfig

MRB_OK, MRB_EINVAL, MRB_ENOMEM, MRB_ECAPACITY, MRB_ECUDA, MRB_ETIMEOUT, MRB_ENONPHYS = range(7)
FP64, FP32_ACC64 = 0, 1
TAG_KEEP, TAG_REFINE, TAG_COARSEN = 0, 1, -1
NB, NS, NV = 16, 24, 5

_lock = threading.Lock()
_lib = None


class MrbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mrb error {code}: {msg}")
        self.code = code


class MrbConfig(ctypes.Structure):
    _fields_ = [
        ("n_instances", ctypes.c_int32),
        ("base_blocks", ctypes.c_int32 * 3),
        ("lmax", ctypes.c_int32 * 256),
        ("bc", ctypes.c_int32 * 6),
        ("precision", ctypes.c_int32),
        ("recon", ctypes.c_int32),
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
        ("mlp_weights", ctypes.c_void_p),
        ("mlp_tau", ctypes.c_double),
        ("stream", ctypes.c_void_p),
        ("lts", ctypes.c_int32),
    ]


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libmrb.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
            ci = ctypes.c_int
            sigs = {
                "mrb_pool_bytes": (sz, [vp, i64]),
                "mrb_init_blocks": (ci, [vp, vp, sz, ctypes.POINTER(vp)]),
                "mrb_n_blocks": (ci, [vp, i32, i32, vp]),
                "mrb_list_blocks": (ci, [vp, i32, i32, vp, vp, i64, vp]),
                "mrb_set_state": (ci, [vp, vp, i64, vp]),
                "mrb_set_cons": (ci, [vp, vp, i64, vp]),
                "mrb_get_state": (ci, [vp, vp, i64, vp, i32]),
                "mrb_get_records": (ci, [vp, vp, i64, vp, i32]),
                "mrb_fill_halos": (ci, [vp]),
                "mrb_compute_rhs": (ci, [vp, vp]),
                "mrb_rk_stage": (ci, [vp, i32, vp]),
                "mrb_cfl_dt": (ci, [vp, vp]),
                "mrb_mr_project": (ci, [vp]),
                "mrb_mr_predict_and_tag": (ci, [vp, i32, vp, vp]),
                "mrb_remesh": (ci, [vp, vp, vp]),
                "mrb_step": (ci, [vp, i32, vp]),
                "mrb_refine_level": (ci, [vp, i32, vp]),
                "mrb_refine_keys": (ci, [vp, vp, i64, vp]),
                "mrb_sums": (ci, [vp, vp]),
                "mrb_flux_census": (ci, [vp, vp]),
                "mrb_neighbors": (ci, [vp, vp, i64, vp]),
                "mrb_profile": (ci, [vp, i32]),
                "mrb_get_tune": (ci, [vp, vp]),
                "mrb_set_tune": (ci, [vp, vp]),
                "mrb_autotune": (ci, [vp, i32, vp]),
                "mrb_profile_read": (ci, [vp, vp, vp, vp]),
                "mrb_block_sums_noalloc": (ci, [vp, i64, vp, ctypes.c_double, vp, vp]),
                "mrb_measure_peaks": (ci, [vp, i32]),
                "mrb_face_samples": (ci, [vp, ctypes.c_float, i64, vp, vp, vp, i64, vp]),
                "mrb_learned_stats": (ci, [vp, vp, vp, i32]),
                "mrb_mlp_logits": (ci, [vp, vp, i64, vp, vp]),
                "mrb_mlp_threshold": (ci, [vp, vp, i64, ctypes.c_double, vp, vp, vp]),
                "mrb_mlp_train_step": (ci, [vp, vp, vp, i32, vp, vp, i64, ctypes.c_float, ctypes.c_float, vp, vp, vp,
                                            vp]),
                "mrb_status": (ci, [vp]),
                "mrb_sync": (ci, [vp]),
                "mrb_clear_status": (ci, [vp]),
                "mrb_destroy": (ci, [vp]),
                "mrb_last_error": (ctypes.c_char_p, [vp]),
            }
            for name, (res, args) in sigs.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def make_config(cfg: RunConfig, stream_ptr: int = 0) -> MrbConfig:
    c = MrbConfig()
    c.n_instances = int(cfg.n_instances)
    for d in range(3):
        c.base_blocks[d] = int(cfg.base_blocks[d])
        c.domain_lo[d] = float(cfg.domain_lo[d])
        c.gravity[d] = float(cfg.gravity[d])
    for i in range(c.n_instances):
        c.lmax[i] = cfg.lmax_of(i)
    for s in range(6):
        c.bc[s] = int(cfg.bc[s])
    c.precision = int(cfg.precision)
    c.recon = int(cfg.recon)
    c.rk_stages = int(getattr(cfg, "rk_stages", 3))
    c.flux = int(getattr(cfg, "flux", 0))
    c.dx0 = float(cfg.dx0)
    c.gamma = float(cfg.gamma)
    c.B = float(cfg.B)
    c.cfl = float(cfg.cfl)
    c.eps = float(cfg.eps)
    c.mu = float(getattr(cfg, "mu", 0.0))
    c.mlp_weights = None
    c.mlp_tau = float(cfg.mlp_tau)
    c.stream = stream_ptr or None
    c.lts = int(getattr(cfg, "lts", 0))
    return c


def _ptr(t) -> int:
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def measure_peaks() -> dict:
    """FP32 (scalar and packed x2) and FP64 FMA, conversion and rsqrt throughputs of the current GPU."""
    out = np.zeros(8)
    rc = lib().mrb_measure_peaks(out.ctypes.data, 8)
    if rc != MRB_OK:
        raise MrbError(rc, "mrb_measure_peaks failed")
    keys = ["fp32_tflops", "fp64_tflops", "d2f_tps", "f2d_tps", "rsqrt_tps", "sm_count", "sm_clock_mhz", "fp32x2_tflops"]
    return {k: float(v) for k, v in zip(keys, out)}


MLP_NPARAM = 1601
MLP_WORK_FLOATS = 512 * (MLP_NPARAM + 1)


def mlp_logits(params, feats, stream=None):
    """Selector logits (tensor cores) of feats [n][16] (float32, device)."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    n = feats.shape[0]
    out = torch.empty(max(n, 1), dtype=torch.float32, device=feats.device)
    rc = lib().mrb_mlp_logits(params.data_ptr(), feats.data_ptr(), n, out.data_ptr(), st.cuda_stream)
    if rc != MRB_OK:
        raise MrbError(rc, "mrb_mlp_logits failed")
    return out[:n]


def mlp_threshold(logits, labels, q, stream=None) -> float:
    """The q-quantile of the label-1 logits (mrb_mlp_threshold): the selector's
    threshold tau, below which a face goes to the linear scheme."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    n = logits.shape[0]
    work = torch.empty(256, dtype=torch.int64, device=logits.device)
    out = ctypes.c_float()
    rc = lib().mrb_mlp_threshold(logits.data_ptr(), labels.data_ptr(), n, float(q), work.data_ptr(),
                                 ctypes.byref(out), st.cuda_stream)
    if rc != MRB_OK:
        raise MrbError(rc, "mrb_mlp_threshold failed")
    return float(out.value)


class MlpTrainer:
    """Adam state and scratch for mrb_mlp_train_step."""

    def __init__(self, params, device="cuda"):
        import torch
        self.torch = torch
        self.params = params
        self.m = torch.zeros(MLP_NPARAM, dtype=torch.float32, device=device)
        self.v = torch.zeros(MLP_NPARAM, dtype=torch.float32, device=device)
        self.work = torch.empty(MLP_WORK_FLOATS, dtype=torch.float32, device=device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        self.t = 0

    def step(self, feats, labels, pos_weight=1.0, lr=1e-3, grad=None):
        st = self.torch.cuda.current_stream()
        if lr > 0:
            self.t += 1
        rc = lib().mrb_mlp_train_step(self.params.data_ptr(), self.m.data_ptr(), self.v.data_ptr(), max(self.t, 1),
                                      feats.data_ptr(), labels.data_ptr(), feats.shape[0], float(pos_weight),
                                      float(lr), self.work.data_ptr(), self.loss.data_ptr(),
                                      grad.data_ptr() if grad is not None else None, st.cuda_stream)
        if rc != MRB_OK:
            raise MrbError(rc, "mrb_mlp_train_step failed")
        return self.loss


def pool_bytes(cfg: RunConfig, n_slots: int) -> int:
    c = make_config(cfg)
    return int(lib().mrb_pool_bytes(ctypes.byref(c), int(n_slots)))


class Context:
    """An mrb context plus the torch-allocated block pool it lives in."""

    def __init__(self, cfg: RunConfig, n_slots: int, stream=None, device="cuda", mlp_params=None):
        import torch

        # every step runs in the library's CUDA kernels: there is no CPU path
        if torch.device(device).type != "cuda":
            raise ValueError(f"the block pool must live in CUDA device memory, not on {device!r}")
        if not torch.cuda.is_available():
            raise RuntimeError("mrb needs a CUDA device (sm_103a); it has no CPU fallback")
        self.cfg = cfg
        self.torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._c = make_config(cfg, self.stream.cuda_stream)
        self.mlp_params = mlp_params
        if mlp_params is not None:
            self._c.mlp_weights = mlp_params.data_ptr()
        nbytes = int(lib().mrb_pool_bytes(ctypes.byref(self._c), int(n_slots)))
        if nbytes == 0:
            raise MrbError(MRB_EINVAL, "invalid configuration")
        self.pool = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        base = self.pool.data_ptr()
        aligned = (base + 255) & ~255
        h = ctypes.c_void_p()
        self._rc(lib().mrb_init_blocks(ctypes.byref(self._c), aligned, nbytes, ctypes.byref(h)), None)
        self._h = h
        self.n_slots = n_slots

    def _rc(self, rc, h="self"):
        if rc != MRB_OK:
            handle = self._h if h == "self" else None
            msg = lib().mrb_last_error(handle)
            raise MrbError(rc, msg.decode() if msg else "")

    def close(self):
        """Destroy the context and drop its block pool (the memory returns to
        torch's allocator once no other reference holds it)."""
        if getattr(self, "_h", None):
            lib().mrb_destroy(self._h)
            self._h = None
            self.pool = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- topology
    def n_blocks(self, level=-1, leaves_only=True) -> int:
        n = ctypes.c_int64()
        self._rc(lib().mrb_n_blocks(self._h, level, int(leaves_only), ctypes.byref(n)))
        return int(n.value)

    def list_blocks(self, level=-1, leaves_only=True):
        n = self.n_blocks(level, leaves_only)
        keys = np.zeros(n, dtype=np.uint64)
        geo = np.zeros((n, 4), dtype=np.int64)
        cnt = ctypes.c_int64()
        self._rc(lib().mrb_list_blocks(self._h, level, int(leaves_only), keys.ctypes.data, geo.ctypes.data, n,
                                       ctypes.byref(cnt)))
        return keys, geo

    def keys(self, level=-1, leaves_only=True):
        return self.list_blocks(level, leaves_only)[0]

    def geometry(self, level=-1, leaves_only=True):
        return self.list_blocks(level, leaves_only)[1]

    def n_leaves(self) -> int:
        return self.n_blocks(-1, True)

    # ---- state
    def set_state(self, keys, prim):
        torch = self.torch
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        if not torch.is_tensor(prim):
            prim = torch.from_numpy(np.ascontiguousarray(prim, dtype=np.float64))
        prim = prim.to(device=self.pool.device, dtype=torch.float64).contiguous()
        assert tuple(prim.shape) == (len(keys), NV, NB, NB, NB)
        self._rc(lib().mrb_set_state(self._h, keys.ctypes.data, len(keys), prim.data_ptr()))
        self._keep = prim

    def set_cons(self, keys, cons):
        torch = self.torch
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        if not torch.is_tensor(cons):
            cons = torch.from_numpy(np.ascontiguousarray(cons, dtype=np.float64))
        cons = cons.to(device=self.pool.device, dtype=torch.float64).contiguous()
        assert tuple(cons.shape) == (len(keys), NV, NB, NB, NB)
        self._rc(lib().mrb_set_cons(self._h, keys.ctypes.data, len(keys), cons.data_ptr()))
        self._keep = cons

    def get_state(self, keys=None, with_halo=False, out=None):
        torch = self.torch
        if keys is None:
            keys = self.keys()
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        n = NS if with_halo else NB
        if out is None:
            out = torch.empty((len(keys), NV, n, n, n), dtype=torch.float64, device=self.pool.device)
        self._rc(lib().mrb_get_state(self._h, keys.ctypes.data, len(keys), out.data_ptr(), int(with_halo)))
        return out

    def get_records(self, keys=None, fresh=False):
        """FP32 primitive records [n][6][16][16][16] of the listed blocks'
        internal cells (mixed-precision contexts): as kept, or converted
        afresh from the FP64 state."""
        torch = self.torch
        if keys is None:
            keys = self.keys()
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        out = torch.empty((len(keys), 6, NB, NB, NB), dtype=torch.float32, device=self.pool.device)
        self._rc(lib().mrb_get_records(self._h, keys.ctypes.data, len(keys), out.data_ptr(), int(fresh)))
        return out

    # ---- steps (same names as the C ABI)
    def fill_halos(self):
        self._rc(lib().mrb_fill_halos(self._h))

    def compute_rhs(self, out=None):
        torch = self.torch
        if out is None:
            out = torch.empty((self.n_leaves(), NV, NB, NB, NB), dtype=torch.float64, device=self.pool.device)
        self._rc(lib().mrb_compute_rhs(self._h, out.data_ptr()))
        return out

    def rk_stage(self, stage: int, dt):
        self._rc(lib().mrb_rk_stage(self._h, int(stage), dt.data_ptr()))

    def cfl_dt(self, out=None):
        torch = self.torch
        if out is None:
            out = torch.empty(self.cfg.n_instances, dtype=torch.float64, device=self.pool.device)
        self._rc(lib().mrb_cfl_dt(self._h, out.data_ptr()))
        return out

    def mr_project(self):
        self._rc(lib().mrb_mr_project(self._h))

    def mr_predict_and_tag(self, allow_refine=True, with_delta=True):
        torch = self.torch
        n = self.n_leaves()
        tags = torch.empty(max(n, 1), dtype=torch.int8, device=self.pool.device)
        delta = torch.empty(max(n, 1), dtype=torch.float64, device=self.pool.device) if with_delta else None
        self._rc(lib().mrb_mr_predict_and_tag(self._h, int(allow_refine), tags.data_ptr(),
                                              delta.data_ptr() if delta is not None else None))
        return tags[:n], (delta[:n] if delta is not None else None)

    def remesh(self, tags) -> int:
        torch = self.torch
        if not torch.is_tensor(tags):
            tags = torch.from_numpy(np.ascontiguousarray(tags, dtype=np.int8))
        tags = tags.to(device=self.pool.device, dtype=torch.int8).contiguous()
        assert tags.numel() == self.n_leaves()
        n = ctypes.c_int64()
        self._rc(lib().mrb_remesh(self._h, tags.data_ptr() if tags.numel() else None, ctypes.byref(n)))
        return int(n.value)

    def refine_level(self, level) -> int:
        n = ctypes.c_int64()
        self._rc(lib().mrb_refine_level(self._h, int(level), ctypes.byref(n)))
        return int(n.value)

    def refine_keys(self, keys) -> int:
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        n = ctypes.c_int64()
        self._rc(lib().mrb_refine_keys(self._h, keys.ctypes.data, len(keys), ctypes.byref(n)))
        return int(n.value)

    def step(self, nsteps=1, dt_hist=None):
        self._rc(lib().mrb_step(self._h, int(nsteps), dt_hist.data_ptr() if dt_hist is not None else None))

    def sums(self, out=None):
        torch = self.torch
        if out is None:
            out = torch.empty((self.cfg.n_instances, NV), dtype=torch.float64, device=self.pool.device)
        self._rc(lib().mrb_sums(self._h, out.data_ptr()))
        return out

    def flux_census(self) -> np.ndarray:
        """Faces where each characteristic field takes the LLF split ([0..4])
        and the number of faces ([5]), over every leaf face (halos filled)."""
        out = np.zeros(6, dtype=np.uint64)
        self._rc(lib().mrb_flux_census(self._h, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def neighbors(self, keys):
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        out = np.zeros((len(keys), 27), dtype=np.uint64)
        self._rc(lib().mrb_neighbors(self._h, keys.ctypes.data, len(keys), out.ctypes.data))
        return out

    def get_tune(self):
        q = np.zeros(5, dtype=np.int32)
        self._rc(lib().mrb_get_tune(self._h, q.ctypes.data))
        return [int(x) for x in q]

    def set_tune(self, params):
        q = np.ascontiguousarray(params, dtype=np.int32)
        assert q.shape == (5,)
        self._rc(lib().mrb_set_tune(self._h, q.ctypes.data))

    def autotune(self, reps=3):
        """Scheduling-only autotuner (mrb_autotune): returns the chosen launch
        shapes and the default / tuned times (ms) of the stage kernel(s), one
        halo fill and one averaging pass."""
        t = np.zeros(6)
        self._rc(lib().mrb_autotune(self._h, int(reps), t.ctypes.data))
        return {"params": self.get_tune(), "stage_ms": (t[0], t[1]), "fill_ms": (t[2], t[3]),
                "project_ms": (t[4], t[5])}

    def profile(self, enable=True):
        self._rc(lib().mrb_profile(self._h, int(enable)))

    def profile_read(self):
        ms = ctypes.c_double()
        n_rhs = ctypes.c_int64()
        n_k = ctypes.c_int64()
        self._rc(lib().mrb_profile_read(self._h, ctypes.byref(ms), ctypes.byref(n_rhs), ctypes.byref(n_k)))
        return float(ms.value), int(n_rhs.value), int(n_k.value)

    def face_samples(self, tau_lab=1e-3, stride=1, cap=None, with_where=False):
        torch = self.torch
        faces = self.n_leaves() * 3 * 17 * 256
        n = (faces + stride - 1) // stride if cap is None else min(cap, (faces + stride - 1) // stride)
        feats = torch.empty((max(n, 1), 16), dtype=torch.float32, device=self.pool.device)
        labels = torch.empty(max(n, 1), dtype=torch.uint8, device=self.pool.device)
        where = torch.empty(max(n, 1), dtype=torch.int64, device=self.pool.device) if with_where else None
        cnt = ctypes.c_int64()
        self._rc(lib().mrb_face_samples(self._h, float(tau_lab), int(stride), feats.data_ptr(), labels.data_ptr(),
                                        where.data_ptr() if where is not None else None, n, ctypes.byref(cnt)))
        k = int(cnt.value)
        return feats[:k], labels[:k], (where[:k] if where is not None else None)

    def learned_stats(self, reset=True):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        self._rc(lib().mrb_learned_stats(self._h, ctypes.byref(a), ctypes.byref(b), int(reset)))
        return int(a.value), int(b.value)

    def status(self) -> int:
        return int(lib().mrb_status(self._h))

    def sync(self):
        self._rc(lib().mrb_sync(self._h))

    def clear_status(self):
        self._rc(lib().mrb_clear_status(self._h))


def init_tree(ctx, ic, allow_coarsen=True, with_keys=False):
    """Alg. (Initialization): impose the initial condition on level 0, then for
    m = 1 .. lmax refine every block of level m-1, impose the initial condition
    on level m and, for m > 1, coarsen sibling groups whose details are below
    eps_m.  `ic(cfg, geo) -> prim[n, 5, 16, 16, 16]` (host numpy), or
    `ic(cfg, geo, keys)` with `with_keys` (batched instances: the instance is
    key >> 56)."""
    if with_keys:
        ic_k = ic
    else:
        def ic_k(c, geo, keys):
            return ic(c, geo)
    torch = ctx.torch
    cfg = ctx.cfg
    lmax = max(cfg.lmax_of(i) for i in range(cfg.n_instances))
    keys, geo = ctx.list_blocks(0)
    ctx.set_state(keys, ic_k(cfg, geo, keys))
    for m in range(1, lmax + 1):
        ctx.refine_level(m - 1)
        keys, geo = ctx.list_blocks(m)
        ctx.set_state(keys, ic_k(cfg, geo, keys))
        if m > 1 and allow_coarsen:
            ctx.fill_halos()
            tags, _ = ctx.mr_predict_and_tag(allow_refine=False, with_delta=False)
            ctx.remesh(tags)
    ctx.mr_project()
    torch.cuda.current_stream().synchronize()


def restore_tree(ctx, node_keys):
    """Checkpoint / resume: rebuild a saved block tree in a fresh context.
    `node_keys` are all node ids (internal nodes and leaves, as listed by
    keys(leaves_only=False)); leaves whose first child is saved are refined,
    level by level.  The caller then restores every node's state with
    set_cons."""
    want = set(int(k) for k in np.asarray(node_keys, dtype=np.uint64))
    mask56 = (1 << 56) - 1

    def child0(k):
        return ((k & mask56) << 3) | ((k >> 56) << 56)

    while True:
        leaves = [int(k) for k in ctx.keys()]
        sel = np.array([k for k in leaves if child0(k) in want], dtype=np.uint64)
        if len(sel) == 0:
            break
        ctx.refine_keys(sel)
    have = set(int(k) for k in ctx.keys(leaves_only=False))
    if have != want:
        raise MrbError(MRB_EINVAL, "saved ids do not form a tree reachable from level 0")
