"""The C-ABI library builds, loads and exports every function include/mrb.h
declares (no GPU needed: nothing is called that touches a device)."""
import ctypes
import os
import re

import pytest

from paper_2012_04385_gb300 import _build, mrb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(mrb_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    path = _build.build()
    L = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 18
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_header():
    L = mrb.lib()
    for n in declared_functions():
        assert getattr(L, n).argtypes is not None, n


def test_pool_bytes_and_config_checks():
    from paper_2012_04385_gb300 import inputs as I
    cfg = I.sod_config()
    b1 = mrb.pool_bytes(cfg, 1)
    b8 = mrb.pool_bytes(cfg, 8)
    per_slot = (2 * 5 * 24 ** 3 + 5 * 16 ** 3 + 6 * 5 * 256) * 8 + 432 * 4
    assert b8 >= 8 * per_slot and b8 < 8 * per_slot + 4 * 256
    # the mixed-precision path adds the FP32 records of both stage buffers and
    # the FP32 stage increments
    per32 = per_slot + (2 * 6 * 16 ** 3 + 5 * 16 ** 3) * 4
    b32 = mrb.pool_bytes(I.sod_config(precision=I.FP32_ACC64), 8)
    assert b32 >= 8 * per32 and b32 < 8 * per32 + 7 * 256
    assert b1 > 0
    bad = I.sod_config(bc=(1, 0, 1, 1, 1, 1))          # periodic on one side only
    assert mrb.pool_bytes(bad, 8) == 0
    assert mrb.pool_bytes(I.sod_config(lmax=(12,)), 8) == 0
    assert mrb.pool_bytes(cfg, 0) == 0
    # reconstruction and flux choices: every pair valid except the learned
    # selector with a flux other than Roe; out-of-range codes rejected
    for recon in (I.RECON_WENO, I.RECON_LEARNED, I.RECON_LINEAR, I.RECON_TENO, I.RECON_WENOAO):
        for flux in (I.FLUX_ROE, I.FLUX_LLF, I.FLUX_HLLC):
            ok = recon != I.RECON_LEARNED or flux == I.FLUX_ROE
            assert (mrb.pool_bytes(I.sod_config(recon=recon, flux=flux), 8) > 0) == ok, (recon, flux)
    assert mrb.pool_bytes(I.sod_config(recon=5), 8) == 0
    assert mrb.pool_bytes(I.sod_config(flux=3), 8) == 0
    assert mrb.pool_bytes(I.sod_config(flux=-1), 8) == 0


def context_functions():
    """Declared functions whose first parameter is the context."""
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", f)).read(), flags=re.S)
            names += re.findall(r"\bint\s+(mrb_[a-z0-9_]+)\s*\(\s*mrb_ctx\s*\*", src)
    return sorted(set(names))


def test_every_context_call_rejects_a_null_context():
    """Each call that takes a context returns MRB_EINVAL for a null one (and
    leaves a message for mrb_last_error), before touching any device."""
    L = mrb.lib()
    names = context_functions()
    assert len(names) >= 20
    for n in names:
        f = getattr(L, n)
        args = [None if t in (ctypes.c_void_p,) else t(0) for t in f.argtypes]
        assert f(*args) == mrb.MRB_EINVAL, n
        assert L.mrb_last_error(None), n


def test_context_refuses_to_run_without_a_cuda_device():
    """The product path has no CPU fallback: a context on the host, or on a
    machine without a CUDA device, raises before anything is allocated."""
    import torch

    from paper_2012_04385_gb300 import inputs as I
    from paper_2012_04385_gb300 import mrb
    with pytest.raises(ValueError):
        mrb.Context(I.sod_config(), 16, device="cpu")
    if not torch.cuda.is_available():
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            mrb.Context(I.sod_config(), 16)


def test_oracle_and_library_share_no_code():
    """The oracle and the CUDA path are independent: the oracle's C++ includes
    only standard and OpenMP headers, its Python modules import neither the
    product package nor its build; the library's sources include only their
    own headers and CUDA's, and the package's modules never import the
    oracle.  Only the seeded input generators (inputs.py) serve both."""
    import ast
    import glob

    def imports(path):
        mods = set()
        for node in ast.walk(ast.parse(open(path).read())):
            if isinstance(node, ast.Import):
                mods.update(a.name.split(".")[0] for a in node.names)
            elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
                mods.add(node.module.split(".")[0])
        return mods

    for path in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        assert "paper_2012_04385_gb300" not in imports(path), path
    for path in glob.glob(os.path.join(ROOT, "paper_2012_04385_gb300", "*.py")):
        assert "oracle" not in imports(path), path
    inc = re.compile(r'^\s*#\s*include\s*[<"]([^>"]+)[>"]', re.M)
    std = {"algorithm", "cmath", "cstdint", "cstring", "map", "string", "tuple", "vector", "omp.h"}
    assert set(inc.findall(open(os.path.join(ROOT, "oracle", "orc.cpp")).read())) <= std
    csrc = os.path.join(ROOT, "paper_2012_04385_gb300", "csrc")
    own = {os.path.basename(p) for p in glob.glob(os.path.join(csrc, "*.cuh"))} | {"mrb.h"}
    system = {"algorithm", "cmath", "cstdint", "cstdio", "cstring", "exception", "mutex", "string", "vector",
              "cuda_runtime.h", "cuda_bf16.h"}
    for path in glob.glob(os.path.join(csrc, "*.cu")) + glob.glob(os.path.join(csrc, "*.cuh")):
        for h in inc.findall(open(path).read()):
            assert h in own | system, (path, h)
