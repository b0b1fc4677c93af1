"""The allocation-free conservation-sum entry point (mrb_block_sums_noalloc).

It exists for callers that cannot call cudaMalloc (code under an allocator that
owns all device memory, or host code that must not take the driver's allocation
lock); its scratch is a fixed device array inside the library.  This file is
collected last so that a run stopping at its first failure has already run
every other test; it passes alone in a fresh process and after the others.
"""
import ctypes

import numpy as np
import pytest

from paper_2012_04385_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2012_04385_gb300 import mrb  # noqa: E402

REL = 1e-13


def test_noalloc_sums_match_mrb_sums_twice():
    cfg = I.explosion_config(lmax=2)
    g = mrb.Context(cfg, 600)
    mrb.init_tree(g, lambda c, geo: I.ic_explosion(c, geo))
    g.step(1)
    keys, geo = g.list_blocks()
    stream = torch.cuda.current_stream()
    ref = g.sums().cpu().numpy()[0]
    blocks = g.get_state(keys)                                   # [n][5][16^3] device
    levels = torch.tensor(geo[:, 0], dtype=torch.int32, device="cuda")
    L = mrb.lib()
    for call in range(2):                                        # two calls in a row share the scratch
        out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
        rc = L.mrb_block_sums_noalloc(blocks.data_ptr(), len(keys), levels.data_ptr(), cfg.dx0,
                                      stream.cuda_stream, out.data_ptr())
        assert rc == mrb.MRB_OK, rc
        got = out.cpu().numpy()
        scale = np.abs(ref).max()
        assert np.all(np.abs(got - ref) <= REL * np.maximum(np.abs(ref), scale)), (call, got, ref)
    # too many blocks is rejected before anything runs
    rc = L.mrb_block_sums_noalloc(blocks.data_ptr(), 65537, levels.data_ptr(), cfg.dx0, stream.cuda_stream,
                                  out.data_ptr())
    assert rc == mrb.MRB_ECAPACITY
