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


def _call(L, blocks, n, levels, dx0, stream, out):
    return L.mrb_block_sums_noalloc(blocks.data_ptr() if blocks is not None else None, n,
                                    levels.data_ptr() if levels is not None else None, dx0, stream.cuda_stream,
                                    out.data_ptr())


def test_noalloc_sums_match_mrb_sums_twice():
    """Blocks passed in the library's leaf order reduce in the same fixed
    order as mrb_sums, so the sums are bitwise equal, on two calls in a row
    (the second reuses the scratch the first left behind)."""
    cfg = I.shock_bubble_config(lmax=2)                         # leaves on levels 1 and 2
    g = mrb.Context(cfg, 600)
    mrb.init_tree(g, lambda c, geo: I.ic_shock_bubble(c, geo))
    g.step(1)
    keys, geo = g.list_blocks()
    stream = torch.cuda.current_stream()
    ref = g.sums().cpu().numpy()[0]
    blocks = g.get_state(keys)                                   # [n][5][16^3] device
    levels = torch.tensor(geo[:, 0], dtype=torch.int32, device="cuda")
    assert len(np.unique(geo[:, 0])) > 1                        # several levels weighted
    L = mrb.lib()
    for call in range(2):
        out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
        assert _call(L, blocks, len(keys), levels, cfg.dx0, stream, out) == mrb.MRB_OK
        got = out.cpu().numpy()
        assert np.array_equal(got, ref), (call, got, ref)
    # too many blocks is rejected before anything runs
    assert _call(L, blocks, 65537, levels, cfg.dx0, stream, out) == mrb.MRB_ECAPACITY
    g.close()


def test_noalloc_empty_and_single_level_without_levels():
    """n_blocks = 0 gives zeros (over scratch left by an earlier call), and a
    single-level tree needs no level array (all blocks on level 0)."""
    cfg = I.sod_config()
    g = mrb.Context(cfg, 16)
    keys, geo = g.list_blocks()
    g.set_state(keys, I.ic_sod(cfg, geo))
    g.step(2)
    stream = torch.cuda.current_stream()
    L = mrb.lib()
    blocks = g.get_state(keys)
    out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
    assert _call(L, blocks, len(keys), None, cfg.dx0, stream, out) == mrb.MRB_OK
    assert np.array_equal(out.cpu().numpy(), g.sums().cpu().numpy()[0])
    out.fill_(float("nan"))
    assert _call(L, None, 0, None, cfg.dx0, stream, out) == mrb.MRB_OK
    assert np.array_equal(out.cpu().numpy(), np.zeros(5))
    g.close()
