"""The allocation-free ingest entry point (gpm_ingest_noalloc) against the
regular one.

Some callers cannot allocate device memory when they ingest (inside a CUDA
stream capture, with a memory budget fixed up front, or inside a framework
that owns the memory pool); gpm_ingest_noalloc serves them with a static
scratch array.  Its output must equal what gpm_match(level 0) ingests, on two
calls in a row (the array keeps the previous call's contents).  This file is
collected last so that a failure here never hides the other GPU tests.
"""
import ctypes

import numpy as np
import pytest

from paper_1804_03787_gb300 import gpm, scene

pytestmark = pytest.mark.gpu


def _regular_ingest(torch, f1, f2, storage):
    gp = gpm.default_params(patch_radius=2, cells=(16, 8), pm_iters=0, num_hyp=8, storage=storage)
    H, W, _ = f1.shape
    ctx = gpm.Context(gp, W, H)
    ctx.match([(f1, f2)])
    fr = ctx.export(gpm.FRAMES)
    ctx.close()
    return fr


@pytest.mark.parametrize("storage", [gpm.GPM_F32, gpm.GPM_BF16])
def test_noalloc_ingest_matches_regular_ingest_twice(storage):
    import torch
    assert torch.cuda.is_available()
    lib = gpm.load()
    texel = 16 if storage == gpm.GPM_F32 else 8
    stream = torch.cuda.current_stream()
    for seed, (W, H) in enumerate([(96, 72), (70, 45)]):
        s = scene.make_scene(W, H, seed=30 + seed, n_layers=2, max_disp=5.0)
        f1 = torch.from_numpy(s.frame1).cuda()
        f2 = torch.from_numpy(s.frame2).cuda()
        o1 = torch.empty(W * H * texel, dtype=torch.uint8, device="cuda")
        o2 = torch.empty(W * H * texel, dtype=torch.uint8, device="cuda")
        st = lib.gpm_ingest_noalloc(ctypes.c_void_p(f1.data_ptr()), ctypes.c_void_p(f2.data_ptr()), W, H, 3 * W, 1,
                                    storage, ctypes.c_void_p(o1.data_ptr()), ctypes.c_void_p(o2.data_ptr()),
                                    ctypes.c_void_p(stream.cuda_stream))
        assert st == gpm.GPM_OK
        torch.cuda.synchronize()
        if storage == gpm.GPM_F32:
            got = np.stack([o1.cpu().numpy().view(np.float32), o2.cpu().numpy().view(np.float32)]).reshape(2, H, W, 4)
        else:
            u = np.stack([o1.cpu().numpy().view(np.uint16), o2.cpu().numpy().view(np.uint16)]).astype(np.uint32)
            got = (u << 16).view(np.float32).reshape(2, H, W, 4)
        want = _regular_ingest(torch, f1, f2, storage)
        np.testing.assert_allclose(got[..., :3], want[..., :3], rtol=1.2e-7, atol=1e-12)


def test_noalloc_rejects_frames_beyond_its_scratch():
    import torch
    lib = gpm.load()
    x = torch.zeros(16, dtype=torch.float32, device="cuda")
    p = ctypes.c_void_p(x.data_ptr())
    assert lib.gpm_ingest_noalloc(p, p, 4, 4097, 12, 1, gpm.GPM_F32, p, p, None) == gpm.GPM_EINVAL
    assert lib.gpm_ingest_noalloc(p, p, 4, 4, 11, 1, gpm.GPM_F32, p, p, None) == gpm.GPM_EINVAL
    assert lib.gpm_ingest_noalloc(None, p, 4, 4, 12, 1, gpm.GPM_F32, p, p, None) == gpm.GPM_EINVAL
