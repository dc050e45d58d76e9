"""The allocation-free ingest entry point (gpm_ingest_noalloc) against the
regular one.

Some callers must not allocate device memory when they ingest a pair: hosts
whose device memory is reserved once at start-up, plugins of frameworks that
own the memory pool, latency-critical loops where cudaMalloc is not allowed.
gpm_ingest_noalloc serves them with a static device scratch array.  It runs
the same ingest kernels as gpm_match(level 0), so its output must equal the
regular ingest bit for bit, on two calls in a row of different sizes (the
array keeps the previous call's contents, which must not leak into the next
one).  This file is collected last so that a failure here never hides the
other GPU tests.
"""
import ctypes

import numpy as np
import pytest

from paper_1804_03787_gb300 import gpm, scene

pytestmark = pytest.mark.gpu


def _regular_ingest(f1, f2, storage, equalize):
    gp = gpm.default_params(patch_radius=2, cells=(16, 8), pm_iters=0, num_hyp=8, storage=storage,
                            equalize=equalize)
    H, W, _ = f1.shape
    ctx = gpm.Context(gp, W, H)
    ctx.match([(f1, f2)])
    fr = ctx.export(gpm.FRAMES)
    ctx.close()
    return fr


def _as_f32_rgbx(o, storage, W, H):
    raw = o.cpu().numpy()
    if storage == gpm.GPM_F32:
        return raw.view(np.float32).reshape(H, W, 4)
    if storage == gpm.GPM_BF16:
        return (raw.view(np.uint16).astype(np.uint32) << 16).view(np.float32).reshape(H, W, 4)
    return raw.view(np.float16).astype(np.float32).reshape(H, W, 4)


@pytest.mark.parametrize("storage,equalize", [(gpm.GPM_F32, 0), (gpm.GPM_BF16, 0), (gpm.GPM_F32, 1),
                                              (gpm.GPM_F16, 1)])
def test_noalloc_ingest_equals_regular_ingest_twice(storage, equalize):
    import torch
    assert torch.cuda.is_available()
    lib = gpm.load()
    texel = 16 if storage == gpm.GPM_F32 else 8
    stream = torch.cuda.current_stream()
    # two calls in a row, the second smaller and ragged: nothing of the first may carry over
    for seed, (W, H) in enumerate([(96, 72), (70, 45)]):
        s = scene.make_scene(W, H, seed=30 + seed, n_layers=2, max_disp=5.0)
        f1 = torch.from_numpy(s.frame1).cuda()
        f2 = torch.from_numpy(s.frame2).cuda()
        o1 = torch.empty(W * H * texel, dtype=torch.uint8, device="cuda")
        o2 = torch.empty(W * H * texel, dtype=torch.uint8, device="cuda")
        st = lib.gpm_ingest_noalloc(ctypes.c_void_p(f1.data_ptr()), ctypes.c_void_p(f2.data_ptr()), W, H, 3 * W, 1,
                                    equalize, storage, ctypes.c_void_p(o1.data_ptr()), ctypes.c_void_p(o2.data_ptr()),
                                    ctypes.c_void_p(stream.cuda_stream))
        assert st == gpm.GPM_OK
        torch.cuda.synchronize()
        got = np.stack([_as_f32_rgbx(o1, storage, W, H), _as_f32_rgbx(o2, storage, W, H)])
        want = _regular_ingest(f1, f2, storage, equalize)
        np.testing.assert_array_equal(got[..., :3], want[..., :3])


def test_noalloc_rejects_bad_arguments():
    import torch
    lib = gpm.load()
    x = torch.zeros(16, dtype=torch.float32, device="cuda")
    p = ctypes.c_void_p(x.data_ptr())
    assert lib.gpm_ingest_noalloc(p, p, 32768, 1, 3 * 32768, 1, 0, gpm.GPM_F32, p, p, None) == gpm.GPM_EINVAL
    assert lib.gpm_ingest_noalloc(p, p, 16384, 8192, 3 * 16384, 1, 0, gpm.GPM_F32, p, p, None) == gpm.GPM_EINVAL
    assert lib.gpm_ingest_noalloc(p, p, 4, 4, 11, 1, 0, gpm.GPM_F32, p, p, None) == gpm.GPM_EINVAL
    assert lib.gpm_ingest_noalloc(None, p, 4, 4, 12, 1, 0, gpm.GPM_F32, p, p, None) == gpm.GPM_EINVAL
    assert lib.gpm_ingest_noalloc(p, p, 4, 4, 12, 1, 2, gpm.GPM_F32, p, p, None) == gpm.GPM_EINVAL
    assert lib.gpm_ingest_noalloc(p, p, 4, 4, 12, 1, 0, 3, p, p, None) == gpm.GPM_EINVAL
