"""GPU edge cases: degenerate inputs, the smallest and a large frame, and calls the library must refuse.

Constant frames make every patch cost exactly zero, so every decision is exact on both sides: the GPU result
must equal the oracle's bit for bit (PatchMatch keeps the random initial field on ties, no window finds a
plane, every pixel is occluded).  Identical frames are the zero-motion case.  A frame of exactly the largest
window's size has one window per axis at that level; a ragged size just above it gets a border-flush window.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_1804_03787_gb300 import gpm, scene

from _parity import end_to_end_stats, final_map_check, oracle_frames, oracle_params, ransac_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need a CUDA device"
    gpm.load()
    return t


def _dev(torch, f1, f2):
    return torch.from_numpy(np.ascontiguousarray(f1, np.float32)).cuda(), \
        torch.from_numpy(np.ascontiguousarray(f2, np.float32)).cuda()


def _both(torch, gp, f1, f2):
    H, W = f1.shape[:2]
    ctx = gpm.Context(gp, W, H)
    flows, occs = ctx.run([_dev(torch, f1, f2)])
    torch.cuda.synchronize()
    g = (flows[0].cpu().numpy(), occs[0].cpu().numpy())
    R = O.run(oracle_params(gp, W, H), f1, f2)
    o = (R.flow[0].reshape(H, W, 2), R.occ[0].reshape(H, W))
    return ctx, g, o


def test_constant_frames_exactly_equal_oracle(torch):
    f = np.full((48, 64, 3), 0.4, np.float32)
    gp = gpm.default_params(patch_radius=2, cells=(16, 8), pm_iters=2, num_hyp=64)
    ctx, (gf, go), (of, oo) = _both(torch, gp, f, f.copy())
    np.testing.assert_array_equal(gf, of)
    np.testing.assert_array_equal(go, oo)
    assert (go == 1).all()  # no plane anywhere: every pixel keeps its (random) NNF offset, occluded
    P = oracle_params(gp, 64, 48)
    frames, _ = oracle_frames(P, f, f)
    vx, vy, _ = O.pm_init(P, frames[0][0], frames[0][1], 0)
    np.testing.assert_array_equal(gf[..., 0].reshape(-1), vx)
    np.testing.assert_array_equal(gf[..., 1].reshape(-1), vy)
    ctx.close()


def test_identical_frames_zero_motion(torch):
    s = scene.tiny_scene(4)
    gp = gpm.default_params()
    ctx, (gf, go), (of, oo) = _both(torch, gp, s.frame1, s.frame1.copy())
    agree = np.mean(np.hypot(*(gf - of).transpose(2, 0, 1)) < 1e-4)
    assert agree > 0.95, agree
    # the zero field is the answer: nearly every pixel gets a plane within 0.05 px of it (the least-squares refit
    # also takes NNF offsets within the RANSAC threshold, so a plane need not be the exact identity), and nearly
    # none is occluded
    assert np.mean(np.hypot(*gf.transpose(2, 0, 1)) < 0.05) > 0.97
    assert go.mean() < 0.03
    ctx.close()


@pytest.mark.parametrize("W,H", [(32, 32), (33, 35)])
def test_smallest_frames_end_to_end(torch, W, H):
    """Frames of the largest window's size (one window per axis at level 1) and a ragged size just above."""
    s = scene.make_scene(W, H, seed=W + H, n_layers=1, max_disp=3.0, affine=True)
    gp = gpm.default_params()
    ctx, (gf, go), (of, oo) = _both(torch, gp, s.frame1, s.frame2)
    agree = np.mean(np.hypot(*(gf - of).transpose(2, 0, 1)) < 1e-4)
    assert agree > 0.95, agree
    assert np.mean(go == oo) > 0.95
    ctx.close()


@pytest.mark.parametrize("W,H", [(1920, 1080), (3840, 2160)])
def test_large_frame_final_map(torch, W, H):
    """1920x1080 (the largest serving size) and 3840x2160 pairs in the benchmark configuration: the final map's
    properties on sampled pixels."""
    s = scene.make_scene(W, H, seed=7, n_layers=6, max_disp=64.0, affine=False, area_frac=(0.02, 0.08))
    gp = gpm.default_params(patch_radius=4, cells=(64, 32, 16, 8), pm_iters=8, num_hyp=512)
    P = oracle_params(gp, W, H)
    frames, _ = oracle_frames(P, s.frame1, s.frame2)
    ctx = gpm.Context(gp, W, H)
    flows, occs = ctx.run([_dev(torch, s.frame1, s.frame2)])
    torch.cuda.synchronize()
    n_plane, n_checked = final_map_check(ctx, P, frames, flows[0], occs[0], samples=3000, seed=5)
    assert n_plane > 2000 and n_checked > 1500, (n_plane, n_checked)
    e = np.hypot(*(flows[0].cpu().numpy() - s.flow).transpose(2, 0, 1))
    assert e[s.occ == 0].mean() < 3.0
    ctx.close()


def test_invalid_calls_are_refused(torch):
    gp = gpm.default_params()
    ctx = gpm.Context(gp, 64, 48)
    # stage order: planes before any matching, matching a level before fitting it
    with pytest.raises(gpm.GpmError):
        ctx.fit_planes(1)
    s = scene.make_scene(64, 48, seed=1, n_layers=1, max_disp=3.0, affine=True)
    ctx.match([_dev(torch, s.frame1, s.frame2)])
    with pytest.raises(gpm.GpmError):
        ctx.match(None, 1)
    with pytest.raises(gpm.GpmError):
        ctx.fit_planes(2)
    # frames smaller than the largest window, or larger than the context's limits
    with pytest.raises(gpm.GpmError):
        ctx.match([_dev(torch, np.zeros((20, 64, 3)), np.zeros((20, 64, 3)))])
    with pytest.raises(gpm.GpmError):
        ctx.match([_dev(torch, np.zeros((48, 80, 3)), np.zeros((48, 80, 3)))])
    # an empty batch
    with pytest.raises(gpm.GpmError):
        ctx.match([])
    # a frame dtype outside gpm_dtype, through the C ABI
    f1, f2 = _dev(torch, s.frame1, s.frame2)
    bad = gpm.Pair(64, 48, 3 * 64, f1.data_ptr(), f2.data_ptr(), 0, 7)
    assert ctx.lib.gpm_match(ctx.h, ctypes.byref(bad), 1, 0) == gpm.GPM_EINVAL
    assert "dtype" in ctx.lib.gpm_last_error(ctx.h).decode()
    # the context stays usable after refused calls
    flows, occs = ctx.run([_dev(torch, s.frame1, s.frame2)])
    torch.cuda.synchronize()
    assert np.isfinite(flows[0].cpu().numpy()).all()
    ctx.close()


def test_device_consistency_flag_reports_bad_imported_labels(torch):
    """GPM_EINTERNAL: labels imported with a model id beyond the model table (and one with a non-finite flow) are
    caught on the device, those pixels get no plane, gpm_sync reports the check once, and the context then runs a
    whole pair as before (nothing read outside the model table)."""
    gp = gpm.default_params()
    s = scene.make_scene(64, 48, seed=2, n_layers=1, max_disp=3.0, affine=True)
    ctx = gpm.Context(gp, 64, 48)
    ctx.match([_dev(torch, s.frame1, s.frame2)])
    ctx.fit_planes(1)
    m, L, f = ctx.export(gpm.LABELS)
    n_models = ctx.export(gpm.MODELS).shape[1]
    m = m.copy()
    f = f.copy()
    m[0, 5] = n_models + 7
    m[1, 9] = -3
    m[0, 11] = 0
    f[0, 11] = (np.inf, 0.0)
    ctx.import_state_raw(gpm.LABELS, (m, L, f), stage=1)
    with pytest.raises(gpm.GpmError) as e:
        ctx.sync()
    assert e.value.status == gpm.GPM_EINTERNAL
    ctx.sync()  # reported once, then cleared
    got, _, _ = ctx.export(gpm.LABELS)
    assert got[0, 5] == -1 and got[1, 9] == -1 and got[0, 11] == -1
    flows, occs = ctx.run([_dev(torch, s.frame1, s.frame2)])
    ctx.sync()
    assert np.isfinite(flows[0].cpu().numpy()).all()
    ctx.close()


def test_profile_select_brackets_only_the_chosen_classes(torch):
    """gpm_profile_select: only the chosen kernel classes are timed, evaluations are counted only on request, and
    a bit beyond the last class is refused."""
    s = scene.tiny_scene(1)
    ctx = gpm.Context(gpm.default_params(), 128, 96)
    ctx.profile_select(["pm_sweep"], count_evals=False)
    ctx.profile_read()
    ctx.run([_dev(torch, s.frame1, s.frame2)])
    prof, evals = ctx.profile_read()
    assert prof["pm_sweep"][0] > 0 and prof["pm_sweep"][1] > 0
    assert all(ms == 0 and n == 0 for k, (ms, n) in prof.items() if k != "pm_sweep")
    assert evals == (0,) * gpm.COUNTERS
    ctx.profile_enable(True)
    ctx.profile_read()
    ctx.run([_dev(torch, s.frame1, s.frame2)])
    prof, evals = ctx.profile_read()
    assert all(prof[k][1] > 0 for k in ("pm_sweep", "pm_sweep_plane", "ransac", "assign", "final"))
    assert all(e > 0 for e in evals)
    # the initial field (one evaluation per pixel and direction) and the recosts of the plane levels
    assert evals[gpm.COUNT_INIT] > 2 * 128 * 96
    # taps actually summed: at most (2r + 1)^2 per evaluation, at least the first 32 (r = 3)
    for ev, taps in ((gpm.COUNT_SWEEP0, gpm.COUNT_SWEEP0_TAPS), (gpm.COUNT_SWEEP_PLANE, gpm.COUNT_SWEEP_PLANE_TAPS)):
        assert 32 * evals[ev] <= evals[taps] <= 49 * evals[ev], (evals[ev], evals[taps])
    with pytest.raises(gpm.GpmError):
        ctx._check(ctx.lib.gpm_profile_select(ctx.h, 1 << len(gpm.PROF_CLASSES), 0), "gpm_profile_select")
    ctx.close()


# ---------------------------------------------------------------- plane validity on hand-built matches
def _validity_nnf(S, scenarios, seed):
    """NNF of an SxS frame whose disjoint 8x8 windows at (x0, y0) carry the given match sets (zero offsets
    elsewhere). Kinds: ('shear', n_in): x' = x + (y - y0) - 4, y' = y - 2 (orientation kept, scale 1), with the
    other 64 - n_in matches moved to random targets at least 4 px from it; 'mirror': x' = 2 x0 + 7 - x;
    'scale2': twice the distance from (x0 + 2, y0 + 2); 'proj': (p - o) / w + o - 8 with w = 1 - (x - x0) / 10.5,
    rounded. Every target stays inside the frame."""
    rng = np.random.default_rng(seed)
    vx = np.zeros((S, S), np.int32)
    vy = np.zeros((S, S), np.int32)
    for (x0, y0), kind in scenarios.items():
        ys, xs = np.mgrid[y0:y0 + 8, x0:x0 + 8]
        if kind == "mirror":
            tx, ty = 2 * x0 + 7 - xs, ys
        elif kind == "scale2":
            tx, ty = 2 * (xs - x0) + x0 - 4, 2 * (ys - y0) + y0 - 4
        elif kind == "proj":
            w = 1 - (xs - x0) / 10.5
            tx, ty = np.round((xs - x0) / w) + x0 - 8, np.round((ys - y0) / w) + y0 - 8
        else:
            tx, ty = xs + (ys - y0) - 4, ys - 2
            out = rng.permutation(64)[kind[1]:]
            for k in out:
                r, c = divmod(k, 8)
                while True:
                    qx, qy = rng.integers(x0 - 8, x0 + 16), rng.integers(y0 - 8, y0 + 16)
                    if max(abs(qx - tx[r, c]), abs(qy - ty[r, c])) >= 4:
                        break
                tx[r, c], ty[r, c] = qx, qy
        assert tx.min() >= 0 and ty.min() >= 0 and tx.max() < S and ty.max() < S
        vx[y0:y0 + 8, x0:x0 + 8] = tx - xs
        vy[y0:y0 + 8, x0:x0 + 8] = ty - ys
    return vx.reshape(-1), vy.reshape(-1)


@pytest.mark.parametrize("r,min_in,scenarios", [
    (2, 8, {(8, 8): ("shear", 13), (16, 8): ("shear", 12), (24, 8): "mirror", (32, 8): "scale2",
            (8, 16): "proj", (16, 16): ("shear", 64), (24, 16): ("shear", 20)}),
    (4, 20, {(8, 8): ("shear", 20), (16, 8): ("shear", 19), (8, 16): "proj"}),
])
def test_plane_validity_rules_on_hand_built_matches(torch, r, min_in, scenarios):
    """Readings R12/R14 through the C ABI: a 48x48 frame pair whose disjoint interior 8x8 windows carry match
    sets built to sit on either side of a validity rule (support of at least max(min_inliers, N/5), orientation,
    scale range, denominator over the window grown by r). The GPU's stage-1 fit of every window equals the
    oracle's (support, winner, refit and geometry flags, H to 1e-6) except where the oracle logged a near tie,
    and each built window is valid or not as the rule says."""
    S = 48
    f = np.full((S, S, 3), 0.5, np.float32)
    gp = gpm.default_params(patch_radius=r, cells=(8,), pm_iters=1, num_hyp=4000, min_inliers=min_in)
    P = oracle_params(gp, S, S)
    vx, vy = _validity_nnf(S, scenarios, seed=r)
    ctx = gpm.Context(gp, S, S)
    ctx.match([_dev(torch, f, f)])
    nnf = np.stack([np.stack([vx, vy], 1)] * 2).astype(np.int32)
    ctx.import_state(gpm.NNF, nnf, level=0)
    ctx.fit_planes(1)
    gmh, gmi = ctx.export(gpm.MODELS), ctx.export(gpm.MODEL_INFO)
    ctx.close()
    nx = len(O.grid_axis(S, 8))
    ids = np.arange(0, 2 * int(O.cell_base(P)[1]), 2)
    frame = np.asarray(f, np.float64)
    for d in range(2):
        mh, mi = O.empty_models(P)
        O.fit_level(P, frame, frame, d, 1, 1, vx, vy, None, mh, mi)
        ok = ransac_equal(gmh[d], gmi[d], mh, mi, ids)
        tie = (mi[ids, O.MI_FLAGS] & O.F_AMBIG) > 0
        assert not (~ok & ~tie).any(), f"dir {d}: windows {ids[~ok & ~tie] // 2} differ"
        for (x0, y0), kind in scenarios.items():
            m = ((y0 // 4) * nx + x0 // 4) * 2
            if kind == "scale2":                       # scale 2 = scale_max: decided by rounding, logged as a tie
                assert mi[m, O.MI_FLAGS] & O.F_AMBIG and gmi[d][m, O.MI_COUNT] == 64
                continue
            if kind == "mirror":
                want = False
            elif kind == "proj":
                want = r + 7 < 10.5                    # denominator positive at the grown window's far corners
            else:
                want = kind[1] >= min_in and 5 * kind[1] >= 64
                assert mi[m, O.MI_COUNT] == kind[1], (kind, mi[m])
            # the rule on the oracle; on the GPU wherever the oracle logged no near tie (then both sides agree)
            sides = (mi[m],) if tie[m // 2] else (mi[m], gmi[d][m])
            for side in sides:
                assert bool(side[O.MI_FLAGS] & O.F_BAD_GEOM) == (not want), ((x0, y0), kind, d, side)


@pytest.mark.parametrize("kw", [dict(num_hyp=1), dict(num_hyp=4096, min_inliers=4), dict(fill_iters=0, pm_iters=1)])
def test_parameter_extremes_end_to_end(torch, kw):
    """The tiny configuration at the ends of the parameter ranges the library accepts (one RANSAC hypothesis per
    window; the most hypotheses with the smallest support; no fill and a single PatchMatch iteration): the whole
    method against the oracle, with the bars of the tiny end-to-end test (plane pixels: EPE within 1e-3 px)."""
    s = scene.tiny_scene(2)
    gp = gpm.default_params(**kw)
    ctx = gpm.Context(gp, 128, 96)
    flows, _ = ctx.run([_dev(torch, s.frame1, s.frame2)])
    torch.cuda.synchronize()
    R = O.run(oracle_params(gp, 128, 96), s.frame1, s.frame2)
    st = end_to_end_stats(ctx, R, flows[0].cpu().numpy(), R.flow[0].reshape(96, 128, 2), s.flow, s.occ, 96, 128)
    ctx.close()
    print(kw, {k: round(v, 5) for k, v in st.items()})
    # the same plane decision: the flows agree within the FP32 mapping's error, the EPE within 1e-3 px
    assert st["same_share"] > 0.6 and st["same_max_flow_diff"] < 1e-3, st
    assert abs(st["epe_same_gpu"] - st["epe_same_oracle"]) <= 1e-3, st
    # different plane decisions (near ties between overlapping windows' fits of one surface) are few
    assert st["label_agree"] > 0.98 and st["plane_agree"] > 0.97, st
    assert st["agree"] > 0.95 and abs(st["epe_gpu"] - st["epe_oracle"]) < 0.05, st