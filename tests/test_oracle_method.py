"""Pins of the FP64 oracle's method steps against invariants, hand-built cases
and scenes whose answer is known.

* PatchMatch: the exhaustive-search NNF (independent numpy brute force) is a
  fixed point of a red-black iteration, and PatchMatch from a random start
  reaches it on most pixels.
* A single global homography scene: every window fits the generating plane
  (to the integer-NNF rounding limit), every mapped pixel is assigned, the
  symmetry cue passes, the flow matches the generating map.
* Cues, merge, NNF update and fill on hand-built label maps.
* Whole method on synthetic scenes with exact ground truth.
"""
import numpy as np
import pytest

import oracle as O
from paper_1804_03787_gb300 import scene


# ---------------------------------------------------------------- PatchMatch
def _brute_nnf(src, tgt, r):
    """Exhaustive square-patch NNF by numpy: argmin over every in-frame target,
    ties to the lowest (ty, tx)."""
    H, W, _ = src.shape
    pad_s = np.pad(src, ((r, r), (r, r), (0, 0)), mode="edge")
    # patches of the source, clamped at the border
    ps = np.stack([pad_s[r + dy:r + dy + H, r + dx:r + dx + W] for dy in range(-r, r + 1) for dx in range(-r, r + 1)], 0)
    vx = np.zeros((H, W), np.int32)
    vy = np.zeros((H, W), np.int32)
    best = np.full((H, W), np.inf)
    ys, xs = np.mgrid[0:H, 0:W]
    taps = [(dy, dx) for dy in range(-r, r + 1) for dx in range(-r, r + 1)]
    for ty in range(H):
        for tx in range(W):
            ox, oy = tx - xs, ty - ys
            acc = np.zeros((H, W))
            for k, (dy, dx) in enumerate(taps):
                sx, sy = np.clip(xs + dx, 0, W - 1), np.clip(ys + dy, 0, H - 1)
                qx, qy = np.clip(sx + ox, 0, W - 1), np.clip(sy + oy, 0, H - 1)
                acc += np.abs(ps[k] - tgt[qy, qx]).sum(-1)
            acc /= 3 * len(taps)
            upd = acc < best
            best[upd] = acc[upd]
            vx[upd] = ox[upd]
            vy[upd] = oy[upd]
    return vx.reshape(-1), vy.reshape(-1), best.reshape(-1)


@pytest.mark.parametrize("r", [1, 2, 3])
def test_exhaustive_nnf_is_patchmatch_fixed_point(r):
    rng = np.random.default_rng(10 + r)
    H, W = 12, 16
    src = rng.random((H, W, 3))
    tgt = np.roll(src, (1, 2), axis=(0, 1)) * 0.9 + 0.1 * rng.random((H, W, 3))
    vx, vy, best = _brute_nnf(src, tgt, r)
    P = O.Params(W, H, patch_radius=r)
    cost = np.zeros(W * H)
    O.pm_recost(P, src, tgt, 0, None, None, None, vx, vy, cost)
    np.testing.assert_allclose(cost, best, rtol=1e-12, atol=0)
    vx2, vy2, c2 = vx.copy(), vy.copy(), cost.copy()
    for it in range(2):
        for ph in range(2):
            O.pm_sweep(P, src, tgt, 0, 0, it, ph, None, None, None, vx2, vy2, c2)
    np.testing.assert_array_equal(vx2, vx)
    np.testing.assert_array_equal(vy2, vy)


def test_patchmatch_converges_toward_exhaustive_nnf():
    """From random offsets, 8 red-black iterations reach the exhaustive NNF on
    most pixels of a textured pair; costs never increase."""
    s = scene.make_scene(32, 24, seed=3, n_layers=1, max_disp=4.0, affine=True, noise=0.0, gain=(1, 1))
    src, tgt = s.frame1.astype(np.float64), s.frame2.astype(np.float64)
    r = 2
    vx, vy, best = _brute_nnf(src, tgt, r)
    P = O.Params(32, 24, patch_radius=r)
    ux, uy, c = O.pm_init(P, src, tgt, 0)
    prev = c.copy()
    for it in range(8):
        for ph in range(2):
            O.pm_sweep(P, src, tgt, 0, 0, it, ph, None, None, None, ux, uy, c)
        assert np.all(c <= prev + 1e-15)
        prev = c.copy()
    agree = np.mean((ux == vx) & (uy == vy))
    assert agree >= 0.9, agree
    assert np.all(c >= best - 1e-12)


def test_propagation_takes_offsets_from_each_of_the_four_neighbours():
    """Sec. 3.1 (PatchMatch propagation): the target frame is the source moved by (3, 2), so that offset costs
    exactly zero inside the frame, and every pixel holds the offset (0, 0) except one neighbour of each test pixel
    (left, right, upper or lower in turn), which holds (3, 2). One half-step of the red-black sweep gives every
    test pixel (3, 2): from whichever side it is offered (random search alone would rarely hit that exact offset)."""
    W, H, r = 48, 40, 1
    rng = np.random.default_rng(21)
    src = rng.random((H, W, 3))
    tgt = np.roll(src, (2, 3), axis=(0, 1))
    P = O.Params(W, H, patch_radius=r)
    vx, vy = np.zeros(W * H, np.int32), np.zeros(W * H, np.int32)
    tests = [(x, y) for y in range(4, H - 5, 4) for x in range(4, W - 6, 4)]
    for j, (x, y) in enumerate(tests):
        dx, dy = ((-1, 0), (1, 0), (0, -1), (0, 1))[j % 4]
        vx[(y + dy) * W + x + dx], vy[(y + dy) * W + x + dx] = 3, 2
    cost = np.zeros(W * H)
    O.pm_recost(P, src, tgt, 0, None, None, None, vx, vy, cost)
    O.pm_sweep(P, src, tgt, 0, 0, 0, 0, None, None, None, vx, vy, cost)
    ids = np.array([y * W + x for x, y in tests])
    got = np.stack([vx[ids], vy[ids]], 1)
    for k in range(4):
        np.testing.assert_array_equal(got[k::4], np.tile([3, 2], (len(ids[k::4]), 1)), err_msg=f"neighbour {k}")
    assert (cost[ids] == 0).all()


def test_distortion_plane_is_the_home_window_model():
    """Reading R9: at a level >= 1 a pixel's patch is distorted by the plane of its home window, the window whose
    central half [x0 + s/4, x0 + 3s/4) holds it (the first or last window beyond the grid's ends): its
    residual-stage plane if valid, else its first-stage plane, else none. Windows of 8 px at stride 4 over a
    24 px row start at 0, 4, 8, 12, 16, so pixels 0-5 are homed in window 0, 6-9 in 1, 10-13 in 2, 14-17 in
    3 and 18-23 in 4. Each window carries a different zoom, so a wrong home changes the cost."""
    W, H, r = 24, 8, 1
    P = O.Params(W, H, patch_radius=r, cells=(8,))
    assert list(O.grid_axis(W, 8)) == [0, 4, 8, 12, 16] and list(O.grid_axis(H, 8)) == [0]
    rng = np.random.default_rng(8)
    src, tgt = rng.random((H, W, 3)), rng.random((H, W, 3))

    def zoom(z):
        return np.diag([z, z, 1.0])

    mh, mi = O.empty_models(P)
    for c in range(5):
        mh[2 * c] = zoom(1.0 + 0.1 * c).reshape(9)                 # first stage of window c
    mh[2 * 2 + 1] = zoom(0.7).reshape(9)                           # residual stage of window 2
    mi[[0, 2, 4, 5, 8], O.MI_VALID] = 1                            # window 3: no valid plane
    home = [0] * 6 + [1] * 4 + [2] * 4 + [3] * 4 + [4] * 6
    plane = {0: zoom(1.0), 1: zoom(1.1), 2: zoom(0.7), 3: None, 4: zoom(1.4)}
    vx = rng.integers(-2, 3, W * H).astype(np.int32)
    vy = rng.integers(-2, 3, W * H).astype(np.int32)
    cost = np.zeros(W * H)
    O.pm_recost(P, src, tgt, 1, mh, mi, np.zeros(W * H, np.uint8), vx, vy, cost)
    for y in (0, 3, 7):
        for x in range(W):
            i = y * W + x
            want = O.patch_cost(P, src, tgt, x, y, int(vx[i]), int(vy[i]), plane[home[x]])
            assert cost[i] == want, (x, y, home[x])


def test_pm_init_targets_inside_frame_and_deterministic():
    P = O.Params(40, 30, patch_radius=1, seed=77)
    f = np.random.default_rng(0).random((30, 40, 3))
    a = O.pm_init(P, f, f, 0)
    b = O.pm_init(P, f, f, 0)
    c = O.pm_init(P, f, f, 1)
    ys, xs = np.divmod(np.arange(40 * 30), 40)
    assert np.all((xs + a[0] >= 0) & (xs + a[0] < 40) & (ys + a[1] >= 0) & (ys + a[1] < 30))
    np.testing.assert_array_equal(a[0], b[0])
    assert np.mean(a[0] == c[0]) < 0.2   # the two directions draw independent streams


# ---------------------------------------------------------------- single-plane scene
def _plane_scene(W, H, Hm, key=12345):
    ys, xs = np.mgrid[0:H, 0:W].astype(float)
    tex = lambda x, y: np.stack([scene.value_noise(x, y, key + 17 * c, period=16.0) for c in range(3)], -1)
    f1 = tex(xs, ys)
    Hi = np.linalg.inv(Hm)
    qx, qy = scene.apply_h(Hi, xs, ys)
    f2 = tex(qx, qy)
    return f1, f2


def _round_nnf(Hm, W, H):
    ys, xs = np.divmod(np.arange(W * H), W)
    X, Y = scene.apply_h(Hm, xs.astype(float), ys.astype(float))
    vx = np.floor(X - xs + 0.5).astype(np.int32)
    vy = np.floor(Y - ys + 0.5).astype(np.int32)
    ok = (xs + vx >= 0) & (xs + vx < W) & (ys + vy >= 0) & (ys + vy < H)
    vx[~ok] = 0
    vy[~ok] = 0
    return vx, vy, X - xs, Y - ys


def test_single_plane_scene_is_recovered_and_assigned():
    W, H = 96, 64
    Hm = scene.h_from_points(np.array([[0, 0], [95, 0], [95, 63], [0, 63]], float),
                             np.array([[2, 1], [97, -1], [94, 66], [-1, 62]], float))
    f1, f2 = _plane_scene(W, H, Hm)
    P = O.Params(W, H, patch_radius=2, cells=(32,), num_hyp=128, eps=0.03)
    vx0, vy0, fx, fy = _round_nnf(Hm, W, H)
    vx1, vy1, _, _ = _round_nnf(np.linalg.inv(Hm), W, H)
    mh, mi = [O.empty_models(P) for _ in range(2)], None
    labs = []
    for d, (vx, vy, src, tgt) in enumerate([(vx0, vy0, f1, f2), (vx1, vy1, f2, f1)]):
        mh_d, mi_d = mh[d]
        O.fit_level(P, src, tgt, d, 1, 1, vx, vy, None, mh_d, mi_d)
        lab = O.Labels.empty(W * H, P.eps)
        O.assign(P, src, tgt, 1, 1, mh_d, mi_d, None, lab)
        labs.append(lab)
    mh0, mi0 = mh[0]
    fitted = mi0[::2, O.MI_FLAGS] & O.F_FITTED
    assert fitted.all()
    assert mi0[::2, O.MI_VALID].all()
    # every window's plane is the generating map to the integer-rounding limit
    ys, xs = np.divmod(np.arange(W * H), W)
    gx, gy = O.grid_axis(W, 32), O.grid_axis(H, 32)
    for c in range(mi0.shape[0] // 2):
        x0, y0 = gx[c % len(gx)], gy[c // len(gx)]
        win = (xs >= x0) & (xs < x0 + 32) & (ys >= y0) & (ys < y0 + 32)
        Hc = mh0[2 * c].reshape(3, 3)
        X, Y = scene.apply_h(Hc, xs.astype(float), ys.astype(float))
        err = np.hypot(X - xs - fx, Y - ys - fy)[win]
        # the matches are rounded to integers (error up to 0.71 px each)
        assert err.max() < 1.0 and err.mean() < 0.3, (c, err.max(), err.mean())
    # every pixel whose true target lies inside the frame (1 px margin) is assigned
    X, Y = xs + fx, ys + fy
    inside = (X >= 1) & (X <= W - 2) & (Y >= 1) & (Y <= H - 2)
    assert np.all(labs[0].m[inside] >= 0)
    err = np.hypot(labs[0].fx - fx, labs[0].fy - fy)[labs[0].m >= 0]
    assert err.max() < 1.0 and err.mean() < 0.3
    # the symmetry cue passes for every plane
    O.cue_counts(P, 1, 1, labs[0], labs[1], mi0)
    nas, nsy = mi0[::2, O.MI_NASSIGN], mi0[::2, O.MI_NSYM]
    assert np.all(nsy >= P.eta * nas) and nas.sum() >= inside.sum()
    O.cue_invalidate(P, 1, 1, mi0)
    assert mi0[::2, O.MI_VALID].all()


def test_overlap_cue_discards_colour_inconsistent_plane():
    """Geometrically perfect matches between unrelated frames: RANSAC accepts the
    plane, but almost none of its inliers are colour inliers, so kappa discards it."""
    rng = np.random.default_rng(8)
    W, H = 32, 32
    f1, f2 = rng.random((H, W, 3)), rng.random((H, W, 3))
    P = O.Params(W, H, patch_radius=1, cells=(16,), num_hyp=64)
    T = np.array([[1, 0, 2], [0, 1, 1], [0, 0, 1.0]])
    vx, vy, _, _ = _round_nnf(T, W, H)
    mh, mi = O.empty_models(P)
    O.fit_level(P, f1, f2, 0, 1, 1, vx, vy, None, mh, mi)
    assert mi[0, O.MI_VALID] == 1 and mi[0, O.MI_NRC] < P.kappa * mi[0, O.MI_COUNT]
    O.cue_invalidate(P, 1, 1, mi)
    assert mi[0, O.MI_VALID] == 0 and mi[0, O.MI_FLAGS] & O.F_BAD_KAPPA


def test_symmetry_cue_discards_asymmetric_plane():
    """Forward labels say +3 px, backward labels say +3 px too (not -3): no pixel
    is forward-backward symmetric, the plane is discarded (eta)."""
    W, H = 32, 16
    P = O.Params(W, H, cells=(16,))
    n = W * H
    lab = O.Labels(np.zeros(n, np.int32), np.full(n, 0.01), np.full(n, 3.0), np.zeros(n))
    other = O.Labels(np.zeros(n, np.int32), np.full(n, 0.01), np.full(n, 3.0), np.zeros(n))
    mh, mi = O.empty_models(P)
    mi[:, O.MI_VALID] = 1
    mi[:, O.MI_COUNT] = 10
    mi[:, O.MI_NRC] = 10
    O.cue_counts(P, 1, 1, lab, other, mi)
    assert mi[0, O.MI_NASSIGN] == n and mi[0, O.MI_NSYM] == 0
    other.fx[:] = -3.0
    O.cue_counts(P, 1, 1, lab, other, mi)
    assert mi[0, O.MI_NSYM] == n - 3 * H     # the last 3 columns land outside the frame
    other.fx[:] = 3.0
    O.cue_counts(P, 1, 1, lab, other, mi)
    O.cue_invalidate(P, 1, 1, mi)
    assert mi[0, O.MI_VALID] == 0 and mi[0, O.MI_FLAGS] & O.F_BAD_FB


# ---------------------------------------------------------------- hand-built label maps
def test_many_to_one_flags_the_worse_of_two_motions():
    W, H = 10, 1
    P = O.Params(W, H, patch_radius=1, cells=(2,))
    n = W
    lab = O.Labels.empty(n, P.eps)
    # p=1 (flow +4) and p=7 (flow -2) both land on q=5; p=7 has the lower L -> p=1 occluded
    # p=4 (flow +1.2) also rounds to q=5 with a flow close to p=7's? no: 1.2 vs -2 differ -> flagged
    # p=6 (flow -1.4, rounds to 5) differs from p=7's flow by 0.6 < t_fb -> same motion, kept
    for p, f, L, m in [(1, 4.0, 0.03, 2), (7, -2.0, 0.01, 4), (4, 1.2, 0.02, 6), (6, -1.4, 0.02, 4), (8, 1.0, 0.05, 8)]:
        lab.m[p], lab.fx[p], lab.L[p] = m, f, L
    cue = np.zeros(n, np.uint8)
    O.many_to_one(P, lab, cue)
    assert list(np.flatnonzero(cue)) == [1, 4]
    assert lab.m[1] == -1 and lab.m[4] == -1 and lab.m[7] == 4 and lab.m[6] == 4 and lab.m[8] == 8


def test_many_to_one_targets_round_half_up():
    """Reading R17's target q = round(p + f), rounding halves up: p = 2 with flow 2.5 lands on q = 5, as does
    p = 7 with flow -2; their flows differ by 4.5 >= t_fb, so the one with the higher L (p = 2) is occluded.
    Truncating instead would send p = 2 to 4, with no conflict."""
    P = O.Params(10, 1, patch_radius=1, cells=(2,))
    lab = O.Labels.empty(10, P.eps)
    for p, f, L, m in [(2, 2.5, 0.03, 2), (7, -2.0, 0.01, 4)]:
        lab.m[p], lab.fx[p], lab.L[p] = m, f, L
    cue = np.zeros(10, np.uint8)
    O.many_to_one(P, lab, cue)
    assert list(np.flatnonzero(cue)) == [2] and lab.m[2] == -1 and lab.m[7] == 4


def test_symmetry_count_reads_the_target_rounded_half_up():
    """Sec. 3.4 cue (1) with reading R17's rounding: p = 2 with flow 2.5 looks up the other direction at
    q = round(4.5) = 5, where the flow is -2.5 (symmetric); at 4, where truncation would look, the flow is +9.
    Pixel 6 with flow 1 meets -1 at 7 (symmetric). Both count as assigned and symmetric."""
    P = O.Params(10, 2, patch_radius=1, cells=(2,), fb_px=1.0)
    n = 20
    lab, other = O.Labels.empty(n, P.eps), O.Labels.empty(n, P.eps)
    for p, f in [(2, 2.5), (6, 1.0)]:
        lab.m[p], lab.fx[p] = 4, f
    for q, f in [(5, -2.5), (4, 9.0), (7, -1.0)]:
        other.m[q], other.fx[q] = 0, f
    _, mi = O.empty_models(P)
    O.cue_counts(P, 1, 1, lab, other, mi)
    assert mi[4, O.MI_NASSIGN] == 2 and mi[4, O.MI_NSYM] == 2


def test_merge_keeps_coarse_unless_clearly_better_and_nnf_update_rounds_half_up():
    P = O.Params(4, 1, cells=(2,), beta=0.015)
    acc = O.Labels(np.array([-1, 5, 5, 5], np.int32), np.array([0.06, 0.03, 0.03, 0.03]),
                   np.array([0, 1.0, 1.0, 1.0]), np.zeros(4))
    lab = O.Labels(np.array([7, 7, 7, -1], np.int32), np.array([0.04, 0.02, 0.01, 0.0]),
                   np.array([2.5, -1.5, 0.49, 9.0]), np.array([-0.5, 0.5, -2.5, 0.0]))
    O.merge(P, lab, acc)
    assert list(acc.m) == [7, 5, 7, 5]
    vx, vy, fr = np.zeros(4, np.int32), np.zeros(4, np.int32), np.zeros(4, np.uint8)
    O.nnf_update(P, acc, vx, vy, fr)
    assert list(vx) == [3, 1, 0, 1] and list(vy) == [0, 0, -2, 0] and list(fr) == [1, 1, 1, 1]


def test_fill_front_advances_one_pixel_per_jacobi_iteration():
    """A global plane assigned everywhere except a hole: after k iterations
    exactly the hole pixels within 4-neighbour distance k of the assigned region
    are filled (cue-flagged pixels never are)."""
    W, H = 24, 20
    Hm = np.array([[1, 0, 2.0], [0, 1, 1.0], [0, 0, 1.0]])
    f1, f2 = _plane_scene(W, H, Hm)
    P = O.Params(W, H, cells=(8,), eps=0.05)
    mh, mi = O.empty_models(P)
    mh[0] = Hm.reshape(9) / np.linalg.norm(Hm)
    mi[0, O.MI_VALID] = 1
    n = W * H
    ys, xs = np.divmod(np.arange(n), W)
    hole = (xs >= 6) & (xs < 16) & (ys >= 5) & (ys < 15)
    acc = O.Labels(np.where(hole, -1, 0).astype(np.int32), np.full(n, 0.001), np.full(n, 2.0), np.full(n, 1.0))
    cue = np.zeros(n, np.uint8)
    cue[(xs == 10) & (ys == 10)] = O.CUE_M2O
    # city-block distance from the assigned region
    dist = np.minimum.reduce([xs - 5, 16 - xs, ys - 4, 15 - ys])
    for k in (1, 2, 3):
        a = acc.copy()
        P.fill_iters = k
        O.fill(P, f1, f2, mh, mi, cue, a)
        want = ~hole | (dist <= k)
        want[(xs == 10) & (ys == 10)] = False
        np.testing.assert_array_equal(a.m >= 0, want)
        np.testing.assert_allclose(a.fx[hole & want], 2.0, atol=1e-12)


# ---------------------------------------------------------------- whole method on known scenes
def _evaluate(s, R):
    H, W = s.occ.shape
    f = R.flow[0].reshape(H, W, 2)
    occ = R.occ[0].reshape(H, W)
    epe = np.hypot(*(f - s.flow).transpose(2, 0, 1))
    tp = ((occ == 1) & (s.occ == 1)).sum()
    return dict(epe_nocc=float(epe[s.occ == 0].mean()), assigned=float((R.acc[0].m >= 0).mean()),
                prec=tp / max(occ.sum(), 1), rec=tp / max(s.occ.sum(), 1))


def test_translating_layer_scene_occlusion_and_flow():
    """Static background, one textured layer translated by an integer vector:
    the plane flow is exact on non-occluded pixels and the occluded strip is found."""
    W, H = 96, 72
    key = 999
    ys, xs = np.mgrid[0:H, 0:W].astype(float)
    tex = lambda k, x, y: np.stack([0.2 + 0.6 * scene.value_noise(x, y, k + 31 * c, period=12.0) for c in range(3)], -1)
    rect = lambda x, y: (x >= 30) & (x < 62) & (y >= 20) & (y < 52)
    t = 6
    f1 = np.where(rect(xs, ys)[..., None], tex(key, xs, ys), tex(key + 1, xs, ys))
    f2 = np.where(rect(xs - t, ys)[..., None], tex(key, xs - t, ys), tex(key + 1, xs, ys))
    gt = np.zeros((H, W, 2))
    gt[rect(xs, ys), 0] = t
    occ_gt = (~rect(xs, ys)) & rect(xs - t, ys)   # background covered in frame 2
    s = scene.Scene(frame1=f1.astype(np.float32), frame2=f2.astype(np.float32), flow=gt.astype(np.float32),
                    occ=occ_gt.astype(np.uint8), layer_id=rect(xs, ys).astype(np.int16))
    # accuracy of the method, not of one random stream: eight Philox keys, bounds on the mean (measured: EPE
    # 0.035 px, recall 0.97, precision 0.93) and a floor for each stream (the worst: recall 0.86)
    ms = []
    for seed in range(8):
        P = O.Params(W, H, patch_radius=3, cells=(32, 16, 8), gain_normalize=0, seed=seed)
        ms.append(_evaluate(s, O.run(P, s.frame1, s.frame2)))
    mean = {k: float(np.mean([m[k] for m in ms])) for k in ms[0]}
    assert mean["epe_nocc"] < 0.05 and all(m["epe_nocc"] < 0.1 for m in ms), ms
    assert mean["rec"] > 0.9 and all(m["rec"] > 0.8 for m in ms), ms
    assert mean["prec"] > 0.8 and all(m["prec"] > 0.6 for m in ms), ms


@pytest.mark.parametrize("seed", [0, 1])
def test_tiny_config_accuracy_against_ground_truth(seed):
    """128x96 scenes (2 layers, affine motion up to 8 px), r=3, cells 32/16/8,
    4 iterations, 256 hypotheses.  Accuracy bounds recorded from the first
    runs with margin: planes cover most pixels, EPE on visible pixels stays
    at the integer-NNF fitting limit."""
    s = scene.tiny_scene(seed)
    P = O.Params(128, 96)
    R = O.run(P, s.frame1, s.frame2)
    m = _evaluate(s, R)
    assert m["assigned"] > 0.9, m
    assert m["epe_nocc"] < 0.6, m
    if s.occ.mean() > 0.05:
        assert m["rec"] > 0.5, m


def _pipeline_level1(seed=0):
    """The tiny configuration run through level 1 of Algorithm 1 (the level's restricted PatchMatch included)."""
    s = scene.tiny_scene(seed)
    P = O.Params(128, 96, seed=seed)
    return P, O.run(P, s.frame1, s.frame2, stop_after=1)


@pytest.mark.parametrize("seed", [0, 1])
def test_pipeline_discards_every_stage_one_plane_that_fails_a_cue(seed):
    """Sec. 3.4 in the pipeline: after level 1, no first-stage model whose symmetric fraction is below eta or
    whose RANSAC / colour overlap is below kappa is still valid, and some models were judged (the scene has
    occlusions, so the rule is exercised)."""
    P, R = _pipeline_level1(seed)
    cb = O.cell_base(P)
    judged = failed = 0
    for d in range(2):
        for c in range(int(cb[0]), int(cb[1])):
            f = R.mi[d][2 * c]
            if not (f[O.MI_FLAGS] & O.F_FITTED):
                continue
            fails = (f[O.MI_NASSIGN] > 0 and f[O.MI_NSYM] < P.eta * f[O.MI_NASSIGN]) or \
                f[O.MI_NRC] < P.kappa * f[O.MI_COUNT]
            judged += 1
            failed += bool(fails)
            if fails:
                assert f[O.MI_VALID] == 0, (d, c, f.tolist())
    assert judged > 20 and failed > 0, (judged, failed)


@pytest.mark.parametrize("seed", [0, 1])
def test_pipeline_residual_stage_fits_the_pixels_stage_one_left(seed):
    """Sec. 3.2 in the pipeline: at level 1 each window's second-stage fit takes exactly the window's pixels
    that the first stage left without a plane (its RANSAC input size), in both directions."""
    P, R = _pipeline_level1(seed)
    W, H = P.width, P.height
    s = P.cells[0]
    xs, ys = O.grid_axis(W, s), O.grid_axis(H, s)
    cb = O.cell_base(P)
    some = 0
    for d in range(2):
        left = (R.extra["stage1_m"][d] < 0).reshape(H, W)
        assert 0 < left.sum() < W * H
        for cy, y0 in enumerate(ys):
            for cx, x0 in enumerate(xs):
                c = int(cb[0]) + cy * len(xs) + cx
                want = int(left[y0:y0 + s, x0:x0 + s].sum())
                assert R.mi[d][2 * c + 1][O.MI_NIN] == want, (d, cx, cy, want, R.mi[d][2 * c + 1].tolist())
                some += 0 < want < s * s
    assert some > 0


def test_pipeline_freezes_assigned_pixels_and_fills_from_neighbours():
    """Algorithm 1 as run end to end: after each level a pixel with a plane holds the rounded plane flow in its
    NNF (Sec. 3.3.1) and keeps it through that level's restricted PatchMatch (Sec. 3.3.2); the final
    model-propagation fill (Sec. 3.4.1) keeps every plane assigned before it, gives new planes only to pixels
    within fill_iters 4-neighbour steps of one, each one of the planes held before the fill, and does fill some."""
    s = scene.make_scene(96, 72, seed=6, n_layers=3, max_disp=6.0, affine=True)
    P = O.Params(96, 72, patch_radius=2, cells=(32, 16), pm_iters=3, num_hyp=128, fill_iters=3)
    W, H, n = 96, 72, 96 * 72
    for stop in (1, 2):
        R = O.run(P, s.frame1, s.frame2, stop_after=stop)
        for d in range(2):
            a = R.acc[d]
            on = a.m >= 0
            assert on.mean() > 0.3
            np.testing.assert_array_equal(R.vx[d][on], np.floor(a.fx[on] + 0.5).astype(np.int32))
            np.testing.assert_array_equal(R.vy[d][on], np.floor(a.fy[on] + 0.5).astype(np.int32))
    pre = O.run(P, s.frame1, s.frame2, stop_after=2)
    post = O.run(P, s.frame1, s.frame2)
    filled_any = False
    for d in range(2):
        before, after = pre.acc[d].m, post.acc[d].m
        np.testing.assert_array_equal(after[before >= 0], before[before >= 0])
        new = (before < 0) & (after >= 0)
        filled_any |= bool(new.any())
        near = (before >= 0).reshape(H, W)
        for _ in range(P.fill_iters):
            g = near.copy()
            g[1:] |= near[:-1]
            g[:-1] |= near[1:]
            g[:, 1:] |= near[:, :-1]
            g[:, :-1] |= near[:, 1:]
            near = g
        assert not (new & ~near.reshape(-1)).any()
        assert np.isin(after[new], before[before >= 0]).all()
    assert filled_any


def test_run_is_deterministic():
    s = scene.make_scene(64, 48, seed=4, n_layers=2, max_disp=5.0)
    P = O.Params(64, 48, patch_radius=2, cells=(16, 8), num_hyp=64, pm_iters=2)
    a = O.run(P, s.frame1, s.frame2)
    b = O.run(P, s.frame1, s.frame2)
    for d in range(2):
        np.testing.assert_array_equal(a.flow[d], b.flow[d])
        np.testing.assert_array_equal(a.mi[d], b.mi[d])


def test_fit_cells_equals_fit_level_on_its_windows():
    """The per-window fit used by the full-size GPU checks is the whole-level fit restricted to the listed
    windows, for both stages (stage 2 on a residual mask), and leaves every other model slot untouched."""
    s = scene.make_scene(64, 48, seed=5, n_layers=2, max_disp=5.0, affine=True)
    P = O.Params(64, 48, patch_radius=2, cells=(16, 8), pm_iters=2, num_hyp=64)
    R = O.run(P, s.frame1, s.frame2, stop_after=0)
    a = np.asarray(s.frame1, np.float64)
    b = np.asarray(s.frame2, np.float64) * O.gain(P, a, s.frame2)
    rng = np.random.default_rng(0)
    resid = (rng.random(64 * 48) < 0.4).astype(np.uint8)
    cb = O.cell_base(P)
    for level in (1, 2):
        count = int(cb[level] - cb[level - 1])
        cells = sorted(rng.choice(count, 5, replace=False).tolist())
        for stage, mask in ((1, None), (2, resid)):
            mh, mi = O.empty_models(P)
            O.fit_level(P, a, b, 0, level, stage, R.vx[0], R.vy[0], mask, mh, mi)
            mh2, mi2 = O.empty_models(P)
            O.fit_cells(P, a, b, 0, level, stage, R.vx[0], R.vy[0], mask, cells, mh2, mi2)
            ids = (int(cb[level - 1]) + np.asarray(cells)) * 2 + stage - 1
            np.testing.assert_array_equal(mh2[ids], mh[ids])
            np.testing.assert_array_equal(mi2[ids], mi[ids])
            others = np.setdiff1d(np.arange(len(mi2)), ids)
            assert not mi2[others].any() and not mh2[others].any()


def test_fill_takes_the_lowest_model_id_among_equal_neighbours():
    """Sec. 3.4.1 with reading R24: a pixel without a plane takes, from its 4-neighbours, the plane with the lowest
    colour error below eps, the lowest model id among errors within 1e-6. On identical constant frames every
    identity plane has error 0: the hole between models 5 (left) and 3 (right) takes 3; a neighbour whose plane
    maps the pixel outside the frame offers nothing, though its id (1) is lower and the clamped sample matches."""
    W, H = 5, 1
    P = O.Params(W, H, cells=(2,), fill_iters=1, eps=0.05)
    f = np.full((H, W, 3), 0.5)
    n = W
    mh = np.zeros((8, 9))
    for m in (3, 5):
        mh[m] = np.eye(3).reshape(9)
    mh[1] = np.array([1, 0, 9.0, 0, 1, 0, 0, 0, 1])               # moves every pixel 9 px right, out of the frame
    mi = np.zeros((8, O.MI), np.int32)
    acc = O.Labels.empty(n, P.eps)
    acc.m[:] = [5, -1, 3, -1, 1]
    cue = np.zeros(n, np.uint8)
    O.fill(P, f, f, mh, mi, cue, acc)
    assert list(acc.m) == [5, 3, 3, 3, 1]                            # pixel 3: model 3 from the left, not 1
    assert acc.L[1] == 0 and acc.L[3] == 0


def test_fill_and_final_log_their_near_ties():
    """The near-tie logs of the fill and of the final map (Sec. 3.4.1): a choice whose colour error lies within
    the band of eps (1e-5 relative, 2e-6 absolute) is marked; a pixel that looked at a marked neighbour is marked;
    a clear choice is not.  In the final map an occlusion decision within the band of occ_thresh, or a target
    within the band of the frame edge, is marked.  Dyadic colours make every error exact."""
    W, H = 7, 1
    P = O.Params(W, H, cells=(2,), fill_iters=1, eps=0.25)
    src = np.full((H, W, 3), 0.5)
    tgt = src.copy()
    tgt[0, 1] += 0.25 - 2.0 ** -22                  # pixel 1: error just below eps
    mh = np.zeros((8, 9))
    for m in (3, 4, 5):
        mh[m] = np.eye(3).reshape(9)
    mi = np.zeros((8, O.MI), np.int32)
    acc = O.Labels.empty(W, P.eps)
    acc.m[:] = [5, -1, -1, 3, -1, -1, 4]
    cue = np.zeros(W, np.uint8)
    amb = np.zeros(W, np.uint8)
    amb[6] = 1                                       # pixel 6's own label rests on a near tie upstream
    O.fill(P, src, tgt, mh, mi, cue, acc, amb)
    assert list(acc.m) == [5, 5, 3, 3, 3, 4, 4]
    assert list(amb) == [0, 1, 0, 0, 0, 1, 1]
    W = 4
    P = O.Params(W, H, cells=(2,), occ_thresh=0.25)
    src = np.full((H, W, 3), 0.5)
    tgt = src.copy()
    tgt[0, 0] += 0.25 - 2.0 ** -22                  # pixel 0: warp error just below the threshold
    tgt[0, 1] += 0.125                               # pixel 1: clearly below
    acc = O.Labels.empty(W, P.eps)
    acc.m[:] = [3, 3, -1, 3]
    acc.fx[3] = 1e-3                                 # pixel 3 lands on the edge of the 1e-3 px frame tolerance
    amb = np.zeros(W, np.uint8)
    vx = np.zeros(W, np.int32)
    flow, occ = O.final(P, src, tgt, acc, vx, vx.copy(), np.zeros(W, np.uint8), amb)
    assert list(occ) == [0, 0, 1, 0]
    assert list(amb) == [1, 0, 0, 1]


def test_final_map_flow_source_and_occlusion_rule_on_hand_built_state():
    """Sec. 3.4.1 and readings R20/R23: the flow is the plane's where a pixel has one, else its NNF offset; a pixel
    is occluded without a plane, under the many-to-one cue, outside the frame (beyond 1e-3 px) or where the warp
    error is not below the threshold. Dyadic colours make every warp error exact, so the threshold is hit exactly."""
    W, H = 8, 2
    P = O.Params(W, H, cells=(2,), occ_thresh=0.25)
    rng = np.random.default_rng(3)
    src = rng.integers(0, 5, (H, W, 3)) / 8.0
    tgt = rng.integers(0, 5, (H, W, 3)) / 8.0
    tgt[0, 2:] = src[0, :W - 2]                     # row 0 of the target: row 0 of the source moved 2 px right
    tgt[0, 5] = src[0, 3] + 0.125                   # warp error of x=3 below the threshold
    tgt[0, 6] = src[0, 4] + 0.25                    # warp error of x=4 exactly at it
    src[0, 7] = (tgt[0, 6] + tgt[0, 7]) / 2         # x=7 lands half-way between target pixels 6 and 7
    src[1, 0], src[1, 1] = tgt[0, 0], tgt[0, 1]     # row 1 pixels 0 and 1 map one row up
    n = W * H
    acc = O.Labels.empty(n, P.eps)
    vx, vy = np.full(n, 2, np.int32), np.full(n, -3, np.int32)
    cue = np.zeros(n, np.uint8)
    for x, fx in ((0, 2.0), (2, 2.0), (3, 2.0), (4, 2.0), (5, 2.0), (6, 2.0), (7, -0.5)):
        acc.m[x], acc.fx[x] = 3, fx
    cue[2] = O.CUE_M2O
    for x, fy in ((0, -1.0), (1, -1.0005), (2, -1.002)):
        acc.m[W + x], acc.fy[W + x] = 5, fy
    flow, occ = O.final(P, src, tgt, acc, vx, vy, cue)
    exp_occ = [0, 1, 1, 0, 1, 0, 1, 0,             # row 0: no plane at 1, cue at 2, at threshold 4, outside 6
               0, 0, 1, 1, 1, 1, 1, 1]             # row 1: 1 px beyond the top is inside the tolerance, 2e-3 is not
    assert list(occ) == exp_occ
    exp_fx = [2, 2, 2, 2, 2, 2, 2, -0.5] + [0, 0, 0, 2, 2, 2, 2, 2]
    exp_fy = [0, -3, 0, 0, 0, 0, 0, 0] + [-1.0, -1.0005, -1.002, -3, -3, -3, -3, -3]
    np.testing.assert_array_equal(flow[:, 0], np.float32(exp_fx))
    np.testing.assert_array_equal(flow[:, 1], np.float32(exp_fy))


def test_edge_aware_fill_evaluates_the_seed_plane_at_the_pixel():
    """Reading R28: a pixel without a plane takes its seed's plane evaluated at its own position, or the seed's
    flow where that plane's denominator is not positive; pixels with a plane or without a seed keep their flow.
    The projective plane w = 1 - x/4 maps (x, y) to (x, y) / w, so its flows are known in closed form."""
    W, H = 6, 2
    P = O.Params(W, H, cells=(2,))
    mh, _ = O.empty_models(P)
    mh[0] = 3.0 * np.array([1, 0, 2, 0, 1, -1, 0, 0, 1.0])      # translation by (2, -1), homogeneous scale 3
    mh[1] = np.array([1, 0, 0, 0, 1, 0, -0.25, 0, 1.0])
    n = W * H
    acc = O.Labels.empty(n, P.eps)
    acc.m[0], acc.fx[0] = 0, 7.0
    acc.m[W + 5], acc.fx[W + 5], acc.fy[W + 5] = 1, 9.5, -3.25
    seed = np.full(n, -1, np.int32)
    seed[1:5] = 0
    seed[W:W + 5] = W + 5
    flow = (100 + np.arange(2 * n, dtype=np.float32)).reshape(n, 2)
    before = flow.copy()
    O.interp_flow(P, mh, acc, seed, flow)
    np.testing.assert_array_equal(flow[1:5], np.float32([[2, -1]] * 4))
    for i in (0, 5, W + 5):                                      # a plane of its own, or no seed
        np.testing.assert_array_equal(flow[i], before[i])
    exp = np.float32([[0, 0], [1 / 3, 1 / 3], [2, 1], [9, 3], [9.5, -3.25]])   # x = 0..4 of row 1; w = 0 at x = 4
    np.testing.assert_allclose(flow[W:W + 5], exp, rtol=0, atol=1e-7)


def test_assignment_rules_on_hand_built_windows():
    """Eq. 3-4 with readings R23/R24 on three 4 px windows (x = 0-3, 2-5, 4-7) over an 8x4 frame pair: the source
    is black and the target grey, so a translation's colour error at p is the target's grey level at the mapped
    pixel, exact in dyadic values. A pixel takes, over its covering windows in order, the valid plane that maps
    it into the frame with a positive denominator and an error below eps; a later window displaces the current
    one only if its error is lower by more than 1e-6. The residual stage uses the second model slot of each
    window and only the masked pixels."""
    W, H, eps = 8, 4, 0.5
    P = O.Params(W, H, cells=(4,), eps=eps)
    assert list(O.grid_axis(W, 4)) == [0, 2, 4] and list(O.grid_axis(H, 4)) == [0]
    t = np.full((H, W), 0.75)
    t[0] = [0.25, 0.5, 0.25, 0.25, 0.25 - 2**-21, 0.125, 0.125 - 2**-19, 0.0625]
    t[1, 1] = 0.0
    t[2] = [0.125, 0.25, 0.125, 0.25, 0.0, 0.25, 0.25, 0.25]
    src = np.zeros((H, W, 3))
    tgt = np.repeat(t[:, :, None], 3, axis=2)

    def tr(a):
        return np.array([1, 0, a, 0, 1, 0, 0, 0, 1.0])

    mh, mi = O.empty_models(P)
    mh[0], mh[2], mh[4] = 2 * tr(0), tr(1), tr(2)                  # stage 1 of windows 0, 1, 2 (model ids 0, 2, 4)
    mh[1], mh[3] = tr(1), tr(0)                                    # stage 2 of windows 0, 1
    mh[5] = np.array([0, 0, -1, 0, 0, -1, 0, 0, -1.0])             # maps every pixel to (1, 1), but w = -1
    mi[[0, 1, 2, 4, 5], O.MI_VALID] = 1                            # model 3 (window 1, stage 2) is invalid
    n = W * H
    lab = O.Labels.empty(n, eps)
    amb = np.zeros(n, np.uint8)
    O.assign(P, src, tgt, 1, 1, mh, mi, None, lab, amb)
    r0 = slice(0, W)
    # x = 0: only window 0; 1: error equals eps; 2: equal errors, the first window keeps it; 3: lower by 2^-21
    # only; 4: lower by 2^-19; 5: much lower; 6, 7: the +2 translation leaves the frame
    assert list(lab.m[r0]) == [0, -1, 0, 0, 4, 4, -1, -1]
    np.testing.assert_array_equal(lab.L[r0], [0.25, eps, 0.25, 0.25, 0.125 - 2**-19, 0.0625, eps, eps])
    np.testing.assert_array_equal(lab.fx[r0], [0, 0, 0, 0, 2, 2, 0, 0])
    assert not lab.fy.any()
    assert list(amb[r0]) == [0, 1, 1, 1, 1, 0, 0, 0]                 # the ties and the eps boundary are logged
    assert list(lab.m[W:2 * W]) == [-1, 0, -1, -1, -1, -1, -1, -1]     # row 1: only the black target pixel (1, 1)
    assert list(lab.m[2 * W:3 * W]) == [0, 0, 0, 2, 2, 2, -1, -1]      # row 2: x = 3 lower later, x = 4 a tie
    assert (lab.m[3 * W:] == -1).all()
    # residual stage on row 2 only; the other rows keep what they held
    lab2 = O.Labels(np.full(n, 77, np.int32), np.full(n, 9.0), np.full(n, 5.0), np.full(n, 6.0))
    mask = np.zeros(n, np.uint8)
    mask[2 * W:3 * W] = 1
    O.assign(P, src, tgt, 1, 2, mh, mi, mask, lab2)
    r2 = slice(2 * W, 3 * W)
    # x = 2 would prefer the invalid identity of window 1; x = 4..7 would map to the black pixel (1, 1) if the
    # negative denominator were ignored
    assert list(lab2.m[r2]) == [1, 1, 1, 1, -1, -1, -1, -1]
    np.testing.assert_array_equal(lab2.L[r2], [0.25, 0.125, 0.25, 0.0, eps, eps, eps, eps])
    np.testing.assert_array_equal(lab2.fx[r2], [1, 1, 1, 1, 0, 0, 0, 0])
    keep = mask == 0
    assert (lab2.m[keep] == 77).all() and (lab2.L[keep] == 9).all() and (lab2.fx[keep] == 5).all()
