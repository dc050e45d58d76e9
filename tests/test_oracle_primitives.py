"""Pins of the FP64 oracle's primitives against facts fixed outside the oracle.

Each test names what it pins and against what: published known-answer
vectors, closed forms (bilinear interpolation reproduces affine functions),
independent brute force, and exact recovery of generating homographies.
"""
import itertools
import os

import numpy as np
import pytest

import oracle as O
from paper_1804_03787_gb300 import scene

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox
def test_philox_known_answers():
    """Philox4x32-10 reproduces the Random123 known-answer vectors."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


# ---------------------------------------------------------------- window grid
def _grid_closed_form(n, s):
    """Positions 0, s/2, ... with pos + s <= n, then n - s if not yet flush."""
    h = s // 2
    k = (n - s) // h + 1
    extra = 1 if (k - 1) * h + s < n else 0
    return k + extra


@pytest.mark.parametrize("n,s", [(128, 32), (96, 32), (128, 8), (96, 16), (1024, 64), (436, 64), (436, 8),
                                 (1920, 16), (1080, 64), (64, 64), (65, 64)])
def test_grid_counts_and_overlap(n, s):
    """Sec. 3.1.2: windows overlap their predecessor by half and cover the frame."""
    pos = O.grid_axis(n, s)
    assert len(pos) == _grid_closed_form(n, s)
    assert pos[0] == 0 and pos[-1] + s == n
    d = np.diff(pos)
    if len(d):
        assert np.all(d[:-1] == s // 2) and 0 < d[-1] <= s // 2
    cover = np.zeros(n, int)
    for p in pos:
        cover[p:p + s] += 1
    assert cover.min() >= 1 and cover.max() <= 3


def test_cell_totals_of_the_two_workloads():
    """Cell counts: 128x96 with cells 32/16/8 -> 35+165+713; 1024x436 with 64/32/16/8 -> 36,502."""
    P = O.Params(128, 96, cells=(32, 16, 8))
    assert list(O.cell_base(P)) == [0, 35, 200, 913]
    P = O.Params(1024, 436, cells=(64, 32, 16, 8))
    cb = O.cell_base(P)
    assert list(np.diff(cb)) == [403, 1701, 6858, 27540] and cb[-1] == 36502


# ---------------------------------------------------------------- bilinear sampling
def test_bilinear_reproduces_affine_ramp():
    """Bilinear interpolation is exact for affine images: I(x,y) = a x + b y + e."""
    H, W = 9, 13
    ys, xs = np.mgrid[0:H, 0:W].astype(float)
    a, b, e = np.array([0.03, -0.01, 0.02]), np.array([0.015, 0.02, -0.005]), np.array([0.2, 0.5, 0.4])
    img = xs[..., None] * a + ys[..., None] * b + e
    rng = np.random.default_rng(0)
    for _ in range(50):
        X, Y = rng.uniform(0, W - 1), rng.uniform(0, H - 1)
        np.testing.assert_allclose(O.sample_bilinear(img, X, Y), a * X + b * Y + e, rtol=0, atol=1e-14)


def test_bilinear_integer_points_and_clamping():
    rng = np.random.default_rng(1)
    img = rng.random((7, 5, 3))
    for y in range(7):
        for x in range(5):
            np.testing.assert_array_equal(O.sample_bilinear(img, x, y), img[y, x])
    np.testing.assert_array_equal(O.sample_bilinear(img, -3.2, 2), img[2, 0])
    np.testing.assert_array_equal(O.sample_bilinear(img, 10.0, 100.0), img[6, 4])


# ---------------------------------------------------------------- warped patch cost
def _square_cost(src, tgt, r, px, py, vx, vy):
    """Independent square-patch PatchMatch cost: mean |I1(clamp(p+d)) - I2(clamp(clamp(p+d)+v))|."""
    H, W, _ = src.shape
    acc = 0.0
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            sx, sy = min(max(px + dx, 0), W - 1), min(max(py + dy, 0), H - 1)
            tx, ty = min(max(sx + vx, 0), W - 1), min(max(sy + vy, 0), H - 1)
            acc += np.abs(src[sy, sx] - tgt[ty, tx]).sum()
    return acc / (3 * (2 * r + 1) ** 2)


def test_identity_and_translation_planes_reduce_to_square_patch():
    """An identity (or pure translation) plane gives exactly the square-patch cost."""
    rng = np.random.default_rng(2)
    H, W, r = 20, 24, 3
    src, tgt = rng.random((H, W, 3)), rng.random((H, W, 3))
    P = O.Params(W, H, patch_radius=r)
    T = np.array([[1, 0, 7.25], [0, 1, -3.5], [0, 0, 1.0]])
    for px, py, vx, vy in [(0, 0, 3, 4), (10, 10, -5, 2), (23, 19, -20, -15), (5, 18, 7, -1), (12, 3, 0, 0)]:
        ref = _square_cost(src, tgt, r, px, py, vx, vy)
        assert O.patch_cost(P, src, tgt, px, py, vx, vy) == pytest.approx(ref, rel=1e-14, abs=0)
        assert O.patch_cost(P, src, tgt, px, py, vx, vy, np.eye(3)) == pytest.approx(ref, rel=1e-14, abs=0)
        assert O.patch_cost(P, src, tgt, px, py, vx, vy, T) == pytest.approx(ref, rel=1e-12, abs=0)


def test_warped_cost_closed_form_on_projective_ramp():
    """Target frame = affine ramp R, source frame I1(p) = R(G p) for a homography G.

    The patch of p warped by G with integer offset v samples R at
    G(s) + e, e = p + v - G(p) the same for every tap, so the cost is
    mean_c |a_c e_x + b_c e_y| exactly (bilinear reproduces the ramp).
    """
    H, W, r = 40, 48, 3
    a, b, e0 = np.array([0.004, -0.003, 0.002]), np.array([0.002, 0.003, -0.004]), np.array([0.4, 0.5, 0.6])
    ys, xs = np.mgrid[0:H, 0:W].astype(float)
    tgt = xs[..., None] * a + ys[..., None] * b + e0
    G = np.array([[1.05, 0.03, 2.3], [-0.02, 0.97, 1.7], [4e-4, -3e-4, 1.0]])
    w = G[2, 0] * xs + G[2, 1] * ys + G[2, 2]
    gx, gy = (G[0, 0] * xs + G[0, 1] * ys + G[0, 2]) / w, (G[1, 0] * xs + G[1, 1] * ys + G[1, 2]) / w
    src = gx[..., None] * a + gy[..., None] * b + e0
    P = O.Params(W, H, patch_radius=r)
    for px, py in [(10, 10), (20, 15), (30, 25), (12, 28)]:
        wp = G[2, 0] * px + G[2, 1] * py + G[2, 2]
        Gx, Gy = (G[0, 0] * px + G[0, 1] * py + G[0, 2]) / wp, (G[1, 0] * px + G[1, 1] * py + G[1, 2]) / wp
        for vx, vy in [(round(Gx - px), round(Gy - py)), (round(Gx - px) + 1, round(Gy - py) - 2)]:
            ex, ey = px + vx - Gx, py + vy - Gy
            want = np.abs(a * ex + b * ey).mean()
            got = O.patch_cost(P, src, tgt, px, py, vx, vy, G)
            assert got == pytest.approx(want, rel=1e-9, abs=1e-15)


# ---------------------------------------------------------------- homography solvers
def _norm(H):
    H = np.asarray(H, float)
    return H / np.linalg.norm(H) * np.sign(H[2, 2])


def _rand_h(rng):
    src = np.array([[0, 0], [40, 0], [40, 40], [0, 40]], float)
    dst = src + rng.uniform(-8, 8, size=(4, 2))
    from paper_1804_03787_gb300.scene import h_from_points
    return h_from_points(src, dst)


def _apply(H, p):
    w = H[2, 0] * p[:, 0] + H[2, 1] * p[:, 1] + H[2, 2]
    return np.stack([(H[0, 0] * p[:, 0] + H[0, 1] * p[:, 1] + H[0, 2]) / w,
                     (H[1, 0] * p[:, 0] + H[1, 1] * p[:, 1] + H[1, 2]) / w], 1)


def test_minimal_and_refit_recover_generating_homography():
    """Noise-free real-valued correspondences give back the generating H to 1e-9."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        Hg = _rand_h(rng)
        p = rng.uniform(0, 40, size=(50, 2))
        q = _apply(Hg, p)
        np.testing.assert_allclose(_norm(O.h_minimal(p[:4], q[:4])), _norm(Hg), atol=1e-9)
        np.testing.assert_allclose(_norm(O.h_dlt(p, q)), _norm(Hg), atol=1e-9)


def test_minimal_solver_rejects_collinear_sample():
    p = np.array([[0, 0], [1, 1], [2, 2], [5, 0]], float)
    assert O.h_minimal(p, p + 1) is None


def test_exact_centre_denominator_test_against_fp64_solver():
    """The exact test that a sample's homography has a zero denominator at the window centre, against the
    FP64 minimal solver (pinned above): samples built from an integer H whose third row vanishes at the centre
    are caught; a 1 px change of one target and random samples are not, and for those the solver's
    denominator at the centre is far from zero."""
    rng = np.random.default_rng(11)
    for s in (8, 16, 64, 96):
        for _ in range(40):
            x0, y0 = int(rng.integers(0, 900)), int(rng.integers(0, 300))
            cx2, cy2 = 2 * x0 + s - 1, 2 * y0 + s - 1          # twice the centre
            # third row (2, 0, -cx2) or (0, 2, -cy2): the denominator is 2x - cx2 (odd, +-1 next to the centre)
            use_x = bool(rng.integers(0, 2))
            row3 = np.array([2, 0, -cx2]) if use_x else np.array([0, 2, -cy2])
            Hi = np.vstack([rng.integers(-3, 4, size=(2, 3)), row3]).astype(float)
            # two source points on each line next to the centre: denominator -1 or +1, integer targets
            a, b = (cx2 - 1) // 2, (cx2 + 1) // 2
            c, e = (cy2 - 1) // 2, (cy2 + 1) // 2
            ys = rng.choice(np.arange(y0, y0 + s), 2, replace=False)
            xs = rng.choice(np.arange(x0, x0 + s), 2, replace=False)
            src = (np.array([[a, ys[0]], [a, ys[1]], [b, ys[0]], [b, ys[1]]]) if use_x
                   else np.array([[xs[0], c], [xs[1], c], [xs[0], e], [xs[1], e]]))
            dst = np.rint(_apply(Hi, src.astype(float))).astype(int)
            np.testing.assert_allclose(_apply(Hi, src.astype(float)), dst, atol=1e-9)
            Hm = O.h_minimal(src.astype(float), dst.astype(float))
            if Hm is None:  # three target points on a line: not a hypothesis at all
                continue
            Hm = np.asarray(Hm, float).reshape(3, 3)
            den_c = (Hm[2, 0] * cx2 + Hm[2, 1] * cy2 + 2 * Hm[2, 2]) / 2
            assert abs(den_c) < 1e-9 * np.abs(Hm[2]).sum() * (abs(cx2) + abs(cy2) + 2)
            assert O.den_zero_at_centre(src, dst, x0, y0, s)
            d2 = dst.copy()
            d2[3, 0] += 1
            H2 = O.h_minimal(src.astype(float), d2.astype(float))
            if H2 is not None:
                H2 = np.asarray(H2, float).reshape(3, 3)
                if abs(H2[2, 0] * cx2 + H2[2, 1] * cy2 + 2 * H2[2, 2]) > 1e-6 * np.abs(H2[2]).sum():
                    assert not O.den_zero_at_centre(src, d2, x0, y0, s)
    for _ in range(300):
        s = 64
        x0, y0 = int(rng.integers(0, 900)), int(rng.integers(0, 300))
        src = np.stack([rng.integers(x0, x0 + s, 4), rng.integers(y0, y0 + s, 4)], 1)
        dst = src + rng.integers(-60, 61, size=(4, 2))
        Hm = O.h_minimal(src.astype(float), dst.astype(float))
        if Hm is None:
            continue
        Hm = np.asarray(Hm, float).reshape(3, 3)
        den_c = Hm[2, 0] * (x0 + (s - 1) / 2) + Hm[2, 1] * (y0 + (s - 1) / 2) + Hm[2, 2]
        if abs(den_c) > 1e-9 * np.abs(Hm[2]).sum() * 1000:
            assert not O.den_zero_at_centre(src, dst, x0, y0, s)


def test_dlt_is_least_squares_optimal_under_noise():
    """With noise, the refit has smaller algebraic residual than the generating H
    (it minimises ||A h|| over unit h in normalised coordinates)."""
    rng = np.random.default_rng(4)
    Hg = _rand_h(rng)
    p = rng.uniform(0, 40, size=(200, 2))
    q = _apply(Hg, p) + rng.normal(0, 0.3, size=(200, 2))
    Hd = O.h_dlt(p, q)
    err_d = np.linalg.norm(_apply(Hd, p) - q, axis=1).mean()
    err_g = np.linalg.norm(_apply(Hg, p) - q, axis=1).mean()
    assert err_d <= err_g * 1.01
    assert np.abs(_apply(Hd, p) - _apply(Hg, p)).max() < 0.3


def test_normalised_dlt_is_similarity_covariant():
    """Hartley & Zisserman's argument for normalising (Sec. 3.1.2 fits planes by the normalised DLT): with both
    point sets centred and scaled to a fixed mean distance, the least-squares homography of noisy matches moves
    with the data under similarities: fitting S p -> S' q gives S' H S^-1 for the H that p -> q gives (up to
    scale). An unnormalised or uncentred DLT does not have this property."""
    rng = np.random.default_rng(12)
    Hg = _rand_h(rng)
    p = rng.uniform(0, 40, size=(60, 2))
    q = _apply(Hg, p) + rng.normal(0, 0.5, size=(60, 2))

    def sim(theta, scale, tx, ty):
        c, s_ = np.cos(theta) * scale, np.sin(theta) * scale
        return np.array([[c, -s_, tx], [s_, c, ty], [0, 0, 1.0]])

    S, Sq = sim(0.5, 3.0, 100.0, -50.0), sim(-1.1, 0.4, -7.0, 220.0)
    H1 = O.h_dlt(p, q)
    H2 = O.h_dlt(_apply(S, p), _apply(Sq, q))
    np.testing.assert_allclose(_norm(H2), _norm(Sq @ H1 @ np.linalg.inv(S)), atol=1e-9)


def _affine_nnf(W, H, A):
    ys, xs = np.divmod(np.arange(W * H), W)
    q = _apply(A, np.stack([xs, ys], 1).astype(float))
    return xs, ys, np.round(q[:, 0] - xs).astype(np.int32), np.round(q[:, 1] - ys).astype(np.int32)


# an integer shear + translation: maps integer pixels to integer pixels
A_INT = np.array([[1, 1, 2], [0, 1, -1], [0, 0, 1]], float)


def test_exhaustive_consensus_matches_brute_force():
    """On a tiny match set, RANSAC with many hypotheses reaches the best
    consensus that brute force over all C(N,4) subsets reaches."""
    rng = np.random.default_rng(5)
    W, H, s = 8, 8, 4
    P = O.Params(W, H, patch_radius=1, cells=(s,), num_hyp=4000, min_inliers=4, ransac_px=1.5)
    xs, ys, vx, vy = _affine_nnf(W, H, A_INT)
    win = (xs < s) & (ys < s)
    out = np.flatnonzero(win)[rng.permutation(s * s)[:6]]
    vx[out] += (rng.integers(3, 6, size=6) * rng.choice([-1, 1], size=6)).astype(np.int32)
    vy[out] += (rng.integers(3, 6, size=6) * rng.choice([-1, 1], size=6)).astype(np.int32)
    mh, mi = O.empty_models(P)
    frame = np.zeros((H, W, 3))
    O.fit_level(P, frame, frame, 0, 1, 1, vx, vy, None, mh, mi)
    idx = np.flatnonzero(win)
    ps = np.stack([xs[idx], ys[idx]], 1).astype(float)
    qs = ps + np.stack([vx[idx], vy[idx]], 1)
    best = 0
    for comb in itertools.combinations(range(len(idx)), 4):
        Hc = O.h_minimal(ps[list(comb)], qs[list(comb)])
        if Hc is None:
            continue
        # orientation: denominator positive at the window centre
        c = (s - 1) / 2.0
        Hc = Hc * np.sign(Hc[2, 0] * c + Hc[2, 1] * c + Hc[2, 2])
        with np.errstate(all="ignore"):
            w = Hc[2, 0] * ps[:, 0] + Hc[2, 1] * ps[:, 1] + Hc[2, 2]
            r2 = ((_apply(Hc, ps) - qs) ** 2).sum(1)
        best = max(best, int(((r2 < 2.25) & (w > 0)).sum()))
    assert best >= 10
    assert mi[0, O.MI_BESTSCORE] == best and mi[0, O.MI_NIN] == 16


def test_ransac_ties_keep_the_lowest_hypothesis():
    """Reading R21: with every match an exact inlier of one integer map, every non-degenerate hypothesis scores
    all 64 matches. Hypothesis k draws the same sample whatever the count K (its counter is k), so the fit with
    K = 1 shows hypothesis 0 is such a one; with K = 512 the tie must still go to hypothesis 0."""
    s = 8
    P1 = O.Params(s, s, patch_radius=1, cells=(s,), num_hyp=1)
    Pk = O.Params(s, s, patch_radius=1, cells=(s,), num_hyp=512)
    _, _, vx, vy = _affine_nnf(s, s, A_INT)
    frame = np.zeros((s, s, 3))
    for P, n_hyp in ((P1, 1), (Pk, 512)):
        mh, mi = O.empty_models(P)
        O.fit_level(P, frame, frame, 0, 1, 1, vx, vy, None, mh, mi)
        assert mi[0, O.MI_BESTK] == 0 and mi[0, O.MI_BESTSCORE] == 64, (n_hyp, mi[0])


def test_residual_stage_fits_only_the_masked_matches():
    """Sec. 3.2: the second stage fits a window's unassigned pixels only. Here the masked pixels (about 40 %)
    follow an integer shear and the others a plain shift; stage 1 finds the majority's shift, stage 2 the
    shear, on exactly the masked matches."""
    s = 8
    rng = np.random.default_rng(13)
    xs, ys, vx, vy = _affine_nnf(s, s, A_INT)
    mask = (rng.random(s * s) < 0.4).astype(np.uint8)
    vx[mask == 0], vy[mask == 0] = -4, 3       # at least 4 px from the shear's offset (y + 2, -1) everywhere
    P = O.Params(s, s, patch_radius=1, cells=(s,), num_hyp=512)
    frame = np.zeros((s, s, 3))
    mh, mi = O.empty_models(P)
    O.fit_level(P, frame, frame, 0, 1, 1, vx, vy, None, mh, mi)
    O.fit_level(P, frame, frame, 0, 1, 2, vx, vy, mask, mh, mi)
    shift = np.array([[1, 0, -4], [0, 1, 3], [0, 0, 1.0]])
    assert mi[0, O.MI_NIN] == 64 and mi[0, O.MI_COUNT] == 64 - int(mask.sum())
    np.testing.assert_allclose(_norm(mh[0].reshape(3, 3)), _norm(shift), atol=1e-9)
    assert mi[1, O.MI_NIN] == int(mask.sum()) and mi[1, O.MI_COUNT] == int(mask.sum())
    np.testing.assert_allclose(_norm(mh[1].reshape(3, 3)), _norm(A_INT), atol=1e-9)


def test_ransac_recovers_integer_affine_with_outliers():
    """30 % gross outliers: the refit on the consensus set is the generating map to 1e-9."""
    rng = np.random.default_rng(6)
    W, H, s = 32, 32, 16
    P = O.Params(W, H, patch_radius=1, cells=(s,), num_hyp=256)
    xs, ys, vx, vy = _affine_nnf(W, H, A_INT)
    win = (xs < s) & (ys < s)
    out = np.flatnonzero(win)[rng.permutation(s * s)[:77]]
    vx[out] += (rng.integers(4, 9, size=77) * rng.choice([-1, 1], size=77)).astype(np.int32)
    vy[out] += (rng.integers(4, 9, size=77) * rng.choice([-1, 1], size=77)).astype(np.int32)
    mh, mi = O.empty_models(P)
    frame = np.zeros((H, W, 3))
    O.fit_level(P, frame, frame, 0, 1, 1, vx, vy, None, mh, mi)
    assert mi[0, O.MI_COUNT] == 256 - 77 and mi[0, O.MI_NIN] == 256 and mi[0, O.MI_VALID] == 1
    assert mi[0, O.MI_FLAGS] & O.F_REFIT
    np.testing.assert_allclose(_norm(mh[0].reshape(3, 3)), _norm(A_INT), atol=1e-9)


# ---------------------------------------------------------------- HSV histogram equalisation (Sec. 4.2)
def test_hsv_conversion_matches_the_library_routine():
    """The oracle's hexcone conversion against Python's colorsys, both ways, incl. grays, black and primaries."""
    import colorsys
    rng = np.random.default_rng(5)
    cols = [tuple(c) for c in rng.random((300, 3))] + [(0, 0, 0), (1, 1, 1), (0.3, 0.3, 0.3), (1, 0, 0),
                                                        (0, 1, 0), (0, 0, 1), (1, 1, 0), (0, 1, 1), (1, 0, 1)]
    for c in cols:
        h, s, v = O.rgb_to_hsv(*c)
        H, S, V = colorsys.rgb_to_hsv(*c)
        assert abs(h - H) < 1e-12 and abs(s - S) < 1e-12 and abs(v - V) < 1e-12, (c, (h, s, v), (H, S, V))
        np.testing.assert_allclose(O.hsv_to_rgb(h, s, v), colorsys.hsv_to_rgb(H, S, V), atol=1e-12)
        np.testing.assert_allclose(O.hsv_to_rgb(h, s, v), c, atol=1e-12)


def test_v_lut_closed_form():
    """Four V levels in distinct bins with counts 10, 20, 30, 40: cumulative 10, 30, 60, 100, so the
    equalised values are (cdf - 10) / 90 = 0, 2/9, 5/9, 1."""
    levels = [0.1, 0.3, 0.55, 0.8]
    counts = [10, 20, 30, 40]
    px = np.concatenate([np.full((c, 3), v) for v, c in zip(levels, counts)]).reshape(1, 100, 3)
    P = O.Params(100, 1)
    ok, lut = O.v_lut(P, px)
    assert ok
    bins = [int(np.floor(256 * v)) for v in levels]
    np.testing.assert_allclose(lut[bins], [0.0, 2 / 9, 5 / 9, 1.0], atol=1e-15)
    # a frame with one occupied bin is left unchanged
    flat = np.full((4, 5, 3), 0.42)
    ok, _ = O.v_lut(O.Params(5, 4), flat)
    assert not ok
    np.testing.assert_array_equal(O.hsv_equalize(O.Params(5, 4), flat), flat)


def test_hsv_equalize_keeps_hue_and_saturation_and_orders_value():
    """Per pixel: H and S unchanged (colorsys), V replaced by the LUT value of its bin, monotone in V."""
    import colorsys
    rng = np.random.default_rng(8)
    W, H = 23, 17
    img = rng.random((H, W, 3)) ** 2
    img[0, 0] = 0.0
    P = O.Params(W, H)
    out = O.hsv_equalize(P, img)
    ok, lut = O.v_lut(P, img)
    assert ok
    vin, vout = [], []
    for y in range(H):
        for x in range(W):
            hi, si, vi = colorsys.rgb_to_hsv(*img[y, x])
            ho, so, vo = colorsys.rgb_to_hsv(*out[y, x])
            if vi > 0 and si > 0 and vo > 0:
                assert abs(hi - ho) < 1e-9 and abs(si - so) < 1e-9
            assert abs(vo - lut[min(255, int(np.floor(256 * vi)))]) < 1e-12
            vin.append(vi)
            vout.append(vo)
    order = np.argsort(vin, kind="stable")
    assert np.all(np.diff(np.asarray(vout)[order]) >= -1e-12)
    # the equalised values fill [0, 1]: lowest occupied bin -> 0, highest -> 1
    assert min(vout) == 0.0 and abs(max(vout) - 1.0) < 1e-12


def test_pipeline_equalises_both_frames_first():
    """run(equalize=1) on a pair equals run(equalize=0) on the pair equalised beforehand."""
    s = scene.make_scene(40, 32, seed=3, n_layers=1, max_disp=3.0, affine=True)
    P1 = O.Params(40, 32, patch_radius=2, cells=(16, 8), pm_iters=2, num_hyp=32, equalize=1)
    P0 = O.Params(40, 32, patch_radius=2, cells=(16, 8), pm_iters=2, num_hyp=32, equalize=0)
    R1 = O.run(P1, s.frame1, s.frame2)
    R0 = O.run(P0, O.hsv_equalize(P0, s.frame1), O.hsv_equalize(P0, s.frame2))
    np.testing.assert_array_equal(R1.flow[0], R0.flow[0])
    np.testing.assert_array_equal(R1.occ[0], R0.occ[0])


# ---------------------------------------------------------------- census data term (Sec. 6)
def _census_bit(dx, dy):
    """Bit index of the neighbour at (dx, dy) in the 5x5 window, raster order without the centre."""
    k = (dy + 2) * 5 + (dx + 2)
    return k if k < 12 else k - 1


def test_census_closed_forms():
    """Constant frame: every code 0.  One dark pixel in a flat bright frame: its code is 0 and each pixel within
    2 of it has exactly the bit pointing at it.  One bright pixel: its code has all 24 bits, the rest are 0."""
    W, H = 11, 9
    P = O.Params(W, H)
    flat = np.full((H, W, 3), 0.6)
    assert not O.census(P, flat)[..., 0].any()
    dark = flat.copy()
    dark[4, 5] = 0.1
    c = O.census(P, dark)[..., 0].astype(np.int64)
    for y in range(H):
        for x in range(W):
            a, b = 5 - x, 4 - y  # the dark pixel relative to (x, y)
            want = (1 << _census_bit(a, b)) if (max(abs(a), abs(b)) <= 2 and (a, b) != (0, 0)) else 0
            assert c[y, x] == want, (x, y, c[y, x], want)
    bright = flat.copy()
    bright[4, 5] = 0.9
    c = O.census(P, bright)[..., 0].astype(np.int64)
    assert c[4, 5] == (1 << 24) - 1 and np.count_nonzero(c) == 1


def test_census_invariant_under_monotone_grey_changes():
    """Codes compare greys only: a strictly increasing map of a grey frame, or a gain of 2 (exact), keeps them."""
    rng = np.random.default_rng(4)
    W, H = 19, 13
    P = O.Params(W, H)
    t = rng.random((H, W))
    grey = np.repeat(t[..., None], 3, axis=2)
    c0 = O.census(P, grey)
    np.testing.assert_array_equal(O.census(P, grey ** 2), c0)
    np.testing.assert_array_equal(O.census(P, np.sqrt(grey) + 0.25), c0)
    colour = rng.random((H, W, 3))
    np.testing.assert_array_equal(O.census(P, 2.0 * colour), O.census(P, colour))


def test_census_cost_finds_an_integer_shift_exhaustively():
    """Hamming patch cost on code frames: zero at offset 0 against itself, and on a frame against its copy shifted
    by (3, -2) the exhaustive argmin over offsets is that shift at interior pixels."""
    rng = np.random.default_rng(11)
    W, H = 28, 22
    P = O.Params(W, H, patch_radius=2, census=1)
    f1 = rng.random((H, W, 3))
    f2 = np.roll(f1, shift=(-2, 3), axis=(0, 1))  # f2(x + 3, y - 2) = f1(x, y)
    c1, c2 = O.census(P, f1), O.census(P, f2)
    assert O.patch_cost(P, c1, c1, 10, 10, 0, 0) == 0.0
    for (x, y) in [(9, 8), (12, 11), (15, 9)]:
        best = min(((O.patch_cost(P, c1, c2, x, y, vx, vy), (vx, vy))
                    for vy in range(-5, 6) for vx in range(-5, 6)))
        assert best[1] == (3, -2) and best[0] == 0.0


def test_pipeline_census_level0_uses_code_frames():
    """run(census=1) stopped after level 0 equals PatchMatch run directly on the census code frames."""
    s = scene.make_scene(36, 28, seed=6, n_layers=1, max_disp=3.0, affine=True)
    P = O.Params(36, 28, patch_radius=2, cells=(16, 8), pm_iters=2, num_hyp=32, census=1)
    R = O.run(P, s.frame1, s.frame2, stop_after=0)
    c1, c2 = O.census(P, s.frame1), O.census(P, s.frame2)
    n = 36 * 28
    frozen = np.zeros(n, np.uint8)
    for d, (src, tgt) in enumerate([(c1, c2), (c2, c1)]):
        vx, vy, cost = O.pm_init(P, src, tgt, d)
        for it in range(P.pm_iters):
            for ph in range(2):
                O.pm_sweep(P, src, tgt, d, 0, it, ph, None, None, frozen, vx, vy, cost)
        np.testing.assert_array_equal(R.vx[d], vx)
        np.testing.assert_array_equal(R.vy[d], vy)
        np.testing.assert_array_equal(R.cost[d], cost)


# ---------------------------------------------------------------- edge-aware fill of unassigned pixels
def _nearest_seeds_dijkstra(q, seeds, W, H):
    """Reference seeds: exact geodesic distance (step 256 + |q_i - q_j| between 4-neighbours) from each seed by
    Dijkstra, the lowest distance winning, then the lowest seed index."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import dijkstra
    n = W * H
    rows, cols, wts = [], [], []
    for y in range(H):
        for x in range(W):
            i = y * W + x
            for (nx, ny) in ((x + 1, y), (x, y + 1)):
                if nx < W and ny < H:
                    j = ny * W + nx
                    w = 256 + abs(int(q[i]) - int(q[j]))
                    rows += [i, j]
                    cols += [j, i]
                    wts += [w, w]
    G = coo_matrix((wts, (rows, cols)), shape=(n, n)).tocsr()
    D = dijkstra(G, indices=sorted(seeds))
    best = np.full(n, -1)
    bd = np.full(n, np.inf)
    for k, s in enumerate(sorted(seeds)):  # ascending index: a tie keeps the earlier (lower) seed
        better = D[k] < bd
        best[better] = s
        bd[better] = D[k][better]
    return best


def test_fill_seeds_flat_frame_are_manhattan_nearest():
    rng = np.random.default_rng(2)
    W, H = 17, 11
    P = O.Params(W, H)
    am = np.full(W * H, -1, np.int32)
    seeds = rng.choice(W * H, 6, replace=False)
    am[seeds] = 0
    got = O.interp_seeds(P, np.full((H, W, 3), 0.3), am)
    ys, xs = np.divmod(np.arange(W * H), W)
    for i in range(W * H):
        d = [(abs(xs[i] - xs[s]) + abs(ys[i] - ys[s]), s) for s in seeds]
        assert got[i] == min(d)[1], (i, got[i], min(d))


def test_fill_seeds_respect_an_edge():
    """Two regions split by a vertical edge (grey steps of 2000 across it): pixels take the seed on their own
    side even when the other one is closer, exactly as the geodesic reference says."""
    W, H = 20, 9
    P = O.Params(W, H)
    img = np.zeros((H, W, 3))
    img[:, 10:] = 0.7  # q jumps by floor(1024 * 2.1) = 2150
    q = np.floor(1024.0 * img.sum(-1)).astype(np.int64).reshape(-1)
    am = np.full(W * H, -1, np.int32)
    left, right = 4 * W + 0, 4 * W + 11
    am[[left, right]] = 0
    got = O.interp_seeds(P, img, am)
    want = _nearest_seeds_dijkstra(q, [left, right], W, H)
    np.testing.assert_array_equal(got, want)
    assert got[4 * W + 9] == left  # 2 px from the right seed across the edge, 9 px from the left one


def test_fill_seeds_grey_quantisation_decides_a_close_call():
    """Reading R28's grey levels q = floor(1024 (R + G + B)) decide a close call: on a 7-pixel row with seeds at
    both ends, pixel 3 is three steps from each; the left path crosses q 0 -> 512 (a grey sum of 0.5), the right
    one q 512 -> 1 (a grey sum of 0.000977, so q = 1). The right path is cheaper by one, so pixel 3 takes the
    right seed; with equal costs the lower seed index (the left) would win."""
    P = O.Params(7, 1)
    img = np.zeros((1, 7, 3))
    img[0, 2:5, 0] = 0.5
    img[0, 5:, 0] = 0.000977
    am = np.array([0, -1, -1, -1, -1, -1, 0], np.int32)
    assert list(O.interp_seeds(P, img, am)) == [0, 0, 0, 6, 6, 6, 6]


def test_pipeline_fill_changes_only_unassigned_flows():
    s = scene.make_scene(48, 36, seed=12, n_layers=2, max_disp=4.0, affine=True)
    kw = dict(patch_radius=2, cells=(16, 8), pm_iters=2, num_hyp=32)
    R0 = O.run(O.Params(48, 36, **kw), s.frame1, s.frame2)
    R1 = O.run(O.Params(48, 36, interp=1, **kw), s.frame1, s.frame2)
    for d in range(2):
        assigned = R0.acc[d].m >= 0
        f0, f1 = R0.flow[d].reshape(-1, 2), R1.flow[d].reshape(-1, 2)
        np.testing.assert_array_equal(R0.occ[d], R1.occ[d])
        same = np.all(f0 == f1, axis=1)
        assert same.mean() > 0.5 and not same.all()
        assert same[assigned].all()


def _fit_one_window(s, vx, vy, **kw):
    P = O.Params(s, s, cells=(s,), num_hyp=4000, **{"patch_radius": 1, **kw})
    mh, mi = O.empty_models(P)
    frame = np.zeros((s, s, 3))
    O.fit_level(P, frame, frame, 0, 1, 1, vx, vy, None, mh, mi)
    return mh[0].reshape(3, 3), mi[0]


def test_plane_validity_support_orientation_and_scale():
    """Readings R12 and R14 on one 8x8 window (64 matches): a plane is valid iff its consensus has at least
    min_inliers and at least a fifth of the matches (13 of 64 is enough, 12 is not), it keeps orientation
    (det J > 0 at the centre) and its scale sqrt(det J) lies in [scale_min, scale_max]; a fitted but invalid
    plane carries the bad-geometry flag, and a scale at a bound is logged as a near tie."""
    s = 8
    xs, ys, vx0, vy0 = _affine_nnf(s, s, A_INT)                     # orientation kept, scale exactly 1
    rng = np.random.default_rng(11)
    for n_in, min_in, valid in ((13, 8, 1), (12, 8, 0), (20, 20, 1), (20, 21, 0)):
        vx, vy = vx0.copy(), vy0.copy()
        out = rng.permutation(s * s)[n_in:]
        vx[out] += (rng.integers(4, 9, size=out.size) * rng.choice([-1, 1], size=out.size)).astype(np.int32)
        vy[out] += (rng.integers(4, 9, size=out.size) * rng.choice([-1, 1], size=out.size)).astype(np.int32)
        _, mi = _fit_one_window(s, vx, vy, min_inliers=min_in)
        assert mi[O.MI_NIN] == 64 and mi[O.MI_COUNT] == n_in, (n_in, mi)
        assert mi[O.MI_VALID] == valid and bool(mi[O.MI_FLAGS] & O.F_BAD_GEOM) == (not valid), (n_in, min_in, mi)
    for smin, smax, valid in ((0.999, 1.001, 1), (1.001, 2.0, 0), (0.5, 0.999, 0)):
        _, mi = _fit_one_window(s, vx0, vy0, scale_min=smin, scale_max=smax)
        assert mi[O.MI_COUNT] == 64 and mi[O.MI_VALID] == valid, (smin, smax, mi)
    # a mirror image: all 64 matches agree, but the orientation flips
    _, _, vx, vy = _affine_nnf(s, s, np.array([[-1, 0, 7], [0, 1, 0], [0, 0, 1]], float))
    _, mi = _fit_one_window(s, vx, vy)
    assert mi[O.MI_COUNT] == 64 and mi[O.MI_FLAGS] & O.F_FITTED and not mi[O.MI_VALID]
    # scale exactly 2 = scale_max: valid or not by rounding, so the fit is logged as a near tie
    _, _, vx, vy = _affine_nnf(s, s, np.array([[2, 0, 0], [0, 2, 0], [0, 0, 1]], float))
    _, mi = _fit_one_window(s, vx, vy)
    assert mi[O.MI_COUNT] == 64 and mi[O.MI_FLAGS] & O.F_AMBIG


def test_plane_validity_denominator_on_the_grown_window():
    """Reading R14: the denominator of a projective plane must stay positive over the window grown by the patch
    radius r. With w = 1 - x/12 (zero at x = 12) and targets rounded to pixels, the fitted plane of an 8x8 window
    is valid for r = 3 (grown corners at x = 10) and invalid for r = 6 (x = 13), its scale at the centre, about
    1.7, inside [0.5, 2] either way."""
    s = 8
    ys, xs = np.divmod(np.arange(s * s), s)
    w = 1 - xs / 12.0
    vx = (np.round(xs / w) - xs).astype(np.int32)
    vy = (np.round(ys / w) - ys).astype(np.int32)
    for r, valid in ((3, 1), (6, 0)):
        Hf, mi = _fit_one_window(s, vx, vy, patch_radius=r)
        assert mi[O.MI_COUNT] >= 60 and mi[O.MI_FLAGS] & O.F_FITTED, (r, mi)
        Hn = Hf / Hf[2, 2]
        assert abs(Hn[2, 0] + 1 / 12) < 5e-3 and abs(Hn[2, 1]) < 5e-3, Hn   # the fit is the generating plane
        assert mi[O.MI_VALID] == valid, (r, mi)
