"""Shared helpers of the GPU parity tests: parameter mirroring between the
CUDA library and the oracle, and the near-tie bookkeeping.

Near-tie rule: a comparison of two floating-point values is ambiguous when the
FP64 oracle sees them closer than 1e-5 relative; an integer or label result
of the FP32 GPU path may differ from the oracle's only where the oracle logged
such an ambiguity upstream of it.
"""
import numpy as np

import oracle as O
from paper_1804_03787_gb300.gpm import LABELS as LABELS_KIND, MODELS as MODELS_KIND

TIE = 1e-5


def f32(x: float) -> float:
    """The float32 value the GPU compares against, as the oracle's threshold."""
    return float(np.float32(x))


def oracle_params(gp, W, H, pair_id=0) -> O.Params:
    cells = tuple(gp.cell_size[i] for i in range(gp.num_scales))
    return O.Params(W, H, patch_radius=gp.patch_radius, cells=cells, pm_iters=gp.pm_iters, num_hyp=gp.num_hyp,
                    eps=f32(gp.eps), ransac_px=f32(gp.ransac_px), fb_px=f32(gp.fb_px), eta=f32(gp.eta),
                    kappa=f32(gp.kappa), beta=f32(gp.beta), occ_thresh=f32(gp.occ_thresh),
                    scale_min=f32(gp.scale_min), scale_max=f32(gp.scale_max), min_inliers=gp.min_inliers,
                    fill_iters=gp.fill_iters, gain_normalize=gp.gain_normalize, pm_init=gp.pm_init, seed=gp.seed,
                    pair_id=pair_id, equalize=gp.equalize, census=gp.census, interp=gp.interp)


def oracle_frames(P: O.Params, f1, f2):
    """Source/target frames of both directions as the oracle sees them."""
    a = np.asarray(f1, np.float64)
    b = np.asarray(f2, np.float64)
    g = O.gain(P, a, b) if P.gain_normalize else 1.0
    b = b * g
    return [(a, b), (b, a)], g


def dilate(mask2d: np.ndarray, radius: int) -> np.ndarray:
    """Manhattan dilation (4-neighbour steps) of a boolean image."""
    m = mask2d.copy()
    for _ in range(radius):
        n = m.copy()
        n[1:] |= m[:-1]
        n[:-1] |= m[1:]
        n[:, 1:] |= m[:, :-1]
        n[:, :-1] |= m[:, 1:]
        m = n
    return m


def norm_h(H):
    H = np.asarray(H, np.float64).reshape(3, 3)
    return H / np.linalg.norm(H)


def rel_close(a, b, rel=1e-5, floor=1e-7, atol=0.0):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b) <= rel * np.maximum(np.maximum(np.abs(a), np.abs(b)), floor) + atol


# A colour error (eq. 3) is a mean of |texel - bilinear sample| over 3
# channels of values in [0, 1]; in FP32 each sample carries a few ulp(1)
# (~6e-8 each) of rounding, so its bound is absolute: 1e-6.
COLOUR_ATOL = 1e-6


# RANSAC outputs of a model that depend only on its window's matches (and, for the colour overlap, the frames)
RANSAC_FIELDS = [O.MI_COUNT, O.MI_NIN, O.MI_BESTK, O.MI_BESTSCORE, O.MI_NRC]


def ransac_equal(gmh, gmi, omh, omi, ids):
    """Per model: the RANSAC outputs (support, input size, winner, refit/geometry flags, colour overlap) and
    H within 1e-6 after normalisation."""
    ok = np.ones(len(ids), bool)
    geo = O.F_FITTED | O.F_REFIT | O.F_BAD_GEOM
    for k, m in enumerate(ids):
        a, b = gmi[m], omi[m]
        if any(a[f] != b[f] for f in RANSAC_FIELDS) or (a[O.MI_FLAGS] & geo) != (b[O.MI_FLAGS] & geo):
            ok[k] = False
        elif b[O.MI_FLAGS] & O.F_FITTED and np.abs(norm_h(gmh[m]) - norm_h(omh[m])).max() > 1e-6:
            ok[k] = False
    return ok


def final_map_check(ctx, P, frames, flow_t, occ_t, samples, seed):
    """Properties of a final flow and occlusion map (Sec. 3.4.1) on sampled pixels of direction 0: a pixel with a
    plane carries that model's mapping of it (to 1e-3 px) and is occluded iff its many-to-one cue is set, its
    target leaves the frame, or its colour error at the target reaches the threshold; a pixel without a plane keeps
    its NNF offset and is occluded.  Samples within 1e-5 of the threshold or 1e-3 px of the border are skipped.
    Returns (pixels with a plane, pixels whose occlusion bit was checked)."""
    W, H = P.width, P.height
    flow = flow_t.cpu().numpy().reshape(-1, 2)
    occ = occ_t.cpu().numpy().reshape(-1)
    from paper_1804_03787_gb300 import gpm
    m = ctx.export(gpm.LABELS)[0][0]
    mh = ctx.export(gpm.MODELS)[0]
    cue = ctx.export(gpm.CUES)[0]
    nnf = ctx.export(gpm.NNF)[0]
    src, tgt = frames[0]
    thr = P.occ_thresh
    rng = np.random.default_rng(seed)
    n_plane = n_checked = 0
    for i in rng.choice(W * H, min(samples, W * H), replace=False):
        x, y = int(i % W), int(i // W)
        if m[i] < 0:
            assert flow[i, 0] == nnf[i, 0] and flow[i, 1] == nnf[i, 1] and occ[i] == 1, (x, y)
            continue
        n_plane += 1
        h = mh[m[i]]
        w = h[6] * x + h[7] * y + h[8]
        X, Y = (h[0] * x + h[1] * y + h[2]) / w, (h[3] * x + h[4] * y + h[5]) / w
        assert abs(flow[i, 0] - (X - x)) < 1e-3 and abs(flow[i, 1] - (Y - y)) < 1e-3, (x, y, flow[i], X - x, Y - y)
        if cue[i] & O.CUE_M2O:
            assert occ[i] == 1
            continue
        Xg, Yg = x + float(flow[i, 0]), y + float(flow[i, 1])
        if min(abs(Xg), abs(Xg - (W - 1)), abs(Yg), abs(Yg - (H - 1))) < 1e-3:
            continue
        if not (0 <= Xg <= W - 1 and 0 <= Yg <= H - 1):
            assert occ[i] == 1, (x, y)
            continue
        delta = float(np.abs(src[y, x] - O.sample_bilinear(tgt, Xg, Yg)).mean())
        if abs(delta - thr) < 1e-5:
            continue
        assert occ[i] == (1 if delta >= thr else 0), (x, y, delta, thr, occ[i])
        n_checked += 1
    return n_plane, n_checked


def end_to_end_stats(ctx, R, gflow, oflow, gt, occ_gt, H, W):
    """End-to-end comparison of the whole method (direction 0): pixels with a plane on both sides, where the
    paper's final flow is the plane's mapping (Sec. 3.4.1), and the rest, which keep an NNF offset from the random
    search (any near tie upstream can change such an offset by many pixels).  Returns a dict of the agreement
    fractions and the EPE (against the scenes' ground truth, non-occluded pixels) of each side on each set."""
    gm = ctx.export(LABELS_KIND)[0][0].reshape(H, W)
    om = R.acc[0].m.reshape(H, W)
    both = (gm >= 0) & (om >= 0)
    d = np.hypot(*(gflow - oflow).transpose(2, 0, 1))
    eg = np.hypot(*(gflow - gt).transpose(2, 0, 1))
    eo = np.hypot(*(oflow - gt).transpose(2, 0, 1))
    vis = occ_gt == 0
    pv = both & vis
    # the same plane on both sides (the same model, fitted to the same homography): the same decision, so the
    # flows differ only by FP32 against FP64 arithmetic
    gmh, omh = ctx.export(MODELS_KIND)[0], R.mh[0]
    nm = omh.shape[0]
    hs = np.array([np.abs(norm_h(gmh[m]) - norm_h(omh[m])).max() < 1e-6 if omh[m].any() else False
                   for m in range(nm)])
    same = (gm == om) & (gm >= 0) & hs[np.clip(gm, 0, nm - 1)]
    sv = same & vis
    return dict(agree=float(np.mean(d < 1e-4)), plane_share=float(both.mean()),
                plane_agree=float(np.mean(d[both] < 1e-4)), plane_flow_diff=float(d[both].mean()),
                epe_plane_gpu=float(eg[pv].mean()), epe_plane_oracle=float(eo[pv].mean()),
                same_share=float(same.mean()), same_max_flow_diff=float(d[same].max()) if same.any() else 0.0,
                epe_same_gpu=float(eg[sv].mean()), epe_same_oracle=float(eo[sv].mean()),
                epe_gpu=float(eg[vis].mean()), epe_oracle=float(eo[vis].mean()),
                label_agree=float(np.mean(gm == om)))
