"""Shared helpers of the GPU parity tests: parameter mirroring between the
CUDA library and the oracle, and the near-tie bookkeeping.

Near-tie rule: a comparison of two floating-point values is ambiguous when the
FP64 oracle sees them closer than 1e-5 relative; an integer or label result
of the FP32 GPU path may differ from the oracle's only where the oracle logged
such an ambiguity upstream of it.
"""
import numpy as np

import oracle as O

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
