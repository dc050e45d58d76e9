"""FP64 CPU oracle for Multi-Scale Generalized Plane Match (arXiv 1804.03787).

TEST INFRASTRUCTURE.  A plain, slow, step-by-step restatement of the method
in double precision (C, compiled with gcc, loaded with ctypes).  Only the
tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg use
it; the CUDA library never does, and the two share no code.

Parity pins: every public function here is pinned by ``tests/test_oracle_*``
against closed forms, brute force, hand-built cases or invariants (see each
test's docstring); ``tests/test_oracle_mutants.py`` plants plausible mistakes
in copies of the C source and checks that the pins catch every one.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

MAX_SCALES = 8
MI = 12
MI_VALID, MI_COUNT, MI_NIN, MI_BESTK, MI_BESTSCORE, MI_FLAGS, MI_NRC, MI_NASSIGN, MI_NSYM, MI_AMB, MI_GAP10 = range(11)
F_FITTED, F_REFIT, F_AMBIG, F_BAD_FB, F_BAD_KAPPA, F_BAD_GEOM = 1, 2, 4, 8, 16, 32
CUE_M2O = 1


class _Params(C.Structure):
    _fields_ = [("W", C.c_int32), ("H", C.c_int32), ("r", C.c_int32), ("num_scales", C.c_int32),
                ("cell", C.c_int32 * MAX_SCALES), ("pm_iters", C.c_int32), ("num_hyp", C.c_int32),
                ("min_inliers", C.c_int32), ("fill_iters", C.c_int32), ("gain_normalize", C.c_int32),
                ("pm_init", C.c_int32), ("equalize", C.c_int32), ("census", C.c_int32), ("interp", C.c_int32), ("pad1", C.c_int32),
                ("eps", C.c_double), ("ransac_px", C.c_double),
                ("fb_px", C.c_double), ("eta", C.c_double), ("kappa", C.c_double), ("beta", C.c_double),
                ("occ_thresh", C.c_double), ("scale_min", C.c_double), ("scale_max", C.c_double),
                ("seed", C.c_uint64), ("pair_id", C.c_uint32), ("pad", C.c_uint32)]


@dataclass
class Params:
    """Method parameters (names follow the paper where it names them)."""
    width: int
    height: int
    patch_radius: int = 3            # r: 3 -> 7x7 patches (Sec. 4)
    cells: tuple = (32, 16, 8)       # window side per level, coarse to fine
    pm_iters: int = 4
    num_hyp: int = 256               # RANSAC hypotheses per window
    eps: float = 0.06                # epsilon of eq. 4
    ransac_px: float = 1.5           # RANSAC inlier radius t
    fb_px: float = 1.0               # forward-backward tolerance
    eta: float = 0.5                 # symmetric-overlap threshold (Sec. 3.4)
    kappa: float = 0.5               # RANSAC / colour inlier overlap threshold
    beta: float = 0.015              # coarse-level priority margin
    occ_thresh: float = 0.06         # final warp-error occlusion threshold
    scale_min: float = 0.5
    scale_max: float = 2.0
    min_inliers: int = 8
    fill_iters: int = 8
    gain_normalize: int = 1
    pm_init: int = 1
    equalize: int = 0                # HSV V-channel histogram equalisation of both frames (Sec. 4.2)
    census: int = 0                  # census data term for the level-0 NNF (Sec. 6)
    interp: int = 0                  # edge-aware fill of the pixels left without a plane
    seed: int = 0
    pair_id: int = 0

    def c(self) -> _Params:
        p = _Params()
        p.W, p.H, p.r = self.width, self.height, self.patch_radius
        p.num_scales = len(self.cells)
        for i, s in enumerate(self.cells):
            p.cell[i] = s
        p.pm_iters, p.num_hyp, p.min_inliers, p.fill_iters = self.pm_iters, self.num_hyp, self.min_inliers, self.fill_iters
        p.gain_normalize, p.pm_init, p.equalize = self.gain_normalize, self.pm_init, self.equalize
        p.census, p.interp = self.census, self.interp
        p.eps, p.ransac_px, p.fb_px, p.eta, p.kappa = self.eps, self.ransac_px, self.fb_px, self.eta, self.kappa
        p.beta, p.occ_thresh, p.scale_min, p.scale_max = self.beta, self.occ_thresh, self.scale_min, self.scale_max
        p.seed, p.pair_id = self.seed & 0xFFFFFFFFFFFFFFFF, self.pair_id & 0xFFFFFFFF
        return p


_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        P = C.POINTER
        d, i32, u8, u32 = P(C.c_double), P(C.c_int32), P(C.c_uint8), P(C.c_uint32)
        pp = P(_Params)
        sig = {
            "orc_philox4x32_10": (None, [u32, u32, u32]),
            "orc_grid_axis": (C.c_int, [C.c_int, C.c_int, i32]),
            "orc_total_cells": (C.c_int, [pp, i32]),
            "orc_sample_bilinear": (None, [d, C.c_int, C.c_int, C.c_double, C.c_double, d]),
            "orc_patch_cost": (C.c_double, [pp, d, d, C.c_int, C.c_int, C.c_int, C.c_int, d]),
            "orc_pm_init": (None, [pp, d, d, C.c_int, i32, i32, d]),
            "orc_pm_recost": (None, [pp, d, d, C.c_int, d, i32, u8, i32, i32, d]),
            "orc_pm_sweep": (None, [pp, d, d, C.c_int, C.c_int, C.c_int, C.c_int, d, i32, u8, i32, i32, d, d]),
            "orc_h_minimal": (C.c_int, [d, d, d]),
            "orc_h_dlt": (C.c_int, [C.c_int, d, d, d]),
            "orc_fit_level": (None, [pp, d, d, C.c_int, C.c_int, C.c_int, i32, i32, u8, d, i32]),
            "orc_den_zero_at_centre": (C.c_int, [i32, i32, i32, i32, C.c_int, C.c_int, C.c_int]),
            "orc_fit_cells": (None, [pp, d, d, C.c_int, C.c_int, C.c_int, i32, i32, u8, i32, C.c_int, d, i32]),
            "orc_assign": (None, [pp, d, d, C.c_int, C.c_int, d, i32, u8, i32, d, d, d, u8]),
            "orc_cue_counts": (None, [pp, C.c_int, C.c_int, i32, d, d, i32, d, d, i32, u8]),
            "orc_cue_invalidate": (None, [pp, C.c_int, C.c_int, i32]),
            "orc_many_to_one": (None, [pp, i32, d, d, d, u8, u8]),
            "orc_merge": (None, [pp, i32, d, d, d, i32, d, d, d, u8]),
            "orc_nnf_update": (None, [pp, i32, d, d, i32, i32, u8]),
            "orc_fill": (None, [pp, d, d, d, i32, u8, i32, d, d, d, u8]),
            "orc_final": (None, [pp, d, d, i32, d, d, i32, i32, u8, P(C.c_float), u8, u8]),
            "orc_gain": (C.c_double, [pp, d, d]),
            "orc_rgb_to_hsv": (None, [C.c_double, C.c_double, C.c_double, d, d, d]),
            "orc_hsv_to_rgb": (None, [C.c_double, C.c_double, C.c_double, d, d, d]),
            "orc_v_lut": (C.c_int, [pp, d, d]),
            "orc_hsv_equalize": (None, [pp, d, d]),
            "orc_census": (None, [pp, d, d]),
            "orc_grey_q": (None, [pp, d, i32]),
            "orc_interp_seeds": (None, [pp, i32, i32, i32]),
            "orc_interp_flow": (None, [pp, d, i32, d, d, i32, P(C.c_float)]),
            "orc_run": (None, [pp, d, d, C.c_void_p, C.c_int]),
            "orc_eval_count": (C.c_longlong, [C.c_int]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


def eval_count(reset: bool = True) -> int:
    """Patch costs the oracle evaluated since the last reset (timing instrumentation)."""
    return int(lib().orc_eval_count(1 if reset else 0))


def set_threads(n: int) -> None:
    """OpenMP threads of the oracle's parallel loops (results do not depend on it)."""
    import ctypes.util
    gomp = C.CDLL(ctypes.util.find_library("gomp") or "libgomp.so.1")
    gomp.omp_set_num_threads(int(n))


def max_threads() -> int:
    import ctypes.util
    gomp = C.CDLL(ctypes.util.find_library("gomp") or "libgomp.so.1")
    return int(gomp.omp_get_max_threads())


def _p(a: np.ndarray | None, ct):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "arrays passed to the oracle must be C-contiguous"
    return a.ctypes.data_as(C.POINTER(ct))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- primitives
def philox4x32_10(counter, key) -> np.ndarray:
    c = np.asarray(counter, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(out, C.c_uint32))
    return out


def grid_axis(n: int, s: int) -> np.ndarray:
    cnt = lib().orc_grid_axis(n, s, None)
    pos = np.zeros(max(cnt, 1), dtype=np.int32)
    lib().orc_grid_axis(n, s, _p(pos, C.c_int32))
    return pos[:cnt]


def cell_base(P: Params) -> np.ndarray:
    cb = np.zeros(MAX_SCALES + 1, dtype=np.int32)
    lib().orc_total_cells(C.byref(P.c()), _p(cb, C.c_int32))
    return cb[: len(P.cells) + 1]


def sample_bilinear(img: np.ndarray, X: float, Y: float) -> np.ndarray:
    img = _f64(img)
    out = np.zeros(3)
    lib().orc_sample_bilinear(_p(img, C.c_double), img.shape[1], img.shape[0], X, Y, _p(out, C.c_double))
    return out


def patch_cost(P: Params, src, tgt, px, py, vx, vy, G=None) -> float:
    src, tgt = _f64(src), _f64(tgt)
    g = None if G is None else _f64(np.asarray(G).reshape(9))
    return lib().orc_patch_cost(C.byref(P.c()), _p(src, C.c_double), _p(tgt, C.c_double), px, py, vx, vy,
                                _p(g, C.c_double))


def h_minimal(src, dst):
    s, d = _f64(src).reshape(8), _f64(dst).reshape(8)
    H = np.zeros(9)
    ok = lib().orc_h_minimal(_p(s, C.c_double), _p(d, C.c_double), _p(H, C.c_double))
    return (H.reshape(3, 3) if ok else None)


def h_dlt(src, dst):
    s, d = _f64(src), _f64(dst)
    n = s.shape[0]
    H = np.zeros(9)
    ok = lib().orc_h_dlt(n, _p(s.reshape(-1), C.c_double), _p(d.reshape(-1), C.c_double), _p(H, C.c_double))
    return (H.reshape(3, 3) if ok else None)


def rgb_to_hsv(r: float, g: float, b: float):
    h, s, v = C.c_double(), C.c_double(), C.c_double()
    lib().orc_rgb_to_hsv(r, g, b, C.byref(h), C.byref(s), C.byref(v))
    return h.value, s.value, v.value


def hsv_to_rgb(h: float, s: float, v: float):
    r, g, b = C.c_double(), C.c_double(), C.c_double()
    lib().orc_hsv_to_rgb(h, s, v, C.byref(r), C.byref(g), C.byref(b))
    return r.value, g.value, b.value


def v_lut(P: Params, rgb):
    """(changed?, 256 equalised V values by bin) of one HxWx3 frame (Sec. 4.2)."""
    lut = np.zeros(256)
    ok = lib().orc_v_lut(C.byref(P.c()), _p(_f64(rgb), C.c_double), _p(lut, C.c_double))
    return bool(ok), lut


def hsv_equalize(P: Params, rgb):
    """One frame with its V histogram equalised, H and S kept (Sec. 4.2)."""
    a = _f64(rgb)
    out = np.zeros_like(a)
    lib().orc_hsv_equalize(C.byref(P.c()), _p(a, C.c_double), _p(out, C.c_double))
    return out


def census(P: Params, rgb):
    """Census code frame of one HxWx3 frame: (code, 0, 0) per pixel, 24-bit 5x5 codes (Sec. 6)."""
    a = _f64(rgb)
    out = np.zeros_like(a)
    lib().orc_census(C.byref(P.c()), _p(a, C.c_double), _p(out, C.c_double))
    return out


def interp_seeds(P: Params, rgb, am):
    """Seed (nearest assigned pixel in geodesic distance, -1 if none) of every pixel, for the edge-aware fill."""
    n = P.width * P.height
    q = np.zeros(n, np.int32)
    lib().orc_grey_q(C.byref(P.c()), _p(_f64(rgb), C.c_double), _p(q, C.c_int32))
    seed = np.zeros(n, np.int32)
    lib().orc_interp_seeds(C.byref(P.c()), _p(q, C.c_int32), _p(np.ascontiguousarray(am, np.int32), C.c_int32),
                           _p(seed, C.c_int32))
    return seed


def interp_flow(P: Params, mh, acc: "Labels", seed, flow):
    """Edge-aware fill: flows (n x 2 float32, updated in place) of the pixels without a plane from their seeds."""
    lib().orc_interp_flow(C.byref(P.c()), _p(_f64(mh), C.c_double), _p(acc.m, C.c_int32), _p(acc.fx, C.c_double),
                          _p(acc.fy, C.c_double), _p(np.ascontiguousarray(seed, np.int32), C.c_int32),
                          _p(flow, C.c_float))
    return flow


def gain(P: Params, f1, f2) -> float:
    return lib().orc_gain(C.byref(P.c()), _p(_f64(f1), C.c_double), _p(_f64(f2), C.c_double))


# ---------------------------------------------------------------- state
@dataclass
class Labels:
    m: np.ndarray
    L: np.ndarray
    fx: np.ndarray
    fy: np.ndarray

    @staticmethod
    def empty(n: int, eps: float) -> "Labels":
        return Labels(np.full(n, -1, np.int32), np.full(n, eps), np.zeros(n), np.zeros(n))

    def copy(self) -> "Labels":
        return Labels(self.m.copy(), self.L.copy(), self.fx.copy(), self.fy.copy())


def n_models(P: Params) -> int:
    return 2 * int(cell_base(P)[-1])


def empty_models(P: Params):
    n = n_models(P)
    return np.zeros((n, 9)), np.zeros((n, MI), dtype=np.int32)


# ---------------------------------------------------------------- stages
def pm_init(P: Params, src, tgt, direction: int):
    n = P.width * P.height
    vx, vy, cost = np.zeros(n, np.int32), np.zeros(n, np.int32), np.zeros(n)
    lib().orc_pm_init(C.byref(P.c()), _p(_f64(src), C.c_double), _p(_f64(tgt), C.c_double), direction,
                      _p(vx, C.c_int32), _p(vy, C.c_int32), _p(cost, C.c_double))
    return vx, vy, cost


def pm_recost(P: Params, src, tgt, level, mh, mi, frozen, vx, vy, cost):
    lib().orc_pm_recost(C.byref(P.c()), _p(_f64(src), C.c_double), _p(_f64(tgt), C.c_double), level,
                        _p(mh, C.c_double), _p(mi, C.c_int32), _p(frozen, C.c_uint8),
                        _p(vx, C.c_int32), _p(vy, C.c_int32), _p(cost, C.c_double))


def pm_sweep(P: Params, src, tgt, direction, level, it, phase, mh, mi, frozen, vx, vy, cost, amb=None):
    lib().orc_pm_sweep(C.byref(P.c()), _p(_f64(src), C.c_double), _p(_f64(tgt), C.c_double), direction, level, it,
                       phase, _p(mh, C.c_double), _p(mi, C.c_int32), _p(frozen, C.c_uint8), _p(vx, C.c_int32),
                       _p(vy, C.c_int32), _p(cost, C.c_double), _p(amb, C.c_double))


def fit_level(P: Params, src, tgt, direction, level, stage, vx, vy, resid, mh, mi):
    lib().orc_fit_level(C.byref(P.c()), _p(_f64(src), C.c_double), _p(_f64(tgt), C.c_double), direction, level, stage,
                        _p(vx, C.c_int32), _p(vy, C.c_int32), _p(resid, C.c_uint8), _p(mh, C.c_double),
                        _p(mi, C.c_int32))


def den_zero_at_centre(src, dst, x0: int, y0: int, s: int) -> bool:
    """Exact test: the homography of 4 integer point pairs (4 x 2 each) has a zero denominator at the centre of
    the window of side s at (x0, y0)."""
    a = np.ascontiguousarray(src, np.int32).reshape(4, 2)
    b = np.ascontiguousarray(dst, np.int32).reshape(4, 2)
    sx, sy, tx, ty = (np.ascontiguousarray(v) for v in (a[:, 0], a[:, 1], b[:, 0], b[:, 1]))
    return bool(lib().orc_den_zero_at_centre(_p(sx, C.c_int32), _p(sy, C.c_int32), _p(tx, C.c_int32),
                                             _p(ty, C.c_int32), x0, y0, s))


def fit_cells(P: Params, src, tgt, direction, level, stage, vx, vy, resid, cells, mh, mi):
    """fit_level restricted to the listed windows of the level (their model slots of mh / mi are written)."""
    cells = np.ascontiguousarray(cells, np.int32)
    lib().orc_fit_cells(C.byref(P.c()), _p(_f64(src), C.c_double), _p(_f64(tgt), C.c_double), direction, level,
                        stage, _p(np.ascontiguousarray(vx, np.int32), C.c_int32),
                        _p(np.ascontiguousarray(vy, np.int32), C.c_int32), _p(resid, C.c_uint8),
                        _p(cells, C.c_int32), len(cells), _p(mh, C.c_double), _p(mi, C.c_int32))


def assign(P: Params, src, tgt, level, stage, mh, mi, mask, lab: Labels, amb=None):
    lib().orc_assign(C.byref(P.c()), _p(_f64(src), C.c_double), _p(_f64(tgt), C.c_double), level, stage,
                     _p(mh, C.c_double), _p(mi, C.c_int32), _p(mask, C.c_uint8), _p(lab.m, C.c_int32),
                     _p(lab.L, C.c_double), _p(lab.fx, C.c_double), _p(lab.fy, C.c_double), _p(amb, C.c_uint8))


def cue_counts(P: Params, level, stage, lab: Labels, other: Labels, mi, amb=None):
    lib().orc_cue_counts(C.byref(P.c()), level, stage, _p(lab.m, C.c_int32), _p(lab.fx, C.c_double),
                         _p(lab.fy, C.c_double), _p(other.m, C.c_int32), _p(other.fx, C.c_double),
                         _p(other.fy, C.c_double), _p(mi, C.c_int32), _p(amb, C.c_uint8))


def cue_invalidate(P: Params, level, stage, mi):
    lib().orc_cue_invalidate(C.byref(P.c()), level, stage, _p(mi, C.c_int32))


def many_to_one(P: Params, lab: Labels, cue, amb=None):
    lib().orc_many_to_one(C.byref(P.c()), _p(lab.m, C.c_int32), _p(lab.L, C.c_double), _p(lab.fx, C.c_double),
                          _p(lab.fy, C.c_double), _p(cue, C.c_uint8), _p(amb, C.c_uint8))


def merge(P: Params, lab: Labels, acc: Labels, amb=None):
    lib().orc_merge(C.byref(P.c()), _p(lab.m, C.c_int32), _p(lab.L, C.c_double), _p(lab.fx, C.c_double),
                    _p(lab.fy, C.c_double), _p(acc.m, C.c_int32), _p(acc.L, C.c_double), _p(acc.fx, C.c_double),
                    _p(acc.fy, C.c_double), _p(amb, C.c_uint8))


def nnf_update(P: Params, acc: Labels, vx, vy, frozen):
    lib().orc_nnf_update(C.byref(P.c()), _p(acc.m, C.c_int32), _p(acc.fx, C.c_double), _p(acc.fy, C.c_double),
                         _p(vx, C.c_int32), _p(vy, C.c_int32), _p(frozen, C.c_uint8))


def fill(P: Params, src, tgt, mh, mi, cue, acc: Labels, amb=None):
    """Model-propagation fill (Sec. 3.4.1) of acc in place; amb (uint8 per pixel, optional): the near-tie log,
    read and extended (see orc_fill)."""
    lib().orc_fill(C.byref(P.c()), _p(_f64(src), C.c_double), _p(_f64(tgt), C.c_double), _p(mh, C.c_double),
                   _p(mi, C.c_int32), _p(cue, C.c_uint8), _p(acc.m, C.c_int32), _p(acc.L, C.c_double),
                   _p(acc.fx, C.c_double), _p(acc.fy, C.c_double), _p(amb, C.c_uint8))


def final(P: Params, src, tgt, acc: Labels, vx, vy, cue, amb=None):
    """Final flow and occlusion map (Sec. 3.4.1); amb as in fill, extended with the occlusion decisions that
    rest on a near tie."""
    n = P.width * P.height
    flow = np.zeros((n, 2), np.float32)
    occ = np.zeros(n, np.uint8)
    lib().orc_final(C.byref(P.c()), _p(_f64(src), C.c_double), _p(_f64(tgt), C.c_double), _p(acc.m, C.c_int32),
                    _p(acc.fx, C.c_double), _p(acc.fy, C.c_double), _p(vx, C.c_int32), _p(vy, C.c_int32),
                    _p(cue, C.c_uint8), _p(flow, C.c_float), _p(occ, C.c_uint8), _p(amb, C.c_uint8))
    return flow, occ


# ---------------------------------------------------------------- whole method
class _State(C.Structure):
    _fields_ = [(n, C.c_void_p * 2) for n in
                ("vx", "vy", "cost", "mh", "mi", "am", "aL", "afx", "afy", "cue", "flow", "occ", "s1m")]


@dataclass
class Result:
    vx: list
    vy: list
    cost: list
    mh: list
    mi: list
    acc: list
    cue: list
    flow: list
    occ: list
    extra: dict = field(default_factory=dict)


def run(P: Params, f1, f2, stop_after: int = -1, init_nnf=None) -> Result:
    """Whole method on one pair; ``init_nnf`` = ((vx0, vy0), (vx1, vy1)) with P.pm_init = 0."""
    f1, f2 = _f64(f1), _f64(f2)
    assert f1.shape == (P.height, P.width, 3) and f2.shape == f1.shape
    n = P.width * P.height
    nm = n_models(P)
    R = Result(vx=[], vy=[], cost=[], mh=[], mi=[], acc=[], cue=[], flow=[], occ=[])
    st = _State()
    for d in range(2):
        if init_nnf is not None:
            vx = np.ascontiguousarray(init_nnf[d][0], np.int32).reshape(n).copy()
            vy = np.ascontiguousarray(init_nnf[d][1], np.int32).reshape(n).copy()
        else:
            vx, vy = np.zeros(n, np.int32), np.zeros(n, np.int32)
        R.vx.append(vx)
        R.vy.append(vy)
        R.cost.append(np.zeros(n))
        R.mh.append(np.zeros((nm, 9)))
        R.mi.append(np.zeros((nm, MI), np.int32))
        R.acc.append(Labels.empty(n, P.eps))
        R.cue.append(np.zeros(n, np.uint8))
        R.flow.append(np.zeros((n, 2), np.float32))
        R.occ.append(np.zeros(n, np.uint8))
        for name, arr in (("vx", vx), ("vy", vy), ("cost", R.cost[d]), ("mh", R.mh[d]), ("mi", R.mi[d]),
                          ("am", R.acc[d].m), ("aL", R.acc[d].L), ("afx", R.acc[d].fx), ("afy", R.acc[d].fy),
                          ("cue", R.cue[d]), ("flow", R.flow[d]), ("occ", R.occ[d])):
            getattr(st, name)[d] = arr.ctypes.data
        # the first-stage labels of the last level run (Sec. 3.2's residual region is where they are -1)
        R.extra.setdefault("stage1_m", []).append(np.full(n, -1, np.int32))
        st.s1m[d] = R.extra["stage1_m"][d].ctypes.data
    lib().orc_run(C.byref(P.c()), _p(f1, C.c_double), _p(f2, C.c_double), C.cast(C.pointer(st), C.c_void_p),
                  stop_after)
    return R
