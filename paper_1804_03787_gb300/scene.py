"""Seeded synthetic piecewise-planar scenes with exact ground truth.

This module only *generates inputs*: it holds none of the matching method's
arithmetic (no patch cost, no PatchMatch, no homography fitting).  Both the
CUDA path and the CPU oracle consume what it produces, so it lives on its own.

The scenes stand in for the MPI-Sintel frames the paper evaluates on (Sec. 4):
the same 1024x436 frame size, large motion, zoom, occlusion and illumination
change, but rendered from known planar layers so that the flow and occlusion
ground truth is exact.

Recipe (all randomness from ``numpy.random.default_rng(seed)``):

* background: fractal value noise, 5 octaves, base period 32 px, persistence
  0.5, lacunarity 2, smoothstep interpolation, one independent noise per
  channel around a random base colour;
* ``n_layers`` textured planar layers: random convex quads covering
  ``area_frac`` (default 5-25 %) of the frame each, z-ordered (later layers on top), each with its own noise
  texture and base colour;
* motion: each layer moves by a random affine map (``affine=True``: three
  corners perturbed) or homography (four corners perturbed) whose corner
  displacements are at most ``max_disp`` px; the background moves by a mild
  homography (corner displacements at most ``bg_disp`` px);
* frame 1 is painted in z-order; frame 2 samples each pixel by mapping it back
  through the inverse motion of the topmost layer that covers it, evaluating
  the continuous texture there (no raster resampling);
* ground-truth flow ``f(p) = H_z(p) p - p`` for the topmost layer ``z(p)`` of
  frame 1; ground-truth occlusion: ``p + f(p)`` leaves the frame or another
  layer is on top there in frame 2;
* photometrics: frame 2 multiplied by a gain ``g ~ U[gain_lo, gain_hi]`` (and, if
  ``gamma`` != 1, raised to that power: a non-uniform illumination change),
  Gaussian noise of std ``noise`` on both frames, clamped to [0, 1], stored as
  float32 HxWx3.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser (Steele et al. 2014) on uint64 arrays."""
    z = z.astype(np.uint64, copy=True)
    z ^= z >> np.uint64(30)
    z *= np.uint64(0xBF58476D1CE4E5B9)
    z ^= z >> np.uint64(27)
    z *= np.uint64(0x94D049BB133111EB)
    z ^= z >> np.uint64(31)
    return z


def _lattice(key: int, gx: np.ndarray, gy: np.ndarray) -> np.ndarray:
    """Deterministic value in [0, 1) for integer lattice points."""
    with np.errstate(over="ignore"):
        h = _mix64(np.uint64(key & 0xFFFFFFFFFFFFFFFF) ^ (gx.astype(np.int64).astype(np.uint64) * np.uint64(0x9E3779B97F4A7C15)))
        h = _mix64(h ^ (gy.astype(np.int64).astype(np.uint64) * np.uint64(0xC2B2AE3D27D4EB4F)))
    return (h >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def value_noise(x: np.ndarray, y: np.ndarray, key: int, octaves: int = 5,
                period: float = 32.0, persistence: float = 0.5, lacunarity: float = 2.0) -> np.ndarray:
    """Fractal value noise at continuous points, in [0, 1]."""
    total = np.zeros(np.broadcast(x, y).shape)
    amp, norm, per = 1.0, 0.0, period
    for o in range(octaves):
        u = x / per
        v = y / per
        gx = np.floor(u)
        gy = np.floor(v)
        fx = u - gx
        fy = v - gy
        sx = fx * fx * (3.0 - 2.0 * fx)
        sy = fy * fy * (3.0 - 2.0 * fy)
        k = key * 1315423911 + o * 2654435761
        a = _lattice(k, gx, gy)
        b = _lattice(k, gx + 1, gy)
        c = _lattice(k, gx, gy + 1)
        d = _lattice(k, gx + 1, gy + 1)
        total += amp * ((1 - sy) * ((1 - sx) * a + sx * b) + sy * ((1 - sx) * c + sx * d))
        norm += amp
        amp *= persistence
        per /= lacunarity
    return total / norm


def apply_h(H: np.ndarray, x: np.ndarray, y: np.ndarray):
    """Map points through a 3x3 homography (FP64)."""
    w = H[2, 0] * x + H[2, 1] * y + H[2, 2]
    return (H[0, 0] * x + H[0, 1] * y + H[0, 2]) / w, (H[1, 0] * x + H[1, 1] * y + H[1, 2]) / w


def h_from_points(src: np.ndarray, dst: np.ndarray) -> np.ndarray:
    """Homography through 4 point pairs (exact linear solve, h33 = 1)."""
    A = np.zeros((8, 8))
    b = np.zeros(8)
    for i in range(4):
        x, y = src[i]
        u, v = dst[i]
        A[2 * i] = [x, y, 1, 0, 0, 0, -u * x, -u * y]
        A[2 * i + 1] = [0, 0, 0, x, y, 1, -v * x, -v * y]
        b[2 * i] = u
        b[2 * i + 1] = v
    h = np.linalg.solve(A, b)
    return np.append(h, 1.0).reshape(3, 3)


def affine_from_points(src: np.ndarray, dst: np.ndarray) -> np.ndarray:
    """Affine map through 3 point pairs, as a 3x3 matrix."""
    A = np.zeros((6, 6))
    b = np.zeros(6)
    for i in range(3):
        x, y = src[i]
        u, v = dst[i]
        A[2 * i] = [x, y, 1, 0, 0, 0]
        A[2 * i + 1] = [0, 0, 0, x, y, 1]
        b[2 * i] = u
        b[2 * i + 1] = v
    h = np.linalg.solve(A, b)
    return np.array([[h[0], h[1], h[2]], [h[3], h[4], h[5]], [0.0, 0.0, 1.0]])


def _inside_convex(quad: np.ndarray, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Points inside a counter-clockwise convex quad (boundary included)."""
    ok = np.ones(np.broadcast(x, y).shape, dtype=bool)
    for i in range(4):
        ax, ay = quad[i]
        bx, by = quad[(i + 1) % 4]
        ok &= (bx - ax) * (y - ay) - (by - ay) * (x - ax) >= 0
    return ok


def _random_quad(rng, W: int, H: int, area_frac=(0.05, 0.25)) -> np.ndarray:
    while True:
        area = rng.uniform(*area_frac) * W * H
        aspect = rng.uniform(0.5, 2.0)
        hw = 0.5 * math.sqrt(area * aspect)
        hh = 0.5 * math.sqrt(area / aspect)
        hw = min(hw, 0.45 * W)
        hh = min(hh, 0.45 * H)
        cx = rng.uniform(0.1 * W, 0.9 * W)
        cy = rng.uniform(0.1 * H, 0.9 * H)
        th = rng.uniform(0, math.pi)
        c, s = math.cos(th), math.sin(th)
        base = np.array([[-hw, -hh], [hw, -hh], [hw, hh], [-hw, hh]])
        jit = rng.uniform(-0.15, 0.15, size=(4, 2)) * min(hw, hh)
        pts = base + jit
        quad = np.stack([cx + c * pts[:, 0] - s * pts[:, 1], cy + s * pts[:, 0] + c * pts[:, 1]], axis=1)
        # orient counter-clockwise in image coordinates (y down): positive cross products
        cr = [(quad[(i + 1) % 4, 0] - quad[i, 0]) * (quad[(i + 2) % 4, 1] - quad[(i + 1) % 4, 1])
              - (quad[(i + 1) % 4, 1] - quad[i, 1]) * (quad[(i + 2) % 4, 0] - quad[(i + 1) % 4, 0]) for i in range(4)]
        if all(v > 0 for v in cr):
            return quad
        if all(v < 0 for v in cr):
            return quad[::-1].copy()


def _random_motion(rng, quad: np.ndarray, max_disp: float, affine: bool) -> np.ndarray:
    for _ in range(100):
        d = rng.uniform(-1, 1, size=(4, 2))
        n = np.linalg.norm(d, axis=1, keepdims=True)
        d = np.where(n > 1, d / np.maximum(n, 1e-12), d) * max_disp
        if affine:
            M = affine_from_points(quad[:3], quad[:3] + d[:3])
        else:
            M = h_from_points(quad, quad + d)
        cx, cy = apply_h(M, quad[:, 0], quad[:, 1])
        disp = np.hypot(cx - quad[:, 0], cy - quad[:, 1])
        if affine and disp.max() > max_disp:
            continue
        # keep the layer orientation (no fold-over) and a moderate zoom
        J = M[:2, :2] - np.outer([cx.mean(), cy.mean()], M[2, :2])
        det = np.linalg.det(M) / (M[2, 0] * quad[:, 0].mean() + M[2, 1] * quad[:, 1].mean() + M[2, 2]) ** 3
        if 0.6 < det < 1.6 and np.all(M[2, 0] * quad[:, 0] + M[2, 1] * quad[:, 1] + M[2, 2] > 0.3):
            return M
    return np.eye(3)


@dataclass
class Scene:
    frame1: np.ndarray          # float32 HxWx3 in [0,1]
    frame2: np.ndarray          # float32 HxWx3 in [0,1]
    flow: np.ndarray            # float32 HxWx2, forward ground truth
    occ: np.ndarray             # uint8 HxW, 1 = occluded in frame 2
    layer_id: np.ndarray        # int16 HxW, topmost layer of frame 1 (-1 = background)
    motions: list = field(default_factory=list)   # 3x3 FP64 homographies, layers then background last
    quads: list = field(default_factory=list)
    gain: float = 1.0
    seed: int = 0

    @property
    def occluded_fraction(self) -> float:
        return float(self.occ.mean())


def make_scene(width: int, height: int, seed: int = 0, n_layers: int = 2, max_disp: float = 8.0,
               affine: bool = False, bg_disp: float | None = None, gain: tuple = (0.8, 1.2),
               noise: float = 2.0 / 255.0, area_frac: tuple = (0.05, 0.25), gamma: float = 1.0) -> Scene:
    """Render one seeded frame pair with exact flow and occlusion ground truth."""
    rng = np.random.default_rng(seed)
    W, H = int(width), int(height)
    if bg_disp is None:
        bg_disp = max_disp / 8.0
    key = int(rng.integers(1, 2**62))
    frame_quad = np.array([[0, 0], [W - 1, 0], [W - 1, H - 1], [0, H - 1]], dtype=np.float64)
    bg_motion = _random_motion(rng, frame_quad, bg_disp, affine) if bg_disp > 0 else np.eye(3)
    bg_base = rng.uniform(0.25, 0.75, size=3)
    quads, motions, bases = [], [], []
    for k in range(n_layers):
        q = _random_quad(rng, W, H, area_frac)
        quads.append(q)
        motions.append(_random_motion(rng, q, max_disp, affine))
        bases.append(rng.uniform(0.15, 0.85, size=3))

    def texture(k: int, x: np.ndarray, y: np.ndarray) -> np.ndarray:
        base = bg_base if k < 0 else bases[k]
        out = np.empty(x.shape + (3,))
        for ch in range(3):
            n = value_noise(x, y, key + 7919 * (k + 2) + 104729 * ch)
            out[..., ch] = base[ch] + 0.9 * (n - 0.5)
        return out

    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    # frame 1: painter's order
    z1 = np.full((H, W), -1, dtype=np.int16)
    for k, q in enumerate(quads):
        z1[_inside_convex(q, xs, ys)] = k
    f1 = np.empty((H, W, 3))
    for k in range(-1, n_layers):
        m = z1 == k
        if m.any():
            f1[m] = texture(k, xs[m], ys[m])

    inv = [np.linalg.inv(M) for M in motions]
    inv_bg = np.linalg.inv(bg_motion)

    def top_in_frame2(qx: np.ndarray, qy: np.ndarray) -> np.ndarray:
        z = np.full(qx.shape, -1, dtype=np.int16)
        for k in range(n_layers):
            px, py = apply_h(inv[k], qx, qy)
            z[_inside_convex(quads[k], px, py)] = k
        return z

    # frame 2: backward map each pixel through the inverse motion of its topmost layer
    z2 = top_in_frame2(xs, ys)
    f2 = np.empty((H, W, 3))
    for k in range(-1, n_layers):
        m = z2 == k
        if m.any():
            px, py = apply_h(inv_bg if k < 0 else inv[k], xs[m], ys[m])
            f2[m] = texture(k, px, py)

    # ground truth
    flow = np.empty((H, W, 2))
    for k in range(-1, n_layers):
        m = z1 == k
        if m.any():
            qx, qy = apply_h(bg_motion if k < 0 else motions[k], xs[m], ys[m])
            flow[m, 0] = qx - xs[m]
            flow[m, 1] = qy - ys[m]
    qx = xs + flow[..., 0]
    qy = ys + flow[..., 1]
    out = (qx < 0) | (qx > W - 1) | (qy < 0) | (qy > H - 1)
    occ = out | (top_in_frame2(qx, qy) != z1)

    g = float(rng.uniform(*gain))
    f2 = f2 * g
    if gamma != 1.0:  # a non-uniform illumination change of frame 2: I -> I^gamma
        f2 = np.clip(f2, 0.0, 1.0) ** gamma
    f1 = f1 + rng.normal(0.0, noise, size=f1.shape)
    f2 = f2 + rng.normal(0.0, noise, size=f2.shape)
    f1 = np.clip(f1, 0.0, 1.0).astype(np.float32)
    f2 = np.clip(f2, 0.0, 1.0).astype(np.float32)
    return Scene(frame1=np.ascontiguousarray(f1), frame2=np.ascontiguousarray(f2),
                 flow=flow.astype(np.float32), occ=occ.astype(np.uint8), layer_id=z1,
                 motions=motions + [bg_motion], quads=quads, gain=g, seed=seed)


# Named workloads: sizes and scene statistics of the paper's benchmark shape
# (Sec. 4: MPI-Sintel frames are 1024x436) and of the small parity case.
def tiny_scene(seed: int = 0) -> Scene:
    """128x96 pair, 2 layers, affine motion up to 8 px."""
    return make_scene(128, 96, seed=seed, n_layers=2, max_disp=8.0, affine=True)


def benchmark_scene(seed: int = 0) -> Scene:
    """1024x436 pair, 6 layers, homographies up to 64 px, gain and noise.

    Layers cover 2-8 % of the frame each, which puts the occluded fraction at
    about 7-14 % (mean near 10 %) over seeds 0-7."""
    return make_scene(1024, 436, seed=seed, n_layers=6, max_disp=64.0, affine=False,
                      area_frac=(0.02, 0.08))


def mixed_size_scene(seed: int, sizes=((256, 192), (512, 384), (1024, 436), (1280, 720)),
                     layers=(3, 8), max_disp: float = 96.0) -> Scene:
    """One pair of a mixed-size batch: size uniform over ``sizes``, 3-8 layers."""
    rng = np.random.default_rng(10_000 + seed)
    W, H = sizes[int(rng.integers(len(sizes)))]
    nl = int(rng.integers(layers[0], layers[1] + 1))
    return make_scene(W, H, seed=seed, n_layers=nl, max_disp=max_disp)
