// Device-side building blocks shared by the GB300 kernels: counter-based
// random numbers, frame texel loads, bilinear sampling, window geometry and
// the FP32 evaluation form of a plane homography.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gpm {

constexpr int kMaxCell = 96;  // largest window side (its matches fill 144 KiB of shared memory in RANSAC)
// Border of the padded frame copies read by the level-0 PatchMatch: the
// largest patch radius.  Every tap of a candidate whose target pixel is in
// the frame then lies inside the padded copy, whose border replicates the
// edge texels, so a tap reads what clamping its coordinates would read.
constexpr int kPad = 4;
constexpr int kMI = 12;  // integer fields per model (layout of GPM_MODEL_INFO)
// A warped sample point counts as inside the frame up to this far (px)
// beyond the border: clamped bilinear sampling is continuous there, and
// identity planes on the border then never split on rounding.
constexpr float kFrameTol = 1e-3f;
// A later plane displaces the current best one only if its robust loss is
// lower by more than this: planes of one surface fitted in overlapping
// windows give equal losses up to rounding, and the first window keeps them.
constexpr float kLTie = 1e-6f;
enum { MI_VALID = 0, MI_COUNT, MI_NIN, MI_BESTK, MI_BESTSCORE, MI_FLAGS, MI_NRC, MI_NASSIGN, MI_NSYM, MI_AMB };
enum { F_FITTED = 1, F_REFIT = 2, F_AMBIG = 4, F_BAD_FB = 8, F_BAD_KAPPA = 16, F_BAD_GEOM = 32 };
enum { CUE_M2O = 1 };

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds, each two
// 32x32->64 products whose halves are mixed with the other counter words and
// the key; the key advances by the Weyl constants after every round.
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                        uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint4(c0, c1, c2, c3);
}

// Counter words: (element index, sub-index, stream tag, pair id).
__host__ __device__ __forceinline__ uint32_t stream_tag(int purpose, int dir, int level, int stage) {
    return ((uint32_t)purpose << 24) | ((uint32_t)dir << 16) | ((uint32_t)level << 8) | (uint32_t)stage;
}
enum { RNG_INIT = 1, RNG_SEARCH = 2, RNG_RANSAC = 3 };

// Uniform integer in [0, n) from a 32-bit random word: floor(u * n / 2^32)
// (one multiply-high instead of an integer division).
__device__ __forceinline__ uint32_t bounded_u32(uint32_t u, uint32_t n) { return __umulhi(u, n); }

// ---------------------------------------------------------------- frames
// Frames live as RGBX texels: FP32 float4 (16 B), or FP16 / BF16 x4 (8 B).
template <int ST>
__device__ __forceinline__ float4 ldpix(const void* base, int i);
template <>
__device__ __forceinline__ float4 ldpix<0>(const void* base, int i) {
    return __ldg(reinterpret_cast<const float4*>(base) + i);
}
template <>
__device__ __forceinline__ float4 ldpix<1>(const void* base, int i) {
    const uint2 u = __ldg(reinterpret_cast<const uint2*>(base) + i);
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
template <>
__device__ __forceinline__ float4 ldpix<2>(const void* base, int i) {
    const uint2 u = __ldg(reinterpret_cast<const uint2*>(base) + i);
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
}

// The raw texel type of a storage type, and loads of texels held in shared memory.
template <int ST>
struct TexelOf {
    using type = uint2;
};
template <>
struct TexelOf<0> {
    using type = float4;
};
template <int ST>
__device__ __forceinline__ float4 ldpix_shared(const void* base, int i);
template <>
__device__ __forceinline__ float4 ldpix_shared<0>(const void* base, int i) {
    return reinterpret_cast<const float4*>(base)[i];
}
template <>
__device__ __forceinline__ float4 ldpix_shared<1>(const void* base, int i) {
    const uint2 u = reinterpret_cast<const uint2*>(base)[i];
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
template <>
__device__ __forceinline__ float4 ldpix_shared<2>(const void* base, int i) {
    const uint2 u = reinterpret_cast<const uint2*>(base)[i];
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
}

// A texel at a shared-memory byte address (a 32-bit shared-window address, as from __cvta_generic_to_shared).
template <int ST>
__device__ __forceinline__ float4 ldpix_shared_addr(unsigned addr);
template <>
__device__ __forceinline__ float4 ldpix_shared_addr<0>(unsigned addr) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr));
    return v;
}
template <int ST>
__device__ __forceinline__ uint2 ld_shared_u2(unsigned addr) {
    uint2 u;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(u.x), "=r"(u.y) : "r"(addr));
    return u;
}
template <>
__device__ __forceinline__ float4 ldpix_shared_addr<1>(unsigned addr) {
    const uint2 u = ld_shared_u2<1>(addr);
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
template <>
__device__ __forceinline__ float4 ldpix_shared_addr<2>(unsigned addr) {
    const uint2 u = ld_shared_u2<2>(addr);
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
}

// Bilinear blend of the four texels around a point with fractions (fx, fy).
__device__ __forceinline__ float3 blend4(float4 a, float4 b, float4 c, float4 d, float fx, float fy) {
    const float gx = 1.f - fx, gy = 1.f - fy;
    float3 o;
    o.x = gy * (gx * a.x + fx * b.x) + fy * (gx * c.x + fx * d.x);
    o.y = gy * (gx * a.y + fx * b.y) + fy * (gx * c.y + fx * d.y);
    o.z = gy * (gx * a.z + fx * b.z) + fy * (gx * c.z + fx * d.z);
    return o;
}

// Bilinear sample at X = ix + fx, Y = iy + fy (fx, fy in [0,1)), the point
// first clamped to [0, W-1] x [0, H-1].
template <int ST>
__device__ __forceinline__ float3 bilinear(const void* img, int W, int H, int ix, float fx, int iy, float fy) {
    if (ix < 0) {
        ix = 0;
        fx = 0.f;
    } else if (ix >= W - 1) {
        ix = W - 1;
        fx = 0.f;
    }
    if (iy < 0) {
        iy = 0;
        fy = 0.f;
    } else if (iy >= H - 1) {
        iy = H - 1;
        fy = 0.f;
    }
    const int ix1 = min(ix + 1, W - 1), iy1 = min(iy + 1, H - 1);
    const float4 a = ldpix<ST>(img, iy * W + ix), b = ldpix<ST>(img, iy * W + ix1);
    const float4 c = ldpix<ST>(img, iy1 * W + ix), d = ldpix<ST>(img, iy1 * W + ix1);
    return blend4(a, b, c, d, fx, fy);
}

__device__ __forceinline__ float absdiff3(float4 a, float3 b) {
    return fabsf(a.x - b.x) + fabsf(a.y - b.y) + fabsf(a.z - b.z);
}

// ---------------------------------------------------------------- window grid
// Windows of side s at stride h = s/2 from 0, plus one flush with the far
// border when the regular ones stop short of it (Sec. 3.1.2: half overlap).
struct AxisGrid {
    int n_reg;   // regular windows at i * h
    int extra;   // 1 if a last window sits at size - s
    int count;   // n_reg + extra
    int last;    // position of the extra window
};
struct LevelGeom {
    int s, h, base;  // side, stride, index of the level's first window in the model table
    AxisGrid gx, gy;
    __host__ __device__ int ncells() const { return gx.count * gy.count; }
};

__host__ __device__ inline AxisGrid make_axis(int n, int s) {
    AxisGrid a;
    const int h = s / 2;
    if (s <= 0 || n < s) {
        a.n_reg = a.extra = a.count = 0;
        a.last = 0;
        return a;
    }
    a.n_reg = (n - s) / h + 1;
    a.extra = ((a.n_reg - 1) * h + s < n) ? 1 : 0;
    a.count = a.n_reg + a.extra;
    a.last = n - s;
    return a;
}
__host__ __device__ __forceinline__ int win_pos(const AxisGrid& a, int h, int i) {
    return i < a.n_reg ? i * h : a.last;
}
// Windows covering coordinate x, ascending: returns count (<= 3) and fills idx.
__device__ __forceinline__ int covering(const AxisGrid& a, int s, int h, int x, int idx[3]) {
    int k = 0;
    int lo = x - s + 1 > 0 ? (x - s + 1 + h - 1) / h : 0;
    int hi = min(x / h, a.n_reg - 1);
    for (int i = lo; i <= hi && k < 2; ++i) idx[k++] = i;
    if (a.extra && x >= a.last) idx[k++] = a.n_reg;
    return k;
}
// The same windows as a range (no array, so it stays in registers): window
// k < count is first + k while k < nreg, then the extra window.
__device__ __forceinline__ int covering_range(const AxisGrid& a, int s, int h, int x, int& first, int& nreg) {
    const int lo = x - s + 1 > 0 ? (x - s + 1 + h - 1) / h : 0;
    const int hi = min(x / h, a.n_reg - 1);
    first = lo;
    nreg = max(0, min(hi - lo + 1, 2));
    return nreg + ((a.extra && x >= a.last) ? 1 : 0);
}
__device__ __forceinline__ int covering_at(const AxisGrid& a, int first, int nreg, int k) {
    return k < nreg ? first + k : a.n_reg;
}
// Home window: the window whose central half holds x.
__device__ __forceinline__ int home_index(const AxisGrid& a, int s, int h, int x) {
    const int t = x - s / 4;
    int i = t >= 0 ? t / h : -1;
    return min(max(i, 0), a.count - 1);
}

// ---------------------------------------------------------------- plane models
// FP32 evaluation form of a homography, in coordinates local to the window
// origin o = (x0 + s/2, y0 + s/2), scaled so that the denominator is 1 at the
// window centre (o - 0.5).  With u = p - o:
//   e = den - 1 = e0 + g0 ux + g1 uy,
//   flow D(u) = H(u) - u = t + (S - t e) / (1 + e),
//   S_x = b0 ux + h1 uy - ux e, S_y = h3 ux + b4 uy - uy e,
// where b0 = h0 - 1, b4 = h4 - 1 and the translation t = (h2, h5) is kept as
// a hi/lo pair of floats.  Every term but t is small near the window, so the
// flow keeps ~1e-7 px absolute accuracy even for 100+ px motions.
struct __align__(16) Mef {
    float b0, h1, h2h, h2l;
    float h3, b4, h5h, h5l;
    float g0, g1, e0, ef;   // ef: rounding bound of the inlier test f (mef_set_bounds), 0 if unset
    int ox, oy, valid, eden;  // eden: the bits of the denominator's rounding bound (float)
};

// Splits a flow component t_hi + c (c small) into integer k and fraction f in [0,1).
__device__ __forceinline__ void split_flow(float th, float c, int& k, float& f) {
    float t = floorf(th + c);
    f = (th - t) + c;
    if (f < 0.f) {
        f += 1.f;
        t -= 1.f;
    } else if (f >= 1.f) {
        f -= 1.f;
        t += 1.f;
    }
    k = (int)t;
}

// Flow of the model at local integer point u.  Returns false if the
// projective denominator is not positive.  (kx + fx, ky + fy) = D(u).
__device__ __forceinline__ bool mef_flow(const Mef& m, float ux, float uy, int& kx, float& fx, int& ky, float& fy) {
    const float e = m.e0 + m.g0 * ux + m.g1 * uy;
    const float den = 1.f + e;
    if (!(den > 0.f)) return false;
    const float Sx = m.b0 * ux + m.h1 * uy - ux * e;
    const float Sy = m.h3 * ux + m.b4 * uy - uy * e;
    const float rden = __frcp_rn(den);  // one reciprocal (about 1e-7 px on these small terms)
    const float cx = m.h2l + (Sx - m.h2h * e) * rden;
    const float cy = m.h5l + (Sy - m.h5h * e) * rden;
    split_flow(m.h2h, cx, kx, fx);
    split_flow(m.h5h, cy, ky, fy);
    return true;
}

// Same, as rounded offset v = floor(D + 0.5) and remainder r = D - v in [-0.5, 0.5).
__device__ __forceinline__ void round_split(int k, float f, int& v, float& r) {
    if (f >= 0.5f) {
        v = k + 1;
        r = f - 1.f;
    } else {
        v = k;
        r = f;
    }
}

// ---- certified residual tests
// The FP32 inlier test below decides f = n.n - t2 den^2 < 0 (and den > 0).
// A first-order bound of its rounding, valid over a whole window, lets a
// kernel know when the FP32 sign could differ from the exact one; such a test
// is then decided again in FP64 (hyp_inlier_fp64).  Coefficients of the form
// carry at most 4 units of 2^-24 (u) relative error, each operation one.  With
// U >= |u| and V >= |v| over the window's matches, A = |e0| + (|g0| + |g1|) U
// (so |e| <= A, den <= 1 + A), B = (|b0| + |h1| + |h3| + |b4|) U, the error of
// a component of n is at most u (3 |n_c| + D_c), D_x + D_y <= 10 B + 24 U A +
// 18 V A + 4 (|h2l| + |h5l|), and that of den at most u (6 A + 1).  A test
// whose exact sign differs from the FP32 one has |f| within the error, so
// n.n is within 10 % of t2 den^2 there; then
//   |df| <= u den (12.6 t2 den + 2.1 t (D_x + D_y) + 12 t2 A),
// taken twice for margin with den <= 1 + A.  If the bound is not small
// against t2 (strongly projective or far-reaching hypotheses) every test of
// the hypothesis is decided in FP64.
__device__ __forceinline__ void mef_set_bounds(Mef& m, float U, float V, float t2) {
    // FP32 arithmetic on non-negative terms (a few roundings, covered by the 1.001 factor)
    const float u = 5.9604644775390625e-08f;
    const float t = sqrtf(t2);
    const float A = fabsf(m.e0) + (fabsf(m.g0) + fabsf(m.g1)) * U;
    const float B = (fabsf(m.b0) + fabsf(m.h1) + fabsf(m.h3) + fabsf(m.b4)) * U;
    // At a possible flip |n| <= 1.05 t den, and n = den (D(u) - v) with D(u) = (h + S) / den the model's flow,
    // so the match's offset is within 1.05 t of D(u), |D_x| + |D_y| <= (|h2| + |h5| + B + 2 U A) / (1 - A): the
    // offsets that matter are bounded by the model, whatever far-off (random) matches the window holds.
    const float h25 = fabsf(m.h2h) + fabsf(m.h5h) + fabsf(m.h2l) + fabsf(m.h5l);
    if (A < 0.5f) V = fminf(V, (h25 + B + 2.f * U * A) / (1.f - A) + 2.2f * t);
    const float D = 10.f * B + (24.f * U + 18.f * V) * A + 4.f * (fabsf(m.h2l) + fabsf(m.h5l));
    const float dmax = 1.f + A;
    float ef = 2.f * u * dmax * (12.6f * t2 * dmax + 2.1f * t * D + 12.f * t2 * A) * 1.001f;
    if (!(ef < 0.05f * t2)) ef = 1e30f;  // too loose for the window: each test takes its own bound (mef_inlier_pt)
    m.ef = ef;
    m.eden = __float_as_int(2.f * u * (6.f * A + 1.f) * 1.001f);
}

// Squared-residual test of a match (u, u + v) against the model:
// ||H(u) - (u + v)||^2 < t2, evaluated as n^2 < t2 den^2 with den > 0.
__device__ __forceinline__ bool mef_inlier(const Mef& m, float ux, float uy, float vx, float vy, float t2) {
    const float e = m.e0 + m.g0 * ux + m.g1 * uy;
    const float den = 1.f + e;
    const float Sx = m.b0 * ux + m.h1 * uy - ux * e;
    const float Sy = m.h3 * ux + m.b4 * uy - uy * e;
    const float nx = ((m.h2h - vx) + m.h2l) + Sx - vx * e;
    const float ny = ((m.h5h - vy) + m.h5l) + Sy - vy * e;
    return den > 0.f && nx * nx + ny * ny < t2 * den * den;
}

// The same test, and unc: the FP32 decision may differ from the exact one (the
// bounds of mef_set_bounds), so the caller decides it again in FP64.
__device__ __forceinline__ bool mef_inlier_c(const Mef& m, float ux, float uy, float vx, float vy, float t2,
                                             bool& unc) {
    const float e = m.e0 + m.g0 * ux + m.g1 * uy;
    const float den = 1.f + e;
    const float Sx = m.b0 * ux + m.h1 * uy - ux * e;
    const float Sy = m.h3 * ux + m.b4 * uy - uy * e;
    const float nx = ((m.h2h - vx) + m.h2l) + Sx - vx * e;
    const float ny = ((m.h5h - vy) + m.h5l) + Sy - vy * e;
    const float n2 = nx * nx + ny * ny, rhs = t2 * den * den;
    unc = fabsf(n2 - rhs) <= m.ef || fabsf(den) <= __int_as_float(m.eden);
    return den > 0.f && n2 < rhs;
}

// A hypothesis whose window-wide bound is too loose (strongly projective, or
// far-reaching matches against a large local scale).
__device__ __forceinline__ bool mef_loose(const Mef& m) { return m.ef >= 1e29f; }

// The inlier test with the bound of mef_set_bounds taken at this match alone
// (A, B, |u|, |v| and n of the match instead of the window's maxima), for
// loose hypotheses.  unc as in mef_inlier_c.
__device__ __forceinline__ bool mef_inlier_pt(const Mef& m, float ux, float uy, float vx, float vy, float t2,
                                              bool& unc) {
    const float e = m.e0 + m.g0 * ux + m.g1 * uy;
    const float den = 1.f + e;
    const float Sx = m.b0 * ux + m.h1 * uy - ux * e;
    const float Sy = m.h3 * ux + m.b4 * uy - uy * e;
    const float nx = ((m.h2h - vx) + m.h2l) + Sx - vx * e;
    const float ny = ((m.h5h - vy) + m.h5l) + Sy - vy * e;
    const float n2 = nx * nx + ny * ny, rhs = t2 * den * den;
    const float u = 5.9604644775390625e-08f;
    const float A = fabsf(m.e0) + fabsf(m.g0 * ux) + fabsf(m.g1 * uy);
    const float B = fabsf(m.b0 * ux) + fabsf(m.h1 * uy) + fabsf(m.h3 * ux) + fabsf(m.b4 * uy);
    const float Um = fmaxf(fabsf(ux), fabsf(uy)), Vm = fmaxf(fabsf(vx), fabsf(vy));
    const float D = 10.f * B + (24.f * Um + 18.f * Vm) * A + 4.f * (fabsf(m.h2l) + fabsf(m.h5l));
    const float eden = 2.f * u * (6.f * A + 1.f) * 1.0001f;
    const float dd = fabsf(den) + eden;
    // the error of f at this match with its own n (the terms of mef_set_bounds without the assumption that
    // n.n is near t2 den^2): 2 |n_c| dn_c + d(t2 den^2) + the rounding of f, twice for margin
    const float n1 = fabsf(nx) + fabsf(ny);
    const float ef = 2.f * u * (8.f * n2 + 2.f * n1 * D + 12.f * t2 * dd * A + 8.f * t2 * dd * dd + 4.f * u * D * D) *
                     1.0001f;
    unc = fabsf(n2 - rhs) <= ef || fabsf(den) <= eden;
    return den > 0.f && n2 < rhs;
}

// Exact-arithmetic stand-in for the residual test: H in window-local
// coordinates as doubles (any positive scale, oriented so that the
// denominator is positive at the window centre), the test in FP64 without a
// division: den = h6 ux + h7 uy + h8 > 0 and |h_xy . (u, 1) - (u + v) den|^2
// < t2 den^2.  Its rounding is some 1e-15 of the terms, far inside the
// 1e-5 near-tie band of the comparison.
__device__ __forceinline__ bool hyp_inlier_fp64(const double* Hl, float ux, float uy, float vx, float vy, double t2) {
    const double x = ux, y = uy, qx = (double)ux + (double)vx, qy = (double)uy + (double)vy;
    const double w = Hl[6] * x + Hl[7] * y + Hl[8];
    if (!(w > 0.0)) return false;
    const double nx = Hl[0] * x + Hl[1] * y + Hl[2] - qx * w;
    const double ny = Hl[3] * x + Hl[4] * y + Hl[5] - qy * w;
    return nx * nx + ny * ny < t2 * w * w;
}

// mef_inlier for two matches at once on the packed FP32x2 pipe: each
// coefficient of the evaluation form in both halves of a float2, and the
// same operations as mef_inlier in each half (one rounding each, as there).
struct Mef2 {
    float2 b0, h1, h2h, h2l, h3, b4, h5h, h5l, g0, g1, e0;
};
__device__ __forceinline__ Mef2 mef2_of(const Mef& m) {
    Mef2 r;
    r.b0 = make_float2(m.b0, m.b0);
    r.h1 = make_float2(m.h1, m.h1);
    r.h2h = make_float2(m.h2h, m.h2h);
    r.h2l = make_float2(m.h2l, m.h2l);
    r.h3 = make_float2(m.h3, m.h3);
    r.b4 = make_float2(m.b4, m.b4);
    r.h5h = make_float2(m.h5h, m.h5h);
    r.h5l = make_float2(m.h5l, m.h5l);
    r.g0 = make_float2(m.g0, m.g0);
    r.g1 = make_float2(m.g1, m.g1);
    r.e0 = make_float2(m.e0, m.e0);
    return r;
}
__device__ __forceinline__ void mef_inlier2(const Mef2& m, const float4& a, const float4& b, float t2, bool& ia,
                                            bool& ib) {
    const float2 ux = make_float2(a.x, b.x), uy = make_float2(a.y, b.y);
    const float2 vx = make_float2(a.z, b.z), vy = make_float2(a.w, b.w);
    const float2 m1 = make_float2(-1.f, -1.f);
    const float2 e = __ffma2_rn(m.g1, uy, __ffma2_rn(m.g0, ux, m.e0));
    const float2 den = __fadd2_rn(make_float2(1.f, 1.f), e);
    const float2 ne = __fmul2_rn(e, m1);
    const float2 sx = __ffma2_rn(ux, ne, __ffma2_rn(m.h1, uy, __fmul2_rn(m.b0, ux)));
    const float2 sy = __ffma2_rn(uy, ne, __ffma2_rn(m.b4, uy, __fmul2_rn(m.h3, ux)));
    const float2 nx = __ffma2_rn(vx, ne, __fadd2_rn(__fadd2_rn(__ffma2_rn(vx, m1, m.h2h), m.h2l), sx));
    const float2 ny = __ffma2_rn(vy, ne, __fadd2_rn(__fadd2_rn(__ffma2_rn(vy, m1, m.h5h), m.h5l), sy));
    const float2 n2 = __ffma2_rn(nx, nx, __fmul2_rn(ny, ny));
    const float2 rhs = __fmul2_rn(__fmul2_rn(make_float2(t2, t2), den), den);
    ia = den.x > 0.f && n2.x < rhs.x;
    ib = den.y > 0.f && n2.y < rhs.y;
}
// The same with the uncertainty flags of mef_inlier_c (ef, eden: the form's bounds).
__device__ __forceinline__ void mef_inlier2_c(const Mef2& m, float ef, float eden, const float4& a, const float4& b,
                                              float t2, bool& ia, bool& ib, bool& ua, bool& ub) {
    const float2 ux = make_float2(a.x, b.x), uy = make_float2(a.y, b.y);
    const float2 vx = make_float2(a.z, b.z), vy = make_float2(a.w, b.w);
    const float2 m1 = make_float2(-1.f, -1.f);
    const float2 e = __ffma2_rn(m.g1, uy, __ffma2_rn(m.g0, ux, m.e0));
    const float2 den = __fadd2_rn(make_float2(1.f, 1.f), e);
    const float2 ne = __fmul2_rn(e, m1);
    const float2 sx = __ffma2_rn(ux, ne, __ffma2_rn(m.h1, uy, __fmul2_rn(m.b0, ux)));
    const float2 sy = __ffma2_rn(uy, ne, __ffma2_rn(m.b4, uy, __fmul2_rn(m.h3, ux)));
    const float2 nx = __ffma2_rn(vx, ne, __fadd2_rn(__fadd2_rn(__ffma2_rn(vx, m1, m.h2h), m.h2l), sx));
    const float2 ny = __ffma2_rn(vy, ne, __fadd2_rn(__fadd2_rn(__ffma2_rn(vy, m1, m.h5h), m.h5l), sy));
    const float2 n2 = __ffma2_rn(nx, nx, __fmul2_rn(ny, ny));
    const float2 rhs = __fmul2_rn(__fmul2_rn(make_float2(t2, t2), den), den);
    ia = den.x > 0.f && n2.x < rhs.x;
    ib = den.y > 0.f && n2.y < rhs.y;
    const float2 f = __fadd2_rn(n2, __fmul2_rn(rhs, m1));
    ua = fabsf(f.x) <= ef || fabsf(den.x) <= eden;
    ub = fabsf(f.y) <= ef || fabsf(den.y) <= eden;
}

// Local homography (double, rows, maps u -> local target) to the evaluation
// form.  Orientation and scale: denominator +1 at the window centre
// (-0.5, -0.5).  Returns false if that denominator is zero.
__host__ __device__ inline bool make_mef(const double* Hl, int ox, int oy, Mef& m) {
    const double dc = Hl[8] - 0.5 * (Hl[6] + Hl[7]);
    if (!(dc != 0.0)) return false;
    const double k = 1.0 / dc;
    double h[9];
    for (int i = 0; i < 9; ++i) h[i] = Hl[i] * k;
    m.b0 = (float)(h[0] - 1.0);
    m.h1 = (float)h[1];
    m.h2h = (float)h[2];
    m.h2l = (float)(h[2] - (double)m.h2h);
    m.h3 = (float)h[3];
    m.b4 = (float)(h[4] - 1.0);
    m.h5h = (float)h[5];
    m.h5l = (float)(h[5] - (double)m.h5h);
    m.g0 = (float)h[6];
    m.g1 = (float)h[7];
    m.e0 = (float)(h[8] - 1.0);
    m.ef = 0.f;
    m.ox = ox;
    m.oy = oy;
    m.eden = 0;
    return true;
}

// absolute H = T(o) Hl T(-o), unit Frobenius norm, positive denominator at
// the window centre (o - 0.5).
__host__ __device__ inline void local_to_abs(const double* Hl, int ox, int oy, double* Ha) {
    // Hl' = Hl * T(-o): columns: c2' = c2 - ox c0 - oy c1
    double t[9];
    for (int r = 0; r < 3; ++r) {
        t[r * 3 + 0] = Hl[r * 3 + 0];
        t[r * 3 + 1] = Hl[r * 3 + 1];
        t[r * 3 + 2] = Hl[r * 3 + 2] - ox * Hl[r * 3 + 0] - oy * Hl[r * 3 + 1];
    }
    // T(o) * t: rows: r0 += ox r2, r1 += oy r2
    for (int c = 0; c < 3; ++c) {
        Ha[0 * 3 + c] = t[0 * 3 + c] + ox * t[2 * 3 + c];
        Ha[1 * 3 + c] = t[1 * 3 + c] + oy * t[2 * 3 + c];
        Ha[2 * 3 + c] = t[2 * 3 + c];
    }
    const double cx = ox - 0.5, cy = oy - 0.5;
    const double w = Ha[6] * cx + Ha[7] * cy + Ha[8];
    double f = 0;
    for (int i = 0; i < 9; ++i) f += Ha[i] * Ha[i];
    f = 1.0 / sqrt(f);
    if (w < 0) f = -f;
    for (int i = 0; i < 9; ++i) Ha[i] *= f;
}

// local H = T(-o) Ha T(o)
__host__ __device__ inline void abs_to_local(const double* Ha, int ox, int oy, double* Hl) {
    double t[9];
    for (int r = 0; r < 3; ++r) {
        t[r * 3 + 0] = Ha[r * 3 + 0];
        t[r * 3 + 1] = Ha[r * 3 + 1];
        t[r * 3 + 2] = Ha[r * 3 + 2] + ox * Ha[r * 3 + 0] + oy * Ha[r * 3 + 1];
    }
    for (int c = 0; c < 3; ++c) {
        Hl[0 * 3 + c] = t[0 * 3 + c] - ox * t[2 * 3 + c];
        Hl[1 * 3 + c] = t[1 * 3 + c] - oy * t[2 * 3 + c];
        Hl[2 * 3 + c] = t[2 * 3 + c];
    }
}

// ---------------------------------------------------------------- per-pair device view
struct Labels {
    int* m;      // model id, -1 = none
    float* L;    // robust loss of eq. 4
    int2* v;     // rounded plane flow
    float2* r;   // plane flow minus v, in [-0.5, 0.5)
};

// Per-window record of the RANSAC refit, filled in three launches (fit,
// solve, finish) and reused by every level and stage.
struct __align__(16) RefitWork {
    long long mom[24];      // exact DLT moments of the winner's inliers about (cx, cy, cu, cv)
    __int128 hx[9];         // the winning hypothesis, exact
    Mef mef0, mef1;         // evaluation forms (origin 0) of the winner and of the refit, with test bounds
    double hl_r[9];         // the refit in window-local coordinates, denominator 1 at the window centre (FP64 tests)
    double ds, dt;          // sums of the inliers' distances to the source / target centroids
    double ha_w[9], ha_r[9];  // absolute homographies of the winner and of the refit
    int cx, cy, cu, cv;     // integer centres of the moments
    int status;             // 2: refit pending (set by the fit), else the window is final
    int nin;                // winner's inliers
    int refit_ok, geo_w, geo_r;
    float vmax;             // largest |offset| component among the window's matches (test bounds)
    int pad[2];
};

struct PairView {
    int W, H, n;
    int m_models;         // models per direction (bound of every model id)
    uint32_t pair_id;
    const void* img[2];   // ingested I1, I2 (RGBX in storage type)
    const void* imgp[2];  // the same, (W + 2 kPad) x (H + 2 kPad) with replicated borders (level-0 PatchMatch)
    float4* box[2];       // per pixel, the RGB sums over its square patch of clamped taps (level-0 lower bound)
    int Wp;               // row length of imgp
    int2* nnf[2];
    float* cost[2];
    uint8_t* frozen[2];
    uint8_t* cue[2];
    uint8_t* resid[2];
    Labels acc[2], tent[2], st1[2], lvl[2];
    double* mh[2];        // [m][9] absolute homographies
    Mef* mef[2];          // [m]
    int* mi[2];           // [m][kMI]
    int* list[2];         // unfrozen pixel indices, colour 0 then colour 1
    int* list_count;      // [2 dirs][2 colours]
    int* flag;            // device consistency flag: set (non-zero) by a check that failed, read by gpm_sync
    unsigned long long* m2o_key[2];
    RefitWork* rw[2];     // [cells of the largest level]
    uint32_t* code[2];    // census codes of each frame (census data term)
    int* gq;              // floor(1024 (R + G + B)) of frame 1 as given (edge-aware fill)
    unsigned long long* evals;  // [PM evaluations level 0, levels >= 1, RANSAC residual tests], or nullptr
};

// The pairs of a launch, passed by value as a __grid_constant__ kernel
// parameter: one launch of a stage covers up to kBatch pairs (blockIdx.z
// selects the pair), each with its views and level geometries.  Reading them
// from the constant bank keeps them out of registers and free of aliasing
// with the kernels' stores (a table in global memory cost the 1024x436 step
// ~1.5 ms of reloads), and no host copy enters the stream, so a whole
// multi-pair pipeline can be captured in one CUDA graph.
constexpr int kMaxScales = 8;  // GPM_MAX_SCALES
constexpr int kBatch = 8;
struct Batch {
    PairView pv[kBatch];
    LevelGeom geo[kBatch][kMaxScales];  // level l at index l - 1
    __host__ __device__ __forceinline__ const PairView& view(int z) const { return pv[z]; }
    __host__ __device__ __forceinline__ LevelGeom geom(int z, int level) const {
        return level > 0 ? geo[z][level - 1] : LevelGeom{};
    }
};
// The block's pair view, copied once from the kernel's parameter table into shared memory.  Fields read from the
// table itself, indexed by blockIdx.z, are constant-bank loads at each use (a kernel's registers cannot hold them
// all); from shared memory they are plain loads.  Every thread of the block must call it: it ends with a barrier.
__device__ __forceinline__ const PairView& shared_view(const Batch& bt, PairView& dst) {
    static_assert(sizeof(PairView) % 4 == 0, "word copy");
    const int* s = reinterpret_cast<const int*>(&bt.view(blockIdx.z));
    int* d = reinterpret_cast<int*>(&dst);
    const int nt = blockDim.x * blockDim.y * blockDim.z;
    const int t = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    for (int e = t; e < (int)(sizeof(PairView) / 4); e += nt) d[e] = s[e];
    __syncthreads();
    return dst;
}
// The caller's flow and occlusion buffers of the pairs of one final-map launch (kernel parameters).
struct FinalOut {
    float* flow[kBatch];
    uint8_t* occ[kBatch];
};

}  // namespace gpm
