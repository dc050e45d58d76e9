// RANSAC hypotheses without double precision.
//
// GB300 runs FP64 at a small fraction of its FP32 rate, and a 4-point
// homography in FP64 was the bottleneck of the per-window fit.  Here the
// projective-basis solution H ~ B adj(A) (see minimal_h in
// kernels_planes.cu) is formed exactly in 128-bit integers -- window-local
// coordinates keep every entry below 2^89 -- and the FP32 evaluation form is
// derived from exact integer numerators with one rounding each; the
// translation, which needs ~1e-7 px absolute accuracy on flows of hundreds of
// pixels, is split into hi + lo with an exact integer remainder.
#pragma once

#include <stdint.h>

#include "common.cuh"

namespace gpm {

typedef __int128 i128;
typedef unsigned __int128 u128;

// Integer -> float without conversion instructions (on GB300 conversions
// from 64-bit integers issue on the slow FP64 pipe): a value below 2^23 ORed
// into the mantissa of 2^23 is exact, so a 32-bit limb is two 16-bit halves
// and one fused multiply-add (correctly rounded).
__host__ __device__ __forceinline__ float u16_to_float(uint32_t v) {
#ifdef __CUDA_ARCH__
    return __int_as_float(0x4B000000u | v) - 8388608.f;
#else
    return (float)v;
#endif
}
__host__ __device__ __forceinline__ float u32_to_float(uint32_t v) {
#ifdef __CUDA_ARCH__
    return __fmaf_rn(u16_to_float(v >> 16), 65536.f, u16_to_float(v & 0xFFFFu));
#else
    return (float)v;
#endif
}

// Float near a 128-bit integer below 2^96 in magnitude (ours stay below 2^92):
// the 32-bit limbs combined by fused multiply-adds, within about 1 ulp -- every
// caller tolerates that (the translation is corrected by an exact remainder).
__host__ __device__ __forceinline__ float i128_to_float(i128 x) {
    const bool neg = x < 0;
    const u128 u = neg ? (u128)0 - (u128)x : (u128)x;  // magnitude: no cancellation between limbs
    const uint32_t l0 = (uint32_t)u, l1 = (uint32_t)(u >> 32), l2 = (uint32_t)(u >> 64);
#ifdef __CUDA_ARCH__
    const float f = __fmaf_rn(u32_to_float(l2), 18446744073709551616.f,
                              __fmaf_rn(u32_to_float(l1), 4294967296.f, u32_to_float(l0)));
#else
    const float f = (float)l2 * 18446744073709551616.f + (float)l1 * 4294967296.f + (float)l0;
#endif
    return neg ? -f : f;
}

// 4-point homography, exact: H = B adj(A) with the projective bases of the
// source points (A) and target points (B); window-local integer coordinates
// (|source| <= 48, |target| < 2^15).
__host__ __device__ inline void minimal_h_exact(const int* px, const int* py, const int* qx, const int* qy,
                                                i128* H) {
    int A[9];
    {
        const int x1 = px[0], x2 = px[1], x3 = px[2], y1 = py[0], y2 = py[1], y3 = py[2];
        const int l0 = (y2 - y3) * px[3] + (x3 - x2) * py[3] + (x2 * y3 - x3 * y2);
        const int l1 = (y3 - y1) * px[3] + (x1 - x3) * py[3] + (x3 * y1 - x1 * y3);
        const int l2 = (y1 - y2) * px[3] + (x2 - x1) * py[3] + (x1 * y2 - x2 * y1);
        A[0] = l0 * x1; A[1] = l1 * x2; A[2] = l2 * x3;
        A[3] = l0 * y1; A[4] = l1 * y2; A[5] = l2 * y3;
        A[6] = l0;      A[7] = l1;      A[8] = l2;
    }
    int64_t mu[3];
    {
        const int64_t x1 = qx[0], x2 = qx[1], x3 = qx[2], y1 = qy[0], y2 = qy[1], y3 = qy[2];
        mu[0] = (y2 - y3) * qx[3] + (x3 - x2) * qy[3] + (x2 * y3 - x3 * y2);
        mu[1] = (y3 - y1) * qx[3] + (x1 - x3) * qy[3] + (x3 * y1 - x1 * y3);
        mu[2] = (y1 - y2) * qx[3] + (x2 - x1) * qy[3] + (x1 * y2 - x2 * y1);
    }
    int64_t adj[9];
    adj[0] = (int64_t)A[4] * A[8] - (int64_t)A[5] * A[7];
    adj[1] = (int64_t)A[2] * A[7] - (int64_t)A[1] * A[8];
    adj[2] = (int64_t)A[1] * A[5] - (int64_t)A[2] * A[4];
    adj[3] = (int64_t)A[5] * A[6] - (int64_t)A[3] * A[8];
    adj[4] = (int64_t)A[0] * A[8] - (int64_t)A[2] * A[6];
    adj[5] = (int64_t)A[2] * A[3] - (int64_t)A[0] * A[5];
    adj[6] = (int64_t)A[3] * A[7] - (int64_t)A[4] * A[6];
    adj[7] = (int64_t)A[1] * A[6] - (int64_t)A[0] * A[7];
    adj[8] = (int64_t)A[0] * A[4] - (int64_t)A[1] * A[3];
    // H = Q diag(mu) adj(A) = Q C with C = diag(mu) adj(A).  Bounds for windows
    // up to 96 px (|source| <= 48) and frames up to 32767 px (|target| < 2^15):
    // |A| < 2^19.4, |adj| < 2^39.8, |mu| < 2^32.6, so C needs 128 bits
    // (< 2^72.4) and |H| < 2^89 (Q holds 16-bit coordinates, last row 1).
    i128 Cm[9];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) Cm[k * 3 + c] = (i128)mu[k] * adj[k * 3 + c];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        H[0 * 3 + c] = Cm[c] * qx[0] + Cm[3 + c] * qx[1] + Cm[6 + c] * qx[2];
        H[1 * 3 + c] = Cm[c] * qy[0] + Cm[3 + c] * qy[1] + Cm[6 + c] * qy[2];
        H[2 * 3 + c] = Cm[c] + Cm[3 + c] + Cm[6 + c];
    }
}

// num / den (den > 0) as hi + lo floats: hi the rounded quotient, lo the
// quotient of the exact integer remainder.
__host__ __device__ inline void split_ratio(i128 num, i128 den, float rden, float& hi, float& lo) {
    hi = i128_to_float(num) * rden;
    lo = 0.f;
    const float a = hi < 0 ? -hi : hi;
    if (!(a >= 9.5367431640625e-07f && a < 1048576.f)) return;  // 2^-20 <= |hi| < 2^20, else hi alone
    int e;
#ifdef __CUDA_ARCH__
    const float mant = frexpf(hi, &e);
#else
    const float mant = __builtin_frexpf(hi, &e);
#endif
    const int m = (int)(mant * 16777216.f);  // hi = m * 2^(e - 24), exactly
    const int sh = 24 - e;                   // in [4, 44]
    const i128 R = num * ((i128)1 << sh) - (i128)m * den;
#ifdef __CUDA_ARCH__
    lo = __fmul_rn(i128_to_float(R) * rden, __int_as_float((127 - sh) << 23));
#else
    lo = (i128_to_float(R) * rden) * __builtin_ldexpf(1.f, -sh);
#endif
}

// Evaluation form (origin 0) of the exact homography; false if its
// denominator vanishes at the window centre.
__host__ __device__ inline bool make_mef_exact(const i128* Hin, Mef& m) {
    i128 H[9];
    i128 dc2 = 2 * Hin[8] - (Hin[6] + Hin[7]);  // twice the denominator at the centre (-0.5, -0.5)
    if (dc2 == 0) return false;
    const bool flip = dc2 < 0;
    for (int k = 0; k < 9; ++k) H[k] = flip ? -Hin[k] : Hin[k];
    if (flip) dc2 = -dc2;
    const float rd = 1.f / i128_to_float(dc2);  // one reciprocal, then products (about 1 ulp each)
    m.b0 = i128_to_float(2 * H[0] - dc2) * rd;
    m.h1 = i128_to_float(2 * H[1]) * rd;
    split_ratio(2 * H[2], dc2, rd, m.h2h, m.h2l);
    m.h3 = i128_to_float(2 * H[3]) * rd;
    m.b4 = i128_to_float(2 * H[4] - dc2) * rd;
    split_ratio(2 * H[5], dc2, rd, m.h5h, m.h5l);
    m.g0 = i128_to_float(2 * H[6]) * rd;
    m.g1 = i128_to_float(2 * H[7]) * rd;
    m.e0 = i128_to_float(2 * H[8] - dc2) * rd;
    m.ef = 0.f;
    m.ox = 0;
    m.oy = 0;
    m.valid = 0;
    m.eden = 0;
    return true;
}

// Bit length of a 128-bit magnitude (0 for zero).
__host__ __device__ __forceinline__ int u128_bits(u128 u) {
    const uint64_t hi = (uint64_t)(u >> 64), lo = (uint64_t)u;
#ifdef __CUDA_ARCH__
    return hi ? 128 - __clzll((long long)hi) : (lo ? 64 - __clzll((long long)lo) : 0);
#else
    return hi ? 128 - __builtin_clzll(hi) : (lo ? 64 - __builtin_clzll(lo) : 0);
#endif
}

// The 9 entries of an exact homography as doubles scaled by one power of two
// (the largest magnitude in [1, 2)), each truncated to 53 significant bits,
// with every sign flipped when flip is set.  Built from integer operations
// alone: the exponent and mantissa fields are assembled directly (on GB300 a
// 64-bit integer conversion or an FP64 divide issues on the slow FP64 pipe).
__host__ __device__ inline void exact_to_double_pow2(const i128* H, double* D, bool flip) {
    int bl[9], E = 0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const u128 u = H[k] < 0 ? (u128)0 - (u128)H[k] : (u128)H[k];
        bl[k] = u128_bits(u);
        E = bl[k] > E ? bl[k] : E;
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const bool neg = H[k] < 0;
        const u128 u = neg ? (u128)0 - (u128)H[k] : (u128)H[k];
        uint64_t bits = 0;
        if (bl[k] > 0) {
            // m: the leading 53 bits, value m 2^(bl - 53); scaled by 2^-E: m 2^(bl - E - 53), whose biased
            // exponent field is bl - E + 1022 + 1 (>= 897 for magnitudes below 2^127: always normal)
            const uint64_t m = bl[k] > 53 ? (uint64_t)(u >> (bl[k] - 53)) : (uint64_t)u << (53 - bl[k]);
            bits = ((uint64_t)(bl[k] - E + 1023) << 52) | (m & 0xFFFFFFFFFFFFFull);
            if (neg != flip) bits |= 0x8000000000000000ull;
        }
#ifdef __CUDA_ARCH__
        D[k] = __longlong_as_double((long long)bits);
#else
        __builtin_memcpy(&D[k], &bits, 8);
#endif
    }
}

// The first n entries of an exact homography as doubles (unnormalised).
__host__ __device__ inline void exact_to_double(const i128* H, double* D, int n = 9) {
    for (int k = 0; k < n; ++k) {
        const bool neg = H[k] < 0;
        const u128 u = neg ? (u128)0 - (u128)H[k] : (u128)H[k];
        const double v = (double)(uint64_t)(u >> 64) * 18446744073709551616.0 + (double)(uint64_t)u;
        D[k] = neg ? -v : v;
    }
}

}  // namespace gpm
