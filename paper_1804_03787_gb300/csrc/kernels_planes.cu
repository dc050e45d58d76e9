// Plane kernels (sm_103a): per-window RANSAC with least-squares refit,
// assignment by colour consistency, occlusion cues, merge, NNF update, model
// propagation fill and the final flow / occlusion map.
#include <float.h>

#include "common.cuh"
#include "hyp_exact.cuh"
#include "kernels.h"
#include "../../include/gpm.h"

namespace gpm {

constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------- 4-point homography
// Exact projective basis construction (hyp_exact.cuh): with P = [p1 p2 p3]
// (homogeneous columns) and lambda = adj(P) p4, A = P diag(lambda) maps the
// projective basis e1, e2, e3, (1,1,1) onto p1..p4 up to scale; likewise B
// for the targets, and H ~ B adj(A).
__device__ __forceinline__ bool collinear3(int ax, int ay, int bx, int by, int cx, int cy) {
    return (long long)(bx - ax) * (cy - ay) - (long long)(by - ay) * (cx - ax) == 0;
}

__device__ __forceinline__ void mat3_mul(const double* A, const double* B, double* C) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) C[i * 3 + j] = A[i * 3] * B[j] + A[i * 3 + 1] * B[3 + j] + A[i * 3 + 2] * B[6 + j];
}

// X = i + f (f in [0,1)) lies in [-kFrameTol, n - 1 + kFrameTol].
__device__ __forceinline__ bool in_frame_tol(int i, float f, int n) {
    if (i >= 0 && i < n - 1) return true;
    if (i == n - 1) return f <= kFrameTol;
    if (i == -1) return f >= 1.f - kFrameTol;
    return false;
}

// Target sample position of pixel (px, py) under a plane: integer base and
// fraction; false if the denominator is not positive or the point leaves the
// frame (tolerance kFrameTol).
__device__ __forceinline__ bool plane_target(const Mef& m, int px, int py, int W, int H, int& ix, float& fx, int& iy,
                                             float& fy, int& kx, int& ky) {
    if (!mef_flow(m, (float)(px - m.ox), (float)(py - m.oy), kx, fx, ky, fy)) return false;
    ix = px + kx;
    iy = py + ky;
    return in_frame_tol(ix, fx, W) && in_frame_tol(iy, fy, H);
}

template <int ST>
__device__ __forceinline__ float colour_delta(const void* src, const void* tgt, int W, int H, int px, int py, int ix,
                                              float fx, int iy, float fy) {
    const float4 a = ldpix<ST>(src, py * W + px);
    const float3 b = bilinear<ST>(tgt, W, H, ix, fx, iy, fy);
    return absdiff3(a, b) / 3.f;
}

// First-order bound of the FP32 error of the position mef_flow gives for local point u (the sum of the x and y
// errors, px): every term of the flow carries a few units of 2^-24 of its own size.
__device__ __forceinline__ float mef_pos_bound(const Mef& m, float ux, float uy) {
    const float ea = fabsf(m.e0) + fabsf(m.g0 * ux) + fabsf(m.g1 * uy);
    const float den = 1.f + m.e0 + m.g0 * ux + m.g1 * uy;
    const float sx = fabsf(m.b0 * ux) + fabsf(m.h1 * uy) + fabsf(ux) * ea + fabsf(m.h2h) * ea;
    const float sy = fabsf(m.h3 * ux) + fabsf(m.b4 * uy) + fabsf(uy) * ea + fabsf(m.h5h) * ea;
    const float d = fabsf(m.h2h) + fabsf(m.h5h) + (sx + sy) / fmaxf(den, 1e-30f);
    return 16.f * 5.9604644775390625e-08f * (sx + sy + d * (1.f + ea)) / fmaxf(den, 1e-30f) +
           1.1920928955078125e-07f * (fabsf(m.h2h) + fabsf(m.h5h));
}

// The colour-overlap decision of one RANSAC inlier in FP64: the local model Hl
// (denominator positive at the window centre) maps p, the frame test with the
// same tolerance, then eq. 3's colour error from the stored texels, bilinear
// with the point clamped into the frame.  Returns 1 if delta < eps.
template <int ST>
__device__ __noinline__ int colour_overlap_fp64(const double* Hl, const void* src, const void* tgt, int W, int H,
                                                int ox, int oy, int px, int py, float eps) {
    const double ux = px - ox, uy = py - oy;
    const double w = Hl[6] * ux + Hl[7] * uy + Hl[8];
    if (!(w > 0.0)) return 0;
    const double X = ox + (Hl[0] * ux + Hl[1] * uy + Hl[2]) / w, Y = oy + (Hl[3] * ux + Hl[4] * uy + Hl[5]) / w;
    if (!(X >= -(double)kFrameTol && X <= W - 1 + (double)kFrameTol && Y >= -(double)kFrameTol &&
          Y <= H - 1 + (double)kFrameTol))
        return 0;
    const double cxp = fmin(fmax(X, 0.0), (double)(W - 1)), cyp = fmin(fmax(Y, 0.0), (double)(H - 1));
    const int ix = min((int)floor(cxp), W - 1), iy = min((int)floor(cyp), H - 1);
    const double fx = cxp - ix, fy = cyp - iy;
    const int ix1 = min(ix + 1, W - 1), iy1 = min(iy + 1, H - 1);
    const float4 a = ldpix<ST>(tgt, iy * W + ix), b = ldpix<ST>(tgt, iy * W + ix1);
    const float4 c = ldpix<ST>(tgt, iy1 * W + ix), d = ldpix<ST>(tgt, iy1 * W + ix1);
    const float4 p = ldpix<ST>(src, py * W + px);
    const double gx = 1.0 - fx, gy = 1.0 - fy;
    const double r = gy * (gx * a.x + fx * b.x) + fy * (gx * c.x + fx * d.x);
    const double g = gy * (gx * a.y + fx * b.y) + fy * (gx * c.y + fx * d.y);
    const double bb = gy * (gx * a.z + fx * b.z) + fy * (gx * c.z + fx * d.z);
    const double delta = (fabs(p.x - r) + fabs(p.y - g) + fabs(p.z - bb)) / 3.0;
    return delta < (double)eps;
}

// ---------------------------------------------------------------- cooperating groups
// One window is processed by a group: a warp (windows up to 16 x 16) or a
// whole block.  The group provides rank, size, barrier, sums and the scan
// used to compact the residual matches in raster order.
struct WarpGroup {
    static constexpr int size = 32;
    __device__ int rank() const { return threadIdx.x & 31; }
    __device__ void sync() const { __syncwarp(); }
    __device__ double sum(double v) const {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
        return v;
    }
    __device__ int sum(int v) const {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
        return v;
    }
    __device__ unsigned long long max(unsigned long long v) const {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long o = __shfl_xor_sync(FULL, v, off);
            v = o > v ? o : v;
        }
        return v;
    }
    __device__ long long sum(long long v) const {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
        return v;
    }
    __device__ bool any(bool p) const { return __any_sync(FULL, p); }
    // exclusive prefix of `take` over the group and the total
    __device__ int scan(bool take, int& total) const {
        const unsigned b = __ballot_sync(FULL, take);
        total = __popc(b);
        return __popc(b & ((1u << rank()) - 1));
    }
};

template <int NT>
struct BlockGroup {
    static constexpr int size = NT;
    double* red_d;
    int* red_i;
    unsigned long long* red_u;
    __device__ int rank() const { return threadIdx.x; }
    __device__ void sync() const { __syncthreads(); }
    __device__ double sum(double v) const {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red_d[threadIdx.x >> 5] = v;
        __syncthreads();
        double t = 0;
        for (int w = 0; w < NT / 32; ++w) t += red_d[w];  // fixed order: same bits on every thread
        return t;
    }
    __device__ int sum(int v) const {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red_i[threadIdx.x >> 5] = v;
        __syncthreads();
        int t = 0;
        for (int w = 0; w < NT / 32; ++w) t += red_i[w];
        return t;
    }
    __device__ bool any(bool p) const { return __syncthreads_or(p) != 0; }
    __device__ long long sum(long long v) const {  // exact: integer addition in any order
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red_u[threadIdx.x >> 5] = (unsigned long long)v;
        __syncthreads();
        unsigned long long t = 0;
        for (int w = 0; w < NT / 32; ++w) t += red_u[w];
        return (long long)t;
    }
    __device__ unsigned long long max(unsigned long long v) const {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long o = __shfl_xor_sync(FULL, v, off);
            v = o > v ? o : v;
        }
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red_u[threadIdx.x >> 5] = v;
        __syncthreads();
        unsigned long long t = 0;
        for (int w = 0; w < NT / 32; ++w) t = red_u[w] > t ? red_u[w] : t;
        return t;
    }
    __device__ int scan(bool take, int& total) const {
        const unsigned b = __ballot_sync(FULL, take);
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        __syncthreads();
        if (lane == 0) red_i[warp] = __popc(b);
        __syncthreads();
        int off = 0;
        total = 0;
        for (int w = 0; w < NT / 32; ++w) {
            if (w < warp) off += red_i[w];
            total += red_i[w];
        }
        return off + __popc(b & ((1u << lane) - 1));
    }
};

// ---------------------------------------------------------------- least-squares refit (one thread per window)
// Entry (r, c) of the normalised DLT normal matrix A^T A from the 24 moments
// mom[a * 6 + q] = sum w_a zz^T[q] (w in {1, u, v, u^2 + v^2}, zz^T entries
// q in {x^2, xy, x, y^2, y, 1}): rows/columns 0-2 hold the b b^T block, 3-5
// the a a^T block, 6-8 the (u, v)-weighted blocks of the rows a = (0, -z, v z)
// and b = (z, 0, -u z).
__device__ __forceinline__ double dlt_entry(const double* mom, int r, int c) {
    const int br = r / 3, bc = c / 3, ir = r % 3, ic = c % 3;
    const int lo = ir < ic ? ir : ic, hi = ir < ic ? ic : ir;
    const int q = lo == 0 ? hi : (lo == 1 ? (hi == 1 ? 3 : 4) : 5);
    if (br == bc) return br < 2 ? mom[q] : mom[18 + q];
    if ((br == 0 && bc == 2) || (br == 2 && bc == 0)) return -mom[6 + q];
    if ((br == 1 && bc == 2) || (br == 2 && bc == 1)) return -mom[12 + q];
    return 0.0;
}

// Plane geometry checks of a local homography (rows, maps u -> local
// target): denominator positive on the window grown by the patch radius and
// local area scale sqrt(det J) at the window centre in [scale_min, scale_max].
__device__ __forceinline__ bool plane_geometry_ok(const double* Hl, int s, int r, double scale_min, double scale_max) {
    const double dc = Hl[8] - 0.5 * (Hl[6] + Hl[7]);
    const double rdc = 1.0 / dc;
    double hn[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) hn[q] = Hl[q] * rdc;
    bool ok = true;
    const double cxs[2] = {-(double)(s / 2) - r, (double)(s / 2) - 1 + r};
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
            if (!(hn[6] * cxs[a] + hn[7] * cxs[b] + hn[8] > 0)) ok = false;
    const double uc = -0.5;
    const double X = hn[0] * uc + hn[1] * uc + hn[2], Y = hn[3] * uc + hn[4] * uc + hn[5];
    const double j00 = hn[0] - X * hn[6], j01 = hn[1] - X * hn[7];
    const double j10 = hn[3] - Y * hn[6], j11 = hn[4] - Y * hn[7];
    const double det = j00 * j11 - j01 * j10;
    // sqrt(det) in [scale_min, scale_max], compared without the root
    return ok && det > 0 && det >= scale_min * scale_min && det <= scale_max * scale_max;
}

// 1 / sqrt(n) for a positive normal double: an FP32 estimate refined by two
// Newton steps (relative error ~1e-16), far fewer FP64 operations than a
// correctly rounded square root and division.  Inverse iteration only needs a
// scale close to the unit norm.
__device__ __forceinline__ double rsqrt_nr(double n) {
    if (!(n > 1e-30 && n < 1e30)) return 1.0 / sqrt(n);  // outside the FP32 estimate's range
    double r = (double)rsqrtf((float)n);
#pragma unroll
    for (int k = 0; k < 2; ++k) r = fma(0.5 * r, fma(-n * r, r, 1.0), r);
    return r;
}

// Cholesky factor (lower, packed, in place) of the symmetric matrix in A;
// rd[j] = 1 / L[j][j].  The diagonal roots come from an FP32 estimate and
// Newton steps (rsqrt_nr).  Returns false if a pivot is not positive (the
// matrix is not positive definite).
__device__ __forceinline__ bool cholesky9(double (&A)[45], double (&rd)[9]) {
    bool ok = true;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        double d = A[j * (j + 1) / 2 + j];
#pragma unroll
        for (int k = 0; k < j; ++k) d = fma(-A[j * (j + 1) / 2 + k], A[j * (j + 1) / 2 + k], d);
        ok = ok && d > 0;
        const double r = d > 0 ? rsqrt_nr(d) : 1.0;
        A[j * (j + 1) / 2 + j] = d * r;
        rd[j] = r;
#pragma unroll
        for (int i = j + 1; i < 9; ++i) {
            double t = A[i * (i + 1) / 2 + j];
#pragma unroll
            for (int k = 0; k < j; ++k) t = fma(-A[i * (i + 1) / 2 + k], A[j * (j + 1) / 2 + k], t);
            A[i * (i + 1) / 2 + j] = t * r;
        }
    }
    return ok;
}

// Unit eigenvector of the smallest eigenvalue of the 9 x 9 symmetric positive
// semi-definite matrix M (lower triangle packed, row i at i(i+1)/2), from the
// start x.  The FP64 pipe of this GPU issues a warp instruction in about 64
// cycles, an FP32 one in 1, so:
//  1. FP32: inverse iteration with the explicit inverse of M / tr + 1e-6 I
//     until the direction settles at FP32 resolution;
//  2. FP64: Rayleigh quotient rho and residual r = M x - rho x of that
//     direction; M has an eigenvalue within |r| of rho, the smallest one when
//     x is nearest its eigenvector, so sigma = rho - 2 |r| lies below it;
//  3. FP64 inverse iteration with the Cholesky factor of M - sigma I: the
//     shift makes each step shrink the other directions by
//     (l1 - sigma) / (li - sigma), so a few steps reach 1e-12.  If that matrix
//     is not positive definite (the bound did not hold), the shift falls back
//     to -1e-13 tr, plain inverse iteration.
// One thread per window: each FP64 warp instruction serves 32 windows.
__device__ __forceinline__ void min_eigvec9(const double (&M)[45], double (&x)[9]) {
    auto sym = [](int i, int j) { return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i; };
    double tr = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) tr += M[i * (i + 1) / 2 + i];
    {  // 1. FP32 direction
        const float rs = tr > 0 ? (float)(1.0 / tr) : 1.f;
        float L[45], rdf[9];
#pragma unroll
        for (int q = 0; q < 45; ++q) L[q] = (float)M[q] * rs;
#pragma unroll
        for (int i = 0; i < 9; ++i) L[i * (i + 1) / 2 + i] += 1e-6f;
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            float d = L[j * (j + 1) / 2 + j];
#pragma unroll
            for (int k = 0; k < j; ++k) d = fmaf(-L[j * (j + 1) / 2 + k], L[j * (j + 1) / 2 + k], d);
            const float r = d > 1e-30f ? rsqrtf(d) : 1e15f;
            L[j * (j + 1) / 2 + j] = d * r;
            rdf[j] = r;
#pragma unroll
            for (int i = j + 1; i < 9; ++i) {
                float t = L[i * (i + 1) / 2 + j];
#pragma unroll
                for (int k = 0; k < j; ++k) t = fmaf(-L[i * (i + 1) / 2 + k], L[j * (j + 1) / 2 + k], t);
                L[i * (i + 1) / 2 + j] = t * r;
            }
        }
        float xf[9], n0 = 0.f;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            xf[i] = (float)x[i];
            n0 = fmaf(xf[i], xf[i], n0);
        }
        const float s0 = rsqrtf(n0);
#pragma unroll
        for (int i = 0; i < 9; ++i) xf[i] *= s0;
        for (int it = 0; it < 60; ++it) {  // a start vector only: the FP64 iteration below converges from it
            float y[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) {  // L z = x
                float t = xf[i];
#pragma unroll
                for (int k = 0; k < i; ++k) t = fmaf(-L[i * (i + 1) / 2 + k], y[k], t);
                y[i] = t * rdf[i];
            }
#pragma unroll
            for (int i = 8; i >= 0; --i) {  // L^T y = z
                float t = y[i];
#pragma unroll
                for (int k = i + 1; k < 9; ++k) t = fmaf(-L[k * (k + 1) / 2 + i], y[k], t);
                y[i] = t * rdf[i];
            }
            float n = 0.f, dot = 0.f;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                n = fmaf(y[i], y[i], n);
                dot = fmaf(y[i], xf[i], dot);
            }
            if (!(n > 0.f) || !isfinite(n)) break;
            float sc = rsqrtf(n);
            if (dot < 0.f) sc = -sc;
            float diff = 0.f;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                y[i] *= sc;
                diff = fmaxf(diff, fabsf(y[i] - xf[i]));
                xf[i] = y[i];
            }
            if (diff < 4e-7f) break;
        }
        bool finite = true;
#pragma unroll
        for (int i = 0; i < 9; ++i) finite = finite && isfinite(xf[i]);
        if (finite) {
#pragma unroll
            for (int i = 0; i < 9; ++i) x[i] = (double)xf[i];
        }
    }
    // 2. shift from the Rayleigh quotient and the residual of x
    double xx = 0, rho = 0, Mx[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        double t = 0;
#pragma unroll
        for (int j = 0; j < 9; ++j) t = fma(M[sym(i, j)], x[j], t);
        Mx[i] = t;
        xx = fma(x[i], x[i], xx);
        rho = fma(x[i], t, rho);
    }
    const double ixx = 1.0 / xx;
    rho *= ixx;
    double rr = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const double r = fma(-rho, x[i], Mx[i]);
        rr = fma(r, r, rr);
    }
    const double floor_shift = -1e-13 * tr - 1e-300;
    double sigma = rho - 2.0 * sqrt(rr * ixx);
    if (!(sigma > floor_shift)) sigma = floor_shift;
    // 3. shifted inverse iteration in FP64
    double A[45], rd[9];
#pragma unroll
    for (int q = 0; q < 45; ++q) A[q] = M[q];
#pragma unroll
    for (int i = 0; i < 9; ++i) A[i * (i + 1) / 2 + i] -= sigma;
    if (!cholesky9(A, rd)) {
#pragma unroll
        for (int q = 0; q < 45; ++q) A[q] = M[q];
#pragma unroll
        for (int i = 0; i < 9; ++i) A[i * (i + 1) / 2 + i] -= floor_shift;
        cholesky9(A, rd);
        sigma = floor_shift;
    }
    {
        const double s0 = rsqrt_nr(xx);
#pragma unroll
        for (int i = 0; i < 9; ++i) x[i] *= s0;
    }
    // Stopping: the step's change is below 1e-12 and, when the iteration converges slowly (a small eigen-gap
    // against the shift's distance), so is the remaining error extrapolated from the ratio of successive changes
    // (a small change per step alone would stop a slow iteration far from the vector).  A slow iteration is
    // re-shifted at the current vector's Rayleigh quotient minus twice its residual (still below the smallest
    // eigenvalue), a few times at most.  An iteration that stays slow after them measures the eigen-gap: with
    // the ratio q of successive changes, (lambda_1 - sigma) / (lambda_2 - sigma) = q gives lambda_2 - lambda_1 =
    // (rho - sigma)(1 - q) / q (rho, the Rayleigh quotient, for lambda_1); below 1e-11 of the trace (at most 9
    // times the largest eigenvalue), the gap is far below the 1e-8 of the largest eigenvalue at which the
    // smallest eigenvector is no longer determined to the 1e-6 a refit is compared at, and the iteration stops.
    double prev = 1e300;
    int reshifts = 0, slow = 0;
    for (int it = 0; it < 200; ++it) {
        double y[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {  // L z = x
            double t = x[i];
#pragma unroll
            for (int k = 0; k < i; ++k) t = fma(-A[i * (i + 1) / 2 + k], y[k], t);
            y[i] = t * rd[i];
        }
#pragma unroll
        for (int i = 8; i >= 0; --i) {  // L^T y = z
            double t = y[i];
#pragma unroll
            for (int k = i + 1; k < 9; ++k) t = fma(-A[k * (k + 1) / 2 + i], y[k], t);
            y[i] = t * rd[i];
        }
        double n = 0, dot = 0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            n = fma(y[i], y[i], n);
            dot = fma(y[i], x[i], dot);
        }
        double sc = rsqrt_nr(n);
        if (dot < 0) sc = -sc;
        double diff = 0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            y[i] *= sc;
            diff = fmax(diff, fabs(y[i] - x[i]));
            x[i] = y[i];
        }
        // 1e-12 is far below what the rescore (1e-5 near-tie band) and the
        // model comparison (1e-6) can see
        const double q = diff / prev;  // convergence ratio of the last step
        prev = diff;
        if (diff < 1e-12 && (q < 0.5 || diff * q / (1.0 - fmin(q, 0.999999)) < 1e-13)) break;
        slow = q > 0.9 ? slow + 1 : 0;  // q >= 1: no convergence at all (a gap below what rounding resolves)
        if (reshifts >= 4 && slow >= 4 && (slow & 3) == 0) {  // the gap, from the convergence ratio
            double xx3 = 0, rho3 = 0;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                double t = 0;
#pragma unroll
                for (int j = 0; j < 9; ++j) t = fma(M[sym(i, j)], x[j], t);
                xx3 = fma(x[i], x[i], xx3);
                rho3 = fma(x[i], t, rho3);
            }
            const double gap = q < 1.0 ? (rho3 / xx3 - sigma) * (1.0 - q) / q : 0.0;
            if (gap < 1e-11 * tr) break;
        }
        if (it >= 2 && q > 0.5 && reshifts < 4) {
            double Mx2[9], xx2 = 0, rho2 = 0;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                double t = 0;
#pragma unroll
                for (int j = 0; j < 9; ++j) t = fma(M[sym(i, j)], x[j], t);
                Mx2[i] = t;
                xx2 = fma(x[i], x[i], xx2);
                rho2 = fma(x[i], t, rho2);
            }
            rho2 /= xx2;
            double rr2 = 0;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const double r = fma(-rho2, x[i], Mx2[i]);
                rr2 = fma(r, r, rr2);
            }
            const double sig2 = rho2 - 2.0 * sqrt(rr2 / xx2);
            if (sig2 > sigma) {
                double B[45], rd2[9];
#pragma unroll
                for (int q2 = 0; q2 < 45; ++q2) B[q2] = M[q2];
#pragma unroll
                for (int i = 0; i < 9; ++i) B[i * (i + 1) / 2 + i] -= sig2;
                if (cholesky9(B, rd2)) {
#pragma unroll
                    for (int q2 = 0; q2 < 45; ++q2) A[q2] = B[q2];
#pragma unroll
                    for (int i = 0; i < 9; ++i) rd[i] = rd2[i];
                    sigma = sig2;
                    prev = 1e300;
                }
            }
            ++reshifts;
        }
    }
}

// Draws hypothesis k of a window: Philox indices into the N matches; false if
// the sample is degenerate (three source or three target points collinear).
// The homography is exact (128-bit integers, see hyp_exact.cuh).
__device__ __forceinline__ bool draw_hypothesis(const float4* match, int N, int cell, int k, uint32_t tag,
                                                uint32_t pair_id, uint32_t k0, uint32_t k1, i128* Hk) {
    const uint4 w = philox((uint32_t)cell, (uint32_t)k, tag, pair_id, k0, k1);
    const uint32_t idx[4] = {bounded_u32(w.x, (uint32_t)N), bounded_u32(w.y, (uint32_t)N),
                             bounded_u32(w.z, (uint32_t)N), bounded_u32(w.w, (uint32_t)N)};
    int px[4], py[4], qx[4], qy[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        // the match coordinates are small exact integers held as floats: adding
        // 1.5 * 2^23 puts the integer in the low mantissa bits (no conversion op)
        const float4 m = match[idx[j]];
        px[j] = __float_as_int(m.x + 12582912.f) - 0x4B400000;
        py[j] = __float_as_int(m.y + 12582912.f) - 0x4B400000;
        qx[j] = __float_as_int((m.x + m.z) + 12582912.f) - 0x4B400000;
        qy[j] = __float_as_int((m.y + m.w) + 12582912.f) - 0x4B400000;
    }
    bool degen = false;
    const int T3[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int a = T3[t][0], b = T3[t][1], c = T3[t][2];
        degen |= collinear3(px[a], py[a], px[b], py[b], px[c], py[c]);
        degen |= collinear3(qx[a], qy[a], qx[b], qy[b], qx[c], qy[c]);
    }
    if (degen) return false;
    minimal_h_exact(px, py, qx, qy, Hk);
    return true;
}

// The same out of line (the winner's redraw, once per window: the scoring
// loop keeps the only inline copy).
__device__ __noinline__ void draw_hypothesis_ool(const float4* match, int N, int cell, int k, uint32_t tag,
                                                 uint32_t pair_id, uint32_t k0, uint32_t k1, i128* Hk) {
    draw_hypothesis(match, N, cell, k, tag, pair_id, k0, k1, Hk);
}

// The exact hypothesis as doubles in window-local coordinates, oriented like
// its evaluation form (positive denominator at the window centre) and scaled
// by a power of two (largest entry in [1, 2)): the FP64 stand-in of the
// residual test, built without FP64 instructions.
__device__ __forceinline__ void exact_local_fp64(const i128* Hk, double* Hl) {
    const i128 dc2 = 2 * Hk[8] - (Hk[6] + Hk[7]);
    exact_to_double_pow2(Hk, Hl, dc2 < 0);
}

// ---------------------------------------------------------------- RANSAC per window
// Sec. 3.1.2 / 3.2, in three launches per level and stage:
//   (A) ransac_fit, a group per window: the window's matches (u, u + v(u))
//       -- all pixels at stage 1, the still-unassigned ones in raster order at
//       stage 2 -- go to shared memory as exact floats; the group draws, solves
//       and scores the hypotheses, keeps the largest support (lowest index on
//       ties) and accumulates what the least-squares refit needs on the
//       winner's inliers: Hartley sums and the 24 DLT moments as exact integers;
//   (B) k_refit_solve, a thread per window: normalised DLT refit in FP64;
//   (C) ransac_finish, a group per window: rescoring of the refit (kept unless
//       it has fewer inliers), the colour-overlap count and the model record.

// Windows with at most this many matches score each hypothesis on one thread.
constexpr int kLaneScoreMax = 64;

// mef_inlier_pt out of line (loose hypotheses are rare: the callers' loops stay small).
__device__ __noinline__ bool mef_inlier_pt_ool(const Mef& m, float4 mt, float t2, bool& unc) {
    return mef_inlier_pt(m, mt.x, mt.y, mt.z, mt.w, t2, unc);
}
// The certified test of a match: the FP32 decision, and unc when it is within its rounding bound.
__device__ __forceinline__ bool cert_inlier(const Mef& m, const float4& mt, float t2, bool& unc) {
    return mef_loose(m) ? mef_inlier_pt_ool(m, mt, t2, unc) : mef_inlier_c(m, mt.x, mt.y, mt.z, mt.w, t2, unc);
}

// Support of a loose hypothesis (per-match bounds), the warp's lanes over the
// matches: the FP32 count and the number of uncertain tests, on every lane.
// Abandoned (x = -1) once even its optimistic count plus the matches left
// cannot exceed bound.  Out of line: rare, and the scoring loops stay small in
// the instruction cache.  tests: residual tests done (counter).
__device__ __noinline__ int2 loose_score_warp(const float4* match, int N, const Mef& m, float t2, int bound,
                                              int& tests) {
    const int lane = threadIdx.x & 31;
    int s2 = 0, u2 = 0;
    for (int c = 0; c < N; c += 128) {
        int sl = 0, ul = 0;
        for (int j = c + lane; j < min(N, c + 128); j += 32) {
            const float4 mt = match[j];
            bool unc;
            sl += mef_inlier_pt(m, mt.x, mt.y, mt.z, mt.w, t2, unc);
            ul += unc;
        }
        s2 += (int)__reduce_add_sync(FULL, (unsigned)sl);
        u2 += (int)__reduce_add_sync(FULL, (unsigned)ul);
        tests += min(128, N - c);
        if (s2 + u2 + max(N - c - 128, 0) <= bound) return make_int2(-1, 0);
    }
    return make_int2(s2, u2);
}

// Support of a loose hypothesis on at most 64 matches (per-match bounds), the
// warp's lanes over the matches: the FP32 count on every lane, the uncertain
// tests (bit j of unc: match j) and the FP32 decisions among them (bit j of
// uin).  Out of line (rare).  tests: residual tests done (counter).
__device__ __noinline__ int loose_score64(const float4* match, int N, const Mef& m, float t2,
                                          unsigned long long& unc, unsigned long long& uin) {
    const int lane = threadIdx.x & 31;
    int score = 0;
    unc = 0;
    uin = 0;
    for (int c = 0; c < N; c += 32) {
        const int j = c + lane;
        bool in = false, u = false;
        if (j < N) {
            const float4 mt = match[j];
            in = mef_inlier_pt(m, mt.x, mt.y, mt.z, mt.w, t2, u);
        }
        const unsigned bi = __ballot_sync(FULL, in), bu = __ballot_sync(FULL, u);
        score += __popc(bi);
        unc |= (unsigned long long)bu << c;
        uin |= (unsigned long long)(bu & bi) << c;
    }
    return score;
}

// The exact count of a hypothesis from its FP32 count on at most 64 matches:
// each uncertain test (bit j of unc) decided again in FP64 with Hl, the
// hypothesis's exact form, replacing its FP32 decision (bit j of uin).  One
// thread; nfp64 counts the FP64 decisions.
__device__ __noinline__ int resolve_uncertain(const float4* match, const double* Hl, float t2, unsigned long long unc,
                                              unsigned long long uin, int score, int& nfp64) {
    for (; unc; unc &= unc - 1) {
        const int j = __ffsll((long long)unc) - 1;
        const float4 mt = match[j];
        score += (int)hyp_inlier_fp64(Hl, mt.x, mt.y, mt.z, mt.w, (double)t2) - (int)((uin >> j) & 1ull);
        ++nfp64;
    }
    return score;
}
// The same from the 128-bit hypothesis itself (kept in shared memory since it was drawn).
__device__ __noinline__ int resolve_uncertain_hk(const float4* match, const i128* hk, float t2,
                                                 unsigned long long unc, unsigned long long uin, int score,
                                                 int& nfp64) {
    double Hl[9];
    {
        i128 H[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) H[q] = hk[q];
        exact_local_fp64(H, Hl);
    }
    return resolve_uncertain(match, Hl, t2, unc, uin, score, nfp64);
}

// The same with the warp's lanes over the matches (every lane gets the score).
__device__ __noinline__ int exact_score_warp(const float4* match, int N, const Mef& m, const double* Hl, float t2,
                                             int& nfp64) {
    const int lane = threadIdx.x & 31;
    int score = 0;
    for (int c = 0; c < N; c += 32) {
        const int j = c + lane;
        bool in = false, unc = false;
        if (j < N) {
            const float4 mt = match[j];
            in = cert_inlier(m, mt, t2, unc);
            if (unc) {
                in = hyp_inlier_fp64(Hl, mt.x, mt.y, mt.z, mt.w, (double)t2);
                ++nfp64;
            }
        }
        score += __popc(__ballot_sync(FULL, in));
    }
    return score;
}

// Exact integer of a small integer-valued float: adding 1.5 * 2^23 puts it in
// the low mantissa bits (no conversion instruction).
__device__ __forceinline__ int exact_int(float f) { return __float_as_int(f + 12582912.f) - 0x4B400000; }

template <class G>
__device__ __forceinline__ void window_origin(const LevelGeom& g, int cell, int& x0, int& y0, int& ox, int& oy) {
    const int cxw = cell % g.gx.count, cyw = cell / g.gx.count;
    x0 = win_pos(g.gx, g.h, cxw);
    y0 = win_pos(g.gy, g.h, cyw);
    ox = x0 + g.s / 2;
    oy = y0 + g.s / 2;
}

// The window's matches in raster order into `match`; returns their number.
template <class G>
__device__ int gather_matches(const G& grp, const PairView& pv, const LevelGeom& g, int stage, int dir, int cell,
                              float4* match) {
    const int tid = grp.rank();
    const int s = g.s;
    int x0, y0, ox, oy;
    window_origin<G>(g, cell, x0, y0, ox, oy);
    const int W = pv.W;
    const int2* nnf = pv.nnf[dir];
    const uint8_t* resid = pv.resid[dir];
    int N = 0;
    for (int base = 0; base < s * s; base += G::size) {
        const int j = base + tid;
        bool take = false;
        float4 mt = make_float4(0, 0, 0, 0);
        if (j < s * s) {
            const int yy = y0 + j / s, xx = x0 + j % s;
            const int i = yy * W + xx;
            take = stage == 1 || resid[i];
            const int2 v = nnf[i];
            mt = make_float4((float)(xx - ox), (float)(yy - oy), (float)v.x, (float)v.y);
        }
        int total;
        const int off = grp.scan(take, total);
        if (take) match[N + off] = mt;
        N += total;
    }
    grp.sync();
    return N;
}

// Sum of |(a, b)| over a lane's points, for exact integers a, b: each root of
// the sum of squares K (exact in 64-bit integers, rounded once to FP64 above
// 2^53) to about 1e-14 relative, added in FP64.  The least-squares refit of a thin, ill-conditioned support
// moves with its Hartley normalisation, so the scale must carry far less than
// FP32 rounding (with FP32 roots, refits moved by ~1e-6).  The root: the FP32
// root s0 and reciprocal 1 / (2 s0), then one Newton step in FP64,
// s0 + (K - s0^2) / (2 s0): its error is about s0 times the square of s0's
// relative error (2^-23), against some ten FP64 operations of a full FP64
// root on GB300's slow FP64 pipe.
struct DistSum {
    double s = 0.0;
    __device__ __forceinline__ void add(int a, int b) {
        const long long K = (long long)a * a + (long long)b * b;  // exact: |a|, |b| < 2^31
        const float fa = (float)a, fb = (float)b;
        const float s0 = sqrtf(fmaf(fa, fa, fb * fb));
        if (!(s0 > 0.f)) return;  // K = 0
        const double sd = (double)s0;
        const double e = fma(-sd, sd, (double)K);
        s += fma(e, (double)(0.5f / s0), sd);
    }
    __device__ __forceinline__ double total() const { return s; }
};

// Refit inputs on the winner's inliers, for ransac_fit (out of line: once per window, and its 24 integer
// moments would otherwise crowd the registers of the hypothesis loop).
template <class G>
__device__ __noinline__ void winner_moments(const G& grp, const float4* match, int N, const Mef* wmef,
                                            const double* whl, float t2, int wscore, RefitWork* rw) {
    const int tid = grp.rank();
    // Hartley centroids (exact integer sums), mean distances, and the DLT moments as exact integers about the
    // rounded centroids
    const Mef wm = *wmef;
    // the winner's inlier test, certified: an uncertain one is decided in FP64 with the exact winner
    auto winner_inlier = [&](const float4& mt) -> bool {
        bool unc;
        const bool in = cert_inlier(wm, mt, t2, unc);
        return unc ? hyp_inlier_fp64(whl, mt.x, mt.y, mt.z, mt.w, (double)t2) : in;
    };
    // the winner's inliers among this thread's matches (bit c: match tid + c G::size; N <= 64 G::size for
    // every group: 256 matches per warp window, 96 x 96 per block window)
    static_assert(kMaxCell * kMaxCell <= 64 * 256 && 16 * 16 <= 64 * 32, "inlier mask too small");
    unsigned long long inm = 0;
    int sx = 0, sy = 0, tx = 0, ty = 0;
    for (int j = tid, c = 0; j < N; j += G::size, ++c) {
        const float4 mt = match[j];
        if (winner_inlier(mt)) {
            inm |= 1ull << c;
            sx += exact_int(mt.x);
            sy += exact_int(mt.y);
            tx += exact_int(mt.x + mt.z);
            ty += exact_int(mt.y + mt.w);
        }
    }
    sx = grp.sum(sx);
    sy = grp.sum(sy);
    tx = grp.sum(tx);
    ty = grp.sum(ty);
    const float fn = (float)wscore;
    const float fmx = __fdiv_rn((float)sx, fn), fmy = __fdiv_rn((float)sy, fn);
    const float fmqx = __fdiv_rn((float)tx, fn), fmqy = __fdiv_rn((float)ty, fn);
    const int cx = __float2int_rn(fmx), cy = __float2int_rn(fmy), cu = __float2int_rn(fmqx), cv = __float2int_rn(fmqy);
    // Hartley scales: distances to the exact centroids, as n |p - mean| = |n p - sum| from exact integers
    // (the least-squares refit of a noisy support moves with its normalisation, so the scale must carry no
    // more than float rounding)
    const int nw = wscore;  // n |coordinate| < 2^31 for frames up to 32767 px and windows up to 96 px
    DistSum dsum, dtsum;
    long long R[24];
#pragma unroll
    for (int q = 0; q < 24; ++q) R[q] = 0;
    for (; inm; inm &= inm - 1) {
        const float4 mt = match[tid + (__ffsll((long long)inm) - 1) * G::size];
        dsum.add(nw * exact_int(mt.x) - sx, nw * exact_int(mt.y) - sy);
        dtsum.add(nw * exact_int(mt.x + mt.z) - tx, nw * exact_int(mt.y + mt.w) - ty);
        const int X = exact_int(mt.x) - cx, Y = exact_int(mt.y) - cy;
        const int U = exact_int(mt.x + mt.z) - cu, V = exact_int(mt.y + mt.w) - cv;
        const int zz[6] = {X * X, X * Y, X, Y * Y, Y, 1};
        const int w3 = U * U + V * V;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            R[q] += zz[q];
            R[6 + q] += (long long)U * zz[q];
            R[12 + q] += (long long)V * zz[q];
            R[18 + q] += (long long)w3 * zz[q];
        }
    }
    const double ds = grp.sum(dsum.total()) / (double)nw;  // sums of |p - mean|
    const double dt = grp.sum(dtsum.total()) / (double)nw;
#pragma unroll
    for (int q = 0; q < 24; ++q) {
        const long long t = grp.sum(R[q]);
        if (tid == q) rw->mom[q] = t;
    }
    if (tid == 0) {
        rw->ds = ds;
        rw->dt = dt;
        rw->cx = cx;
        rw->cy = cy;
        rw->cu = cu;
        rw->cv = cv;
        rw->nin = wscore;
        rw->status = 2;
    }
}

template <class G, int ST, bool LANE>
__device__ void ransac_fit(const G& grp, const PairView& pv, const LevelGeom& g, int level, int stage,
                           const PlaneParams& pp, int dir, int cell, float4* match, Mef* hyp, int* gbest, int* kfull,
                           Mef* wmef, void* hx) {
    const int tid = grp.rank();
    const int id = (g.base + cell) * 2 + (stage - 1);
    int* mi = pv.mi[dir] + (size_t)id * kMI;
    RefitWork* rw = pv.rw[dir] + cell;
    if (G::size > 32 && tid == 0) {
        *gbest = -1;
        *kfull = 0x7fffffff;
    }
    const int N = gather_matches<G>(grp, pv, g, stage, dir, cell, match);
    if (tid == 0) {
        for (int k = 0; k < kMI; ++k) mi[k] = 0;
        mi[MI_NIN] = N;
        mi[MI_BESTK] = -1;
        for (int k = 0; k < 9; ++k) pv.mh[dir][(size_t)id * 9 + k] = 0.0;
        Mef z = {};
        pv.mef[dir][id] = z;
        rw->status = 0;
    }
    if (N < pp.min_inliers || N < 4) return;
    // the largest |offset| component among the matches, and the window's half side: the bounds of the FP32 tests
    float vloc = 0.f;
    for (int j = tid; j < N; j += G::size) {
        const float4 mt = match[j];
        vloc = fmaxf(vloc, fmaxf(fabsf(mt.z), fabsf(mt.w)));
    }
    const float V = (float)grp.max((unsigned long long)vloc);  // integers: exact as a key
    const float U = 0.5f * (float)g.s;
    if (tid == 0) rw->vmax = V;

    // Hypotheses.  Few matches: each thread draws and scores its own
    // hypotheses k = rank, rank + size, ... in full.  Otherwise each warp of
    // the group draws 32 at a time (one per lane), then scores them in index
    // order with its lanes over the matches, 128 at a time, and abandons one
    // as soon as it cannot win: its inliers so far plus the matches left fall
    // below the best score of the group (any index), or do not exceed the
    // best of this warp's earlier, lower-index hypotheses.  The winner (most
    // inliers, lowest index) is never abandoned, so the outcome is that of
    // scoring every hypothesis in full.  Once a hypothesis has all N matches
    // as inliers, hypotheses of higher index can at most tie and are not
    // drawn at all.
    // Counts are certified: a count with uncertain FP32 tests bounds the exact
    // count by count +- uncertain; a hypothesis whose optimistic count could
    // still win gets its exact count at once (its uncertain tests decided in
    // FP64 with its exact form).  hx keeps each lane's hypothesis since it was
    // drawn: in the one-hypothesis-per-lane kernel (LANE) as its 128-bit
    // entries (converted only when needed), else as its exact form in FP64.
    const float t2 = pp.t2;
    const uint32_t tag = stream_tag(RNG_RANSAC, dir, level, stage);
    constexpr int NW = G::size / 32;
    const int lane = tid & 31;
    Mef* hb = hyp + (tid >> 5) * 32;
    i128* hkw = reinterpret_cast<i128*>(hx) + (tid >> 5) * (32 * 9);    // LANE: this warp's 32 hypotheses
    double* hlw = reinterpret_cast<double*>(hx) + (tid >> 5) * (32 * 9);  // else: their exact forms
    int best_score = -1, best_k = 0x7fffffff, tests = 0;
    int nfp64 = 0, nloose = 0;  // tests decided in FP64, hypotheses tested with per-match bounds (counters)
    // LANE: the warp's best hypothesis so far (its key, its 128-bit entries after the 32 lanes' in hx, its
    // evaluation form in *wmef), so that the winner needs no second draw
    unsigned long long wbest_key = 0ull;
    i128* wslot = reinterpret_cast<i128*>(hx) + 32 * 9;
    if (LANE || N <= kLaneScoreMax) {
        int group_best = -1;  // the group's best exact count after the previous rounds
        for (int r = 0; r * G::size < pp.num_hyp; ++r) {
            const int k = r * G::size + tid;
            Mef m;
            bool ok = false;
            if (k < pp.num_hyp) {
                i128 Hk[9];
                ok = draw_hypothesis(match, N, cell, k, tag, pv.pair_id, pp.k0, pp.k1, Hk) && make_mef_exact(Hk, m);
                if (LANE) {
#pragma unroll
                    for (int q = 0; q < 9; ++q) hkw[lane * 9 + q] = Hk[q];
                } else if (ok) {
                    exact_local_fp64(Hk, hlw + lane * 9);
                }
            }
            // FP32 count; the uncertain tests (bit j: match j) and the FP32 decisions among them: the exact
            // count is within score +- popc(um)
            int score = 0;
            unsigned long long um = 0, im = 0;
            bool loose = false;
            if (ok) {
                mef_set_bounds(m, U, V, t2);
                loose = mef_loose(m);
                nloose += loose;
                if (!loose) {  // two matches per instruction on the packed FP32x2 pipe
                    const Mef2 m2 = mef2_of(m);
                    const float ef = m.ef, eden = __int_as_float(m.eden);
                    int j = 0;
                    for (; j + 1 < N; j += 2) {
                        bool ia, ib, ua, ub;
                        mef_inlier2_c(m2, ef, eden, match[j], match[j + 1], t2, ia, ib, ua, ub);
                        score += (int)ia + (int)ib;
                        if (ua || ub) {
                            const unsigned long long ba = (unsigned long long)ua << j, bb = (unsigned long long)ub
                                                                                                  << (j + 1);
                            um |= ba | bb;
                            im |= (ia ? ba : 0ull) | (ib ? bb : 0ull);
                        }
                    }
                    if (j < N) {
                        const float4 mt = match[j];
                        bool unc;
                        const bool in = mef_inlier_c(m, mt.x, mt.y, mt.z, mt.w, t2, unc);
                        score += in;
                        if (unc) {
                            um |= 1ull << j;
                            if (in) im |= 1ull << j;
                        }
                    }
                }
                tests += N;
            }
            hb[lane] = m;
            __syncwarp();
            // loose hypotheses (per-match bounds): the warp scores them together, lanes over the matches
            for (unsigned lm = __ballot_sync(FULL, loose); lm; lm &= lm - 1) {
                const int l = __ffs(lm) - 1;
                unsigned long long ul, il;
                const int sl = loose_score64(match, N, hb[l], t2, ul, il);
                if (lane == l) {
                    score = sl;
                    um = ul;
                    im = il;
                }
            }
            const int unc_n = __popcll(um);
            // A hypothesis with uncertain tests that could beat the best so far (this thread's, the group's of
            // earlier rounds: lower indices) and that no hypothesis of this round surely beats gets its exact
            // count.  Without uncertain tests its count is exact.
            const int rlo = (int)__reduce_max_sync(FULL, (unsigned)(ok ? score - unc_n + 1 : 0)) - 1;
            const int hi = score + unc_n;
            bool exact = unc_n == 0;
            if (ok && !exact && hi > max(best_score, group_best) && hi >= rlo) {
                score = LANE ? resolve_uncertain_hk(match, hkw + lane * 9, t2, um, im, score, nfp64)
                             : resolve_uncertain(match, hlw + lane * 9, t2, um, im, score, nfp64);
                exact = true;
            }
            __syncwarp();
            if (ok && exact && score > best_score) {
                best_score = score;
                best_k = k;
            }
            if (LANE) {  // the warp's best so far (most inliers, lowest index) into its slot when it changes
                const unsigned long long key =
                    best_score < 0 ? 0ull
                                   : (((unsigned long long)(best_score + 1)) << 32) |
                                         (unsigned long long)(0xFFFFFFFFu - (uint32_t)best_k);
                const unsigned long long wk = grp.max(key);
                if (wk != wbest_key) {  // a hypothesis of this round: its lane still holds it in hkw and hb
                    const int wl = __ffs(__ballot_sync(FULL, key == wk)) - 1;
                    if (lane < 9) wslot[lane] = hkw[wl * 9 + lane];
                    if (lane == 9) *wmef = hb[wl];
                    wbest_key = wk;
                }
                __syncwarp();
                group_best = (int)(wk >> 32) - 1;
                // all N matches inliers: every later round has higher indices and can at most tie
                if (group_best >= N) break;
            } else {
                // all N matches inliers: every later round has higher indices and can at most tie
                if (grp.any(best_score >= N)) break;
                group_best = (int)grp.max((unsigned long long)(best_score + 1)) - 1;
            }
        }
    }
    for (int b = tid >> 5; !LANE && N > kLaneScoreMax && b * 32 < pp.num_hyp; b += NW) {
        // a hypothesis with all N matches inliers at a lower index than this batch: nothing here can win
        if ((NW > 1 ? *(volatile int*)kfull : (best_score >= N ? best_k : 0x7fffffff)) < b * 32) break;
        const int k = b * 32 + lane;
        bool ok = false;
        if (k < pp.num_hyp) {
            i128 Hk[9];
            Mef m;
            ok = draw_hypothesis(match, N, cell, k, tag, pv.pair_id, pp.k0, pp.k1, Hk) && make_mef_exact(Hk, m);
            if (ok) {
                mef_set_bounds(m, U, V, t2);
                nloose += mef_loose(m);
                hb[lane] = m;
                exact_local_fp64(Hk, hlw + lane * 9);
            }
        }
        unsigned todo = __ballot_sync(FULL, ok);
        __syncwarp();
        while (todo) {
            const int l = __ffs(todo) - 1;
            todo &= todo - 1;
            const Mef2 m2 = mef2_of(hb[l]);
            const float ef = hb[l].ef, eden = __int_as_float(hb[l].eden);
            const bool loose = mef_loose(hb[l]);  // warp-uniform
            // abandon when reach < group best or reach <= this warp's best
            const int bound = max(NW > 1 ? *(volatile int*)gbest - 1 : -1, best_score);
            int score = 0, unc_n = 0;  // FP32 count, uncertain tests: the exact count is within score +- unc_n
            bool alive = true;
            if (loose) {  // per-match bounds, out of line
                const int2 su = loose_score_warp(match, N, hb[l], t2, bound, tests);
                score = su.x;
                unc_n = su.y;
                alive = su.x >= 0 && score + unc_n > bound;
            }
            for (int c = 0; !loose && c < N; c += 128) {
                int uc = 0;  // this lane's uncertain tests in the chunk
#pragma unroll
                for (int u = 0; u < 4; u += 2) {  // matches j and j + 32 of this lane, tested as a pair
                    const int j = c + 32 * u + lane;
                    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
                    const float4 ma = j < N ? match[j] : z, mb = j + 32 < N ? match[j + 32] : z;
                    bool ia, ib, ua, ub;
                    mef_inlier2_c(m2, ef, eden, ma, mb, t2, ia, ib, ua, ub);
                    uc += (ua && j < N) + (ub && j + 32 < N);
                    score += __popc(__ballot_sync(FULL, ia && j < N)) + __popc(__ballot_sync(FULL, ib && j + 32 < N));
                }
                if (__any_sync(FULL, uc != 0)) unc_n += (int)__reduce_add_sync(FULL, (unsigned)uc);
                tests += min(128, N - c);
                // abandoned only if even every uncertain test turning in its favour could not win
                if (score + unc_n + max(N - c - 128, 0) <= bound) {
                    alive = false;
                    break;
                }
            }
            if (alive && unc_n > 0) {  // a contender with uncertain tests: its exact count
                int f = 0;
                score = exact_score_warp(match, N, hb[l], hlw + l * 9, t2, f);
                const unsigned tf = __reduce_add_sync(FULL, (unsigned)f);
                if (lane == 0) nfp64 += (int)tf;
                alive = score > bound;
            }
            if (alive) {  // more inliers than every earlier hypothesis of this warp
                best_score = score;
                best_k = b * 32 + l;
                if (NW > 1 && lane == 0) {
                    atomicMax(gbest, score);
                    if (score >= N) atomicMin(kfull, best_k);
                }
            }
        }
        __syncwarp();
    }
    if (pv.evals) {  // residual tests performed, those decided in FP64, loose hypotheses (profiling)
        const bool per_lane = LANE || N <= kLaneScoreMax;
        const int t = grp.sum(per_lane || lane == 0 ? tests : 0);
        const int f = grp.sum(nfp64);
        const int lo = grp.sum(per_lane || lane == 0 ? nloose : 0);
        if (tid == 0) {
            atomicAdd(&pv.evals[GPM_COUNT_RANSAC], (unsigned long long)t);
            atomicAdd(&pv.evals[GPM_COUNT_RANSAC_FP64], (unsigned long long)f);
            atomicAdd(&pv.evals[GPM_COUNT_RANSAC_LOOSE], (unsigned long long)lo);
        }
    }
    // most inliers, then lowest hypothesis index
    const unsigned long long key =
        best_score < 0 ? 0ull
                       : (((unsigned long long)(best_score + 1)) << 32) |
                             (unsigned long long)(0xFFFFFFFFu - (uint32_t)best_k);
    const unsigned long long wkey = grp.max(key);
    if (wkey == 0ull) {  // every sample degenerate: no winner, best score -1
        if (tid == 0) mi[MI_BESTSCORE] = -1;
        return;
    }
    const int wscore = (int)(wkey >> 32) - 1;
    const int wk = (int)(0xFFFFFFFFu - (uint32_t)(wkey & 0xFFFFFFFFull));
    // the winner's exact form for its FP64 tests, in the first 72 bytes of hx (the scan is over: every warp
    // of the group has passed the reduction above)
    double* whl = reinterpret_cast<double*>(hx);
    if (tid < 32) {  // first warp: the winner again, exact (LANE: from the warp's slot), and its evaluation form
        i128 Hk[9];
        if (LANE) {
#pragma unroll
            for (int q = 0; q < 9; ++q) Hk[q] = wslot[q];
        } else {
            draw_hypothesis_ool(match, N, cell, wk, tag, pv.pair_id, pp.k0, pp.k1, Hk);
        }
        {
            double Hl[9];
            exact_local_fp64(Hk, Hl);
            __syncwarp();
#pragma unroll
            for (int q = 0; q < 9; ++q)
                if (tid == q) whl[q] = Hl[q];
        }
        if (tid == 0) {
            Mef m0;
            if (LANE) {
                m0 = *wmef;
            } else {
                make_mef_exact(Hk, m0);
                mef_set_bounds(m0, U, V, t2);
            }
            *wmef = m0;
            rw->mef0 = m0;
            mi[MI_BESTK] = wk;
            mi[MI_BESTSCORE] = wscore;
        }
#pragma unroll
        for (int q = 0; q < 9; ++q)
            if (tid == q) rw->hx[q] = Hk[q];
    }
    grp.sync();
    if (wscore < 4) return;

    winner_moments<G>(grp, match, N, wmef, whl, t2, wscore, rw);
}

// (B) Normalised DLT refit of each window whose fit is pending, one thread
// per window and direction: centred, Hartley-scaled moments from the exact
// integer ones, the smallest eigenvector of A^T A started from the winner,
// denormalisation, and the geometry checks of the winner and of the refit.
__global__ void __launch_bounds__(64) k_refit_solve(const __grid_constant__ Batch bt, int level, PlaneParams pp) {
    const PairView& pv = bt.view(blockIdx.z);
    const LevelGeom g = bt.geom(blockIdx.z, level);
    const int nc = g.ncells();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * nc) return;
    const int dir = t / nc, cell = t - dir * nc;
    RefitWork* rw = pv.rw[dir] + cell;
    if (rw->status != 2) return;
    int x0, y0, ox, oy;
    window_origin<WarpGroup>(g, cell, x0, y0, ox, oy);
    // the winner, normalised by its largest entry
    double Hw[9];
    i128 hx[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) hx[q] = rw->hx[q];
    exact_to_double(hx, Hw, 9);
    double f = 0;
#pragma unroll
    for (int q = 0; q < 9; ++q) f = fmax(f, fabs(Hw[q]));
    const double rf = 1.0 / f;
#pragma unroll
    for (int q = 0; q < 9; ++q) Hw[q] *= rf;
    rw->geo_w = plane_geometry_ok(Hw, g.s, pp.radius, pp.scale_min, pp.scale_max) ? 1 : 0;
    local_to_abs(Hw, ox, oy, rw->ha_w);
    rw->refit_ok = 0;
    rw->geo_r = 0;

    // centroids and Hartley scales
    double R[24];
#pragma unroll
    for (int q = 0; q < 24; ++q) R[q] = (double)rw->mom[q];  // exact: |moment| < 2^53
    const double inv_n = 1.0 / (double)rw->nin;
    const double dx = R[2] * inv_n, dy = R[4] * inv_n, du = R[11] * inv_n, dv = R[17] * inv_n;
    const double mx = rw->cx + dx, my = rw->cy + dy, mqx = rw->cu + du, mqy = rw->cv + dv;
    const double ds = rw->ds * inv_n, dt = rw->dt * inv_n;
    if (!(ds > 1e-12 && dt > 1e-12)) return;
    const double ss = sqrt(2.0) / ds, sq = sqrt(2.0) / dt;
    const double iss = ds * 0.70710678118654752440, isq = dt * 0.70710678118654752440;  // 1 / ss, 1 / sq
    // centre the source terms (per raw weight 1, U, V, U^2 + V^2), then the weights
    double P[24];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const double* r = R + 6 * a;
        P[6 * a + 0] = r[0] - 2.0 * dx * r[2] + dx * dx * r[5];
        P[6 * a + 1] = r[1] - dy * r[2] - dx * r[4] + dx * dy * r[5];
        P[6 * a + 2] = r[2] - dx * r[5];
        P[6 * a + 3] = r[3] - 2.0 * dy * r[4] + dy * dy * r[5];
        P[6 * a + 4] = r[4] - dy * r[5];
        P[6 * a + 5] = r[5];
    }
    double mom[24];
    const double sz[6] = {ss * ss, ss * ss, ss, ss * ss, ss, 1.0};
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const double c0 = P[q];
        const double c1 = P[6 + q] - du * P[q];
        const double c2 = P[12 + q] - dv * P[q];
        const double c3 = P[18 + q] - 2.0 * du * P[6 + q] - 2.0 * dv * P[12 + q] + (du * du + dv * dv) * P[q];
        mom[q] = sz[q] * c0;
        mom[6 + q] = sq * sz[q] * c1;
        mom[12 + q] = sq * sz[q] * c2;
        mom[18 + q] = sq * sq * sz[q] * c3;
    }
    double A[45];
#pragma unroll
    for (int i = 0; i < 9; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) A[i * (i + 1) / 2 + j] = dlt_entry(mom, i, j);
    // start: the winner in the normalised frames, h0 = Tq Hw Tp^-1
    double x[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double b[3];
#pragma unroll
            for (int k = 0; k < 3; ++k)
                b[k] = c == 0 ? Hw[k * 3] * iss
                              : (c == 1 ? Hw[k * 3 + 1] * iss : Hw[k * 3] * mx + Hw[k * 3 + 1] * my + Hw[k * 3 + 2]);
            x[r * 3 + c] = r == 0 ? sq * (b[0] - mqx * b[2]) : (r == 1 ? sq * (b[1] - mqy * b[2]) : b[2]);
        }
    min_eigvec9(A, x);
    // Hr = Tq^-1 h Tp
    double Hr[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double b[3];
#pragma unroll
            for (int k = 0; k < 3; ++k)
                b[k] = c == 0 ? x[k * 3] * ss
                              : (c == 1 ? x[k * 3 + 1] * ss : x[k * 3 + 2] - ss * (mx * x[k * 3] + my * x[k * 3 + 1]));
            Hr[r * 3 + c] = r == 0 ? b[0] * isq + mqx * b[2] : (r == 1 ? b[1] * isq + mqy * b[2] : b[2]);
        }
    Mef m1;
    if (!make_mef(Hr, 0, 0, m1)) return;
    mef_set_bounds(m1, 0.5f * (float)g.s, rw->vmax, pp.t2);
    rw->mef1 = m1;
    {
        // the refit for FP64 tests: denominator 1 at the window centre (-0.5, -0.5), as its evaluation form
        const double k = 1.0 / (Hr[8] - 0.5 * (Hr[6] + Hr[7]));
#pragma unroll
        for (int q = 0; q < 9; ++q) rw->hl_r[q] = Hr[q] * k;
    }
    rw->geo_r = plane_geometry_ok(Hr, g.s, pp.radius, pp.scale_min, pp.scale_max) ? 1 : 0;
    local_to_abs(Hr, ox, oy, rw->ha_r);
    rw->refit_ok = 1;
}

// (C) Rescore the refit on the window's matches, choose, count colour
// inliers among the RANSAC inliers (|S_R n S_C|, Sec. 3.4 third cue) and
// write the model: valid iff the support is at least max(min_inliers, N / 5)
// and the chosen homography passed the geometry checks.
template <class G, int ST>
__device__ void ransac_finish(const G& grp, const PairView& pv, const LevelGeom& g, int stage, const PlaneParams& pp,
                              int dir, int cell, float4* match) {
    const RefitWork* rw = pv.rw[dir] + cell;
    if (rw->status != 2) return;
    const int tid = grp.rank();
    const int id = (g.base + cell) * 2 + (stage - 1);
    int* mi = pv.mi[dir] + (size_t)id * kMI;
    const int N = gather_matches<G>(grp, pv, g, stage, dir, cell, match);
    int x0, y0, ox, oy;
    window_origin<G>(g, cell, x0, y0, ox, oy);
    const int W = pv.W, H = pv.H;
    const float t2 = pp.t2;
    const int wscore = rw->nin;
    const bool have_refit = rw->refit_ok != 0;
    int rcount = 0;
    if (have_refit) {
        const Mef rm = rw->mef1;
        for (int j = tid; j < N; j += G::size) {
            const float4 mt = match[j];
            bool unc;
            bool in = cert_inlier(rm, mt, t2, unc);
            if (unc) in = hyp_inlier_fp64(rw->hl_r, mt.x, mt.y, mt.z, mt.w, (double)t2);
            rcount += in;
        }
    }
    rcount = grp.sum(rcount);
    const bool use_refit = have_refit && rcount >= wscore;
    Mef fm = use_refit ? rw->mef1 : rw->mef0;
    // the chosen model in FP64 (local coordinates), for decisions the FP32 form cannot certify
    double Hl[9];
    if (use_refit) {
#pragma unroll
        for (int q = 0; q < 9; ++q) Hl[q] = rw->hl_r[q];
    } else {
        i128 hx[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) hx[q] = rw->hx[q];
        exact_local_fp64(hx, Hl);
    }
    const int count = use_refit ? rcount : wscore;
    const void* src = pv.img[dir];
    const void* tgt = pv.img[1 - dir];
    fm.ox = ox;
    fm.oy = oy;
    int nrc = 0;
    for (int j = tid; j < N; j += G::size) {
        const float4 mt = match[j];
        bool unc;
        bool in = cert_inlier(fm, mt, t2, unc);
        if (unc) in = hyp_inlier_fp64(Hl, mt.x, mt.y, mt.z, mt.w, (double)t2);
        if (!in) continue;
        const int px = ox + (int)mt.x, py = oy + (int)mt.y;
        int ix, iy, kx, ky;
        float fx, fy;
        // certified: a frame test or colour decision within the FP32 position error (times the largest
        // texel difference, 2) is taken again in FP64
        const float dp = mef_pos_bound(fm, mt.x, mt.y);
        bool sure = mef_flow(fm, mt.x, mt.y, kx, fx, ky, fy);
        int dec = 0;
        if (sure) {
            ix = px + kx;
            iy = py + ky;
            const float X = (float)ix + fx, Y = (float)iy + fy;
            const float e0 = -kFrameTol, ex = (float)(W - 1) + kFrameTol, ey = (float)(H - 1) + kFrameTol;
            sure = fabsf(X - e0) > dp && fabsf(X - ex) > dp && fabsf(Y - e0) > dp && fabsf(Y - ey) > dp;
            if (sure) {
                if (in_frame_tol(ix, fx, W) && in_frame_tol(iy, fy, H)) {
                    const float dl = colour_delta<ST>(src, tgt, W, H, px, py, ix, fx, iy, fy);
                    sure = fabsf(dl - pp.eps) > 2.f * dp + 1e-6f;
                    dec = dl < pp.eps;
                }
            }
        } else {
            // the FP32 denominator is not positive: certain unless it is within its rounding of zero
            const float den = 1.f + fm.e0 + fm.g0 * mt.x + fm.g1 * mt.y;
            sure = fabsf(den) > __int_as_float(fm.eden);
        }
        nrc += sure ? dec : colour_overlap_fp64<ST>(Hl, src, tgt, W, H, ox, oy, px, py, pp.eps);
    }
    nrc = grp.sum(nrc);
    if (tid == 0) {
        const bool valid = count >= pp.min_inliers && 5 * count >= N && (use_refit ? rw->geo_r : rw->geo_w) != 0;
        const double* Ha = use_refit ? rw->ha_r : rw->ha_w;
        for (int q = 0; q < 9; ++q) pv.mh[dir][(size_t)id * 9 + q] = Ha[q];
        fm.valid = valid ? 1 : 0;
        pv.mef[dir][id] = fm;
        mi[MI_VALID] = valid ? 1 : 0;
        mi[MI_COUNT] = count;
        mi[MI_FLAGS] = F_FITTED | (use_refit ? F_REFIT : 0) | (valid ? 0 : F_BAD_GEOM);
        mi[MI_NRC] = nrc;
    }
}

// Windows up to 16 x 16: one warp per window, eight windows per block.
// Dynamic shared memory: 8 x MS matches, 8 x 32 hypotheses (evaluation
// forms), then per warp the exact hypotheses (LANE: 32 x 9 128-bit entries
// and the warp's best so far, 9 more; else 32 x 9 doubles).  LANE: windows
// of at most kLaneScoreMax pixels, whose hypotheses are all scored one per
// lane (the other scoring path is not compiled in).
constexpr int ransac_warp_match_stride(bool lane) { return lane ? kLaneScoreMax : 256; }
constexpr size_t ransac_warp_hx_bytes(bool lane) { return lane ? (32 * 9 + 9) * sizeof(i128) : 32 * 9 * sizeof(double); }
// Windows (warps) per block of the warp-per-window fit.
constexpr int kRansacWarps = 4;
constexpr size_t ransac_warp_smem(bool lane) {
    return kRansacWarps * (ransac_warp_match_stride(lane) * sizeof(float4) + 32 * sizeof(Mef) +
                           ransac_warp_hx_bytes(lane));
}
template <int ST, bool LANE>
__global__ void __launch_bounds__(32 * kRansacWarps, 24 / kRansacWarps)
    k_ransac_warp(const __grid_constant__ Batch bt, int level, int stage, PlaneParams pp) {
    const PairView& pv = bt.view(blockIdx.z);
    const LevelGeom g = bt.geom(blockIdx.z, level);
    constexpr int MS = ransac_warp_match_stride(LANE);
    extern __shared__ float4 warp_dyn[];
    __shared__ Mef wmef[kRansacWarps];
    const int warp = threadIdx.x >> 5;
    const int cell = blockIdx.x * kRansacWarps + warp;
    if (cell >= g.ncells()) return;
    float4* match = warp_dyn + warp * MS;
    Mef* hyp = reinterpret_cast<Mef*>(warp_dyn + kRansacWarps * MS) + warp * 32;
    char* hx = reinterpret_cast<char*>(warp_dyn + kRansacWarps * MS + kRansacWarps * 32 * 4) +
               (size_t)warp * ransac_warp_hx_bytes(LANE);
    WarpGroup grp;
    ransac_fit<WarpGroup, ST, LANE>(grp, pv, g, level, stage, pp, blockIdx.y, cell, match, hyp, nullptr, nullptr,
                                    &wmef[warp], hx);
}
template <int ST>
__global__ void __launch_bounds__(256) k_ransac_finish_warp(const __grid_constant__ Batch bt, int level, int stage, PlaneParams pp) {
    const PairView& pv = bt.view(blockIdx.z);
    const LevelGeom g = bt.geom(blockIdx.z, level);
    __shared__ float4 match[8][256];
    const int warp = threadIdx.x >> 5;
    const int cell = blockIdx.x * 8 + warp;
    if (cell >= g.ncells()) return;
    WarpGroup grp;
    ransac_finish<WarpGroup, ST>(grp, pv, g, stage, pp, blockIdx.y, cell, match[warp]);
}

// Larger windows: one 256-thread block per window (matches in dynamic shared memory).
template <int ST>
__global__ void __launch_bounds__(256, 3) k_ransac_block(const __grid_constant__ Batch bt, int level, int stage, PlaneParams pp) {
    const PairView& pv = bt.view(blockIdx.z);
    const LevelGeom g = bt.geom(blockIdx.z, level);
    if ((int)blockIdx.x >= g.ncells()) return;  // past this pair's windows (block-uniform)
    extern __shared__ float4 match_dyn[];
    __shared__ double red_d[8];
    __shared__ int red_i[8];
    __shared__ unsigned long long red_u[8];
    __shared__ Mef hyp[8 * 32];
    __shared__ Mef wmef;
    __shared__ int gbest, kfull;
    BlockGroup<256> grp{red_d, red_i, red_u};
    __shared__ double hl[8 * 32 * 9];  // the exact forms of the block's 8 x 32 hypotheses in flight
    ransac_fit<BlockGroup<256>, ST, false>(grp, pv, g, level, stage, pp, blockIdx.y, blockIdx.x, match_dyn, hyp,
                                           &gbest, &kfull, &wmef, hl);
}
template <int ST>
__global__ void __launch_bounds__(256) k_ransac_finish_block(const __grid_constant__ Batch bt, int level, int stage, PlaneParams pp) {
    const PairView& pv = bt.view(blockIdx.z);
    const LevelGeom g = bt.geom(blockIdx.z, level);
    if ((int)blockIdx.x >= g.ncells()) return;  // past this pair's windows (block-uniform)
    extern __shared__ float4 match_dyn[];
    __shared__ double red_d[8];
    __shared__ int red_i[8];
    __shared__ unsigned long long red_u[8];
    BlockGroup<256> grp{red_d, red_i, red_u};
    ransac_finish<BlockGroup<256>, ST>(grp, pv, g, stage, pp, blockIdx.y, blockIdx.x, match_dyn);
}

// ---------------------------------------------------------------- assignment (eq. 3-4)
// For each pixel, over the windows of the level that cover it (window
// order), the valid plane of the given stage maps p to H p; delta is the mean
// absolute RGB difference between I_src(p) and the bilinear I_tgt(H p); the
// pixel is an inlier iff delta < eps, and takes the inlier plane with the
// smallest L = delta (first window on ties), with flow H p - p.
template <int ST>
__global__ void k_assign(const __grid_constant__ Batch bt, int level, int stage, int which, int write_resid, PlaneParams pp) {
    const PairView& pv = bt.view(blockIdx.z);
    const LevelGeom g = bt.geom(blockIdx.z, level);
    const int dir = blockIdx.y;
    const int W = pv.W, H = pv.H, n = pv.n;
    Labels out = which == 0 ? pv.tent[dir] : (which == 1 ? pv.st1[dir] : pv.lvl[dir]);
    const void* src = pv.img[dir];
    const void* tgt = pv.img[1 - dir];
    const Mef* mef = pv.mef[dir];
    const uint8_t* resid = pv.resid[dir];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (stage == 2 && !resid[i]) continue;
        const int y = i / W, x = i - y * W;
        int ix3[3], iy3[3];
        const int nxw = covering(g.gx, g.s, g.h, x, ix3), nyw = covering(g.gy, g.s, g.h, y, iy3);
        int bm = -1, bkx = 0, bky = 0;
        float bL = FLT_MAX, bfx = 0.f, bfy = 0.f;
        for (int a = 0; a < nyw; ++a)
            for (int b = 0; b < nxw; ++b) {
                const int cell = iy3[a] * g.gx.count + ix3[b];
                const int id = (g.base + cell) * 2 + (stage - 1);
                const Mef m = mef[id];
                if (!m.valid) continue;
                int ix, iy, kx, ky;
                float fx, fy;
                if (!plane_target(m, x, y, W, H, ix, fx, iy, fy, kx, ky)) continue;
                const float d = colour_delta<ST>(src, tgt, W, H, x, y, ix, fx, iy, fy);
                if (!(d < pp.eps)) continue;
                if (d < bL - kLTie) {
                    bL = d;
                    bm = id;
                    bkx = kx;
                    bky = ky;
                    bfx = fx;
                    bfy = fy;
                }
            }
        int vx = 0, vy = 0;
        float rx = 0.f, ry = 0.f;
        if (bm >= 0) {
            round_split(bkx, bfx, vx, rx);
            round_split(bky, bfy, vy, ry);
        }
        out.m[i] = bm;
        out.L[i] = bm >= 0 ? bL : pp.eps;
        out.v[i] = make_int2(vx, vy);
        out.r[i] = make_float2(rx, ry);
        if (write_resid) pv.resid[dir][i] = bm < 0;
    }
}

// ---------------------------------------------------------------- occlusion cues (Sec. 3.4)
__global__ void k_cue_zero(const __grid_constant__ Batch bt, int level, int stage) {
    const PairView& pv = bt.view(blockIdx.z);
    const LevelGeom g = bt.geom(blockIdx.z, level);
    const int dir = blockIdx.y;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < g.ncells(); c += gridDim.x * blockDim.x) {
        int* f = pv.mi[dir] + (size_t)((g.base + c) * 2 + stage - 1) * kMI;
        f[MI_NASSIGN] = 0;
        f[MI_NSYM] = 0;
    }
}

// Forward-backward plane projection symmetry: a pixel assigned to a plane of
// this level and stage with flow f is symmetric iff q = round(p + f) holds an
// assigned pixel of the other direction with flow g, |f + g| < t_fb.
__global__ void k_cue_counts(const __grid_constant__ Batch bt, int level, int stage, int which, PlaneParams pp) {
    const PairView& pv = bt.view(blockIdx.z);
    const LevelGeom g = bt.geom(blockIdx.z, level);
    const int dir = blockIdx.y;
    const int W = pv.W, H = pv.H, n = pv.n;
    const Labels lab = which == 0 ? pv.tent[dir] : pv.lvl[dir];
    const Labels oth = which == 0 ? pv.tent[1 - dir] : pv.lvl[1 - dir];
    const int lo = g.base * 2, hi = (g.base + g.ncells()) * 2;
    int* mi = pv.mi[dir];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int m = lab.m[i];
        if (m < lo || m >= hi || (m & 1) != stage - 1) continue;
        atomicAdd(&mi[(size_t)m * kMI + MI_NASSIGN], 1);
        const int y = i / W, x = i - y * W;
        const int2 v = lab.v[i];
        const int qx = x + v.x, qy = y + v.y;
        if (qx < 0 || qx >= W || qy < 0 || qy >= H) continue;
        const int j = qy * W + qx;
        if (oth.m[j] < 0) continue;
        const int2 w = oth.v[j];
        const float2 r = lab.r[i], s = oth.r[j];
        const float ex = (float)(v.x + w.x) + (r.x + s.x);
        const float ey = (float)(v.y + w.y) + (r.y + s.y);
        if (ex * ex + ey * ey < pp.fb2) atomicAdd(&mi[(size_t)m * kMI + MI_NSYM], 1);
    }
}

// Discard planes failing the symmetry cue (eta) or the RANSAC/colour overlap cue (kappa).
__global__ void k_cue_invalidate(const __grid_constant__ Batch bt, int level, int stage, PlaneParams pp) {
    const PairView& pv = bt.view(blockIdx.z);
    const LevelGeom g = bt.geom(blockIdx.z, level);
    const int dir = blockIdx.y;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < g.ncells(); c += gridDim.x * blockDim.x) {
        const int id = (g.base + c) * 2 + stage - 1;
        int* f = pv.mi[dir] + (size_t)id * kMI;
        if (!f[MI_VALID]) continue;
        bool bad = false;
        if (f[MI_NASSIGN] > 0 && (float)f[MI_NSYM] < pp.eta * (float)f[MI_NASSIGN]) {
            f[MI_FLAGS] |= F_BAD_FB;
            bad = true;
        }
        if ((float)f[MI_NRC] < pp.kappa * (float)f[MI_COUNT]) {
            f[MI_FLAGS] |= F_BAD_KAPPA;
            bad = true;
        }
        if (bad) {
            f[MI_VALID] = 0;
            pv.mef[dir][id].valid = 0;
        }
    }
}

// Many-to-one: per target q = round(p + f), the lowest (L, index) keeps it;
// a loser whose flow differs from the winner's by t_fb or more is occluded.
__global__ void k_m2o_init(const __grid_constant__ Batch bt) {
    const PairView& pv = bt.view(blockIdx.z);
    const int dir = blockIdx.y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < pv.n; i += gridDim.x * blockDim.x)
        pv.m2o_key[dir][i] = ~0ull;
}
__global__ void k_m2o_claim(const __grid_constant__ Batch bt) {
    const PairView& pv = bt.view(blockIdx.z);
    const int dir = blockIdx.y;
    const int W = pv.W, n = pv.n;
    const Labels lab = pv.lvl[dir];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (lab.m[i] < 0) continue;
        const int y = i / W, x = i - y * W;
        const int2 v = lab.v[i];
        if (x + v.x < 0 || x + v.x >= W || y + v.y < 0 || y + v.y >= pv.H) continue;
        const int q = (y + v.y) * W + (x + v.x);
        const unsigned long long key = ((unsigned long long)__float_as_uint(lab.L[i]) << 32) | (unsigned)i;
        atomicMin(&pv.m2o_key[dir][q], key);
    }
}
__global__ void k_m2o_resolve(const __grid_constant__ Batch bt, PlaneParams pp) {
    const PairView& pv = bt.view(blockIdx.z);
    const int dir = blockIdx.y;
    const int W = pv.W, n = pv.n;
    const Labels lab = pv.lvl[dir];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (lab.m[i] < 0) continue;
        const int y = i / W, x = i - y * W;
        const int2 v = lab.v[i];
        if (x + v.x < 0 || x + v.x >= W || y + v.y < 0 || y + v.y >= pv.H) continue;
        const int q = (y + v.y) * W + (x + v.x);
        const int w = (int)(pv.m2o_key[dir][q] & 0xFFFFFFFFull);
        if (w == i) continue;
        const int2 vw = lab.v[w];
        const float2 r = lab.r[i], rw = lab.r[w];
        const float ex = (float)(v.x - vw.x) + (r.x - rw.x);
        const float ey = (float)(v.y - vw.y) + (r.y - rw.y);
        if (!(ex * ex + ey * ey < pp.fb2)) {
            lab.m[i] = -1;
            pv.cue[dir][i] |= CUE_M2O;
        }
    }
}

// Sec. 3.3 merge with coarse priority, then the NNF update of Sec. 3.3.1.
__global__ void k_merge_update(const __grid_constant__ Batch bt, PlaneParams pp) {
    const PairView& pv = bt.view(blockIdx.z);
    const int dir = blockIdx.y;
    const int n = pv.n;
    const Labels lab = pv.lvl[dir], acc = pv.acc[dir];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int m = lab.m[i];
        int am = acc.m[i];
        if (m >= 0 && (am < 0 || lab.L[i] < acc.L[i] - pp.beta)) {
            acc.m[i] = m;
            acc.L[i] = lab.L[i];
            acc.v[i] = lab.v[i];
            acc.r[i] = lab.r[i];
            am = m;
        }
        pv.frozen[dir][i] = am >= 0;
        if (am >= 0) pv.nnf[dir][i] = acc.v[i];
    }
}

// ---------------------------------------------------------------- fill and final map (Sec. 3.4.1)
// One Jacobi iteration: labels from acc into tent (flip = 0) or from tent into acc (flip = 1).
template <int ST>
__global__ void k_fill(const __grid_constant__ Batch bt, int flip, PlaneParams pp) {
    const PairView& pv = bt.view(blockIdx.z);
    const int dir = blockIdx.y;
    const int W = pv.W, H = pv.H, n = pv.n;
    const Labels cur = flip ? pv.tent[dir] : pv.acc[dir], nxt = flip ? pv.acc[dir] : pv.tent[dir];
    const void* src = pv.img[dir];
    const void* tgt = pv.img[1 - dir];
    const Mef* mef = pv.mef[dir];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int cm = cur.m[i];
        int bm = cm, bkx = 0, bky = 0;
        float bL = cur.L[i], bfx = 0.f, bfy = 0.f;
        bool filled = false;
        if (cm < 0 && !(pv.cue[dir][i] & CUE_M2O)) {
            const int y = i / W, x = i - y * W;
            bm = -1;
            bL = FLT_MAX;
            for (int k = 0; k < 4; ++k) {
                const int xx = x + (k == 0 ? -1 : (k == 1 ? 1 : 0));
                const int yy = y + (k == 2 ? -1 : (k == 3 ? 1 : 0));
                if (xx < 0 || xx >= W || yy < 0 || yy >= H) continue;
                const int m = cur.m[yy * W + xx];
                if (m < 0 || m >= pv.m_models) continue;
                const Mef mm = mef[m];
                int ix, iy, kx, ky;
                float fx, fy;
                if (!plane_target(mm, x, y, W, H, ix, fx, iy, fy, kx, ky)) continue;
                const float d = colour_delta<ST>(src, tgt, W, H, x, y, ix, fx, iy, fy);
                if (!(d < pp.eps)) continue;
                if (d < bL - kLTie || (fabsf(d - bL) <= kLTie && m < bm)) {
                    bL = d;
                    bm = m;
                    bkx = kx;
                    bky = ky;
                    bfx = fx;
                    bfy = fy;
                }
            }
            filled = bm >= 0;
            if (!filled) bL = cur.L[i];
        }
        nxt.m[i] = bm;
        nxt.L[i] = bL;
        if (filled) {
            int vx, vy;
            float rx, ry;
            round_split(bkx, bfx, vx, rx);
            round_split(bky, bfy, vy, ry);
            nxt.v[i] = make_int2(vx, vy);
            nxt.r[i] = make_float2(rx, ry);
        } else {
            nxt.v[i] = cur.v[i];
            nxt.r[i] = cur.r[i];
        }
    }
}

// ---------------------------------------------------------------- edge-aware fill of unassigned pixels
// Each pixel left without a plane takes the plane of the assigned pixel
// nearest in geodesic distance (steps 256 + |q_i - q_j| between
// 4-neighbours, q = floor(1024 (R + G + B)) of frame 1 as given).  Integer
// distances by fast sweeping: rounds of four in-place scans in the order rows
// left to right, rows right to left, columns top to bottom, columns bottom to
// top; an offer wins with a lower distance, or an equal one from a lower seed
// index.
// Scratch of the edge-aware fill (the many-to-one keys and the pixel lists are idle by then): distances and seeds.
__device__ __forceinline__ long long* seed_dist(const PairView& pv) { return reinterpret_cast<long long*>(pv.m2o_key[0]); }
__device__ __forceinline__ int* seed_of(const PairView& pv) { return pv.list[0]; }
__global__ void k_seed_init(const __grid_constant__ Batch bt) {
    const PairView& pv = bt.view(blockIdx.z);
    const int* am = pv.acc[0].m;
    const int n = pv.n;
    long long* dist = seed_dist(pv);
    int* seed = seed_of(pv);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        dist[i] = am[i] >= 0 ? 0 : (1ll << 62);
        seed[i] = am[i] >= 0 ? i : -1;
    }
}
// One walk along a line (a row or a column): relax each pixel from the one
// before it.  The previous pixel's (distance, seed, grey) stays in registers,
// so the loop-carried chain is integer arithmetic only; the next chunk of U
// pixels is loaded before the current chunk is stored (disjoint pixels), so
// the loads run ahead of the chain.  Every register of a chunk is defined,
// also past the end of the line (those slots are never used).
template <int U>
__device__ __forceinline__ void seed_walk(const int* q, long long* dist, int* seed, int64_t i0, int64_t step, int len) {
    long long dp = dist[i0];
    int sp = seed[i0], qp = q[i0];
    long long dn[U];
    int sn[U], qn[U];
    int cnt = min(U, len - 1);
#pragma unroll
    for (int j = 0; j < U; ++j) {
        dn[j] = 0, sn[j] = -1, qn[j] = 0;
        if (j < cnt) {
            const int64_t i = i0 + (int64_t)(1 + j) * step;
            dn[j] = dist[i], sn[j] = seed[i], qn[j] = q[i];
        }
    }
    for (int m = 1; m < len; m += U) {
        long long dc[U];
        int sc[U], qc[U];
        const int cur = cnt;
        cnt = min(U, len - (m + U));  // pixels in the next chunk (<= 0 past the end)
#pragma unroll
        for (int j = 0; j < U; ++j) {
            dc[j] = dn[j], sc[j] = sn[j], qc[j] = qn[j];
            if (j < cnt) {
                const int64_t i = i0 + (int64_t)(m + U + j) * step;
                dn[j] = dist[i], sn[j] = seed[i], qn[j] = q[i];
            }
        }
#pragma unroll
        for (int j = 0; j < U; ++j) {
            if (j < cur) {
                if (sp >= 0) {
                    const long long c = dp + 256 + (long long)abs(qc[j] - qp);
                    if (c < dc[j] || (c == dc[j] && sp < sc[j])) {
                        const int64_t i = i0 + (int64_t)(m + j) * step;
                        dc[j] = c, sc[j] = sp;
                        dist[i] = c, seed[i] = sp;
                    }
                }
                dp = dc[j], sp = sc[j], qp = qc[j];
            }
        }
    }
}
// cols = 0: one thread per row, left to right then right to left; cols = 1:
// one thread per column, top to bottom then bottom to top (a warp's loads of
// one step are then coalesced).  Lines are disjoint, so fusing a line's two
// scans keeps the order of four whole-frame scans.
__global__ void k_seed_lines(const __grid_constant__ Batch bt, int cols) {
    const PairView& pv = bt.view(blockIdx.z);
    const int* q = pv.gq;
    long long* dist = seed_dist(pv);
    int* seed = seed_of(pv);
    const int W = pv.W, H = pv.H;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (!cols) {
        if (t >= H) return;
        seed_walk<8>(q, dist, seed, (int64_t)t * W, 1, W);
        seed_walk<8>(q, dist, seed, (int64_t)t * W + W - 1, -1, W);
    } else {
        if (t >= W) return;
        seed_walk<8>(q, dist, seed, t, W, H);
        seed_walk<8>(q, dist, seed, (int64_t)(H - 1) * W + t, -(int64_t)W, H);
    }
}

// Final flow (plane flow, else the NNF offset, else with a seed the seed's
// plane at this pixel) and occlusion: no plane, a cue flag, or colour error
// after warping by the final flow >= occ_thresh.
template <int ST>
__global__ void k_final(const __grid_constant__ Batch bt, PlaneParams pp, int interp, const __grid_constant__ FinalOut out) {
    const PairView& pv = bt.view(blockIdx.z);
    const int dir = 0;
    const int* seed = interp ? seed_of(pv) : nullptr;
    float* flow = out.flow[blockIdx.z];
    uint8_t* occ = out.occ[blockIdx.z];
    const int W = pv.W, H = pv.H, n = pv.n;
    const Labels acc = pv.acc[dir];
    const void* src = pv.img[dir];
    const void* tgt = pv.img[1 - dir];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int y = i / W, x = i - y * W;
        int bx, by;
        float fx, fy;
        const bool as = acc.m[i] >= 0;
        if (as) {
            const int2 v = acc.v[i];
            const float2 r = acc.r[i];
            flow[2 * i] = (float)v.x + r.x;
            flow[2 * i + 1] = (float)v.y + r.y;
            bx = x + v.x + (r.x < 0.f ? -1 : 0);
            fx = r.x < 0.f ? r.x + 1.f : r.x;
            by = y + v.y + (r.y < 0.f ? -1 : 0);
            fy = r.y < 0.f ? r.y + 1.f : r.y;
        } else {
            const int2 v = pv.nnf[dir][i];
            flow[2 * i] = (float)v.x;
            flow[2 * i + 1] = (float)v.y;
            bx = x + v.x;
            by = y + v.y;
            fx = fy = 0.f;
            const int sd = seed ? seed[i] : -1;
            if (sd >= 0) {  // edge-aware fill: the seed's plane here, or the seed's flow
                const Mef m = pv.mef[dir][acc.m[sd]];
                int kx, ky;
                float gx, gy;
                if (mef_flow(m, (float)(x - m.ox), (float)(y - m.oy), kx, gx, ky, gy)) {
                    flow[2 * i] = (float)kx + gx;
                    flow[2 * i + 1] = (float)ky + gy;
                } else {
                    const int2 vs = acc.v[sd];
                    const float2 rs = acc.r[sd];
                    flow[2 * i] = (float)vs.x + rs.x;
                    flow[2 * i + 1] = (float)vs.y + rs.y;
                }
            }
        }
        bool o = !as || (pv.cue[dir][i] & CUE_M2O);
        if (!in_frame_tol(bx, fx, W) || !in_frame_tol(by, fy, H))
            o = true;
        else if (!(colour_delta<ST>(src, tgt, W, H, x, y, bx, fx, by, fy) < pp.occ_thresh))
            o = true;
        occ[i] = o ? 1 : 0;
    }
}

// ---------------------------------------------------------------- state import / export helpers
// Evaluation forms of imported absolute homographies.
__global__ void k_import_models(const __grid_constant__ Batch bt, int nlev, int m) {
    const PairView& pv = bt.view(blockIdx.z);
    const LevelGeom* geoms = bt.geo[blockIdx.z];
    const int dir = blockIdx.y;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < m; id += gridDim.x * blockDim.x) {
        const int cell_all = id >> 1;
        int l = 0;
        while (l + 1 < nlev && geoms[l + 1].base <= cell_all) ++l;
        const LevelGeom g = geoms[l];
        const int cell = cell_all - g.base;
        const int cx = cell % g.gx.count, cy = cell / g.gx.count;
        const int ox = win_pos(g.gx, g.h, cx) + g.s / 2, oy = win_pos(g.gy, g.h, cy) + g.s / 2;
        double Hl[9];
        abs_to_local(pv.mh[dir] + (size_t)id * 9, ox, oy, Hl);
        Mef f = {};
        const bool ok = make_mef(Hl, ox, oy, f);
        f.valid = ok && pv.mi[dir][(size_t)id * kMI + MI_VALID] ? 1 : 0;
        pv.mef[dir][id] = f;
    }
}

// labels <-> (model, L, flow) with flow = v + r in double
__global__ void k_labels_export(Labels l, int n, int* om, float* oL, double* of) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        om[i] = l.m[i];
        oL[i] = l.L[i];
        of[2 * i] = (double)l.v[i].x + (double)l.r[i].x;
        of[2 * i + 1] = (double)l.v[i].y + (double)l.r[i].y;
    }
}
__global__ void k_labels_import(Labels l, int n, int m, const int* im, const float* iL, const double* iF,
                                int* flag) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int id = im[i];
        const double fx = iF[2 * i], fy = iF[2 * i + 1];
        // |flow| < 2^30 (and finite): the rounded offset fits an int
        const bool flow_ok = fabs(fx) < 1073741824.0 && fabs(fy) < 1073741824.0;
        if (id < -1 || id >= m || (id >= 0 && !flow_ok)) {
            *flag = 1;
            id = -1;
        }
        l.m[i] = id;
        l.L[i] = iL[i];
        if (flow_ok) {
            const double vx = floor(fx + 0.5), vy = floor(fy + 0.5);
            l.v[i] = make_int2((int)vx, (int)vy);
            l.r[i] = make_float2((float)(fx - vx), (float)(fy - vy));
        } else {
            l.v[i] = make_int2(0, 0);
            l.r[i] = make_float2(0.f, 0.f);
        }
    }
}

// ---------------------------------------------------------------- launchers
// Every launch covers np pairs (blockIdx.z); grids are sized for the largest pair, and each block past its own
// pair's pixels or windows does nothing.
template <int ST>
static void launch_ransac_st(const Batch& bt, int np, int level, int s, int max_cells, int stage,
                             const PlaneParams& pp, cudaStream_t st) {
    const int nc = max_cells;
    if (s <= 16) {
        static bool wattr_set = false;
        if (!wattr_set) {
            cudaFuncSetAttribute(k_ransac_warp<ST, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)ransac_warp_smem(false));
            cudaFuncSetAttribute(k_ransac_warp<ST, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)ransac_warp_smem(true));
            wattr_set = true;
        }
        const dim3 fgrid((nc + kRansacWarps - 1) / kRansacWarps, 2, np), grid((nc + 7) / 8, 2, np);
        if (s * s <= kLaneScoreMax)
            k_ransac_warp<ST, true><<<fgrid, 32 * kRansacWarps, ransac_warp_smem(true), st>>>(bt, level, stage, pp);
        else
            k_ransac_warp<ST, false><<<fgrid, 32 * kRansacWarps, ransac_warp_smem(false), st>>>(bt, level, stage, pp);
        k_refit_solve<<<dim3((2 * nc + 63) / 64, 1, np), 64, 0, st>>>(bt, level, pp);
        k_ransac_finish_warp<ST><<<grid, 256, 0, st>>>(bt, level, stage, pp);
        return;
    }
    const size_t smem = (size_t)s * s * sizeof(float4);
    static bool attr_set = false;
    if (!attr_set) {
        const int mx = kMaxCell * kMaxCell * (int)sizeof(float4);  // the largest window's matches
        cudaFuncSetAttribute(k_ransac_block<ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_ransac_finish_block<ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        attr_set = true;
    }
    k_ransac_block<ST><<<dim3(nc, 2, np), 256, smem, st>>>(bt, level, stage, pp);
    k_refit_solve<<<dim3((2 * nc + 63) / 64, 1, np), 64, 0, st>>>(bt, level, pp);
    k_ransac_finish_block<ST><<<dim3(nc, 2, np), 256, smem, st>>>(bt, level, stage, pp);
}
void launch_ransac(const Batch& bt, int np, int level, int s, int max_cells, int stage, const PlaneParams& pp,
                   cudaStream_t st) {
    switch (pp.storage) {
        case 0: launch_ransac_st<0>(bt, np, level, s, max_cells, stage, pp, st); break;
        case 1: launch_ransac_st<1>(bt, np, level, s, max_cells, stage, pp, st); break;
        case 2: launch_ransac_st<2>(bt, np, level, s, max_cells, stage, pp, st); break;
    }
}

void launch_assign(const Batch& bt, int np, int level, int stage, int which, int write_resid, const PlaneParams& pp,
                   int grid_blocks, cudaStream_t st) {
    const dim3 grid(grid_blocks, 2, np);
    switch (pp.storage) {
        case 0: k_assign<0><<<grid, 256, 0, st>>>(bt, level, stage, which, write_resid, pp); break;
        case 1: k_assign<1><<<grid, 256, 0, st>>>(bt, level, stage, which, write_resid, pp); break;
        case 2: k_assign<2><<<grid, 256, 0, st>>>(bt, level, stage, which, write_resid, pp); break;
    }
}

void launch_cues(const Batch& bt, int np, int level, int max_cells, int stage, int which, const PlaneParams& pp,
                 int grid_blocks, cudaStream_t st) {
    const int cb = (max_cells + 255) / 256;
    k_cue_zero<<<dim3(cb, 2, np), 256, 0, st>>>(bt, level, stage);
    k_cue_counts<<<dim3(grid_blocks, 2, np), 256, 0, st>>>(bt, level, stage, which, pp);
    k_cue_invalidate<<<dim3(cb, 2, np), 256, 0, st>>>(bt, level, stage, pp);
}

void launch_many_to_one(const Batch& bt, int np, const PlaneParams& pp, int grid_blocks, cudaStream_t st) {
    k_m2o_init<<<dim3(grid_blocks, 2, np), 256, 0, st>>>(bt);
    k_m2o_claim<<<dim3(grid_blocks, 2, np), 256, 0, st>>>(bt);
    k_m2o_resolve<<<dim3(grid_blocks, 2, np), 256, 0, st>>>(bt, pp);
}

void launch_merge_update(const Batch& bt, int np, const PlaneParams& pp, int grid_blocks, cudaStream_t st) {
    k_merge_update<<<dim3(grid_blocks, 2, np), 256, 0, st>>>(bt, pp);
}

// Label sets of a pair: 0 acc, 1 tent, 2 st1, 3 lvl.
__device__ __forceinline__ Labels label_set(const PairView& pv, int set, int dir) {
    return set == 0 ? pv.acc[dir] : (set == 1 ? pv.tent[dir] : (set == 2 ? pv.st1[dir] : pv.lvl[dir]));
}
__global__ void k_copy_labels(const __grid_constant__ Batch bt, int from, int to) {
    const PairView& pv = bt.view(blockIdx.z);
    const int dir = blockIdx.y;
    const Labels a = label_set(pv, from, dir), b = label_set(pv, to, dir);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < pv.n; i += gridDim.x * blockDim.x) {
        b.m[i] = a.m[i];
        b.L[i] = a.L[i];
        b.v[i] = a.v[i];
        b.r[i] = a.r[i];
    }
}
void launch_copy_labels(const Batch& bt, int np, int from, int to, int grid_blocks, cudaStream_t st) {
    k_copy_labels<<<dim3(grid_blocks, 2, np), 256, 0, st>>>(bt, from, to);
}

void launch_fill(const Batch& bt, int np, const PlaneParams& pp, int iters, int grid_blocks, cudaStream_t st) {
    // ping-pong between acc and tent (tent is free after the last level)
    const dim3 grid(grid_blocks, 2, np);
    for (int it = 0; it < iters; ++it) {
        switch (pp.storage) {
            case 0: k_fill<0><<<grid, 256, 0, st>>>(bt, it & 1, pp); break;
            case 1: k_fill<1><<<grid, 256, 0, st>>>(bt, it & 1, pp); break;
            case 2: k_fill<2><<<grid, 256, 0, st>>>(bt, it & 1, pp); break;
        }
    }
    if (iters & 1) launch_copy_labels(bt, np, 1, 0, grid_blocks, st);  // the result sits in tent
}

void launch_fill_seeds(const Batch& bt, int np, int max_w, int max_h, int rounds, int grid_blocks, cudaStream_t st) {
    k_seed_init<<<dim3(grid_blocks, 1, np), 256, 0, st>>>(bt);
    for (int r = 0; r < rounds; ++r) {
        k_seed_lines<<<dim3((max_h + 31) / 32, 1, np), 32, 0, st>>>(bt, 0);
        k_seed_lines<<<dim3((max_w + 31) / 32, 1, np), 32, 0, st>>>(bt, 1);
    }
}

void launch_final(const Batch& bt, int np, const PlaneParams& pp, int interp, const FinalOut& out, int grid_blocks,
                  cudaStream_t st) {
    const dim3 grid(grid_blocks, 1, np);
    switch (pp.storage) {
        case 0: k_final<0><<<grid, 256, 0, st>>>(bt, pp, interp, out); break;
        case 1: k_final<1><<<grid, 256, 0, st>>>(bt, pp, interp, out); break;
        case 2: k_final<2><<<grid, 256, 0, st>>>(bt, pp, interp, out); break;
    }
}

// Clears the models of every window of every level (model ids below m_models).
__global__ void k_reset_models(const __grid_constant__ Batch bt) {
    const PairView& pv = bt.view(blockIdx.z);
    const int dir = blockIdx.y;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < pv.m_models; id += gridDim.x * blockDim.x) {
#pragma unroll
        for (int q = 0; q < 9; ++q) pv.mh[dir][(size_t)id * 9 + q] = 0.0;
        pv.mef[dir][id] = Mef{};
#pragma unroll
        for (int q = 0; q < kMI; ++q) pv.mi[dir][(size_t)id * kMI + q] = 0;
    }
}
void launch_reset_models(const Batch& bt, int np, int max_models, cudaStream_t st) {
    if (max_models <= 0) return;  // no plane levels: no model table (an empty grid is not a launch)
    k_reset_models<<<dim3((max_models + 255) / 256, 2, np), 256, 0, st>>>(bt);
}

__global__ void k_reset_labels(const __grid_constant__ Batch bt, float eps) {
    const PairView& pv = bt.view(blockIdx.z);
    const int dir = blockIdx.y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < pv.n; i += gridDim.x * blockDim.x) {
        pv.acc[dir].m[i] = -1;
        pv.acc[dir].L[i] = eps;
        pv.acc[dir].v[i] = make_int2(0, 0);
        pv.acc[dir].r[i] = make_float2(0.f, 0.f);
        pv.cue[dir][i] = 0;
        pv.frozen[dir][i] = 0;
    }
}
__global__ void k_frozen_from_labels(const __grid_constant__ Batch bt) {
    const PairView& pv = bt.view(blockIdx.z);
    const int dir = blockIdx.y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < pv.n; i += gridDim.x * blockDim.x)
        pv.frozen[dir][i] = pv.acc[dir].m[i] >= 0;
}
void launch_frozen_from_labels(const Batch& bt, int np, int grid_blocks, cudaStream_t st) {
    k_frozen_from_labels<<<dim3(grid_blocks, 2, np), 256, 0, st>>>(bt);
}

void launch_reset_labels(const Batch& bt, int np, float eps, int grid_blocks, cudaStream_t st) {
    k_reset_labels<<<dim3(grid_blocks, 2, np), 256, 0, st>>>(bt, eps);
}

template <int ST>
__global__ void k_frames_export(const __grid_constant__ Batch bt, float* dst) {
    const PairView& pv = bt.view(blockIdx.z);
    const int dir = blockIdx.y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < pv.n; i += gridDim.x * blockDim.x) {
        const float4 a = ldpix<ST>(pv.img[dir], i);
        reinterpret_cast<float4*>(dst)[(size_t)dir * pv.n + i] = a;
    }
}
void launch_frames_export(const Batch& bt, int n, int storage, float* dst, cudaStream_t st) {
    const dim3 grid((n + 255) / 256, 2);
    switch (storage) {
        case 0: k_frames_export<0><<<grid, 256, 0, st>>>(bt, dst); break;
        case 1: k_frames_export<1><<<grid, 256, 0, st>>>(bt, dst); break;
        case 2: k_frames_export<2><<<grid, 256, 0, st>>>(bt, dst); break;
    }
}

void launch_import_models(const Batch& bt, int nlev, int m, cudaStream_t st) {
    if (m <= 0) return;  // no model table
    k_import_models<<<dim3((m + 255) / 256, 2), 256, 0, st>>>(bt, nlev, m);
}

void launch_labels_export(const Labels& l, int n, int* om, float* oL, double* of, cudaStream_t st) {
    k_labels_export<<<(n + 255) / 256, 256, 0, st>>>(l, n, om, oL, of);
}
void launch_labels_import(const Labels& l, int n, int m, const int* im, const float* iL, const double* iF, int* flag,
                          cudaStream_t st) {
    k_labels_import<<<(n + 255) / 256, 256, 0, st>>>(l, n, m, im, iL, iF, flag);
}

}  // namespace gpm
