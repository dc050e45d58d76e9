// Plane kernels (sm_103a): per-window RANSAC with least-squares refit,
// assignment by colour consistency, occlusion cues, merge, NNF update, model
// propagation fill and the final flow / occlusion map.
#include <float.h>

#include "common.cuh"
#include "kernels.h"

namespace gpm {

constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------- block reductions
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0;
    for (int w = 0; w < NT / 32; ++w) t += red[w];  // fixed order: same bits on every thread
    return t;
}
template <int NT>
__device__ __forceinline__ int block_count(int v, int* red) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    int t = 0;
    for (int w = 0; w < NT / 32; ++w) t += red[w];
    return t;
}

// ---------------------------------------------------------------- 4-point homography
// Exact projective basis construction: with P = [p1 p2 p3] (homogeneous
// columns) and lambda = adj(P) p4, A = P diag(lambda) maps the projective
// basis e1, e2, e3, (1,1,1) onto p1..p4 up to scale; likewise B for the
// targets, and H ~ B adj(A).  Coordinates are window-local integers, so all
// of it up to adj(A) and B is exact integer arithmetic; only the final
// product is rounded (FP64).  Sign and scale are fixed later.
__device__ __forceinline__ void minimal_h(const int* px, const int* py, const int* qx, const int* qy, double* H) {
    long long aP[9], aQ[9];
    {
        const long long x1 = px[0], x2 = px[1], x3 = px[2], y1 = py[0], y2 = py[1], y3 = py[2];
        aP[0] = y2 - y3; aP[1] = x3 - x2; aP[2] = x2 * y3 - x3 * y2;
        aP[3] = y3 - y1; aP[4] = x1 - x3; aP[5] = x3 * y1 - x1 * y3;
        aP[6] = y1 - y2; aP[7] = x2 - x1; aP[8] = x1 * y2 - x2 * y1;
    }
    {
        const long long x1 = qx[0], x2 = qx[1], x3 = qx[2], y1 = qy[0], y2 = qy[1], y3 = qy[2];
        aQ[0] = y2 - y3; aQ[1] = x3 - x2; aQ[2] = x2 * y3 - x3 * y2;
        aQ[3] = y3 - y1; aQ[4] = x1 - x3; aQ[5] = x3 * y1 - x1 * y3;
        aQ[6] = y1 - y2; aQ[7] = x2 - x1; aQ[8] = x1 * y2 - x2 * y1;
    }
    long long l[3], mu[3];
    for (int i = 0; i < 3; ++i) {
        l[i] = aP[3 * i] * px[3] + aP[3 * i + 1] * py[3] + aP[3 * i + 2];
        mu[i] = aQ[3 * i] * qx[3] + aQ[3 * i + 1] * qy[3] + aQ[3 * i + 2];
    }
    long long A[9];
    for (int c = 0; c < 3; ++c) {
        A[0 * 3 + c] = l[c] * px[c];
        A[1 * 3 + c] = l[c] * py[c];
        A[2 * 3 + c] = l[c];
    }
    long long adjA[9];
    adjA[0] = A[4] * A[8] - A[5] * A[7];
    adjA[1] = A[2] * A[7] - A[1] * A[8];
    adjA[2] = A[1] * A[5] - A[2] * A[4];
    adjA[3] = A[5] * A[6] - A[3] * A[8];
    adjA[4] = A[0] * A[8] - A[2] * A[6];
    adjA[5] = A[2] * A[3] - A[0] * A[5];
    adjA[6] = A[3] * A[7] - A[4] * A[6];
    adjA[7] = A[1] * A[6] - A[0] * A[7];
    adjA[8] = A[0] * A[4] - A[1] * A[3];
    double B[9], dA[9];
    for (int c = 0; c < 3; ++c) {
        B[0 * 3 + c] = (double)(mu[c] * qx[c]);
        B[1 * 3 + c] = (double)(mu[c] * qy[c]);
        B[2 * 3 + c] = (double)mu[c];
    }
    for (int k = 0; k < 9; ++k) dA[k] = (double)adjA[k];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            H[r * 3 + c] = fma(B[r * 3], dA[c], fma(B[r * 3 + 1], dA[3 + c], B[r * 3 + 2] * dA[6 + c]));
}

__device__ __forceinline__ bool collinear3(int ax, int ay, int bx, int by, int cx, int cy) {
    return (long long)(bx - ax) * (cy - ay) - (long long)(by - ay) * (cx - ax) == 0;
}

// Smallest-eigenvalue eigenvector of a symmetric positive semi-definite 9x9
// matrix by inverse iteration on M + sigma I (one Cholesky factorisation,
// then repeated triangular solves), started from x.
__device__ void min_eigvec_inverse_iteration(const double* M, double* x) {
    double tr = 0;
    for (int i = 0; i < 9; ++i) tr += M[i * 9 + i];
    const double sigma = 1e-13 * tr + 1e-300;
    double L[81];
    for (int i = 0; i < 81; ++i) L[i] = 0;
    for (int j = 0; j < 9; ++j) {
        double d = M[j * 9 + j] + sigma;
        for (int k = 0; k < j; ++k) d -= L[j * 9 + k] * L[j * 9 + k];
        d = d > 0 ? sqrt(d) : 1e-150;
        L[j * 9 + j] = d;
        for (int i = j + 1; i < 9; ++i) {
            double s = M[i * 9 + j];
            for (int k = 0; k < j; ++k) s -= L[i * 9 + k] * L[j * 9 + k];
            L[i * 9 + j] = s / d;
        }
    }
    double nx = 0;
    for (int i = 0; i < 9; ++i) nx += x[i] * x[i];
    nx = 1.0 / sqrt(nx);
    for (int i = 0; i < 9; ++i) x[i] *= nx;
    for (int it = 0; it < 60; ++it) {
        double y[9];
        for (int i = 0; i < 9; ++i) {  // L y = x
            double s = x[i];
            for (int k = 0; k < i; ++k) s -= L[i * 9 + k] * y[k];
            y[i] = s / L[i * 9 + i];
        }
        for (int i = 8; i >= 0; --i) {  // L^T z = y
            double s = y[i];
            for (int k = i + 1; k < 9; ++k) s -= L[k * 9 + i] * y[k];
            y[i] = s / L[i * 9 + i];
        }
        double n = 0, dot = 0;
        for (int i = 0; i < 9; ++i) {
            n += y[i] * y[i];
            dot += y[i] * x[i];
        }
        n = 1.0 / sqrt(n);
        if (dot < 0) n = -n;
        double diff = 0;
        for (int i = 0; i < 9; ++i) {
            y[i] *= n;
            diff = fmax(diff, fabs(y[i] - x[i]));
            x[i] = y[i];
        }
        if (diff < 1e-15) break;
    }
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
// fraction; false if the denominator is not positive or the point leaves
// [0, W-1] x [0, H-1].
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

// ---------------------------------------------------------------- RANSAC per window
// Sec. 3.1.2 / 3.2: one block per window and direction.  The window's
// matches (u, u + v(u)) -- all pixels at stage 1, the still-unassigned ones in
// raster order at stage 2 -- sit in shared memory as exact floats; each
// thread draws, solves and scores hypotheses k = tid, tid + NT, ...; the
// block keeps the largest support (lowest k on ties), refits it by the
// normalised DLT on its inliers and keeps the refit unless it has fewer.
template <int NT, int ST>
__global__ void __launch_bounds__(NT) k_ransac(PairView pv, LevelGeom g, int level, int stage, PlaneParams pp) {
    extern __shared__ float4 sm_match[];
    __shared__ double red_d[NT / 32];
    __shared__ int red_i[NT / 32];
    __shared__ unsigned long long s_best;
    __shared__ double s_Hw[9], s_Hr[9];
    __shared__ double s_M[81];
    __shared__ Mef s_mef[2];
    __shared__ int s_woff[NT / 32 + 1];
    __shared__ int s_refit_ok;

    const int dir = blockIdx.y;
    const int cell = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cxw = cell % g.gx.count, cyw = cell / g.gx.count;
    const int s = g.s;
    const int x0 = win_pos(g.gx, g.h, cxw), y0 = win_pos(g.gy, g.h, cyw);
    const int ox = x0 + s / 2, oy = y0 + s / 2;
    const int W = pv.W, H = pv.H;
    const int id = (g.base + cell) * 2 + (stage - 1);
    int* mi = pv.mi[dir] + (size_t)id * kMI;
    const int2* nnf = pv.nnf[dir];
    const uint8_t* resid = pv.resid[dir];

    // gather the window's matches in raster order
    int N = 0;
    for (int base = 0; base < s * s; base += NT) {
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
        const unsigned b = __ballot_sync(FULL, take);
        if (lane == 0) s_woff[warp] = __popc(b);
        __syncthreads();
        if (tid == 0) {
            int acc = 0;
            for (int w = 0; w < NT / 32; ++w) {
                const int c = s_woff[w];
                s_woff[w] = acc;
                acc += c;
            }
            s_woff[NT / 32] = acc;
        }
        __syncthreads();
        if (take) sm_match[N + s_woff[warp] + __popc(b & ((1u << lane) - 1))] = mt;
        N += s_woff[NT / 32];
        __syncthreads();
    }

    if (tid == 0) {
        for (int k = 0; k < kMI; ++k) mi[k] = 0;
        mi[MI_NIN] = N;
        mi[MI_BESTK] = -1;
        for (int k = 0; k < 9; ++k) pv.mh[dir][(size_t)id * 9 + k] = 0.0;
        Mef z = {};
        pv.mef[dir][id] = z;
    }
    if (N < pp.min_inliers || N < 4) return;

    // hypotheses
    const float t2 = pp.t2;
    const uint32_t tag = stream_tag(RNG_RANSAC, dir, level, stage);
    int best_score = -1, best_k = 0x7fffffff;
    double bH[9];
    for (int k = tid; k < pp.num_hyp; k += NT) {
        const uint4 w = philox((uint32_t)cell, (uint32_t)k, tag, pv.pair_id, pp.k0, pp.k1);
        const uint32_t idx[4] = {w.x % (uint32_t)N, w.y % (uint32_t)N, w.z % (uint32_t)N, w.w % (uint32_t)N};
        int px[4], py[4], qx[4], qy[4];
        for (int j = 0; j < 4; ++j) {
            const float4 m = sm_match[idx[j]];
            px[j] = (int)m.x;
            py[j] = (int)m.y;
            qx[j] = (int)(m.x + m.z);
            qy[j] = (int)(m.y + m.w);
        }
        bool degen = false;
        const int T3[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int a = T3[t][0], b = T3[t][1], c = T3[t][2];
            degen |= collinear3(px[a], py[a], px[b], py[b], px[c], py[c]);
            degen |= collinear3(qx[a], qy[a], qx[b], qy[b], qx[c], qy[c]);
        }
        if (degen) continue;
        double Hk[9];
        minimal_h(px, py, qx, qy, Hk);
        Mef m;
        if (!make_mef(Hk, 0, 0, m)) continue;
        int score = 0;
        for (int j = 0; j < N; ++j) {
            const float4 mt = sm_match[j];
            score += mef_inlier(m, mt.x, mt.y, mt.z, mt.w, t2);
        }
        if (score > best_score) {
            best_score = score;
            best_k = k;
            for (int q = 0; q < 9; ++q) bH[q] = Hk[q];
        }
    }
    // block argmax: most inliers, then lowest hypothesis index
    if (tid == 0) s_best = 0ull;
    __syncthreads();
    const unsigned long long key =
        best_score < 0 ? 0ull
                       : (((unsigned long long)(best_score + 1)) << 32) |
                             (unsigned long long)(0xFFFFFFFFu - (uint32_t)best_k);
    if (key) atomicMax(&s_best, key);
    __syncthreads();
    const unsigned long long wkey = s_best;
    if (wkey == 0ull) return;
    const int wscore = (int)(wkey >> 32) - 1;
    const int wk = (int)(0xFFFFFFFFu - (uint32_t)(wkey & 0xFFFFFFFFull));
    if (best_k == wk) {
        for (int q = 0; q < 9; ++q) s_Hw[q] = bH[q];
        make_mef(bH, 0, 0, s_mef[0]);
    }
    __syncthreads();
    if (tid == 0) {
        mi[MI_BESTK] = wk;
        mi[MI_BESTSCORE] = wscore;
    }
    if (wscore < 4) return;

    // least-squares refit: Hartley normalisation of the winner's inliers
    const Mef wm = s_mef[0];
    double sx = 0, sy = 0, tx = 0, ty = 0;
    for (int j = tid; j < N; j += NT) {
        const float4 mt = sm_match[j];
        if (mef_inlier(wm, mt.x, mt.y, mt.z, mt.w, t2)) {
            sx += mt.x;
            sy += mt.y;
            tx += mt.x + mt.z;
            ty += mt.y + mt.w;
        }
    }
    sx = block_sum<NT>(sx, red_d);
    sy = block_sum<NT>(sy, red_d);
    tx = block_sum<NT>(tx, red_d);
    ty = block_sum<NT>(ty, red_d);
    const double inv_n = 1.0 / (double)wscore;
    const double mx = sx * inv_n, my = sy * inv_n, mqx = tx * inv_n, mqy = ty * inv_n;
    double ds = 0, dt = 0;
    for (int j = tid; j < N; j += NT) {
        const float4 mt = sm_match[j];
        if (mef_inlier(wm, mt.x, mt.y, mt.z, mt.w, t2)) {
            const double a = mt.x - mx, b = mt.y - my;
            ds += sqrt(a * a + b * b);
            const double c = (double)mt.x + mt.z - mqx, d = (double)mt.y + mt.w - mqy;
            dt += sqrt(c * c + d * d);
        }
    }
    ds = block_sum<NT>(ds, red_d) * inv_n;
    dt = block_sum<NT>(dt, red_d) * inv_n;
    const bool norm_ok = ds > 1e-12 && dt > 1e-12;
    const double ss = norm_ok ? sqrt(2.0) / ds : 1.0, sq = norm_ok ? sqrt(2.0) / dt : 1.0;
    // The normalised DLT rows of a pair (z = (x, y, 1) source, (u, v) target)
    // are a = (0, -z, v z) and b = (z, 0, -u z); their outer products sum to
    // blocks of S[w] = sum w z z^T with w in {1, u, v, u^2 + v^2}: 24 moments.
    double mom[24];
#pragma unroll
    for (int q = 0; q < 24; ++q) mom[q] = 0;
    for (int j = tid; j < N; j += NT) {
        const float4 mt = sm_match[j];
        if (!mef_inlier(wm, mt.x, mt.y, mt.z, mt.w, t2)) continue;
        const double x = ss * (mt.x - mx), y = ss * (mt.y - my);
        const double u = sq * ((double)mt.x + mt.z - mqx), v = sq * ((double)mt.y + mt.w - mqy);
        const double mm[6] = {x * x, x * y, x, y * y, y, 1.0};
        const double ww[4] = {1.0, u, v, u * u + v * v};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 6; ++b) mom[a * 6 + b] = fma(ww[a], mm[b], mom[a * 6 + b]);
    }
#pragma unroll
    for (int q = 0; q < 24; ++q) mom[q] = block_sum<NT>(mom[q], red_d);
    if (tid == 0) {
        s_refit_ok = 0;
        if (norm_ok) {
            const int map[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
            double* M = s_M;
            for (int q = 0; q < 81; ++q) M[q] = 0;
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) {
                    const int e = map[r][c];
                    const double S = mom[e], Su = mom[6 + e], Sv = mom[12 + e], Suv = mom[18 + e];
                    M[r * 9 + c] = S;
                    M[(3 + r) * 9 + (3 + c)] = S;
                    M[r * 9 + (6 + c)] = -Su;
                    M[(6 + c) * 9 + r] = -Su;
                    M[(3 + r) * 9 + (6 + c)] = -Sv;
                    M[(6 + c) * 9 + (3 + r)] = -Sv;
                    M[(6 + r) * 9 + (6 + c)] = Suv;
                }
            // start from the winning hypothesis in the normalised frames
            const double Tp[9] = {ss, 0, -ss * mx, 0, ss, -ss * my, 0, 0, 1};
            const double Tqi[9] = {1 / sq, 0, mqx, 0, 1 / sq, mqy, 0, 0, 1};
            const double Tq[9] = {sq, 0, -sq * mqx, 0, sq, -sq * mqy, 0, 0, 1};
            const double Tpi[9] = {1 / ss, 0, mx, 0, 1 / ss, my, 0, 0, 1};
            double t1[9], h0[9];
            mat3_mul(Tq, s_Hw, t1);
            mat3_mul(t1, Tpi, h0);
            min_eigvec_inverse_iteration(M, h0);
            double Hr[9];
            mat3_mul(Tqi, h0, t1);
            mat3_mul(t1, Tp, Hr);
            for (int q = 0; q < 9; ++q) s_Hr[q] = Hr[q];
            s_refit_ok = make_mef(Hr, 0, 0, s_mef[1]) ? 1 : 0;
        }
    }
    __syncthreads();
    int rcount = 0;
    const bool have_refit = s_refit_ok != 0;
    if (have_refit) {
        const Mef rm = s_mef[1];
        for (int j = tid; j < N; j += NT) {
            const float4 mt = sm_match[j];
            rcount += mef_inlier(rm, mt.x, mt.y, mt.z, mt.w, t2);
        }
    }
    rcount = block_count<NT>(rcount, red_i);
    const bool use_refit = have_refit && rcount >= wscore;
    Mef fm = s_mef[use_refit ? 1 : 0];
    const int count = use_refit ? rcount : wscore;

    // colour inliers among the RANSAC inliers: |S_R n S_C| (Sec. 3.4, third cue)
    const void* src = pv.img[dir];
    const void* tgt = pv.img[1 - dir];
    fm.ox = ox;
    fm.oy = oy;
    int nrc = 0;
    for (int j = tid; j < N; j += NT) {
        const float4 mt = sm_match[j];
        if (!mef_inlier(fm, mt.x, mt.y, mt.z, mt.w, t2)) continue;
        const int px = ox + (int)mt.x, py = oy + (int)mt.y;
        int ix, iy, kx, ky;
        float fx, fy;
        if (!plane_target(fm, px, py, W, H, ix, fx, iy, fy, kx, ky)) continue;
        nrc += colour_delta<ST>(src, tgt, W, H, px, py, ix, fx, iy, fy) < pp.eps;
    }
    nrc = block_count<NT>(nrc, red_i);

    if (tid == 0) {
        const double* Hl = use_refit ? s_Hr : s_Hw;
        // orientation/scale of the evaluation form: denominator 1 at the window centre
        const double dc = Hl[8] - 0.5 * (Hl[6] + Hl[7]);
        double hn[9];
        for (int q = 0; q < 9; ++q) hn[q] = Hl[q] / dc;
        // plane validity: support, positive denominator on the window grown by
        // the patch radius, local area scale at the centre within range
        bool valid = count >= pp.min_inliers && 5 * count >= N;
        const int r = pp.radius;
        const double cxs[2] = {-(double)(s / 2) - r, (double)(s / 2) - 1 + r};
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                if (!(hn[6] * cxs[a] + hn[7] * cxs[b] + hn[8] > 0)) valid = false;
        {
            const double uc = -0.5;
            const double X = hn[0] * uc + hn[1] * uc + hn[2], Y = hn[3] * uc + hn[4] * uc + hn[5];
            const double j00 = hn[0] - X * hn[6], j01 = hn[1] - X * hn[7];
            const double j10 = hn[3] - Y * hn[6], j11 = hn[4] - Y * hn[7];
            const double det = j00 * j11 - j01 * j10;
            if (!(det > 0)) valid = false;
            else {
                const double sc = sqrt(det);
                if (!(sc >= (double)pp.scale_min && sc <= (double)pp.scale_max)) valid = false;
            }
        }
        double Ha[9];
        local_to_abs(Hl, ox, oy, Ha);
        for (int q = 0; q < 9; ++q) pv.mh[dir][(size_t)id * 9 + q] = Ha[q];
        fm.valid = valid ? 1 : 0;
        pv.mef[dir][id] = fm;
        mi[MI_VALID] = valid ? 1 : 0;
        mi[MI_COUNT] = count;
        mi[MI_FLAGS] = F_FITTED | (use_refit ? F_REFIT : 0) | (valid ? 0 : F_BAD_GEOM);
        mi[MI_NRC] = nrc;
    }
}

// ---------------------------------------------------------------- assignment (eq. 3-4)
// For each pixel, over the windows of the level that cover it (window
// order), the valid plane of the given stage maps p to H p; delta is the mean
// absolute RGB difference between I_src(p) and the bilinear I_tgt(H p); the
// pixel is an inlier iff delta < eps, and takes the inlier plane with the
// smallest L = delta (first window on ties), with flow H p - p.
template <int ST>
__global__ void k_assign(PairView pv, LevelGeom g, int stage, int which, int write_resid, PlaneParams pp) {
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
__global__ void k_cue_zero(PairView pv, LevelGeom g, int stage) {
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
__global__ void k_cue_counts(PairView pv, LevelGeom g, int stage, int which, PlaneParams pp) {
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
__global__ void k_cue_invalidate(PairView pv, LevelGeom g, int stage, PlaneParams pp) {
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
__global__ void k_m2o_claim(PairView pv) {
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
__global__ void k_m2o_resolve(PairView pv, PlaneParams pp) {
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
__global__ void k_merge_update(PairView pv, PlaneParams pp) {
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
template <int ST>
__global__ void k_fill(PairView pv, Labels cur0, Labels cur1, Labels nxt0, Labels nxt1, PlaneParams pp) {
    const int dir = blockIdx.y;
    const int W = pv.W, H = pv.H, n = pv.n;
    const Labels cur = dir ? cur1 : cur0, nxt = dir ? nxt1 : nxt0;
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

// Final flow (plane flow, else the NNF offset) and occlusion: no plane, a
// cue flag, or colour error after warping by the final flow >= occ_thresh.
template <int ST>
__global__ void k_final(PairView pv, int dir, PlaneParams pp, float* flow, uint8_t* occ) {
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
__global__ void k_import_models(PairView pv, LevelGeom* geoms, int nlev, int m) {
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
__global__ void k_labels_import(Labels l, int n, const int* im, const float* iL, const double* iF) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        l.m[i] = im[i];
        l.L[i] = iL[i];
        const double fx = iF[2 * i], fy = iF[2 * i + 1];
        const double vx = floor(fx + 0.5), vy = floor(fy + 0.5);
        l.v[i] = make_int2((int)vx, (int)vy);
        l.r[i] = make_float2((float)(fx - vx), (float)(fy - vy));
    }
}

// ---------------------------------------------------------------- launchers
template <int ST>
static void launch_ransac_st(const PairView& pv, const LevelGeom& g, int level, int stage, const PlaneParams& pp,
                             cudaStream_t st) {
    constexpr int NT = 256;
    const size_t smem = (size_t)g.s * g.s * sizeof(float4);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_ransac<NT, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024 + 1024);
        attr_set = true;
    }
    k_ransac<NT, ST><<<dim3(g.ncells(), 2), NT, smem, st>>>(pv, g, level, stage, pp);
}
void launch_ransac(const PairView& pv, const LevelGeom& g, int level, int stage, const PlaneParams& pp,
                   cudaStream_t st) {
    switch (pp.storage) {
        case 0: launch_ransac_st<0>(pv, g, level, stage, pp, st); break;
        case 1: launch_ransac_st<1>(pv, g, level, stage, pp, st); break;
        case 2: launch_ransac_st<2>(pv, g, level, stage, pp, st); break;
    }
}

void launch_assign(const PairView& pv, const LevelGeom& g, int stage, int which, int write_resid,
                   const PlaneParams& pp, int grid_blocks, cudaStream_t st) {
    const dim3 grid(grid_blocks, 2);
    switch (pp.storage) {
        case 0: k_assign<0><<<grid, 256, 0, st>>>(pv, g, stage, which, write_resid, pp); break;
        case 1: k_assign<1><<<grid, 256, 0, st>>>(pv, g, stage, which, write_resid, pp); break;
        case 2: k_assign<2><<<grid, 256, 0, st>>>(pv, g, stage, which, write_resid, pp); break;
    }
}

void launch_cues(const PairView& pv, const LevelGeom& g, int stage, int which, const PlaneParams& pp,
                 int grid_blocks, cudaStream_t st) {
    const int cb = (g.ncells() + 255) / 256;
    k_cue_zero<<<dim3(cb, 2), 256, 0, st>>>(pv, g, stage);
    k_cue_counts<<<dim3(grid_blocks, 2), 256, 0, st>>>(pv, g, stage, which, pp);
    k_cue_invalidate<<<dim3(cb, 2), 256, 0, st>>>(pv, g, stage, pp);
}

void launch_many_to_one(const PairView& pv, const PlaneParams& pp, int grid_blocks, cudaStream_t st) {
    cudaMemsetAsync(pv.m2o_key[0], 0xFF, sizeof(unsigned long long) * pv.n, st);
    cudaMemsetAsync(pv.m2o_key[1], 0xFF, sizeof(unsigned long long) * pv.n, st);
    k_m2o_claim<<<dim3(grid_blocks, 2), 256, 0, st>>>(pv);
    k_m2o_resolve<<<dim3(grid_blocks, 2), 256, 0, st>>>(pv, pp);
}

void launch_merge_update(const PairView& pv, const PlaneParams& pp, int grid_blocks, cudaStream_t st) {
    k_merge_update<<<dim3(grid_blocks, 2), 256, 0, st>>>(pv, pp);
}

void launch_fill(const PairView& pv, const PlaneParams& pp, int iters, int grid_blocks, Labels tmp, cudaStream_t st) {
    (void)tmp;
    // ping-pong between acc and tent (tent is free after the last level)
    Labels a0 = pv.acc[0], a1 = pv.acc[1], b0 = pv.tent[0], b1 = pv.tent[1];
    for (int it = 0; it < iters; ++it) {
        const dim3 grid(grid_blocks, 2);
        switch (pp.storage) {
            case 0: k_fill<0><<<grid, 256, 0, st>>>(pv, a0, a1, b0, b1, pp); break;
            case 1: k_fill<1><<<grid, 256, 0, st>>>(pv, a0, a1, b0, b1, pp); break;
            case 2: k_fill<2><<<grid, 256, 0, st>>>(pv, a0, a1, b0, b1, pp); break;
        }
        Labels t0 = a0, t1 = a1;
        a0 = b0;
        a1 = b1;
        b0 = t0;
        b1 = t1;
    }
    if (iters & 1) {  // result sits in tent: copy back into acc
        for (int d = 0; d < 2; ++d) {
            const Labels s = d ? pv.tent[1] : pv.tent[0], t = d ? pv.acc[1] : pv.acc[0];
            cudaMemcpyAsync(t.m, s.m, sizeof(int) * pv.n, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(t.L, s.L, sizeof(float) * pv.n, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(t.v, s.v, sizeof(int2) * pv.n, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(t.r, s.r, sizeof(float2) * pv.n, cudaMemcpyDeviceToDevice, st);
        }
    }
}

void launch_final(const PairView& pv, const PlaneParams& pp, float* flow, uint8_t* occ, int grid_blocks,
                  cudaStream_t st) {
    switch (pp.storage) {
        case 0: k_final<0><<<grid_blocks, 256, 0, st>>>(pv, 0, pp, flow, occ); break;
        case 1: k_final<1><<<grid_blocks, 256, 0, st>>>(pv, 0, pp, flow, occ); break;
        case 2: k_final<2><<<grid_blocks, 256, 0, st>>>(pv, 0, pp, flow, occ); break;
    }
}

__global__ void k_reset_labels(PairView pv, float eps) {
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
void launch_reset_labels(const PairView& pv, float eps, int grid_blocks, cudaStream_t st) {
    k_reset_labels<<<dim3(grid_blocks, 2), 256, 0, st>>>(pv, eps);
}

template <int ST>
__global__ void k_frames_export(PairView pv, float* dst) {
    const int dir = blockIdx.y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < pv.n; i += gridDim.x * blockDim.x) {
        const float4 a = ldpix<ST>(pv.img[dir], i);
        reinterpret_cast<float4*>(dst)[(size_t)dir * pv.n + i] = a;
    }
}
void launch_frames_export(const PairView& pv, int storage, float* dst, cudaStream_t st) {
    const dim3 grid((pv.n + 255) / 256, 2);
    switch (storage) {
        case 0: k_frames_export<0><<<grid, 256, 0, st>>>(pv, dst); break;
        case 1: k_frames_export<1><<<grid, 256, 0, st>>>(pv, dst); break;
        case 2: k_frames_export<2><<<grid, 256, 0, st>>>(pv, dst); break;
    }
}

void launch_import_models(const PairView& pv, const LevelGeom* geoms, int nlev, int m, cudaStream_t st) {
    k_import_models<<<dim3((m + 255) / 256, 2), 256, 0, st>>>(pv, const_cast<LevelGeom*>(geoms), nlev, m);
}

void launch_labels_export(const Labels& l, int n, int* om, float* oL, double* of, cudaStream_t st) {
    k_labels_export<<<(n + 255) / 256, 256, 0, st>>>(l, n, om, oL, of);
}
void launch_labels_import(const Labels& l, int n, const int* im, const float* iL, const double* iF, cudaStream_t st) {
    k_labels_import<<<(n + 255) / 256, 256, 0, st>>>(l, n, im, iL, iF);
}

}  // namespace gpm
