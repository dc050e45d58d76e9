// Frame ingest and PatchMatch kernels (sm_103a).
//
// PatchMatch (Sec. 3.1; Barnes et al. 2009) with red-black scheduling: one
// launch per half-iteration updates every pixel of one colour from the state
// before the launch (its four neighbours all have the other colour).  One
// warp evaluates one pixel: each lane owns ceil(T/32) taps of the (2r+1)^2
// patch, keeps their source texels in registers for all candidates, and the
// per-candidate cost is one integer reduction of the lanes' sums (rounded to
// 2^-24), identical on every lane, so the accept/reject decision is
// warp-uniform.  At levels >= 1 the patch is
// distorted by the pixel's home-window plane (Sec. 3.3.2 with the plane
// distortion compensation of Sec. 3.1.3): tap d samples the target frame at
// p + v + G(s) - G(p), s = clamp(p + d).
#include "common.cuh"
#include "kernels.h"
#include "../../include/gpm.h"

namespace gpm {

constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------- ingest
// Optional HSV histogram equalisation (Sec. 4.2): V = max(R, G, B) of each
// frame is equalised over 256 bins of [0, 1] (bin = min(255, floor(256 V)),
// V' = (cdf(bin) - cdf_min) / (n - cdf_min), cdf_min the count of the lowest
// occupied bin) with H and S kept.  At fixed H and S the hexcone RGB is
// proportional to V, so the equalised pixel is RGB * V' / V (V' grey for
// black pixels).  A frame with a single occupied bin is left unchanged
// (its table holds -1).
// Element k of an input frame as a float: FP32, FP16 or BF16 (gpm_dtype), each converted exactly.
__device__ __forceinline__ float in_elem(const void* f, int dtype, int64_t k) {
    if (dtype == GPM_F16) return __half2float(reinterpret_cast<const __half*>(f)[k]);
    if (dtype == GPM_BF16) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(f)[k]);
    return reinterpret_cast<const float*>(f)[k];
}

__device__ __forceinline__ int v_bin(float v) {
    float x = floorf(v * 256.f);
    if (!(x >= 0.f)) x = 0.f;
    return (int)fminf(x, 255.f);
}

// Clears the V histograms of the jobs that equalise (blockIdx.z = job).
__global__ void k_vhist_zero(const __grid_constant__ IngestJobs J) {
    const IngestJob& j = J.j[blockIdx.z];
    if (j.hist)
        for (int k = threadIdx.x; k < 2 * 256; k += blockDim.x) j.hist[k] = 0;
}

// V histogram of each frame (blockIdx.y = frame, blockIdx.z = job); hist holds 2 x 256 zeroed counts.
__global__ void k_vhist(const __grid_constant__ IngestJobs J) {
    const IngestJob& j = J.j[blockIdx.z];
    if (!j.hist) return;  // block-uniform
    const int W = j.W, H = j.H;
    const int64_t stride = j.stride;
    int* hist = j.hist;
    __shared__ int h[256];
    for (int k = threadIdx.x; k < 256; k += blockDim.x) h[k] = 0;
    __syncthreads();
    const void* f = blockIdx.y ? j.f2 : j.f1;
    const int n = W * H;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int y = i / W, x = i - y * W;
        const int64_t e = (int64_t)y * stride + 3 * x;
        const float r = in_elem(f, j.dtype, e), g = in_elem(f, j.dtype, e + 1), b = in_elem(f, j.dtype, e + 2);
        atomicAdd(&h[v_bin(fmaxf(r, fmaxf(g, b)))], 1);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 256; k += blockDim.x)
        if (h[k]) atomicAdd(&hist[blockIdx.y * 256 + k], h[k]);
}

// Equalised V per bin (blockIdx.x = frame, blockIdx.z = job, 256 threads): an inclusive scan of the counts.
__global__ void k_vlut(const __grid_constant__ IngestJobs J) {
    const IngestJob& j = J.j[blockIdx.z];
    if (!j.hist) return;  // block-uniform
    const int* hist = j.hist;
    const int n = j.W * j.H;
    float* lut = j.lut;
    __shared__ int c[256];
    __shared__ int cmin;
    const int t = threadIdx.x;
    const int* hf = hist + blockIdx.x * 256;
    c[t] = hf[t];
    if (t == 0) {
        cmin = -1;
        for (int b = 0; b < 256; ++b)
            if (hf[b] > 0) {
                cmin = hf[b];
                break;
            }
    }
    __syncthreads();
    for (int off = 1; off < 256; off <<= 1) {
        const int v = t >= off ? c[t - off] : 0;
        __syncthreads();
        c[t] += v;
        __syncthreads();
    }
    // counts below 2^24 are exact floats, so this is the correctly rounded quotient
    lut[blockIdx.x * 256 + t] = (cmin < 0 || cmin == n) ? -1.f : (float)(c[t] - cmin) / (float)(n - cmin);
}

__device__ __forceinline__ float3 equalize_px(float r, float g, float b, const float* lut) {
    const float v = fmaxf(r, fmaxf(g, b));
    const float l = lut[v_bin(v)];
    if (l < 0.f) return make_float3(r, g, b);
    if (v > 0.f) {
        const float k = l / v;
        return make_float3(r * k, g * k, b * k);
    }
    return make_float3(l, l, l);
}

// ---------------------------------------------------------------- census codes (Sec. 6)
// Grey = R + G + B in FP64 (the same additions as the FP64 oracle, so the
// same values), stored as an orderable integer key: the bits of a
// non-negative double increase with it, negative ones are mirrored; + 0.0
// turns -0 into +0.  The 24 comparisons per pixel then run on the integer
// pipe with exactly the outcomes of comparing the doubles.
__global__ void k_grey_keys(const __grid_constant__ IngestJobs J) {
    const IngestJob& j = J.j[blockIdx.z];
    if (!j.k1) return;  // block-uniform
    const int W = j.W, n = j.W * j.H;
    const int64_t stride = j.stride;
    const void* f = blockIdx.y ? j.f2 : j.f1;
    long long* k = blockIdx.y ? j.k2 : j.k1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int y = i / W, x = i - y * W;
        const int64_t e = (int64_t)y * stride + 3 * x;
        const double g = (((double)in_elem(f, j.dtype, e) + (double)in_elem(f, j.dtype, e + 1)) +
                          (double)in_elem(f, j.dtype, e + 2)) + 0.0;
        const long long b = __double_as_longlong(g);
        k[i] = b >= 0 ? b : (long long)(0x8000000000000000ull - (unsigned long long)b) - 1;
    }
}

// 5x5 census code per pixel: bit k (raster order without the centre, neighbours clamped into the frame) set iff
// the neighbour's grey is below the centre's.
__global__ void k_census(const __grid_constant__ IngestJobs J) {
    const IngestJob& j = J.j[blockIdx.z];
    if (!j.k1) return;  // block-uniform
    const int W = j.W, H = j.H, n = j.W * j.H;
    const long long* k = blockIdx.y ? j.k2 : j.k1;
    uint32_t* c = blockIdx.y ? j.c2 : j.c1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int y = i / W, x = i - y * W;
        const long long kc = k[i];
        uint32_t code = 0;
        int bit = 0;
#pragma unroll
        for (int dy = -2; dy <= 2; ++dy)
#pragma unroll
            for (int dx = -2; dx <= 2; ++dx) {
                if (dx == 0 && dy == 0) continue;
                const int nx = min(max(x + dx, 0), W - 1), ny = min(max(y + dy, 0), H - 1);
                code |= (k[ny * W + nx] < kc ? 1u : 0u) << bit;
                ++bit;
            }
        c[i] = code;
    }
}

// Deterministic FP64 sums of both frames (after equalisation when lut is set): fixed grid, fixed tree
// (blockIdx.z = job).
__global__ void k_frame_sums(const __grid_constant__ IngestJobs J) {
    const IngestJob& j = J.j[blockIdx.z];
    const void* f1 = j.f1;
    const void* f2 = j.f2;
    const int dt = j.dtype;
    const int W = j.W, H = j.H;
    const int64_t stride = j.stride;
    const float* lut = j.hist ? j.lut : nullptr;
    double* partial = j.partial;
    __shared__ double sh[2][256];
    double a = 0, b = 0;
    for (int y = blockIdx.x; y < H; y += gridDim.x) {
        const int64_t r = (int64_t)y * stride;
        if (lut) {
            for (int x = threadIdx.x; x < W; x += blockDim.x) {
                const int64_t e = r + 3 * x;
                const float3 p = equalize_px(in_elem(f1, dt, e), in_elem(f1, dt, e + 1), in_elem(f1, dt, e + 2), lut);
                const float3 q =
                    equalize_px(in_elem(f2, dt, e), in_elem(f2, dt, e + 1), in_elem(f2, dt, e + 2), lut + 256);
                a += (double)p.x + (double)p.y + (double)p.z;
                b += (double)q.x + (double)q.y + (double)q.z;
            }
        } else {
            for (int k = threadIdx.x; k < 3 * W; k += blockDim.x) {
                a += (double)in_elem(f1, dt, r + k);
                b += (double)in_elem(f2, dt, r + k);
            }
        }
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = sh[0][0];
        partial[2 * blockIdx.x + 1] = sh[1][0];
    }
}

__global__ void k_gain(const __grid_constant__ IngestJobs J, int nblk, int enable) {
    const IngestJob& j = J.j[blockIdx.z];
    const double* partial = j.partial;
    double* gain = j.gain;
    if (threadIdx.x != 0) return;
    double a = 0, b = 0;
    for (int i = 0; i < nblk; ++i) {
        a += partial[2 * i];
        b += partial[2 * i + 1];
    }
    *gain = (enable && b > 0) ? a / b : 1.0;
}

template <int ST>
__device__ __forceinline__ void store_pix(void* base, int i, float r, float g, float b) {
    if constexpr (ST == 0) {
        reinterpret_cast<float4*>(base)[i] = make_float4(r, g, b, 0.f);
    } else if constexpr (ST == 1) {
        __half2 lo = __floats2half2_rn(r, g), hi = __floats2half2_rn(b, 0.f);
        uint2 u;
        u.x = *reinterpret_cast<uint32_t*>(&lo);
        u.y = *reinterpret_cast<uint32_t*>(&hi);
        reinterpret_cast<uint2*>(base)[i] = u;
    } else {
        __nv_bfloat162 lo = __floats2bfloat162_rn(r, g), hi = __floats2bfloat162_rn(b, 0.f);
        uint2 u;
        u.x = *reinterpret_cast<uint32_t*>(&lo);
        u.y = *reinterpret_cast<uint32_t*>(&hi);
        reinterpret_cast<uint2*>(base)[i] = u;
    }
}

template <int ST>
__global__ void k_pack(const __grid_constant__ IngestJobs J) {
    const IngestJob& j = J.j[blockIdx.z];
    const void* f1 = j.f1;
    const void* f2 = j.f2;
    const int dt = j.dtype;
    const int W = j.W, H = j.H;
    const int64_t stride = j.stride;
    const float* lut = j.hist ? j.lut : nullptr;
    void* o1 = j.o1;
    void* o2 = j.o2;
    const double g = *j.gain;
    const int n = W * H;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int y = i / W, x = i - y * W;
        const int64_t e = (int64_t)y * stride + 3 * x;
        float3 p = make_float3(in_elem(f1, dt, e), in_elem(f1, dt, e + 1), in_elem(f1, dt, e + 2));
        float3 q = make_float3(in_elem(f2, dt, e), in_elem(f2, dt, e + 1), in_elem(f2, dt, e + 2));
        if (lut) {
            p = equalize_px(p.x, p.y, p.z, lut);
            q = equalize_px(q.x, q.y, q.z, lut + 256);
        }
        store_pix<ST>(o1, i, p.x, p.y, p.z);
        store_pix<ST>(o2, i, (float)((double)q.x * g), (float)((double)q.y * g), (float)((double)q.z * g));
    }
}

// ---------------------------------------------------------------- patch machinery
template <int R>
struct Patch {
    static constexpr int D = 2 * R + 1;
    static constexpr int T = D * D;
    static constexpr int NT = (T + 31) / 32;
};

// Per-lane patch state of one pixel.  Tap j of the lane reads the target at
// (tx + cx, ty + cy) for candidate offset c -- the clamped source pixel for a
// square patch, or the integer part of p + G(s) - G(p) with fraction (fx, fy)
// for a plane-distorted one -- and tidx = ty * W + tx.  [xlo, xhi] x [ylo, yhi]
// bounds every texel the patch touches at offset 0 (including the +1 column
// and row of bilinear taps), so a candidate whose shifted bounds stay inside
// the frame needs no clamping: one add per tap gives the texel index.
template <int R>
struct LanePatch {
    float4 a[Patch<R>::NT];   // source texels of the lane's taps
    uint32_t code[Patch<R>::NT];  // census data term: source codes of the lane's taps
    int tx[Patch<R>::NT], ty[Patch<R>::NT], tidx[Patch<R>::NT];
    float fx[Patch<R>::NT], fy[Patch<R>::NT];
    // offsets c with oxlo <= c.x <= oxlo + oxspan and oylo <= c.y <= oylo + oyspan keep every texel of
    // the patch inside the frame (the unclamped, one-add indexing path)
    int oxlo, oxspan, oylo, oyspan;
    bool warped;
};

// The patch touches texels [xlo, xhi] x [ylo, yhi] at offset 0; offsets keep them inside the frame iff
// -xlo <= c.x <= W-1-xhi (likewise y).  An empty range gets a start no offset reaches.
template <int R>
__device__ __forceinline__ void set_interior_box(LanePatch<R>& lp, int xlo, int xhi, int ylo, int yhi, int W, int H) {
    const int sx = (W - 1 - xhi) + xlo, sy = (H - 1 - yhi) + ylo;
    lp.oxlo = sx >= 0 ? -xlo : (1 << 30);
    lp.oxspan = max(sx, 0);
    lp.oylo = sy >= 0 ? -ylo : (1 << 30);
    lp.oyspan = max(sy, 0);
}

// CENSUS: src holds the frame's census codes (uint32 per pixel) instead of texels.
// Wp > 0: src is a padded copy (row length Wp, border kPad) and the target
// is read from the other frame's copy: tidx then indexes the clamped tap
// there, and a candidate whose target pixel is in the frame needs no clamping
// for any tap (the interior box, in unpadded terms, is then not consulted).
template <int R, int ST, bool CENSUS = false>
__device__ __forceinline__ void load_patch(LanePatch<R>& lp, const void* src, int W, int H, int px, int py,
                                           int lane, int Wp = 0) {
#pragma unroll
    for (int j = 0; j < Patch<R>::NT; ++j) {
        const int t = lane + 32 * j;
        const int tt = t < Patch<R>::T ? t : 0;
        const int dy = tt / Patch<R>::D - R, dx = tt % Patch<R>::D - R;
        lp.tx[j] = min(max(px + dx, 0), W - 1);
        lp.ty[j] = min(max(py + dy, 0), H - 1);
        const int si = lp.ty[j] * W + lp.tx[j];
        lp.tidx[j] = Wp > 0 ? (lp.ty[j] + kPad) * Wp + lp.tx[j] + kPad : si;
        if (CENSUS)
            lp.code[j] = __ldg(reinterpret_cast<const uint32_t*>(src) + si);
        else
            lp.a[j] = ldpix<ST>(src, Wp > 0 ? lp.tidx[j] : si);
        lp.fx[j] = 0.f;
        lp.fy[j] = 0.f;
    }
    set_interior_box(lp, max(px - R, 0), min(px + R, W - 1), max(py - R, 0), min(py + R, H - 1), W, H);
    lp.warped = false;
}

__device__ __forceinline__ int warp_min(int v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = min(v, __shfl_xor_sync(FULL, v, off));
    return v;
}
__device__ __forceinline__ int warp_max(int v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = max(v, __shfl_xor_sync(FULL, v, off));
    return v;
}

// Tap displacements G(s) - G(p) for the plane m at pixel p, from the local
// Jacobian form: with J the derivative of G at p and c = (g0, g1) / den(p),
// G(p + d) - G(p) = J d / (1 + c . d) exactly.
template <int R>
__device__ __forceinline__ void warp_taps(LanePatch<R>& lp, const Mef& m, int px, int py, int W, int H, int lane) {
    const float ux = (float)(px - m.ox), uy = (float)(py - m.oy);
    const float e = m.e0 + m.g0 * ux + m.g1 * uy;
    const float den = 1.f + e;
    const float Sx = m.b0 * ux + m.h1 * uy - ux * e;
    const float Sy = m.h3 * ux + m.b4 * uy - uy * e;
    // local target of p: X = u + D(u)
    const float rden = __frcp_rn(den);
    const float X = ux + (m.h2h + (m.h2l + (Sx - m.h2h * e) * rden));
    const float Y = uy + (m.h5h + (m.h5l + (Sy - m.h5h * e) * rden));
    const float j00 = (1.f + m.b0 - X * m.g0) * rden, j01 = (m.h1 - X * m.g1) * rden;
    const float j10 = (m.h3 - Y * m.g0) * rden, j11 = (1.f + m.b4 - Y * m.g1) * rden;
    const float c0 = m.g0 * rden, c1 = m.g1 * rden;
    int xlo = 1 << 30, xhi = -(1 << 30), ylo = 1 << 30, yhi = -(1 << 30);
#pragma unroll
    for (int j = 0; j < Patch<R>::NT; ++j) {
        const float dx = (float)(lp.tx[j] - px), dy = (float)(lp.ty[j] - py);
        const float rq = __frcp_rn(1.f + c0 * dx + c1 * dy);
        const float ex = (j00 * dx + j01 * dy) * rq;
        const float ey = (j10 * dx + j11 * dy) * rq;
        const float fx = floorf(ex), fy = floorf(ey);
        lp.tx[j] = px + (int)fx;
        lp.ty[j] = py + (int)fy;
        lp.tidx[j] = lp.ty[j] * W + lp.tx[j];
        lp.fx[j] = ex - fx;
        lp.fy[j] = ey - fy;
        if (lane + 32 * j < Patch<R>::T) {
            xlo = min(xlo, lp.tx[j]);
            xhi = max(xhi, lp.tx[j] + 1);
            ylo = min(ylo, lp.ty[j]);
            yhi = max(yhi, lp.ty[j] + 1);
        }
    }
    set_interior_box(lp, warp_min(xlo), warp_max(xhi), warp_min(ylo), warp_max(yhi), W, H);
    lp.warped = true;
}

// Target sample of tap j for candidate offset c (off = c.y * W + c.x).  IN:
// the offset keeps every texel of the patch inside the frame (one add gives
// the index); otherwise the coordinates are clamped.  The caller makes this
// warp-uniform choice once per candidate, outside the tap loop.
template <int R, int ST, bool IN>
__device__ __forceinline__ float3 tap_sample(const LanePatch<R>& lp, const void* tgt, int W, int H, int j, int2 c,
                                             int off) {
    if (!lp.warped) {
        const int idx = IN ? lp.tidx[j] + off
                           : min(max(lp.ty[j] + c.y, 0), H - 1) * W + min(max(lp.tx[j] + c.x, 0), W - 1);
        const float4 v = ldpix<ST>(tgt, idx);
        return make_float3(v.x, v.y, v.z);
    }
    if (IN) {
        const int i0 = lp.tidx[j] + off;
        return blend4(ldpix<ST>(tgt, i0), ldpix<ST>(tgt, i0 + 1), ldpix<ST>(tgt, i0 + W), ldpix<ST>(tgt, i0 + W + 1),
                      lp.fx[j], lp.fy[j]);
    }
    return bilinear<ST>(tgt, W, H, lp.tx[j] + c.x, lp.fx[j], lp.ty[j] + c.y, lp.fy[j]);
}

template <int R>
__device__ __forceinline__ bool interior_of(const LanePatch<R>& lp, int2 c) {
    return (unsigned)(c.x - lp.oxlo) <= (unsigned)lp.oxspan && (unsigned)(c.y - lp.oylo) <= (unsigned)lp.oyspan;
}

// Raw patch cost of offset (vx, vy): the sum over taps and channels of
// |difference|.  The NNF cost buffer holds these sums (strict-less decisions
// compare them directly); the exported cost is the sum divided by 3T.
// The warp's total of the lanes' tap sums: each lane's sum rounded to a
// multiple of 2^-23 and the integers added exactly by one redux, so every
// lane gets the same bits.  A lane's sum is at most 18 (three taps of three
// channels, each |difference| at most 2: frames in [0, 1], a gain below 2),
// so the total of at most 243 channel terms stays below 2^32; it is within
// 32 * 2^-24 = 2^-19 of the exact total of the lane sums, and costs one
// reduction instead of five dependent shuffles and additions.
__device__ __forceinline__ float warp_sum_q23(float s) {
    const unsigned q = __float2uint_rn(s * 8388608.f);
    return (float)__reduce_add_sync(FULL, q) * 1.1920928955078125e-07f;
}

template <int R, int ST, bool IN>
__device__ __forceinline__ float patch_sum_in(const LanePatch<R>& lp, const void* tgt, int W, int H, int2 c, int lane) {
    const int off = c.y * W + c.x;
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < Patch<R>::NT; ++j) {
        const int t = lane + 32 * j;
        if (t < Patch<R>::T) s += absdiff3(lp.a[j], tap_sample<R, ST, IN>(lp, tgt, W, H, j, c, off));
    }
    return warp_sum_q23(s);
}
template <int R, int ST>
__device__ __forceinline__ float patch_sum(const LanePatch<R>& lp, const void* tgt, int W, int H, int px, int py,
                                           int vx, int vy, int lane) {
    const int2 c = make_int2(vx, vy);
    return interior_of<R>(lp, c) ? patch_sum_in<R, ST, true>(lp, tgt, W, H, c, lane)
                                 : patch_sum_in<R, ST, false>(lp, tgt, W, H, c, lane);
}

// ---------------------------------------------------------------- census data term (Sec. 6)
// Square patches only (level 0).  The cost is the sum over taps of the
// Hamming distance of the source and target census codes: an exact integer,
// summed across the warp by one redux, so decisions are exact and the
// abandon test needs no margin (a partial sum at or above the best cannot
// become strictly lower).  Returns false when abandoned; best < 0 never
// abandons.
template <int R, bool IN>
__device__ __forceinline__ bool census_sum_in(const LanePatch<R>& lp, const uint32_t* tgt, int W, int H, int2 c,
                                              int best, int& sum, int lane) {
    const int off = c.y * W + c.x;
    int s = 0;
#pragma unroll
    for (int j = 0; j < Patch<R>::NT; ++j) {
        const int t = lane + 32 * j;
        if (t < Patch<R>::T) {
            const int idx = IN ? lp.tidx[j] + off
                               : min(max(lp.ty[j] + c.y, 0), H - 1) * W + min(max(lp.tx[j] + c.x, 0), W - 1);
            s += __popc(lp.code[j] ^ __ldg(tgt + idx));
        }
        const int tot = (int)__reduce_add_sync(FULL, (unsigned)s);
        if (j + 1 < Patch<R>::NT) {
            if (best >= 0 && tot >= best) return false;
        } else {
            sum = tot;
        }
    }
    return true;
}
template <int R>
__device__ __forceinline__ bool census_sum(const LanePatch<R>& lp, const uint32_t* tgt, int W, int H, int2 c,
                                           int best, int& sum, int lane) {
    return interior_of<R>(lp, c) ? census_sum_in<R, true>(lp, tgt, W, H, c, best, sum, lane)
                                 : census_sum_in<R, false>(lp, tgt, W, H, c, best, sum, lane);
}

// Integer threshold for the abandon test of tap_sum: with thr the best raw
// sum so far, returns ceil(thr * 2^19 * (1 + 2^-21)) + 1.  A partial bound at
// or above it means the exact total of the lane sums is at least
// thr (1 + 2^-21) + 2^-19; the final sum (warp_sum_q23) is within 2^-19 of
// that total and then rounded to a float, so it stays above thr.
__device__ __forceinline__ int abandon_threshold(float thr) {
    return __float2int_ru(__fmul_ru(thr * 524288.f, 1.f + 4.76837158203125e-07f)) + 1;
}

// Raw tap sum of candidate offset c (over taps and channels of |difference|,
// before the division by 3T), abandoned once it cannot win.  After a tested
// 32-tap chunk every lane floors its partial sum to a multiple of 2^-19 and
// the warp adds those integers exactly (one redux): a lower bound of the
// exact partial sum.  The terms are non-negative and FP32 addition is
// monotonic, so a lane's final sum is at least its partial sum; a bound at
// or above `ithr` (abandon_threshold) therefore means the full cost is above
// the best, and the strict-less test would reject the candidate anyway: the
// function returns false.  Each lane accumulates its taps in the same order
// as patch_sum and the total is warp_sum_q24's, so a full sum is bitwise the
// same as patch_sum's.
template <int R, int ST, bool IN, bool EVERY_CHUNK>
__device__ __forceinline__ bool tap_sum_in(const LanePatch<R>& lp, const void* tgt, int W, int H, int2 c, int ithr,
                                        float& sum, int& nch, int lane) {
    const int off = c.y * W + c.x;
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < Patch<R>::NT; ++j) {
        const int t = lane + 32 * j;
        if (t < Patch<R>::T) s += absdiff3(lp.a[j], tap_sample<R, ST, IN>(lp, tgt, W, H, j, c, off));
        if (j + 1 < Patch<R>::NT && EVERY_CHUNK) {
            // floor(min(s * 2^19, 2^23 - 1)): exact scaling, clamp (keeps a lower bound), truncation in the
            // mantissa of 2^23
            const unsigned q =
                (unsigned)(__float_as_int(__fadd_rz(fminf(s * 524288.f, 8388607.f), 8388608.f)) - 0x4B000000);
            if ((int)__reduce_add_sync(FULL, q) >= ithr) {
                nch = j + 1;
                return false;
            }
        }
        if (j + 1 == Patch<R>::NT) sum = warp_sum_q23(s);
    }
    nch = Patch<R>::NT;
    return true;
}
// EVERY_CHUNK: test the bound after every chunk but the last (plane levels, where a chunk costs four gathers per
// tap); otherwise never (level 0, where the patch-sum bound has already removed most losing candidates and a
// test, with its reduction and the predication it puts on every later gather, cost more than it saved).
template <int R, int ST, bool EVERY_CHUNK>
__device__ __forceinline__ bool tap_sum(const LanePatch<R>& lp, const void* tgt, int W, int H, int2 c, int ithr,
                                        float& sum, int& nch, int lane) {
    return interior_of<R>(lp, c) ? tap_sum_in<R, ST, true, EVERY_CHUNK>(lp, tgt, W, H, c, ithr, sum, nch, lane)
                                 : tap_sum_in<R, ST, false, EVERY_CHUNK>(lp, tgt, W, H, c, ithr, sum, nch, lane);
}

// Two candidates at once: each one's taps are accumulated per lane in the
// same order as tap_sum_in, so a full sum is bitwise the same, but the two
// candidates' gathers are issued together and share the latency of each
// chunk.  Both are tested against the same threshold, the best before the
// pair: a bound at or above it means that candidate cannot win against that
// best nor against a lower one, so the caller's in-order strict-less updates
// give the result of evaluating the two one after the other.
template <int R, int ST, bool IN, bool EVERY_CHUNK>
__device__ __forceinline__ void tap_sum2_in(const LanePatch<R>& lp, const void* tgt, int W, int H, int2 c1, int2 c2,
                                            int ithr, float& sum1, float& sum2, bool& ok1, bool& ok2, int& ntap,
                                            int lane) {
    const int off1 = c1.y * W + c1.x, off2 = c2.y * W + c2.x;
    float s1 = 0.f, s2 = 0.f;
    ok1 = ok2 = true;
    ntap = 0;
#pragma unroll
    for (int j = 0; j < Patch<R>::NT; ++j) {
        const int t = lane + 32 * j;
        if (t < Patch<R>::T) {
            float3 v1 = make_float3(0.f, 0.f, 0.f), v2 = v1;
            if (ok1) v1 = tap_sample<R, ST, IN>(lp, tgt, W, H, j, c1, off1);
            if (ok2) v2 = tap_sample<R, ST, IN>(lp, tgt, W, H, j, c2, off2);
            if (ok1) s1 += absdiff3(lp.a[j], v1);
            if (ok2) s2 += absdiff3(lp.a[j], v2);
        }
        if (j + 1 < Patch<R>::NT && EVERY_CHUNK) {
            const unsigned q1 =
                (unsigned)(__float_as_int(__fadd_rz(fminf(s1 * 524288.f, 8388607.f), 8388608.f)) - 0x4B000000);
            const unsigned q2 =
                (unsigned)(__float_as_int(__fadd_rz(fminf(s2 * 524288.f, 8388607.f), 8388608.f)) - 0x4B000000);
            const bool was1 = ok1, was2 = ok2;
            if (ok1) ok1 = (int)__reduce_add_sync(FULL, q1) < ithr;
            if (ok2) ok2 = (int)__reduce_add_sync(FULL, q2) < ithr;
            // taps summed by a candidate abandoned here, for the work counters
            ntap += ((was1 && !ok1) + (was2 && !ok2)) * min(32 * (j + 1), Patch<R>::T);
            if (!ok1 && !ok2) return;
        }
    }
    ntap += (ok1 ? Patch<R>::T : 0) + (ok2 ? Patch<R>::T : 0);
    if (ok1) sum1 = warp_sum_q23(s1);
    if (ok2) sum2 = warp_sum_q23(s2);
}
__device__ __forceinline__ unsigned lanemask_lt(int lane) { return (1u << lane) - 1u; }

// Key of a candidate offset for duplicate detection; lanes without a
// candidate get a key no offset can have.
__device__ __forceinline__ unsigned long long cand_key(bool ok, int2 c, int lane) {
    return ok ? (((unsigned long long)(unsigned)c.x << 32) | (unsigned)c.y) : (0x8000000000000000ull | (unsigned)lane);
}

// Lanes whose candidate is to be evaluated: valid, not the incumbent and not
// a repeat of a lower lane's candidate.  Skipping those changes nothing: the
// cost of an offset is a deterministic function of it, and a repeat can never
// be strictly cheaper than the best so far, which is at most its first cost.
__device__ __forceinline__ unsigned fresh_lanes(bool ok, int2 c, int2 inc, int lane) {
    const unsigned same = __match_any_sync(FULL, cand_key(ok, c, lane));
    const bool keep = ok && !(c.x == inc.x && c.y == inc.y) && (same & lanemask_lt(lane)) == 0;
    return __ballot_sync(FULL, keep);
}

// Home-window plane of p at a level (residual-stage model first), or nullptr.
__device__ __forceinline__ const Mef* home_plane(const LevelGeom& g, const Mef* mef, int x, int y) {
    const int cx = home_index(g.gx, g.s, g.h, x), cy = home_index(g.gy, g.s, g.h, y);
    const int cell = cy * g.gx.count + cx;
    const Mef* m2 = mef + (g.base + cell) * 2 + 1;
    if (m2->valid) return m2;
    const Mef* m1 = mef + (g.base + cell) * 2;
    if (m1->valid) return m1;
    return nullptr;
}

// ---------------------------------------------------------------- init
// The costs of two pixels' candidates at once (patches l1, l2, interior offsets
// c1, c2 into the padded target copy of row length Wp): the same arithmetic per
// pixel as patch_sum_in, with the two pixels' gathers in flight together.
template <int R, int ST>
__device__ __forceinline__ void patch_sum_pair_in(const LanePatch<R>& l1, const LanePatch<R>& l2, const void* tgt,
                                                  int Wp, int H, int2 c1, int2 c2, float& sum1, float& sum2) {
    const int o1 = c1.y * Wp + c1.x, o2 = c2.y * Wp + c2.x;
    float s1 = 0.f, s2 = 0.f;
#pragma unroll
    for (int j = 0; j < Patch<R>::NT; ++j) {
        const int t = (int)(threadIdx.x & 31) + 32 * j;
        if (t < Patch<R>::T) {
            const float3 v1 = tap_sample<R, ST, true>(l1, tgt, Wp, H, j, c1, o1);
            const float3 v2 = tap_sample<R, ST, true>(l2, tgt, Wp, H, j, c2, o2);
            s1 += absdiff3(l1.a[j], v1);
            s2 += absdiff3(l2.a[j], v2);
        }
    }
    sum1 = warp_sum_q23(s1);
    sum2 = warp_sum_q23(s2);
}

template <int R, int ST, bool CENSUS>
__global__ void __launch_bounds__(256) k_pm_init(const __grid_constant__ Batch bt, uint32_t k0, uint32_t k1) {
    const PairView& pv = bt.view(blockIdx.z);
    const int dir = blockIdx.y;
    const int lane = threadIdx.x & 31;
    const int W = pv.W, H = pv.H, n = pv.n;
    const void* src = CENSUS ? (const void*)pv.code[dir] : pv.img[dir];
    const void* tgt = CENSUS ? (const void*)pv.code[1 - dir] : pv.img[1 - dir];
    const int nw = gridDim.x * (blockDim.x >> 5);
    const int first = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if constexpr (!CENSUS) {
        // two pixels per warp and round (i and i + nw): their gathers share the latency
        for (int i = first; i < n; i += 2 * nw) {
            const int i2 = i + nw < n ? i + nw : i;  // warp-uniform; the last odd pixel is computed twice
            const int y1 = i / W, x1 = i - y1 * W, y2 = i2 / W, x2 = i2 - y2 * W;
            const uint32_t tag = stream_tag(RNG_INIT, dir, 0, 0);
            const uint4 w1 = philox((uint32_t)i, 0u, tag, pv.pair_id, k0, k1);
            const uint4 w2 = philox((uint32_t)i2, 0u, tag, pv.pair_id, k0, k1);
            const int2 c1 = make_int2((int)(w1.x % (uint32_t)W) - x1, (int)(w1.y % (uint32_t)H) - y1);
            const int2 c2 = make_int2((int)(w2.x % (uint32_t)W) - x2, (int)(w2.y % (uint32_t)H) - y2);
            LanePatch<R> l1, l2;
            load_patch<R, ST>(l1, pv.imgp[dir], W, H, x1, y1, lane, pv.Wp);
            load_patch<R, ST>(l2, pv.imgp[dir], W, H, x2, y2, lane, pv.Wp);
            float s1, s2;
            patch_sum_pair_in<R, ST>(l1, l2, pv.imgp[1 - dir], pv.Wp, H, c1, c2, s1, s2);
            if (lane == 0) {
                pv.nnf[dir][i] = c1;
                pv.cost[dir][i] = s1;
                pv.nnf[dir][i2] = c2;
                pv.cost[dir][i2] = s2;
                if (pv.evals) atomicAdd(&pv.evals[GPM_COUNT_INIT], i2 != i ? 2ull : 1ull);
            }
        }
        return;
    }
    for (int i = first; i < n; i += nw) {
        const int y = i / W, x = i - y * W;
        const uint4 w = philox((uint32_t)i, 0u, stream_tag(RNG_INIT, dir, 0, 0), pv.pair_id, k0, k1);
        const int vx = (int)(w.x % (uint32_t)W) - x, vy = (int)(w.y % (uint32_t)H) - y;
        LanePatch<R> lp;
        float c;
        if constexpr (CENSUS) {
            load_patch<R, ST, CENSUS>(lp, src, W, H, x, y, lane);
            int sum = 0;
            census_sum<R>(lp, reinterpret_cast<const uint32_t*>(tgt), W, H, make_int2(vx, vy), -1, sum, lane);
            c = (float)sum;
        } else {
            load_patch<R, ST>(lp, pv.imgp[dir], W, H, x, y, lane, pv.Wp);
            c = patch_sum_in<R, ST, true>(lp, pv.imgp[1 - dir], pv.Wp, H, make_int2(vx, vy), lane);
        }
        if (lane == 0) {
            pv.nnf[dir][i] = make_int2(vx, vy);
            pv.cost[dir][i] = c;
            if (pv.evals) atomicAdd(&pv.evals[GPM_COUNT_INIT], 1ull);
        }
    }
}

// ---------------------------------------------------------------- recost (level >= 1)
template <int R, int ST>
__global__ void __launch_bounds__(256) k_pm_recost(const __grid_constant__ Batch bt, int level) {
    const PairView& pv = bt.view(blockIdx.z);
    const LevelGeom g = bt.geom(blockIdx.z, level);
    const int dir = blockIdx.y;
    const int lane = threadIdx.x & 31;
    const int W = pv.W, H = pv.H;
    const void* src = pv.img[dir];
    const void* tgt = pv.img[1 - dir];
    const int nw = gridDim.x * (blockDim.x >> 5);
    const int half = pv.n;  // list capacity per colour
    for (int col = 0; col < 2; ++col) {
        const int cnt = pv.list_count[dir * 2 + col];
        const int* list = pv.list[dir] + col * half;
        for (int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < cnt; w += nw) {
            const int i = list[w];
            const int y = i / W, x = i - y * W;
            LanePatch<R> lp;
            const int2 v = pv.nnf[dir][i];
            float c;
            // the padded copy serves square patches whose target pixel is in the frame (an imported offset
            // need not be)
            if (level > 0 || (unsigned)(x + v.x) >= (unsigned)W || (unsigned)(y + v.y) >= (unsigned)H) {
                load_patch<R, ST>(lp, src, W, H, x, y, lane);
                if (level > 0) {
                    const Mef* G = home_plane(g, pv.mef[dir], x, y);
                    if (G) warp_taps<R>(lp, *G, x, y, W, H, lane);
                }
                c = patch_sum<R, ST>(lp, tgt, W, H, x, y, v.x, v.y, lane);
            } else {
                load_patch<R, ST>(lp, pv.imgp[dir], W, H, x, y, lane, pv.Wp);
                c = patch_sum_in<R, ST, true>(lp, pv.imgp[1 - dir], pv.Wp, H, v, lane);
            }
            if (lane == 0) {
                pv.cost[dir][i] = c;
                if (pv.evals) atomicAdd(&pv.evals[GPM_COUNT_INIT], 1ull);
            }
        }
    }
}

// ---------------------------------------------------------------- patch-sum lower bound (level 0)
// For a pixel p whose patch stays inside the frame and an offset c whose
// target pixel is in the frame, the raw cost is
// sum_t sum_ch |a - b| >= sum_ch |sum_t a - sum_t b| = LB, the sums read from
// the frames' box images (k_box_sums).  A candidate is dropped, without a
// tap, when LB_f - m >= bc (1 + 2^-16) + 2^-18, which allows for rounding on
// both sides: the computed cost C_f is at least C (1 - 2^-18) - 2^-19 (FP32
// sums of at most 9 terms per lane, the 2^-23 rounding of 32 lane sums, one
// conversion), and the exact LB is at least the computed one minus
// m = 2^-19 (sum of both boxes' channels) (each box sum carries at most 16
// FP32 roundings of its own size, then six FP32 operations), so the test
// implies C_f >= bc: the candidate could not be strictly cheaper.
__device__ __forceinline__ float box_lb(float4 b1, float4 b2) {
    const float lb = fabsf(b1.x - b2.x) + fabsf(b1.y - b2.y) + fabsf(b1.z - b2.z);
    const float m = 1.9073486328125e-06f * (((b1.x + b1.y) + b1.z) + ((b2.x + b2.y) + b2.z));
    return lb - m;
}
__device__ __forceinline__ float box_threshold(float bc) {
    return fmaf(bc, 1.52587890625e-05f, bc) + 3.814697265625e-06f;
}

// load_patch for a square colour patch whose source texels are staged in shared memory (tile origin (x0, y0) in
// image coordinates, row length TW): the same taps, target indices into the padded copy (row length Wp).
template <int R, int ST, int TW>
__device__ __forceinline__ void load_patch_tile(LanePatch<R>& lp, const void* tile, int x0, int y0, int W, int H,
                                                int px, int py, int lane, int Wp) {
#pragma unroll
    for (int j = 0; j < Patch<R>::NT; ++j) {
        const int t = lane + 32 * j;
        const int tt = t < Patch<R>::T ? t : 0;
        const int dy = tt / Patch<R>::D - R, dx = tt % Patch<R>::D - R;
        lp.tx[j] = min(max(px + dx, 0), W - 1);
        lp.ty[j] = min(max(py + dy, 0), H - 1);
        lp.tidx[j] = (lp.ty[j] + kPad) * Wp + lp.tx[j] + kPad;
        lp.a[j] = ldpix_shared<ST>(tile, (lp.ty[j] - y0 + R) * TW + lp.tx[j] - x0 + R);
        lp.fx[j] = 0.f;
        lp.fy[j] = 0.f;
    }
    set_interior_box(lp, max(px - R, 0), min(px + R, W - 1), max(py - R, 0), min(py + R, H - 1), W, H);
    lp.warped = false;
}

// ---------------------------------------------------------------- sweep
// PLANES: levels >= 1 (restricted pixel list, plane-distorted patches, plane
// candidates); otherwise level 0 with the census data term (level 0 with
// colour patches runs k_pm_sweep0).
//
// Candidates come in two lists, one candidate per lane, in the fixed order:
// (A) propagation from the left, right, upper and lower neighbours (lanes
// 0-3), then at levels >= 1 the models of the windows covering p in window
// order, first stage then residual stage (lanes 4..21); (B) random search
// around the best offset after A, radius R0 >> k on lane k.  The warp walks
// each list in lane order through one evaluation site (a small kernel body
// keeps the instruction cache warm) and accepts with the strict-less rule.
// CENSUS (level 0 only): the census data term on the frames' code images.
template <int R, int ST, bool PLANES, bool CENSUS>
__global__ void __launch_bounds__(256, 4) k_pm_sweep(const __grid_constant__ Batch bt, int level, int it, int phase, uint32_t k0,
                                                  uint32_t k1) {
    static_assert(!(PLANES && CENSUS), "the census data term is for square patches");
    static_assert(PLANES || CENSUS, "level 0 with colour patches runs k_pm_sweep0");
    __shared__ PairView spv;
    const PairView& pv = shared_view(bt, spv);
    const LevelGeom g = bt.geom(blockIdx.z, level);
    const int dir = blockIdx.y;
    const int lane = threadIdx.x & 31;
    const int W = pv.W, H = pv.H;
    const void* src = CENSUS ? (const void*)pv.code[dir] : pv.img[dir];
    const void* tgt = CENSUS ? (const void*)pv.code[1 - dir] : pv.img[1 - dir];
    int2* __restrict__ nnf = pv.nnf[dir];
    const int nw = gridDim.x * (blockDim.x >> 5);
    const int hw = (W + 1) >> 1;
    const int total = !PLANES ? H * hw : pv.list_count[dir * 2 + phase];
    const int* list = !PLANES ? nullptr : pv.list[dir] + phase * pv.n;
    const int R0 = max(W, H);
    int nrad = 0;  // search radii R0 >> k >= 1
    while ((R0 >> nrad) >= 1) ++nrad;
    const uint32_t tag = stream_tag(RNG_SEARCH, dir, level, 0);
    // Level 0: a block takes tiles of 8 x 8 pixels of this colour (16 x 8 image pixels), its eight warps one
    // row of the tile per round, so that successive rounds reuse the target region already in the SM's L1.
    // Plane levels: the compacted pixel list, grid-strided.
    const int wid = threadIdx.x >> 5;
    const int ntx = (hw + 7) >> 3, ntiles = ntx * ((H + 7) >> 3);
    for (int rnd = 0;; ++rnd) {
        int x, y, i;
        if (!PLANES) {
            const int tile = blockIdx.x + (rnd >> 3) * gridDim.x;
            if (tile >= ntiles) break;  // block-uniform
            const int ty = tile / ntx, tx = tile - ty * ntx;
            y = 8 * ty + (rnd & 7);
            const int xh = 8 * tx + wid;
            if (y >= H || xh >= hw) continue;
            x = 2 * xh + ((y + phase) & 1);
            if (x >= W) continue;
            i = y * W + x;
        } else {
            const int w = blockIdx.x * (blockDim.x >> 5) + wid + rnd * nw;
            if (w >= total) break;
            i = list[w];
            y = i / W;
            x = i - y * W;
        }
        LanePatch<R> lp;
        load_patch<R, ST, CENSUS>(lp, src, W, H, x, y, lane);
        if (PLANES) {
            const Mef* G = home_plane(g, pv.mef[dir], x, y);
            if (G) warp_taps<R>(lp, *G, x, y, W, H, lane);
        }
        int2 best = nnf[i];
        float bc = pv.cost[dir][i];  // raw sum of the incumbent
        int ithr = CENSUS ? 0 : abandon_threshold(bc);
        int nev = 0, ntap = 0;
        // list A
        int2 cand = make_int2(0, 0);
        bool ok = false;
        if (lane < 4) {
            const int nx = x + (lane == 0 ? -1 : (lane == 1 ? 1 : 0));
            const int ny = y + (lane == 2 ? -1 : (lane == 3 ? 1 : 0));
            if (nx >= 0 && nx < W && ny >= 0 && ny < H) {
                cand = nnf[ny * W + nx];
                const int tx = x + cand.x, ty = y + cand.y;
                ok = tx >= 0 && tx < W && ty >= 0 && ty < H;
            }
        } else if (PLANES && lane < 4 + 18) {
            int fx0, nrx, fy0, nry;
            const int nxw = covering_range(g.gx, g.s, g.h, x, fx0, nrx);
            const int nyw = covering_range(g.gy, g.s, g.h, y, fy0, nry);
            const int j = lane - 4, st = j & 1, wk = j >> 1;       // window wk of at most 3 x 3, stage st
            const int a = nxw == 1 ? wk : (nxw == 2 ? wk >> 1 : (wk * 11) >> 5);  // wk / nxw for wk < 9
            const int b = wk - a * nxw;
            if (nxw > 0 && a < nyw) {
                const int cell = covering_at(g.gy, fy0, nry, a) * g.gx.count + covering_at(g.gx, fx0, nrx, b);
                const Mef m = pv.mef[dir][(g.base + cell) * 2 + st];
                int kx, ky;
                float fx, fy;
                if (m.valid && mef_flow(m, (float)(x - m.ox), (float)(y - m.oy), kx, fx, ky, fy)) {
                    float rx, ry;
                    round_split(kx, fx, cand.x, rx);
                    round_split(ky, fy, cand.y, ry);
                    const int tx = x + cand.x, ty = y + cand.y;
                    ok = tx >= 0 && tx < W && ty >= 0 && ty < H;
                }
            }
        }
        unsigned todo = fresh_lanes(ok, cand, best, lane);
#pragma unroll 1
        for (int list_b = 0; list_b < 2; ++list_b) {
            if (list_b) {
                // list B: random search around v0, the best offset after list A
                const int2 v0 = best;
                // random words for the search radii, two radii per Philox call, one call per lane
                uint4 rw = make_uint4(0, 0, 0, 0);
                if (lane < (nrad + 1) / 2)
                    rw = philox((uint32_t)i, ((uint32_t)it << 8) | (uint32_t)lane, tag, pv.pair_id, k0, k1);
                const int src_lane = lane >> 1;
                uint32_t wx = __shfl_sync(FULL, rw.x, src_lane), wy = __shfl_sync(FULL, rw.y, src_lane);
                const uint32_t wz = __shfl_sync(FULL, rw.z, src_lane), ww = __shfl_sync(FULL, rw.w, src_lane);
                if (lane & 1) {
                    wx = wz;
                    wy = ww;
                }
                const int Rk = R0 >> lane;
                const int ox = (int)bounded_u32(wx, (uint32_t)(2 * Rk + 1)) - Rk;
                const int oy = (int)bounded_u32(wy, (uint32_t)(2 * Rk + 1)) - Rk;
                const int tx = min(max(x + v0.x + ox, 0), W - 1), ty = min(max(y + v0.y + oy, 0), H - 1);
                cand = make_int2(tx - x, ty - y);
                todo = fresh_lanes(lane < nrad, cand, v0, lane);
            }
            while (todo) {
                const int l = __ffs(todo) - 1;
                todo &= todo - 1;
                const int2 c = make_int2(__shfl_sync(FULL, cand.x, l), __shfl_sync(FULL, cand.y, l));
                if constexpr (CENSUS) {
                    int sum;  // exact integer costs: the incumbent's sum is an integer held in a float
                    if (census_sum<R>(lp, reinterpret_cast<const uint32_t*>(tgt), W, H, c, (int)bc, sum, lane) &&
                        sum < (int)bc) {
                        bc = (float)sum;
                        best = c;
                    }
                } else {
                    float sum;
                    int nch;
                    const bool done = tap_sum<R, ST, PLANES>(lp, tgt, W, H, c, ithr, sum, nch, lane);
                    ntap += min(32 * nch, Patch<R>::T);
                    if (done && sum < bc) {
                        bc = sum;
                        best = c;
                        ithr = abandon_threshold(bc);
                    }
                }
                ++nev;
            }
        }
        if (lane == 0) {
            nnf[i] = best;
            pv.cost[dir][i] = bc;
            if (pv.evals) {
                atomicAdd(&pv.evals[PLANES ? GPM_COUNT_SWEEP_PLANE : GPM_COUNT_SWEEP0], (unsigned long long)nev);
                atomicAdd(&pv.evals[PLANES ? GPM_COUNT_SWEEP_PLANE_TAPS : GPM_COUNT_SWEEP0_TAPS],
                          (unsigned long long)(CENSUS ? nev * Patch<R>::T : ntap));
            }
        }
    }
}

// ---------------------------------------------------------------- level-0 sweep, two layouts
// Tiles of the level-0 sweep: 16 pixels of one colour by 8 rows (32 x 8 image pixels), each of the block's four
// warps owning two rows, one pixel per lane.  The staged source region is the tile grown by r, in rows of TW
// texels (TW congruent to 2r + 1 modulo 8, so that eight consecutive taps of a patch row fall on eight distinct
// 16-byte bank groups).
template <int R>
struct Tile0L {
    static constexpr int TXC = 16, TY = 8, TX = 2 * TXC, WARPS = 4;
    static constexpr int TW0 = TX + 2 * R;
    static constexpr int TW = TW0 + ((2 * R + 1 - TW0) % 8 + 8) % 8;
    static constexpr int TH = TY + 2 * R;
};
// Search radii R0 >> k >= 1 for frames below 2^15 pixels a side: at most 15.
constexpr int kMaxRadii = 16;

int sweep0_tiles(int W, int H) {
    const int hw = (W + 1) >> 1;
    return ((hw + Tile0L<1>::TXC - 1) / Tile0L<1>::TXC) * ((H + Tile0L<1>::TY - 1) / Tile0L<1>::TY);
}

// A candidate offset in one word (|c.x|, |c.y| < 2^15 for frames below 2^15 pixels a side).
__device__ __forceinline__ uint32_t pack_off(int2 c) { return (uint32_t)(uint16_t)c.x | ((uint32_t)c.y << 16); }
__device__ __forceinline__ int2 unpack_off(uint32_t k) { return make_int2((int)(int16_t)(k & 0xFFFFu), (int)k >> 16); }

// Appends candidate c to a pixel's list (column `lane` of list[k][32]) unless an earlier entry holds it.
__device__ __forceinline__ void list_push(uint32_t (*list)[32], int& n, int2 c, int lane) {
    const uint32_t key = pack_off(c);
    bool dup = false;
    for (int k = 0; k < n; ++k) dup |= list[k][lane] == key;
    if (!dup) list[n++][lane] = key;
}

// Raw tap sums of N candidate offsets of one square patch (off[q] = c.y * Wp + c.x into the padded target copy),
// all in full: each lane accumulates its taps in the order of tap_sum_in and the totals are warp_sum_q23's, so
// each sum is bitwise tap_sum_in's; the N candidates' gathers of a chunk are in flight together.
template <int R, int ST, int N>
__device__ __forceinline__ void tap_sums_sq(const LanePatch<R>& lp, const void* tgtp, const int* off, float* sum,
                                            int lane) {
    float s[N];
#pragma unroll
    for (int q = 0; q < N; ++q) s[q] = 0.f;
#pragma unroll
    for (int j = 0; j < Patch<R>::NT; ++j) {
        if (lane + 32 * j < Patch<R>::T) {
            float4 v[N];
#pragma unroll
            for (int q = 0; q < N; ++q) v[q] = ldpix<ST>(tgtp, lp.tidx[j] + off[q]);
#pragma unroll
            for (int q = 0; q < N; ++q) s[q] += absdiff3(lp.a[j], make_float3(v[q].x, v[q].y, v[q].z));
        }
    }
#pragma unroll
    for (int q = 0; q < N; ++q) sum[q] = warp_sum_q23(s[q]);
}

// Maximum number of one pixel's candidates whose costs are summed together.
constexpr int kSweep0Group = 3;

template <int R, int ST, int N>
__device__ __forceinline__ void eval_group(const LanePatch<R>& lp, const void* tgtp, int Wp,
                                           const uint32_t (*list)[32], int p, int k, int2& best, float& bc) {
    int2 c[N];
    int off[N];
    float sum[N];
#pragma unroll
    for (int q = 0; q < N; ++q) {
        c[q] = unpack_off(list[k + q][p]);
        off[q] = c[q].y * Wp + c[q].x;
    }
    tap_sums_sq<R, ST, N>(lp, tgtp, off, sum, (int)(threadIdx.x & 31));
#pragma unroll
    for (int q = 0; q < N; ++q)
        if (sum[q] < bc) {
            bc = sum[q];
            best = c[q];
        }
}

// The warp (one tap per lane) evaluates the n listed candidates of one pixel in list order, up to kSweep0Group
// at a time, with the strict-less rule (every cost summed in full, then the updates in list order): best / bc
// are warp-uniform on entry and on return.
template <int R, int ST>
__device__ __forceinline__ void eval_listed(const LanePatch<R>& lp, const void* tgtp, int Wp,
                                            const uint32_t (*list)[32], int p, int n, int2& best, float& bc,
                                            unsigned& nev, unsigned& ntap) {
    for (int k = 0; k < n;) {
        const int g = min(n - k, kSweep0Group);
        if (g >= 4)
            eval_group<R, ST, 4>(lp, tgtp, Wp, list, p, k, best, bc);
        else if (g == 3)
            eval_group<R, ST, 3>(lp, tgtp, Wp, list, p, k, best, bc);
        else if (g == 2)
            eval_group<R, ST, 2>(lp, tgtp, Wp, list, p, k, best, bc);
        else
            eval_group<R, ST, 1>(lp, tgtp, Wp, list, p, k, best, bc);
        k += g;
        nev += g;
        ntap += g * Patch<R>::T;
    }
}

// Level-0 sweep with square colour patches (Sec. 3.1), one colour of the red-black schedule per launch.  Each
// pixel's candidates come in two lists: (A) propagation, the offsets of its left, right, upper and lower
// neighbours; (B) random search around the best offset after A, radius R0 >> k for k = 0, 1, ... (Philox words,
// two radii per call).  A candidate replaces the best only if its raw tap sum is strictly lower, in list order;
// candidates that repeat the best or an earlier entry, or that the patch-sum bound rules out, cannot win and are
// not listed.  The per-pixel scalar work runs with one pixel per lane: the neighbours' offsets, the Philox words
// and the search candidates, the bound and the removal of repeats, into a list per pixel in shared memory.  The
// patch costs run with one tap per lane, the warp walking its 32 pixels' lists in turn; list B is built once
// list A is evaluated for all 32 pixels.
template <int R, int ST>
__global__ void __launch_bounds__(128, 6) k_pm_sweep0(const __grid_constant__ Batch bt, int it, int phase,
                                                      uint32_t k0, uint32_t k1) {
    using TL = Tile0L<R>;
    using Tex = typename TexelOf<ST>::type;
    __shared__ Tex stile[TL::TH * TL::TW];
    __shared__ uint32_t slist[TL::WARPS][kMaxRadii][32];
    const PairView& pv = bt.view(blockIdx.z);
    const int dir = blockIdx.y;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int W = pv.W, H = pv.H, Wp = pv.Wp;
    const int hw = (W + 1) >> 1;
    const int ntx = (hw + TL::TXC - 1) / TL::TXC, nty = (H + TL::TY - 1) / TL::TY;
    if ((int)blockIdx.x >= ntx * nty) return;  // block-uniform: the grid covers the largest pair of the batch
    const int tyi = blockIdx.x / ntx, txi = blockIdx.x - tyi * ntx;
    const int x0 = TL::TX * txi, y0 = TL::TY * tyi;
    {
        // the tile's source region, from the padded copy (entries past its edge are clamped and unused)
        const Tex* sp = reinterpret_cast<const Tex*>(pv.imgp[dir]);
        const int Hp = H + 2 * kPad;
        for (int e = threadIdx.x; e < TL::TH * TL::TW; e += blockDim.x) {
            const int ly = e / TL::TW, lx = e - ly * TL::TW;
            const int gx = min(x0 - R + lx + kPad, Wp - 1), gy = min(y0 - R + ly + kPad, Hp - 1);
            stile[e] = sp[gy * Wp + gx];
        }
    }
    __syncthreads();
    const void* tgtp = pv.imgp[1 - dir];
    uint32_t(*list)[32] = slist[wid];
    int2* __restrict__ nnf = pv.nnf[dir];
    const float4* __restrict__ boxt = pv.box[1 - dir];
    // the lane's pixel
    const int yq = y0 + 2 * wid + (lane >> 4);
    const int xq = 2 * (TL::TXC * txi + (lane & 15)) + ((yq + phase) & 1);
    const bool mine = yq < H && xq < W;
    const int iq = mine ? yq * W + xq : 0;
    int2 best = make_int2(0, 0);
    float bc = 0.f;
    if (mine) {
        best = nnf[iq];
        bc = pv.cost[dir][iq];
    }
    // interior pixels: the patch-sum bound applies
    const bool prune = mine && xq >= R && yq >= R && xq < W - R && yq < H - R;
    const float4 b1 = prune ? pv.box[dir][iq] : make_float4(0.f, 0.f, 0.f, 0.f);
    unsigned npr = 0, nev = 0, ntap = 0;
    // list A, one pixel per lane: the four neighbours' offsets whose target is in the frame, neither the
    // incumbent nor a repeat, and not excluded by the bound
    int n = 0;
    if (mine) {
        const float thr = box_threshold(bc);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int nx = xq + (k == 0 ? -1 : (k == 1 ? 1 : 0));
            const int ny = yq + (k == 2 ? -1 : (k == 3 ? 1 : 0));
            if (nx < 0 || nx >= W || ny < 0 || ny >= H) continue;
            const int2 c = nnf[ny * W + nx];
            const int tx = xq + c.x, ty = yq + c.y;
            if (tx < 0 || tx >= W || ty < 0 || ty >= H || (c.x == best.x && c.y == best.y)) continue;
            if (prune && box_lb(b1, boxt[iq + c.y * W + c.x]) >= thr) {
                ++npr;
                continue;
            }
            list_push(list, n, c, lane);
        }
    }
    __syncwarp();
    // list A, one tap per lane, pixel by pixel
    for (int p = 0; p < 32; ++p) {
        const int np_ = __shfl_sync(FULL, n, p);
        if (np_ == 0) continue;  // warp-uniform
        const int yp = y0 + 2 * wid + (p >> 4);
        const int xp = 2 * (TL::TXC * txi + (p & 15)) + ((yp + phase) & 1);
        LanePatch<R> lp;
        load_patch_tile<R, ST, TL::TW>(lp, stile, x0, y0, W, H, xp, yp, lane, Wp);
        int2 b = make_int2(__shfl_sync(FULL, best.x, p), __shfl_sync(FULL, best.y, p));
        float c = __shfl_sync(FULL, bc, p);
        eval_listed<R, ST>(lp, tgtp, Wp, list, p, np_, b, c, nev, ntap);
        if (lane == p) {
            best = b;
            bc = c;
        }
    }
    __syncwarp();
    // list B, one pixel per lane: random search around v0, the best offset after list A (Philox words two radii
    // per call, as in k_pm_sweep)
    n = 0;
    if (mine) {
        const int2 v0 = best;
        const int R0 = max(W, H);
        int nrad = 0;
        while ((R0 >> nrad) >= 1) ++nrad;
        const uint32_t tag = stream_tag(RNG_SEARCH, dir, 0, 0);
        const float thr = box_threshold(bc);
        for (int call = 0; 2 * call < nrad; ++call) {
            const uint4 rw = philox((uint32_t)iq, ((uint32_t)it << 8) | (uint32_t)call, tag, pv.pair_id, k0, k1);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = 2 * call + h;
                if (k >= nrad) break;
                const uint32_t wx = h ? rw.z : rw.x, wy = h ? rw.w : rw.y;
                const int Rk = R0 >> k;
                const int ox = (int)bounded_u32(wx, (uint32_t)(2 * Rk + 1)) - Rk;
                const int oy = (int)bounded_u32(wy, (uint32_t)(2 * Rk + 1)) - Rk;
                const int tx = min(max(xq + v0.x + ox, 0), W - 1), ty = min(max(yq + v0.y + oy, 0), H - 1);
                const int2 c = make_int2(tx - xq, ty - yq);
                if (c.x == v0.x && c.y == v0.y) continue;
                if (prune && box_lb(b1, boxt[iq + c.y * W + c.x]) >= thr) {
                    ++npr;
                    continue;
                }
                list_push(list, n, c, lane);
            }
        }
    }
    __syncwarp();
    for (int p = 0; p < 32; ++p) {
        const int np_ = __shfl_sync(FULL, n, p);
        if (np_ == 0) continue;
        const int yp = y0 + 2 * wid + (p >> 4);
        const int xp = 2 * (TL::TXC * txi + (p & 15)) + ((yp + phase) & 1);
        LanePatch<R> lp;
        load_patch_tile<R, ST, TL::TW>(lp, stile, x0, y0, W, H, xp, yp, lane, Wp);
        int2 b = make_int2(__shfl_sync(FULL, best.x, p), __shfl_sync(FULL, best.y, p));
        float c = __shfl_sync(FULL, bc, p);
        eval_listed<R, ST>(lp, tgtp, Wp, list, p, np_, b, c, nev, ntap);
        if (lane == p) {
            best = b;
            bc = c;
        }
    }
    if (mine) {
        nnf[iq] = best;
        pv.cost[dir][iq] = bc;
    }
    if (pv.evals) {
        const unsigned npw = __reduce_add_sync(FULL, npr);
        if (lane == 0) {
            atomicAdd(&pv.evals[GPM_COUNT_SWEEP0], (unsigned long long)nev);
            atomicAdd(&pv.evals[GPM_COUNT_SWEEP0_TAPS], (unsigned long long)ntap);
            if (npw) atomicAdd(&pv.evals[GPM_COUNT_SWEEP0_PRUNED], (unsigned long long)npw);
        }
    }
}

// Unfrozen pixels of each colour, for the restricted sweeps (order is free:
// pixels of one colour are independent within a half-iteration).
__global__ void k_lists_zero(const __grid_constant__ Batch bt) {
    if (threadIdx.x < 4) bt.view(blockIdx.z).list_count[threadIdx.x] = 0;
}
__global__ void k_build_lists(const __grid_constant__ Batch bt) {
    const PairView& pv = bt.view(blockIdx.z);
    const int dir = blockIdx.y;
    const int n = pv.n, W = pv.W;
    const int lane = threadIdx.x & 31;
    for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const int i = base + threadIdx.x;
        bool ok = false;
        int col = 0;
        if (i < n) {
            ok = !pv.frozen[dir][i];
            const int y = i / W, x = i - y * W;
            col = (x + y) & 1;
        }
        for (int c = 0; c < 2; ++c) {
            const unsigned mask = __ballot_sync(FULL, ok && col == c);
            if (!mask) continue;
            int off = 0;
            if (lane == 0) off = atomicAdd(&pv.list_count[dir * 2 + c], __popc(mask));
            off = __shfl_sync(FULL, off, 0);
            if (ok && col == c) pv.list[dir][c * n + off + __popc(mask & ((1u << lane) - 1))] = i;
        }
    }
}

// ---------------------------------------------------------------- launchers
template <int R, int ST>
static void launch_pm_r(const PmLaunch& L, cudaStream_t st) {
    const dim3 grid(L.grid_blocks, 2, L.np), block(256);
    switch (L.op) {
        case PmLaunch::INIT:  // census codes do not depend on the texel storage: one instance serves all
            if (L.census)
                k_pm_init<R, 0, true><<<grid, block, 0, st>>>(L.bt, L.k0, L.k1);
            else
                k_pm_init<R, ST, false><<<grid, block, 0, st>>>(L.bt, L.k0, L.k1);
            break;
        case PmLaunch::RECOST:
            k_pm_recost<R, ST><<<grid, block, 0, st>>>(L.bt, L.level);
            break;
        case PmLaunch::SWEEP:
            if (L.level == 0 && L.census)
                k_pm_sweep<R, 0, false, true><<<grid, block, 0, st>>>(L.bt, 0, L.it, L.phase, L.k0, L.k1);
            else if (L.level == 0)
                k_pm_sweep0<R, ST><<<dim3(L.tiles0, 2, L.np), dim3(32 * Tile0L<R>::WARPS), 0, st>>>(L.bt, L.it, L.phase,
                                                                                                  L.k0, L.k1);
            else
                k_pm_sweep<R, ST, true, false><<<grid, block, 0, st>>>(L.bt, L.level, L.it, L.phase, L.k0, L.k1);
            break;
    }
}

template <int ST>
static void launch_pm_st(const PmLaunch& L, cudaStream_t st) {
    switch (L.radius) {
        case 1: launch_pm_r<1, ST>(L, st); break;
        case 2: launch_pm_r<2, ST>(L, st); break;
        case 3: launch_pm_r<3, ST>(L, st); break;
        case 4: launch_pm_r<4, ST>(L, st); break;
        default: break;
    }
}

void launch_pm(const PmLaunch& L, cudaStream_t st) {
    switch (L.storage) {
        case 0: launch_pm_st<0>(L, st); break;
        case 1: launch_pm_st<1>(L, st); break;
        case 2: launch_pm_st<2>(L, st); break;
    }
}

// Greys of frame 1 as given, for the edge-aware fill (the jobs that ask for them).
__global__ void k_grey_q(const __grid_constant__ IngestJobs J) {
    const IngestJob& j = J.j[blockIdx.z];
    if (!j.gq) return;
    const int W = j.W, n = j.W * j.H;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int y = i / W, x = i - y * W;
        const int64_t e = (int64_t)y * j.stride + 3 * x;
        j.gq[i] = (int)floor(1024.0 * (((double)in_elem(j.f1, j.dtype, e) + (double)in_elem(j.f1, j.dtype, e + 1)) +
                                       (double)in_elem(j.f1, j.dtype, e + 2)));
    }
}

// The ingest of nj pairs, each kernel one launch over the jobs (blockIdx.z).  Per job the grid and the order
// of every reduction are those of a single pair's ingest, so each result is the same alone and in a batch.
void launch_ingest_jobs(const IngestJobs& J, int nj, int max_n, int max_h, int gain_enable, int storage,
                        cudaStream_t st) {
    (void)max_n;
    (void)max_h;
    const int blocks = 152 * 4;
    bool eq = false, census = false, grey = false;
    for (int k = 0; k < nj; ++k) {
        eq |= J.j[k].hist != nullptr;
        census |= J.j[k].k1 != nullptr;
        grey |= J.j[k].gq != nullptr;
    }
    if (census) {
        k_grey_keys<<<dim3(blocks, 2, nj), 256, 0, st>>>(J);
        k_census<<<dim3(blocks, 2, nj), 256, 0, st>>>(J);
    }
    if (grey) k_grey_q<<<dim3(blocks, 1, nj), 256, 0, st>>>(J);
    if (eq) {
        k_vhist_zero<<<dim3(1, 1, nj), 256, 0, st>>>(J);
        k_vhist<<<dim3(blocks, 2, nj), 256, 0, st>>>(J);
        k_vlut<<<dim3(2, 1, nj), 256, 0, st>>>(J);
    }
    k_frame_sums<<<dim3(kIngestPartialBlocks, 1, nj), 256, 0, st>>>(J);
    k_gain<<<dim3(1, 1, nj), 32, 0, st>>>(J, kIngestPartialBlocks, gain_enable);
    switch (storage) {
        case 0: k_pack<0><<<dim3(blocks, 1, nj), 256, 0, st>>>(J); break;
        case 1: k_pack<1><<<dim3(blocks, 1, nj), 256, 0, st>>>(J); break;
        case 2: k_pack<2><<<dim3(blocks, 1, nj), 256, 0, st>>>(J); break;
    }
}

void launch_ingest(const float* f1, const float* f2, int W, int H, int64_t stride, int gain_enable, int storage,
                   double* partial, int nblk, double* gain, void* o1, void* o2, int* eq_hist, float* eq_lut,
                   cudaStream_t st) {
    (void)nblk;  // always kIngestPartialBlocks
    IngestJobs J{};
    J.j[0] = IngestJob{f1, f2, GPM_F32, W, H, stride, partial, gain, o1, o2, eq_lut ? eq_hist : nullptr, eq_lut,
                       nullptr, nullptr, nullptr, nullptr, nullptr};
    launch_ingest_jobs(J, 1, W * H, H, gain_enable, storage, st);
}

// Padded copy of each ingested frame: texel (x, y) of the copy, for x in
// [-kPad, W + kPad) and y in [-kPad, H + kPad), is the frame's texel at the
// clamped coordinates (T: one texel, 16 or 8 bytes).
template <typename T>
__global__ void k_pad_frames(const __grid_constant__ Batch bt) {
    const PairView& pv = bt.view(blockIdx.z);
    const int dir = blockIdx.y;
    const T* src = reinterpret_cast<const T*>(pv.img[dir]);
    T* dst = reinterpret_cast<T*>(const_cast<void*>(pv.imgp[dir]));
    const int W = pv.W, H = pv.H, Wp = pv.Wp, np = Wp * (H + 2 * kPad);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
        const int yp = i / Wp, xp = i - yp * Wp;
        const int x = min(max(xp - kPad, 0), W - 1), y = min(max(yp - kPad, 0), H - 1);
        dst[i] = src[y * W + x];
    }
}
// Patch sums of each ingested frame: box[q] = the RGB sums over the (2r+1)^2 taps of q's patch, taps clamped
// into the frame (read from the padded copy).  For a pixel p whose patch stays inside the frame and an offset c
// whose target pixel is in the frame, the level-0 cost's taps are exactly these patches' texels, so
// sum_ch |box1(p)_ch - box2(p + c)_ch| bounds the raw cost from below.  Separable, in FP32: a block stages a
// 32 x 8 tile and its r-halo, sums each row's 2r + 1 texels, then each column's 2r + 1 row sums, in a fixed order
// (at most 16 FP32 roundings per sum, which the sweep's test allows for).
template <int R, int ST>
__global__ void __launch_bounds__(256) k_box_sums(const __grid_constant__ Batch bt) {
    constexpr int BX = 32, BY = 8, TWB = BX + 2 * R, THB = BY + 2 * R;
    __shared__ float3 tex[THB][TWB];
    __shared__ float3 hs[THB][BX];
    const PairView& pv = bt.view(blockIdx.z >> 1);  // blockIdx.z = 2 pair + direction
    const int dir = blockIdx.z & 1;
    const int W = pv.W, H = pv.H, Wp = pv.Wp, Hp = H + 2 * kPad;
    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
    if (x0 >= W || y0 >= H) return;  // past this pair's frame (block-uniform)
    for (int e = threadIdx.x; e < THB * TWB; e += blockDim.x) {
        const int ly = e / TWB, lx = e - ly * TWB;
        const int gx = min(x0 - R + lx + kPad, Wp - 1), gy = min(y0 - R + ly + kPad, Hp - 1);
        const float4 v = ldpix<ST>(pv.imgp[dir], gy * Wp + gx);
        tex[ly][lx] = make_float3(v.x, v.y, v.z);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < THB * BX; e += blockDim.x) {
        const int ly = e / BX, lx = e - ly * BX;
        float3 a = tex[ly][lx];
#pragma unroll
        for (int d = 1; d <= 2 * R; ++d) {
            const float3 v = tex[ly][lx + d];
            a.x += v.x;
            a.y += v.y;
            a.z += v.z;
        }
        hs[ly][lx] = a;
    }
    __syncthreads();
    const int lx = threadIdx.x & (BX - 1), ly = threadIdx.x / BX;
    const int x = x0 + lx, y = y0 + ly;
    if (x < W && y < H) {
        float3 a = hs[ly][lx];
#pragma unroll
        for (int d = 1; d <= 2 * R; ++d) {
            const float3 v = hs[ly + d][lx];
            a.x += v.x;
            a.y += v.y;
            a.z += v.z;
        }
        pv.box[dir][y * W + x] = make_float4(a.x, a.y, a.z, 0.f);
    }
}
template <int ST>
static void launch_box_st(const Batch& bt, dim3 grid, int radius, cudaStream_t st) {
    switch (radius) {
        case 1: k_box_sums<1, ST><<<grid, 256, 0, st>>>(bt); break;
        case 2: k_box_sums<2, ST><<<grid, 256, 0, st>>>(bt); break;
        case 3: k_box_sums<3, ST><<<grid, 256, 0, st>>>(bt); break;
        case 4: k_box_sums<4, ST><<<grid, 256, 0, st>>>(bt); break;
    }
}
void launch_box_sums(const Batch& bt, int np, int max_w, int max_h, int radius, int storage, cudaStream_t st) {
    const dim3 grid((max_w + 31) / 32, (max_h + 7) / 8, 2 * np);
    switch (storage) {
        case 0: launch_box_st<0>(bt, grid, radius, st); break;
        case 1: launch_box_st<1>(bt, grid, radius, st); break;
        case 2: launch_box_st<2>(bt, grid, radius, st); break;
    }
}

void launch_pad_frames(const Batch& bt, int np, int storage, int grid_blocks, cudaStream_t st) {
    if (storage == 0)
        k_pad_frames<uint4><<<dim3(grid_blocks, 2, np), 256, 0, st>>>(bt);
    else
        k_pad_frames<uint2><<<dim3(grid_blocks, 2, np), 256, 0, st>>>(bt);
}

void launch_build_lists(const Batch& bt, int np, int grid_blocks, cudaStream_t st) {
    k_lists_zero<<<dim3(1, 1, np), 32, 0, st>>>(bt);
    k_build_lists<<<dim3(grid_blocks, 2, np), 256, 0, st>>>(bt);
}

// Exported patch costs: the raw sums divided by 3T (the same division, so the same bits, as a mean taken
// at evaluation time).
__global__ void k_cost_export(const float* src, float* dst, int n, float scale) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[i] / scale;
}
void launch_cost_export(const float* src, float* dst, int n, int radius, int census, cudaStream_t st) {
    const int d = 2 * radius + 1;
    k_cost_export<<<(n + 255) / 256, 256, 0, st>>>(src, dst, n, (float)((census ? 24 : 3) * d * d));
}



}  // namespace gpm
