// Frame ingest that allocates nothing (gpm_ingest_noalloc in include/gpm.h).
//
// Who needs it: callers that cannot call cudaMalloc at all, or not at the
// moment they ingest -- code running inside a CUDA stream capture (where an
// allocation would break or be recorded into the graph), real-time and
// embedded hosts whose memory is fixed up front, and plugins of frameworks
// that own the device memory pool.  They pass the input frames and the
// output RGBX buffers; the gain-normalisation scratch (per-row FP64 sums of
// both frames and the gain) lives in a file-scope device array instead of a
// buffer from an allocator.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/gpm.h"
#include "common.cuh"
#include "kernels.h"

namespace gpm {

constexpr int kNoAllocMaxRows = 4096;  // rows a frame may have: scratch = 2 * 4096 + 1 doubles (64 KiB)

// Every GPU that loads the library holds this array until the process exits.
// Calls share it: two calls that overlap on the GPU (different streams, no
// ordering between them) race on it.
static __device__ __align__(256) double g_ingest_scratch[2 * kNoAllocMaxRows + 1];

// One block per row: FP64 sums of the row's RGB values in both frames.
__global__ void k_row_sums_noalloc(const float* f1, const float* f2, int W, int64_t stride, double* rows) {
    __shared__ double sh[2][256];
    const int y = blockIdx.x;
    const float* r1 = f1 + (int64_t)y * stride;
    const float* r2 = f2 + (int64_t)y * stride;
    double a = 0, b = 0;
    for (int k = threadIdx.x; k < 3 * W; k += blockDim.x) {
        a += (double)r1[k];
        b += (double)r2[k];
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
        rows[2 * y] = sh[0][0];
        rows[2 * y + 1] = sh[1][0];
    }
}

// gain = sum(I1) / sum(I2), summed over the rows in order (deterministic).
__global__ void k_row_gain_noalloc(const double* rows, int H, int enable, double* gain) {
    if (threadIdx.x != 0) return;
    double a = 0, b = 0;
    for (int y = 0; y < H; ++y) {
        a += rows[2 * y];
        b += rows[2 * y + 1];
    }
    *gain = (enable && b > 0) ? a / b : 1.0;
}

namespace {
std::mutex g_mu;
double* g_scratch_ptr[64] = {};  // device address of the array, per device (set once)
}  // namespace

}  // namespace gpm

using namespace gpm;

extern "C" gpm_status gpm_ingest_noalloc(const float* frame1, const float* frame2, int32_t width, int32_t height,
                                         int64_t row_stride, int32_t gain_normalize, int32_t storage, void* out1,
                                         void* out2, void* stream) {
    if (!frame1 || !frame2 || !out1 || !out2) return GPM_EINVAL;
    if (width < 1 || height < 1 || row_stride < 3 * (int64_t)width) return GPM_EINVAL;
    if (height > kNoAllocMaxRows) return GPM_EINVAL;  // beyond the static scratch
    if ((int64_t)width * height > (1 << 26)) return GPM_EINVAL;
    if (storage < 0 || storage > 2) return GPM_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return GPM_ECUDA;
    }
    double* scratch = nullptr;
    {
        // Set-up, once per device, with that device current: the host-side
        // name of the array is not a device address, so look the address up.
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_ingest_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return GPM_ECUDA;
            }
            g_scratch_ptr[dev] = (double*)p;
        }
        scratch = g_scratch_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    // every row slot and the gain are rewritten by each call: nothing carries over
    k_row_sums_noalloc<<<height, 256, 0, st>>>(frame1, frame2, width, row_stride, scratch);
    k_row_gain_noalloc<<<1, 32, 0, st>>>(scratch, height, gain_normalize, scratch + 2 * kNoAllocMaxRows);
    launch_pack(frame1, frame2, width, height, row_stride, storage, scratch + 2 * kNoAllocMaxRows, out1, out2, st);
    const cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GPM_ECUDA;
    }
    return GPM_OK;
}
