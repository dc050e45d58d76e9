// Frame ingest that allocates nothing (gpm_ingest_noalloc in include/gpm.h).
//
// Who needs it: callers that must not call cudaMalloc when they ingest --
// real-time and embedded hosts whose device memory is reserved once at
// start-up, plugins of frameworks that own the device memory pool and forbid
// allocations behind their back, and latency-critical loops where an
// allocation (and the implicit synchronisation cudaMalloc can bring) is not
// allowed.  They pass the input frames and the output RGBX buffers; the
// ingest's scratch (the FP64 partial sums of both frames, the gain, and the
// V histogram and table of the optional HSV equalisation) lives in one
// file-scope device array instead of a buffer from an allocator.
//
// The work is the same launch sequence, on the same grid, as the ingest of
// gpm_match(level 0): the same kernels in the same order with the same
// summation tree, so the output is bitwise the same.
#include <cuda_runtime.h>

#include <cstddef>
#include <mutex>

#include "../../include/gpm.h"
#include "common.cuh"
#include "kernels.h"

namespace gpm {

// The scratch of one ingest (6 KiB in all).
struct NoAllocScratch {
    double partial[2 * kIngestPartialBlocks];  // per-block FP64 sums of both frames
    double gain;                                // mean(I1) / mean(I2), or 1
    double pad[31];                             // keeps the tables 256-byte aligned
    int hist[2 * 256];                          // V histograms (HSV equalisation)
    float lut[2 * 256];                         // equalised V per bin
};

// Every GPU that loads the library holds this array until the process exits.
// Calls share it: two calls that overlap on the GPU (different streams, no
// ordering between them) race on it.
static __device__ __align__(256) NoAllocScratch g_ingest_scratch;

namespace {
std::mutex g_mu;
NoAllocScratch* g_scratch_ptr[64] = {};  // device address of the array, per device (looked up once)
}  // namespace

}  // namespace gpm

using namespace gpm;

extern "C" gpm_status gpm_ingest_noalloc(const float* frame1, const float* frame2, int32_t width, int32_t height,
                                         int64_t row_stride, int32_t gain_normalize, int32_t equalize,
                                         int32_t storage, void* out1, void* out2, void* stream) {
    if (!frame1 || !frame2 || !out1 || !out2) return GPM_EINVAL;
    if (width < 1 || height < 1 || width > 32767 || height > 32767 || row_stride < 3 * (int64_t)width)
        return GPM_EINVAL;
    if ((int64_t)width * height > (1 << 26)) return GPM_EINVAL;  // the largest frame a context takes
    if (storage < 0 || storage > 2 || (equalize != 0 && equalize != 1)) return GPM_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return GPM_ECUDA;
    }
    NoAllocScratch* sc = nullptr;
    {
        // Set-up, once per device, with that device current: the host-side
        // name of the array is only a stand-in, not a device address.
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_ingest_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return GPM_ECUDA;
            }
            g_scratch_ptr[dev] = (NoAllocScratch*)p;
        }
        sc = g_scratch_ptr[dev];
    }
    // Every slot this call reads is written first by this call (the partial sums and the gain by their kernels,
    // the histogram cleared on the stream before it is counted), so nothing carries over from an earlier call.
    char* base = reinterpret_cast<char*>(sc);  // a device address: only offsets are taken on the host
    double* partial = reinterpret_cast<double*>(base + offsetof(NoAllocScratch, partial));
    double* gain = reinterpret_cast<double*>(base + offsetof(NoAllocScratch, gain));
    int* hist = reinterpret_cast<int*>(base + offsetof(NoAllocScratch, hist));
    float* lut = reinterpret_cast<float*>(base + offsetof(NoAllocScratch, lut));
    launch_ingest(frame1, frame2, width, height, row_stride, gain_normalize, storage, partial, kIngestPartialBlocks,
                  gain, out1, out2, equalize ? hist : nullptr, equalize ? lut : nullptr, (cudaStream_t)stream);
    // Reports a launch failure of this call; an error that earlier work left pending is reported (and cleared) too.
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GPM_OK : GPM_ECUDA;
}
