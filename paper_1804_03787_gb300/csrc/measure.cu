// Measurement aid (gpm_fp32_peak_probe in include/gpm.h): a kernel that
// keeps every FP32 lane busy with fused multiply-adds, so that the FP32
// lane-operation peak that the PatchMatch kernels' roofline divides by is
// measured on the device at hand rather than taken from nominal figures.
#include <cuda_runtime.h>

#include "../../include/gpm.h"

namespace gpm {

// Eight independent FMA chains per thread (enough to cover the FMA latency
// with a few warps per scheduler), 64 FMAs per chain per iteration.
__global__ void __launch_bounds__(256) k_fma_probe(int iters, float a, float b, float* sink) {
    float x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 64; ++r) {
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = fmaf(x[k], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace gpm

extern "C" gpm_status gpm_fp32_peak_probe(int32_t blocks, int32_t iters, float* sink, void* stream) {
    if (blocks < 1 || blocks > (1 << 20) || iters < 1 || iters > (1 << 20) || !sink) return GPM_EINVAL;
    gpm::k_fma_probe<<<blocks, 256, 0, (cudaStream_t)stream>>>(iters, 0.999f, 1e-3f, sink);
    return cudaGetLastError() == cudaSuccess ? GPM_OK : GPM_ECUDA;
}
