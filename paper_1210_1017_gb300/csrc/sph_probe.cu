// FP32 issue-rate probe: the measured denominator of the interaction's
// roofline (the interaction is bound by the plain FP32/integer pipes, not by
// the tensor cores, so its peak is the rate of fused multiply-adds the SMs
// can issue).  The paper has no counterpart; this is a measurement helper.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sph.h"

namespace {

constexpr int kChains = 8;     // independent dependency chains per thread
constexpr int kUnroll = 16;    // steps of every chain per loop iteration

// Each thread advances kChains independent recurrences a <- a*m + c
// (a fixed point at 1 keeps the values normal) kUnroll times per iteration:
// kChains * kUnroll = 128 fused multiply-adds per thread and iteration,
// against one compare-and-branch.  The sum is stored so nothing is dead.
__global__ void __launch_bounds__(256) k_fma_probe(float* __restrict__ out, uint32_t iters,
                                                   float m, float c) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.0f + (float)(threadIdx.x + k) * 0x1p-12f;
    for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], m, c);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int sph_fma_probe(float* d_out, uint32_t blocks, uint32_t iters, void* stream) {
    if (!d_out || blocks == 0 || iters == 0) return SPH_ERR_INVALID_ARG;
    k_fma_probe<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        d_out, iters, 1.0f - 0x1p-20f, 0x1p-20f);
    return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}
