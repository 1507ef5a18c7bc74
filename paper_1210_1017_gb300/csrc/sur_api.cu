// C ABI of the surrogate (include/sur.h).
#include "../../include/sph.h"
#include "../../include/sur.h"
#include "sur_internal.cuh"

using namespace sur;

namespace {
constexpr uint32_t kWgradBlocks = 3 * 152;   // three blocks per SM
}

extern "C" {

int sur_linear(const void* A, const void* Bt, const float* bias, uint32_t M, uint32_t K,
               uint32_t N, int epilogue, const void* res, void* out_bf16, float* out_f32,
               void* stream) {
    if (!A || !Bt || (!out_bf16 && !out_f32)) return SPH_ERR_INVALID_ARG;
    if ((epilogue == kEpiResidual || epilogue == kEpiReluMask) && !res) return SPH_ERR_INVALID_ARG;
    if (epilogue != kEpiNone && epilogue != kEpiRelu && epilogue != kEpiResidual &&
        epilogue != kEpiReluMask)
        return SPH_ERR_INVALID_ARG;
    LinearArgs g = {};
    g.A = static_cast<const __nv_bfloat16*>(A);
    g.Bt = static_cast<const __nv_bfloat16*>(Bt);
    g.bias = bias;
    g.M = M;
    g.epi = epilogue;
    g.res = static_cast<const __nv_bfloat16*>(res);
    g.out_bf16 = static_cast<__nv_bfloat16*>(out_bf16);
    g.out_f32 = out_f32;
    g.ldo = N;
    if (!launch_linear((int)K, (int)N, g, static_cast<cudaStream_t>(stream)))
        return SPH_ERR_INVALID_ARG;
    return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}

uint64_t sur_wgrad_scratch_bytes(uint32_t N) {
    return (uint64_t)kWgradBlocks * 128 * N * sizeof(float);
}

int sur_wgrad(const void* P, const void* Q, uint32_t M, uint32_t N, float scale, float* dW,
              void* scratch, uint64_t scratch_bytes, void* stream) {
    if (!P || !Q || !dW || !scratch) return SPH_ERR_INVALID_ARG;
    if (scratch_bytes < sur_wgrad_scratch_bytes(N)) return SPH_ERR_WORKSPACE;
    WgradArgs g = {};
    g.X = static_cast<const __nv_bfloat16*>(P);
    g.dY = static_cast<const __nv_bfloat16*>(Q);
    g.M = M;
    g.partial = static_cast<float*>(scratch);
    g.nparts = kWgradBlocks;
    g.dW = dW;
    g.scale = scale;
    if (!launch_wgrad((int)N, g, static_cast<cudaStream_t>(stream))) return SPH_ERR_INVALID_ARG;
    return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}

}  // extern "C"
