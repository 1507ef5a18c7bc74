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

int sur_edge_layer(const void* E, const void* W1t, const void* W2t, const float* b1,
                   const float* b2, const void* P, const void* Q, const uint32_t* src,
                   const uint32_t* dst, uint32_t M, void* Z, void* Eout, void* stream) {
    if (!E || !W1t || !W2t || !b1 || !b2 || !P || !Q || !src || !dst || !Eout)
        return SPH_ERR_INVALID_ARG;
    const void* ptrs[] = {E, W1t, W2t, P, Q, Eout, b1, b2};
    for (const void* q : ptrs)
        if (reinterpret_cast<uintptr_t>(q) % 16u) return SPH_ERR_INVALID_ARG;
    if (Z && reinterpret_cast<uintptr_t>(Z) % 16u) return SPH_ERR_INVALID_ARG;
    EdgeArgs g = {};
    g.E = static_cast<const __nv_bfloat16*>(E);
    g.W1t = static_cast<const __nv_bfloat16*>(W1t);
    g.W2t = static_cast<const __nv_bfloat16*>(W2t);
    g.b1 = b1;
    g.b2 = b2;
    g.P = static_cast<const __nv_bfloat16*>(P);
    g.Q = static_cast<const __nv_bfloat16*>(Q);
    g.src = src;
    g.dst = dst;
    g.M = M;
    g.Z = static_cast<__nv_bfloat16*>(Z);
    g.Eout = static_cast<__nv_bfloat16*>(Eout);
    launch_edge_layer(g, static_cast<cudaStream_t>(stream));
    return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}

int sur_edge_encoder(const void* X, const void* W1t, const void* W2t, const float* b1,
                     const float* b2, uint32_t M, void* Z, void* Eout, void* stream) {
    if (!X || !W1t || !W2t || !b1 || !b2 || !Eout) return SPH_ERR_INVALID_ARG;
    const void* ptrs[] = {X, W1t, W2t, Eout};
    for (const void* q : ptrs)
        if (reinterpret_cast<uintptr_t>(q) % 16u) return SPH_ERR_INVALID_ARG;
    if (Z && reinterpret_cast<uintptr_t>(Z) % 16u) return SPH_ERR_INVALID_ARG;
    EdgeArgs g = {};
    g.E = static_cast<const __nv_bfloat16*>(X);
    g.W1t = static_cast<const __nv_bfloat16*>(W1t);
    g.W2t = static_cast<const __nv_bfloat16*>(W2t);
    g.b1 = b1;
    g.b2 = b2;
    g.M = M;
    g.Z = static_cast<__nv_bfloat16*>(Z);
    g.Eout = static_cast<__nv_bfloat16*>(Eout);
    launch_edge_encoder(g, static_cast<cudaStream_t>(stream));
    return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}

}  // extern "C"
