// Private declarations of the surrogate network's CUDA code.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace sur {

enum Epilogue : int {
    kEpiNone = 0,       // acc (+ bias)
    kEpiRelu = 1,       // relu(acc + bias)
    kEpiResidual = 2,   // res + acc + bias
    kEpiEdge1 = 3,      // relu(acc + P[src] + Q[dst] + bias): factorised edge-MLP input
    kEpiReluMask = 4,   // acc where res > 0, else 0 (backward through a ReLU)
    kEpiAccum = 5,      // out_f32 += acc (+ bias): gradient accumulation
};

struct LinearArgs {
    const __nv_bfloat16* A;     // M x K, row-major (row stride lda; 0 = K)
    uint32_t lda;
    const __nv_bfloat16* Bt;    // N x K, row-major (the layer's weights transposed)
    const float* bias;          // N or null
    uint32_t M;
    int epi;
    const __nv_bfloat16* res;   // M x N (residual / ReLU mask source), row stride ldr (0 = N)
    uint32_t ldr;
    const __nv_bfloat16* gp;    // node x N gathered at src (kEpiEdge1)
    const __nv_bfloat16* gq;    // node x N gathered at dst (kEpiEdge1)
    const uint32_t* src;
    const uint32_t* dst;
    __nv_bfloat16* out_bf16;    // M x ldo (may be null)
    float* out_f32;             // M x ldo (may be null)
    uint32_t ldo;
    uint32_t* status;           // bit 0: a bounded wait gave up
};

// D[128 x N] = P^T Q summed over rows [0, M): P is M x 128, Q is M x N (bf16,
// row-major with the given leading dimensions); dW = scale * D.
struct WgradArgs {
    const __nv_bfloat16* X;     // P (row stride ldp; 0 = 128)
    const __nv_bfloat16* dY;    // Q (row stride ldq; 0 = N)
    uint32_t ldp, ldq;
    uint32_t M;
    float* partial;             // nparts x 128 x N scratch
    uint32_t nparts;
    float* dW;                  // 128 x N
    float scale;
    uint32_t* status;
};

// Fused edge update of one message-passing layer over M edges (latent 128):
//   z  = relu(e W1c + b1 + P[src] + Q[dst])      (stored to Z when Z != null)
//   e' = e + z W2 + b2                           (stored to Eout)
// W1t, W2t: the weights transposed (N x K, K-major), bf16.
struct EdgeArgs {
    const __nv_bfloat16* E;
    const __nv_bfloat16* W1t;
    const __nv_bfloat16* W2t;
    const float* b1;
    const float* b2;
    const __nv_bfloat16* P;
    const __nv_bfloat16* Q;
    const uint32_t* src;
    const uint32_t* dst;
    uint32_t M;
    __nv_bfloat16* Z;
    __nv_bfloat16* Eout;
    uint32_t* status;
};

int num_sms();
bool launch_linear(int K, int N, const LinearArgs& g, cudaStream_t st);
void launch_edge_layer(const EdgeArgs& g, cudaStream_t st);
// The edge encoder in one kernel: E (M x 16) -> Eout = relu(E W1 + b1) W2 + b2
// (z = relu(E W1 + b1) to Z when Z != null); P, Q, src, dst unused.
void launch_edge_encoder(const EdgeArgs& g, cudaStream_t st);
bool launch_wgrad(int N, const WgradArgs& g, cudaStream_t st);

}  // namespace sur
