/*
 * sur.h -- C ABI of the learned surrogate in libsph.so: a message-passing
 * network on the radius-2h neighbour graph of the SPH cell list that
 * advances particle state several SPH steps per call (the configured
 * "learned surrogate" pattern; the paper itself has no learned component).
 * Its dense layers run on the tcgen05 tensor cores in BF16 with FP32
 * accumulation, forward and backward.
 *
 * Conventions as in sph.h: SPH_OK / SPH_ERR_* return codes, caller-owned
 * device memory, async on the given stream unless marked "sync".
 */
#ifndef SUR_H
#define SUR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Epilogues of sur_linear. */
#define SUR_EPI_NONE      0   /* out = A B^T + bias                          */
#define SUR_EPI_RELU      1   /* out = relu(A B^T + bias)                    */
#define SUR_EPI_RESIDUAL  2   /* out = res + A B^T + bias                    */
#define SUR_EPI_RELU_MASK 4   /* out = (res > 0) ? A B^T : 0 (ReLU backward) */

/* One dense layer on the tensor cores: A is M x K bf16 (row-major), Bt is
 * N x K bf16 (row-major: the weights transposed), bias N floats or NULL, res
 * M x N bf16 (for the residual / mask epilogues).  Writes out_bf16 and/or
 * out_f32 (M x N row-major; NULL to skip).  Supported (K, N): (16, 128),
 * (128, 128), (256, 128), (128, 16), (16, 16), (128, 256).  All pointers
 * 16-byte aligned.  Async. */
int sur_linear(const void *d_A, const void *d_Bt, const float *d_bias,
               uint32_t M, uint32_t K, uint32_t N, int epilogue,
               const void *d_res, void *d_out_bf16, float *d_out_f32,
               void *stream);

/* Weight gradient on the tensor cores: dW = scale * P^T Q summed over rows
 * 0..M-1, P is M x 128 bf16, Q is M x N bf16 (N = 128 or 16), dW 128 x N
 * float.  scratch of sur_wgrad_scratch_bytes(N) bytes; the sum over row
 * tiles is taken per block in tensor memory and across blocks in a fixed
 * order (deterministic).  Async. */
uint64_t sur_wgrad_scratch_bytes(uint32_t N);
int sur_wgrad(const void *d_P, const void *d_Q, uint32_t M, uint32_t N,
              float scale, float *d_dW, void *d_scratch,
              uint64_t scratch_bytes, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SUR_H */
