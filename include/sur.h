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

#include "sph.h"

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

/* The fused edge update of one message-passing layer (the network's hot
 * kernel) on its own, over M edges of latent width 128 (all arrays device,
 * bf16 row-major unless noted, 16-byte aligned):
 *   z  = relu(E W1 + b1 + P[src] + Q[dst])   -> Z (M x 128; may be NULL)
 *   E' = E + z W2 + b2                        -> Eout (M x 128)
 * W1t, W2t: the 128 x 128 weights transposed (row n holds output n); b1, b2:
 * float[128]; P, Q: node tables (rows indexed by src[m], dst[m], uint32).
 * bf16 inputs, fp32 accumulation on the tensor cores, results rounded to
 * bf16.  Async on `stream`.  SPH_ERR_INVALID_ARG for NULL or unaligned
 * pointers. */
int sur_edge_layer(const void *d_E, const void *d_W1t, const void *d_W2t,
                   const float *d_b1, const float *d_b2, const void *d_P,
                   const void *d_Q, const uint32_t *d_src, const uint32_t *d_dst,
                   uint32_t M, void *d_Z, void *d_Eout, void *stream);

/* The network's edge encoder (its first two layers) in one kernel, over M
 * edges (all arrays device, 16-byte aligned):
 *   z  = relu(X W1 + b1)   -> Z (M x 128 bf16; may be NULL)
 *   E0 = z W2 + b2         -> Eout (M x 128 bf16)
 * X: M x 16 bf16 edge features; W1t: 128 x 16 and W2t: 128 x 128 bf16 (the
 * weights transposed: row n holds output n); b1, b2: float[128].  z is
 * rounded to bf16 before the second product, so the results are those of
 * two sur_linear calls (SUR_EPI_RELU, then SUR_EPI_NONE with bf16 output)
 * without the round trip of z through memory.  Async on `stream`.
 * SPH_ERR_INVALID_ARG for NULL or unaligned pointers. */
int sur_edge_encoder(const void *d_X, const void *d_W1t, const void *d_W2t,
                     const float *d_b1, const float *d_b2, uint32_t M, void *d_Z,
                     void *d_Eout, void *stream);

/* ---- the network -------------------------------------------------------
 * Nodes: the particles of an SPH context (sph.h) in its current sorted order,
 * with cells built.  Edges: every ordered pair within 2h (the FP64 predicate
 * of the cell list), or within radius * 2h for a sparser graph.  Node input: the particle's last five velocities (a
 * history array indexed by particle id: hist[id][15], oldest first) / v_scale
 * and its boundary flag; edge input: (r_i - r_j)/2h and |r_i - r_j|/2h.
 * A sparser graph keeps only the pairs closer than radius * 2h (radius in
 * (0, 1); 0 or 1 = the full support): fewer edges per node and a smaller
 * receptive field per layer.
 * Latent width 128; `layers` message-passing layers of
 *   e' = e + W2 relu(W1a h_i + W1b h_j + W1c e + b1) + b2
 *   h' = h + W4 relu(W3 [h, sum_j e'_ij] + b3) + b4,
 * decoder W6 relu(W5 h + b5) + b6 -> normalised acceleration (3 of 16
 * outputs); a = out * a_std + a_mean.  Parameters are one flat float array
 * (per layer W[kin][kout] then b[kout]; layer order: node encoder 2, edge
 * encoder 2, per message-passing layer W1a, W1b, W1c+b1, W2+b2, W3+b3,
 * W4+b4, then decoder 2).  Every dense layer runs on the tensor cores
 * (bf16 inputs, fp32 accumulation), forward and backward. */
typedef struct sur_config {
    uint32_t layers;           /* message-passing layers                     */
    uint32_t max_nodes;        /* particles of the largest graph             */
    uint32_t max_edges;        /* edges of the largest graph                 */
    uint32_t train;            /* keep activations for sur_backward          */
    float v_scale;             /* velocity normalisation [m/s]               */
    float a_mean[3], a_std[3]; /* acceleration normalisation [m/s^2]         */
    float dt_s;                /* time advanced per sur_advance call [s]     */
    float radius;              /* edge radius / 2h; 0 or 1 = 2h (the SPH
                                  neighbour relation), else in (0, 1)       */
} sur_config;

typedef struct sur_ctx sur_ctx;
struct sph_ctx;

uint64_t sur_param_count(const sur_config *cfg);
uint64_t sur_query_bytes(const sur_config *cfg);   /* device workspace size */
int sur_init(const sur_config *cfg, void *d_workspace, uint64_t bytes,
             void *stream, sur_ctx **out);          /* sync; params zero      */
int sur_set_params(sur_ctx *ctx, const float *host, uint64_t count); /* sync; resets Adam */
int sur_get_params(sur_ctx *ctx, float *host, uint64_t count);       /* sync */
int sur_get_grads(sur_ctx *ctx, float *host, uint64_t count);        /* sync */

/* Forward pass on the SPH context's particles; d_hist as above (device, n x
 * 15 floats by id).  d_acc (device, n x 3 by id, may be NULL) receives the
 * predicted acceleration.  Sync (reads the edge count). */
int sur_forward(sur_ctx *ctx, struct sph_ctx *sph, const float *d_hist,
                float *d_acc);

/* Gradients of loss = mean over fluid particles of |out - target|^2 (out
 * and target normalised accelerations; d_target device, n x 3 by id) with
 * respect to all parameters, from the last sur_forward (train contexts).
 * Writes the loss to *loss (host).  Sync. */
int sur_backward(sur_ctx *ctx, struct sph_ctx *sph, const float *d_target,
                 float *loss);

/* One Adam step on the parameters with the gradients of sur_backward. */
int sur_adam(sur_ctx *ctx, float lr, float beta1, float beta2, float eps);

/* One surrogate call: forward, then semi-implicit Euler over dt_s of the
 * SPH context's fluid particles (v += a dt_s, r += v dt_s; boundary and
 * excluded particles stay) and a shift of the velocity history.  The SPH
 * context's cells are stale afterwards (call sph_build_cells).  Sync. */
int sur_advance(sur_ctx *ctx, struct sph_ctx *sph, float *d_hist);

/* A training sample from seven saved frames of the SPH context's particles
 * (d_frames: device, 7 x n x 3 float64 by id, frame f = x at time
 * t_k + (f - 5) dt_s).  Input frames 1..5 get random-walk noise (per frame
 * increments N(0, sigma^2/5) from a counter-based SplitMix64/Box-Muller
 * stream of `seed`, so x^k has std sigma; boundary particles none).
 * Writes (device, by id): d_pos n x 3 float64 = noisy x^k; d_vel n x 3 =
 * (x~^k - x~^{k-1}) / dt_s; d_hist n x 15 = the five finite-difference
 * velocities, oldest first; d_target n x 3 = ((x^{k+1} - 2 x~^k +
 * x~^{k-1}) / dt_s^2 - a_mean) / a_std, the normalised acceleration that
 * sur_advance needs to land on the clean x^{k+1}.  Async. */
int sur_make_sample(sur_ctx *ctx, struct sph_ctx *sph, const double *d_frames,
                    double sigma, uint64_t seed, double *d_pos, float *d_vel,
                    float *d_hist, float *d_target);

/* ncalls surrogate calls (each: cell rebuild if needed, then sur_advance);
 * after every save_every calls (and the last) the stream is synchronised
 * and cb(user, call, t) runs, t = call * dt_s, from which the caller may
 * read the state (sph_download, sph_download_by_id); a non-zero return
 * stops early (still SPH_OK).  The cells are rebuilt at the end.  cb may
 * be NULL.  Sync. */
int sur_rollout(sur_ctx *ctx, struct sph_ctx *sph, float *d_hist,
                uint32_t ncalls, uint32_t save_every, sph_snapshot_fn cb,
                void *user);

uint32_t sur_num_edges(const sur_ctx *ctx);
/* The graph of the last sur_forward, in the particle order of the SPH
 * context at that call (its cell order): rowptr[n + 1] (CSR row starts of
 * the receiving particles i) and col[sur_num_edges] (the sending particles
 * j of each row, with |r_i - r_j| < 2h by the FP64 predicate of Sec. 3.1),
 * both caller-owned host arrays.  SPH_ERR_STATE before the first forward.
 * Sync. */
int sur_read_graph(sur_ctx *ctx, uint32_t *rowptr, uint32_t *col);
const char *sur_last_error(const sur_ctx *ctx);
void sur_destroy(sur_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* SUR_H */
