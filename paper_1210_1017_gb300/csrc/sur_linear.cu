// Linear layers of the surrogate network on the tcgen05 tensor cores:
//   out[m, :] = epilogue( A[m, :] * B^T + bias )     (A: M x K bf16, B: N x K bf16)
// with the epilogues the message-passing network needs (bias, ReLU,
// residual add, the factorised edge-MLP input with gathered node terms, the
// ReLU mask of the backward pass) fused after the tcgen05.ld of the fp32
// accumulator.  Also the weight gradient dW = X^T dY, reduced over rows in
// TMEM per block and then across blocks in a fixed order.
#include <cuda_bf16.h>

#include "sur_gemm.cuh"
#include "sur_internal.cuh"

namespace sur {

namespace {

template <int N>
__device__ __forceinline__ constexpr uint32_t tmem_cols() {
    return N <= 32 ? 32u : (N <= 64 ? 64u : (N <= 128 ? 128u : 256u));
}

// Issue the asynchronous copies of a (128 x K) bf16 tile (rows past nrows
// zero-filled) into the canonical K-major layout; consecutive threads take
// consecutive rows of one 16-byte column piece.
template <int K, int THR = 128>
__device__ __forceinline__ void issue_rows(unsigned char* dst, const __nv_bfloat16* src,
                                           uint32_t row0, uint32_t nrows, uint32_t ld) {
#pragma unroll
    for (int c = threadIdx.x; c < 128 * (K / 8); c += THR) {
        const int r = c & 127, gk = c >> 7;
        const bool ok = row0 + r < nrows;
        const __nv_bfloat16* p = ok ? src + (size_t)(row0 + r) * ld + gk * 8 : src;
        cp_async16(dst + kmajor_offset(r, gk * 8, K), p, ok);
    }
}

__device__ __forceinline__ void unpack8(const uint4& u, float* f) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float2 t = __bfloat1622float2(h[q]);
        f[2 * q] = t.x;
        f[2 * q + 1] = t.y;
    }
}

// Epilogue operands of one row and NP columns, in registers: bf16 rows in
// a (residual, ReLU mask, P[src]) and b (Q[dst]); an fp32 row (gradient
// accumulation) spans a then b.
template <int NP>
struct EpiOps {
    uint4 a[NP / 8];
    uint4 b[NP / 8];
};

template <int N, int NP>
__device__ __forceinline__ void epi_load(EpiOps<NP>& o, const LinearArgs& g, uint32_t m,
                                         uint32_t gi, uint32_t gj, uint32_t ldr, int col0) {
    switch (g.epi) {
        case kEpiEdge1: {
            const uint4* p = reinterpret_cast<const uint4*>(g.gp + (size_t)gi * N + col0);
            const uint4* q = reinterpret_cast<const uint4*>(g.gq + (size_t)gj * N + col0);
#pragma unroll
            for (int i = 0; i < NP / 8; ++i) {
                o.a[i] = p[i];
                o.b[i] = q[i];
            }
            break;
        }
        case kEpiResidual:
        case kEpiReluMask: {
            const uint4* p = reinterpret_cast<const uint4*>(g.res + (size_t)m * ldr + col0);
#pragma unroll
            for (int i = 0; i < NP / 8; ++i) o.a[i] = p[i];
            break;
        }
        case kEpiAccum: {
            const uint4* p = reinterpret_cast<const uint4*>(g.out_f32 + (size_t)m * g.ldo + col0);
#pragma unroll
            for (int i = 0; i < NP / 8; ++i) {
                o.a[i] = p[i];
                o.b[i] = p[NP / 8 + i];
            }
            break;
        }
        default: break;
    }
}

// Forward-type GEMM with fused epilogue; persistent over 128-row tiles.  The
// A tile is double-buffered: the copies of the next tile are in flight while
// the tensor cores multiply the current one and the epilogue drains it.
// Block size of k_linear: 256 threads (the two warps sharing a TMEM lane
// quarter split the output columns) when N >= 32, else 128.
template <int N>
__host__ __device__ constexpr int linear_threads() { return N >= 32 ? 256 : 128; }

template <int K, int N>
__global__ void __launch_bounds__(linear_threads<N>(), 1) k_linear(const LinearArgs g) {
    constexpr int THR = linear_threads<N>();
    constexpr int NCOL = N / (THR / 128);             // output columns per thread
    extern __shared__ __align__(128) unsigned char s_raw[];
    __shared__ __align__(16) float s_bias[N];          // read by every row: staged once
    unsigned char* sb = s_raw;                        // N x K (weights)
    unsigned char* sa0 = s_raw + N * K * 2;           // 2 x (128 x K)
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    if (w == 0) tmem_alloc(&s_tmem, tmem_cols<N>());
    if (tid == 0) mbar_init1(&s_bar);
    const uint32_t lda = g.lda ? g.lda : (uint32_t)K;
    const uint32_t ldr = g.ldr ? g.ldr : (uint32_t)N;
    const uint32_t ntiles = (g.M + 127) / 128;
    // weights and the first tile
    for (int c = tid; c < N * (K / 8); c += THR) {
        const int r = c % N, gk = c / N;
        cp_async16(sb + kmajor_offset(r, gk * 8, K), g.Bt + (size_t)r * K + gk * 8, true);
    }
    for (int c = tid; c < N; c += THR) s_bias[c] = g.bias ? g.bias[c] : 0.f;
    if (blockIdx.x < ntiles) issue_rows<K, THR>(sa0, g.A, blockIdx.x * 128, g.M, lda);
    cp_async_commit();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    uint32_t phase = 0, buf = 0;
    bool ok = true;
    for (uint32_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, buf ^= 1u) {
        unsigned char* sa = sa0 + buf * (128 * K * 2);
        cp_async_wait_all();
        fence_async_shared();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int s = 0; s < K / 16; ++s) {
                const uint64_t ad = smem_desc(sm_addr(sa) + s * 256, kLBO, (K / 8) * 128);
                const uint64_t bd = smem_desc(sm_addr(sb) + s * 256, kLBO, (K / 8) * 128);
                tc_mma(tmem, ad, bd, idesc_bf16(N), s > 0 ? 1u : 0u);
            }
            tc_commit(&s_bar);
        }
        // next tile into the other buffer (its last reader, the previous
        // tile's MMA, has completed)
        const uint32_t next = tile + gridDim.x;
        if (next < ntiles) issue_rows<K, THR>(sa0 + (buf ^ 1u) * (128 * K * 2), g.A, next * 128, g.M, lda);
        cp_async_commit();
        // this thread's row and columns: its epilogue operands load while the MMA runs
        const int wq = w & 3, col0 = (w >> 2) * NCOL;
        const uint32_t m = tile * 128 + wq * 32 + lane;
        const bool valid = m < g.M;
        uint32_t gi = 0, gj = 0;
        if (g.epi == kEpiEdge1 && valid) {
            gi = g.src[m];
            gj = g.dst[m];
        }
        constexpr int NP = NCOL < 128 ? NCOL : 128;   // columns per epilogue pass
        EpiOps<NP> op;
        if (valid) epi_load<N, NP>(op, g, m, gi, gj, ldr, col0);
        const bool got = mbar_wait(&s_bar, phase);
        ok = __syncthreads_and(got) != 0;
        if (!ok) {
            if (tid == 0 && g.status) atomicOr(g.status, 1u);
            break;
        }
        phase ^= 1u;
        tc_fence_after();
#pragma unroll
        for (int h = 0; h < NCOL / NP; ++h) {
            if (h > 0 && valid) epi_load<N, NP>(op, g, m, gi, gj, ldr, col0 + h * NP);
#pragma unroll
            for (int cl = 0; cl < NP; cl += 16) {
                const int c0 = col0 + h * NP + cl;
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(wq * 32) << 16) + c0, v);
                if (!valid) continue;
                if (g.bias) {
                    const float4* b4 = reinterpret_cast<const float4*>(s_bias + c0);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 b = b4[q];
                        v[4 * q] += b.x;
                        v[4 * q + 1] += b.y;
                        v[4 * q + 2] += b.z;
                        v[4 * q + 3] += b.w;
                    }
                }
                float t[16], u[16];
                switch (g.epi) {
                    case kEpiEdge1:   // relu(acc + P[src] + Q[dst] + b)
                        unpack8(op.a[cl / 8], t);
                        unpack8(op.a[cl / 8 + 1], t + 8);
                        unpack8(op.b[cl / 8], u);
                        unpack8(op.b[cl / 8 + 1], u + 8);
#pragma unroll
                        for (int i = 0; i < 16; ++i) v[i] = fmaxf(v[i] + t[i] + u[i], 0.f);
                        break;
                    case kEpiRelu:
#pragma unroll
                        for (int i = 0; i < 16; ++i) v[i] = fmaxf(v[i], 0.f);
                        break;
                    case kEpiResidual:
                        unpack8(op.a[cl / 8], t);
                        unpack8(op.a[cl / 8 + 1], t + 8);
#pragma unroll
                        for (int i = 0; i < 16; ++i) v[i] += t[i];
                        break;
                    case kEpiReluMask:   // backward through a ReLU: keep where act > 0
                        unpack8(op.a[cl / 8], t);
                        unpack8(op.a[cl / 8 + 1], t + 8);
#pragma unroll
                        for (int i = 0; i < 16; ++i) v[i] = t[i] > 0.f ? v[i] : 0.f;
                        break;
                    case kEpiAccum:
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int k = cl / 4 + q;
                            const uint4 x = k < NP / 8 ? op.a[k % (NP / 8)] : op.b[k % (NP / 8)];
                            v[4 * q] += __uint_as_float(x.x);
                            v[4 * q + 1] += __uint_as_float(x.y);
                            v[4 * q + 2] += __uint_as_float(x.z);
                            v[4 * q + 3] += __uint_as_float(x.w);
                        }
                        break;
                    default: break;
                }
                if (g.out_f32) {
                    float4* o = reinterpret_cast<float4*>(g.out_f32 + (size_t)m * g.ldo + c0);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        o[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                }
                if (g.out_bf16) {
                    __nv_bfloat162 hh[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) hh[q] = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
                    uint4* o = reinterpret_cast<uint4*>(g.out_bf16 + (size_t)m * g.ldo + c0);
                    o[0] = *reinterpret_cast<uint4*>(&hh[0]);
                    o[1] = *reinterpret_cast<uint4*>(&hh[4]);
                }
            }
        }
        tc_fence_before();
        __syncthreads();
    }
    cp_async_wait_all();
    __syncthreads();
    if (w == 0) tmem_dealloc(tmem, tmem_cols<N>());
}

// Transposed staging in two halves: the global loads of a (128-row x C)
// tile into registers (each job: 8 rows of one 8-column block), then the
// register transpose into the (C x 128) K-major tile in shared memory.
template <int C>
struct TRegs {
    static constexpr int kJobs = (C / 8) * 16;
    static constexpr int kPer = (kJobs + 127) / 128;
    uint4 v[kPer][8];
};

template <int C>
__device__ __forceinline__ void load_t(TRegs<C>& r, const __nv_bfloat16* src, uint32_t row0,
                                       uint32_t nrows, uint32_t ld) {
#pragma unroll
    for (int jj = 0; jj < TRegs<C>::kPer; ++jj) {
        const int j = threadIdx.x + jj * 128;
        const int cb = j % (C / 8), rg = j / (C / 8);
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) {
            const uint32_t m = row0 + rg * 8 + rr;
            r.v[jj][rr] = make_uint4(0u, 0u, 0u, 0u);
            if (j < TRegs<C>::kJobs && m < nrows)
                r.v[jj][rr] = *reinterpret_cast<const uint4*>(src + (size_t)m * ld + cb * 8);
        }
    }
}

template <int C>
__device__ __forceinline__ void store_t(unsigned char* dst, const TRegs<C>& r) {
#pragma unroll
    for (int jj = 0; jj < TRegs<C>::kPer; ++jj) {
        const int j = threadIdx.x + jj * 128;
        if (j >= TRegs<C>::kJobs) continue;
        const int cb = j % (C / 8), rg = j / (C / 8);
        __nv_bfloat16 t[8][8];
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) {
            const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&r.v[jj][rr]);
#pragma unroll
            for (int cc = 0; cc < 8; ++cc) t[cc][rr] = e[cc];
        }
#pragma unroll
        for (int cc = 0; cc < 8; ++cc)
            *reinterpret_cast<uint4*>(dst + kmajor_offset(cb * 8 + cc, rg * 8, 128)) =
                *reinterpret_cast<const uint4*>(t[cc]);
    }
}

// Weight gradient dW[C x N] = X^T dY over rows [0, M): X is M x C, dY is
// M x N (bf16, row-major).  Block b accumulates the row tiles b, b + grid,
// ... in TMEM (C = 128 rows of the MMA, one MMA chain per tile), then writes
// its partial; k_wgrad_reduce adds the partials in block order.  The loads
// of the next tile are in flight while the tensor cores work on this one.
template <int N>
__global__ void __launch_bounds__(128) k_wgrad(const WgradArgs g) {
    extern __shared__ __align__(128) unsigned char s_raw[];
    unsigned char* sa = s_raw;                  // X^T tile: 128 x 128 (features x rows)
    unsigned char* sb = s_raw + 128 * 128 * 2;  // dY^T tile: N x 128
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    if (w == 0) tmem_alloc(&s_tmem, tmem_cols<N>());
    if (tid == 0) mbar_init1(&s_bar);
    const uint32_t ldp = g.ldp ? g.ldp : 128u, ldq = g.ldq ? g.ldq : (uint32_t)N;
    const uint32_t ntiles = (g.M + 127) / 128;
    TRegs<128> rx;
    TRegs<N> ry;
    if (blockIdx.x < ntiles) {
        load_t<128>(rx, g.X, blockIdx.x * 128, g.M, ldp);
        load_t<N>(ry, g.dY, blockIdx.x * 128, g.M, ldq);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    uint32_t phase = 0, first = 1;
    bool ok = true;
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        store_t<128>(sa, rx);
        store_t<N>(sb, ry);
        fence_async_shared();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int s = 0; s < 128 / 16; ++s) {
                const uint64_t ad = smem_desc(sm_addr(sa) + s * 256, kLBO, 16 * 128);
                const uint64_t bd = smem_desc(sm_addr(sb) + s * 256, kLBO, 16 * 128);
                tc_mma(tmem, ad, bd, idesc_bf16(N), (first && s == 0) ? 0u : 1u);
            }
            tc_commit(&s_bar);
        }
        first = 0;
        const uint32_t next = tile + gridDim.x;
        if (next < ntiles) {
            load_t<128>(rx, g.X, next * 128, g.M, ldp);
            load_t<N>(ry, g.dY, next * 128, g.M, ldq);
        }
        const bool got = mbar_wait(&s_bar, phase);
        ok = __syncthreads_and(got) != 0;
        if (!ok) {
            if (tid == 0 && g.status) atomicOr(g.status, 1u);
            break;
        }
        phase ^= 1u;
        tc_fence_before();
        __syncthreads();
    }
    tc_fence_after();
    float* part = g.partial + (size_t)blockIdx.x * 128 * N;
    const uint32_t r = w * 32 + lane;   // feature row of dW
#pragma unroll 1
    for (int c0 = 0; c0 < N; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(w * 32) << 16) + c0, v);
        float4* o = reinterpret_cast<float4*>(part + (size_t)r * N + c0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const bool z = first || !ok;
            o[q] = z ? make_float4(0.f, 0.f, 0.f, 0.f)
                     : make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (w == 0) tmem_dealloc(tmem, tmem_cols<N>());
}

__global__ void k_wgrad_reduce(const float* __restrict__ partial, int nparts, int count,
                               float* __restrict__ out, float scale) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    float s = 0.f;
    for (int b = 0; b < nparts; ++b) s += partial[(size_t)b * count + i];
    out[i] = s * scale;
}


// The network's edge encoder (its two edge layers) in one kernel, per
// 128-edge tile: tcgen05 MMA 1 (x W1, K = 16: the edge features) into TMEM
// columns [0, 128); the first epilogue writes z = relu(acc + b1) as the
// K-major A operand of MMA 2 in shared memory (and to global memory for the
// backward pass); MMA 2 (z W2) into columns [128, 256); the second epilogue
// writes e0 = acc + b2.  z never reaches HBM in inference.  The x tile is
// double-buffered (the next tile's copies in flight during this one).  256
// threads, two blocks per SM (76 KB of shared memory and 256 TMEM columns
// each): the two warps that share a TMEM lane quarter split the columns.
constexpr int kEncK = 16;
constexpr size_t kEncSmem = (size_t)128 * kEncK * 2 * 3 + (size_t)128 * 128 * 2 * 2;   // W1, 2 x x; W2, z

__global__ void __launch_bounds__(256, 2) k_edge_encoder(const EdgeArgs g) {
    constexpr int K1 = kEncK, N = 128, NT = 256, CW = 64;   // CW: epilogue columns per thread
    constexpr uint32_t T = 128 * 128 * 2;          // bytes of one 128 x 128 bf16 tile
    constexpr uint32_t T1 = 128 * K1 * 2;          // bytes of one 128 x K1 tile
    extern __shared__ __align__(128) unsigned char s_raw[];
    unsigned char* sw1 = s_raw;                    // W1^T, N x K1
    unsigned char* sw2 = sw1 + T1;                 // W2^T, N x N
    unsigned char* sz = sw2 + T;                   // z tile
    unsigned char* sa0 = sz + T;                   // 2 x x tile
    __shared__ __align__(16) float s_b1[128], s_b2[128];
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    if (w == 0) tmem_alloc(&s_tmem, 256);
    if (tid == 0) mbar_init1(&s_bar);
    const uint32_t ntiles = (g.M + 127) / 128;
    for (int c = tid; c < N * (K1 / 8); c += NT) {
        const int r = c % N, gk = c / N;
        cp_async16(sw1 + kmajor_offset(r, gk * 8, K1), g.W1t + (size_t)r * K1 + gk * 8, true);
    }
    for (int c = tid; c < N * (N / 8); c += NT) {
        const int r = c % N, gk = c / N;
        cp_async16(sw2 + kmajor_offset(r, gk * 8, N), g.W2t + (size_t)r * N + gk * 8, true);
    }
    if (tid < 128) {
        s_b1[tid] = g.b1[tid];
        s_b2[tid] = g.b2[tid];
    }
    if (blockIdx.x < ntiles) issue_rows<K1, NT>(sa0, g.E, blockIdx.x * 128, g.M, K1);
    cp_async_commit();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const int wq = w & 3, part = w >> 2;                 // lane quarter, column half
    const uint32_t lane_base = tmem + ((uint32_t)(wq * 32) << 16);
    uint32_t phase = 0, buf = 0;
    bool ok = true;
    for (uint32_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, buf ^= 1u) {
        unsigned char* sa = sa0 + buf * T1;
        cp_async_wait_all();                       // x of this tile (and the weights)
        fence_async_shared();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int s = 0; s < K1 / 16; ++s) {
                const uint64_t ad = smem_desc(sm_addr(sa) + s * 256, kLBO, (K1 / 8) * 128);
                const uint64_t bd = smem_desc(sm_addr(sw1) + s * 256, kLBO, (K1 / 8) * 128);
                tc_mma(tmem, ad, bd, idesc_bf16(N), s > 0 ? 1u : 0u);
            }
            tc_commit(&s_bar);
        }
        // the next tile's x into the other buffer (its last reader, the
        // previous tile's MMA 1, has completed)
        const uint32_t next = tile + gridDim.x;
        if (next < ntiles) issue_rows<K1, NT>(sa0 + (buf ^ 1u) * T1, g.E, next * 128, g.M, K1);
        cp_async_commit();
        const int r = wq * 32 + lane;              // this thread's row of the tile
        const uint32_t m = tile * 128 + r;
        const bool valid = m < g.M;
        bool got = mbar_wait(&s_bar, phase);
        ok = __syncthreads_and(got) != 0;
        if (!ok) break;
        phase ^= 1u;
        tc_fence_after();
        // epilogue 1: z = relu(acc + b1) -> shared (MMA 2) and global
#pragma unroll 2
        for (int c0 = part * CW; c0 < part * CW + CW; c0 += 16) {
            float v[16];
            tmem_ld16(lane_base + c0, v);
            const float2* b2v = reinterpret_cast<const float2*>(s_b1 + c0);
            __nv_bfloat162 hh[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float2 a = __fadd2_rn(make_float2(v[2 * q], v[2 * q + 1]), b2v[q]);
                hh[q] = __floats2bfloat162_rn(fmaxf(a.x, 0.f), fmaxf(a.y, 0.f));
            }
            const uint4 z0 = *reinterpret_cast<uint4*>(&hh[0]);
            const uint4 z1 = *reinterpret_cast<uint4*>(&hh[4]);
            *reinterpret_cast<uint4*>(sz + kmajor_offset(r, c0, N)) = z0;
            *reinterpret_cast<uint4*>(sz + kmajor_offset(r, c0 + 8, N)) = z1;
            if (g.Z && valid) {
                uint4* o = reinterpret_cast<uint4*>(g.Z + (size_t)m * N + c0);
                o[0] = z0;
                o[1] = z1;
            }
        }
        fence_async_shared();
        tc_fence_before();
        __syncthreads();                           // z complete
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int s = 0; s < N / 16; ++s) {
                const uint64_t ad = smem_desc(sm_addr(sz) + s * 256, kLBO, (N / 8) * 128);
                const uint64_t bd = smem_desc(sm_addr(sw2) + s * 256, kLBO, (N / 8) * 128);
                tc_mma(tmem + 128, ad, bd, idesc_bf16(N), s > 0 ? 1u : 0u);
            }
            tc_commit(&s_bar);
        }
        got = mbar_wait(&s_bar, phase);
        ok = __syncthreads_and(got) != 0;
        if (!ok) break;
        phase ^= 1u;
        tc_fence_after();
        // epilogue 2: e0 = acc + b2
#pragma unroll 2
        for (int c0 = part * CW; c0 < part * CW + CW; c0 += 16) {
            float v[16];
            tmem_ld16(lane_base + 128 + c0, v);
            if (!valid) continue;
            const float2* b2v = reinterpret_cast<const float2*>(s_b2 + c0);
            __nv_bfloat162 hh[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float2 a = __fadd2_rn(make_float2(v[2 * q], v[2 * q + 1]), b2v[q]);
                hh[q] = __floats2bfloat162_rn(a.x, a.y);
            }
            uint4* o = reinterpret_cast<uint4*>(g.Eout + (size_t)m * N + c0);
            o[0] = *reinterpret_cast<uint4*>(&hh[0]);
            o[1] = *reinterpret_cast<uint4*>(&hh[4]);
        }
        tc_fence_before();
        __syncthreads();
    }
    if (!ok && tid == 0 && g.status) atomicOr(g.status, 1u);
    cp_async_wait_all();
    __syncthreads();
    if (w == 0) tmem_dealloc(tmem, 256);
}

// Named barrier of one half of a 512-thread block (ids 1 and 2, 256 threads),
// and its AND-reduction over a predicate.
__device__ __forceinline__ void half_sync(int h) {
    asm volatile("bar.sync %0, 256;" ::"r"(h + 1) : "memory");
}

__device__ __forceinline__ bool half_and(int h, bool v) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, %2, 256, p;\n"
        " selp.u32 %0, 1, 0, q;\n}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(h + 1)
        : "memory");
    return r != 0;
}

// The fused edge update of a message-passing layer, per 128-edge tile:
//   z = relu(e W1c + b1 + P[src] + Q[dst]),  e' = e + z W2 + b2
// (MMA 1 into TMEM, z written as MMA 2's K-major operand in shared memory and
// to Z when training, MMA 2, the residual e read back from the staged tile),
// as two independent halves of 256 threads that share the weights: half h
// takes the tiles 2 b + h, 2 b + h + 2 grid, ... of block b with its own
// mbarrier, its own 256 TMEM columns (accumulators of MMA 1 and MMA 2) and
// its own named barrier, so one half's MMAs, copies and barriers overlap the
// other half's epilogues.  Per half: the e tile, and the P[src] rows that z
// overwrites; the Q[dst] rows go to registers (each thread's row and 64
// columns): the next tile's are loaded while this tile's MMA 2 and second
// epilogue run.  The next tile's e and P[src] copies are issued at the end
// of a tile, the row indices a tile ahead.
constexpr size_t kEdgePPSmem = (size_t)6 * 128 * 128 * 2;   // W1c, W2, 2 x (e, P/z)

__global__ void __launch_bounds__(512, 1) k_edge_pp(const EdgeArgs g) {
    constexpr int N = 128;
    constexpr uint32_t T = 128 * 128 * 2;
    extern __shared__ __align__(128) unsigned char s_raw[];
    __shared__ __align__(16) float s_b1[128], s_b2[128];
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int h = tid >> 8, lt = tid & 255;              // half, thread within the half
    unsigned char* sw1 = s_raw;                          // W1c^T
    unsigned char* sw2 = s_raw + T;                      // W2^T
    unsigned char* se = s_raw + (2 + h) * T;             // e tile of this half
    unsigned char* spz = s_raw + (4 + h) * T;            // P[src] rows, then z
    if (w == 0) tmem_alloc(&s_tmem, 512);
    if (tid == 0) {
        mbar_init1(&s_bar[0]);
        mbar_init1(&s_bar[1]);
    }
    for (int c = tid; c < N * (N / 8); c += 512) {
        const int r = c % N, gk = c / N;
        cp_async16(sw1 + kmajor_offset(r, gk * 8, N), g.W1t + (size_t)r * N + gk * 8, true);
        cp_async16(sw2 + kmajor_offset(r, gk * 8, N), g.W2t + (size_t)r * N + gk * 8, true);
    }
    if (tid < 128) {
        s_b1[tid] = g.b1[tid];
        s_b2[tid] = g.b2[tid];
    }
    const uint32_t ntiles = (g.M + 127) / 128;
    const uint32_t stride = 2 * gridDim.x;
    const int wq = w & 3, part = (w >> 2) & 1;           // lane quarter, column half
    const int r = wq * 32 + lane;                        // epilogue row of this thread
    const uint32_t gr = (uint32_t)(lt & 127);            // gather row of this thread
    const int gh = lt >> 7;                              // its half of the row's pieces
    // copies of one tile's e and P[src] rows by this half
    auto issue_tile = [&](uint32_t t, uint32_t srow) {
#pragma unroll
        for (int c = lt; c < 128 * (N / 8); c += 256) {
            const int rr = c & 127, gk = c >> 7;
            const bool ok = t * 128 + rr < g.M;
            const __nv_bfloat16* p = ok ? g.E + (size_t)(t * 128 + rr) * N + gk * 8 : g.E;
            cp_async16(se + kmajor_offset(rr, gk * 8, N), p, ok);
        }
        const bool ok = t * 128 + gr < g.M;
        const __nv_bfloat16* p = ok ? g.P + (size_t)srow * N : g.P;
#pragma unroll
        for (int gk = 8 * gh; gk < 8 * gh + 8; ++gk)
            cp_async16(spz + kmajor_offset(gr, gk * 8, N), p + gk * 8, ok);
    };
    // this thread's 64 columns of one Q[dst] row
    uint4 qv[8];
    auto load_q = [&](uint32_t t, uint32_t drow) {
        const bool ok = t * 128 + r < g.M;
        const uint4* q = reinterpret_cast<const uint4*>(g.Q + (size_t)(ok ? drow : 0u) * N + part * 64);
#pragma unroll
        for (int k = 0; k < 8; ++k) qv[k] = ok ? __ldg(q + k) : make_uint4(0u, 0u, 0u, 0u);
    };
    uint32_t tile = 2 * blockIdx.x + (uint32_t)h;
    uint32_t nsrc = 0, ndst = 0;                         // rows of the half's next tile
    if (tile < ntiles) {
        const uint32_t mg = tile * 128 + gr, me = tile * 128 + (uint32_t)r;
        issue_tile(tile, mg < g.M ? g.src[mg] : 0u);
        load_q(tile, me < g.M ? g.dst[me] : 0u);
        const uint32_t nt = tile + stride;
        if (nt < ntiles) {
            if (nt * 128 + gr < g.M) nsrc = g.src[nt * 128 + gr];
            if (nt * 128 + (uint32_t)r < g.M) ndst = g.dst[nt * 128 + r];
        }
    }
    cp_async_commit();
    cp_async_wait_all();                                 // weights of both halves, first tiles
    fence_async_shared();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem + (uint32_t)(h * 256);
    const uint32_t lane_base = tmem + ((uint32_t)(wq * 32) << 16);
    uint32_t phase = 0;
    bool ok = true;
    for (; tile < ntiles && ok; tile += stride) {
        cp_async_wait_all();                             // e, P[src] of this tile
        fence_async_shared();
        tc_fence_before();
        half_sync(h);
        if (lt == 0) {
            tc_fence_after();
#pragma unroll
            for (int s = 0; s < N / 16; ++s) {
                const uint64_t ad = smem_desc(sm_addr(se) + s * 256, kLBO, (N / 8) * 128);
                const uint64_t bd = smem_desc(sm_addr(sw1) + s * 256, kLBO, (N / 8) * 128);
                tc_mma(tmem, ad, bd, idesc_bf16(N), s > 0 ? 1u : 0u);
            }
            tc_commit(&s_bar[h]);
        }
        const uint32_t m = tile * 128 + (uint32_t)r;
        const bool valid = m < g.M;
        const uint32_t next = tile + stride;
        bool got = mbar_wait(&s_bar[h], phase);
        ok = half_and(h, got);
        if (!ok) break;
        phase ^= 1u;
        tc_fence_after();
        // epilogue 1: z = relu(((acc + b1) + P[src]) + Q[dst]) over the P rows, and to Z
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int c0 = part * 64 + 16 * k;
            float v[16];
            tmem_ld16(lane_base + c0, v);
            float t[16], u[16];
            unpack8(*reinterpret_cast<const uint4*>(spz + kmajor_offset(r, c0, N)), t);
            unpack8(*reinterpret_cast<const uint4*>(spz + kmajor_offset(r, c0 + 8, N)), t + 8);
            unpack8(qv[2 * k], u);
            unpack8(qv[2 * k + 1], u + 8);
            const float2* b2v = reinterpret_cast<const float2*>(s_b1 + c0);
            __nv_bfloat162 hh[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                float2 a = __fadd2_rn(make_float2(v[2 * q], v[2 * q + 1]), b2v[q]);
                a = __fadd2_rn(a, make_float2(t[2 * q], t[2 * q + 1]));
                a = __fadd2_rn(a, make_float2(u[2 * q], u[2 * q + 1]));
                hh[q] = __floats2bfloat162_rn(fmaxf(a.x, 0.f), fmaxf(a.y, 0.f));
            }
            const uint4 z0 = *reinterpret_cast<uint4*>(&hh[0]);
            const uint4 z1 = *reinterpret_cast<uint4*>(&hh[4]);
            *reinterpret_cast<uint4*>(spz + kmajor_offset(r, c0, N)) = z0;
            *reinterpret_cast<uint4*>(spz + kmajor_offset(r, c0 + 8, N)) = z1;
            if (g.Z && valid) {
                uint4* o = reinterpret_cast<uint4*>(g.Z + (size_t)m * N + c0);
                o[0] = z0;
                o[1] = z1;
            }
        }
        fence_async_shared();
        tc_fence_before();
        half_sync(h);                                    // z complete
        if (lt == 0) {
            tc_fence_after();
#pragma unroll
            for (int s = 0; s < N / 16; ++s) {
                const uint64_t ad = smem_desc(sm_addr(spz) + s * 256, kLBO, (N / 8) * 128);
                const uint64_t bd = smem_desc(sm_addr(sw2) + s * 256, kLBO, (N / 8) * 128);
                tc_mma(tmem + 128, ad, bd, idesc_bf16(N), s > 0 ? 1u : 0u);
            }
            tc_commit(&s_bar[h]);
        }
        // the next tile's Q[dst] rows into registers, the rows of the one after
        uint32_t nsrc2 = 0, ndst2 = 0;
        if (next < ntiles) {
            load_q(next, ndst);
            const uint32_t n2 = next + stride;
            if (n2 < ntiles) {
                if (n2 * 128 + gr < g.M) nsrc2 = __ldg(g.src + n2 * 128 + gr);
                if (n2 * 128 + (uint32_t)r < g.M) ndst2 = __ldg(g.dst + n2 * 128 + r);
            }
        }
        got = mbar_wait(&s_bar[h], phase);
        ok = half_and(h, got);
        if (!ok) break;
        phase ^= 1u;
        tc_fence_after();
        // epilogue 2: e' = (acc + b2) + e
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int c0 = part * 64 + 16 * k;
            float v[16];
            tmem_ld16(lane_base + 128 + c0, v);
            if (!valid) continue;
            float t[16];
            unpack8(*reinterpret_cast<const uint4*>(se + kmajor_offset(r, c0, N)), t);
            unpack8(*reinterpret_cast<const uint4*>(se + kmajor_offset(r, c0 + 8, N)), t + 8);
            const float2* b2v = reinterpret_cast<const float2*>(s_b2 + c0);
            __nv_bfloat162 hh[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                float2 a = __fadd2_rn(make_float2(v[2 * q], v[2 * q + 1]), b2v[q]);
                a = __fadd2_rn(a, make_float2(t[2 * q], t[2 * q + 1]));
                hh[q] = __floats2bfloat162_rn(a.x, a.y);
            }
            uint4* o = reinterpret_cast<uint4*>(g.Eout + (size_t)m * N + c0);
            o[0] = *reinterpret_cast<uint4*>(&hh[0]);
            o[1] = *reinterpret_cast<uint4*>(&hh[4]);
        }
        tc_fence_before();
        half_sync(h);                                    // e and z tiles free
        if (next < ntiles) issue_tile(next, nsrc);
        cp_async_commit();
        nsrc = nsrc2;
        ndst = ndst2;
    }
    if (!ok && lt == 0 && g.status) atomicOr(g.status, 1u);
    cp_async_wait_all();
    __syncthreads();
    if (w == 0) tmem_dealloc(s_tmem, 512);
}

template <int K, int N>
size_t linear_smem() { return (size_t)2 * 128 * K * 2 + (size_t)N * K * 2; }

template <int K, int N>
void launch_linear_t(const LinearArgs& g, int sms, cudaStream_t st) {
    static bool init = false;
    const size_t smem = linear_smem<K, N>();
    if (!init) {
        cudaFuncSetAttribute(k_linear<K, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        init = true;
    }
    // resident blocks per SM: shared memory, registers and the SM's 512
    // TMEM columns
    static int per_sm = 0;
    if (!per_sm) {
        cudaFuncAttributes fa{};
        cudaFuncGetAttributes(&fa, k_linear<K, N>);
        const int cols = N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : 256));
        const int by_smem = (int)((228u * 1024u) / (smem + fa.sharedSizeBytes + 1024u));
        const int by_regs = fa.numRegs > 0 ? 65536 / (linear_threads<N>() * fa.numRegs) : 1;
        per_sm = by_smem < by_regs ? by_smem : by_regs;
        if (per_sm > 512 / cols) per_sm = 512 / cols;
        if (per_sm < 1) per_sm = 1;
    }
    const uint32_t tiles = (g.M + 127) / 128;
    uint32_t grid = (uint32_t)(sms * per_sm);
    if (grid > tiles) grid = tiles ? tiles : 1;
    k_linear<K, N><<<grid, linear_threads<N>(), smem, st>>>(g);
}

template <int N>
void launch_wgrad_t(const WgradArgs& g, int sms, cudaStream_t st) {
    static bool init = false;
    const size_t smem = (size_t)128 * 128 * 2 + (size_t)N * 128 * 2;
    if (!init) {
        cudaFuncSetAttribute(k_wgrad<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        init = true;
    }
    const uint32_t tiles = (g.M + 127) / 128;
    uint32_t grid = (uint32_t)g.nparts;
    if (grid > tiles) grid = tiles ? tiles : 1;
    k_wgrad<N><<<grid, 128, smem, st>>>(g);
    const int count = 128 * N;
    k_wgrad_reduce<<<(count + 255) / 256, 256, 0, st>>>(g.partial, (int)grid, count, g.dW, g.scale);
}

int g_sms = 0;

}  // namespace

int num_sms() {
    if (!g_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_sms <= 0) g_sms = 1;
    }
    return g_sms;
}

bool launch_linear(int K, int N, const LinearArgs& g, cudaStream_t st) {
    const int sms = num_sms();
    if (g.M == 0) return true;
    if (K == 16 && N == 128) launch_linear_t<16, 128>(g, sms, st);
    else if (K == 128 && N == 128) launch_linear_t<128, 128>(g, sms, st);
    else if (K == 256 && N == 128) launch_linear_t<256, 128>(g, sms, st);
    else if (K == 128 && N == 16) launch_linear_t<128, 16>(g, sms, st);
    else if (K == 16 && N == 16) launch_linear_t<16, 16>(g, sms, st);
    else if (K == 128 && N == 256) launch_linear_t<128, 256>(g, sms, st);
    else return false;
    return true;
}

// The layer: two halves per block, one block per SM (192 KB of shared memory,
// the SM's 512 TMEM columns).
void launch_edge_layer(const EdgeArgs& g, cudaStream_t st) {
    static bool init = false;
    if (!init) {
        cudaFuncSetAttribute(k_edge_pp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEdgePPSmem);
        init = true;
    }
    if (g.M == 0) return;
    const uint32_t tiles = (g.M + 127) / 128;
    uint32_t grid = (uint32_t)num_sms();
    if (grid > (tiles + 1) / 2) grid = (tiles + 1) / 2;
    k_edge_pp<<<grid, 512, kEdgePPSmem, st>>>(g);
}

// The encoder: two 256-thread blocks per SM.
void launch_edge_encoder(const EdgeArgs& g, cudaStream_t st) {
    static bool init = false;
    if (!init) {
        cudaFuncSetAttribute(k_edge_encoder, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEncSmem);
        init = true;
    }
    if (g.M == 0) return;
    const uint32_t tiles = (g.M + 127) / 128;
    uint32_t grid = (uint32_t)(num_sms() * 2);
    if (grid > tiles) grid = tiles;
    k_edge_encoder<<<grid, 256, kEncSmem, st>>>(g);
}

bool launch_wgrad(int N, const WgradArgs& g, cudaStream_t st) {
    if (N == 128) launch_wgrad_t<128>(g, num_sms(), st);
    else if (N == 16) launch_wgrad_t<16>(g, num_sms(), st);
    else return false;
    return true;
}

}  // namespace sur
