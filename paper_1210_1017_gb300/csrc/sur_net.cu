// The learned surrogate: a message-passing network on the radius-2h
// neighbour graph of the SPH cell list (encoder, `layers` message-passing
// layers, decoder), forward, backward and Adam, with every dense layer on the
// tcgen05 tensor cores (sur_linear.cu) and the graph work in the kernels here.
//
// Nodes are the particles of an SPH context in its (cell, id)-sorted order;
// inputs and outputs are indexed by particle id.  Node input: the last five
// velocities / v_scale and the boundary flag (16 features).  Edge input:
// (r_i - r_j) / 2h and |r_i - r_j| / 2h (padded to 16).  Latent width 128.
//   edge update: e' = e + W2 relu(W1a h_i + W1b h_j + W1c e + b1) + b2
//   node update: h' = h + W4 relu(W3 [h, sum_j e'_ij] + b3) + b4
//   decoder:     out = W6 relu(W5 h + b5) + b6   (first 3 of 16 outputs: the
//                normalised acceleration)
#include <math.h>
#include <string.h>

#include <string>
#include <vector>

#include "../../include/sph.h"
#include "../../include/sur.h"
#include "sph_ctx.cuh"
#include "sur_internal.cuh"

using namespace sur;

namespace {

constexpr int L = 128;       // latent width
constexpr int KIN = 16;      // padded input width of the encoders
constexpr int KOUT = 16;     // padded decoder output width
constexpr uint32_t kWgradParts = 3 * 152;   // three blocks per SM

struct Layer {
    int kin, kout;
    bool bias;
    size_t w_off, b_off;     // offsets in the flat parameter array
    __nv_bfloat16* Wt;       // kout x kin (forward operand)
    __nv_bfloat16* W;        // kin x kout (backward operand)
};

__global__ void k_cast_bf16(const float* __restrict__ in, __nv_bfloat16* __restrict__ out,
                            size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        out[i] = __float2bfloat16_rn(in[i]);
}

// W (kin x kout, fp32 row-major) -> bf16 W and bf16 W^T.
__global__ void k_refresh(const float* __restrict__ w, int kin, int kout, __nv_bfloat16* W,
                          __nv_bfloat16* Wt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kin * kout) return;
    const int r = i / kout, c = i % kout;
    const __nv_bfloat16 v = __float2bfloat16_rn(w[i]);
    W[i] = v;
    Wt[(size_t)c * kin + r] = v;
}

// ----------------------------------------------------------------- graph --

// Neighbours j != i with |r_ij|^2 < r2 (FP64 predicate; r2 = (2h)^2 as the
// SPH cell list defines neighbours, or (radius 2h)^2 for a sparser graph),
// visited in ascending sorted index: the 9 rows of cells around i's cell in
// (z, y) order, cells in x order.
//
// The predicate is decided in FP32 where that is exact: with the positions
// relative to their own cell origins (posc, rounded once from FP64) and
// whole-cell offsets, each coordinate difference is within 6 roundings of
// 2^-24 of a cell (3.6e-7 cs), so |d2_32 - d2_64| < 2 sqrt(3) r 3.6e-7 cs +
// 1.8e-7 r^2, below 1.3e-5 r2 for r >= 0.1 cs.  So d2_32 < `inside` (r2
// (1 - 2^-12)) is inside and d2_32 >= `outside` (r2 (1 + 2^-12)) or not
// finite is outside;
// the caller widens both to "always ask FP64" for radii below 0.1 cell.
// Candidates in between take the FP64 arithmetic of the predicate as
// written.  The edge features (bfloat16) come from the FP32 differences.
// FP64 instructions run at 1/64 of the FP32 rate on this GPU.
template <int MODE>
__global__ void k_graph(const sph::Dev d, const double* __restrict__ x, const double* __restrict__ y,
                        const double* __restrict__ z, const float4* __restrict__ posc,
                        const uint32_t* __restrict__ key, const uint32_t* __restrict__ off,
                        uint32_t* __restrict__ cnt, const uint32_t* __restrict__ rowptr,
                        uint32_t* __restrict__ col, uint32_t* __restrict__ src,
                        __nv_bfloat16* __restrict__ xe, double inv2h, double r2, float inside,
                        float outside) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    const uint32_t n_in = off[d.ncells];
    if (i >= n_in) {
        if (MODE == 0) cnt[i] = 0;
        return;
    }
    const uint32_t k = key[i];
    uint32_t lo = 0, hi = d.n_inst;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (d.cell_base[mid] <= k) lo = mid;
        else hi = mid;
    }
    const sph::Inst& I = d.inst[lo];
    const uint32_t lk = k - I.cell_base;
    const int cx = (int)(lk % (uint32_t)I.ncx);
    const uint32_t t = lk / (uint32_t)I.ncx;
    const int cy = (int)(t % (uint32_t)I.ncy), cz = (int)(t / (uint32_t)I.ncy);
    const double xi = x[i], yi = y[i], zi = z[i];
    const float4 pi = posc[i];
    const float inv2hf = (float)inv2h;
    const int xlo = cx > 0 ? cx - 1 : 0, xhi = cx + 1 < I.ncx ? cx + 1 : I.ncx - 1;
    uint32_t c = 0, e = MODE ? rowptr[i] : 0u;
    for (int zz = cz - 1; zz <= cz + 1; ++zz) {
        if (zz < 0 || zz >= I.ncz) continue;
        const float qz = fmaf((float)(cz - zz), d.csf, pi.z);
        for (int yy = cy - 1; yy <= cy + 1; ++yy) {
            if (yy < 0 || yy >= I.ncy) continue;
            const float qy = fmaf((float)(cy - yy), d.csf, pi.y);
            const uint32_t rb = I.cell_base + (uint32_t)I.ncx * ((uint32_t)yy + (uint32_t)I.ncy * zz);
            for (int xx = xlo; xx <= xhi; ++xx) {
                const float qx = fmaf((float)(cx - xx), d.csf, pi.x);
                const uint32_t s = off[rb + xx], en = off[rb + xx + 1];
                for (uint32_t j = s; j < en; ++j) {
                    if (j == i) continue;
                    const float4 pj = posc[j];
                    const float fx = qx - pj.x, fy = qy - pj.y, fz = qz - pj.z;
                    const float d2f = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
                    // outside, or not finite (the FP64 predicate rejects those too)
                    if (!(d2f < outside)) continue;
                    if (!(d2f < inside)) {
                        const double dx = __dsub_rn(xi, x[j]);
                        const double dy = __dsub_rn(yi, y[j]);
                        const double dz = __dsub_rn(zi, z[j]);
                        const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                                                    __dmul_rn(dz, dz));
                        if (!(d2 < r2)) continue;
                    }
                    if (MODE) {
                        // the edge inputs are bfloat16: the FP32 differences (within
                        // 3.6e-7 of a cell of the FP64 ones) round to the bfloat16 of
                        // the FP64 value except where that lies within this error of
                        // a rounding midpoint (one bfloat16 step then)
                        col[e] = j;
                        src[e] = i;
                        // one 32-byte row: (x, y, z, |r|) / 2h, then zeros
                        const __nv_bfloat162 f01 = __floats2bfloat162_rn(fx * inv2hf, fy * inv2hf);
                        const __nv_bfloat162 f23 =
                            __floats2bfloat162_rn(fz * inv2hf, sqrtf(d2f) * inv2hf);
                        uint4* f = reinterpret_cast<uint4*>(xe + (size_t)e * KIN);
                        f[0] = make_uint4(*reinterpret_cast<const uint32_t*>(&f01),
                                          *reinterpret_cast<const uint32_t*>(&f23), 0u, 0u);
                        f[1] = make_uint4(0u, 0u, 0u, 0u);
                        ++e;
                    }
                    ++c;
                }
            }
        }
    }
    if (MODE == 0) cnt[i] = c;
}

// rev[e] = index of the edge (j, i) in row j (rows are sorted ascending).
__global__ void k_graph_rev(uint32_t E, const uint32_t* __restrict__ rowptr,
                            const uint32_t* __restrict__ col, const uint32_t* __restrict__ src,
                            uint32_t* __restrict__ rev) {
    const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const uint32_t i = src[e], j = col[e];
    uint32_t lo = rowptr[j], hi = rowptr[j + 1];
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (col[mid] < i) lo = mid + 1;
        else hi = mid;
    }
    rev[e] = lo;
}

// Node inputs: five velocities (history indexed by particle id, oldest
// first) / v_scale, boundary flag.
__global__ void k_node_features(const sph::Dev d, const uint32_t* __restrict__ id,
                                const float* __restrict__ hist, double inv_v,
                                __nv_bfloat16* __restrict__ xn) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    const uint32_t pid = id[i];
    uint32_t lo = 0, hi = d.n_inst;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (d.id_base[mid] <= pid) lo = mid;
        else hi = mid;
    }
    const bool bound = pid < d.inst[lo].id_fluid;
    __nv_bfloat16* f = xn + (size_t)i * KIN;
#pragma unroll
    for (int q = 0; q < 15; ++q) f[q] = __double2bfloat16((double)hist[(size_t)pid * 15 + q] * inv_v);
    f[15] = __float2bfloat16_rn(bound ? 1.f : 0.f);
}

// out[i, 0:128] = sum over the edges of row i of e[edge, 0:128] (fp32 sum in
// edge order, one warp per node, 4 features per lane).
template <typename T>
__global__ void k_rowsum(uint32_t n, const uint32_t* __restrict__ rowptr, const T* __restrict__ e,
                         const uint32_t* __restrict__ perm, __nv_bfloat16* out_bf, float* out_f,
                         uint32_t ldo) {
    const uint32_t node = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (node >= n) return;
    // each lane sums its 4 columns over the node's edges in edge order; one
    // 8-byte (bf16) or 16-byte (fp32) load per edge and lane, several edges
    // in flight
    float s[4] = {0.f, 0.f, 0.f, 0.f};
    const uint32_t k0 = rowptr[node], k1 = rowptr[node + 1];
#pragma unroll 4
    for (uint32_t k = k0; k < k1; ++k) {
        const uint32_t ed = perm ? perm[k] : k;
        if constexpr (sizeof(T) == 2) {
            const uint2 u = __ldg(reinterpret_cast<const uint2*>(e + (size_t)ed * L) + lane);
            const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
            const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
            s[0] += a.x;
            s[1] += a.y;
            s[2] += b.x;
            s[3] += b.y;
        } else {
            const float4 u = __ldg(reinterpret_cast<const float4*>(e + (size_t)ed * L) + lane);
            s[0] += u.x;
            s[1] += u.y;
            s[2] += u.z;
            s[3] += u.w;
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (out_bf) out_bf[(size_t)node * ldo + lane * 4 + q] = __float2bfloat16_rn(s[q]);
        if (out_f) out_f[(size_t)node * ldo + lane * 4 + q] = s[q];
    }
}

// out[i] += in[i] (fp32), and a bf16 copy of the sum.
__global__ void k_add_gather(size_t count, float* __restrict__ acc, const float* __restrict__ node,
                             const uint32_t* __restrict__ src, uint32_t ldn,
                             __nv_bfloat16* __restrict__ out_bf) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count;
         t += (size_t)gridDim.x * blockDim.x) {
        const size_t e = t / L, c = t % L;
        float v = acc[t];
        if (node) v += node[(size_t)src[e] * ldn + c];
        acc[t] = v;
        out_bf[t] = __float2bfloat16_rn(v);
    }
}

// Column sums of an (M x C) matrix into grad[0:C] (block partials in a fixed
// order, then one block adds them).
template <typename T>
__global__ void k_colsum_part(uint32_t M, int C, const T* __restrict__ in, uint32_t ld,
                              float* __restrict__ part) {
    const int c = threadIdx.x;   // blockDim = C
    float s = 0.f;
#pragma unroll 8
    for (uint32_t m = blockIdx.x; m < M; m += gridDim.x) {
        if constexpr (sizeof(T) == 2) s += __bfloat162float(in[(size_t)m * ld + c]);
        else s += in[(size_t)m * ld + c];
    }
    part[(size_t)blockIdx.x * C + c] = s;
}

__global__ void k_colsum_final(int nparts, int C, const float* __restrict__ part,
                               float* __restrict__ out, float scale) {
    const int c = threadIdx.x;
    if (c >= C) return;
    float s = 0.f;
    for (int b = 0; b < nparts; ++b) s += part[(size_t)b * C + c];
    out[c] = s * scale;
}

// Loss over fluid nodes and its gradient: out (n x 16 fp32, sorted order),
// target (by id, n x 3).  dOUT (bf16, n x 16) = 2 (out - target) / n_fluid.
__global__ void k_loss(const sph::Dev d, const uint32_t* __restrict__ id,
                       const float* __restrict__ out, const float* __restrict__ target,
                       const uint32_t* __restrict__ off, float inv_nf,
                       __nv_bfloat16* __restrict__ dout, float* __restrict__ part) {
    __shared__ float s_sum[256];
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (i < d.n) {
        const uint32_t n_in = off[d.ncells];
        const uint32_t pid = id[i];
        uint32_t lo = 0, hi = d.n_inst;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (d.id_base[mid] <= pid) lo = mid;
            else hi = mid;
        }
        const bool fluid = i < n_in && pid >= d.inst[lo].id_fluid;
#pragma unroll
        for (int c = 0; c < KOUT; ++c) {
            float g = 0.f;
            if (fluid && c < 3) {
                const float r = out[(size_t)i * KOUT + c] - target[(size_t)pid * 3 + c];
                l += r * r;
                g = 2.f * r * inv_nf;
            }
            dout[(size_t)i * KOUT + c] = __float2bfloat16_rn(g);
        }
    }
    s_sum[threadIdx.x] = l;
    __syncthreads();
    for (int st = 128; st; st >>= 1) {
        if (threadIdx.x < st) s_sum[threadIdx.x] += s_sum[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s_sum[0];
}

__global__ void k_loss_final(int nparts, const float* __restrict__ part, float inv_nf,
                             float* __restrict__ loss) {
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int b = 0; b < nparts; ++b) s += part[b];
    *loss = (float)(s * inv_nf);
}

__global__ void k_adam(size_t n, float* __restrict__ w, const float* __restrict__ g,
                       float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// Output (sorted order, normalised) -> by id, denormalised acceleration.
__global__ void k_write_out(const sph::Dev d, const uint32_t* __restrict__ id,
                            const float* __restrict__ out, float3 am, float3 as,
                            float* __restrict__ acc_by_id) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    const uint32_t pid = id[i];
    acc_by_id[(size_t)pid * 3 + 0] = out[(size_t)i * KOUT + 0] * as.x + am.x;
    acc_by_id[(size_t)pid * 3 + 1] = out[(size_t)i * KOUT + 1] * as.y + am.y;
    acc_by_id[(size_t)pid * 3 + 2] = out[(size_t)i * KOUT + 2] * as.z + am.z;
}

// Semi-implicit Euler over dt_s for fluid particles of the SPH state (sorted
// order): v += a dt, r += v dt (FP64 positions); boundary and excluded
// particles stay.  The velocity history (by id) shifts by one.
__global__ void k_advance(const sph::Dev d, const uint32_t* __restrict__ id, double* x, double* y,
                          double* z, float4* vr, const uint32_t* __restrict__ off,
                          const float* __restrict__ acc_by_id, float* hist, float dt) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    const uint32_t pid = id[i];
    uint32_t lo = 0, hi = d.n_inst;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (d.id_base[mid] <= pid) lo = mid;
        else hi = mid;
    }
    const bool fluid = i < off[d.ncells] && pid >= d.inst[lo].id_fluid;
    float4 v = vr[i];
    if (fluid) {
        v.x += acc_by_id[(size_t)pid * 3 + 0] * dt;
        v.y += acc_by_id[(size_t)pid * 3 + 1] * dt;
        v.z += acc_by_id[(size_t)pid * 3 + 2] * dt;
        x[i] += (double)(v.x * dt);
        y[i] += (double)(v.y * dt);
        z[i] += (double)(v.z * dt);
        vr[i] = v;
    }
    float* h = hist + (size_t)pid * 15;
#pragma unroll
    for (int q = 0; q < 12; ++q) h[q] = h[q + 3];
    h[12] = fluid ? v.x : 0.f;
    h[13] = fluid ? v.y : 0.f;
    h[14] = fluid ? v.z : 0.f;
}

inline uint32_t nblk(size_t n, uint32_t t) { return (uint32_t)((n + t - 1) / t); }

// ---------------------------------------------------------- training data --

// SplitMix64 finaliser (Steele, Lea & Flood, 2014) as a counter-based
// generator: the 64-bit output for counter k under a seed.
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// One standard normal per counter (Box-Muller on two 32-bit uniforms).
__device__ __forceinline__ double normal01(uint64_t seed, uint64_t k) {
    const uint64_t r = splitmix64(seed ^ splitmix64(k));
    const double u1 = ((double)(uint32_t)(r >> 32) + 1.0) * (1.0 / 4294967296.0);   // (0, 1]
    const double u2 = (double)(uint32_t)r * (1.0 / 4294967296.0);                    // [0, 1)
    return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

// A training sample from seven saved frames by id (f = 0..6 hold
// x^{k-5} .. x^{k+1}, spaced dt): random-walk noise on the input frames
// (increments of std sigma / sqrt(5) from frame 1 on, so x^k carries std
// sigma; boundary particles none), finite-difference velocities of the
// noisy frames, and the acceleration that brings the noisy x^k to the clean
// x^{k+1} under semi-implicit Euler, normalised.
__global__ void k_make_sample(const sph::Dev d, const double* __restrict__ frames, uint32_t n,
                              double sigma, uint64_t seed, double dt, float3 am, float3 as,
                              double* __restrict__ pos, float* __restrict__ vel,
                              float* __restrict__ hist, float* __restrict__ target) {
    const uint32_t pid = blockIdx.x * blockDim.x + threadIdx.x;
    if (pid >= n) return;
    uint32_t lo = 0, hi = d.n_inst;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (d.id_base[mid] <= pid) lo = mid;
        else hi = mid;
    }
    const bool bound = pid < d.inst[lo].id_fluid;
    const double step_sd = bound ? 0.0 : sigma / sqrt(5.0);
    const double inv_dt = 1.0 / dt;
    const float amv[3] = {am.x, am.y, am.z}, asv[3] = {as.x, as.y, as.z};
    for (int a = 0; a < 3; ++a) {
        double xt[6];
        double walk = 0.0;
        for (int f = 0; f < 6; ++f) {
            if (f > 0 && step_sd > 0.0)
                walk += step_sd * normal01(seed, ((uint64_t)pid * 8u + (uint64_t)f) * 4u + (uint64_t)a);
            xt[f] = frames[((size_t)f * n + pid) * 3 + a] + walk;
        }
        for (int f = 1; f < 6; ++f)
            hist[(size_t)pid * 15 + (f - 1) * 3 + a] = (float)((xt[f] - xt[f - 1]) * inv_dt);
        const double x6 = frames[((size_t)6 * n + pid) * 3 + a];
        const double acc = (x6 - 2.0 * xt[5] + xt[4]) * inv_dt * inv_dt;
        pos[(size_t)pid * 3 + a] = xt[5];
        vel[(size_t)pid * 3 + a] = (float)((xt[5] - xt[4]) * inv_dt);
        target[(size_t)pid * 3 + a] = (float)((acc - (double)amv[a]) / (double)asv[a]);
    }
}

// out (cols x rows) = in (rows x cols)^T
__global__ void k_transpose(const float* __restrict__ in, int rows, int cols, float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * cols) return;
    const int r = i / cols, c = i % cols;
    out[(size_t)c * rows + r] = in[i];
}
inline uint32_t gridcap(size_t n, uint32_t t) {
    const size_t b = (n + t - 1) / t;
    return (uint32_t)(b > 4096 ? 4096 : (b ? b : 1));
}

struct Carve {
    char* base;
    size_t used = 0;
    template <typename T>
    T* take(size_t count) {
        used = (used + 255) / 256 * 256;
        T* p = base ? (T*)(base + used) : nullptr;
        used += count * sizeof(T);
        return p;
    }
};

}  // namespace

struct sur_ctx {
    sur_config cfg;
    cudaStream_t st = nullptr;
    std::vector<Layer> layers;
    size_t nparams = 0;
    int NL = 0;
    // parameters
    float *w, *g, *m, *v;
    unsigned long long adam_t = 0;
    // graph
    uint32_t *cnt, *rowptr, *bsum, *col, *src, *rev;
    uint32_t n = 0, E = 0;
    // activations (train: one per layer; inference: ping-pong)
    __nv_bfloat16 *xn, *xe, *en1, *ee1;
    std::vector<__nv_bfloat16*> XN, Ebuf, Z1, Y1;
    __nv_bfloat16 *P, *Q, *D1;
    float* out;
    // backward
    float *dH, *dXN, *dE, *partial, *colpart, *losspart, *loss;
    __nv_bfloat16 *dHb, *dY1, *dEb, *dpre, *dPb, *dQb, *dD1, *dout, *dEe1, *dEn1;
    float *acc;   // predicted acceleration by id (n x 3)
    float* wg_tmp;   // 128 x 128 scratch for transposed weight gradients
    bool have_forward = false;
    std::string err;
};

namespace {

void build_layers(sur_ctx* c) {
    c->layers.clear();
    size_t off = 0;
    auto add = [&](int kin, int kout, bool bias) {
        Layer l{};
        l.kin = kin;
        l.kout = kout;
        l.bias = bias;
        l.w_off = off;
        off += (size_t)kin * kout;
        l.b_off = off;
        if (bias) off += kout;
        c->layers.push_back(l);
    };
    add(KIN, L, true);  // 0 encoder node 1
    add(L, L, true);    // 1 encoder node 2
    add(KIN, L, true);  // 2 encoder edge 1
    add(L, L, true);    // 3 encoder edge 2
    for (int l = 0; l < c->NL; ++l) {
        add(L, L, false);     // W1a (h_i)
        add(L, L, false);     // W1b (h_j)
        add(L, L, true);      // W1c (e), b1
        add(L, L, true);      // W2, b2
        add(2 * L, L, true);  // W3, b3
        add(L, L, true);      // W4, b4
    }
    add(L, L, true);     // decoder 1
    add(L, KOUT, true);  // decoder 2
    c->nparams = off;
}

size_t carve(sur_ctx* c, void* base) {
    Carve cv{(char*)base};
    const size_t N = c->cfg.max_nodes, E = c->cfg.max_edges;
    const bool train = c->cfg.train != 0;
    const int NL = c->NL;
    c->w = cv.take<float>(c->nparams);
    c->g = cv.take<float>(c->nparams);
    c->m = cv.take<float>(c->nparams);
    c->v = cv.take<float>(c->nparams);
    for (Layer& l : c->layers) {
        l.Wt = cv.take<__nv_bfloat16>((size_t)l.kin * l.kout);
        l.W = cv.take<__nv_bfloat16>((size_t)l.kin * l.kout);
    }
    c->cnt = cv.take<uint32_t>(N + 1);
    c->rowptr = cv.take<uint32_t>(N + 2);
    c->bsum = cv.take<uint32_t>(sph::scan_bsum_count(N + 1));
    c->col = cv.take<uint32_t>(E);
    c->src = cv.take<uint32_t>(E);
    c->rev = cv.take<uint32_t>(E);
    c->xn = cv.take<__nv_bfloat16>(N * KIN);
    c->xe = cv.take<__nv_bfloat16>(E * KIN);
    c->en1 = cv.take<__nv_bfloat16>(N * L);
    c->ee1 = train ? cv.take<__nv_bfloat16>(E * L) : nullptr;   // encoder hidden layer (backward only)
    const int nx = train ? NL + 1 : 2, ne = train ? NL + 1 : 2, nz = train ? NL : 0;
    c->XN.assign(nx, nullptr);
    c->Ebuf.assign(ne, nullptr);
    c->Z1.assign(nz, nullptr);
    c->Y1.assign(train ? NL : 1, nullptr);
    for (auto& p : c->XN) p = cv.take<__nv_bfloat16>(N * 2 * L);
    for (auto& p : c->Ebuf) p = cv.take<__nv_bfloat16>(E * L);
    for (auto& p : c->Z1) p = cv.take<__nv_bfloat16>(E * L);
    for (auto& p : c->Y1) p = cv.take<__nv_bfloat16>(N * L);
    c->P = cv.take<__nv_bfloat16>(N * L);
    c->Q = cv.take<__nv_bfloat16>(N * L);
    c->D1 = cv.take<__nv_bfloat16>(N * L);
    c->out = cv.take<float>(N * KOUT);
    c->acc = cv.take<float>(N * 3);
    c->partial = cv.take<float>((size_t)kWgradParts * L * L);
    c->colpart = cv.take<float>((size_t)1024 * 2 * L);
    c->losspart = cv.take<float>(nblk(N, 256) + 1);
    c->loss = cv.take<float>(1);
    c->wg_tmp = cv.take<float>((size_t)L * L);
    if (train) {
        c->dH = cv.take<float>(N * L);
        c->dXN = cv.take<float>(N * 2 * L);
        c->dE = cv.take<float>(E * L);
        c->dHb = cv.take<__nv_bfloat16>(N * L);
        c->dY1 = cv.take<__nv_bfloat16>(N * L);
        c->dEb = cv.take<__nv_bfloat16>(E * L);
        c->dpre = cv.take<__nv_bfloat16>(E * L);
        c->dPb = cv.take<__nv_bfloat16>(N * L);
        c->dQb = cv.take<__nv_bfloat16>(N * L);
        c->dD1 = cv.take<__nv_bfloat16>(N * L);
        c->dout = cv.take<__nv_bfloat16>(N * KOUT);
        c->dEe1 = cv.take<__nv_bfloat16>(E * L);
        c->dEn1 = cv.take<__nv_bfloat16>(N * L);
    }
    return (cv.used + 255) / 256 * 256;
}

int fail(sur_ctx* c, int code, const char* msg) {
    if (c) c->err = msg;
    return code;
}

int linear(sur_ctx* c, const __nv_bfloat16* A, uint32_t lda, const Layer& l, bool use_W,
           uint32_t M, int epi, const __nv_bfloat16* res, uint32_t ldr, __nv_bfloat16* out_bf,
           float* out_f, uint32_t ldo, bool with_bias = true) {
    LinearArgs g = {};
    g.A = A;
    g.lda = lda;
    // forward: out = A W (+ b) uses W^T as the K-major operand; backward:
    // dX = dY W^T uses W itself
    g.Bt = use_W ? l.W : l.Wt;
    g.bias = (!use_W && with_bias && l.bias) ? c->w + l.b_off : nullptr;
    g.M = M;
    g.epi = epi;
    g.res = res;
    g.ldr = ldr;
    g.out_bf16 = out_bf;
    g.out_f32 = out_f;
    g.ldo = ldo;
    const int K = use_W ? l.kout : l.kin, N = use_W ? l.kin : l.kout;
    if (!launch_linear(K, N, g, c->st)) return fail(c, SPH_ERR_INVALID_ARG, "unsupported layer shape");
    return SPH_OK;
}

// The fused edge update of one layer: z = relu(e W1c + b1 + P[src] + Q[dst])
// (kept for the backward pass when z != null), e' = e + z W2 + b2.
void edge_layer(sur_ctx* c, const Layer& l1, const Layer& l2, const __nv_bfloat16* e,
                __nv_bfloat16* z, __nv_bfloat16* e_out) {
    EdgeArgs g = {};
    g.E = e;
    g.W1t = l1.Wt;
    g.W2t = l2.Wt;
    g.b1 = c->w + l1.b_off;
    g.b2 = c->w + l2.b_off;
    g.P = c->P;
    g.Q = c->Q;
    g.src = c->src;
    g.dst = c->col;
    g.M = c->E;
    g.Z = z;
    g.Eout = e_out;
    launch_edge_layer(g, c->st);
}

// The two edge-encoder layers in one kernel: e0 = relu(xe W + b) W' + b'
// (the hidden activation kept for the backward pass when z != null).
void edge_encoder(sur_ctx* c, const Layer& l1, const Layer& l2, __nv_bfloat16* z, __nv_bfloat16* e0) {
    EdgeArgs g = {};
    g.E = c->xe;
    g.W1t = l1.Wt;
    g.W2t = l2.Wt;
    g.b1 = c->w + l1.b_off;
    g.b2 = c->w + l2.b_off;
    g.M = c->E;
    g.Z = z;
    g.Eout = e0;
    launch_edge_encoder(g, c->st);
}

// grad of W (kin x kout) += X^T dY over M rows (X: M x kin with stride ldx,
// dY: M x kout with stride ldy); kin = 16 layers are computed as (dY^T X)^T.
void wgrad(sur_ctx* c, const Layer& l, const __nv_bfloat16* X, uint32_t ldx,
           const __nv_bfloat16* dY, uint32_t ldy, uint32_t M, int kin_half = -1) {
    WgradArgs g = {};
    g.M = M;
    g.partial = c->partial;
    g.nparts = kWgradParts;
    g.scale = 1.f;
    float* dst = c->g + l.w_off;
    if (l.kin == KIN) {
        // D[128 x 16] = dY^T X = (dW)^T, then transposed into dW (16 x 128)
        g.X = dY;
        g.ldp = ldy;
        g.dY = X;
        g.ldq = ldx;
        g.dW = c->wg_tmp;
        launch_wgrad(KIN, g, c->st);
        k_transpose<<<nblk((size_t)KIN * L, 256), 256, 0, c->st>>>(c->wg_tmp, L, KIN, dst);
        return;
    }
    g.X = X;
    g.ldp = ldx;
    g.dY = dY;
    g.ldq = ldy;
    g.dW = dst + (kin_half > 0 ? (size_t)kin_half * L * l.kout : 0);
    launch_wgrad(l.kout, g, c->st);
}

}  // namespace

namespace {

void colsum(sur_ctx* c, const void* in, bool bf16, uint32_t M, int C, uint32_t ld, float* out) {
    const uint32_t parts = M == 0 ? 1u : (M < 1024u ? M : 1024u);
    if (bf16)
        k_colsum_part<__nv_bfloat16><<<parts, C, 0, c->st>>>(M, C, (const __nv_bfloat16*)in, ld, c->colpart);
    else
        k_colsum_part<float><<<parts, C, 0, c->st>>>(M, C, (const float*)in, ld, c->colpart);
    k_colsum_final<<<1, C, 0, c->st>>>((int)parts, C, c->colpart, out, 1.f);
}

void cast(sur_ctx* c, const float* in, __nv_bfloat16* out, size_t n) {
    k_cast_bf16<<<gridcap(n, 256), 256, 0, c->st>>>(in, out, n);
}

void refresh_all(sur_ctx* c) {
    for (Layer& l : c->layers)
        k_refresh<<<nblk((size_t)l.kin * l.kout, 256), 256, 0, c->st>>>(c->w + l.w_off, l.kin, l.kout,
                                                                        l.W, l.Wt);
}

// dst (n x 128, stride 128) += src (n x 128, stride lds)
__global__ void k_add_strided(uint32_t n, float* __restrict__ dst, const float* __restrict__ src,
                              uint32_t lds) {
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t >= (size_t)n * L) return;
    const size_t i = t / L, c = t % L;
    dst[t] += src[i * lds + c];
}

int check(sur_ctx* c, const char* what) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        c->err = std::string(what) + ": " + cudaGetErrorString(e);
        return SPH_ERR_CUDA;
    }
    return SPH_OK;
}

int forward(sur_ctx* c, sph_ctx* s, const float* hist) {
    if (!s->cells_valid) return fail(c, SPH_ERR_STATE, "SPH cells not built");
    if (!s->ids_dense) return fail(c, SPH_ERR_STATE, "by-id arrays need every id below n");
    if (s->n > c->cfg.max_nodes) return fail(c, SPH_ERR_INVALID_ARG, "more particles than max_nodes");
    const uint32_t n = s->n;
    c->n = n;
    cudaStream_t st = c->st;
    const sph::Dev& d = s->d;
    const int cur = s->cur;
    const double inv2h = 1.0 / (2.0 * s->p.h);
    // the SPH predicate's (2h)^2 itself, or (radius 2h)^2 rounded once
    const float rad = c->cfg.radius;
    const double r2 = (rad > 0.f && rad < 1.f)
                          ? ((double)rad * (2.0 * s->p.h)) * ((double)rad * (2.0 * s->p.h))
                          : s->d.r2max_d;
    const uint32_t* key = s->key[s->skey];
    // the FP32 decision margins of k_graph (FP64 for every candidate below
    // a tenth of a cell)
    const bool fp32_ok = r2 >= 0.01 * (2.0 * s->p.h) * (2.0 * s->p.h);
    const float inside = fp32_ok ? (float)r2 * (1.0f - 0x1p-12f) : -1.0f;
    const float outside = fp32_ok ? (float)r2 * (1.0f + 0x1p-12f) : INFINITY;
    k_graph<0><<<nblk(n, 128), 128, 0, st>>>(d, s->x[cur], s->y[cur], s->z[cur], s->posc, key,
                                             s->off, c->cnt, nullptr, nullptr, nullptr, nullptr,
                                             inv2h, r2, inside, outside);
    sph::launch_scan(c->cnt, n, c->bsum, c->rowptr, st);
    uint32_t E = 0;
    cudaMemcpyAsync(&E, c->rowptr + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return check(c, "graph count");
    if (E > c->cfg.max_edges) return fail(c, SPH_ERR_CAPACITY, "more edges than max_edges");
    c->E = E;
    k_graph<1><<<nblk(n, 128), 128, 0, st>>>(d, s->x[cur], s->y[cur], s->z[cur], s->posc, key,
                                             s->off, nullptr, c->rowptr, c->col, c->src, c->xe,
                                             inv2h, r2, inside, outside);
    if (c->cfg.train && E) k_graph_rev<<<nblk(E, 256), 256, 0, st>>>(E, c->rowptr, c->col, c->src, c->rev);
    k_node_features<<<nblk(n, 256), 256, 0, st>>>(d, s->id[cur], hist, 1.0 / (double)c->cfg.v_scale, c->xn);
    const std::vector<Layer>& Ls = c->layers;
    const bool train = c->cfg.train != 0;
    int rc;
    // encoders
    if ((rc = linear(c, c->xn, 0, Ls[0], false, n, kEpiRelu, nullptr, 0, c->en1, nullptr, L))) return rc;
    if ((rc = linear(c, c->en1, 0, Ls[1], false, n, kEpiNone, nullptr, 0, c->XN[0], nullptr, 2 * L))) return rc;
    edge_encoder(c, Ls[2], Ls[3], train ? c->ee1 : nullptr, c->Ebuf[0]);
    // message passing
    for (int l = 0; l < c->NL; ++l) {
        __nv_bfloat16* xn_cur = c->XN[train ? l : l % 2];
        __nv_bfloat16* xn_next = c->XN[train ? l + 1 : (l + 1) % 2];
        __nv_bfloat16* e_in = c->Ebuf[train ? l : l % 2];
        __nv_bfloat16* e_out = c->Ebuf[train ? l + 1 : (l + 1) % 2];
        __nv_bfloat16* z1 = train ? c->Z1[l] : nullptr;
        __nv_bfloat16* y1 = c->Y1[train ? l : 0];
        const Layer* w = &Ls[4 + 6 * l];
        if ((rc = linear(c, xn_cur, 2 * L, w[0], false, n, kEpiNone, nullptr, 0, c->P, nullptr, L))) return rc;
        if ((rc = linear(c, xn_cur, 2 * L, w[1], false, n, kEpiNone, nullptr, 0, c->Q, nullptr, L))) return rc;
        edge_layer(c, w[2], w[3], e_in, train ? z1 : nullptr, e_out);
        k_rowsum<__nv_bfloat16><<<nblk((size_t)n * 32, 256), 256, 0, st>>>(n, c->rowptr, e_out, nullptr,
                                                                           xn_cur + L, nullptr, 2 * L);
        if ((rc = linear(c, xn_cur, 0, w[4], false, n, kEpiRelu, nullptr, 0, y1, nullptr, L))) return rc;
        if ((rc = linear(c, y1, 0, w[5], false, n, kEpiResidual, xn_cur, 2 * L, xn_next, nullptr, 2 * L)))
            return rc;
    }
    __nv_bfloat16* h_last = c->XN[train ? c->NL : c->NL % 2];
    const Layer* dec = &Ls[4 + 6 * c->NL];
    if ((rc = linear(c, h_last, 2 * L, dec[0], false, n, kEpiRelu, nullptr, 0, c->D1, nullptr, L))) return rc;
    if ((rc = linear(c, c->D1, 0, dec[1], false, n, kEpiNone, nullptr, 0, nullptr, c->out, KOUT))) return rc;
    c->have_forward = true;
    return check(c, "sur_forward");
}

int backward(sur_ctx* c, sph_ctx* s, const float* target, float* loss_host) {
    if (!c->cfg.train) return fail(c, SPH_ERR_STATE, "context not created for training");
    if (!c->have_forward) return fail(c, SPH_ERR_STATE, "no forward pass to differentiate");
    cudaStream_t st = c->st;
    const uint32_t n = c->n, E = c->E;
    const std::vector<Layer>& Ls = c->layers;
    const sph::Dev& d = s->d;
    const int cur = s->cur;
    // fluid count for the mean
    uint32_t nf = 0;
    {
        // count fluid in-domain particles on the host side from the tables
        uint32_t n_in = 0;
        cudaMemcpyAsync(&n_in, s->off + s->tab.ncells, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        uint64_t nb = 0;
        for (size_t q = 0; q < s->tab.inst.size(); ++q) nb += s->tab.inst[q].id_fluid - s->tab.inst[q].id_base;
        nf = n_in > nb ? (uint32_t)(n_in - nb) : 1u;
    }
    const float inv_nf = 1.f / (float)nf;
    cudaMemsetAsync(c->g, 0, c->nparams * sizeof(float), st);
    const uint32_t lb = nblk(n, 256);
    k_loss<<<lb, 256, 0, st>>>(d, s->id[cur], c->out, target, s->off, inv_nf, c->dout, c->losspart);
    k_loss_final<<<1, 32, 0, st>>>((int)lb, c->losspart, inv_nf, c->loss);
    int rc;
    // decoder
    const Layer* dec = &Ls[4 + 6 * c->NL];
    __nv_bfloat16* h_last = c->XN[c->NL];
    colsum(c, c->dout, true, n, KOUT, KOUT, c->g + dec[1].b_off);
    wgrad(c, dec[1], c->D1, L, c->dout, KOUT, n);
    if ((rc = linear(c, c->dout, 0, dec[1], true, n, kEpiReluMask, c->D1, L, c->dD1, nullptr, L))) return rc;
    colsum(c, c->dD1, true, n, L, L, c->g + dec[0].b_off);
    wgrad(c, dec[0], h_last, 2 * L, c->dD1, L, n);
    if ((rc = linear(c, c->dD1, 0, dec[0], true, n, kEpiNone, nullptr, 0, nullptr, c->dH, L))) return rc;
    cudaMemsetAsync(c->dE, 0, (size_t)E * L * sizeof(float), st);
    for (int l = c->NL - 1; l >= 0; --l) {
        const Layer* w = &Ls[4 + 6 * l];
        __nv_bfloat16* xn_cur = c->XN[l];
        __nv_bfloat16* e_in = c->Ebuf[l];
        __nv_bfloat16* z1 = c->Z1[l];
        __nv_bfloat16* y1 = c->Y1[l];
        // node update h' = h + W4 relu(W3 [h, agg] + b3) + b4
        cast(c, c->dH, c->dHb, (size_t)n * L);
        colsum(c, c->dH, false, n, L, L, c->g + w[5].b_off);
        wgrad(c, w[5], y1, L, c->dHb, L, n);
        if ((rc = linear(c, c->dHb, 0, w[5], true, n, kEpiReluMask, y1, L, c->dY1, nullptr, L))) return rc;
        colsum(c, c->dY1, true, n, L, L, c->g + w[4].b_off);
        wgrad(c, w[4], xn_cur, 2 * L, c->dY1, L, n, 0);
        wgrad(c, w[4], xn_cur + L, 2 * L, c->dY1, L, n, 1);
        if ((rc = linear(c, c->dY1, 0, w[4], true, n, kEpiNone, nullptr, 0, nullptr, c->dXN, 2 * L))) return rc;
        k_add_strided<<<nblk((size_t)n * L, 256), 256, 0, st>>>(n, c->dH, c->dXN, 2 * L);
        // aggregation and edge update e' = e + W2 relu(pre) + b2
        k_add_gather<<<gridcap((size_t)E * L, 256), 256, 0, st>>>((size_t)E * L, c->dE, c->dXN + L,
                                                                  c->src, 2 * L, c->dEb);
        colsum(c, c->dE, false, E, L, L, c->g + w[3].b_off);
        wgrad(c, w[3], z1, L, c->dEb, L, E);
        if ((rc = linear(c, c->dEb, 0, w[3], true, E, kEpiReluMask, z1, L, c->dpre, nullptr, L))) return rc;
        colsum(c, c->dpre, true, E, L, L, c->g + w[2].b_off);
        wgrad(c, w[2], e_in, L, c->dpre, L, E);
        if ((rc = linear(c, c->dpre, 0, w[2], true, E, kEpiAccum, nullptr, 0, nullptr, c->dE, L))) return rc;
        // pre = W1a h_i + W1b h_j + ...: sums over the edges of i and of j
        k_rowsum<__nv_bfloat16><<<nblk((size_t)n * 32, 256), 256, 0, st>>>(n, c->rowptr, c->dpre, nullptr,
                                                                           c->dPb, nullptr, L);
        k_rowsum<__nv_bfloat16><<<nblk((size_t)n * 32, 256), 256, 0, st>>>(n, c->rowptr, c->dpre, c->rev,
                                                                           c->dQb, nullptr, L);
        wgrad(c, w[0], xn_cur, 2 * L, c->dPb, L, n);
        wgrad(c, w[1], xn_cur, 2 * L, c->dQb, L, n);
        if ((rc = linear(c, c->dPb, 0, w[0], true, n, kEpiAccum, nullptr, 0, nullptr, c->dH, L))) return rc;
        if ((rc = linear(c, c->dQb, 0, w[1], true, n, kEpiAccum, nullptr, 0, nullptr, c->dH, L))) return rc;
    }
    // encoders
    cast(c, c->dE, c->dEb, (size_t)E * L);
    colsum(c, c->dE, false, E, L, L, c->g + Ls[3].b_off);
    wgrad(c, Ls[3], c->ee1, L, c->dEb, L, E);
    if ((rc = linear(c, c->dEb, 0, Ls[3], true, E, kEpiReluMask, c->ee1, L, c->dEe1, nullptr, L))) return rc;
    colsum(c, c->dEe1, true, E, L, L, c->g + Ls[2].b_off);
    wgrad(c, Ls[2], c->xe, KIN, c->dEe1, L, E);
    cast(c, c->dH, c->dHb, (size_t)n * L);
    colsum(c, c->dH, false, n, L, L, c->g + Ls[1].b_off);
    wgrad(c, Ls[1], c->en1, L, c->dHb, L, n);
    if ((rc = linear(c, c->dHb, 0, Ls[1], true, n, kEpiReluMask, c->en1, L, c->dEn1, nullptr, L))) return rc;
    colsum(c, c->dEn1, true, n, L, L, c->g + Ls[0].b_off);
    wgrad(c, Ls[0], c->xn, KIN, c->dEn1, L, n);
    if (loss_host) {
        cudaMemcpyAsync(loss_host, c->loss, sizeof(float), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) return check(c, "sur_backward");
    }
    return check(c, "sur_backward");
}

}  // namespace

extern "C" {

uint64_t sur_param_count(const sur_config* cfg) {
    if (!cfg) return 0;
    sur_ctx tmp;
    tmp.NL = (int)cfg->layers;
    build_layers(&tmp);
    return tmp.nparams;
}

uint64_t sur_query_bytes(const sur_config* cfg) {
    if (!cfg || cfg->layers == 0 || cfg->max_nodes == 0) return 0;
    sur_ctx tmp;
    tmp.cfg = *cfg;
    tmp.NL = (int)cfg->layers;
    build_layers(&tmp);
    return carve(&tmp, nullptr);
}

int sur_init(const sur_config* cfg, void* ws, uint64_t bytes, void* stream, sur_ctx** out) {
    if (!cfg || !out || !ws || cfg->layers == 0 || cfg->layers > 64 || cfg->max_nodes == 0 ||
        !(cfg->v_scale > 0.f) || !(cfg->radius >= 0.f && cfg->radius <= 1.f) ||
        ((uintptr_t)ws % 256) != 0)
        return SPH_ERR_INVALID_ARG;
    sur_ctx* c = new sur_ctx();
    c->cfg = *cfg;
    c->NL = (int)cfg->layers;
    c->st = (cudaStream_t)stream;
    build_layers(c);
    if (carve(c, ws) > bytes) {
        delete c;
        return SPH_ERR_WORKSPACE;
    }
    cudaMemsetAsync(c->w, 0, 4 * c->nparams * sizeof(float), c->st);
    refresh_all(c);
    if (cudaStreamSynchronize(c->st) != cudaSuccess) {
        delete c;
        return SPH_ERR_CUDA;
    }
    *out = c;
    return SPH_OK;
}

int sur_set_params(sur_ctx* c, const float* host, uint64_t count) {
    if (!c || !host || count != c->nparams) return SPH_ERR_INVALID_ARG;
    cudaMemcpyAsync(c->w, host, count * sizeof(float), cudaMemcpyHostToDevice, c->st);
    cudaMemsetAsync(c->m, 0, count * sizeof(float), c->st);
    cudaMemsetAsync(c->v, 0, count * sizeof(float), c->st);
    c->adam_t = 0;
    refresh_all(c);
    return cudaStreamSynchronize(c->st) == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}

int sur_get_params(sur_ctx* c, float* host, uint64_t count) {
    if (!c || !host || count != c->nparams) return SPH_ERR_INVALID_ARG;
    cudaMemcpyAsync(host, c->w, count * sizeof(float), cudaMemcpyDeviceToHost, c->st);
    return cudaStreamSynchronize(c->st) == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}

int sur_get_grads(sur_ctx* c, float* host, uint64_t count) {
    if (!c || !host || count != c->nparams) return SPH_ERR_INVALID_ARG;
    cudaMemcpyAsync(host, c->g, count * sizeof(float), cudaMemcpyDeviceToHost, c->st);
    return cudaStreamSynchronize(c->st) == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}

int sur_forward(sur_ctx* c, sph_ctx* s, const float* d_hist, float* d_acc) {
    if (!c || !s || !d_hist) return SPH_ERR_INVALID_ARG;
    int rc = forward(c, s, d_hist);
    if (rc) return rc;
    const float3 am = make_float3(c->cfg.a_mean[0], c->cfg.a_mean[1], c->cfg.a_mean[2]);
    const float3 as = make_float3(c->cfg.a_std[0], c->cfg.a_std[1], c->cfg.a_std[2]);
    if (d_acc)
        k_write_out<<<nblk(s->n, 256), 256, 0, c->st>>>(s->d, s->id[s->cur], c->out, am, as, d_acc);
    return check(c, "sur_forward");
}

int sur_backward(sur_ctx* c, sph_ctx* s, const float* d_target, float* loss) {
    if (!c || !s || !d_target) return SPH_ERR_INVALID_ARG;
    return backward(c, s, d_target, loss);
}

int sur_adam(sur_ctx* c, float lr, float beta1, float beta2, float eps) {
    if (!c) return SPH_ERR_INVALID_ARG;
    c->adam_t += 1;
    const float c1 = 1.f - powf(beta1, (float)c->adam_t);
    const float c2 = 1.f - powf(beta2, (float)c->adam_t);
    k_adam<<<gridcap(c->nparams, 256), 256, 0, c->st>>>(c->nparams, c->w, c->g, c->m, c->v, lr, beta1,
                                                        beta2, eps, c1, c2);
    refresh_all(c);
    return check(c, "sur_adam");
}

int sur_advance(sur_ctx* c, sph_ctx* s, float* d_hist) {
    if (!c || !s || !d_hist) return SPH_ERR_INVALID_ARG;
    int rc = forward(c, s, d_hist);
    if (rc) return rc;
    const float3 am = make_float3(c->cfg.a_mean[0], c->cfg.a_mean[1], c->cfg.a_mean[2]);
    const float3 as = make_float3(c->cfg.a_std[0], c->cfg.a_std[1], c->cfg.a_std[2]);
    const int cur = s->cur;
    k_write_out<<<nblk(s->n, 256), 256, 0, c->st>>>(s->d, s->id[cur], c->out, am, as, c->acc);
    k_advance<<<nblk(s->n, 256), 256, 0, c->st>>>(s->d, s->id[cur], s->x[cur], s->y[cur], s->z[cur],
                                                  s->vr[cur], s->off, c->acc, d_hist, c->cfg.dt_s);
    s->cells_valid = false;
    sph::drop_pending_counts(s, c->st);
    s->pre_state = 0;
    // a Verlet context has no earlier state for the surrogate's result: its
    // next SPH step is an Euler step
    cudaMemsetAsync(s->i_vphase, 0, s->n_inst * sizeof(uint32_t), c->st);
    return check(c, "sur_advance");
}

int sur_make_sample(sur_ctx* c, sph_ctx* s, const double* d_frames, double sigma,
                    uint64_t seed, double* d_pos, float* d_vel, float* d_hist, float* d_target) {
    if (!c || !s || !d_frames || !d_pos || !d_vel || !d_hist || !d_target || !(sigma >= 0.0) ||
        !(c->cfg.dt_s > 0.f))
        return SPH_ERR_INVALID_ARG;
    if (s->n > c->cfg.max_nodes) return fail(c, SPH_ERR_INVALID_ARG, "more particles than max_nodes");
    const float3 am = make_float3(c->cfg.a_mean[0], c->cfg.a_mean[1], c->cfg.a_mean[2]);
    const float3 as = make_float3(c->cfg.a_std[0], c->cfg.a_std[1], c->cfg.a_std[2]);
    k_make_sample<<<nblk(s->n, 256), 256, 0, c->st>>>(s->d, d_frames, s->n, sigma, seed,
                                                      (double)c->cfg.dt_s, am, as, d_pos, d_vel,
                                                      d_hist, d_target);
    return check(c, "sur_make_sample");
}

int sur_rollout(sur_ctx* c, sph_ctx* s, float* d_hist, uint32_t ncalls, uint32_t save_every,
                sph_snapshot_fn cb, void* user) {
    if (!c || !s || !d_hist) return SPH_ERR_INVALID_ARG;
    if (!(c->cfg.dt_s > 0.f)) return fail(c, SPH_ERR_INVALID_ARG, "dt_s must be positive");
    if (save_every == 0) save_every = ncalls ? ncalls : 1;
    double t = 0.0;
    for (uint32_t k = 1; k <= ncalls; ++k) {
        if (!s->cells_valid) {
            const int rc = sph_build_cells(s);
            if (rc) return fail(c, rc, "cell rebuild failed");
        }
        const int rc = sur_advance(c, s, d_hist);
        if (rc) return rc;
        t += (double)c->cfg.dt_s;
        if (cb && (k % save_every == 0 || k == ncalls)) {
            if (cudaStreamSynchronize(c->st) != cudaSuccess) return check(c, "sur_rollout");
            if (cb(user, k, t)) break;
        }
    }
    const int rc = sph_build_cells(s);
    if (rc) return fail(c, rc, "cell rebuild failed");
    return check(c, "sur_rollout");
}

uint32_t sur_num_edges(const sur_ctx* c) { return c ? c->E : 0; }

int sur_read_graph(sur_ctx* c, uint32_t* rowptr, uint32_t* col) {
    if (!c || !rowptr || !col) return SPH_ERR_INVALID_ARG;
    if (!c->have_forward) {
        c->err = "no graph yet (call sur_forward first)";
        return SPH_ERR_STATE;
    }
    cudaError_t e = cudaMemcpyAsync(rowptr, c->rowptr, ((size_t)c->n + 1) * sizeof(uint32_t),
                                    cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess && c->E)
        e = cudaMemcpyAsync(col, c->col, (size_t)c->E * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                            c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) {
        c->err = std::string("read graph: ") + cudaGetErrorString(e);
        return SPH_ERR_CUDA;
    }
    return SPH_OK;
}

const char* sur_last_error(const sur_ctx* c) { return c ? c->err.c_str() : "NULL context"; }

void sur_destroy(sur_ctx* c) { delete c; }

}  // extern "C"
