// Per-step kernels of the weakly compressible SPH hot path on sm_103a:
// cell labels, reorder with the id tie-break, the 27-cell pair interaction
// (Eqs. 7 and 9 with the Tait law and artificial viscosity of Sec. 2.2),
// the CFL reductions (Sec. 3.3), the symplectic predictor/corrector, FP64
// neighbour counts and FP64 conservation sums.  Every kernel serves an
// ensemble of independent instances (see sph_internal.cuh); a single
// simulation is the ensemble of one.
#include <cuda_fp16.h>
#include <math.h>
#include <stdlib.h>

#include <mutex>

#include "sph_internal.cuh"

namespace sph {

namespace {

constexpr uint32_t kFull = 0xffffffffu;

__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Index q with base[q] <= v < base[q + 1] (base has n + 1 ascending entries).
__device__ __forceinline__ uint32_t find_instance(const uint32_t* __restrict__ base, uint32_t n,
                                                  uint32_t v) {
    uint32_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(base + mid) <= v) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Sec. 3.1 cell label: floor((x - x0) * (1/(2h))) per axis in FP64, each
// operation rounded as written; label = cell_base + cx + ncx (cy + ncy cz)
// in the particle's instance.  Outside its grid (or non-finite) -> ncells.
__device__ __forceinline__ uint32_t cell_key(const Dev& d, const Inst& I, double x, double y,
                                             double z) {
    const double tx = __dmul_rn(__dsub_rn(x, I.x0), d.inv_cs);
    const double ty = __dmul_rn(__dsub_rn(y, I.y0), d.inv_cs);
    const double tz = __dmul_rn(__dsub_rn(z, I.z0), d.inv_cs);
    // t in [0, nc) <=> floor(t) in [0, nc) for finite t (the conversion
    // saturates far outside); infinities and NaNs (exponent all ones) are
    // out.  The range test thus runs on integers, not on the FP64 pipe.
    const bool finite = ((uint32_t)__double2hiint(tx) & 0x7ff00000u) != 0x7ff00000u &&
                        ((uint32_t)__double2hiint(ty) & 0x7ff00000u) != 0x7ff00000u &&
                        ((uint32_t)__double2hiint(tz) & 0x7ff00000u) != 0x7ff00000u;
    const int cx = __double2int_rd(tx), cy = __double2int_rd(ty), cz = __double2int_rd(tz);
    const bool in = finite && cx >= 0 && cx < I.ncx && cy >= 0 && cy < I.ncy && cz >= 0 &&
                    cz < I.ncz;
    if (!in) return d.ncells;
    return I.cell_base + (uint32_t)cx +
           (uint32_t)I.ncx * ((uint32_t)cy + (uint32_t)I.ncy * (uint32_t)cz);
}

__host__ __device__ __forceinline__ uint32_t digit_mask(int pass, int bits_total) {
    int b = bits_total - 8 * pass;
    b = b > 8 ? 8 : (b < 0 ? 0 : b);
    return (1u << b) - 1u;
}

// Count a label into the per-cell histogram (one atomic per distinct label
// in the warp) and into the block's digit histograms of the radix sort.
__device__ __forceinline__ void count_key(bool valid, uint32_t key, uint32_t* cnt,
                                          uint32_t* s_hist, int passes, int bits) {
    const uint32_t act = __ballot_sync(kFull, valid);
    if (valid) {
        const uint32_t peers = __match_any_sync(act, key);
        if ((threadIdx.x & 31) == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&cnt[key], __popc(peers));
        for (int p = 0; p < passes; ++p)
            atomicAdd(&s_hist[p * 256 + ((key >> (8 * p)) & digit_mask(p, bits))], 1u);
    }
}

__device__ __forceinline__ void flush_hist(uint32_t* s_hist, uint32_t* hist, int passes) {
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += blockDim.x)
        if (s_hist[i]) atomicAdd(&hist[i], s_hist[i]);
}

__device__ __forceinline__ void zero_hist(uint32_t* s_hist) {
    for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) s_hist[i] = 0;
    __syncthreads();
}

__device__ __forceinline__ int bits_for(uint32_t ncells) {
    return 32 - __clz(ncells);   // labels run 0..ncells
}

__global__ void __launch_bounds__(256) k_keys(const Dev d, const double* __restrict__ x,
                                              const double* __restrict__ y,
                                              const double* __restrict__ z,
                                              const uint32_t* __restrict__ id, uint32_t n,
                                              uint32_t* __restrict__ key, uint32_t* cnt,
                                              uint32_t* hist, int passes) {
    __shared__ uint32_t s_hist[4 * 256];
    zero_hist(s_hist);
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < n;
    uint32_t k = 0;
    if (valid) {
        const uint32_t q = find_instance(d.id_base, d.n_inst, id[i]);
        k = cell_key(d, d.inst[q], x[i], y[i], z[i]);
        key[i] = k;
    }
    count_key(valid, k, cnt, s_hist, passes, bits_for(d.ncells));
    flush_hist(s_hist, hist, passes);
}

// Tait pressure over density squared, P = B [(rho/rho0)^7 - 1] / rho^2, in
// FP32.  (rho/rho0)^7 - 1 is expanded in x = (rho - rho0)/rho0 so that it
// keeps its relative accuracy near the free surface, where it cancels.
__device__ __forceinline__ float p_over_rho2(const Dev& d, float B, float rho) {
    const float x = (rho - d.rho0) * d.inv_rho0;
    const float poly =
        x * (7.f + x * (21.f + x * (35.f + x * (35.f + x * (21.f + x * (7.f + x))))));
    return B * poly / (rho * rho);
}

constexpr uint32_t kMaxSeg = 4096;   // largest cell the id tie-break handles

// Sec. 3.1 reorder.  Thread k takes the k-th pair of the cell sort (grouped
// by cell, any order inside a cell), ranks its particle by id among the
// particles of the same cell, and moves the particle's state to (cell start
// + rank): the result is ordered by (label, id) whatever the order inside
// the cells was.  Also writes the FP32 position relative to the cell's
// origin and P = p/rho^2.
__global__ void __launch_bounds__(256) k_reorder(const Dev d, const ReorderArgs a) {
    pdl_wait();
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool valid = k < d.n;
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) a.hist_to_zero[i] = 0;
    uint32_t c = 0, v = 0, myid = 0, s = 0, e = 0;
    if (valid) {
        c = a.skey[k];
        v = a.sval[k];
        if (!in_bounds(c <= d.ncells && v < d.n, d.status)) {
            c = d.ncells;
            v = k;
        }
        myid = a.sid[v];
        s = a.off[c];
        e = a.off[c + 1];
    }
    const bool big = (e - s) > kMaxSeg;
    const uint32_t wbase = k - lane;
    uint32_t rank = 0;
#pragma unroll 8
    for (int t = 0; t < 32; ++t) {
        const uint32_t oid = __shfl_sync(kFull, myid, t);
        const uint32_t j = wbase + t;
        if (j >= s && j < e && oid < myid) ++rank;
    }
    if (valid && !big && e - s > 1) {
        const uint32_t lo_end = e < wbase ? e : wbase;
        for (uint32_t j = s; j < lo_end; ++j) rank += a.sid[a.sval[j]] < myid;
        for (uint32_t j = (s > wbase + 32 ? s : wbase + 32); j < e; ++j)
            rank += a.sid[a.sval[j]] < myid;
    }
    if (!valid) return;
    if (big) {
        rank = k - s;
        atomicOr(a.status, kStatusCapacity);
    }
    const uint32_t dst = s + rank;
    if (!in_bounds(dst < d.n, d.status)) return;
    const double x = a.sx[v], y = a.sy[v], z = a.sz[v];
    const float4 vr = a.svr[v];
    a.dx[dst] = x;
    a.dy[dst] = y;
    a.dz[dst] = z;
    a.dvr[dst] = vr;
    a.did[dst] = myid;
    if (a.spx) {
        a.dpx[dst] = a.spx[v];
        a.dpy[dst] = a.spy[v];
        a.dpz[dst] = a.spz[v];
    }
    if (a.spvr) a.dpvr[dst] = a.spvr[v];
    float4 pc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (c < d.ncells) {
        const Inst& I = d.inst[find_instance(d.cell_base, d.n_inst, c)];
        const uint32_t lc = c - I.cell_base;
        const uint32_t cx = lc % (uint32_t)I.ncx;
        const uint32_t t = lc / (uint32_t)I.ncx;
        const uint32_t cy = t % (uint32_t)I.ncy;
        const uint32_t cz = t / (uint32_t)I.ncy;
        pc.x = __double2float_rn(x - (I.x0 + (double)cx * d.cs));
        pc.y = __double2float_rn(y - (I.y0 + (double)cy * d.cs));
        pc.z = __double2float_rn(z - (I.z0 + (double)cz * d.cs));
        pc.w = p_over_rho2(d, I.B, vr.w);
    }
    a.posc[dst] = pc;
}

// ----------------------------------------------------------- interaction --

constexpr uint32_t kIdxMask = (1u << 26) - 1;
constexpr uint32_t kWaitLimit = 1u << 22;

// Shape of one interaction variant: W warps per block (units of W*32
// particles), STAGE staged candidates, WCAP hit-mask words per lane.  Dynamic
// shared memory: staged posc and velrhop (STAGE float4 each), the staged
// positions in half precision (one uint4 of three half2 per candidate pair),
// then per warp WCAP x 32 hit-mask words and WCAP word descriptors.  The
// global-memory fallback keeps 32-bit lists of kFallbackCap entries per lane
// in the staging area.
constexpr int kFallbackCap = 64;   // at most; fewer when the staging area is small

template <int W, int STAGE, int WCAP>
struct Shape {
    static constexpr size_t stage_bytes = (size_t)STAGE * 2 * sizeof(float4);
    static constexpr int fb_cap =
        stage_bytes / ((size_t)W * 32 * sizeof(uint32_t)) < (size_t)kFallbackCap
            ? (int)(stage_bytes / ((size_t)W * 32 * sizeof(uint32_t)))
            : kFallbackCap;
    static constexpr size_t half_bytes = (size_t)STAGE / 2 * sizeof(uint4);
    static constexpr size_t word_bytes = (size_t)W * WCAP * 32 * sizeof(uint32_t);
    static constexpr size_t smem = stage_bytes + half_bytes + word_bytes +
                                   (size_t)W * WCAP * sizeof(uint32_t);
    static_assert(fb_cap >= 16 && (size_t)W * fb_cap * 32 * sizeof(uint32_t) <= stage_bytes,
                  "fallback lists must fit in the staging area");
    static_assert(STAGE <= (1 << 16) && STAGE % 2 == 0, "staged index must fit 16 bits");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// 1-D bulk copy global -> shared (TMA engine), completion counted on bar.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}" : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of bar; false if it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    for (uint32_t k = 0; k < kWaitLimit; ++k)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

struct PairAcc {
    float ax, ay, az, dr, mu;
    float npf;       // pairs counted by the FP32 test (exact below 2^24)
    uint32_t np;
};

// The sign bits (15 and 31) of a and of b, each spread over one byte of the
// result (0xff if set): byte 0 <- a bit 15, 1 <- a bit 31, 2 <- b bit 15,
// 3 <- b bit 31 (prmt selects a byte and, with the selector's high bit,
// replicates that byte's sign bit).
__device__ __forceinline__ uint32_t sign_bytes(uint32_t a, uint32_t b) {
    uint32_t r;
    asm("prmt.b32 %0, %1, %2, 0xFDB9;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}

// Hit-mask bits of the slots [0, lim) of a 32-candidate word (slot s at
// bit 8 (s mod 4) + s / 4), for lim = 0 .. 32.
struct KeepTable {
    uint32_t v[33];
};
constexpr KeepTable make_keep_table() {
    KeepTable t{};
    for (int lim = 0; lim <= 32; ++lim) {
        uint32_t k = 0;
        for (int sl = 0; sl < lim; ++sl) k |= 1u << (8 * (sl & 3) + (sl >> 2));
        t.v[lim] = k;
    }
    return t;
}
__constant__ KeepTable c_keep = make_keep_table();

// Pair terms of Eqs. 7 and 9 for i (pi, vi) and j (pj, vj) at offset
// (dx, dy, dz) = r_i - r_j.  MOM: evaluate the momentum terms (a warp-uniform
// choice).  They are accumulated for every particle; the caller keeps them
// only for fluid particles, since boundary particles never move (Sec. 2.3).
// A pair with v_ij = 0 whose offset lies outside the support (the particle
// itself, placed 4 cells away) contributes exactly nothing and is not
// counted, which lets lane work be padded with it.  Masks are products with
// 0 or 1 rather than selects, keeping the integer/logic pipe free.
// KERN: 0 Wendland C2, 1 cubic spline (Sec. 2.2).
template <int KERN, bool MOM, bool CHECK = false>
__device__ __forceinline__ void pair_terms(const Dev& d, float c0, const float4& pi,
                                           const float4& vi, float ci, float dx, float dy, float dz,
                                           const float4& pj, const float4& vj, PairAcc& s) {
    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    // CHECK: the entry came from the conservative half-precision pre-filter;
    // the FP32 neighbour test (the same predicate as the candidate test of the
    // global-memory path) decides and counts the pair: use = [d2 < (2h)^2],
    // the saturated sign of 2^100 ((2h)^2 - d2), exact (power-of-two scaling)
    const float use = CHECK ? __saturatef(fmaf(d2, -0x1p100f, d.r2max * 0x1p100f)) : 1.f;
    if (CHECK) s.npf += use;
    // grad_i W = F r_ij.  Wendland C2: F = -5 aD/h^2 (1 - q/2)^3.  Cubic
    // spline: F = aD/h^2 (9/4 q - 3) for q < 1, -3/4 aD/h^2 (2 - q)^2 / q
    // for 1 <= q < 2 (a select: the outer piece is infinite at q = 0).
    const float q = sqrt_approx(d2) * d.inv_h;
    float shape;
    if (KERN == 1) {
        const float wo = 2.0f - q;
        const float outer = -0.75f * (wo * wo) * rcp_approx(q);
        const float inner = fmaf(2.25f, q, -3.0f);
        shape = q < 1.0f ? inner : outer;
    } else {
        const float wq = fmaf(-0.5f, q, 1.0f);
        shape = wq * wq * wq;
    }
    const float F = CHECK ? d.fc * shape * use : d.fc * shape;
    const float dvx = vi.x - vj.x, dvy = vi.y - vj.y, dvz = vi.z - vj.z;
    const float vr = fmaf(dvx, dx, fmaf(dvy, dy, dvz * dz));
    s.dr = fmaf(vr, F, s.dr);                                      // Eq. 7
    if (MOM) {
        const float nu = d.h * vr * rcp_approx(d2 + d.eta2);       // Sec. 2.2
        const float rrj = vj.w * d.inv_rho0;
        const float cj = c0 * rrj * rrj * rrj;
        // Pi_ij only for approaching pairs (v_ij . r_ij < 0, the sign of nu)
        const float visc = -d.alpha * (ci + cj) * fminf(nu, 0.f) * rcp_approx(vi.w + vj.w);
        const float f = (pi.w + pj.w + visc) * F;                  // Eq. 9
        s.ax = fmaf(-f, dx, s.ax);
        s.ay = fmaf(-f, dy, s.ay);
        s.az = fmaf(-f, dz, s.az);
        s.mu = fmaxf(s.mu, CHECK ? fabsf(nu) * use : fabsf(nu));
    }
}

// Sec. 3.3 reductions, by one block once every interaction block has
// published its counters (pairs, candidates, status bits) and atomically
// raised the per-instance maxima: the counters are summed (integer sums and
// maxima do not depend on the order), then per instance
//   dt = CFL min( sqrt(h / max|a|), h / (max c + max mu) )
// (0 for instances that are done), and the maxima are cleared for the next
// evaluation.  Loads bypass L1 (the partials may come from the same kernel).
// Run by a block of at most 256 threads (an interaction block).
__device__ void reduce_counters_and_dt(const Dev& d, const ReduceArgs& a, int set_dt) {
    __shared__ unsigned long long s_u[8][3];
    __shared__ uint32_t s_b[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    unsigned long long pf = 0, pb = 0, nc = 0;
    uint32_t bad = 0;
    for (uint32_t i = threadIdx.x; i < a.nparts; i += blockDim.x) {
        const uint4 u = __ldcg(a.part_u + i);
        pf += u.x;
        nc += u.y;
        bad |= u.z;
        pb += u.w;
    }
    for (int o = 16; o; o >>= 1) {
        pf += __shfl_xor_sync(kFull, pf, o);
        pb += __shfl_xor_sync(kFull, pb, o);
        nc += __shfl_xor_sync(kFull, nc, o);
        bad |= __shfl_xor_sync(kFull, bad, o);
    }
    if (lane == 0) {
        s_u[w][0] = pf;
        s_u[w][1] = pb;
        s_u[w][2] = nc;
        s_b[w] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long qf = 0, qb = 0, qc = 0;
        uint32_t bb = 0;
        for (int k = 0; k < nw; ++k) {
            qf += s_u[k][0];
            qb += s_u[k][1];
            qc += s_u[k][2];
            bb |= s_b[k];
        }
        a.counters[0] += qf + qb;
        a.counters[1] += qc;
        a.counters[2] = qf + qb;
        a.counters[3] = qc;
        a.counters[4] = qf;
        a.counters[5] = qb;
        a.counters[6] += qf;
        a.counters[7] += qb;
        if (bb) atomicOr(a.status, bb);
    }
    for (uint32_t q = threadIdx.x; q < d.n_inst; q += blockDim.x) {
        uint32_t* tm = d.is.terms + 3 * q;
        const float fa = __uint_as_float(__ldcg(tm + 0));
        const float fc = __uint_as_float(__ldcg(tm + 1));
        const float fm = __uint_as_float(__ldcg(tm + 2));
        const double amax = sqrt((double)fa);
        if (set_dt) {
            double dt = 0.0;
            if (!d.is.done[q]) {
                if (d.dt_fixed > 0.0) {
                    dt = d.dt_fixed;
                } else {
                    const double dtf = amax > 0.0 ? sqrt(d.h_d / amax) : INFINITY;
                    const double dtc = d.h_d / ((double)fc + (double)fm);
                    dt = d.cfl * (dtf < dtc ? dtf : dtc);
                }
            }
            d.is.dt[q] = dt;
            d.is.last[3 * q + 0] = (float)amax;
            d.is.last[3 * q + 1] = fc;
            d.is.last[3 * q + 2] = fm;
        }
        tm[0] = 0u;
        tm[1] = 0u;
        tm[2] = 0u;
    }
}

// Packed accumulators of two pair streams (the two pairs a lane evaluates
// per step of the pair phase), one in each half of a float2.  The momentum
// sums hold +sum f r_ij (the caller negates once at the end; negation is
// exact, so this equals summing the negated terms).
struct PairAcc2 {
    float2 ax, ay, az, dr, npf;
    float mu;
};

__device__ __forceinline__ float2 ff2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }

// pair_terms<KERN, true, true> for two pairs at once, with the Blackwell
// packed FP32 operations (__ffma2_rn, __fadd2_rn, __fmul2_rn: two FP32
// results per instruction, each rounded as the scalar operation); the
// square roots, reciprocals, min/max and the saturated support test stay
// scalar.  Same arithmetic per pair as pair_terms.
template <int KERN, bool MOM>
__device__ __forceinline__ void pair_terms2(const Dev& d, float c0, const float4& pi,
                                            const float4& vi, float ci, float2 dx, float2 dy,
                                            float2 dz, const float4& pa, const float4& va,
                                            const float4& pb, const float4& vb, PairAcc2& s) {
    const float2 d2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
    const float r2s = d.r2max * 0x1p100f;
    const float2 use = ff2(__saturatef(fmaf(d2.x, -0x1p100f, r2s)),
                           __saturatef(fmaf(d2.y, -0x1p100f, r2s)));
    s.npf = __fadd2_rn(s.npf, use);
    const float2 q = __fmul2_rn(ff2(sqrt_approx(d2.x), sqrt_approx(d2.y)), dup2(d.inv_h));
    float2 shape;
    if (KERN == 1) {
        const float2 wo = __ffma2_rn(q, dup2(-1.0f), dup2(2.0f));
        const float2 outer =
            __fmul2_rn(__fmul2_rn(dup2(-0.75f), __fmul2_rn(wo, wo)), ff2(rcp_approx(q.x), rcp_approx(q.y)));
        const float2 inner = __ffma2_rn(dup2(2.25f), q, dup2(-3.0f));
        shape = ff2(q.x < 1.0f ? inner.x : outer.x, q.y < 1.0f ? inner.y : outer.y);
    } else {
        const float2 wq = __ffma2_rn(dup2(-0.5f), q, dup2(1.0f));
        shape = __fmul2_rn(__fmul2_rn(wq, wq), wq);
    }
    const float2 F = __fmul2_rn(__fmul2_rn(dup2(d.fc), shape), use);
    const float2 m1 = dup2(-1.0f);
    const float2 dvx = __ffma2_rn(ff2(va.x, vb.x), m1, dup2(vi.x));
    const float2 dvy = __ffma2_rn(ff2(va.y, vb.y), m1, dup2(vi.y));
    const float2 dvz = __ffma2_rn(ff2(va.z, vb.z), m1, dup2(vi.z));
    const float2 vr = __ffma2_rn(dvx, dx, __ffma2_rn(dvy, dy, __fmul2_rn(dvz, dz)));
    s.dr = __ffma2_rn(vr, F, s.dr);                                 // Eq. 7
    if (MOM) {
        const float2 de = __fadd2_rn(d2, dup2(d.eta2));
        const float2 nu = __fmul2_rn(__fmul2_rn(dup2(d.h), vr), ff2(rcp_approx(de.x), rcp_approx(de.y)));
        const float2 rrj = __fmul2_rn(ff2(va.w, vb.w), dup2(d.inv_rho0));
        const float2 cj = __fmul2_rn(__fmul2_rn(__fmul2_rn(dup2(c0), rrj), rrj), rrj);
        const float2 rs = __fadd2_rn(dup2(vi.w), ff2(va.w, vb.w));
        const float2 nmin = ff2(fminf(nu.x, 0.f), fminf(nu.y, 0.f));
        const float2 visc = __fmul2_rn(
            __fmul2_rn(__fmul2_rn(dup2(-d.alpha), __fadd2_rn(dup2(ci), cj)), nmin),
            ff2(rcp_approx(rs.x), rcp_approx(rs.y)));
        const float2 f = __fmul2_rn(__fadd2_rn(__fadd2_rn(dup2(pi.w), ff2(pa.w, pb.w)), visc), F);
        s.ax = __ffma2_rn(f, dx, s.ax);                              // Eq. 9 (sign later)
        s.ay = __ffma2_rn(f, dy, s.ay);
        s.az = __ffma2_rn(f, dz, s.az);
        s.mu = fmaxf(s.mu, fmaxf(fabsf(nu.x) * use.x, fabsf(nu.y) * use.y));
    }
}

// Sec. 3.2.  One block takes work units in turn: up to W*32 consecutive
// sorted particles of one row of cells (same instance, cy, cz) spanning at
// most kSpan cells with no more than two empty cells in a row, so the
// candidates of all of them lie in 9 contiguous, compact runs of the sorted
// arrays (the neighbouring rows, cells [first cx - 1, last cx + 1]).  Those
// runs are copied to shared memory with bulk asynchronous copies; their y, z
// are then shifted into the frame of the unit's row, so a candidate's offset
// from particle i only needs i's own cell offset in x.  Each warp then tests
// every candidate of its lanes' cells in half precision (one broadcast
// shared-memory load per two candidates, all lanes) against a conservative
// threshold, keeps the hits as per-lane mask words, and evaluates the pair
// terms from the masks with all lanes busy, applying the exact FP32 test
// |r_ij| < 2h there.  Positions are relative to the particles' own cell
// origins (FP32), plus whole-cell offsets.  A unit whose runs do not fit the
// staging area reads its candidates from global memory instead (FP32 test,
// 32-bit lists).  Units of instances that are done are skipped.
// SPLIT warps share each group of 32 particles: warp w takes particles
// (w % W) * 32 + lane of the unit and every SPLIT-th candidate cell of each
// neighbour row r, starting at cell xlo + (w / W + r) % SPLIT (the rotation
// evens out the parts' shares when a warp's cell range is odd; every lane
// keeps a similar share of its own neighbours in each part); the parts' sums
// are added in a fixed order at the end.  More warps per block at the same
// staging footprint.
template <int W, int STAGE, int WCAP, int MINB, bool COUNTS, int SPLIT, int KERN, bool PK,
          bool TU, bool DYN>
__global__ void __launch_bounds__(W * SPLIT * 32, MINB) k_interact(const Dev d, const InteractArgs a) {
    pdl_wait();
    constexpr int NT = W * SPLIT * 32;
    constexpr int FBCAP = Shape<W * SPLIT, STAGE, WCAP>::fb_cap;   // fallback list slots
    extern __shared__ __align__(128) unsigned char s_raw[];
    float4* s_p = reinterpret_cast<float4*>(s_raw);
    float4* s_v = s_p + STAGE;
    uint4* s_h = reinterpret_cast<uint4*>(s_v + STAGE);            // STAGE / 2 candidate pairs
    uint32_t* s_words = reinterpret_cast<uint32_t*>(s_h + STAGE / 2);
    uint32_t* s_desc = s_words + W * SPLIT * WCAP * 32;
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ uint32_t s_rs[9], s_len[9], s_base[10];
    // cell offsets of the 9 runs (DYN: two buffers, the next unit's filled
    // by asynchronous copies while this one is worked on)
    __shared__ uint32_t s_offb[DYN ? 2 : 1][9][kSpan + 3];
    __shared__ int s_okb[DYN ? 2 : 1][9];
    __shared__ uint32_t s_nui[2];                // DYN: next unit, by parity of k
    __shared__ int s_mode;
    __shared__ uint32_t s_ru[W * SPLIT][4];
    __shared__ float s_comb[SPLIT > 1 ? (SPLIT - 1) * W * 32 : 1][8];   // parts 1.. sums

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) mbar_init(&s_bar, 1);
    __syncthreads();
    const uint32_t nunits = *a.n_units;
    uint32_t phase = 0;
    uint32_t t_np = 0, t_nb = 0, t_nc = 0, t_bad = 0;   // counters over this block's units
    // DYN: units are taken from a counter (the first one is blockIdx.x), and
    // the next unit's record, end labels and cell offsets are fetched while
    // this one is worked on.  pf: the next unit's record is in nx_*; pf_off:
    // its offsets are in buffer sb ^ 1.  Every value is block-uniform.
    uint32_t k_unit = 0;
    bool pf = false, pf_off = false;
    int sb = 0;
    uint2 nx_unit = make_uint2(0u, 0u);
    uint32_t nx_k0 = 0u, nx_kl = 0u;
    for (uint32_t ui = blockIdx.x; ui < nunits;) {
    uint32_t (*s_off)[kSpan + 3] = s_offb[DYN ? sb : 0];
    int* s_ok = s_okb[DYN ? sb : 0];
    if (DYN && tid == 0) s_nui[k_unit & 1u] = gridDim.x + atomicAdd(a.sched, 1u);
    uint2 unit;
    uint32_t key0, keyl = 0u;
    if (DYN && pf) {
        unit = nx_unit;
        key0 = nx_k0;
        keyl = nx_kl;
    } else {
        unit = a.units[ui];
        key0 = __ldg(a.key + unit.x);
        if (DYN) keyl = __ldg(a.key + unit.y - 1);
    }
    const bool have_off = DYN && pf_off;
    pf = false;
    pf_off = false;
    const uint32_t i0 = unit.x, i1 = unit.y;
    if (!in_bounds(i0 < i1 && i1 <= d.n && i1 - i0 <= (uint32_t)(W * 32), d.status)) break;
    const uint32_t q = find_instance(d.cell_base, d.n_inst, key0);
    if (__ldg(d.is.done + q)) {                      // block-uniform
        if (DYN) {
            __syncthreads();                         // s_nui written
            ui = s_nui[k_unit & 1u];
            ++k_unit;
        } else {
            ui += gridDim.x;
        }
        continue;
    }
    const Inst& I = d.inst[q];
    const int ncx = I.ncx, ncy = I.ncy, ncz = I.ncz;
    const float c0 = I.c0;
    const uint32_t lkey0 = key0 - I.cell_base;
    const uint32_t lrow = lkey0 / (uint32_t)ncx;
    const uint32_t rowbase = I.cell_base + lrow * (uint32_t)ncx;   // global label of (0, cy, cz)
    const int cy = (int)(lrow % (uint32_t)ncy), cz = (int)(lrow / (uint32_t)ncy);
    const int xb = (int)(key0 - rowbase);
    const int xe = (int)((DYN ? keyl : __ldg(a.key + i1 - 1)) - rowbase);
    const int ulo = xb > 0 ? xb - 1 : 0;
    const int uhi = xe + 1 < ncx ? xe + 1 : ncx - 1;
    const int nce = uhi - ulo + 2;                 // offsets per neighbour row
    if (!have_off) {
        // cell offsets of the 9 neighbour rows (each thread derives its
        // row's base label itself: no barrier before the loads)
        for (int r9 = tid; r9 < 9 * nce; r9 += NT) {
            const int r = r9 / nce, c = r9 - r * nce;
            const int yy = cy + r % 3 - 1, zz = cz + r / 3 - 1;
            const bool ok = yy >= 0 && yy < ncy && zz >= 0 && zz < ncz;
            const uint32_t rb =
                I.cell_base + (uint32_t)ncx * ((uint32_t)yy + (uint32_t)ncy * (uint32_t)zz);
            s_off[r][c] = ok ? __ldg(a.off + rb + ulo + c) : 0u;
            if (c == 0) s_ok[r] = ok;
        }
        __syncthreads();
    }
    // staging plan and copies by the first warp: lane r < 9 owns run r
    if (w == 0) {
        const uint32_t len = lane < 9 ? s_off[lane][nce - 1] - s_off[lane][0] : 0u;
        uint32_t incl = len;
#pragma unroll
        for (int o = 1; o < 16; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        const uint32_t base = incl - len;
        const uint32_t total = __shfl_sync(kFull, incl, 8);
        if (lane < 9) {
            s_base[lane] = base;
            s_rs[lane] = s_off[lane][0];
            s_len[lane] = len;
        }
        if (lane == 0) {
            s_base[9] = total;
            s_mode = total <= (uint32_t)STAGE;
            if (total <= (uint32_t)STAGE)
                mbar_expect_tx(&s_bar, total * 2u * (uint32_t)sizeof(float4));
        }
        __syncwarp();
        // the expected byte count is registered before any copy is issued
        if (total <= (uint32_t)STAGE && lane < 18) {
            const int r = lane >> 1;
            const uint32_t rl = __shfl_sync(0x3ffffu, len, r);
            const uint32_t rbase = __shfl_sync(0x3ffffu, base, r);
            const uint32_t rs = s_off[r][0];
            if (rl) {
                if (lane & 1)
                    bulk_g2s(s_v + rbase, a.velrhop + rs, rl * (uint32_t)sizeof(float4), &s_bar);
                else
                    bulk_g2s(s_p + rbase, a.posc + rs, rl * (uint32_t)sizeof(float4), &s_bar);
            }
        }
    }
    // own particle, while the copies are in flight
    const int part = w / W;
    const uint32_t i = i0 + (uint32_t)((w % W) * 32 + lane);
    const bool valid = i < i1;
    float4 pi = make_float4(0.f, 0.f, 0.f, 0.f), vi = make_float4(0.f, 0.f, 0.f, 1.f);
    int cx = 0;
    bool fluid = false;
    if (valid) {
        pi = a.posc[i];
        vi = a.velrhop[i];
        cx = (int)(__ldg(a.key + i) - rowbase);
        fluid = a.id[i] >= I.id_fluid;
    }
    const float rri = vi.w * d.inv_rho0;
    const float ci = c0 * rri * rri * rri;
    PairAcc acc = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0u};
    uint32_t ncand = 0;
    __syncthreads();
    const bool staged = s_mode != 0;
    // DYN: the next unit (taken by thread 0 at the top of this one) and its
    // record; its end labels follow once the record has landed
    uint32_t nui = 0u;
    if (DYN) {
        nui = s_nui[k_unit & 1u];
        if (nui < nunits) nx_unit = a.units[nui];
    }
    if (staged) {
        const bool got = mbar_wait_bounded(&s_bar, phase);
        if (__syncthreads_or(!got) != 0) {
            if (tid == 0) atomicOr(a.status, kStatusTimeout);
            mbar_wait_bounded(&s_bar, phase);   // let copies in flight land first
            break;
        }
        phase ^= 1u;
        if (DYN && nui < nunits) {
            nx_k0 = __ldg(a.key + nx_unit.x);
            nx_kl = __ldg(a.key + nx_unit.y - 1);
            pf = true;
        }
        // one pass over candidate pairs: shift the staged y, z into the
        // frame of this unit's row (the run r of a candidate gives the
        // offsets), then keep half-precision copies in cell units (cell =
        // 2h = 1) centred on the cell (minus 1/2), two candidates per uint4:
        // (x0, x1), (y0, y1), (z0, z1) and their squared norms (k0, k1),
        // computed from the rounded coordinates
        const float inv_cs = 1.0f / d.csf;
        const uint32_t nst = s_base[9];
        for (uint32_t k = tid; 2 * k < nst; k += NT) {
            float4 pp[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const uint32_t j = 2 * k + (uint32_t)e;
                if (j >= nst) {
                    pp[e] = pp[0];
                    continue;
                }
                int r = 0;
#pragma unroll
                for (int q2 = 1; q2 < 9; ++q2) r += s_base[q2] <= j ? 1 : 0;
                float4 v = s_p[j];
                v.y += (float)(r % 3 - 1) * d.csf;
                v.z += (float)(r / 3 - 1) * d.csf;
                s_p[j] = v;
                pp[e] = v;
            }
            const __half2 hx = __floats2half2_rn(fmaf(pp[0].x, inv_cs, -0.5f),
                                                 fmaf(pp[1].x, inv_cs, -0.5f));
            const __half2 hy = __floats2half2_rn(fmaf(pp[0].y, inv_cs, -0.5f),
                                                 fmaf(pp[1].y, inv_cs, -0.5f));
            const __half2 hz = __floats2half2_rn(fmaf(pp[0].z, inv_cs, -0.5f),
                                                 fmaf(pp[1].z, inv_cs, -0.5f));
            const float2 fx = __half22float2(hx), fy = __half22float2(hy), fz = __half22float2(hz);
            const __half2 hk = __floats2half2_rn(fmaf(fx.x, fx.x, fmaf(fy.x, fy.x, fz.x * fz.x)),
                                                 fmaf(fx.y, fx.y, fmaf(fy.y, fy.y, fz.y * fz.y)));
            s_h[k] = make_uint4(*reinterpret_cast<const uint32_t*>(&hx),
                                *reinterpret_cast<const uint32_t*>(&hy),
                                *reinterpret_cast<const uint32_t*>(&hz),
                                *reinterpret_cast<const uint32_t*>(&hk));
        }
        __syncthreads();
        if (DYN && pf) {
            // the next unit's cell offsets into the other buffer (asynchronous
            // 4-byte copies, waited for before this unit's last barrier)
            const uint32_t nq = find_instance(d.cell_base, d.n_inst, nx_k0);
            const Inst& J = d.inst[nq];
            const int jcx = J.ncx, jcy = J.ncy, jcz = J.ncz;
            const uint32_t jrow = (nx_k0 - J.cell_base) / (uint32_t)jcx;
            const uint32_t jbase = J.cell_base + jrow * (uint32_t)jcx;
            const int jy = (int)(jrow % (uint32_t)jcy), jz = (int)(jrow / (uint32_t)jcy);
            const int jxb = (int)(nx_k0 - jbase), jxe = (int)(nx_kl - jbase);
            const int jlo = jxb > 0 ? jxb - 1 : 0;
            const int jhi = jxe + 1 < jcx ? jxe + 1 : jcx - 1;
            const int jnce = jhi - jlo + 2;
            uint32_t (*o2)[kSpan + 3] = s_offb[sb ^ 1];
            int* ok2 = s_okb[sb ^ 1];
            for (int r9 = tid; r9 < 9 * jnce; r9 += NT) {
                const int r = r9 / jnce, c = r9 - r * jnce;
                const int yy = jy + r % 3 - 1, zz = jz + r / 3 - 1;
                const bool ok = yy >= 0 && yy < jcy && zz >= 0 && zz < jcz;
                if (ok) {
                    const uint32_t rb =
                        J.cell_base + (uint32_t)jcx * ((uint32_t)yy + (uint32_t)jcy * (uint32_t)zz);
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                                     smem_u32(&o2[r][c])),
                                 "l"(a.off + rb + jlo + c)
                                 : "memory");
                } else {
                    o2[r][c] = 0u;
                }
                if (c == 0) ok2[r] = ok;
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
            pf_off = true;
        }
    }

    const uint32_t act = __ballot_sync(kFull, valid);
    if (act) {
        const int wxmin = __reduce_min_sync(kFull, valid ? cx : 0x7fffffff);
        const int wxmax = __reduce_max_sync(kFull, valid ? cx : -1);
        const int xlo = wxmin > 0 ? wxmin - 1 : 0;
        const int xhi = wxmax + 1 < ncx ? wxmax + 1 : ncx - 1;
        uint32_t cnt = 0;
        if (staged) {
            // candidate test in half precision, two candidates per
            // instruction, against a conservative threshold (cell units,
            // centred coordinates q of particle i and p of the candidate:
            // |q - p|^2 - thr = (|p|^2 + (|q|^2 - thr)) - 2 q.p < 0, thr =
            // 1 + 2^-6, one add and three fused multiply-adds); each lane
            // keeps one 32-bit hit mask per word of 32 staged candidates
            // (bit 8k + j: candidate base + 4j + k).  The pair phase applies
            // the exact FP32 test.  Rounding:
            // for |q - p| <= 1 every intermediate stays below 8, so the
            // computed value exceeds the exact one by at most 7.8e-3, and the
            // rounded coordinates move |q - p|^2 by at most 2.6e-3: a pair
            // within the support always tests negative.
            uint32_t* wl = s_words + w * (WCAP * 32) + lane;
            uint32_t* wd = s_desc + w * WCAP;
            PairAcc2 acc2 = {dup2(0.f), dup2(0.f), dup2(0.f), dup2(0.f), dup2(0.f), 0.f};
            const uint32_t self = valid ? s_base[4] + (i - s_rs[4]) : 0u;
            const bool anyfluid = __any_sync(kFull, fluid);
            const float inv_cs = 1.0f / d.csf;
            const float thr = 1.0f + 1.0f / 64.0f;
            // y and z of i, centred and rounded; -2 q_y, -2 q_z (exact)
            const __half2 hqy = __float2half2_rn(fmaf(pi.y, inv_cs, -0.5f));
            const __half2 hqz = __float2half2_rn(fmaf(pi.z, inv_cs, -0.5f));
            const float qy = __low2float(hqy), qz = __low2float(hqz);
            const float qyz2 = fmaf(qy, qy, qz * qz) - thr;
            const __half2 m2qy = __float2half2_rn(-2.0f * qy);
            const __half2 m2qz = __float2half2_rn(-2.0f * qz);
            uint32_t nw = 0, lane_hits = 0;
            uint32_t lane_nz = 0;   // bit w: stored word w holds hits of this lane
            static_assert(WCAP <= 32, "one bit per stored word");
            // pair phase over the stored words: each lane pops its own hits,
            // two per iteration; lanes that run out are padded with i itself,
            // placed 4 cells away (no contribution, not counted)
            auto flush = [&]() {
                __syncwarp();   // the words and lane 0's descriptors are written
                const uint32_t mx = __reduce_max_sync(kFull, lane_hits);
                uint32_t nz = lane_nz, cm = 0, jb = 0;
                float qxw = 0.f;                         // i's x in the word's cell frame
                const float qpad = fmaf(4.0f, d.csf, pi.x);   // pads: i itself, out of range
                constexpr int kPop = 2;   // pairs per iteration (independent chains)
                // the lane's next hit (its staged index and i's x in that
                // word's cell frame), or the pad i itself, out of range
                auto pop = [&](uint32_t& j, float& qx) {
                    if (cm == 0 && nz != 0) {
                        const uint32_t wi = __ffs(nz) - 1;
                        nz &= nz - 1;
                        cm = wl[wi * 32];
                        const uint32_t dsc = wd[wi];
                        jb = dsc & 0xffffu;
                        qxw = fmaf((float)(cx - (ulo + (int)(dsc >> 16))), d.csf, pi.x);
                    }
                    if (cm) {
                        const uint32_t b = 31u - __clz(cm);
                        cm ^= 1u << b;
                        j = jb + 4u * b - 31u * (b >> 3);
                        qx = qxw;
                    } else {
                        j = self;
                        qx = qpad;
                    }
                };
                for (uint32_t t = 0; t < mx; t += kPop) {
                    uint32_t j2[kPop];
                    float qx2[kPop];
#pragma unroll
                    for (int k = 0; k < kPop; ++k) pop(j2[k], qx2[k]);
                    float4 pp[kPop], vv[kPop];
#pragma unroll
                    for (int k = 0; k < kPop; ++k) {
                        if (!in_bounds(j2[k] < s_base[9], d.status)) {
                            j2[k] = self;
                            qx2[k] = qpad;
                        }
                        pp[k] = s_p[j2[k]];
                        vv[k] = s_v[j2[k]];
                    }
                    if (PK) {
                        const float2 m1 = dup2(-1.0f);
                        const float2 dx2 = __ffma2_rn(ff2(pp[0].x, pp[1].x), m1, ff2(qx2[0], qx2[1]));
                        const float2 dy2 = __ffma2_rn(ff2(pp[0].y, pp[1].y), m1, dup2(pi.y));
                        const float2 dz2 = __ffma2_rn(ff2(pp[0].z, pp[1].z), m1, dup2(pi.z));
                        if (anyfluid)
                            pair_terms2<KERN, true>(d, c0, pi, vi, ci, dx2, dy2, dz2, pp[0], vv[0],
                                                    pp[1], vv[1], acc2);
                        else
                            pair_terms2<KERN, false>(d, c0, pi, vi, ci, dx2, dy2, dz2, pp[0], vv[0],
                                                     pp[1], vv[1], acc2);
                    } else if (anyfluid) {
#pragma unroll
                        for (int k = 0; k < kPop; ++k)
                            pair_terms<KERN, true, true>(d, c0, pi, vi, ci, qx2[k] - pp[k].x,
                                                         pi.y - pp[k].y, pi.z - pp[k].z, pp[k],
                                                         vv[k], acc);
                    } else {
#pragma unroll
                        for (int k = 0; k < kPop; ++k)
                            pair_terms<KERN, false, true>(d, c0, pi, vi, ci, qx2[k] - pp[k].x,
                                                          pi.y - pp[k].y, pi.z - pp[k].z, pp[k],
                                                          vv[k], acc);
                    }
                }
                __syncwarp();   // every lane is done reading before the words are reused
                acc.np += (uint32_t)acc.npf;
                acc.npf = 0.f;
                if (PK) {
                    acc.np += (uint32_t)acc2.npf.x + (uint32_t)acc2.npf.y;
                    acc2.npf = dup2(0.f);
                }
                nw = 0;
                lane_hits = 0;
                lane_nz = 0;
            };
            for (int r = 0; r < 9; ++r) {
                if (!s_ok[r]) continue;
                const uint32_t rs = s_rs[r], sb = s_base[r];
                for (int xx = xlo + (part + r) % SPLIT; xx <= xhi; xx += SPLIT) {
                    const uint32_t gs = s_off[r][xx - ulo], ge = s_off[r][xx - ulo + 1];
                    const int ox = cx - xx;
                    const bool adj = valid && ox >= -1 && ox <= 1;
                    if (adj) ncand += ge - gs;
                    if (gs == ge) continue;
                    // x of i in the candidate cell's frame, centred and
                    // rounded; |q|^2 - thr
                    const __half2 hqx =
                        __float2half2_rn(fmaf(fmaf((float)ox, d.csf, pi.x), inv_cs, -0.5f));
                    const float qx = __low2float(hqx);
                    const __half2 hc = __float2half2_rn(fmaf(qx, qx, qyz2));
                    const __half2 m2qx = __float2half2_rn(-2.0f * qx);
                    const uint32_t s0 = sb + (gs - rs), e0 = sb + (ge - rs);
                    for (uint32_t base = s0 & ~1u; base < e0; base += 32) {
                        if (nw == (uint32_t)WCAP) flush();
                        const uint32_t lim = e0 - base < 32u ? e0 - base : 32u;   // slots in use
                        const uint32_t npair = (lim + 1) >> 1;
                        const uint4* hp = s_h + (base >> 1);
                        // the sign bits of r^2 - thr for two candidate pairs
                        // (four candidates) spread into one byte each (all
                        // ones or zero), then one bit of each byte kept: bit
                        // 8k + j <-> candidate base + 4j + k.  A pair slot
                        // past the word's end is read (inside the shared
                        // allocation) and masked below.
                        auto test_pair = [&](const uint4 hv) {
                            const __half2 kc = __hadd2(*reinterpret_cast<const __half2*>(&hv.w), hc);
                            const __half2 r2t = __hfma2(
                                m2qx, *reinterpret_cast<const __half2*>(&hv.x),
                                __hfma2(m2qy, *reinterpret_cast<const __half2*>(&hv.y),
                                        __hfma2(m2qz, *reinterpret_cast<const __half2*>(&hv.z), kc)));
                            return *reinterpret_cast<const uint32_t*>(&r2t);
                        };
                        uint32_t m = 0;
                        // TU: a word of five or more candidate pairs tests its
                        // first eight pairs without a bound test between them
                        // (their loads can all be in flight), then the rest
                        uint32_t jj0 = 0;
                        if (TU && npair >= 5) {
#pragma unroll
                            for (uint32_t jj = 0; jj < 4; ++jj) {
                                const uint32_t sa = test_pair(hp[2 * jj]), sb = test_pair(hp[2 * jj + 1]);
                                m |= sign_bytes(sa, sb) & (0x01010101u << jj);
                            }
                            jj0 = 4;
                        }
#pragma unroll
                        for (uint32_t jj = 0; jj < 8; ++jj) {
                            if (jj < jj0) continue;
                            if (2 * jj >= npair) break;
                            const uint32_t sa = test_pair(hp[2 * jj]), sb = test_pair(hp[2 * jj + 1]);
                            m |= sign_bytes(sa, sb) & (0x01010101u << jj);
                        }
                        // slots outside [s0, e0) and lanes not adjacent to the cell
                        uint32_t keep = c_keep.v[lim];
                        if (base < s0) keep &= ~1u;
                        m = adj ? (m & keep) : 0u;
                        if (__any_sync(kFull, m != 0u)) {
                            wl[nw * 32] = m;
                            if (lane == 0) wd[nw] = base | ((uint32_t)(xx - ulo) << 16);
                            lane_hits += __popc(m);
                            lane_nz |= (m != 0u ? 1u : 0u) << nw;
                            ++nw;
                        }
                    }
                }
            }
            flush();
            if (PK) {
                // the two streams' sums, in a fixed order (momentum negated once)
                acc.ax -= acc2.ax.x + acc2.ax.y;
                acc.ay -= acc2.ay.x + acc2.ay.y;
                acc.az -= acc2.az.x + acc2.az.y;
                acc.dr += acc2.dr.x + acc2.dr.y;
                acc.mu = fmaxf(acc.mu, acc2.mu);
            }
        } else {
            // candidates straight from global memory (unit too large to stage)
            uint32_t* lst = reinterpret_cast<uint32_t*>(s_raw) + w * (FBCAP * 32);
            auto flush = [&]() {
                const uint32_t mx = __reduce_max_sync(kFull, cnt);
                for (uint32_t t = 0; t < mx; ++t) {
                    if (t < cnt) {
                        const uint32_t e = lst[t * 32 + lane];
                        uint32_t j = e & kIdxMask;
                        if (!in_bounds(j < d.n, d.status)) j = i;
                        const float ox = (float)((int)((e >> 26) & 3u) - 1);
                        const float oy = (float)((int)((e >> 28) & 3u) - 1);
                        const float oz = (float)((int)(e >> 30) - 1);
                        const float4 pj = __ldg(a.posc + j);
                        const float4 vj = __ldg(a.velrhop + j);
                        pair_terms<KERN, true>(d, c0, pi, vi, ci, fmaf(ox, d.csf, pi.x) - pj.x,
                                               fmaf(oy, d.csf, pi.y) - pj.y,
                                               fmaf(oz, d.csf, pi.z) - pj.z, pj, vj, acc);
                    }
                }
                acc.np += cnt;
                cnt = 0;
            };
            for (int r = 0; r < 9; ++r) {
                if (!s_ok[r]) continue;
                const int dy = r % 3 - 1, dz = r / 3 - 1;
                const float qy = fmaf((float)(-dy), d.csf, pi.y);
                const float qz = fmaf((float)(-dz), d.csf, pi.z);
                const uint32_t code_yz = ((uint32_t)(1 - dy) << 28) | ((uint32_t)(1 - dz) << 30);
                for (int xx = xlo + (part + r) % SPLIT; xx <= xhi; xx += SPLIT) {
                    const uint32_t gs = s_off[r][xx - ulo], ge = s_off[r][xx - ulo + 1];
                    const int ox = cx - xx;
                    const bool adj = valid && ox >= -1 && ox <= 1;
                    if (adj) ncand += ge - gs;
                    if (gs == ge) continue;
                    const float qx = fmaf((float)ox, d.csf, pi.x);
                    const uint32_t code = code_yz | ((uint32_t)(ox + 1) << 26);
                    for (uint32_t c0i = gs; c0i < ge; c0i += FBCAP) {
                        const uint32_t c1 = (ge - c0i) > (uint32_t)FBCAP ? c0i + FBCAP : ge;
                        if (__reduce_max_sync(kFull, cnt) + (c1 - c0i) > (uint32_t)FBCAP) flush();
#pragma unroll 4
                        for (uint32_t j = c0i; j < c1; ++j) {
                            const float4 pj = __ldg(a.posc + j);
                            const float dx = qx - pj.x, dy2 = qy - pj.y, dz2 = qz - pj.z;
                            const float d2 = fmaf(dx, dx, fmaf(dy2, dy2, dz2 * dz2));
                            if (adj && d2 < d.r2max) {
                                lst[cnt * 32 + lane] = j | code;
                                ++cnt;
                            }
                        }
                    }
                }
            }
            flush();
        }
    }

    if (SPLIT > 1) {
        // parts 1 .. SPLIT-1 hand their sums to part 0, which adds them in
        // part order (a fixed order: the result does not depend on timing)
        const int slot = (w % W) * 32 + lane;
        if (part > 0) {
            float* c = s_comb[(part - 1) * W * 32 + slot];
            c[0] = acc.ax;
            c[1] = acc.ay;
            c[2] = acc.az;
            c[3] = acc.dr;
            c[4] = acc.mu;
            c[5] = __uint_as_float(acc.np);
            c[6] = __uint_as_float(ncand);
        }
        __syncthreads();
        if (part == 0) {
#pragma unroll
            for (int pp = 1; pp < SPLIT; ++pp) {
                const float* c = s_comb[(pp - 1) * W * 32 + slot];
                acc.ax += c[0];
                acc.ay += c[1];
                acc.az += c[2];
                acc.dr += c[3];
                acc.mu = fmaxf(acc.mu, c[4]);
                acc.np += __float_as_uint(c[5]);
                ncand += __float_as_uint(c[6]);
            }
        }
    }
    const bool owner = part == 0;                   // writes this particle's results
    const float m = d.mass;
    // boundary particles keep gravity only (their momentum sums are dropped)
    const float4 out = make_float4(fmaf(m, fluid ? acc.ax : 0.f, d.gx),
                                   fmaf(m, fluid ? acc.ay : 0.f, d.gy),
                                   fmaf(m, fluid ? acc.az : 0.f, d.gz), m * acc.dr);
    const uint32_t npairs = (valid && owner) ? acc.np - 1u : 0u;   // without the pair (i, i)
    if (valid && owner) {
        a.ace[i] = out;
        if (COUNTS) a.nnb[i] = npairs;
    }
    // this instance's CFL maxima (non-negative floats order like their bits)
    float am = (valid && fluid) ? out.x * out.x + out.y * out.y + out.z * out.z : 0.f;
    if (!(am == am)) am = 0.f;
    float cm = valid ? ci : 0.f;
    float mm = (valid && fluid) ? acc.mu : 0.f;
    for (int o = 16; o; o >>= 1) {
        am = fmaxf(am, __shfl_xor_sync(kFull, am, o));
        cm = fmaxf(cm, __shfl_xor_sync(kFull, cm, o));
        mm = fmaxf(mm, __shfl_xor_sync(kFull, mm, o));
    }
    if (lane == 0 && act && owner) {
        atomicMax(d.is.terms + 3 * q + 0, __float_as_uint(am));
        atomicMax(d.is.terms + 3 * q + 1, __float_as_uint(cm));
        atomicMax(d.is.terms + 3 * q + 2, __float_as_uint(mm));
    }
    t_bad |= (valid && owner && !(isfinite(out.x) && isfinite(out.y) && isfinite(out.z) &&
                                  isfinite(out.w)))
                 ? kStatusNonFinite
                 : 0u;
    t_np += fluid ? npairs : 0u;
    t_nb += fluid ? 0u : npairs;
    t_nc += owner ? ncand : 0u;
    if (DYN && pf_off) asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();   // the next unit overwrites the shared staging
    if (DYN) {
        ui = nui;
        ++k_unit;
        if (pf_off) sb ^= 1;
    } else {
        ui += gridDim.x;
    }
    }
    if (DYN) {
        // the last block to finish rearms the unit counter for the next launch
        // (every block's last take precedes its finish ticket)
        __threadfence();
        if (tid == 0 && atomicAdd(a.sched + 1, 1u) == gridDim.x - 1u) {
            a.sched[0] = 0u;
            a.sched[1] = 0u;
        }
    }

    uint32_t np = t_np, nb = t_nb, nc = t_nc, bad = t_bad;
    for (int o = 16; o; o >>= 1) {
        np += __shfl_xor_sync(kFull, np, o);
        nb += __shfl_xor_sync(kFull, nb, o);
        nc += __shfl_xor_sync(kFull, nc, o);
        bad |= __shfl_xor_sync(kFull, bad, o);
    }
    if (lane == 0) {
        s_ru[w][0] = np;
        s_ru[w][1] = nc;
        s_ru[w][2] = bad;
        s_ru[w][3] = nb;
    }
    __syncthreads();
    if (tid == 0) {
        uint4 u = make_uint4(0u, 0u, 0u, 0u);
        for (int k = 0; k < W * SPLIT; ++k) {
            u.x += s_ru[k][0];
            u.y += s_ru[k][1];
            u.z |= s_ru[k][2];
            u.w += s_ru[k][3];
        }
        a.part_u[blockIdx.x] = u;
    }
    if (a.ticket) {
        // the last block to finish runs the Sec. 3.3 reductions (every
        // thread's maxima atomics and thread 0's partials fenced first)
        __shared__ bool s_lastblk;
        __threadfence();
        __syncthreads();
        if (tid == 0) s_lastblk = atomicAdd(a.ticket, 1u) == gridDim.x - 1u;
        __syncthreads();
        if (s_lastblk) {
            __threadfence();
            reduce_counters_and_dt(d, a.red, a.set_dt);
            if (tid == 0) *a.ticket = 0u;
        }
    }
}

// Staged-candidate prefix sums of each row: for row r and x in [0, ncx],
// csum[I.cell_base + lr ncx + r + x] = sum over the 9 neighbour rows (dy, dz
// in {-1, 0, 1}, inside the instance) of off[row + x].  The particles of the
// 9 runs of cells [x0, x1) then number csum[x1] - csum[x0].  One block per
// row, threads along x (coalesced).
__global__ void __launch_bounds__(128) k_row_csum(const Dev d, const uint32_t* __restrict__ off,
                                                  uint32_t* __restrict__ csum) {
    pdl_wait();
    const uint32_t r = blockIdx.x;
    const Inst& I = d.inst[find_instance(d.row_base, d.n_inst, r)];
    const int ncx = I.ncx;
    const uint32_t lr = r - I.row_base;
    const int cy = (int)(lr % (uint32_t)I.ncy), cz = (int)(lr / (uint32_t)I.ncy);
    uint32_t* out = csum + I.cell_base + (size_t)lr * (uint32_t)ncx + r;
    for (int x = threadIdx.x; x <= ncx; x += blockDim.x) {
        uint32_t t = 0;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int yy = cy + k % 3 - 1, zz = cz + k / 3 - 1;
            if (yy >= 0 && yy < I.ncy && zz >= 0 && zz < I.ncz)
                t += __ldg(off + I.cell_base +
                           ((size_t)zz * (uint32_t)I.ncy + (uint32_t)yy) * (uint32_t)ncx + x);
        }
        out[x] = t;
    }
}

// Work units.  A row of cells is cut into units of consecutive particles:
// a unit closes before a cell that lies more than 3 cells past the unit's
// last non-empty cell (so no unit spans an empty stretch), when it would
// reach kSpan cells, when its staged candidates (the 9 neighbour rows over
// cells [first - 1, last + 1]) would exceed the staging area of the
// interaction variant in use (d.stage), or when it holds d.unit particles
// (the variant's block size).  One thread walks one (global) row, reading
// the offsets and staged-candidate sums in chunks of kUnitChunk cells (all
// loads of a chunk in flight together); mode 0 counts the units of each
// row, mode 1 writes them at the row's offset (uint2: first particle, end).
constexpr int kUnitChunk = 16;

// The walk of row r: its units (mode 1 writes them from units[out]).  With
// SCS the row's staged-candidate sums are read from `csum` itself (the
// caller's shared-memory copy, indexes 0..ncx) instead of the global array.
template <int MODE, bool SCS = false>
__device__ __forceinline__ uint32_t unit_walk(const Dev& d, const uint32_t* __restrict__ off,
                                              const uint32_t* __restrict__ csum, uint32_t r,
                                              uint32_t out,
                                              uint2* __restrict__ units) {
    const Inst& I = d.inst[find_instance(d.row_base, d.n_inst, r)];
    const int ncx = I.ncx;
    const uint32_t lr = r - I.row_base;
    const uint32_t* o = off + I.cell_base + (size_t)lr * (uint32_t)ncx;
    const uint32_t* cs = SCS ? csum : csum + I.cell_base + (size_t)lr * (uint32_t)ncx + r;
    uint32_t n = 0;
    uint32_t start = 0xffffffffu;
    uint32_t base = 0;   // cs[first - 1] of the open unit (clamped at 0)
    int lo = 0, last = 0;
    uint32_t a = __ldg(o);
    for (int x0 = 0; x0 < ncx; x0 += kUnitChunk) {
        // ob[k] = o[x + 1], cc[k] = cs[x - 1], cc[k + 3] = cs[x + 2] for
        // x = x0 + k (indexes clamped to [0, ncx])
        uint32_t ob[kUnitChunk], cc[kUnitChunk + 3];
#pragma unroll
        for (int k = 0; k < kUnitChunk; ++k) {
            const int xi = x0 + 1 + k;
            ob[k] = __ldg(o + (xi < ncx ? xi : ncx));
        }
#pragma unroll
        for (int k = 0; k < kUnitChunk + 3; ++k) {
            const int xi = x0 - 1 + k;
            const int xc = xi < 0 ? 0 : (xi < ncx ? xi : ncx);
            cc[k] = SCS ? cs[xc] : __ldg(cs + xc);
        }
#pragma unroll
        for (int k = 0; k < kUnitChunk; ++k) {
            const int x = x0 + k;
            const uint32_t b = ob[k];
            if (x < ncx && a != b) {
                if (start != 0xffffffffu &&
                    (x - last > 3 || x - lo >= kSpan || cc[k + 3] - base > (uint32_t)d.stage)) {
                    if (MODE && in_bounds(out + n < d.units_cap, d.status)) units[out + n] = make_uint2(start, a);
                    ++n;
                    start = 0xffffffffu;
                }
                if (start == 0xffffffffu) {
                    start = a;
                    lo = x;
                    base = cc[k];
                }
                last = x;
                while (b - start > (uint32_t)d.unit) {
                    if (MODE && in_bounds(out + n < d.units_cap, d.status)) units[out + n] = make_uint2(start, start + d.unit);
                    ++n;
                    start += d.unit;
                    lo = x;
                    base = cc[k];
                }
            }
            if (x < ncx) a = b;
        }
    }
    if (start != 0xffffffffu) {
        if (MODE && in_bounds(out + n < d.units_cap, d.status)) units[out + n] = make_uint2(start, a);
        ++n;
    }
    return n;
}

template <int MODE>
__global__ void __launch_bounds__(128) k_units(const Dev d, const uint32_t* __restrict__ off,
                                               const uint32_t* __restrict__ csum,
                                               uint32_t* __restrict__ ucnt,
                                               const uint32_t* __restrict__ uoff,
                                               uint2* __restrict__ units) {
    pdl_wait();
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= d.nrows) return;
    const uint32_t n = unit_walk<MODE>(d, off, csum, r, MODE ? uoff[r] : 0u, units);
    if (!MODE) ucnt[r] = n;
}

// The unit list of a grid of few rows in one launch (d.nrows <= kFusedRows,
// rows of at most kFusedNcx cells): one warp per row, rows taken in launch
// order from a ticket.  The warp sums the row's 9 neighbour-row offsets into
// shared memory (k_row_csum's sums), lane 0 counts the row's units, a
// decoupled look-back over the rows before it (tile_lookback, one word per
// row holding its unit count) gives the row's first unit, and lane 0 writes
// the units.  The warp of the last row writes the total and rearms the
// ticket and the epoch: its look-back ended on a prefix, so every row has
// taken its ticket and read the epoch by then.  A look-back that gave up
// leaves a partial prefix, never above the true one, so every write stays
// inside the unit array.
constexpr uint32_t kFusedRows = 8192;
constexpr int kFusedNcx = 1023;
constexpr int kFusedWarps = 4;
constexpr uint32_t kRowSpinLimit = 1u << 20;   // polls of a row's look-back

// Self-test of the failure path: one warp runs the look-back of row 1
// against a row 0 whose word stays zero (never published), so the wait gives
// up after `limit` polls.
__global__ void k_row_lookback_selftest(const unsigned long long* zeroed, uint32_t limit,
                                        uint32_t* err) {
    tile_lookback(zeroed, 1u, 1u, limit, err);
}

__global__ void __launch_bounds__(kFusedWarps * 32) k_units_fused(const Dev d,
                                                                   const uint32_t* __restrict__ off,
                                                                   const UnitsFusedArgs a) {
    pdl_wait();
    __shared__ uint32_t s_cs[kFusedWarps][kFusedNcx + 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (blockIdx.x * kFusedWarps + w >= d.nrows) return;   // exactly nrows tickets
    uint32_t r = 0, ep = 0;
    if (lane == 0) {
        r = atomicAdd(a.ctl, 1u);
        ep = *reinterpret_cast<volatile uint32_t*>(a.ctl + 1) & 0x3fffffffu;
    }
    r = __shfl_sync(kFull, r, 0);
    ep = __shfl_sync(kFull, ep, 0);
    const Inst& I = d.inst[find_instance(d.row_base, d.n_inst, r)];
    const int ncx = I.ncx;
    const uint32_t lr = r - I.row_base;
    const int cy = (int)(lr % (uint32_t)I.ncy), cz = (int)(lr / (uint32_t)I.ncy);
    uint32_t* cs = s_cs[w];
    for (int x = lane; x <= ncx; x += 32) {
        uint32_t t = 0;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int yy = cy + k % 3 - 1, zz = cz + k / 3 - 1;
            if (yy >= 0 && yy < I.ncy && zz >= 0 && zz < I.ncz)
                t += __ldg(off + I.cell_base +
                           ((size_t)zz * (uint32_t)I.ncy + (uint32_t)yy) * (uint32_t)ncx + x);
        }
        cs[x] = t;
    }
    __syncwarp();
    uint32_t n = 0;
    if (lane == 0) n = unit_walk<0, true>(d, off, cs, r, 0u, nullptr);
    n = __shfl_sync(kFull, n, 0);
    const unsigned long long tag = (unsigned long long)ep << 34;
    uint32_t excl = 0;
    if (r > 0) {
        if (lane == 0) st_relaxed64(a.words + r, tag | (1ull << 32) | n);
        excl = tile_lookback(a.words, r, ep, kRowSpinLimit, a.err);
    }
    if (lane == 0) {
        st_relaxed64(a.words + r, tag | (2ull << 32) | (excl + n));
        unit_walk<1, true>(d, off, cs, r, excl, a.units);
        if (r == d.nrows - 1) {
            *a.total = excl + n;
            a.ctl[0] = 0u;
            a.ctl[1] = ep + 1u;
        }
    }
}

// Symplectic predictor (half step) for sorted particle k, then its new
// label.  Boundary particles keep r and v (Sec. 2.3); excluded particles
// (k >= in-domain count) are left untouched.  Each particle uses its
// instance's step size (0 once the instance is done).
__global__ void __launch_bounds__(256) k_predict(const Dev d, const IntegrateArgs a) {
    pdl_wait();
    __shared__ uint32_t s_hist[4 * 256];
    zero_hist(s_hist);
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = k < d.n;
    uint32_t key = 0;
    if (valid) {
        const uint32_t n_in = a.off[d.ncells];
        double x = a.x[k], y = a.y[k], z = a.z[k];
        float4 vr = a.velrhop[k];
        a.px[k] = x;
        a.py[k] = y;
        a.pz[k] = z;
        a.pvr[k] = vr;
        key = d.ncells;
        if (k < n_in) {
            const uint32_t id = a.id[k];
            const uint32_t q = find_instance(d.id_base, d.n_inst, id);
            const Inst& I = d.inst[q];
            const float hdt = (float)(0.5 * d.is.dt[q]);
            const float4 ac = a.ace[k];
            if (id >= I.id_fluid) {
                x += (double)(hdt * vr.x);
                y += (double)(hdt * vr.y);
                z += (double)(hdt * vr.z);
                vr.x = fmaf(hdt, ac.x, vr.x);
                vr.y = fmaf(hdt, ac.y, vr.y);
                vr.z = fmaf(hdt, ac.z, vr.z);
                a.x[k] = x;
                a.y[k] = y;
                a.z[k] = z;
            }
            vr.w = fmaf(hdt, ac.w, vr.w);
            a.velrhop[k] = vr;
            key = cell_key(d, I, x, y, z);
        }
        a.key[k] = key;
    }
    count_key(valid, key, a.cnt, s_hist, a.passes, bits_for(d.ncells));
    flush_hist(s_hist, a.hist, a.passes);
}

// Symplectic corrector from the start state (pre arrays, reordered like the
// current state) and the half-step rates, then the new label.  Threads
// k < n_inst also advance instance k's time and step count.
__global__ void __launch_bounds__(256) k_correct(const Dev d, const IntegrateArgs a) {
    pdl_wait();
    __shared__ uint32_t s_hist[4 * 256];
    zero_hist(s_hist);
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = k < d.n;
    uint32_t key = 0;
    if (valid) {
        const uint32_t n_in = a.off[d.ncells];
        key = d.ncells;
        if (k < n_in) {
            const uint32_t id = a.id[k];
            const uint32_t q = find_instance(d.id_base, d.n_inst, id);
            const Inst& I = d.inst[q];
            const double dt = d.is.dt[q];
            const float dtf = (float)dt;
            const float hdt = (float)(0.5 * dt);
            double x = a.x[k], y = a.y[k], z = a.z[k];
            const float4 ac = a.ace[k];
            const float4 pv = a.pvr[k];
            float4 vr = a.velrhop[k];
            if (id >= I.id_fluid) {
                const float ux = fmaf(dtf, ac.x, pv.x);
                const float uy = fmaf(dtf, ac.y, pv.y);
                const float uz = fmaf(dtf, ac.z, pv.z);
                x = a.px[k] + (double)(hdt * (ux + pv.x));
                y = a.py[k] + (double)(hdt * (uy + pv.y));
                z = a.pz[k] + (double)(hdt * (uz + pv.z));
                a.x[k] = x;
                a.y[k] = y;
                a.z[k] = z;
                vr.x = ux;
                vr.y = uy;
                vr.z = uz;
            }
            const float eps = -(ac.w * dtf) / vr.w;
            vr.w = pv.w * ((2.f - eps) / (2.f + eps));
            a.velrhop[k] = vr;
            key = cell_key(d, I, x, y, z);
        }
        a.key[k] = key;
    }
    if (k < d.n_inst && !d.is.done[k]) {
        const double t = d.is.t[k] + d.is.dt[k];
        d.is.t[k] = t;
        d.is.steps[k] += 1ull;
        if (t >= d.inst[k].t_end) d.is.done[k] = 1u;
    }
    count_key(valid, key, a.cnt, s_hist, a.passes, bits_for(d.ncells));
    flush_hist(s_hist, a.hist, a.passes);
}

// Verlet step of Sec. 3.3 (the SPHysics form) for sorted particle k, from
// the rates at S^n and (v, rho) one step earlier (a.pvr, sorted like the
// state), then the new label:
//   fluid:   r1 = r + dt v + dt^2/2 a (increment in FP32, r in FP64)
//            v1 = v_prev + 2 dt a   (leapfrog) | v + dt a   (Euler step)
//   all:     rho1 = rho_prev + 2 dt drho       | rho + dt drho
// The member's Verlet phase picks the Euler step (phase 0).  a.pvr_out
// receives the (v, rho) on entry.  Members that are done (dt = 0) and
// excluded particles keep their state.
__global__ void __launch_bounds__(256) k_verlet(const Dev d, const IntegrateArgs a) {
    pdl_wait();
    __shared__ uint32_t s_hist[4 * 256];
    zero_hist(s_hist);
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = k < d.n;
    uint32_t key = 0;
    if (valid) {
        const uint32_t n_in = a.off[d.ncells];
        key = d.ncells;
        if (k < n_in) {
            const uint32_t id = a.id[k];
            const uint32_t q = find_instance(d.id_base, d.n_inst, id);
            const Inst& I = d.inst[q];
            const double dt = d.is.dt[q];
            double x = a.x[k], y = a.y[k], z = a.z[k];
            const float4 vr = a.velrhop[k];
            if (dt > 0.0) {
                const bool euler = d.is.vphase[q] == 0u;
                const float4 pv = euler ? vr : a.pvr[k];
                const float dtf = (float)dt;
                const float dtv = euler ? dtf : (float)(2.0 * dt);
                const float hdt2 = (float)(0.5 * dt * dt);
                const float4 ac = a.ace[k];
                float4 nv = vr;
                if (id >= I.id_fluid) {
                    x += (double)fmaf(hdt2, ac.x, dtf * vr.x);
                    y += (double)fmaf(hdt2, ac.y, dtf * vr.y);
                    z += (double)fmaf(hdt2, ac.z, dtf * vr.z);
                    a.x[k] = x;
                    a.y[k] = y;
                    a.z[k] = z;
                    nv.x = fmaf(dtv, ac.x, pv.x);
                    nv.y = fmaf(dtv, ac.y, pv.y);
                    nv.z = fmaf(dtv, ac.z, pv.z);
                }
                nv.w = fmaf(dtv, ac.w, pv.w);
                a.velrhop[k] = nv;
                a.pvr_out[k] = vr;
            }
            key = cell_key(d, I, x, y, z);
        }
        a.key[k] = key;
    }
    count_key(valid, key, a.cnt, s_hist, a.passes, bits_for(d.ncells));
    flush_hist(s_hist, a.hist, a.passes);
}

// After k_verlet: each running member's time, step count and Verlet phase
// (0 again after verlet_every steps) advance.
__global__ void __launch_bounds__(256) k_verlet_advance(const Dev d) {
    pdl_wait();
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < d.n_inst && !d.is.done[q]) {
        const double t = d.is.t[q] + d.is.dt[q];
        d.is.t[q] = t;
        d.is.steps[q] += 1ull;
        const uint32_t ph = d.is.vphase[q] + 1u;
        d.is.vphase[q] = ph >= d.verlet_every ? 0u : ph;
        if (t >= d.inst[q].t_end) d.is.done[q] = 1u;
    }
}

// Neighbour counts with the FP64 predicate (dx*dx + dy*dy) + dz*dz < (2h)^2,
// every operation rounded as written.
__global__ void __launch_bounds__(256) k_counts_fp64(const Dev d, const double* __restrict__ x,
                                                     const double* __restrict__ y,
                                                     const double* __restrict__ z,
                                                     const uint32_t* __restrict__ key,
                                                     const uint32_t* __restrict__ off,
                                                     uint32_t* __restrict__ out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    const uint32_t n_in = off[d.ncells];
    if (i >= n_in) {
        out[i] = 0;
        return;
    }
    const uint32_t k = key[i];
    const Inst& I = d.inst[find_instance(d.cell_base, d.n_inst, k)];
    const uint32_t lk = k - I.cell_base;
    const int cx = (int)(lk % (uint32_t)I.ncx);
    const uint32_t t = lk / (uint32_t)I.ncx;
    const int cy = (int)(t % (uint32_t)I.ncy), cz = (int)(t / (uint32_t)I.ncy);
    const double xi = x[i], yi = y[i], zi = z[i];
    const int xlo = cx > 0 ? cx - 1 : 0, xhi = cx + 1 < I.ncx ? cx + 1 : I.ncx - 1;
    uint32_t c = 0;
    for (int zz = cz - 1; zz <= cz + 1; ++zz) {
        if (zz < 0 || zz >= I.ncz) continue;
        for (int yy = cy - 1; yy <= cy + 1; ++yy) {
            if (yy < 0 || yy >= I.ncy) continue;
            const uint32_t rb =
                I.cell_base + (uint32_t)I.ncx * ((uint32_t)yy + (uint32_t)I.ncy * zz);
            const uint32_t s = off[rb + xlo], e = off[rb + xhi + 1];
            for (uint32_t j = s; j < e; ++j) {
                if (j == i) continue;
                const double dx = __dsub_rn(xi, x[j]);
                const double dy = __dsub_rn(yi, y[j]);
                const double dz = __dsub_rn(zi, z[j]);
                const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                                            __dmul_rn(dz, dz));
                c += d2 < d.r2max_d;
            }
        }
    }
    out[i] = c;
}

// FP64 conservation sums, per block in a fixed order, then combined in block
// order by one block.
__global__ void __launch_bounds__(256) k_diag_part(const Dev d, const double* __restrict__ x,
                                                   const double* __restrict__ y,
                                                   const double* __restrict__ z,
                                                   const float4* __restrict__ vr,
                                                   const uint32_t* __restrict__ id,
                                                   const uint32_t* __restrict__ off,
                                                   double* __restrict__ part) {
    __shared__ double s[256][8];
    const uint32_t n_in = off[d.ncells];
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const double m = d.mass_d;
    const double rho0 = d.rho0_d;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < d.n; k += gridDim.x * blockDim.x) {
        if (k >= n_in) {
            acc[7] += 1.0;
            continue;
        }
        const uint32_t pid = id[k];
        const Inst& I = d.inst[find_instance(d.id_base, d.n_inst, pid)];
        const float4 v = vr[k];
        const double rho = v.w;
        const double B = I.B_d;
        acc[0] += m;
        // e(rho) = B [ ((rho/rho0)^6 - 1) / (6 rho0) + 1/rho - 1/rho0 ]
        const double rr = rho / rho0, r2 = rr * rr, r6 = r2 * r2 * r2;
        acc[6] += m * B * ((r6 - 1.0) / (6.0 * rho0) + 1.0 / rho - 1.0 / rho0);
        if (pid >= I.id_fluid) {
            acc[1] += m * v.x;
            acc[2] += m * v.y;
            acc[3] += m * v.z;
            acc[4] += 0.5 * m * ((double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z);
            acc[5] -= m * (d.g_d[0] * x[k] + d.g_d[1] * y[k] + d.g_d[2] * z[k]);
        }
    }
    for (int q = 0; q < 8; ++q) s[threadIdx.x][q] = acc[q];
    __syncthreads();
    for (int st = 128; st; st >>= 1) {
        if (threadIdx.x < st)
            for (int q = 0; q < 8; ++q) s[threadIdx.x][q] += s[threadIdx.x + st][q];
        __syncthreads();
    }
    if (threadIdx.x < 8) part[blockIdx.x * 8 + threadIdx.x] = s[0][threadIdx.x];
}

__global__ void k_diag_final(const double* __restrict__ part, int nparts, double* __restrict__ out) {
    if (threadIdx.x >= 8) return;
    double a = 0.0;
    for (int b = 0; b < nparts; ++b) a += part[b * 8 + threadIdx.x];
    out[threadIdx.x] = a;
}

// Free-surface front (the front position of the dam-break results): per
// instance, the largest x of the in-domain fluid particles with zlo <= z <
// zhi.  Maxima are kept as order-preserving 64-bit images of the FP64 x (a
// maximum does not depend on the order of the updates); 0 stands for "no
// particle".  Each thread folds its particles of one instance before an
// atomic, and a warp whose lanes agree on the instance folds once more.
__device__ __forceinline__ unsigned long long ordered_bits(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

__global__ void __launch_bounds__(256) k_front(const Dev d, const double* __restrict__ x,
                                               const double* __restrict__ z,
                                               const uint32_t* __restrict__ id,
                                               const uint32_t* __restrict__ off, double zlo,
                                               double zhi, unsigned long long* __restrict__ out) {
    const uint32_t n_in = off[d.ncells];
    uint32_t qc = 0xffffffffu;
    unsigned long long best = 0;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n_in; k += gridDim.x * blockDim.x) {
        const double zk = z[k];
        if (!(zk >= zlo && zk < zhi)) continue;
        const uint32_t pid = id[k];
        const uint32_t q = find_instance(d.id_base, d.n_inst, pid);
        if (pid < d.inst[q].id_fluid) continue;
        if (q != qc) {
            if (best) atomicMax(out + qc, best);
            qc = q;
            best = 0;
        }
        const unsigned long long b = ordered_bits(x[k]);
        best = b > best ? b : best;
    }
    const uint32_t q0 = __shfl_sync(kFull, qc, 0);
    if (__all_sync(kFull, qc == q0 || best == 0)) {
        for (int o = 16; o; o >>= 1) {
            const unsigned long long t = __shfl_xor_sync(kFull, best, o);
            best = t > best ? t : best;
        }
        if ((threadIdx.x & 31) == 0 && best) atomicMax(out + q0, best);
    } else if (best) {
        atomicMax(out + qc, best);
    }
}

// Device-side step loop (sph_step): the conditional WHILE node of the step
// graph runs its body (`body` steps) again while k_loop_ctrl leaves its
// condition at 1.  k_loop_init arms the counter before each launch.
__global__ void k_loop_init(uint32_t* ctr, uint32_t nsteps) {
    ctr[0] = 0u;
    ctr[1] = nsteps;
}

__global__ void __launch_bounds__(256) k_loop_ctrl(cudaGraphConditionalHandle h, uint32_t* ctr,
                                                   const uint32_t* __restrict__ done,
                                                   uint32_t n_inst, uint32_t body) {
    pdl_wait();
    int running = 0;
    for (uint32_t q = threadIdx.x; q < n_inst; q += blockDim.x) running |= done[q] == 0u;
    running = __syncthreads_or(running);
    if (threadIdx.x == 0) {
        const uint32_t k = ctr[0] + body;
        ctr[0] = k;
        // another body while it fits the steps asked and a member still runs
        cudaGraphSetConditional(h, (running && k + body <= ctr[1]) ? 1u : 0u);
    }
}

inline uint32_t blocks_for(uint32_t n, uint32_t t) { return n ? (n + t - 1) / t : 1; }

}  // namespace

void launch_keys(const Dev& d, const double* x, const double* y, const double* z,
                 const uint32_t* id, uint32_t n, uint32_t* key, uint32_t* cnt, uint32_t* hist,
                 int passes, cudaStream_t st) {
    k_keys<<<blocks_for(n, 256), 256, 0, st>>>(d, x, y, z, id, n, key, cnt, hist, passes);
}

void launch_reorder(const Dev& d, const ReorderArgs& a, cudaStream_t st) {
    launch_pdl(k_reorder, blocks_for(d.n, 256), 256, 0, st, d, a);
}

// Upper bound on the number of units: every unit but the last of its row
// either holds the unit size (at least kMinUnit particles) or closes before a
// non-empty cell (a gap, the span limit or the staging limit), and a row has
// no more such closures than non-empty cells (at most min(n, ncells) in all).
uint32_t max_units(uint32_t n, uint32_t nrows, uint64_t ncells) {
    const uint64_t cells = ncells < n ? ncells : n;
    return (uint32_t)((n + kMinUnit - 1) / kMinUnit + cells + nrows);
}

namespace {

using KernelPtr = void (*)(const Dev, const InteractArgs);

struct Variant {
    int warps;              // warps of particles (the unit is warps x 32 particles)
    int split;              // warps per group of 32 particles
    int stage;              // staged candidates
    KernelPtr fn[2][2];     // [kernel: Wendland C2, cubic spline][with counts]
    size_t smem;
    int grid;   // persistent grid on this GPU (set by prepare_interact)
};

// (warps, staged candidates, hit-mask words per lane, resident blocks per SM
// that the shared memory allows -- also the register budget hint)
#define SPH_VARIANT_D(Wv, Sv, Cv, Bv, Pv, PKv, TUv, Dv)                               \
    Variant {                                                                        \
        Wv, Pv, Sv,                                                                  \
            {{k_interact<Wv, Sv, Cv, Bv, false, Pv, 0, PKv, TUv, Dv>,                \
              k_interact<Wv, Sv, Cv, Bv, true, Pv, 0, PKv, TUv, Dv>},                \
             {k_interact<Wv, Sv, Cv, Bv, false, Pv, 1, PKv, TUv, Dv>,                \
              k_interact<Wv, Sv, Cv, Bv, true, Pv, 1, PKv, TUv, Dv>}},               \
            Shape<Wv * Pv, Sv, Cv>::smem, 0                                          \
    }
#define SPH_VARIANT_T(Wv, Sv, Cv, Bv, Pv, PKv, TUv) \
    SPH_VARIANT_D(Wv, Sv, Cv, Bv, Pv, PKv, TUv, false)
#define SPH_VARIANT(Wv, Sv, Cv, Bv, Pv, PKv) SPH_VARIANT_T(Wv, Sv, Cv, Bv, Pv, PKv, false)

Variant g_variants[kNumVariants] = {
    SPH_VARIANT(4, 2048, 24, 2, 2, false),   // 128-particle units, two warps per 32 particles
    SPH_VARIANT(4, 2048, 32, 2, 1, false),   // 128-particle units
    SPH_VARIANT(3, 1280, 16, 3, 2, false),   // 96-particle units, two warps per 32, three per SM
    SPH_VARIANT(3, 1408, 16, 3, 2, false),
    SPH_VARIANT(2, 1280, 24, 3, 2, false),   // 64-particle units, two warps per 32 particles
    SPH_VARIANT(4, 1792, 20, 2, 2, false),
    SPH_VARIANT(3, 1152, 24, 4, 1, false),   // 96-particle units, four blocks per SM
    // the same shapes with the pair terms of two pairs in packed FP32
    SPH_VARIANT(4, 2048, 24, 2, 2, true),
    SPH_VARIANT(3, 1408, 16, 3, 2, true),
    SPH_VARIANT(4, 1792, 20, 2, 2, true),
    // packed, and the candidate test's first eight pairs of a word unconditional
    SPH_VARIANT_T(4, 2048, 24, 2, 2, true, true),
    SPH_VARIANT_T(3, 1408, 16, 3, 2, true, true),
    // 32-particle units shared by four warps, four blocks per SM: shorter
    // dependent chains per unit for small systems (fewer units than SMs)
    SPH_VARIANT_T(1, 1024, 12, 4, 4, true, true),
    // units taken from a counter, the next unit's record and cell offsets
    // fetched during the current one
    SPH_VARIANT_D(4, 2048, 24, 2, 2, true, true, true),
    SPH_VARIANT_D(3, 1408, 16, 3, 2, true, true, true),
    SPH_VARIANT_D(1, 1024, 12, 4, 4, true, true, true),
};

}  // namespace

int variant_unit(int v) { return g_variants[v].warps * 32; }

int variant_stage(int v) { return g_variants[v].stage; }

// Persistent grid: every resident block of the variant on this GPU.
uint32_t interact_grid(int v) { return (uint32_t)g_variants[v].grid; }

namespace {

__global__ void k_pdl_probe() { pdl_wait(); }

bool g_pdl = false;
std::once_flag g_pdl_once;

// Whether the driver takes programmatic launches inside a captured
// conditional node's body (the device-side step loop): capture two of them
// into a WHILE node whose condition starts at 0 (the body never runs), then
// instantiate and launch the graph.  Every failure here is a host-side error
// code, cleared before returning.
bool probe_pdl() {
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    bool ok = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    do {
        if (cudaGraphCreate(&graph, 0) != cudaSuccess) break;
        cudaGraphConditionalHandle h;
        if (cudaGraphConditionalHandleCreate(&h, graph, 0u, cudaGraphCondAssignDefault) !=
            cudaSuccess)
            break;
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        if (cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np) != cudaSuccess) break;
        cudaGraph_t body = np.conditional.phGraph_out[0];
        if (cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            break;
        g_pdl = true;   // launch_pdl reads it
        const cudaError_t e1 = launch_pdl(k_pdl_probe, 1, 32, 0, s);
        const cudaError_t e2 = launch_pdl(k_pdl_probe, 1, 32, 0, s);
        g_pdl = false;
        const cudaError_t e3 = cudaStreamEndCapture(s, &body);
        if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) break;
        if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) break;
        if (cudaGraphLaunch(exec, s) != cudaSuccess) break;
        if (cudaStreamSynchronize(s) != cudaSuccess) break;
        ok = true;
    } while (false);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(s);
    cudaGetLastError();
    return ok;
}

}  // namespace

bool pdl_enabled() { return g_pdl; }

void prepare_interact() {
    std::call_once(g_pdl_once, [] {
        const char* e = getenv("SPH_PDL");
        const bool want = !(e && e[0] == '0');
        g_pdl = want && probe_pdl();
    });
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (Variant& v : g_variants) {
        for (int k = 0; k < 2; ++k)
            for (int c = 0; c < 2; ++c)
                cudaFuncSetAttribute(v.fn[k][c], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)v.smem);
        // one grid for both kernels of the shape: the smaller residency
        int per_sm = 0;
        for (int k = 0; k < 2; ++k) {
            int r = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, v.fn[k][0], v.warps * v.split * 32,
                                                          v.smem);
            per_sm = k == 0 || r < per_sm ? r : per_sm;
        }
        v.grid = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
    }
}

void launch_interact(const Dev& d, const InteractArgs& a, bool counts, cudaStream_t st) {
    const Variant& v = g_variants[d.variant];
    launch_pdl(v.fn[d.kern == 1 ? 1 : 0][counts ? 1 : 0], v.grid, v.warps * v.split * 32, v.smem,
               st, d, a);
}

void launch_row_lookback_selftest(unsigned long long* zeroed, uint32_t limit, uint32_t* err,
                                  cudaStream_t st) {
    cudaMemsetAsync(zeroed, 0, sizeof(unsigned long long), st);
    k_row_lookback_selftest<<<1, 32, 0, st>>>(zeroed, limit, err);
}

bool units_fit_one_launch(uint32_t nrows, int max_ncx) {
    return nrows <= kFusedRows && max_ncx <= kFusedNcx;
}

bool units_fused(const Dev& d) { return d.units_fused != 0; }

void launch_units(const Dev& d, const uint32_t* off, uint32_t* csum, uint32_t* ucnt,
                  uint32_t* ubsum, uint32_t* uoff, uint2* units, unsigned long long* urow,
                  uint32_t* uctl, uint32_t* err, cudaStream_t st) {
    if (units_fused(d)) {
        const UnitsFusedArgs a = {units, uoff + d.nrows, urow, uctl, err};
        launch_pdl(k_units_fused, (d.nrows + kFusedWarps - 1) / kFusedWarps, kFusedWarps * 32, 0,
                   st, d, off, a);
        return;
    }
    launch_pdl(k_row_csum, d.nrows, 128, 0, st, d, off, csum);
    launch_pdl(k_units<0>, blocks_for(d.nrows, 128), 128, 0, st, d, off, csum, ucnt, uoff, units);
    launch_scan(ucnt, d.nrows, ubsum, uoff, st);
    launch_pdl(k_units<1>, blocks_for(d.nrows, 128), 128, 0, st, d, off, csum, ucnt, uoff, units);
}

void launch_predict(const Dev& d, const IntegrateArgs& a, cudaStream_t st) {
    launch_pdl(k_predict, blocks_for(d.n, 256), 256, 0, st, d, a);
}

void launch_correct(const Dev& d, const IntegrateArgs& a, cudaStream_t st) {
    const uint32_t n = d.n > d.n_inst ? d.n : d.n_inst;
    launch_pdl(k_correct, blocks_for(n, 256), 256, 0, st, d, a);
}

void launch_verlet(const Dev& d, const IntegrateArgs& a, cudaStream_t st) {
    launch_pdl(k_verlet, blocks_for(d.n, 256), 256, 0, st, d, a);
    launch_pdl(k_verlet_advance, blocks_for(d.n_inst, 256), 256, 0, st, d);
}

void launch_counts_fp64(const Dev& d, const double* x, const double* y, const double* z,
                        const uint32_t* key, const uint32_t* off, uint32_t* out,
                        cudaStream_t st) {
    k_counts_fp64<<<blocks_for(d.n, 256), 256, 0, st>>>(d, x, y, z, key, off, out);
}

void launch_diag(const Dev& d, const double* x, const double* y, const double* z,
                 const float4* vr, const uint32_t* id, const uint32_t* off, double* partial,
                 double* out, cudaStream_t st) {
    k_diag_part<<<kDiagBlocks, 256, 0, st>>>(d, x, y, z, vr, id, off, partial);
    k_diag_final<<<1, 32, 0, st>>>(partial, kDiagBlocks, out);
}

void launch_loop_init(uint32_t* ctr, uint32_t nsteps, cudaStream_t st) {
    k_loop_init<<<1, 1, 0, st>>>(ctr, nsteps);
}

void launch_loop_ctrl(cudaGraphConditionalHandle h, uint32_t* ctr, const uint32_t* done,
                      uint32_t n_inst, uint32_t body, cudaStream_t st) {
    launch_pdl(k_loop_ctrl, 1, 256, 0, st, h, ctr, done, n_inst, body);
}

void launch_front(const Dev& d, const double* x, const double* z, const uint32_t* id,
                  const uint32_t* off, double zlo, double zhi, unsigned long long* out,
                  cudaStream_t st) {
    cudaMemsetAsync(out, 0, d.n_inst * sizeof(unsigned long long), st);
    k_front<<<kDiagBlocks, 256, 0, st>>>(d, x, z, id, off, zlo, zhi, out);
}

}  // namespace sph
