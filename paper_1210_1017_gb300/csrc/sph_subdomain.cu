// Sub-domain selection of Sec. 4.2-4.3 on one GPU: the data a sub-domain of
// a one-dimensional decomposition along x sends to its neighbours (the edge
// particles that build their halos, or the particles that migrated), found
// the way the paper does it: a labelling kernel, a radix sort of the
// particles by (label, id), and a copy of the labelled ones.
//
// Only the labelled particles are sorted: the labelling kernel compacts
// them (their slots come from a warp-aggregated counter, so their order is
// arbitrary), a four-pass sort by id and a stable one-pass sort by label then
// give the (label, id) order of the paper's worked example for any 32-bit
// ids.  The state itself keeps its cell order.
#include <string.h>

#include "sph_ctx.cuh"

namespace sph {

namespace {

constexpr uint32_t kFull = 0xffffffffu;
constexpr uint32_t kIdxBits = 26;                     // state index < 2^26
constexpr uint32_t kIdxMask = (1u << kIdxBits) - 1u;

// Order-preserving integer image of a finite double: a < b exactly when
// ordered(a) < ordered(b), with -0 and +0 both 0.  The labels compare these
// on the integer pipe (GB300 issues FP64 instructions at 1/64 of the FP32
// rate, which would bound this pass instead of HBM).
__host__ __device__ __forceinline__ long long ordered(long long bits) {
    const long long mag = bits & 0x7fffffffffffffffLL;
    return bits < 0 ? -mag : mag;
}

struct SubLabelArgs {
    const double* x;
    const uint32_t* id;
    const uint32_t* off;      // cell offsets: off[ncells] = in-domain count
    uint32_t ncells, n;
    int mode;
    long long xlo, xhi, lo_edge, hi_edge;   // ordered images of the bounds
    uint32_t* key;            // id of each selected particle
    uint32_t* val;            // (label << 26) | state index
    uint32_t* cnt;            // [0] in-domain count, [1..2] per label, [3] selected
};

// Label of state entry k (in-domain entries k < off[ncells] only).  Only
// warps holding labelled particles touch the counters (label 0 is the rest
// of the in-domain count), so the pass stays a read of x.
__global__ void __launch_bounds__(256) k_sub_label(const SubLabelArgs a) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t l = 0;
    if (k < a.n) {
        const uint32_t n_in = a.off[a.ncells];
        if (k == 0) a.cnt[0] = n_in;
        if (k < n_in) {
            const long long x = ordered(__double_as_longlong(a.x[k]));
            if (a.mode == SPH_SUBDOMAIN_EDGE) {
                if (x >= a.xlo && x < a.lo_edge) l = 1;
                else if (x >= a.hi_edge && x < a.xhi) l = 2;
            } else {
                if (x < a.xlo) l = 1;
                else if (x >= a.xhi) l = 2;
            }
        }
    }
    const uint32_t m1 = __ballot_sync(kFull, l == 1u);
    const uint32_t m2 = __ballot_sync(kFull, l == 2u);
    const uint32_t sel = m1 | m2;
    if (sel == 0u) return;                       // warp-uniform
    uint32_t base = 0;
    if (lane == 0) {
        if (m1) atomicAdd(a.cnt + 1, __popc(m1));
        if (m2) atomicAdd(a.cnt + 2, __popc(m2));
        base = atomicAdd(a.cnt + 3, __popc(sel));
    }
    base = __shfl_sync(kFull, base, 0);
    if (l != 0u) {
        const uint32_t slot = base + __popc(sel & ((1u << lane) - 1u));
        a.key[slot] = a.id[k];
        a.val[slot] = (l << kIdxBits) | k;
    }
}

// Keys and values of the second (label) sort from the id-sorted pairs.
__global__ void __launch_bounds__(256) k_sub_relabel(const uint32_t* __restrict__ val_in,
                                                     uint32_t m, uint32_t* __restrict__ key_out,
                                                     uint32_t* __restrict__ val_out) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m) {
        const uint32_t v = val_in[t];
        key_out[t] = v >> kIdxBits;
        val_out[t] = v & kIdxMask;
    }
}

// Copy of the selected particles' state in the sorted order.
__global__ void __launch_bounds__(256) k_sub_gather(const uint32_t* __restrict__ sidx, uint32_t m,
                                                    const double* __restrict__ x,
                                                    const double* __restrict__ y,
                                                    const double* __restrict__ z,
                                                    const float4* __restrict__ vr,
                                                    const uint32_t* __restrict__ id,
                                                    double* __restrict__ pos3,
                                                    float* __restrict__ vel3,
                                                    float* __restrict__ rho,
                                                    uint32_t* __restrict__ ids) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m) {
        const uint32_t k = sidx[t];
        pos3[3 * (size_t)t + 0] = x[k];
        pos3[3 * (size_t)t + 1] = y[k];
        pos3[3 * (size_t)t + 2] = z[k];
        const float4 v = vr[k];
        vel3[3 * (size_t)t + 0] = v.x;
        vel3[3 * (size_t)t + 1] = v.y;
        vel3[3 * (size_t)t + 2] = v.z;
        rho[t] = v.w;
        ids[t] = id[k];
    }
}

inline uint32_t blocks256(uint32_t n) { return n ? (n + 255u) / 256u : 1u; }

}  // namespace

}  // namespace sph

using namespace sph;

extern "C" int sph_subdomain_select(sph_ctx* c, int mode, double xlo, double xhi,
                                    uint32_t* counts, uint32_t capacity, double* pos, float* vel,
                                    float* rho, uint32_t* ids) {
    const TraceRange trace("sph_subdomain_select");
    if (!c) return SPH_ERR_INVALID_ARG;
    if (!counts) return fail(c, SPH_ERR_INVALID_ARG, "NULL counts");
    if (mode != SPH_SUBDOMAIN_EDGE && mode != SPH_SUBDOMAIN_MIGRATE)
        return fail(c, SPH_ERR_INVALID_ARG, "unknown sub-domain mode");
    if (!(xhi > xlo)) return fail(c, SPH_ERR_INVALID_ARG, "empty sub-domain");
    const double cs = 2.0 * c->p.h;
    if (mode == SPH_SUBDOMAIN_EDGE && !(xhi - xlo >= 2.0 * cs))
        return fail(c, SPH_ERR_INVALID_ARG, "sub-domain narrower than its two edges (4h)");
    if (c->n_inst != 1) return fail(c, SPH_ERR_STATE, "sub-domains of a single simulation only");
    if (!c->have_state || !c->cells_valid) return fail(c, SPH_ERR_STATE, "cells not built");
    cudaStream_t st = c->st;
    const uint32_t n = c->n;

    SubLabelArgs la;
    la.x = c->x[c->cur];
    la.id = c->id[c->cur];
    la.off = c->off;
    la.ncells = (uint32_t)c->ncells;
    la.n = n;
    la.mode = mode;
    // xlo + 2h and xhi - 2h rounded once in FP64, then mapped
    const double bounds[4] = {xlo, xhi, xlo + cs, xhi - cs};
    long long ob[4];
    for (int i = 0; i < 4; ++i) {
        long long b;
        memcpy(&b, &bounds[i], sizeof(b));
        ob[i] = ordered(b);
    }
    la.xlo = ob[0];
    la.xhi = ob[1];
    la.lo_edge = ob[2];
    la.hi_edge = ob[3];
    la.key = c->sub_key[0];
    la.val = c->sub_val[0];
    la.cnt = c->sub_cnt;
    cudaMemsetAsync(c->sub_cnt, 0, 4 * sizeof(uint32_t), st);
    k_sub_label<<<blocks256(n), 256, 0, st>>>(la);
    int rc = cuda_check(c, cudaGetLastError(), "sub-domain labels");
    if (rc) return rc;
    uint32_t cnt[4] = {0, 0, 0, 0};
    cudaMemcpyAsync(cnt, c->sub_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, st);
    rc = cuda_check(c, cudaStreamSynchronize(st), "sub-domain counts");
    if (rc) return rc;
    counts[0] = cnt[0] - cnt[1] - cnt[2];
    counts[1] = cnt[1];
    counts[2] = cnt[2];
    const uint32_t m = cnt[3];
    if (m > capacity) return fail(c, SPH_ERR_CAPACITY, "output capacity below the selected count");
    if (m == 0) return SPH_OK;

    // sort A: by id (32 bits, 4 passes); sort B: stable by label (1 pass)
    const uint32_t tiles = os_tiles(m);
    uint32_t* ctr = c->sub_os;                 // 5 tile counters
    uint32_t* status = c->sub_os + 5;          // 5 passes x tiles x 256
    cudaMemsetAsync(c->sub_hist, 0, 5 * 256 * sizeof(uint32_t), st);
    cudaMemsetAsync(c->sub_os, 0, (5 + (size_t)5 * tiles * 256) * sizeof(uint32_t), st);
    launch_digit_hist(c->sub_key[0], m, 4, 32, c->sub_hist, st);
    int src = 0;
    for (int p = 0; p < 4; ++p) {
        launch_onesweep_pass(c->sub_key[src], c->sub_val[src], c->sub_key[1 - src],
                             c->sub_val[1 - src], m, p, 32, c->sub_hist, status, ctr, c->status,
                             st);
        src = 1 - src;
    }
    // after four passes the pairs are back in [0]
    k_sub_relabel<<<blocks256(m), 256, 0, st>>>(c->sub_val[0], m, c->sub_key[1], c->sub_val[1]);
    launch_digit_hist(c->sub_key[1], m, 1, 2, c->sub_hist + 4 * 256, st);
    launch_onesweep_pass(c->sub_key[1], c->sub_val[1], c->sub_key[0], c->sub_val[0], m, 0, 2,
                         c->sub_hist + 4 * 256, status + (size_t)4 * tiles * 256, ctr + 4,
                         c->status, st);
    // gather into the transfer staging (ids into the free key buffer)
    double* spos = c->stage_pos;
    float* svel = c->stage_vr;
    float* srho = c->stage_vr + 3 * (size_t)n;
    uint32_t* sids = c->sub_key[1];
    k_sub_gather<<<blocks256(m), 256, 0, st>>>(c->sub_val[0], m, c->x[c->cur], c->y[c->cur],
                                               c->z[c->cur], c->vr[c->cur], c->id[c->cur], spos,
                                               svel, srho, sids);
    rc = cuda_check(c, cudaGetLastError(), "sub-domain sort and gather");
    if (rc) return rc;
    // cudaMemcpyDefault: host or device destinations (unified addressing)
    if (pos) cudaMemcpyAsync(pos, spos, 3 * (size_t)m * sizeof(double), cudaMemcpyDefault, st);
    if (vel) cudaMemcpyAsync(vel, svel, 3 * (size_t)m * sizeof(float), cudaMemcpyDefault, st);
    if (rho) cudaMemcpyAsync(rho, srho, (size_t)m * sizeof(float), cudaMemcpyDefault, st);
    if (ids) cudaMemcpyAsync(ids, sids, (size_t)m * sizeof(uint32_t), cudaMemcpyDefault, st);
    return cuda_check(c, cudaStreamSynchronize(st), "sub-domain copy");
}
