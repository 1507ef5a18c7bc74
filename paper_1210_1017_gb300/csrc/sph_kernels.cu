// Per-step kernels of the weakly compressible SPH hot path on sm_103a:
// cell labels, reorder with the id tie-break, the 27-cell pair interaction
// (Eqs. 7 and 9 with the Tait law and artificial viscosity of Sec. 2.2),
// the CFL reductions (Sec. 3.3), the symplectic predictor/corrector, FP64
// neighbour counts and FP64 conservation sums.
#include <math.h>

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

// Sec. 3.1 cell label: floor((x - x0) * (1/(2h))) per axis in FP64, each
// operation rounded as written; label = cx + ncx (cy + ncy cz).  Outside the
// grid (or non-finite) -> ncells.
__device__ __forceinline__ uint32_t cell_key(const Dev& d, double x, double y, double z) {
    const double tx = __dmul_rn(__dsub_rn(x, d.x0), d.inv_cs);
    const double ty = __dmul_rn(__dsub_rn(y, d.y0), d.inv_cs);
    const double tz = __dmul_rn(__dsub_rn(z, d.z0), d.inv_cs);
    const bool in = (tx >= 0.0) && (tx < (double)d.ncx) && (ty >= 0.0) &&
                    (ty < (double)d.ncy) && (tz >= 0.0) && (tz < (double)d.ncz);
    if (!in) return d.ncells;
    const int cx = __double2int_rd(tx), cy = __double2int_rd(ty), cz = __double2int_rd(tz);
    return (uint32_t)cx + (uint32_t)d.ncx * ((uint32_t)cy + (uint32_t)d.ncy * (uint32_t)cz);
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
                                              const double* __restrict__ z, uint32_t n,
                                              uint32_t* __restrict__ key, uint32_t* cnt,
                                              uint32_t* hist, int passes) {
    __shared__ uint32_t s_hist[4 * 256];
    zero_hist(s_hist);
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < n;
    uint32_t k = 0;
    if (valid) {
        k = cell_key(d, x[i], y[i], z[i]);
        key[i] = k;
    }
    count_key(valid, k, cnt, s_hist, passes, bits_for(d.ncells));
    flush_hist(s_hist, hist, passes);
}

// Tait pressure over density squared, P = B [(rho/rho0)^7 - 1] / rho^2, in
// FP32.  (rho/rho0)^7 - 1 is expanded in x = (rho - rho0)/rho0 so that it
// keeps its relative accuracy near the free surface, where it cancels.
__device__ __forceinline__ float p_over_rho2(const Dev& d, float rho) {
    const float x = (rho - d.rho0) * d.inv_rho0;
    const float poly =
        x * (7.f + x * (21.f + x * (35.f + x * (35.f + x * (21.f + x * (7.f + x))))));
    return d.B * poly / (rho * rho);
}

constexpr uint32_t kMaxSeg = 4096;   // largest cell the id tie-break handles

// Sec. 3.1 reorder.  Thread k takes the k-th pair of the radix sort (stable
// by the previous order), ranks its particle by id among the particles of
// the same cell, and moves the particle's state to (cell start + rank): the
// result is ordered by (label, id) whatever the previous order was.  Also
// writes the FP32 position relative to the cell's origin and P = p/rho^2.
__global__ void __launch_bounds__(256) k_reorder(const Dev d, const ReorderArgs a) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool valid = k < d.n;
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) a.hist_to_zero[i] = 0;
    uint32_t c = 0, v = 0, myid = 0, s = 0, e = 0;
    if (valid) {
        c = a.skey[k];
        v = a.sval[k];
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
        a.dpvr[dst] = a.spvr[v];
    }
    float4 pc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (c < d.ncells) {
        const uint32_t cx = c % (uint32_t)d.ncx;
        const uint32_t t = c / (uint32_t)d.ncx;
        const uint32_t cy = t % (uint32_t)d.ncy;
        const uint32_t cz = t / (uint32_t)d.ncy;
        pc.x = __double2float_rn(x - (d.x0 + (double)cx * d.cs));
        pc.y = __double2float_rn(y - (d.y0 + (double)cy * d.cs));
        pc.z = __double2float_rn(z - (d.z0 + (double)cz * d.cs));
        pc.w = p_over_rho2(d, vr.w);
    }
    a.posc[dst] = pc;
}

// ----------------------------------------------------------- interaction --

constexpr int kIWarps = 4;          // warps per block
constexpr int kCap = 96;            // neighbour-list slots per lane
constexpr uint32_t kIdxMask = (1u << 26) - 1;

// Sec. 3.2.  Each warp owns 32 consecutive (sorted) particles i.  For the
// lanes that share a row of cells (same cy, cz) it walks the 9 neighbouring
// rows; in each row the cells [min cx - 1, max cx + 1] are contiguous in the
// sorted arrays.  Phase 1 tests every candidate j (one load, broadcast to
// all lanes) against each lane's particle and appends hits (|r_ij| < 2h) to
// the lane's list in shared memory, tagged with the cell offset between i
// and j.  Phase 2 walks the lists with all lanes busy and accumulates the
// pair terms of Eqs. 7 and 9.  Distances use positions relative to each
// particle's own cell origin plus whole-cell offsets, in FP32.
template <bool COUNTS>
__global__ void __launch_bounds__(kIWarps * 32) k_interact(const Dev d, const InteractArgs a) {
    extern __shared__ uint32_t s_dyn[];
    __shared__ float s_rf[kIWarps][3];
    __shared__ uint32_t s_ru[kIWarps][4];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t* lst = s_dyn + w * (kCap * 32);
    const uint32_t n_in = a.off[d.ncells];
    const uint32_t i = (blockIdx.x * kIWarps + w) * 32 + lane;
    const bool valid = i < n_in;

    float4 pi = make_float4(0.f, 0.f, 0.f, 0.f), vi = make_float4(0.f, 0.f, 0.f, 1.f);
    int cx = 0, cy = 0, cz = 0;
    bool fluid = false;
    if (valid) {
        pi = a.posc[i];
        vi = a.velrhop[i];
        const uint32_t k = a.key[i];
        cx = (int)(k % (uint32_t)d.ncx);
        const uint32_t t = k / (uint32_t)d.ncx;
        cy = (int)(t % (uint32_t)d.ncy);
        cz = (int)(t / (uint32_t)d.ncy);
        fluid = a.id[i] >= d.n_bound;
    }
    const float rri = vi.w * d.inv_rho0;
    const float ci = d.c0 * rri * rri * rri;
    float ax = 0.f, ay = 0.f, az = 0.f, dr = 0.f, mu = 0.f;
    uint32_t cnt = 0, npairs = 0, nbpairs = 0, ncand = 0;

    auto flush = [&]() {
        const uint32_t mx = __reduce_max_sync(kFull, cnt);
        for (uint32_t t = 0; t < mx; ++t) {
            if (t < cnt) {
                const uint32_t e = lst[t * 32 + lane];
                const uint32_t j = e & kIdxMask;
                const float ox = (float)((int)((e >> 26) & 3u) - 1);
                const float oy = (float)((int)((e >> 28) & 3u) - 1);
                const float oz = (float)((int)(e >> 30) - 1);
                const float4 pj = __ldg(a.posc + j);
                const float4 vj = __ldg(a.velrhop + j);
                const float dx = fmaf(ox, d.csf, pi.x) - pj.x;
                const float dy = fmaf(oy, d.csf, pi.y) - pj.y;
                const float dz = fmaf(oz, d.csf, pi.z) - pj.z;
                const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                // Wendland C2: grad_i W = F r_ij, F = -5 aD/h^2 (1 - q/2)^3
                const float q = sqrt_approx(d2) * d.inv_h;
                const float wq = fmaf(-0.5f, q, 1.0f);
                const float F = d.fc * (wq * wq * wq);
                const float dvx = vi.x - vj.x, dvy = vi.y - vj.y, dvz = vi.z - vj.z;
                const float vr = fmaf(dvx, dx, fmaf(dvy, dy, dvz * dz));
                dr = fmaf(vr, F, dr);                                  // Eq. 7
                if (fluid) {
                    // boundary particles never move (Sec. 2.3): their
                    // acceleration is not needed
                    const float nu = d.h * vr * rcp_approx(d2 + d.eta2);   // Sec. 2.2
                    const float rrj = vj.w * d.inv_rho0;
                    const float cj = d.c0 * rrj * rrj * rrj;
                    const float visc =
                        vr < 0.f ? -d.alpha * (ci + cj) * nu * rcp_approx(vi.w + vj.w) : 0.f;
                    const float s = (pi.w + pj.w + visc) * F;              // Eq. 9
                    ax = fmaf(-s, dx, ax);
                    ay = fmaf(-s, dy, ay);
                    az = fmaf(-s, dz, az);
                    mu = fmaxf(mu, fabsf(nu));
                    ++npairs;
                } else {
                    ++nbpairs;
                }
            }
        }
        cnt = 0;
    };

    uint32_t todo = __ballot_sync(kFull, valid);
    while (todo) {
        const int leader = __ffs(todo) - 1;
        const int myrow = cy + d.ncy * cz;
        const int row = __shfl_sync(kFull, myrow, leader);
        const bool inrow = valid && myrow == row;
        todo &= ~__ballot_sync(kFull, inrow);
        const int xmin = __reduce_min_sync(kFull, inrow ? cx : 0x7fffffff);
        const int xmax = __reduce_max_sync(kFull, inrow ? cx : -1);
        const int rcy = row % d.ncy, rcz = row / d.ncy;
        const int xlo = xmin > 0 ? xmin - 1 : 0;
        const int xhi = xmax + 1 < d.ncx ? xmax + 1 : d.ncx - 1;
        for (int zz = rcz - 1; zz <= rcz + 1; ++zz) {
            if (zz < 0 || zz >= d.ncz) continue;
            for (int yy = rcy - 1; yy <= rcy + 1; ++yy) {
                if (yy < 0 || yy >= d.ncy) continue;
                const uint32_t rbase = (uint32_t)d.ncx * ((uint32_t)yy + (uint32_t)d.ncy * zz);
                const float qy = fmaf((float)(cy - yy), d.csf, pi.y);
                const float qz = fmaf((float)(cz - zz), d.csf, pi.z);
                const uint32_t code_yz =
                    ((uint32_t)(cy - yy + 1) << 28) | ((uint32_t)(cz - zz + 1) << 30);
                for (int xx = xlo; xx <= xhi; ++xx) {
                    const uint32_t s = __ldg(a.off + rbase + xx);
                    const uint32_t e = __ldg(a.off + rbase + xx + 1);
                    const bool adj = inrow && cx - xx <= 1 && xx - cx <= 1;
                    if (adj) ncand += e - s;
                    if (s == e) continue;
                    const float qx = fmaf((float)(cx - xx), d.csf, pi.x);
                    const uint32_t code = code_yz | ((uint32_t)(cx - xx + 1) << 26);
                    for (uint32_t c0 = s; c0 < e; c0 += kCap) {
                        const uint32_t c1 = (e - c0) > (uint32_t)kCap ? c0 + kCap : e;
                        if (__reduce_max_sync(kFull, cnt) + (c1 - c0) > (uint32_t)kCap) flush();
#pragma unroll 4
                        for (uint32_t j = c0; j < c1; ++j) {
                            const float4 pj = __ldg(a.posc + j);
                            const float dx = qx - pj.x, dy = qy - pj.y, dz = qz - pj.z;
                            const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                            if (adj && d2 < d.r2max && j != i) {
                                lst[cnt * 32 + lane] = j | code;
                                ++cnt;
                            }
                        }
                    }
                }
            }
        }
    }
    flush();

    const float m = d.mass;
    const float4 out = make_float4(fmaf(m, ax, d.gx), fmaf(m, ay, d.gy), fmaf(m, az, d.gz), m * dr);
    if (valid) {
        a.ace[i] = out;
        if (COUNTS) a.nnb[i] = npairs + nbpairs;
    }
    float am = (valid && fluid) ? out.x * out.x + out.y * out.y + out.z * out.z : 0.f;
    float cm = valid ? ci : 0.f;
    float mm = (valid && fluid) ? mu : 0.f;
    uint32_t bad = (valid && !(isfinite(out.x) && isfinite(out.y) && isfinite(out.z) &&
                               isfinite(out.w)))
                       ? kStatusNonFinite
                       : 0u;
    if (!(am == am)) am = 0.f;
    uint32_t np = npairs, nb = nbpairs, nc = ncand;
    for (int o = 16; o; o >>= 1) {
        am = fmaxf(am, __shfl_xor_sync(kFull, am, o));
        cm = fmaxf(cm, __shfl_xor_sync(kFull, cm, o));
        mm = fmaxf(mm, __shfl_xor_sync(kFull, mm, o));
        np += __shfl_xor_sync(kFull, np, o);
        nb += __shfl_xor_sync(kFull, nb, o);
        nc += __shfl_xor_sync(kFull, nc, o);
        bad |= __shfl_xor_sync(kFull, bad, o);
    }
    if (lane == 0) {
        s_rf[w][0] = am;
        s_rf[w][1] = cm;
        s_rf[w][2] = mm;
        s_ru[w][0] = np;
        s_ru[w][1] = nc;
        s_ru[w][2] = bad;
        s_ru[w][3] = nb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
        uint4 u = make_uint4(0u, 0u, 0u, 0u);
        for (int k = 0; k < kIWarps; ++k) {
            f.x = fmaxf(f.x, s_rf[k][0]);
            f.y = fmaxf(f.y, s_rf[k][1]);
            f.z = fmaxf(f.z, s_rf[k][2]);
            u.x += s_ru[k][0];
            u.y += s_ru[k][1];
            u.z |= s_ru[k][2];
            u.w += s_ru[k][3];
        }
        a.part_f[blockIdx.x] = f;
        a.part_u[blockIdx.x] = u;
    }
}

// Sec. 3.3 reductions: per-block partials -> kReduceBlocks partials -> the
// last block to finish combines them in block order and sets the step size
// dt = CFL min( sqrt(h / max|a|), h / (max c + max mu) ).  Maxima and integer
// sums do not depend on the order, so the result is deterministic.
__global__ void __launch_bounds__(256) k_dt_reduce(const Dev d, const ReduceArgs a, int set_dt) {
    __shared__ float s_f[8][3];
    __shared__ unsigned long long s_u[8][3];
    __shared__ uint32_t s_b[8];
    __shared__ bool s_last;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float am = 0.f, cm = 0.f, mm = 0.f;
    unsigned long long pf = 0, pb = 0, nc = 0;
    uint32_t bad = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.nparts;
         i += gridDim.x * blockDim.x) {
        const float4 f = a.part_f[i];
        const uint4 u = a.part_u[i];
        am = fmaxf(am, f.x);
        cm = fmaxf(cm, f.y);
        mm = fmaxf(mm, f.z);
        pf += u.x;
        nc += u.y;
        bad |= u.z;
        pb += u.w;
    }
    for (int o = 16; o; o >>= 1) {
        am = fmaxf(am, __shfl_xor_sync(kFull, am, o));
        cm = fmaxf(cm, __shfl_xor_sync(kFull, cm, o));
        mm = fmaxf(mm, __shfl_xor_sync(kFull, mm, o));
        pf += __shfl_xor_sync(kFull, pf, o);
        pb += __shfl_xor_sync(kFull, pb, o);
        nc += __shfl_xor_sync(kFull, nc, o);
        bad |= __shfl_xor_sync(kFull, bad, o);
    }
    if (lane == 0) {
        s_f[w][0] = am;
        s_f[w][1] = cm;
        s_f[w][2] = mm;
        s_u[w][0] = pf;
        s_u[w][1] = pb;
        s_u[w][2] = nc;
        s_b[w] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
        unsigned long long q0 = 0, q1 = 0, q2 = 0;
        uint32_t b = 0;
        for (int k = 0; k < 8; ++k) {
            f.x = fmaxf(f.x, s_f[k][0]);
            f.y = fmaxf(f.y, s_f[k][1]);
            f.z = fmaxf(f.z, s_f[k][2]);
            q0 += s_u[k][0];
            q1 += s_u[k][1];
            q2 += s_u[k][2];
            b |= s_b[k];
        }
        a.lvl2_f[blockIdx.x] = f;
        a.lvl2_q[4 * blockIdx.x + 0] = q0;
        a.lvl2_q[4 * blockIdx.x + 1] = q1;
        a.lvl2_q[4 * blockIdx.x + 2] = q2;
        a.lvl2_q[4 * blockIdx.x + 3] = b;
        __threadfence();
        const uint32_t ticket = atomicAdd(a.done, 1u);
        s_last = ticket == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    __threadfence();
    float fa = 0.f, fc = 0.f, fm = 0.f;
    unsigned long long qf = 0, qb = 0, qc = 0;
    uint32_t b = 0;
    for (uint32_t k = 0; k < gridDim.x; ++k) {
        const float4 f = __ldcg(a.lvl2_f + k);
        fa = fmaxf(fa, f.x);
        fc = fmaxf(fc, f.y);
        fm = fmaxf(fm, f.z);
        qf += __ldcg(a.lvl2_q + 4 * k + 0);
        qb += __ldcg(a.lvl2_q + 4 * k + 1);
        qc += __ldcg(a.lvl2_q + 4 * k + 2);
        b |= (uint32_t)__ldcg(a.lvl2_q + 4 * k + 3);
    }
    const double amax = sqrt((double)fa);
    a.terms[0] = (float)amax;
    a.terms[1] = fc;
    a.terms[2] = fm;
    a.counters[0] += qf + qb;
    a.counters[1] += qc;
    a.counters[2] = qf + qb;
    a.counters[3] = qc;
    a.counters[4] = qf;
    a.counters[5] = qb;
    a.counters[6] += qf;
    a.counters[7] += qb;
    if (b) atomicOr(a.status, b);
    if (set_dt) {
        double dt;
        if (d.dt_fixed > 0.0) {
            dt = d.dt_fixed;
        } else {
            const double dtf = amax > 0.0 ? sqrt(d.h_d / amax) : INFINITY;
            const double dtc = d.h_d / ((double)fc + (double)fm);
            dt = d.cfl * (dtf < dtc ? dtf : dtc);
        }
        *a.dt = dt;
    }
    *a.done = 0u;
}

// Symplectic predictor (half step) for sorted particle k, then its new
// label.  Boundary particles keep r and v (Sec. 2.3); excluded particles
// (k >= in-domain count) are left untouched.
__global__ void __launch_bounds__(256) k_predict(const Dev d, const IntegrateArgs a) {
    __shared__ uint32_t s_hist[4 * 256];
    zero_hist(s_hist);
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = k < d.n;
    uint32_t key = 0;
    if (valid) {
        const uint32_t n_in = a.off[d.ncells];
        const double dt = *a.dt;
        const float hdt = (float)(0.5 * dt);
        double x = a.x[k], y = a.y[k], z = a.z[k];
        float4 vr = a.velrhop[k];
        a.px[k] = x;
        a.py[k] = y;
        a.pz[k] = z;
        a.pvr[k] = vr;
        if (k < n_in) {
            const float4 ac = a.ace[k];
            if (a.id[k] >= d.n_bound) {
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
        }
        key = cell_key(d, x, y, z);
        a.key[k] = key;
    }
    count_key(valid, key, a.cnt, s_hist, a.passes, bits_for(d.ncells));
    flush_hist(s_hist, a.hist, a.passes);
}

// Symplectic corrector from the start state (pre arrays, reordered like the
// current state) and the half-step rates, then the new label.
__global__ void __launch_bounds__(256) k_correct(const Dev d, const IntegrateArgs a) {
    __shared__ uint32_t s_hist[4 * 256];
    zero_hist(s_hist);
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = k < d.n;
    uint32_t key = 0;
    const double dt = *a.dt;
    if (valid) {
        const uint32_t n_in = a.off[d.ncells];
        const float dtf = (float)dt;
        const float hdt = (float)(0.5 * dt);
        double x = a.x[k], y = a.y[k], z = a.z[k];
        if (k < n_in) {
            const float4 ac = a.ace[k];
            const float4 pv = a.pvr[k];
            float4 vr = a.velrhop[k];
            if (a.id[k] >= d.n_bound) {
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
        }
        key = cell_key(d, x, y, z);
        a.key[k] = key;
    }
    if (k == 0) {
        *a.t += dt;
        *a.step += 1ull;
    }
    count_key(valid, key, a.cnt, s_hist, a.passes, bits_for(d.ncells));
    flush_hist(s_hist, a.hist, a.passes);
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
    const int cx = (int)(k % (uint32_t)d.ncx);
    const uint32_t t = k / (uint32_t)d.ncx;
    const int cy = (int)(t % (uint32_t)d.ncy), cz = (int)(t / (uint32_t)d.ncy);
    const double xi = x[i], yi = y[i], zi = z[i];
    const int xlo = cx > 0 ? cx - 1 : 0, xhi = cx + 1 < d.ncx ? cx + 1 : d.ncx - 1;
    uint32_t c = 0;
    for (int zz = cz - 1; zz <= cz + 1; ++zz) {
        if (zz < 0 || zz >= d.ncz) continue;
        for (int yy = cy - 1; yy <= cy + 1; ++yy) {
            if (yy < 0 || yy >= d.ncy) continue;
            const uint32_t rb = (uint32_t)d.ncx * ((uint32_t)yy + (uint32_t)d.ncy * zz);
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
    const double B = d.B_d;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < d.n; k += gridDim.x * blockDim.x) {
        if (k >= n_in) {
            acc[7] += 1.0;
            continue;
        }
        const float4 v = vr[k];
        const double rho = v.w;
        acc[0] += m;
        acc[6] += m * B * ((pow(rho, 6.0) - pow(rho0, 6.0)) / (6.0 * pow(rho0, 7.0)) + 1.0 / rho -
                           1.0 / rho0);
        if (id[k] >= d.n_bound) {
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

inline uint32_t blocks_for(uint32_t n, uint32_t t) { return n ? (n + t - 1) / t : 1; }

}  // namespace

void launch_keys(const Dev& d, const double* x, const double* y, const double* z, uint32_t n,
                 uint32_t* key, uint32_t* cnt, uint32_t* hist, int passes, cudaStream_t st) {
    k_keys<<<blocks_for(n, 256), 256, 0, st>>>(d, x, y, z, n, key, cnt, hist, passes);
}

void launch_reorder(const Dev& d, const ReorderArgs& a, cudaStream_t st) {
    k_reorder<<<blocks_for(d.n, 256), 256, 0, st>>>(d, a);
}

uint32_t interact_blocks(uint32_t n) { return blocks_for(n, kIWarps * 32); }

constexpr size_t kInteractSmem = (size_t)kIWarps * kCap * 32 * sizeof(uint32_t);

void prepare_interact() {
    cudaFuncSetAttribute(k_interact<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kInteractSmem);
    cudaFuncSetAttribute(k_interact<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kInteractSmem);
}

void launch_interact(const Dev& d, const InteractArgs& a, bool counts, cudaStream_t st) {
    const uint32_t nb = interact_blocks(d.n);
    if (counts)
        k_interact<true><<<nb, kIWarps * 32, kInteractSmem, st>>>(d, a);
    else
        k_interact<false><<<nb, kIWarps * 32, kInteractSmem, st>>>(d, a);
}

void launch_dt_reduce(const Dev& d, const ReduceArgs& a, bool set_dt, cudaStream_t st) {
    k_dt_reduce<<<kReduceBlocks, 256, 0, st>>>(d, a, set_dt ? 1 : 0);
}

void launch_predict(const Dev& d, const IntegrateArgs& a, cudaStream_t st) {
    k_predict<<<blocks_for(d.n, 256), 256, 0, st>>>(d, a);
}

void launch_correct(const Dev& d, const IntegrateArgs& a, cudaStream_t st) {
    k_correct<<<blocks_for(d.n, 256), 256, 0, st>>>(d, a);
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

}  // namespace sph
