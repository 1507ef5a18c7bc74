// C ABI of libsph.so (declared in include/sph.h): context, workspace
// layout, the ensemble table, the step sequence and its CUDA-graph capture,
// host transfers.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <string>
#include <vector>

#include "../../include/sph.h"
#include "sph_ctx.cuh"
#include "sph_internal.cuh"

using namespace sph;

namespace {

constexpr size_t kAlign = 256;
constexpr uint32_t kMaxGridBlocks = 4096;   // partials of the persistent interaction
constexpr uint32_t kMaxInstances = 1u << 16;

// Bump allocator over the caller's workspace (base may be null when only
// the size is wanted).
struct Carver {
    char* base;
    size_t used = 0;
    explicit Carver(void* b) : base((char*)b) {}
    template <typename T>
    T* take(size_t count) {
        used = (used + kAlign - 1) / kAlign * kAlign;
        T* p = base ? (T*)(base + used) : nullptr;
        used += count * sizeof(T);
        return p;
    }
};

int bit_length(uint64_t v) {
    int b = 0;
    while (v) {
        ++b;
        v >>= 1;
    }
    return b;
}

__global__ void k_unpack(uint32_t n, const double* __restrict__ pos, const float* __restrict__ vel,
                         const float* __restrict__ rho, double* x, double* y, double* z,
                         float4* vr, const uint32_t* __restrict__ id, uint32_t* id_flag) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (id[i] >= n) atomicOr(id_flag, 1u);
    x[i] = pos[3 * (size_t)i];
    y[i] = pos[3 * (size_t)i + 1];
    z[i] = pos[3 * (size_t)i + 2];
    vr[i] = make_float4(vel[3 * (size_t)i], vel[3 * (size_t)i + 1], vel[3 * (size_t)i + 2], rho[i]);
}

// k_unpack for a pipelined upload: the ids come from the staging slot too.
__global__ void k_unpack_ids(uint32_t n, const double* __restrict__ pos,
                             const float* __restrict__ vel, const float* __restrict__ rho,
                             const uint32_t* __restrict__ ids, double* x, double* y, double* z,
                             float4* vr, uint32_t* id, uint32_t* id_flag) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t k = ids[i];
    if (k >= n) atomicOr(id_flag, 1u);
    id[i] = k;
    x[i] = pos[3 * (size_t)i];
    y[i] = pos[3 * (size_t)i + 1];
    z[i] = pos[3 * (size_t)i + 2];
    vr[i] = make_float4(vel[3 * (size_t)i], vel[3 * (size_t)i + 1], vel[3 * (size_t)i + 2], rho[i]);
}

// Scatter by id (every id < n, distinct).
__global__ void k_pack_by_id(uint32_t n, const double* __restrict__ x, const double* __restrict__ y,
                             const double* __restrict__ z, const float4* __restrict__ vr,
                             const uint32_t* __restrict__ id, double* pos, float* vel, float* rho) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t k = id[i];
    if (k >= n) return;
    pos[3 * (size_t)k] = x[i];
    pos[3 * (size_t)k + 1] = y[i];
    pos[3 * (size_t)k + 2] = z[i];
    const float4 v = vr[i];
    vel[3 * (size_t)k] = v.x;
    vel[3 * (size_t)k + 1] = v.y;
    vel[3 * (size_t)k + 2] = v.z;
    rho[k] = v.w;
}

__global__ void k_pack(uint32_t n, const double* __restrict__ x, const double* __restrict__ y,
                       const double* __restrict__ z, const float4* __restrict__ vr, double* pos,
                       float* vel, float* rho, const uint32_t* __restrict__ id = nullptr,
                       uint32_t* ids = nullptr) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (ids) ids[i] = id[i];
    pos[3 * (size_t)i] = x[i];
    pos[3 * (size_t)i + 1] = y[i];
    pos[3 * (size_t)i + 2] = z[i];
    const float4 v = vr[i];
    vel[3 * (size_t)i] = v.x;
    vel[3 * (size_t)i + 1] = v.y;
    vel[3 * (size_t)i + 2] = v.z;
    rho[i] = v.w;
}

}  // namespace

namespace {

int validate_shared(const sph_params* p) {
    if (!p) return SPH_ERR_INVALID_ARG;
    if (!(p->h > 0.0) || !(p->rho0 > 0.0) || !(p->mass > 0.0) || !(p->cfl > 0.0) ||
        !(p->alpha >= 0.0) || !(p->eta2_coef > 0.0))
        return SPH_ERR_INVALID_ARG;
    if (p->gamma != 7.0) return SPH_ERR_INVALID_ARG;   // Tait law of Sec. 2.2
    if ((p->scheme & ~(SPH_SCHEME_CUBIC | SPH_SCHEME_VERLET)) != 0u || p->reserved != 0u)
        return SPH_ERR_INVALID_ARG;
    return SPH_OK;
}

// Build the ensemble table (host side); validates every member.
int build_table(const sph_params* p, const sph_instance* inst, uint32_t n_inst, Table* t) {
    int rc = validate_shared(p);
    if (rc) return rc;
    if (!inst || n_inst == 0 || n_inst > kMaxInstances) return SPH_ERR_INVALID_ARG;
    const double cs = 2.0 * p->h;
    t->inst.assign(n_inst, Inst{});
    t->cell_base.assign(n_inst + 1, 0);
    t->row_base.assign(n_inst + 1, 0);
    t->id_base.assign(n_inst + 1, 0);
    uint64_t cells = 0, rows = 0, ids = 0;
    int max_ncx = 1;
    for (uint32_t q = 0; q < n_inst; ++q) {
        const sph_instance& s = inst[q];
        if (!(s.c0 > 0.0) || s.n_particles == 0 || s.n_bound > s.n_particles)
            return SPH_ERR_INVALID_ARG;
        Inst& I = t->inst[q];
        int nc[3];
        for (int a = 0; a < 3; ++a) {
            if (!(s.dmax[a] > s.dmin[a])) return SPH_ERR_INVALID_ARG;
            const double v = ceil((s.dmax[a] - s.dmin[a]) / cs);
            if (!(v >= 1.0) || v > 65535.0) return SPH_ERR_INVALID_ARG;
            nc[a] = (int)v;
        }
        I.x0 = s.dmin[0];
        I.y0 = s.dmin[1];
        I.z0 = s.dmin[2];
        I.t_end = s.t_end;
        I.ncx = nc[0];
        I.ncy = nc[1];
        I.ncz = nc[2];
        I.cell_base = (uint32_t)cells;
        I.row_base = (uint32_t)rows;
        I.id_base = (uint32_t)ids;
        I.id_fluid = (uint32_t)(ids + s.n_bound);
        I.id_end = (uint32_t)(ids + s.n_particles);
        I.c0 = (float)s.c0;
        I.B = (float)(s.c0 * s.c0 * p->rho0 / p->gamma);
        I.B_d = s.c0 * s.c0 * p->rho0 / p->gamma;
        t->cell_base[q] = I.cell_base;
        t->row_base[q] = I.row_base;
        t->id_base[q] = I.id_base;
        cells += (uint64_t)nc[0] * nc[1] * nc[2];
        rows += (uint64_t)nc[1] * nc[2];
        ids += s.n_particles;
        if (nc[0] > max_ncx) max_ncx = nc[0];
        if (cells >= (1ull << 31) || ids >= kMaxParticles) return SPH_ERR_INVALID_ARG;
    }
    t->cell_base[n_inst] = (uint32_t)cells;
    t->row_base[n_inst] = (uint32_t)rows;
    t->id_base[n_inst] = (uint32_t)ids;
    t->ncells = cells;
    t->nrows = rows;
    t->n = ids;
    t->max_ncx = max_ncx;
    return SPH_OK;
}

sph_instance single_instance(const sph_params* p, uint32_t n) {
    sph_instance s;
    memset(&s, 0, sizeof(s));
    for (int a = 0; a < 3; ++a) {
        s.dmin[a] = p->dmin[a];
        s.dmax[a] = p->dmax[a];
    }
    s.c0 = p->c0;
    s.t_end = INFINITY;
    s.n_particles = n;
    s.n_bound = p->n_bound;
    return s;
}

// Lay out every device buffer; with base == nullptr only sizes are computed.
size_t carve(sph_ctx* c, void* base, uint32_t n, const Table& t, int passes) {
    Carver cv(base);
    const uint32_t n_inst = (uint32_t)t.inst.size();
    for (int b = 0; b < 2; ++b) {
        c->x[b] = cv.take<double>(n);
        c->y[b] = cv.take<double>(n);
        c->z[b] = cv.take<double>(n);
        c->vr[b] = cv.take<float4>(n);
        c->id[b] = cv.take<uint32_t>(n);
        c->px[b] = cv.take<double>(3 * (size_t)n);   // x, y, z of the start state
        c->py[b] = c->px[b] ? c->px[b] + n : nullptr;
        c->pz[b] = c->px[b] ? c->px[b] + 2 * (size_t)n : nullptr;
        c->pvr[b] = cv.take<float4>(n);
        c->key[b] = cv.take<uint32_t>(n);
        c->val[b] = cv.take<uint32_t>(n);
    }
    c->posc = cv.take<float4>(n);
    c->ace = cv.take<float4>(n);
    c->stage_pos = cv.take<double>(3 * (size_t)n);
    c->stage_vr = cv.take<float>(4 * (size_t)n);
    c->nnb = cv.take<uint32_t>(n);
    c->nnb64 = cv.take<uint32_t>(n);
    c->cnt = cv.take<uint32_t>(t.ncells + 1);
    c->off = cv.take<uint32_t>(t.ncells + 2);
    c->cscan_words = cv.take<unsigned long long>(scan_bsum_count(t.ncells + 1));
    c->cscan_ctl = cv.take<uint32_t>(2);
    c->hist = cv.take<uint32_t>(4 * 256);
    const uint32_t tiles = os_tiles(n);
    (void)passes;
    // status words the failure-path self-test runs its look-back against
    c->os_bytes = 4 * sizeof(uint32_t) + 256 * sizeof(uint32_t);
    c->tilectr = cv.take<uint32_t>(c->os_bytes / sizeof(uint32_t));
    c->os_status = c->tilectr ? c->tilectr + 4 : nullptr;
    for (int b = 0; b < 2; ++b) {
        c->sub_key[b] = cv.take<uint32_t>(n);
        c->sub_val[b] = cv.take<uint32_t>(n);
    }
    c->sub_hist = cv.take<uint32_t>(5 * 256);
    c->sub_os_bytes = 5 * sizeof(uint32_t) + (size_t)5 * tiles * 256 * sizeof(uint32_t);
    c->sub_os = cv.take<uint32_t>(c->sub_os_bytes / sizeof(uint32_t));
    c->sub_cnt = cv.take<uint32_t>(4);
    c->csum = cv.take<uint32_t>(t.ncells + t.nrows + 1);
    c->ucnt = cv.take<uint32_t>(t.nrows + 1);
    c->uoff = cv.take<uint32_t>(t.nrows + 2);
    c->ubsum = cv.take<uint32_t>(scan_bsum_count(t.nrows + 1));
    c->urow = cv.take<unsigned long long>(t.nrows);
    c->uctl = cv.take<uint32_t>(2);
    c->units_cap = max_units(n, (uint32_t)t.nrows, t.ncells);
    c->units = cv.take<uint2>(c->units_cap);
    c->part_u = cv.take<uint4>(kMaxGridBlocks);
    // ticket of the interaction's last block, then the unit counter and
    // finish ticket of the counter-scheduled interaction variants
    c->done = cv.take<uint32_t>(4);
    c->status = cv.take<uint32_t>(1);
    c->id_flag = cv.take<uint32_t>(1);
    c->diag_out = cv.take<double>(8);
    c->diag_part = cv.take<double>(8 * kDiagBlocks);
    c->front = cv.take<unsigned long long>(n_inst);
    c->loop_ctr = cv.take<uint32_t>(4);
    c->counters = cv.take<unsigned long long>(8);
    c->d_inst = cv.take<Inst>(n_inst);
    c->d_cell_base = cv.take<uint32_t>(n_inst + 1);
    c->d_row_base = cv.take<uint32_t>(n_inst + 1);
    c->d_id_base = cv.take<uint32_t>(n_inst + 1);
    c->i_dt = cv.take<double>(n_inst);
    c->i_t = cv.take<double>(n_inst);
    c->i_done = cv.take<uint32_t>(n_inst);
    c->i_steps = cv.take<unsigned long long>(n_inst);
    c->i_terms = cv.take<uint32_t>(3 * (size_t)n_inst);
    c->i_last = cv.take<float>(3 * (size_t)n_inst);
    c->i_vphase = cv.take<uint32_t>(n_inst);
    return (cv.used + kAlign - 1) / kAlign * kAlign;
}

Dev make_dev(const sph_ctx* c) {
    const sph_params* p = &c->p;
    Dev d;
    memset(&d, 0, sizeof(d));
    d.status = c->status;
    d.units_cap = c->units_cap;
    const double cs = 2.0 * p->h;
    d.inst = c->d_inst;
    d.cell_base = c->d_cell_base;
    d.row_base = c->d_row_base;
    d.id_base = c->d_id_base;
    d.n_inst = c->n_inst;
    d.is.dt = c->i_dt;
    d.is.t = c->i_t;
    d.is.done = c->i_done;
    d.is.steps = c->i_steps;
    d.is.terms = c->i_terms;
    d.is.last = c->i_last;
    d.is.vphase = c->i_vphase;
    d.inv_cs = 1.0 / cs;
    d.cs = cs;
    d.r2max_d = cs * cs;
    d.h_d = p->h;
    d.cfl = p->cfl;
    d.dt_fixed = p->dt_fixed;
    d.mass_d = p->mass;
    d.rho0_d = p->rho0;
    for (int k = 0; k < 3; ++k) d.g_d[k] = p->gravity[k];
    d.ncells = (uint32_t)c->tab.ncells;
    d.nrows = (uint32_t)c->tab.nrows;
    d.n = c->n;
    d.max_ncx = c->tab.max_ncx;
    d.variant = c->variant;
    d.unit = variant_unit(c->variant);
    d.stage = variant_stage(c->variant);
    d.units_fused = c->units_one ? 1 : 0;
    d.csf = (float)cs;
    d.h = (float)p->h;
    d.inv_h = (float)(1.0 / p->h);
    d.r2max = (float)(cs * cs);
    d.eta2 = (float)(p->eta2_coef * p->h * p->h);
    d.kern = (p->scheme & SPH_SCHEME_CUBIC) ? 1 : 0;
    if (d.kern == 1) {
        const double aD = 1.0 / (M_PI * p->h * p->h * p->h);   // cubic spline
        d.fc = (float)(aD / (p->h * p->h));
    } else {
        const double aD = 21.0 / (16.0 * M_PI * p->h * p->h * p->h);   // Wendland C2
        d.fc = (float)(-5.0 * aD / (p->h * p->h));
    }
    d.verlet_every = p->verlet_every ? p->verlet_every : 40u;
    d.alpha = (float)p->alpha;
    d.rho0 = (float)p->rho0;
    d.inv_rho0 = (float)(1.0 / p->rho0);
    d.mass = (float)p->mass;
    d.gx = (float)p->gravity[0];
    d.gy = (float)p->gravity[1];
    d.gz = (float)p->gravity[2];
    return d;
}

// Sort the labels in key[0] (counted into cnt/hist by the label kernel),
// scan the counts into cell offsets, cut the rows into interaction work
// units and reorder the state (and the start state when with_pre).
void rebuild_after_keys(sph_ctx* c, bool with_pre) {
    cudaStream_t st = c->st;
    launch_scan_cells(c->d, c->cnt, c->off, c->cscan_words, c->cscan_ctl, c->status, st);
    // the interaction's unit list needs only the cell offsets: on the fork
    // stream it runs beside the scatter and the reorder (joined below)
    const bool fork = c->st_units != nullptr;
    if (fork) {
        cudaEventRecord(c->ev_fork, st);
        cudaStreamWaitEvent(c->st_units, c->ev_fork, 0);
        launch_units(c->d, c->off, c->csum, c->ucnt, c->ubsum, c->uoff, c->units, c->urow,
                     c->uctl, c->status, c->st_units);
        cudaEventRecord(c->ev_join, c->st_units);
    }
    // the labels are in key[0]; one counting-sort pass groups the particles
    // by cell into (key[1], val[1]) and the reorder applies the id tie-break
    launch_cell_scatter(c->key[0], c->n, c->off, c->cnt, c->key[1], c->val[1], c->status, st);
    const int src = 1;
    c->skey = src;
    if (!fork)
        launch_units(c->d, c->off, c->csum, c->ucnt, c->ubsum, c->uoff, c->units, c->urow,
                     c->uctl, c->status, st);
    ReorderArgs ra;
    memset(&ra, 0, sizeof(ra));
    ra.skey = c->key[src];
    ra.sval = c->val[src];
    ra.off = c->off;
    const int s = c->cur, d = 1 - c->cur;
    ra.sx = c->x[s];
    ra.sy = c->y[s];
    ra.sz = c->z[s];
    ra.svr = c->vr[s];
    ra.sid = c->id[s];
    ra.dx = c->x[d];
    ra.dy = c->y[d];
    ra.dz = c->z[d];
    ra.dvr = c->vr[d];
    ra.did = c->id[d];
    if (with_pre) {
        ra.spx = c->px[0];
        ra.spy = c->py[0];
        ra.spz = c->pz[0];
        ra.spvr = c->pvr[0];
        ra.dpx = c->px[1];
        ra.dpy = c->py[1];
        ra.dpz = c->pz[1];
        ra.dpvr = c->pvr[1];
    } else if (c->verlet) {
        ra.spvr = c->pvr[0];   // (v, rho) one step earlier
        ra.dpvr = c->pvr[1];
    }
    ra.posc = c->posc;
    ra.hist_to_zero = c->hist;
    ra.status = c->status;
    launch_reorder(c->d, ra, st);
    if (fork) cudaStreamWaitEvent(st, c->ev_join, 0);
    c->cur = d;
}

void enqueue_interact(sph_ctx* c, bool counts, bool set_dt) {
    InteractArgs ia;
    ia.units = c->units;
    ia.n_units = c->uoff + c->tab.nrows;
    ia.status = c->status;
    ia.posc = c->posc;
    ia.velrhop = c->vr[c->cur];
    ia.key = c->key[c->skey];
    ia.id = c->id[c->cur];
    ia.off = c->off;
    ia.ace = c->ace;
    ia.nnb = c->nnb;
    ia.part_u = c->part_u;
    // the Sec. 3.3 reductions run in the interaction's last block
    ia.ticket = c->done;
    ia.sched = c->done + 1;
    ia.red.part_u = c->part_u;
    ia.red.nparts = c->nparts;
    ia.red.counters = c->counters;
    ia.red.status = c->status;
    ia.set_dt = set_dt ? 1 : 0;
    launch_interact(c->d, ia, counts, c->st);
}

IntegrateArgs integrate_args(sph_ctx* c, int pre) {
    IntegrateArgs a;
    a.off = c->off;
    a.x = c->x[c->cur];
    a.y = c->y[c->cur];
    a.z = c->z[c->cur];
    a.velrhop = c->vr[c->cur];
    a.id = c->id[c->cur];
    a.ace = c->ace;
    a.px = c->px[pre];
    a.py = c->py[pre];
    a.pz = c->pz[pre];
    a.pvr = c->pvr[pre];
    a.pvr_out = c->pvr[0];
    a.key = c->key[0];
    a.cnt = c->cnt;
    a.hist = c->hist;
    a.passes = 0;   // the cell sort needs the per-cell counts only
    return a;
}

void enqueue_build(sph_ctx* c) {
    if (!c->keys_ready) {
        launch_keys(c->d, c->x[c->cur], c->y[c->cur], c->z[c->cur], c->id[c->cur], c->n,
                    c->key[0], c->cnt, c->hist, 0, c->st);
    }
    const bool with_pre = c->pre_state == 1;
    rebuild_after_keys(c, with_pre);
    if (with_pre) c->pre_state = 2;
    c->keys_ready = false;
    c->cells_valid = true;
}

// One full step on the current buffers (state starts and ends in c->cur).
void enqueue_step(sph_ctx* c) {
    if (c->verlet) {
        enqueue_interact(c, false, true);
        launch_verlet(c->d, integrate_args(c, 1), c->st);
        c->keys_ready = true;
        enqueue_build(c);
        return;
    }
    enqueue_interact(c, false, true);
    launch_predict(c->d, integrate_args(c, 0), c->st);
    c->keys_ready = true;
    c->pre_state = 1;
    enqueue_build(c);
    enqueue_interact(c, false, false);
    launch_correct(c->d, integrate_args(c, 1), c->st);
    c->keys_ready = true;
    c->pre_state = 0;
    enqueue_build(c);
}

void release_fork_stream(sph_ctx* c) {
    if (c->st_units) {
        cudaStreamSynchronize(c->st_units);
        cudaStreamDestroy(c->st_units);
    }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    c->st_units = nullptr;
    c->ev_fork = c->ev_join = nullptr;
}

int post_launch(sph_ctx* c, const char* what) {
    return cuda_check(c, cudaGetLastError(), what);
}

int query(const sph_params* params, const sph_instance* inst, uint32_t n_inst, sph_sizes* out) {
    if (!out) return SPH_ERR_INVALID_ARG;
    sph_ctx tmp;
    int rc = build_table(params, inst, n_inst, &tmp.tab);
    if (rc) return rc;
    const int bits = bit_length(tmp.tab.ncells);
    const int passes = (bits + 7) / 8;
    out->workspace_bytes = carve(&tmp, nullptr, (uint32_t)tmp.tab.n, tmp.tab, passes);
    out->ncells = tmp.tab.ncells;
    out->ncx = (uint32_t)tmp.tab.inst[0].ncx;
    out->ncy = (uint32_t)tmp.tab.inst[0].ncy;
    out->ncz = (uint32_t)tmp.tab.inst[0].ncz;
    out->sort_passes = 1u;   // one counting-sort pass over the whole label
    return SPH_OK;
}

int init(const sph_params* params, const sph_instance* inst, uint32_t n_inst, void* ws,
         uint64_t ws_bytes, void* stream, sph_ctx** out) {
    if (!out) return SPH_ERR_INVALID_ARG;
    *out = nullptr;
    sph_ctx* c = new sph_ctx();
    int rc = build_table(params, inst, n_inst, &c->tab);
    if (rc) {
        delete c;
        return rc;
    }
    if (!ws || ((uintptr_t)ws % kAlign) != 0) {
        delete c;
        return SPH_ERR_WORKSPACE;
    }
    c->p = *params;
    c->verlet = (params->scheme & SPH_SCHEME_VERLET) != 0u;
    c->n = (uint32_t)c->tab.n;
    c->n_inst = n_inst;
    c->st = (cudaStream_t)stream;
    c->ncells = c->tab.ncells;
    c->bits = bit_length(c->ncells);
    c->passes = (c->bits + 7) / 8;
    const size_t need = carve(c, ws, c->n, c->tab, c->passes);
    if (ws_bytes < need) {
        delete c;
        return SPH_ERR_WORKSPACE;
    }
    c->tiles = os_tiles(c->n);
    {
        // the one-launch unit list for grids of few, short rows, unless the
        // environment sets SPH_UNITS_FUSED=0 when the context is created
        const char* e = getenv("SPH_UNITS_FUSED");
        c->units_one = !(e && e[0] == '0') &&
                       units_fit_one_launch((uint32_t)c->tab.nrows, c->tab.max_ncx);
    }
    prepare_interact();
    for (int v = 0; v < kNumVariants; ++v) {
        if (interact_grid(v) == 0 || interact_grid(v) > kMaxGridBlocks) {
            delete c;
            return SPH_ERR_CUDA;
        }
    }
    c->nparts = interact_grid(c->variant);
    c->d = make_dev(c);
    cudaStream_t st = c->st;
    cudaMemcpyAsync(c->d_inst, c->tab.inst.data(), n_inst * sizeof(Inst), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(c->d_cell_base, c->tab.cell_base.data(), (n_inst + 1) * sizeof(uint32_t),
                    cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(c->d_row_base, c->tab.row_base.data(), (n_inst + 1) * sizeof(uint32_t),
                    cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(c->d_id_base, c->tab.id_base.data(), (n_inst + 1) * sizeof(uint32_t),
                    cudaMemcpyHostToDevice, st);
    std::vector<double> dt0(n_inst, params->dt_fixed > 0.0 ? params->dt_fixed : 0.0);
    cudaMemcpyAsync(c->i_dt, dt0.data(), n_inst * sizeof(double), cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(c->i_t, 0, n_inst * sizeof(double), st);
    cudaMemsetAsync(c->i_done, 0, n_inst * sizeof(uint32_t), st);
    cudaMemsetAsync(c->i_steps, 0, n_inst * sizeof(unsigned long long), st);
    cudaMemsetAsync(c->i_terms, 0, 3 * (size_t)n_inst * sizeof(uint32_t), st);
    cudaMemsetAsync(c->i_last, 0, 3 * (size_t)n_inst * sizeof(float), st);
    cudaMemsetAsync(c->i_vphase, 0, n_inst * sizeof(uint32_t), st);
    cudaMemsetAsync(c->cnt, 0, (c->ncells + 1) * sizeof(uint32_t), st);
    cudaMemsetAsync(c->hist, 0, 4 * 256 * sizeof(uint32_t), st);
    cudaMemsetAsync(c->done, 0, 4 * sizeof(uint32_t), st);
    cudaMemsetAsync(c->status, 0, sizeof(uint32_t), st);
    cudaMemsetAsync(c->counters, 0, 8 * sizeof(unsigned long long), st);
    cudaMemsetAsync(c->urow, 0, (size_t)c->tab.nrows * sizeof(unsigned long long), st);
    cudaMemsetAsync(c->uctl, 0, 2 * sizeof(uint32_t), st);
    cudaMemsetAsync(c->cscan_words, 0, scan_bsum_count(c->ncells + 1) * sizeof(unsigned long long),
                    st);
    cudaMemsetAsync(c->cscan_ctl, 0, 2 * sizeof(uint32_t), st);
    rc = cuda_check(c, cudaStreamSynchronize(st), "sph_init");
    if (rc) {
        delete c;
        return rc;
    }
    {
        // the unit-list fork stream (not on the legacy default stream, or
        // when the environment sets SPH_FORK_UNITS=0 at context creation)
        const char* e = getenv("SPH_FORK_UNITS");
        if (st != nullptr && !(e && e[0] == '0')) {
            const bool ok =
                cudaStreamCreateWithFlags(&c->st_units, cudaStreamNonBlocking) == cudaSuccess &&
                cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
                cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) == cudaSuccess;
            if (!ok) {
                cudaGetLastError();
                release_fork_stream(c);
            }
        }
    }
    *out = c;
    return SPH_OK;
}

}  // namespace

extern "C" {

int sph_query_sizes(const sph_params* params, uint32_t n, sph_sizes* out) {
    if (!params || n == 0 || n >= kMaxParticles) return SPH_ERR_INVALID_ARG;
    const sph_instance one = single_instance(params, n);
    return query(params, &one, 1, out);
}

int sph_query_sizes_batch(const sph_params* params, const sph_instance* inst, uint32_t n_inst,
                          sph_sizes* out) {
    return query(params, inst, n_inst, out);
}

int sph_init(const sph_params* params, uint32_t n, void* ws, uint64_t ws_bytes, void* stream,
             sph_ctx** out) {
    if (!out) return SPH_ERR_INVALID_ARG;
    *out = nullptr;
    if (!params || n == 0 || n >= kMaxParticles) return SPH_ERR_INVALID_ARG;
    const sph_instance one = single_instance(params, n);
    return init(params, &one, 1, ws, ws_bytes, stream, out);
}

int sph_init_batch(const sph_params* params, const sph_instance* inst, uint32_t n_inst, void* ws,
                   uint64_t ws_bytes, void* stream, sph_ctx** out) {
    return init(params, inst, n_inst, ws, ws_bytes, stream, out);
}

int sph_instance_state(sph_ctx* c, double* t, double* dt, uint32_t* done, uint64_t* steps) {
    if (!c) return SPH_ERR_INVALID_ARG;
    const size_t m = c->n_inst;
    cudaStream_t st = c->st;
    if (t) cudaMemcpyAsync(t, c->i_t, m * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (dt) cudaMemcpyAsync(dt, c->i_dt, m * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (done) cudaMemcpyAsync(done, c->i_done, m * sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (steps) cudaMemcpyAsync(steps, c->i_steps, m * sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
    return cuda_check(c, cudaStreamSynchronize(st), "instance state");
}

int sph_set_instance_state(sph_ctx* c, const double* t, const uint64_t* steps) {
    if (!c) return SPH_ERR_INVALID_ARG;
    if (!t) return fail(c, SPH_ERR_INVALID_ARG, "NULL time array");
    const size_t m = c->n_inst;
    std::vector<uint32_t> done(m);
    for (size_t q = 0; q < m; ++q) {
        if (!std::isfinite(t[q]) || t[q] < 0.0) return fail(c, SPH_ERR_INVALID_ARG, "bad member time");
        done[q] = t[q] >= c->tab.inst[q].t_end ? 1u : 0u;
    }
    cudaStream_t st = c->st;
    cudaMemcpyAsync(c->i_t, t, m * sizeof(double), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(c->i_done, done.data(), m * sizeof(uint32_t), cudaMemcpyHostToDevice, st);
    if (steps)
        cudaMemcpyAsync(c->i_steps, steps, m * sizeof(uint64_t), cudaMemcpyHostToDevice, st);
    return cuda_check(c, cudaStreamSynchronize(st), "set instance state");
}

int sph_upload(sph_ctx* c, const double* pos, const float* vel, const float* rho,
               const uint32_t* ids) {
    const TraceRange trace("sph_upload");
    if (!c || !pos || !vel || !rho || !ids) return fail(c, SPH_ERR_INVALID_ARG, "NULL argument");
    const size_t n = c->n;
    cudaStream_t st = c->st;
    double* dpos = c->stage_pos;
    float* dvel = c->stage_vr;
    float* drho = c->stage_vr + 3 * n;
    // cudaMemcpyDefault: host or device source (unified addressing)
    int rc = cuda_check(c, cudaMemcpyAsync(dpos, pos, 3 * n * sizeof(double), cudaMemcpyDefault, st), "upload pos");
    if (rc) return rc;
    cudaMemcpyAsync(dvel, vel, 3 * n * sizeof(float), cudaMemcpyDefault, st);
    cudaMemcpyAsync(drho, rho, n * sizeof(float), cudaMemcpyDefault, st);
    cudaMemcpyAsync(c->id[c->cur], ids, n * sizeof(uint32_t), cudaMemcpyDefault, st);
    cudaMemsetAsync(c->id_flag, 0, sizeof(uint32_t), st);
    // Verlet: the first step after an upload has no earlier state (Euler)
    cudaMemsetAsync(c->i_vphase, 0, c->n_inst * sizeof(uint32_t), st);
    drop_pending_counts(c, st);
    k_unpack<<<(uint32_t)((n + 255) / 256), 256, 0, st>>>(c->n, dpos, dvel, drho, c->x[c->cur],
                                                         c->y[c->cur], c->z[c->cur], c->vr[c->cur],
                                                         c->id[c->cur], c->id_flag);
    rc = post_launch(c, "upload");
    if (rc) return rc;
    uint32_t flag = 1;
    cudaMemcpyAsync(&flag, c->id_flag, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    c->have_state = true;
    c->cells_valid = false;
    c->keys_ready = false;
    c->pre_state = 0;
    rc = cuda_check(c, cudaStreamSynchronize(st), "upload sync");
    c->ids_dense = rc == SPH_OK && flag == 0;
    c->ids_pending = false;
    return rc;
}

int sph_build_cells(sph_ctx* c) {
    const TraceRange trace("sph_build_cells");
    if (!c) return SPH_ERR_INVALID_ARG;
    if (!c->have_state) return fail(c, SPH_ERR_STATE, "no state uploaded");
    enqueue_build(c);
    return post_launch(c, "build_cells");
}

int sph_interact(sph_ctx* c, uint32_t flags) {
    const TraceRange trace("sph_interact");
    if (!c) return SPH_ERR_INVALID_ARG;
    if (!c->cells_valid) return fail(c, SPH_ERR_STATE, "cells not built");
    // at the half step (predictor pending) the step size stays the one set
    // by the evaluation at the start of the step, as in sph_step
    enqueue_interact(c, (flags & SPH_INTERACT_COUNTS) != 0, c->pre_state != 2);
    return post_launch(c, "interact");
}

int sph_predict(sph_ctx* c) {
    const TraceRange trace("sph_predict");
    if (!c) return SPH_ERR_INVALID_ARG;
    if (c->verlet) return fail(c, SPH_ERR_STATE, "predict on a Verlet context");
    if (!c->cells_valid) return fail(c, SPH_ERR_STATE, "cells not built");
    launch_predict(c->d, integrate_args(c, 0), c->st);
    c->keys_ready = true;
    c->pre_state = 1;
    c->cells_valid = false;
    return post_launch(c, "predict");
}

int sph_correct(sph_ctx* c) {
    const TraceRange trace("sph_correct");
    if (!c) return SPH_ERR_INVALID_ARG;
    if (c->verlet) return fail(c, SPH_ERR_STATE, "correct on a Verlet context");
    if (!c->cells_valid || c->pre_state != 2)
        return fail(c, SPH_ERR_STATE, "correct needs predict, build_cells and interact first");
    launch_correct(c->d, integrate_args(c, 1), c->st);
    c->keys_ready = true;
    c->pre_state = 0;
    c->cells_valid = false;
    return post_launch(c, "correct");
}

int sph_verlet(sph_ctx* c) {
    const TraceRange trace("sph_verlet");
    if (!c) return SPH_ERR_INVALID_ARG;
    if (!c->verlet) return fail(c, SPH_ERR_STATE, "verlet on a symplectic context");
    if (!c->cells_valid) return fail(c, SPH_ERR_STATE, "verlet needs build_cells and interact first");
    launch_verlet(c->d, integrate_args(c, 1), c->st);
    c->keys_ready = true;
    c->cells_valid = false;
    return post_launch(c, "verlet");
}

// The loop graph of start parity g: a conditional WHILE node whose body is
// `body` steps followed by k_loop_ctrl (captured from the same enqueue
// functions as the single-step graphs).  The body must end on the parity it
// started from.
static int build_loop_graph(sph_ctx* c, int g, uint32_t body) {
    cudaGraph_t graph = nullptr;
    int rc = cuda_check(c, cudaGraphCreate(&graph, 0), "loop graph create");
    if (rc) return rc;
    cudaGraphConditionalHandle h;
    rc = cuda_check(c, cudaGraphConditionalHandleCreate(&h, graph, 1u, cudaGraphCondAssignDefault),
                    "conditional handle");
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (!rc) rc = cuda_check(c, cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np),
                             "conditional node");
    if (!rc) {
        cudaGraph_t bodyg = np.conditional.phGraph_out[0];
        rc = cuda_check(c, cudaStreamBeginCaptureToGraph(c->st, bodyg, nullptr, nullptr, 0,
                                                         cudaStreamCaptureModeThreadLocal),
                        "begin body capture");
        if (!rc) {
            for (uint32_t s = 0; s < body; ++s) enqueue_step(c);
            launch_loop_ctrl(h, c->loop_ctr, c->i_done, c->n_inst, body, c->st);
            rc = cuda_check(c, cudaStreamEndCapture(c->st, &bodyg), "end body capture");
        }
    }
    if (!rc && c->cur != g) rc = fail(c, SPH_ERR_STATE, "loop body changed buffer parity");
    if (!rc) rc = cuda_check(c, cudaGraphInstantiate(&c->loop_graph[g], graph, 0), "instantiate loop");
    cudaGraphDestroy(graph);
    return rc;
}

int sph_step(sph_ctx* c, uint32_t nsteps) {
    const TraceRange trace("sph_step");
    if (!c) return SPH_ERR_INVALID_ARG;
    if (!c->have_state) return fail(c, SPH_ERR_STATE, "no state uploaded");
    c->pre_state = 0;
    if (!c->cells_valid) {
        enqueue_build(c);
        int rc = post_launch(c, "build_cells");
        if (rc) return rc;
    }
    if (nsteps == 0) return SPH_OK;
    if (c->st == nullptr) {
        for (uint32_t s = 0; s < nsteps; ++s) enqueue_step(c);
        return post_launch(c, "step");
    }
    // Two or more steps: one launch of the loop graph, whose WHILE node runs
    // bodies of one symplectic step (which returns to its buffer parity) or
    // two Verlet steps on the device until the steps asked are done or every
    // member has reached its end time; a remaining odd Verlet step takes the
    // single-step graph below.
    const uint32_t body = c->verlet ? 2u : 1u;
    uint32_t looped = 0;
    if (nsteps >= 2u * body || (!c->verlet && nsteps >= 2u)) {
        looped = nsteps / body * body;
        const int g = c->cur;
        if (!c->loop_graph[g]) {
            int rc = build_loop_graph(c, g, body);
            if (rc) return rc;
        }
        launch_loop_init(c->loop_ctr, looped, c->st);
        int rc = post_launch(c, "loop init");
        if (rc) return rc;
        rc = cuda_check(c, cudaGraphLaunch(c->loop_graph[g], c->st), "loop graph launch");
        if (rc) return rc;
    }
    // One graph per state-buffer parity the step starts from.  A symplectic
    // step rebuilds twice and ends on the parity it started from; a Verlet
    // step rebuilds once, so its steps alternate between the two graphs.
    for (uint32_t s = looped; s < nsteps; ++s) {
        const int g = c->cur;
        if (!c->graph[g]) {
            cudaGraph_t graph;
            int rc = cuda_check(c, cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal),
                                "begin capture");
            if (rc) return rc;
            enqueue_step(c);   // host bookkeeping advances as the graph will
            rc = cuda_check(c, cudaStreamEndCapture(c->st, &graph), "end capture");
            if (rc) return rc;
            rc = cuda_check(c, cudaGraphInstantiate(&c->graph[g], graph, 0), "instantiate");
            cudaGraphDestroy(graph);
            if (rc) return rc;
            if ((c->cur != g) != c->verlet)
                return fail(c, SPH_ERR_STATE, "step changed buffer parity");
        } else if (c->verlet) {
            c->cur = 1 - g;
        }
        int rc = cuda_check(c, cudaGraphLaunch(c->graph[g], c->st), "graph launch");
        if (rc) return rc;
    }
    return SPH_OK;
}

int sph_rollout(sph_ctx* c, uint32_t nsteps, uint32_t save_every, sph_snapshot_fn cb,
                void* user) {
    const TraceRange trace("sph_rollout");
    if (!c) return SPH_ERR_INVALID_ARG;
    if (save_every == 0) save_every = nsteps ? nsteps : 1;
    uint32_t done = 0;
    while (done < nsteps) {
        const uint32_t k = (nsteps - done) < save_every ? (nsteps - done) : save_every;
        int rc = sph_step(c, k);
        if (rc) return rc;
        done += k;
        rc = cuda_check(c, cudaStreamSynchronize(c->st), "rollout sync");
        if (rc) return rc;
        // the device status word at every save boundary: a non-finite rate,
        // a wait that gave up or a capacity overflow ends the rollout here
        rc = sph_check(c);
        if (rc) return rc;
        if (cb) {
            double t = 0.0;
            unsigned long long s = 0;
            cudaMemcpy(&t, c->i_t, sizeof(double), cudaMemcpyDeviceToHost);
            cudaMemcpy(&s, c->i_steps, sizeof(s), cudaMemcpyDeviceToHost);
            if (cb(user, s, t)) break;
        }
    }
    return SPH_OK;
}

int sph_download(sph_ctx* c, double* pos, float* vel, float* rho, uint32_t* ids) {
    const TraceRange trace("sph_download");
    if (!c) return SPH_ERR_INVALID_ARG;
    if (!c->have_state) return fail(c, SPH_ERR_STATE, "no state uploaded");
    const size_t n = c->n;
    cudaStream_t st = c->st;
    double* dpos = c->stage_pos;
    float* dv = c->stage_vr;
    float* dr = dv + 3 * n;
    k_pack<<<(uint32_t)((n + 255) / 256), 256, 0, st>>>(c->n, c->x[c->cur], c->y[c->cur],
                                                       c->z[c->cur], c->vr[c->cur], dpos, dv, dr);
    int rc = post_launch(c, "download pack");
    if (rc) return rc;
    // cudaMemcpyDefault: host or device destination (unified addressing)
    if (pos) cudaMemcpyAsync(pos, dpos, 3 * n * sizeof(double), cudaMemcpyDefault, st);
    if (vel) cudaMemcpyAsync(vel, dv, 3 * n * sizeof(float), cudaMemcpyDefault, st);
    if (rho) cudaMemcpyAsync(rho, dr, n * sizeof(float), cudaMemcpyDefault, st);
    if (ids) cudaMemcpyAsync(ids, c->id[c->cur], n * sizeof(uint32_t), cudaMemcpyDefault, st);
    return cuda_check(c, cudaStreamSynchronize(st), "download");
}

int sph_download_by_id(sph_ctx* c, double* pos, float* vel, float* rho) {
    const TraceRange trace("sph_download_by_id");
    if (!c) return SPH_ERR_INVALID_ARG;
    if (!c->have_state) return fail(c, SPH_ERR_STATE, "no state uploaded");
    if (c->ids_pending) {
        const int rc = sph_sync_transfers(c);
        if (rc) return rc;
    }
    if (!c->ids_dense) return fail(c, SPH_ERR_STATE, "ids are not all below n");
    const size_t n = c->n;
    cudaStream_t st = c->st;
    double* dpos = c->stage_pos;
    float* dv = c->stage_vr;
    float* dr = dv + 3 * n;
    k_pack_by_id<<<(uint32_t)((n + 255) / 256), 256, 0, st>>>(
        c->n, c->x[c->cur], c->y[c->cur], c->z[c->cur], c->vr[c->cur], c->id[c->cur], dpos, dv, dr);
    int rc = post_launch(c, "download_by_id pack");
    if (rc) return rc;
    if (pos) cudaMemcpyAsync(pos, dpos, 3 * n * sizeof(double), cudaMemcpyDefault, st);
    if (vel) cudaMemcpyAsync(vel, dv, 3 * n * sizeof(float), cudaMemcpyDefault, st);
    if (rho) cudaMemcpyAsync(rho, dr, n * sizeof(float), cudaMemcpyDefault, st);
    return cuda_check(c, cudaStreamSynchronize(st), "download_by_id");
}

uint64_t sph_array_bytes(const sph_ctx* c, int which) {
    if (!c) return 0;
    switch (which) {
        case SPH_ARRAY_KEY:
        case SPH_ARRAY_NNB:
        case SPH_ARRAY_NNB64: return (uint64_t)c->n * 4;
        case SPH_ARRAY_CELL_OFF: return (c->ncells + 2) * 4;
        case SPH_ARRAY_ACE:
        case SPH_ARRAY_POSC: return (uint64_t)c->n * 16;
        case SPH_ARRAY_PREV: return c->verlet ? (uint64_t)c->n * 16 : 0;
        case SPH_ARRAY_DT: return 8ull * c->n_inst;
        case SPH_ARRAY_UNITS: return 4ull + 8ull * c->units_cap;
        default: return 0;
    }
}

int sph_read_array(sph_ctx* c, int which, void* host, uint64_t bytes) {
    if (!c || !host) return fail(c, SPH_ERR_INVALID_ARG, "NULL argument");
    const uint64_t want = sph_array_bytes(c, which);
    if (want == 0 || bytes != want) return fail(c, SPH_ERR_INVALID_ARG, "bad array id or size");
    if (which == SPH_ARRAY_UNITS) {
        if (!c->cells_valid) return fail(c, SPH_ERR_STATE, "cells not built");
        // the count, then the units; entries past the count are left as they are
        uint32_t* h = static_cast<uint32_t*>(host);
        int rc = cuda_check(c, cudaMemcpyAsync(h, c->uoff + c->tab.nrows, 4, cudaMemcpyDeviceToHost,
                                               c->st), "read unit count");
        if (!rc) rc = cuda_check(c, cudaMemcpyAsync(h + 1, c->units, 8ull * c->units_cap,
                                                    cudaMemcpyDeviceToHost, c->st), "read units");
        if (rc) return rc;
        return cuda_check(c, cudaStreamSynchronize(c->st), "read array sync");
    }
    const void* src = nullptr;
    switch (which) {
        case SPH_ARRAY_KEY: src = c->key[c->skey]; break;
        case SPH_ARRAY_CELL_OFF: src = c->off; break;
        case SPH_ARRAY_ACE: src = c->ace; break;
        case SPH_ARRAY_NNB: src = c->nnb; break;
        case SPH_ARRAY_NNB64: src = c->nnb64; break;
        case SPH_ARRAY_POSC: src = c->posc; break;
        case SPH_ARRAY_DT: src = c->i_dt; break;
        // in the state's order: after a rebuild the reordered copy
        case SPH_ARRAY_PREV: src = c->cells_valid ? c->pvr[1] : c->pvr[0]; break;
    }
    int rc = cuda_check(c, cudaMemcpyAsync(host, src, bytes, cudaMemcpyDeviceToHost, c->st), "read array");
    if (rc) return rc;
    return cuda_check(c, cudaStreamSynchronize(c->st), "read array sync");
}

int sph_neighbour_counts_fp64(sph_ctx* c) {
    const TraceRange trace("sph_neighbour_counts_fp64");
    if (!c) return SPH_ERR_INVALID_ARG;
    if (!c->cells_valid) return fail(c, SPH_ERR_STATE, "cells not built");
    launch_counts_fp64(c->d, c->x[c->cur], c->y[c->cur], c->z[c->cur], c->key[c->skey], c->off,
                       c->nnb64, c->st);
    return post_launch(c, "counts_fp64");
}

int sph_diagnostics(sph_ctx* c, sph_diag* out) {
    const TraceRange trace("sph_diagnostics");
    if (!c || !out) return fail(c, SPH_ERR_INVALID_ARG, "NULL argument");
    memset(out, 0, sizeof(*out));
    if (c->have_state && c->cells_valid) {
        launch_diag(c->d, c->x[c->cur], c->y[c->cur], c->z[c->cur], c->vr[c->cur], c->id[c->cur],
                    c->off, c->diag_part, c->diag_out, c->st);
        int rc = post_launch(c, "diag");
        if (rc) return rc;
    }
    double dsum[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double t = 0, dt = 0;
    unsigned long long cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0}, step = 0;
    float terms[4] = {0, 0, 0, 0};
    uint32_t status = 0;
    cudaStream_t st = c->st;
    if (c->have_state && c->cells_valid)
        cudaMemcpyAsync(dsum, c->diag_out, sizeof(dsum), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&t, c->i_t, sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&dt, c->i_dt, sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(cnt, c->counters, sizeof(cnt), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&step, c->i_steps, sizeof(step), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(terms, c->i_last, 3 * sizeof(float), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&status, c->status, sizeof(status), cudaMemcpyDeviceToHost, st);
    int rc = cuda_check(c, cudaStreamSynchronize(st), "diagnostics");
    if (rc) return rc;
    out->t = t;
    out->dt = dt;
    out->mass = dsum[0];
    out->momentum[0] = dsum[1];
    out->momentum[1] = dsum[2];
    out->momentum[2] = dsum[3];
    out->kinetic = dsum[4];
    out->potential = dsum[5];
    out->internal = dsum[6];
    out->n_out = (uint32_t)dsum[7];
    out->step = step;
    out->pairs_total = cnt[0];
    out->candidates_total = cnt[1];
    out->pairs_last = cnt[2];
    out->candidates_last = cnt[3];
    out->pairs_fluid_last = cnt[4];
    out->pairs_boundary_last = cnt[5];
    out->pairs_fluid_total = cnt[6];
    out->pairs_boundary_total = cnt[7];
    out->status = status;
    out->amax = terms[0];
    out->cmax = terms[1];
    out->mumax = terms[2];
    return SPH_OK;
}

int sph_front(sph_ctx* c, double z_lo, double z_hi, double* front) {
    const TraceRange trace("sph_front");
    if (!c || !front) return fail(c, SPH_ERR_INVALID_ARG, "NULL argument");
    if (!(z_lo < z_hi)) return fail(c, SPH_ERR_INVALID_ARG, "need z_lo < z_hi");
    if (!c->have_state || !c->cells_valid) return fail(c, SPH_ERR_STATE, "cells not built");
    launch_front(c->d, c->x[c->cur], c->z[c->cur], c->id[c->cur], c->off, z_lo, z_hi, c->front,
                 c->st);
    int rc = post_launch(c, "front");
    if (rc) return rc;
    std::vector<unsigned long long> img(c->n_inst);
    rc = cuda_check(c, cudaMemcpyAsync(img.data(), c->front, c->n_inst * sizeof(unsigned long long),
                                       cudaMemcpyDeviceToHost, c->st), "front copy");
    if (rc) return rc;
    rc = cuda_check(c, cudaStreamSynchronize(c->st), "front sync");
    if (rc) return rc;
    for (uint32_t q = 0; q < c->n_inst; ++q) {
        const unsigned long long u = img[q];
        if (u == 0) {
            front[q] = -INFINITY;
            continue;
        }
        const unsigned long long b = (u & 0x8000000000000000ull) ? (u & 0x7fffffffffffffffull) : ~u;
        memcpy(&front[q], &b, sizeof(double));
    }
    return SPH_OK;
}

int sph_check(sph_ctx* c) {
    if (!c) return SPH_ERR_INVALID_ARG;
    uint32_t status = 0;
    int rc = cuda_check(c, cudaMemcpyAsync(&status, c->status, sizeof(status), cudaMemcpyDeviceToHost, c->st), "check");
    if (rc) return rc;
    rc = cuda_check(c, cudaStreamSynchronize(c->st), "check sync");
    if (rc) return rc;
    if (status & SPH_STATUS_TIMEOUT)
        return fail(c, SPH_ERR_TIMEOUT, "a bounded device wait gave up (radix-sort look-back or staging copy)");
    if (status & SPH_STATUS_NONFINITE) return fail(c, SPH_ERR_NONFINITE, "non-finite interaction result");
    if (status & SPH_STATUS_CAPACITY) return fail(c, SPH_ERR_CAPACITY, "a cell exceeded the id tie-break capacity");
    if (status & SPH_STATUS_BOUNDS)
        return fail(c, SPH_ERR_BOUNDS, "a kernel index was out of range (checked build)");
    return SPH_OK;
}

int sph_clear_status(sph_ctx* c) {
    if (!c) return SPH_ERR_INVALID_ARG;
    int rc = cuda_check(c, cudaMemsetAsync(c->status, 0, sizeof(uint32_t), c->st), "clear status");
    if (rc) return rc;
    return cuda_check(c, cudaStreamSynchronize(c->st), "clear status sync");
}

int sph_selftest_timeout(sph_ctx* c, uint32_t polls) {
    if (!c) return SPH_ERR_INVALID_ARG;
    if (polls == 0 || polls > (1u << 20)) return fail(c, SPH_ERR_INVALID_ARG, "polls must be 1..2^20");
    // status words reserved for this test (zeroed by the launch)
    launch_lookback_selftest(c->os_status, polls, c->status, c->st);
    int rc = post_launch(c, "selftest");
    if (rc) return rc;
    return cuda_check(c, cudaStreamSynchronize(c->st), "selftest sync");
}

int sph_units_selftest_timeout(sph_ctx* c, uint32_t polls) {
    if (!c) return SPH_ERR_INVALID_ARG;
    if (polls == 0 || polls > (1u << 20)) return fail(c, SPH_ERR_INVALID_ARG, "polls must be 1..2^20");
    // a word of the sort self-test's reserved status area (zeroed by the launch)
    launch_row_lookback_selftest(reinterpret_cast<unsigned long long*>(c->os_status), polls,
                                 c->status, c->st);
    int rc = post_launch(c, "units selftest");
    if (rc) return rc;
    return cuda_check(c, cudaStreamSynchronize(c->st), "units selftest sync");
}

uint32_t sph_num_variants(void) { return (uint32_t)kNumVariants; }

int sph_pdl_enabled(void) { return pdl_enabled() ? 1 : 0; }

int sph_set_variant(sph_ctx* c, uint32_t v) {
    if (!c || v >= (uint32_t)kNumVariants) return fail(c, SPH_ERR_INVALID_ARG, "bad variant");
    if ((int)v == c->variant) return SPH_OK;
    c->variant = (int)v;
    c->nparts = interact_grid(c->variant);
    c->d = make_dev(c);
    for (int g = 0; g < 2; ++g) {
        if (c->graph[g]) cudaGraphExecDestroy(c->graph[g]);
        c->graph[g] = nullptr;
        if (c->loop_graph[g]) cudaGraphExecDestroy(c->loop_graph[g]);
        c->loop_graph[g] = nullptr;
    }
    // the work units depend on the block shape: recut them for the current cells
    if (c->cells_valid) launch_units(c->d, c->off, c->csum, c->ucnt, c->ubsum, c->uoff, c->units,
                                     c->urow, c->uctl, c->status, c->st);
    return post_launch(c, "set variant");
}

int sph_autotune(sph_ctx* c, uint32_t reps, float* ms_per_variant, uint32_t* best) {
    const TraceRange trace("sph_autotune");
    if (!c) return SPH_ERR_INVALID_ARG;
    if (!c->cells_valid) return fail(c, SPH_ERR_STATE, "cells not built");
    if (reps == 0) reps = 3;
    const int start = c->variant;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = INFINITY;
    int best_v = start;
    for (int v = 0; v < kNumVariants; ++v) {
        int rc = sph_set_variant(c, (uint32_t)v);
        if (rc) return rc;
        InteractArgs ia;
        ia.units = c->units;
        ia.n_units = c->uoff + c->tab.nrows;
        ia.status = c->status;
        ia.posc = c->posc;
        ia.velrhop = c->vr[c->cur];
        ia.key = c->key[c->skey];
        ia.id = c->id[c->cur];
        ia.off = c->off;
        ia.ace = c->ace;
        ia.nnb = c->nnb;
        ia.part_u = c->part_u;
        ia.ticket = nullptr;   // timing only: no counters, no step size
        ia.sched = c->done + 1;
        launch_interact(c->d, ia, false, c->st);   // warm
        cudaEventRecord(e0, c->st);
        for (uint32_t r = 0; r < reps; ++r) launch_interact(c->d, ia, false, c->st);
        cudaEventRecord(e1, c->st);
        rc = cuda_check(c, cudaEventSynchronize(e1), "autotune");
        if (rc) return rc;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= (float)reps;
        if (ms_per_variant) ms_per_variant[v] = ms;
        if (ms < best_ms) {
            best_ms = ms;
            best_v = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // the timing launches left running maxima behind; clear them
    cudaMemsetAsync(c->i_terms, 0, 3 * (size_t)c->n_inst * sizeof(uint32_t), c->st);
    if (best) *best = (uint32_t)best_v;
    return sph_set_variant(c, (uint32_t)best_v);
}

uint32_t sph_kernels_per_step(const sph_ctx* c) {
    if (!c) return 0;
    // the cell scan is one launch; another scan is 3 kernels, or 1 when the
    // array fits one scan block
    const uint32_t cell_scan = 1u;
    // the unit list: one launch for a grid of few rows, else row sums, count,
    // scan, fill
    const uint32_t unit_scan = scan_bsum_count(c->tab.nrows) == 1 ? 1u : 3u;
    const uint32_t unit_list = c->units_one ? 1u : 3u + unit_scan;
    // one rebuild: cell scan + 1 counting-sort scatter + unit list + reorder
    const uint32_t rebuild = cell_scan + 1u + unit_list + 1u;
    // Verlet: interact (with the CFL reduction) + update + member advance + rebuild
    if (c->verlet) return 1u + 2u + rebuild;
    // symplectic: 2 interactions (with the CFL reduction) + predict + correct + 2 rebuilds
    return 2u + 2u + 2u * rebuild;
}

const char* sph_last_error(const sph_ctx* c) { return c ? c->err.c_str() : "NULL context"; }

// --- pipelined transfers -------------------------------------------------

namespace {

// One staging slot: positions (3n f64), velocities (3n f32), densities (n
// f32), ids (n u32), each sub-array 256-byte aligned.
struct XferSlot {
    double* pos;
    float *vel, *rho;
    uint32_t* ids;
};

uint64_t xfer_slot_bytes(uint32_t n) {
    Carver cv(nullptr);
    cv.take<double>(3 * (size_t)n);
    cv.take<float>(3 * (size_t)n);
    cv.take<float>(n);
    cv.take<uint32_t>(n);
    return (cv.used + kAlign - 1) / kAlign * kAlign;
}

XferSlot xfer_slot(sph_ctx* c, int s) {
    Carver cv(c->xfer + (size_t)s * c->xfer_slot);
    XferSlot x;
    x.pos = cv.take<double>(3 * (size_t)c->n);
    x.vel = cv.take<float>(3 * (size_t)c->n);
    x.rho = cv.take<float>(c->n);
    x.ids = cv.take<uint32_t>(c->n);
    return x;
}

}  // namespace

// Waits for the copy streams and destroys them and their events (each
// handle only if it was created).
static void release_transfer_streams(sph_ctx* c) {
    for (cudaStream_t* s : {&c->s_h2d, &c->s_d2h}) {
        if (*s) {
            cudaStreamSynchronize(*s);
            cudaStreamDestroy(*s);
            *s = nullptr;
        }
    }
    for (cudaEvent_t* e : {&c->ev_up_loaded[0], &c->ev_up_loaded[1], &c->ev_up_free[0],
                           &c->ev_up_free[1], &c->ev_dn_packed, &c->ev_dn_free}) {
        if (*e) {
            cudaEventDestroy(*e);
            *e = nullptr;
        }
    }
    c->xfer = nullptr;
}

uint64_t sph_async_transfer_bytes(const sph_ctx* c) {
    if (!c) return 0;
    return 3 * xfer_slot_bytes(c->n);
}

int sph_enable_async_transfers(sph_ctx* c, void* d_buf, uint64_t bytes) {
    if (!c || !d_buf) return SPH_ERR_INVALID_ARG;
    if (((uintptr_t)d_buf % kAlign) != 0 || bytes < sph_async_transfer_bytes(c))
        return fail(c, SPH_ERR_WORKSPACE, "transfer buffer too small or not 256-byte aligned");
    if (c->s_h2d) {
        // a new buffer: everything that used the old one has finished
        int rc = sph_sync_transfers(c);
        if (rc) return rc;
    } else {
        const unsigned fl = cudaEventDisableTiming;
        bool ok = cudaStreamCreateWithFlags(&c->s_h2d, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&c->s_d2h, cudaStreamNonBlocking) == cudaSuccess;
        for (int s = 0; s < 2 && ok; ++s)
            ok = cudaEventCreateWithFlags(&c->ev_up_loaded[s], fl) == cudaSuccess &&
                 cudaEventCreateWithFlags(&c->ev_up_free[s], fl) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&c->ev_dn_packed, fl) == cudaSuccess &&
             cudaEventCreateWithFlags(&c->ev_dn_free, fl) == cudaSuccess;
        if (!ok) {
            const cudaError_t e = cudaGetLastError();
            release_transfer_streams(c);   // what was created; pipelined calls stay off
            return cuda_check(c, e != cudaSuccess ? e : cudaErrorUnknown, "transfer streams");
        }
    }
    c->xfer = static_cast<unsigned char*>(d_buf);
    c->xfer_slot = xfer_slot_bytes(c->n);
    c->up_slot = 0;
    return SPH_OK;
}

int sph_upload_async(sph_ctx* c, const double* pos, const float* vel, const float* rho,
                     const uint32_t* ids) {
    const TraceRange trace("sph_upload_async");
    if (!c || !pos || !vel || !rho || !ids) return fail(c, SPH_ERR_INVALID_ARG, "NULL argument");
    if (!c->xfer) return fail(c, SPH_ERR_STATE, "pipelined transfers not enabled");
    const size_t n = c->n;
    const int s = c->up_slot;
    const XferSlot u = xfer_slot(c, s);
    cudaStream_t st = c->st, h = c->s_h2d;
    // the slot's previous upload has been unpacked
    cudaStreamWaitEvent(h, c->ev_up_free[s], 0);
    int rc = cuda_check(c, cudaMemcpyAsync(u.pos, pos, 3 * n * sizeof(double), cudaMemcpyDefault, h),
                        "upload pos");
    if (rc) return rc;
    cudaMemcpyAsync(u.vel, vel, 3 * n * sizeof(float), cudaMemcpyDefault, h);
    cudaMemcpyAsync(u.rho, rho, n * sizeof(float), cudaMemcpyDefault, h);
    cudaMemcpyAsync(u.ids, ids, n * sizeof(uint32_t), cudaMemcpyDefault, h);
    cudaEventRecord(c->ev_up_loaded[s], h);
    // the unpack replaces the state in stream order, after the copies
    cudaStreamWaitEvent(st, c->ev_up_loaded[s], 0);
    cudaMemsetAsync(c->id_flag, 0, sizeof(uint32_t), st);
    cudaMemsetAsync(c->i_vphase, 0, c->n_inst * sizeof(uint32_t), st);
    drop_pending_counts(c, st);
    k_unpack_ids<<<(uint32_t)((n + 255) / 256), 256, 0, st>>>(
        c->n, u.pos, u.vel, u.rho, u.ids, c->x[c->cur], c->y[c->cur], c->z[c->cur], c->vr[c->cur],
        c->id[c->cur], c->id_flag);
    rc = post_launch(c, "upload_async");
    if (rc) return rc;
    cudaEventRecord(c->ev_up_free[s], st);
    c->up_slot ^= 1;
    c->have_state = true;
    c->cells_valid = false;
    c->keys_ready = false;
    c->pre_state = 0;
    c->ids_pending = true;
    return cuda_check(c, cudaGetLastError(), "upload_async");
}

int sph_download_async(sph_ctx* c, double* pos, float* vel, float* rho, uint32_t* ids) {
    const TraceRange trace("sph_download_async");
    if (!c) return SPH_ERR_INVALID_ARG;
    if (!c->have_state) return fail(c, SPH_ERR_STATE, "no state uploaded");
    if (!c->xfer) return fail(c, SPH_ERR_STATE, "pipelined transfers not enabled");
    const size_t n = c->n;
    const XferSlot dn = xfer_slot(c, 2);
    cudaStream_t st = c->st, h = c->s_d2h;
    // the previous download's copies out of the slot have finished
    cudaStreamWaitEvent(st, c->ev_dn_free, 0);
    k_pack<<<(uint32_t)((n + 255) / 256), 256, 0, st>>>(c->n, c->x[c->cur], c->y[c->cur],
                                                       c->z[c->cur], c->vr[c->cur], dn.pos, dn.vel,
                                                       dn.rho, c->id[c->cur], dn.ids);
    int rc = post_launch(c, "download_async pack");
    if (rc) return rc;
    cudaEventRecord(c->ev_dn_packed, st);
    cudaStreamWaitEvent(h, c->ev_dn_packed, 0);
    if (pos) cudaMemcpyAsync(pos, dn.pos, 3 * n * sizeof(double), cudaMemcpyDefault, h);
    if (vel) cudaMemcpyAsync(vel, dn.vel, 3 * n * sizeof(float), cudaMemcpyDefault, h);
    if (rho) cudaMemcpyAsync(rho, dn.rho, n * sizeof(float), cudaMemcpyDefault, h);
    if (ids) cudaMemcpyAsync(ids, dn.ids, n * sizeof(uint32_t), cudaMemcpyDefault, h);
    cudaEventRecord(c->ev_dn_free, h);
    return cuda_check(c, cudaGetLastError(), "download_async");
}

int sph_sync_transfers(sph_ctx* c) {
    const TraceRange trace("sph_sync_transfers");
    if (!c) return SPH_ERR_INVALID_ARG;
    int rc = SPH_OK;
    if (c->s_h2d) {
        rc = cuda_check(c, cudaStreamSynchronize(c->s_h2d), "h2d stream");
        if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->s_d2h), "d2h stream");
    }
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->st), "stream");
    if (!rc && c->ids_pending) {
        uint32_t flag = 1;
        rc = cuda_check(c, cudaMemcpy(&flag, c->id_flag, sizeof(uint32_t), cudaMemcpyDeviceToHost),
                        "id check");
        c->ids_dense = rc == SPH_OK && flag == 0;
        c->ids_pending = false;
    }
    return rc;
}

void sph_destroy(sph_ctx* c) {
    if (!c) return;
    // work still queued may read the workspace or the transfer buffer, which
    // the caller frees after this call
    cudaStreamSynchronize(c->st);
    for (int g = 0; g < 2; ++g) {
        if (c->graph[g]) cudaGraphExecDestroy(c->graph[g]);
        if (c->loop_graph[g]) cudaGraphExecDestroy(c->loop_graph[g]);
    }
    release_transfer_streams(c);
    release_fork_stream(c);
    delete c;
}

uint64_t sph_radix_sort_scratch_bytes(uint32_t n) {
    Carver cv(nullptr);
    cv.take<uint32_t>(n);       // temporary keys
    cv.take<uint32_t>(n);       // temporary values
    cv.take<uint32_t>(4 * 256); // digit histograms
    cv.take<uint32_t>(4 + (size_t)4 * os_tiles(n) * 256);   // tile counters + status
    cv.take<uint32_t>(1);       // error word
    return (cv.used + kAlign - 1) / kAlign * kAlign;
}

int sph_radix_sort_pairs(const uint32_t* kin, const uint32_t* vin, uint32_t* kout, uint32_t* vout,
                         uint32_t n, uint32_t key_bits, void* scratch, uint64_t scratch_bytes,
                         void* stream) {
    if (!kin || !kout || !vout || !scratch) return SPH_ERR_INVALID_ARG;
    if (key_bits == 0 || key_bits > 32 || n >= (1u << 30)) return SPH_ERR_INVALID_ARG;
    if (((uintptr_t)scratch % kAlign) != 0 || scratch_bytes < sph_radix_sort_scratch_bytes(n))
        return SPH_ERR_WORKSPACE;
    if (n == 0) return SPH_OK;
    cudaStream_t st = (cudaStream_t)stream;
    Carver cv(scratch);
    uint32_t* tk = cv.take<uint32_t>(n);
    uint32_t* tv = cv.take<uint32_t>(n);
    uint32_t* hist = cv.take<uint32_t>(4 * 256);
    const uint32_t tiles = os_tiles(n);
    uint32_t* tilectr = cv.take<uint32_t>(4 + (size_t)4 * tiles * 256);
    uint32_t* err = cv.take<uint32_t>(1);
    const int passes = ((int)key_bits + 7) / 8;
    cudaMemsetAsync(hist, 0, 4 * 256 * sizeof(uint32_t), st);
    cudaMemsetAsync(tilectr, 0, (4 + (size_t)passes * tiles * 256) * sizeof(uint32_t), st);
    cudaMemsetAsync(err, 0, sizeof(uint32_t), st);
    launch_digit_hist(kin, n, passes, (int)key_bits, hist, st);
    // ping-pong so that the last pass lands in the outputs
    const uint32_t* ck = kin;
    const uint32_t* cv_ = vin;
    for (int p = 0; p < passes; ++p) {
        const bool to_out = ((passes - 1 - p) % 2) == 0;
        uint32_t* ok = to_out ? kout : tk;
        uint32_t* ov = to_out ? vout : tv;
        launch_onesweep_pass(ck, cv_, ok, ov, n, p, (int)key_bits, hist, tilectr + 4, tilectr, err, st);
        ck = ok;
        cv_ = ov;
    }
    return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}

// The error word of a scratch laid out by sph_radix_sort_pairs for n pairs.
static uint32_t* sort_err_word(void* scratch, uint32_t n) {
    Carver cv(scratch);
    cv.take<uint32_t>(n);
    cv.take<uint32_t>(n);
    cv.take<uint32_t>(4 * 256);
    cv.take<uint32_t>(4 + (size_t)4 * os_tiles(n) * 256);
    return cv.take<uint32_t>(1);
}

static int sort_scratch_args(const void* scratch, uint64_t scratch_bytes, uint32_t n) {
    if (!scratch || n == 0 || n >= (1u << 30)) return SPH_ERR_INVALID_ARG;
    if (((uintptr_t)scratch % kAlign) != 0 || scratch_bytes < sph_radix_sort_scratch_bytes(n))
        return SPH_ERR_WORKSPACE;
    return SPH_OK;
}

int sph_radix_sort_status(const void* d_scratch, uint64_t scratch_bytes, uint32_t n,
                          void* stream) {
    int rc = sort_scratch_args(d_scratch, scratch_bytes, n);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t word = 0;
    if (cudaMemcpyAsync(&word, sort_err_word(const_cast<void*>(d_scratch), n), sizeof(word),
                        cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return SPH_ERR_CUDA;
    return (word & kStatusTimeout) ? SPH_ERR_TIMEOUT : SPH_OK;
}

int sph_radix_sort_selftest_timeout(void* d_scratch, uint64_t scratch_bytes, uint32_t n,
                                    uint32_t polls, void* stream) {
    int rc = sort_scratch_args(d_scratch, scratch_bytes, n);
    if (rc) return rc;
    if (polls == 0 || polls > (1u << 20)) return SPH_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    Carver cv(d_scratch);
    cv.take<uint32_t>(n);
    cv.take<uint32_t>(n);
    cv.take<uint32_t>(4 * 256);
    uint32_t* tilectr = cv.take<uint32_t>(4 + (size_t)4 * os_tiles(n) * 256);
    uint32_t* err = cv.take<uint32_t>(1);
    cudaMemsetAsync(err, 0, sizeof(uint32_t), st);
    // tile 1 of the first pass waits on tile 0's status words, zeroed here
    // and published by nobody
    launch_lookback_selftest(tilectr + 4, polls, err, st);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
        return SPH_ERR_CUDA;
    return SPH_OK;
}

}  // extern "C"
