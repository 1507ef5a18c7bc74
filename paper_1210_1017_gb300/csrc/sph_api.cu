// C ABI of libsph.so (declared in include/sph.h): context, workspace
// layout, the step sequence and its CUDA-graph capture, host transfers.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "../../include/sph.h"
#include "sph_internal.cuh"

using namespace sph;

namespace {

constexpr size_t kAlign = 256;
constexpr uint32_t kMaxGridBlocks = 4096;   // partials of the persistent interaction

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
                         float4* vr) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    x[i] = pos[3 * (size_t)i];
    y[i] = pos[3 * (size_t)i + 1];
    z[i] = pos[3 * (size_t)i + 2];
    vr[i] = make_float4(vel[3 * (size_t)i], vel[3 * (size_t)i + 1], vel[3 * (size_t)i + 2], rho[i]);
}

__global__ void k_pack(uint32_t n, const double* __restrict__ x, const double* __restrict__ y,
                       const double* __restrict__ z, const float4* __restrict__ vr, double* pos,
                       float* vel, float* rho) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
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

struct sph_ctx {
    sph_params p;
    Dev d;
    uint32_t n = 0;
    cudaStream_t st = nullptr;
    int bits = 0, passes = 0;
    uint32_t tiles = 0, nparts = 0;
    uint64_t ncells = 0;
    uint32_t ncx_ = 1;        // cells per row (set before carving)
    // state, double-buffered for the reorder gather
    double *x[2], *y[2], *z[2];
    float4* vr[2];
    uint32_t* id[2];
    // start-of-step state: [0] written by the predictor, [1] after the
    // mid-step reorder (read by the corrector)
    double *px[2], *py[2], *pz[2];
    float4* pvr[2];
    float4 *posc, *ace;
    double* stage_pos;       // host transfer staging: 3n doubles
    float* stage_vr;         // 4n floats (velocity, then density)
    uint32_t *key[2], *val[2];
    uint32_t *cnt, *off, *bsum, *hist, *tilectr, *os_status, *nnb, *nnb64;
    uint32_t *ucnt, *uoff, *ubsum;   // work units of the interaction
    uint2* units;
    float4 *part_f, *lvl2_f;
    uint4* part_u;
    unsigned long long* lvl2_q;
    uint32_t *done, *status;
    double *dt, *t, *diag_out, *diag_part;
    float* terms;
    unsigned long long *counters, *step;
    size_t os_bytes = 0;
    // bookkeeping
    int cur = 0;             // state buffer index
    int skey = 0;            // key/val buffer holding the last sort result
    bool have_state = false;
    bool cells_valid = false;
    bool keys_ready = false; // labels + histograms already computed
    int pre_state = 0;       // 0 none, 1 in px[0] (unsorted), 2 in px[1] (sorted)
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    std::string err;
};

namespace {

int fail(sph_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

int cuda_check(sph_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return SPH_OK;
    return fail(c, SPH_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int validate(const sph_params* p, uint32_t n, uint64_t* ncells, uint32_t nc[3], std::string* why) {
    if (!p) {
        *why = "params is NULL";
        return SPH_ERR_INVALID_ARG;
    }
    if (n == 0 || n >= kMaxParticles) {
        *why = "n_particles must be in [1, 2^26)";
        return SPH_ERR_INVALID_ARG;
    }
    if (!(p->h > 0.0) || !(p->rho0 > 0.0) || !(p->c0 > 0.0) || !(p->mass > 0.0) ||
        !(p->cfl > 0.0) || !(p->alpha >= 0.0) || !(p->eta2_coef > 0.0)) {
        *why = "h, rho0, c0, mass, cfl, eta2_coef must be > 0 and alpha >= 0";
        return SPH_ERR_INVALID_ARG;
    }
    if (p->gamma != 7.0) {
        *why = "gamma must be 7 (Tait law of Sec. 2.2)";
        return SPH_ERR_INVALID_ARG;
    }
    const double cs = 2.0 * p->h;
    uint64_t total = 1;
    for (int a = 0; a < 3; ++a) {
        if (!(p->dmax[a] > p->dmin[a])) {
            *why = "dmax must exceed dmin on every axis";
            return SPH_ERR_INVALID_ARG;
        }
        const double t = ceil((p->dmax[a] - p->dmin[a]) / cs);
        if (!(t >= 1.0) || t > 65535.0) {
            *why = "grid must have 1..65535 cells per axis";
            return SPH_ERR_INVALID_ARG;
        }
        nc[a] = (uint32_t)t;
        total *= nc[a];
    }
    if (total >= (1ull << 31)) {
        *why = "cell grid must have fewer than 2^31 cells";
        return SPH_ERR_INVALID_ARG;
    }
    *ncells = total;
    return SPH_OK;
}

// Lay out every device buffer; with base == nullptr only sizes are computed.
size_t carve(sph_ctx* c, void* base, uint32_t n, uint64_t ncells, int passes) {
    Carver cv(base);
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
    c->cnt = cv.take<uint32_t>(ncells + 1);
    c->off = cv.take<uint32_t>(ncells + 2);
    c->bsum = cv.take<uint32_t>(scan_bsum_count(ncells + 1));
    c->hist = cv.take<uint32_t>(4 * 256);
    const uint32_t tiles = os_tiles(n);
    c->os_bytes = 4 * sizeof(uint32_t) + (size_t)passes * tiles * 256 * sizeof(uint32_t);
    c->tilectr = cv.take<uint32_t>(c->os_bytes / sizeof(uint32_t));
    c->os_status = c->tilectr ? c->tilectr + 4 : nullptr;
    const uint32_t nrows = (uint32_t)(ncells / c->ncx_);
    c->ucnt = cv.take<uint32_t>(nrows + 1);
    c->uoff = cv.take<uint32_t>(nrows + 2);
    c->ubsum = cv.take<uint32_t>(scan_bsum_count(nrows + 1));
    c->units = cv.take<uint2>(max_units(n, nrows, c->ncx_));
    const uint32_t np = kMaxGridBlocks;
    c->part_f = cv.take<float4>(np);
    c->part_u = cv.take<uint4>(np);
    c->lvl2_f = cv.take<float4>(kReduceBlocks);
    c->lvl2_q = cv.take<unsigned long long>(4 * kReduceBlocks);
    c->done = cv.take<uint32_t>(1);
    c->status = cv.take<uint32_t>(1);
    c->dt = cv.take<double>(1);
    c->t = cv.take<double>(1);
    c->diag_out = cv.take<double>(8);
    c->diag_part = cv.take<double>(8 * kDiagBlocks);
    c->terms = cv.take<float>(4);
    c->counters = cv.take<unsigned long long>(8);
    c->step = cv.take<unsigned long long>(1);
    return (cv.used + kAlign - 1) / kAlign * kAlign;
}

Dev make_dev(const sph_params* p, uint32_t n, const uint32_t nc[3], uint64_t ncells) {
    Dev d;
    memset(&d, 0, sizeof(d));
    const double cs = 2.0 * p->h;
    d.x0 = p->dmin[0];
    d.y0 = p->dmin[1];
    d.z0 = p->dmin[2];
    d.inv_cs = 1.0 / cs;
    d.cs = cs;
    d.r2max_d = cs * cs;
    d.h_d = p->h;
    d.cfl = p->cfl;
    d.dt_fixed = p->dt_fixed;
    d.ncx = (int)nc[0];
    d.ncy = (int)nc[1];
    d.ncz = (int)nc[2];
    d.ncells = (uint32_t)ncells;
    d.n = n;
    d.n_bound = p->n_bound;
    d.csf = (float)cs;
    d.h = (float)p->h;
    d.inv_h = (float)(1.0 / p->h);
    d.r2max = (float)(cs * cs);
    d.eta2 = (float)(p->eta2_coef * p->h * p->h);
    const double aD = 21.0 / (16.0 * M_PI * p->h * p->h * p->h);
    d.fc = (float)(-5.0 * aD / (p->h * p->h));
    d.alpha = (float)p->alpha;
    d.c0 = (float)p->c0;
    d.rho0 = (float)p->rho0;
    d.inv_rho0 = (float)(1.0 / p->rho0);
    d.B = (float)(p->c0 * p->c0 * p->rho0 / p->gamma);
    d.mass = (float)p->mass;
    d.mass_d = p->mass;
    d.rho0_d = p->rho0;
    d.B_d = p->c0 * p->c0 * p->rho0 / p->gamma;
    for (int k = 0; k < 3; ++k) d.g_d[k] = p->gravity[k];
    d.gx = (float)p->gravity[0];
    d.gy = (float)p->gravity[1];
    d.gz = (float)p->gravity[2];
    return d;
}

// Sort the labels in key[0] (counted into cnt/hist by the label kernel),
// scan the counts into cell offsets and reorder the state (and the start
// state when with_pre).
void rebuild_after_keys(sph_ctx* c, bool with_pre) {
    cudaStream_t st = c->st;
    launch_scan_cells(c->d, c->cnt, c->bsum, c->off, st);
    cudaMemsetAsync(c->tilectr, 0, c->os_bytes, st);
    int src = 0;
    for (int p = 0; p < c->passes; ++p) {
        launch_onesweep_pass(c->key[src], p == 0 ? nullptr : c->val[src], c->key[1 - src],
                             c->val[1 - src], c->n, p, c->bits, c->hist,
                             c->os_status, c->tilectr, c->status, st);
        src = 1 - src;
    }
    c->skey = src;
    launch_units(c->d, c->off, c->ucnt, c->ubsum, c->uoff, c->units, st);
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
    }
    ra.posc = c->posc;
    ra.hist_to_zero = c->hist;
    ra.status = c->status;
    launch_reorder(c->d, ra, st);
    c->cur = d;
}

void enqueue_interact(sph_ctx* c, bool counts, bool set_dt) {
    InteractArgs ia;
    ia.units = c->units;
    ia.n_units = c->uoff + (c->ncells / c->ncx_);
    ia.status = c->status;
    ia.posc = c->posc;
    ia.velrhop = c->vr[c->cur];
    ia.key = c->key[c->skey];
    ia.id = c->id[c->cur];
    ia.off = c->off;
    ia.ace = c->ace;
    ia.nnb = c->nnb;
    ia.part_f = c->part_f;
    ia.part_u = c->part_u;
    launch_interact(c->d, ia, counts, c->st);
    ReduceArgs ra;
    ra.part_f = c->part_f;
    ra.part_u = c->part_u;
    ra.nparts = c->nparts;
    ra.lvl2_f = c->lvl2_f;
    ra.lvl2_q = c->lvl2_q;
    ra.done = c->done;
    ra.dt = c->dt;
    ra.terms = c->terms;
    ra.counters = c->counters;
    ra.status = c->status;
    launch_dt_reduce(c->d, ra, set_dt, c->st);
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
    a.dt = c->dt;
    a.t = c->t;
    a.step = c->step;
    a.key = c->key[0];
    a.cnt = c->cnt;
    a.hist = c->hist;
    a.passes = c->passes;
    return a;
}

void enqueue_build(sph_ctx* c) {
    if (!c->keys_ready) {
        launch_keys(c->d, c->x[c->cur], c->y[c->cur], c->z[c->cur], c->n, c->key[0], c->cnt,
                    c->hist, c->passes, c->st);
    }
    const bool with_pre = c->pre_state == 1;
    rebuild_after_keys(c, with_pre);
    if (with_pre) c->pre_state = 2;
    c->keys_ready = false;
    c->cells_valid = true;
}

// One full step on the current buffers (state starts and ends in c->cur).
void enqueue_step(sph_ctx* c) {
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

int post_launch(sph_ctx* c, const char* what) {
    return cuda_check(c, cudaGetLastError(), what);
}

}  // namespace

extern "C" {

int sph_query_sizes(const sph_params* params, uint32_t n, sph_sizes* out) {
    if (!out) return SPH_ERR_INVALID_ARG;
    uint64_t ncells;
    uint32_t nc[3];
    std::string why;
    int rc = validate(params, n, &ncells, nc, &why);
    if (rc) return rc;
    sph_ctx tmp;
    tmp.ncx_ = nc[0];
    const int bits = bit_length(ncells);
    const int passes = (bits + 7) / 8;
    out->workspace_bytes = carve(&tmp, nullptr, n, ncells, passes);
    out->ncells = ncells;
    out->ncx = nc[0];
    out->ncy = nc[1];
    out->ncz = nc[2];
    out->sort_passes = (uint32_t)passes;
    return SPH_OK;
}

int sph_init(const sph_params* params, uint32_t n, void* ws, uint64_t ws_bytes, void* stream,
             sph_ctx** out) {
    if (!out) return SPH_ERR_INVALID_ARG;
    *out = nullptr;
    uint64_t ncells;
    uint32_t nc[3];
    std::string why;
    int rc = validate(params, n, &ncells, nc, &why);
    if (rc) return rc;
    if (!ws || ((uintptr_t)ws % kAlign) != 0) return SPH_ERR_WORKSPACE;
    sph_ctx* c = new sph_ctx();
    c->p = *params;
    c->n = n;
    c->st = (cudaStream_t)stream;
    c->ncells = ncells;
    c->bits = bit_length(ncells);
    c->passes = (c->bits + 7) / 8;
    c->ncx_ = nc[0];
    const size_t need = carve(c, ws, n, ncells, c->passes);
    if (ws_bytes < need) {
        delete c;
        return SPH_ERR_WORKSPACE;
    }
    c->tiles = os_tiles(n);
    prepare_interact();
    c->nparts = interact_grid();
    if (c->nparts == 0 || c->nparts > kMaxGridBlocks) {
        delete c;
        return SPH_ERR_CUDA;
    }
    c->d = make_dev(params, n, nc, ncells);
    cudaStream_t st = c->st;
    cudaMemsetAsync(c->cnt, 0, (ncells + 1) * sizeof(uint32_t), st);
    cudaMemsetAsync(c->hist, 0, 4 * 256 * sizeof(uint32_t), st);
    cudaMemsetAsync(c->done, 0, sizeof(uint32_t), st);
    cudaMemsetAsync(c->status, 0, sizeof(uint32_t), st);
    cudaMemsetAsync(c->t, 0, sizeof(double), st);
    cudaMemsetAsync(c->counters, 0, 8 * sizeof(unsigned long long), st);
    cudaMemsetAsync(c->step, 0, sizeof(unsigned long long), st);
    cudaMemsetAsync(c->terms, 0, 4 * sizeof(float), st);
    const double dt0 = params->dt_fixed > 0.0 ? params->dt_fixed : 0.0;
    cudaMemcpyAsync(c->dt, &dt0, sizeof(double), cudaMemcpyHostToDevice, st);
    rc = cuda_check(c, cudaStreamSynchronize(st), "sph_init");
    if (rc) {
        delete c;
        return rc;
    }
    *out = c;
    return SPH_OK;
}

int sph_upload(sph_ctx* c, const double* pos, const float* vel, const float* rho,
               const uint32_t* ids) {
    if (!c || !pos || !vel || !rho || !ids) return fail(c, SPH_ERR_INVALID_ARG, "NULL argument");
    const size_t n = c->n;
    cudaStream_t st = c->st;
    double* dpos = c->stage_pos;
    float* dvel = c->stage_vr;
    float* drho = c->stage_vr + 3 * n;
    int rc = cuda_check(c, cudaMemcpyAsync(dpos, pos, 3 * n * sizeof(double), cudaMemcpyHostToDevice, st), "upload pos");
    if (rc) return rc;
    cudaMemcpyAsync(dvel, vel, 3 * n * sizeof(float), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(drho, rho, n * sizeof(float), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(c->id[c->cur], ids, n * sizeof(uint32_t), cudaMemcpyHostToDevice, st);
    k_unpack<<<(uint32_t)((n + 255) / 256), 256, 0, st>>>(c->n, dpos, dvel, drho, c->x[c->cur],
                                                         c->y[c->cur], c->z[c->cur], c->vr[c->cur]);
    rc = post_launch(c, "upload");
    if (rc) return rc;
    c->have_state = true;
    c->cells_valid = false;
    c->keys_ready = false;
    c->pre_state = 0;
    return cuda_check(c, cudaStreamSynchronize(st), "upload sync");
}

int sph_build_cells(sph_ctx* c) {
    if (!c) return SPH_ERR_INVALID_ARG;
    if (!c->have_state) return fail(c, SPH_ERR_STATE, "no state uploaded");
    enqueue_build(c);
    return post_launch(c, "build_cells");
}

int sph_interact(sph_ctx* c, uint32_t flags) {
    if (!c) return SPH_ERR_INVALID_ARG;
    if (!c->cells_valid) return fail(c, SPH_ERR_STATE, "cells not built");
    // at the half step (predictor pending) the step size stays the one set
    // by the evaluation at the start of the step, as in sph_step
    enqueue_interact(c, (flags & SPH_INTERACT_COUNTS) != 0, c->pre_state != 2);
    return post_launch(c, "interact");
}

int sph_predict(sph_ctx* c) {
    if (!c) return SPH_ERR_INVALID_ARG;
    if (!c->cells_valid) return fail(c, SPH_ERR_STATE, "cells not built");
    launch_predict(c->d, integrate_args(c, 0), c->st);
    c->keys_ready = true;
    c->pre_state = 1;
    c->cells_valid = false;
    return post_launch(c, "predict");
}

int sph_correct(sph_ctx* c) {
    if (!c) return SPH_ERR_INVALID_ARG;
    if (!c->cells_valid || c->pre_state != 2)
        return fail(c, SPH_ERR_STATE, "correct needs predict, build_cells and interact first");
    launch_correct(c->d, integrate_args(c, 1), c->st);
    c->keys_ready = true;
    c->pre_state = 0;
    c->cells_valid = false;
    return post_launch(c, "correct");
}

int sph_step(sph_ctx* c, uint32_t nsteps) {
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
    const int g = c->cur;
    if (!c->graph[g]) {
        cudaGraph_t graph;
        int rc = cuda_check(c, cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal),
                            "begin capture");
        if (rc) return rc;
        enqueue_step(c);
        rc = cuda_check(c, cudaStreamEndCapture(c->st, &graph), "end capture");
        if (rc) return rc;
        rc = cuda_check(c, cudaGraphInstantiate(&c->graph[g], graph, 0), "instantiate");
        cudaGraphDestroy(graph);
        if (rc) return rc;
        if (c->cur != g) return fail(c, SPH_ERR_STATE, "step changed buffer parity");
    }
    for (uint32_t s = 0; s < nsteps; ++s) {
        int rc = cuda_check(c, cudaGraphLaunch(c->graph[g], c->st), "graph launch");
        if (rc) return rc;
    }
    return SPH_OK;
}

int sph_rollout(sph_ctx* c, uint32_t nsteps, uint32_t save_every, sph_snapshot_fn cb,
                void* user) {
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
        if (cb) {
            double t = 0.0;
            unsigned long long s = 0;
            cudaMemcpy(&t, c->t, sizeof(double), cudaMemcpyDeviceToHost);
            cudaMemcpy(&s, c->step, sizeof(s), cudaMemcpyDeviceToHost);
            if (cb(user, s, t)) break;
        }
    }
    return SPH_OK;
}

int sph_download(sph_ctx* c, double* pos, float* vel, float* rho, uint32_t* ids) {
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
    if (pos) cudaMemcpyAsync(pos, dpos, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (vel) cudaMemcpyAsync(vel, dv, 3 * n * sizeof(float), cudaMemcpyDeviceToHost, st);
    if (rho) cudaMemcpyAsync(rho, dr, n * sizeof(float), cudaMemcpyDeviceToHost, st);
    if (ids) cudaMemcpyAsync(ids, c->id[c->cur], n * sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    return cuda_check(c, cudaStreamSynchronize(st), "download");
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
        case SPH_ARRAY_DT: return 8;
        default: return 0;
    }
}

int sph_read_array(sph_ctx* c, int which, void* host, uint64_t bytes) {
    if (!c || !host) return fail(c, SPH_ERR_INVALID_ARG, "NULL argument");
    const uint64_t want = sph_array_bytes(c, which);
    if (want == 0 || bytes != want) return fail(c, SPH_ERR_INVALID_ARG, "bad array id or size");
    const void* src = nullptr;
    switch (which) {
        case SPH_ARRAY_KEY: src = c->key[c->skey]; break;
        case SPH_ARRAY_CELL_OFF: src = c->off; break;
        case SPH_ARRAY_ACE: src = c->ace; break;
        case SPH_ARRAY_NNB: src = c->nnb; break;
        case SPH_ARRAY_NNB64: src = c->nnb64; break;
        case SPH_ARRAY_POSC: src = c->posc; break;
        case SPH_ARRAY_DT: src = c->dt; break;
    }
    int rc = cuda_check(c, cudaMemcpyAsync(host, src, bytes, cudaMemcpyDeviceToHost, c->st), "read array");
    if (rc) return rc;
    return cuda_check(c, cudaStreamSynchronize(c->st), "read array sync");
}

int sph_neighbour_counts_fp64(sph_ctx* c) {
    if (!c) return SPH_ERR_INVALID_ARG;
    if (!c->cells_valid) return fail(c, SPH_ERR_STATE, "cells not built");
    launch_counts_fp64(c->d, c->x[c->cur], c->y[c->cur], c->z[c->cur], c->key[c->skey], c->off,
                       c->nnb64, c->st);
    return post_launch(c, "counts_fp64");
}

int sph_diagnostics(sph_ctx* c, sph_diag* out) {
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
    cudaMemcpyAsync(&t, c->t, sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&dt, c->dt, sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(cnt, c->counters, sizeof(cnt), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&step, c->step, sizeof(step), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(terms, c->terms, sizeof(terms), cudaMemcpyDeviceToHost, st);
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

int sph_check(sph_ctx* c) {
    if (!c) return SPH_ERR_INVALID_ARG;
    uint32_t status = 0;
    int rc = cuda_check(c, cudaMemcpyAsync(&status, c->status, sizeof(status), cudaMemcpyDeviceToHost, c->st), "check");
    if (rc) return rc;
    rc = cuda_check(c, cudaStreamSynchronize(c->st), "check sync");
    if (rc) return rc;
    if (status & SPH_STATUS_TIMEOUT) return fail(c, SPH_ERR_TIMEOUT, "radix sort look-back gave up");
    if (status & SPH_STATUS_NONFINITE) return fail(c, SPH_ERR_NONFINITE, "non-finite interaction result");
    if (status & SPH_STATUS_CAPACITY) return fail(c, SPH_ERR_CAPACITY, "a cell exceeded the id tie-break capacity");
    return SPH_OK;
}

uint32_t sph_kernels_per_step(const sph_ctx* c) {
    if (!c) return 0;
    // 2 x (interact + reduce) + predict + correct
    // + 2 x (3 cell scan + passes + 5 unit list + reorder)
    return 2u * 2u + 2u + 2u * (3u + (uint32_t)c->passes + 5u + 1u);
}

const char* sph_last_error(const sph_ctx* c) { return c ? c->err.c_str() : "NULL context"; }

void sph_destroy(sph_ctx* c) {
    if (!c) return;
    for (int g = 0; g < 2; ++g)
        if (c->graph[g]) cudaGraphExecDestroy(c->graph[g]);
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

}  // extern "C"
