// The SPH context (private to libsph.so; shared by the SPH and surrogate
// translation units).
#pragma once
#include <nvtx3/nvToolsExt.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sph.h"
#include "sph_internal.cuh"

namespace sph {

// Host view of the ensemble: the device table plus its search arrays.
struct Table {
    std::vector<Inst> inst;
    std::vector<uint32_t> cell_base, row_base, id_base;   // n_inst + 1 each
    uint64_t ncells = 0, nrows = 0, n = 0;
    int max_ncx = 1;
};

}  // namespace sph

struct sph_ctx {
    sph_params p;
    sph::Dev d;
    sph::Table tab;
    uint32_t n = 0, n_inst = 1;
    cudaStream_t st = nullptr;
    int bits = 0, passes = 0;
    uint32_t tiles = 0, nparts = 0;
    uint64_t ncells = 0;
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
    uint32_t *cnt, *off, *hist, *tilectr, *os_status, *nnb, *nnb64;
    uint32_t *ucnt, *uoff, *ubsum;   // work units of the interaction
    uint32_t* csum;                  // staged-candidate prefix sums per row
    unsigned long long* cscan_words; // one-launch cell scan: look-back word per tile
    uint32_t* cscan_ctl;             // one-launch cell scan: tile ticket, launch epoch
    unsigned long long* urow;        // one-launch unit list: look-back word per row
    uint32_t* uctl;                  // one-launch unit list: row ticket, launch epoch
    bool units_one = false;          // build the unit list in one launch
    uint32_t units_cap = 0;          // capacity of `units`
    uint2* units;
    uint4* part_u;
    uint32_t *done, *status;
    uint32_t* id_flag;       // set by the upload when some id >= n
    // sub-domain selection (Sec. 4.3): ping-pong (key, value) arrays of the
    // selected particles for the radix sorts, their digit histograms (4
    // passes by id + 1 by label), tile counters and look-back status, and
    // the label counters
    uint32_t *sub_key[2], *sub_val[2];
    uint32_t *sub_hist, *sub_os, *sub_cnt;
    size_t sub_os_bytes = 0;
    double *diag_out, *diag_part;
    unsigned long long* front;   // per-member front images (sph_front)
    unsigned long long* counters;
    // ensemble table and per-member state (device)
    sph::Inst* d_inst;
    uint32_t *d_cell_base, *d_row_base, *d_id_base;
    double *i_dt, *i_t;
    uint32_t *i_done, *i_terms;
    unsigned long long* i_steps;
    float* i_last;
    uint32_t* i_vphase;      // Verlet phase per member
    size_t os_bytes = 0;
    // bookkeeping
    int variant = 0;         // interaction block shape (see sph_autotune)
    int cur = 0;             // state buffer index
    int skey = 0;            // key/val buffer holding the last sort result
    bool have_state = false;
    bool ids_dense = false;  // every id < n (ids then index by-id arrays)
    bool cells_valid = false;
    bool keys_ready = false; // labels + histograms already computed
    int pre_state = 0;       // 0 none, 1 in px[0] (unsorted), 2 in px[1] (sorted)
    bool verlet = false;     // Verlet integrator: pvr[0] / pvr[1] hold (v, rho) one
                             // step earlier, before / after the reorder
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    // sph_step(n): one graph per start parity whose conditional WHILE node
    // repeats a body of loop_body steps on the device (see sph_step)
    cudaGraphExec_t loop_graph[2] = {nullptr, nullptr};
    uint32_t* loop_ctr = nullptr;   // [0] steps done in this launch, [1] steps asked
    // a second stream for the unit list: after the cell scan each rebuild
    // forks the unit-list kernels onto it and joins them before the
    // interaction, so they run beside the cell scatter and the reorder (both
    // only need the cell offsets); null on the legacy default stream
    cudaStream_t st_units = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // pipelined transfers (sph_enable_async_transfers): a caller-owned buffer
    // of three staging slots (two for uploads, one for downloads), a copy
    // stream per direction and the events that order them with c->st
    unsigned char* xfer = nullptr;
    uint64_t xfer_slot = 0;          // bytes per slot
    cudaStream_t s_h2d = nullptr, s_d2h = nullptr;
    cudaEvent_t ev_up_loaded[2] = {nullptr, nullptr}, ev_up_free[2] = {nullptr, nullptr};
    cudaEvent_t ev_dn_packed = nullptr, ev_dn_free = nullptr;
    int up_slot = 0;                 // upload slot of the next sph_upload_async
    bool ids_pending = false;        // ids_dense not yet read back after an async upload
    std::string err;
};

namespace sph {

// Host-side range around a C-ABI call (NVTX, header-only): profilers that
// read NVTX (nsys timelines, ncu --nvtx-include) see which call enqueued
// which kernels.  Without an attached tool a push/pop is a null check.
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

// The state is being replaced (an upload, a surrogate advance): labels that
// sph_predict / sph_correct / sph_verlet computed and counted into the
// per-cell counts for the next rebuild no longer apply.  Clear those counts,
// since the next rebuild counts the new labels from zero.
inline void drop_pending_counts(sph_ctx* c, cudaStream_t st) {
    if (c->keys_ready) cudaMemsetAsync(c->cnt, 0, (c->ncells + 1) * sizeof(uint32_t), st);
    c->keys_ready = false;
}

// Record a one-line error message on the context and return the code.
inline int fail(sph_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

// SPH_OK, or SPH_ERR_CUDA with the runtime's message.
inline int cuda_check(sph_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return SPH_OK;
    return fail(c, SPH_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace sph

