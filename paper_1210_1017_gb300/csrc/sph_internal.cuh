// Private declarations shared by the CUDA translation units of libsph.so.
//
// A context holds an ensemble of one or more independent simulations
// ("instances") that share the smoothing length, particle mass and the
// physical constants except c0, and run in lockstep: one cell sort, one
// interaction launch and one integrator launch serve all of them.  Instance
// q owns the particle ids [id_base, id_end) (boundary particles first) and
// the global cell labels [cell_base, cell_base + ncx ncy ncz); its rows of
// cells (cy, cz) are the global rows [row_base, row_base + ncy ncz).  A
// single simulation is the ensemble of one.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

namespace sph {

constexpr uint32_t kStatusTimeout = 1u;
constexpr uint32_t kStatusNonFinite = 2u;
constexpr uint32_t kStatusCapacity = 4u;
constexpr uint32_t kStatusBounds = 8u;

// The checked build (compiled with -DSPH_CHECKED, loaded as
// libsph_checked.so) tests the array indexes its kernels compute (staged
// and global candidate indexes, gather and scatter slots, cell offsets, the
// unit list) before using them.  An index out of range sets kStatusBounds
// in the context's status word and the access is skipped (the index is
// replaced by a safe one), so a wrong index is reported, never followed and
// never trapped.  In the normal build the tests compile away.
#ifdef SPH_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

// True when ok; otherwise (checked build only) records kStatusBounds.
__device__ __forceinline__ bool in_bounds(bool ok, uint32_t* status) {
    if (kChecked && !ok) {
        atomicOr(status, kStatusBounds);
        return false;
    }
    return true;
}

// Largest particle count (FP64 counts and ids stay within 32 bits with room).
constexpr uint32_t kMaxParticles = 1u << 26;

// One instance of the ensemble (device table entry).
struct Inst {
    double x0, y0, z0;      // grid origin
    double t_end;           // the instance stops (dt = 0) once t >= t_end
    int ncx, ncy, ncz;
    uint32_t cell_base;
    uint32_t row_base;
    uint32_t id_base;
    uint32_t id_fluid;      // ids in [id_base, id_fluid) are boundary particles
    uint32_t id_end;
    float c0;               // reference speed of sound
    float B;                // Tait stiffness c0^2 rho0 / gamma
    double B_d;             // the same in FP64 (conservation sums)
};

// Per-instance device state.
struct InstState {
    double* dt;             // step size of the current step
    double* t;              // simulated time
    uint32_t* done;         // 1 once t >= t_end
    unsigned long long* steps;
    uint32_t* terms;        // 3 per instance, float bits of the running maxima of
                            // |a|^2, c and mu over the current evaluation
    float* last;            // 3 per instance: max |a|, max c, max mu of the last one
    uint32_t* vphase;       // Verlet: steps since the last Euler step (0: the next
                            // step is an Euler step); reset by an upload
};

// Per-context constants handed to kernels by value.
struct Dev {
    const Inst* inst;
    const uint32_t* cell_base;   // n_inst + 1 entries (last = ncells)
    const uint32_t* row_base;    // n_inst + 1 entries (last = nrows)
    const uint32_t* id_base;     // n_inst + 1 entries (last = n)
    uint32_t n_inst;
    InstState is;
    double inv_cs;         // 1 / (2h), rounded once (cell label arithmetic)
    double cs;             // 2h
    double r2max_d;        // (2h)^2 rounded once (FP64 neighbour predicate)
    double h_d, cfl, dt_fixed;
    double mass_d, rho0_d;
    double g_d[3];
    uint32_t ncells;       // all instances' cells; also the label of excluded particles
    uint32_t nrows;        // all instances' rows of cells
    uint32_t n;
    int max_ncx;
    int variant;           // interaction variant (block shape) in use
    int unit;              // its unit size in particles
    int stage;             // its staging capacity in candidates
    int units_fused;       // the unit list is built in one launch (k_units_fused)
    uint32_t units_cap;    // capacity of the unit list
    uint32_t* status;      // the context's device status word
    float csf;             // 2h
    float h, inv_h;
    float r2max;           // (2h)^2 in FP32
    float eta2;            // eta^2
    float fc;              // gradient factor: -5 aD/h^2 (Wendland C2) or aD/h^2
                           // (cubic spline, aD = 1/(pi h^3))
    int kern;              // 0: Wendland C2, 1: cubic spline (Sec. 2.2)
    uint32_t verlet_every; // Verlet: an Euler step every this many steps
    float alpha, rho0, inv_rho0, mass;
    float gx, gy, gz;
};

// Stream-ordered launchers (defined in the .cu files).
void launch_keys(const Dev& d, const double* x, const double* y, const double* z,
                 const uint32_t* id, uint32_t n, uint32_t* key, uint32_t* cnt, uint32_t* hist,
                 int passes, cudaStream_t st);
// Cell offsets from the per-cell counts (kept: the cell sort's scatter
// counts them back down) in one launch (launch_scan_onepass).
void launch_scan_cells(const Dev& d, uint32_t* cnt, uint32_t* off, unsigned long long* words,
                       uint32_t* ctl, uint32_t* err, cudaStream_t st);
// out[i] = in[0] + ... + in[i-1] for i = 0..m (m + 1 outputs); clears in[]
// unless zero_in is false.
void launch_scan(uint32_t* in, uint64_t m, uint32_t* bsum, uint32_t* out, cudaStream_t st,
                 bool zero_in = true);
// The same in one launch, with a decoupled look-back between tiles: words
// holds scan_bsum_count(m) look-back words and ctl a ticket and an epoch,
// all zero before the first launch and kept by the caller between launches
// (one set per stream of successive scans).  A look-back that gives up sets
// kStatusTimeout in *err.
void launch_scan_onepass(uint32_t* in, uint64_t m, uint32_t* out, bool zero_in,
                         unsigned long long* words, uint32_t* ctl, uint32_t* err,
                         cudaStream_t st);
// One-pass counting sort of the cell labels (keys; values = input index)
// into (kout, vout), from the per-cell counts cnt (counted back to zero) and
// the cell offsets off.  Order inside a cell is arbitrary.
void launch_cell_scatter(const uint32_t* key, uint32_t n, const uint32_t* off, uint32_t* cnt,
                         uint32_t* kout, uint32_t* vout, uint32_t* status, cudaStream_t st);
uint32_t scan_bsum_count(uint64_t m);

// Radix sort
constexpr int kOsThreads = 256;
constexpr int kOsItems = 16;
constexpr int kOsTile = kOsThreads * kOsItems;
inline uint32_t os_tiles(uint32_t n) { return (n + kOsTile - 1) / kOsTile; }
void launch_digit_hist(const uint32_t* keys, uint32_t n, int passes, int bits_total,
                       uint32_t* hist, cudaStream_t st);
// Failure-path self-test: the radix sort's look-back waits on 256 status
// words that nothing sets (zeroed here) and gives up after `limit` polls,
// setting kStatusTimeout in *err.
void launch_lookback_selftest(uint32_t* zeroed256, uint32_t limit, uint32_t* err,
                              cudaStream_t st);
void launch_onesweep_pass(const uint32_t* kin, const uint32_t* vin, uint32_t* kout,
                          uint32_t* vout, uint32_t n, int pass, int bits_total,
                          const uint32_t* hist, uint32_t* status, uint32_t* tilectr,
                          uint32_t* err, cudaStream_t st);

struct ReorderArgs {
    const uint32_t* skey;
    const uint32_t* sval;
    const uint32_t* off;
    const double *sx, *sy, *sz;
    const float4* svr;
    const uint32_t* sid;
    const double *spx, *spy, *spz;   // pre state (may be null)
    const float4* spvr;
    double *dx, *dy, *dz;
    float4* dvr;
    uint32_t* did;
    double *dpx, *dpy, *dpz;
    float4* dpvr;
    float4* posc;
    uint32_t* hist_to_zero;          // cleared for the next rebuild
    uint32_t* status;
};
void launch_reorder(const Dev& d, const ReorderArgs& a, cudaStream_t st);

// Interaction work unit: up to `unit` consecutive particles of one row of
// cells spanning at most kSpan cells (uint2: first particle, end).  The unit
// size is the block size of the interaction variant in use.
constexpr int kSpan = 32;
constexpr int kMinUnit = 32;
constexpr int kNumVariants = 16;

struct ReduceArgs {
    const uint4* part_u;
    uint32_t nparts;
    // [0] pairs total, [1] candidates total, [2] pairs last, [3] candidates
    // last, [4] fluid-i pairs last, [5] boundary-i pairs last, [6] fluid-i
    // pairs total, [7] boundary-i pairs total
    unsigned long long* counters;
    uint32_t* status;
};

struct InteractArgs {
    const uint2* units;
    const uint32_t* n_units;
    uint32_t* status;
    const float4* posc;
    const float4* velrhop;
    const uint32_t* key;
    const uint32_t* id;
    const uint32_t* off;
    float4* ace;
    uint32_t* nnb;        // may be null
    uint4* part_u;        // per block (persistent grid): fluid-i pairs, candidates,
                          // status bits, boundary-i pairs
    uint32_t* ticket;     // non-null: the last block runs the Sec. 3.3 reductions
                          // (zero on entry, left at zero)
    uint32_t* sched;      // unit counter and finish ticket of the variants that
                          // take units from a counter (zero on entry, left at zero)
    ReduceArgs red;
    int set_dt;
};
uint32_t max_units(uint32_t n, uint32_t nrows, uint64_t ncells);   // bound on units
int variant_unit(int variant);               // particles per unit of a variant
int variant_stage(int variant);              // staged candidates of a variant
uint32_t interact_grid(int variant);         // blocks of its persistent launch
// Grids of few, short rows build the unit list in one launch (row sums,
// counts, a look-back over rows, the fill); others take row sums, counts, a
// scan and the fill as separate launches.
struct UnitsFusedArgs {
    uint2* units;
    uint32_t* total;                 // number of units (uoff[nrows])
    unsigned long long* words;       // per-row look-back words (nrows)
    uint32_t* ctl;                   // row ticket, launch epoch (zero at init)
    uint32_t* err;                   // device status word
};
bool units_fused(const Dev& d);
bool units_fit_one_launch(uint32_t nrows, int max_ncx);   // the grid qualifies
// Failure-path self-test: the one-launch unit list's row look-back waits on
// a word that nothing publishes (zeroed here) and gives up after `limit`
// polls, setting kStatusTimeout in *err.
void launch_row_lookback_selftest(unsigned long long* zeroed, uint32_t limit, uint32_t* err,
                                  cudaStream_t st);
void launch_units(const Dev& d, const uint32_t* off, uint32_t* csum, uint32_t* ucnt,
                  uint32_t* ubsum, uint32_t* uoff, uint2* units, unsigned long long* urow,
                  uint32_t* uctl, uint32_t* err, cudaStream_t st);
// Once per context (current device): opt in to the shared memory and size
// the persistent grid from the device's SM count and occupancy.
void prepare_interact();
void launch_interact(const Dev& d, const InteractArgs& a, bool counts, cudaStream_t st);

// Decoupled look-back over tiles handed out in launch order (the one-launch
// unit list's rows, the one-launch scan's tiles).  A tile's word is
// epoch << 34 | flag << 32 | value, flag 1 for the tile's own total and 2
// for the inclusive prefix through it; the epoch (launch number mod 2^30)
// makes words of earlier launches read as not yet published, so the words
// are never cleared.  tile_lookback returns the sum over tiles 0 .. r-1 (the
// whole warp; lane j reads tile p - j of a window of 32 below the next
// unread tile p).  A wait that sees no progress for `limit` polls sets
// kStatusTimeout in *err and returns the partial sum, which never exceeds
// the true one.
__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t tile_lookback(const unsigned long long* words, uint32_t r,
                                                  uint32_t ep, uint32_t limit, uint32_t* err) {
    constexpr unsigned kAll = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    uint32_t excl = 0, spins = 0;
    int64_t p = (int64_t)r - 1;
    while (true) {
        const int64_t q = p - lane;
        uint32_t flag = 2u, val = 0u;   // before tile 0: a prefix of 0
        if (q >= 0) {
            const unsigned long long s = ld_relaxed64(words + q);
            flag = (uint32_t)(s >> 34) == ep ? (uint32_t)(s >> 32) & 3u : 0u;
            val = (uint32_t)s;
        }
        const uint32_t waiting = __ballot_sync(kAll, flag == 0u);
        const uint32_t prefix = __ballot_sync(kAll, flag == 2u);
        const int fw = waiting ? __ffs(waiting) - 1 : 32;
        const int fp = prefix ? __ffs(prefix) - 1 : 32;
        if (fp < fw) return excl + __reduce_add_sync(kAll, lane <= fp ? val : 0u);
        excl += __reduce_add_sync(kAll, lane < fw ? val : 0u);
        p -= fw;
        if (fw == 0 && ++spins > limit) {
            if (lane == 0) atomicOr(err, kStatusTimeout);
            return excl;
        }
    }
}

// Programmatic dependent launch of the step's kernels: a kernel launched
// with it may be scheduled while the previous kernel of its stream drains,
// and it calls pdl_wait() before touching global memory; that returns once
// the previous kernel has completed and its writes are visible.  Since every
// such kernel waits first, each also completes after all earlier work of the
// stream.  pdl_enabled() is decided once per process by prepare_interact:
// off when the environment sets SPH_PDL=0 or when the driver does not accept
// the launches inside a captured conditional node's body.
bool pdl_enabled();
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
template <typename... K, typename... A>
inline cudaError_t launch_pdl(void (*k)(K...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, A&&... args) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 1u : 0u;
    return cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
}


struct IntegrateArgs {
    const uint32_t* off;     // for the in-domain count
    double *x, *y, *z;
    float4* velrhop;
    const uint32_t* id;
    const float4* ace;
    double *px, *py, *pz;    // pre state: written by predict, read by correct
    float4* pvr;
    float4* pvr_out;         // Verlet: receives (v, rho) on entry
    uint32_t* key;
    uint32_t* cnt;
    uint32_t* hist;
    int passes;
};
void launch_predict(const Dev& d, const IntegrateArgs& a, cudaStream_t st);
void launch_correct(const Dev& d, const IntegrateArgs& a, cudaStream_t st);
// Verlet: pvr holds (v, rho) one step earlier (sorted like the state),
// pvr_out receives the state's (v, rho) on entry; px.. are unused.  Then
// each member's time, step count and Verlet phase advance.
void launch_verlet(const Dev& d, const IntegrateArgs& a, cudaStream_t st);

void launch_counts_fp64(const Dev& d, const double* x, const double* y, const double* z,
                        const uint32_t* key, const uint32_t* off, uint32_t* out,
                        cudaStream_t st);

// FP64 conservation sums over all instances: out[0..7] = mass, px, py, pz,
// kinetic, potential, internal, n_out (as double).
constexpr int kDiagBlocks = 152;
void launch_diag(const Dev& d, const double* x, const double* y, const double* z,
                 const float4* vr, const uint32_t* id, const uint32_t* off,
                 double* partial, double* out, cudaStream_t st);
// Device-side step loop: arm the counter (ctr[0] = 0, ctr[1] = nsteps); after
// each body of `body` steps, count it and set the WHILE condition to "another
// body fits and some member is still running".
void launch_loop_init(uint32_t* ctr, uint32_t nsteps, cudaStream_t st);
void launch_loop_ctrl(cudaGraphConditionalHandle h, uint32_t* ctr, const uint32_t* done,
                      uint32_t n_inst, uint32_t body, cudaStream_t st);
void launch_front(const Dev& d, const double* x, const double* z, const uint32_t* id,
                  const uint32_t* off, double zlo, double zhi, unsigned long long* out,
                  cudaStream_t st);

}  // namespace sph
