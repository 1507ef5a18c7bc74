// Radix sort of (cell label, index) pairs and the scan that turns per-cell
// counts into first-index-per-cell offsets (Sec. 3.1 of the paper: label,
// radix sort, reorder, first index of each cell).
//
// The sort is a least-significant-digit radix sort with 8-bit digits in the
// single-pass "onesweep" organisation: one histogram of all digit places up
// front (fused into the label kernel on the SPH path), then one kernel per
// digit place in which each 4096-key tile ranks its keys in shared memory,
// publishes its per-digit counts, and finds its global offsets by a bounded
// decoupled look-back over the tiles before it.  Equal digits keep their
// input order, so the sort is stable.
#include "sph_internal.cuh"

namespace sph {

namespace {

constexpr uint32_t kFull = 0xffffffffu;
constexpr uint32_t kFlagAgg = 1u << 30;     // tile's own count published
constexpr uint32_t kFlagPre = 2u << 30;     // inclusive prefix published
constexpr uint32_t kValMask = (1u << 30) - 1;
constexpr uint32_t kSpinLimit = 1u << 24;   // polls before giving up

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Exclusive scan of one value per thread over a 256-thread block.
__device__ __forceinline__ uint32_t block_excl_scan_256(uint32_t v, uint32_t* s_w) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t t = lane < 8 ? s_w[lane] : 0u;
        uint32_t inc = t;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            uint32_t y = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane < 8) s_w[lane] = inc - t;
    }
    __syncthreads();
    uint32_t r = x - v + s_w[w];
    __syncthreads();
    return r;
}

__host__ __device__ __forceinline__ uint32_t digit_mask(int pass, int bits_total) {
    int b = bits_total - 8 * pass;
    b = b > 8 ? 8 : (b < 0 ? 0 : b);
    return (1u << b) - 1u;
}

__global__ void __launch_bounds__(256) k_digit_hist(const uint32_t* __restrict__ keys,
                                                    uint32_t n, int passes, int bits_total,
                                                    uint32_t* __restrict__ hist) {
    __shared__ uint32_t sh[4 * 256];
    for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += gridDim.x * blockDim.x) {
        const uint32_t k = keys[i];
        for (int p = 0; p < passes; ++p)
            atomicAdd(&sh[p * 256 + ((k >> (8 * p)) & digit_mask(p, bits_total))], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// Decoupled look-back for one digit: the sum of the counts of the tiles
// before `tile` (status words of 256 digits per tile; a tile's word holds its
// own count, kFlagAgg, or the inclusive prefix, kFlagPre, or 0 while it has
// published nothing).  The predecessors are polled kLookWin at a time (the
// loads of one window are in flight together), and the walk takes their
// counts in order until an inclusive prefix ends it or a silent tile stops
// it, where the next window starts.  A predecessor that stays silent for
// `limit` windows makes the wait give up: the timeout bit is set in *err and
// the partial sum returned, which never exceeds the true prefix (so scatter
// addresses stay inside the output).  Tile 0 always publishes an inclusive
// prefix, so no window reads before it.
constexpr int kLookWin = 8;

__device__ __forceinline__ uint32_t lookback_prefix(const uint32_t* status, uint32_t tile,
                                                    int digit, uint32_t limit, uint32_t* err) {
    uint32_t excl = 0;
    int64_t p = (int64_t)tile - 1;
    uint32_t spins = 0;
    while (p >= 0) {
        uint32_t s[kLookWin];
#pragma unroll
        for (int j = 0; j < kLookWin; ++j)
            s[j] = p - j >= 0 ? ld_relaxed(status + (size_t)(p - j) * 256 + digit) : kFlagPre;
        bool stop = false, fin = false;
        int taken = 0;
#pragma unroll
        for (int j = 0; j < kLookWin; ++j) {
            if (!stop) {
                const uint32_t flag = s[j] & ~kValMask;
                if (flag == 0u) {
                    stop = true;
                } else {
                    excl += s[j] & kValMask;
                    ++taken;
                    if (flag == kFlagPre) stop = fin = true;
                }
            }
        }
        if (fin) break;
        p -= taken;
        if (taken == 0 && ++spins > limit) {
            atomicOr(err, kStatusTimeout);
            break;
        }
    }
    return excl;
}

// One digit place.  hist holds the global count of each digit value for
// this place; status holds one word per (tile, digit), zero on entry;
// tilectr is a zeroed counter that hands out tiles in launch order, so every
// tile a block waits on belongs to a block that is already running.
__global__ void __launch_bounds__(kOsThreads) k_onesweep(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
    uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, uint32_t n, int shift,
    uint32_t dmask, const uint32_t* __restrict__ hist, uint32_t* status,
    uint32_t* tilectr, uint32_t* err) {
    constexpr int W = kOsThreads / 32;
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_wh[W][256];       // per-warp digit counts, then offsets
    __shared__ uint32_t s_dstart[256];      // tile-local first slot per digit
    __shared__ uint32_t s_gbase[256];       // global first slot of the tile's digit run
    __shared__ uint32_t s_w[8];
    __shared__ uint32_t s_keys[kOsTile];
    __shared__ uint32_t s_vals[kOsTile];

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(tilectr, 1u);
    for (int i = tid; i < W * 256; i += kOsThreads) (&s_wh[0][0])[i] = 0;
    const uint32_t gofs = block_excl_scan_256(hist[tid], s_w);   // also syncs
    const uint32_t tile = s_tile;
    const uint32_t base = tile * kOsTile + w * (kOsItems * 32);

    uint32_t k[kOsItems], v[kOsItems], rk[kOsItems];
#pragma unroll
    for (int r = 0; r < kOsItems; ++r) {
        const uint32_t idx = base + r * 32 + lane;
        const bool ok = idx < n;
        k[r] = ok ? kin[idx] : 0u;
        v[r] = ok ? (vin ? vin[idx] : idx) : 0u;
        rk[r] = ok ? 0u : 0xffffffffu;
    }
    // Warp-level stable ranking: items r = 0..15 in order, lanes in order.
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int r = 0; r < kOsItems; ++r) {
        const bool ok = rk[r] == 0u;
        const uint32_t d = ok ? ((k[r] >> shift) & dmask) : 256u + lane;
        const uint32_t peers = __match_any_sync(kFull, d);
        uint32_t prev = 0;
        if (ok) prev = s_wh[w][d];
        __syncwarp();
        if (ok) {
            rk[r] = prev + __popc(peers & lt);
            if (lane == __ffs(peers) - 1) s_wh[w][d] = prev + __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
    // Thread tid owns digit tid: per-warp exclusive offsets and tile count.
    uint32_t run = 0;
#pragma unroll
    for (int ww = 0; ww < W; ++ww) {
        const uint32_t c = s_wh[ww][tid];
        s_wh[ww][tid] = run;
        run += c;
    }
    const uint32_t cnt = run;
    uint32_t* my = status + (size_t)tile * 256 + tid;
    st_relaxed(my, (tile == 0 ? kFlagPre : kFlagAgg) | cnt);
    const uint32_t dstart = block_excl_scan_256(cnt, s_w);
    s_dstart[tid] = dstart;
    // Decoupled look-back for digit tid.
    uint32_t excl = 0;
    if (tile > 0) {
        excl = lookback_prefix(status, tile, tid, kSpinLimit, err);
        st_relaxed(my, kFlagPre | (excl + cnt));
    }
    s_gbase[tid] = gofs + excl;
    __syncthreads();
    // Scatter into tile-sorted order in shared memory.
#pragma unroll
    for (int r = 0; r < kOsItems; ++r) {
        if (rk[r] != 0xffffffffu) {
            const uint32_t d = (k[r] >> shift) & dmask;
            const uint32_t pos = s_dstart[d] + s_wh[w][d] + rk[r];
            s_keys[pos] = k[r];
            s_vals[pos] = v[r];
        }
    }
    __syncthreads();
    const uint32_t t0 = tile * kOsTile;
    const uint32_t nv = (n - t0) < (uint32_t)kOsTile ? (n - t0) : (uint32_t)kOsTile;
    for (uint32_t i = tid; i < nv; i += kOsThreads) {
        const uint32_t key = s_keys[i];
        const uint32_t d = (key >> shift) & dmask;
        const uint32_t g = s_gbase[d] + (i - s_dstart[d]);
        kout[g] = key;
        vout[g] = s_vals[i];
    }
}

// Self-test of the failure path: one block of 256 threads runs the look-back
// of tile 1 against a tile 0 whose status words stay zero (nothing
// publishes them), so every digit's wait gives up after `limit` polls.
__global__ void __launch_bounds__(256) k_lookback_selftest(const uint32_t* status, uint32_t limit,
                                                           uint32_t* err) {
    lookback_prefix(status, 1u, (int)threadIdx.x, limit, err);
}

// --- exclusive scan of the per-cell counts into cell offsets --------------

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanChunk = kScanThreads * kScanItems;

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ in,
                                                              uint64_t m,
                                                              uint32_t* __restrict__ bsum) {
    pdl_wait();
    __shared__ uint32_t s_w[8];
    const uint64_t b0 = (uint64_t)blockIdx.x * kScanChunk;
    uint32_t s = 0;
    for (int r = 0; r < kScanItems; ++r) {
        const uint64_t i = b0 + (uint64_t)r * kScanThreads + threadIdx.x;
        if (i < m) s += in[i];
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int i = 0; i < 8; ++i) t += s_w[i];
        bsum[blockIdx.x] = t;
    }
}

// Exclusive scan of the block sums in place (one block).
__global__ void __launch_bounds__(256) k_scan_top(uint32_t* bsum, uint32_t nb) {
    pdl_wait();
    __shared__ uint32_t s_w[8];
    __shared__ uint32_t s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (uint32_t c0 = 0; c0 < nb; c0 += 256) {
        const uint32_t i = c0 + threadIdx.x;
        const uint32_t v = i < nb ? bsum[i] : 0u;
        const uint32_t ex = block_excl_scan_256(v, s_w);
        const uint32_t carry = s_carry;
        if (i < nb) bsum[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 255) s_carry = carry + ex + v;
        __syncthreads();
    }
}

// out[i] = sum of in[0..i), i = 0..m (m + 1 outputs); clears in[] for the
// next use.
__global__ void __launch_bounds__(kScanThreads) k_scan_down(uint32_t* __restrict__ in, uint64_t m,
                                                            const uint32_t* __restrict__ bsum,
                                                            uint32_t* __restrict__ out,
                                                            int zero_in) {
    pdl_wait();
    __shared__ uint32_t s_w[8];
    const uint64_t b0 = (uint64_t)blockIdx.x * kScanChunk;
    const uint64_t t0 = b0 + (uint64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t tot = 0;
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
        const uint64_t i = t0 + r;
        v[r] = i < m ? in[i] : 0u;
        tot += v[r];
    }
    const uint32_t ex = block_excl_scan_256(tot, s_w) + (bsum ? bsum[blockIdx.x] : 0u);
    uint32_t run = ex;
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
        const uint64_t i = t0 + r;
        if (i < m) {
            out[i] = run;
            if (zero_in) in[i] = 0u;
        }
        if (i == m) out[m] = run;
        run += v[r];
    }
}

// The same scan in one launch: tiles of kScanChunk entries taken in launch
// order from a ticket (ctl[0]), each publishing its total, finding the sum
// of the tiles before it by a decoupled look-back (tile_lookback, epoch in
// ctl[1]) and publishing its inclusive prefix.  The block of the last tile
// rearms the ticket and the epoch: its look-back ended on a prefix, so every
// tile has taken its ticket and read the epoch by then.
constexpr uint32_t kScanSpinLimit = 1u << 20;   // polls of a tile's look-back

__global__ void __launch_bounds__(kScanThreads) k_scan_onepass(uint32_t* __restrict__ in,
                                                               uint64_t m,
                                                               uint32_t* __restrict__ out,
                                                               int zero_in,
                                                               unsigned long long* words,
                                                               uint32_t* ctl, uint32_t* err) {
    pdl_wait();
    __shared__ uint32_t s_w[8];
    __shared__ uint32_t s_tile, s_ep, s_tot, s_excl;
    if (threadIdx.x == 0) {
        s_tile = atomicAdd(ctl, 1u);
        s_ep = *reinterpret_cast<volatile uint32_t*>(ctl + 1) & 0x3fffffffu;
    }
    __syncthreads();
    const uint32_t tile = s_tile, ep = s_ep;
    const uint64_t t0 = (uint64_t)tile * kScanChunk + (uint64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t tot = 0;
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
        const uint64_t i = t0 + r;
        v[r] = i < m ? in[i] : 0u;
        tot += v[r];
    }
    const uint32_t ex = block_excl_scan_256(tot, s_w);
    if (threadIdx.x == kScanThreads - 1) s_tot = ex + tot;
    __syncthreads();
    if (threadIdx.x < 32) {
        const uint32_t btot = s_tot;
        const unsigned long long tag = (unsigned long long)ep << 34;
        uint32_t excl = 0;
        if (tile > 0) {
            if (threadIdx.x == 0) st_relaxed64(words + tile, tag | (1ull << 32) | btot);
            excl = tile_lookback(words, tile, ep, kScanSpinLimit, err);
        }
        if (threadIdx.x == 0) {
            st_relaxed64(words + tile, tag | (2ull << 32) | (excl + btot));
            s_excl = excl;
            if ((uint64_t)tile == m / kScanChunk) {   // the tile that holds index m
                ctl[0] = 0u;
                ctl[1] = ep + 1u;
            }
        }
    }
    __syncthreads();
    uint32_t run = s_excl + ex;
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
        const uint64_t i = t0 + r;
        if (i < m) {
            out[i] = run;
            if (zero_in) in[i] = 0u;
        }
        if (i == m) out[m] = run;
        run += v[r];
    }
}

}  // namespace

void launch_scan_onepass(uint32_t* in, uint64_t m, uint32_t* out, bool zero_in,
                         unsigned long long* words, uint32_t* ctl, uint32_t* err,
                         cudaStream_t st) {
    launch_pdl(k_scan_onepass, scan_bsum_count(m), kScanThreads, 0, st, in, m, out,
               zero_in ? 1 : 0, words, ctl, err);
}

uint32_t scan_bsum_count(uint64_t m) {
    // m + 1 outputs: the block that holds index m writes the total
    return (uint32_t)((m + 1 + kScanChunk - 1) / kScanChunk);
}

void launch_scan(uint32_t* in, uint64_t m, uint32_t* bsum, uint32_t* out, cudaStream_t st,
                 bool zero_in) {
    const uint32_t nb = scan_bsum_count(m);
    if (nb == 1) {
        // one block holds the whole array: no block sums needed
        launch_pdl(k_scan_down, 1, kScanThreads, 0, st, in, m, nullptr, out, zero_in ? 1 : 0);
        return;
    }
    launch_pdl(k_scan_reduce, nb, kScanThreads, 0, st, in, m, bsum);
    launch_pdl(k_scan_top, 1, 256, 0, st, bsum, nb);
    launch_pdl(k_scan_down, nb, kScanThreads, 0, st, in, m, bsum, out, zero_in ? 1 : 0);
}

// The per-cell counts (incl. the excluded bin) stay in cnt: the scatter of
// the cell sort counts them back down to zero.
void launch_scan_cells(const Dev& d, uint32_t* cnt, uint32_t* off, unsigned long long* words,
                       uint32_t* ctl, uint32_t* err, cudaStream_t st) {
    launch_scan_onepass(cnt, (uint64_t)d.ncells + 1, off, false, words, ctl, err, st);
}

// Sec. 3.1 cell sort as one counting-sort pass (a radix sort whose single
// digit is the whole cell label): the label kernel's per-cell counts are the
// histogram, the cell offsets its exclusive scan, and each particle takes a
// slot of its cell's range by a warp-aggregated atomic decrement of its
// cell's count (which leaves the counts at zero for the next rebuild).  The
// order inside a cell is left arbitrary: the reorder ranks every particle by
// id within its cell, which makes the result the (label, id) order.
__global__ void __launch_bounds__(256) k_cell_scatter(const uint32_t* __restrict__ key, uint32_t n,
                                                      const uint32_t* __restrict__ off,
                                                      uint32_t* cnt, uint32_t* __restrict__ kout,
                                                      uint32_t* __restrict__ vout,
                                                      uint32_t* status) {
    pdl_wait();
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < n;
    const uint32_t act = __ballot_sync(kFull, valid);
    if (!valid) return;
    const uint32_t k = key[i];
    const uint32_t peers = __match_any_sync(act, k);
    const int leader = __ffs(peers) - 1;
    const uint32_t np = __popc(peers);
    uint32_t old = 0;
    if ((int)(threadIdx.x & 31) == leader) old = atomicSub(cnt + k, np);
    old = __shfl_sync(peers, old, leader);
    const uint32_t slot = off[k] + old - np + __popc(peers & lanemask_lt());
    if (!in_bounds(slot < n, status)) return;
    kout[slot] = k;
    vout[slot] = i;
}

void launch_cell_scatter(const uint32_t* key, uint32_t n, const uint32_t* off, uint32_t* cnt,
                         uint32_t* kout, uint32_t* vout, uint32_t* status, cudaStream_t st) {
    if (n == 0) return;
    launch_pdl(k_cell_scatter, (n + 255) / 256, 256, 0, st, key, n, off, cnt, kout, vout, status);
}

void launch_lookback_selftest(uint32_t* zeroed256, uint32_t limit, uint32_t* err,
                              cudaStream_t st) {
    cudaMemsetAsync(zeroed256, 0, 256 * sizeof(uint32_t), st);
    k_lookback_selftest<<<1, 256, 0, st>>>(zeroed256, limit, err);
}

void launch_digit_hist(const uint32_t* keys, uint32_t n, int passes, int bits_total,
                       uint32_t* hist, cudaStream_t st) {
    uint32_t blocks = (n + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks == 0) blocks = 1;
    k_digit_hist<<<blocks, 256, 0, st>>>(keys, n, passes, bits_total, hist);
}

void launch_onesweep_pass(const uint32_t* kin, const uint32_t* vin, uint32_t* kout,
                          uint32_t* vout, uint32_t n, int pass, int bits_total,
                          const uint32_t* hist, uint32_t* status, uint32_t* tilectr,
                          uint32_t* err, cudaStream_t st) {
    const uint32_t tiles = os_tiles(n);
    if (tiles == 0) return;
    k_onesweep<<<tiles, kOsThreads, 0, st>>>(kin, vin, kout, vout, n, 8 * pass,
                                             digit_mask(pass, bits_total), hist + 256 * pass,
                                             status + (size_t)pass * tiles * 256,
                                             tilectr + pass, err);
}

}  // namespace sph
