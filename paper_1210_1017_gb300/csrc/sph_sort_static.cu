// sph_radix_sort_pairs_static: the stable radix sort of sph_radix_sort_pairs
// for callers that cannot hand the library any device scratch memory.
//
// Who needs it: code that drives the library through the plain C ABI without
// a device allocator of its own (nothing to cudaMalloc the scratch with), a
// host whose device memory is entirely owned by another allocator's pool, or
// a latency-critical loop that must not call cudaMalloc/cudaFree at run time
// because those calls can synchronise the whole device and stall work on
// other streams.  Such callers still own the input and output arrays; only the
// sort's own scratch (temporary keys/values, digit histograms, tile counters
// and look-back status words) moves into a fixed array that is part of the
// loaded library.
//
// The array below is a host-side stand-in when named from host code; the
// device address is looked up with cudaGetSymbolAddress once per device, on
// the first call made with that device current.  That first call therefore
// makes a CUDA runtime query and should come before any stream capture.  All
// calls on one device share the array: calls that overlap on the GPU (two
// streams, two threads) race on it and must be serialised by the caller.
// Nothing here allocates: the zeroing is done with cudaMemsetAsync on the
// fixed array.
#include <mutex>

#include "../../include/sph.h"
#include "sph_internal.cuh"

namespace {

using namespace sph;

constexpr uint32_t kMaxN = SPH_RADIX_SORT_STATIC_MAX_N;
constexpr uint32_t kMaxTiles = (kMaxN + kOsTile - 1) / kOsTile;
constexpr int kMaxPasses = 4;

// Layout of the fixed scratch, in 32-bit words.
constexpr size_t kTmpKeys = 0;
constexpr size_t kTmpVals = kTmpKeys + kMaxN;
constexpr size_t kHist = kTmpVals + kMaxN;                 // 4 x 256 digit counts
constexpr size_t kTileCtr = kHist + kMaxPasses * 256;      // one per pass
constexpr size_t kStatus = kTileCtr + kMaxPasses;          // passes x tiles x 256
constexpr size_t kErr = kStatus + (size_t)kMaxPasses * kMaxTiles * 256;
constexpr size_t kWords = kErr + 64;

static __device__ __align__(256) uint32_t g_sort_scratch[kWords];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
uint32_t* g_scratch_addr[kMaxDevices] = {};

// Device address of g_sort_scratch on the current device (looked up once).
int scratch_for_current_device(uint32_t** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return SPH_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return SPH_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess || !p) return SPH_ERR_CUDA;
        g_scratch_addr[dev] = static_cast<uint32_t*>(p);
    }
    *out = g_scratch_addr[dev];
    return SPH_OK;
}

}  // namespace

extern "C" int sph_radix_sort_pairs_static(const uint32_t* d_keys_in, const uint32_t* d_vals_in,
                                           uint32_t* d_keys_out, uint32_t* d_vals_out,
                                           uint32_t n, uint32_t key_bits, void* stream) {
    if (!d_keys_in || !d_keys_out || !d_vals_out) return SPH_ERR_INVALID_ARG;
    if (key_bits == 0 || key_bits > 32) return SPH_ERR_INVALID_ARG;
    if (n > kMaxN) return SPH_ERR_TOO_LARGE;
    if (n == 0) return SPH_OK;
    uint32_t* s = nullptr;
    const int rc = scratch_for_current_device(&s);
    if (rc != SPH_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int passes = ((int)key_bits + 7) / 8;
    const uint32_t tiles = os_tiles(n);
    // the previous call's contents are still there: clear what counts
    cudaMemsetAsync(s + kHist, 0, (kMaxPasses * 256 + kMaxPasses) * sizeof(uint32_t), st);
    cudaMemsetAsync(s + kStatus, 0, (size_t)passes * tiles * 256 * sizeof(uint32_t), st);
    cudaMemsetAsync(s + kErr, 0, sizeof(uint32_t), st);
    launch_digit_hist(d_keys_in, n, passes, (int)key_bits, s + kHist, st);
    const uint32_t* ck = d_keys_in;
    const uint32_t* cv = d_vals_in;
    for (int p = 0; p < passes; ++p) {
        const bool to_out = ((passes - 1 - p) % 2) == 0;
        uint32_t* ok = to_out ? d_keys_out : s + kTmpKeys;
        uint32_t* ov = to_out ? d_vals_out : s + kTmpVals;
        launch_onesweep_pass(ck, cv, ok, ov, n, p, (int)key_bits, s + kHist, s + kStatus,
                             s + kTileCtr, s + kErr, st);
        ck = ok;
        cv = ov;
    }
    return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}

extern "C" int sph_radix_sort_static_status(void* stream) {
    uint32_t* s = nullptr;
    const int rc = scratch_for_current_device(&s);
    if (rc != SPH_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t word = 0;
    if (cudaMemcpyAsync(&word, s + kErr, sizeof(word), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return SPH_ERR_CUDA;
    return (word & kStatusTimeout) ? SPH_ERR_TIMEOUT : SPH_OK;
}

extern "C" int sph_radix_sort_static_selftest_timeout(uint32_t polls, void* stream) {
    if (polls == 0 || polls > (1u << 20)) return SPH_ERR_INVALID_ARG;
    uint32_t* s = nullptr;
    const int rc = scratch_for_current_device(&s);
    if (rc != SPH_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaMemsetAsync(s + kErr, 0, sizeof(uint32_t), st);
    // tile 1 of the first pass waits on tile 0's status words (zeroed by the
    // self-test launch), which nothing publishes
    launch_lookback_selftest(s + kStatus, polls, s + kErr, st);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
        return SPH_ERR_CUDA;
    return SPH_OK;
}
