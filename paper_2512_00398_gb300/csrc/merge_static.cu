// merge_static.cu -- candidate merging without any device allocation.
//
// Some callers cannot allocate device memory at the time they merge: a
// real-time pipeline that forbids allocation once it has started (cudaMalloc
// can block for milliseconds and can fail when the device is full), or code
// embedded in a host framework that owns every byte of device memory.  For
// them hp_merge_static runs the same merge kernels as hp_merge, but all of
// their scratch lives in one file-scope device array of fixed size, reserved
// when the library is loaded and held on every GPU that loads it until the
// process exits.  The caller still provides the raw candidates, their count,
// the per-trial sigmas, the output buffer and, to learn of a raw count beyond
// the buffer it passed, an optional device status word.
#include <mutex>

#include "../../include/hp.h"
#include "common.cuh"

namespace hp {
namespace {

constexpr int64_t kStaticMaxRaw = HP_MERGE_STATIC_MAX_RAW;
constexpr int64_t kStaticPad = (kStaticMaxRaw + kSortChunk - 1) / kSortChunk * kSortChunk;
constexpr int64_t kStaticBlocks = kStaticPad / 1024 + 2;

// Byte offsets of every scratch array inside the static buffer (256-aligned).
constexpr size_t al(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kOffKeys0 = 0;
constexpr size_t kOffKeys1 = al(kOffKeys0 + kStaticPad * 8);
constexpr size_t kOffVals0 = al(kOffKeys1 + kStaticPad * 8);
constexpr size_t kOffVals1 = al(kOffVals0 + kStaticPad * 8);
constexpr size_t kOffParent = al(kOffVals1 + kStaticPad * 8);
constexpr size_t kOffBest = al(kOffParent + kStaticPad * 4);
constexpr size_t kOffRep = al(kOffBest + kStaticPad * 8);
constexpr size_t kOffMembers = al(kOffRep + kStaticPad * 4);
constexpr size_t kOffDmLo = al(kOffMembers + kStaticPad * 4);
constexpr size_t kOffDmHi = al(kOffDmLo + kStaticPad * 4);
constexpr size_t kOffTLo = al(kOffDmHi + kStaticPad * 4);
constexpr size_t kOffTHi = al(kOffTLo + kStaticPad * 8);
constexpr size_t kOffScan = al(kOffTHi + kStaticPad * 8);
constexpr size_t kOffBlockSums = al(kOffScan + kStaticPad * 4);
constexpr size_t kOffNClamped = al(kOffBlockSums + kStaticBlocks * 4);
constexpr size_t kOffWidths = al(kOffNClamped + 8);
constexpr size_t kStaticBytes = al(kOffWidths + kMaxWidths * 4);

// The scratch itself.  In host code this name is only a stand-in for the
// symbol: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_merge_scratch[kStaticBytes];

struct WidthList {
    int32_t w[kMaxWidths];
};

// Copies the boxcar ladder from the kernel parameters into the scratch, so no
// host-to-device copy (and no staging buffer) is needed.
__global__ void put_widths_kernel(WidthList wl, int nw, int32_t* dst) {
    if (threadIdx.x < (unsigned)nw) dst[threadIdx.x] = wl.w[threadIdx.x];
}

// Device address of g_merge_scratch per device, resolved once per device (the
// first call on it) and kept for the life of the process; a device reset
// (cudaDeviceReset) reloads the module and would leave this address stale.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};

int scratch_address(unsigned char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HP_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return HP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_merge_scratch) != cudaSuccess || !p) return HP_ERR_CUDA;
        g_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_addr[dev];
    return HP_OK;
}

}  // namespace
}  // namespace hp

extern "C" int hp_merge_static(const hp_raw_cand* raw_dev, const int64_t* nraw_dev,
                               int64_t raw_capacity, const double* sigma_dev,
                               const int* boxcar_widths, int nw, int dm_tol, int64_t t_gap,
                               int w_tol, void* stream, hp_cand_buf* cand_out,
                               int32_t* status_dev) {
    using namespace hp;
    if (!raw_dev || !nraw_dev || !sigma_dev || !boxcar_widths || !cand_out || !cand_out->data ||
        !cand_out->count || cand_out->capacity < 0)
        return HP_ERR_INVALID_ARG;
    if (raw_capacity < 0 || raw_capacity > kStaticMaxRaw) return HP_ERR_INVALID_ARG;
    // the same bounds as the plan's merge parameters (HP_PARAM_DM_TOL, T_GAP, W_TOL)
    if (nw < 1 || nw > kMaxWidths || dm_tol < 0 || dm_tol > kMaxDMs || w_tol < 0 ||
        w_tol > kMaxWidths || t_gap > kMaxMergeGap || t_gap < -kMaxMergeGap)
        return HP_ERR_INVALID_ARG;
    WidthList wl = {};
    int32_t wmax = 0;
    for (int k = 0; k < nw; ++k) {
        if (boxcar_widths[k] < 1 || boxcar_widths[k] > kMaxWidth) return HP_ERR_INVALID_ARG;
        if (k > 0 && boxcar_widths[k] <= boxcar_widths[k - 1]) return HP_ERR_INVALID_ARG;
        wl.w[k] = boxcar_widths[k];
        wmax = boxcar_widths[k];
    }
    unsigned char* base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    int32_t* widths = reinterpret_cast<int32_t*>(base + kOffWidths);
    put_widths_kernel<<<1, kMaxWidths, 0, s>>>(wl, nw, widths);
    if (cudaGetLastError() != cudaSuccess) return HP_ERR_CUDA;

    // Every scratch word the merge kernels read is written earlier in the same
    // call (keys, union-find state, cluster statistics, scan sums), so nothing
    // left by a previous call needs clearing.
    MergeArgs m;
    m.raw = raw_dev;
    m.nraw = nraw_dev;
    m.cap = raw_capacity;
    m.sigma = sigma_dev;
    m.widths = widths;
    m.nw = nw;
    m.wmax = wmax;
    m.dm_tol = dm_tol;
    m.t_gap = t_gap;
    m.w_tol = w_tol;
    m.keys[0] = reinterpret_cast<uint64_t*>(base + kOffKeys0);
    m.keys[1] = reinterpret_cast<uint64_t*>(base + kOffKeys1);
    m.vals[0] = reinterpret_cast<int64_t*>(base + kOffVals0);
    m.vals[1] = reinterpret_cast<int64_t*>(base + kOffVals1);
    m.parent = reinterpret_cast<int32_t*>(base + kOffParent);
    m.best_bits = reinterpret_cast<uint64_t*>(base + kOffBest);
    m.rep = reinterpret_cast<int32_t*>(base + kOffRep);
    m.members = reinterpret_cast<int32_t*>(base + kOffMembers);
    m.dm_lo = reinterpret_cast<int32_t*>(base + kOffDmLo);
    m.dm_hi = reinterpret_cast<int32_t*>(base + kOffDmHi);
    m.t_lo = reinterpret_cast<unsigned long long*>(base + kOffTLo);
    m.t_hi = reinterpret_cast<unsigned long long*>(base + kOffTHi);
    m.scan = reinterpret_cast<int32_t*>(base + kOffScan);
    m.block_sums = reinterpret_cast<int32_t*>(base + kOffBlockSums);
    m.n_clamped = reinterpret_cast<int64_t*>(base + kOffNClamped);
    m.trial_start = nullptr;   // friends found by search over the whole sorted list
    m.ndm = 0;
    m.out = cand_out->data;
    m.out_cap = cand_out->capacity;
    m.out_count = cand_out->count;
    // a raw count beyond raw_capacity merges the first raw_capacity entries and
    // latches HP_ERR_CAND_OVERFLOW here (when the caller gave a status word)
    m.status = status_dev;
    int64_t launches = 0;
    return launch_merge(m, s, &launches) == cudaSuccess ? HP_OK : HP_ERR_CUDA;
}
