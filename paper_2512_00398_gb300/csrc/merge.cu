// merge.cu -- candidate merging and clustering on sm_103a (Section II-B,
// "Candidate Merging and Clustering"; Algorithm 1, last stage).
//
// Friends-of-friends over (trial, time window, width): two raw candidates are
// friends iff |d_i - d_j| <= dm_tol, |k_i - k_j| <= w_tol and their boxcar
// windows [t, t + W) lie within t_gap samples:
//   max(t_i, t_j) - min(t_i + W_i, t_j + W_j) <= t_gap.
// Clusters are connected components, so the result does not depend on the
// (atomic, unordered) order in which the detection kernel appended them.
//
//   1. keys (dm << 43 | sample << 5 | width) and exact sums S, padded with
//      UINT64_MAX; bitonic sort of 2048-key chunks in shared memory, then
//      merge passes that place every key by a binary search in the partner
//      run (keys are unique, so ranks are exact).
//   2. each candidate scans the sorted keys of trials d .. d + dm_tol whose
//      windows can touch its own and links friends with a lock-free
//      union-find that always hangs the larger root under the smaller one, so
//      every root is the smallest index (= smallest key) of its cluster.
//   3. per cluster: member count, trial and time ranges, and the member with
//      the largest S/N = S / (sigma * sqrt(W)), computed in FP64 with
//      correctly rounded operations (ties: smallest key).
//   4. roots are compacted in index order with a device-wide scan.
#include <algorithm>
#include <atomic>
#include <climits>

#include "common.cuh"

namespace hp {
namespace {

constexpr int kSortThreads = 1024;   // 2 keys per thread
constexpr uint64_t kPad = ~0ull;

__device__ __forceinline__ int key_dm(uint64_t k) { return (int)(k >> kKeyDmShift); }
__device__ __forceinline__ int64_t key_sample(uint64_t k) {
    return (int64_t)((k >> kKeySampleShift) & ((1ull << (kKeyDmShift - kKeySampleShift)) - 1));
}
__device__ __forceinline__ int key_width(uint64_t k) {
    return (int)(k & ((1u << kKeySampleShift) - 1));
}

// The element-wise kernels walk the list with a grid stride: their grids are
// sized for the capacity only up to one resident wave, so a short list does not
// pay for tens of thousands of empty blocks (the link kernel keeps one thread
// per candidate).
#define FOR_EACH(i, n) \
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); \
         i += (int64_t)gridDim.x * blockDim.x)

__global__ void init_keys_kernel(MergeArgs a) {
    const int64_t nr = *a.nraw;
    const int64_t n = nr < a.cap ? nr : a.cap;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *a.n_clamped = n;
        if (nr > a.cap) latch_status(a.status, HP_ERR_CAND_OVERFLOW);
    }
    const int64_t padded = (n + kSortChunk - 1) / kSortChunk * kSortChunk;
    FOR_EACH(i, padded) {
        if (i < n) {
            const hp_raw_cand c = a.raw[i];
            a.keys[0][i] = ((uint64_t)c.dm_idx << kKeyDmShift) |
                           ((uint64_t)c.sample << kKeySampleShift) | (uint64_t)c.width_idx;
            a.vals[0][i] = c.S;
        } else {
            a.keys[0][i] = kPad;
            a.vals[0][i] = 0;
        }
    }
}

__global__ void __launch_bounds__(kSortThreads) chunk_sort_kernel(uint64_t* __restrict__ keys,
                                                                  int64_t* __restrict__ vals,
                                                                  const int64_t* __restrict__ n_ptr) {
    __shared__ uint64_t sk[kSortChunk];
    __shared__ int64_t sv[kSortChunk];
    const int64_t n = *n_ptr;
    // chunks blockIdx.x, blockIdx.x + gridDim.x, ... below n (block-uniform)
    for (int64_t base = (int64_t)blockIdx.x * kSortChunk; base < n;
         base += (int64_t)gridDim.x * kSortChunk) {
        for (int i = threadIdx.x; i < kSortChunk; i += blockDim.x) {
            sk[i] = keys[base + i];
            sv[i] = vals[base + i];
        }
        __syncthreads();
        for (int size = 2; size <= kSortChunk; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int i = threadIdx.x; i < kSortChunk; i += blockDim.x) {
                    const int j = i ^ stride;
                    if (j > i) {
                        const bool up = (i & size) == 0;
                        const uint64_t ki = sk[i], kj = sk[j];
                        if ((ki > kj) == up) {
                            sk[i] = kj;
                            sk[j] = ki;
                            const int64_t t = sv[i];
                            sv[i] = sv[j];
                            sv[j] = t;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (int i = threadIdx.x; i < kSortChunk; i += blockDim.x) {
            keys[base + i] = sk[i];
            vals[base + i] = sv[i];
        }
        __syncthreads();   // sk, sv are refilled with the next chunk
    }
}

__global__ void merge_pass_kernel(const uint64_t* __restrict__ ks, const int64_t* __restrict__ vs,
                                  uint64_t* __restrict__ kd, int64_t* __restrict__ vd,
                                  const int64_t* __restrict__ n_ptr, int64_t run) {
    const int64_t n = *n_ptr;
    FOR_EACH(i, n) {
        const int64_t r = i / run;
        const int64_t ps = (r ^ 1) * run;
        const uint64_t key = ks[i];
        if (ps >= n) {
            kd[i] = key;
            vd[i] = vs[i];
            continue;
        }
        int64_t lo = ps, hi = min(ps + run, n);   // count partner keys < key
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (ks[mid] < key) lo = mid + 1; else hi = mid;
        }
        const int64_t dst = min(r, r ^ 1) * run + (i - r * run) + (lo - ps);
        kd[dst] = key;
        vd[dst] = vs[i];
    }
}

__global__ void uf_init_kernel(MergeArgs a) {
    FOR_EACH(i, *a.n_clamped) {
        a.parent[i] = (int32_t)i;
        a.best_bits[i] = 0;
        a.rep[i] = INT_MAX;
        a.members[i] = 0;
        a.dm_lo[i] = INT_MAX;
        a.dm_hi[i] = INT_MIN;
        a.t_lo[i] = ~0ull;
        a.t_hi[i] = 0;
    }
}

__device__ __forceinline__ int32_t uf_find(int32_t* parent, int32_t x) {
    int32_t p = parent[x];
    while (p != x) {
        const int32_t g = parent[p];
        if (g != p) atomicCAS(&parent[x], p, g);   // path halving, keeps parent < child
        x = p;
        p = parent[x];
    }
    return x;
}

__device__ void uf_union(int32_t* parent, int32_t a, int32_t b) {
    while (true) {
        a = uf_find(parent, a);
        b = uf_find(parent, b);
        if (a == b) return;
        if (a > b) { const int32_t t = a; a = b; b = t; }
        if (atomicCAS(&parent[b], b, a) == b) return;   // b was still a root
    }
}

__device__ __forceinline__ int64_t lower_bound_key(const uint64_t* k, int64_t n, uint64_t key) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (k[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// trial_start[d] = the first sorted entry of trial d or later (d = ndm: n)
__global__ void trial_start_kernel(MergeArgs a, const uint64_t* __restrict__ keys) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d > a.ndm) return;
    const int64_t n = *a.n_clamped;
    a.trial_start[d] = d == a.ndm ? n : lower_bound_key(keys, n, (uint64_t)d << kKeyDmShift);
}

__global__ void link_kernel(MergeArgs a, const uint64_t* __restrict__ keys) {
    const int64_t n = *a.n_clamped;
    FOR_EACH(i, n) {
        const uint64_t ki = keys[i];
        const int di = key_dm(ki), wi = key_width(ki);
        const int64_t ti = key_sample(ki);
        const int64_t ei = ti + a.widths[wi];
        const int64_t t_first = ti - (int64_t)a.wmax - a.t_gap;
        const int64_t t_last = ei + a.t_gap;
        for (int dd = di; dd <= di + a.dm_tol; ++dd) {
            // the friends j > i: in i's own trial the entries after i, in a later
            // trial from the first entry at t_first (searched within that trial's
            // entries when the per-trial table is there)
            int64_t j0;
            if (dd == di) {
                j0 = i + 1;
            } else {
                const uint64_t lo_key = ((uint64_t)dd << kKeyDmShift) |
                                        ((uint64_t)(t_first > 0 ? t_first : 0) << kKeySampleShift);
                if (a.trial_start) {
                    if (dd >= a.ndm) break;
                    const int64_t b0 = a.trial_start[dd], b1 = a.trial_start[dd + 1];
                    j0 = b0 + lower_bound_key(keys + b0, b1 - b0, lo_key);
                } else {
                    j0 = lower_bound_key(keys, n, lo_key);
                }
            }
            for (int64_t j = j0; j < n; ++j) {
                const uint64_t kj = keys[j];
                if (key_dm(kj) != dd) break;
                const int64_t tj = key_sample(kj);
                if (tj > t_last) break;
                const int wj = key_width(kj);
                if (abs(wi - wj) > a.w_tol) continue;
                const int64_t ej = tj + a.widths[wj];
                const int64_t gap = max(ti, tj) - min(ei, ej);
                if (gap <= a.t_gap) uf_union(a.parent, (int32_t)i, (int32_t)j);
            }
        }
    }
}

__global__ void compress_kernel(MergeArgs a) {
    FOR_EACH(i, *a.n_clamped) a.parent[i] = uf_find(a.parent, (int32_t)i);
}

__device__ __forceinline__ double cand_snr(const MergeArgs& a, uint64_t key, int64_t S) {
    if (a.sigw) return __ddiv_rn((double)S, a.sigw[(int64_t)key_dm(key) * a.nw + key_width(key)]);
    const double sg = a.sigma[key_dm(key)];
    const double sw = __dsqrt_rn((double)a.widths[key_width(key)]);
    return __ddiv_rn((double)S, __dmul_rn(sg, sw));
}

__global__ void stats_kernel(MergeArgs a, const uint64_t* __restrict__ keys,
                             const int64_t* __restrict__ vals) {
    FOR_EACH(i, *a.n_clamped) {
        const int32_t r = a.parent[i];
        const uint64_t k = keys[i];
        const double snr = cand_snr(a, k, vals[i]);
        atomicMax(reinterpret_cast<unsigned long long*>(&a.best_bits[r]),
                  (unsigned long long)__double_as_longlong(snr));
        atomicAdd(&a.members[r], 1);
        atomicMin(&a.dm_lo[r], key_dm(k));
        atomicMax(&a.dm_hi[r], key_dm(k));
        const unsigned long long t = (unsigned long long)key_sample(k);
        atomicMin(&a.t_lo[r], t);
        atomicMax(&a.t_hi[r], t + (unsigned long long)a.widths[key_width(k)]);
    }
}

__global__ void rep_kernel(MergeArgs a, const uint64_t* __restrict__ keys,
                           const int64_t* __restrict__ vals) {
    FOR_EACH(i, *a.n_clamped) {
        const int32_t r = a.parent[i];
        const double snr = cand_snr(a, keys[i], vals[i]);
        if ((unsigned long long)__double_as_longlong(snr) == (unsigned long long)a.best_bits[r])
            atomicMin(&a.rep[r], (int32_t)i);
    }
}

// roots -> per-block counts; single-block scan of the counts; scatter.  A
// logical block is kScanBlock consecutive entries; only the ceil(n / kScanBlock)
// logical blocks below n are counted, scanned and scattered, each CTA taking
// logical blocks blockIdx.x, blockIdx.x + gridDim.x, ...
constexpr int kScanBlock = 1024;

__global__ void __launch_bounds__(kScanBlock) root_count_kernel(MergeArgs a) {
    __shared__ int32_t cnt;
    const int64_t n = *a.n_clamped;
    for (int64_t lb = blockIdx.x; lb * kScanBlock < n; lb += gridDim.x) {
        if (threadIdx.x == 0) cnt = 0;
        __syncthreads();
        const int64_t i = lb * kScanBlock + threadIdx.x;
        const bool root = i < n && a.parent[i] == (int32_t)i;
        const unsigned b = __ballot_sync(0xffffffffu, root);
        if ((threadIdx.x & 31) == 0 && b) atomicAdd(&cnt, __popc(b));
        __syncthreads();
        if (threadIdx.x == 0) a.block_sums[lb] = cnt;
        __syncthreads();   // cnt is cleared for the next logical block
    }
}

__global__ void __launch_bounds__(1024) block_scan_kernel(MergeArgs a) {
    __shared__ int32_t warp_tot[32];
    __shared__ int32_t carry;
    const int64_t nblocks = (*a.n_clamped + kScanBlock - 1) / kScanBlock;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < nblocks; b0 += 1024) {
        const int64_t i = b0 + threadIdx.x;
        const int32_t v = i < nblocks ? a.block_sums[i] : 0;
        int32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t u = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += u;
        }
        if (lane == 31) warp_tot[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int32_t w = warp_tot[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t u = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += u;
            }
            warp_tot[lane] = w;
        }
        __syncthreads();
        const int32_t c = carry;
        const int32_t incl = x + c + (warp > 0 ? warp_tot[warp - 1] : 0);
        if (i < nblocks) a.block_sums[i] = incl - v;   // exclusive
        __syncthreads();
        if (threadIdx.x == 1023) carry = incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) *a.out_count = carry;
}

__global__ void __launch_bounds__(kScanBlock) scatter_kernel(MergeArgs a,
                                                             const uint64_t* __restrict__ keys,
                                                             const int64_t* __restrict__ vals) {
    __shared__ int32_t warp_cnt[32];
    const int64_t n = *a.n_clamped;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t lb = blockIdx.x; lb * kScanBlock < n; lb += gridDim.x) {
        const int64_t i = lb * kScanBlock + threadIdx.x;
        const bool root = i < n && a.parent[i] == (int32_t)i;
        const unsigned b = __ballot_sync(0xffffffffu, root);
        if (lane == 0) warp_cnt[warp] = __popc(b);
        __syncthreads();
        int32_t before = 0;
        for (int w = 0; w < warp; ++w) before += warp_cnt[w];
        __syncthreads();   // warp_cnt is rewritten for the next logical block
        if (!root) continue;
        const int64_t slot = (int64_t)a.block_sums[lb] + before + __popc(b & ((1u << lane) - 1));
        if (slot >= a.out_cap) continue;
        const int32_t rp = a.rep[i];
        const uint64_t kr = keys[rp];
        hp_cand c;
        c.dm_idx = key_dm(kr);
        c.width_idx = key_width(kr);
        c.sample = key_sample(kr);
        c.snr = (float)cand_snr(a, kr, vals[rp]);
        c.members = a.members[i];
        c.dm_lo = a.dm_lo[i];
        c.dm_hi = a.dm_hi[i];
        c.t_lo = (int64_t)a.t_lo[i];
        c.t_hi = (int64_t)a.t_hi[i];
        a.out[slot] = c;
    }
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// One resident wave of a strided kernel's blocks on the current device (its
// blocks per SM at full occupancy x the SM count), looked up once per kernel;
// a larger grid would leave a partial second wave with the same fixed share of
// work per thread.
template <class K>
int64_t wave(K kernel, int threads, std::atomic<int>& cache) {
    int v = cache.load(std::memory_order_relaxed);
    if (v == 0) {
        int dev = 0, sms = 0, per = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, 0) != cudaSuccess) {
            (void)cudaGetLastError();
            v = 1024;
        } else {
            v = std::max(1, sms * per);
        }
        cache.store(v, std::memory_order_relaxed);
    }
    return v;
}

std::atomic<int> g_wave[12];

}  // namespace

int merge_sort_passes(int64_t cap) {
    int p = 0;
    for (int64_t run = kSortChunk; run < cap; run <<= 1) ++p;
    return p;
}

cudaError_t launch_merge(const MergeArgs& a_in, cudaStream_t s, int64_t* nlaunch) {
    MergeArgs a = a_in;
    cudaError_t e;
    if (a.cap <= 0) {
        return cudaMemsetAsync(a.out_count, 0, sizeof(int64_t), s);
    }
    const int64_t padded_cap = ceil_div(a.cap, kSortChunk) * kSortChunk;
    // grids of at most one resident wave; the kernels stride over the rest
    const int64_t g256 = ceil_div(padded_cap, 256);
    auto grid = [&](auto kernel, int threads, int64_t blocks, int id) {
        return (unsigned)std::min<int64_t>(blocks, wave(kernel, threads, g_wave[id]));
    };
    ++*nlaunch;
    init_keys_kernel<<<grid(init_keys_kernel, 256, g256, 0), 256, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ++*nlaunch;
    chunk_sort_kernel<<<grid(chunk_sort_kernel, kSortThreads, padded_cap / kSortChunk, 1),
                        kSortThreads, 0, s>>>(a.keys[0], a.vals[0], a.n_clamped);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int cur = 0;
    for (int64_t run = kSortChunk; run < a.cap; run <<= 1) {
        ++*nlaunch;
        merge_pass_kernel<<<grid(merge_pass_kernel, 256, g256, 2), 256, 0, s>>>(
            a.keys[cur], a.vals[cur], a.keys[cur ^ 1],
                                               a.vals[cur ^ 1], a.n_clamped, run);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        cur ^= 1;
    }
    const uint64_t* keys = a.keys[cur];
    const int64_t* vals = a.vals[cur];
    ++*nlaunch;
    uf_init_kernel<<<grid(uf_init_kernel, 256, g256, 3), 256, 0, s>>>(a);
    if (a.trial_start) {
        ++*nlaunch;
        trial_start_kernel<<<(unsigned)ceil_div((int64_t)a.ndm + 1, 256), 256, 0, s>>>(a, keys);
    }
    ++*nlaunch;
    // one candidate per thread: the friend scans' work is heavy-tailed (dense
    // clusters), which the block scheduler balances and a fixed stride does not
    link_kernel<<<(unsigned)g256, 256, 0, s>>>(a, keys);
    ++*nlaunch;
    compress_kernel<<<grid(compress_kernel, 256, g256, 5), 256, 0, s>>>(a);
    ++*nlaunch;
    stats_kernel<<<grid(stats_kernel, 256, g256, 6), 256, 0, s>>>(a, keys, vals);
    ++*nlaunch;
    rep_kernel<<<grid(rep_kernel, 256, g256, 7), 256, 0, s>>>(a, keys, vals);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t nblocks = ceil_div(padded_cap, kScanBlock);
    ++*nlaunch;
    root_count_kernel<<<grid(root_count_kernel, kScanBlock, nblocks, 8), kScanBlock, 0, s>>>(a);
    ++*nlaunch;
    block_scan_kernel<<<1, 1024, 0, s>>>(a);
    ++*nlaunch;
    scatter_kernel<<<grid(scatter_kernel, kScanBlock, nblocks, 9), kScanBlock, 0, s>>>(a, keys, vals);
    return cudaGetLastError();
}

}  // namespace hp
