// search.cu -- the per-trial stages of Algorithm 1 on sm_103a: baseline
// removal, normalisation, boxcar matched filtering and peak detection
// (Section II-B).  Every trial of every DM is processed by one grid, not a
// loop of small per-trial launches.
//
//   baseline  median mode: remedian levels (medians of five, lower median
//             for a trailing partial group) and integer linear interpolation
//             between block centres; mean mode: moving mean over +-H samples
//             with floor division.  Both are exact integers.
//   sigma     1.482602218505602 * median |y|, the median found exactly from a
//             histogram of |y| (exact bins below 4096, then a second pass
//             inside the coarse bucket holding the median when needed).
//   boxcars   S_W(t) = P(t + W) - P(t) from an int64 prefix sum kept in shared
//             memory for a tile of starts plus a halo of the widest boxcar.
//   peaks     S_W(t) >= ceil(thr * sigma * sqrt(W)) (the FP64 limit rounded up
//             once per trial and width, so the per-sample test is an exact
//             integer compare); one candidate per maximal run, at the largest
//             S (first on ties), appended with an atomic counter.
#include <climits>

#include "common.cuh"

namespace hp {
namespace {

constexpr double kMadToSigma = 1.482602218505602;
constexpr int64_t kNever = LLONG_MAX;

// ------------------------------------------------------------- remedian
__device__ __forceinline__ int32_t lower_median_small(const int32_t* v, int r) {
    if (r >= 5) {
        int32_t a = v[0], b = v[1], c = v[2], d = v[3], e = v[4];
#define CS(x, y) { int32_t lo_ = min(x, y); int32_t hi_ = max(x, y); x = lo_; y = hi_; }
        CS(a, b); CS(d, e); CS(c, e); CS(c, d); CS(a, d); CS(a, c); CS(b, e); CS(b, d); CS(b, c);
#undef CS
        return c;
    }
    if (r == 4) {
        const int32_t p = min(v[0], v[1]), P = max(v[0], v[1]);
        const int32_t q = min(v[2], v[3]), Q = max(v[2], v[3]);
        return min(max(p, q), min(P, Q));
    }
    if (r == 3) return max(min(v[0], v[1]), min(max(v[0], v[1]), v[2]));
    if (r == 2) return min(v[0], v[1]);
    return v[0];
}

__constant__ int64_t kPow5[14] = {1, 5, 25, 125, 625, 3125, 15625, 78125, 390625, 1953125,
                                  9765625, 48828125, 244140625, 1220703125};

// q (<= 5) remedian levels over chunks of 5^q values; one value per chunk.
__global__ void __launch_bounds__(256) remedian_pass_kernel(const int32_t* __restrict__ in,
                                                            int64_t in_pitch, int64_t n_in, int q,
                                                            int32_t* __restrict__ out,
                                                            int64_t out_pitch) {
    __shared__ int32_t buf[2][3125];
    const int trial = blockIdx.y;
    const int64_t chunk = kPow5[q];
    const int64_t base = (int64_t)blockIdx.x * chunk;
    int cnt = (int)min(chunk, n_in - base);
    const int32_t* src = in + (int64_t)trial * in_pitch + base;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) buf[0][i] = src[i];
    __syncthreads();
    int cur = 0;
    for (int l = 0; l < q; ++l) {
        const int m = (cnt + 4) / 5;
        for (int i = threadIdx.x; i < m; i += blockDim.x)
            buf[cur ^ 1][i] = lower_median_small(&buf[cur][5 * i], min(5, cnt - 5 * i));
        __syncthreads();
        cur ^= 1;
        cnt = m;
    }
    if (threadIdx.x == 0) out[(int64_t)trial * out_pitch + blockIdx.x] = buf[cur][0];
}

// ------------------------------------------------------- baseline walkers
// Exact baseline b(t) evaluated at consecutive samples t, t+1, ...
struct MedianWalker {
    const int32_t* m;
    int64_t M, P, half;
    int64_t t, next, base, q, r, dq, dr;
    bool interior;

    __device__ void init(int64_t t_) {
        t = t_;
        const int64_t c_last = P * (M - 1) + half;
        if (M == 1 || t <= half) {
            base = m[0]; q = 0; interior = false;
            next = (M == 1) ? LLONG_MAX : half + 1;
            return;
        }
        if (t >= c_last) {
            base = m[M - 1]; q = 0; interior = false; next = LLONG_MAX;
            return;
        }
        const int64_t j = (t - half) / P;
        const int64_t cj = P * j + half;
        const int64_t delta = (int64_t)m[j + 1] - (int64_t)m[j];
        const int64_t num = delta * (t - cj);
        q = floor_div_pos(num, P);
        r = num - q * P;
        dq = floor_div_pos(delta, P);
        dr = delta - dq * P;
        base = m[j];
        interior = true;
        next = cj + P;
    }
    __device__ __forceinline__ int64_t value() const { return base + q; }
    __device__ __forceinline__ void step() {
        ++t;
        if (t == next) { init(t); return; }
        if (interior) {
            q += dq;
            r += dr;
            if (r >= P) { r -= P; ++q; }
        }
    }
};

struct MeanWalker {
    const int32_t* D;
    const int64_t* pre;    // pre[j] = sum of D[0 .. 32 j)
    int64_t n, H, t, sum, cnt;

    __device__ int64_t prefix(int64_t p) const {
        const int64_t blk = p >> 5;
        int64_t s = pre[blk];
        for (int64_t i = blk << 5; i < p; ++i) s += D[i];
        return s;
    }
    __device__ void init(int64_t t_) {
        t = t_;
        const int64_t lo = max((int64_t)0, t - H), hi = min(n - 1, t + H);
        sum = prefix(hi + 1) - prefix(lo);
        cnt = hi - lo + 1;
    }
    __device__ __forceinline__ int64_t value() const { return floor_div_pos(sum, cnt); }
    __device__ __forceinline__ void step() {
        ++t;
        const int64_t add = t + H;
        if (add <= n - 1) { sum += D[add]; ++cnt; }
        const int64_t rem = t - H - 1;
        if (rem >= 0) { sum -= D[rem]; --cnt; }
    }
};

struct BaselineCtx {
    int mode;
    const int32_t* knots;   // median: level-L values, row stride knot_pitch
    int64_t knot_pitch, M, P, half;
    const int64_t* pre;     // mean: block prefix rows, stride pre_pitch
    int64_t pre_pitch, H;
};

struct Walker {
    int mode;
    MedianWalker med;
    MeanWalker mean;
    __device__ void setup(const BaselineCtx& c, const int32_t* Drow, int64_t n, int trial) {
        mode = c.mode;
        if (mode == 0) {
            med.m = c.knots + (int64_t)trial * c.knot_pitch;
            med.M = c.M; med.P = c.P; med.half = c.half;
        } else {
            mean.D = Drow; mean.pre = c.pre + (int64_t)trial * c.pre_pitch;
            mean.n = n; mean.H = c.H;
        }
    }
    __device__ void init(int64_t t) { if (mode == 0) med.init(t); else mean.init(t); }
    __device__ __forceinline__ int64_t value() const { return mode == 0 ? med.value() : mean.value(); }
    __device__ __forceinline__ void step() { if (mode == 0) med.step(); else mean.step(); }
};

// ------------------------------------------------------ mean-mode prefix
__global__ void __launch_bounds__(256) mean_blocksum_kernel(const int32_t* __restrict__ D,
                                                            int64_t pitch, int64_t n,
                                                            int64_t* __restrict__ pre,
                                                            int64_t pre_pitch) {
    const int trial = blockIdx.y;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // 32-sample block
    const int64_t nb = (n + 31) / 32;
    if (j >= nb) return;
    const int32_t* row = D + (int64_t)trial * pitch;
    int64_t s = 0;
    for (int64_t i = j * 32; i < min(n, j * 32 + 32); ++i) s += row[i];
    pre[(int64_t)trial * pre_pitch + j + 1] = s;
}

__global__ void __launch_bounds__(1024) mean_scan_kernel(int64_t* __restrict__ pre,
                                                         int64_t pre_pitch, int64_t nb) {
    __shared__ int64_t warp_tot[32];
    __shared__ int64_t carry;
    int64_t* row = pre + (int64_t)blockIdx.x * pre_pitch;
    if (threadIdx.x == 0) { carry = 0; row[0] = 0; }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t base = 1; base <= nb; base += 1024) {
        const int64_t i = base + threadIdx.x;
        int64_t v = i <= nb ? row[i] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        if (lane == 31) warp_tot[warp] = v;
        __syncthreads();
        if (warp == 0) {
            int64_t w = warp_tot[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t u = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += u;
            }
            warp_tot[lane] = w;
        }
        __syncthreads();
        const int64_t c = carry;
        v += c + (warp > 0 ? warp_tot[warp - 1] : 0);
        if (i <= nb) row[i] = v;
        __syncthreads();
        if (threadIdx.x == 1023) carry = v;
        __syncthreads();
    }
}

// -------------------------------------------------------- |y| histogram
constexpr int kHistChunk = 8192;   // samples per block (256 threads x 32)

__device__ __forceinline__ int hist_bin(int64_t v) {
    return v < kHistFine ? (int)v : kHistFine + (int)min(v >> 12, (int64_t)(kHistFine - 1));
}

__global__ void __launch_bounds__(256) mad_hist_kernel(const int32_t* __restrict__ D,
                                                       int64_t pitch, int64_t n, BaselineCtx bc,
                                                       uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[kHistBins];
    const int trial = blockIdx.y;
    for (int i = threadIdx.x; i < kHistBins; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int32_t* row = D + (int64_t)trial * pitch;
    const int64_t t_begin = (int64_t)blockIdx.x * kHistChunk + threadIdx.x * 32;
    const int64_t t_end = min(n, t_begin + 32);
    if (t_begin < t_end) {
        Walker w;
        w.setup(bc, row, n, trial);
        w.init(t_begin);
        for (int64_t t = t_begin; t < t_end; ++t) {
            int64_t y = (int64_t)row[t] - w.value();
            if (y < 0) y = -y;
            atomicAdd(&h[hist_bin(y)], 1u);
            w.step();
        }
    }
    __syncthreads();
    uint32_t* g = hist + (int64_t)trial * kHistBins;
    for (int i = threadIdx.x; i < kHistBins; i += blockDim.x)
        if (h[i]) atomicAdd(&g[i], h[i]);
}

// Block-wide search of the bin holding rank k (0-based) in a histogram of
// `bins` counts.  Returns the bin and the count of all earlier bins.
__device__ void find_rank_bin(const uint32_t* __restrict__ hrow, int bins, int64_t k, int* bin_out,
                              int64_t* before_out) {
    __shared__ int64_t part[1024];
    __shared__ int s_bin;
    __shared__ int64_t s_before;
    const int per = (bins + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per;
    int64_t mine = 0;
    for (int b = b0; b < min(bins, b0 + per); ++b) mine += hrow[b];
    part[threadIdx.x] = mine;
    if (threadIdx.x == 0) { s_bin = -1; s_before = 0; }
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {   // inclusive Hillis-Steele scan
        const int64_t v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    const int64_t incl = part[threadIdx.x];
    const int64_t excl = incl - mine;
    if (excl <= k && k < incl) {
        int64_t c = excl;
        for (int b = b0; b < min(bins, b0 + per); ++b) {
            if (k < c + hrow[b]) { s_bin = b; s_before = c; break; }
            c += hrow[b];
        }
    }
    __syncthreads();
    *bin_out = s_bin;
    *before_out = s_before;
}

__global__ void __launch_bounds__(1024) mad_select_kernel(uint32_t* __restrict__ hist, int64_t n,
                                                          int32_t* __restrict__ bucket,
                                                          int64_t* __restrict__ rank,
                                                          int64_t* __restrict__ mad) {
    const int trial = blockIdx.x;
    uint32_t* hrow = hist + (int64_t)trial * kHistBins;
    const int64_t k = (n - 1) / 2;
    int bin;
    int64_t before;
    find_rank_bin(hrow, kHistBins, k, &bin, &before);
    if (threadIdx.x == 0) {
        if (bin < kHistFine) {
            mad[trial] = bin;
            bucket[trial] = -1;
        } else {
            bucket[trial] = bin - kHistFine;
            rank[trial] = k - before;
        }
    }
    __syncthreads();
    if (bin >= kHistFine)   // reuse the row for the refinement histogram
        for (int i = threadIdx.x; i < kHistFine; i += blockDim.x) hrow[i] = 0;
}

__global__ void __launch_bounds__(256) mad_refine_hist_kernel(const int32_t* __restrict__ D,
                                                              int64_t pitch, int64_t n,
                                                              BaselineCtx bc,
                                                              const int32_t* __restrict__ bucket,
                                                              uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[kHistFine];
    const int trial = blockIdx.y;
    const int32_t B = bucket[trial];
    if (B < 0) return;
    for (int i = threadIdx.x; i < kHistFine; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int32_t* row = D + (int64_t)trial * pitch;
    const int64_t t_begin = (int64_t)blockIdx.x * kHistChunk + threadIdx.x * 32;
    const int64_t t_end = min(n, t_begin + 32);
    if (t_begin < t_end) {
        Walker w;
        w.setup(bc, row, n, trial);
        w.init(t_begin);
        for (int64_t t = t_begin; t < t_end; ++t) {
            int64_t y = (int64_t)row[t] - w.value();
            if (y < 0) y = -y;
            if ((y >> 12) == B) atomicAdd(&h[y & 4095], 1u);
            w.step();
        }
    }
    __syncthreads();
    uint32_t* g = hist + (int64_t)trial * kHistBins;
    for (int i = threadIdx.x; i < kHistFine; i += blockDim.x)
        if (h[i]) atomicAdd(&g[i], h[i]);
}

__global__ void __launch_bounds__(1024) mad_refine_select_kernel(
    const uint32_t* __restrict__ hist, const int32_t* __restrict__ bucket,
    const int64_t* __restrict__ rank, int64_t* __restrict__ mad) {
    const int trial = blockIdx.x;
    const int32_t B = bucket[trial];
    if (B < 0) return;
    int bin;
    int64_t before;
    find_rank_bin(hist + (int64_t)trial * kHistBins, kHistFine, rank[trial], &bin, &before);
    if (threadIdx.x == 0) mad[trial] = ((int64_t)B << 12) + bin;
}

// sigma and the integer thresholds ceil(thr * sigma * sqrt(W)) per (trial, width)
__global__ void sigma_kernel(const int64_t* __restrict__ mad, int ndm,
                             const int32_t* __restrict__ widths, int nw, float thr,
                             double* __restrict__ sigma, int64_t* __restrict__ tint) {
    const int trial = blockIdx.x * blockDim.x + threadIdx.x;
    if (trial >= ndm) return;
    const double sg = __dmul_rn(kMadToSigma, (double)mad[trial]);
    sigma[trial] = sg;
    for (int k = 0; k < nw; ++k) {
        int64_t v = kNever;
        if (sg > 0.0) {
            const double lim = __dmul_rn(__dmul_rn((double)thr, sg), __dsqrt_rn((double)widths[k]));
            v = (int64_t)ceil(lim);
        }
        tint[(int64_t)trial * nw + k] = v;
    }
}

// ------------------------------------------------------------ detection
constexpr int kDetectThreads = 512;
constexpr int kDetectPer = kDetectTile / kDetectThreads;   // starts per thread

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t* warp_tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t u = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += u;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t u = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += u;
        }
        warp_tot[lane] = w;
    }
    __syncthreads();
    return x - v + (warp > 0 ? warp_tot[warp - 1] : 0);
}

__device__ __forceinline__ void emit(const SearchArgs& a, int trial, int k, int64_t t, int64_t S) {
    const unsigned long long idx = atomicAdd(reinterpret_cast<unsigned long long*>(a.raw_count), 1ull);
    if ((int64_t)idx < a.raw_cap) {
        hp_raw_cand c;
        c.dm_idx = trial;
        c.width_idx = k;
        c.sample = t;
        c.S = S;
        a.raw[idx] = c;
    }
}

__global__ void __launch_bounds__(kDetectThreads) detect_kernel(const __grid_constant__ SearchArgs a,
                                                                BaselineCtx bc) {
    extern __shared__ int64_t P[];   // P[i] = sum of y over samples [base, base + i)
    __shared__ int64_t warp_tot[32];
    const int trial = blockIdx.y;
    const int64_t n = a.nout;
    const int64_t t0 = (int64_t)blockIdx.x * kDetectTile;
    const int64_t base = t0 - 1;
    const int64_t len = min((int64_t)kDetectTile + a.wmax, n - base);
    const int32_t* row = a.D + (int64_t)trial * a.pitch;
    const int tid = threadIdx.x;

    // y over [base, base + len) -> P[1 .. len], then a block-wide prefix sum
    const int64_t per = (len + kDetectThreads - 1) / kDetectThreads;
    const int64_t i0 = min(len, tid * per), i1 = min(len, i0 + per);
    int64_t local = 0;
    if (i0 < i1) {
        Walker w;
        w.setup(bc, row, n, trial);
        int64_t s = base + i0;
        if (s < 0) {                       // the slot before sample 0 holds y = 0
            P[i0 + 1] = 0;
            ++s;
        }
        if (s < base + i1) w.init(s);
        for (; s < base + i1; ++s) {
            const int64_t y = (int64_t)row[s] - w.value();
            P[s - base + 1] = y;
            local += y;
            w.step();
        }
    }
    const int64_t off = block_exclusive_scan(local, warp_tot);
    int64_t run = off;
    for (int64_t i = i0; i < i1; ++i) {
        run += P[i + 1];
        P[i + 1] = run;
    }
    if (tid == 0) P[0] = 0;
    __syncthreads();

    for (int k = 0; k < a.nw; ++k) {
        const int64_t thr_k = a.tint[(int64_t)trial * a.nw + k];
        if (thr_k == kNever) continue;
        const int64_t W = a.widths[k];
        const int64_t last = n - W;                     // last valid boxcar start
        const int64_t ta = t0 + (int64_t)tid * kDetectPer;
        const int64_t tb = min(ta + kDetectPer, min(t0 + kDetectTile, last + 1));
        if (ta >= tb) continue;
        bool prev = false;
        if (ta > 0) prev = (P[ta - 1 - base + W] - P[ta - 1 - base]) >= thr_k;
        for (int64_t t = ta; t < tb; ++t) {
            const int64_t S = P[t - base + W] - P[t - base];
            const bool above = S >= thr_k;
            if (above && !prev) {
                // this thread owns the run that starts at t: follow it to its end
                int64_t best_t = t, best_S = S, Sp = S;
                int64_t u = t + 1;
                bool slow = false;
                Walker wa, wb;                          // y(u-1) leaving, y(u+W-1) entering
                for (; u <= last; ++u) {
                    int64_t Su;
                    if (!slow && u - base + W <= len) {
                        Su = P[u - base + W] - P[u - base];
                    } else {
                        if (!slow) {
                            slow = true;
                            wa.setup(bc, row, n, trial);
                            wb.setup(bc, row, n, trial);
                            wa.init(u - 1);
                            wb.init(u - 1 + W);
                        }
                        Su = Sp - ((int64_t)row[u - 1] - wa.value()) +
                             ((int64_t)row[u - 1 + W] - wb.value());
                        wa.step();
                        wb.step();
                    }
                    if (Su < thr_k) break;
                    if (Su > best_S) { best_S = Su; best_t = u; }
                    Sp = Su;
                }
                emit(a, trial, k, best_t, best_S);
            }
            prev = above;
        }
    }
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

cudaError_t launch_search(const SearchArgs& a, cudaStream_t s, int64_t* nlaunch) {
    cudaError_t e;
    const int64_t n = a.nout;
    const int ndm = a.ndm;
    if (ndm <= 0 || n <= 0) return cudaSuccess;
    if ((e = cudaMemsetAsync(a.raw_count, 0, sizeof(int64_t), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(a.hist, 0, (size_t)ndm * kHistBins * 4, s)) != cudaSuccess) return e;

    BaselineCtx bc{};
    bc.mode = a.baseline_mode;
    if (a.baseline_mode == 0) {
        const int L = a.levels;
        int64_t P = 1;
        for (int l = 0; l < L; ++l) P *= 5;
        if (L == 0) {
            bc.knots = a.D;
            bc.knot_pitch = a.pitch;
            bc.M = n;
        } else {
            const int32_t* in = a.D;
            int64_t in_pitch = a.pitch, n_in = n;
            int32_t* bufs[2] = {a.lvl_a, a.lvl_b};
            const int64_t pitches[2] = {a.lvl_pitch_a, a.lvl_pitch_b};
            int left = L, which = 0;
            while (left > 0) {
                const int q = left < 5 ? left : 5;
                int64_t chunk = 1;
                for (int l = 0; l < q; ++l) chunk *= 5;
                const int64_t n_out = ceil_div(n_in, chunk);
                int32_t* out = bufs[which];
                const int64_t out_pitch = which == 0 ? pitches[0] : pitches[1];
                if (n_out > out_pitch) return cudaErrorInvalidValue;
                ++*nlaunch;
                remedian_pass_kernel<<<dim3((unsigned)n_out, ndm), 256, 0, s>>>(in, in_pitch, n_in, q,
                                                                            out, out_pitch);
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
                in = out;
                in_pitch = out_pitch;
                n_in = n_out;
                which ^= 1;
                left -= q;
            }
            bc.knots = in;
            bc.knot_pitch = in_pitch;
            bc.M = n_in;
        }
        bc.P = P;
        bc.half = (P - 1) / 2;
    } else {
        bc.pre = a.mean_pre;
        bc.pre_pitch = a.mean_pitch;
        bc.H = a.win / 2;
        const int64_t nb = ceil_div(n, 32);
        ++*nlaunch;
        mean_blocksum_kernel<<<dim3((unsigned)ceil_div(nb, 256), ndm), 256, 0, s>>>(a.D, a.pitch, n,
                                                                                 a.mean_pre, a.mean_pitch);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        ++*nlaunch;
        mean_scan_kernel<<<ndm, 1024, 0, s>>>(a.mean_pre, a.mean_pitch, nb);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }

    const dim3 hgrid((unsigned)ceil_div(n, kHistChunk), ndm);
    ++*nlaunch;
    mad_hist_kernel<<<hgrid, 256, 0, s>>>(a.D, a.pitch, n, bc, a.hist);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ++*nlaunch;
    mad_select_kernel<<<ndm, 1024, 0, s>>>(a.hist, n, a.refine_bucket, a.refine_rank, a.mad);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ++*nlaunch;
    mad_refine_hist_kernel<<<hgrid, 256, 0, s>>>(a.D, a.pitch, n, bc, a.refine_bucket, a.hist);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ++*nlaunch;
    mad_refine_select_kernel<<<ndm, 1024, 0, s>>>(a.hist, a.refine_bucket, a.refine_rank, a.mad);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ++*nlaunch;
    sigma_kernel<<<(unsigned)ceil_div(ndm, 128), 128, 0, s>>>(a.mad, ndm, a.widths, a.nw, a.thr,
                                                              a.sigma, a.tint);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;

    const size_t smem = ((size_t)kDetectTile + (size_t)a.wmax + 2) * sizeof(int64_t);
    if ((e = cudaFuncSetAttribute(detect_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
        return e;
    const dim3 dgrid((unsigned)ceil_div(n, kDetectTile), ndm);
    ++*nlaunch;
    detect_kernel<<<dgrid, kDetectThreads, smem, s>>>(a, bc);
    return cudaGetLastError();
}

}  // namespace hp
