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
#include <type_traits>

#include "common.cuh"

namespace hp {
namespace {

constexpr double kMadToSigma = 1.482602218505602;
constexpr int64_t kNever = LLONG_MAX;

// ------------------------------------------------------------- remedian
__device__ __forceinline__ int32_t lower_median_small(const int32_t* v, int r) {
    if (r >= 5) return median5(v[0], v[1], v[2], v[3], v[4]);
    if (r == 4) {
        const int32_t p = min(v[0], v[1]), P = max(v[0], v[1]);
        const int32_t q = min(v[2], v[3]), Q = max(v[2], v[3]);
        return min(max(p, q), min(P, Q));
    }
    if (r == 3) return max(min(v[0], v[1]), min(max(v[0], v[1]), v[2]));
    if (r == 2) return min(v[0], v[1]);
    return v[0];
}

// Second-level remedian values the dedispersion could not form: the group of
// 25 samples straddling each edge k bt of its time tiles (0 < k < ntt, unless
// the edge is a multiple of 25) and a last partial group (lower medians of a
// short group, as in the passes below).  Thread k of row `trial`, k in 1..ntt.
__global__ void __launch_bounds__(128) level2_fixup_kernel(const int32_t* __restrict__ D,
                                                           int64_t pitch, int64_t n, int64_t bt,
                                                           int32_t* __restrict__ lv,
                                                           int64_t lv_pitch) {
    const int trial = blockIdx.y;
    const int64_t ntt = (n + bt - 1) / bt;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < 1 || k > ntt) return;
    int64_t g;
    if (k < ntt) {
        const int64_t e = k * bt;   // e < n
        if (e % 25 == 0) return;
        g = e / 25;
    } else {
        g = (n - 1) / 25;
        if (25 * g + 25 <= n) return;
    }
    const int32_t* row = D + (int64_t)trial * pitch + 25 * g;
    const int cnt = (int)min((int64_t)25, n - 25 * g);
    const int nm = (cnt + 4) / 5;
    int32_t m[5];
    for (int j = 0; j < nm; ++j) {
        int32_t v[5];
        const int r = min(5, cnt - 5 * j);
        for (int i = 0; i < r; ++i) v[i] = row[5 * j + i];
        m[j] = lower_median_small(v, r);
    }
    lv[(int64_t)trial * lv_pitch + g] = lower_median_small(m, nm);
}

__constant__ int64_t kPow5[14] = {1, 5, 25, 125, 625, 3125, 15625, 78125, 390625, 1953125,
                                  9765625, 48828125, 244140625, 1220703125};

// q (<= 5) remedian levels over chunks of 5^q values; one value per chunk.
// A block takes the chunks blockIdx.x, blockIdx.x + gridDim.x, ... of one
// trial; the loads of its next chunk are in flight while the current chunk's
// levels are formed in shared memory.
constexpr int kRemThreads = 256;
constexpr int kRemPer = (3125 + kRemThreads - 1) / kRemThreads;   // values per thread
constexpr int kRemChunksPerBlock = 8;

__global__ void __launch_bounds__(kRemThreads) remedian_pass_kernel(const int32_t* __restrict__ in,
                                                                   int64_t in_pitch, int64_t n_in,
                                                                   int q, int32_t* __restrict__ out,
                                                                   int64_t out_pitch, int64_t n_out) {
    __shared__ int32_t buf[2][3125];
    const int trial = blockIdx.y;
    const int64_t chunk = kPow5[q];
    const int32_t* row = in + (int64_t)trial * in_pitch;
    int32_t v[kRemPer];
    auto load = [&](int64_t c) {
        const int64_t base = c * chunk;
        const int cnt = (int)min(chunk, n_in - base);
#pragma unroll
        for (int u = 0; u < kRemPer; ++u) {
            const int i = (int)threadIdx.x + u * kRemThreads;
            v[u] = i < cnt ? __ldg(row + base + i) : 0;
        }
    };
    int64_t c = blockIdx.x;
    if (c < n_out) load(c);
    for (; c < n_out; c += gridDim.x) {
        int cnt = (int)min(chunk, n_in - c * chunk);
#pragma unroll
        for (int u = 0; u < kRemPer; ++u) {
            const int i = (int)threadIdx.x + u * kRemThreads;
            if (i < cnt) buf[0][i] = v[u];
        }
        if (c + gridDim.x < n_out) load(c + gridDim.x);
        __syncthreads();
        int cur = 0, l = 0;
        // levels with more than 32 medians: the whole block, a barrier each
        for (; l < q && cnt > 160; ++l) {
            const int m = (cnt + 4) / 5;
            for (int i = threadIdx.x; i < m; i += blockDim.x)
                buf[cur ^ 1][i] = lower_median_small(&buf[cur][5 * i], min(5, cnt - 5 * i));
            __syncthreads();
            cur ^= 1;
            cnt = m;
        }
        // the rest (at most 32 medians per level) in the first warp
        if (threadIdx.x < 32) {
            for (; l < q; ++l) {
                const int m = (cnt + 4) / 5;
                if ((int)threadIdx.x < m)
                    buf[cur ^ 1][threadIdx.x] =
                        lower_median_small(&buf[cur][5 * threadIdx.x], min(5, cnt - 5 * (int)threadIdx.x));
                __syncwarp();
                cur ^= 1;
                cnt = m;
            }
            if (threadIdx.x == 0) out[(int64_t)trial * out_pitch + c] = buf[cur][0];
        }
        __syncthreads();   // buf is rewritten with the next chunk
    }
}

// ------------------------------------------------------- baseline walkers
// Exact baseline b(t) evaluated at consecutive samples t, t+1, ...

// The median baseline interpolates linearly between knots P samples apart:
// within an interval b(t) = m_j + floor(delta (t - c_j) / P), kept as the
// quotient q and remainder r of that division and advanced by the quotient
// and remainder of delta / P per sample.  I is the integer type of the
// per-sample state: int32 when P < 2^30 (then r + dr < 2P < 2^31, and q lies
// between 0 and delta (P - 1) / P, inside int32 for series within +-2^30),
// int64 otherwise; the set-up is 64-bit either way.
template <typename I>
struct MedianWalkerT {
    const int32_t* m;
    int64_t M, P, half;
    int64_t next;          // the sample at which the walker is set up again
    I base, q, r, dq, dr, PI;
    int32_t left;          // samples until then
    bool interior;

    __device__ void init(int64_t t) {
        const int64_t c_last = P * (M - 1) + half;
        int64_t nx;
        PI = (I)P;
        if (M == 1 || t <= half) {
            base = m[0]; q = 0; r = 0; dq = 0; dr = 0; interior = false;
            nx = (M == 1) ? LLONG_MAX : half + 1;
        } else if (t >= c_last) {
            base = m[M - 1]; q = 0; r = 0; dq = 0; dr = 0; interior = false;
            nx = LLONG_MAX;
        } else {
            const int64_t j = (t - half) / P;
            const int64_t cj = P * j + half;
            const int64_t delta = (int64_t)m[j + 1] - (int64_t)m[j];
            const int64_t num = delta * (t - cj);
            const int64_t q64 = floor_div_pos(num, P);
            const int64_t dq64 = floor_div_pos(delta, P);
            q = (I)q64;
            r = (I)(num - q64 * P);
            dq = (I)dq64;
            dr = (I)(delta - dq64 * P);
            base = m[j];
            interior = true;
            nx = cj + P;
        }
        next = nx;
        left = (int32_t)min(nx - t, (int64_t)1 << 30);
    }
    __device__ __forceinline__ int64_t value() const { return (int64_t)(base + q); }
    __device__ __forceinline__ void step() {
        if (--left == 0) { init(next); return; }
        if (interior) {
            q += dq;
            r += dr;
            if (r >= PI) { r -= PI; ++q; }
        }
    }
    // y = v - b over the next N samples when no new interval starts among them
    // (left > N): the plain update, which the flat parts (dq = dr = 0) share;
    // f(y) for each
    template <int N, class F>
    __device__ __forceinline__ void subtract_run(int32_t (&v)[N], F&& f) {
        I q_ = q, r_ = r;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            v[i] = (int32_t)((int64_t)v[i] - (int64_t)(base + q_));
            f(v[i]);
            q_ += dq;
            r_ += dr;
            if (r_ >= PI) { r_ -= PI; ++q_; }
        }
        q = q_;
        r = r_;
        left -= N;
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

// Walker<0> / Walker<2>: running-median baseline; Walker<1>: moving-mean baseline.  The
// mode is uniform per launch, so the kernels are instantiated per mode.
template <int MODE> struct Walker;

// median mode with knots less than 2^30 samples apart (every practical case)
template <> struct Walker<0> : MedianWalkerT<int32_t> {
    __device__ void setup(const BaselineCtx& c, const int32_t*, int64_t, int trial) {
        m = c.knots + (int64_t)trial * c.knot_pitch;
        M = c.M; P = c.P; half = c.half;
    }
};

// median mode, knots 2^30 samples apart or more
template <> struct Walker<2> : MedianWalkerT<int64_t> {
    __device__ void setup(const BaselineCtx& c, const int32_t*, int64_t, int trial) {
        m = c.knots + (int64_t)trial * c.knot_pitch;
        M = c.M; P = c.P; half = c.half;
    }
};

template <> struct Walker<1> : MeanWalker {
    __device__ void setup(const BaselineCtx& c, const int32_t* Drow, int64_t n_, int trial) {
        D = Drow; pre = c.pre + (int64_t)trial * c.pre_pitch;
        n = n_; H = c.H;
    }
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

// The 32 samples of one thread's chunk, with 16-byte loads when the row is
// 16-byte aligned (pitch a multiple of 4 and an aligned base).
__device__ __forceinline__ void load_chunk32(const int32_t* __restrict__ row, int64_t t_begin,
                                             int64_t t_end, bool vec, int32_t (&v)[32]) {
    if (vec && t_end - t_begin == 32) {
        const int4* p = reinterpret_cast<const int4*>(row + t_begin);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int4 x = __ldg(p + q);
            v[4 * q] = x.x; v[4 * q + 1] = x.y; v[4 * q + 2] = x.z; v[4 * q + 3] = x.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < 32; ++q) v[q] = t_begin + q < t_end ? row[t_begin + q] : 0;
    }
}

// Histogram of |y| per trial; also writes y = D - b (int32: |D|, |b| < 2^21)
// for the passes after it.  A block takes kHistBlock consecutive samples of
// one trial; each thread walks kHistSpan consecutive samples with one baseline
// walker (set up once, its divisions amortised over the span), kHistStep at a
// time: every byte it loads is used, and the block's shared bins are cleared
// and flushed once per kHistBlock samples.  Each thread reads a step before it
// writes it, so Y may alias D (median mode, whose walker reads only the knots).
constexpr int kHistThreads = 256;
constexpr int kHistSpan = 256;                           // samples per thread
constexpr int kHistStep = 16;                            // samples per load step
constexpr int kHistBlock = kHistThreads * kHistSpan;     // samples per block

template <int MODE>
__global__ void __launch_bounds__(kHistThreads, 4) mad_hist_kernel(const int32_t* D, int64_t pitch,
                                                                int64_t n, BaselineCtx bc, int vec,
                                                                uint32_t* __restrict__ hist,
                                                                int32_t* Y, int64_t ypitch,
                                                                int yvec) {
    __shared__ uint32_t h[kHistBins];
    __shared__ __align__(16) int4 tile[kHistThreads / 32][32 * kHistStep / 4];
    const int trial = blockIdx.y;
    for (int i = threadIdx.x; i < kHistBins; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int32_t* row = D + (int64_t)trial * pitch;
    int32_t* yrow = Y + (int64_t)trial * ypitch;
    const int64_t blk0 = (int64_t)blockIdx.x * kHistBlock;
    // first sample of step 0 and the distance between steps
    const int64_t s_first = blk0 + (int64_t)threadIdx.x * kHistSpan;
    constexpr int64_t stride = kHistStep;
    if (vec && yvec && blk0 + kHistBlock <= n) {
        // Whole block, aligned rows: a warp moves the step's 32 pieces of 16
        // samples (one per lane, a span apart) through shared memory, eight whole
        // 64-byte pieces per load or store instruction; lane l then reads its own
        // piece.  16-byte slot of (piece p, quarter c): 4p + (c ^ ((p >> 1) & 3)),
        // so that both the eight lanes of a cooperative access (pieces p, p + 1,
        // quarters 0-3) and eight lanes reading their own pieces (p .. p + 7, one
        // quarter) touch eight distinct 16-byte bank groups.
        const int lane = threadIdx.x & 31;
        int4* T = tile[threadIdx.x >> 5];
        const int64_t wbase = blk0 + (int64_t)(threadIdx.x & ~31) * kHistSpan;
        auto slot = [](int p, int c) { return 4 * p + (c ^ ((p >> 1) & 3)); };
        int4 g[4];
        auto gload = [&](int j) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int p = (lane >> 2) + 8 * k, c = lane & 3;
                g[k] = __ldg(reinterpret_cast<const int4*>(row + wbase + (int64_t)p * kHistSpan +
                                                           j * kHistStep) + c);
            }
        };
        Walker<MODE> w;
        w.setup(bc, row, n, trial);
        w.init(s_first);
        gload(0);
        for (int j = 0; j < kHistSpan / kHistStep; ++j) {
            __syncwarp();
#pragma unroll
            for (int k = 0; k < 4; ++k) T[slot((lane >> 2) + 8 * k, lane & 3)] = g[k];
            __syncwarp();
            if (j + 1 < kHistSpan / kHistStep) gload(j + 1);
            int32_t v[kHistStep];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int4 x = T[slot(lane, c)];
                v[4 * c] = x.x; v[4 * c + 1] = x.y; v[4 * c + 2] = x.z; v[4 * c + 3] = x.w;
            }
            auto count = [&](int32_t y) {
                const uint32_t m = y < 0 ? 0u - (uint32_t)y : (uint32_t)y;
                atomicAdd(&h[m < (uint32_t)kHistFine ? (int)m
                                                     : kHistFine + (int)min(m >> 12, (uint32_t)(kHistFine - 1))],
                          1u);
            };
            bool fast = false;
            if constexpr (MODE != 1) fast = w.left > kHistStep;
            if (fast) {
                if constexpr (MODE != 1) w.subtract_run(v, count);
            } else {
#pragma unroll
                for (int q = 0; q < kHistStep; ++q) {
                    const int32_t y = (int32_t)((int64_t)v[q] - w.value());
                    v[q] = y;
                    count(y);
                    w.step();
                }
            }
#pragma unroll
            for (int c = 0; c < 4; ++c)
                T[slot(lane, c)] = make_int4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
            __syncwarp();
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int p = (lane >> 2) + 8 * k, c = lane & 3;
                reinterpret_cast<int4*>(yrow + wbase + (int64_t)p * kHistSpan + j * kHistStep)[c] =
                    T[slot(p, c)];
            }
        }
    } else if (s_first < n) {
        Walker<MODE> w;
        w.setup(bc, row, n, trial);
        w.init(s_first);
        for (int j = 0; j < kHistSpan / kHistStep; ++j) {
            const int64_t s = s_first + j * stride;
            if (s >= n) break;
            const int64_t t_end = min(n, s + kHistStep);
            int32_t v[kHistStep];
            const bool whole = s + kHistStep <= n;
            if (vec && whole) {
                const int4* p = reinterpret_cast<const int4*>(row + s);
#pragma unroll
                for (int q = 0; q < kHistStep / 4; ++q) {
                    const int4 x = __ldg(p + q);
                    v[4 * q] = x.x; v[4 * q + 1] = x.y; v[4 * q + 2] = x.z; v[4 * q + 3] = x.w;
                }
            } else {
#pragma unroll
                for (int q = 0; q < kHistStep; ++q) v[q] = s + q < t_end ? row[s + q] : 0;
            }
#pragma unroll
            for (int q = 0; q < kHistStep; ++q) {
                if (whole || s + q < t_end) {
                    const int32_t y = (int32_t)((int64_t)v[q] - w.value());
                    v[q] = y;
                    const uint32_t m = y < 0 ? 0u - (uint32_t)y : (uint32_t)y;
                    atomicAdd(&h[m < (uint32_t)kHistFine ? (int)m
                                                         : kHistFine + (int)min(m >> 12, (uint32_t)(kHistFine - 1))],
                              1u);
                    w.step();
                }
            }
            if (yvec && whole) {
                int4* p = reinterpret_cast<int4*>(yrow + s);
#pragma unroll
                for (int q = 0; q < kHistStep / 4; ++q)
                    p[q] = make_int4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            } else {
#pragma unroll
                for (int q = 0; q < kHistStep; ++q)
                    if (s + q < t_end) yrow[s + q] = v[q];
            }
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
                                                          int64_t* __restrict__ mad,
                                                          int64_t* __restrict__ ybound) {
    const int trial = blockIdx.x;
    uint32_t* hrow = hist + (int64_t)trial * kHistBins;
    const int64_t k = (n - 1) / 2;
    if (ybound) {
        // an upper bound of max |y| from the highest non-empty bin: exact below
        // kHistFine, the top of a coarse bin above, none for the last coarse bin
        __shared__ int s_top;
        if (threadIdx.x == 0) s_top = -1;
        __syncthreads();
        int top = -1;
        for (int b = threadIdx.x; b < kHistBins; b += blockDim.x)
            if (hrow[b]) top = b;
        if (top >= 0) atomicMax(&s_top, top);
        __syncthreads();
        if (threadIdx.x == 0) {
            const int t = s_top;
            ybound[trial] = t < 0 ? 0
                          : t < kHistFine ? (int64_t)t
                          : t == kHistBins - 1 ? -1
                          : ((int64_t)(t - kHistFine + 1) << 12) - 1;
        }
    }
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

__global__ void __launch_bounds__(256) mad_refine_hist_kernel(const int32_t* __restrict__ Y,
                                                              int64_t ypitch, int64_t n, int yvec,
                                                              const int32_t* __restrict__ bucket,
                                                              uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[kHistFine];
    const int trial = blockIdx.y;
    const int32_t B = bucket[trial];
    if (B < 0) return;
    for (int i = threadIdx.x; i < kHistFine; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int32_t* yrow = Y + (int64_t)trial * ypitch;
    const int64_t t_begin = (int64_t)blockIdx.x * kHistChunk + threadIdx.x * 32;
    const int64_t t_end = min(n, t_begin + 32);
    if (t_begin < t_end) {
        int32_t v[32];
        load_chunk32(yrow, t_begin, t_end, yvec != 0, v);
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            if (t_begin + q < t_end) {
                const int64_t y = v[q] < 0 ? -(int64_t)v[q] : (int64_t)v[q];
                if ((y >> 12) == B) atomicAdd(&h[y & 4095], 1u);
            }
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
constexpr int kDetectThreads = 256;
constexpr int kDetectPer = kDetectTile / kDetectThreads;   // starts per thread

// Every boxcar sum of this trial fits int32 with room to spare: its |y| bound
// times (the widest boxcar + 32) stays below 2^31 - 1 (the 32-bit detection's
// group bound adds two 15-sample partial sums to a boxcar sum).
__device__ __forceinline__ bool narrow_trial(const SearchArgs& a, int trial) {
    if (!a.ybound) return false;
    const int64_t yb = a.ybound[trial];
    return yb >= 0 && yb * (a.ybound_w + 32) < (int64_t)INT32_MAX;
}


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
        c.sample = t * a.sample_mul + a.t_offset;
        c.S = S;
        a.raw[idx] = c;
    }
}

// Follow the run of above-threshold starts that begins at ts with the whole
// warp (32 starts per step).  Returns false with the run's largest S and first
// position, or true when the run continues past the tile halo: then *tail_u is
// the first start not yet examined (the run goes on at least to tail_u - 1).
template <typename BoxcarFn>
__device__ __forceinline__ bool follow_run(int64_t ts, int64_t last, int64_t base, int64_t len,
                                           int64_t W, int64_t thr, BoxcarFn boxcar, int lane,
                                           int64_t* best_S_out, int64_t* best_t_out,
                                           int64_t* tail_u) {
    int64_t best_S = LLONG_MIN, best_t = ts;
    bool tail = false;
    for (int64_t u0 = ts;; u0 += 32) {
        const int64_t u = u0 + lane;
        const bool inr = u <= last && u - base + W <= len;
        int64_t Su = 0;
        bool ab = false;
        if (inr) {
            Su = boxcar(u);
            ab = Su >= thr;
        }
        const unsigned stop = __ballot_sync(0xffffffffu, !ab);
        const int first = stop ? __ffs(stop) - 1 : 32;
        int64_t cs = (lane < first) ? Su : LLONG_MIN;
        int64_t ct = u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int64_t os = __shfl_down_sync(0xffffffffu, cs, o);
            const int64_t ot = __shfl_down_sync(0xffffffffu, ct, o);
            if (os > cs || (os == cs && ot < ct)) { cs = os; ct = ot; }
        }
        cs = __shfl_sync(0xffffffffu, cs, 0);
        ct = __shfl_sync(0xffffffffu, ct, 0);
        if (cs > best_S) { best_S = cs; best_t = ct; }
        if (!stop) continue;
        const int64_t ue = u0 + first;                 // first start not seen above
        tail = ue <= last && ue - base + W > len;
        *tail_u = ue;
        break;
    }
    *best_S_out = best_S;
    *best_t_out = best_t;
    return tail;
}

// follow_run for sums that fit int32 (the 32-bit detection): 4 consecutive
// starts per lane, 128 per warp step, the running maximum in 32 bits.
template <class BoxcarFn>
__device__ __forceinline__ bool follow_run32(int64_t ts, int64_t last, int64_t base, int64_t len,
                                             int64_t W, int32_t thr, BoxcarFn boxcar, int lane,
                                             int64_t* best_S_out, int64_t* best_t_out,
                                             int64_t* tail_u) {
    int32_t best_S = INT32_MIN;
    int64_t best_t = ts;
    bool tail = false;
    for (int64_t u0 = ts;; u0 += 128) {
        const int64_t ub = u0 + 4 * lane;
        int32_t Sv[4];
        int lane_first = 4;                      // first of this lane's starts not above
#pragma unroll
        for (int e = 3; e >= 0; --e) {
            const int64_t u = ub + e;
            const bool inr = u <= last && u - base + W <= len;
            Sv[e] = inr ? boxcar(u) : 0;
            if (!(inr && Sv[e] >= thr)) lane_first = e;
        }
        const unsigned stop = __ballot_sync(0xffffffffu, lane_first < 4);
        const int first_lane = stop ? __ffs(stop) - 1 : 32;
        const int lim = lane < first_lane ? 4 : (lane == first_lane ? lane_first : 0);
        int32_t cs = INT32_MIN;
        int ct = 4 * lane;                       // start offset from u0
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (e < lim && Sv[e] > cs) { cs = Sv[e]; ct = 4 * lane + e; }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int32_t os = __shfl_down_sync(0xffffffffu, cs, o);
            const int ot = __shfl_down_sync(0xffffffffu, ct, o);
            if (os > cs || (os == cs && ot < ct)) { cs = os; ct = ot; }
        }
        cs = __shfl_sync(0xffffffffu, cs, 0);
        ct = __shfl_sync(0xffffffffu, ct, 0);
        if (cs > best_S) { best_S = cs; best_t = u0 + ct; }
        if (!stop) continue;
        const int64_t ue = u0 + 4 * first_lane + __shfl_sync(0xffffffffu, lane_first, first_lane);
        tail = ue <= last && ue - base + W > len;
        *tail_u = ue;
        break;
    }
    *best_S_out = best_S;
    *best_t_out = best_t;
    return tail;
}

// One tile of starts of one trial with an int64 prefix (the trials that
// detect32_kernel cannot take).
__device__ void detect_tile(const SearchArgs& a, int trial, int64_t tile) {
    extern __shared__ int64_t P[];   // P[i] = sum of y over samples [base, base + i)
    __shared__ int64_t warp_tot[32];
    __shared__ int64_t warp_max[32];
    __shared__ unsigned above_bits[kDetectThreads / 32][kDetectPer];
    __shared__ int64_t thr_s[kMaxWidths];     // this trial's integer thresholds
    __shared__ int32_t width_s[kMaxWidths];
    const int64_t n = a.nout;
    const int64_t t0 = tile * kDetectTile;
    const int64_t base = t0 - 1;
    const int len = (int)min((int64_t)kDetectTile + a.wmax, n - base);   // <= tile + kMaxWidth
    const int32_t* yrow = a.Y + (int64_t)trial * a.ypitch;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < a.nw) {
        thr_s[tid] = a.tint[(int64_t)trial * a.nw + tid];
        width_s[tid] = a.widths[tid];
    }

    // y over [base, base + len) into P[1 ..] with coalesced loads, a batch of
    // independent loads in flight per thread (the slot before sample 0 holds
    // y = 0), then one contiguous chunk per thread (an odd chunk length keeps
    // the 16 threads of a half-warp on distinct banks) and a block prefix sum
    constexpr int kLoadBatch = 8;
    for (int ib = tid; ib < len; ib += kLoadBatch * kDetectThreads) {
        int32_t v[kLoadBatch];
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
            const int i = ib + u * kDetectThreads;
            const int64_t s = base + i;
            v[u] = (i < len && s >= 0) ? __ldg(yrow + s) : 0;
        }
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
            const int i = ib + u * kDetectThreads;
            if (i < len) P[i + 1] = (int64_t)v[u];
        }
    }
    __syncthreads();
    const int per = ((len + kDetectThreads - 1) / kDetectThreads) | 1;
    const int i0 = min(len, tid * per), i1 = min(len, i0 + per);
    int64_t local = 0, ymax = 0;
    for (int i = i0; i < i1; ++i) {
        const int64_t y = P[i + 1];
        local += y;
        ymax = max(ymax, y < 0 ? -y : y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ymax = max(ymax, __shfl_xor_sync(0xffffffffu, ymax, o));
    if (lane == 0) warp_max[warp] = ymax;
    const int64_t off = block_exclusive_scan(local, warp_tot);   // (synchronises)
    int64_t run = off;
    for (int i = i0; i < i1; ++i) {
        run += P[i + 1];
        P[i + 1] = run;
    }
    if (tid == 0) P[0] = 0;
    __syncthreads();
    int64_t tile_max = 0;
    for (int w = 0; w < kDetectThreads / 32; ++w) tile_max = max(tile_max, warp_max[w]);
    // every boxcar sum of this tile fits int32, so wrapped 32-bit prefix
    // differences are exact
    const bool narrow = tile_max * (int64_t)a.wmax < (int64_t)INT32_MAX;
    const uint32_t* P32 = reinterpret_cast<const uint32_t*>(P);   // low word of P[i]: P32[2 i]

    // starts handled by this thread: t = t0 + j * kDetectThreads + tid
    const int i_first = tid + 1;                                  // t - base for j = 0
    uint32_t pr[kDetectPer];
#pragma unroll
    for (int j = 0; j < kDetectPer; ++j) {
        const int i = i_first + j * kDetectThreads;
        pr[j] = (narrow && i <= len) ? P32[2 * i] : 0u;
    }

    // the block that holds start nwin - 1 reports the carry flags
    const bool carry_here = a.carry_out && a.nwin - 1 >= t0 && a.nwin - 1 < t0 + kDetectTile;
    for (int k = 0; k < a.nw; ++k) {
        const int64_t thr_k = thr_s[k];
        if (thr_k == kNever) {
            if (carry_here && tid == 0) a.carry_out[(int64_t)trial * a.nw + k] = 0;
            continue;
        }
        // a run at start 0 continues one the previous gulp already reported
        const bool cin = a.carry_in && t0 == 0 && a.carry_in[(int64_t)trial * a.nw + k];
        const int Wi = width_s[k];
        const int64_t W = Wi;
        const int64_t last = n - W;                     // last valid boxcar start
        const int64_t tend = min(t0 + kDetectTile, last + 1);
        auto box64 = [&](int64_t u) { return P[u - base + W] - P[u - base]; };
        auto box32 = [&](int64_t u) {
            const int i = (int)(u - base);
            return (int64_t)(int32_t)(P32[2 * (i + Wi)] - P32[2 * i]);
        };
        if (carry_here && tid == 0)    // is start nwin - 1 above threshold?
            a.carry_out[(int64_t)trial * a.nw + k] =
                a.nwin - 1 < tend && box64(a.nwin - 1) >= thr_k;
        if (t0 >= tend) continue;
        const int32_t thr32 = (int32_t)min(thr_k, (int64_t)INT32_MAX);
        const bool full = t0 + kDetectTile <= tend;     // every start of the tile is valid
        // hot loop: only the above-threshold mask of each warp-wide group of
        // starts (runs are rare; their starts are found below)
        unsigned any = 0;
        if (narrow) {
#pragma unroll
            for (int j = 0; j < kDetectPer; ++j) {
                const int i = i_first + j * kDetectThreads;
                bool above = (int32_t)(P32[2 * (i + Wi)] - pr[j]) >= thr32;
                if (!full) above = above && t0 + (int64_t)(i - 1) < tend;
                const unsigned bits = __ballot_sync(0xffffffffu, above);
                if (lane == 0) above_bits[warp][j] = bits;
                any |= bits;
            }
        } else {
#pragma unroll 1
            for (int j = 0; j < kDetectPer; ++j) {
                const int64_t t = t0 + (int64_t)j * kDetectThreads + tid;
                const bool above = t < tend && box64(t) >= thr_k;
                const unsigned bits = __ballot_sync(0xffffffffu, above);
                if (lane == 0) above_bits[warp][j] = bits;
                any |= bits;
            }
        }
        if (!any) continue;
        __syncwarp();
        // runs are rare: follow each with the whole warp outside the unrolled loop
#pragma unroll 1
        for (int j = 0; j < kDetectPer; ++j) {
            const unsigned bits = above_bits[warp][j];
            if (!bits) continue;
            const int64_t tg = t0 + (int64_t)j * kDetectThreads + warp * 32;   // group base
            // a start opens a run when its left neighbour is below threshold (for
            // lane 0 the neighbour is start tg - 1 of the group before)
            const bool left = tg > 0 && (narrow ? box32(tg - 1) : box64(tg - 1)) >= thr_k;
            unsigned starts = bits & ~((bits << 1) | (left ? 1u : 0u));
            // streamed search: runs must begin inside the window [0, nwin), and a
            // run at start 0 that the previous gulp left open is not reported again
            if (a.nwin < tg + 32) starts &= a.nwin <= tg ? 0u : (1u << (int)(a.nwin - tg)) - 1u;
            if (cin && tg == 0) starts &= ~1u;
            while (starts) {
                const int L = __ffs(starts) - 1;
                starts &= starts - 1;
                int64_t bS, bt, tu = 0;
                const bool tail =
                    narrow ? follow_run(tg + L, last, base, len, W, thr_k, box32, lane, &bS, &bt, &tu)
                           : follow_run(tg + L, last, base, len, W, thr_k, box64, lane, &bS, &bt, &tu);
                if (lane == 0) {
                    if (!tail) {
                        emit(a, trial, k, bt, bS);
                    } else {
                        // rare: the run leaves the tile halo; tail_kernel finishes it
                        const unsigned long long q = atomicAdd(
                            reinterpret_cast<unsigned long long*>(a.tail_count), 1ull);
                        if ((int64_t)q < a.tail_cap) {
                            TailRec r;
                            r.trial = trial;
                            r.k = k;
                            r.u = tu;
                            r.S_prev = box64(tu - 1);
                            r.best_S = bS;
                            r.best_t = bt;
                            a.tails[q] = r;
                        } else {
                            latch_status(a.status, HP_ERR_CAND_OVERFLOW);
                        }
                    }
                }
            }
        }
        __syncwarp();
    }
}

// Blocks loop over the tiles of their trial, a few blocks per trial: the
// trials this kernel takes are rare, and the others leave at once.
constexpr int kDetectBlocksPerTrial = 8;
__global__ void __launch_bounds__(kDetectThreads) detect_kernel(const __grid_constant__ SearchArgs a) {
    const int trial = blockIdx.y;
    if (narrow_trial(a, trial)) return;   // detect32_kernel takes the trial
    const int64_t ntiles = (a.nout + kDetectTile - 1) / kDetectTile;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        detect_tile(a, trial, tile);
        __syncthreads();   // the shared prefix and bit masks are rebuilt for the next tile
    }
}

// ------------------------------------------------ detection, 32-bit prefix
// For trials whose every boxcar sum fits int32 (ybound * widest boxcar <
// 2^31 - 1).  A block walks one segment of a trial's starts in chunks of 2048
// (128 threads, 16 consecutive starts each), keeping the prefix of y as
// wrapping 32-bit sums (a difference of two is the exact boxcar sum) in a
// shared-memory ring that holds the chunk, 16 samples before it and the
// widest boxcar after it.  Each chunk adds 2048 prefix entries, from loads
// issued while the previous chunk was tested, so every sample is loaded and
// summed once per segment.  A thread's first prefix index is a multiple of 16:
// for a width that is a multiple of 16 it reads the 16 sums it needs with four
// 16-byte loads (the 16-byte quarters of each 64-byte ring row are swizzled so
// that the 8 lanes of a quarter-warp hit distinct banks), widths of 1, 2, 4, 8
// come from its own registers, and a start costs one three-input add and half
// a three-input AND per width.  Widths that are multiples of 16 are first
// tested per group of 16 starts against an upper bound: with P the prefix,
// g = 16 starts from entry k, and M+ / M- the largest / smallest of
// P[j + i] - P[j] over i < 16 for the group at j (kept per group when the
// prefix is written),
//   max_i S_W(k + i) <= P[k + W] - P[k] + M+(k + W) - M-(k),
// so one add and a sign test clear the whole group and only groups whose bound
// reaches the threshold take the exact test.  The hot loop only notes that
// some start is above threshold; the rare warps with one find the run starts
// and follow each run (as detect_kernel), runs leaving the ring go to
// tail_kernel.
constexpr int kDWThreads = 128;
constexpr int kDWPer = 16;                          // consecutive starts per thread
constexpr int kDWChunk = kDWThreads * kDWPer;       // starts per chunk
constexpr int kDWLead = 16;                         // prefix entries before a segment's first start

// Exclusive prefix of v over the block's threads, and in *total the block's
// sum; one barrier: every warp adds up the warp totals before it itself.
__device__ __forceinline__ uint32_t block_exclusive_scan32(uint32_t v, uint32_t* warp_tot,
                                                           uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += u;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    uint32_t before = 0, all = 0;
#pragma unroll
    for (int i = 0; i < kDWThreads / 32; ++i) {
        const uint32_t t = warp_tot[i];
        before += i < warp ? t : 0u;
        all += t;
    }
    *total = all;
    return x - v + before;
}

// q[i] = the prefix entry W after p[i], for W up to 16: from this thread's own
// 16 entries p and the next 16, nx
template <int W>
__device__ __forceinline__ void shifted16(const uint32_t (&p)[16], const uint32_t (&nx)[16],
                                          uint32_t (&q)[16]) {
#pragma unroll
    for (int i = 0; i < 16; ++i) q[i] = i + W < 16 ? p[i + W] : nx[i + W - 16];
}

// The prefix ring: entry k at position k & mask; the 16-byte quarter of each
// 64-byte row is XOR-ed with bits 1-2 of the row index.
struct Ring {
    uint32_t* A;
    int mask;
    __device__ __forceinline__ static int swz(int r) { return r ^ (((r >> 5) & 3) << 2); }
    __device__ __forceinline__ uint32_t get(int64_t k) const { return A[swz((int)(k & mask))]; }
    // the 16 entries of the row at position r (a multiple of 16)
    __device__ __forceinline__ void get16(int r, uint32_t (&v)[16]) const {
        const int x = ((r >> 5) & 3) << 2;
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const uint4 u = *reinterpret_cast<const uint4*>(&A[r + ((4 * h) ^ x)]);
            v[4 * h] = u.x; v[4 * h + 1] = u.y; v[4 * h + 2] = u.z; v[4 * h + 3] = u.w;
        }
    }
    __device__ __forceinline__ void put16(int r, const uint32_t (&v)[16]) const {
        const int x = ((r >> 5) & 3) << 2;
#pragma unroll
        for (int h = 0; h < 4; ++h)
            *reinterpret_cast<uint4*>(&A[r + ((4 * h) ^ x)]) =
                make_uint4(v[4 * h], v[4 * h + 1], v[4 * h + 2], v[4 * h + 3]);
    }
};

__global__ void __launch_bounds__(kDWThreads) detect32_kernel(const __grid_constant__ SearchArgs a,
                                                              int64_t seg, int ring_words) {
    extern __shared__ __align__(16) uint32_t ring_mem[];
    __shared__ uint32_t warp_tot[32];
    __shared__ int32_t thr_s[kMaxWidths];           // INT32_MAX: this width finds nothing
    __shared__ int32_t width_s[kMaxWidths];
    __shared__ int2 wt_s[kMaxWidths];               // {W, threshold} of the widths that can fire:
    __shared__ int nlive, nexact;                   // [0, nexact) tested exactly, the rest by group bound
    __shared__ int32_t thr_p2[4];                   // widths 1, 2, 4, 8 (INT32_MAX: not searched)
    const int trial = blockIdx.y;
    if (!narrow_trial(a, trial)) return;             // detect_kernel takes the trial
    const int64_t n = a.nout;
    const int64_t S0 = (int64_t)blockIdx.x * seg;    // this block's starts [S0, S1)
    if (S0 >= n) return;
    const int64_t S1 = min(n, S0 + seg);
    const int64_t base = S0 - kDWLead;                // prefix entry k sums y over [base, base + k)
    const int32_t* yrow = a.Y + (int64_t)trial * a.ypitch;
    const bool vec = (a.ypitch & 3) == 0 && (reinterpret_cast<uintptr_t>(a.Y) & 15u) == 0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const Ring R{ring_mem, ring_words - 1};
    // per group of 16 ring entries: {P at its first entry, M+}, and M-
    uint2* gpm = reinterpret_cast<uint2*>(ring_mem + ring_words);
    int32_t* gmn = reinterpret_cast<int32_t*>(gpm + (ring_words >> 4));
    if (tid < a.nw) {
        const int64_t tk = a.tint[(int64_t)trial * a.nw + tid];
        thr_s[tid] = (int32_t)min(tk, (int64_t)INT32_MAX);
        width_s[tid] = a.widths[tid];
    }
    if (tid == 0) {
        // widths 1, 2, 4, 8 apart (tested from registers with fixed shifts), then
        // the other widths below 16 or not multiples of 16, then the multiples of 16
        for (int j = 0; j < 4; ++j) thr_p2[j] = INT32_MAX;
        int m = 0;
        for (int pass = 0; pass < 2; ++pass) {
            for (int k = 0; k < a.nw; ++k) {
                const int64_t tk = a.tint[(int64_t)trial * a.nw + k];
                const int W = a.widths[k];
                if (tk >= (int64_t)INT32_MAX) continue;
                const bool p2 = W == 1 || W == 2 || W == 4 || W == 8;
                if (pass == 0 && p2) thr_p2[31 - __clz(W)] = (int32_t)tk;
                else if (!p2 && ((W & 15) == 0) == (pass == 1)) wt_s[m++] = make_int2(W, (int)tk);
            }
            if (pass == 0) nexact = m;
        }
        nlive = m;
    }

    // y of the 16 samples before prefix entries f + 16 tid .. (0 outside the series)
    uint32_t v[16];
    auto load = [&](int64_t f) {
        const int64_t s0 = base + f + kDWPer * tid;
        if (vec && s0 >= 0 && s0 + 16 <= n) {
            const int4* q = reinterpret_cast<const int4*>(yrow + s0);
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int4 x = __ldg(q + h);
                v[4 * h] = x.x; v[4 * h + 1] = x.y; v[4 * h + 2] = x.z; v[4 * h + 3] = x.w;
            }
        } else {
#pragma unroll
            for (int e = 0; e < 16; ++e)
                v[e] = (s0 + e >= 0 && s0 + e < n) ? (uint32_t)__ldg(yrow + s0 + e) : 0u;
        }
    };
    // prefix entries f .. f + kDWChunk - 1 from the loaded v (synchronises)
    uint32_t carry = 0;
    auto put = [&](int64_t f) {
        uint32_t ex[16];
        uint32_t run = 0;
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            ex[e] = run;
            run += v[e];
        }
        // the group's M+ and M- (partial sums of at most 15 samples: exact int32)
        int32_t mx = 0, mn = 0;
#pragma unroll
        for (int e = 1; e < 16; e += 2) {
            const int32_t x0 = (int32_t)ex[e];
            const int32_t x1 = e + 1 < 16 ? (int32_t)ex[e + 1] : 0;
            mx = __vimax3_s32(mx, x0, x1);
            mn = __vimin3_s32(mn, x0, x1);
        }
        uint32_t chunk_total;
        const uint32_t off = carry + block_exclusive_scan32(run, warp_tot, &chunk_total);
#pragma unroll
        for (int e = 0; e < 16; ++e) ex[e] += off;
        const int pos = (int)((f + kDWPer * tid) & R.mask);
        R.put16(pos, ex);
        gpm[pos >> 4] = make_uint2(off, (uint32_t)mx);
        gmn[pos >> 4] = mn;
        carry += chunk_total;
        __syncthreads();   // ring entries visible; warp_tot free for the next scan
    };
    // entries [0, f0) before the first chunk: the chunk, the lead and the widest boxcar
    const int64_t f0 = (kDWLead + kDWChunk + (int64_t)a.wmax + 1 + kDWChunk - 1) / kDWChunk * kDWChunk;
    int64_t f = 0;
    for (; f < f0; f += kDWChunk) {
        load(f);
        put(f);
    }
    const int64_t nchunks = (S1 - S0 + kDWChunk - 1) / kDWChunk;
    if (nchunks > 1) load(f);                         // the next chunk's new samples, in flight
    const bool cin_any = a.carry_in && S0 == 0;

    for (int64_t c = 0; c < nchunks; ++c) {
        const int64_t t0 = S0 + c * kDWChunk;
        const int64_t kb = c * kDWChunk + kDWLead + kDWPer * tid;   // prefix index of start tb
        const int64_t tb = t0 + kDWPer * tid;                        // this thread's first start
        const int64_t tmax = S1 - 1;                                 // last start of the segment
        const int64_t len = min(f - 1, n - base);                    // highest prefix entry held
        const int pos0 = (int)(kb & R.mask);
        uint32_t p[16], nx[16];
        R.get16(pos0, p);
        R.get16((pos0 + 16) & R.mask, nx);
        // the prefix entry W after each of this thread's starts
        auto ahead = [&](int W, uint32_t (&q)[16]) {
            if ((W & 15) == 0) {
                R.get16((pos0 + W) & R.mask, q);
            } else if (W == 1) {
                shifted16<1>(p, nx, q);
            } else if (W == 2) {
                shifted16<2>(p, nx, q);
            } else if (W == 4) {
                shifted16<4>(p, nx, q);
            } else if (W == 8) {
                shifted16<8>(p, nx, q);
            } else {
#pragma unroll
                for (int i = 0; i < 16; ++i) q[i] = R.get(kb + W + i);
            }
        };
        // hot loop: does some width have an above-threshold start among this
        // thread's 16?  When the whole chunk is valid for every width, the AND
        // of S - thr over the starts has its sign bit clear iff some S >= thr (a
        // wrapped difference can only add a false alarm, which the exact pass
        // below clears); otherwise starts past the segment or the series are masked.
        uint32_t hit = 0;
        const bool full = t0 + kDWChunk - 1 <= tmax && t0 + kDWChunk - 1 <= n - a.wmax;
        if (full) {
            const int nl = nlive, ne = nexact;
            // widths 1, 2, 4, 8: the sums W ahead are this thread's own entries
            auto test_p2 = [&](auto wc) {
                constexpr int W = decltype(wc)::value;
                constexpr int j = W == 1 ? 0 : W == 2 ? 1 : W == 4 ? 2 : 3;
                const uint32_t thr = (uint32_t)thr_p2[j];
                if (thr == (uint32_t)INT32_MAX) return;
                uint32_t acc = 0xffffffffu;
#pragma unroll
                for (int i = 0; i < 16; i += 2) {
                    const uint32_t q0 = i + W < 16 ? p[i + W] : nx[i + W - 16];
                    const uint32_t q1 = i + 1 + W < 16 ? p[i + 1 + W] : nx[i + 1 + W - 16];
                    acc &= (q0 - p[i] - thr) & (q1 - p[i + 1] - thr);
                }
                if ((int32_t)acc >= 0) hit = 1u;
            };
            test_p2(std::integral_constant<int, 1>{});
            test_p2(std::integral_constant<int, 2>{});
            test_p2(std::integral_constant<int, 4>{});
            test_p2(std::integral_constant<int, 8>{});
            for (int k = 0; k < ne; ++k) {
                const int2 wt = wt_s[k];
                const uint32_t thr = (uint32_t)wt.y;
                uint32_t q[16];
                ahead(wt.x, q);
                uint32_t acc = 0xffffffffu;
#pragma unroll
                for (int i = 0; i < 16; i += 2)
                    acc &= (q[i] - p[i] - thr) & (q[i + 1] - p[i + 1] - thr);
                if ((int32_t)acc >= 0) hit = 1u;
            }
            // widths that are multiples of 16: the group bound first.  If a start
            // fires, bound - thr lies in [0, (W + 30) * |y| bound] < 2^31 (narrow
            // trial), so its sign bit is clear; a set sign bit clears the group.
            const uint32_t base0 = p[0] + (uint32_t)gmn[pos0 >> 4];
            for (int k = ne; k < nl; ++k) {
                const int2 wt = wt_s[k];
                const int r = (pos0 + wt.x) & R.mask;
                const uint2 g = gpm[r >> 4];
                if ((int32_t)(g.x + g.y - base0 - (uint32_t)wt.y) >= 0) {
                    const uint32_t thr = (uint32_t)wt.y;
                    uint32_t q[16];
                    R.get16(r, q);
                    uint32_t acc = 0xffffffffu;
#pragma unroll
                    for (int i = 0; i < 16; i += 2)
                        acc &= (q[i] - p[i] - thr) & (q[i + 1] - p[i + 1] - thr);
                    if ((int32_t)acc >= 0) hit = 1u;
                }
            }
            // the exact pass below wants the widths: find them on a hit (rare)
            if (hit) {
                hit = 0;
                for (int k = 0; k < a.nw; ++k) {
                    const int32_t thr = thr_s[k];
                    if (thr == INT32_MAX) continue;
                    uint32_t q[16];
                    ahead(width_s[k], q);
                    bool any = false;
#pragma unroll
                    for (int i = 0; i < 16; ++i) any |= (int32_t)(q[i] - p[i]) >= thr;
                    if (any) hit |= 1u << k;
                }
            }
        } else {
            for (int k = 0; k < a.nw; ++k) {
                const int32_t thr = thr_s[k];
                if (thr == INT32_MAX) continue;
                const int W = width_s[k];
                const int64_t lim = min(tmax, n - W) - tb;   // starts tb + i, i <= lim, are tested
                uint32_t q[16];
                ahead(W, q);
                bool any = false;
#pragma unroll
                for (int i = 0; i < 16; ++i) any |= i <= lim && (int32_t)(q[i] - p[i]) >= thr;
                if (any) hit |= 1u << k;
            }
        }

        // the block that holds start nwin - 1 reports the carry flags
        if (a.carry_out && tid == 0 && a.nwin - 1 >= t0 && a.nwin - 1 < t0 + kDWChunk &&
            a.nwin - 1 < S1) {
            const int64_t i = a.nwin - 1 - base;
            for (int k = 0; k < a.nw; ++k) {
                const int W = width_s[k];
                const bool above = thr_s[k] != INT32_MAX && a.nwin - 1 <= n - W &&
                                   (int32_t)(R.get(i + W) - R.get(i)) >= thr_s[k];
                a.carry_out[(int64_t)trial * a.nw + k] = above ? 1 : 0;
            }
        }

        if (__any_sync(0xffffffffu, hit != 0)) {
            // rare: run starts and runs of the widths some lane flagged
            unsigned todo = __reduce_or_sync(0xffffffffu, hit);
            while (todo) {
                const int k = __ffs(todo) - 1;
                todo &= todo - 1;
                const int32_t thr = thr_s[k];
                const int W = width_s[k];
                const int64_t last = n - W;
                const int64_t lim = min(tmax, last) - tb;
                uint32_t q[16];
                ahead(W, q);
                unsigned above = 0;
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (i <= lim && (int32_t)(q[i] - p[i]) >= thr) above |= 1u << i;
                // a start opens a run when the start before it is below threshold:
                // the previous lane's last start, or for lane 0 start tb - 1
                const unsigned prev = __shfl_up_sync(0xffffffffu, above, 1);
                bool left;
                if (lane > 0) {
                    left = (prev >> 15) & 1u;
                } else {
                    const int64_t tl = tb - 1;            // its prefix entry kb - 1 is held
                    left = tl >= 0 && tl <= last &&
                           (int32_t)(R.get(kb - 1 + W) - R.get(kb - 1)) >= thr;
                }
                unsigned starts = above & ~((above << 1) | (left ? 1u : 0u)) & 0xffffu;
                // streamed search: runs begin inside the window, and a run at start 0
                // that the previous gulp left open is not reported again
                if (a.nwin < tb + 16) starts &= a.nwin <= tb ? 0u : (1u << (int)(a.nwin - tb)) - 1u;
                if (cin_any && tb == 0 && a.carry_in[(int64_t)trial * a.nw + k]) starts &= ~1u;
                unsigned lanes = __ballot_sync(0xffffffffu, starts != 0);
                auto box32 = [&](int64_t u) {
                    const int64_t i = u - base;
                    return (int32_t)(R.get(i + W) - R.get(i));
                };
                while (lanes) {
                    const int L = __ffs(lanes) - 1;
                    lanes &= lanes - 1;
                    unsigned sL = __shfl_sync(0xffffffffu, starts, L);
                    const int64_t tL = t0 + (int64_t)kDWPer * (warp * 32 + L);
                    while (sL) {
                        const int e = __ffs(sL) - 1;
                        sL &= sL - 1;
                        int64_t bS, bt, tu = 0;
                        const bool tail = follow_run32(tL + e, last, base, len, (int64_t)W,
                                                       thr, box32, lane, &bS, &bt, &tu);
                        if (lane == 0) {
                            if (!tail) {
                                emit(a, trial, k, bt, bS);
                            } else {
                                const unsigned long long qi = atomicAdd(
                                    reinterpret_cast<unsigned long long*>(a.tail_count), 1ull);
                                if ((int64_t)qi < a.tail_cap) {
                                    TailRec r;
                                    r.trial = trial;
                                    r.k = k;
                                    r.u = tu;
                                    r.S_prev = box32(tu - 1);
                                    r.best_S = bS;
                                    r.best_t = bt;
                                    a.tails[qi] = r;
                                } else {
                                    latch_status(a.status, HP_ERR_CAND_OVERFLOW);
                                }
                            }
                        }
                    }
                }
            }
        }
        __syncthreads();                              // chunk c tested everywhere
        if (c + 1 < nchunks) {
            put(f);                                   // the samples loaded during chunk c
            f += kDWChunk;
            if (c + 2 < nchunks) load(f);             // in flight while chunk c + 1 is tested
        }
    }
}

// Runs that leave the detect tile's halo or the ring: continue each one from
// y in global memory, then emit it.  A warp per run, 128 starts per step (4
// consecutive per lane): S(v) = S(v - 1) - y(v - 1) + y(v - 1 + W), so the
// step's sums are S(u - 1) plus a lane-local then warp prefix sum of those
// differences; the run ends at the first start below threshold (or past the
// last start), and its candidate is the largest S before that (ties: the
// earliest start).
constexpr int kTailPer = 4;

__global__ void tail_kernel(const __grid_constant__ SearchArgs a) {
    const int64_t cnt = min(*a.tail_count, a.tail_cap);
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < cnt; q += warps) {
        const TailRec r = a.tails[q];
        const int64_t n = a.nout;
        const int32_t* yrow = a.Y + (int64_t)r.trial * a.ypitch;
        const int64_t W = a.widths[r.k];
        const int64_t last = n - W;
        const int64_t thr = a.tint[(int64_t)r.trial * a.nw + r.k];
        int64_t best_S = r.best_S, best_t = r.best_t, Sp = r.S_prev;
        for (int64_t v0 = r.u; v0 <= last; v0 += 32 * kTailPer) {
            const int64_t vb = v0 + kTailPer * lane;
            int64_t c[kTailPer];
            int64_t run = 0;
#pragma unroll
            for (int e = 0; e < kTailPer; ++e) {
                const int64_t v = vb + e;
                if (v <= last) run += (int64_t)__ldg(yrow + v - 1 + W) - (int64_t)__ldg(yrow + v - 1);
                c[e] = run;                                  // inclusive, lane-local
            }
            int64_t x = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t u = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += u;
            }
            const int64_t before = Sp + x - run;             // S(vb - 1)
            int lane_first = kTailPer;                       // first start below threshold
#pragma unroll
            for (int e = kTailPer - 1; e >= 0; --e)
                if (!(vb + e <= last && before + c[e] >= thr)) lane_first = e;
            const unsigned stop = __ballot_sync(0xffffffffu, lane_first < kTailPer);
            const int first_lane = stop ? __ffs(stop) - 1 : 32;
            const int lim = lane < first_lane ? kTailPer : (lane == first_lane ? lane_first : 0);
            int64_t cs = LLONG_MIN, ct = vb;
#pragma unroll
            for (int e = 0; e < kTailPer; ++e)
                if (e < lim && before + c[e] > cs) { cs = before + c[e]; ct = vb + e; }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const int64_t os = __shfl_down_sync(0xffffffffu, cs, o);
                const int64_t ot = __shfl_down_sync(0xffffffffu, ct, o);
                if (os > cs || (os == cs && ot < ct)) { cs = os; ct = ot; }
            }
            cs = __shfl_sync(0xffffffffu, cs, 0);
            ct = __shfl_sync(0xffffffffu, ct, 0);
            if (cs > best_S) { best_S = cs; best_t = ct; }
            if (stop) break;
            Sp += __shfl_sync(0xffffffffu, x, 31);
        }
        if (lane == 0) emit(a, r.trial, r.k, best_t, best_S);
    }
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ------------------------------------------------- per-width sigmas
// The lower median of |S_k(t)| over the starts 0 <= t <= n - W_k of every
// (trial, width), exact, by radix selection (WsigState).  Each histogram
// pass rebuilds the boxcar sums of a tile of up to 16384 starts (one block of
// 1024 threads) from a prefix of y over the tile and its halo in
// shared memory and counts one digit of every value still in the running,
// per width into one shared histogram.  The first pass counts v >> s0 below
// 4096 (and v >> (s0 + 12) above, up to 4095), with s0 chosen from the
// trial's MAD and sqrt(W) so that the values spread over ~1000 bins (few
// same-bin atomics) and narrow widths finish in that pass; later passes count
// the next (up to) 12 bits below the digits fixed so far.  A median in the
// last first-pass bin (values beyond what that pass resolves) restarts from
// the top digit of the 36-bit range.
constexpr int kWsigThreads = 1024;
constexpr int kWsigTileMax = 16384;   // starts per block (fewer when the halo is wide)
constexpr int kWsigBins = 2 * 4096;
constexpr int kWsigTop = 36;          // |S| < 2^36 (checked)
constexpr int kWsigPasses = 4;        // first pass + at most three 12-bit digits

__device__ __forceinline__ int wsig_bin(const WsigState& st, uint64_t v) {
    if (st.level == 1) {
        const uint64_t key = v >> st.shift;
        return key < 4096 ? (int)key : 4096 + (int)min(v >> (st.shift + 12), (uint64_t)4095);
    }
    if ((int64_t)(v >> st.shift) != st.prefix) return -1;
    const int d = min(12, st.shift);
    return (int)((v >> (st.shift - d)) & ((1u << d) - 1u));
}

__global__ void wsig_init_kernel(const __grid_constant__ SearchArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)a.ndm * a.nw) return;
    const int32_t W = a.widths[i % a.nw];
    const int64_t m = a.nout - W + 1;                     // starts
    // first-pass shift: log2 of the expected median, MAD * sqrt(W), less 9
    const int64_t mad = a.mad[i / a.nw];
    const int lm = 63 - __clzll((unsigned long long)max(mad, (int64_t)1));
    const int lw = (31 - __clz(W)) / 2;
    WsigState st;
    st.level = m > 0 ? 1 : 0;
    st.shift = min(max(lm + lw - 9, 0), kWsigTop - 12);
    st.prefix = 0;
    st.rank = m > 0 ? (m - 1) / 2 : 0;
    a.wstate[i] = st;
    if (m <= 0) a.wmad[i] = 0;
}

__global__ void __launch_bounds__(kWsigThreads) wsig_hist_kernel(const __grid_constant__ SearchArgs a,
                                                                 int level, int tile) {
    extern __shared__ int64_t P[];   // P[i] = sum of y over samples [t0, t0 + i)
    __shared__ uint32_t h[kWsigBins];
    __shared__ int64_t warp_tot[32];
    __shared__ int64_t warp_max[32];
    __shared__ int bin_lo, bin_hi;
    const int trial = blockIdx.y;
    const WsigState* st = a.wstate + (int64_t)trial * a.nw;
    bool any = false;
    for (int k = 0; k < a.nw; ++k) any = any || st[k].level == level;
    if (!any) return;                                     // the whole block
    const int64_t n = a.nout;
    const int64_t t0 = (int64_t)blockIdx.x * tile;
    const int len = (int)min((int64_t)tile + a.wmax - 1, n - t0);
    const int32_t* yrow = a.Y + (int64_t)trial * a.ypitch + t0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < len; i += blockDim.x) P[i + 1] = (int64_t)yrow[i];
    __syncthreads();
    const int per = ((len + (int)blockDim.x - 1) / (int)blockDim.x) | 1;
    const int i0 = min(len, tid * per), i1 = min(len, i0 + per);
    int64_t local = 0, ymax = 0;
    for (int i = i0; i < i1; ++i) {
        const int64_t y = P[i + 1];
        local += y;
        ymax = max(ymax, y < 0 ? -y : y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ymax = max(ymax, __shfl_xor_sync(0xffffffffu, ymax, o));
    if (lane == 0) warp_max[warp] = ymax;
    int64_t run = block_exclusive_scan(local, warp_tot);  // (synchronises)
    for (int i = i0; i < i1; ++i) {
        run += P[i + 1];
        P[i + 1] = run;
    }
    if (tid == 0) {
        P[0] = 0;
        bin_lo = kWsigBins;
        bin_hi = -1;
    }
    __syncthreads();
    int64_t tile_max = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tile_max = max(tile_max, warp_max[w]);
    // every boxcar sum of this tile fits int32: wrapped 32-bit differences of
    // the prefix's low words are exact
    const bool narrow = tile_max * (int64_t)a.wmax < (int64_t)INT32_MAX;
    const uint32_t* P32 = reinterpret_cast<const uint32_t*>(P);   // low word of P[i]: P32[2 i]
    for (int i = tid; i < kWsigBins; i += blockDim.x) h[i] = 0;
    for (int k = 0; k < a.nw; ++k) {
        const WsigState sk = st[k];
        if (sk.level != level) continue;                  // uniform over the block
        __syncthreads();
        const int W = a.widths[k];
        const int t_end = (int)min((int64_t)tile, n - W + 1 - t0);   // starts of this tile
        int lo = kWsigBins, hi = -1;
        bool big = false;
        if (narrow) {
            // every |S| < 2^31: the digit in 32-bit arithmetic (a shift of 31
            // or more leaves 0)
            const int sh = sk.shift;
            const uint32_t s1 = (uint32_t)min(sh, 31), s2 = (uint32_t)min(sh + 12, 31);
            const bool z1 = sh >= 31, z2 = sh + 12 >= 31;
            const int d = min(12, sh);
            const uint32_t s3 = (uint32_t)min(sh - d, 31);
            const bool z3 = sh - d >= 31;
            const uint32_t mask = (1u << d) - 1u;
            const bool reach = sk.prefix < ((int64_t)1 << 31);   // a 31-bit value can match
            const uint32_t pre = (uint32_t)sk.prefix;
            if (level == 1) {
                for (int t = tid; t < t_end; t += blockDim.x) {
                    const int32_t S = (int32_t)(P32[2 * (t + W)] - P32[2 * t]);
                    const uint32_t v = S < 0 ? 0u - (uint32_t)S : (uint32_t)S;
                    const uint32_t k1 = z1 ? 0u : v >> s1;
                    const int b = k1 < 4096u ? (int)k1 : 4096 + (int)min(z2 ? 0u : v >> s2, 4095u);
                    atomicAdd(&h[b], 1u);
                    lo = min(lo, b);
                    hi = max(hi, b);
                }
            } else if (reach) {
                for (int t = tid; t < t_end; t += blockDim.x) {
                    const int32_t S = (int32_t)(P32[2 * (t + W)] - P32[2 * t]);
                    const uint32_t v = S < 0 ? 0u - (uint32_t)S : (uint32_t)S;
                    if ((z1 ? 0u : v >> s1) == pre) {
                        const int b = (int)((z3 ? 0u : v >> s3) & mask);
                        atomicAdd(&h[b], 1u);
                        lo = min(lo, b);
                        hi = max(hi, b);
                    }
                }
            }
        } else {
            for (int t = tid; t < t_end; t += blockDim.x) {
                const int64_t S = P[t + W] - P[t];
                const uint64_t v = S < 0 ? (uint64_t)(-S) : (uint64_t)S;
                big = big || v >= ((uint64_t)1 << kWsigTop);
                const int b = wsig_bin(sk, v);
                if (b >= 0) {
                    atomicAdd(&h[b], 1u);
                    lo = min(lo, b);
                    hi = max(hi, b);
                }
            }
        }
        if (big) latch_status(a.status, HP_ERR_INVALID_ARG);   // |S| beyond the 36-bit range
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if (lane == 0 && hi >= 0) {
            atomicMin(&bin_lo, lo);
            atomicMax(&bin_hi, hi);
        }
        __syncthreads();
        const int b0 = bin_lo, b1 = bin_hi;
        __syncthreads();                                  // every thread has read the range
        if (tid == 0) {
            bin_lo = kWsigBins;
            bin_hi = -1;
        }
        // flush the touched bins and clear them for the next width
        uint32_t* g = a.whist + ((int64_t)trial * a.nw + k) * kWsigBins;
        for (int i = b0 + tid; i <= b1; i += blockDim.x) {
            const uint32_t c = h[i];
            if (c) {
                atomicAdd(&g[i], c);
                h[i] = 0;
            }
        }
    }
}

__global__ void __launch_bounds__(1024) wsig_select_kernel(const __grid_constant__ SearchArgs a,
                                                           int level) {
    const int64_t idx = blockIdx.x;                       // trial * nw + k
    WsigState st = a.wstate[idx];
    if (st.level != level) return;                        // the whole block
    uint32_t* hrow = a.whist + idx * kWsigBins;
    const int nbins = level == 1 ? kWsigBins : 1 << min(12, st.shift);
    int bin;
    int64_t before;
    find_rank_bin(hrow, nbins, st.rank, &bin, &before);
    if (threadIdx.x == 0) {
        if (level == 1 && bin == kWsigBins - 1) {
            // beyond what the first pass resolves: every digit from the top
            st.prefix = 0;
            st.shift = kWsigTop;
        } else if (level == 1) {
            st.prefix = bin < 4096 ? bin : bin - 4096;
            st.shift = bin < 4096 ? st.shift : st.shift + 12;
            st.rank -= before;
        } else {
            const int d = min(12, st.shift);
            st.prefix = (st.prefix << d) | bin;
            st.shift -= d;
            st.rank -= before;
        }
        st.level = level + 1;
        if (st.shift == 0) {
            a.wmad[idx] = st.prefix;
            st.level = 0;
        }
        a.wstate[idx] = st;
    }
    __syncthreads();
    if (a.wstate[idx].level != 0)   // the next pass counts into the first bins
        for (int i = threadIdx.x; i < 4096; i += blockDim.x) hrow[i] = 0;
}

// sigma_k and the integer thresholds ceil(thr * sigma_k)
__global__ void wsig_sigma_kernel(const __grid_constant__ SearchArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)a.ndm * a.nw) return;
    const double sg = __dmul_rn(kMadToSigma, (double)a.wmad[i]);
    a.sigw[i] = sg;
    a.tint[i] = sg > 0.0 ? (int64_t)ceil(__dmul_rn((double)a.thr, sg)) : kNever;
}

cudaError_t launch_width_sigma(const SearchArgs& a, cudaStream_t s, int64_t* nlaunch) {
    cudaError_t e;
    const int64_t pairs = (int64_t)a.ndm * a.nw;
    if ((e = cudaMemsetAsync(a.whist, 0, (size_t)pairs * kWsigBins * 4, s)) != cudaSuccess) return e;
    ++*nlaunch;
    wsig_init_kernel<<<(unsigned)ceil_div(pairs, 256), 256, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the widest tile whose prefix (tile + halo) fits beside the static arrays
    int tile = kWsigTileMax;
    while (tile > 1024 && ((size_t)tile + a.wmax + 1) * sizeof(int64_t) > (size_t)190 * 1024) tile /= 2;
    const size_t smem = ((size_t)tile + (size_t)a.wmax + 1) * sizeof(int64_t);
    if ((e = cudaFuncSetAttribute(wsig_hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
        return e;
    const dim3 hgrid((unsigned)ceil_div(a.nout, tile), a.ndm);
    for (int level = 1; level <= kWsigPasses; ++level) {
        ++*nlaunch;
        wsig_hist_kernel<<<hgrid, kWsigThreads, smem, s>>>(a, level, tile);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        ++*nlaunch;
        wsig_select_kernel<<<(unsigned)pairs, 1024, 0, s>>>(a, level);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    ++*nlaunch;
    wsig_sigma_kernel<<<(unsigned)ceil_div(pairs, 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}


// ------------------------------------------------- decimated boxcars
// Thresholds of the decimated widths move to their level's table (kNever in
// the every-start pass); level l takes the widths with W / decimate == dec_q[l]
// as boxcars of W / q samples on its scrunched series.
__global__ void decim_split_kernel(const __grid_constant__ SearchArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)a.ndm * a.nw) return;
    const int k = (int)(i % a.nw);
    const int32_t W = a.widths[k];
    const int32_t q = (W > a.decimate && W % a.decimate == 0) ? W / a.decimate : 1;
    const int64_t thr = a.tint[i];
    for (int l = 0; l < a.ndec; ++l) {
        a.tint_lv[(int64_t)l * a.ndm * a.nw + i] = q == a.dec_q[l] ? thr : kNever;
        if (i < a.nw) a.widths_lv[(int64_t)l * a.nw + k] = q == a.dec_q[l] ? W / q : 1;
    }
    if (q > 1) a.tint[i] = kNever;
}

// dst[d][m] = sum of src[d][m f .. m f + f), m < n_dst (int32: |y| < 2^21 and
// f * q <= 1024 keep the sums below 2^31)
__global__ void __launch_bounds__(256) scrunch_kernel(const int32_t* __restrict__ src,
                                                      int64_t src_pitch, int64_t n_src, int f,
                                                      int32_t* __restrict__ dst, int64_t dst_pitch,
                                                      int64_t n_dst) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int d = blockIdx.y;
    if (m >= n_dst || (m + 1) * f > n_src) return;
    const int32_t* r = src + (int64_t)d * src_pitch + m * f;
    int64_t acc = 0;
    for (int i = 0; i < f; ++i) acc += r[i];
    dst[(int64_t)d * dst_pitch + m] = (int32_t)acc;
}

cudaError_t launch_detect(const SearchArgs& a, cudaStream_t s, int64_t* nlaunch) {
    cudaError_t e;
    if (a.nout <= 0) return cudaSuccess;
    const size_t smem = ((size_t)kDetectTile + (size_t)a.wmax + 2) * sizeof(int64_t);
    if ((e = cudaFuncSetAttribute(detect_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
        return e;
    const dim3 dgrid((unsigned)std::min<int64_t>(ceil_div(a.nout, kDetectTile), kDetectBlocksPerTrial),
                     a.ndm);
    ++*nlaunch;
    detect_kernel<<<dgrid, kDetectThreads, smem, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the trials whose boxcar sums all fit int32 (nearly all): a block per
    // segment of a trial, about 10 000 blocks, at least 4 chunks per segment
    const int64_t f0 = ceil_div(kDWLead + kDWChunk + (int64_t)a.wmax + 1, kDWChunk) * kDWChunk;
    int ring = 64;
    while (ring < f0) ring <<= 1;
    // the ring, then per group of 16 entries {P, M+} and M-
    const size_t smem32 = (size_t)ring * sizeof(uint32_t) + (size_t)(ring / 16) * 12;
    if ((e = cudaFuncSetAttribute(detect32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem32)) != cudaSuccess)
        return e;
    const int64_t chunks = ceil_div(a.nout, kDWChunk);
    const int64_t nseg = std::max<int64_t>(1, std::min<int64_t>(ceil_div(10000, a.ndm), chunks / 4));
    const int64_t seg = ceil_div(chunks, nseg) * kDWChunk;
    const dim3 dgrid32((unsigned)ceil_div(a.nout, seg), a.ndm);
    ++*nlaunch;
    detect32_kernel<<<dgrid32, kDWThreads, smem32, s>>>(a, seg, ring);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ++*nlaunch;
    tail_kernel<<<2048, 128, 0, s>>>(a);   // a warp per run; idle warps leave at once
    return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_walkers(const SearchArgs& a, const BaselineCtx& bc, cudaStream_t s,
                           int64_t* nlaunch) {
    cudaError_t e;
    const int64_t n = a.nout;
    const int ndm = a.ndm;
    const dim3 hgrid((unsigned)ceil_div(n, kHistChunk), ndm);
    const int vec = ((a.pitch & 3) == 0) && (((uintptr_t)a.D & 15u) == 0);
    const int yvec = ((a.ypitch & 3) == 0) && (((uintptr_t)a.Y & 15u) == 0);
    ++*nlaunch;
    mad_hist_kernel<MODE><<<dim3((unsigned)ceil_div(n, kHistBlock), ndm), kHistThreads, 0, s>>>(
        a.D, a.pitch, n, bc, vec, a.hist, a.Y, a.ypitch, yvec);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ++*nlaunch;
    mad_select_kernel<<<ndm, 1024, 0, s>>>(a.hist, n, a.refine_bucket, a.refine_rank, a.mad,
                                           a.ybound);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ++*nlaunch;
    mad_refine_hist_kernel<<<hgrid, 256, 0, s>>>(a.Y, a.ypitch, n, yvec, a.refine_bucket, a.hist);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ++*nlaunch;
    mad_refine_select_kernel<<<ndm, 1024, 0, s>>>(a.hist, a.refine_bucket, a.refine_rank, a.mad);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ++*nlaunch;
    sigma_kernel<<<(unsigned)ceil_div(ndm, 128), 128, 0, s>>>(a.mad, ndm, a.widths, a.nw, a.thr,
                                                              a.sigma, a.tint);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (a.stats_only) return cudaSuccess;
    if (a.width_sigma && (e = launch_width_sigma(a, s, nlaunch)) != cudaSuccess) return e;
    if (a.ndec > 0) {
        // the decimated widths leave the every-start pass for their own levels
        ++*nlaunch;
        decim_split_kernel<<<(unsigned)ceil_div((int64_t)ndm * a.nw, 256), 256, 0, s>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = launch_detect(a, s, nlaunch)) != cudaSuccess) return e;
    for (int l = 0; l < a.ndec; ++l) {
        // series summed in blocks of q, from the previous level when q divides
        const int q = a.dec_q[l];
        const int qp = l > 0 && q % a.dec_q[l - 1] == 0 ? a.dec_q[l - 1] : 1;
        const int32_t* src = qp > 1 ? a.ydec + a.dec_off[l - 1] : a.Y;
        const int64_t src_pitch = qp > 1 ? a.dec_pitch[l - 1] : a.ypitch;
        const int64_t n_src = n / qp, n_l = n / q;
        ++*nlaunch;
        scrunch_kernel<<<dim3((unsigned)ceil_div(n_l, 256), ndm), 256, 0, s>>>(
            src, src_pitch, n_src, q / qp, a.ydec + a.dec_off[l], a.dec_pitch[l], n_l);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        SearchArgs al = a;
        al.Y = a.ydec + a.dec_off[l];
        al.ypitch = a.dec_pitch[l];
        al.nout = n_l;
        al.nwin = n_l;
        al.widths = a.widths_lv + (int64_t)l * a.nw;
        al.wmax = a.decimate;
        al.tint = a.tint_lv + (int64_t)l * ndm * a.nw;
        al.sample_mul = q;
        al.carry_in = nullptr;
        al.carry_out = nullptr;
        if ((e = cudaMemsetAsync(a.tail_count, 0, sizeof(int64_t), s)) != cudaSuccess) return e;
        if ((e = launch_detect(al, s, nlaunch)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_search(const SearchArgs& a, cudaStream_t s, int64_t* nlaunch) {
    cudaError_t e;
    const int64_t n = a.nout;
    const int ndm = a.ndm;
    if (ndm <= 0 || n <= 0) return cudaSuccess;
    if (!a.stats_only) {
        if ((e = cudaMemsetAsync(a.raw_count, 0, sizeof(int64_t), s)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(a.tail_count, 0, sizeof(int64_t), s)) != cudaSuccess) return e;
    }
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
            int left = L;
            if (a.lv2 != nullptr && L >= 2) {
                // the dedispersion formed the second level of every group inside
                // one of its time tiles; the straddling groups come from D
                const int64_t ntt = ceil_div(n, a.lv2_bt);
                ++*nlaunch;
                level2_fixup_kernel<<<dim3((unsigned)ceil_div(ntt + 1, 128), ndm), 128, 0, s>>>(
                    a.D, a.pitch, n, a.lv2_bt, a.lv2, a.lv2_pitch);
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
                in = a.lv2;
                in_pitch = a.lv2_pitch;
                n_in = ceil_div(n, 25);
                left = L - 2;
            }
            int32_t* bufs[2] = {a.lvl_a, a.lvl_b};
            const int64_t pitches[2] = {a.lvl_pitch_a, a.lvl_pitch_b};
            int which = 0;
            while (left > 0) {
                const int q = left < 5 ? left : 5;
                int64_t chunk = 1;
                for (int l = 0; l < q; ++l) chunk *= 5;
                const int64_t n_out = ceil_div(n_in, chunk);
                int32_t* out = bufs[which];
                const int64_t out_pitch = which == 0 ? pitches[0] : pitches[1];
                if (n_out > out_pitch) return cudaErrorInvalidValue;
                ++*nlaunch;
                const int64_t gx = ceil_div(n_out, kRemChunksPerBlock);
                remedian_pass_kernel<<<dim3((unsigned)gx, ndm), kRemThreads, 0, s>>>(
                    in, in_pitch, n_in, q, out, out_pitch, n_out);
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

    if (a.baseline_mode != 0) return launch_walkers<1>(a, bc, s, nlaunch);
    return bc.P < ((int64_t)1 << 30) ? launch_walkers<0>(a, bc, s, nlaunch)
                                     : launch_walkers<2>(a, bc, s, nlaunch);
}

}  // namespace hp
