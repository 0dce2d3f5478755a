// Top-k compression codec of Sec. 4.1.5 (its classical steps): the spectrum
// c = G_N x, the k coefficients of largest magnitude of every vector (as
// (index, value) pairs, ordered by |c| descending and, between equal
// magnitudes, by the larger index first), and the reconstruction
// G_N^dagger of the spectrum that holds only those pairs.
//
// Selection: every coefficient gets the composite key (|c|^2 bits, index).
// |c|^2 >= 0, so its IEEE bit pattern orders like the value; the index makes
// every key distinct and ranks equal magnitudes by the larger index.  A radix
// select over 8-bit digits of the composite key, most significant first,
// finds for every vector the smallest key T among its k largest: each pass
// histograms the digit of the keys that still match the chosen prefix and
// picks the digit at which the count from the top reaches the number still
// needed.  A vector is finished once the chosen bucket holds exactly that
// number (T's lower bits are then zero), at the latest after the last digit.
// The coefficients with key >= T are collected (exactly k), one CTA per
// vector sorts them by key descending, and the values are gathered.
// Before the radix passes, one pass over the spectrum histograms the top 12
// bits of the keys and collects every coefficient whose top bits reach an
// estimated bucket: the bucket that a sample of every 32nd coefficient puts
// a little below the k-th largest key.  The exact histogram then shows
// whether the estimate was low enough (the bucket of the k-th largest key is
// not below it); if not, a second pass collects from that exact bucket.
// Either way the list contains all the k largest keys, typically a few
// times k long.  The radix passes and the final
// collection then read the candidates instead of the spectrum.  A vector whose
// candidates exceed the list's capacity (many equal magnitudes) keeps reading
// its spectrum; the result is the same either way.
// |c|^2 is formed with explicit round-to-nearest products and sum (no fused
// multiply-add), so the decision can be reproduced in the same precision.
#include <algorithm>
#include <cmath>

#include "gtt_plan.h"
#include "gtt_sparse.cuh"
#include "gtt_types.cuh"

namespace gtt {

constexpr int kTopkMax = 4096;   // k per vector (one CTA sorts them in shared memory)
constexpr int kTopkSortThreads = 1024;
constexpr int kTopkBins = 4096;           // buckets of the pre-pass: the top 12 bits of the key
constexpr uint32_t kTopkCandCap = 65536;  // candidate list capacity per vector
constexpr int kTopkSample = 32;           // the threshold estimate samples one coefficient in 32:
constexpr int kTopkSampleRun = 32;        // runs of 32 consecutive ones, every 1024

template <typename T> struct KeyOf;
template <> struct KeyOf<float> {
    using K = uint32_t;
    static __device__ __forceinline__ K key(float v) { return __float_as_uint(__fmul_rn(v, v)); }
};
template <> struct KeyOf<c64> {
    using K = uint32_t;
    static __device__ __forceinline__ K key(c64 v) {
        return __float_as_uint(__fadd_rn(__fmul_rn(v.re, v.re), __fmul_rn(v.im, v.im)));
    }
};
template <> struct KeyOf<double> {
    using K = unsigned long long;
    static __device__ __forceinline__ K key(double v) { return (K)__double_as_longlong(__dmul_rn(v, v)); }
};
template <> struct KeyOf<c128> {
    using K = unsigned long long;
    static __device__ __forceinline__ K key(c128 v) {
        return (K)__double_as_longlong(__dadd_rn(__dmul_rn(v.re, v.re), __dmul_rn(v.im, v.im)));
    }
};

struct TopkState {
    unsigned long long key_prefix;  // chosen key bits (lower bits zero)
    uint32_t idx_prefix;            // chosen index bits (lower bits zero)
    uint32_t need;                  // how many keys of the current bucket are still to be taken
    uint32_t done;                  // 1: the threshold T = (key_prefix, idx_prefix) is final
    uint32_t count;                 // keys collected so far
    uint32_t fast;                  // 1: selected from a short candidate list by one sort
};

// Digit `pass` of the composite key: the key's KB bits (KB / 8 digits), then
// the index's 32 bits (4 digits), most significant first.  match: the key's
// bits above the digit equal the prefix chosen so far.
template <typename K>
__device__ __forceinline__ bool digit_of(K key, uint32_t idx, int pass, const TopkState &st, uint32_t *d) {
    constexpr int KB = 8 * (int)sizeof(K), KD = KB / 8;
    if (pass < KD) {
        const int shift = KB - 8 * (pass + 1);
        const K mask = pass == 0 ? (K)0 : (K)(~(K)0) << (KB - 8 * pass);
        if ((key & mask) != (K)st.key_prefix) return false;
        *d = (uint32_t)(key >> shift) & 255u;
        return true;
    }
    const int q = pass - KD;
    if (key != (K)st.key_prefix) return false;
    const uint32_t mask = q == 0 ? 0u : ~0u << (32 - 8 * q);
    if ((idx & mask) != st.idx_prefix) return false;
    *d = (idx >> (24 - 8 * q)) & 255u;
    return true;
}

// fn(element, index) over this CTA's share of one vector (grid-stride over
// blockIdx.x): 16-byte loads when the vector is a whole number of 16-byte
// chunks (so every vector of the batch starts on a 16-byte boundary), else
// one element at a time.
template <typename T, typename F>
__device__ __forceinline__ void topk_for_each(const T *v, long long N, F fn) {
    constexpr int CE = 16 / (int)sizeof(T);
    const long long stride = (long long)gridDim.x * blockDim.x;
    if (N % CE == 0) {
        const int4 *v4 = reinterpret_cast<const int4 *>(v);
        const long long nch = N / CE;
#pragma unroll 2
        for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nch; c += stride) {
            const int4 raw = v4[c];
            const T *x = reinterpret_cast<const T *>(&raw);
#pragma unroll
            for (int i = 0; i < CE; ++i) fn(x[i], c * CE + i);
        }
    } else {
        for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += stride) fn(v[e], e);
    }
}

// Estimate pass: histogram of the top 12 key bits of a sample of vector
// blockIdx.y, runs of kTopkSampleRun consecutive coefficients (whole cache
// lines for a warp) every kTopkSample * kTopkSampleRun.
template <typename T>
__global__ void __launch_bounds__(256) gtt_topk_sample_kernel(const T *spec, long long N, uint32_t *sbins) {
    using K = typename KeyOf<T>::K;
    constexpr int SH = 8 * (int)sizeof(K) - 12;
    constexpr long long kPeriod = (long long)kTopkSample * kTopkSampleRun;
    __shared__ uint32_t h[kTopkBins];
    for (int i = threadIdx.x; i < kTopkBins; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const long long item = blockIdx.y, ns = (N + kPeriod - 1) / kPeriod * kTopkSampleRun;
    const T *v = spec + item * N;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < ns; j += (long long)gridDim.x * blockDim.x) {
        const long long e = (j / kTopkSampleRun) * kPeriod + j % kTopkSampleRun;
        if (e < N) atomicAdd(&h[(uint32_t)(KeyOf<T>::key(v[e]) >> SH)], 1u);
    }
    __syncthreads();
    uint32_t *g = sbins + item * kTopkBins;
    for (int i = threadIdx.x; i < kTopkBins; i += blockDim.x)
        if (h[i]) atomicAdd(&g[i], h[i]);
}

// The bucket of vector blockIdx.x that holds its k-th largest key (the
// counts of the buckets from the top reach k there).  With est (the exact
// histogram after an estimated collection): redo = the exact bucket lies
// below the estimate, and the vector's candidate count restarts at 0 for the
// collection from the exact bucket.
__global__ void __launch_bounds__(256) gtt_topk_binscan_kernel(long long k, const uint32_t *bins, uint32_t *thr,
                                                               const uint32_t *est, uint32_t *cand_n,
                                                               uint32_t *redo) {
    constexpr int PER = kTopkBins / 256;
    const long long item = blockIdx.x;
    const uint32_t *g = bins + item * kTopkBins;
    const uint32_t tid = threadIdx.x;
    const unsigned long long kk = (unsigned long long)k;
    __shared__ uint32_t h[kTopkBins];
    __shared__ unsigned long long suf[256];
    for (int i = tid; i < kTopkBins; i += 256) h[i] = g[i];
    __syncthreads();
    uint32_t sum = 0;
    for (int i = 0; i < PER; ++i) sum += h[tid * PER + i];
    suf[tid] = sum;
    __syncthreads();
    // suf[c] = count of the keys in chunks c .. 255 (a suffix sum in 8 steps)
    for (int d = 1; d < 256; d <<= 1) {
        const unsigned long long add = tid + d < 256u ? suf[tid + d] : 0ull;
        __syncthreads();
        suf[tid] += add;
        __syncthreads();
    }
    // the chunk where the count from the top reaches k (one thread), or chunk 0
    // with bucket 0 when the vector holds fewer keys than k
    const unsigned long long above_chunk = tid < 255u ? suf[tid + 1] : 0ull;
    const bool mine = (suf[tid] >= kk && above_chunk < kk) || (tid == 0 && suf[0] < kk);
    if (mine) {
        unsigned long long above = above_chunk;
        int bin = (int)tid * PER;
        for (int b = (int)tid * PER + PER - 1; b >= (int)tid * PER && suf[0] >= kk; --b) {
            if (above + h[b] >= kk) {
                bin = b;
                break;
            }
            above += h[b];
        }
        thr[item] = (uint32_t)bin;
        if (est) {
            const bool again = (uint32_t)bin < est[item];
            redo[item] = again ? 1u : 0u;
            if (again) cand_n[item] = 0u;
        }
    }
}

// Pre-pass 2: the candidates of vector blockIdx.y, every coefficient whose
// top 12 key bits reach its threshold bucket (cand_n counts them all; at most
// cap are stored).
// With bins: also the exact histogram of the top 12 key bits (the estimated
// collection).  With redo: only the vectors whose estimate was too high.
template <typename T>
__global__ void __launch_bounds__(256) gtt_topk_cand_kernel(const T *spec, long long N, const uint32_t *thr,
                                                            uint32_t cap, uint32_t *cand_n,
                                                            typename KeyOf<T>::K *cand_key, uint32_t *cand_idx,
                                                            uint32_t *bins, const uint32_t *redo) {
    using K = typename KeyOf<T>::K;
    constexpr int SH = 8 * (int)sizeof(K) - 12;
    __shared__ uint32_t h[kTopkBins];
    const long long item = blockIdx.y;
    if (redo && !redo[item]) return;  // uniform over the CTA
    if (bins) {
        for (int i = threadIdx.x; i < kTopkBins; i += blockDim.x) h[i] = 0;
        __syncthreads();
    }
    const uint32_t tb = thr[item];
    const T *v = spec + item * N;
    topk_for_each<T>(v, N, [&](const T &x, long long e) {
        const K key = KeyOf<T>::key(x);
        if (bins) atomicAdd(&h[(uint32_t)(key >> SH)], 1u);
        if ((uint32_t)(key >> SH) >= tb) {
            const uint32_t slot = atomicAdd(&cand_n[item], 1u);
            if (slot < cap) {
                cand_key[item * cap + slot] = key;
                cand_idx[item * cap + slot] = (uint32_t)e;
            }
        }
    });
    if (bins) {
        __syncthreads();
        uint32_t *g = bins + item * kTopkBins;
        for (int i = threadIdx.x; i < kTopkBins; i += blockDim.x)
            if (h[i]) atomicAdd(&g[i], h[i]);
    }
}

// Histogram of digit `pass` over the matching keys of vector blockIdx.y.
// The scan of digit `pass` for one vector: pick the digit whose bucket holds
// the threshold, update the state, clear the histogram.  Run by thread 0.
template <typename K>
__device__ void topk_scan_digit(int pass, TopkState *state, uint32_t *h) {
    constexpr int KB = 8 * (int)sizeof(K), KD = KB / 8;
    TopkState st = *state;
    uint32_t above = 0;
    for (int d = 255; d >= 0; --d) {
        const uint32_t c = __ldcg(&h[d]);
        if (above + c >= st.need) {  // the threshold lies in bucket d
            if (pass < KD)
                st.key_prefix |= (unsigned long long)d << (KB - 8 * (pass + 1));
            else
                st.idx_prefix |= (uint32_t)d << (24 - 8 * (pass - KD));
            st.need -= above;
            if (c == st.need) st.done = 1u;  // the whole bucket is taken
            break;
        }
        above += c;
    }
    *state = st;
}

// Histogram of digit `pass` over the matching keys of vector blockIdx.y; the
// CTA of the vector that finishes last picks the digit (topk_scan_digit) and
// clears the histogram and its arrival count for the next pass.  The keys
// come from the vector's candidates when they all fit the list (cand_n <=
// cap), else from its spectrum.
template <typename T>
__global__ void __launch_bounds__(256) gtt_topk_hist_kernel(const T *spec, long long N, int pass,
                                                            TopkState *state, uint32_t *hist, uint32_t *arrive,
                                                            uint32_t cap, const uint32_t *cand_n,
                                                            const typename KeyOf<T>::K *cand_key,
                                                            const uint32_t *cand_idx) {
    using K = typename KeyOf<T>::K;
    const long long item = blockIdx.y;
    const TopkState st = state[item];
    if (st.done) return;
    __shared__ uint32_t h[256];
    __shared__ bool last;
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t nc = cand_n[item];
    if (nc <= cap) {
        const K *ck = cand_key + item * cap;
        const uint32_t *ci = cand_idx + item * cap;
        for (long long e = blockIdx.x * 256ll + threadIdx.x; e < nc; e += (long long)gridDim.x * 256) {
            uint32_t d;
            if (digit_of<K>(ck[e], ci[e], pass, st, &d)) atomicAdd(&h[d], 1u);
        }
    } else {
        const T *v = spec + item * N;
        for (long long e = blockIdx.x * 256ll + threadIdx.x; e < N; e += (long long)gridDim.x * 256) {
            uint32_t d;
            if (digit_of<K>(KeyOf<T>::key(v[e]), (uint32_t)e, pass, st, &d)) atomicAdd(&h[d], 1u);
        }
    }
    __syncthreads();
    uint32_t *g = hist + item * 256;
    if (h[threadIdx.x]) atomicAdd(&g[threadIdx.x], h[threadIdx.x]);
    __threadfence();  // this CTA's counts before its arrival
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&arrive[item], 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();  // every CTA's counts are in
    if (threadIdx.x == 0) {
        topk_scan_digit<K>(pass, &state[item], g);
        arrive[item] = 0u;
    }
    __syncthreads();
    g[threadIdx.x] = 0u;
}

// Collect the keys >= T of vector blockIdx.y (exactly k of them).
template <typename T>
__global__ void __launch_bounds__(256) gtt_topk_collect_kernel(const T *spec, long long N, long long k,
                                                               TopkState *state,
                                                               typename KeyOf<T>::K *sel_key, uint32_t *sel_idx,
                                                               uint32_t cap, const uint32_t *cand_n,
                                                               const typename KeyOf<T>::K *cand_key,
                                                               const uint32_t *cand_idx) {
    using K = typename KeyOf<T>::K;
    const long long item = blockIdx.y;
    if (state[item].fast) return;
    const K tk = (K)state[item].key_prefix;
    const uint32_t ti = state[item].idx_prefix;
    auto take = [&](K key, uint32_t idx) {
        if (key > tk || (key == tk && idx >= ti)) {
            const uint32_t slot = atomicAdd(&state[item].count, 1u);
            if (slot < (uint32_t)k) {
                sel_key[item * k + slot] = key;
                sel_idx[item * k + slot] = idx;
            }
        }
    };
    const uint32_t nc = cand_n[item];
    if (nc <= cap) {
        for (long long e = blockIdx.x * 256ll + threadIdx.x; e < nc; e += (long long)gridDim.x * 256)
            take(cand_key[item * cap + e], cand_idx[item * cap + e]);
    } else {
        const T *v = spec + item * N;
        for (long long e = blockIdx.x * 256ll + threadIdx.x; e < N; e += (long long)gridDim.x * 256)
            take(KeyOf<T>::key(v[e]), (uint32_t)e);
    }
}

// Bitonic sort of the P2 (a power of two) pairs (sk, si) in shared memory
// into output order: entries with a real index first, then key descending,
// then index descending (padding entries carry index kTopkPad).  When P2 equals
// the size of the last merge, that merge runs in output order over the whole
// array.
constexpr uint32_t kTopkPad = 0xFFFFFFFFu;  // index of a padding entry (real indices are < 2^32 - 1)
template <typename K> __device__ void topk_bitonic(K *sk, uint32_t *si, int P2) {
    auto before = [&](int a, int b) {
        const bool va = si[a] != kTopkPad, vb = si[b] != kTopkPad;
        if (va != vb) return va;
        if (sk[a] != sk[b]) return sk[a] > sk[b];
        return si[a] > si[b];
    };
    for (int size = 2; size <= P2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < P2; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool desc = (i & size) == 0;  // this run sorts in output order
                    if (desc ? before(j, i) : before(i, j)) {
                        const K tk = sk[i];
                        sk[i] = sk[j];
                        sk[j] = tk;
                        const uint32_t ti = si[i];
                        si[i] = si[j];
                        si[j] = ti;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Sort the k collected (key, index) pairs of vector blockIdx.x and write the
// indices and the gathered values (vectors selected by the fast sort are done).
template <typename T>
__global__ void __launch_bounds__(kTopkSortThreads) gtt_topk_sort_kernel(const T *spec, long long N, long long k,
                                                                         const typename KeyOf<T>::K *sel_key,
                                                                         const uint32_t *sel_idx, long long *out_idx,
                                                                         T *out_val, const TopkState *state) {
    using K = typename KeyOf<T>::K;
    __shared__ K sk[kTopkMax];
    __shared__ uint32_t si[kTopkMax];
    const long long item = blockIdx.x;
    if (state[item].fast) return;
    int P2 = 1;
    while (P2 < k) P2 <<= 1;
    for (int i = threadIdx.x; i < P2; i += blockDim.x) {
        const bool ok = i < k;
        sk[i] = ok ? sel_key[item * k + i] : (K)0;
        si[i] = ok ? sel_idx[item * k + i] : kTopkPad;
    }
    __syncthreads();
    topk_bitonic<K>(sk, si, P2);
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        out_idx[item * k + i] = (long long)si[i];
        out_val[item * k + i] = spec[item * N + si[i]];
    }
}

// A vector whose candidate list holds at most kTopkMax entries: sort the whole
// list in one CTA, write its first k entries and mark the vector done, so the
// radix passes, the collection and the sort above pass it by.
// The list may be longer (an estimated collection): only the candidates in
// or above the exact bucket of the k-th largest key (thr) take part, as long
// as they fit.
template <typename T>
__global__ void __launch_bounds__(kTopkSortThreads) gtt_topk_fastsort_kernel(const T *spec, long long N, long long k,
                                                                             uint32_t cap, const uint32_t *cand_n,
                                                                             const typename KeyOf<T>::K *cand_key,
                                                                             const uint32_t *cand_idx,
                                                                             long long *out_idx, T *out_val,
                                                                             TopkState *state, const uint32_t *thr) {
    using K = typename KeyOf<T>::K;
    constexpr int SH = 8 * (int)sizeof(K) - 12;
    __shared__ K sk[kTopkMax];
    __shared__ uint32_t si[kTopkMax];
    __shared__ uint32_t s_n;
    const long long item = blockIdx.x;
    const uint32_t nc = cand_n[item];
    if (nc > cap) return;  // the radix passes select this vector (uniform over the CTA)
    const uint32_t tb = thr[item];
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nc; i += blockDim.x) {
        const K key = cand_key[item * cap + i];
        if ((uint32_t)(key >> SH) >= tb) {
            const uint32_t slot = atomicAdd(&s_n, 1u);
            if (slot < (uint32_t)kTopkMax) {
                sk[slot] = key;
                si[slot] = cand_idx[item * cap + i];
            }
        }
    }
    __syncthreads();
    const uint32_t m = s_n;
    if (m > (uint32_t)kTopkMax) return;  // too many in the exact bucket: the radix passes (uniform)
    int P2 = 1;
    while (P2 < (int)m) P2 <<= 1;
    for (int i = (int)m + threadIdx.x; i < P2; i += blockDim.x) {
        sk[i] = (K)0;
        si[i] = kTopkPad;
    }
    __syncthreads();
    topk_bitonic<K>(sk, si, P2);
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        out_idx[item * k + i] = (long long)si[i];
        out_val[item * k + i] = spec[item * N + si[i]];
    }
    if (threadIdx.x == 0) {
        state[item].done = 1u;
        state[item].fast = 1u;
    }
}

// y[item][idx[item][j]] = val[item][j] (y zeroed beforehand).
template <typename T>
__global__ void __launch_bounds__(256) gtt_topk_scatter_kernel(const long long *idx, const T *val, long long k,
                                                               long long items, long long N, T *y) {
    const long long total = items * k;
    for (long long u = blockIdx.x * 256ll + threadIdx.x; u < total; u += (long long)gridDim.x * 256) {
        const long long item = u / k, i = idx[u];
        if (i >= 0 && i < N) y[item * N + i] = val[u];  // indices outside [0, N) are skipped
    }
}

template <typename T> struct TopkKernels {
    static const void *sample() { return (const void *)&gtt_topk_sample_kernel<T>; }
    static const void *cand() { return (const void *)&gtt_topk_cand_kernel<T>; }
    static const void *hist() { return (const void *)&gtt_topk_hist_kernel<T>; }
    static const void *collect() { return (const void *)&gtt_topk_collect_kernel<T>; }
    static const void *sort() { return (const void *)&gtt_topk_sort_kernel<T>; }
    static const void *fastsort() { return (const void *)&gtt_topk_fastsort_kernel<T>; }
    static const void *scatter() { return (const void *)&gtt_topk_scatter_kernel<T>; }
    static constexpr int key_bytes = (int)sizeof(typename KeyOf<T>::K);
};

template <typename T>
static gtt_status_t topk_select(gtt_plan_s *P, const void *spec, long long k, long long *out_idx, void *out_val,
                                cudaStream_t s) {
    using TK = TopkKernels<T>;
    const long long B = P->batch, N = P->N;
    const int KB = TK::key_bytes;
    // the candidate pre-passes pay off on long vectors; shorter ones run the
    // radix passes on the spectrum directly
    const bool use_cand = N >= 16ll * kTopkCandCap;
    const uint32_t cap = use_cand ? kTopkCandCap : 0u;
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    // workspace: states, radix histograms, collected keys and indices, candidate
    // counts; with the pre-passes also bucket counts, thresholds and the lists
    const size_t st_bytes = al((size_t)B * sizeof(TopkState));
    const size_t h_bytes = al((size_t)B * 256 * sizeof(uint32_t));
    const size_t key_bytes = al((size_t)B * k * KB);
    const size_t sidx_bytes = al((size_t)B * k * sizeof(uint32_t));
    const size_t cn_bytes = al((size_t)B * sizeof(uint32_t));
    const size_t ar_bytes = al((size_t)B * sizeof(uint32_t));
    const size_t bins_bytes = use_cand ? al((size_t)B * kTopkBins * sizeof(uint32_t)) : 0;  // sample, then exact
    const size_t thr_bytes = use_cand ? al((size_t)B * sizeof(uint32_t)) : 0;               // estimate, exact, redo
    const size_t ckey_bytes = use_cand ? al((size_t)B * cap * KB) : 0;
    const size_t cidx_bytes = use_cand ? al((size_t)B * cap * sizeof(uint32_t)) : 0;
    const size_t need =
        st_bytes + h_bytes + key_bytes + sidx_bytes + cn_bytes + ar_bytes + 2 * bins_bytes + 3 * thr_bytes +
        ckey_bytes + cidx_bytes;
    if (P->ws_topk_bytes < need) {
        if (P->ws_topk) cudaFree(P->ws_topk);
        P->ws_topk = nullptr;
        P->ws_topk_bytes = 0;
        cudaError_t e = cudaMalloc(&P->ws_topk, need);
        if (e != cudaSuccess) {
            P->ws_topk = nullptr;
            return set_error(GTT_ERR_ALLOC, std::string("top-k workspace: ") + cudaGetErrorString(e));
        }
        P->ws_topk_bytes = need;
    }
    unsigned char *w = static_cast<unsigned char *>(P->ws_topk);
    TopkState *state = reinterpret_cast<TopkState *>(w);
    w += st_bytes;
    uint32_t *hist = reinterpret_cast<uint32_t *>(w);
    w += h_bytes;
    void *sel_key = w;
    w += key_bytes;
    uint32_t *sel_idx = reinterpret_cast<uint32_t *>(w);
    w += sidx_bytes;
    uint32_t *cand_n = reinterpret_cast<uint32_t *>(w);
    w += cn_bytes;
    uint32_t *arrive = reinterpret_cast<uint32_t *>(w);  // CTAs of a vector done with the current digit
    w += ar_bytes;
    uint32_t *sbins = reinterpret_cast<uint32_t *>(w);
    w += bins_bytes;
    uint32_t *bins = reinterpret_cast<uint32_t *>(w);
    w += bins_bytes;
    uint32_t *thr_est = reinterpret_cast<uint32_t *>(w);
    w += thr_bytes;
    uint32_t *thr = reinterpret_cast<uint32_t *>(w);
    w += thr_bytes;
    uint32_t *redo = reinterpret_cast<uint32_t *>(w);
    w += thr_bytes;
    void *cand_key = w;
    w += ckey_bytes;
    uint32_t *cand_idx = reinterpret_cast<uint32_t *>(w);
    // initial state: nothing chosen, k needed; no candidates (a count above
    // cap sends every pass to the spectrum)
    std::vector<TopkState> init((size_t)B);
    for (TopkState &t : init) t = TopkState{0ull, 0u, (uint32_t)k, 0u, 0u, 0u};
    cudaError_t e = cudaMemcpyAsync(state, init.data(), (size_t)B * sizeof(TopkState), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(hist, 0, h_bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(arrive, 0, ar_bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cand_n, use_cand ? 0 : 0xFF, (size_t)B * sizeof(uint32_t), s);
    if (e == cudaSuccess && use_cand) e = cudaMemsetAsync(sbins, 0, 2 * bins_bytes, s);  // both histograms
    if (e != cudaSuccess) return cuda_error(e, "top-k workspace set-up");
    // pass geometry: blocks per vector so the whole batch fills the GPU
    const long long per_item = std::max<long long>(1, std::min<long long>((N + 2047) / 2048,
                                                                           (8ll * P->num_sms + B - 1) / B));
    const dim3 grid((unsigned)per_item, (unsigned)B);
    const void *sp = spec;
    long long n = N, kk = k;
    uint32_t cp = cap;
    gtt_status_t st;
    if (use_cand) {
        // the estimate: the bucket where a sample of every kTopkSample-th key
        // reaches k / kTopkSample plus four standard deviations and 8, so that
        // the k-th largest key is very rarely above it
        const double kf = (double)k / kTopkSample;
        long long m = (long long)std::ceil(kf + 4.0 * std::sqrt(kf) + 8.0);
        uint32_t *nil = nullptr;
        void *sargs[3] = {(void *)&sp, (void *)&n, (void *)&sbins};
        st = launch_timed(P, TK::sample(), grid, dim3(256), sargs, 0, s, "gtt_topk_sample_kernel");
        if (st != GTT_OK) return st;
        void *eargs[6] = {(void *)&m, (void *)&sbins, (void *)&thr_est, (void *)&nil, (void *)&nil, (void *)&nil};
        st = launch_timed(P, (const void *)&gtt_topk_binscan_kernel, dim3((unsigned)B), dim3(256), eargs, 0, s,
                          "gtt_topk_binscan_kernel");
        if (st != GTT_OK) return st;
        // one pass: the exact histogram and the candidates from the estimate
        void *c1args[9] = {(void *)&sp,       (void *)&n,        (void *)&thr_est, (void *)&cp, (void *)&cand_n,
                           (void *)&cand_key, (void *)&cand_idx, (void *)&bins,    (void *)&nil};
        st = launch_timed(P, TK::cand(), grid, dim3(256), c1args, 0, s, "gtt_topk_cand_kernel");
        if (st != GTT_OK) return st;
        void *targs[6] = {(void *)&kk, (void *)&bins, (void *)&thr, (void *)&thr_est, (void *)&cand_n,
                          (void *)&redo};
        st = launch_timed(P, (const void *)&gtt_topk_binscan_kernel, dim3((unsigned)B), dim3(256), targs, 0, s,
                          "gtt_topk_binscan_kernel");
        if (st != GTT_OK) return st;
        // the vectors whose estimate was above their exact bucket collect again
        void *c2args[9] = {(void *)&sp,       (void *)&n,        (void *)&thr, (void *)&cp,  (void *)&cand_n,
                           (void *)&cand_key, (void *)&cand_idx, (void *)&nil, (void *)&redo};
        st = launch_timed(P, TK::cand(), grid, dim3(256), c2args, 0, s, "gtt_topk_cand_kernel");
        if (st != GTT_OK) return st;
        void *fargs[11] = {(void *)&sp,       (void *)&n,        (void *)&kk,      (void *)&cp,
                           (void *)&cand_n,   (void *)&cand_key, (void *)&cand_idx, (void *)&out_idx,
                           (void *)&out_val,  (void *)&state,    (void *)&thr};
        st = launch_timed(P, TK::fastsort(), dim3((unsigned)B), dim3(kTopkSortThreads), fargs, 0, s,
                          "gtt_topk_fastsort_kernel");
        if (st != GTT_OK) return st;
    }
    const int passes = KB + 4;  // key digits, then index digits
    for (int pass = 0; pass < passes; ++pass) {
        int ps = pass;
        void *hargs[10] = {(void *)&sp, (void *)&n,      (void *)&ps,       (void *)&state,   (void *)&hist,
                           (void *)&arrive, (void *)&cp, (void *)&cand_n, (void *)&cand_key, (void *)&cand_idx};
        st = launch_timed(P, TK::hist(), grid, dim3(256), hargs, 0, s, "gtt_topk_hist_kernel");
        if (st != GTT_OK) return st;
    }
    void *cargs[10] = {(void *)&sp,      (void *)&n,  (void *)&kk,     (void *)&state,    (void *)&sel_key,
                       (void *)&sel_idx, (void *)&cp, (void *)&cand_n, (void *)&cand_key, (void *)&cand_idx};
    st = launch_timed(P, TK::collect(), grid, dim3(256), cargs, 0, s, "gtt_topk_collect_kernel");
    if (st != GTT_OK) return st;
    void *oargs[8] = {(void *)&sp,      (void *)&n,       (void *)&kk,      (void *)&sel_key,
                      (void *)&sel_idx, (void *)&out_idx, (void *)&out_val, (void *)&state};
    return launch_timed(P, TK::sort(), dim3((unsigned)B), dim3(kTopkSortThreads), oargs, 0, s, "gtt_topk_sort_kernel");
}

template <typename T>
static gtt_status_t topk_scatter(gtt_plan_s *P, const long long *idx, const void *val, long long k, void *y,
                                 cudaStream_t s) {
    long long kk = k, items = P->batch, n = P->N;
    const long long total = items * k;
    const int grid = (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, 8ll * P->num_sms));
    void *args[6] = {(void *)&idx, (void *)&val, (void *)&kk, (void *)&items, (void *)&n, (void *)&y};
    return launch_timed(P, TopkKernels<T>::scatter(), dim3(grid), dim3(256), args, 0, s, "gtt_topk_scatter_kernel");
}

// The reconstruction's first pass on the kept pairs only (gtt_sparse.cuh),
// when the first pass is a CUDA-core or TMA pass (their stages are the sparse
// kernel's) on contiguous tiles that divide a vector.  Returns false, with
// nothing launched, when it does not apply.
static bool sparse_first_applies(gtt_plan_s *P, long long k) {
    if (P->mixed || P->passes.empty() || k > kSparseMaxK) return false;
    const PassPlan &pp = P->passes[0];
    if (pp.tc.on || pp.tcx.on || pp.mix.on || pp.m0 != 0) return false;
    if (!pp.tma.on && pp.name.compare(0, 15, "gtt_pass_kernel") != 0) return false;  // e.g. the b = 8 tile kernel
    const PassParams &p = pp.params;
    if (p.L != (long long)p.r || P->N % p.tile_elems != 0 || P->N / p.tile_elems >= (long long)kSparseNoTile)
        return false;
    return sparse_first_kernel((int)P->dtype, P->b, pp.D) != nullptr;
}

static gtt_status_t sparse_first_pass(gtt_plan_s *P, const long long *idx, const void *val, long long k, void *y,
                                      cudaStream_t s) {
    const long long B = P->batch, N = P->N;
    const size_t need = (size_t)B * k * sizeof(unsigned long long);
    if (P->ws_topk_bytes < need) {  // the selection workspace, grown for the sorted pairs
        if (P->ws_topk) cudaFree(P->ws_topk);
        P->ws_topk = nullptr;
        P->ws_topk_bytes = 0;
        cudaError_t e = cudaMalloc(&P->ws_topk, need);
        if (e != cudaSuccess) {
            P->ws_topk = nullptr;
            return set_error(GTT_ERR_ALLOC, std::string("top-k workspace: ") + cudaGetErrorString(e));
        }
        P->ws_topk_bytes = need;
    }
    unsigned long long *sorted = static_cast<unsigned long long *>(P->ws_topk);
    PassPlan &pp = P->passes[0];
    PassParams prm = pp.params;
    prm.err = P->dev_err;
    uint32_t te = prm.tile_elems;
    long long kk = k, n = N;
    void *sargs[5] = {(void *)&idx, (void *)&kk, (void *)&n, (void *)&te, (void *)&sorted};
    gtt_status_t st = launch_timed(P, sparse_sort_kernel(), dim3((unsigned)B),
                                   dim3(kSparseSortThreads), sargs, 0, s, "gtt_sparse_sort_kernel");
    if (st != GTT_OK) return st;
    const void *kern = sparse_first_kernel((int)P->dtype, P->b, pp.D);
    cudaError_t e = allow_max_smem(kern, P->smem_optin);
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute");
    void *fargs[8] = {(void *)&idx, (void *)&val, (void *)&sorted, (void *)&kk,
                      (void *)&n,   (void *)&y,   (void *)&prm,    (void *)P->Wa.data()};
    st = launch_timed(P, kern, dim3((unsigned)k, (unsigned)B), dim3(pp.block), fargs, pp.smem, s,
                      "gtt_sparse_first_kernel");
    if (st != GTT_OK) return st;
    return run_passes_from(P, P->Wa, y, s, 1);
}

} // namespace gtt

using namespace gtt;

static gtt_status_t topk_check(gtt_plan_t P, long long k) {
    if (!P) return set_error(GTT_ERR_INVALID_ARG, "NULL plan");
    if (P->dtype == GTT_I32) return set_error(GTT_ERR_UNSUPPORTED, "top-k compression needs a floating-point dtype");
    if (k < 1 || k > P->N || k > kTopkMax)
        return set_error(GTT_ERR_INVALID_ARG, "k must be in [1, min(N, " + std::to_string(kTopkMax) + ")]");
    if (P->N >= 0xFFFFFFFFll) return set_error(GTT_ERR_UNSUPPORTED, "vectors of 2^32 - 1 elements or more");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev != P->device) return set_error(GTT_ERR_INVALID_ARG, "current CUDA device differs from the plan's device");
    return GTT_OK;
}

extern "C" gtt_status_t gtt_compress(gtt_plan_t P, const void *x, void *spectrum, long long k, long long *indices,
                                     void *values, gtt_stream_t stream) {
    gtt_status_t st = topk_check(P, k);
    if (st != GTT_OK) return st;
    if (!x || !spectrum || !indices || !values) return set_error(GTT_ERR_INVALID_ARG, "NULL pointer");
    if (((uintptr_t)x & 15u) || ((uintptr_t)spectrum & 15u) || ((uintptr_t)indices & 7u) ||
        ((uintptr_t)values & 15u))
        return set_error(GTT_ERR_INVALID_ARG, "misaligned pointer");
    cudaStream_t s = (cudaStream_t)stream;
    st = run_passes(P, P->Wf, x, spectrum, s);
    if (st != GTT_OK) return st;
    switch (P->dtype) {
    case GTT_F32: return topk_select<float>(P, spectrum, k, indices, values, s);
    case GTT_F64: return topk_select<double>(P, spectrum, k, indices, values, s);
    case GTT_C64: return topk_select<c64>(P, spectrum, k, indices, values, s);
    case GTT_C128: return topk_select<c128>(P, spectrum, k, indices, values, s);
    default: return set_error(GTT_ERR_UNSUPPORTED, "dtype");
    }
}

extern "C" gtt_status_t gtt_decompress(gtt_plan_t P, const long long *indices, const void *values, long long k,
                                       void *y, gtt_stream_t stream) {
    gtt_status_t st = topk_check(P, k);
    if (st != GTT_OK) return st;
    if (!indices || !values || !y) return set_error(GTT_ERR_INVALID_ARG, "NULL pointer");
    if (((uintptr_t)y & 15u) || ((uintptr_t)indices & 7u) || ((uintptr_t)values & 15u))
        return set_error(GTT_ERR_INVALID_ARG, "misaligned pointer");
    cudaStream_t s = (cudaStream_t)stream;
    st = zero_range(P, y, 0, P->N, s);
    if (st != GTT_OK) return st;
    if (sparse_first_applies(P, k)) return sparse_first_pass(P, indices, values, k, y, s);
    switch (P->dtype) {
    case GTT_F32: st = topk_scatter<float>(P, indices, values, k, y, s); break;
    case GTT_F64: st = topk_scatter<double>(P, indices, values, k, y, s); break;
    case GTT_C64: st = topk_scatter<c64>(P, indices, values, k, y, s); break;
    case GTT_C128: st = topk_scatter<c128>(P, indices, values, k, y, s); break;
    default: st = set_error(GTT_ERR_UNSUPPORTED, "dtype");
    }
    if (st != GTT_OK) return st;
    return run_passes(P, P->Wa, y, y, s);
}
