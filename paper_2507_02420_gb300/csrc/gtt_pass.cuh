// Fused multi-digit pass of the fast GTT (Sec. 3, Algorithm 1; cost
// structure of Sec. 3.1).
//
// Algorithm 1 applies W to one base-b digit at a time (a "mode").  Modes act
// on different digits, so they commute, and any set of them can be applied to
// a tile that holds every fibre of those digits.  One launch of this kernel
// applies the modes [m0, m0 + g) of a batch of vectors in ONE read and ONE
// write of HBM:
//
//   element index e = hi * (L*M) + row * L + lo,   L = b^m0, M = b^g,
//   row = the g transformed digits, lo = the m0 lower digits.
//
// A tile fixes `hi` and a run of r consecutive `lo` values (r divides L), so it
// is M rows of r contiguous elements at stride L.  r = L (in particular the
// first pass, m0 = 0) makes the tile one contiguous block.
//
// Inside a tile (staged in shared memory) the g digits are processed in
// register stages of D digits: each thread gathers B^D elements -- the full
// fibres of D digits -- into registers, applies W to each of those digits
// (W read from the constant bank), and writes them back.  The last stage's
// window is slid down so it stays inside the g digits; a per-stage mask says
// which of its digits are applied there.
#pragma once
#include <type_traits>

#include "gtt_types.cuh"

namespace gtt {

constexpr int kMaxStages = 24;
constexpr int kPassMaxThreads = 512;

struct PassParams {
    long long total;      // batch * N elements
    long long L;          // b^m0: stride of the first transformed digit
    long long tiles;      // end of the tile range of this launch (total / (M * r) for a whole pass)
    long long tile_begin; // first tile of this launch (0 for a whole pass)
    uint32_t r;           // run length
    uint32_t M;           // b^g
    uint32_t tile_elems;  // M * r
    uint32_t lo_blocks;   // L / r (fits 32 bits: <= 2^31)
    FastDiv div_lo_blocks;
    FastDiv div_r;
    FastDiv div_cpr;      // division by r / (16-byte chunk elements), vec_mode 2
    int vec_mode;         // 0 element-wise, 1 contiguous 16-byte chunks, 2 row-chunked 16-byte
    int nstages;
    int stage_a[kMaxStages];     // first digit (within the g) of the stage's register window
    int stage_mask[kMaxStages];  // bit k set: apply W to window digit k in this stage
    uint32_t stage_strideA[kMaxStages];  // r * b^a
    FastDiv stage_divBa[kMaxStages];     // division by b^a
    int *err;             // the plan's status word (bounds checks of the debug build)
};

// smem position of tile element e: one pad element after every B^D elements,
// which turns the power-of-two lane strides of the first stage into odd ones.
template <int PADEVERY> __device__ __forceinline__ uint32_t spos(uint32_t e) {
    return e + e / PADEVERY;
}

// Complex64 digits of radix 5 .. SMAX use scalar FMAs when W is a kernel
// parameter (CW): the packed form's (re, re) / (-im, im) pairs of such a
// matrix do not stay in registers, and moving each pair into registers before
// its packed FMA costs more than the packing saves, while a scalar FMA takes
// its W entry straight from the constant bank.  Measured per forward on
// b^n x batch transforms: b = 5 904 -> 850 us, b = 8 1462 -> 1328 us, b = 7
// even, b = 16 1934 -> 2000 us (so SMAX = 8 here; the mixed-radix kernel,
// whose stages take W from parameter slots, gains at 16 too and passes 16).
// FP32 keeps its packed row pairs: scalar FMAs measured slower there (b = 16
// 1032 -> 1502 us, b = 12 281 -> 437 us).  With W in shared memory a pair is
// one load either way, and the packed forms stay.  Both forms do the same
// operations in the same order.
template <typename T, int B, int D, int K, bool CW = true, int SMAX = 8>
__device__ __forceinline__ void apply_digit(T (&v)[cpow(B, D)], const WMat<T, B> &W) {
    constexpr int S = cpow(B, K);
    constexpr bool scalar = CW && std::is_same<T, c64>::value && B >= 5 && B <= SMAX;
#pragma unroll
    for (int o = 0; o < cpow(B, D) / B; ++o) {
        const int base = (o / S) * S * B + (o % S);
        if constexpr (std::is_same<T, c64>::value && !scalar) {
            // packed FP32x2: the same operations, in the same order, as mul/fma_acc
            float2 in[B], sw[B];
#pragma unroll
            for (int j = 0; j < B; ++j) {
                in[j] = make_float2(v[base + j * S].re, v[base + j * S].im);
                sw[j] = make_float2(v[base + j * S].im, v[base + j * S].re);
            }
            // inputs outermost: the B accumulators advance together (independent
            // chains between dependent FMAs); each output still sums j = 0..B-1 in order
            float2 acc[B];
#pragma unroll
            for (int i = 0; i < B; ++i) acc[i] = __ffma2_rn(W.wa[i * B], in[0], make_float2(0.f, 0.f));
#pragma unroll
            for (int i = 0; i < B; ++i) acc[i] = __ffma2_rn(W.wb[i * B], sw[0], acc[i]);
#pragma unroll
            for (int j = 1; j < B; ++j) {
#pragma unroll
                for (int i = 0; i < B; ++i) acc[i] = __ffma2_rn(W.wa[i * B + j], in[j], acc[i]);
#pragma unroll
                for (int i = 0; i < B; ++i) acc[i] = __ffma2_rn(W.wb[i * B + j], sw[j], acc[i]);
            }
#pragma unroll
            for (int i = 0; i < B; ++i) v[base + i * S] = c64{acc[i].x, acc[i].y};
        } else if constexpr (std::is_same<T, float>::value && B % 2 == 0 && !scalar) {
            float2 in[B];
#pragma unroll
            for (int j = 0; j < B; ++j) in[j] = make_float2(v[base + j * S], v[base + j * S]);
            float2 acc[B / 2];
#pragma unroll
            for (int ip = 0; ip < B / 2; ++ip) acc[ip] = __ffma2_rn(W.wp[ip * B], in[0], make_float2(0.f, 0.f));
#pragma unroll
            for (int j = 1; j < B; ++j)
#pragma unroll
                for (int ip = 0; ip < B / 2; ++ip) acc[ip] = __ffma2_rn(W.wp[ip * B + j], in[j], acc[ip]);
#pragma unroll
            for (int ip = 0; ip < B / 2; ++ip) {
                v[base + 2 * ip * S] = acc[ip].x;
                v[base + (2 * ip + 1) * S] = acc[ip].y;
            }
        } else {
            T in[B];
#pragma unroll
            for (int j = 0; j < B; ++j) in[j] = v[base + j * S];
#pragma unroll
            for (int i = 0; i < B; ++i) {
                T acc = mul(W.w[i * B], in[0]);
#pragma unroll
                for (int j = 1; j < B; ++j) acc = fma_acc(W.w[i * B + j], in[j], acc);
                v[base + i * S] = acc;
            }
        }
    }
}

// Apply W to every register digit K < D whose bit is set in `mask` (CW: W is
// a kernel parameter, false: W is in shared memory).
template <typename T, int B, int D, int K = 0, bool CW = true>
__device__ __forceinline__ void apply_window(T (&v)[cpow(B, D)], int mask, const WMat<T, B> &W) {
    if constexpr (K < D) {
        if (mask & (1 << K)) apply_digit<T, B, D, K, CW>(v, W);
        apply_window<T, B, D, K + 1, CW>(v, mask, W);
    }
}

template <typename T> struct Vec16;  // 16-byte chunk of T
template <> struct Vec16<float> { static constexpr int n = 4; };
template <> struct Vec16<uint32_t> { static constexpr int n = 4; };
template <> struct Vec16<double> { static constexpr int n = 2; };
template <> struct Vec16<c64> { static constexpr int n = 2; };
template <> struct Vec16<c128> { static constexpr int n = 1; };

template <typename T>
__device__ __forceinline__ void load16(const T *g, T (&out)[Vec16<T>::n]) {
    int4 raw = *reinterpret_cast<const int4 *>(g);
    *reinterpret_cast<int4 *>(out) = raw;
}
template <typename T>
__device__ __forceinline__ void store16(T *g, const T (&in)[Vec16<T>::n]) {
    *reinterpret_cast<int4 *>(g) = *reinterpret_cast<const int4 *>(in);
}

template <typename T, int B, int D>
__global__ void __launch_bounds__(kPassMaxThreads)
gtt_pass_kernel(const T *in, T *out, PassParams p, WMat<T, B> W) {
    constexpr int RB = cpow(B, D);   // elements per register block
    constexpr int CE = Vec16<T>::n;  // elements per 16-byte chunk
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s = reinterpret_cast<T *>(smem_raw);
    // smem slot of tile element e (padded), and global element offsets, checked in the debug build
    const uint32_t smem_elems = p.tile_elems + p.tile_elems / cpow(B, D) + 1;
#define SP(e) GTT_CHECKED(spos<RB>(e), smem_elems, p.err)
#define GI(off, w) GTT_CHECKED(off, p.total - base - (w) + 1, p.err)

    const uint32_t tid = threadIdx.x, nth = blockDim.x;
    const uint32_t tile_elems = p.tile_elems, r = p.r;
    const long long LM = p.L * (long long)p.M;

    for (long long t = p.tile_begin + blockIdx.x; t < p.tiles; t += gridDim.x) {
        const long long hi = t / p.lo_blocks;
        const uint32_t lob = (uint32_t)(t - hi * p.lo_blocks);
        const long long base = hi * LM + (long long)lob * r;
        const T *gin = in + base;

        // ---- HBM -> smem
        if (p.vec_mode == 1) {  // contiguous tile, 16-byte chunks
            for (uint32_t c = tid; c < tile_elems / CE; c += nth) {
                T v[CE];
                load16(gin + GI((size_t)c * CE, CE), v);
#pragma unroll
                for (int i = 0; i < CE; ++i) s[SP(c * CE + i)] = v[i];
            }
        } else if (p.vec_mode == 2) {  // rows of r elements, r % CE == 0
            const uint32_t cpr = r / CE;
            for (uint32_t c = tid; c < tile_elems / CE; c += nth) {
                const uint32_t row = p.div_cpr.div(c), cc = c - row * cpr;
                T v[CE];
                load16(gin + GI((long long)row * p.L + cc * CE, CE), v);
#pragma unroll
                for (int i = 0; i < CE; ++i) s[SP(row * r + cc * CE + i)] = v[i];
            }
        } else if (p.L == (long long)r) {
            // contiguous, but not in whole 16-byte chunks (odd radices): the
            // elements up to the first 16-byte boundary one by one, then
            // chunks, then the rest
            const uint32_t head = min(tile_elems, (uint32_t)((CE - ((uintptr_t)gin / sizeof(T)) % CE) % CE));
            const uint32_t nch = (tile_elems - head) / CE, mid_end = head + nch * CE;
            for (uint32_t e = tid; e < head; e += nth) s[SP(e)] = gin[GI(e, 1)];
            for (uint32_t c = tid; c < nch; c += nth) {
                T v[CE];
                load16(gin + GI(head + (size_t)c * CE, CE), v);
#pragma unroll
                for (int i = 0; i < CE; ++i) s[SP(head + c * CE + i)] = v[i];
            }
            for (uint32_t e = mid_end + tid; e < tile_elems; e += nth) s[SP(e)] = gin[GI(e, 1)];
        } else {
            for (uint32_t e = tid; e < tile_elems; e += nth) {
                const uint32_t row = p.div_r.div(e), col = e - row * r;
                s[SP(e)] = gin[GI((long long)row * p.L + col, 1)];
            }
        }
        __syncthreads();

        // ---- register stages
        const uint32_t nslots = tile_elems / RB;
        for (int st = 0; st < p.nstages; ++st) {
            const uint32_t strideA = p.stage_strideA[st];   // r * b^a
            const int mask = p.stage_mask[st];
            for (uint32_t slot = tid; slot < nslots; slot += nth) {
                // slot -> (col, low digits below the window, digits above it)
                const uint32_t rest = p.div_r.div(slot);
                const uint32_t col = slot - rest * r;
                const uint32_t high = p.stage_divBa[st].div(rest);
                const uint32_t low = rest - high * p.stage_divBa[st].d;
                const uint32_t e0 = high * (strideA * RB) + low * r + col;
                T v[RB];
#pragma unroll
                for (int q = 0; q < RB; ++q) v[q] = s[SP(e0 + q * strideA)];
                apply_window<T, B, D>(v, mask, W);
#pragma unroll
                for (int q = 0; q < RB; ++q) s[SP(e0 + q * strideA)] = v[q];
            }
            __syncthreads();
        }

        // ---- smem -> HBM
        T *gout = out + base;
        if (p.vec_mode == 1) {
            for (uint32_t c = tid; c < tile_elems / CE; c += nth) {
                T v[CE];
#pragma unroll
                for (int i = 0; i < CE; ++i) v[i] = s[SP(c * CE + i)];
                store16(gout + GI((size_t)c * CE, CE), v);
            }
        } else if (p.vec_mode == 2) {
            const uint32_t cpr = r / CE;
            for (uint32_t c = tid; c < tile_elems / CE; c += nth) {
                const uint32_t row = p.div_cpr.div(c), cc = c - row * cpr;
                T v[CE];
#pragma unroll
                for (int i = 0; i < CE; ++i) v[i] = s[SP(row * r + cc * CE + i)];
                store16(gout + GI((long long)row * p.L + cc * CE, CE), v);
            }
        } else if (p.L == (long long)r) {  // contiguous, not in whole chunks: as the load
            const uint32_t head = min(tile_elems, (uint32_t)((CE - ((uintptr_t)gout / sizeof(T)) % CE) % CE));
            const uint32_t nch = (tile_elems - head) / CE, mid_end = head + nch * CE;
            for (uint32_t e = tid; e < head; e += nth) gout[GI(e, 1)] = s[SP(e)];
            for (uint32_t c = tid; c < nch; c += nth) {
                T v[CE];
#pragma unroll
                for (int i = 0; i < CE; ++i) v[i] = s[SP(head + c * CE + i)];
                store16(gout + GI(head + (size_t)c * CE, CE), v);
            }
            for (uint32_t e = mid_end + tid; e < tile_elems; e += nth) gout[GI(e, 1)] = s[SP(e)];
        } else {
            for (uint32_t e = tid; e < tile_elems; e += nth) {
                const uint32_t row = p.div_r.div(e), col = e - row * r;
                gout[GI((long long)row * p.L + col, 1)] = s[SP(e)];
            }
        }
        __syncthreads();
    }
#undef SP
#undef GI
}

} // namespace gtt
