// Element types and arithmetic for the GTT kernels.
//
// Complex values are stored interleaved (re, im), matching the C ABI's C64 /
// C128 layouts.  The integer type is uint32_t: the ABI's int32 data with
// arithmetic that wraps modulo 2^32, so results are exact bit patterns.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gtt {

struct __align__(8) c64 {
    float re, im;
};
struct __align__(16) c128 {
    double re, im;
};

template <typename T> struct Traits;
template <> struct Traits<float> {
    static constexpr bool complex = false;
    using real = float;
};
template <> struct Traits<double> {
    static constexpr bool complex = false;
    using real = double;
};
template <> struct Traits<c64> {
    static constexpr bool complex = true;
    using real = float;
};
template <> struct Traits<c128> {
    static constexpr bool complex = true;
    using real = double;
};
template <> struct Traits<uint32_t> {
    static constexpr bool complex = false;
    using real = uint32_t;
};

// acc = w * v
__device__ __forceinline__ float mul(float w, float v) { return w * v; }
__device__ __forceinline__ double mul(double w, double v) { return w * v; }
__device__ __forceinline__ uint32_t mul(uint32_t w, uint32_t v) { return w * v; }
__device__ __forceinline__ c64 mul(c64 w, c64 v) {
    c64 r;
    r.re = __fmul_rn(w.re, v.re);
    r.im = __fmul_rn(w.re, v.im);
    r.re = __fmaf_rn(-w.im, v.im, r.re);
    r.im = __fmaf_rn(w.im, v.re, r.im);
    return r;
}
__device__ __forceinline__ c128 mul(c128 w, c128 v) {
    c128 r;
    r.re = __dmul_rn(w.re, v.re);
    r.im = __dmul_rn(w.re, v.im);
    r.re = __fma_rn(-w.im, v.im, r.re);
    r.im = __fma_rn(w.im, v.re, r.im);
    return r;
}

// acc += w * v
__device__ __forceinline__ float fma_acc(float w, float v, float acc) { return __fmaf_rn(w, v, acc); }
__device__ __forceinline__ double fma_acc(double w, double v, double acc) { return __fma_rn(w, v, acc); }
__device__ __forceinline__ uint32_t fma_acc(uint32_t w, uint32_t v, uint32_t acc) { return acc + w * v; }
__device__ __forceinline__ c64 fma_acc(c64 w, c64 v, c64 acc) {
    acc.re = __fmaf_rn(w.re, v.re, acc.re);
    acc.im = __fmaf_rn(w.re, v.im, acc.im);
    acc.re = __fmaf_rn(-w.im, v.im, acc.re);
    acc.im = __fmaf_rn(w.im, v.re, acc.im);
    return acc;
}
__device__ __forceinline__ c128 fma_acc(c128 w, c128 v, c128 acc) {
    acc.re = __fma_rn(w.re, v.re, acc.re);
    acc.im = __fma_rn(w.re, v.im, acc.im);
    acc.re = __fma_rn(-w.im, v.im, acc.re);
    acc.im = __fma_rn(w.im, v.re, acc.im);
    return acc;
}

// a + b
__device__ __forceinline__ float add_(float a, float b) { return a + b; }
__device__ __forceinline__ double add_(double a, double b) { return a + b; }
__device__ __forceinline__ c64 add_(c64 a, c64 b) { return c64{a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ c128 add_(c128 a, c128 b) { return c128{a.re + b.re, a.im + b.im}; }

// Index checks of the debug build (compiled with -DGTT_DEBUG into
// libgtt_debug.so; the release library has none).  An index outside
// [0, n) sets bit 1 (value 2) of the plan's status word and is replaced by 0,
// a location inside the buffer, so the kernel goes on without touching memory
// it does not own; gtt_plan_check reports the violation.  Nothing traps.
#ifdef GTT_DEBUG
__device__ __forceinline__ long long gtt_dbg_index(long long i, long long n, int *err) {
    if (i < 0 || i >= n) {
        if (err) atomicOr(err, 2);
        return 0;
    }
    return i;
}
#define GTT_CHECKED(i, n, err) (::gtt::gtt_dbg_index((long long)(i), (long long)(n), (err)))
#else
#define GTT_CHECKED(i, n, err) (i)
#endif

// Compile-time integer power.
__host__ __device__ constexpr int cpow(int b, int e) { return e == 0 ? 1 : b * cpow(b, e - 1); }

// Base matrix passed by value as a kernel parameter, so that every W[i][j]
// with compile-time (i, j) is read straight from the constant bank.
template <typename T, int B> struct WMat {
    T w[B * B];
};
// complex64 adds, for the packed FP32x2 FMAs of apply_digit, the pairs
// wa = (re, re) and wb = (-im, im) of every entry: one complex MAC is then
// acc += wa * (v.re, v.im) followed by acc += wb * (v.im, v.re).
template <int B> struct WMat<c64, B> {
    c64 w[B * B];
    float2 wa[B * B];
    float2 wb[B * B];
};
// FP32 with even B adds the row pairs wp[(i/2)*B + j] = (W[i][j], W[i+1][j]),
// so two outputs of a fibre advance with one packed FMA.
template <int B> struct WMat<float, B> {
    float w[B * B];
    float2 wp[(B % 2 == 0) ? B * B / 2 : 1];
};

// Unsigned 32-bit division by a runtime divisor d >= 1 via a precomputed
// multiplier (the round-up method of Granlund and Montgomery, "Division by
// invariant integers using multiplication", PLDI 1994):
//   l = ceil(log2 d),  m = floor(2^32 (2^l - d) / d) + 1,
//   q = (t + ((n - t) >> 1)) >> (l - 1)  with t = umulhi(m, n)   (d > 1),
// exact for every 32-bit n.
struct FastDiv {
    uint32_t d, m;
    int l;
    __host__ void init(uint32_t dd) {
        d = dd;
        l = 0;
        while ((1ull << l) < dd) ++l;
        m = (uint32_t)((((1ull << 32) * ((1ull << l) - dd)) / dd) + 1);
    }
    __device__ __forceinline__ uint32_t div(uint32_t n) const {
        if (d == 1) return n;
        uint32_t t = __umulhi(m, n);
        return (t + ((n - t) >> 1)) >> (l - 1);
    }
};

} // namespace gtt
