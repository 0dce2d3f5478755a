// Multi-factor passes of the heterogeneous transform G = W_0 (x) ... (x) W_{n-1}
// (the remark after Def. 2.3): one launch applies several factors, each to
// its own digit of the index, in one HBM round trip.
//
// The digits of a mixed-radix index have different radices, so the uniform
// pass kernel (one compile-time B for every digit of a pass) cannot hold more
// than one of them.  Here a tile holds every fibre of g consecutive digits
// with radices R_0 .. R_{g-1} (fastest first) -- M = R_0 ... R_{g-1} rows (times
// `kblk` blocks) of r contiguous elements at stride L, as in gtt_pass.cuh --
// and stage k applies its factor along digit k, whose tile stride is
// r * R_0 ... R_{k-1}.  Each stage dispatches on its radix and its position to
// a compile-time fibre of R_k registers and a compile-time slot of the kernel
// parameters that holds its factor, so every factor entry is read straight
// from the constant bank, as in the uniform pass kernel.
#pragma once
#include "gtt_pass.cuh"

namespace gtt {

constexpr int kMixMaxStages = 4;
constexpr int kMixThreads = 256;

// CTAs per SM the register budget aims at: three for 4- and 8-byte types
// (measured best for complex64: 948 us against 963 us at two on the 9-factor
// workload); two for the FP64 types, whose large-radix fibres spill at three.
template <typename T> __host__ __device__ constexpr int mix_min_blocks() {
    return (std::is_same<T, double>::value || std::is_same<T, c128>::value) ? 2 : 3;
}

// Factor slots in the parameters: one WMat<T, 16> each (a smaller factor uses
// the start of its slot); three for the 16-byte-entry layouts, else four.
template <typename T> __host__ __device__ constexpr int mix_slots() { return sizeof(WMat<T, 16>) >= 4096 ? 3 : 4; }

struct MixedParams {
    PassParams p;        // tile geometry (M = product of the stage radices x blocks); p.nstages unused
    int nst;             // stages, one per digit of the pass, fastest digit first
    int pad_shift;       // tile element e sits at e + (e >> pad_shift) in shared memory
    uint32_t smem_elems; // tile slots including the padding
    int rad[kMixMaxStages];            // radix of the stage's digit
    uint32_t stride[kMixMaxStages];    // tile stride of that digit: r x (product of the radices below it)
    FastDiv div_blow[kMixMaxStages];   // division by the product of the radices below it
};

// Kernel parameters: the geometry, then the factor of stage k in w[k]
// (W_k, or W_k^H for the adjoint), in the WMat<T, R_k> layout.
template <typename T> struct MixedArgs {
    MixedParams m;
    WMat<T, 16> w[mix_slots<T>()];
};

// One stage: every fibre of the stage's digit through its factor (radix B,
// parameter slot ST).
template <typename T, int B, int ST>
__device__ __forceinline__ void mixed_stage(T *__restrict__ s, const MixedArgs<T> &a) {
    constexpr int st = ST;
    const MixedParams &m = a.m;
    const WMat<T, B> &W = *reinterpret_cast<const WMat<T, B> *>(&a.w[ST]);
    const uint32_t tid = threadIdx.x, nth = blockDim.x;
    const uint32_t r = m.p.r, S = m.stride[st], nslots = m.p.tile_elems / B;
    const FastDiv div_r = m.p.div_r, div_blow = m.div_blow[st];
    const int ps = m.pad_shift;
    for (uint32_t slot = tid; slot < nslots; slot += nth) {
        // slot -> (column of the run, digits below the stage's, digits above it)
        const uint32_t rest = div_r.div(slot), col = slot - rest * r;
        const uint32_t high = div_blow.div(rest), low = rest - high * div_blow.d;
        const uint32_t e0 = high * (S * B) + low * r + col;
        T v[B];
#pragma unroll
        for (int q = 0; q < B; ++q) {
            const uint32_t e = e0 + q * S;
            v[q] = s[GTT_CHECKED(e + (e >> ps), m.smem_elems, m.p.err)];
        }
        apply_digit<T, B, 1, 0, true, 16>(v, W);  // complex64: scalar FMAs from radix 5 on
#pragma unroll
        for (int q = 0; q < B; ++q) {
            const uint32_t e = e0 + q * S;
            s[GTT_CHECKED(e + (e >> ps), m.smem_elems, m.p.err)] = v[q];
        }
    }
}

template <typename T, int B>
__device__ __forceinline__ void mixed_stage_slot(T *s, const MixedArgs<T> &a, int st) {
    switch (st) {
    case 0: mixed_stage<T, B, 0>(s, a); break;
    case 1: mixed_stage<T, B, 1>(s, a); break;
    case 2: mixed_stage<T, B, 2>(s, a); break;
    default:
        if constexpr (mix_slots<T>() > 3) mixed_stage<T, B, 3>(s, a);
        break;
    }
}

template <typename T>
__device__ __forceinline__ void mixed_stage_any(T *s, const MixedArgs<T> &a, int st) {
    switch (a.m.rad[st]) {
    case 2: mixed_stage_slot<T, 2>(s, a, st); break;
    case 3: mixed_stage_slot<T, 3>(s, a, st); break;
    case 4: mixed_stage_slot<T, 4>(s, a, st); break;
    case 5: mixed_stage_slot<T, 5>(s, a, st); break;
    case 6: mixed_stage_slot<T, 6>(s, a, st); break;
    case 7: mixed_stage_slot<T, 7>(s, a, st); break;
    case 8: mixed_stage_slot<T, 8>(s, a, st); break;
    case 9: mixed_stage_slot<T, 9>(s, a, st); break;
    case 10: mixed_stage_slot<T, 10>(s, a, st); break;
    case 11: mixed_stage_slot<T, 11>(s, a, st); break;
    case 12: mixed_stage_slot<T, 12>(s, a, st); break;
    case 13: mixed_stage_slot<T, 13>(s, a, st); break;
    case 14: mixed_stage_slot<T, 14>(s, a, st); break;
    case 15: mixed_stage_slot<T, 15>(s, a, st); break;
    case 16: mixed_stage_slot<T, 16>(s, a, st); break;
    default: break;
    }
}

// One pass over tiles.
template <typename T>
__global__ void __launch_bounds__(kMixThreads, mix_min_blocks<T>())
gtt_mixed_pass_kernel(const T *in, T *out, const __grid_constant__ MixedArgs<T> a) {
    constexpr int CE = Vec16<T>::n;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s = reinterpret_cast<T *>(smem_raw);
    const MixedParams &m = a.m;
    const PassParams &p = m.p;
    const int ps = m.pad_shift;
#define SP(e) GTT_CHECKED((e) + ((e) >> ps), m.smem_elems, p.err)
#define GI(off, w) GTT_CHECKED(off, p.total - base - (w) + 1, p.err)

    const uint32_t tid = threadIdx.x, nth = blockDim.x;

    const uint32_t tile_elems = p.tile_elems, r = p.r;
    const long long LM = p.L * (long long)p.M;
    for (long long t = p.tile_begin + blockIdx.x; t < p.tiles; t += gridDim.x) {
        const long long hi = t / p.lo_blocks;
        const uint32_t lob = (uint32_t)(t - hi * p.lo_blocks);
        const long long base = hi * LM + (long long)lob * r;
        const T *gin = in + base;

        // ---- HBM -> smem (the load forms of gtt_pass_kernel)
        if (p.vec_mode == 1) {
            for (uint32_t c = tid; c < tile_elems / CE; c += nth) {
                T v[CE];
                load16(gin + GI((size_t)c * CE, CE), v);
#pragma unroll
                for (int i = 0; i < CE; ++i) s[SP(c * CE + i)] = v[i];
            }
        } else if (p.vec_mode == 2) {
            const uint32_t cpr = r / CE;
            for (uint32_t c = tid; c < tile_elems / CE; c += nth) {
                const uint32_t row = p.div_cpr.div(c), cc = c - row * cpr;
                T v[CE];
                load16(gin + GI((long long)row * p.L + cc * CE, CE), v);
#pragma unroll
                for (int i = 0; i < CE; ++i) s[SP(row * r + cc * CE + i)] = v[i];
            }
        } else if (p.L == (long long)r) {
            // contiguous, not in whole 16-byte chunks (odd radices): the head
            // up to a 16-byte boundary element by element, then chunks, then the rest
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

        for (int st = 0; st < m.nst; ++st) {
            mixed_stage_any<T>(s, a, st);
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

// Kernel entry for a dtype code (gtt_dtype_t), instantiated in gtt_mixed_inst_*.cu,
// and the layout of its parameters: total bytes, offset of w[0], bytes per slot.
size_t mixed_args_bytes(int dtype, size_t *w_offset, size_t *slot_bytes, int *slots);
const void *mixed_kernel_f64();
const void *mixed_kernel_f32();
const void *mixed_kernel_c64();
const void *mixed_kernel_c128();
const void *mixed_kernel_u32();
inline const void *mixed_kernel(int dtype) {
    switch (dtype) {
    case 0: return mixed_kernel_f64();
    case 1: return mixed_kernel_f32();
    case 2: return mixed_kernel_c64();
    case 3: return mixed_kernel_c128();
    case 4: return mixed_kernel_u32();
    default: return nullptr;
    }
}

} // namespace gtt
