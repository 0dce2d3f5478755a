// Reverse-mode derivative of y = G_N x, one pass (a group of modes) at a time.
//
// No counterpart in the paper.  With a_0 = x, a_{k+1} = P_k a_k (W applied to
// digit k) and g_{k+1} = dL/da_{k+1}, PyTorch's conjugate convention gives
//     g_k = P_k^H g_{k+1}        (W^H applied to digit k),
//     dW += sum over the fibres of digit k of g_{k+1}[i] * conj(a_k[j]).
// A backward pass covers the modes [m0, m0+g) of the forward schedule's tile
// geometry (the same (hi, run) tiles as gtt_pass_kernel).  Per tile it loads
// the pass's input activation a_{m0} and the gradient g_{m0+g}, recomputes
// a_{m0+1} .. a_{m0+g-1} into shared memory, then walks the digits in reverse.
//
// dW partials: each fibre is handled by a group of B/R consecutive threads;
// thread `ib` of the group owns dW rows [ib*R, ib*R + R) and keeps R x B
// accumulators in registers across every tile the CTA processes.  At the end
// the CTA sums its threads' partials in a fixed order and writes one b x b
// partial per CTA; gtt_dw_reduce_kernel adds the partials of all CTAs and
// passes in a fixed order, so dW is bitwise reproducible.
#pragma once
#include <type_traits>

#include "gtt_pass.cuh"

namespace gtt {

constexpr int kBwdThreads = 256;

__device__ __forceinline__ float conj_(float v) { return v; }
__device__ __forceinline__ double conj_(double v) { return v; }
__device__ __forceinline__ c64 conj_(c64 v) { return c64{v.re, -v.im}; }
__device__ __forceinline__ c128 conj_(c128 v) { return c128{v.re, -v.im}; }

template <typename T> __device__ __forceinline__ T zero_() { return T{}; }

// v[i] for a runtime i, as unrolled selects (keeps v in registers)
template <typename T, int B> __device__ __forceinline__ T pick(const T (&v)[B], int i) {
    T r = v[0];
#pragma unroll
    for (int q = 1; q < B; ++q)
        if (q == i) r = v[q];
    return r;
}

// Rows of dW per thread: the largest R dividing B with B/R a power of two
// and R*B accumulators within budget (64 real / 32 complex); odd B: R = B.
__host__ __device__ constexpr int bwd_rows(int B, bool cplx) {
    int budget = cplx ? 32 : 64;
    int R = B;
    while (R * B > budget && R % 2 == 0) R /= 2;
    return R;
}

template <typename T, int B, int R>
__global__ void __launch_bounds__(kBwdThreads)
gtt_backward_pass_kernel(const T *act_in, const T *grad_out, T *grad_in, T *dw_part, PassParams p,
                         int g, WMat<T, B> W, WMat<T, B> WH) {
    constexpr int GS = B / R;  // threads per fibre group
    constexpr int CE = Vec16<T>::n;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s = reinterpret_cast<T *>(smem_raw);
    const uint32_t tile = p.tile_elems, r = p.r;
    const uint32_t tstride = tile + tile / B + 1;  // padded tile size in elements
    T *G = s + (size_t)g * tstride;               // gradient tile; A_k at s + k*tstride

    const uint32_t tid = threadIdx.x, nth = blockDim.x;
    const long long LM = p.L * (long long)p.M;
    const uint32_t nfib = tile / B;

    T acc[R][B];
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < B; ++j) acc[i][j] = zero_<T>();

    for (long long t = p.tile_begin + blockIdx.x; t < p.tiles; t += gridDim.x) {
        const long long hi = t / p.lo_blocks;
        const uint32_t lob = (uint32_t)(t - hi * p.lo_blocks);
        const long long base = hi * LM + (long long)lob * r;
        if (p.vec_mode != 0) {  // 16-byte chunks: contiguous tile (1) or rows of r, r % CE == 0 (2)
            const uint32_t cpr = p.vec_mode == 1 ? tile / CE : r / CE;
            const long long rstride = p.vec_mode == 1 ? 0 : p.L;
            for (uint32_t c = tid; c < tile / CE; c += nth) {
                const uint32_t row = p.vec_mode == 1 ? 0u : p.div_cpr.div(c), cc = c - row * cpr;
                const long long ga = GTT_CHECKED(base + (long long)row * rstride + cc * CE, p.total - CE + 1, p.err);
                T va[CE], vg[CE];
                load16(act_in + ga, va);
                load16(grad_out + ga, vg);
                const uint32_t e0 = p.vec_mode == 1 ? c * CE : row * r + cc * CE;
#pragma unroll
                for (int i = 0; i < CE; ++i) {
                    s[spos<B>(e0 + i)] = va[i];
                    G[spos<B>(e0 + i)] = vg[i];
                }
            }
        } else {
            for (uint32_t e = tid; e < tile; e += nth) {
                const uint32_t row = p.div_r.div(e), col = e - row * r;
                const long long ga = GTT_CHECKED(base + (long long)row * p.L + col, p.total, p.err);
                s[spos<B>(e)] = act_in[ga];
                G[spos<B>(e)] = grad_out[ga];
            }
        }
        __syncthreads();

        // Window element q of a fibre sits at spos(e0 + q * strideA).  That is
        // linear in q when strideA is a multiple of B, or 1 with e0 a multiple
        // of B (always the case for power-of-b runs): spos(e0) + q * step.
        // forward recompute: A_{k+1} = mode k applied to A_k, k = 0 .. g-2
        for (int k = 0; k + 1 < g; ++k) {
            const T *A = s + (size_t)k * tstride;
            T *An = s + (size_t)(k + 1) * tstride;
            const uint32_t strideA = p.stage_strideA[k];
            const bool lin = strideA == 1u || strideA % B == 0u;
            const uint32_t step = strideA == 1u ? 1u : strideA + strideA / B;
            for (uint32_t f = tid; f < nfib; f += nth) {
                const uint32_t rest = p.div_r.div(f), col = f - rest * r;
                const uint32_t high = p.stage_divBa[k].div(rest);
                const uint32_t low = rest - high * p.stage_divBa[k].d;
                const uint32_t e0 = high * (strideA * B) + low * r + col;
                auto body = [&](auto pos) {
                    T v[B];
#pragma unroll
                    for (int q = 0; q < B; ++q) v[q] = A[pos(q)];
                    apply_window<T, B, 1>(v, 1, W);
#pragma unroll
                    for (int q = 0; q < B; ++q) An[pos(q)] = v[q];
                };
                if (lin) {
                    const uint32_t sb = spos<B>(e0);
                    body([&](int q) { return sb + (uint32_t)q * step; });
                } else {
                    body([&](int q) { return spos<B>(e0 + (uint32_t)q * strideA); });
                }
            }
            __syncthreads();
        }

        // reverse sweep over the pass's digits
        for (int k = g - 1; k >= 0; --k) {
            const T *A = s + (size_t)k * tstride;
            const uint32_t strideA = p.stage_strideA[k];
            const bool lin = strideA == 1u || strideA % B == 0u;
            const uint32_t step = strideA == 1u ? 1u : strideA + strideA / B;
            for (uint32_t slot = tid; slot < nfib * GS; slot += nth) {
                const uint32_t f = slot / GS, ib = slot % GS;
                const uint32_t rest = p.div_r.div(f), col = f - rest * r;
                const uint32_t high = p.stage_divBa[k].div(rest);
                const uint32_t low = rest - high * p.stage_divBa[k].d;
                const uint32_t e0 = high * (strideA * B) + low * r + col;
                auto body = [&](auto pos) {
                    T a[B], gv[B];
#pragma unroll
                    for (int q = 0; q < B; ++q) {
                        a[q] = conj_(A[pos(q)]);
                        gv[q] = G[pos(q)];
                    }
                    T gn[R];
                    if constexpr (std::is_same<T, float>::value && B % 2 == 0 && GS == 1) {
                        // packed FP32x2, the same operations in the same order as below:
                        // dW row i, columns (j, j+1); g' rows (i, i+1) from W^H's row pairs
#pragma unroll
                        for (int i = 0; i < B; ++i) {
                            const float2 gi2 = make_float2(gv[i], gv[i]);
#pragma unroll
                            for (int j = 0; j < B; j += 2) {
                                const float2 c = __ffma2_rn(gi2, make_float2(a[j], a[j + 1]),
                                                            make_float2(acc[i][j], acc[i][j + 1]));
                                acc[i][j] = c.x;
                                acc[i][j + 1] = c.y;
                            }
                        }
#pragma unroll
                        for (int ip = 0; ip < B / 2; ++ip) {
                            float2 sum = __fmul2_rn(WH.wp[ip * B], make_float2(gv[0], gv[0]));
#pragma unroll
                            for (int j = 1; j < B; ++j) sum = __ffma2_rn(WH.wp[ip * B + j], make_float2(gv[j], gv[j]), sum);
                            gn[2 * ip] = sum.x;
                            gn[2 * ip + 1] = sum.y;
                        }
                    } else {
#pragma unroll
                        for (int ii = 0; ii < R; ++ii) {
                            const int i = (int)ib * R + ii;
                            const T gi = GS == 1 ? gv[ii] : pick<T, B>(gv, i);
                            // dW[i][j] += g[i] * conj(a[j])
#pragma unroll
                            for (int j = 0; j < B; ++j) acc[ii][j] = fma_acc(gi, a[j], acc[ii][j]);
                            // g'[i] = sum_j W^H[i][j] g[j]
                            T sum = mul(WH.w[i * B], gv[0]);
#pragma unroll
                            for (int j = 1; j < B; ++j) sum = fma_acc(WH.w[i * B + j], gv[j], sum);
                            gn[ii] = sum;
                        }
                    }
                    if (GS > 1) __syncwarp(__activemask());
#pragma unroll
                    for (int ii = 0; ii < R; ++ii) G[pos((int)ib * R + ii)] = gn[ii];
                };
                if (lin) {
                    const uint32_t sb = spos<B>(e0);
                    body([&](int q) { return sb + (uint32_t)q * step; });
                } else {
                    body([&](int q) { return spos<B>(e0 + (uint32_t)q * strideA); });
                }
            }
            __syncthreads();
        }

        if (p.vec_mode != 0) {
            const uint32_t cpr = p.vec_mode == 1 ? tile / CE : r / CE;
            const long long rstride = p.vec_mode == 1 ? 0 : p.L;
            for (uint32_t c = tid; c < tile / CE; c += nth) {
                const uint32_t row = p.vec_mode == 1 ? 0u : p.div_cpr.div(c), cc = c - row * cpr;
                const uint32_t e0 = p.vec_mode == 1 ? c * CE : row * r + cc * CE;
                T v[CE];
#pragma unroll
                for (int i = 0; i < CE; ++i) v[i] = G[spos<B>(e0 + i)];
                store16(grad_in + GTT_CHECKED(base + (long long)row * rstride + cc * CE, p.total - CE + 1, p.err), v);
            }
        } else {
            for (uint32_t e = tid; e < tile; e += nth) {
                const uint32_t row = p.div_r.div(e), col = e - row * r;
                grad_in[GTT_CHECKED(base + (long long)row * p.L + col, p.total, p.err)] = G[spos<B>(e)];
            }
        }
        __syncthreads();
    }

    // CTA reduction of the per-thread partials, fixed order
    T *red = s;  // nth * R * B elements (the host sizes smem for it)
#pragma unroll
    for (int ii = 0; ii < R; ++ii)
#pragma unroll
        for (int j = 0; j < B; ++j) red[(size_t)tid * R * B + ii * B + j] = acc[ii][j];
    __syncthreads();
    for (uint32_t e = tid; e < (uint32_t)(B * B); e += nth) {
        const uint32_t i = e / B, j = e % B, ib = i / R, ii = i % R;
        T sum = zero_<T>();
        for (uint32_t th = ib; th < nth; th += GS) sum = add_(sum, red[(size_t)th * R * B + ii * B + j]);
        dw_part[(size_t)blockIdx.x * B * B + e] = sum;
    }
}

// dW[e] = sum over parts of part[q][e], accumulated in double: one warp per
// entry, lane l adds parts l, l+32, l+64, ... in order, then a fixed butterfly
// combines the lanes, so the result is the same on every run.
constexpr int kDwEntriesPerBlock = 8;  // warps of a 256-thread block

__device__ __forceinline__ double warp_sum_fixed(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__global__ void __launch_bounds__(32 * kDwEntriesPerBlock) gtt_dw_reduce_kernel(const T *parts, int nparts, int bb, T *dW) {
    const int e = blockIdx.x * kDwEntriesPerBlock + (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
    if (e >= bb) return;  // whole warps leave together
    if constexpr (Traits<T>::complex) {
        double re = 0.0, im = 0.0;
        for (int q = lane; q < nparts; q += 32) {
            re += (double)parts[(size_t)q * bb + e].re;
            im += (double)parts[(size_t)q * bb + e].im;
        }
        re = warp_sum_fixed(re);
        im = warp_sum_fixed(im);
        if (lane == 0) {
            T out;
            out.re = (typename Traits<T>::real)re;
            out.im = (typename Traits<T>::real)im;
            dW[e] = out;
        }
    } else {
        double acc = 0.0;
        for (int q = lane; q < nparts; q += 32) acc += (double)parts[(size_t)q * bb + e];
        acc = warp_sum_fixed(acc);
        if (lane == 0) dW[e] = (T)acc;
    }
}

} // namespace gtt
