// FP32 passes with b = 8 on tiles of 4096 elements (four base-8 digits), the
// top G of which a pass transforms; the low 4 - G digits are a run of
// r = 8^(4-G) contiguous elements.  Two kernels share the tile machinery:
//   - gtt_forward_b8_kernel<G>: a forward (or adjoint) pass, Algorithm 1's
//     mode loop (Sec. 3) over the tile's top G digits;
//   - gtt_backward_b8_kernel<G>: the reverse-mode pass (no counterpart in the
//     paper; PyTorch's convention: g_k = W^T applied to digit k of g_{k+1},
//     and dW += sum over the fibres of digit k of g_{k+1}[i] a_k[j]), which
//     computes what gtt_backward_pass_kernel computes for these shapes.
// The tile geometry is fixed at compile time:
//   - element e = d0 + 8 d1 + 64 d2 + 512 d3 of the tile sits in shared
//     memory at bwd8_pos(e) = e ^ 8 ((e >> 6) mod 4) ^ 4 ((e >> 5) mod 2);
//     with one fibre per thread, every access of every digit is free of bank
//     conflicts (digit 0 as two 16-byte loads per fibre, the others as 32-bit
//     accesses whose 32 lanes hit 32 banks), and 16-byte chunks stay whole;
//   - a fibre's 8 offsets are a per-fibre base combined with compile-time
//     constants, so a mode costs no division or multiplication;
//   - the next tile's inputs are loaded with cp.async into a second buffer
//     (pair) while this one is worked on.
// Forward, per tile: each of the G digits in turn, in place, 2 of the 512
// fibres of a digit per thread; the tile is stored as 16-byte chunks.
// Backward, per tile: the activations entering digits 1 .. G-1 of the pass are
// recomputed into shared memory (W applied forward), then the digits are
// walked in reverse, each thread owning 2 of the 512 fibres of a digit:
// dW accumulates in 64 registers per thread across all the CTA's tiles and
// g' = W^T g is written over g in place.  The CTA's 256 partials are summed
// in a fixed order at the end, as in gtt_backward_pass_kernel, so dW is
// bitwise repeatable.
#pragma once
#include "gtt_pass.cuh"

namespace gtt {

constexpr int kBwd8Tile = 4096;
constexpr int kBwd8Threads = 256;

__device__ __forceinline__ uint32_t bwd8_pos(uint32_t e) {
    return e ^ (((e >> 6) & 3u) << 3) ^ (((e >> 5) & 1u) << 2);
}

// Shared memory of the b = 8 backward pass with G transformed digits: two
// activation tiles and two gradient tiles (double-buffered loads) and the
// recomputed activations of digits 1 .. G-1; the final reduction reuses it.
__host__ __device__ constexpr size_t bwd8_smem_bytes(int G) {
    return (size_t)(4 + (G - 1)) * kBwd8Tile * 4 > (size_t)kBwd8Threads * 64 * 4
               ? (size_t)(4 + (G - 1)) * kBwd8Tile * 4
               : (size_t)kBwd8Threads * 64 * 4;
}

// Offsets (in floats) of fibre f of tile digit T: element q of the fibre is
// tile element e0 + q 8^T with e0 = (f / 8^T) 8^(T+1) + f mod 8^T.
//   T = 0: e0 = 8 f; the fibre is two 16-byte chunks, at bwd8_pos(e0) and
//          bwd8_pos(e0 + 4) (returned in off[0], off[4]);
//   T = 1: e0 has bits 3..5 clear, so bwd8_pos(e0 + 8 q) =
//          (e0 ^ 8 ((e0 >> 6) mod 4)) ^ (8 q ^ 4 (q / 4));
//   T = 2: bits 6..8 carry q, bit 5 comes from f: bwd8_pos(e0 + 64 q) =
//          (e0 ^ 4 ((e0 >> 5) mod 2) ^ 8 (q mod 4)) + 64 q;
//   T = 3: bwd8_pos(e0 + 512 q) = bwd8_pos(e0) + 512 q.
template <int T>
__device__ __forceinline__ void bwd8_fibre(uint32_t f, uint32_t (&off)[8]) {
    constexpr uint32_t SH = 3u * T;
    const uint32_t e0 = ((f >> SH) << (SH + 3u)) | (f & ((1u << SH) - 1u));
    if (T == 0) {
        off[0] = bwd8_pos(e0);
        off[4] = bwd8_pos(e0 + 4u);
    } else if (T == 1) {
        const uint32_t base = e0 ^ (((e0 >> 6) & 3u) << 3);
#pragma unroll
        for (uint32_t q = 0; q < 8; ++q) off[q] = base ^ ((q << 3) ^ ((q >> 2) << 2));
    } else if (T == 2) {
        const uint32_t base = e0 ^ (((e0 >> 5) & 1u) << 2);
#pragma unroll
        for (uint32_t q = 0; q < 8; ++q) off[q] = (base ^ ((q & 3u) << 3)) + 64u * q;
    } else {
        const uint32_t base = bwd8_pos(e0);
#pragma unroll
        for (uint32_t q = 0; q < 8; ++q) off[q] = base + 512u * q;
    }
}

template <int T>
__device__ __forceinline__ void bwd8_load(const float *S, const uint32_t (&off)[8], float (&v)[8]) {
    if (T == 0) {
        const float4 lo = *reinterpret_cast<const float4 *>(S + off[0]);
        const float4 hi = *reinterpret_cast<const float4 *>(S + off[4]);
        v[0] = lo.x, v[1] = lo.y, v[2] = lo.z, v[3] = lo.w;
        v[4] = hi.x, v[5] = hi.y, v[6] = hi.z, v[7] = hi.w;
    } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = S[off[q]];
    }
}

template <int T>
__device__ __forceinline__ void bwd8_store(float *S, const uint32_t (&off)[8], const float (&v)[8]) {
    if (T == 0) {
        *reinterpret_cast<float4 *>(S + off[0]) = make_float4(v[0], v[1], v[2], v[3]);
        *reinterpret_cast<float4 *>(S + off[4]) = make_float4(v[4], v[5], v[6], v[7]);
    } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) S[off[q]] = v[q];
    }
}

// y = W x along the fibre (forward recompute): output pairs (i, i+1) from the
// row pairs of W, packed FP32x2, the FMAs in the order j = 0..7
__device__ __forceinline__ void bwd8_forward(const float (&a)[8], float (&y)[8], const WMat<float, 8> &W) {
#pragma unroll
    for (int ip = 0; ip < 4; ++ip) {
        float2 s = __fmul2_rn(W.wp[ip * 8], make_float2(a[0], a[0]));
#pragma unroll
        for (int j = 1; j < 8; ++j) s = __ffma2_rn(W.wp[ip * 8 + j], make_float2(a[j], a[j]), s);
        y[2 * ip] = s.x;
        y[2 * ip + 1] = s.y;
    }
}

// One digit of the reverse sweep for one fibre: dW[i][j] += g[i] a[j], then
// g'[i] = sum_j W^T[i][j] g[j], written over g
template <int T>
__device__ __forceinline__ void bwd8_reverse(const float *A, float *Gs, uint32_t f, float2 (&acc)[8][4],
                                             const WMat<float, 8> &WH) {
    uint32_t off[8];
    bwd8_fibre<T>(f, off);
    float a[8], gv[8], gn[8];
    bwd8_load<T>(A, off, a);
    bwd8_load<T>(Gs, off, gv);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float2 gi2 = make_float2(gv[i], gv[i]);
#pragma unroll
        for (int jp = 0; jp < 4; ++jp) acc[i][jp] = __ffma2_rn(gi2, make_float2(a[2 * jp], a[2 * jp + 1]), acc[i][jp]);
    }
    bwd8_forward(gv, gn, WH);
    bwd8_store<T>(Gs, off, gn);
}

// Forward recompute of one fibre of tile digit T: An = W applied to A.
template <int T>
__device__ __forceinline__ void bwd8_recompute(const float *A, float *An, uint32_t f, const WMat<float, 8> &W) {
    uint32_t off[8];
    bwd8_fibre<T>(f, off);
    float a[8], y[8];
    bwd8_load<T>(A, off, a);
    bwd8_forward(a, y, W);
    bwd8_store<T>(An, off, y);
}

// Forward digits T >= 1 with two fibres per thread: fibres 2p and 2p + 1
// differ in tile digit 0 only, so their elements sit side by side (bwd8_pos
// leaves bit 0 alone) and one 64-bit access serves both: half the
// shared-memory instructions of two single-fibre calls (4 us faster on a
// 4-digit pass of 67 M elements; the backward measured no gain from it).
template <int T>
__device__ __forceinline__ void bwd8_recompute2(const float *A, float *An, uint32_t pr, const WMat<float, 8> &W) {
    static_assert(T >= 1, "pairs differ in tile digit 0");
    uint32_t off[8];
    bwd8_fibre<T>(2u * pr, off);
    float ax[8], ay[8], yx[8], yy[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float2 v = *reinterpret_cast<const float2 *>(A + off[q]);
        ax[q] = v.x, ay[q] = v.y;
    }
    bwd8_forward(ax, yx, W);
    bwd8_forward(ay, yy, W);
#pragma unroll
    for (int q = 0; q < 8; ++q) *reinterpret_cast<float2 *>(An + off[q]) = make_float2(yx[q], yy[q]);
}

// Activation entering the pass's digit K: the loaded tile for K = 0, else the
// recomputed tile K - 1 after the four load buffers.
template <int K> __device__ __forceinline__ float *bwd8_act(float *act0, float *sm) {
    return K == 0 ? act0 : sm + (3 + K) * kBwd8Tile;
}

// The pass's digit k is tile digit 4 - G + k; K runs over the pass's digits.
template <int G, int K>
__device__ __forceinline__ void bwd8_recompute_all(float *act0, float *sm, const WMat<float, 8> &W) {
    if constexpr (K + 1 < G) {
#pragma unroll 1
        for (uint32_t i = 0; i < 2; ++i)
            bwd8_recompute<4 - G + K>(bwd8_act<K>(act0, sm), bwd8_act<K + 1>(act0, sm), threadIdx.x + 256u * i, W);
        __syncthreads();
        bwd8_recompute_all<G, K + 1>(act0, sm, W);
    }
}

template <int G, int K>
__device__ __forceinline__ void bwd8_reverse_all(float *act0, float *sm, float *Gs, float2 (&acc)[8][4],
                                                 const WMat<float, 8> &WH) {
    if constexpr (K >= 0) {
#pragma unroll 1
        for (uint32_t i = 0; i < 2; ++i)
            bwd8_reverse<4 - G + K>(bwd8_act<K>(act0, sm), Gs, threadIdx.x + 256u * i, acc, WH);
        __syncthreads();
        bwd8_reverse_all<G, K - 1>(act0, sm, Gs, acc, WH);
    }
}

template <int G>
__global__ void __launch_bounds__(kBwd8Threads, 2)
gtt_backward_b8_kernel(const float *act_in, const float *grad_out, float *grad_in, float *dw_part, PassParams p,
                       int g_unused, WMat<float, 8> W, WMat<float, 8> WH) {
    (void)g_unused;
    constexpr uint32_t kLogR = 3u * (4u - G);  // run length r = 8^(4-G)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *sm = reinterpret_cast<float *>(smem_raw);
    // [act 0][act 1][grad 0][grad 1][a_1 .. a_{G-1}]
    auto actb = [&](int s) { return sm + s * kBwd8Tile; };
    auto gradb = [&](int s) { return sm + (2 + s) * kBwd8Tile; };
    const uint32_t tid = threadIdx.x;
    const long long LM = p.L * (long long)p.M;

    float2 acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int jp = 0; jp < 4; ++jp) acc[i][jp] = make_float2(0.f, 0.f);

    auto tile_base = [&](long long t) {
        const long long hi = t / p.lo_blocks;
        const uint32_t lob = (uint32_t)(t - hi * p.lo_blocks);
        return hi * LM + ((long long)lob << kLogR);
    };
    // global offset of the 16-byte chunk c of a tile: rows of r elements at stride L
    auto chunk_off = [&](long long gb, uint32_t c) {
        const uint32_t e = 4u * c;
        return gb + (long long)(e >> kLogR) * p.L + (e & ((1u << kLogR) - 1u));
    };
    auto issue_load = [&](long long t, int s) {
        if (t < p.tiles) {
            const long long gb = tile_base(t);
#pragma unroll
            for (int i = 0; i < kBwd8Tile / 4 / kBwd8Threads; ++i) {
                const uint32_t c = tid + (uint32_t)i * kBwd8Threads;
                const long long go = GTT_CHECKED(chunk_off(gb, c), p.total - 3, p.err);
                const uint32_t so = GTT_CHECKED(bwd8_pos(4u * c), kBwd8Tile - 3, p.err);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(actb(s) + so)),
                             "l"(act_in + go)
                             : "memory");
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(gradb(s) + so)),
                             "l"(grad_out + go)
                             : "memory");
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };

    const long long step = gridDim.x;
    int s = 0;
    issue_load(p.tile_begin + blockIdx.x, 0);
    for (long long t = p.tile_begin + blockIdx.x; t < p.tiles; t += step) {
        issue_load(t + step, s ^ 1);                          // the next tile, into the other pair
        asm volatile("cp.async.wait_group 1;" ::: "memory");  // this tile's copies are complete
        __syncthreads();
        bwd8_recompute_all<G, 0>(actb(s), sm, W);
        bwd8_reverse_all<G, G - 1>(actb(s), sm, gradb(s), acc, WH);
        // the input gradient of this tile, back to global memory
        const long long gb = tile_base(t);
#pragma unroll
        for (int i = 0; i < kBwd8Tile / 4 / kBwd8Threads; ++i) {
            const uint32_t c = tid + (uint32_t)i * kBwd8Threads;
            const float4 v = *reinterpret_cast<const float4 *>(gradb(s) + bwd8_pos(4u * c));
            *reinterpret_cast<float4 *>(grad_in + GTT_CHECKED(chunk_off(gb, c), p.total - 3, p.err)) = v;
        }
        __syncthreads();  // the pair is read before the load two tiles ahead lands in it
        s ^= 1;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();

    // CTA reduction of the per-thread partials, fixed order (thread 0 first)
    float *red = sm;  // 256 x 64 floats
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int jp = 0; jp < 4; ++jp)
            *reinterpret_cast<float2 *>(red + (size_t)tid * 64 + i * 8 + 2 * jp) = acc[i][jp];
    __syncthreads();
    if (tid < 64) {
        float sum = 0.f;
        for (uint32_t th = 0; th < kBwd8Threads; ++th) sum += red[(size_t)th * 64 + tid];
        dw_part[(size_t)blockIdx.x * 64 + tid] = sum;
    }
}

// Shared memory of the b = 8 forward pass: the tile and the next one.
constexpr size_t kFwd8Smem = 2 * kBwd8Tile * 4;

// Tile digits LO .. LO + G - 1 in turn, in place.
template <int G, int LO, int K>
__device__ __forceinline__ void fwd8_digits(float *S, const WMat<float, 8> &W) {
    if constexpr (K < G) {
        if constexpr (LO + K >= 1)
            bwd8_recompute2<LO + K>(S, S, threadIdx.x, W);
        else
#pragma unroll 1
            for (uint32_t i = 0; i < 2; ++i) bwd8_recompute<LO + K>(S, S, threadIdx.x + 256u * i, W);
        __syncthreads();
        fwd8_digits<G, LO, K + 1>(S, W);
    }
}

// y = W applied to G digits of every tile (the adjoint passes W^H): the top G
// tile digits over runs of 8^(4-G) elements (BOT = false; G = 4 only on the
// first pass, whose tiles are contiguous: the 16-byte chunk copies need runs
// of at least 4 elements), or, on the first
// pass, the bottom G digits of 8^(4-G) consecutive blocks of 8^G elements
// (BOT = true: a contiguous 4096-element tile).  In place is allowed: a tile
// is read whole before it is written, and tiles are disjoint.
template <int G, bool BOT>
__global__ void __launch_bounds__(kBwd8Threads, 4) gtt_forward_b8_kernel(const float *in, float *out, PassParams p,
                                                                         WMat<float, 8> W) {
    constexpr uint32_t kLogR = BOT ? 0u : 3u * (4u - G);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *sm = reinterpret_cast<float *>(smem_raw);
    const uint32_t tid = threadIdx.x;
    const long long LM = p.L * (long long)p.M;
    auto tile_base = [&](long long t) {
        if (BOT) return t * (long long)kBwd8Tile;  // contiguous tiles
        const long long hi = t / p.lo_blocks;
        const uint32_t lob = (uint32_t)(t - hi * p.lo_blocks);
        return hi * LM + ((long long)lob << kLogR);
    };
    auto chunk_off = [&](long long gb, uint32_t c) {
        const uint32_t e = 4u * c;
        if (BOT) return gb + (long long)e;
        return gb + (long long)(e >> kLogR) * p.L + (e & ((1u << kLogR) - 1u));
    };
    auto issue_load = [&](long long t, int s) {
        if (t < p.tiles) {
            const long long gb = tile_base(t);
#pragma unroll
            for (int i = 0; i < kBwd8Tile / 4 / kBwd8Threads; ++i) {
                const uint32_t c = tid + (uint32_t)i * kBwd8Threads;
                const long long go = GTT_CHECKED(chunk_off(gb, c), p.total - 3, p.err);
                const uint32_t so = GTT_CHECKED(bwd8_pos(4u * c), kBwd8Tile - 3, p.err);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                                 (uint32_t)__cvta_generic_to_shared(sm + s * kBwd8Tile + so)),
                             "l"(in + go)
                             : "memory");
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    const long long step = gridDim.x;
    int s = 0;
    issue_load(p.tile_begin + blockIdx.x, 0);
    for (long long t = p.tile_begin + blockIdx.x; t < p.tiles; t += step) {
        issue_load(t + step, s ^ 1);
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        __syncthreads();
        float *S = sm + s * kBwd8Tile;
        fwd8_digits<G, BOT ? 0 : 4 - G, 0>(S, W);
        const long long gb = tile_base(t);
#pragma unroll
        for (int i = 0; i < kBwd8Tile / 4 / kBwd8Threads; ++i) {
            const uint32_t c = tid + (uint32_t)i * kBwd8Threads;
            const float4 v = *reinterpret_cast<const float4 *>(S + bwd8_pos(4u * c));
            *reinterpret_cast<float4 *>(out + GTT_CHECKED(chunk_off(gb, c), p.total - 3, p.err)) = v;
        }
        __syncthreads();  // the buffer is read before the load two tiles ahead lands in it
        s ^= 1;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
}

} // namespace gtt
