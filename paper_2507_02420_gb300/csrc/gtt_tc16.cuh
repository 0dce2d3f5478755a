// b = 16 mode passes on the 5th-generation tensor cores (tcgen05), FP32 data,
// BF16 products of 3-piece splits accumulated in FP32 in tensor memory.
//
// Each mode of Algorithm 1 (Sec. 3) with b = 16 is the contraction
// Y = X W^T over the mode's digit: for every fibre m, y_m[n] = sum_k W[n][k] x_m[k].
// A tile holds 4096 FP32 elements, i.e. three base-16 digits (h0, h1, h2); the
// pass transforms the top g of them (the rest is a run of r = 16^(3-g)
// contiguous elements).  Per mode, the 256 fibres of the tile are the MMA's
// M dimension (two M = 128 blocks), the digit is K = 16, and W gives N.
//
// Precision: x = x0 + x1 + x2 and W = W0 + W1 + W2 with BF16 pieces
// (round-to-nearest splits of the FP32 residuals).  The six products whose
// order is at most 2^-16 relative are accumulated in two FP32 partial sums:
//   C0 = x0 W0,  C12 = x0 W1 + x0 W2 + x1 W0 + x1 W1 + x2 W0,
// and y = C12 + C0 on readback.  The x pieces go to tensor memory
// (tcgen05.st, two BF16 per column; the MMA reads A from there) and B is
// [W0|W1|W2] in shared memory: x0 [W0|W1] (N = 32) starts C0 and C12, and
// four N = 16 MMAs add the other terms to C12.  The tensor core adds each
// MMA's sum into its FP32 accumulator with truncation; C12 is about 2^-8 of
// y, so that costs at most about 2^-29 of y per mode.  The dropped terms are
// below 2^-24 relative, so the result matches FP32 to within a few ulps.
// The two-piece variant (NP = 2: x = x0 + x1, W = W0 + W1, products x0 W0,
// x0 W1, x1 W0 into C0 and C1, y = C1 + C0) leaves the x residual and x1 W1,
// about 2^-16 relative per mode: the cheaper, less accurate reading of "bf16x3"
// (BF16X2 in the C ABI), kept for the precision comparison.
// The TF32 variant (NP = 0, TF32X3 in the C ABI): x = x0 + x1 with x0 = x
// rounded to TF32 (to nearest on the bit pattern) and x1 = x - x0, W = W0 + W1
// (TF32 pieces rounded on the host); the two A pieces go to tensor memory
// (tcgen05.st; the MMA reads A from there), and x0 [W0|W1] (N = 32) plus
// x1 W0 (N = 16) accumulate C0 and C1, y = C1 + C0.  About 2^-21 relative per
// mode: fewer instructions per element than the BF16 splits, within 1e-6.
//
// Shared-memory operands (K-major, no swizzle): core matrices of 8 rows x 16
// bytes, the two K-halves 128 bytes apart (leading byte offset) and 8-row
// groups 256 bytes apart (stride byte offset).  Only BF16X2 keeps its A pieces
// there; the other variants hold A in tensor memory.  One elected thread issues the
// MMAs; tcgen05.commit signals an mbarrier; every wait is bounded.
#pragma once
#include <cuda_bf16.h>

#include "gtt_tma.cuh"

namespace gtt {

constexpr int kTcThreads = 256;
constexpr int kTcTile = 4096;
constexpr int kTcBufs = 3;                   // tile ring: the tile in work and two prefetched
constexpr uint32_t kTcTileBytes = kTcTile * 4;
constexpr uint32_t kTcTmemCols = 128;        // two M blocks x 64 columns
constexpr uint32_t kTcPieceBytes = 8192;     // one BF16 piece of the A operand: 256 rows x 16
constexpr uint32_t kTcWBytes = 2048;         // B operand: 48 rows x 16 BF16 (1536 bytes), or 32 rows x 16 TF32
constexpr uint32_t kTcWBf16Bytes = 1536, kTcWTf32Bytes = 2048;
// ring, A pieces (BF16X2; the others keep A in tensor memory), B
// operand, mbarrier + TMEM slot, and slack for 128-byte alignment
__host__ __device__ constexpr size_t tc_smem_per_cta(int np) {
    return kTcBufs * kTcTileBytes + (np == 2 ? 2 * kTcPieceBytes : 0) + kTcWBytes + 16 + 128;
}
constexpr size_t kTcSmemPerCta = tc_smem_per_cta(3);

struct TcParams {
    PassParams p;              // tile geometry: tile_elems = 4096, r = 16^(3-g)
    int g;                     // transformed digits: the top g of the tile's three
    const unsigned char *wpieces;  // 48 rows x 16 BF16 (W0, W1, W2 rows), K-major core-matrix layout
    int *err;
};

__device__ __forceinline__ uint64_t umma_sdesc(uint32_t saddr_bytes) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr_bytes & 0x3FFFF) >> 4);
    d |= (uint64_t)(128u >> 4) << 16;  // leading byte offset: next core matrix along K
    d |= (uint64_t)(256u >> 4) << 32;  // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;            // descriptor version for tcgen05
    return d;
}

// instruction descriptor: FP32 accumulate, BF16 A and B, both K-major, M = 128
__host__ __device__ constexpr uint32_t umma_idesc(int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                     d_tmem),
                 "l"(a), "l"(b), "r"(idesc), "r"(acc)
                 : "memory");
}

// K-major TF32 B operand (32 rows x 16): core matrices of 8 rows x 16 bytes,
// K-neighbours 128 bytes apart, 8-row groups 512 bytes apart
__device__ __forceinline__ uint64_t umma_sdesc_tf32(uint32_t saddr_bytes) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr_bytes & 0x3FFFF) >> 4);
    d |= (uint64_t)(128u >> 4) << 16;
    d |= (uint64_t)(512u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}
__host__ __device__ constexpr uint32_t umma_idesc_tf32(int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
// D (tensor memory) += A (tensor memory) * B (shared memory)^T, BF16
__device__ __forceinline__ void umma_bf16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(
                     d_tmem),
                 "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
                 : "memory");
}
// D (tensor memory) += A (tensor memory) * B (shared memory)^T, TF32
__device__ __forceinline__ void umma_tf32_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(
                     d_tmem),
                 "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
                 : "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(v[0]),
                 "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// byte offset of element (row m, k) in a K-major core-matrix operand
__device__ __forceinline__ uint32_t kmaj_off(uint32_t m, uint32_t k) {
    return (m >> 3) * 256u + (k >> 3) * 128u + (m & 7u) * 16u + (k & 7u) * 2u;
}

// Tile buffer layout.  Element (h2, h1, h0) of a tile sits at float index
//   256 h2 + 16 R + 4 ((h0 / 4) ^ (R / 2 mod 4)) + h0 mod 4,   R = h1 ^ (h2 mod 2):
// rows of 16 are swapped in pairs on odd h2 and their 4-float chunks XOR-permuted.
// Every 16-byte chunk of the tile stays 16 contiguous bytes (so the global
// loads are 16-byte copies), and the fibres of all three modes are read and
// written without bank conflicts: mode 0 (along h0) as 4 x 128-bit accesses
// per thread, modes 1 and 2 as 32-bit accesses whose 32 lanes hit 32 banks.
__device__ __forceinline__ uint32_t tc_pos(uint32_t h2, uint32_t h1, uint32_t h0) {
    const uint32_t R = h1 ^ (h2 & 1u);
    return h2 * 256u + R * 16u + ((((h0 >> 2) ^ (R >> 1)) & 3u) << 2) + (h0 & 3u);
}

// Float offsets of the 16 elements of fibre m for mode D (the fibre runs along
// digit D; m enumerates the other two digits, lower digit first).  For D = 0
// only off[0], off[4], off[8], off[12] are used: the starts of 4 chunks.
template <int D>
__device__ __forceinline__ void tc_fibre(uint32_t m, uint32_t (&off)[16]) {
    if (D == 0) {
        const uint32_t h1 = m & 15u, h2 = m >> 4;
#pragma unroll
        for (int k = 0; k < 16; ++k) off[k] = tc_pos(h2, h1, (uint32_t)k);
    } else if (D == 1) {
        // with p = h2 mod 2: 16 (k ^ p) = 16 k + 16 p for even k and 16 k - 16 p
        // for odd k, and the chunk term depends on k / 2 mod 4 only
        const uint32_t h0 = m & 15u, h2 = m >> 4, p = h2 & 1u, c = h0 >> 2;
        const uint32_t be = h2 * 256u + 16u * p + (h0 & 3u), bo = h2 * 256u - 16u * p + (h0 & 3u);
#pragma unroll
        for (int k = 0; k < 16; ++k)
            off[k] = ((k & 1) ? bo : be) + 16u * (uint32_t)k + ((c ^ ((uint32_t)(k >> 1) & 3u)) << 2);
    } else {
        // R = h1 ^ (k mod 2); the chunk term uses R / 2 = h1 / 2 for both parities
        const uint32_t h0 = m & 15u, h1 = m >> 4, c = h0 >> 2;
        const uint32_t chunk = ((c ^ (h1 >> 1)) & 3u) << 2;
        const uint32_t pe = 16u * h1 + chunk + (h0 & 3u), po = 16u * (h1 ^ 1u) + chunk + (h0 & 3u);
#pragma unroll
        for (int k = 0; k < 16; ++k) off[k] = ((k & 1) ? po : pe) + 256u * (uint32_t)k;
    }
}

struct TcCtx {
    uint32_t colA0 = 0;    // TF32 variant: A0 column offset within the thread's M block (A1 at +16)
    uint32_t m;            // fibre of this thread (= row of the A operand)
    uint32_t tmem;         // base of the TMEM allocation (lane 0, first column)
    uint32_t tmem_row;     // this thread's accumulator row: its lane, its M block's columns
    uint32_t a_smem, bar;  // A operand pieces and the MMA-completion mbarrier (shared addresses)
    uint64_t descB;
    unsigned char *A;
};

// One mode of the tile in S: read fibre m, split it into three BF16 pieces
// (the A operand), run the BF16x3 MMAs into TMEM, and write y_m back to S
// (D < 2) or, for the last mode, straight to global memory at o[n * stride_n].
// Returns false in a thread whose wait for the MMA completion timed out.
template <int D, int NP>
__device__ __forceinline__ bool tc_mode(const TcCtx &c, float *S, uint32_t &phase, float *o, long long stride_n) {
    uint32_t off[16];
    tc_fibre<D>(c.m, off);
    float v[16];
    if (D == 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 t = *reinterpret_cast<const float4 *>(S + off[4 * q]);
            v[4 * q] = t.x, v[4 * q + 1] = t.y, v[4 * q + 2] = t.z, v[4 * q + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = S[off[k]];
    }
    // split into pieces: TF32 (NP = 0) into tensor memory, BF16 K-major into
    // shared memory; residuals x - piece are exact
    const float2 neg1 = make_float2(-1.f, -1.f);
    if constexpr (NP == 0) {
        uint32_t t0[16], t1[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const uint32_t u = (__float_as_uint(v[k]) + 0x1000u) & 0xFFFFE000u;  // to nearest TF32
            t0[k] = u;
            t1[k] = __float_as_uint(v[k] - __uint_as_float(u));
        }
        tmem_st16(c.tmem_row + c.colA0, t0);
        tmem_st16(c.tmem_row + c.colA0 + 16u, t1);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    uint32_t pc[3][8];  // NP = 3: the pieces as packed BF16 pairs, k = 2j (low half) and 2j + 1
#pragma unroll
    for (int h = 0; h < (NP == 0 ? 0 : 2); ++h) {
        uint32_t w0[4], w1[4], w2[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float2 x = make_float2(v[8 * h + 2 * q], v[8 * h + 2 * q + 1]);
            const __nv_bfloat162 p0 = __floats2bfloat162_rn(x.x, x.y);
            const uint32_t u0 = *reinterpret_cast<const uint32_t *>(&p0);
            const float2 r1 = __ffma2_rn(make_float2(__uint_as_float(u0 << 16), __uint_as_float(u0 & 0xFFFF0000u)), neg1, x);
            const __nv_bfloat162 p1 = __floats2bfloat162_rn(r1.x, r1.y);
            const uint32_t u1 = *reinterpret_cast<const uint32_t *>(&p1);
            const float2 r2 = __ffma2_rn(make_float2(__uint_as_float(u1 << 16), __uint_as_float(u1 & 0xFFFF0000u)), neg1, r1);
            const __nv_bfloat162 p2 = __floats2bfloat162_rn(r2.x, r2.y);
            w0[q] = u0;
            w1[q] = u1;
            w2[q] = *reinterpret_cast<const uint32_t *>(&p2);
        }
        if (NP == 3) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                pc[0][4 * h + q] = w0[q];
                pc[1][4 * h + q] = w1[q];
                pc[2][4 * h + q] = w2[q];
            }
        } else {
            const uint32_t ko = kmaj_off(c.m, 8 * h);
            *reinterpret_cast<uint4 *>(c.A + ko) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
            *reinterpret_cast<uint4 *>(c.A + kTcPieceBytes + ko) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
        }
    }
    if (NP == 3) {  // pieces p in columns 8p .. 8p + 7 of the thread's row (two BF16 per column)
        tmem_st8(c.tmem_row, pc[0]);
        tmem_st8(c.tmem_row + 8u, pc[1]);
        tmem_st8(c.tmem_row + 16u, pc[2]);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    if (NP == 2) fence_proxy_async();  // generic-proxy writes of A, visible to the tensor core
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (uint32_t b2 = 0; b2 < 2; ++b2) {
            const uint32_t dcol = c.tmem + b2 * 64u;
            const uint32_t aoff = c.a_smem + b2 * 4096u;  // rows 128 b2 .. (16 groups x 256 B)
            if (NP == 0) {
                // M block b2: A0 in columns 64 b2 .. +15, A1 in +16 .. +31, D in +32 .. +63
                const uint32_t a0 = c.tmem + b2 * 64u, d = a0 + 32u;
#pragma unroll
                for (uint32_t s = 0; s < 2; ++s)  // x0 [W0|W1]^T into D[0:32]
                    umma_tf32_ts(d, a0 + 8u * s, c.descB + ((256u * s) >> 4), umma_idesc_tf32(32), s > 0);
#pragma unroll
                for (uint32_t s = 0; s < 2; ++s)  // + x1 W0^T into D[0:16]
                    umma_tf32_ts(d, a0 + 16u + 8u * s, c.descB + ((256u * s) >> 4), umma_idesc_tf32(16), 1u);
            } else if (NP == 3) {
                // M block b2: pieces x0, x1, x2 in columns 64 b2 + 0, 8, 16; C0 in
                // +32 .. +47, C12 in +48 .. +63.  B rows 16p .. 16p + 15 hold W_p
                // (8-row groups 256 bytes apart: W_p starts 512 p bytes in).
                const uint32_t a0 = c.tmem + b2 * 64u, d = a0 + 32u;
                umma_bf16_ts(d, a0, c.descB, umma_idesc(32), 0u);                              // x0 [W0|W1]
                umma_bf16_ts(d + 16u, a0, c.descB + (1024u >> 4), umma_idesc(16), 1u);         // + x0 W2
                umma_bf16_ts(d + 16u, a0 + 8u, c.descB, umma_idesc(16), 1u);                   // + x1 W0
                umma_bf16_ts(d + 16u, a0 + 8u, c.descB + (512u >> 4), umma_idesc(16), 1u);     // + x1 W1
                umma_bf16_ts(d + 16u, a0 + 16u, c.descB, umma_idesc(16), 1u);                  // + x2 W0
            } else {
                umma_bf16(dcol, umma_sdesc(aoff), c.descB, umma_idesc(32), 0u);
                umma_bf16(dcol + 16u, umma_sdesc(aoff + kTcPieceBytes), c.descB, umma_idesc(16), 1u);
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(c.bar)
                     : "memory");
    }
    // every thread waits for the MMAs itself; an expired wait is voted on at the
    // next tile's barrier (the CTA then stops), so no barrier is needed here
    const bool ok = mbar_wait(c.bar, phase);
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    float c0[16], c1[16];
    const uint32_t drow = c.tmem_row + (NP == 2 ? 0u : 32u);  // this thread's accumulator row
    tmem_ld16(drow, c0);
    tmem_ld16(drow + 16u, c1);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    float y[16];
#pragma unroll
    for (int n = 0; n < 16; n += 2) {
        const float2 s = __fadd2_rn(make_float2(c1[n], c1[n + 1]), make_float2(c0[n], c0[n + 1]));
        y[n] = s.x, y[n + 1] = s.y;
    }
    if (D == 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            *reinterpret_cast<float4 *>(S + off[4 * q]) = make_float4(y[4 * q], y[4 * q + 1], y[4 * q + 2], y[4 * q + 3]);
    } else if (D == 1) {
#pragma unroll
        for (int n = 0; n < 16; ++n) S[off[n]] = y[n];
    } else {
#pragma unroll
        for (int n = 0; n < 16; ++n) o[n * stride_n] = y[n];
    }
    // the next mode issues MMAs into the same TMEM columns only after its own
    // barrier, which every thread reaches after finishing these loads
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    // y_m in S, visible to the next mode.  Mode 0 -> mode 1 stays inside a
    // warp: element (h2, h1, h0) is written by thread h1 + 16 h2 and read by
    // thread h0 + 16 h2, both in warp h2 / 2.  Mode 1 -> mode 2 crosses warps.
    if (D == 0) __syncwarp();
    if (D == 1) __syncthreads();
    return ok;
}

// Pass over tiles of three base-16 digits whose top G are transformed (G = 3:
// contiguous tiles of the first pass; G = 2, 1: runs of r = 16, 256 elements).
template <int G, int NP>
__global__ void __launch_bounds__(kTcThreads, 3) gtt_tc16_pass_kernel(const float *in, float *out, TcParams tp) {
    constexpr uint32_t kLogR = 4u * (3u - G);  // run length r = 16^(3-G)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t raw = smem_addr(smem_raw);
    unsigned char *base = smem_raw + ((128u - (raw & 127u)) & 127u);
    float *ring = reinterpret_cast<float *>(base);
    unsigned char *A = base + kTcBufs * kTcTileBytes;
    unsigned char *Bw = A + (NP == 2 ? 2 * kTcPieceBytes : 0);
    uint64_t *bar = reinterpret_cast<uint64_t *>(Bw + kTcWBytes);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(Bw + kTcWBytes + 8);
    const PassParams &p = tp.p;
    const uint32_t tid = threadIdx.x, warp = tid >> 5;

    for (uint32_t i = tid; i < kTcWBytes / 16; i += kTcThreads)
        reinterpret_cast<int4 *>(Bw)[i] = reinterpret_cast<const int4 *>(tp.wpieces)[i];
    if (tid == 0) {
        mbar_init(smem_addr(bar), 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"(kTcTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    TcCtx c;
    c.m = tid;  // fibre of this thread in every mode; warp w reads TMEM lanes 32 (w mod 4) ..
    c.tmem = tmem;
    c.tmem_row = tmem + (((warp & 3u) * 32u) << 16) + (warp >> 2) * 64u;
    c.a_smem = smem_addr(A);
    c.bar = smem_addr(bar);
    c.descB = NP == 0 ? umma_sdesc_tf32(smem_addr(Bw)) : umma_sdesc(smem_addr(Bw));
    c.A = A;
    uint32_t phase = 0;
    bool failed = false, bad = false;

    const long long LM = p.L * (long long)p.M;
    const long long G0 = p.tile_begin + blockIdx.x, step = gridDim.x;
    auto tile_base = [&](long long t) {
        const long long hi = t / p.lo_blocks;
        const uint32_t lob = (uint32_t)(t - hi * p.lo_blocks);
        return hi * LM + ((long long)lob << kLogR);
    };
    // 16-byte copies of tile t into ring slot s (one commit group, empty past the end)
    auto issue_load = [&](long long t, int s) {
        if (t < p.tiles) {
            const long long gb = tile_base(t);
            float *Sb = ring + s * kTcTile;
#pragma unroll
            for (int i = 0; i < kTcTile / 4 / kTcThreads; ++i) {
                const uint32_t cc = tid + (uint32_t)i * kTcThreads, e = cc * 4u;
                const uint32_t row = e >> kLogR, col = e & ((1u << kLogR) - 1u);
                const float *src = in + GTT_CHECKED(gb + (long long)row * p.L + col, p.total - 3, tp.err);
                const uint32_t dst = smem_addr(Sb + GTT_CHECKED(tc_pos(cc >> 6, (cc >> 2) & 15u, (cc & 3u) * 4u), kTcTile - 3, tp.err));
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };

    // last mode: element m + 256 n of the tile is row m / r + n (256 / r), column m mod r
    const uint32_t rowm = c.m >> kLogR, colm = c.m & ((1u << kLogR) - 1u);
    const long long stride_n = (long long)(256u >> kLogR) * p.L;
    issue_load(G0, 0);
    issue_load(G0 + step, 1);
    int slot = 0;
    for (long long t = G0; t < p.tiles; t += step) {
        issue_load(t + 2 * step, slot == 0 ? 2 : slot - 1);
        asm volatile("cp.async.wait_group 2;" ::: "memory");  // tile t's group is complete
        if (__syncthreads_or(bad)) {  // uniform: an MMA wait of the last tile expired somewhere
            failed = true;
            break;
        }
        float *S = ring + slot * kTcTile;
        float *o = out + tile_base(t) + (long long)rowm * p.L + colm;
#ifdef GTT_DEBUG
        long long stride_o = stride_n;
        if (tile_base(t) + (long long)rowm * p.L + colm + 15 * stride_n >= p.total) {  // last-mode stores stay inside
            atomicOr(tp.err, 2);
            o = out;
            stride_o = 0;
        }
#define stride_n stride_o
#endif
        if (G == 3) bad |= !tc_mode<0, NP>(c, S, phase, o, stride_n);
        if (G >= 2) bad |= !tc_mode<1, NP>(c, S, phase, o, stride_n);
        bad |= !tc_mode<2, NP>(c, S, phase, o, stride_n);
#ifdef GTT_DEBUG
#undef stride_n
#endif
        slot = slot == 2 ? 0 : slot + 1;
    }
    if (!failed && __syncthreads_or(bad)) failed = true;  // the last tile's vote
    asm volatile("cp.async.wait_all;" ::: "memory");  // no copy may land after the CTA leaves
    if (failed && tid == 0) atomicExch(tp.err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols));
}

} // namespace gtt
