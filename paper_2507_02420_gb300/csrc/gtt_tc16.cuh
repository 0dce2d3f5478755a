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
// order is at most 2^-16 relative are accumulated in three FP32 partial sums:
//   C0 = x0 W0,  C1 = x0 W1 + x1 W0,  C2 = x0 W2 + x1 W1 + x2 W0,
// computed by three MMAs against the concatenated B operands
//   x0 . [W0|W1|W2] (N = 48), x1 . [W0|W1] (N = 32, into C1 C2), x2 . W0 (N = 16, into C2),
// and y = (C2 + C1) + C0 on readback.  The dropped terms are below 2^-24
// relative, so the result matches FP32 to within a few ulps.
//
// Operands (shared memory, K-major, no swizzle): core matrices of 8 rows x 16
// bytes, the two K-halves 128 bytes apart (leading byte offset) and 8-row
// groups 256 bytes apart (stride byte offset).  One elected thread issues the
// MMAs; tcgen05.commit signals an mbarrier; every wait is bounded.
#pragma once
#include <cuda_bf16.h>

#include "gtt_tma.cuh"

namespace gtt {

constexpr int kTcThreads = 256;
constexpr int kTcTile = 4096;
constexpr uint32_t kTcTmemCols = 128;       // two M blocks x 64 columns (48 used)
constexpr size_t kTcSmemPerCta = 65536;      // two fp32 tiles, three BF16 pieces, W pieces: 3 CTAs/SM

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

__device__ __forceinline__ uint32_t tc_spos(uint32_t e) { return e + (e >> 4); }

__global__ void __launch_bounds__(kTcThreads, 1) gtt_tc16_pass_kernel(const float *in, float *out, TcParams tp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t raw = smem_addr(smem_raw);
    const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
    unsigned char *base = smem_raw + pad;
    float *S0 = reinterpret_cast<float *>(base);                       // two tiles of 4096 + 256 floats
    float *S1 = reinterpret_cast<float *>(base + 17408);
    unsigned char *A = base + 2 * 17408;                               // 3 pieces x 8 KiB
    unsigned char *Bw = A + 3 * 8192;                                  // 1536 bytes
    uint64_t *bar = reinterpret_cast<uint64_t *>(Bw + 1536);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(Bw + 1536 + 8);
    const PassParams &p = tp.p;
    const uint32_t tid = threadIdx.x, warp = tid >> 5;

    for (uint32_t i = tid; i < 1536 / 16; i += kTcThreads)
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
    const uint64_t descB = umma_sdesc(smem_addr(Bw));
    uint32_t phase = 0;
    bool failed = false;

    const uint32_t r = p.r;
    const long long LM = p.L * (long long)p.M;
    const uint32_t m = tid;          // fibre of this thread in every mode
    const uint32_t blk = warp >> 2;  // M block (TMEM column range) of this warp
    const uint32_t lane_base = (warp & 3u) * 32u;

    // asynchronous copy of tile t into the padded buffer Sb (one commit group)
    auto issue_load = [&](long long t, float *Sb) {
        const long long hi = t / p.lo_blocks;
        const uint32_t lob = (uint32_t)(t - hi * p.lo_blocks);
        const long long gb = hi * LM + (long long)lob * r;
        for (uint32_t c = tid; c < kTcTile / 4; c += kTcThreads) {
            // 4 consecutive elements: same row (r in {1, 16, 256}), same 16-element pad group
            const uint32_t e = c * 4, row = p.div_r.div(e), col = e - row * r;
            const float *src = in + gb + (long long)row * p.L + col;
            const uint32_t dst = smem_addr(&Sb[tc_spos(e)]);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst + 4u * i), "l"(src + i) : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };

    int buf = 0;
    if (p.tile_begin + blockIdx.x < p.tiles) issue_load(p.tile_begin + blockIdx.x, S0);
    for (long long t = p.tile_begin + blockIdx.x; t < p.tiles && !failed; t += gridDim.x, buf ^= 1) {
        float *S = buf ? S1 : S0;
        const long long hi = t / p.lo_blocks;
        const uint32_t lob = (uint32_t)(t - hi * p.lo_blocks);
        const long long gbase = hi * LM + (long long)lob * r;
        // prefetch the next tile into the other buffer, then wait for this one
        if (t + gridDim.x < p.tiles) {
            issue_load(t + gridDim.x, buf ? S0 : S1);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();

        for (int d = 3 - tp.g; d < 3; ++d) {
            // this thread's fibre: the other two hex digits (a < c) are m % 16, m / 16
            const int a = d == 0 ? 1 : 0, c = d == 2 ? 1 : 2;
            const uint32_t sd = 1u << (4 * d), sa = 1u << (4 * a), sc = 1u << (4 * c);
            const uint32_t e0 = (m & 15u) * sa + (m >> 4) * sc;
            float v[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] = S[tc_spos(e0 + k * sd)];
            // split into three BF16 pieces, written K-major (two 16-byte rows per piece)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t w0[4], w1[4], w2[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float xa = v[8 * h + 2 * q], xb = v[8 * h + 2 * q + 1];
                    const __nv_bfloat162 p0 = __floats2bfloat162_rn(xa, xb);
                    const float ra = xa - __low2float(p0), rb = xb - __high2float(p0);
                    const __nv_bfloat162 p1 = __floats2bfloat162_rn(ra, rb);
                    const float sa2 = ra - __low2float(p1), sb2 = rb - __high2float(p1);
                    const __nv_bfloat162 p2 = __floats2bfloat162_rn(sa2, sb2);
                    w0[q] = *reinterpret_cast<const uint32_t *>(&p0);
                    w1[q] = *reinterpret_cast<const uint32_t *>(&p1);
                    w2[q] = *reinterpret_cast<const uint32_t *>(&p2);
                }
                const uint32_t off = kmaj_off(m, 8 * h);
                *reinterpret_cast<uint4 *>(A + off) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
                *reinterpret_cast<uint4 *>(A + 8192 + off) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
                *reinterpret_cast<uint4 *>(A + 16384 + off) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
            }
            fence_proxy_async();
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (uint32_t b2 = 0; b2 < 2; ++b2) {
                    const uint32_t dcol = tmem + b2 * 64u;
                    const uint32_t aoff = smem_addr(A) + b2 * 4096u;  // rows 128*b2 .. (16 groups x 256 B)
                    umma_bf16(dcol, umma_sdesc(aoff), descB, umma_idesc(48), 0u);
                    umma_bf16(dcol + 16u, umma_sdesc(aoff + 8192u), descB, umma_idesc(32), 1u);
                    umma_bf16(dcol + 32u, umma_sdesc(aoff + 16384u), descB, umma_idesc(16), 1u);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_addr(bar))
                             : "memory");
            }
            const bool ok = mbar_wait(smem_addr(bar), phase);
            phase ^= 1u;
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            float c0[16], c1[16], c2[16];
            const uint32_t taddr = tmem + (lane_base << 16) + blk * 64u;
            tmem_ld16(taddr, c0);
            tmem_ld16(taddr + 16u, c1);
            tmem_ld16(taddr + 32u, c2);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (d < 2) {
#pragma unroll
                for (int n = 0; n < 16; ++n) S[tc_spos(e0 + n * sd)] = (c2[n] + c1[n]) + c0[n];
            } else {
                // last mode (digit h2): element m + 256 n sits at row (m/r) + n (256/r),
                // column m % r; across a warp the stores are contiguous runs
                const uint32_t rowm = p.div_r.div(m), colm = m - rowm * r;
                const long long stride_n = (long long)(256u / r) * p.L;
                float *o = out + gbase + (long long)rowm * p.L + colm;
#pragma unroll
                for (int n = 0; n < 16; ++n) o[n * stride_n] = (c2[n] + c1[n]) + c0[n];
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
        }
        if (failed) break;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");  // no copy may land after the CTA leaves
    if (failed && tid == 0) atomicExch(tp.err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols));
}

} // namespace gtt
