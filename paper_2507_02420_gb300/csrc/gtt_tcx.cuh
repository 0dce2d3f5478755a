// Complex (complex64) mode passes of the fast GTT for b = 4 on the
// 5th-generation tensor cores: pairs of base-4 digits act as one base-16
// digit, transformed with the 16 x 16 matrix W (x) W (Def. 2.3: the Kronecker
// power factors over any grouping of adjacent digits), and each such mode of
// Algorithm 1 (Sec. 3) is the contraction Y = X (W (x) W)^T over the fibres of
// the digit pair.
//
// Complex arithmetic as real: a fibre of 16 complex values is a row of 32
// interleaved reals x[2l + c], and the 16 x 16 complex M becomes the 32 x 32
// real R with R[2j][2l] = R[2j+1][2l+1] = Re M[j][l], R[2j][2l+1] = -Im M[j][l],
// R[2j+1][2l] = Im M[j][l], so y = R x gives the interleaved output.
//
// Precision (TF32, three products): x = x0 + x1 with x0 = x truncated to TF32
// (the low 13 mantissa bits cleared) and x1 = x - x0 (exact in FP32; the tensor
// core reads it as TF32), R = R0 + R1 with TF32 pieces rounded on the host.  The
// accumulator holds x0 R0^T + x1 R0^T in columns 0..31 and x0 R1^T in 32..63;
// y is their FP32 sum.  Per mode the result is within about 2^-20 of FP32.
//
// A tile is 4096 complex (32 KiB); a cluster of four CTAs (one per SM) holds
// four tiles that differ in one more base-4 digit, the cluster digit.  A pass
// covers 7 digits (contiguous: digits 0..5 in the tile, digit 6 across the
// cluster) or 6 digits (strided: digits m0..m0+4 in the tile -- two base-16
// modes and one base-4 digit on CUDA cores -- and digit m0+5 across the
// cluster) in one HBM round trip.
//
// Work of a CTA (one CTA per SM: a cluster launch of a kernel that allocates
// tensor memory gets one CTA per SM): 16 warps in two slots of 8; a slot takes
// every other tile of the CTA's list.  For its tile a slot
//   1. runs the base-16 modes as two M = 128 groups of 128 fibres, each group
//      with its own tensor-memory columns (the A operand of the MMA comes from
//      tensor memory), MMA issue and completion barrier: a thread reads its
//      fibre from the tile, writes the two pieces to tensor memory
//      (tcgen05.st), the group's leader issues 4 + 4 MMAs (K = 8) against
//      [R0 ; R1] in shared memory, and each thread reads its accumulator row
//      back (tcgen05.ld) and writes y to the tile in place;
//   2. sends the tile's quarter q (after the last mode, or after the base-4
//      digit of strided tiles) to CTA q of the cluster with asynchronous
//      distributed-shared-memory stores (st.async) that complete on CTA q's
//      exchange-buffer barrier;
//   3. refills its tile buffer with the tile three ahead (TMA for contiguous
//      tiles, 16-byte cp.async copies into a bank-spread layout for strided
//      ones);
//   4. once all four CTAs' quarters of the tile have arrived in this CTA's
//      exchange buffer, applies W to the cluster digit on CUDA cores, writes
//      the results to global memory, and tells all four CTAs that the buffer
//      is free again.
// Every wait is bounded.  An expired wait raises the plan's error flag and sets
// the CTA's abort flag; the CTA then skips its work but still makes its
// arrivals (never more than a barrier phase expects), so its peers never wait
// for it, and leaves through the final cluster barrier.
#pragma once
#include <cuda.h>

#include "gtt_tma.cuh"

namespace gtt {

constexpr int kTcxTile = 4096;                     // complex elements per CTA tile
constexpr uint32_t kTcxTileBytes = kTcxTile * 8;   // 32 KiB
constexpr int kTcxCluster = 4;
constexpr uint32_t kTcxBBytes = 64 * 32 * 4;       // [R0 ; R1]: 64 rows x 32 TF32, K-major

struct TcxParams {
    long long ctiles;          // cluster tiles of this launch
    // strided geometry (digits m0 .. m0+5): element = hi*stride_hi + top*stride_top + row*L + lo
    long long L, stride_top, stride_hi;
    uint32_t lo_runs;          // L / 4: runs of 4 consecutive low indices
    FastDiv div_lo_runs;
    const float *bmat;         // [R0 ; R1] in the K-major core-matrix layout (kTcxBBytes)
    float2 wa[16], wb[16];     // W (or W^H) of the base-4 digits on CUDA cores: (re, re) and (-im, im)
    int *err;
};

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ uint64_t tcx_bdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(128u >> 4) << 16;   // leading byte offset: next core matrix along K
    d |= (uint64_t)(1024u >> 4) << 32;  // stride byte offset: next 8-row group (8 core matrices along K = 32)
    d |= (uint64_t)1 << 46;             // descriptor version for tcgen05
    return d;
}
// instruction descriptor: FP32 accumulate, TF32 A and B, both K-major, M = 128
__host__ __device__ constexpr uint32_t tcx_idesc(int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
// D (tensor memory) += A (tensor memory) * B (shared memory)^T
__device__ __forceinline__ void tcx_mma(uint32_t d, uint32_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
                 "r"(a), "l"(b), "r"(id), "r"(acc)
                 : "memory");
}
__device__ __forceinline__ void tcx_st32(uint32_t taddr, const uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]),
        "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]),
        "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
        : "memory");
}
__device__ __forceinline__ void tcx_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
          "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
}
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_id_x() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_count_x() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}
// every thread of every CTA of the cluster; orders shared-memory writes before
// the barrier with reads after it, across the cluster
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t map_to_rank(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}
__device__ __forceinline__ float4 ld_cluster_f4(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr)
                 : "memory");
    return v;
}
// Strided tiles: 1024 rows of 4 complex (32 bytes); 16-byte chunk (row, cp)
// (cp = column pair) is stored at chunk (2 row + cp) ^ g(row) with g taking
// bits 2 ^ 6, 4 and 5 of the row into chunk bits 0, 1 and 2.  The fibres of
// both base-16 modes (row bits 0-3 and 4-7) and the 16-byte row accesses of
// the base-4 digit (row bits 8-9) then reach every bank evenly.
__device__ __forceinline__ uint32_t sx_chunk(uint32_t row, uint32_t cp) {
    const uint32_t g = (((row >> 2) ^ (row >> 6)) & 1u) | (((row >> 4) & 3u) << 1);
    return (2u * row + cp) ^ g;
}

// acc += w * x (complex), with w given as the pairs (re, re) and (-im, im)
__device__ __forceinline__ float2 cmac(float2 acc, float2 wa, float2 wb, float2 x) {
    acc = __ffma2_rn(wa, x, acc);
    return __ffma2_rn(wb, make_float2(x.y, x.x), acc);
}

// The TF32 two-piece split of a fibre and its tensor-memory store (A0, A1).
__device__ __forceinline__ void tcx_store_pieces(uint32_t trow, uint32_t colA0, const float (&v)[32]) {
    uint32_t t0[32], t1[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const uint32_t u = __float_as_uint(v[k]) & 0xFFFFE000u;
        t0[k] = u;
        t1[k] = __float_as_uint(v[k] - __uint_as_float(u));
    }
    tcx_st32(trow + colA0, t0);
    tcx_st32(trow + colA0 + 32u, t1);
}


constexpr int kTcxSlots = 2;                       // tiles in flight per CTA
constexpr int kTcxBlock = kTcxSlots * 256;         // 16 warps: 4 per scheduler, up to 128 registers
constexpr int kTcxNbS = 3;                         // tile buffers per CTA
constexpr int kTcxNbX = 3;                         // exchange buffers per CTA (4 x 8 KiB each)
constexpr uint32_t kTcxTmemCols = 512;             // 4 groups x (A0 32 + A1 32 + D 64)
constexpr int kTcxBars = kTcxNbS + 2 * kTcxNbX + 4;

__host__ __device__ constexpr size_t tcx_smem_bytes() {
    return (size_t)(kTcxNbS + kTcxNbX) * kTcxTileBytes + kTcxBBytes + 8 * kTcxBars + 16 + 1024;
}

// named barriers: 1, 2 = the 256 threads of a slot; 3..6 = the 128 threads of a group
__device__ __forceinline__ void slot_sync(uint32_t slot) {
    if (slot == 0)
        asm volatile("bar.sync 1, 256;" ::: "memory");
    else
        asm volatile("bar.sync 2, 256;" ::: "memory");
}
__device__ __forceinline__ void group_sync(uint32_t gi) {
    switch (gi) {
    case 0: asm volatile("bar.sync 3, 128;" ::: "memory"); break;
    case 1: asm volatile("bar.sync 4, 128;" ::: "memory"); break;
    case 2: asm volatile("bar.sync 5, 128;" ::: "memory"); break;
    default: asm volatile("bar.sync 6, 128;" ::: "memory"); break;
    }
}

// Arrive (release, cluster scope) on the mbarrier at the same shared offset in
// CTA `rank` of the cluster.
__device__ __forceinline__ void remote_arrive(uint32_t bar_local, uint32_t rank) {
    const uint32_t r = map_to_rank(bar_local, rank);
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(r) : "memory");
}
// Bounded wait with acquire at cluster scope (arrivals made by other CTAs).
__device__ __forceinline__ bool mbar_wait_cluster(uint32_t bar, uint32_t parity, volatile int *abort) {
    for (uint32_t i = 0; i < kSpinLimit; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((i & 255u) == 255u && *abort) return false;
    }
    return false;
}
// 16 bytes to the shared memory of another CTA of the cluster (addr and bar are
// cluster addresses); the transfer completes on that CTA's mbarrier.
__device__ __forceinline__ void st_async16(uint32_t addr, float4 v, uint32_t bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(addr),
                 "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(bar)
                 : "memory");
}

// Per-thread state of a tensor-core mode.
struct TcxMode {
    uint32_t tmem, trow, colA0, colD, mma_bar, gi, tt;
    uint64_t bdesc;
    int *err;  // the plan's status word (bounds checks of the debug build)
};

// Float offset, in a contiguous tile, of element kk of this thread's fibre in
// base-16 mode MODE (rows of 16 complex in the 128B swizzle; tile element
// e = d0 + 16 d1 + 256 d2; the thread's fibre is fixed by tt).
template <int MODE> __device__ __forceinline__ uint32_t contig_off(uint32_t tt, int kk) {
    uint32_t s, c2;
    if (MODE == 0) {
        s = tt;
        c2 = (uint32_t)kk;
    } else if (MODE == 1) {
        s = (uint32_t)kk + 16u * (tt >> 4);
        c2 = tt & 15u;
    } else {
        s = (tt >> 4) + 16u * (uint32_t)kk;
        c2 = tt & 15u;
    }
    return 2u * (s * 16u + ((((c2 >> 1) ^ s) & 7u) << 1) + (c2 & 1u));
}
// Float offset, in a strided tile, of element kk of this thread's fibre in mode MODE (row bits 4 MODE .. 4 MODE + 3).
template <int MODE> __device__ __forceinline__ uint32_t strided_off(uint32_t tt, int kk) {
    const uint32_t col = tt & 3u;
    const uint32_t row = MODE == 0 ? (uint32_t)kk + 16u * (tt >> 2) : ((tt >> 2) & 15u) + 16u * (uint32_t)kk + 256u * (tt >> 6);
    return 2u * (sx_chunk(row, col >> 1) * 2u + (col & 1u));
}

// One base-16 mode on this thread's fibre: read it from the tile, run the MMAs
// of its group, and return y in v.  Returns false if the CTA is aborting.
template <bool CONTIG, int MODE>
__device__ __forceinline__ void tcx_mode_mma(const TcxMode &c, const float *S, float (&v)[32], uint32_t &mma_phase,
                                             bool &ok, volatile int *abort_flag) {
    const bool run = ok && !*abort_flag;
    if (run) {
        if (CONTIG && MODE == 0) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float4 t = *reinterpret_cast<const float4 *>(S + 4u * (c.tt * 8u + ((uint32_t)q ^ (c.tt & 7u))));
                v[4 * q] = t.x, v[4 * q + 1] = t.y, v[4 * q + 2] = t.z, v[4 * q + 3] = t.w;
            }
        } else {
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
                const float2 t = *reinterpret_cast<const float2 *>(
                    S + GTT_CHECKED(CONTIG ? contig_off<MODE>(c.tt, kk) : strided_off<MODE>(c.tt, kk), 2 * kTcxTile - 1, c.err));
                v[2 * kk] = t.x, v[2 * kk + 1] = t.y;
            }
        }
        tcx_store_pieces(c.trow, c.colA0, v);
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    group_sync(c.gi);
    if ((c.tt & 127u) == 0 && ok && !*abort_flag) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a0 = c.tmem + c.colA0, d = c.tmem + c.colD;
#pragma unroll
        for (uint32_t s = 0; s < 4; ++s)  // x0 [R0 | R1]^T into D[0:64]
            tcx_mma(d, a0 + 8u * s, c.bdesc + ((256u * s) >> 4), tcx_idesc(64), s > 0);
#pragma unroll
        for (uint32_t s = 0; s < 4; ++s)  // + x1 R0^T into D[0:32]
            tcx_mma(d, a0 + 32u + 8u * s, c.bdesc + ((256u * s) >> 4), tcx_idesc(32), 1u);
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(c.mma_bar)
                     : "memory");
    }
    if (ok && !*abort_flag && !mbar_wait_or_abort(c.mma_bar, mma_phase, abort_flag)) {
        ok = false;
        *abort_flag = 1;
    }
    mma_phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok && !*abort_flag) {
        uint32_t c0[32], c1[32];
        tcx_ld32(c.trow + c.colD, c0);
        tcx_ld32(c.trow + c.colD + 32u, c1);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int kk = 0; kk < 32; kk += 2) {
            const float2 sum = __fadd2_rn(make_float2(__uint_as_float(c0[kk]), __uint_as_float(c0[kk + 1])),
                                          make_float2(__uint_as_float(c1[kk]), __uint_as_float(c1[kk + 1])));
            v[kk] = sum.x, v[kk + 1] = sum.y;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
// Write y of this thread's fibre back to the tile (mode MODE's positions).
template <bool CONTIG, int MODE>
__device__ __forceinline__ void tcx_write_back(uint32_t tt, float *S, const float (&v)[32], int *err) {
    if (CONTIG && MODE == 0) {
#pragma unroll
        for (int q = 0; q < 8; ++q)
            *reinterpret_cast<float4 *>(S + 4u * (tt * 8u + ((uint32_t)q ^ (tt & 7u)))) =
                make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else {
#pragma unroll
        for (int kk = 0; kk < 16; ++kk)
            *reinterpret_cast<float2 *>(S + GTT_CHECKED(CONTIG ? contig_off<MODE>(tt, kk) : strided_off<MODE>(tt, kk),
                                                        2 * kTcxTile - 1, err)) = make_float2(v[2 * kk], v[2 * kk + 1]);
    }
}

template <bool CONTIG>
__global__ void __cluster_dims__(kTcxCluster, 1, 1) __launch_bounds__(kTcxBlock, 1)
gtt_tcx_pass_kernel(const __grid_constant__ CUtensorMap tin, const float2 *in, float2 *out, const TcxParams p) {
    constexpr int NBS = kTcxNbS, NBX = kTcxNbX;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t raw = smem_addr(smem_raw);
    const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
    unsigned char *base = smem_raw + pad;
    const uint32_t base_s = raw + pad;
    float *ring = reinterpret_cast<float *>(base);                      // tile buffers
    const uint32_t xring = base_s + NBS * kTcxTileBytes;                // exchange buffers: [src 4][1024 complex]
    float *Bs = reinterpret_cast<float *>(base + (NBS + NBX) * kTcxTileBytes);
    const uint32_t bars = base_s + (NBS + NBX) * kTcxTileBytes + kTcxBBytes;
    const uint32_t sfull = bars, xfull = bars + 8u * NBS, xfree = xfull + 8u * NBX, mmab = xfree + 8u * NBX;
    unsigned char *flags = base + (NBS + NBX) * kTcxTileBytes + kTcxBBytes + 8 * kTcxBars;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(flags);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(flags + 8);
    const uint32_t tid = threadIdx.x, warp = tid >> 5;
    const uint32_t rank = cluster_rank(), cid = cluster_id_x(), ncl = cluster_count_x();
    const long long my_tiles = (long long)cid < p.ctiles ? (p.ctiles - 1 - cid) / ncl + 1 : 0;
    const uint32_t slot = warp >> 3, gi = warp >> 2, tt = tid & 255u;

    for (uint32_t i = tid; i < kTcxBBytes / 16; i += kTcxBlock)
        reinterpret_cast<int4 *>(Bs)[i] = reinterpret_cast<const int4 *>(p.bmat)[i];
    if (tid == 0) {
        for (int i = 0; i < NBS; ++i) mbar_init(sfull + 8u * i, CONTIG ? 1u : 256u);
        for (int i = 0; i < NBX; ++i) {
            mbar_init(xfull + 8u * i, 1);
            mbar_init(xfree + 8u * i, kTcxCluster);
        }
        for (int i = 0; i < 4; ++i) mbar_init(mmab + 8u * i, 1);
        *abort_flag = 0;
        fence_mbar_init();
        // the first NBX tiles' exchange buffers expect 4 x 8 KiB each
        for (int i = 0; i < NBX && i < my_tiles; ++i) mbar_expect_tx(xfull + 8u * i, kTcxTileBytes);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"(kTcxTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_proxy_async();  // B written by the generic proxy, read by the tensor core
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // every CTA of the cluster has started (its barriers exist) before any remote access
    cluster_sync_all();

    bool ok = true;
    auto live = [&]() { return ok && !*abort_flag; };
    auto fail = [&]() {
        ok = false;
        *abort_flag = 1;
    };
    // strided tiles: origin of the tile of cluster tile ct with cluster digit `top`
    auto strided_origin = [&](long long ct, uint32_t top) -> long long {
        const long long hi = ct / p.lo_runs;
        const uint32_t j = (uint32_t)(ct - hi * (long long)p.lo_runs);
        return hi * p.stride_hi + (long long)top * p.stride_top + 4ll * j;
    };
    // load tile k into buffer k mod NBS: TMA by tt 0 of the calling slot, or
    // 8 cp.async per thread of the slot (one arrival per thread on sfull)
    auto load_tile = [&](long long k, bool whole_cta) {
        const int buf = (int)(k % NBS);
        const uint32_t bar = sfull + 8u * buf;
        const long long ct = cid + k * (long long)ncl;
        if constexpr (CONTIG) {
            if ((whole_cta ? tid : tt) == 0) {
                if (live()) {
                    fence_proxy_async();  // earlier generic accesses to the buffer before the TMA write
                    mbar_expect_tx(bar, kTcxTileBytes);
                    tma_load_2d(base_s + buf * kTcxTileBytes, &tin, bar, 0, (int)((4 * ct + rank) * 256));
                } else {
                    mbar_arrive(bar);  // nothing is loaded: release the waiting slot
                }
            }
        } else {
            if (!whole_cta || tid < 256u) {
                const uint32_t t = whole_cta ? tid : tt;
                if (live()) {
                    const float2 *src = in + strided_origin(ct, rank);
                    const uint32_t dst0 = base_s + buf * kTcxTileBytes;
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const uint32_t q = t + 256u * (uint32_t)i, row = q >> 1, cp = q & 1u;
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst0 + sx_chunk(row, cp) * 16u),
                                     "l"(src + (long long)row * p.L + 2 * cp)
                                     : "memory");
                    }
                }
                asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
            }
        }
    };
    for (long long k = 0; k < NBS && k < my_tiles; ++k) load_tile(k, true);

    TcxMode mc;
    mc.tmem = *tmem_slot;
    mc.trow = mc.tmem + (((warp & 3u) * 32u) << 16);  // this thread's lane
    mc.colA0 = gi * 128u;
    mc.colD = mc.colA0 + 64u;
    mc.mma_bar = mmab + 8u * gi;
    mc.gi = gi;
    mc.tt = tt;
    mc.bdesc = tcx_bdesc(smem_addr(Bs));
    mc.err = p.err;
    uint32_t mma_phase = 0;

    for (long long k = slot; k < my_tiles; k += kTcxSlots) {
        const int buf = (int)(k % NBS), bx = (int)(k % NBX);
        float *S = ring + buf * (kTcxTileBytes / 4);
        const long long ct = cid + k * (long long)ncl;
        if (live() && !mbar_wait_or_abort(sfull + 8u * buf, (uint32_t)((k / NBS) & 1), abort_flag)) fail();
        slot_sync(slot);
        // ---- base-16 modes; the exchange buffers of tile k (our slot `rank` in
        // CTA h's buffer bx) are free once every CTA has consumed tile k - NBX
        auto wait_xfree = [&]() {
            if (k >= NBX && live() && !mbar_wait_cluster(xfree + 8u * bx, (uint32_t)(((k / NBX) - 1) & 1), abort_flag))
                fail();
        };
        auto xdst = [&](uint32_t h, uint32_t idx) {  // cluster address of complex idx of our slot in CTA h
            return map_to_rank(xring + bx * kTcxTileBytes + (rank * 1024u + idx) * 8u, h);
        };
        float v[32];
        if constexpr (CONTIG) {
            tcx_mode_mma<true, 0>(mc, S, v, mma_phase, ok, abort_flag);
            if (live()) tcx_write_back<true, 0>(tt, S, v, p.err);
            slot_sync(slot);
            tcx_mode_mma<true, 1>(mc, S, v, mma_phase, ok, abort_flag);
            if (live()) tcx_write_back<true, 1>(tt, S, v, p.err);
            slot_sync(slot);
            tcx_mode_mma<true, 2>(mc, S, v, mma_phase, ok, abort_flag);
            wait_xfree();
            if (live()) {
                // y[d2], d2 = 0..15, of position tt + 256 d2: quarter d2 / 4 goes to CTA d2 / 4
                // as complex 4 tt .. 4 tt + 3 of our slot
#pragma unroll
                for (uint32_t h = 0; h < 4; ++h) {
                    const uint32_t dst = xdst(h, 4u * tt), bar = map_to_rank(xfull + 8u * bx, h);
                    st_async16(dst, make_float4(v[8 * h], v[8 * h + 1], v[8 * h + 2], v[8 * h + 3]), bar);
                    st_async16(dst + 16u, make_float4(v[8 * h + 4], v[8 * h + 5], v[8 * h + 6], v[8 * h + 7]), bar);
                }
            }
        } else {
            tcx_mode_mma<false, 0>(mc, S, v, mma_phase, ok, abort_flag);
            if (live()) tcx_write_back<false, 0>(tt, S, v, p.err);
            slot_sync(slot);
            tcx_mode_mma<false, 1>(mc, S, v, mma_phase, ok, abort_flag);
            if (live()) tcx_write_back<false, 1>(tt, S, v, p.err);
            slot_sync(slot);
            // the base-4 digit of row bits 8-9 on CUDA cores; output row tt + 256 o goes to
            // CTA o as complex 4 tt .. 4 tt + 3 of our slot
            wait_xfree();
            if (live()) {
                float4 x[4][2];
#pragma unroll
                for (int h = 0; h < 4; ++h)
#pragma unroll
                    for (uint32_t cp = 0; cp < 2; ++cp)
                        x[h][cp] = *reinterpret_cast<const float4 *>(S + 4u * sx_chunk(tt + 256u * h, cp));
#pragma unroll
                for (uint32_t o = 0; o < 4; ++o) {
                    float2 a[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) a[i] = make_float2(0.f, 0.f);
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const float2 wa = p.wa[o * 4 + h], wb = p.wb[o * 4 + h];
                        a[0] = cmac(a[0], wa, wb, make_float2(x[h][0].x, x[h][0].y));
                        a[1] = cmac(a[1], wa, wb, make_float2(x[h][0].z, x[h][0].w));
                        a[2] = cmac(a[2], wa, wb, make_float2(x[h][1].x, x[h][1].y));
                        a[3] = cmac(a[3], wa, wb, make_float2(x[h][1].z, x[h][1].w));
                    }
                    const uint32_t dst = xdst(o, 4u * tt), bar = map_to_rank(xfull + 8u * bx, o);
                    st_async16(dst, make_float4(a[0].x, a[0].y, a[1].x, a[1].y), bar);
                    st_async16(dst + 16u, make_float4(a[2].x, a[2].y, a[3].x, a[3].y), bar);
                }
            }
        }
        // ---- the tile buffer is no longer read: refill it with tile k + NBS
        slot_sync(slot);
        if (k + NBS < my_tiles) load_tile(k + NBS, false);
        // ---- the cluster digit: wait for the four quarters of tile k in our exchange buffer
        bool landed = false;
        if (live()) {
            landed = mbar_wait_or_abort(xfull + 8u * bx, (uint32_t)((k / NBX) & 1), abort_flag);
            if (!landed) fail();
        }
        if (live()) {
            const float *X = reinterpret_cast<const float *>(base + (NBS + bx) * kTcxTileBytes);
            const uint32_t m = tt;  // complex 4 m .. 4 m + 3 of every source slot h (source CTA h: cluster digit h)
            float4 x[4][2];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                x[h][0] = *reinterpret_cast<const float4 *>(X + (h * 1024u + 4u * m) * 2u);
                x[h][1] = *reinterpret_cast<const float4 *>(X + (h * 1024u + 4u * m) * 2u + 4u);
            }
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                float2 a[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = make_float2(0.f, 0.f);
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const float2 wa = p.wa[o * 4 + h], wb = p.wb[o * 4 + h];
                    a[0] = cmac(a[0], wa, wb, make_float2(x[h][0].x, x[h][0].y));
                    a[1] = cmac(a[1], wa, wb, make_float2(x[h][0].z, x[h][0].w));
                    a[2] = cmac(a[2], wa, wb, make_float2(x[h][1].x, x[h][1].y));
                    a[3] = cmac(a[3], wa, wb, make_float2(x[h][1].z, x[h][1].w));
                }
                if constexpr (CONTIG) {
                    // complex j of the group: position m + 256 (4 rank + j) of tile o
                    float2 *dst = out + GTT_CHECKED(ct * (long long)(4 * kTcxTile) + (long long)o * kTcxTile + 1024ll * rank + m,
                                                    p.ctiles * 4 * kTcxTile - 768, p.err);
#pragma unroll
                    for (int j = 0; j < 4; ++j) dst[256 * j] = a[j];
                } else {
                    // row 256 rank + m, columns 0..3, cluster digit o
                    float2 *dst = out + GTT_CHECKED(strided_origin(ct, (uint32_t)o) + (long long)(256u * rank + m) * p.L,
                                                    p.ctiles * 4 * kTcxTile - 3, p.err);
                    reinterpret_cast<float4 *>(dst)[0] = make_float4(a[0].x, a[0].y, a[1].x, a[1].y);
                    reinterpret_cast<float4 *>(dst)[1] = make_float4(a[2].x, a[2].y, a[3].x, a[3].y);
                }
            }
        }
        slot_sync(slot);  // every thread of the slot is done with the exchange buffer
        if (tt == 0) {
            // the arrival for tile k + NBX (never onto a phase that did not complete)
            if (landed && k + NBX < my_tiles) mbar_expect_tx(xfull + 8u * bx, kTcxTileBytes);
#pragma unroll
            for (uint32_t h = 0; h < (uint32_t)kTcxCluster; ++h) remote_arrive(xfree + 8u * bx, h);
        }
    }
    if (!ok && tt == 0) atomicExch(p.err, 1);
    // no copy may land after the CTA leaves: the last load into each tile buffer has completed
    if constexpr (CONTIG) {
        if (tid == 0)
            for (long long k = my_tiles > NBS ? my_tiles - NBS : 0; k < my_tiles; ++k)
                mbar_wait(sfull + 8u * (uint32_t)(k % NBS), (uint32_t)((k / NBS) & 1));
    } else {
        asm volatile("cp.async.wait_all;" ::: "memory");
    }
    // every CTA of the cluster is done with the others' buffers and barriers before any exits
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    cluster_sync_all();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(mc.tmem), "r"(kTcxTmemCols));
}

} // namespace gtt
