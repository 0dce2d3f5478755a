// TMA-pipelined pass of the fast GTT (Sec. 3, Algorithm 1: a group of modes
// applied in one HBM round trip; same tile geometry as gtt_pass_kernel).
//
// Persistent CTAs walk their tiles through a ring of `nbuf` shared-memory
// buffers.  The CTA is kTmaThreads compute threads plus one producer warp.
// The producer's lane 0 issues the tensor-memory-accelerator copies: a
// cp.async.bulk.tensor load per buffer (completion counted on the buffer's
// "full" mbarrier), and, once every compute thread has arrived on the
// buffer's "empty" mbarrier, the cp.async.bulk.tensor store of the finished
// tile, then (when the store has read the buffer) the load of the tile nbuf
// ahead.  The compute threads never wait for a copy other than their next
// tile's load, and synchronise their register stages on a named barrier that
// the producer does not take part in.
//
// Shared-memory layout: rows of 128 bytes in the TMA 128B swizzle (16-byte
// chunk c of row s sits at chunk c ^ (s & 7)); every buffer is 1024-byte
// aligned.  A tile is either contiguous (the first pass: its M elements are
// M*es/128 consecutive rows) or strided (M rows of r elements, r*es a
// multiple of 128: column block cb of 128 bytes occupies rows
// [cb*M, cb*M + M)).  The swizzle makes both the row-wise accesses of the
// lowest digits and the column-wise accesses of higher digits conflict-free.
//
// Every mbarrier wait is bounded (kSpinLimit polls); on expiry the kernel
// records the error in p.err, drains its own copies and returns.
#pragma once
#include <cuda.h>

#include "gtt_pass.cuh"

namespace gtt {

constexpr int kTmaThreads = 256;               // compute threads
constexpr int kTmaBlock = kTmaThreads + 32;     // plus the producer warp
constexpr int kTmaMaxBuf = 4;
// shared memory past the tile ring: full and empty mbarriers, the abort flag
constexpr int kTmaBarBytes = 16 * kTmaMaxBuf + 16;
constexpr uint32_t kSpinLimit = 1u << 24;

// CTAs per SM the register allocation is sized for: three when the register
// window is small (<= 16 elements, <= 128 bytes of data per thread, b <= 8),
// else one.
__host__ __device__ constexpr int tma_min_blocks(int es, int B, int D) {
    return (B <= 8 && cpow(B, D) <= 16 && cpow(B, D) * es <= 128) ? 3 : 1;
}

constexpr int kTmaXorStages = 8;  // stages that can use the table-driven address form

struct TmaParams {
    long long tiles;          // end of this launch's tile range
    long long tile_begin;     // first tile of this launch's range
    uint32_t M, r, tile_elems, lo_blocks, tile_bytes;
    uint32_t rows_per_box;    // rows per TMA box (<= 256)
    uint32_t boxes_per_cb;    // boxes per column block
    uint32_t cbs;             // column blocks (strided); 1 for contiguous tiles
    uint32_t units_per_elem;  // tensor-map units per element (2 for 16-byte types)
    int nbuf;
    FastDiv div_lo_blocks, div_r;
    int nstages;
    int stage_mask[kMaxStages];
    uint32_t stage_Ba[kMaxStages];  // b^a of the stage's window start a
    FastDiv stage_divBa[kMaxStages];
    int stage_addr[kMaxStages];       // address form of the stage (kAddr*)
    uint32_t stage_stride[kMaxStages];  // bytes between register elements (kAddrStride)
    uint32_t stage_fq[kTmaXorStages][16];  // swizzled offset of register element q (kAddrXor)
    int *err;  // device flag: 1 = an mbarrier wait expired
};

// How a stage's register elements map to swizzled shared memory (chosen on
// the host from the tile geometry):
//   kAddrGeneral  any layout: the full swizzle formula per element;
//   kAddrStride   the swizzle phase (row mod 8) and the byte in the row are the
//                 same for every element: a fixed byte stride;
//   kAddrRowXor   element q sits q rows after a row that is a multiple of 8, at
//                 the same byte: the 16-byte chunk index is XORed with q mod 8;
//   kAddrXor      any power-of-two geometry: the byte offset of a tile element
//                 is a GF(2)-linear function F of its index bits (bit moves and
//                 the 128B-swizzle XOR), and the window base and q * Ba occupy
//                 disjoint bits, so offset(q) = F(base) ^ F(q * Ba), with the
//                 second term tabulated per stage on the host (stage_fq).
constexpr int kAddrGeneral = 0, kAddrStride = 1, kAddrRowXor = 2, kAddrXor = 3;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait; returns false if the phase did not complete in time.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t i = 0; i < kSpinLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(dst), "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(dst), "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, uint32_t src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%2, %3}], [%1];" ::"l"((uint64_t)map),
                 "r"(src), "r"(x), "r"(y)
                 : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, uint32_t src, int x, int y, int z) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"((uint64_t)map),
                 "r"(src), "r"(x), "r"(y), "r"(z)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// Bounded wait that also gives up once *abort is set by another thread.
__device__ __forceinline__ bool mbar_wait_or_abort(uint32_t bar, uint32_t parity, volatile int *abort) {
    for (uint32_t i = 0; i < kSpinLimit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255u) == 255u && *abort) return false;
    }
    return false;
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// barrier 1 over the compute threads only
__device__ __forceinline__ void compute_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kTmaThreads) : "memory"); }
// barrier 1 over the compute threads, returning whether any of them passed true
__device__ __forceinline__ bool compute_any(bool v) {
    uint32_t r;
    asm volatile("{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
                 : "=r"(r)
                 : "r"((uint32_t)v), "n"(kTmaThreads)
                 : "memory");
    return r != 0;
}

// Byte offset of (swizzle row s, byte ccb within the row's 128 bytes).
__device__ __forceinline__ uint32_t swz(uint32_t s, uint32_t ccb) {
    return (s << 7) + ((((ccb >> 4) ^ s) & 7u) << 4) + (ccb & 15u);
}

template <typename T, bool CONTIG> struct TmaTile {
    static constexpr uint32_t ES = sizeof(T);
    static constexpr uint32_t R128 = 128 / ES;  // elements per 128-byte row
    // byte offset of tile element (row, col)
    __device__ __forceinline__ static uint32_t off(uint32_t row, uint32_t col, uint32_t M) {
        if constexpr (CONTIG) {
            return swz(row / R128, (row % R128) * ES);
        } else {
            return swz((col / R128) * M + row, (col % R128) * ES);
        }
    }
};

template <typename T, int B, int D, bool CONTIG>
__global__ void __launch_bounds__(kTmaBlock, tma_min_blocks((int)sizeof(T), B, D))
gtt_tma_pass_kernel(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tout,
                    TmaParams p, WMat<T, B> W) {
    constexpr int RB = cpow(B, D);
    constexpr int CE = 16 / (int)sizeof(T);
    using Tile = TmaTile<T, CONTIG>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t raw = smem_addr(smem_raw);
    const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
    unsigned char *sbase = smem_raw + pad;              // generic pointer, 1024-aligned in shared space
    const uint32_t sbase_s = raw + pad;                  // shared-window address of the same byte
    const uint32_t full = sbase_s + (uint32_t)p.nbuf * p.tile_bytes;  // nbuf mbarriers: tile loaded
    const uint32_t empty = full + 8u * kTmaMaxBuf;                    // nbuf mbarriers: tile computed
    volatile int *abort_flag = reinterpret_cast<volatile int *>(sbase + (size_t)p.nbuf * p.tile_bytes + 16 * kTmaMaxBuf);

    const uint32_t tid = threadIdx.x;
    const long long range = p.tiles - p.tile_begin;
    const long long my_tiles = blockIdx.x < range ? (range - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (tid == 0) {
        for (int i = 0; i < p.nbuf; ++i) {
            mbar_init(full + 8u * i, 1);
            mbar_init(empty + 8u * i, kTmaThreads);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();

    if (tid >= (uint32_t)kTmaThreads) {
        // ---- producer warp: lane 0 issues every copy of this CTA ----
        if (tid == (uint32_t)kTmaThreads) {
            auto issue_load = [&](long long j) {
                const long long t = p.tile_begin + blockIdx.x + j * (long long)gridDim.x;
                const int buf = (int)(j % p.nbuf);
                const uint32_t bar = full + 8u * buf;
                const uint32_t dst = sbase_s + (uint32_t)buf * p.tile_bytes;
                mbar_expect_tx(bar, p.tile_bytes);
                if constexpr (CONTIG) {
                    const long long row0 = t * (long long)(p.tile_bytes >> 7);
                    for (uint32_t k = 0; k < p.boxes_per_cb; ++k)
                        tma_load_2d(dst + k * p.rows_per_box * 128u, &tin, bar, 0,
                                    (int)(row0 + (long long)k * p.rows_per_box));
                } else {
                    const long long hi = t / p.lo_blocks;
                    const uint32_t lob = (uint32_t)(t - hi * p.lo_blocks);
                    for (uint32_t cb = 0; cb < p.cbs; ++cb)
                        for (uint32_t k = 0; k < p.boxes_per_cb; ++k) {
                            const int x = (int)((lob * p.r + cb * Tile::R128) * p.units_per_elem);
                            tma_load_3d(dst + (cb * p.M + k * p.rows_per_box) * 128u, &tin, bar, x,
                                        (int)(k * p.rows_per_box), (int)hi);
                        }
                }
            };
            auto issue_store = [&](long long j) {
                const long long t = p.tile_begin + blockIdx.x + j * (long long)gridDim.x;
                const uint32_t src = sbase_s + (uint32_t)(j % p.nbuf) * p.tile_bytes;
                if constexpr (CONTIG) {
                    const long long row0 = t * (long long)(p.tile_bytes >> 7);
                    for (uint32_t k = 0; k < p.boxes_per_cb; ++k)
                        tma_store_2d(&tout, src + k * p.rows_per_box * 128u, 0,
                                     (int)(row0 + (long long)k * p.rows_per_box));
                } else {
                    const long long hi = t / p.lo_blocks;
                    const uint32_t lob = (uint32_t)(t - hi * p.lo_blocks);
                    for (uint32_t cb = 0; cb < p.cbs; ++cb)
                        for (uint32_t k = 0; k < p.boxes_per_cb; ++k) {
                            const int x = (int)((lob * p.r + cb * Tile::R128) * p.units_per_elem);
                            tma_store_3d(&tout, src + (cb * p.M + k * p.rows_per_box) * 128u, x,
                                         (int)(k * p.rows_per_box), (int)hi);
                        }
                }
                bulk_commit();
            };
            long long issued = 0;
            for (; issued < my_tiles && issued < p.nbuf; ++issued) issue_load(issued);
            bool failed = false;
            for (long long i = 0; i < my_tiles; ++i) {
                const int buf = (int)(i % p.nbuf);
                if (!mbar_wait_or_abort(empty + 8u * buf, (uint32_t)((i / p.nbuf) & 1), abort_flag)) {
                    failed = true;
                    break;
                }
                issue_store(i);
                if (i + p.nbuf < my_tiles) {
                    bulk_wait_read_all();  // the store has read the buffer: refill it
                    issue_load(i + p.nbuf);
                    ++issued;
                }
            }
            if (failed) {
                atomicExch(p.err, 1);
                *abort_flag = 1;
                // the last load issued into each buffer must land before the CTA leaves
                for (long long j = issued > p.nbuf ? issued - p.nbuf : 0; j < issued; ++j)
                    mbar_wait(full + 8u * (uint32_t)(j % p.nbuf), (uint32_t)((j / p.nbuf) & 1));
            }
            bulk_wait_all();
        }
    } else {
        // ---- compute threads: register stages on the tile in the buffer ----
        const uint32_t nth = kTmaThreads;
        for (long long i = 0; i < my_tiles; ++i) {
            const int buf = (int)(i % p.nbuf);
            const bool ok = mbar_wait_or_abort(full + 8u * buf, (uint32_t)((i / p.nbuf) & 1), abort_flag);
            if (compute_any(!ok)) {  // uniform over the compute threads
                if (tid == 0) {
                    atomicExch(p.err, 1);
                    *abort_flag = 1;
                }
                break;
            }
            unsigned char *tb = sbase + (size_t)buf * p.tile_bytes;
            // byte offset of an element of T in the tile, checked in the debug build
#define TB(off) GTT_CHECKED(off, p.tile_bytes - sizeof(T) + 1, p.err)

            const uint32_t nslots = p.tile_elems / RB;
            for (int st = 0; st < p.nstages; ++st) {
                const uint32_t Ba = p.stage_Ba[st];
                const int mask = p.stage_mask[st];
                for (uint32_t slot = tid; slot < nslots; slot += nth) {
                    const uint32_t rest = p.div_r.div(slot);
                    const uint32_t col = slot - rest * p.r;
                    const uint32_t high = p.stage_divBa[st].div(rest);
                    const uint32_t low = rest - high * Ba;
                    const uint32_t row0 = low + high * Ba * RB;
                    T v[RB];
                    if constexpr (CONTIG && (RB % CE == 0)) {
                        if (Ba == 1) {  // the window holds the lowest digits: 16-byte chunks
#pragma unroll
                            for (int q = 0; q < RB; q += CE)
                                *reinterpret_cast<int4 *>(&v[q]) =
                                    *reinterpret_cast<const int4 *>(tb + GTT_CHECKED(Tile::off(row0 + q, 0, p.M), p.tile_bytes - 15, p.err));
                            apply_window<T, B, D>(v, mask, W);
#pragma unroll
                            for (int q = 0; q < RB; q += CE)
                                *reinterpret_cast<int4 *>(tb + GTT_CHECKED(Tile::off(row0 + q, 0, p.M), p.tile_bytes - 15, p.err)) =
                                    *reinterpret_cast<const int4 *>(&v[q]);
                            continue;
                        }
                    }
                    const int form = p.stage_addr[st];
                    if (form == kAddrXor) {
                        const uint32_t a0 = Tile::off(row0, col, p.M);
                        const uint32_t *fq = p.stage_fq[st];
#pragma unroll
                        for (int q = 0; q < RB; ++q) v[q] = *reinterpret_cast<const T *>(tb + TB(a0 ^ fq[q]));
                        apply_window<T, B, D>(v, mask, W);
#pragma unroll
                        for (int q = 0; q < RB; ++q) *reinterpret_cast<T *>(tb + TB(a0 ^ fq[q])) = v[q];
                    } else if (form == kAddrStride) {
                        unsigned char *a0 = tb + Tile::off(row0, col, p.M);
                        const uint32_t stride = p.stage_stride[st];
#pragma unroll
                        for (int q = 0; q < RB; ++q) v[q] = *reinterpret_cast<const T *>(tb + TB((a0 - tb) + q * stride));
                        apply_window<T, B, D>(v, mask, W);
#pragma unroll
                        for (int q = 0; q < RB; ++q) *reinterpret_cast<T *>(tb + TB((a0 - tb) + q * stride)) = v[q];
                    } else if (form == kAddrRowXor) {
                        // swizzle row of element 0 (a multiple of 8) and its byte in the row
                        const uint32_t off0 = Tile::off(row0, col, p.M);  // chunk phase 0 at q = 0
                        unsigned char *rbase = tb + (off0 & ~127u) + (off0 & 15u);
                        const uint32_t c = (off0 >> 4) & 7u;
#pragma unroll
                        for (int q = 0; q < RB; ++q)
                            v[q] = *reinterpret_cast<const T *>(tb + TB((rbase - tb) + q * 128 + (((c ^ (uint32_t)q) & 7u) << 4)));
                        apply_window<T, B, D>(v, mask, W);
#pragma unroll
                        for (int q = 0; q < RB; ++q)
                            *reinterpret_cast<T *>(tb + TB((rbase - tb) + q * 128 + (((c ^ (uint32_t)q) & 7u) << 4))) = v[q];
                    } else {
#pragma unroll
                        for (int q = 0; q < RB; ++q)
                            v[q] = *reinterpret_cast<const T *>(tb + TB(Tile::off(row0 + q * Ba, col, p.M)));
                        apply_window<T, B, D>(v, mask, W);
#pragma unroll
                        for (int q = 0; q < RB; ++q)
                            *reinterpret_cast<T *>(tb + TB(Tile::off(row0 + q * Ba, col, p.M))) = v[q];
                    }
                }
                if (st + 1 < p.nstages) compute_sync();
            }
#undef TB
            fence_proxy_async();  // this thread's smem writes, visible to the TMA store
            mbar_arrive(empty + 8u * buf);
        }
    }
    __syncthreads();
}

} // namespace gtt
