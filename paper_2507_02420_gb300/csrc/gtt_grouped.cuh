// Grouped persistent launch: many transforms of uneven b, n and dtype in one
// kernel (each transform is the fast GTT of Sec. 3 with its own W).  The
// group's graph runs the requests under 2 MiB here and the larger ones as
// chains of their shapes' pass kernels beside it (gtt_grouped.cu).
//
// The work list is a sequence of segments; a segment is one pass of one
// request, split into tiles (the tile geometry of gtt_pass_kernel).  CTAs take
// work items (segment, tile) from a global atomic counter in list order (a
// table maps every item to its segment); a CTA fetches its next item's index
// while it works on the current one, and waits for that item's dependency only
// after the current item is complete.  A
// segment of pass p > 0 may only start once every tile of pass p-1 of the same
// request is done; the host orders the list so that pass p of request q comes
// `lag` requests after pass p-1 of q, so the wait is normally already
// satisfied and the previous pass's output is still in L2.  The waits always
// end: items are taken in list order, so every awaited item has been taken by
// a running CTA, which either works on it (an item in work waits for nothing)
// or holds it as its next item and reaches it after finishing its current one;
// a wait only ever points to earlier items, so no cycle forms.  Each wait is
// still bounded (kGroupSpinLimit polls) and an expiry raises the error flag.
//
// W of every request lives in a device blob (the kernels' parameter layout);
// an item copies its W into shared memory unless the previous item of the CTA
// had the same W.  Tile data is read with L2-coherent loads (ld.global.cg, 16
// bytes wide where the tile rows allow): an earlier pass on another SM wrote it.
#pragma once
#include "gtt_internal.h"

namespace gtt {

constexpr int kGroupMaxPass = 6;
constexpr int kGroupThreads = 128;
constexpr uint32_t kGroupSpinLimit = 1u << 26;

struct GroupPass {
    PassParams p;
    int D;
};

struct GroupReq {
    const void *x;
    void *y;
    int b, dtype, npass, w_off;
    int w_bytes, pad_;  // size of this request's W in the blob (a multiple of 16)
    GroupPass pass[kGroupMaxPass];
};

struct GroupSeg {
    int req, pass, dep;  // dep: segment that must complete first, -1 if none
    unsigned int dep_tiles;  // tiles of segment dep (what done[dep] must reach)
    long long first_item, tiles;
};

struct GroupArgs {
    const GroupReq *reqs;
    const GroupSeg *segs;
    const unsigned int *item_seg;      // segment of every work item
    int nsegs;
    long long total_items;
    const unsigned char *wblob;
    unsigned long long *work_counter;  // zeroed before every launch
    unsigned int *done;                // tiles completed per segment, zeroed before every launch
    int *err;
    int w_smem_bytes;                  // bytes reserved for W at the start of shared memory
};

template <typename T> __device__ __forceinline__ T ld_cg(const T *p) {
    if constexpr (sizeof(T) == 4) {
        unsigned v = __ldcg(reinterpret_cast<const unsigned *>(p));
        return *reinterpret_cast<T *>(&v);
    } else {
        unsigned long long v = __ldcg(reinterpret_cast<const unsigned long long *>(p));
        return *reinterpret_cast<T *>(&v);
    }
}

// Ask L2 for one item's input tile (M rows of r elements at stride L) before
// it is read: a bulk prefetch per 16-byte aligned row (one for a contiguous
// tile), else one line prefetch per 128-byte line of the row.  The DRAM reads
// of the whole tile then start at once instead of one per load in turn.  L2
// is the coherence point, so a prefetch never yields stale data.
__device__ __forceinline__ void group_prefetch(const unsigned char *in, int es, const PassParams &p, long long t) {
    const uint32_t tid = threadIdx.x, nth = blockDim.x;
    const long long hi = t / p.lo_blocks;
    const uint32_t lob = (uint32_t)(t - hi * p.lo_blocks);
    const long long base = hi * p.L * (long long)p.M + (long long)lob * p.r;
    const bool contig = p.L == (long long)p.r || p.M == 1;
    const uint32_t rows = contig ? 1u : p.M;
    const uint32_t row_bytes = (contig ? p.tile_elems : p.r) * (uint32_t)es;
    for (uint32_t row = tid; row < rows; row += nth) {
        const unsigned char *a = in + (base + (long long)row * p.L) * es;
        if ((((uintptr_t)a | row_bytes) & 15u) == 0) {
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"(row_bytes) : "memory");
        } else {
            const uintptr_t end = (uintptr_t)a + row_bytes;
            for (uintptr_t l = (uintptr_t)a & ~(uintptr_t)127; l < end; l += 128)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(l));
        }
    }
}

// One tile of one pass (shared-memory staging as in gtt_pass_kernel).
template <typename T, int B, int D>
__device__ __noinline__ void group_tile(const T *in, T *out, const PassParams &p, long long t, T *__restrict__ s,
                                        const WMat<T, B> &W) {
    constexpr int RB = cpow(B, D);
    constexpr int CE = Vec16<T>::n;
    const uint32_t tid = threadIdx.x, nth = blockDim.x;
    // the pass parameters live in global memory, and stores to the tile would
    // otherwise force the compiler to read them again: read each one once
    // (the tile is restrict-qualified as well; in and out may be the same)
    const uint32_t tile_elems = p.tile_elems, r = p.r;
    const long long L = p.L;
    const int vec_mode = p.vec_mode, nstages = p.nstages;
    const FastDiv div_r = p.div_r, div_cpr = p.div_cpr;
    const long long hi = t / p.lo_blocks;
    const uint32_t lob = (uint32_t)(t - hi * p.lo_blocks);
    const long long base = hi * L * (long long)p.M + (long long)lob * r;
    if (vec_mode != 0) {  // 16-byte chunks: contiguous tile (1) or rows of r, r % CE == 0 (2)
        const uint32_t cpr = vec_mode == 1 ? tile_elems / CE : r / CE;
        const long long rstride = vec_mode == 1 ? 0 : L;
#pragma unroll 4
        for (uint32_t c = tid; c < tile_elems / CE; c += nth) {
            const uint32_t row = vec_mode == 1 ? 0u : div_cpr.div(c), cc = c - row * cpr;
            const int4 raw = __ldcg(reinterpret_cast<const int4 *>(
                in + GTT_CHECKED(base + (long long)row * rstride + cc * CE, p.total - CE + 1, p.err)));
            const T *v = reinterpret_cast<const T *>(&raw);
            const uint32_t e0 = vec_mode == 1 ? c * CE : row * r + cc * CE;
#pragma unroll
            for (int i = 0; i < CE; ++i) s[spos<RB>(e0 + i)] = v[i];
        }
    } else if (L == (long long)r) {
        // contiguous, but not in whole 16-byte chunks (odd b): the elements up to
        // the first 16-byte boundary one by one, then chunks, then the rest
        const T *src = in + base;
        const uint32_t head = min(tile_elems, (uint32_t)((CE - ((uintptr_t)src / sizeof(T)) % CE) % CE));
        const uint32_t nch = (tile_elems - head) / CE, mid_end = head + nch * CE;
        for (uint32_t e = tid; e < head; e += nth) s[spos<RB>(e)] = ld_cg(src + e);
#pragma unroll 4
        for (uint32_t c = tid; c < nch; c += nth) {
            const int4 raw = __ldcg(reinterpret_cast<const int4 *>(src + head + c * CE));
            const T *v = reinterpret_cast<const T *>(&raw);
#pragma unroll
            for (int i = 0; i < CE; ++i) s[spos<RB>(head + c * CE + i)] = v[i];
        }
        for (uint32_t e = mid_end + tid; e < tile_elems; e += nth) s[spos<RB>(e)] = ld_cg(src + e);
    } else {
#pragma unroll 4
        for (uint32_t e = tid; e < tile_elems; e += nth) {
            const uint32_t row = div_r.div(e), col = e - row * r;
            s[spos<RB>(e)] = ld_cg(in + GTT_CHECKED(base + (long long)row * L + col, p.total, p.err));
        }
    }
    __syncthreads();
    const uint32_t nslots = tile_elems / RB;
    for (int st = 0; st < nstages; ++st) {
        const uint32_t strideA = p.stage_strideA[st];
        const int mask = p.stage_mask[st];
        const FastDiv div_ba = p.stage_divBa[st];
        for (uint32_t slot = tid; slot < nslots; slot += nth) {
            const uint32_t rest = div_r.div(slot);
            const uint32_t col = slot - rest * r;
            const uint32_t high = div_ba.div(rest);
            const uint32_t low = rest - high * div_ba.d;
            const uint32_t e0 = high * (strideA * RB) + low * r + col;
            T v[RB];
#pragma unroll
            for (int q = 0; q < RB; ++q) v[q] = s[spos<RB>(e0 + q * strideA)];
            apply_window<T, B, D, 0, false>(v, mask, W);  // W in shared memory: packed forms
#pragma unroll
            for (int q = 0; q < RB; ++q) s[spos<RB>(e0 + q * strideA)] = v[q];
        }
        __syncthreads();
    }
    if (vec_mode != 0) {
        const uint32_t cpr = vec_mode == 1 ? tile_elems / CE : r / CE;
        const long long rstride = vec_mode == 1 ? 0 : L;
        for (uint32_t c = tid; c < tile_elems / CE; c += nth) {
            const uint32_t row = vec_mode == 1 ? 0u : div_cpr.div(c), cc = c - row * cpr;
            const uint32_t e0 = vec_mode == 1 ? c * CE : row * r + cc * CE;
            T v[CE];
#pragma unroll
            for (int i = 0; i < CE; ++i) v[i] = s[spos<RB>(e0 + i)];
            store16(out + GTT_CHECKED(base + (long long)row * rstride + cc * CE, p.total - CE + 1, p.err), v);
        }
    } else if (L == (long long)r) {  // contiguous, not in whole chunks: as the load
        T *dst = out + base;
        const uint32_t head = min(tile_elems, (uint32_t)((CE - ((uintptr_t)dst / sizeof(T)) % CE) % CE));
        const uint32_t nch = (tile_elems - head) / CE, mid_end = head + nch * CE;
        for (uint32_t e = tid; e < head; e += nth) dst[e] = s[spos<RB>(e)];
        for (uint32_t c = tid; c < nch; c += nth) {
            T v[CE];
#pragma unroll
            for (int i = 0; i < CE; ++i) v[i] = s[spos<RB>(head + c * CE + i)];
            store16(dst + head + c * CE, v);
        }
        for (uint32_t e = mid_end + tid; e < tile_elems; e += nth) dst[e] = s[spos<RB>(e)];
    } else {
        for (uint32_t e = tid; e < tile_elems; e += nth) {
            const uint32_t row = div_r.div(e), col = e - row * r;
            out[base + (long long)row * L + col] = s[spos<RB>(e)];
        }
    }
}

template <typename T, int B>
__device__ __forceinline__ void group_dispatch_d(const GroupReq &rq, const GroupPass &gp, long long t,
                                                 unsigned char *smem, int w_smem_bytes, bool first) {
    constexpr int DM = dmax_bytes((int)sizeof(T), B);
    const T *in = reinterpret_cast<const T *>(first ? rq.x : (const void *)rq.y);
    T *out = reinterpret_cast<T *>(rq.y);
    const WMat<T, B> &W = *reinterpret_cast<const WMat<T, B> *>(smem);
    T *s = reinterpret_cast<T *>(smem + w_smem_bytes);
    if (gp.D == DM)
        group_tile<T, B, DM>(in, out, gp.p, t, s, W);
    else
        group_tile<T, B, 1>(in, out, gp.p, t, s, W);
}

template <typename T>
__device__ __forceinline__ void group_dispatch(const GroupReq &rq, const GroupPass &gp, long long t,
                                               unsigned char *smem, int w_smem_bytes, bool first) {
    switch (rq.b) {
    case 2: group_dispatch_d<T, 2>(rq, gp, t, smem, w_smem_bytes, first); break;
    case 3: group_dispatch_d<T, 3>(rq, gp, t, smem, w_smem_bytes, first); break;
    case 4: group_dispatch_d<T, 4>(rq, gp, t, smem, w_smem_bytes, first); break;
    case 5: group_dispatch_d<T, 5>(rq, gp, t, smem, w_smem_bytes, first); break;
    case 6: group_dispatch_d<T, 6>(rq, gp, t, smem, w_smem_bytes, first); break;
    case 7: group_dispatch_d<T, 7>(rq, gp, t, smem, w_smem_bytes, first); break;
    case 8: group_dispatch_d<T, 8>(rq, gp, t, smem, w_smem_bytes, first); break;
    case 16: group_dispatch_d<T, 16>(rq, gp, t, smem, w_smem_bytes, first); break;
    default: break;
    }
}

__global__ void __launch_bounds__(kGroupThreads, 4) gtt_grouped_kernel(GroupArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_item;
    __shared__ int s_seg, s_woff;
    const uint32_t tid = threadIdx.x;
    long long next = 0;  // thread 0: the item taken ahead of the current one
    if (tid == 0) {
        next = (long long)atomicAdd(a.work_counter, 1ull);
        s_woff = -1;
    }
    for (;;) {
        if (tid == 0) {
            const long long item = next;
            int seg = 0;
            if (item < a.total_items) {
                // take the next item now; its dependency is waited for only
                // after this item is complete, so a CTA never blocks while it
                // holds an unfinished item
                next = (long long)atomicAdd(a.work_counter, 1ull);
                seg = (int)a.item_seg[item];
                const int dep = a.segs[seg].dep;
                if (dep >= 0) {  // bounded wait for the previous pass of this request
                    const unsigned int need = a.segs[seg].dep_tiles;
                    uint32_t spins = 0;
                    while (*((volatile unsigned int *)&a.done[dep]) < need) {
                        if (++spins > kGroupSpinLimit) {
                            atomicExch(a.err, 1);
                            break;
                        }
                        __nanosleep(64);
                    }
                    __threadfence();
                }
            }
            s_item = item;
            s_seg = seg;
        }
        __syncthreads();
        const long long item = s_item;
        if (item >= a.total_items) break;
        const GroupSeg &sg = a.segs[s_seg];
        const GroupReq &rq = a.reqs[sg.req];
        const GroupPass &gp = rq.pass[sg.pass];
        group_prefetch(reinterpret_cast<const unsigned char *>(sg.pass == 0 ? rq.x : (const void *)rq.y),
                       rq.dtype == 1 ? 4 : 8, gp.p, item - sg.first_item);
        // W of this request into shared memory, unless it is already there
        const bool new_w = rq.w_off != s_woff;
        if (new_w) {
            const int wb = rq.w_bytes;
            const int4 *src = reinterpret_cast<const int4 *>(a.wblob + rq.w_off);
            int4 *dst = reinterpret_cast<int4 *>(smem);
            for (int i = tid; i < wb / 16; i += blockDim.x) dst[i] = src[i];
        }
        __syncthreads();
        if (tid == 0 && new_w) s_woff = rq.w_off;  // read again only after the next barrier
        const long long t = item - sg.first_item;
        if (rq.dtype == 1)
            group_dispatch<float>(rq, gp, t, smem, a.w_smem_bytes, sg.pass == 0);
        else
            group_dispatch<c64>(rq, gp, t, smem, a.w_smem_bytes, sg.pass == 0);
        __threadfence();  // this thread's stores before the completion count
        __syncthreads();
        if (tid == 0) atomicAdd(&a.done[s_seg], 1u);
    }
}

} // namespace gtt
