// The first pass of the inverse on a sparse spectrum (gtt_decompress, the
// reconstruction of Sec. 4.1.5).
//
// The spectrum to reconstruct holds k values per vector and zeros elsewhere.
// The inverse's first pass works on contiguous tiles, and a tile of zeros
// stays zero, so only the tiles that hold kept indices need the pass: the
// output buffer is zero-filled, the kept pairs are sorted by tile, and one
// CTA per touched tile builds the tile in shared memory from its pairs,
// applies the pass's register stages (the same stages, in the same order, as
// the pass kernels, so every value equals the dense pass's; a zero tile gives
// zeros either way, up to the sign of zero) and writes it.  The remaining
// passes then run as usual.
#pragma once
#include "gtt_pass.cuh"

namespace gtt {

constexpr int kSparseSortThreads = 1024;
constexpr int kSparseMaxK = 4096;
constexpr uint32_t kSparseNoTile = 0xFFFFFFFFu;  // tile number of an index outside [0, N)

// Sort the k kept pairs of every vector by (tile, pair number) (one CTA per
// vector, gtt_sparse.cu): key = tile << 32 | j, with tile = idx / tile_elems,
// or kSparseNoTile for an index outside [0, N); k <= kSparseMaxK.  Kernel
// arguments: (const long long *idx, long long k, long long N, uint32_t
// tile_elems, unsigned long long *sorted).
const void *sparse_sort_kernel();

// CTA (c, item): if sorted position c holds the first pair of its tile, build
// that tile of the first pass from the tile's pairs, run the pass's stages
// and write the tile to y (zero-filled beforehand).  Contiguous tiles only
// (the first pass); with repeated indices one of their values is kept.
template <typename T, int B, int D>
__global__ void __launch_bounds__(kPassMaxThreads)
gtt_sparse_first_kernel(const long long *idx, const T *val, const unsigned long long *sorted, long long k,
                        long long N, T *y, PassParams p, WMat<T, B> W) {
    constexpr int RB = cpow(B, D);
    constexpr int CE = Vec16<T>::n;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s = reinterpret_cast<T *>(smem_raw);
    const uint32_t smem_elems = p.tile_elems + p.tile_elems / RB + 1;
#define SP(e) GTT_CHECKED(spos<RB>(e), smem_elems, p.err)
    const long long item = blockIdx.y, c = blockIdx.x;
    const unsigned long long *keys = sorted + item * k;
    const uint32_t tile = (uint32_t)(keys[c] >> 32);
    if (tile == kSparseNoTile || (c > 0 && (uint32_t)(keys[c - 1] >> 32) == tile)) return;  // uniform over the CTA
    const uint32_t tid = threadIdx.x, nth = blockDim.x, tile_elems = p.tile_elems;
    const long long tbase = (long long)tile * tile_elems;
    for (uint32_t e = tid; e < smem_elems; e += nth) s[e] = T{};
    __syncthreads();
    for (long long q = c + tid; q < k && (uint32_t)(keys[q] >> 32) == tile; q += nth) {
        const uint32_t j = (uint32_t)keys[q];
        s[SP(idx[item * k + j] - tbase)] = val[item * k + j];
    }
    __syncthreads();

    // the pass's register stages (gtt_pass_kernel), on the tile in shared memory
    const uint32_t nslots = tile_elems / RB;
    for (int st = 0; st < p.nstages; ++st) {
        const uint32_t strideA = p.stage_strideA[st];
        const int mask = p.stage_mask[st];
        for (uint32_t slot = tid; slot < nslots; slot += nth) {
            const uint32_t rest = p.div_r.div(slot);
            const uint32_t col = slot - rest * p.r;
            const uint32_t high = p.stage_divBa[st].div(rest);
            const uint32_t low = rest - high * p.stage_divBa[st].d;
            const uint32_t e0 = high * (strideA * RB) + low * p.r + col;
            T v[RB];
#pragma unroll
            for (int q = 0; q < RB; ++q) v[q] = s[SP(e0 + q * strideA)];
            apply_window<T, B, D>(v, mask, W);
#pragma unroll
            for (int q = 0; q < RB; ++q) s[SP(e0 + q * strideA)] = v[q];
        }
        __syncthreads();
    }

    T *gout = y + item * N + tbase;
    if (tile_elems % CE == 0) {
        for (uint32_t ch = tid; ch < tile_elems / CE; ch += nth) {
            T v[CE];
#pragma unroll
            for (int i = 0; i < CE; ++i) v[i] = s[SP(ch * CE + i)];
            store16(gout + ch * CE, v);
        }
    } else {
        for (uint32_t e = tid; e < tile_elems; e += nth) gout[e] = s[SP(e)];
    }
#undef SP
}

// Kernel entry for (dtype, b, D), or nullptr (b not in {2, 4, 8, 16}, I32, or
// D neither 1 nor dmax_bytes(es, b)).
const void *sparse_first_kernel(int dtype, int b, int D);

} // namespace gtt
