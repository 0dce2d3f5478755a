// Instantiations of the sparse first-pass kernel (gtt_sparse.cuh) for the
// power-of-two bases and the floating-point types.
#include "gtt_internal.h"
#include "gtt_sparse.cuh"

namespace gtt {

// The sort of the kept pairs (declared in gtt_sparse.cuh); one CTA per vector.
__global__ void __launch_bounds__(kSparseSortThreads)
gtt_sparse_sort_kernel(const long long *idx, long long k, long long N, uint32_t tile_elems,
                       unsigned long long *sorted) {
    __shared__ unsigned long long s[kSparseMaxK];
    const long long item = blockIdx.x;
    int P2 = 1;
    while (P2 < k) P2 <<= 1;
    for (int i = threadIdx.x; i < P2; i += blockDim.x) {
        unsigned long long key = ~0ull;
        if (i < k) {
            const long long e = idx[item * k + i];
            const uint32_t tile = (e >= 0 && e < N) ? (uint32_t)(e / tile_elems) : kSparseNoTile;
            key = ((unsigned long long)tile << 32) | (uint32_t)i;
        }
        s[i] = key;
    }
    __syncthreads();
    // bitonic sort, ascending
    for (int size = 2; size <= P2; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < P2; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const unsigned long long a = s[i], b = s[j];
                    if ((a > b) == ((i & size) == 0)) {
                        s[i] = b;
                        s[j] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < k; i += blockDim.x) sorted[item * k + i] = s[i];
}

const void *sparse_sort_kernel() { return (const void *)&gtt_sparse_sort_kernel; }

template <typename T, int B> static const void *pick_sparse(int d) {
    constexpr int DM = dmax_bytes((int)sizeof(T), B);
    if (d == DM) return (const void *)&gtt_sparse_first_kernel<T, B, DM>;
    if (d == 1) return (const void *)&gtt_sparse_first_kernel<T, B, 1>;
    return nullptr;
}

template <typename T> static const void *pick_sparse_b(int b, int d) {
    switch (b) {
    case 2: return pick_sparse<T, 2>(d);
    case 4: return pick_sparse<T, 4>(d);
    case 8: return pick_sparse<T, 8>(d);
    case 16: return pick_sparse<T, 16>(d);
    default: return nullptr;
    }
}

const void *sparse_first_kernel(int dtype, int b, int D) {
    switch (dtype) {
    case 0: return pick_sparse_b<double>(b, D);
    case 1: return pick_sparse_b<float>(b, D);
    case 2: return pick_sparse_b<c64>(b, D);
    case 3: return pick_sparse_b<c128>(b, D);
    default: return nullptr;
    }
}

} // namespace gtt
