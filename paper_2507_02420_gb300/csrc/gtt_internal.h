// Internal interface between the C-ABI layer and the kernel translation units.
#pragma once
#include "gtt_tma.cuh"

namespace gtt {

// dtype codes follow gtt_dtype_t: 0 F64, 1 F32, 2 C64, 3 C128, 4 I32.
inline int elem_size(int dtype) {
    switch (dtype) {
    case 0: return 8;
    case 1: return 4;
    case 2: return 8;
    case 3: return 16;
    case 4: return 4;
    default: return 0;
    }
}

// Register-window depth D of the pass kernel: the largest D with B^D elements
// of the type fitting a ~32-register budget (B^D <= 32 for 4-byte types,
// <= 16 for 8-byte types, <= 9 for 16-byte types).
__host__ __device__ constexpr int dmax_bytes(int es, int b) {
    return es == 4 ? (b == 2 ? 5 : b == 3 ? 3 : (b == 4 || b == 5) ? 2 : 1)
         : es == 8 ? (b == 2 ? 4 : (b == 3 || b == 4) ? 2 : 1)
                   : (b == 2 ? 3 : b == 3 ? 2 : 1);
}

// Kernel entry for (dtype, b, D); D must be 1 or dmax_bytes(es, b).  nullptr
// if no such instantiation exists.
const void *pass_kernel_f64(int b, int d);
const void *pass_kernel_f32(int b, int d);
const void *pass_kernel_c64(int b, int d);
const void *pass_kernel_c128(int b, int d);
const void *pass_kernel_u32(int b, int d);

inline const void *pass_kernel(int dtype, int b, int d) {
    switch (dtype) {
    case 0: return pass_kernel_f64(b, d);
    case 1: return pass_kernel_f32(b, d);
    case 2: return pass_kernel_c64(b, d);
    case 3: return pass_kernel_c128(b, d);
    case 4: return pass_kernel_u32(b, d);
    default: return nullptr;
    }
}

} // namespace gtt

namespace gtt {
// Backward pass kernels and the dW reduction (floating-point types only).
const void *bwd_kernel_f64(int b);
const void *bwd_kernel_f32(int b);
const void *bwd_kernel_c64(int b);
const void *bwd_kernel_c128(int b);
const void *dw_reduce_kernel_f64();
const void *dw_reduce_kernel_f32();
const void *dw_reduce_kernel_c64();
const void *dw_reduce_kernel_c128();

inline const void *bwd_kernel(int dtype, int b) {
    switch (dtype) {
    case 0: return bwd_kernel_f64(b);
    case 1: return bwd_kernel_f32(b);
    case 2: return bwd_kernel_c64(b);
    case 3: return bwd_kernel_c128(b);
    default: return nullptr;
    }
}
inline const void *dw_reduce_kernel(int dtype) {
    switch (dtype) {
    case 0: return dw_reduce_kernel_f64();
    case 1: return dw_reduce_kernel_f32();
    case 2: return dw_reduce_kernel_c64();
    case 3: return dw_reduce_kernel_c128();
    default: return nullptr;
    }
}
// rows of dW per backward thread (mirrors bwd_rows in gtt_bwd.cuh)
inline int bwd_rows_host(int b, bool cplx) {
    int budget = cplx ? 32 : 64;
    int R = b;
    while (R * b > budget && R % 2 == 0) R /= 2;
    return R;
}
} // namespace gtt

namespace gtt {
// TMA-pipelined pass kernels (gtt_tma.cuh): b in {2, 4, 8, 16}, D in {1, dmax},
// contiguous or strided tiles.  nullptr when not instantiated.
const void *tma_kernel_f64(int b, int d, bool contig);
const void *tma_kernel_f32(int b, int d, bool contig);
const void *tma_kernel_c64(int b, int d, bool contig);
const void *tma_kernel_c128(int b, int d, bool contig);
const void *tma_kernel_u32(int b, int d, bool contig);

inline const void *tma_kernel(int dtype, int b, int d, bool contig) {
    switch (dtype) {
    case 0: return tma_kernel_f64(b, d, contig);
    case 1: return tma_kernel_f32(b, d, contig);
    case 2: return tma_kernel_c64(b, d, contig);
    case 3: return tma_kernel_c128(b, d, contig);
    case 4: return tma_kernel_u32(b, d, contig);
    default: return nullptr;
    }
}
} // namespace gtt
