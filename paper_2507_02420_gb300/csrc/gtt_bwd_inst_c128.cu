// Backward-kernel instantiations for element type c128.
#include "gtt_bwd_inst.cuh"

namespace gtt {
const void *bwd_kernel_c128(int b) { return pick_bwd_b<c128>(b); }
const void *dw_reduce_kernel_c128() { return (const void *)&gtt_dw_reduce_kernel<c128>; }
} // namespace gtt
