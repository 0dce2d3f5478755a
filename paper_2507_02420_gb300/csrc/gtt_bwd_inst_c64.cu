// Backward-kernel instantiations for element type c64.
#include "gtt_bwd_inst.cuh"

namespace gtt {
const void *bwd_kernel_c64(int b) { return pick_bwd_b<c64>(b); }
const void *dw_reduce_kernel_c64() { return (const void *)&gtt_dw_reduce_kernel<c64>; }
} // namespace gtt
