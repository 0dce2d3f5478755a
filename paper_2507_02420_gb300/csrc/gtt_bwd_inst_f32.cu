// Backward-kernel instantiations for element type float.
#include "gtt_bwd_inst.cuh"

namespace gtt {
const void *bwd_kernel_f32(int b) { return pick_bwd_b<float>(b); }
const void *dw_reduce_kernel_f32() { return (const void *)&gtt_dw_reduce_kernel<float>; }
} // namespace gtt
