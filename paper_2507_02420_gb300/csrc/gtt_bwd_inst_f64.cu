// Backward-kernel instantiations for element type double.
#include "gtt_bwd_inst.cuh"

namespace gtt {
const void *bwd_kernel_f64(int b) { return pick_bwd_b<double>(b); }
const void *dw_reduce_kernel_f64() { return (const void *)&gtt_dw_reduce_kernel<double>; }
} // namespace gtt
