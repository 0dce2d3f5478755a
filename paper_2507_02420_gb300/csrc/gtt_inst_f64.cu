// Pass-kernel instantiations for element type double.
#include "gtt_inst.cuh"

namespace gtt {
const void *pass_kernel_f64(int b, int d) { return pick_pass_b<double>(b, d); }
} // namespace gtt
