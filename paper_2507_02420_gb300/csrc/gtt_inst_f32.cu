// Pass-kernel instantiations for element type float.
#include "gtt_inst.cuh"

namespace gtt {
const void *pass_kernel_f32(int b, int d) { return pick_pass_b<float>(b, d); }
} // namespace gtt
