// Pass-kernel instantiations for element type uint32_t.
#include "gtt_inst.cuh"

namespace gtt {
const void *pass_kernel_u32(int b, int d) { return pick_pass_b<uint32_t>(b, d); }
} // namespace gtt
