// Pass-kernel instantiations for element type c64.
#include "gtt_inst.cuh"

namespace gtt {
const void *pass_kernel_c64(int b, int d) { return pick_pass_b<c64>(b, d); }
} // namespace gtt
