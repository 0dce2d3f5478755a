// Pass-kernel instantiations for element type c128.
#include "gtt_inst.cuh"

namespace gtt {
const void *pass_kernel_c128(int b, int d) { return pick_pass_b<c128>(b, d); }
} // namespace gtt
