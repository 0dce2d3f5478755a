// Multi-factor mixed-radix pass kernel for element type c64.
#include "gtt_mixed.cuh"

namespace gtt {
const void *mixed_kernel_c64() { return (const void *)&gtt_mixed_pass_kernel<c64>; }
} // namespace gtt
