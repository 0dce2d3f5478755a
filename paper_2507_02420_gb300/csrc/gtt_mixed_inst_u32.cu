// Multi-factor mixed-radix pass kernel for element type u32.
#include "gtt_mixed.cuh"

namespace gtt {
const void *mixed_kernel_u32() { return (const void *)&gtt_mixed_pass_kernel<uint32_t>; }
} // namespace gtt
