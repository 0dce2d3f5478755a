// Multi-factor mixed-radix pass kernel for element type c128.
#include "gtt_mixed.cuh"

namespace gtt {
const void *mixed_kernel_c128() { return (const void *)&gtt_mixed_pass_kernel<c128>; }
} // namespace gtt
