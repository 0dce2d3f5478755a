// Multi-factor mixed-radix pass kernel for element type f32.
#include "gtt_mixed.cuh"

namespace gtt {
const void *mixed_kernel_f32() { return (const void *)&gtt_mixed_pass_kernel<float>; }
} // namespace gtt
