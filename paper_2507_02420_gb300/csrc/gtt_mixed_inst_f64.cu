// Multi-factor mixed-radix pass kernel for element type f64.
#include "gtt_mixed.cuh"

namespace gtt {
const void *mixed_kernel_f64() { return (const void *)&gtt_mixed_pass_kernel<double>; }
} // namespace gtt
