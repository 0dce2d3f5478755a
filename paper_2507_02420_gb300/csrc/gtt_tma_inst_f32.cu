// TMA pass-kernel instantiations for element type float.
#include "gtt_tma_inst.cuh"

namespace gtt {
const void *tma_kernel_f32(int b, int d, bool contig) { return pick_tma_b<float>(b, d, contig); }
} // namespace gtt
