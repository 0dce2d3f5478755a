// TMA pass-kernel instantiations for element type double.
#include "gtt_tma_inst.cuh"

namespace gtt {
const void *tma_kernel_f64(int b, int d, bool contig) { return pick_tma_b<double>(b, d, contig); }
} // namespace gtt
