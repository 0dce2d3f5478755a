// TMA pass-kernel instantiations for element type c64.
#include "gtt_tma_inst.cuh"

namespace gtt {
const void *tma_kernel_c64(int b, int d, bool contig) { return pick_tma_b<c64>(b, d, contig); }
} // namespace gtt
