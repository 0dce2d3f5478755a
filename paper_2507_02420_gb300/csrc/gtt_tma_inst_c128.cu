// TMA pass-kernel instantiations for element type c128.
#include "gtt_tma_inst.cuh"

namespace gtt {
const void *tma_kernel_c128(int b, int d, bool contig) { return pick_tma_b<c128>(b, d, contig); }
} // namespace gtt
