// TMA pass-kernel instantiations for element type uint32_t.
#include "gtt_tma_inst.cuh"

namespace gtt {
const void *tma_kernel_u32(int b, int d, bool contig) { return pick_tma_b<uint32_t>(b, d, contig); }
} // namespace gtt
