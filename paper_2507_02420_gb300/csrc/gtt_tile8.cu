// Host side of the b = 8 FP32 forward tile kernel (gtt_tile8.cuh): which
// passes it takes and their launch shape.
#include <algorithm>
#include <string>

#include "gtt_plan.h"
#include "gtt_tile8.cuh"

namespace gtt {

static const void *fwd8_kernel(int g, bool bot) {
    if (bot) return g == 3 ? (const void *)&gtt_forward_b8_kernel<3, true>
                    : g == 2 ? (const void *)&gtt_forward_b8_kernel<2, true> : (const void *)&gtt_forward_b8_kernel<1, true>;
    return g == 4 ? (const void *)&gtt_forward_b8_kernel<4, false>
         : g == 3 ? (const void *)&gtt_forward_b8_kernel<3, false>
         : g == 2 ? (const void *)&gtt_forward_b8_kernel<2, false> : (const void *)&gtt_forward_b8_kernel<1, false>;
}

// A pass of an FP32 b = 8 plan whose tile is 4096 elements runs on the tile
// kernel: g digits over runs of 8^(4-g) (the top g of the tile's four
// digits), or, on the first pass, g digits of 8^(4-g) consecutive blocks (the
// bottom g).  Returns false, leaving the pass as it is, for other passes.
bool tile8_attach(gtt_plan_s *P, PassPlan *pp) {
    if (P->dtype != GTT_F32 || P->b != 8 || P->mixed || pp->factor >= 0) return false;
    const int g = pp->g;
    if (g < 1 || g > 4 || pp->params.tile_elems != (uint32_t)kBwd8Tile) return false;
    long long r4 = 1;
    for (int i = g; i < 4; ++i) r4 *= 8;
    // the kernel moves 16-byte chunks of 4 consecutive tile elements, so a
    // later pass needs runs of at least 8 elements (g <= 3); the first pass
    // has contiguous tiles
    bool bot;
    if (pp->m0 == 0)
        bot = g < 4;  // r = 8^(4-g) consecutive blocks (g = 4: the whole tile)
    else if (g <= 3 && pp->r == r4 && pp->params.r == (uint32_t)r4)
        bot = false;
    else
        return false;
    if (pp->m0 == 0 && pp->r != r4) return false;
    const void *k = fwd8_kernel(g, bot);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kBwd8Threads, kFwd8Smem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return false;
    }
    pp->kern = k;
    pp->block = kBwd8Threads;
    pp->smem = kFwd8Smem;
    pp->ctas_per_sm = per_sm;
    pp->grid = (int)std::min<long long>((long long)per_sm * P->num_sms, pp->params.tiles);
    pp->name = "gtt_forward_b8_kernel<" + std::to_string(g) + (bot ? ",bottom>" : ">");
    pp->tma.on = false;
    return true;
}

} // namespace gtt
