// Instantiates gtt_tma_pass_kernel<T, B, D, CONTIG> for B in {2, 4, 8, 16}.
#pragma once
#include "gtt_internal.h"

namespace gtt {

template <typename T, int B> const void *pick_tma(int d, bool contig) {
    constexpr int DM = dmax_bytes((int)sizeof(T), B);
    if (d == DM) return contig ? (const void *)&gtt_tma_pass_kernel<T, B, DM, true>
                               : (const void *)&gtt_tma_pass_kernel<T, B, DM, false>;
    if (d == 1) return contig ? (const void *)&gtt_tma_pass_kernel<T, B, 1, true>
                              : (const void *)&gtt_tma_pass_kernel<T, B, 1, false>;
    return nullptr;
}

template <typename T> const void *pick_tma_b(int b, int d, bool contig) {
    switch (b) {
    case 2: return pick_tma<T, 2>(d, contig);
    case 4: return pick_tma<T, 4>(d, contig);
    case 8: return pick_tma<T, 8>(d, contig);
    case 16: return pick_tma<T, 16>(d, contig);
    default: return nullptr;
    }
}

} // namespace gtt
