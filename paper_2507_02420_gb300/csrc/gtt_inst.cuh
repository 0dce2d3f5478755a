// Instantiates gtt_pass_kernel<T, B, D> for B = 2..16 and D in {1, dmax}.
#pragma once
#include "gtt_internal.h"

namespace gtt {

template <typename T, int B> const void *pick_pass(int d) {
    constexpr int DM = dmax_bytes((int)sizeof(T), B);
    if (d == DM) return (const void *)&gtt_pass_kernel<T, B, DM>;
    if (d == 1) return (const void *)&gtt_pass_kernel<T, B, 1>;
    return nullptr;
}

template <typename T> const void *pick_pass_b(int b, int d) {
    switch (b) {
    case 2: return pick_pass<T, 2>(d);
    case 3: return pick_pass<T, 3>(d);
    case 4: return pick_pass<T, 4>(d);
    case 5: return pick_pass<T, 5>(d);
    case 6: return pick_pass<T, 6>(d);
    case 7: return pick_pass<T, 7>(d);
    case 8: return pick_pass<T, 8>(d);
    case 9: return pick_pass<T, 9>(d);
    case 10: return pick_pass<T, 10>(d);
    case 11: return pick_pass<T, 11>(d);
    case 12: return pick_pass<T, 12>(d);
    case 13: return pick_pass<T, 13>(d);
    case 14: return pick_pass<T, 14>(d);
    case 15: return pick_pass<T, 15>(d);
    case 16: return pick_pass<T, 16>(d);
    default: return nullptr;
    }
}

} // namespace gtt
