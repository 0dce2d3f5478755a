// Instantiates the backward pass kernel for B = 2..16 and the dW reduction.
#pragma once
#include "gtt_bwd.cuh"

namespace gtt {

template <typename T, int B> const void *pick_bwd() {
    return (const void *)&gtt_backward_pass_kernel<T, B, bwd_rows(B, Traits<T>::complex)>;
}

template <typename T> const void *pick_bwd_b(int b) {
    switch (b) {
    case 2: return pick_bwd<T, 2>();
    case 3: return pick_bwd<T, 3>();
    case 4: return pick_bwd<T, 4>();
    case 5: return pick_bwd<T, 5>();
    case 6: return pick_bwd<T, 6>();
    case 7: return pick_bwd<T, 7>();
    case 8: return pick_bwd<T, 8>();
    case 9: return pick_bwd<T, 9>();
    case 10: return pick_bwd<T, 10>();
    case 11: return pick_bwd<T, 11>();
    case 12: return pick_bwd<T, 12>();
    case 13: return pick_bwd<T, 13>();
    case 14: return pick_bwd<T, 14>();
    case 15: return pick_bwd<T, 15>();
    case 16: return pick_bwd<T, 16>();
    default: return nullptr;
    }
}

} // namespace gtt
