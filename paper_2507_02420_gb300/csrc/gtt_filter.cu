// gtt_filter: natural-order spectral filtering (Sec. 4.3.2, the classical
// reading of Algorithm 3): y = G_N^dagger (mask * G_N x), where the mask keeps
// the coefficients of index p < cut (low-pass) or p >= cut (high-pass) of
// every vector of the batch and zeroes the others.
//
// The forward passes write the spectrum into y; one write-only kernel zeroes
// the masked coefficient range of every vector (it reads nothing); the
// adjoint passes then run in place on y.  The adjoint's first pass works on
// contiguous tiles, and a tile inside the zeroed range stays zero, so that
// pass runs only on the tiles that meet the kept range (the same values: a
// zero tile gives zeros either way, up to the sign of zero).
#include <algorithm>

#include "gtt_plan.h"

namespace gtt {

// Zero words [lo, hi) of every one of `items` rows of `row_words` 32-bit words
// (V = 4: 16-byte stores, all three counts multiples of 4; V = 1: 4-byte).
template <int V>
__global__ void __launch_bounds__(256) gtt_zero_range_kernel(uint32_t *data, long long items, long long row_words,
                                                             long long lo, long long hi) {
    const long long span = (hi - lo) / V;
    const long long total = items * span;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < total;
         u += (long long)gridDim.x * blockDim.x) {
        const long long item = u / span, off = u - item * span;
        uint32_t *p = data + item * row_words + lo + off * V;
        if constexpr (V == 4)
            *reinterpret_cast<uint4 *>(p) = make_uint4(0u, 0u, 0u, 0u);
        else
            *p = 0u;
    }
}

gtt_status_t zero_range(gtt_plan_s *P, void *y, long long lo_el, long long hi_el, cudaStream_t s) {
    if (hi_el <= lo_el) return GTT_OK;
    const long long wpe = P->es / 4;  // 32-bit words per element
    long long row = P->N * wpe, lo = lo_el * wpe, hi = hi_el * wpe;
    const bool vec = row % 4 == 0 && lo % 4 == 0 && hi % 4 == 0;
    const long long units = P->batch * (hi - lo) / (vec ? 4 : 1);
    const int grid = (int)std::max<long long>(1, std::min<long long>((units + 255) / 256, 8ll * P->num_sms));
    uint32_t *d = static_cast<uint32_t *>(y);
    long long items = P->batch;
    void *args[5] = {(void *)&d, (void *)&items, (void *)&row, (void *)&lo, (void *)&hi};
    const void *k = vec ? (const void *)&gtt_zero_range_kernel<4> : (const void *)&gtt_zero_range_kernel<1>;
    return launch_timed(P, k, dim3(grid), dim3(256), args, 0, s, "gtt_zero_range_kernel");
}

} // namespace gtt

using namespace gtt;

extern "C" gtt_status_t gtt_filter(gtt_plan_t P, const void *x, void *y, long long cut, int keep_low,
                                   gtt_stream_t stream) {
    if (!P) return set_error(GTT_ERR_INVALID_ARG, "NULL plan");
    if (!x || !y) return set_error(GTT_ERR_INVALID_ARG, "NULL data pointer");
    if (((uintptr_t)x & 15u) || ((uintptr_t)y & 15u))
        return set_error(GTT_ERR_INVALID_ARG, "data pointers must be 16-byte aligned");
    if (cut < 0 || cut > P->N) return set_error(GTT_ERR_INVALID_ARG, "cut must be in [0, N]");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev != P->device) return set_error(GTT_ERR_INVALID_ARG, "current CUDA device differs from the plan's device");
    cudaStream_t s = (cudaStream_t)stream;
    // spectrum
    gtt_status_t st = run_passes(P, P->Wf, x, y, s);
    if (st != GTT_OK) return st;
    // zero the masked coefficients: [cut, N) for a low-pass, [0, cut) for a high-pass
    st = keep_low ? zero_range(P, y, cut, P->N, s) : zero_range(P, y, 0, cut, s);
    if (st != GTT_OK) return st;
    // back to the signal domain
    const PassPlan &p0 = P->passes[0];
    const long long te = p0.params.tile_elems;
    if (p0.tcx.on || p0.m0 != 0 || p0.params.L != (long long)p0.params.r || P->N % te != 0 || P->batch > 16)
        return run_passes(P, P->Wa, y, y, s);
    const long long lo = keep_low ? 0 : cut, hi = keep_low ? cut : P->N;
    for (long long v = 0; v < P->batch; ++v) {
        const long long t0 = (v * P->N + lo) / te, t1 = (v * P->N + hi + te - 1) / te;
        if (t1 > t0) {
            st = run_pass_range(P, 0, P->Wa, y, y, s, t0, t1);
            if (st != GTT_OK) return st;
        }
    }
    return run_passes_from(P, P->Wa, y, s, 1);
}
