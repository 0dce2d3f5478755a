// gtt_backward_noalloc: gtt_backward without any device allocation.
//
// Who needs it: callers that must not allocate device memory from inside the
// library -- for example code running under a framework's caching allocator
// that has already reserved the device's memory (a stray cudaMalloc can fail
// or fragment the pool), or latency-critical loops where cudaMalloc/cudaFree
// would synchronize the device.  gtt_backward allocates its dW-partial
// scratch (and, in some cases, data-sized work buffers) on first use; this
// variant takes the dW-partial scratch from a fixed array in the library's
// own device globals and needs no data-sized buffer.  It launches the same
// kernels in the same order as gtt_backward with a caller-provided dx (the
// checkpoint pass on the TMA kernel where the geometry allows it), so its
// results are bitwise equal to gtt_backward's.
//
// The scratch is a file-scope `static __device__` array of
// kNoAllocScratchBytes; every GPU that loads the library keeps it until the
// process exits.  In host code the array's name is only a host-side stand-in,
// so every call looks up its device address with cudaGetSymbolAddress (with
// the plan's device current; no address is cached, so a reset context cannot
// leave a stale one) and passes it to the kernels.  All calls share the one
// array: calls whose kernels overlap on the GPU (different streams, or
// different plans on the same device at the same time) race on it.  Every
// call overwrites the partials it reads, so nothing has to start at zero.
#include <cstring>
#include <string>

#include "gtt_bwd.cuh"
#include "gtt_plan.h"

using namespace gtt;

namespace {

constexpr size_t kNoAllocScratchBytes = 1u << 20;  // 1 MiB of dW partials
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch on the current device.
gtt_status_t scratch_address(void **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress of the static scratch");
    *out = p;
    return GTT_OK;
}

} // namespace

extern "C" gtt_status_t gtt_backward_noalloc(gtt_plan_t P, const void *x, const void *dy, void *dx,
                                             void *dW, gtt_stream_t stream) {
    if (!P) return set_error(GTT_ERR_INVALID_ARG, "NULL plan");
    if (P->mixed) return set_error(GTT_ERR_UNSUPPORTED, "not available for mixed-radix plans");
    if (P->dtype == GTT_I32) return set_error(GTT_ERR_UNSUPPORTED, "backward needs a floating-point dtype");
    if (!x || !dy || !dx)
        return set_error(GTT_ERR_INVALID_ARG, "gtt_backward_noalloc needs x, dy and dx (dx holds its checkpoint)");
    if (dx == dy) return set_error(GTT_ERR_INVALID_ARG, "gtt_backward_noalloc needs dx distinct from dy");
    if (dx == x) return set_error(GTT_ERR_INVALID_ARG, "gtt_backward_noalloc needs dx distinct from x");
    auto al = [](const void *p) { return ((uintptr_t)p & 15u) == 0; };
    if (!al(x) || !al(dy) || !al(dx) || (dW && !al(dW)))
        return set_error(GTT_ERR_INVALID_ARG, "pointers must be 16-byte aligned");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev != P->device) return set_error(GTT_ERR_INVALID_ARG, "current CUDA device differs from the plan's device");
    gtt_status_t st;
    void *scratch = nullptr;
    st = scratch_address(&scratch);
    if (st != GTT_OK) return st;
    if (!P->bwd_ready) {
        st = make_bwd_schedule(P, kBwdSmemBudget);  // host-side set-up, no allocation on the device
        if (st != GTT_OK) return st;
    }
    const int m = (int)P->bwd.size();
    if (m > 2)
        return set_error(GTT_ERR_INVALID_ARG,
                         "gtt_backward_noalloc: this transform needs " + std::to_string(m) +
                             " backward passes; more than 2 need a data-sized checkpoint buffer (use gtt_backward)");
    int nparts = 0;
    for (const BwdPass &bp : P->bwd) nparts += bp.grid;
    const size_t need = (size_t)nparts * P->b * P->b * P->es;
    if (need > kNoAllocScratchBytes)
        return set_error(GTT_ERR_INVALID_ARG, "gtt_backward_noalloc: dW partials need " + std::to_string(need) +
                                                  " bytes, above the static scratch of " +
                                                  std::to_string(kNoAllocScratchBytes) + " bytes");
    cudaStream_t s = (cudaStream_t)stream;
    void *CK = m == 2 ? dx : nullptr;  // a^(1) lives in dx until the last pass overwrites it
    const std::vector<unsigned char> &Wf = P->Wf, &Wa = P->Wa;
    size_t part_off = 0;
    for (int j = m - 1; j >= 0; --j) {
        const BwdPass &bp = P->bwd[j];
        const void *A = x;
        if (j == 1) {  // a^(1) = forward pass 0 of the backward schedule, into dx
            PassPlan &fp = P->bwd[0].fwd;
            const void *in = x;
            void *outp = CK;
            if (fp.tma.on) {
                st = tma_run(P, fp, Wf, in, outp, s, 0, fp.params.tiles);
            } else {
                PassParams fpp = fp.params;
                fpp.err = P->dev_err;
                void *args[4] = {(void *)&in, (void *)&outp, (void *)&fpp, (void *)Wf.data()};
                st = launch_timed(P, fp.kern, dim3(fp.grid), dim3(fp.block), args, fp.smem, s, fp.name);
            }
            if (st != GTT_OK) return st;
            A = CK;
        }
        const void *Gin = (j == m - 1) ? dy : (const void *)dx;
        void *Gout = dx;
        char *dwp = (char *)scratch + part_off * P->b * P->b * P->es;
        int g = bp.g;
        PassParams gp = bp.geo.params;
        gp.err = P->dev_err;
        void *args[8] = {(void *)&A, (void *)&Gin, (void *)&Gout, (void *)&dwp,
                         (void *)&gp, (void *)&g, (void *)Wf.data(), (void *)Wa.data()};
        st = launch_timed(P, bp.kern, dim3(bp.grid), dim3(kBwdThreads), args, bp.smem, s, bp.name);
        if (st != GTT_OK) return st;
        part_off += bp.grid;
    }
    if (dW) {
        const void *rk = dw_reduce_kernel((int)P->dtype);
        const void *parts = scratch;
        int bb = P->b * P->b;
        void *args[4] = {(void *)&parts, (void *)&nparts, (void *)&bb, (void *)&dW};
        st = launch_timed(P, rk, dim3((bb + kDwEntriesPerBlock - 1) / kDwEntriesPerBlock), dim3(32 * kDwEntriesPerBlock),
                          args, 0, s, "gtt_dw_reduce_kernel");
        if (st != GTT_OK) return st;
    }
    return GTT_OK;
}
