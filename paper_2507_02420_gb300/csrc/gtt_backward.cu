// gtt_backward: reverse-mode derivative of y = G_N x (no counterpart in the
// paper; PyTorch's conjugate convention).
//
// The backward uses its own schedule of passes, sized so a tile plus the
// recomputed activations of its digits fit shared memory.  Pass j needs the
// activation a^(j) entering it and the gradient leaving it:
//   - a^(0) = x; a^(j), j >= 1, is recomputed by running forward passes
//     0..j-1 of the same schedule (on the TMA pass kernel where the geometry
//     allows it);
//   - the gradient buffer is dx (or a plan-owned buffer when dx is NULL); the
//     last pass reads dy, every pass writes its input gradient in place.
// Checkpoints: with two passes, a^(1) is computed once into dx (when dx is
// distinct from dy) or a plan-owned buffer.  With three passes and a gradient
// buffer distinct from dy, a^(1) goes to the checkpoint buffer and a^(2) to
// the gradient buffer, which the first backward pass reads as its activation
// and overwrites, tile by tile, with its gradient (a tile is read whole before
// it is written).  Otherwise a^(j) is recomputed into the checkpoint buffer
// before each pass.
// dW partials (one b x b block per CTA and pass) are summed in a fixed order.
#include <algorithm>
#include <cstring>
#include <string>

#include "gtt_bwd.cuh"
#include "gtt_tile8.cuh"
#include "gtt_plan.h"

using namespace gtt;

namespace gtt {

static long long ipow_ll(int b, int e) {
    long long r = 1;
    for (int i = 0; i < e; ++i) r *= b;
    return r;
}

// Shared memory of a backward pass: (g+1) padded tiles, or the per-thread
// partial buffer of the final CTA reduction, whichever is larger.
static size_t bwd_smem_bytes(int b, int g, long long tile, int es, bool cplx) {
    const size_t tstride = (size_t)(tile + tile / b + 1);
    const size_t tiles = (size_t)(g + 1) * tstride * es;
    const size_t red = (size_t)kBwdThreads * bwd_rows_host(b, cplx) * b * es;
    return (std::max(tiles, red) + 15) / 16 * 16;
}

static const void *bwd8_kernel(int g) {
    return g == 4 ? (const void *)&gtt_backward_b8_kernel<4>
                  : g == 3 ? (const void *)&gtt_backward_b8_kernel<3>
                           : g == 2 ? (const void *)&gtt_backward_b8_kernel<2> : (const void *)&gtt_backward_b8_kernel<1>;
}

gtt_status_t make_bwd_schedule(gtt_plan_s *P, size_t smem_budget) {
    const int b = P->b, n = P->n, es = P->es;
    const bool cplx = P->dtype == GTT_C64 || P->dtype == GTT_C128;
    const int DM = dmax_bytes(es, b);
    const void *bk_generic = bwd_kernel((int)P->dtype, b);
    if (!bk_generic) return set_error(GTT_ERR_UNSUPPORTED, "no backward kernel for this dtype");
    // FP32, b = 8: the fixed 4096-element tile kernel; the first pass takes
    // digits 0-3, later passes at most 3 digits, so their runs are at least
    // 8 elements (32 bytes)
    const bool b8 = P->dtype == GTT_F32 && b == 8 && n >= 4;
    std::vector<BwdPass> out;
    int m0 = 0;
    while (m0 < n) {
        long long r = 1;
        const long long L = ipow_ll(b, m0);
        int g = 1;
        if (b8) {
            g = m0 == 0 ? 4 : std::min(3, n - m0);
            r = ipow_ll(8, 4 - g);
        } else if (m0 == 0) {
            while (m0 + g < n && bwd_smem_bytes(b, g + 1, ipow_ll(b, g + 1), es, cplx) <= smem_budget) ++g;
        } else {
            // fewer passes first: as many modes as fit with runs of at least one
            // 32-byte sector, then the longest runs (up to a 128-byte line, more
            // on the last pass) that still fit with those modes
            while (r * b <= L && r * es < 32) r *= b;
            while (m0 + g < n && bwd_smem_bytes(b, g + 1, ipow_ll(b, g + 1) * r, es, cplx) <= smem_budget) ++g;
            while (r * b <= L && (r * es < 128 || m0 + g == n) &&
                   bwd_smem_bytes(b, g, ipow_ll(b, g) * r * b, es, cplx) <= smem_budget)
                r *= b;
        }
        BwdPass bp;
        bp.g = g;
        gtt_status_t st = build_pass(P, m0, g, r, 1, &bp.geo);  // D = 1: one stage per digit
        if (st != GTT_OK) return st;
        st = build_pass(P, m0, g, r, g >= DM ? DM : 1, &bp.fwd);  // forward recompute of a^(j+1)
        if (st != GTT_OK) return st;
        if (!tile8_attach(P, &bp.fwd) && P->use_tma)
            tma_attach(P, &bp.fwd, P->tma_nbuf);  // stays on the CUDA-core kernel if ineligible
        const void *bk = b8 ? bwd8_kernel(g) : bk_generic;
        bp.kern = bk;
        bp.smem = b8 ? bwd8_smem_bytes(g) : bwd_smem_bytes(b, g, ipow_ll(b, g) * r, es, cplx);
        if (bp.smem > 227 * 1024) return set_error(GTT_ERR_UNSUPPORTED, "backward tile exceeds shared memory");
        cudaError_t e;
        e = allow_max_smem(bk, P->smem_optin);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(bk, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute (backward)");
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bk, kBwdThreads, bp.smem);
        if (e != cudaSuccess) return cuda_error(e, "occupancy query (backward)");
        if (per_sm < 1) return set_error(GTT_ERR_UNSUPPORTED, "backward kernel cannot be resident");
        bp.grid = (int)std::min<long long>((long long)per_sm * P->num_sms, bp.geo.params.tiles);
        static const char *tnames[] = {"f64", "f32", "c64", "c128", "u32"};
        bp.name = b8 ? "gtt_backward_b8_kernel<" + std::to_string(g) + ">"
                     : std::string("gtt_backward_pass_kernel<") + tnames[(int)P->dtype] + "," +
                           std::to_string(b) + "," + std::to_string(bwd_rows_host(b, cplx)) + ">";
        out.push_back(bp);
        m0 += g;
    }
    P->bwd = out;
    P->bwd_ready = true;
    return GTT_OK;
}

static gtt_status_t ensure_buffer(void **buf, size_t *have, size_t need, const char *what) {
    if (*buf && *have >= need) return GTT_OK;
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *have = 0;
    cudaError_t e = cudaMalloc(buf, need);
    if (e != cudaSuccess) {
        *buf = nullptr;
        return set_error(GTT_ERR_ALLOC, std::string(what) + ": " + cudaGetErrorString(e));
    }
    *have = need;
    return GTT_OK;
}

} // namespace gtt

// ckpt: the activation entering the second backward pass, saved by
// gtt_forward_saving (two-pass schedules), or NULL to recompute it.
static gtt_status_t backward_impl(gtt_plan_t P, const void *x, const void *ckpt, const void *dy, void *dx, void *dW,
                                  gtt_stream_t stream) {
    if (!P) return set_error(GTT_ERR_INVALID_ARG, "NULL plan");
    if (P->mixed) return set_error(GTT_ERR_UNSUPPORTED, "not available for mixed-radix plans");
    if (P->dtype == GTT_I32) return set_error(GTT_ERR_UNSUPPORTED, "backward needs a floating-point dtype");
    if (!x || !dy) return set_error(GTT_ERR_INVALID_ARG, "NULL x or dy");
    if (dx && dx == x) return set_error(GTT_ERR_INVALID_ARG, "dx must not alias x_saved");
    auto al = [](const void *p) { return ((uintptr_t)p & 15u) == 0; };
    if (!al(x) || !al(dy) || (dx && !al(dx)) || (dW && !al(dW)))
        return set_error(GTT_ERR_INVALID_ARG, "pointers must be 16-byte aligned");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev != P->device) return set_error(GTT_ERR_INVALID_ARG, "current CUDA device differs from the plan's device");
    cudaStream_t s = (cudaStream_t)stream;
    gtt_status_t st;
    if (!P->bwd_ready) {
        st = make_bwd_schedule(P, kBwdSmemBudget);
        if (st != GTT_OK) return st;
    }
    const int m = (int)P->bwd.size();
    if (ckpt) {
        if (saving_boundary(P) < 0)
            return set_error(GTT_ERR_UNSUPPORTED, "this plan keeps no checkpoint (use gtt_backward)");
        if (((uintptr_t)ckpt & 15u) || ckpt == x || ckpt == dy)
            return set_error(GTT_ERR_INVALID_ARG, "ckpt must be 16-byte aligned and distinct from x and dy");
    }
    const size_t data_bytes = (size_t)P->total * P->es;
    // gradient buffer
    void *GB = dx;
    if (!GB) {
        st = ensure_buffer(&P->ws_grad, &P->ws_grad_bytes, data_bytes, "backward gradient buffer");
        if (st != GTT_OK) return st;
        GB = P->ws_grad;
    }
    // checkpoint buffer
    void *CK = nullptr;
    const bool two_ck = m == 3 && GB != dy;  // a^(2) parked in the gradient buffer
    if (m >= 2 && !ckpt) {
        if (m == 2 && dx && dx != dy) {
            CK = dx;
        } else {
            st = ensure_buffer(&P->ws_ck, &P->ws_ck_bytes, data_bytes, "backward checkpoint buffer");
            if (st != GTT_OK) return st;
            CK = P->ws_ck;
        }
    }
    // dW partials: one b*b block per CTA per pass
    int nparts = 0;
    for (const BwdPass &bp : P->bwd) nparts += bp.grid;
    st = ensure_buffer(&P->ws_dw, &P->ws_dw_bytes, (size_t)nparts * P->b * P->b * P->es, "dW partials");
    if (st != GTT_OK) return st;

    const std::vector<unsigned char> &Wf = P->Wf, &Wa = P->Wa;
    auto fwd_pass = [&](int q, const void *in, void *outp) -> gtt_status_t {
        PassPlan &fp = P->bwd[q].fwd;
        if (fp.tma.on) return tma_run(P, fp, Wf, in, outp, s, 0, fp.params.tiles);
        PassParams fpp = fp.params;
        fpp.err = P->dev_err;
        void *args[4] = {(void *)&in, (void *)&outp, (void *)&fpp, (void *)Wf.data()};
        return launch_timed(P, fp.kern, dim3(fp.grid), dim3(fp.block), args, fp.smem, s, fp.name);
    };
    // activations entering each backward pass, computed up front when they fit
    std::vector<const void *> act(m, x);
    bool upfront = false;
    if (ckpt) {
        act[1] = ckpt;  // m == 2: nothing to recompute
        upfront = true;
    } else if (m == 2 || two_ck) {
        st = fwd_pass(0, x, CK);
        if (st != GTT_OK) return st;
        act[1] = CK;
        if (two_ck) {
            st = fwd_pass(1, CK, GB);
            if (st != GTT_OK) return st;
            act[2] = GB;
        }
        upfront = true;
    }
    size_t part_off = 0;
    for (int j = m - 1; j >= 0; --j) {
        const BwdPass &bp = P->bwd[j];
        const void *A = act[j];
        if (!upfront && j >= 1) {  // a^(j): forward passes 0..j-1 into CK
            for (int q = 0; q < j; ++q) {
                st = fwd_pass(q, q == 0 ? x : (const void *)CK, CK);
                if (st != GTT_OK) return st;
            }
            A = CK;
        }
        const void *Gin = (j == m - 1) ? dy : (const void *)GB;
        void *Gout = GB;
        char *dwp = (char *)P->ws_dw + part_off * P->b * P->b * P->es;
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
        const void *parts = P->ws_dw;
        int bb = P->b * P->b;
        void *args[4] = {(void *)&parts, (void *)&nparts, (void *)&bb, (void *)&dW};
        st = launch_timed(P, rk, dim3((bb + kDwEntriesPerBlock - 1) / kDwEntriesPerBlock), dim3(32 * kDwEntriesPerBlock), args, 0, s, "gtt_dw_reduce_kernel");
        if (st != GTT_OK) return st;
    }
    return GTT_OK;
}

extern "C" gtt_status_t gtt_backward(gtt_plan_t P, const void *x, const void *dy, void *dx, void *dW,
                                     gtt_stream_t stream) {
    return backward_impl(P, x, nullptr, dy, dx, dW, stream);
}

extern "C" gtt_status_t gtt_backward_saved(gtt_plan_t P, const void *x, const void *ckpt, const void *dy, void *dx,
                                           void *dW, gtt_stream_t stream) {
    if (!ckpt) return set_error(GTT_ERR_INVALID_ARG, "NULL ckpt");
    return backward_impl(P, x, ckpt, dy, dx, dW, stream);
}
