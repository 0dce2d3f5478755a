// Host side of the b = 16 tensor-core passes (gtt_tc16.cuh): the BF16x3
// schedule, the split W operands, and the launch.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "gtt_plan.h"
#include "gtt_tc16.cuh"

namespace gtt {

// B operand: rows n = 16p + i hold piece p of row i of M (M = W for the
// forward, W^T for the adjoint), K-major core-matrix layout, 48 x 16 BF16.
static void split_w_pieces(const float *M, int transpose, unsigned char *out) {
    memset(out, 0, 1536);
    for (int n = 0; n < 48; ++n)
        for (int k = 0; k < 16; ++k) {
            const int p = n / 16, i = n % 16;
            const float w = transpose ? M[k * 16 + i] : M[i * 16 + k];
            const __nv_bfloat16 w0 = __float2bfloat16_rn(w);
            const float r1 = w - __bfloat162float(w0);
            const __nv_bfloat16 w1 = __float2bfloat16_rn(r1);
            const float r2 = r1 - __bfloat162float(w1);
            const __nv_bfloat16 w2 = __float2bfloat16_rn(r2);
            const __nv_bfloat16 piece = p == 0 ? w0 : p == 1 ? w1 : w2;
            const size_t off = (n / 8) * 256 + (k / 8) * 128 + (n % 8) * 16 + (k % 8) * 2;
            memcpy(out + off, &piece, 2);
        }
}

// Round a float to TF32 (10 explicit mantissa bits), to nearest with ties away
// from zero, on its bit pattern (the same rule the kernel applies to x).
static float round_tf32_host(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    u = (u + 0x1000u) & 0xFFFFE000u;
    memcpy(&f, &u, 4);
    return f;
}

// TF32 B operand: rows n = 16p + i hold piece p (W0, then W1 = W - W0) of row i
// of M (W, or W^T for the adjoint), K-major core-matrix layout, 32 x 16 TF32.
static void split_w_pieces_tf32(const float *M, int transpose, unsigned char *out) {
    memset(out, 0, kTcWTf32Bytes);
    for (int n = 0; n < 32; ++n)
        for (int k = 0; k < 16; ++k) {
            const int p = n / 16, i = n % 16;
            const float w = transpose ? M[k * 16 + i] : M[i * 16 + k];
            const float w0 = round_tf32_host(w);
            const float w1 = round_tf32_host(w - w0);
            const float piece = p == 0 ? w0 : w1;
            const size_t off = (n / 8) * 512 + (k / 4) * 128 + (n % 8) * 16 + (k % 4) * 4;
            memcpy(out + off, &piece, 4);
        }
}

// Device layout of the weight pieces: BF16 forward and adjoint (1536 bytes
// each), then TF32 forward and adjoint (2048 bytes each).
static size_t wpieces_offset(int np, bool adjoint) {
    return np == 0 ? 2 * kTcWBf16Bytes + (adjoint ? kTcWTf32Bytes : 0) : (adjoint ? kTcWBf16Bytes : 0);
}

gtt_status_t tc_upload_w(gtt_plan_s *P) {
    constexpr size_t total = 2 * kTcWBf16Bytes + 2 * kTcWTf32Bytes;
    if (!P->d_wpieces) {
        cudaError_t e = cudaMalloc(&P->d_wpieces, total);
        if (e != cudaSuccess) {
            P->d_wpieces = nullptr;
            return set_error(GTT_ERR_ALLOC, "tensor-core weight pieces");
        }
    }
    unsigned char host[total];
    const float *W = reinterpret_cast<const float *>(P->Wf.data());  // element layout prefix
    split_w_pieces(W, 0, host);
    split_w_pieces(W, 1, host + kTcWBf16Bytes);
    split_w_pieces_tf32(W, 0, host + 2 * kTcWBf16Bytes);
    split_w_pieces_tf32(W, 1, host + 2 * kTcWBf16Bytes + kTcWTf32Bytes);
    cudaError_t e = cudaMemcpy(P->d_wpieces, host, sizeof host, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_error(e, "uploading tensor-core weight pieces");
    return GTT_OK;
}

static const void *tc_kernel(int g, int np) {
    if (np == 0)
        return g == 3 ? (const void *)&gtt_tc16_pass_kernel<3, 0>
                      : g == 2 ? (const void *)&gtt_tc16_pass_kernel<2, 0> : (const void *)&gtt_tc16_pass_kernel<1, 0>;
    if (np == 2)
        return g == 3 ? (const void *)&gtt_tc16_pass_kernel<3, 2>
                      : g == 2 ? (const void *)&gtt_tc16_pass_kernel<2, 2> : (const void *)&gtt_tc16_pass_kernel<1, 2>;
    return g == 3 ? (const void *)&gtt_tc16_pass_kernel<3, 3>
                  : g == 2 ? (const void *)&gtt_tc16_pass_kernel<2, 3> : (const void *)&gtt_tc16_pass_kernel<1, 3>;
}

// CTAs of a tensor-core pass kernel per SM, from the register and shared-memory
// budgets (the occupancy query under-reports kernels that allocate tensor
// memory), capped by the 4 x 128 TMEM columns of an SM; 0 on failure
static int tc_residency(gtt_plan_s *P, const void *k, int np) {
    if (allow_max_smem(k, P->smem_optin) != cudaSuccess ||
        cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess)
        return 0;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) return 0;
    int regs_per_sm = 0, smem_per_sm = 0;
    cudaDeviceGetAttribute(&regs_per_sm, cudaDevAttrMaxRegistersPerMultiprocessor, P->device);
    cudaDeviceGetAttribute(&smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, P->device);
    const int by_regs = regs_per_sm / std::max(1, fa.numRegs * kTcThreads);
    const int by_smem = smem_per_sm / (int)(tc_smem_per_cta(np) + 1024);
    return std::min(std::min(by_regs, by_smem), 4);
}

// CTAs per SM at most, by variant (TF32X3; BF16X2 and BF16X3) and pass
// (g = 1, 2, 3).  Measured on b16_n6_batch64: the g = 2 pass (64-byte runs at
// a 16 KiB stride) slows down with more resident CTAs -- TF32X3 2112 / 1910 /
// 1649 us at 4 / 3 / 2 CTAs per SM, BF16X3 1930 / 1627 / 1837 us -- while the
// g = 3 pass is fastest at 4 (1591 against 1744 us at 3).
static int tc_ctas_cap(int np, int g) {
    static const int cap[2][3] = {{4, 2, 4}, {4, 3, 4}};
    return cap[np == 0 ? 0 : 1][g - 1];
}

// Tensor-core schedule for b = 16, n >= 3: digits (3, r=1), then (2, r=16)
// passes, and a final (1, r=256) pass when one digit is left.
gtt_status_t make_tc_schedule(gtt_plan_s *P, int np, std::vector<PassPlan> *out) {
    if (P->b != 16 || P->dtype != GTT_F32 || P->n < 3)
        return set_error(GTT_ERR_UNSUPPORTED, "the b = 16 tensor-core paths need b = 16, FP32 and n >= 3");
    std::vector<PassPlan> passes;
    int m0 = 0;
    while (m0 < P->n) {
        const int left = P->n - m0;
        const int g = m0 == 0 ? 3 : (left >= 2 ? 2 : 1);
        const long long r = m0 == 0 ? 1 : (g == 2 ? 16 : 256);
        const void *k = tc_kernel(g, np);
        const int per_sm = std::min(tc_residency(P, k, np), tc_ctas_cap(np, g));
        if (per_sm < 1) return set_error(GTT_ERR_UNSUPPORTED, "tensor-core kernel cannot be resident");
        PassPlan pp;
        gtt_status_t st = build_pass(P, m0, g, r, 1, &pp);
        if (st != GTT_OK) return st;
        pp.tc.on = true;
        pp.tc.g = g;
        pp.tc.kern = k;
        pp.tc.grid = (int)std::min<long long>((long long)per_sm * P->num_sms, pp.params.tiles);
        pp.tc.ctas_per_sm = per_sm;
        pp.tc.block = kTcThreads;
        pp.tc.smem = tc_smem_per_cta(np);
        pp.tc.np = np;
        pp.tc.name = std::string("gtt_tc16_pass_kernel<") + (np == 3 ? "bf16x3" : np == 2 ? "bf16x2" : "tf32x3") + ",g=" +
                     std::to_string(g) + ">";
        passes.push_back(pp);
        m0 += g;
    }
    *out = passes;
    return GTT_OK;
}

gtt_status_t tc_run(gtt_plan_s *P, PassPlan &pp, bool adjoint, const void *in, void *out, cudaStream_t s,
                    long long tile_begin, long long tile_end) {
    TcParams tp;
    memset(&tp, 0, sizeof(tp));
    tp.p = pp.params;
    tp.p.tile_begin = tile_begin;
    tp.p.tiles = tile_end;
    const int grid = (int)std::min<long long>(pp.tc.grid, tile_end - tile_begin);
    tp.g = pp.tc.g;
    tp.wpieces = (const unsigned char *)P->d_wpieces + wpieces_offset(pp.tc.np, adjoint);
    tp.err = P->dev_err;
    void *args[3] = {(void *)&in, (void *)&out, (void *)&tp};
    return launch_timed(P, pp.tc.kern, dim3(grid), dim3(pp.tc.block), args, pp.tc.smem, s, pp.tc.name);
}

} // namespace gtt
