// Host side of the complex64 b = 4 tensor-core passes (gtt_tcx.cuh): the
// TF32 pieces of W (x) W as the MMA's B operand, the schedule (a 7-digit
// contiguous pass, then 6-digit strided passes), tensor maps and launches.
#include <cudaTypedefs.h>

#include <algorithm>
#include <complex>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "gtt_plan.h"
#include "gtt_tcx.cuh"

namespace gtt {

static PFN_cuTensorMapEncodeTiled_v12000 tcx_encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

// Round a float to TF32 (10 explicit mantissa bits), to nearest with ties away
// from zero, on its bit pattern: add half a TF32 unit to the magnitude bits,
// clear the 13 bits below.  (Finite inputs far below FLT_MAX only.)
static float round_tf32(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    u = (u + 0x1000u) & 0xFFFFE000u;
    memcpy(&f, &u, 4);
    return f;
}

// The MMA's B operand for one 16 x 16 complex matrix M: the 32 x 32 real R of
// the complex product (interleaved rows and columns), split as R = R0 + R1
// into TF32 pieces, stored as rows n = 0..31 (R0) and 32..63 (R1) of a 64 x 32
// K-major core-matrix layout (8 rows x 16 bytes; K-neighbour core matrices
// 128 bytes apart, 8-row groups 1024 bytes apart).
static void tcx_b_operand(const std::complex<double> *M, float *out) {
    memset(out, 0, kTcxBBytes);
    for (int n = 0; n < 32; ++n)
        for (int k = 0; k < 32; ++k) {
            const std::complex<double> m = M[(n / 2) * 16 + k / 2];
            const double r = (n % 2 == k % 2) ? m.real() : (n % 2 == 0 ? -m.imag() : m.imag());
            const float r0 = round_tf32((float)r);
            const float r1 = round_tf32((float)(r - (double)r0));
            for (int piece = 0; piece < 2; ++piece) {
                const int row = n + 32 * piece;
                const size_t off = (size_t)(row / 8) * 256 + (size_t)(k / 4) * 32 + (row % 8) * 4 + (k % 4);
                out[off] = piece ? r1 : r0;
            }
        }
}

// W (x) W from the plan's W or W^H bytes (complex64, row-major 4 x 4), in
// double: rows and columns d = h_low + 4 h_high (the higher digit's factor on
// the left, as in Def. 2.3).
static void kron_ww(const std::vector<unsigned char> &Wb, std::complex<double> *M) {
    std::complex<double> w[16];
    for (int i = 0; i < 16; ++i) {
        float re, im;
        memcpy(&re, Wb.data() + 8 * i, 4);
        memcpy(&im, Wb.data() + 8 * i + 4, 4);
        w[i] = {re, im};
    }
    for (int o1 = 0; o1 < 4; ++o1)
        for (int o0 = 0; o0 < 4; ++o0)
            for (int i1 = 0; i1 < 4; ++i1)
                for (int i0 = 0; i0 < 4; ++i0) M[(4 * o1 + o0) * 16 + 4 * i1 + i0] = w[o1 * 4 + i1] * w[o0 * 4 + i0];
}

bool tcx_eligible(const gtt_plan_s *P) {
    return !P->mixed && P->b == 4 && P->dtype == GTT_C64 && P->n >= 7 && (P->n - 7) % 6 == 0;
}

gtt_status_t tcx_upload_w(gtt_plan_s *P) {
    if (!P->d_tcx) {
        cudaError_t e = cudaMalloc(&P->d_tcx, 2 * kTcxBBytes);
        if (e != cudaSuccess) {
            P->d_tcx = nullptr;
            return set_error(GTT_ERR_ALLOC, "TF32 weight pieces");
        }
    }
    std::vector<float> host(2 * kTcxBBytes / 4);
    std::complex<double> M[256];
    kron_ww(P->Wf, M);
    tcx_b_operand(M, host.data());
    kron_ww(P->Wa, M);
    tcx_b_operand(M, host.data() + kTcxBBytes / 4);
    cudaError_t e = cudaMemcpy(P->d_tcx, host.data(), 2 * kTcxBBytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_error(e, "uploading TF32 weight pieces");
    return GTT_OK;
}

template <bool C> static const void *tcx_kernel() {
    return C ? (const void *)&gtt_tcx_pass_kernel<true> : (const void *)&gtt_tcx_pass_kernel<false>;
}

// Clusters of a tcx kernel that are resident at once (0 when it cannot run):
// one CTA per SM -- the cluster launch of a kernel that allocates tensor
// memory places one CTA per SM -- within the GPU's cluster placement limits.
static int tcx_clusters(gtt_plan_s *P, const void *k, size_t smem) {
    if (allow_max_smem(k, P->smem_optin) != cudaSuccess ||
        cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess)
        return 0;
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(kTcxCluster * P->num_sms);
    cfg.blockDim = dim3(kTcxBlock);
    cfg.dynamicSmemBytes = smem;  // the cluster shape is the kernel's compile-time one
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess) return 0;
    return std::min(n, P->num_sms / kTcxCluster);
}

// Schedule: pass 0 covers digits 0..6 (contiguous tiles of 4^6, digit 6 across
// the cluster), then passes of 6 digits m0..m0+5 (runs of 4 low elements,
// digits m0..m0+4 in the tile, m0+5 across the cluster).
gtt_status_t make_tcx_schedule(gtt_plan_s *P, std::vector<PassPlan> *out) {
    if (!tcx_eligible(P)) return set_error(GTT_ERR_UNSUPPORTED, "TF32X3 needs b = 4, complex64 and n = 7 + 6k");
    if (!tcx_encode_fn()) return set_error(GTT_ERR_UNSUPPORTED, "tensor-map encoding is not available");
    if (P->total / 16 > (1ll << 31)) return set_error(GTT_ERR_UNSUPPORTED, "data too large for 32-bit TMA rows");
    std::vector<PassPlan> passes;
    int m0 = 0;
    while (m0 < P->n) {
        const bool contig = m0 == 0;
        const int g = contig ? 7 : 6;
        const void *k = contig ? tcx_kernel<true>() : tcx_kernel<false>();
        const size_t smem = tcx_smem_bytes();
        if (smem > (size_t)P->smem_optin) return set_error(GTT_ERR_UNSUPPORTED, "tcx tile ring exceeds shared memory");
        const int maxc = tcx_clusters(P, k, smem);
        if (maxc < 1) return set_error(GTT_ERR_UNSUPPORTED, "tcx kernel cannot be resident");
        PassPlan pp;
        memset(&pp.params, 0, sizeof(pp.params));
        pp.m0 = m0;
        pp.g = g;
        pp.r = contig ? 1 : 4;
        pp.D = 1;
        long long L = 1;
        for (int i = 0; i < m0; ++i) L *= 4;
        TcxPass &t = pp.tcx;
        t.on = true;
        t.contig = contig;
        t.kern = k;
        t.smem = smem;
        t.ctiles = P->total / (4 * kTcxTile);
        t.grid = (int)std::min<long long>(maxc, t.ctiles) * kTcxCluster;
        t.L = L;
        t.name = std::string("gtt_tcx_pass_kernel<c64,4,") + (contig ? "contig" : "strided") + ">";
        pp.params.tile_elems = 4 * kTcxTile;  // per cluster
        pp.params.tiles = t.ctiles;
        pp.params.total = P->total;
        pp.params.L = L;
        pp.params.M = contig ? 4 * kTcxTile : 4096;
        pp.params.r = (uint32_t)pp.r;
        passes.push_back(pp);
        m0 += g;
    }
    *out = passes;
    return GTT_OK;
}

static gtt_status_t tcx_encode(gtt_plan_s *P, const void *ptr, CUtensorMap *map) {
    cuuint64_t dims[2] = {16, (cuuint64_t)(P->total / 16)};
    cuuint64_t strides[1] = {128};
    cuuint32_t box[2] = {16, 256};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = tcx_encode_fn()(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void *>(ptr), dims, strides, box,
                                 estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(GTT_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return GTT_OK;
}

gtt_status_t tcx_run(gtt_plan_s *P, PassPlan &pp, bool adjoint, const void *in, void *outp, cudaStream_t s) {
    TcxPass &t = pp.tcx;
    if (t.contig && t.map_ptr != in) {
        gtt_status_t st = tcx_encode(P, in, &t.map);
        if (st != GTT_OK) return st;
        t.map_ptr = in;
    }
    TcxParams prm;
    memset(&prm, 0, sizeof(prm));
    prm.ctiles = t.ctiles;
    prm.L = t.L;
    prm.stride_top = t.L * 1024;   // 4^(m0+5)
    prm.stride_hi = t.L * 4096;    // 4^(m0+6)
    prm.lo_runs = (uint32_t)(t.L / 4);
    prm.div_lo_runs.init(std::max<uint32_t>(1u, prm.lo_runs));
    prm.bmat = reinterpret_cast<const float *>((const unsigned char *)P->d_tcx + (adjoint ? kTcxBBytes : 0));
    const std::vector<unsigned char> &Wb = adjoint ? P->Wa : P->Wf;  // complex64, row-major 4 x 4
    for (int i = 0; i < 16; ++i) {
        float re, im;
        memcpy(&re, Wb.data() + 8 * i, 4);
        memcpy(&im, Wb.data() + 8 * i + 4, 4);
        prm.wa[i] = make_float2(re, re);
        prm.wb[i] = make_float2(-im, im);
    }
    prm.err = P->dev_err;
    const CUtensorMap *mp = &t.map;  // strided passes do not read it
    const float2 *inp = (const float2 *)in;
    float2 *op = (float2 *)outp;
    void *args[4] = {(void *)mp, (void *)&inp, (void *)&op, (void *)&prm};
    return launch_timed(P, t.kern, dim3(t.grid), dim3(kTcxBlock), args, t.smem, s, t.name);
}

} // namespace gtt
