// C ABI of libgtt (declared in include/gtt.h): plans, schedules, launches.
//
// A plan holds W (and W^H) in the element type, a fusion schedule -- the list
// of passes, each applying a contiguous group of modes of Algorithm 1 in one
// HBM round trip -- and the launch geometry of every pass.
#include <algorithm>
#include <complex>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/gtt.h"
#include "gtt_internal.h"
#include "gtt_plan.h"

using namespace gtt;

static thread_local std::string g_last_error;

namespace gtt {

gtt_status_t set_error(gtt_status_t st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

gtt_status_t cuda_error(cudaError_t e, const char *what) {
    return set_error(GTT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

static long long ipow_ll(int b, int e) {
    long long r = 1;
    for (int i = 0; i < e; ++i) r *= b;
    return r;
}

// Build the launch description of one pass (modes [m0, m0+g), run r, window D).
// The first pass has no lower digits to run over; there r > 1 means tiles of r
// consecutive blocks of b^g contiguous elements (the register stages treat the
// block index like any digit above their window, and leave it untouched).
gtt_status_t build_pass(gtt_plan_s *P, int m0, int g, long long r, int D, PassPlan *out) {
    long long kblk = 1, rr = r;
    if (m0 == 0 && r > 1) {
        kblk = r;
        rr = 1;
    }
    gtt_status_t st = build_pass_geom(P, P->b, ipow_ll(P->b, m0), g, kblk, rr, D, out);
    if (st != GTT_OK) return st;
    out->m0 = m0;
    out->r = r;
    return GTT_OK;
}

// The geometry core: digits of radix b at stride L (the product of the radices
// below them), g of them per tile, kblk consecutive blocks of b^g rows per tile
// (the rows of block hi + 1 follow those of block hi at the same stride L),
// runs of r elements (r divides L), register windows of D digits.
gtt_status_t build_pass_geom(gtt_plan_s *P, int b, long long L, int g, long long kblk, long long r, int D,
                             PassPlan *out) {
    const int es = P->es;
    PassPlan pp;
    pp.g = g;
    pp.D = D;
    pp.r = r;
    const long long M = ipow_ll(b, g) * kblk;
    if (r < 1 || L % r != 0 || g < D || g < 1) return set_error(GTT_ERR_INTERNAL, "bad pass geometry");
    if (P->total % (M * r) != 0) return set_error(GTT_ERR_INVALID_ARG, "blocks per tile must divide the data");
    if (L / r > (1ll << 31) || M * r > (1ll << 24))
        return set_error(GTT_ERR_UNSUPPORTED, "pass geometry exceeds 32-bit tile indexing");
    const long long tile = M * r;
    const int RB = (int)ipow_ll(b, D);
    PassParams &p = pp.params;
    memset(&p, 0, sizeof(p));
    p.total = P->total;
    p.L = L;
    p.tiles = P->total / tile;
    p.r = (uint32_t)r;
    p.M = (uint32_t)M;
    p.tile_elems = (uint32_t)tile;
    p.lo_blocks = (uint32_t)(L / r);
    p.div_lo_blocks.init(p.lo_blocks);
    p.div_r.init((uint32_t)r);
    const int CE = 16 / es;
    if (L == r && tile % CE == 0)
        p.vec_mode = 1;
    else if (r % CE == 0 && L % CE == 0)
        p.vec_mode = 2;
    else
        p.vec_mode = 0;
    p.div_cpr.init(p.vec_mode == 2 ? (uint32_t)(r / CE) : 1u);
    // register stages: windows [s*D, s*D+D), the last slid down to [g-D, g)
    const int S = (g + D - 1) / D;
    if (S > kMaxStages) return set_error(GTT_ERR_INTERNAL, "too many stages");
    p.nstages = S;
    for (int s = 0; s < S; ++s) {
        int a = s * D, mask = (1 << D) - 1;
        if (a + D > g) {
            const int first_new = a;  // digits below were applied by earlier stages
            a = g - D;
            mask = 0;
            for (int k = 0; k < D; ++k)
                if (a + k >= first_new) mask |= 1 << k;
        }
        p.stage_a[s] = a;
        p.stage_mask[s] = mask;
        p.stage_strideA[s] = (uint32_t)(r * ipow_ll(b, a));
        p.stage_divBa[s].init((uint32_t)ipow_ll(b, a));
    }
    pp.kern = pass_kernel((int)P->dtype, b, D);
    if (!pp.kern) return set_error(GTT_ERR_INTERNAL, "no kernel instantiation for (dtype, b, D)");
    const long long nslots = tile / RB;
    int block = (int)std::min<long long>(kPassMaxThreads, ((nslots + 31) / 32) * 32);
    pp.block = std::max(block, 32);
    pp.smem = (size_t)(tile + tile / RB + 1) * es;
    pp.smem = (pp.smem + 15) / 16 * 16;
    if (pp.smem > 227 * 1024) return set_error(GTT_ERR_INTERNAL, "tile exceeds shared memory");
    cudaError_t e;
    e = allow_max_smem(pp.kern, P->smem_optin);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(pp.kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pp.kern, pp.block, pp.smem);
    if (e != cudaSuccess) return cuda_error(e, "occupancy query");
    if (per_sm < 1) return set_error(GTT_ERR_UNSUPPORTED, "pass kernel cannot be resident");
    long long grid = (long long)per_sm * P->num_sms;
    pp.grid = (int)std::min<long long>(grid, p.tiles);
    pp.ctas_per_sm = per_sm;
    static const char *tnames[] = {"f64", "f32", "c64", "c128", "u32"};
    pp.name = std::string("gtt_pass_kernel<") + tnames[(int)P->dtype] + "," + std::to_string(b) +
              "," + std::to_string(D) + ">";
    *out = pp;
    return GTT_OK;
}

// Fixed-rule schedule: greedy passes with tiles of at most max_tile_bytes and
// runs of at least min_run_bytes (when the lower digits allow it).
gtt_status_t make_schedule(gtt_plan_s *P, long long max_tile_bytes, long long min_run_bytes,
                           std::vector<PassPlan> *out) {
    const int b = P->b, n = P->n, es = P->es;
    const int DM = dmax_bytes(es, b);
    long long tmax = std::max<long long>(max_tile_bytes / es, b);
    // FP64 arithmetic runs at a small fraction of the FP32 rate, so a small
    // FP64 / complex128 transform that one or two CTAs would hold is spread
    // over many CTAs instead: tiles of at most b^3 elements, runs of 1.
    // (b = 2, n = 12, FP64: 4 passes of 512 CTAs, 12.5 us per forward in a
    // CUDA graph, against 32 us for one pass on one CTA.)
    if ((P->dtype == GTT_F64 || P->dtype == GTT_C128) && P->total * es <= 2 * max_tile_bytes) {
        tmax = std::min<long long>(tmax, (long long)b * b * b);
        min_run_bytes = 0;
    }
    std::vector<PassPlan> passes;
    // FP32, b = 8, default settings: the tile kernels' schedule, digits 0-3
    // and then at most 3 digits on runs of 8^(4-g) (b8_n7: 245 us per forward
    // against 302 us for the greedy [4, 2, 1])
    if (P->dtype == GTT_F32 && b == 8 && n >= 4 && max_tile_bytes == kDefaultTileBytes &&
        min_run_bytes == kDefaultRunBytes) {
        for (int m = 0; m < n;) {
            const int g = m == 0 ? 4 : std::min(3, n - m);
            long long r = 1;
            for (int i = g; m > 0 && i < 4; ++i) r *= 8;
            PassPlan pp;
            gtt_status_t st = build_pass(P, m, g, r, 1, &pp);
            if (st != GTT_OK) return st;
            if (!tile8_attach(P, &pp) && P->use_tma) tma_attach(P, &pp, P->tma_nbuf);
            passes.push_back(pp);
            m += g;
        }
        *out = passes;
        return GTT_OK;
    }
    int m0 = 0;
    while (m0 < n) {
        long long r = 1;
        if (m0 > 0) {
            // r = b^j, j <= m0: smallest with r*es >= min_run_bytes, keeping b*r <= tmax
            int j = 0;
            while (j < m0 && r * es < min_run_bytes && r * b * b <= tmax) {
                r *= b;
                ++j;
            }
        }
        int g = 0;
        long long M = 1;
        while (m0 + g < n && M * b * r <= tmax) {
            M *= b;
            ++g;
        }
        if (g == 0) g = 1;
        if (m0 > 0) {
            // all remaining digits fit: widen the run to fill the tile
            long long L = 1;
            for (int i = 0; i < m0; ++i) L *= b;
            while (m0 + g == n && r * b <= L && M * r * b <= tmax) r *= b;
        }
        const int D = g >= DM ? DM : 1;
        PassPlan pp;
        gtt_status_t st = build_pass(P, m0, g, r, D, &pp);
        if (st != GTT_OK) return st;
        if (!tile8_attach(P, &pp) && P->use_tma) tma_attach(P, &pp, P->tma_nbuf);
        passes.push_back(pp);
        m0 += g;
    }
    *out = passes;
    return GTT_OK;
}

} // namespace gtt

// ------------------------------------------------------------------ C ABI

// Extend a row-major b x b matrix (element layout) to the kernels' parameter
// layout WMat<T, B>: complex64 appends the pairs (re, re) and (-im, im) of
// every entry; FP32 appends the row pairs (W[2i][j], W[2i+1][j]) (for odd b
// the 4 bytes that align the pair array, then a single unused pair); other
// types use the element layout as it is.  The result has the size of WMat<T, b>.
static void append_packed_pairs(int dtype, int b, std::vector<unsigned char> *Wv) {
    if (dtype == GTT_C64) {
        std::vector<float> ex;
        const float *w = reinterpret_cast<const float *>(Wv->data());
        for (int k = 0; k < b * b; ++k) {
            ex.push_back(w[2 * k]);
            ex.push_back(w[2 * k]);
        }
        for (int k = 0; k < b * b; ++k) {
            ex.push_back(-w[2 * k + 1]);
            ex.push_back(w[2 * k + 1]);
        }
        const unsigned char *p = reinterpret_cast<const unsigned char *>(ex.data());
        Wv->insert(Wv->end(), p, p + ex.size() * sizeof(float));
    } else if (dtype == GTT_F32) {
        std::vector<float> ex;
        const float *w = reinterpret_cast<const float *>(Wv->data());
        if (b % 2 == 0) {
            for (int ip = 0; ip < b / 2; ++ip)
                for (int j = 0; j < b; ++j) {
                    ex.push_back(w[(2 * ip) * b + j]);
                    ex.push_back(w[(2 * ip + 1) * b + j]);
                }
        } else {
            ex.assign(3, 0.f);
        }
        const unsigned char *p = reinterpret_cast<const unsigned char *>(ex.data());
        Wv->insert(Wv->end(), p, p + ex.size() * sizeof(float));
    }
}

// W (host, b x b of the element type) and W^H (the transpose, conjugated for
// complex types), both in the kernels' parameter layout.
static void make_w_params(int dtype, int es, int b, const void *W, std::vector<unsigned char> *Wf,
                          std::vector<unsigned char> *Wa) {
    const size_t wbytes = (size_t)b * b * es;
    Wf->assign((const unsigned char *)W, (const unsigned char *)W + wbytes);
    Wa->resize(wbytes);
    for (int i = 0; i < b; ++i)
        for (int j = 0; j < b; ++j) {
            unsigned char *dst = &(*Wa)[((size_t)i * b + j) * es];
            const unsigned char *src = &(*Wf)[((size_t)j * b + i) * es];
            memcpy(dst, src, es);
            if (dtype == GTT_C64) {
                float im;
                memcpy(&im, dst + 4, 4);
                im = -im;
                memcpy(dst + 4, &im, 4);
            } else if (dtype == GTT_C128) {
                double im;
                memcpy(&im, dst + 8, 8);
                im = -im;
                memcpy(dst + 8, &im, 8);
            }
        }
    append_packed_pairs(dtype, b, Wf);
    append_packed_pairs(dtype, b, Wa);
}

// Kronecker product W_lo (x) W_lo+1 (x) ... (x) W_hi of adjacent factors, in
// the element layout of `dtype` (row-major).  Formed in double (complex
// double) and rounded once; int32 entries multiply modulo 2^32.
static std::vector<unsigned char> kron_factors(int dtype, int es, const std::vector<int> &radices,
                                               const std::vector<size_t> &off, const unsigned char *W, int lo,
                                               int hi) {
    const bool integer = dtype == GTT_I32;
    auto entry = [&](int k, int i) -> std::complex<double> {
        const unsigned char *p = W + off[k] + (size_t)i * es;
        switch (dtype) {
        case GTT_F64: return *reinterpret_cast<const double *>(p);
        case GTT_F32: return *reinterpret_cast<const float *>(p);
        case GTT_C64: return {reinterpret_cast<const float *>(p)[0], reinterpret_cast<const float *>(p)[1]};
        case GTT_C128: return {reinterpret_cast<const double *>(p)[0], reinterpret_cast<const double *>(p)[1]};
        default: return 0.0;
        }
    };
    int m = radices[lo];
    std::vector<std::complex<double>> M((size_t)m * m);
    std::vector<uint32_t> Mi((size_t)m * m);
    for (int i = 0; i < m * m; ++i) {
        M[i] = entry(lo, i);
        if (integer) Mi[i] = (uint32_t)*reinterpret_cast<const int32_t *>(W + off[lo] + (size_t)i * es);
    }
    for (int k = lo + 1; k <= hi; ++k) {
        const int c = radices[k], mc = m * c;
        std::vector<std::complex<double>> N((size_t)mc * mc);
        std::vector<uint32_t> Ni((size_t)mc * mc);
        for (int i1 = 0; i1 < m; ++i1)
            for (int j1 = 0; j1 < m; ++j1)
                for (int i2 = 0; i2 < c; ++i2)
                    for (int j2 = 0; j2 < c; ++j2) {
                        const size_t o = (size_t)(i1 * c + i2) * mc + (j1 * c + j2);
                        if (integer)
                            Ni[o] = Mi[(size_t)i1 * m + j1] *
                                    (uint32_t)*reinterpret_cast<const int32_t *>(W + off[k] + (size_t)(i2 * c + j2) * es);
                        else
                            N[o] = M[(size_t)i1 * m + j1] * entry(k, i2 * c + j2);
                    }
        M.swap(N);
        Mi.swap(Ni);
        m = mc;
    }
    std::vector<unsigned char> out((size_t)m * m * es);
    for (int i = 0; i < m * m; ++i) {
        unsigned char *p = out.data() + (size_t)i * es;
        if (integer) {
            const int32_t v = (int32_t)Mi[i];
            memcpy(p, &v, 4);
        } else if (dtype == GTT_F64) {
            const double v = M[i].real();
            memcpy(p, &v, 8);
        } else if (dtype == GTT_F32) {
            const float v = (float)M[i].real();
            memcpy(p, &v, 4);
        } else if (dtype == GTT_C64) {
            const float v[2] = {(float)M[i].real(), (float)M[i].imag()};
            memcpy(p, v, 8);
        } else {
            const double v[2] = {M[i].real(), M[i].imag()};
            memcpy(p, v, 16);
        }
    }
    return out;
}

// Copy W into the plan: one matrix, or for a mixed plan the factors
// W_0, ..., W_{n-1} back to back; each stage of a mixed pass gets its own
// factor and adjoint (a single factor, or the Kronecker product of the
// adjacent factors it covers) in its slot of the pass's kernel parameters.
static gtt_status_t set_w_bytes(gtt_plan_s *P, const void *W) {
    if (!P->mixed) {
        make_w_params((int)P->dtype, P->es, P->b, W, &P->Wf, &P->Wa);
        return GTT_OK;
    }
    const int n = P->n;
    std::vector<size_t> off(n + 1, 0);  // byte offset of factor k
    for (int k = 0; k < n; ++k) off[k + 1] = off[k] + (size_t)P->radices[k] * P->radices[k] * P->es;
    size_t w_offset = 0, slot_bytes = 0;
    int slots = 0;
    const size_t args_bytes = mixed_args_bytes((int)P->dtype, &w_offset, &slot_bytes, &slots);
    for (PassPlan &pp : P->passes) {
        MixPass &mx = pp.mix;
        mx.args_f.assign(args_bytes, 0);
        mx.args_a.assign(args_bytes, 0);
        memcpy(mx.args_f.data(), &mx.params, sizeof(MixedParams));
        memcpy(mx.args_a.data(), &mx.params, sizeof(MixedParams));
        for (int k = 0; k < mx.params.nst; ++k) {
            const int hi = mx.hi[k], lo = mx.hi[k] - mx.cnt[k] + 1;
            std::vector<unsigned char> f, a;
            if (mx.cnt[k] == 1) {
                make_w_params((int)P->dtype, P->es, P->radices[hi], (const unsigned char *)W + off[hi], &f, &a);
            } else {
                const std::vector<unsigned char> K =
                    kron_factors((int)P->dtype, P->es, P->radices, off, (const unsigned char *)W, lo, hi);
                make_w_params((int)P->dtype, P->es, mx.params.rad[k], K.data(), &f, &a);
            }
            if (k >= slots || f.size() != wmat_size((int)P->dtype, mx.params.rad[k]) || f.size() > slot_bytes)
                return set_error(GTT_ERR_INTERNAL, "factor layout size");
            memcpy(mx.args_f.data() + w_offset + k * slot_bytes, f.data(), f.size());
            memcpy(mx.args_a.data() + w_offset + k * slot_bytes, a.data(), a.size());
        }
    }
    return GTT_OK;
}

extern "C" gtt_status_t gtt_plan_set_w(gtt_plan_t P, const void *W) {
    if (!P || !W) return set_error(GTT_ERR_INVALID_ARG, "NULL plan or W");
    gtt_status_t st = set_w_bytes(P, W);
    if (st != GTT_OK) return st;
    if (P->precision == GTT_PREC_BF16X3 || P->precision == GTT_PREC_BF16X2 ||
        (P->precision == GTT_PREC_TF32X3 && P->b == 16))
        return tc_upload_w(P);
    if (P->precision == GTT_PREC_TF32X3) return tcx_upload_w(P);
    return GTT_OK;
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

static gtt_status_t check_device(gtt_plan_s *P) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev != P->device)
        return set_error(GTT_ERR_INVALID_ARG, "current CUDA device differs from the plan's device");
    return GTT_OK;
}

// AUTO's choice: the tensor-core path where it exists (b = 16, FP32, n >= 3),
// which is faster than the CUDA-core path and at least as accurate; FP32 CUDA
// cores everywhere else.
static bool tc_eligible(const gtt_plan_s *P) { return P->b == 16 && P->dtype == GTT_F32 && P->n >= 3; }

// Back to a CUDA-core schedule (the plan's fixed rule or its explicit passes).
static gtt_status_t use_cuda_core(gtt_plan_s *P) {
    if (P->precision == GTT_PREC_BF16X3 || P->precision == GTT_PREC_BF16X2 || P->precision == GTT_PREC_TF32X3) {
        std::vector<PassPlan> passes;
        gtt_status_t st = P->explicit_g.empty()
                              ? make_schedule(P, P->sched_tile_bytes, P->sched_run_bytes, &passes)
                              : make_explicit_schedule(P, (int)P->explicit_g.size(), P->explicit_g.data(),
                                                       P->explicit_r.data(), &passes);
        if (st != GTT_OK) return st;
        P->passes = passes;
    }
    P->precision = GTT_PREC_FP32;
    return GTT_OK;
}

static gtt_status_t use_complex_tensor_cores(gtt_plan_s *P) {
    std::vector<PassPlan> passes;
    gtt_status_t st = make_tcx_schedule(P, &passes);
    if (st != GTT_OK) return st;
    st = tcx_upload_w(P);
    if (st != GTT_OK) return st;
    P->passes = passes;
    P->precision = GTT_PREC_TF32X3;
    return GTT_OK;
}

static gtt_status_t use_tensor_cores(gtt_plan_s *P, int np = 3) {
    std::vector<PassPlan> passes;
    gtt_status_t st = make_tc_schedule(P, np, &passes);
    if (st != GTT_OK) return st;
    st = tc_upload_w(P);
    if (st != GTT_OK) return st;
    P->passes = passes;
    P->precision = np == 3 ? GTT_PREC_BF16X3 : np == 2 ? GTT_PREC_BF16X2 : GTT_PREC_TF32X3;
    return GTT_OK;
}

static gtt_status_t plan_create(gtt_plan_t *out, int b, int n, const void *W, gtt_dtype_t dtype, long long batch);

extern "C" gtt_status_t gtt_plan_create(gtt_plan_t *out, int b, int n, const void *W,
                                        gtt_dtype_t dtype, long long batch) {
    nvtxRangePushA("gtt_plan_create");
    const gtt_status_t st = plan_create(out, b, n, W, dtype, batch);
    nvtxRangePop();
    return st;
}

static gtt_status_t plan_create(gtt_plan_t *out, int b, int n, const void *W, gtt_dtype_t dtype, long long batch) {
    if (!out || !W) return set_error(GTT_ERR_INVALID_ARG, "NULL out or W");
    *out = nullptr;
    if (b < 2 || b > 16) return set_error(GTT_ERR_INVALID_ARG, "b must be in [2, 16]");
    if (n < 1) return set_error(GTT_ERR_INVALID_ARG, "n must be >= 1");
    if (batch < 1) return set_error(GTT_ERR_INVALID_ARG, "batch must be >= 1");
    if ((int)dtype < 0 || (int)dtype > 4) return set_error(GTT_ERR_INVALID_ARG, "unknown dtype");
    long long N = 1;
    for (int i = 0; i < n; ++i) {
        N *= b;
        if (N > (1ll << 36)) return set_error(GTT_ERR_INVALID_ARG, "N = b^n above 2^36");
    }
    if (N > (1ll << 40) / batch) return set_error(GTT_ERR_INVALID_ARG, "batch * N above 2^40");
    gtt_plan_s *P = new (std::nothrow) gtt_plan_s();
    if (!P) return set_error(GTT_ERR_ALLOC, "host allocation failed");
    P->b = b;
    P->n = n;
    P->dtype = dtype;
    P->batch = batch;
    P->N = N;
    P->total = N * batch;
    P->es = elem_size((int)dtype);
    cudaError_t e = cudaGetDevice(&P->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&P->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->device);
    if (e != cudaSuccess) {
        delete P;
        return cuda_error(e, "device query");
    }
    const size_t wbytes = (size_t)b * b * P->es;
    (void)wbytes;
    set_w_bytes(P, W);
    e = cudaMalloc(&P->dev_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(P->dev_err, 0, sizeof(int));
    if (e != cudaSuccess) {
        if (P->dev_err) cudaFree(P->dev_err);
        delete P;
        return set_error(GTT_ERR_ALLOC, std::string("error flag: ") + cudaGetErrorString(e));
    }
    P->sched_tile_bytes = kDefaultTileBytes;
    P->sched_run_bytes = kDefaultRunBytes;
    gtt_status_t st = make_schedule(P, kDefaultTileBytes, kDefaultRunBytes, &P->passes);
    if (st != GTT_OK) {
        cudaFree(P->dev_err);
        delete P;
        return st;
    }
    // a schedule from the autotune cache replaces the fixed rule; with
    // GTT_AUTOTUNE=on an uncached shape is tuned now
    if (!tune_apply_cached(P)) {
        const char *at = std::getenv("GTT_AUTOTUNE");
        if (at && std::strcmp(at, "on") == 0) autotune(P, 64);
    }
    // the default precision (AUTO): tensor cores where they apply
    if (tc_eligible(P) && use_tensor_cores(P) != GTT_OK) P->precision = GTT_PREC_FP32;
    *out = P;
    return GTT_OK;
}

extern "C" gtt_status_t gtt_plan_create_mixed(gtt_plan_t *out, int n, const int *radices, const void *W,
                                              gtt_dtype_t dtype, long long batch) {
    if (!out || !W || !radices) return set_error(GTT_ERR_INVALID_ARG, "NULL out, radices or W");
    *out = nullptr;
    if (n < 1) return set_error(GTT_ERR_INVALID_ARG, "n must be >= 1");
    if (batch < 1) return set_error(GTT_ERR_INVALID_ARG, "batch must be >= 1");
    if ((int)dtype < 0 || (int)dtype > 4) return set_error(GTT_ERR_INVALID_ARG, "unknown dtype");
    long long N = 1;
    for (int k = 0; k < n; ++k) {
        if (radices[k] < 2 || radices[k] > 16) return set_error(GTT_ERR_INVALID_ARG, "every b_k must be in [2, 16]");
        N *= radices[k];
        if (N > (1ll << 36)) return set_error(GTT_ERR_INVALID_ARG, "N = prod b_k above 2^36");
    }
    if (N > (1ll << 40) / batch) return set_error(GTT_ERR_INVALID_ARG, "batch * N above 2^40");
    gtt_plan_s *P = new (std::nothrow) gtt_plan_s();
    if (!P) return set_error(GTT_ERR_ALLOC, "host allocation failed");
    P->mixed = true;
    P->radices.assign(radices, radices + n);
    P->b = 0;  // no single base
    P->n = n;
    P->dtype = dtype;
    P->batch = batch;
    P->N = N;
    P->total = N * batch;
    P->es = elem_size((int)dtype);
    P->precision = GTT_PREC_FP32;
    cudaError_t e = cudaGetDevice(&P->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&P->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->device);
    if (e != cudaSuccess) {
        delete P;
        return cuda_error(e, "device query");
    }
    // digits, the fastest first: digit j of the natural index has radix
    // b_{n-1-j} and stride prod_{i < j} b_{n-1-i}.  Adjacent digits whose
    // radices multiply to at most 16 first become one digit of that radix
    // (d_j + b_j d_{j+1} + ...), transformed by the Kronecker product of their
    // factors (the slower digit's factor on the left).  Consecutive such digits
    // then share a pass, one stage each, as many as a tile of at most the
    // default tile size holds and the kernel has factor slots for (three or
    // four): the first pass on contiguous tiles of several consecutive blocks,
    // the later ones on M rows of runs of r contiguous elements (r divides the
    // stride L: at least 64 bytes where L allows, then as long as the tile
    // allows).
    struct MDigit {
        int rad, hi, cnt;
    };
    std::vector<MDigit> md;
    for (int j = 0; j < n;) {
        int g = 1, bj = radices[n - 1 - j];
        while (j + g < n && bj * radices[n - 1 - (j + g)] <= 16) bj *= radices[n - 1 - (j + g++)];
        md.push_back({bj, n - 1 - j, g});
        j += g;
    }
    size_t w_offset = 0, slot_bytes = 0;
    int max_stages = 0;  // factor slots in the mixed kernel's parameters
    mixed_args_bytes((int)dtype, &w_offset, &slot_bytes, &max_stages);
    const long long tmax = kDefaultTileBytes / P->es, rmin = std::max(1, 64 / P->es);
    auto smallest_divisor_at_least = [](long long L, long long lo) {
        for (long long d = lo; d < L; ++d)
            if (L % d == 0) return d;
        return L;
    };
    auto largest_divisor_at_most = [](long long L, long long hi) {
        for (long long d = std::min(L, hi); d > 1; --d)
            if (L % d == 0) return d;
        return 1ll;
    };
    auto drop = [&](gtt_status_t st) {
        if (P->dev_err) cudaFree(P->dev_err);
        delete P;
        return st;
    };
    long long L = 1;
    int digit = 0;
    for (size_t i = 0; i < md.size();) {
        long long r = L == 1 ? 1 : smallest_divisor_at_least(L, rmin);
        if (r * md[i].rad > tmax) r = largest_divisor_at_most(L, tmax / md[i].rad);
        long long M = md[i].rad;
        size_t j = i + 1;
        while (j < md.size() && j - i < (size_t)max_stages && M * md[j].rad * r <= tmax) M *= md[j++].rad;
        if (L > 1) r = std::max(r, largest_divisor_at_most(L, tmax / M));  // longer runs where the tile has room
        // the first pass: as many consecutive blocks per tile as it has room for
        // (while the pass keeps at least two tiles per SM)
        long long kblk =
            L == 1 ? largest_divisor_at_most(P->total / M, std::min(tmax / M, P->total / M / (2ll * P->num_sms))) : 1;
        std::vector<int> rad, hi, cnt;
        int digits = 0;
        for (size_t k = i; k < j; ++k) {
            rad.push_back(md[k].rad);
            hi.push_back(md[k].hi);
            cnt.push_back(md[k].cnt);
            digits += md[k].cnt;
        }
        PassPlan pp;
        gtt_status_t st = build_mixed_pass(P, rad, hi, cnt, L, kblk, r, &pp);
        if (st != GTT_OK) return drop(st);
        pp.m0 = digit;
        pp.factor = md[i].hi;
        pp.factors = digits;
        P->passes.push_back(pp);
        L *= M;
        digit += digits;
        i = j;
    }
    gtt_status_t st = set_w_bytes(P, W);
    if (st != GTT_OK) return drop(st);
    e = cudaMalloc(&P->dev_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(P->dev_err, 0, sizeof(int));
    if (e != cudaSuccess) return drop(set_error(GTT_ERR_ALLOC, std::string("error flag: ") + cudaGetErrorString(e)));
    *out = P;
    return GTT_OK;
}

namespace gtt {
// Build an explicit schedule: pass k covers digits[k] modes with runs[k].
gtt_status_t make_explicit_schedule(gtt_plan_s *P, int count, const int *digits, const long long *runs,
                                    std::vector<PassPlan> *out) {
    if (count < 1 || count > 64 || !digits || !runs) return set_error(GTT_ERR_INVALID_ARG, "bad pass list");
    const int b = P->b, es = P->es, DM = dmax_bytes(es, b);
    int m0 = 0;
    std::vector<PassPlan> passes;
    for (int k = 0; k < count; ++k) {
        const int g = digits[k];
        const long long r = runs[k];
        if (g < 1 || m0 + g > P->n) return set_error(GTT_ERR_INVALID_ARG, "pass digits out of range");
        long long L = 1, M = 1;
        for (int i = 0; i < m0; ++i) L *= b;
        for (int i = 0; i < g; ++i) M *= b;
        if (r < 1 || (k > 0 && L % r != 0)) return set_error(GTT_ERR_INVALID_ARG, "run must divide b^m0");
        if (M * r * es > 220 * 1024) return set_error(GTT_ERR_INVALID_ARG, "tile above 220 KiB");
        PassPlan pp;
        gtt_status_t st = build_pass(P, m0, g, r, g >= DM ? DM : 1, &pp);
        if (st != GTT_OK) return st;
        if (!tile8_attach(P, &pp) && P->use_tma) tma_attach(P, &pp, P->tma_nbuf);
        passes.push_back(pp);
        m0 += g;
    }
    if (m0 != P->n) return set_error(GTT_ERR_INVALID_ARG, "pass digits must sum to n");
    *out = passes;
    return GTT_OK;
}
} // namespace gtt

extern "C" gtt_status_t gtt_plan_set_passes(gtt_plan_t P, int count, const int *digits, const long long *runs) {
    if (!P) return set_error(GTT_ERR_INVALID_ARG, "NULL plan");
    if (P->mixed) return set_error(GTT_ERR_UNSUPPORTED, "explicit schedules are for single-base plans");
    std::vector<PassPlan> passes;
    gtt_status_t st = make_explicit_schedule(P, count, digits, runs, &passes);
    if (st != GTT_OK) return st;
    P->passes = passes;
    P->precision = GTT_PREC_FP32;  // a CUDA-core schedule
    P->explicit_g.assign(digits, digits + count);
    P->explicit_r.assign(runs, runs + count);
    return GTT_OK;
}

extern "C" gtt_status_t gtt_plan_set_pipeline(gtt_plan_t P, int use_tma, int nbuf) {
    if (!P) return set_error(GTT_ERR_INVALID_ARG, "NULL plan");
    if (nbuf < 1 || nbuf > kTmaMaxBuf) return set_error(GTT_ERR_INVALID_ARG, "nbuf must be in [1, 4]");
    const bool old_use = P->use_tma;
    const int old_nbuf = P->tma_nbuf;
    P->use_tma = use_tma != 0;
    P->tma_nbuf = nbuf;
    P->bwd_ready = false;  // the backward's recompute passes follow the pipeline choice
    if (P->precision == GTT_PREC_BF16X3 || P->precision == GTT_PREC_BF16X2 || P->precision == GTT_PREC_TF32X3)
        return GTT_OK;  // tensor-core passes stage their own tiles
    if (P->mixed) return GTT_OK;                          // mixed plans run the CUDA-core kernel
    std::vector<PassPlan> passes;
    gtt_status_t st = P->explicit_g.empty()
                          ? make_schedule(P, P->sched_tile_bytes, P->sched_run_bytes, &passes)
                          : make_explicit_schedule(P, (int)P->explicit_g.size(), P->explicit_g.data(),
                                                   P->explicit_r.data(), &passes);
    if (st != GTT_OK) {
        P->use_tma = old_use;
        P->tma_nbuf = old_nbuf;
        return st;
    }
    P->passes = passes;
    return GTT_OK;
}

extern "C" gtt_status_t gtt_plan_set_chunking(gtt_plan_t P, long long elems) {
    if (!P) return set_error(GTT_ERR_INVALID_ARG, "NULL plan");
    if (elems < -1) return set_error(GTT_ERR_INVALID_ARG, "elems must be >= -1");
    P->chunk_elems = elems;
    return GTT_OK;
}

extern "C" gtt_status_t gtt_plan_check(gtt_plan_t P) {
    if (!P) return set_error(GTT_ERR_INVALID_ARG, "NULL plan");
    int flag = 0;
    cudaError_t e = cudaMemcpy(&flag, P->dev_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "reading the error flag");
    if (flag) {
        cudaMemset(P->dev_err, 0, sizeof(int));
        if (flag & 2) return set_error(GTT_ERR_INTERNAL, "an index check of the debug build failed in a kernel of this plan");
        return set_error(GTT_ERR_TIMEOUT, "a bounded device-side wait expired in a kernel of this plan");
    }
    return GTT_OK;
}

extern "C" gtt_status_t gtt_plan_set_precision(gtt_plan_t P, int precision) {
    if (!P) return set_error(GTT_ERR_INVALID_ARG, "NULL plan");
    if (precision == GTT_PREC_FP32) return use_cuda_core(P);
    if (precision == GTT_PREC_BF16X3) return use_tensor_cores(P, 3);
    if (precision == GTT_PREC_BF16X2) return use_tensor_cores(P, 2);
    if (precision == GTT_PREC_TF32X3) return P->b == 16 ? use_tensor_cores(P, 0) : use_complex_tensor_cores(P);
    if (precision == GTT_PREC_AUTO) {
        if (tc_eligible(P) && use_tensor_cores(P) == GTT_OK) return GTT_OK;
        return use_cuda_core(P);
    }
    return set_error(GTT_ERR_INVALID_ARG, "unknown precision");
}

extern "C" gtt_status_t gtt_plan_set_schedule(gtt_plan_t P, long long max_tile_bytes,
                                             long long min_run_bytes) {
    if (!P) return set_error(GTT_ERR_INVALID_ARG, "NULL plan");
    if (P->mixed) return set_error(GTT_ERR_UNSUPPORTED, "schedules are for single-base plans");
    if (max_tile_bytes < 16 || max_tile_bytes > 220 * 1024 || min_run_bytes < 0 ||
        min_run_bytes > max_tile_bytes)
        return set_error(GTT_ERR_INVALID_ARG, "schedule limits out of range");
    std::vector<PassPlan> passes;
    gtt_status_t st = make_schedule(P, max_tile_bytes, min_run_bytes, &passes);
    if (st != GTT_OK) return st;
    P->passes = passes;
    P->precision = GTT_PREC_FP32;  // a CUDA-core schedule
    P->explicit_g.clear();
    P->explicit_r.clear();
    P->sched_tile_bytes = max_tile_bytes;
    P->sched_run_bytes = min_run_bytes;
    return GTT_OK;
}

namespace gtt {
static cudaError_t pool_event(gtt_plan_s *P, cudaEvent_t *ev) {
    if (!P->event_pool.empty()) {
        *ev = P->event_pool.back();
        P->event_pool.pop_back();
        return cudaSuccess;
    }
    return cudaEventCreate(ev);
}

gtt_status_t launch_timed(gtt_plan_s *P, const void *kern, dim3 grid, dim3 block, void **args,
                          size_t smem, cudaStream_t stream, const std::string &name) {
    TimingRecord rec;
    if (P->timing) {
        cudaError_t e = pool_event(P, &rec.start);
        if (e == cudaSuccess) e = pool_event(P, &rec.stop);
        if (e == cudaSuccess) e = cudaEventRecord(rec.start, stream);
        if (e != cudaSuccess) return cuda_error(e, "timing event");
    }
    nvtxRangePushA(name.c_str());  // a named range per launch (no cost unless a profiler listens)
    cudaError_t e = cudaLaunchKernel(kern, grid, block, args, smem, stream);
    nvtxRangePop();
    if (e != cudaSuccess) return cuda_error(e, "kernel launch");
    if (P->timing) {
        e = cudaEventRecord(rec.stop, stream);
        if (e != cudaSuccess) return cuda_error(e, "timing event");
        rec.name = name;
        P->pending.push_back(rec);
    }
    return GTT_OK;
}

// L2-resident chunking for the current schedule.  Passes 0 .. prefix-1 only
// touch digits below s (the largest m0 + g among them), so each of their tiles
// lies in one block of b^s consecutive elements and a block's tiles are
// consecutive in every such pass.  Those passes then run chunk by chunk (a
// chunk = `per_chunk` blocks, at most the chunk size in elements), so that
// each pass after the first reads its input from L2; the remaining passes run
// over the whole data afterwards.  prefix = 0 means no chunking.
struct ChunkPlan {
    size_t prefix = 0;
    long long units = 1, per_chunk = 1;
};

static ChunkPlan chunk_plan(const gtt_plan_s *P) {
    ChunkPlan c;
    long long C = P->chunk_elems;
    if (C == -1) C = P->total * P->es > (96ll << 20) ? (48ll << 20) / P->es : 0;  // 48 MiB chunks
    if (C <= 0 || P->mixed || P->precision == GTT_PREC_TF32X3) return c;
    int top = 0;
    long long block = 1;
    size_t prefix = 0;
    for (size_t i = 0; i < P->passes.size(); ++i) {
        top = std::max(top, P->passes[i].m0 + P->passes[i].g);
        const long long blk = ipow_ll(P->b, top);
        if (blk > C) break;
        // a first-pass tile of several blocks must not straddle a chunk block
        if (P->passes[i].m0 == 0 && blk % P->passes[i].params.tile_elems != 0) break;
        prefix = i + 1;
        block = blk;
    }
    const long long units = P->total / block, per_chunk = std::max(1ll, C / block);
    if (prefix < 2 || per_chunk >= units) return c;  // nothing stays in L2 between passes
    c.prefix = prefix;
    c.units = units;
    c.per_chunk = per_chunk;
    return c;
}

static gtt_status_t run_pass(gtt_plan_s *P, PassPlan &pp, const std::vector<unsigned char> &Wb, const void *in,
                             void *outp, cudaStream_t stream, long long tb, long long te) {
    if (pp.tc.on) return tc_run(P, pp, &Wb == &P->Wa, in, outp, stream, tb, te);
    if (pp.tcx.on) return tcx_run(P, pp, &Wb == &P->Wa, in, outp, stream);
    if (pp.tma.on) return tma_run(P, pp, Wb, in, outp, stream, tb, te);
    if (pp.mix.on) {  // a mixed plan's pass: its stages' factors (or their adjoints) in the parameters
        // (patched in place: the launch copies the parameters, and a plan is
        // used from one host thread at a time)
        std::vector<unsigned char> &prm = &Wb == &P->Wa ? pp.mix.args_a : pp.mix.args_f;
        MixedParams *m = reinterpret_cast<MixedParams *>(prm.data());
        m->p.tile_begin = tb;
        m->p.tiles = te;
        m->p.err = P->dev_err;
        const int grid = (int)std::min<long long>(pp.grid, te - tb);
        void *args[3] = {(void *)&in, (void *)&outp, (void *)prm.data()};
        return launch_timed(P, pp.kern, dim3(grid), dim3(pp.block), args, pp.smem, stream, pp.name);
    }
    PassParams prm = pp.params;
    prm.tile_begin = tb;
    prm.tiles = te;
    prm.err = P->dev_err;
    const int grid = (int)std::min<long long>(pp.grid, te - tb);
    void *args[4] = {(void *)&in, (void *)&outp, (void *)&prm, (void *)Wb.data()};
    return launch_timed(P, pp.kern, dim3(grid), dim3(pp.block), args, pp.smem, stream, pp.name);
}

gtt_status_t run_pass_range(gtt_plan_s *P, size_t i, const std::vector<unsigned char> &Wb, const void *in, void *out,
                            cudaStream_t stream, long long tile_begin, long long tile_end) {
    return run_pass(P, P->passes[i], Wb, in, out, stream, tile_begin, tile_end);
}

gtt_status_t run_passes_from(gtt_plan_s *P, const std::vector<unsigned char> &Wb, void *y, cudaStream_t stream,
                             size_t first) {
    for (size_t i = first; i < P->passes.size(); ++i) {
        gtt_status_t st = run_pass(P, P->passes[i], Wb, y, y, stream, 0, P->passes[i].params.tiles);
        if (st != GTT_OK) return st;
    }
    return GTT_OK;
}

// Launch every pass of the schedule with the given W bytes.
gtt_status_t run_passes(gtt_plan_s *P, const std::vector<unsigned char> &Wb, const void *x, void *y,
                        cudaStream_t stream) {
    const ChunkPlan c = chunk_plan(P);
    for (long long u0 = 0; c.prefix > 0 && u0 < c.units; u0 += c.per_chunk) {
        const long long u1 = std::min(c.units, u0 + c.per_chunk);
        for (size_t i = 0; i < c.prefix; ++i) {
            PassPlan &pp = P->passes[i];
            const long long per_unit = pp.params.tiles / c.units;
            gtt_status_t st = run_pass(P, pp, Wb, i == 0 ? x : (const void *)y, y, stream, u0 * per_unit, u1 * per_unit);
            if (st != GTT_OK) return st;
        }
    }
    for (size_t i = c.prefix; i < P->passes.size(); ++i) {
        gtt_status_t st = run_pass(P, P->passes[i], Wb, i == 0 ? x : (const void *)y, y, stream, 0,
                                   P->passes[i].params.tiles);
        if (st != GTT_OK) return st;
    }
    return GTT_OK;
}
} // namespace gtt

extern "C" gtt_status_t gtt_plan_set_timing(gtt_plan_t P, int enable) {
    if (!P) return set_error(GTT_ERR_INVALID_ARG, "NULL plan");
    P->timing = enable != 0;
    return GTT_OK;
}

extern "C" gtt_status_t gtt_plan_timing(gtt_plan_t P, char *buf, size_t len) {
    if (!P || !buf || len == 0) return set_error(GTT_ERR_INVALID_ARG, "NULL plan or buffer");
    std::vector<std::string> names;
    std::vector<long long> counts;
    std::vector<double> total;
    gtt_status_t st = GTT_OK;
    for (TimingRecord &r : P->pending) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(r.stop);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.start, r.stop);
        if (e != cudaSuccess && st == GTT_OK) st = cuda_error(e, "timing readback");
        size_t k = 0;
        while (k < names.size() && names[k] != r.name) ++k;
        if (k == names.size()) {
            names.push_back(r.name);
            counts.push_back(0);
            total.push_back(0.0);
        }
        counts[k] += 1;
        total[k] += ms;
        P->event_pool.push_back(r.start);
        P->event_pool.push_back(r.stop);
    }
    P->pending.clear();
    std::string s = "{\"kernels\": [";
    for (size_t k = 0; k < names.size(); ++k) {
        char tmp[256];
        snprintf(tmp, sizeof tmp, "%s{\"name\": \"%s\", \"launches\": %lld, \"total_ms\": %.6f}",
                 k ? ", " : "", names[k].c_str(), counts[k], total[k]);
        s += tmp;
    }
    s += "]}";
    snprintf(buf, len, "%s", s.c_str());
    return st;
}

static gtt_status_t transform(gtt_plan_t P, const void *x, void *y, gtt_stream_t stream, bool adjoint) {
    if (!P) return set_error(GTT_ERR_INVALID_ARG, "NULL plan");
    if (!x || !y) return set_error(GTT_ERR_INVALID_ARG, "NULL data pointer");
    if (!aligned16(x) || !aligned16(y)) return set_error(GTT_ERR_INVALID_ARG, "data pointers must be 16-byte aligned");
    gtt_status_t st = check_device(P);
    if (st != GTT_OK) return st;
    return run_passes(P, adjoint ? P->Wa : P->Wf, x, y, (cudaStream_t)stream);
}

extern "C" gtt_status_t gtt_forward(gtt_plan_t P, const void *x, void *y, gtt_stream_t stream) {
    return transform(P, x, y, stream, false);
}

extern "C" gtt_status_t gtt_inverse(gtt_plan_t P, const void *y, void *x, gtt_stream_t stream) {
    return transform(P, y, x, stream, true);
}

namespace gtt {
// Index of the forward pass after which exactly the digits below the
// backward's split digit are applied, or -1 (two-pass backward schedules only).
int saving_boundary(gtt_plan_s *P) {
    if (P->mixed || P->dtype == GTT_I32) return -1;
    if (!P->bwd_ready && make_bwd_schedule(P, kBwdSmemBudget) != GTT_OK) return -1;
    if (P->bwd.size() != 2) return -1;
    const int split = P->bwd[1].geo.m0;
    int done = 0;
    for (size_t i = 0; i < P->passes.size(); ++i) {
        if (P->passes[i].tcx.on) return -1;  // cluster passes cover digits by their own rule
        done += P->passes[i].g;
        if (done == split) return (int)i;
        if (done > split) return -1;
    }
    return -1;
}
} // namespace gtt

extern "C" gtt_status_t gtt_forward_saving(gtt_plan_t P, const void *x, void *y, void *ckpt, gtt_stream_t stream) {
    if (!P) return set_error(GTT_ERR_INVALID_ARG, "NULL plan");
    if (!x || !y || !ckpt) return set_error(GTT_ERR_INVALID_ARG, "NULL data pointer");
    if (!aligned16(x) || !aligned16(y) || !aligned16(ckpt))
        return set_error(GTT_ERR_INVALID_ARG, "data pointers must be 16-byte aligned");
    if (ckpt == x || ckpt == y) return set_error(GTT_ERR_INVALID_ARG, "ckpt must not alias x or y");
    gtt_status_t st = check_device(P);
    if (st != GTT_OK) return st;
    const int k = saving_boundary(P);
    if (k < 0)
        return set_error(GTT_ERR_UNSUPPORTED,
                         "no forward pass boundary at the backward's split digit (use gtt_forward + gtt_backward)");
    cudaStream_t s = (cudaStream_t)stream;
    for (size_t i = 0; i < P->passes.size(); ++i) {
        PassPlan &pp = P->passes[i];
        const void *in = i == 0 ? x : (i <= (size_t)k ? (const void *)ckpt : (i == (size_t)k + 1 ? ckpt : y));
        void *out = i <= (size_t)k ? ckpt : y;
        st = run_pass(P, pp, P->Wf, in, out, s, 0, pp.params.tiles);
        if (st != GTT_OK) return st;
    }
    return GTT_OK;
}

static gtt_status_t transform_host(gtt_plan_t P, const void *xh, void *yh, gtt_stream_t stream,
                                   bool adjoint) {
    if (!P) return set_error(GTT_ERR_INVALID_ARG, "NULL plan");
    if (!xh || !yh) return set_error(GTT_ERR_INVALID_ARG, "NULL host pointer");
    gtt_status_t st = check_device(P);
    if (st != GTT_OK) return st;
    const size_t bytes = (size_t)P->total * P->es;
    if (!P->dstage) {
        cudaError_t e = cudaMalloc(&P->dstage, bytes);
        if (e != cudaSuccess) {
            P->dstage = nullptr;
            return set_error(GTT_ERR_ALLOC, std::string("staging buffer: ") + cudaGetErrorString(e));
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(P->dstage, xh, bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_error(e, "host to device copy");
    st = run_passes(P, adjoint ? P->Wa : P->Wf, P->dstage, P->dstage, s);
    if (st != GTT_OK) return st;
    e = cudaMemcpyAsync(yh, P->dstage, bytes, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_error(e, "device to host copy");
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "stream synchronize");
    return GTT_OK;
}

extern "C" gtt_status_t gtt_forward_host(gtt_plan_t P, const void *x, void *y, gtt_stream_t s) {
    return transform_host(P, x, y, s, false);
}

extern "C" gtt_status_t gtt_inverse_host(gtt_plan_t P, const void *y, void *x, gtt_stream_t s) {
    return transform_host(P, y, x, s, true);
}

extern "C" gtt_status_t gtt_plan_describe(gtt_plan_t P, char *buf, size_t len) {
    if (!P || !buf || len == 0) return set_error(GTT_ERR_INVALID_ARG, "NULL plan or buffer");
    std::string s = "{\"b\": " + std::to_string(P->b) + ", \"n\": " + std::to_string(P->n) +
                    ", \"dtype\": " + std::to_string((int)P->dtype) + ", \"batch\": " +
                    std::to_string(P->batch) + ", \"precision\": \"" +
                    (P->precision == GTT_PREC_BF16X3   ? "bf16x3"
                     : P->precision == GTT_PREC_BF16X2 ? "bf16x2"
                     : P->precision == GTT_PREC_TF32X3 ? "tf32x3"
                                                       : "fp32") +
                    "\", \"launches_per_transform\": " +
                    std::to_string(P->passes.size()) + ", \"passes\": [";
    for (size_t i = 0; i < P->passes.size(); ++i) {
        const PassPlan &pp = P->passes[i];
        const bool t = pp.tma.on;
        char tmp[512];
        snprintf(tmp, sizeof tmp,
                 "%s{\"kernel\": \"%s\", \"m0\": %d, \"g\": %d, \"r\": %lld, \"D\": %d, "
                 "\"tile_bytes\": %lld, \"tiles\": %lld, \"grid\": %d, \"block\": %d, \"smem\": %zu, "
                 "\"ctas_per_sm\": %d, \"vec_mode\": %d, \"tma\": %s, \"nbuf\": %d}",
                 i ? ", " : "",
                 pp.tcx.on ? pp.tcx.name.c_str() : pp.tc.on ? pp.tc.name.c_str() : t ? pp.tma.name.c_str() : pp.name.c_str(),
                 pp.m0, pp.g, pp.r, pp.D, (long long)pp.params.tile_elems * P->es, pp.params.tiles,
                 pp.tcx.on ? pp.tcx.grid : pp.tc.on ? pp.tc.grid : t ? pp.tma.grid : pp.grid,
                 pp.tcx.on ? 512 : pp.tc.on ? pp.tc.block : t ? kTmaBlock : pp.block,
                 pp.tcx.on ? pp.tcx.smem : pp.tc.on ? pp.tc.smem : t ? pp.tma.smem : pp.smem,
                 pp.tcx.on ? 1 : pp.tc.on ? pp.tc.ctas_per_sm : t ? pp.tma.ctas_per_sm : pp.ctas_per_sm, pp.params.vec_mode,
                 t ? "true" : "false", t ? pp.tma.params.nbuf : 0);
        s += tmp;
        if (pp.mix.on) {  // the stages' radices, fastest digit first
            s.pop_back();
            s += ", \"radices\": [";
            for (int k = 0; k < pp.mix.params.nst; ++k)
                s += (k ? ", " : "") + std::to_string(pp.mix.params.rad[k]);
            s += "], \"pad_shift\": " + std::to_string(pp.mix.params.pad_shift) + "}";
        }
    }
    s += "]";
    if (P->bwd_ready) {  // the backward schedule, once a backward call has built it
        s += ", \"backward\": [";
        for (size_t i = 0; i < P->bwd.size(); ++i) {
            const BwdPass &bp = P->bwd[i];
            char tmp[384];
            snprintf(tmp, sizeof tmp,
                     "%s{\"kernel\": \"%s\", \"m0\": %d, \"g\": %d, \"r\": %lld, \"grid\": %d, \"smem\": %zu}",
                     i ? ", " : "", bp.name.c_str(), bp.geo.m0, bp.g, bp.geo.r, bp.grid, bp.smem);
            s += tmp;
        }
        s += "]";
    }
    s += "}";
    snprintf(buf, len, "%s", s.c_str());
    return GTT_OK;
}

extern "C" gtt_status_t gtt_plan_destroy(gtt_plan_t P) {
    if (!P) return GTT_OK;
    if (P->dstage) cudaFree(P->dstage);
    if (P->dev_err) cudaFree(P->dev_err);
    if (P->d_wpieces) cudaFree(P->d_wpieces);
    if (P->d_tcx) cudaFree(P->d_tcx);
    if (P->ws_grad) cudaFree(P->ws_grad);
    if (P->ws_ck) cudaFree(P->ws_ck);
    if (P->ws_dw) cudaFree(P->ws_dw);
    if (P->ws_topk) cudaFree(P->ws_topk);
    for (TimingRecord &r : P->pending) {
        cudaEventDestroy(r.start);
        cudaEventDestroy(r.stop);
    }
    for (cudaEvent_t ev : P->event_pool) cudaEventDestroy(ev);
    delete P;
    return GTT_OK;
}

extern "C" const char *gtt_last_error(void) { return g_last_error.c_str(); }
