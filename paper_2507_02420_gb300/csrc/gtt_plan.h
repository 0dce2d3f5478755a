// Plan object and host-side helpers shared by the C-ABI translation units.
#pragma once
#include <cstring>
#include <string>
#include <vector>

#include "../../include/gtt.h"
#include "gtt_internal.h"
#include "gtt_mixed.cuh"

namespace gtt {

// Default fixed-rule schedule: tiles of at most this many bytes (several CTAs
// per SM) and runs of at least this many contiguous bytes in strided passes.
constexpr long long kDefaultTileBytes = 48 * 1024;
constexpr long long kDefaultRunBytes = 64;

// Multi-factor pass of a mixed-radix plan (gtt_mixed.cuh): one stage per
// digit, stage k applying the Kronecker product of the factors
// W_{hi_k - cnt_k + 1} .. W_{hi_k} (a single factor when cnt_k = 1).
struct MixPass {
    bool on = false;
    MixedParams params;
    std::vector<int> hi, cnt;                  // factors of each stage
    std::vector<unsigned char> args_f, args_a; // kernel parameters (MixedArgs<T>) with the factors or adjoints
    MixPass() { memset(&params, 0, sizeof(params)); }
};

// One pass of a schedule: modes [m0, m0+g) with runs of r elements, register
// windows of D digits, and its launch geometry.
// TMA-pipelined variant of a pass (gtt_tma.cuh); present when the tile
// geometry allows 128-byte TMA rows.  The tensor maps depend on the data
// pointers and are encoded at launch time (cached per pointer pair).
struct TmaPass {
    bool on = false;
    bool contig = false;
    TmaParams params;
    const void *kern = nullptr;
    int grid = 0, ctas_per_sm = 0;
    size_t smem = 0;
    std::string name;
    // tensor-map cache
    const void *map_in_ptr = nullptr, *map_out_ptr = nullptr;
    CUtensorMap map_in, map_out;  // the type carries its own 64-byte alignment
};

// b = 16 tensor-core (BF16x3) variant of a pass (gtt_tc16.cuh).
struct TcPass {
    bool on = false;
    int g = 0;
    int np = 3;  // pieces: 3 (BF16X3), 2 (BF16X2) or 0 (TF32X3)
    const void *kern = nullptr;
    int grid = 0, block = 0, ctas_per_sm = 0;
    size_t smem = 0;
    std::string name;
};

// complex64 b = 4 tensor-core (TF32X3) variant of a pass (gtt_tcx.cuh): a
// cluster of four CTAs per tile group; the contiguous pass keeps a tensor map
// of its input (cached per pointer).
struct TcxPass {
    bool on = false;
    bool contig = false;
    const void *kern = nullptr;
    int grid = 0;
    size_t smem = 0;
    long long ctiles = 0, L = 1;
    std::string name;
    const void *map_ptr = nullptr;
    CUtensorMap map;
    TcxPass() { memset(&map, 0, sizeof(map)); }
};

struct PassPlan {
    int m0 = 0, g = 0, D = 1;
    long long r = 1;
    PassParams params;
    const void *kern = nullptr;
    int grid = 0, block = 0, ctas_per_sm = 0;
    size_t smem = 0;
    std::string name;  // kernel name with its template arguments
    TmaPass tma;
    TcPass tc;
    TcxPass tcx;
    MixPass mix;                           // mixed plans: multi-factor pass (gtt_mixed.cuh)
    int factor = -1;                       // mixed plans: the factor W_k of the pass's fastest digit
    int factors = 1;                       // mixed plans: the factors W_{factor-factors+1} .. W_factor it applies
};

// One pass of the backward schedule: the tile geometry (one stage per digit),
// the matching forward pass used to recompute checkpoints, and the launch.
struct BwdPass {
    PassPlan geo, fwd;
    const void *kern = nullptr;
    int grid = 0, g = 0;
    size_t smem = 0;
    std::string name;
};
constexpr size_t kBwdSmemBudget = 100 * 1024;

// Launch timing: event pairs recorded around each launch when enabled.
struct TimingRecord {
    cudaEvent_t start, stop;
    std::string name;
};

// Raise a kernel's dynamic shared-memory limit to the device's opt-in maximum
// (one limit per kernel, so passes of different tile sizes can share it).
inline cudaError_t allow_max_smem(const void *kern, int optin) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes);
}

gtt_status_t set_error(gtt_status_t st, const std::string &msg);
gtt_status_t cuda_error(cudaError_t e, const char *what);

} // namespace gtt

struct gtt_plan_s {
    int device = 0, num_sms = 0, smem_optin = 0;
    int b = 0, n = 0, es = 0;
    gtt_dtype_t dtype = GTT_F32;
    long long batch = 0, N = 0, total = 0;
    int precision = GTT_PREC_AUTO;
    bool mixed = false;                 // G = W_0 (x) ... (x) W_{n-1} with factor sizes `radices`
    std::vector<int> radices;           // mixed plans: b_k of factor k (factor 0 most significant)
    std::vector<unsigned char> Wf, Wa;  // W and W^H in the element type, row-major
    std::vector<gtt::PassPlan> passes;  // forward/inverse schedule
    void *dstage = nullptr;             // device staging for the host-buffer calls
    std::vector<gtt::BwdPass> bwd;       // backward schedule (built on first use)
    bool bwd_ready = false;
    void *ws_grad = nullptr, *ws_ck = nullptr, *ws_dw = nullptr;  // backward workspace
    size_t ws_grad_bytes = 0, ws_ck_bytes = 0, ws_dw_bytes = 0;
    void *ws_topk = nullptr;                                        // top-k selection workspace
    size_t ws_topk_bytes = 0;
    bool use_tma = true;                 // TMA-pipelined passes where the geometry allows
    int tma_nbuf = 2;                    // shared-memory buffers per CTA in TMA passes
    long long sched_tile_bytes = 0, sched_run_bytes = 0;  // limits of the current schedule
    std::vector<int> explicit_g;         // explicit schedule (gtt_plan_set_passes), else empty
    std::vector<long long> explicit_r;
    int *dev_err = nullptr;              // device flag raised by a bounded wait that expired
    void *d_wpieces = nullptr;           // BF16x3 pieces of W and W^T (b = 16 tensor-core path)
    void *d_tcx = nullptr;               // TF32 pieces of W (x) W and its adjoint (complex b = 4 tensor-core path)
    long long chunk_elems = 0;           // elements per L2-resident chunk (0: off, -1: automatic)
    bool timing = false;
    std::vector<gtt::TimingRecord> pending;  // recorded, not yet read
    std::vector<cudaEvent_t> event_pool;
};

namespace gtt {
gtt_status_t build_pass(gtt_plan_s *P, int m0, int g, long long r, int D, PassPlan *out);
gtt_status_t build_pass_geom(gtt_plan_s *P, int b, long long L, int g, long long kblk, long long r, int D,
                             PassPlan *out);
gtt_status_t make_schedule(gtt_plan_s *P, long long max_tile_bytes, long long min_run_bytes,
                           std::vector<PassPlan> *out);
// Launch `kern` with `args`, recording timing events when the plan asks for it.
gtt_status_t launch_timed(gtt_plan_s *P, const void *kern, dim3 grid, dim3 block, void **args,
                          size_t smem, cudaStream_t stream, const std::string &name);
gtt_status_t make_bwd_schedule(gtt_plan_s *P, size_t smem_budget);
// Forward pass after which the digits below the backward's split are applied
// (gtt_forward_saving's checkpoint), or -1.
int saving_boundary(gtt_plan_s *P);
// Autotuner (gtt_autotune.cu): apply a cached schedule to a plan (true if
// one existed), or time candidates and keep the fastest.
bool tune_apply_cached(gtt_plan_s *P);
gtt_status_t autotune(gtt_plan_s *P, int max_candidates);
gtt_status_t make_explicit_schedule(gtt_plan_s *P, int count, const int *digits, const long long *runs,
                                    std::vector<PassPlan> *out);
// b = 16 tensor-core passes (gtt_tc16.cu)
gtt_status_t tc_upload_w(gtt_plan_s *P);
gtt_status_t make_tc_schedule(gtt_plan_s *P, int np, std::vector<PassPlan> *out);  // np = 3 (BF16X3), 2 (BF16X2), 0 (TF32X3)
gtt_status_t tc_run(gtt_plan_s *P, PassPlan &pp, bool adjoint, const void *in, void *out, cudaStream_t s,
                    long long tile_begin, long long tile_end);
// complex64 b = 4 tensor-core passes (gtt_tcx.cu)
bool tcx_eligible(const gtt_plan_s *P);
gtt_status_t tcx_upload_w(gtt_plan_s *P);
gtt_status_t make_tcx_schedule(gtt_plan_s *P, std::vector<PassPlan> *out);
gtt_status_t tcx_run(gtt_plan_s *P, PassPlan &pp, bool adjoint, const void *in, void *out, cudaStream_t s);
// Mixed-radix plans: a pass over consecutive digits of radices rad[0..] (fastest
// first; stage k applies the factors hi[k] - cnt[k] + 1 .. hi[k]) at stride L,
// runs of r, kblk blocks per tile.
gtt_status_t build_mixed_pass(gtt_plan_s *P, const std::vector<int> &rad, const std::vector<int> &hi,
                              const std::vector<int> &cnt, long long L, long long kblk, long long r, PassPlan *out);
// Bytes of the kernels' parameter layout WMat<T, b> for a dtype code.
size_t wmat_size(int dtype, int b);
// Attach the TMA variant to a forward pass when its geometry allows (true if attached).
bool tma_attach(gtt_plan_s *P, PassPlan *pp, int nbuf);
// FP32 b = 8 passes on 4096-element tiles: the compile-time tile kernel
// (false: the pass is not of that shape and stays as it is)
bool tile8_attach(gtt_plan_s *P, PassPlan *pp);
gtt_status_t tma_run(gtt_plan_s *P, PassPlan &pp, const std::vector<unsigned char> &Wb, const void *in,
                     void *out, cudaStream_t stream, long long tile_begin, long long tile_end);
// Zero elements [lo, hi) of every vector of y (batch x N, the plan's element
// type) with a write-only kernel.
gtt_status_t zero_range(gtt_plan_s *P, void *y, long long lo, long long hi, cudaStream_t s);
gtt_status_t run_passes(gtt_plan_s *P, const std::vector<unsigned char> &Wb, const void *x, void *y,
                        cudaStream_t stream);
// Pass i of the schedule over its tiles [tile_begin, tile_end).
gtt_status_t run_pass_range(gtt_plan_s *P, size_t i, const std::vector<unsigned char> &Wb, const void *in, void *out,
                            cudaStream_t stream, long long tile_begin, long long tile_end);
// Passes first .. end of the schedule, in place on y, over all tiles (no chunking).
gtt_status_t run_passes_from(gtt_plan_s *P, const std::vector<unsigned char> &Wb, void *y, cudaStream_t stream,
                             size_t first);
} // namespace gtt
