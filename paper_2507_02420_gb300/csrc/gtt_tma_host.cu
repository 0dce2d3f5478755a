// Host side of the TMA-pipelined passes: eligibility, launch geometry, tensor
// maps (encoded through the runtime's driver entry point) and launch.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "gtt_plan.h"

namespace gtt {

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

static bool is_pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }

// Host copy of the kernel's tile offset (TmaTile::off): byte offset of tile
// element (row, col) in the 128B-swizzled buffer.
static uint32_t host_swz(uint32_t s, uint32_t ccb) { return (s << 7) + ((((ccb >> 4) ^ s) & 7u) << 4) + (ccb & 15u); }
static uint32_t host_tile_off(bool contig, uint32_t es, uint32_t row, uint32_t col, uint32_t M) {
    const uint32_t R128 = 128 / es;
    return contig ? host_swz(row / R128, (row % R128) * es) : host_swz((col / R128) * M + row, (col % R128) * es);
}

bool tma_attach(gtt_plan_s *P, PassPlan *pp, int nbuf) {
    pp->tma = TmaPass();
    const int b = P->b, es = P->es;
    if (!(b == 2 || b == 4 || b == 8 || b == 16) || nbuf < 1 || nbuf > kTmaMaxBuf) return false;
    if (!encode_fn()) return false;
    const PassParams &cp = pp->params;
    const long long tile_bytes = (long long)cp.tile_elems * es;
    const bool contig = cp.L == 1;  // first pass: tile = M contiguous elements
    if (tile_bytes % 128 != 0) return false;
    TmaParams t;
    memset(&t, 0, sizeof(t));
    t.tiles = cp.tiles;
    t.tile_begin = cp.tile_begin;
    t.M = cp.M;
    t.r = cp.r;
    t.tile_elems = cp.tile_elems;
    t.lo_blocks = cp.lo_blocks;
    t.tile_bytes = (uint32_t)tile_bytes;
    t.units_per_elem = es == 16 ? 2 : 1;
    t.nbuf = nbuf;
    t.div_lo_blocks = cp.div_lo_blocks;
    t.div_r = cp.div_r;
    t.nstages = cp.nstages;
    const bool contig_tile = cp.L == 1;
    const uint32_t R128 = 128 / es;
    long long RB = 1;
    for (int i = 0; i < pp->D; ++i) RB *= b;
    for (int s = 0; s < cp.nstages; ++s) {
        const uint32_t Ba = cp.stage_divBa[s].d;
        t.stage_mask[s] = cp.stage_mask[s];
        t.stage_Ba[s] = Ba;
        t.stage_divBa[s] = cp.stage_divBa[s];
        // address form (see kAddr* in gtt_tma.cuh); M % 8 == 0 is required below
        t.stage_addr[s] = kAddrGeneral;
        t.stage_stride[s] = 0;
        if (s < kTmaXorStages && RB <= 16) {  // b and hence Ba, M, R128 are powers of two
            t.stage_addr[s] = kAddrXor;
            for (long long q = 0; q < RB; ++q)
                t.stage_fq[s][q] = host_tile_off(contig_tile, (uint32_t)es, (uint32_t)(q * Ba), 0, cp.M);
        }
        if (!contig_tile) {
            if (Ba % 8 == 0) {
                t.stage_addr[s] = kAddrStride;
                t.stage_stride[s] = Ba * 128u;
            } else if (Ba == 1 && RB % 8 == 0) {
                t.stage_addr[s] = kAddrRowXor;
            }
        } else if (Ba > 1) {
            if (Ba % (8 * R128) == 0) {
                t.stage_addr[s] = kAddrStride;
                t.stage_stride[s] = Ba * (uint32_t)es;
            } else if (Ba == R128 && RB % 8 == 0) {
                t.stage_addr[s] = kAddrRowXor;
            }
        }
    }
    if (contig) {
        if (cp.r != 1) return false;  // contiguous tiles of the first pass only
        const long long rows_total = P->total * es / 128;
        if ((P->total * es) % 128 != 0 || rows_total > (1ll << 31)) return false;
        const uint32_t tile_rows = (uint32_t)(tile_bytes / 128);
        t.rows_per_box = std::min<uint32_t>(tile_rows, 256);
        if (tile_rows % t.rows_per_box) return false;
        t.boxes_per_cb = tile_rows / t.rows_per_box;
        t.cbs = 1;
    } else {
        if (((long long)cp.r * es) % 128 != 0 || !is_pow2(cp.M)) return false;
        t.rows_per_box = std::min<uint32_t>(cp.M, 256);
        t.boxes_per_cb = cp.M / t.rows_per_box;
        t.cbs = (uint32_t)((long long)cp.r * es / 128);
        const long long H = P->total / (cp.L * (long long)cp.M);
        if (cp.L * (long long)t.units_per_elem > (1ll << 31) || H > (1ll << 31)) return false;
    }
    // every box must land on a 1024-byte boundary (the 128B swizzle repeats
    // every 8 rows): rows per box, and M for column blocks, multiples of 8
    if (t.rows_per_box % 8 != 0 || (!contig && cp.M % 8 != 0)) return false;
    const void *k = tma_kernel((int)P->dtype, b, pp->D, contig);
    if (!k) return false;
    const size_t smem = (size_t)nbuf * tile_bytes + 1024 + kTmaBarBytes;
    if (smem > (size_t)P->smem_optin) return false;
    if (allow_max_smem(k, P->smem_optin) != cudaSuccess) return false;
    if (cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess) return false;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kTmaBlock, smem) != cudaSuccess || per_sm < 1)
        return false;
    TmaPass &tp = pp->tma;
    tp.params = t;
    tp.contig = contig;
    tp.kern = k;
    tp.smem = smem;
    tp.ctas_per_sm = per_sm;
    tp.grid = (int)std::min<long long>((long long)per_sm * P->num_sms, cp.tiles);
    static const char *tnames[] = {"f64", "f32", "c64", "c128", "u32"};
    tp.name = std::string("gtt_tma_pass_kernel<") + tnames[(int)P->dtype] + "," + std::to_string(b) + "," +
              std::to_string(pp->D) + "," + (contig ? "contig" : "strided") + ">";
    tp.on = true;
    return true;
}

static gtt_status_t encode(gtt_plan_s *P, const PassPlan &pp, const void *ptr, CUtensorMap *map) {
    const TmaPass &tp = pp.tma;
    const int es = P->es;
    const CUtensorMapDataType dt = es == 4 ? CU_TENSOR_MAP_DATA_TYPE_UINT32 : CU_TENSOR_MAP_DATA_TYPE_UINT64;
    const cuuint32_t upe = tp.params.units_per_elem;
    const cuuint32_t row_units = (cuuint32_t)(128 / (es == 4 ? 4 : 8));
    CUresult r;
    if (tp.contig) {
        cuuint64_t dims[2] = {row_units, (cuuint64_t)(P->total * es / 128)};
        cuuint64_t strides[1] = {128};
        cuuint32_t box[2] = {row_units, tp.params.rows_per_box};
        cuuint32_t estr[2] = {1, 1};
        r = encode_fn()(map, dt, 2, const_cast<void *>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
        const long long L = pp.params.L, M = pp.params.M;
        cuuint64_t dims[3] = {(cuuint64_t)(L * upe), (cuuint64_t)M, (cuuint64_t)(P->total / (L * M))};
        cuuint64_t strides[2] = {(cuuint64_t)(L * es), (cuuint64_t)(L * M * es)};
        cuuint32_t box[3] = {row_units, tp.params.rows_per_box, 1};
        cuuint32_t estr[3] = {1, 1, 1};
        r = encode_fn()(map, dt, 3, const_cast<void *>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    if (r != CUDA_SUCCESS) return set_error(GTT_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return GTT_OK;
}

gtt_status_t tma_run(gtt_plan_s *P, PassPlan &pp, const std::vector<unsigned char> &Wb, const void *in, void *out,
                     cudaStream_t stream, long long tile_begin, long long tile_end) {
    TmaPass &tp = pp.tma;
    gtt_status_t st;
    if (tp.map_in_ptr != in) {
        st = encode(P, pp, in, &tp.map_in);
        if (st != GTT_OK) return st;
        tp.map_in_ptr = in;
    }
    if (tp.map_out_ptr != out) {
        st = encode(P, pp, out, &tp.map_out);
        if (st != GTT_OK) return st;
        tp.map_out_ptr = out;
    }
    TmaParams prm = tp.params;
    prm.err = P->dev_err;
    prm.tile_begin = tile_begin;
    prm.tiles = tile_end;
    const int grid = (int)std::min<long long>(tp.grid, tile_end - tile_begin);
    void *args[4] = {(void *)&tp.map_in, (void *)&tp.map_out, (void *)&prm, (void *)Wb.data()};
    return launch_timed(P, tp.kern, dim3(grid), dim3(kTmaBlock), args, tp.smem, stream, tp.name);
}

} // namespace gtt
