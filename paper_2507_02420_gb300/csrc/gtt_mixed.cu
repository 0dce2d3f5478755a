// Host side of the multi-factor mixed-radix passes (gtt_mixed.cuh): tile
// geometry, the shared-memory padding, and the launch shape.
#include <algorithm>
#include <climits>
#include <cstddef>
#include <string>

#include "gtt_plan.h"

namespace gtt {

template <typename T> static size_t wmat_size_t(int b) {
    switch (b) {
    case 2: return sizeof(WMat<T, 2>);
    case 3: return sizeof(WMat<T, 3>);
    case 4: return sizeof(WMat<T, 4>);
    case 5: return sizeof(WMat<T, 5>);
    case 6: return sizeof(WMat<T, 6>);
    case 7: return sizeof(WMat<T, 7>);
    case 8: return sizeof(WMat<T, 8>);
    case 9: return sizeof(WMat<T, 9>);
    case 10: return sizeof(WMat<T, 10>);
    case 11: return sizeof(WMat<T, 11>);
    case 12: return sizeof(WMat<T, 12>);
    case 13: return sizeof(WMat<T, 13>);
    case 14: return sizeof(WMat<T, 14>);
    case 15: return sizeof(WMat<T, 15>);
    case 16: return sizeof(WMat<T, 16>);
    default: return 0;
    }
}

// Bytes of the kernels' parameter layout WMat<T, b> for a dtype code.
size_t wmat_size(int dtype, int b) {
    switch (dtype) {
    case GTT_F64: return wmat_size_t<double>(b);
    case GTT_F32: return wmat_size_t<float>(b);
    case GTT_C64: return wmat_size_t<c64>(b);
    case GTT_C128: return wmat_size_t<c128>(b);
    case GTT_I32: return wmat_size_t<uint32_t>(b);
    default: return 0;
    }
}

template <typename T> static size_t args_layout(size_t *w_offset, size_t *slot_bytes, int *slots) {
    *w_offset = offsetof(MixedArgs<T>, w);
    *slot_bytes = sizeof(WMat<T, 16>);
    *slots = mix_slots<T>();
    return sizeof(MixedArgs<T>);
}

size_t mixed_args_bytes(int dtype, size_t *w_offset, size_t *slot_bytes, int *slots) {
    switch (dtype) {
    case GTT_F64: return args_layout<double>(w_offset, slot_bytes, slots);
    case GTT_F32: return args_layout<float>(w_offset, slot_bytes, slots);
    case GTT_C64: return args_layout<c64>(w_offset, slot_bytes, slots);
    case GTT_C128: return args_layout<c128>(w_offset, slot_bytes, slots);
    case GTT_I32: return args_layout<uint32_t>(w_offset, slot_bytes, slots);
    default: return 0;
    }
}

// Shared-memory wavefronts of one warp access in which lane l reads the es
// bytes at element slot pos[l]: a wavefront serves at most 128 bytes (lanes in
// groups of 128 / es), and within a group each bank serves one 4-byte word per
// wavefront.
static int wavefronts(const std::vector<uint64_t> &pos, int es) {
    const int words = es / 4, group = std::max(1, 32 / words);
    int total = 0;
    for (size_t g0 = 0; g0 < pos.size(); g0 += group) {
        std::vector<std::vector<uint64_t>> bank(32);
        for (size_t l = g0; l < std::min(pos.size(), g0 + group); ++l)
            for (int w = 0; w < words; ++w) {
                const uint64_t word = pos[l] * words + w;
                std::vector<uint64_t> &bk = bank[word % 32];
                if (std::find(bk.begin(), bk.end(), word) == bk.end()) bk.push_back(word);
            }
        size_t mx = 1;
        for (const auto &bk : bank) mx = std::max(mx, bk.size());
        total += (int)mx;
    }
    return total;
}

// Padding of the tile in shared memory (one slot after every 2^ps elements):
// the ps whose stage accesses by the first warp take the fewest wavefronts,
// the least padding among equals (ps = 31: none).
static int choose_pad_shift(const MixedParams &m, int es) {
    int best = 31;
    long long best_cost = LLONG_MAX;
    for (int ps : {31, 6, 5, 4, 3, 2}) {
        long long cost = 0;
        long long blow = 1;
        for (int k = 0; k < m.nst; ++k) {
            const uint32_t B = (uint32_t)m.rad[k], S = m.stride[k], nslots = m.p.tile_elems / B;
            const uint32_t lanes = std::min<uint32_t>(32, nslots);
            for (uint32_t q = 0; q < B; ++q) {
                std::vector<uint64_t> pos(lanes);
                for (uint32_t l = 0; l < lanes; ++l) {
                    const uint32_t rest = l / m.p.r, col = l % m.p.r;
                    const uint32_t high = rest / (uint32_t)blow, low = rest % (uint32_t)blow;
                    const uint64_t e = (uint64_t)high * S * B + (uint64_t)low * m.p.r + col + (uint64_t)q * S;
                    pos[l] = e + (e >> ps);
                }
                cost += wavefronts(pos, es);
            }
            blow *= B;
        }
        if (cost < best_cost) {
            best_cost = cost;
            best = ps;
        }
    }
    return best;
}

gtt_status_t build_mixed_pass(gtt_plan_s *P, const std::vector<int> &rad, const std::vector<int> &hi,
                              const std::vector<int> &cnt, long long L, long long kblk, long long r, PassPlan *out) {
    const int es = P->es, g = (int)rad.size();
    size_t w_offset = 0, slot_bytes = 0;
    int slots = 0;
    if (mixed_args_bytes((int)P->dtype, &w_offset, &slot_bytes, &slots) == 0 || g < 1 || g > slots ||
        hi.size() != rad.size() || cnt.size() != rad.size())
        return set_error(GTT_ERR_INTERNAL, "bad mixed pass");
    long long Mg = 1;
    for (int b : rad) Mg *= b;
    const long long M = Mg * kblk, tile = M * r;
    if (r < 1 || kblk < 1 || L % r != 0) return set_error(GTT_ERR_INTERNAL, "bad mixed pass geometry");
    if (P->total % tile != 0) return set_error(GTT_ERR_INTERNAL, "mixed tiles must divide the data");
    if (L / r > (1ll << 31) || tile > (1ll << 24))
        return set_error(GTT_ERR_UNSUPPORTED, "pass geometry exceeds 32-bit tile indexing");
    PassPlan pp;
    pp.g = g;
    pp.D = 1;
    pp.r = r;
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

    MixPass &mx = pp.mix;
    mx.on = true;
    mx.hi = hi;
    mx.cnt = cnt;
    MixedParams &m = mx.params;
    m.p = p;
    m.nst = g;
    long long blow = 1;
    uint32_t max_fibres = 0;
    for (int k = 0; k < g; ++k) {
        if (rad[k] < 2 || rad[k] > 16) return set_error(GTT_ERR_INTERNAL, "mixed radix out of range");
        m.rad[k] = rad[k];
        m.stride[k] = (uint32_t)(r * blow);
        m.div_blow[k].init((uint32_t)blow);
        blow *= rad[k];
        max_fibres = std::max<uint32_t>(max_fibres, (uint32_t)(tile / rad[k]));
    }
    m.pad_shift = choose_pad_shift(m, es);
    m.smem_elems = (uint32_t)(tile + (tile >> m.pad_shift));
    pp.smem = ((size_t)m.smem_elems * es + 15) / 16 * 16;
    if (pp.smem > (size_t)P->smem_optin) return set_error(GTT_ERR_UNSUPPORTED, "mixed tile exceeds shared memory");
    pp.kern = mixed_kernel((int)P->dtype);
    if (!pp.kern) return set_error(GTT_ERR_INTERNAL, "no mixed kernel for this dtype");
    cudaError_t e = allow_max_smem(pp.kern, P->smem_optin);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(pp.kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute");
    pp.block = std::max(32, (int)std::min<uint32_t>(kMixThreads, (max_fibres + 31) / 32 * 32));
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pp.kern, pp.block, pp.smem);
    if (e != cudaSuccess) return cuda_error(e, "occupancy query");
    if (per_sm < 1) return set_error(GTT_ERR_UNSUPPORTED, "mixed pass kernel cannot be resident");
    pp.ctas_per_sm = per_sm;
    pp.grid = (int)std::min<long long>((long long)per_sm * P->num_sms, p.tiles);
    static const char *tnames[] = {"f64", "f32", "c64", "c128", "u32"};
    pp.name = std::string("gtt_mixed_pass_kernel<") + tnames[(int)P->dtype] + ">(";
    for (int k = 0; k < g; ++k) pp.name += (k ? "x" : "") + std::to_string(rad[k]);
    pp.name += ")";
    *out = pp;
    return GTT_OK;
}

} // namespace gtt
