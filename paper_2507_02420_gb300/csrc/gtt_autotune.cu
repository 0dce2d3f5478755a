// Autotuner: pick the fusion schedule (how the n modes are grouped into
// passes, the run length of each strided pass, and the TMA pipeline depth)
// by timing candidates on the device, and remember the winner per
// (GPU, b, n, dtype, batch) in a process-wide cache that can be saved to and
// loaded from a JSON file.  gtt_plan_create consults the cache.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "gtt_plan.h"

namespace gtt {

struct TuneEntry {
    std::vector<int> g;
    std::vector<long long> r;
    int tma = 1, nbuf = 2;
    double us = 0.0;
};

static std::mutex g_cache_mu;
static std::map<std::string, TuneEntry> g_cache;
static bool g_env_loaded = false;

std::string tune_key(const gtt_plan_s *P) {
    cudaDeviceProp prop;
    std::string name = "unknown";
    if (cudaGetDeviceProperties(&prop, P->device) == cudaSuccess) name = prop.name;
    for (char &c : name)
        if (c == '"' || c == '|') c = '_';
    return name + "|b" + std::to_string(P->b) + "|n" + std::to_string(P->n) + "|t" + std::to_string((int)P->dtype) +
           "|batch" + std::to_string(P->batch);
}

// --- minimal reader/writer for the cache file format written below
static bool parse_int_list(const std::string &s, size_t pos, std::vector<long long> *out) {
    size_t a = s.find('[', pos), z = s.find(']', pos);
    if (a == std::string::npos || z == std::string::npos || z < a) return false;
    out->clear();
    std::stringstream ss(s.substr(a + 1, z - a - 1));
    std::string tok;
    while (std::getline(ss, tok, ','))
        if (tok.find_first_of("0123456789") != std::string::npos) out->push_back(std::atoll(tok.c_str()));
    return true;
}

static gtt_status_t load_cache_file(const char *path) {
    std::ifstream f(path);
    if (!f) return set_error(GTT_ERR_INVALID_ARG, std::string("cannot read ") + path);
    std::string line;
    std::map<std::string, TuneEntry> tmp;
    while (std::getline(f, line)) {  // one entry per line
        size_t k = line.find("\"key\": \"");
        if (k == std::string::npos) continue;
        size_t ke = line.find('"', k + 8);
        if (ke == std::string::npos) continue;
        TuneEntry e;
        std::vector<long long> gl, rl, tl, nl;
        size_t pg = line.find("\"digits\""), pr = line.find("\"runs\"");
        if (pg == std::string::npos || pr == std::string::npos) continue;
        if (!parse_int_list(line, pg, &gl) || !parse_int_list(line, pr, &rl) || gl.size() != rl.size() || gl.empty())
            continue;
        for (long long v : gl) e.g.push_back((int)v);
        e.r = rl;
        size_t pt = line.find("\"tma\": ");
        if (pt != std::string::npos) e.tma = std::atoi(line.c_str() + pt + 7);
        size_t pn = line.find("\"nbuf\": ");
        if (pn != std::string::npos) e.nbuf = std::atoi(line.c_str() + pn + 8);
        size_t pu = line.find("\"us\": ");
        if (pu != std::string::npos) e.us = std::atof(line.c_str() + pu + 6);
        tmp[line.substr(k + 8, ke - k - 8)] = e;
    }
    std::lock_guard<std::mutex> lk(g_cache_mu);
    for (auto &kv : tmp) g_cache[kv.first] = kv.second;
    return GTT_OK;
}

static void load_env_cache_once() {
    static std::once_flag once;
    std::call_once(once, [] {
        g_env_loaded = true;
        const char *p = std::getenv("GTT_AUTOTUNE_CACHE");
        if (p && *p) load_cache_file(p);  // a missing file is not an error here
    });
}

// Apply a cached schedule to a fresh plan if one exists (true if applied).
bool tune_apply_cached(gtt_plan_s *P) {
    load_env_cache_once();
    TuneEntry e;
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        auto it = g_cache.find(tune_key(P));
        if (it == g_cache.end()) return false;
        e = it->second;
    }
    const bool old_tma = P->use_tma;
    const int old_nbuf = P->tma_nbuf;
    P->use_tma = e.tma != 0;
    P->tma_nbuf = std::max(1, std::min(kTmaMaxBuf, e.nbuf));
    std::vector<PassPlan> passes;
    if (make_explicit_schedule(P, (int)e.g.size(), e.g.data(), e.r.data(), &passes) != GTT_OK) {
        P->use_tma = old_tma;
        P->tma_nbuf = old_nbuf;
        return false;
    }
    P->passes = passes;
    P->explicit_g = e.g;
    P->explicit_r = e.r;
    return true;
}

// Candidate schedules: compositions of n into at most 4 passes, with a few
// run lengths per strided pass, tiles of 2 KiB .. 200 KiB (all of them, up to
// kEnumCap; autotune ranks them with model_cost before timing any).
constexpr size_t kEnumCap = 20000;
static void enumerate(const gtt_plan_s *P, int m0, std::vector<int> &g, std::vector<long long> &r,
                      std::vector<std::pair<std::vector<int>, std::vector<long long>>> *out, size_t cap) {
    const int b = P->b, n = P->n, es = P->es;
    if (out->size() >= cap) return;
    if (m0 == n) {
        out->push_back({g, r});
        return;
    }
    if (g.size() >= 4) return;
    long long L = 1;
    for (int i = 0; i < m0; ++i) L *= b;
    std::vector<long long> runs;
    if (m0 == 0) {  // blocks per contiguous tile: 1, 2, 4, 8
        for (long long k = 1; k <= 8; k *= 2)
            if (P->total % k == 0) runs.push_back(k);
    } else {
        long long rr = 1;
        bool have32 = false, have128 = false;
        while (rr <= L) {
            if (!have32 && rr * es >= 32) {
                runs.push_back(rr);
                have32 = true;
            }
            if (!have128 && rr * es >= 128) {
                if (runs.empty() || runs.back() != rr) runs.push_back(rr);
                have128 = true;
                if (rr * b <= L) runs.push_back(rr * b);
                break;
            }
            rr *= b;
        }
        if (runs.empty()) runs.push_back(L);
    }
    const int remaining = n - m0;
    for (int gg = remaining; gg >= 1; --gg) {
        long long M = 1;
        for (int i = 0; i < gg; ++i) M *= b;
        for (long long rr : runs) {
            const long long bytes = M * rr * es;
            if (bytes > 200 * 1024) continue;
            if (m0 == 0 && P->total % (M * rr) != 0) continue;
            if (bytes < 2048 && gg < remaining && M * rr < (long long)P->total) continue;
            g.push_back(gg);
            r.push_back(rr);
            enumerate(P, m0 + gg, g, r, out, cap);
            g.pop_back();
            r.pop_back();
        }
    }
}

// Model time of one schedule, used only to rank the candidates before they
// are timed: every pass moves the vector in and out of HBM once and applies g
// modes (b FMAs per element and mode, 4b for complex types); a pass costs the
// larger of the two, raised where its tiles are too big for two CTAs per SM,
// its rows are shorter than a 32-byte sector (or a 128-byte line), or its
// tiles are so small that per-tile overhead shows.
static double model_cost(const gtt_plan_s *P, const std::vector<int> &g, const std::vector<long long> &r) {
    const double total = (double)P->total, es = (double)P->es;
    const bool cplx = P->dtype == GTT_C64 || P->dtype == GTT_C128;
    const bool wide = P->dtype == GTT_F64 || P->dtype == GTT_C128;
    const double fma_rate = wide ? 0.3e12 : 25e12;  // sustained FMAs per second (rough)
    const double mem = 2.0 * total * es / 5.8e12;
    double cost = 0.0;
    int m0 = 0;
    for (size_t k = 0; k < g.size(); ++k) {
        double M = 1.0;
        for (int i = 0; i < g[k]; ++i) M *= P->b;
        const double tile = M * (double)r[k] * es;
        const double comp = total * g[k] * P->b * (cplx ? 4.0 : 1.0) / fma_rate;
        double t = std::max(mem, comp);
        if (tile > 110.0 * 1024) t *= 1.6;
        if (tile < 8192.0) t *= 1.3;
        if (m0 > 0) {
            const double row = (double)r[k] * es;
            if (row < 32.0) t *= 2.0;
            else if (row < 128.0) t *= 1.15;
        }
        cost += t;
        m0 += g[k];
    }
    return cost;
}

// Time `reps` runs of the plan's current passes after one warm-up (microseconds
// per run), or a negative value if a run failed.
static double time_passes(gtt_plan_s *P, void *x, void *y, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, int reps) {
    if (run_passes(P, P->Wf, x, y, s) != GTT_OK) return -1.0;
    cudaEventRecord(e0, s);
    for (int i = 0; i < reps; ++i)
        if (run_passes(P, P->Wf, x, y, s) != GTT_OK) return -1.0;
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms * 1e3 / reps;
}

// Two rounds: the max_candidates schedules with the lowest model cost are
// timed in every pipeline variant (no TMA, TMA with 1..3 buffers) over 3 runs;
// the best kFinalists (schedule, variant) pairs are then timed again over 10
// runs each and the fastest of those is kept.
constexpr int kFinalists = 6;
gtt_status_t autotune(gtt_plan_s *P, int max_candidates) {
    std::vector<std::pair<std::vector<int>, std::vector<long long>>> cands;
    std::vector<int> g;
    std::vector<long long> r;
    enumerate(P, 0, g, r, &cands, kEnumCap);
    if (cands.empty()) return set_error(GTT_ERR_INTERNAL, "no candidate schedule");
    std::vector<std::pair<double, size_t>> ranked;
    for (size_t i = 0; i < cands.size(); ++i) ranked.push_back({model_cost(P, cands[i].first, cands[i].second), i});
    std::stable_sort(ranked.begin(), ranked.end(),
                     [](const std::pair<double, size_t> &a, const std::pair<double, size_t> &b) { return a.first < b.first; });
    if (ranked.size() > (size_t)std::max(1, max_candidates)) ranked.resize((size_t)std::max(1, max_candidates));
    const size_t bytes = (size_t)P->total * P->es;
    void *x = nullptr, *y = nullptr;
    cudaError_t e = cudaMalloc(&x, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&y, bytes);
    if (e != cudaSuccess) {
        if (x) cudaFree(x);
        return set_error(GTT_ERR_ALLOC, "autotune scratch buffers");
    }
    cudaMemset(x, 0, bytes);
    cudaStream_t s;
    cudaEvent_t e0, e1;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const bool save_timing = P->timing;
    P->timing = false;
    const bool old_tma = P->use_tma;
    const int old_nbuf = P->tma_nbuf;
    struct Timed {
        double us;
        size_t cand;
        int variant;
    };
    std::vector<Timed> timed;
    auto prepare = [&](size_t ci, int variant) -> bool {
        P->use_tma = variant > 0;
        P->tma_nbuf = variant > 0 ? variant : 1;
        std::vector<PassPlan> passes;
        const auto &c = cands[ci];
        if (make_explicit_schedule(P, (int)c.first.size(), c.first.data(), c.second.data(), &passes) != GTT_OK)
            return false;
        bool any_tma = false;
        for (auto &pp : passes) any_tma |= pp.tma.on;
        if (variant > 0 && !any_tma) return false;
        P->passes = passes;
        return true;
    };
    for (auto &rk : ranked)
        for (int variant = 0; variant < 4; ++variant) {
            if (!prepare(rk.second, variant)) continue;
            const double us = time_passes(P, x, y, s, e0, e1, 3);
            if (us >= 0.0) timed.push_back({us, rk.second, variant});
        }
    std::sort(timed.begin(), timed.end(), [](const Timed &a, const Timed &b) { return a.us < b.us; });
    if (timed.size() > (size_t)kFinalists) timed.resize(kFinalists);
    TuneEntry best;
    best.us = 1e30;
    for (const Timed &t : timed) {
        if (!prepare(t.cand, t.variant)) continue;
        const double us = time_passes(P, x, y, s, e0, e1, 10);
        if (us >= 0.0 && us < best.us) {
            best.us = us;
            best.g = cands[t.cand].first;
            best.r = cands[t.cand].second;
            best.tma = t.variant > 0;
            best.nbuf = P->tma_nbuf;
        }
    }
    cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    cudaFree(x);
    cudaFree(y);
    P->timing = save_timing;
    if (best.g.empty()) {
        P->use_tma = old_tma;
        P->tma_nbuf = old_nbuf;
        return set_error(GTT_ERR_INTERNAL, "autotune: no candidate ran");
    }
    P->use_tma = best.tma != 0;
    P->tma_nbuf = best.nbuf;
    std::vector<PassPlan> passes;
    gtt_status_t st = make_explicit_schedule(P, (int)best.g.size(), best.g.data(), best.r.data(), &passes);
    if (st != GTT_OK) return st;
    P->passes = passes;
    P->explicit_g = best.g;
    P->explicit_r = best.r;
    std::lock_guard<std::mutex> lk(g_cache_mu);
    g_cache[tune_key(P)] = best;
    return GTT_OK;
}

} // namespace gtt

using namespace gtt;

extern "C" gtt_status_t gtt_plan_autotune(gtt_plan_t P, int max_candidates) {
    if (!P) return set_error(GTT_ERR_INVALID_ARG, "NULL plan");
    if (P->mixed) return set_error(GTT_ERR_UNSUPPORTED, "not available for mixed-radix plans");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != P->device)
        return set_error(GTT_ERR_INVALID_ARG, "current CUDA device differs from the plan's device");
    if (P->precision == GTT_PREC_BF16X3 || P->precision == GTT_PREC_BF16X2 || P->precision == GTT_PREC_TF32X3)
        return GTT_OK;  // a tensor-core path has one schedule
    return autotune(P, max_candidates > 0 ? max_candidates : 64);
}

extern "C" gtt_status_t gtt_autotune_cache_load(const char *path) {
    if (!path) return set_error(GTT_ERR_INVALID_ARG, "NULL path");
    return load_cache_file(path);
}

extern "C" gtt_status_t gtt_autotune_cache_save(const char *path) {
    if (!path) return set_error(GTT_ERR_INVALID_ARG, "NULL path");
    std::ofstream f(path);
    if (!f) return set_error(GTT_ERR_INVALID_ARG, std::string("cannot write ") + path);
    std::lock_guard<std::mutex> lk(g_cache_mu);
    f << "{\"entries\": [\n";
    size_t i = 0;
    for (auto &kv : g_cache) {
        const TuneEntry &e = kv.second;
        f << "{\"key\": \"" << kv.first << "\", \"digits\": [";
        for (size_t k = 0; k < e.g.size(); ++k) f << (k ? ", " : "") << e.g[k];
        f << "], \"runs\": [";
        for (size_t k = 0; k < e.r.size(); ++k) f << (k ? ", " : "") << e.r[k];
        char us[64];
        snprintf(us, sizeof us, "%.3f", e.us);
        f << "], \"tma\": " << e.tma << ", \"nbuf\": " << e.nbuf << ", \"us\": " << us << "}"
          << (++i < g_cache.size() ? "," : "") << "\n";
    }
    f << "]}\n";
    return GTT_OK;
}
