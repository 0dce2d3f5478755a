// Grouped transforms (gtt_group_*): host planning, device tables, CUDA graph.
#include <algorithm>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "gtt_grouped.cuh"
#include "gtt_plan.h"

using namespace gtt;

namespace {
// A request large enough to fill the GPU on its own runs on its shape's plan
// (the TMA / tile pass kernels, with its own W) instead of the persistent
// kernel: a chain of launches per request, the requests spread over
// kGroupSideStreams capture streams, so that chains run side by side, and the
// persistent kernel takes half its CTAs per SM to leave room for them.
// Measured on the 1000-request workload (312 direct requests): 2 MiB and 4
// streams 6.08-6.10 ms against 6.30 with the persistent kernel's full grid,
// 6.66 with 8 streams, 8.84 with 1; 1 MiB and 512 KiB thresholds 6.7-6.8 ms
// (at 8 streams); everything in the persistent kernel 7.98 ms.
constexpr long long kGroupDirectBytes = 2ll << 20;
constexpr int kGroupSideStreams = 4;
struct DirectReq {
    gtt_plan_s *P;                  // the shape's plan (owned by the group)
    std::vector<unsigned char> W;   // this request's W (or W^H) in the kernels' parameter layout
    const void *x;
    void *y;
};
} // namespace

struct gtt_group_s {
    int device = 0, count = 0;
    GroupReq *d_reqs = nullptr;
    GroupSeg *d_segs = nullptr;
    unsigned int *d_item_seg = nullptr;
    unsigned char *d_wblob = nullptr;
    unsigned long long *d_counters = nullptr;  // [0] work counter, then done[nsegs] as uint32
    int *d_err = nullptr;
    size_t counter_bytes = 0;
    GroupArgs args;
    int grid = 0;
    size_t smem = 0;
    long long total_elems = 0;
    int distinct_shapes = 0, max_passes = 0;
    cudaStream_t capture_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<DirectReq> direct;            // requests run as pass chains on their shapes' plans
    std::vector<gtt_plan_s *> direct_plans;   // owned
    cudaStream_t side[kGroupSideStreams] = {};
    cudaEvent_t fork = nullptr, join[kGroupSideStreams] = {};
    long long direct_launches = 0;
};

namespace {

constexpr int kGroupLag = 16;  // pass p of request q follows pass p-1 of request q + lag

gtt_status_t fail(gtt_group_s *G, gtt_status_t st) {
    if (G) {
        if (G->d_reqs) cudaFree(G->d_reqs);
        if (G->d_segs) cudaFree(G->d_segs);
        if (G->d_item_seg) cudaFree(G->d_item_seg);
        if (G->d_wblob) cudaFree(G->d_wblob);
        if (G->d_counters) cudaFree(G->d_counters);
        if (G->d_err) cudaFree(G->d_err);
        if (G->capture_stream) cudaStreamDestroy(G->capture_stream);
        for (gtt_plan_s *P : G->direct_plans) gtt_plan_destroy(P);
        for (int i = 0; i < kGroupSideStreams; ++i) {
            if (G->side[i]) cudaStreamDestroy(G->side[i]);
            if (G->join[i]) cudaEventDestroy(G->join[i]);
        }
        if (G->fork) cudaEventDestroy(G->fork);
        delete G;
    }
    return st;
}

} // namespace

extern "C" gtt_status_t gtt_group_create(gtt_group_t *out, int count, const gtt_request_t *reqs) {
    if (!out || !reqs || count < 1) return set_error(GTT_ERR_INVALID_ARG, "NULL output, requests, or count < 1");
    *out = nullptr;
    gtt_group_s *G = new (std::nothrow) gtt_group_s();
    if (!G) return set_error(GTT_ERR_ALLOC, "host allocation failed");
    cudaError_t e = cudaGetDevice(&G->device);
    if (e != cudaSuccess) return fail(G, cuda_error(e, "cudaGetDevice"));
    G->count = count;

    // one scratch plan per distinct (b, n, dtype) supplies the schedule
    std::map<std::tuple<int, int, int>, gtt_plan_s *> shapes;
    std::vector<GroupReq> hreqs;  // the persistent kernel's requests
    std::vector<const gtt_plan_s *> direct_shape;
    std::vector<unsigned char> wblob;
    size_t max_w = 16, max_tile_smem = 0;
    gtt_status_t st = GTT_OK;
    for (int q = 0; q < count && st == GTT_OK; ++q) {
        const gtt_request_t &R = reqs[q];
        if (R.b < 2 || R.b > 16 || !(R.b <= 8 || R.b == 16) || R.n < 1)
            st = set_error(GTT_ERR_UNSUPPORTED, "group requests need b in 2..8 or 16 and n >= 1");
        else if (R.dtype != GTT_F32 && R.dtype != GTT_C64)
            st = set_error(GTT_ERR_UNSUPPORTED, "group requests support FP32 and complex64");
        else if (!R.W || !R.x || !R.y || ((uintptr_t)R.x & 15) || ((uintptr_t)R.y & 15))
            st = set_error(GTT_ERR_INVALID_ARG, "request pointers must be non-NULL and 16-byte aligned");
        if (st != GTT_OK) break;
        auto key = std::make_tuple(R.b, R.n, (int)R.dtype);
        gtt_plan_s *P = nullptr;
        auto it = shapes.find(key);
        if (it == shapes.end()) {
            gtt_plan_t ph = nullptr;
            st = gtt_plan_create(&ph, R.b, R.n, R.W, R.dtype, 1);
            if (st == GTT_OK) st = gtt_plan_set_precision(ph, GTT_PREC_FP32);  // the grouped kernel's arithmetic
            if (st != GTT_OK) {
                if (ph) gtt_plan_destroy(ph);
                break;
            }
            P = ph;
            if (P->passes.size() > (size_t)kGroupMaxPass) {
                st = set_error(GTT_ERR_UNSUPPORTED, "schedule has too many passes for a group");
                gtt_plan_destroy(ph);
                break;
            }
            shapes[key] = P;
        } else {
            P = it->second;
        }
        // this request's W in the kernels' parameter layout (forward, or W^H for
        // an inverse); the scratch plan supplies the schedule only -- the
        // grouped kernel stages its tiles itself
        gtt_plan_set_w(P, R.W);
        const std::vector<unsigned char> &Wb = R.inverse ? P->Wa : P->Wf;
        if (P->N * P->es >= kGroupDirectBytes) {
            G->direct.push_back(DirectReq{P, Wb, R.x, R.y});
            if (std::find(direct_shape.begin(), direct_shape.end(), P) == direct_shape.end()) direct_shape.push_back(P);
            G->direct_launches += (long long)P->passes.size();
            G->total_elems += P->N;
            continue;
        }
        const size_t off = (wblob.size() + 15) / 16 * 16;
        wblob.resize(off + Wb.size());
        memcpy(wblob.data() + off, Wb.data(), Wb.size());
        max_w = std::max(max_w, (Wb.size() + 15) / 16 * 16);
        hreqs.emplace_back();
        GroupReq &gr = hreqs.back();
        memset(&gr, 0, sizeof(gr));
        gr.x = R.x;
        gr.y = R.y;
        gr.b = R.b;
        gr.dtype = (int)R.dtype;
        gr.npass = (int)P->passes.size();
        gr.w_off = (int)off;
        gr.w_bytes = (int)((Wb.size() + 15) / 16 * 16);
        for (int k = 0; k < gr.npass; ++k) {
            gr.pass[k].p = P->passes[k].params;
            gr.pass[k].D = P->passes[k].D;
            const long long tile = P->passes[k].params.tile_elems;
            long long RB = 1;
            for (int i = 0; i < gr.pass[k].D; ++i) RB *= R.b;
            max_tile_smem = std::max(max_tile_smem, (size_t)(tile + tile / RB + 1) * P->es);
        }
        G->max_passes = std::max(G->max_passes, gr.npass);
        G->total_elems += P->N;
    }
    G->distinct_shapes = (int)shapes.size();
    for (auto &kv : shapes) {
        if (std::find(direct_shape.begin(), direct_shape.end(), kv.second) != direct_shape.end())
            G->direct_plans.push_back(kv.second);  // kept: the direct requests run on it
        else
            gtt_plan_destroy(kv.second);
    }
    if (st != GTT_OK) return fail(G, st);
    wblob.resize(wblob.size() + max_w, 0);  // every W read of max_w bytes stays inside the blob

    // work list: pass p of request q after pass p-1 of request q + lag
    std::vector<GroupSeg> segs;
    const int pcount = (int)hreqs.size();
    std::vector<std::vector<int>> seg_of(pcount, std::vector<int>(kGroupMaxPass, -1));
    long long items = 0;
    for (int t = 0; t < pcount + (G->max_passes - 1) * kGroupLag; ++t)
        for (int p = 0; p < G->max_passes; ++p) {
            const int q = t - p * kGroupLag;
            if (q < 0 || q >= pcount || p >= hreqs[q].npass) continue;
            GroupSeg sg;
            memset(&sg, 0, sizeof(sg));
            sg.req = q;
            sg.pass = p;
            sg.dep = p > 0 ? seg_of[q][p - 1] : -1;
            sg.dep_tiles = p > 0 ? (unsigned int)hreqs[q].pass[p - 1].p.tiles : 0u;
            sg.first_item = items;
            sg.tiles = hreqs[q].pass[p].p.tiles;
            items += sg.tiles;
            seg_of[q][p] = (int)segs.size();
            segs.push_back(sg);
        }

    if (items >= (1ll << 31)) return fail(G, set_error(GTT_ERR_UNSUPPORTED, "too many work items in a group"));
    std::vector<unsigned int> item_seg((size_t)items);
    for (size_t k = 0; k < segs.size(); ++k)
        for (long long i = 0; i < segs[k].tiles; ++i) item_seg[(size_t)(segs[k].first_item + i)] = (unsigned int)k;

    // device tables
    G->counter_bytes = sizeof(unsigned long long) + segs.size() * sizeof(unsigned int);
    // (at least one entry each: a group may have no requests for the persistent kernel)
    e = cudaMalloc(&G->d_reqs, std::max<size_t>(1, hreqs.size()) * sizeof(GroupReq));
    if (e == cudaSuccess) e = cudaMalloc(&G->d_segs, std::max<size_t>(1, segs.size()) * sizeof(GroupSeg));
    if (e == cudaSuccess) e = cudaMalloc(&G->d_item_seg, std::max<size_t>(1, item_seg.size()) * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc(&G->d_wblob, wblob.size());
    if (e == cudaSuccess) e = cudaMalloc(&G->d_counters, G->counter_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&G->d_err, sizeof(int));
    if (e != cudaSuccess) return fail(G, set_error(GTT_ERR_ALLOC, "group device tables"));
    for (GroupReq &gr : hreqs)
        for (int k = 0; k < gr.npass; ++k) gr.pass[k].p.err = G->d_err;  // status word of the debug build's checks
    e = cudaMemcpy(G->d_reqs, hreqs.data(), hreqs.size() * sizeof(GroupReq), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(G->d_segs, segs.data(), segs.size() * sizeof(GroupSeg), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(G->d_item_seg, item_seg.data(), item_seg.size() * sizeof(unsigned int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(G->d_wblob, wblob.data(), wblob.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(G->d_err, 0, sizeof(int));
    if (e != cudaSuccess) return fail(G, cuda_error(e, "group table upload"));

    GroupArgs &a = G->args;
    a.reqs = G->d_reqs;
    a.segs = G->d_segs;
    a.item_seg = G->d_item_seg;
    a.nsegs = (int)segs.size();
    a.total_items = items;
    a.wblob = G->d_wblob;
    a.work_counter = G->d_counters;
    a.done = reinterpret_cast<unsigned int *>(G->d_counters + 1);
    a.err = G->d_err;
    a.w_smem_bytes = (int)max_w;
    G->smem = max_w + (max_tile_smem + 15) / 16 * 16;
    int optin = 0, sms = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, G->device);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, G->device);
    if (G->smem > (size_t)optin) return fail(G, set_error(GTT_ERR_UNSUPPORTED, "group tiles exceed shared memory"));
    const void *k = (const void *)&gtt_grouped_kernel;
    if (allow_max_smem(k, optin) != cudaSuccess ||
        cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess)
        return fail(G, set_error(GTT_ERR_CUDA, "group kernel attribute"));
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kGroupThreads, G->smem);
    if (e != cudaSuccess || per_sm < 1) return fail(G, set_error(GTT_ERR_UNSUPPORTED, "group kernel cannot be resident"));
    G->grid = (G->direct.empty() || per_sm < 2 ? per_sm : per_sm / 2) * sms;
    e = cudaStreamCreateWithFlags(&G->capture_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail(G, cuda_error(e, "capture stream"));
    if (!G->direct.empty()) {
        e = cudaEventCreateWithFlags(&G->fork, cudaEventDisableTiming);
        for (int i = 0; i < kGroupSideStreams && e == cudaSuccess; ++i) {
            e = cudaStreamCreateWithFlags(&G->side[i], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&G->join[i], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return fail(G, cuda_error(e, "side streams"));
        // largest requests first, dealt round-robin over the side streams
        std::stable_sort(G->direct.begin(), G->direct.end(),
                         [](const DirectReq &a, const DirectReq &b) { return a.P->N > b.P->N; });
    }
    *out = G;
    return GTT_OK;
}

static gtt_status_t group_capture(gtt_group_s *G) {
    cudaStream_t s = G->capture_stream;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_error(e, "begin capture");
    gtt_status_t st = GTT_OK;
    const int sides = G->direct.empty() ? 0 : kGroupSideStreams;
    // the side streams fork at the start, so the pass chains of the direct
    // requests run beside the persistent kernel
    if (sides) {
        cudaEventRecord(G->fork, s);
        for (int i = 0; i < sides; ++i) cudaStreamWaitEvent(G->side[i], G->fork, 0);
    }
    if (G->args.total_items > 0) {
        cudaMemsetAsync(G->d_counters, 0, G->counter_bytes, s);
        void *args[1] = {(void *)&G->args};
        cudaLaunchKernel((const void *)&gtt_grouped_kernel, dim3(G->grid), dim3(kGroupThreads), args, G->smem, s);
    }
    for (size_t j = 0; j < G->direct.size() && st == GTT_OK; ++j) {
        DirectReq &r = G->direct[j];
        for (size_t i = 0; i < r.P->passes.size() && st == GTT_OK; ++i)
            st = run_pass_range(r.P, i, r.W, i == 0 ? r.x : (const void *)r.y, r.y, G->side[j % sides], 0,
                                r.P->passes[i].params.tiles);
    }
    for (int i = 0; i < sides; ++i) {
        cudaEventRecord(G->join[i], G->side[i]);
        cudaStreamWaitEvent(s, G->join[i], 0);
    }
    e = cudaStreamEndCapture(s, &G->graph);
    if (st != GTT_OK) {
        if (G->graph) cudaGraphDestroy(G->graph);
        G->graph = nullptr;
        return st;
    }
    if (e != cudaSuccess) return cuda_error(e, "end capture");
    e = cudaGraphInstantiate(&G->exec, G->graph, 0);
    if (e != cudaSuccess) return cuda_error(e, "graph instantiate");
    return GTT_OK;
}

extern "C" gtt_status_t gtt_group_execute(gtt_group_t G, gtt_stream_t stream) {
    if (!G) return set_error(GTT_ERR_INVALID_ARG, "NULL group");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != G->device)
        return set_error(GTT_ERR_INVALID_ARG, "current CUDA device differs from the group's device");
    if (!G->exec) {
        gtt_status_t st = group_capture(G);
        if (st != GTT_OK) return st;
    }
    cudaError_t e = cudaGraphLaunch(G->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_error(e, "graph launch");
    return GTT_OK;
}

extern "C" gtt_status_t gtt_group_check(gtt_group_t G) {
    if (!G) return set_error(GTT_ERR_INVALID_ARG, "NULL group");
    int flag = 0;
    cudaError_t e = cudaMemcpy(&flag, G->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "reading the group error flag");
    for (gtt_plan_s *P : G->direct_plans) {  // the direct requests' pass kernels raise their plan's flag
        int f = 0;
        e = cudaMemcpy(&f, P->dev_err, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_error(e, "reading a plan error flag");
        if (f) cudaMemset(P->dev_err, 0, sizeof(int));
        flag |= f;
    }
    if (flag) {
        cudaMemset(G->d_err, 0, sizeof(int));
        if (flag & 2) return set_error(GTT_ERR_INTERNAL, "an index check of the debug build failed in the grouped kernel");
        return set_error(GTT_ERR_TIMEOUT, "a bounded wait between passes expired in the grouped kernel");
    }
    return GTT_OK;
}

extern "C" gtt_status_t gtt_group_describe(gtt_group_t G, char *buf, size_t len) {
    if (!G || !buf || len == 0) return set_error(GTT_ERR_INVALID_ARG, "NULL group or buffer");
    snprintf(buf, len,
             "{\"requests\": %d, \"elements\": %lld, \"work_items\": %lld, \"segments\": %d, \"distinct_shapes\": %d, "
             "\"max_passes\": %d, \"grid\": %d, \"block\": %d, \"smem\": %zu, \"kernel\": \"gtt_grouped_kernel\", "
             "\"direct_requests\": %zu, \"direct_launches\": %lld, \"direct_streams\": %d}",
             G->count, G->total_elems, G->args.total_items, G->args.nsegs, G->distinct_shapes, G->max_passes,
             G->grid, kGroupThreads, G->smem, G->direct.size(), G->direct_launches,
             G->direct.empty() ? 0 : kGroupSideStreams);
    return GTT_OK;
}

extern "C" gtt_status_t gtt_group_destroy(gtt_group_t G) {
    if (!G) return GTT_OK;
    if (G->exec) cudaGraphExecDestroy(G->exec);
    if (G->graph) cudaGraphDestroy(G->graph);
    return fail(G, GTT_OK);
}
