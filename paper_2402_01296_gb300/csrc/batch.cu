// Batched evaluation: many ciphertext-branch evaluations of different ring
// degrees and shapes replayed as one CUDA graph.
//
// The evaluations are spread over lanes (streams) by the longest-processing-
// time rule on an analytic cost (NTT butterflies and MAC products); each lane
// runs its evaluations one after another on its own slice of the workspace,
// and the lanes run concurrently, so small evaluations fill the device while
// large ones run.  The whole launch sequence is captured once and replayed with
// a single graph launch; nothing waits on the device, so there is no wait to
// bound.
#include <algorithm>
#include <numeric>

#include "device_api.h"

struct bcn_batch {
    std::vector<bcn_batch_item> items;
    std::vector<std::vector<const uint32_t *>> pts;  // copies of the per-item pointer arrays
    int lanes = 0;
    std::vector<int> lane_of;                         // item -> lane
    std::vector<std::vector<int>> lane_items;         // lane -> items in order
    std::vector<size_t> lane_off, lane_bytes;         // workspace slices
    int device = -1;
    cudaStream_t origin = nullptr;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace bcn {
namespace {

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Analytic cost of one evaluation: NTT butterflies of the square layers
// (tensor square: 5 transforms per limb; key switch: dnum + 2 per target
// prime) plus the multiply-accumulates of every layer, per ciphertext word.
double model_cost(const bcn_model *m) {
    const bcn_ctx *c = m->ctx;
    const double N = c->N, logN = c->logN;
    double cost = 0;
    for (const auto &p : m->layers) {
        const double n = p.level;
        cost += (double)p.n_out * p.K * 2 * n * N;  // MAC products
        if (p.square) {
            const double dnum = std::ceil(n / c->alpha), nb = n + c->K;
            const double ntts = 5 * n + nb * (dnum + 2);
            cost += (double)p.n_out * ntts * (N / 2) * logN * 4;  // a butterfly costs about 4 products
        }
    }
    return cost;
}

bcn_status plan(const bcn_batch_item *items, int n, int lanes, std::vector<std::vector<int>> &lane_items,
                std::vector<size_t> &lane_bytes, int *device) {
    if (!items || n < 1 || lanes < 1) return fail(BCN_E_INVAL, "bcn_batch: no items or lanes");
    lanes = std::min(lanes, n);
    int dev = -1;
    std::vector<double> cost(n);
    std::vector<size_t> ws(n);
    for (int i = 0; i < n; i++) {
        const bcn_batch_item &it = items[i];
        if (!it.model || !it.evk_eval || !it.cts || !it.out) return fail(BCN_E_INVAL, "bcn_batch: null item field");
        if (it.model->prof.on) return fail(BCN_E_INVAL, "bcn_batch: disable kernel timing on batched models");
        if (dev < 0) dev = it.model->ctx->device;
        if (it.model->ctx->device != dev || dev < 0)
            return fail(BCN_E_INVAL, "bcn_batch: all items must live on the same device");
        cost[i] = model_cost(it.model);
        bcn_status s = bcn_eval_workspace_bytes(it.model, &ws[i]);
        if (s != BCN_OK) return s;
    }
    // longest processing time first onto the least-loaded lane
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<double> load(lanes, 0.0);
    lane_items.assign(lanes, {});
    lane_bytes.assign(lanes, 0);
    for (int i : order) {
        const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[l] += cost[i];
        lane_items[l].push_back(i);
        lane_bytes[l] = std::max(lane_bytes[l], align256(ws[i]));
    }
    *device = dev;
    return BCN_OK;
}

void destroy_members(bcn_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto e : b->joins) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    for (auto s : b->streams) cudaStreamDestroy(s);
    if (b->origin) cudaStreamDestroy(b->origin);
}

}  // namespace
}  // namespace bcn

using namespace bcn;

extern "C" {

bcn_status bcn_batch_plan(const bcn_batch_item *items, int n_items, int lanes, size_t *workspace_bytes) {
    if (!workspace_bytes) return fail(BCN_E_INVAL, "bcn_batch_plan: null output");
    std::vector<std::vector<int>> li;
    std::vector<size_t> lb;
    int dev = -1;
    bcn_status s = plan(items, n_items, lanes, li, lb, &dev);
    if (s != BCN_OK) return s;
    *workspace_bytes = std::accumulate(lb.begin(), lb.end(), (size_t)0);
    return BCN_OK;
}

bcn_status bcn_batch_create(const bcn_batch_item *items, int n_items, int lanes, void *workspace, size_t ws_bytes,
                            bcn_batch **out) {
    if (!out) return fail(BCN_E_INVAL, "bcn_batch_create: null output");
    *out = nullptr;
    bcn_batch *b = new bcn_batch();
    bcn_status s = plan(items, n_items, lanes, b->lane_items, b->lane_bytes, &b->device);
    if (s != BCN_OK) {
        delete b;
        return s;
    }
    b->lanes = (int)b->lane_items.size();
    size_t need = 0;
    for (size_t l = 0; l < b->lane_bytes.size(); l++) {
        b->lane_off.push_back(need);
        need += b->lane_bytes[l];
    }
    if (ws_bytes < need || (need && !workspace)) {
        delete b;
        return fail(BCN_E_BUDGET, "bcn_batch_create: workspace smaller than bcn_batch_plan's size");
    }
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != b->device) {
        delete b;
        return fail(BCN_E_INVAL, "bcn_batch_create: the items' device must be current");
    }
    b->items.assign(items, items + n_items);
    b->pts.resize(n_items);
    for (int i = 0; i < n_items; i++) {
        int n_add = 0;
        for (const auto &p : items[i].model->layers) n_add += p.add;
        if (n_add && !items[i].pts) {
            delete b;
            return fail(BCN_E_INVAL, "bcn_batch_create: missing feature plaintexts");
        }
        b->pts[i].assign(items[i].pts, items[i].pts + n_add);
        b->items[i].pts = b->pts[i].data();
    }
    auto bail = [&](bcn_status st, const std::string &msg) {
        destroy_members(b);
        delete b;
        return fail(st, msg);
    };
    if (cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
        return bail(BCN_E_CUDA, "bcn_batch_create: stream/event creation failed");
    b->streams.resize(b->lanes, nullptr);
    b->joins.resize(b->lanes, nullptr);
    for (int l = 0; l < b->lanes; l++)
        if (cudaStreamCreateWithFlags(&b->streams[l], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->joins[l], cudaEventDisableTiming) != cudaSuccess)
            return bail(BCN_E_CUDA, "bcn_batch_create: stream/event creation failed");
    // capture: fork from the origin, one evaluation chain per lane, join back
    if (cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return bail(BCN_E_CUDA, "bcn_batch_create: cudaStreamBeginCapture failed");
    bcn_status st = BCN_OK;
    std::string err;
    if (cudaEventRecord(b->fork, b->origin) != cudaSuccess) st = BCN_E_CUDA;
    char *ws = reinterpret_cast<char *>(workspace);
    for (int l = 0; l < b->lanes && st == BCN_OK; l++) {
        if (cudaStreamWaitEvent(b->streams[l], b->fork, 0) != cudaSuccess) {
            st = BCN_E_CUDA;
            break;
        }
        for (int i : b->lane_items[l]) {
            const bcn_batch_item &it = b->items[i];
            st = bcn_eval(it.model, it.evk_eval, it.cts, it.pts, it.out, ws + b->lane_off[l], b->lane_bytes[l],
                          b->streams[l]);
            if (st != BCN_OK) {
                err = bcn_last_error();
                break;
            }
        }
        if (st == BCN_OK && (cudaEventRecord(b->joins[l], b->streams[l]) != cudaSuccess ||
                             cudaStreamWaitEvent(b->origin, b->joins[l], 0) != cudaSuccess))
            st = BCN_E_CUDA;
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(b->origin, &g);
    b->graph = g;
    if (st != BCN_OK) return bail(st, "bcn_batch_create: capture failed: " + err);
    if (ec != cudaSuccess || !g) return bail(BCN_E_CUDA, std::string("bcn_batch_create: ") + cudaGetErrorString(ec));
    if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess)
        return bail(BCN_E_CUDA, "bcn_batch_create: cudaGraphInstantiate failed");
    *out = b;
    return BCN_OK;
}

bcn_status bcn_batch_launch(bcn_batch *b, void *stream) {
    if (!b || !b->exec) return fail(BCN_E_INVAL, "bcn_batch_launch: null batch");
    const cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(BCN_E_CUDA, std::string("bcn_batch_launch: ") + cudaGetErrorString(e));
    return BCN_OK;
}

bcn_status bcn_batch_lanes(const bcn_batch *b, int *lane_of_item) {
    if (!b || !lane_of_item) return fail(BCN_E_INVAL, "bcn_batch_lanes: null argument");
    for (int l = 0; l < b->lanes; l++)
        for (int i : b->lane_items[l]) lane_of_item[i] = l;
    return BCN_OK;
}

bcn_status bcn_batch_destroy(bcn_batch *b) {
    if (!b) return BCN_OK;
    destroy_members(b);
    delete b;
    return BCN_OK;
}

bcn_status bcn_model_cost(const bcn_model *m, double *cost) {
    if (!m || !cost) return fail(BCN_E_INVAL, "bcn_model_cost: null argument");
    *cost = model_cost(m);
    return BCN_OK;
}

}  // extern "C"
