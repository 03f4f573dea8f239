// BWT_F_GRAPH: the whole batch as one CUDA graph, replayed when the block
// layout and buffers repeat (the plan keeps the last few graphs, so callers
// that alternate between buffer sets replay too).
//
// Graph = reset -> first stage (plain: first sort + naming; with
//         BWT_F_LEARNED: the learned first stage) -> set loop condition ->
//         WHILE(cond) { round on bins[0]; IF(another round due) { round on
//         bins[1] } } -> L gather.
// The body holds two rounds so the double-buffered group bins alternate
// inside one fixed graph; the second is skipped when the first finished the
// batch (about twenty launches that would find no work). The conditions
// (groups left, depth below the largest block, no device error, at most 40
// rounds) are computed on the device, so a replay never returns to the host
// between rounds. (Conditional nodes around each round's large-group section
// were measured too: evaluating them cost about what the skipped launches
// did, and more on workloads whose rounds mostly have large groups.)
#include <cstring>
#include <vector>

#include "kernels.h"
#include "plan_internal.h"

using namespace bwt;

#define CKG(call)                                             \
    do {                                                      \
        cudaError_t _e = (call);                              \
        if (_e != cudaSuccess) {                              \
            status = record_cuda(_e, #call);                  \
            goto fail;                                        \
        }                                                     \
    } while (0)

#define CKS(call)                   \
    do {                            \
        status = (call);            \
        if (status != BWT_OK) goto fail; \
    } while (0)

static std::vector<uint64_t> graph_key_of(bwt_plan* p, const uint8_t* d_in, uint8_t* d_L, int32_t* d_primary) {
    std::vector<uint64_t> k = {(uint64_t)(uintptr_t)d_in, (uint64_t)(uintptr_t)d_L, (uint64_t)(uintptr_t)d_primary,
                               (uint64_t)p->rbits, (uint64_t)p->tile, (uint64_t)p->spin_limit,
                               (uint64_t)p->withhold, (uint64_t)p->nb, (uint64_t)p->round_bits};
    k.insert(k.end(), p->h_off, p->h_off + p->nb + 1);
    return k;
}

// Launches a cached graph on the caller's stream and records its event; the
// kernel counts of the call come from the graph's own (filled in by
// graph_stats once the call has finished).
static bwt_status launch_entry(bwt_plan* p, GraphEntry& ge, cudaStream_t st, bool replay) {
    cudaError_t e = cudaGraphLaunch(ge.exec, st);
    if (e != cudaSuccess) return record_cuda(e, "cudaGraphLaunch");
    e = cudaEventRecord(ge.launched, st);
    if (e != cudaSuccess) return record_cuda(e, "cudaEventRecord");
    ge.last_use = ++p->graph_use;
    p->graph_main_kernels = ge.main_kernels;
    p->graph_round_kernels = ge.round_kernels;
    p->graph_large_kernels = ge.large_kernels;
    p->graph_main_radix = ge.main_radix;
    p->graph_large_radix = ge.large_radix;
    p->stats.graph_replayed = replay ? 1u : 0u;
    p->stats.kernel_launches = 0;
    p->stats.radix_launches = 0;
    return BWT_OK;
}

bwt_status bwt::begin_if_capture(cudaStream_t st, cudaStream_t inner, cudaGraphConditionalHandle h) {
    cudaStreamCaptureStatus cst;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(st, &cst, nullptr, &g, &deps, nullptr, &ndeps);
    if (e != cudaSuccess) return record_cuda(e, "cudaStreamGetCaptureInfo");
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if ((e = cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &cp)) != cudaSuccess) return record_cuda(e, "IF node");
    if ((e = cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
        cudaSuccess)
        return record_cuda(e, "cudaStreamUpdateCaptureDependencies");
    e = cudaStreamBeginCaptureToGraph(inner, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    return e == cudaSuccess ? BWT_OK : record_cuda(e, "cudaStreamBeginCaptureToGraph");
}

bwt_status bwt::run_graph(bwt_plan* p, const uint8_t* d_in, uint8_t* d_L, int32_t* d_primary, cudaStream_t st) {
    const bool learned = (p->desc.flags & BWT_F_LEARNED) != 0;
    if (learned) {
        if (!p->have_model) return BWT_ENOMODEL;
        bwt_status s = ensure_learned_buffers(p);  // allocations happen before any capture
        if (s != BWT_OK) return s;
    }
    std::vector<uint64_t> key = graph_key_of(p, d_in, d_L, d_primary);
    for (auto& ge : p->graphs) {
        if (ge.key != key) continue;
        return launch_entry(p, ge, st, true);
    }

    bwt_status status = BWT_OK;
    // capture streams: the main graph, the loop body, the body's second round
    cudaStream_t cs = nullptr, bs = nullptr, rs = nullptr;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t launched = nullptr;
    cudaGraphConditionalHandle cond, cond_r1;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    cudaStreamCaptureStatus cst;
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cudaGraphNode_t cnode;
    cudaGraph_t body, tmp;
    uint64_t k0, k1, k2, k3, k4, r0, r1, r3, r4;

    CKG(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    CKG(cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking));
    CKG(cudaStreamCreateWithFlags(&rs, cudaStreamNonBlocking));
    CKG(cudaGraphCreate(&g, 0));
    CKG(cudaGraphConditionalHandleCreate(&cond, g, 0, 0));
    p->capturing = true;
    CKG(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    k0 = p->stats.kernel_launches;
    r0 = p->stats.radix_launches;
    CKS(reset_ctrl(p, cs));
    if (learned) CKS(enqueue_learned(p, d_in, cs));
    else CKS(enqueue_initial_sort(p, d_in, cs));
    CKG(launch_set_cond_initial(p->ctrl, p->max_n, cond, cs));
    p->stats.kernel_launches++;
    k1 = p->stats.kernel_launches;
    r1 = p->stats.radix_launches;
    CKG(cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps));
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    CKG(cudaGraphAddNode(&cnode, g, deps, nullptr, ndeps, &cp));
    body = cp.conditional.phGraph_out[0];
    CKG(cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies));
    // loop body: a round on bins[0]; then, if another round is due, a round
    // on bins[1] (an IF node, so a finished batch skips it)
    CKG(cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    CKS(enqueue_round(p, 0, nullptr, bs));
    CKG(cudaGraphConditionalHandleCreate(&cond_r1, body, 0, 0));
    CKG(launch_round_end(p->ctrl, 0, p->max_n, cond, cond_r1, 1 | 2 | 4, bs));
    p->stats.kernel_launches++;
    k2 = p->stats.kernel_launches;
    CKS(begin_if_capture(bs, rs, cond_r1));
    CKS(enqueue_round(p, 1, nullptr, rs));
    CKG(launch_round_end(p->ctrl, 1, p->max_n, cond, 0, 1 | 4, rs));
    p->stats.kernel_launches++;
    CKG(cudaStreamEndCapture(rs, &tmp));
    CKG(cudaStreamEndCapture(bs, &body));
    k3 = p->stats.kernel_launches;
    r3 = p->stats.radix_launches;
    {
        NvtxRange nv("gather");
        CKG(launch_gather_L(d_in, p->sa, p->blocks, p->tiles0, p->ntiles0, d_L, d_primary, p->ctrl, cs));
    }
    p->stats.kernel_launches++;
    k4 = p->stats.kernel_launches;
    r4 = p->stats.radix_launches;
    CKG(cudaStreamEndCapture(cs, &g));
    p->capturing = false;
    CKG(cudaGraphInstantiate(&exec, g, 0));
    CKG(cudaEventCreateWithFlags(&launched, cudaEventDisableTiming));
    cudaStreamDestroy(cs);
    cudaStreamDestroy(bs);
    cudaStreamDestroy(rs);
    cs = bs = rs = nullptr;
    {
        // the least recently used graph makes room (its last launch may still run)
        if (p->graphs.size() >= kGraphCache) {
            size_t lru = 0;
            for (size_t i = 1; i < p->graphs.size(); ++i)
                if (p->graphs[i].last_use < p->graphs[lru].last_use) lru = i;
            GraphEntry& old = p->graphs[lru];
            if (old.launched) {
                cudaEventSynchronize(old.launched);
                cudaEventDestroy(old.launched);
            }
            if (old.exec) cudaGraphExecDestroy(old.exec);
            if (old.graph) cudaGraphDestroy(old.graph);
            p->graphs.erase(p->graphs.begin() + (long)lru);
        }
        GraphEntry ge;
        ge.key = std::move(key);
        ge.graph = g;
        ge.exec = exec;
        g = nullptr;
        exec = nullptr;
        ge.main_kernels = (k1 - k0) + (k4 - k3);
        ge.large_kernels = p->cap_large_kernels;
        ge.round_kernels = (k2 - k1) - ge.large_kernels;  // one round and its end kernel, the section aside
        ge.main_radix = (r1 - r0) + (r4 - r3);
        ge.large_radix = p->cap_large_radix;
        ge.launched = launched;
        p->graphs.push_back(std::move(ge));
    }
    return launch_entry(p, p->graphs.back(), st, false);

fail:
    p->capturing = false;
    for (cudaStream_t s : {rs, bs, cs}) {  // innermost captures first
        if (!s) continue;
        cudaGraph_t t = nullptr;
        cudaStreamEndCapture(s, &t);
        cudaStreamDestroy(s);
    }
    if (launched) cudaEventDestroy(launched);
    if (exec) cudaGraphExecDestroy(exec);
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return status;
}

// After a graph run: kernel and round counts from the device control words
// (the rounds whose launches ran).
void bwt::graph_stats(bwt_plan* p) {
    const uint64_t rounds_run = p->h_ctrl[CTRL_BODY_ITERS];
    p->stats.rounds = p->h_ctrl[CTRL_ROUNDS];
    p->stats.kernel_launches =  // + the control-word copy after the graph
        p->graph_main_kernels + rounds_run * (p->graph_round_kernels + p->graph_large_kernels) + 1;
    p->stats.radix_launches = p->graph_main_radix + rounds_run * p->graph_large_radix;
}
