// Step graphs: a list of bubbles — of one or several contexts (parameter points with their
// own grids and models), loop parts and channels — captured once into a CUDA graph and
// replayed as one launch per step.  Bubbles of one context run in list order (they share
// its workspace); the bubbles of different contexts run on separate branches of the graph
// and may overlap on the GPU.  Slot additions run in their context's branch; a join entry
// makes every branch wait for all others (the next loop order of a multiloop step).
#include <algorithm>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "kb_internal.h"

struct kb_graph {
    int device = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<std::pair<kb_ctx*, unsigned long long>> launches;   // kernels per replay, per context
    // each context's memory generation at capture: the graph's kernels hold its workspace,
    // table and record-cache addresses, so it must not run once any of them was replaced
    std::vector<std::pair<kb_ctx*, unsigned long long>> mem_gen;
    unsigned long long kernels = 0;
};

namespace {

struct Branch {
    kb_ctx* ctx;
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    size_t need = 0;
    unsigned long long launches0 = 0;
};

kb_status fail(kb_ctx* ctx, const std::string& msg, kb_status s) {
    if (ctx) ctx->err = msg;
    return s;
}

}  // namespace

extern "C" {

kb_status kb_graph_create(kb_graph** out, const kb_bubble_desc* d, int n) {
    if (!out) return KB_ERR_ARG;
    *out = nullptr;
    if (!d || n < 1) return KB_ERR_ARG;
    kb_ctx* c0 = nullptr;
    for (int i = 0; i < n && !c0; ++i)
        if (d[i].op != KB_OP_JOIN) c0 = d[i].ctx;
    if (!c0) return KB_ERR_ARG;
    std::vector<Branch> br;
    std::map<kb_ctx*, size_t> index;
    int joins = 0;
    for (int i = 0; i < n; ++i) {
        if (d[i].op == KB_OP_JOIN) { ++joins; continue; }
        kb_ctx* c = d[i].ctx;
        if (!c) return fail(c0, "kb_graph_create: null context in descriptor", KB_ERR_ARG);
        if (c->device != c0->device) return fail(c0, "kb_graph_create: contexts on different devices", KB_ERR_ARG);
        if (!c->grids_set || !c->model_set) return fail(c, "kb_graph_create: set grids and model first", KB_ERR_STATE);
        if (d[i].op != KB_OP_BUBBLE && d[i].op != KB_OP_ADD && d[i].op != KB_OP_CACHE && d[i].op != KB_OP_IMAGE &&
            d[i].op != KB_OP_T_SU2 && d[i].op != KB_OP_T_SU2_FINISH)
            return fail(c, "kb_graph_create: unknown entry kind", KB_ERR_ARG);
        if (d[i].op == KB_OP_T_SU2_FINISH) {
            kb_ctx* c2 = d[i].ctx2;
            if (!c2 || d[i].slot2 < 0 || d[i].slot2 >= KB_MAX_SLOTS || !c2->slot_set[d[i].slot2] ||
                !c2->slots[d[i].slot2].cls[KB_CH_A][KB_K3])
                return fail(c, "kb_graph_create: the a-channel K3 source of a T_SU2_FINISH entry is not set",
                            KB_ERR_ARG);
            bool seen = false;
            for (int q = 0; q < i; ++q) seen |= d[q].op != KB_OP_JOIN && d[q].ctx == c2;
            if (!seen)
                return fail(c, "kb_graph_create: the source context of a T_SU2_FINISH entry has no earlier entries",
                            KB_ERR_ARG);
        }
        if (d[i].channel < 0 || d[i].channel > 2 || (d[i].class_mask & ~KB_MASK_ALL) ||
            (d[i].op == KB_OP_CACHE && (d[i].class_mask < 1 || d[i].class_mask > 15)) ||
            (d[i].op == KB_OP_BUBBLE && d[i].precision != KB_PREC_FP64 && d[i].precision != KB_PREC_MIXED))
            return fail(c, "kb_graph_create: descriptor out of range", KB_ERR_ARG);
        if (!index.count(c)) { index[c] = br.size(); br.push_back(Branch{c}); }
        if (d[i].op != KB_OP_BUBBLE && d[i].op != KB_OP_T_SU2) continue;
        Branch& b = br[index[c]];
        size_t need = d[i].op == KB_OP_T_SU2 ? kb_mixed_workspace_need(c, KB_CH_T, d[i].class_mask)
                      : d[i].precision == KB_PREC_FP64 ? kb_fp64_workspace_need(c, d[i].channel, d[i].class_mask)
                                                       : kb_mixed_workspace_need(c, d[i].channel, d[i].class_mask);
        b.need = std::max(b.need, need);
    }
    if (cudaSetDevice(c0->device) != cudaSuccess) return fail(c0, "cudaSetDevice failed", KB_ERR_CUDA);
    // everything that allocates, synchronises or copies happens before the capture
    for (int i = 0; i < n; ++i)
        if (d[i].op == KB_OP_CACHE) {
            kb_status s = kb_vertex_cache_prepare(d[i].ctx, d[i].slot_left, d[i].channel, d[i].class_mask);
            if (s != KB_OK) return s;
        }
    for (auto& b : br) {
        kb_status s = kb_ensure_workspace(b.ctx, b.need, nullptr, true);
        if (s != KB_OK) return s;
        s = kb_fp64_prepare(b.ctx);
        if (s != KB_OK) return s;
    }
    bool any_mixed = false;
    for (int i = 0; i < n; ++i)
        any_mixed |= (d[i].op == KB_OP_BUBBLE && d[i].precision == KB_PREC_MIXED) || d[i].op == KB_OP_T_SU2;
    if (any_mixed && !kb_tc_prepare(c0->device))
        return fail(c0, "kb_graph_create: tensor-core kernel setup failed", KB_ERR_CUDA);
    if (any_mixed && !kb_mixed_prepare(c0->device))
        return fail(c0, "kb_graph_create: mixed-path kernel setup failed", KB_ERR_CUDA);
    // contexts with autotuning on: tune their contraction shapes now (timing is not possible
    // inside a capture); the replays use the tuned split-K factors
    for (int i = 0; i < n; ++i) {
        const kb_bubble_desc& x = d[i];
        if (x.op == KB_OP_T_SU2 && x.ctx->autotune) {
            kb_status s = kb_mixed_tune(x.ctx, KB_CH_T, x.slot_left, x.slot_left, x.class_mask, 0.0, nullptr, true);
            if (s != KB_OK) return s;
            continue;
        }
        if (x.op != KB_OP_BUBBLE || x.precision != KB_PREC_MIXED || !x.ctx->autotune) continue;
        kb_status s = kb_mixed_tune(x.ctx, x.channel, x.slot_left, x.slot_right, x.class_mask, x.beta, nullptr);
        if (s != KB_OK) return s;
    }
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(c0, "kb_graph_create: tuning failed", KB_ERR_CUDA);

    cudaStream_t s0 = nullptr;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join_ev((size_t)joins * br.size(), nullptr);
    int finishes = 0;
    for (int i = 0; i < n; ++i) finishes += d[i].op == KB_OP_T_SU2_FINISH;
    join_ev.resize(join_ev.size() + (size_t)finishes, nullptr);      // one event per finish entry at the end
    kb_status st = KB_OK;
    auto cleanup = [&]() {
        for (auto& b : br) {
            if (b.st) cudaStreamDestroy(b.st);
            if (b.done) cudaEventDestroy(b.done);
        }
        for (auto e : join_ev)
            if (e) cudaEventDestroy(e);
        if (fork) cudaEventDestroy(fork);
        if (s0) cudaStreamDestroy(s0);
    };
    if (cudaStreamCreateWithFlags(&s0, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess) {
        cleanup();
        return fail(c0, "kb_graph_create: stream/event creation failed", KB_ERR_CUDA);
    }
    for (auto& b : br)
        if (cudaStreamCreateWithFlags(&b.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming) != cudaSuccess) {
            cleanup();
            return fail(c0, "kb_graph_create: stream/event creation failed", KB_ERR_CUDA);
        }
    for (auto& e : join_ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            cleanup();
            return fail(c0, "kb_graph_create: stream/event creation failed", KB_ERR_CUDA);
        }
    std::vector<bool> prof(br.size());
    for (size_t i = 0; i < br.size(); ++i) {
        prof[i] = br[i].ctx->prof_on;
        br[i].ctx->prof_on = false;   // no timing events inside a graph
        br[i].launches0 = br[i].ctx->launches;
    }
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        st = fail(c0, "kb_graph_create: cudaStreamBeginCapture failed", KB_ERR_CUDA);
    } else {
        cudaEventRecord(fork, s0);
        for (auto& b : br) cudaStreamWaitEvent(b.st, fork, 0);
        int jn = 0, fn = 0;
        for (int i = 0; i < n && st == KB_OK; ++i) {
            const kb_bubble_desc& x = d[i];
            if (x.op == KB_OP_T_SU2_FINISH) {
                // ctx's branch waits for everything ctx2's branch has so far, then finishes K3
                cudaEvent_t ev = join_ev[(size_t)joins * br.size() + fn++];
                cudaEventRecord(ev, br[index[x.ctx2]].st);
                cudaStreamWaitEvent(br[index[x.ctx]].st, ev, 0);
                const kb::VertexDev& src = x.ctx2->slots[x.slot2];
                st = kb_t_su2_finish(x.ctx, x.out_slot, src.cls[KB_CH_A][KB_K3], src.dt[KB_CH_A][KB_K3], x.alpha,
                                     br[index[x.ctx]].st);
            } else if (x.op == KB_OP_T_SU2) {
                st = kb_bubble_t_su2(x.ctx, x.slot_left, x.out_slot, x.pi_kind, x.class_mask, x.alpha,
                                     br[index[x.ctx]].st);
            } else if (x.op == KB_OP_JOIN) {
                cudaEvent_t* ev = &join_ev[(size_t)jn++ * br.size()];
                for (size_t b = 0; b < br.size(); ++b) cudaEventRecord(ev[b], br[b].st);
                for (size_t b = 0; b < br.size(); ++b)
                    for (size_t o = 0; o < br.size(); ++o)
                        if (o != b) cudaStreamWaitEvent(br[b].st, ev[o], 0);
            } else if (x.op == KB_OP_CACHE) {
                st = kb_vertex_cache_launch(x.ctx, x.slot_left, x.channel, x.class_mask, br[index[x.ctx]].st);
            } else if (x.op == KB_OP_IMAGE) {
                st = kb_vertex_image_impl(x.ctx, x.channel, x.slot_left, x.out_slot, x.class_mask, br[index[x.ctx]].st);
            } else if (x.op == KB_OP_ADD) {
                st = kb_vertex_add_impl(x.ctx, x.channel, x.slot_left, x.out_slot, x.class_mask, x.alpha,
                                        br[index[x.ctx]].st);
            } else {
                st = kb_bubble(x.ctx, x.channel, x.slot_left, x.slot_right, x.out_slot, x.pi_kind, x.class_mask,
                               x.alpha, x.beta, x.precision, br[index[x.ctx]].st);
            }
        }
        for (auto& b : br) {
            cudaEventRecord(b.done, b.st);
            cudaStreamWaitEvent(s0, b.done, 0);
        }
        cudaError_t e = cudaStreamEndCapture(s0, &graph);
        if (st == KB_OK && e != cudaSuccess)
            st = fail(c0, std::string("kb_graph_create: capture failed: ") + cudaGetErrorString(e), KB_ERR_CUDA);
    }
    kb_graph* g = nullptr;
    if (st == KB_OK) {
        g = new (std::nothrow) kb_graph();
        if (!g) st = KB_ERR_OOM;
    }
    for (size_t i = 0; i < br.size(); ++i) {
        unsigned long long k = br[i].ctx->launches - br[i].launches0;
        br[i].ctx->launches = br[i].launches0;   // captured, not run
        br[i].ctx->prof_on = prof[i];
        if (g) {
            g->launches.push_back({br[i].ctx, k});
            g->mem_gen.push_back({br[i].ctx, br[i].ctx->mem_gen});
            g->kernels += k;
        }
    }
    if (st == KB_OK) {
        cudaError_t e = cudaGraphInstantiate(&g->exec, graph, 0);
        if (e != cudaSuccess) {
            st = fail(c0, std::string("kb_graph_create: instantiate failed: ") + cudaGetErrorString(e), KB_ERR_CUDA);
        }
    }
    cudaGetLastError();
    cleanup();
    if (st != KB_OK) {
        if (graph) cudaGraphDestroy(graph);
        delete g;
        return st;
    }
    g->graph = graph;
    g->device = c0->device;
    *out = g;
    return KB_OK;
}

kb_status kb_graph_launch(kb_graph* g, void* stream) {
    if (!g || !g->exec) return KB_ERR_ARG;
    for (auto& p : g->mem_gen)
        if (p.first->mem_gen != p.second) {
            p.first->err = "kb_graph_launch: the context's workspace, tables or record caches changed since the "
                           "capture; create the graph again";
            return KB_ERR_STATE;
        }
    if (cudaSetDevice(g->device) != cudaSuccess) return KB_ERR_CUDA;
    if (cudaGraphLaunch(g->exec, reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) return KB_ERR_CUDA;
    for (auto& p : g->launches) p.first->launches += p.second;
    return KB_OK;
}

kb_status kb_graph_kernel_count(kb_graph* g, unsigned long long* count) {
    if (!g || !count) return KB_ERR_ARG;
    *count = g->kernels;
    return KB_OK;
}

kb_status kb_graph_destroy(kb_graph* g) {
    if (!g) return KB_ERR_ARG;
    cudaSetDevice(g->device);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return KB_OK;
}

}  // extern "C"
