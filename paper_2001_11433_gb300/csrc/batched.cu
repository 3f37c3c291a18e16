// Batched MCE: many independent graphs in one persistent launch.
//
// The graphs are the vertex ranges of a disjoint union, so their per-vertex
// subproblems (Algorithm 5) never mix; one search kernel runs them all and
// reduces count and hash per graph.  A per-graph node budget turns graphs
// that are too large to finish into MCE_EBUDGET instead of a stall.
#include <vector>

#include "mce_host.h"

namespace mce {
namespace {

__global__ void k_graph_of(const int32_t *gptr, int32_t k, int32_t *graph_of) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < k; g += (int64_t)gridDim.x * blockDim.x)
        for (int32_t v = gptr[g]; v < gptr[g + 1]; ++v) graph_of[v] = (int32_t)g;
}

__global__ void k_check_disjoint(const int32_t *row_ptr, const int32_t *col, const int32_t *graph_of, int32_t n,
                                 int32_t *bad) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
        for (int32_t e = row_ptr[x]; e < row_ptr[x + 1]; ++e)
            if (graph_of[col[e]] != graph_of[x]) atomicOr(bad, 1);
}

__global__ void k_graph_status(const unsigned long long *nodes, int32_t k, uint64_t budget, int32_t *status,
                               int32_t *any) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < k; g += (int64_t)gridDim.x * blockDim.x) {
        const bool over = budget && nodes[g] > budget;
        status[g] = over ? MCE_EBUDGET : MCE_OK;
        if (over) atomicOr(any, 1);
    }
}

}  // namespace
}  // namespace mce

using namespace mce;

extern "C" mce_status mce_enumerate_batched(const mce_graph *g, const int32_t *graph_ptr, int32_t k,
                                            const mce_opts *opts, uint64_t *counts, uint64_t *hashes,
                                            int32_t *status, mce_result *total) {
    if (!g || !graph_ptr || k < 1 || !opts || !counts || !hashes || !status || !total) {
        g_last_error = "mce_enumerate_batched: bad arguments";
        return MCE_EINVAL;
    }
    if (graph_ptr[0] != 0 || graph_ptr[k] != g->n) {
        g_last_error = "mce_enumerate_batched: graph_ptr must start at 0 and end at n";
        return MCE_EINVAL;
    }
    for (int32_t i = 0; i < k; ++i)
        if (graph_ptr[i + 1] < graph_ptr[i]) {
            g_last_error = "mce_enumerate_batched: graph_ptr not monotone";
            return MCE_EINVAL;
        }
    cudaStream_t s = (cudaStream_t)opts->stream;
    DevBuf dptr, graph_of, gnodes, bad;
    MCE_TRY(dptr.alloc(((size_t)k + 1) * 4, s));
    MCE_TRY(graph_of.alloc(((size_t)g->n + 1) * 4, s));
    MCE_TRY(gnodes.alloc((size_t)k * 8, s));
    MCE_TRY(bad.alloc(8, s));
    MCE_CUDA(cudaMemcpyAsync(dptr.p, graph_ptr, ((size_t)k + 1) * 4, cudaMemcpyHostToDevice, s));
    MCE_CUDA(cudaMemsetAsync(gnodes.p, 0, (size_t)k * 8, s));
    MCE_CUDA(cudaMemsetAsync(bad.p, 0, 8, s));
    MCE_CUDA(cudaMemsetAsync(counts, 0, (size_t)k * 8, s));
    MCE_CUDA(cudaMemsetAsync(hashes, 0, (size_t)k * 8, s));
    MCE_LAUNCH(k_graph_of, grid_for(k, 128), 128, 0, s, dptr.as<int32_t>(), k, graph_of.as<int32_t>());
    if (g->n)
        MCE_LAUNCH(k_check_disjoint, grid_for(g->n, 256), 256, 0, s, g->row_ptr, g->col, graph_of.as<int32_t>(), g->n,
                   bad.as<int32_t>());
    int32_t hbad = 0;
    MCE_CUDA(cudaMemcpyAsync(&hbad, bad.p, 4, cudaMemcpyDeviceToHost, s));
    MCE_CUDA(cudaStreamSynchronize(s));
    if (hbad) {
        g_last_error = "mce_enumerate_batched: an edge joins two graphs";
        return MCE_EINVAL;
    }
    mce_opts o = *opts;
    o.node_budget = 0;   // the budget applies per graph
    o.pv_count = o.pv_hash = o.pv_nodes = nullptr;
    memset(total, 0, sizeof(*total));
    mce_status st = enumerate(g, &o, total, graph_of.as<int32_t>(), gnodes.as<unsigned long long>(),
                              opts->node_budget, (unsigned long long *)counts, (unsigned long long *)hashes);
    if (st != MCE_OK && st != MCE_EOVERFLOW) return st;
    MCE_CUDA(cudaMemsetAsync(bad.p, 0, 4, s));
    MCE_LAUNCH(k_graph_status, grid_for(k, 256), 256, 0, s, gnodes.as<unsigned long long>(), k, opts->node_budget,
               status, bad.as<int32_t>());
    MCE_CUDA(cudaMemcpyAsync(&hbad, bad.p, 4, cudaMemcpyDeviceToHost, s));
    MCE_CUDA(cudaStreamSynchronize(s));
    if (hbad) total->complete = 0;
    return st;
}

// ------------------------------------------------------------------ reusable batched plan
//
// mce_batched_create prepares everything once (graph ids, rank, Γ+ lists,
// trivial subproblems, the heaviest-first order, every buffer); a run is then
// a fixed sequence of copies, memsets and two kernels on one stream, captured
// into a CUDA graph on its first call and replayed afterwards.  The tuner
// times launch shapes (resident blocks per SM, hand-over interval) on runs
// whose per-graph budget is cut, and keeps the fastest.

namespace mce {
namespace {

__global__ void k_plan_reset(unsigned long long *seq, int64_t qcap, unsigned long long *ctl, unsigned long long pending) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < qcap; i += (int64_t)gridDim.x * blockDim.x)
        seq[i] = (unsigned long long)i;
    if (blockIdx.x == 0 && threadIdx.x < CTL_WORDS) ctl[threadIdx.x] = threadIdx.x == CTL_PENDING ? pending : 0ULL;
}

}  // namespace
}  // namespace mce

struct mce_batched {
    const mce_graph *g = nullptr;
    int32_t k = 0;
    cudaStream_t cap = nullptr;   // private stream the run is captured on
    mce::DevBuf graph_of, rank, up_ptr, up_col, order, out0, out, gcount0, ghash0, gcount, ghash, gnodes, status, any,
        cache, coff;
    mce::BkBuffers bb;
    mce::BkParams P{};
    mce::LaunchShape ls;
    int64_t per_warp = 0, cmax = 0, cache_words = 0;
    uint64_t budget = 0;
    int32_t warp_small = 0;     // small nodes by the whole warp (1) or by the lanes (0)
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    uint64_t launches = 0;
};

namespace mce {
namespace {

// (re)allocate the per-warp buffers for the plan's launch shape
mce_status plan_shape(mce_batched *b, cudaStream_t s) {
    const int64_t nwarps = (int64_t)num_sms() * b->ls.blocks_per_sm * b->ls.warps_per_block;
    BkParams &P = b->P;
    P.gws_words = b->per_warp > b->ls.smem_words ? b->per_warp : 16;
    P.smem_words = b->ls.smem_words;
    P.lp_words = b->ls.lp_words;
    MCE_TRY(alloc_lp_tasks(P, nwarps, s, b->bb));
    MCE_TRY(b->bb.gws.alloc((size_t)nwarps * P.gws_words * 4, s));
    P.gws = b->bb.gws.as<uint32_t>();
    const int64_t wcmax = (b->cmax + 31) / 32;
    P.slot_words = (2 + b->cmax + 4 * wcmax + 3) & ~int64_t(3);
    int64_t cap = ((int64_t)1 << 26) / P.slot_words;
    if (cap > ((int64_t)1 << 16)) cap = (int64_t)1 << 16;
    if (cap < 1024) cap = 1024;
    P.qcap = cap;
    MCE_TRY(b->bb.arena.alloc((size_t)P.qcap * P.slot_words * 4, s));
    MCE_TRY(b->bb.qseq.alloc((size_t)P.qcap * 8, s));
    MCE_TRY(b->bb.taskbuf.alloc((size_t)nwarps * P.slot_words * 4, s));
    MCE_TRY(b->bb.ctl.alloc(CTL_WORDS * 8, s));
    P.arena = b->bb.arena.as<uint32_t>();
    P.qseq = b->bb.qseq.as<unsigned long long>();
    P.taskbuf = b->bb.taskbuf.as<uint32_t>();
    P.ctl = b->bb.ctl.as<unsigned long long>();
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    return MCE_OK;
}

// the stream work of one run (no host synchronisation, no allocation)
mce_status plan_issue(mce_batched *b, cudaStream_t s) {
    BkParams &P = b->P;
    const int32_t n = b->g->n, k = b->k;
    MCE_CUDA(cudaMemcpyAsync(b->out.p, b->out0.p, OUT_WORDS * 8, cudaMemcpyDeviceToDevice, s));
    MCE_CUDA(cudaMemcpyAsync(b->gcount.p, b->gcount0.p, (size_t)k * 8, cudaMemcpyDeviceToDevice, s));
    MCE_CUDA(cudaMemcpyAsync(b->ghash.p, b->ghash0.p, (size_t)k * 8, cudaMemcpyDeviceToDevice, s));
    MCE_CUDA(cudaMemsetAsync(b->gnodes.p, 0, (size_t)k * 8, s));
    MCE_CUDA(cudaMemsetAsync(b->any.p, 0, 4, s));
    if (b->coff.p) MCE_CUDA(cudaMemsetAsync(b->coff.p, 0xff, (size_t)n * 8, s));
    if (P.n_sub > 0) {
        MCE_LAUNCH(k_plan_reset, grid_for(P.qcap, 256), 256, 0, s, P.qseq, P.qcap, P.ctl, (unsigned long long)P.n_sub);
        MCE_TRY(launch_bk(P, b->ls.warps_per_block, b->ls.blocks_per_sm, s));
    } else {
        MCE_CUDA(cudaMemsetAsync(P.ctl, 0, CTL_WORDS * 8, s));
    }
    MCE_LAUNCH(k_graph_status, grid_for(k, 256), 256, 0, s, b->gnodes.as<unsigned long long>(), k, P.graph_budget,
               b->status.as<int32_t>(), b->any.as<int32_t>());
    return MCE_OK;
}

}  // namespace
}  // namespace mce

extern "C" {

mce_status mce_batched_create(const mce_graph *g, const int32_t *graph_ptr, int32_t k, const mce_opts *opts,
                              mce_batched **out) {
    if (!g || !graph_ptr || k < 1 || !opts || !out) {
        g_last_error = "mce_batched_create: bad arguments";
        return MCE_EINVAL;
    }
    if (graph_ptr[0] != 0 || graph_ptr[k] != g->n) {
        g_last_error = "mce_batched_create: graph_ptr must start at 0 and end at n";
        return MCE_EINVAL;
    }
    for (int32_t i = 0; i < k; ++i)
        if (graph_ptr[i + 1] < graph_ptr[i]) {
            g_last_error = "mce_batched_create: graph_ptr not monotone";
            return MCE_EINVAL;
        }
    mce_batched *b = new mce_batched();
    struct Guard {
        mce_batched *&b;
        bool keep = false;
        ~Guard() {
            if (!keep) mce_batched_free(b);
        }
    } guard{b};
    cudaStream_t s = (cudaStream_t)opts->stream;
    const int32_t n = g->n;
    b->g = g;
    b->k = k;
    MCE_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    b->budget = opts->node_budget;
    DevBuf dptr, bad, flag, keys, reqb, tmp;
    MCE_TRY(dptr.alloc(((size_t)k + 1) * 4, s));
    MCE_TRY(b->graph_of.alloc(((size_t)n + 1) * 4, s));
    MCE_TRY(bad.alloc(8, s));
    MCE_CUDA(cudaMemcpyAsync(dptr.p, graph_ptr, ((size_t)k + 1) * 4, cudaMemcpyHostToDevice, s));
    MCE_CUDA(cudaMemsetAsync(bad.p, 0, 8, s));
    MCE_LAUNCH(k_graph_of, grid_for(k, 128), 128, 0, s, dptr.as<int32_t>(), k, b->graph_of.as<int32_t>());
    if (n)
        MCE_LAUNCH(k_check_disjoint, grid_for(n, 256), 256, 0, s, g->row_ptr, g->col, b->graph_of.as<int32_t>(), n,
                   bad.as<int32_t>());
    int32_t hbad = 0;
    MCE_CUDA(cudaMemcpyAsync(&hbad, bad.p, 4, cudaMemcpyDeviceToHost, s));
    MCE_CUDA(cudaStreamSynchronize(s));
    if (hbad) {
        g_last_error = "mce_batched_create: an edge joins two graphs";
        return MCE_EINVAL;
    }
    // rank, Γ+ lists, trivial subproblems, order
    MCE_TRY(b->rank.alloc(((size_t)n + 1) * 4, s));
    MCE_TRY(compute_rank(g, opts, s, b->rank.as<int32_t>()));
    int64_t up_nnz = 0;
    MCE_TRY(build_up_lists(g, b->rank.as<int32_t>(), s, b->up_ptr, b->up_col, &up_nnz));
    for (DevBuf *d : {&b->out0, &b->out}) MCE_TRY(d->alloc(OUT_WORDS * 8, s));
    for (DevBuf *d : {&b->gcount0, &b->ghash0, &b->gcount, &b->ghash, &b->gnodes}) MCE_TRY(d->alloc((size_t)k * 8, s));
    MCE_TRY(b->status.alloc((size_t)k * 4, s));
    MCE_TRY(b->any.alloc(8, s));
    MCE_CUDA(cudaMemsetAsync(b->out0.p, 0, OUT_WORDS * 8, s));
    MCE_CUDA(cudaMemsetAsync(b->gcount0.p, 0, (size_t)k * 8, s));
    MCE_CUDA(cudaMemsetAsync(b->ghash0.p, 0, (size_t)k * 8, s));
    MCE_TRY(flag.alloc(((size_t)n + 1) * 4, s));
    MCE_TRY(keys.alloc(((size_t)n + 1) * 8, s));
    MCE_TRY(reqb.alloc(32, s));
    MCE_CUDA(cudaMemsetAsync(reqb.p, 0, 32, s));
    MCE_TRY(launch_prepass(g, b->up_ptr.as<int32_t>(), opts->hash_seed, nullptr, b->out0.as<unsigned long long>(),
                           flag.as<int32_t>(), keys.as<uint64_t>(), reqb.as<unsigned long long>(),
                           b->graph_of.as<int32_t>(), b->gcount0.as<unsigned long long>(),
                           b->ghash0.as<unsigned long long>(), s));
    MCE_TRY(exclusive_scan_i32(flag.as<int32_t>(), flag.as<int32_t>(), n, s));
    int32_t n_act = 0;
    unsigned long long reqc[4] = {0, 0, 0, 0};
    MCE_CUDA(cudaMemcpyAsync(&n_act, flag.as<int32_t>() + n, 4, cudaMemcpyDeviceToHost, s));
    MCE_CUDA(cudaMemcpyAsync(reqc, reqb.p, 32, cudaMemcpyDeviceToHost, s));
    MCE_CUDA(cudaStreamSynchronize(s));
    MCE_TRY(b->order.alloc(((size_t)n_act + 1) * 4, s));
    if (n_act > 0) {
        MCE_TRY(tmp.alloc((size_t)n_act * 16, s));
        MCE_TRY(launch_order(flag.as<int32_t>(), keys.as<uint64_t>(), n, n_act, g->id_bits, tmp.as<uint64_t>(),
                             b->order.as<int32_t>(), s));
    }
    b->cmax = (int64_t)reqc[1];
    const int64_t cw = (int64_t)reqc[2] < ((int64_t)1 << 30) ? (int64_t)reqc[2] : ((int64_t)1 << 30);
    // as mce_enumerate: the private part only when the cache holds every build
    b->per_warp = (int64_t)reqc[0];
    if (cw == (int64_t)reqc[2]) b->per_warp = (int64_t)reqc[3];
    else if (b->per_warp > ((int64_t)1 << 24))
        b->per_warp = (int64_t)reqc[3] > ((int64_t)1 << 24) ? (int64_t)reqc[3] : ((int64_t)1 << 24);
    BkParams &P = b->P;
    P.mode = BK_MCE;
    P.row_ptr = g->row_ptr;
    P.col = g->col;
    P.up_ptr = b->up_ptr.as<int32_t>();
    P.up_col = b->up_col.as<int32_t>();
    P.rank = b->rank.as<int32_t>();
    P.order = b->order.as<int32_t>();
    P.n_sub = n_act;
    P.graph_of = b->graph_of.as<int32_t>();
    P.graph_nodes = b->gnodes.as<unsigned long long>();
    P.graph_budget = opts->node_budget;
    P.g_count = b->gcount.as<unsigned long long>();
    P.g_hash = b->ghash.as<unsigned long long>();
    P.seed = opts->hash_seed;
    P.out = b->out.as<unsigned long long>();
    P.split = opts->split;
    P.split_nodes = opts->split ? (opts->split_nodes ? opts->split_nodes : 4096u) : 0u;
    P.max_run_ns = (uint64_t)(opts->time_limit_ms ? opts->time_limit_ms : 600000u) * 1000000ULL;
    P.timeout_ns = 60ULL * 1000000000ULL;
    if (cw > 0) {
        MCE_TRY(b->cache.alloc((size_t)cw * 4 + 512, s));
        MCE_TRY(b->coff.alloc((size_t)n * 8, s));
        P.cache = reinterpret_cast<uint32_t *>(((uintptr_t)b->cache.p + 127) & ~(uintptr_t)127);
        P.cache_words = cw;
        P.cache_off = b->coff.as<long long>();
    }
    {
        // With a per-graph budget the lane search would finish its buffered
        // small subtrees past the budget of graphs that run out (measured on
        // GB300: 47 % more tree nodes and a 1.2x longer run on 4,096 G(n, p)),
        // so the whole-warp small search is the default then; a positive
        // lane_search_words asks for the lane search all the same.
        mce_opts o = *opts;
        if (opts->node_budget && opts->lane_search_words <= 0) o.warp_small_search = 1;
        b->ls = launch_shape(&o);
        b->warp_small = o.warp_small_search;
    }
    MCE_TRY(plan_shape(b, s));
    MCE_CUDA(cudaStreamSynchronize(s));
    guard.keep = true;
    *out = b;
    return MCE_OK;
}

mce_status mce_batched_run(mce_batched *b, void *stream) {
    if (!b) return MCE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (!b->exec) {
        // capture the run once; later runs replay it
        MCE_TRY(bk_prepare(b->ls.blocks_per_sm,
                           bk_block_smem_bytes(b->ls.warps_per_block, b->ls.smem_words, b->ls.lp_words)));
        const uint64_t before = g_launches.load(std::memory_order_relaxed);
        // captured on the plan's own stream (the legacy default stream
        // cannot be captured); the graph is launched on the caller's stream
        MCE_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        const mce_status st = plan_issue(b, b->cap);
        // kernels counted at capture are counted again at every replay
        b->launches = g_launches.load(std::memory_order_relaxed) - before;
        g_launches.fetch_sub(b->launches, std::memory_order_relaxed);
        cudaGraph_t gr = nullptr;
        const cudaError_t e = cudaStreamEndCapture(b->cap, &gr);
        if (st != MCE_OK) {
            if (gr) cudaGraphDestroy(gr);
            return st;
        }
        MCE_CUDA(e);
        b->graph = gr;
        MCE_CUDA(cudaGraphInstantiate(&b->exec, gr, 0));
    }
    g_launches.fetch_add(b->launches, std::memory_order_relaxed);
    MCE_CUDA(cudaGraphLaunch(b->exec, s));
    return MCE_OK;
}

mce_status mce_batched_read(mce_batched *b, void *stream, uint64_t *counts, uint64_t *hashes, int32_t *status,
                            mce_result *total) {
    if (!b || !total) return MCE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t k = b->k;
    if (counts) MCE_CUDA(cudaMemcpyAsync(counts, b->gcount.p, (size_t)k * 8, cudaMemcpyDeviceToHost, s));
    if (hashes) MCE_CUDA(cudaMemcpyAsync(hashes, b->ghash.p, (size_t)k * 8, cudaMemcpyDeviceToHost, s));
    if (status) MCE_CUDA(cudaMemcpyAsync(status, b->status.p, (size_t)k * 4, cudaMemcpyDeviceToHost, s));
    int32_t any = 0;
    MCE_CUDA(cudaMemcpyAsync(&any, b->any.p, 4, cudaMemcpyDeviceToHost, s));
    memset(total, 0, sizeof(*total));
    mce_status st = read_result(b->out, b->bb.ctl, s, total);
    total->subproblems = b->P.n_sub;
    if (any) total->complete = 0;
    return st;
}

mce_status mce_batched_tune(mce_batched *b, void *stream, uint64_t tune_budget, int32_t repeats,
                            int32_t *best_blocks_per_sm, uint32_t *best_split_nodes, int32_t *best_warp_small) {
    if (!b || repeats < 1) return MCE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    struct Cand {
        int32_t bps;
        uint32_t split;
        int32_t ws;   // 1 = whole-warp small search, 0 = lane search
    };
    const Cand cands[] = {{2, 4096, 1}, {3, 4096, 1}, {3, 8192, 1}, {4, 4096, 1},
                          {2, 4096, 0}, {2, 12288, 0}, {3, 4096, 0}};
    const uint64_t keep_budget = b->P.graph_budget;
    const LaunchShape keep_ls = b->ls;
    const uint32_t keep_split = b->P.split_nodes;
    if (tune_budget && (keep_budget == 0 || tune_budget < keep_budget)) b->P.graph_budget = tune_budget;
    cudaEvent_t e0, e1;
    MCE_CUDA(cudaEventCreate(&e0));
    MCE_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    Cand bestc = {keep_ls.blocks_per_sm, keep_split, b->warp_small};
    for (const Cand &c : cands) {
        mce_opts o;
        mce_opts_init(&o);
        o.blocks_per_sm = c.bps;
        o.warp_small_search = c.ws;
        b->ls = launch_shape(&o);
        b->P.split_nodes = b->P.split ? c.split : 0u;
        mce_status st = plan_shape(b, s);
        if (st != MCE_OK) break;
        float tsum = 0.f;
        for (int r = 0; r < repeats && st == MCE_OK; ++r) {
            cudaEventRecord(e0, s);
            st = plan_issue(b, s);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            tsum += ms;
        }
        if (st == MCE_OK && tsum < best) {
            best = tsum;
            bestc = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    mce_opts o;
    mce_opts_init(&o);
    o.blocks_per_sm = bestc.bps;
    o.warp_small_search = bestc.ws;
    b->ls = launch_shape(&o);
    b->warp_small = bestc.ws;
    b->P.split_nodes = b->P.split ? bestc.split : 0u;
    b->P.graph_budget = keep_budget;
    MCE_TRY(plan_shape(b, s));
    MCE_CUDA(cudaStreamSynchronize(s));
    if (best_blocks_per_sm) *best_blocks_per_sm = bestc.bps;
    if (best_split_nodes) *best_split_nodes = bestc.split;
    if (best_warp_small) *best_warp_small = bestc.ws;
    return MCE_OK;
}

void mce_batched_free(mce_batched *b) {
    if (!b) return;
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}

}  // extern "C"
