// mce_enumerate_stream: the clique list of a static enumeration streamed to
// the host in chunks, for outputs larger than any device buffer (the
// paper's largest outputs hold billions of maximal cliques).
//
// The rank is computed once.  The vertices are then taken in id order, a
// chunk of subproblems (Algorithm 5) at a time, each chunk enumerated with
// its clique list into one of two device buffers.  While chunk i + 1 runs,
// chunk i's list is copied to pinned host memory on a second stream and then
// handed to the caller's sink, so that the copy overlaps the search.  A chunk
// whose list does not fit is split in half and run again (its partial output
// is discarded); chunks grow again while their lists stay small.
#include <string.h>

#include <vector>

#include "mce_host.h"

namespace mce {
namespace {

__global__ void k_iota_i32(int32_t *a, int32_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = (int32_t)i;
}

struct HostBuf {
    void *p = nullptr;
    ~HostBuf() {
        if (p) cudaFreeHost(p);
    }
};

struct Slot {
    DevBuf off, vtx;
    HostBuf hoff, hvtx;
    cudaEvent_t copied = nullptr;
    int64_t n_cliques = 0, n_words = 0;
    bool pending = false;
    ~Slot() {
        if (copied) cudaEventDestroy(copied);
    }
};

void add_result(mce_result *acc, const mce_result &r) {
    acc->count += r.count;
    acc->hash += r.hash;
    acc->tree_nodes += r.tree_nodes;
    if (r.hist_len > acc->hist_len) acc->hist_len = r.hist_len;
    for (int i = 0; i < r.hist_len; ++i) acc->hist[i] += r.hist[i];
    acc->tasks_split += r.tasks_split;
    acc->subproblems += r.subproblems;
    acc->ms_enum += r.ms_enum;
    acc->ms_search += r.ms_search;
    acc->word_ops += r.word_ops;
    acc->list_cliques += r.list_cliques;
    acc->list_words += r.list_words;
}

}  // namespace
}  // namespace mce

using namespace mce;

extern "C" mce_status mce_enumerate_stream(const mce_graph *g, const mce_opts *opts, int64_t buf_words,
                                           mce_clique_sink sink, void *ctx, mce_result *res) {
    if (!g || !opts || !sink || !res || buf_words < 64 || opts->whole_graph || opts->subset || opts->list_off ||
        opts->pv_count) {
        g_last_error = "mce_enumerate_stream: bad arguments (whole_graph, subset, lists and per-vertex "
                       "outputs are not offered here)";
        return MCE_EINVAL;
    }
    memset(res, 0, sizeof(*res));
    res->complete = 1;
    const int32_t n = g->n;
    if (n == 0) return MCE_OK;
    cudaStream_t s = (cudaStream_t)opts->stream;
    cudaStream_t cs = nullptr;
    MCE_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamDestroy(s); }
    } sg{cs};
    // the rank, once
    DevBuf rank, ids;
    MCE_TRY(rank.alloc((size_t)n * 4, s));
    MCE_TRY(ids.alloc((size_t)n * 4, s));
    cudaEvent_t e0, e1;
    MCE_CUDA(cudaEventCreate(&e0));
    MCE_CUDA(cudaEventCreate(&e1));
    struct EvGuard {
        cudaEvent_t a, b;
        ~EvGuard() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } eg{e0, e1};
    MCE_CUDA(cudaEventRecord(e0, s));
    MCE_TRY(compute_rank(g, opts, s, rank.as<int32_t>()));
    MCE_CUDA(cudaEventRecord(e1, s));
    MCE_LAUNCH(k_iota_i32, grid_for(n, 256), 256, 0, s, ids.as<int32_t>(), n);
    // two list buffers: cliques at most buf_words / 2 (a clique takes >= 2 words)
    const int64_t max_cl = buf_words / 2;
    Slot slot[2];
    // on every return, copies in flight finish before the buffers are freed
    struct CopyGuard {
        cudaStream_t s;
        ~CopyGuard() { cudaStreamSynchronize(s); }
    } cg{cs};
    for (auto &sl : slot) {
        MCE_TRY(sl.off.alloc((size_t)max_cl * 8, s));
        MCE_TRY(sl.vtx.alloc((size_t)buf_words * 4, s));
        MCE_CUDA(cudaMallocHost(&sl.hoff.p, (size_t)max_cl * 8));
        MCE_CUDA(cudaMallocHost(&sl.hvtx.p, (size_t)buf_words * 4));
        MCE_CUDA(cudaEventCreateWithFlags(&sl.copied, cudaEventDisableTiming));
    }
    auto deliver = [&](Slot &sl) -> mce_status {
        if (!sl.pending) return MCE_OK;
        MCE_CUDA(cudaEventSynchronize(sl.copied));
        // offsets within the chunk: the sink gets them as they are
        sink(ctx, (const int64_t *)sl.hoff.p, (const int32_t *)sl.hvtx.p, sl.n_cliques, sl.n_words);
        sl.pending = false;
        return MCE_OK;
    };
    mce_opts oc = *opts;
    oc.rank_kind = MCE_RANK_USER;
    oc.user_rank = rank.as<int32_t>();
    oc.subset_on_host = 0;
    int64_t start = 0, chunk = n < 4096 ? n : 4096;
    int cur = 0;
    while (start < n) {
        const int64_t len = start + chunk <= n ? chunk : n - start;
        Slot &sl = slot[cur];
        MCE_TRY(deliver(sl));   // this buffer's previous list has reached the sink
        oc.subset = ids.as<int32_t>() + start;
        oc.subset_len = len;
        oc.list_off = sl.off.as<int64_t>();
        oc.list_vtx = sl.vtx.as<int32_t>();
        oc.list_max_cliques = max_cl;
        oc.list_max_words = buf_words;
        mce_result r;
        memset(&r, 0, sizeof(r));
        mce_status st = enumerate(g, &oc, &r, nullptr, nullptr, 0, nullptr, nullptr);
        const bool list_full = r.list_cliques > max_cl || r.list_words > buf_words;
        if (st == MCE_EOVERFLOW && list_full) {
            if (len == 1) {
                g_last_error = "mce_enumerate_stream: one subproblem's cliques exceed the buffer";
                return MCE_EOVERFLOW;
            }
            chunk = len / 2;   // run the first half again
            continue;
        }
        if (st != MCE_OK && st != MCE_EBUDGET) return st;
        add_result(res, r);
        if (!r.complete) res->complete = 0;
        // copy the list out on the copy stream, after the search that wrote it
        sl.n_cliques = r.list_cliques;
        sl.n_words = r.list_words;
        MCE_CUDA(cudaEventRecord(sl.copied, s));
        MCE_CUDA(cudaStreamWaitEvent(cs, sl.copied, 0));
        if (sl.n_cliques) {
            MCE_CUDA(cudaMemcpyAsync(sl.hoff.p, sl.off.p, (size_t)sl.n_cliques * 8, cudaMemcpyDeviceToHost, cs));
            MCE_CUDA(cudaMemcpyAsync(sl.hvtx.p, sl.vtx.p, (size_t)sl.n_words * 4, cudaMemcpyDeviceToHost, cs));
        }
        MCE_CUDA(cudaEventRecord(sl.copied, cs));
        sl.pending = true;
        start += len;
        // grow while the list used less than a quarter of the buffer
        if (r.list_words * 4 < buf_words && r.list_cliques * 4 < max_cl) chunk = chunk * 2;
        cur ^= 1;
    }
    MCE_TRY(deliver(slot[cur]));
    MCE_TRY(deliver(slot[cur ^ 1]));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    res->ms_rank = ms;
    return res->complete ? MCE_OK : MCE_EBUDGET;
}
