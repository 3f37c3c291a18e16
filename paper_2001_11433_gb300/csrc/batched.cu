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
