// Host-side declarations shared by the orchestration files.
#pragma once

#include "bk.cuh"

namespace mce {

struct LaunchShape {
    int32_t warps_per_block = 8;
    int32_t blocks_per_sm = 4;
    int32_t smem_words = 0;
    int32_t queue_capacity = 0;   // task ring slots (0 = automatic)
    int32_t lp_words = 0;         // per-warp shared words of the lane-parallel small search (0 = off)
};

LaunchShape launch_shape(const mce_opts *o);
struct BkBuffers {
    DevBuf gws, arena, qseq, taskbuf, ctl, lp_tasks;
};
// task lists of the lane-parallel small search (static MCE only)
mce_status alloc_lp_tasks(BkParams &P, int64_t nwarps, cudaStream_t s, BkBuffers &b);
mce_status run_bk(BkParams &P, const LaunchShape &ls, int64_t req_max, int64_t cmax, cudaStream_t s, BkBuffers &b);
mce_status compute_rank(const mce_graph *g, const mce_opts *o, cudaStream_t s, int32_t *rank);
mce_status read_result(const DevBuf &out, const DevBuf &ctl, cudaStream_t s, mce_result *res);
mce_status enumerate(const mce_graph *g, const mce_opts *o, mce_result *res, const int32_t *graph_of,
                     unsigned long long *graph_nodes, uint64_t graph_budget, unsigned long long *g_count,
                     unsigned long long *g_hash);
// prepass of the per-vertex decomposition (trivial subproblems, sizes, order keys)
mce_status launch_prepass(const mce_graph *g, const int32_t *up_ptr, uint64_t seed, const float *cost,
                          unsigned long long *out, int32_t *flag, uint64_t *keys, unsigned long long *reqc,
                          const int32_t *graph_of, unsigned long long *g_count, unsigned long long *g_hash,
                          cudaStream_t s);
// order of the non-trivial subproblems from the scanned flags and their keys
mce_status launch_order(const int32_t *flag_scan, const uint64_t *keys, int32_t n, int32_t n_act, int32_t idb,
                        uint64_t *tmp2, int32_t *order, cudaStream_t s);
// validate a graph built from a caller CSR (graph.cu)
mce_status check_csr(const mce_graph *g, cudaStream_t s);
// move an incremental state to another stream between batches (imce.cu)
void imce_set_stream(imce_state *S, cudaStream_t s);
// learned cost model (mlp.cu)
mce_status model_predict(const mce_model *m, const float *feat, int32_t rows, int32_t bf16, cudaStream_t s,
                         float *out);

}  // namespace mce
