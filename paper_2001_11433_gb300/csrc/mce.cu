// Static MCE: ParMCE (Algorithm 5) over all vertices.
//
//   1. rank (Section 4.2 keys or a given rank) and Γ+ lists;
//   2. prepass: isolated vertices are maximal cliques {v} (Algorithm 1 with
//      cand = fini = ∅); a vertex with no higher-ranked neighbour but some
//      lower-ranked one has an empty subproblem; the rest are scheduled;
//   3. order the subproblems, heaviest expected first (|Γ+(v)|^2 + 64 deg v:
//      the search and the build, whose scan of the neighbourhood makes hubs
//      with few candidates expensive too; or a learned cost), and run the
//      persistent search kernel.
#include "bk.cuh"
#include "mce_host.h"

namespace mce {

namespace {


__global__ void k_mce_prepass(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ up_ptr, int32_t n,
                              int32_t idb, uint64_t seed, const float *cost, unsigned long long *out,
                              unsigned long long *pv_count, unsigned long long *pv_hash,
                              unsigned long long *pv_nodes, int32_t *flag, uint64_t *keys,
                              unsigned long long *req_max, const int32_t *graph_of, unsigned long long *g_count,
                              unsigned long long *g_hash, int64_t *list_off, int32_t *list_vtx,
                              int64_t list_max_cliques, int64_t list_max_words, const uint8_t *in_subset) {
    unsigned long long cnt = 0, hsh = 0, nodes = 0, req = 0, cmax = 0, shw = 0, prv = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        if (in_subset && !in_subset[v]) {
            flag[v] = 0;
            continue;
        }
        const int32_t w = row_ptr[v + 1] - row_ptr[v];
        const int32_t c = up_ptr[v + 1] - up_ptr[v];
        int32_t f = 0;
        if (w == 0) {
            const uint64_t h = clique_hash_from_sum(vertex_hash((int32_t)v, seed), 1);
            cnt++;
            hsh += h;
            nodes++;
            if (pv_count) {
                pv_count[v] = 1;
                pv_hash[v] = h;
                pv_nodes[v] = 1;
            }
            if (g_count) {
                atomicAdd(&g_count[graph_of[v]], 1ULL);
                atomicAdd(&g_hash[graph_of[v]], (unsigned long long)h);
            }
            if (list_off) {
                const unsigned long long idx = atomicAdd(&out[OUT_LIST_CLIQUES], 1ULL);
                const unsigned long long pos = atomicAdd(&out[OUT_LIST_WORDS], 2ULL);
                if ((int64_t)idx < list_max_cliques && (int64_t)pos + 2 <= list_max_words) {
                    list_off[idx] = (int64_t)pos;
                    list_vtx[pos] = 1;
                    list_vtx[pos + 1] = (int32_t)v;
                } else {
                    atomicOr(&out[OUT_FLAGS], 1ULL);
                }
            }
        } else if (c == 0) {
            nodes++;
            if (pv_count) pv_nodes[v] = 1;
        } else {
            f = 1;
            uint64_t k;
            if (cost) {
                // descending predicted cost: invert the order-preserving float map
                uint32_t b = __float_as_uint(cost[v]);
                b ^= (b >> 31) ? 0xffffffffu : 0x80000000u;
                k = ((uint64_t)(~b) << idb) | (uint64_t)v;
            } else {
                // expected cost: the search grows with c^2 at least, the build
                // with the neighbourhood (each of the w local vertices is scanned)
                const uint64_t est = (uint64_t)c * (uint64_t)c + 64ULL * (uint64_t)w;
                const uint64_t cap = (1ULL << (63 - idb)) - 1;
                k = ((cap - (est < cap ? est : cap)) << idb) | (uint64_t)v;
            }
            keys[v] = k;
            req = max(req, (unsigned long long)bk_ws_words(w, c, BK_MCE));
            cmax = max(cmax, (unsigned long long)c);
            shw += (unsigned long long)bk_shared_words(w, c);
            prv = max(prv, (unsigned long long)bk_private_words(w, c, BK_MCE));
        }
        flag[v] = f;
    }
    for (int o = 16; o; o >>= 1) {
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        hsh += __shfl_xor_sync(0xffffffffu, hsh, o);
        nodes += __shfl_xor_sync(0xffffffffu, nodes, o);
        req = max(req, __shfl_xor_sync(0xffffffffu, req, o));
        cmax = max(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
        shw += __shfl_xor_sync(0xffffffffu, shw, o);
        prv = max(prv, __shfl_xor_sync(0xffffffffu, prv, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (cnt) {
            atomicAdd(&out[OUT_COUNT], cnt);
            atomicAdd(&out[OUT_HASH], hsh);
            atomicAdd(&out[OUT_HIST + 1], cnt);
            atomicMax(&out[OUT_MAXSIZE], 1ULL);
        }
        if (nodes) atomicAdd(&out[OUT_NODES], nodes);
        if (req) atomicMax(req_max, req);
        if (cmax) atomicMax(req_max + 1, cmax);
        if (shw) atomicAdd(req_max + 2, shw);
        if (prv) atomicMax(req_max + 3, prv);
    }
}

__global__ void k_subset_mask(const int32_t *subset, int64_t m, int32_t n, uint8_t *mask, int32_t *bad) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = subset[i];
        if (v < 0 || v >= n) atomicOr(bad, 1);
        else mask[v] = 1;
    }
}

__global__ void k_count_over(const unsigned long long *nodes, int32_t n, uint64_t budget, unsigned long long *cnt) {
    unsigned long long c = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        c += nodes[v] > budget;
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, c);
}

__global__ void k_gather_active(const int32_t *flag_scan, const uint64_t *keys, int32_t n, uint64_t *out) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        if (flag_scan[v + 1] != flag_scan[v]) out[flag_scan[v]] = keys[v];
}

__global__ void k_order_from_keys(const uint64_t *keys, int32_t m, int32_t idb, int32_t *order) {
    const uint64_t mask = (1ULL << idb) - 1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        order[i] = (int32_t)(keys[i] & mask);
}

__global__ void k_set_u64(unsigned long long *p, unsigned long long v) { *p = v; }

// heavy[v] = 1 when the predicted log(1 + tree nodes) reaches thr
__global__ void k_heavy_flags(const float *cost, int32_t n, float thr, uint8_t *heavy) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        heavy[v] = cost[v] >= thr ? 1 : 0;
}

// Whole-graph TTT (Algorithm 3 from K = ∅, cand = V): the root's pivot is a
// vertex of largest degree (|V ∩ Γ(u)| = deg u), smallest id among ties.
__global__ void k_whole_pivot(const int32_t *row_ptr, int32_t n, unsigned long long *best) {
    unsigned long long b = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = ((unsigned long long)(row_ptr[v + 1] - row_ptr[v]) << 32) |
                                     (unsigned long long)(0x7fffffffu - (uint32_t)v);
        b = max(b, k);
    }
    for (int o = 16; o; o >>= 1) b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
    if ((threadIdx.x & 31) == 0) atomicMax(best, b);
}

// key(v) = 1 for the neighbours of the pivot, else 0 (the root's ext, which
// holds the pivot itself); in_ext[v] = 1 - key(v).  k_whole_init, then
// k_whole_mark over the pivot's row.
__global__ void k_whole_init(int32_t n, int64_t *key, uint8_t *in_ext) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        key[v] = 0;
        in_ext[v] = 1;
    }
}

__global__ void k_whole_mark(const int32_t *row_ptr, const int32_t *col, const unsigned long long *best, int64_t *key,
                             uint8_t *in_ext) {
    const int32_t p = (int32_t)(0x7fffffffu - (uint32_t)(*best & 0xffffffffULL));
    for (int32_t e = row_ptr[p] + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x); e < row_ptr[p + 1];
         e += (int32_t)(gridDim.x * blockDim.x)) {
        key[col[e]] = 1;
        in_ext[col[e]] = 0;
    }
}

struct EvPair {
    cudaEvent_t a, b;
    ~EvPair() {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
};

}  // namespace

mce_status launch_prepass(const mce_graph *g, const int32_t *up_ptr, uint64_t seed, const float *cost,
                          unsigned long long *out, int32_t *flag, uint64_t *keys, unsigned long long *reqc,
                          const int32_t *graph_of, unsigned long long *g_count, unsigned long long *g_hash,
                          cudaStream_t s) {
    if (g->n == 0) return MCE_OK;
    MCE_LAUNCH(k_mce_prepass, grid_for(g->n, 256), 256, 0, s, g->row_ptr, up_ptr, g->n, g->id_bits, seed, cost, out,
               (unsigned long long *)nullptr, (unsigned long long *)nullptr, (unsigned long long *)nullptr, flag, keys,
               reqc, graph_of, g_count, g_hash, (int64_t *)nullptr, (int32_t *)nullptr, (int64_t)0, (int64_t)0,
               (const uint8_t *)nullptr);
    return MCE_OK;
}

mce_status launch_order(const int32_t *flag_scan, const uint64_t *keys, int32_t n, int32_t n_act, int32_t idb,
                        uint64_t *tmp2, int32_t *order, cudaStream_t s) {
    uint64_t *act = tmp2, *act_tmp = tmp2 + n_act;
    MCE_LAUNCH(k_gather_active, grid_for(n, 256), 256, 0, s, flag_scan, keys, n, act);
    MCE_TRY(radix_sort_u64(act, act_tmp, n_act, 64, s));
    MCE_LAUNCH(k_order_from_keys, grid_for(n_act, 256), 256, 0, s, act, n_act, idb, order);
    return MCE_OK;
}

LaunchShape launch_shape(const mce_opts *o) {
    LaunchShape ls;
    ls.warps_per_block = (o && o->warps_per_block > 0) ? o->warps_per_block : 8;
    if (ls.warps_per_block > 8) ls.warps_per_block = 8;
    // measured on GB300: two resident blocks of eight warps (128 registers)
    // are the robust choice (Chung-Lu, incremental, sampled R-MAT sets); three
    // (80 registers) win about 10 % on the full R-MAT 18 set only
    ls.blocks_per_sm = (o && o->blocks_per_sm > 0) ? o->blocks_per_sm : 2;
    // shared memory per SM is 228 KB with 1 KB reserved per block; the search
    // kernel also has about 1 KB of static shared memory
    const int64_t per_block = (int64_t)228 * 1024 / ls.blocks_per_sm - 2048;
    int64_t words = (per_block - 2048) / 4 / ls.warps_per_block - BK_PIV_WORDS;
    words &= ~int64_t(3);
    if (words < 0) words = 0;
    // Measured on GB300: the per-warp workspaces hit L1 more often when no
    // shared memory is carved out for them, so slots are opt-in.
    if (!o || o->shared_words <= 0) words = 0;
    else if (o->shared_words < words) words = o->shared_words & ~3;
    ls.smem_words = (int32_t)words;
    // what is left of the block's shared memory goes to the lane-parallel small
    // search, up to 8 KB a warp (below 2 KB a warp it stays off).  Measured on
    // GB300: larger arenas take shared memory from L1, which the lane search's
    // node stacks and the subproblem rows need more (R-MAT 18 and Chung-Lu
    // searches 5-14 % faster at 8 KB than at 12 KB).
    if (!o || !o->warp_small_search) {
        int64_t lp = (per_block - 2048) / 4 / ls.warps_per_block - BK_PIV_WORDS - ls.smem_words;
        if (lp > 2048) lp = 2048;
        if (o && o->lane_search_words > 0 && o->lane_search_words < lp) lp = o->lane_search_words;
        lp &= ~int64_t(1);
        ls.lp_words = lp >= 512 ? (int32_t)lp : 0;
    }
    // the ring's sequence numbers tell "published for ticket p" (p + 1) from
    // "free for ticket p + cap" (p + cap) only when cap >= 2
    ls.queue_capacity = (o && o->queue_capacity > 0) ? (o->queue_capacity < 2 ? 2 : o->queue_capacity) : 0;
    return ls;
}

mce_status alloc_lp_tasks(BkParams &P, int64_t nwarps, cudaStream_t s, BkBuffers &b) {
    if (P.mode != BK_MCE || P.lp_words == 0) {
        P.lp_words = 0;
        P.lp_tasks = nullptr;
        P.lp_task_cap = 0;
        return MCE_OK;
    }
    P.lp_task_cap = BK_LP_TASK_CAP;
    MCE_TRY(b.lp_tasks.alloc((size_t)nwarps * BK_LP_TASK_CAP * BK_LP_TASK_WORDS * 4, s));
    P.lp_tasks = b.lp_tasks.as<uint32_t>();
    return MCE_OK;
}

mce_status run_bk(BkParams &P, const LaunchShape &ls, int64_t req_max, int64_t cmax, cudaStream_t s, BkBuffers &b) {
    const int64_t nwarps = (int64_t)num_sms() * ls.blocks_per_sm * ls.warps_per_block;
    P.gws_words = req_max > ls.smem_words ? req_max : 16;
    P.smem_words = ls.smem_words;
    P.lp_words = ls.lp_words;
    MCE_TRY(alloc_lp_tasks(P, nwarps, s, b));
    MCE_TRY(b.gws.alloc((size_t)nwarps * P.gws_words * 4, s));
    P.gws = b.gws.as<uint32_t>();
    // one ring slot holds (root, depth, path <= c, cand, finic, ext, conf)
    const int64_t wcmax = (cmax + 31) / 32;
    P.slot_words = (2 + cmax + 4 * wcmax + 3) & ~int64_t(3);
    int64_t cap = ((int64_t)1 << 26) / P.slot_words;
    if (cap > ((int64_t)1 << 16)) cap = (int64_t)1 << 16;
    if (cap < 1024) cap = 1024;
    if (ls.queue_capacity > 0) cap = ls.queue_capacity;
    P.qcap = cap;
    MCE_TRY(b.arena.alloc((size_t)P.qcap * P.slot_words * 4, s));
    MCE_TRY(b.qseq.alloc((size_t)P.qcap * 8, s));
    MCE_TRY(b.taskbuf.alloc((size_t)nwarps * P.slot_words * 4, s));
    MCE_TRY(init_queue_seq(b.qseq.as<unsigned long long>(), P.qcap, s));
    MCE_TRY(b.ctl.alloc(CTL_WORDS * sizeof(unsigned long long), s));
    MCE_CUDA(cudaMemsetAsync(b.ctl.p, 0, CTL_WORDS * sizeof(unsigned long long), s));
    P.arena = b.arena.as<uint32_t>();
    P.qseq = b.qseq.as<unsigned long long>();
    P.taskbuf = b.taskbuf.as<uint32_t>();
    P.ctl = b.ctl.as<unsigned long long>();
    MCE_LAUNCH(k_set_u64, 1, 1, 0, s, P.ctl + CTL_PENDING, (unsigned long long)P.n_sub);
    if (P.timeout_ns == 0) P.timeout_ns = 60ULL * 1000000000ULL;
    if (P.max_run_ns == 0) P.max_run_ns = 600ULL * 1000000000ULL;
    return launch_bk(P, ls.warps_per_block, ls.blocks_per_sm, s);
}

mce_status compute_rank(const mce_graph *g, const mce_opts *o, cudaStream_t s, int32_t *rank) {
    const int32_t n = g->n;
    if (n == 0) return MCE_OK;
    switch (o->rank_kind) {
        case MCE_RANK_USER:
            if (!o->user_rank) {
                g_last_error = "MCE_RANK_USER without user_rank";
                return MCE_EINVAL;
            }
            MCE_CUDA(cudaMemcpyAsync(rank, o->user_rank, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
            return MCE_OK;
        case MCE_RANK_LEARNED: {
            if (!o->model) {
                g_last_error = "MCE_RANK_LEARNED without a model";
                return MCE_EINVAL;
            }
            DevBuf feat, score;
            MCE_TRY(feat.alloc((size_t)n * 8 * 4, s));
            MCE_TRY(score.alloc((size_t)n * 4, s));
            MCE_TRY(features(g, model_feature_kind(o->model), s, feat.as<float>()));
            MCE_TRY(model_predict(o->model, feat.as<float>(), n, 1, s, score.as<float>()));
            return rank_from_key_f32(score.as<float>(), n, g->id_bits, s, rank);
        }
        case MCE_RANK_DEGREE:
        case MCE_RANK_DEGEN:
        case MCE_RANK_TRIANGLE: {
            DevBuf key;
            MCE_TRY(key.alloc((size_t)n * 8, s));
            MCE_TRY(vertex_key(g, o->rank_kind, s, key.as<int64_t>()));
            return rank_from_key_i64(key.as<int64_t>(), n, g->id_bits, s, rank);
        }
        default:
            g_last_error = "unknown rank kind";
            return MCE_EINVAL;
    }
}

mce_status read_result(const DevBuf &out, const DevBuf &ctl, cudaStream_t s, mce_result *res) {
    static_assert(OUT_WORDS * 8 < 16384, "output block");
    unsigned long long h[OUT_WORDS];
    unsigned long long c[CTL_WORDS];
    MCE_CUDA(cudaMemcpyAsync(h, out.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    if (ctl.p) MCE_CUDA(cudaMemcpyAsync(c, ctl.p, sizeof(c), cudaMemcpyDeviceToHost, s));
    else for (int i = 0; i < CTL_WORDS; ++i) c[i] = 0;
    MCE_CUDA(cudaStreamSynchronize(s));
    res->count = h[OUT_COUNT];
    res->hash = h[OUT_HASH];
    res->tree_nodes = h[OUT_NODES];
    res->hist_len = (int32_t)(h[OUT_MAXSIZE] ? h[OUT_MAXSIZE] + 1 : 0);
    if (res->hist_len > MCE_HIST_CAP) res->hist_len = MCE_HIST_CAP;
    for (int i = 0; i < MCE_HIST_CAP; ++i) res->hist[i] = i < res->hist_len ? h[OUT_HIST + i] : 0;
    res->list_cliques = (int64_t)h[OUT_LIST_CLIQUES];
    res->list_words = (int64_t)h[OUT_LIST_WORDS];
    res->tasks_split = h[OUT_SPLITS];
    res->word_ops = h[OUT_WORDOPS];
    for (int i = 0; i < 7; ++i) res->stats[i] = h[OUT_BUILD_NS + i];
    res->stats[7] = (c[CTL_T_END] > c[CTL_T_LAST] && c[CTL_T_LAST]) ? c[CTL_T_END] - c[CTL_T_LAST] : 0;
    res->complete = (c[CTL_ABORT] & 3ULL) ? 0 : 1;
    if (c[CTL_ABORT] & 4ULL) {
        g_last_error = "search workspace smaller than a subproblem";
        return MCE_ESTATE;
    }
    if (c[CTL_ABORT] & 2ULL) {
        g_last_error = "a bounded device wait gave up";
        return MCE_ETIMEOUT;
    }
    if (c[CTL_ABORT] & 1ULL) return MCE_EBUDGET;
    if (h[OUT_FLAGS] & 1ULL) return MCE_EOVERFLOW;
    if (h[OUT_FLAGS] & 2ULL) {
        g_last_error = "clique larger than the histogram";
        return MCE_EOVERFLOW;
    }
    return MCE_OK;
}

mce_status enumerate(const mce_graph *g, const mce_opts *o, mce_result *res, const int32_t *graph_of,
                     unsigned long long *graph_nodes, uint64_t graph_budget, unsigned long long *g_count,
                     unsigned long long *g_hash) {
    cudaStream_t s = (cudaStream_t)o->stream;
    const int32_t n = g->n;
    const int32_t idb = g->id_bits;
    cudaEvent_t e0, e1, e2;
    MCE_CUDA(cudaEventCreate(&e0));
    MCE_CUDA(cudaEventCreate(&e1));
    MCE_CUDA(cudaEventCreate(&e2));
    struct EvGuard {
        cudaEvent_t a, b, c;
        ~EvGuard() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
            cudaEventDestroy(c);
        }
    } evg{e0, e1, e2};
    MCE_CUDA(cudaEventRecord(e0, s));
    DevBuf rank, out, up_ptr, up_col, flag, keys, tmp, order, cost, wmask;
    MCE_TRY(rank.alloc((size_t)(n + 1) * 4, s));
    if (o->whole_graph) {
        // Algorithm 3 from K = ∅, cand = V: the root (pivot p of largest degree)
        // has the children q ∈ ext = V \ Γ(p), in increasing id; child q is
        // TTT({q}, Γ(q) minus the earlier ext vertices, Γ(q) ∩ earlier ext),
        // which is the subproblem of q (Algorithm 5) under the rank that puts
        // ext first (by id) and Γ(p) after it (by id).  Every maximal clique
        // has a vertex in ext (else p would extend it).
        if (n > 0) {
            DevBuf best, wkey;
            MCE_TRY(best.alloc(8, s));
            MCE_TRY(wkey.alloc((size_t)n * 8, s));
            MCE_TRY(wmask.alloc((size_t)n + 16, s));
            MCE_CUDA(cudaMemsetAsync(best.p, 0, 8, s));
            MCE_LAUNCH(k_whole_pivot, grid_for(n, 256), 256, 0, s, g->row_ptr, n, best.as<unsigned long long>());
            MCE_LAUNCH(k_whole_init, grid_for(n, 256), 256, 0, s, n, wkey.as<int64_t>(), wmask.as<uint8_t>());
            MCE_LAUNCH(k_whole_mark, 64, 256, 0, s, g->row_ptr, g->col, best.as<unsigned long long>(),
                       wkey.as<int64_t>(), wmask.as<uint8_t>());
            MCE_TRY(rank_from_key_i64(wkey.as<int64_t>(), n, g->id_bits, s, rank.as<int32_t>()));
        }
    } else {
        MCE_TRY(compute_rank(g, o, s, rank.as<int32_t>()));
    }
    MCE_CUDA(cudaEventRecord(e1, s));
    int64_t up_nnz = 0;
    MCE_TRY(build_up_lists(g, rank.as<int32_t>(), s, up_ptr, up_col, &up_nnz));
    const float *costp = nullptr;
    const mce_model *cost_model = o->split_model ? o->split_model : (o->order_by_model ? o->model : nullptr);
    DevBuf heavy;
    if (cost_model && n > 0) {
        DevBuf feat;
        MCE_TRY(feat.alloc((size_t)n * 8 * 4 + 16, s));
        MCE_TRY(cost.alloc((size_t)n * 4 + 16, s));
        MCE_TRY(features(g, model_feature_kind(cost_model), s, feat.as<float>()));
        MCE_TRY(model_predict(cost_model, feat.as<float>(), n, 1, s, cost.as<float>()));
        if (o->order_by_model) costp = cost.as<float>();
        if (o->split_model) {
            MCE_TRY(heavy.alloc((size_t)n + 16, s));
            const float thr = logf(1.0f + (float)(o->heavy_nodes ? o->heavy_nodes : 65536u));
            MCE_LAUNCH(k_heavy_flags, grid_for(n, 256), 256, 0, s, cost.as<float>(), n, thr, heavy.as<uint8_t>());
        }
    }
    MCE_TRY(out.alloc(OUT_WORDS * 8, s));
    MCE_CUDA(cudaMemsetAsync(out.p, 0, OUT_WORDS * 8, s));
    MCE_TRY(flag.alloc((size_t)(n + 1) * 4, s));
    MCE_TRY(keys.alloc((size_t)(n + 1) * 8, s));
    DevBuf reqb, mask;
    MCE_TRY(reqb.alloc(32, s));
    MCE_CUDA(cudaMemsetAsync(reqb.p, 0, 32, s));
    const uint8_t *maskp = nullptr;
    DevBuf hsub;
    const int32_t *subp = o->subset;
    if (o->subset && o->subset_on_host && o->subset_len > 0) {
        MCE_TRY(hsub.alloc((size_t)o->subset_len * 4, s));
        MCE_CUDA(cudaMemcpyAsync(hsub.p, o->subset, (size_t)o->subset_len * 4, cudaMemcpyHostToDevice, s));
        subp = hsub.as<int32_t>();
    }
    if (o->whole_graph) {
        maskp = wmask.as<uint8_t>();
    } else if (o->subset) {
        DevBuf bad;
        MCE_TRY(bad.alloc(4, s));
        MCE_TRY(mask.alloc((size_t)n + 16, s));
        MCE_CUDA(cudaMemsetAsync(mask.p, 0, (size_t)n + 16, s));
        MCE_CUDA(cudaMemsetAsync(bad.p, 0, 4, s));
        if (o->subset_len > 0)
            MCE_LAUNCH(k_subset_mask, grid_for(o->subset_len, 256), 256, 0, s, subp, o->subset_len, n,
                       mask.as<uint8_t>(), bad.as<int32_t>());
        int32_t hb = 0;
        MCE_CUDA(cudaMemcpyAsync(&hb, bad.p, 4, cudaMemcpyDeviceToHost, s));
        MCE_CUDA(cudaStreamSynchronize(s));
        if (hb) {
            g_last_error = "mce_enumerate: subset holds an id outside [0, n)";
            return MCE_EINVAL;
        }
        maskp = mask.as<uint8_t>();
    }
    if (o->pv_count) {
        MCE_CUDA(cudaMemsetAsync(o->pv_count, 0, (size_t)n * 8, s));
        MCE_CUDA(cudaMemsetAsync(o->pv_hash, 0, (size_t)n * 8, s));
        MCE_CUDA(cudaMemsetAsync(o->pv_nodes, 0, (size_t)n * 8, s));
    }
    if (n > 0)
        MCE_LAUNCH(k_mce_prepass, grid_for(n, 256), 256, 0, s, g->row_ptr, up_ptr.as<int32_t>(), n, idb, o->hash_seed,
                   costp, out.as<unsigned long long>(), (unsigned long long *)o->pv_count,
                   (unsigned long long *)o->pv_hash, (unsigned long long *)o->pv_nodes, flag.as<int32_t>(),
                   keys.as<uint64_t>(), reqb.as<unsigned long long>(), graph_of, g_count, g_hash, o->list_off,
                   o->list_vtx, o->list_max_cliques, o->list_max_words, maskp);
    MCE_TRY(exclusive_scan_i32(flag.as<int32_t>(), flag.as<int32_t>(), n, s));
    int32_t n_act = 0;
    unsigned long long reqc[4] = {0, 0, 0, 0};
    MCE_CUDA(cudaMemcpyAsync(&n_act, flag.as<int32_t>() + n, 4, cudaMemcpyDeviceToHost, s));
    MCE_CUDA(cudaMemcpyAsync(reqc, reqb.p, 32, cudaMemcpyDeviceToHost, s));
    MCE_CUDA(cudaStreamSynchronize(s));
    res->subproblems = n_act;
    BkBuffers bb;
    DevBuf subn;
    if (n_act > 0) {
        MCE_TRY(tmp.alloc((size_t)n_act * 8 * 2, s));
        MCE_TRY(order.alloc((size_t)n_act * 4, s));
        uint64_t *act = tmp.as<uint64_t>(), *act_tmp = act + n_act;
        MCE_LAUNCH(k_gather_active, grid_for(n, 256), 256, 0, s, flag.as<int32_t>(), keys.as<uint64_t>(), n, act);
        MCE_TRY(radix_sort_u64(act, act_tmp, n_act, 64, s));
        MCE_LAUNCH(k_order_from_keys, grid_for(n_act, 256), 256, 0, s, act, n_act, idb, order.as<int32_t>());
        BkParams P{};
        P.mode = BK_MCE;
        P.row_ptr = g->row_ptr;
        P.col = g->col;
        P.up_ptr = up_ptr.as<int32_t>();
        P.up_col = up_col.as<int32_t>();
        P.rank = rank.as<int32_t>();
        P.order = order.as<int32_t>();
        P.n_sub = n_act;
        P.graph_of = graph_of;
        P.graph_nodes = graph_nodes;
        P.graph_budget = graph_budget;
        P.g_count = g_count;
        P.g_hash = g_hash;
        P.seed = o->hash_seed;
        P.out = out.as<unsigned long long>();
        P.list_off = o->list_off;
        P.list_vtx = o->list_vtx;
        P.list_max_cliques = o->list_max_cliques;
        P.list_max_words = o->list_max_words;
        P.pv_count = (unsigned long long *)o->pv_count;
        P.pv_hash = (unsigned long long *)o->pv_hash;
        P.pv_nodes = (unsigned long long *)o->pv_nodes;
        P.node_budget = o->node_budget;
        if (o->subproblem_budget) {
            MCE_TRY(subn.alloc((size_t)n * 8, s));
            MCE_CUDA(cudaMemsetAsync(subn.p, 0, (size_t)n * 8, s));
            P.sub_nodes = subn.as<unsigned long long>();
            P.sub_budget = o->subproblem_budget;
        }
        P.split = o->split;
        // measured on GB300 with the lane search: 4,096 keeps every rank of the
        // Chung-Lu graph balanced (12,288 costs the learned rank 18 %), while
        // the R-MAT 18 benchmark set is fastest at 12,288, which it asks for
        P.split_nodes = o->split ? (o->split_nodes ? o->split_nodes : 4096u) : 0u;
        P.sm_limit = o->sm_limit;
        P.lp_hold_waiting = o->lane_hold_waiting;
        if (heavy.p && o->split) {
            P.heavy = heavy.as<uint8_t>();
            P.heavy_split_nodes = o->heavy_split_nodes ? o->heavy_split_nodes : 256u;
        }
        P.max_run_ns = (uint64_t)o->time_limit_ms * 1000000ULL;
        // build cache for every subproblem (up to 2^30 words); when it holds them
        // all, a warp's own workspace only needs the private search state
        DevBuf cache, coff;
        const int64_t cw = (int64_t)reqc[2] < ((int64_t)1 << 30) ? (int64_t)reqc[2] : ((int64_t)1 << 30);
        int64_t per_warp = (int64_t)reqc[0];
        if (cw == (int64_t)reqc[2]) per_warp = (int64_t)reqc[3];
        else if (per_warp > ((int64_t)1 << 24)) per_warp = (int64_t)reqc[3] > ((int64_t)1 << 24) ? (int64_t)reqc[3]
                                                                                                 : ((int64_t)1 << 24);
        if (cw > 0) {
            MCE_TRY(cache.alloc((size_t)cw * 4 + 512, s));
            MCE_TRY(coff.alloc((size_t)n * 8, s));
            MCE_CUDA(cudaMemsetAsync(coff.p, 0xff, (size_t)n * 8, s));
            // 128-byte aligned start
            P.cache = reinterpret_cast<uint32_t *>(((uintptr_t)cache.p + 127) & ~(uintptr_t)127);
            P.cache_words = cw;
            P.cache_off = coff.as<long long>();
        }
        const LaunchShape ls = launch_shape(o);
        cudaEvent_t k0, k1;
        MCE_CUDA(cudaEventCreate(&k0));
        MCE_CUDA(cudaEventCreate(&k1));
        EvPair kg{k0, k1};
        MCE_CUDA(cudaEventRecord(k0, s));
        MCE_TRY(run_bk(P, ls, per_warp, (int64_t)reqc[1], s, bb));
        MCE_CUDA(cudaEventRecord(k1, s));
        MCE_CUDA(cudaEventSynchronize(k1));
        float ks = 0;
        cudaEventElapsedTime(&ks, k0, k1);
        res->ms_search = ks;
    }
    MCE_CUDA(cudaEventRecord(e2, s));
    if (subn.p) {
        DevBuf cnt;
        MCE_TRY(cnt.alloc(8, s));
        MCE_CUDA(cudaMemsetAsync(cnt.p, 0, 8, s));
        MCE_LAUNCH(k_count_over, grid_for(n, 256), 256, 0, s, subn.as<unsigned long long>(), n, o->subproblem_budget,
                   cnt.as<unsigned long long>());
        unsigned long long hc = 0;
        MCE_CUDA(cudaMemcpyAsync(&hc, cnt.p, 8, cudaMemcpyDeviceToHost, s));
        MCE_CUDA(cudaStreamSynchronize(s));
        res->incomplete = (int64_t)hc;
    }
    mce_status st = read_result(out, bb.ctl, s, res);
    if (o->whole_graph && n > 0) res->tree_nodes += 1;   // the root node of the whole-graph tree
    float a = 0, b = 0;
    cudaEventElapsedTime(&a, e0, e1);
    cudaEventElapsedTime(&b, e1, e2);
    res->ms_rank = a;
    res->ms_enum = b;
    return st;
}

}  // namespace mce
