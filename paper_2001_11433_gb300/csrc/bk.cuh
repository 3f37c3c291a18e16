// Persistent warp-cooperative Bron-Kerbosch engine (shared by static and
// incremental enumeration).
#pragma once

#include "internal.cuh"

namespace mce {

// Control block of one persistent launch (uint64 words).  Each word sits on
// its own 128-byte line: idle warps hammer the queue head while busy warps
// poll the others.
enum CtlWord {
    CTL_NEXT = 0 * 16,       // next unclaimed subproblem index
    CTL_QTAIL = 1 * 16,      // ring tickets taken by pushers
    CTL_QHEAD = 2 * 16,      // ring tickets taken by poppers
    CTL_PENDING = 3 * 16,    // subproblems + queued tasks not finished
    CTL_HUNGRY = 4 * 16,     // warps waiting for work
    CTL_CACHE_TOP = 5 * 16,  // words of the build cache in use
    CTL_NODES = 6 * 16,      // tree nodes, for the budget
    CTL_ABORT = 7 * 16,      // 1 = budget, 2 = timeout, 4 = workspace too small, 8 = bad task
    CTL_T_LAST = 8 * 16,     // globaltimer when the last subproblem was claimed
    CTL_T_END = 9 * 16,      // latest globaltimer at which a warp left the launch
    CTL_WORDS = 10 * 16
};

// Output block (uint64 words); the size histogram follows at OUT_HIST.
enum OutWord {
    OUT_COUNT = 0,
    OUT_HASH = 1,
    OUT_NODES = 2,
    OUT_MAXSIZE = 3,
    OUT_LIST_CLIQUES = 4,
    OUT_LIST_WORDS = 5,
    OUT_FLAGS = 6,     // 1 = list overflow, 2 = histogram overflow
    OUT_SPLITS = 7,
    OUT_WORDOPS = 8,
    OUT_BUILD_NS = 9,      // summed over warps: time building subproblems
    OUT_SEARCH_NS = 10,    //                    time searching
    OUT_IDLE_NS = 11,      //                    time waiting for work
    OUT_BUILDS = 12,       // subproblem builds
    OUT_PIECES = 13,       // handed-over pieces run
    OUT_MAXBUSY_NS = 14,   // largest build + search time of one warp
    OUT_NWARPS = 15,
    OUT_HIST = 16,
    OUT_WORDS = 16 + MCE_HIST_CAP
};

// Mode of a subproblem.
enum BkMode {
    BK_MCE = 0,    // ParMCE subproblem of vertex v (Algorithm 5)
    BK_IMCE = 1    // new cliques of edge e_i (Algorithm 6 with the exclusion of Algorithm 7)
};

struct BkParams {
    int32_t mode;
    // graph
    const int32_t *row_ptr, *col;
    const int32_t *up_ptr, *up_col;   // Γ+ lists (by rank for MCE, by degree rank of G+H for IMCE)
    const int32_t *rank;              // MCE only
    // subproblems
    const int32_t *order;             // MCE: vertices; IMCE: edge indices, in processing order
    int32_t n_sub;
    // IMCE: batch edges e_1..e_rho (arrival order) and the new-edge adjacency
    const int32_t *eu, *ev;
    const int32_t *h_ptr, *h_adj, *h_idx;   // per vertex: new neighbours and edge indices
    const int32_t *graph_of;          // batched MCE: graph id of each vertex (or null)
    unsigned long long *graph_nodes;  // batched MCE: tree nodes per graph
    uint64_t graph_budget;
    uint64_t seed;
    // per-warp workspace
    uint32_t *gws;
    int64_t gws_words;
    int32_t smem_words;
    // task ring: qcap slots of slot_words words, sequence numbers, and one
    // private record buffer per warp
    uint32_t *arena;
    int64_t slot_words;
    unsigned long long *qseq;
    int64_t qcap;
    uint32_t *taskbuf;
    // build cache: the warp that opens a subproblem builds its read-only part
    // here and publishes the offset in cache_off[v]; pieces reuse it
    uint32_t *cache;
    int64_t cache_words;
    long long *cache_off;
    unsigned long long *ctl;
    // outputs
    unsigned long long *out;
    int64_t *list_off;
    int32_t *list_vtx;
    int64_t list_max_cliques, list_max_words;
    unsigned long long *pv_count, *pv_hash, *pv_nodes;   // per subproblem id
    unsigned long long *g_count, *g_hash;                // batched: per graph
    uint64_t node_budget;
    unsigned long long *sub_nodes;    // exact nodes per subproblem (with sub_budget)
    uint64_t sub_budget;
    int32_t split;
    uint32_t split_nodes;     // a task hands over a piece after this many nodes (0 = only when warps wait)
    uint64_t timeout_ns;      // bound on any single wait
    uint64_t max_run_ns;      // bound on a warp's time in one launch
    int32_t lp_words;         // per-warp shared words of the lane-parallel small search (0 = off)
    uint32_t *lp_tasks;       // per warp: a stack of lp_task_cap node records (BK_LP_TASK_WORDS each)
    int32_t lp_task_cap;
    int32_t sm_limit;         // blocks on SMs with %smid >= sm_limit do no work (0 = all SMs work)
    const uint8_t *heavy;     // per vertex: 1 = predicted heavy, splits every heavy_split_nodes (or null)
    uint32_t heavy_split_nodes;
    uint32_t lp_hold_waiting; // waiting warps from which small subtrees stay with the whole warp (0 = never)
};

// Words of the read-only part of a built subproblem with w local vertices of
// which c are candidates: a 32-word header (kept vertices W, kept fini f),
// then local ids, bounds, bitset rows, the bound-sorted fini list F0, and one
// bitset over F0 positions per candidate (its lower-ranked neighbours).
// Rounded to 32 words so that every part starts on a 128-byte line.
// Bitset rows are ⌈c/32⌉ words padded to a multiple of 4, so that every row
// starts on a 16-byte boundary and is read as 16-byte vectors.
__host__ __device__ inline int64_t bk_row_stride(int64_t wc) { return (wc + 3) & ~int64_t(3); }
__host__ __device__ inline int64_t bk_align4(int64_t x) { return (x + 3) & ~int64_t(3); }

__host__ __device__ inline int64_t bk_shared_words(int64_t w, int64_t c) {
    const int64_t wc = (c + 31) / 32;
    const int64_t S = bk_row_stride(wc);
    const int64_t wf = (w - c + 31) / 32;
    const int64_t words = bk_align4(32 + 2 * w) + w * S + (w - c) + c * wf;
    return (words + 31) & ~int64_t(31);
}

// Per-warp shared-memory scratch: the wide pivot's cand (64 words) and
// member list of cand ∪ finic (512 16-bit local ids); in the small search
// the same 320 words hold h(C_k) and the frame stack, and 96 more words the
// global and local ids of C and the local ids of X.
constexpr int BK_PIV_WORDS = 64 + 256 + 96;

// Lane-parallel small search: per warp a table of up to BK_LP_MAX_ROOTS
// relabelled small nodes (4 words each, then the next-root counter) and an
// arena for their universes.
constexpr int BK_LP_MAX_ROOTS = 64;
constexpr int BK_LP_TABLE_WORDS = BK_LP_MAX_ROOTS * 4 + 4;
// A node of a small subtree waiting for a lane: root index | depth << 8,
// cand, finc, xs, hash sum (2 words).
constexpr int BK_LP_TASK_WORDS = 6;
constexpr int BK_LP_TASK_CAP = 2048;

// Dynamic shared memory of one search block: 256 histogram bins, the pivot
// scratch of every warp, the optional per-warp workspace slots, then the
// per-warp regions of the lane-parallel small search.
__host__ __device__ inline int64_t bk_block_smem_bytes(int32_t warps_per_block, int32_t smem_words,
                                                       int32_t lp_words) {
    return (int64_t)512 * 4 + (int64_t)warps_per_block * (BK_PIV_WORDS + smem_words + lp_words) * 4;
}

// Frames of the explicit stack: one per clique vertex beyond the seeds,
// at most 511 (a deeper search stops with an error instead of overrunning).
__host__ __device__ inline int64_t bk_depth_cap(int64_t c) { return (c < 511 ? c : 511) + 2; }

// Words of the per-warp search state: F and its scratch, frames, K path,
// and (incremental mode) the exclusion rows.
__host__ __device__ inline int64_t bk_private_words(int64_t w, int64_t c, int32_t mode) {
    const int64_t wc = (c + 31) / 32;
    const int64_t S = bk_row_stride(wc);
    const int64_t fr = 4 * wc + 4;                  // cand, finic, ext, conf + meta
    int64_t words = 2 * (w - c) + bk_depth_cap(c) * fr + (c + 2) + 8;
    if (mode == BK_IMCE) words += (c + 2) * S;
    return (words + 31) & ~int64_t(31);
}

// Workspace words needed by a subproblem (same formula on host and device).
__host__ __device__ inline int64_t bk_ws_words(int64_t w, int64_t c, int32_t mode) {
    return bk_shared_words(w, c) + bk_private_words(w, c, mode);
}

mce_status bk_prepare(int32_t blocks_per_sm, int64_t smem_bytes);
mce_status launch_bk(const BkParams &p, int32_t warps_per_block, int32_t blocks_per_sm, cudaStream_t s);
mce_status init_queue_seq(unsigned long long *seq, int64_t n, cudaStream_t s);

}  // namespace mce
