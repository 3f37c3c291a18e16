/*
 * libmce_gb300 — maximal clique enumeration on one GB300 (sm_103a).
 *
 * Implements the method of Das, Sanei-Mehri and Tirthapura, "Shared-Memory
 * Parallel Maximal Clique Enumeration from Static and Dynamic Graphs":
 *   - static MCE: TTT (Algorithm 1) decomposed into one subproblem per vertex
 *     under a total vertex rank (ParMCE, Algorithm 5), heavy subtrees split
 *     with the prefix rule of ParTTT (Algorithm 3);
 *   - incremental MCE for edge additions: new cliques (Algorithm 6 with the
 *     edge-excluding enumerator of Algorithms 7/9) and subsumed cliques
 *     (Algorithm 8), with the maximal cliques kept in a device hash index.
 *
 * Conventions for every call:
 *   - Vertex ids are int32 in [0, n).  Graphs are simple and undirected
 *     (Section 3); inputs are normalised (self loops dropped, direction
 *     ignored, parallel edges merged; Section 6.1).
 *   - "device" pointers are CUDA device addresses on the current device;
 *     "host" pointers are ordinary host memory (pinned memory is faster).
 *   - The caller owns every buffer it passes; the library never keeps a
 *     caller pointer after a call returns.  Objects created by the library
 *     (mce_graph, mce_model, imce_state) are owned by the caller and freed
 *     with the matching *_free / *_close call.
 *   - Work is issued on `stream` (a cudaStream_t, NULL = legacy default
 *     stream).  Calls that return a summary synchronise that stream once to
 *     read it back; results written to caller device buffers are complete
 *     when the call returns.
 *   - The library allocates its own device scratch with the stream-ordered
 *     allocator and keeps a grow-only workspace per device between calls.
 *   - Errors are returned as mce_status; on any status other than MCE_OK,
 *     MCE_EOVERFLOW or MCE_EBUDGET the output structs are left unspecified.
 *     A CUDA error is reported as MCE_ECUDA and the text is available from
 *     mce_last_error().  No entry point aborts the process.
 *
 * Clique set summary (not part of the paper, which outputs the cliques):
 *   h(v)     = splitmix64(v xor seed)   (splitmix64 as published by Vigna:
 *              z = x + 0x9E3779B97F4A7C15, then the 30/27/31 xor-shift-multiply
 *              finaliser with 0xBF58476D1CE4E5B9 and 0x94D049BB133111EB)
 *   H(K)     = fmix(sum_{v in K} h(v) + |K| * 0x9E3779B97F4A7C15)  (mod 2^64)
 *   Hash(C)  = sum_{K in C} H(K)  (mod 2^64)
 * Both levels are order independent, so no sorting is needed on the device.
 */
#ifndef MCE_GB300_H
#define MCE_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t mce_status;
#define MCE_OK 0
#define MCE_EINVAL (-1)     /* bad argument: null pointer, size, id outside [0, n) */
#define MCE_ENOMEM (-2)     /* device allocation failed */
#define MCE_EOVERFLOW (-3)  /* an optional output buffer was too small; summary still exact */
#define MCE_EBUDGET (-4)    /* node budget exhausted; result marked incomplete */
#define MCE_ETIMEOUT (-5)   /* a bounded device wait gave up; result incomplete */
#define MCE_ECUDA (-6)      /* CUDA runtime error */
#define MCE_ESTATE (-7)     /* object in an unusable state */

/* Largest clique size + 1 that the histogram records. */
#define MCE_HIST_CAP 1024

/* Vertex rank keys (Section 4.2): rank(v) = position of (key(v), id(v)) in
 * ascending lexicographic order; a higher key gives a higher rank. */
enum {
    MCE_RANK_DEGREE = 0,    /* key = degree */
    MCE_RANK_DEGEN = 1,     /* key = core number (degeneracy of v) */
    MCE_RANK_TRIANGLE = 2,  /* key = number of triangles containing v */
    MCE_RANK_LEARNED = 3,   /* key = cost predicted by an mce_model */
    MCE_RANK_USER = 4       /* rank given by the caller (a permutation) */
};

typedef struct mce_graph mce_graph;   /* device-resident CSR */
typedef struct mce_model mce_model;   /* MLP cost model, weights on the device */
typedef struct imce_state imce_state; /* graph + its maximal cliques */

typedef struct {
    int32_t rank_kind;            /* MCE_RANK_* */
    const int32_t *user_rank;     /* device int32[n], a permutation of [0, n) (MCE_RANK_USER) */
    const mce_model *model;       /* MCE_RANK_LEARNED */
    uint64_t node_budget;         /* stop after this many search-tree nodes; 0 = unlimited */
    uint64_t hash_seed;           /* seed of h(v) */
    void *stream;                 /* cudaStream_t */
    /* Optional clique list (device, caller-owned).  Clique i starts at
     * list_vtx[list_off[i]] with its size, followed by its vertex ids in no
     * particular order.  Cliques come in no particular order. */
    int64_t *list_off;            /* int64[list_max_cliques] */
    int32_t *list_vtx;            /* int32[list_max_words] */
    int64_t list_max_cliques;
    int64_t list_max_words;
    /* Optional per-subproblem outputs (device uint64[n], caller-owned): the
     * cliques, hash and tree nodes of the subproblem of each vertex v (the
     * cliques whose lowest-ranked vertex is v). */
    uint64_t *pv_count;
    uint64_t *pv_hash;
    uint64_t *pv_nodes;
    int32_t split;                /* 1 = split heavy subtrees across warps (default) */
    uint32_t split_nodes;         /* with split: a task hands over a piece every this many nodes even
                                     when no warp waits (0 = 4096); pieces also go to waiting warps */
    int32_t order_by_model;       /* 1 = schedule subproblems by the model's prediction */
    int32_t warps_per_block;      /* search warps per block, 1..8 (0 = 8) */
    int32_t blocks_per_sm;        /* resident search blocks per SM, 2..4 (0 = 2: 128 registers a
                                     thread; 3 and 4 trade registers for warps) */
    int32_t shared_words;         /* per-warp shared-memory workspace words (0 = none, the default:
                                     the global workspaces then get the whole L1) */
    uint32_t time_limit_ms;       /* stop the search after this long (MCE_ETIMEOUT); 0 = 600 s */
    /* Optional restriction to the subproblems of some vertices (device
     * int32[subset_len], distinct ids); NULL = every vertex. */
    const int32_t *subset;
    int64_t subset_len;
    int32_t subset_on_host;       /* 1 = subset is host memory (copied in) */
    /* Abandon a subproblem once its search tree passes this many nodes
     * (0 = never).  Node credits are exact, so a subproblem is abandoned iff
     * its tree has more nodes than the budget.  Abandoned subproblems are
     * counted in mce_result.incomplete; the summary then includes their
     * partial output, while per-subproblem outputs identify them
     * (pv_nodes > budget). */
    uint64_t subproblem_budget;
    /* Slots of the device task ring that carries handed-over pieces (0 =
     * automatic: 64 MiB of records, 1024..65536 slots).  A full ring refuses a
     * hand-over and the donor keeps the work, so any capacity gives the same
     * result; values below 2 count as 2. */
    int32_t queue_capacity;
    /* 1 = search every small subtree (at most 32 candidates and 32 fini
     * vertices) with the whole warp, one node at a time; 0 (default) = one
     * small subtree per lane, 32 at a time (static MCE without clique lists).
     * Both give the same trees, node counts and cliques. */
    int32_t warp_small_search;
    /* 1 = ParTTT (Algorithm 3) on the whole graph from K = ∅, cand = V, fini =
     * ∅, instead of the per-vertex decomposition: the root's pivot is a vertex
     * p of largest degree (smallest id), its children are the vertices of
     * ext = V \ Γ(p) in increasing id, and each child's subtree is searched
     * (and split across warps) as a subproblem.  tree_nodes counts the root
     * too and equals Algorithm 1's count on the whole graph.  rank_kind,
     * user_rank and subset are ignored. */
    int32_t whole_graph;
    /* Streaming multiprocessors that take search work (0 = all), for scaling
     * measurements: the whole grid is launched and only blocks on SMs with an
     * id below sm_limit search.  The result does not depend on it. */
    int32_t sm_limit;
    /* Per-warp shared-memory words of the lane-parallel small search (0 =
     * automatic: what the block's shared memory leaves, at most 2048; values
     * below 512 turn it off).  Shared memory comes out of the SM's L1, which
     * also caches the lane search's node stacks. */
    int32_t lane_search_words;
    /* Learned heavy-subtree splitting: a model that predicts log(1 + search-
     * tree nodes) of each subproblem under the rank in use.  When set, the
     * subproblems predicted to pass heavy_nodes (0 = 65536) tree nodes hand
     * pieces of their subtree to other warps every heavy_split_nodes (0 =
     * 256) nodes from the start, instead of every split_nodes; with
     * order_by_model the subproblems also run in decreasing predicted cost
     * (this model's, else `model`'s).  Results do not depend on it. */
    const mce_model *split_model;
    uint32_t heavy_nodes;
    uint32_t heavy_split_nodes;
    /* While at least this many warps wait for work, small subtrees are
     * searched by the whole warp, whose pending children can be handed over,
     * instead of by the lanes (0 = never; measured fastest on GB300, where
     * the lanes' shared node stack keeps small subtrees short). */
    uint32_t lane_hold_waiting;
} mce_opts;

typedef struct {
    uint64_t count;               /* maximal cliques */
    uint64_t hash;                /* Hash(C) */
    uint64_t tree_nodes;          /* search-tree nodes visited (Algorithm 1 calls) */
    int32_t hist_len;             /* largest clique size + 1 */
    int32_t complete;             /* 0 if stopped by the budget or a timeout */
    uint64_t hist[MCE_HIST_CAP];  /* hist[s] = cliques of size s */
    int64_t list_cliques;         /* cliques written to the list */
    int64_t list_words;           /* words written to list_vtx */
    uint64_t tasks_split;         /* subtrees handed to other warps */
    int32_t subproblems;          /* vertices with a non-trivial subproblem */
    float ms_rank;                /* ranking time (key + sort), device time */
    float ms_enum;                /* enumeration time, device time */
    float ms_search;              /* device time of the search kernel alone */
    uint64_t word_ops;            /* algorithmic 32-bit word operations of the search: per
                                     tree node (|cand|+|fini|)*ceil(|cand|/32) AND+POPC for
                                     the pivot and 2*ceil((|cand|+|fini|)/32) per child
                                     searched, plus |K| per clique emitted */
    int64_t incomplete;           /* subproblems abandoned by subproblem_budget */
    uint64_t stats[8];            /* search kernel, summed over warps: [0] ns building subproblems,
                                     [1] ns searching, [2] ns waiting for work, [3] builds,
                                     [4] handed-over pieces run, [5] largest busy ns of one
                                     warp, [6] warps, [7] ns from the last subproblem claim to
                                     the end of the launch */
} mce_result;

/* ---------------------------------------------------------------- misc */

const char *mce_strerror(mce_status s);
/* Text of the last CUDA error seen by this thread, or "". */
const char *mce_last_error(void);
/* Fill *o with defaults: degeneracy rank, no budget, seed 0, split on. */
void mce_opts_init(mce_opts *o);
/* Number of kernels this library has launched in this process. */
uint64_t mce_kernel_launches(void);
/* Failure injection for tests, on the host: after `after` more successful
 * device allocations by this library, the next one fails as if the device
 * were out of memory (MCE_ENOMEM); the injection then disarms itself.
 * after < 0 disarms it.  Every entry point keeps its all-or-nothing promise
 * under such a failure (an incremental state is left as it was). */
void mce_debug_fail_alloc(int64_t after);

/* ---------------------------------------------------------------- graphs */

/* Build the CSR of the simple graph behind m raw pairs (u[i], v[i]).
 * u, v: int32[m], device memory if on_device != 0, else host memory.
 * Self loops are dropped, direction ignored, repeats merged (Section 3,
 * Section 6.1).  Errors: MCE_EINVAL for m < 0, n < 0, n >= 2^30 or an id
 * outside [0, n). */
mce_status mce_graph_create(const int32_t *u, const int32_t *v, int64_t m, int32_t n,
                            int32_t on_device, void *stream, mce_graph **g);

/* Graph from a caller CSR (host if on_device == 0, else device):
 * row_ptr int32[n+1], col int32[nnz], copied into library memory.  It must
 * already be a simple undirected graph (Section 3): row_ptr[0] = 0,
 * row_ptr[n] = nnz, rows strictly increasing, ids in [0, n), no self loop,
 * (x, y) present iff (y, x) is.  Anything else is MCE_EINVAL with the
 * failed properties named in mce_last_error(); nothing is repaired. */
mce_status mce_graph_from_csr(const int32_t *row_ptr, const int32_t *col, int32_t n, int64_t nnz,
                              int32_t on_device, void *stream, mce_graph **g);

/* Copy out the CSR: row_ptr int32[n+1] and col int32[nnz] (device
 * pointers owned by the graph, valid until mce_graph_free). */
mce_status mce_graph_csr(const mce_graph *g, int32_t *n, int64_t *nnz,
                         const int32_t **row_ptr, const int32_t **col);

/* Copy the CSR into caller buffers row_ptr int32[n+1] and col int32[nnz]:
 * host memory if to_host != 0, else device memory. */
mce_status mce_graph_copy_csr(const mce_graph *g, int32_t *row_ptr, int32_t *col, int32_t to_host, void *stream);

void mce_graph_free(mce_graph *g);

/* ---------------------------------------------------------------- ranking */

/* Per-vertex key (Section 4.2) into device int64[n]: kind MCE_RANK_DEGREE
 * (degree), MCE_RANK_DEGEN (core number: v is in the k-core but not the
 * (k+1)-core) or MCE_RANK_TRIANGLE (triangles containing v). */
mce_status mce_vertex_key(const mce_graph *g, int32_t kind, void *stream, int64_t *key);

/* rank_out: device int32[n], rank(v) = position of (key(v), v) in ascending
 * order, for opts->rank_kind. */
mce_status mce_rank(const mce_graph *g, const mce_opts *opts, int32_t *rank_out);

/* ---------------------------------------------------------------- static MCE */

/* All maximal cliques of g (ParMCE, Algorithm 5, with TTT, Algorithm 1, on
 * each subproblem): count, size histogram, set hash, tree nodes; optional
 * clique list and per-subproblem outputs through opts. */
mce_status mce_enumerate(const mce_graph *g, const mce_opts *opts, mce_result *res);

/* All maximal cliques of g streamed to the host, for outputs larger than
 * device memory.  The rank is computed once; the subproblems (Algorithm 5)
 * then run a chunk of vertices at a time with their clique list in one of two
 * device buffers of buf_words words, and while the next chunk runs, the last
 * one's list is copied to pinned host memory and passed to sink(ctx, off, vtx,
 * n_cliques, n_words): clique i starts at vtx[off[i]] with its size, then its
 * vertex ids (host memory owned by the library, valid during the call).  A
 * chunk whose list does not fit is split and run again, so every clique
 * reaches the sink exactly once.  *res is the summary over all chunks.
 * opts->subset, lists, per-subproblem outputs and whole_graph are not
 * offered here (MCE_EINVAL); a single subproblem with more output than
 * buf_words returns MCE_EOVERFLOW.  The sink runs on the calling thread. */
typedef void (*mce_clique_sink)(void *ctx, const int64_t *off, const int32_t *vtx, int64_t n_cliques,
                                int64_t n_words);
mce_status mce_enumerate_stream(const mce_graph *g, const mce_opts *opts, int64_t buf_words, mce_clique_sink sink,
                                void *ctx, mce_result *res);

/* ---------------------------------------------------------------- learned cost model */

/* Per-vertex features, device float[n*8], row-major (MCE_FEATURES_FULL):
 *   0 log1p(degree)              1 core number
 *   2 log1p(triangles)           3 mean log1p(neighbour degree)
 *   4 std log1p(neighbour degree) 5 max log1p(neighbour degree)
 *   6 log1p(#higher-degree-rank neighbours)  7 local clustering 2t/(d(d-1)) */
mce_status mce_features(const mce_graph *g, void *stream, float *feat);
/* Feature sets: MCE_FEATURES_FULL as above (needs core numbers and triangle
 * counts); MCE_FEATURES_LIGHT from one pass over the CSR (degrees only):
 *   0 log1p(d)   1/2/3 mean / std / max log1p(neighbour degree)
 *   4 log1p(#higher-degree-rank neighbours)
 *   5 log1p(sum over neighbours w of min(d, d(w)) / 2)  (a triangle bound)
 *   6 fraction of higher-degree-rank neighbours   7 log1p(sum of neighbour degrees) */
#define MCE_FEATURES_FULL 0
#define MCE_FEATURES_LIGHT 1
mce_status mce_features_kind(const mce_graph *g, int32_t kind, void *stream, float *feat);

/* MLP 8 -> hidden -> hidden -> 1, ReLU, weights initialised from `seed`. */
mce_status mce_model_create(int32_t hidden, uint64_t seed, mce_model **m);
void mce_model_free(mce_model *m);
/* Feature set (MCE_FEATURES_*) the model reads when it ranks or orders
 * subproblems (default MCE_FEATURES_FULL). */
mce_status mce_model_set_features(mce_model *m, int32_t kind);
/* Weights as host float arrays in the order W1[h*8], b1[h], W2[h*h], b2[h],
 * w3[h], b3[1] (row-major, y = W x + b); n_params = 8h + h + h*h + h + h + 1. */
int64_t mce_model_num_params(const mce_model *m);
mce_status mce_model_get(const mce_model *m, float *host_params);
mce_status mce_model_set(mce_model *m, const float *host_params);
/* Mean-squared-error loss and its gradient over `rows` samples (device
 * feat[rows*8], label[rows]) in FP32; grad: host float[n_params]. */
mce_status mce_model_loss_grad(const mce_model *m, const float *feat, const float *label, int32_t rows,
                               void *stream, float *loss, float *host_grad);
/* `epochs` passes of minibatch Adam over device feat/label; *loss_out =
 * last epoch's mean loss. */
mce_status mce_model_train(mce_model *m, const float *feat, const float *label, int32_t rows,
                           int32_t epochs, int32_t batch, float lr, uint64_t seed, void *stream,
                           float *loss_out);
/* Predictions (device float[rows]); bf16 = 1 uses BF16 weights and
 * activations with FP32 accumulation, else FP32. */
mce_status mce_model_predict(const mce_model *m, const float *feat, int32_t rows, int32_t bf16,
                             void *stream, float *out);

/* ---------------------------------------------------------------- batched MCE */

/* Maximal cliques of k disjoint graphs in one persistent launch.  The
 * graphs are the vertex ranges [graph_ptr[i], graph_ptr[i+1]) of the
 * disjoint union described by (u, v, m, n); graph_ptr is host int32[k+1].
 * Per graph (device buffers, caller-owned): counts uint64[k], hashes
 * uint64[k], status int32[k] (MCE_OK, or MCE_EBUDGET when the graph's search
 * trees have more than opts->node_budget nodes in all; node counts are
 * exact, so the status does not depend on timing).  The budget applies per
 * graph; counts and hashes of graphs over it are partial.  *total receives
 * the summary over all graphs. */
mce_status mce_enumerate_batched(const mce_graph *g, const int32_t *graph_ptr, int32_t k,
                                 const mce_opts *opts, uint64_t *counts, uint64_t *hashes,
                                 int32_t *status, mce_result *total);

/* A reusable batched plan: everything that does not change between runs
 * (graph ids, rank, Γ+ lists, trivial subproblems, subproblem order, all
 * device buffers) is prepared once by mce_batched_create; graph_ptr is host
 * int32[k+1] as for mce_enumerate_batched and opts->node_budget is the
 * per-graph budget.  The plan keeps pointers into g, which must outlive it. */
typedef struct mce_batched mce_batched;
mce_status mce_batched_create(const mce_graph *g, const int32_t *graph_ptr, int32_t k, const mce_opts *opts,
                              mce_batched **b);
/* One asynchronous run on `stream` (no host synchronisation, no
 * allocation).  The first run after creation or tuning is captured into a
 * CUDA graph; later runs replay it. */
mce_status mce_batched_run(mce_batched *b, void *stream);
/* Wait for the last run and copy its per-graph results to host arrays
 * (counts uint64[k], hashes uint64[k], status int32[k]; each may be NULL)
 * and the summary over all graphs to *total. */
mce_status mce_batched_read(mce_batched *b, void *stream, uint64_t *counts, uint64_t *hashes, int32_t *status,
                            mce_result *total);
/* Autotuner: times `repeats` runs of each launch shape (resident blocks per
 * SM x hand-over interval x small nodes searched by the whole warp or by the
 * lanes) with the per-graph budget lowered to tune_budget (0 = keep it) and
 * keeps the fastest; the choice is returned (each pointer may be NULL).
 * Without tuning, a plan with a per-graph budget searches small nodes with
 * the whole warp unless lane_search_words > 0: the lane search finishes its
 * buffered small subtrees even past a graph's budget. */
mce_status mce_batched_tune(mce_batched *b, void *stream, uint64_t tune_budget, int32_t repeats,
                            int32_t *best_blocks_per_sm, uint32_t *best_split_nodes, int32_t *best_warp_small);
void mce_batched_free(mce_batched *b);

/* ---------------------------------------------------------------- incremental MCE */

typedef struct {
    int64_t applied;              /* new edges of the batch (ρ) */
    int64_t dropped;              /* self loops, existing edges, repeats */
    uint64_t new_count, new_hash; /* Λnew = C(G+H) \ C(G) */
    uint64_t sub_count, sub_hash; /* Λdel = C(G) \ C(G+H) */
    int32_t new_hist_len, sub_hist_len;
    uint64_t new_hist[MCE_HIST_CAP];
    uint64_t sub_hist[MCE_HIST_CAP];
    uint64_t alive;               /* |C(G+H)| after the batch */
    float ms;                     /* device time of the batch */
} imce_delta;

/* Take a copy of g and compute C(g) into a device clique index. */
mce_status imce_open(const mce_graph *g, const mce_opts *opts, imce_state **s);
/* Add k raw pairs (device if on_device, else host): canonicalise
 * (Algorithm 6 line 2 order = arrival order; self loops, existing edges and
 * repeats dropped), then Λnew (Algorithms 6, 7), Λdel (Algorithm 8), and
 * update the graph and the index.  All or nothing: on an error the state is
 * unchanged.  Optional lists (device, caller-owned; same layout as the
 * mce_opts list) receive Λnew and Λdel when not NULL. */
mce_status imce_add_edges(imce_state *s, const int32_t *u, const int32_t *v, int64_t k,
                          int32_t on_device, imce_delta *out);
/* Delete k raw pairs (device if on_device, else host) from the graph and
 * update C(G).  The batch is canonicalised as for additions (arrival order;
 * self loops, pairs that are not edges of G and repeats dropped and counted in
 * out->dropped; out->applied = deleted edges).  Deletions reduce to additions
 * (Section 5: G = (G - H) + H): out->sub_* describe the removed cliques
 * C(G) \ C(G - H), which are the new cliques of adding H to G - H and are
 * found on G by Algorithms 6 and 7; out->new_* describe the created cliques
 * C(G - H) \ C(G), Algorithm 8's splits of the removed cliques that are
 * maximal in G - H.  All or nothing: on an error the state is unchanged. */
mce_status imce_remove_edges(imce_state *s, const int32_t *u, const int32_t *v, int64_t k,
                             int32_t on_device, imce_delta *out);
/* Current graph (owned by the state). */
const mce_graph *imce_graph(const imce_state *s);
/* Alive cliques of the index into a caller list (layout as mce_opts). */
mce_status imce_cliques(const imce_state *s, int64_t *list_off, int32_t *list_vtx,
                        int64_t max_cliques, int64_t max_words, int64_t *n_cliques, int64_t *n_words);
void imce_close(imce_state *s);

/* ---------------------------------------------------------------- serving loop */

/* Continuous batching of edge batches over device-resident graphs (tenants),
 * each with its clique index.  Section 5 defines one step for G and a batch
 * H, so a tenant runs one batch at a time in submission order; batches of
 * different tenants run concurrently, one per slot (a worker thread with its
 * own CUDA stream).  A batch is admitted when it has arrived, its tenant is
 * idle, a slot is free and its projected device memory (mem_fixed + 16(n+1)
 * + 8(nnz+2k) + 96k bytes) fits mem_budget next to the batches in flight;
 * the oldest arrived batch that does not fit holds back later ones, and a
 * batch is always admitted when nothing is in flight.  Latency is measured
 * from arrival to completion on a host steady clock. */
typedef struct imce_server imce_server;
/* Test hook: when set, the server calls it in place of imce_add_edges (host
 * arrays u, v of k pairs) and tenants carry no device state. */
typedef mce_status (*imce_server_exec_fn)(void *ctx, int32_t tenant, const int32_t *u, const int32_t *v, int64_t k,
                                          imce_delta *out);
typedef struct {
    int32_t slots;             /* concurrent batches, 1..64 (default 4) */
    uint64_t mem_budget;       /* bytes; 0 = 80% of free device memory at create */
    uint64_t mem_fixed;        /* per-batch fixed part of the projection; 0 = 384 MiB */
    imce_server_exec_fn execute;
    void *execute_ctx;
} imce_server_opts;

typedef struct {
    int64_t id;
    int32_t tenant;
    mce_status status;         /* of imce_add_edges for this batch */
    int64_t edges;             /* raw pairs submitted */
    double arrival_ms, admit_ms, done_ms;   /* server clock */
    uint64_t reserved;         /* projected bytes held while in flight */
    imce_delta delta;
} imce_request_info;

typedef struct {
    int64_t completed, failed, edges, applied;
    uint64_t new_cliques, subsumed_cliques;
    double p50_ms, p99_ms, max_ms;          /* latency: arrival -> completion */
    double wait_p50_ms, wait_p99_ms;        /* arrival -> admission */
    double span_ms;                         /* first arrival -> last completion */
    double edges_per_s;                     /* edges / span */
    int32_t max_in_flight;
    uint64_t peak_reserved, mem_budget;
} imce_server_stats;

void imce_server_opts_init(imce_server_opts *o);
mce_status imce_server_create(const imce_server_opts *o, imce_server **s);
/* imce_open(g, opts) into a new tenant; g is copied; *tenant = its index. */
mce_status imce_server_add_tenant(imce_server *s, const mce_graph *g, const mce_opts *opts, int32_t *tenant);
/* Queue k raw pairs (host arrays, copied before return) for a tenant.  The
 * batch arrives at arrival_ms on the server clock (ms since create or the
 * last reset; negative or past = now).  Returns at once; *id names it. */
mce_status imce_server_submit(imce_server *s, int32_t tenant, const int32_t *u, const int32_t *v, int64_t k,
                              double arrival_ms, int64_t *id);
/* Block until batch `id` has finished; returns its status. */
mce_status imce_server_wait(imce_server *s, int64_t id, imce_request_info *info);
/* Block until every submitted batch has finished. */
mce_status imce_server_drain(imce_server *s);
/* Drain, then restart the clock at 0 and the statistics. */
mce_status imce_server_reset_clock(imce_server *s);
/* Statistics over the batches finished since create or the last reset. */
mce_status imce_server_stats_get(imce_server *s, imce_server_stats *st);
/* The tenant's state (owned by the server; use only while it is idle). */
imce_state *imce_server_tenant(imce_server *s, int32_t tenant);
/* Drain, stop the workers and close every tenant. */
void imce_server_free(imce_server *s);

/* ---------------------------------------------------------------- no-allocation entry point */

/* Size of the fixed device scratch array used by mce_enumerate_noalloc. */
#define MCE_NOALLOC_SCRATCH_BYTES (64u << 20)

/* Static maximal clique enumeration that allocates no memory.  The paper has
 * no counterpart; this exists for callers that cannot allocate device memory
 * when they enumerate (an allocator that owns all device memory, a service
 * that must not grow after start-up).
 *
 * row_ptr int32[n+1] and col int32[nnz]: a simple undirected graph as CSR
 * on the device, rows sorted (e.g. from mce_graph_csr); rank int32[n]: a
 * permutation of [0, n) on the device (e.g. from mce_rank).  Both are checked
 * on the device before anything reads through them (row_ptr[0] = 0,
 * row_ptr[n] = nnz, row_ptr non-decreasing, ids in [0, n), rows strictly
 * increasing, no self loop, (x, y) present iff (y, x) is, rank values in
 * [0, n) and distinct); a failed check returns MCE_EINVAL with the property
 * named in mce_last_error().  Subproblems run
 * in vertex order; the result (count, hash, histogram, tree nodes) equals
 * mce_enumerate with the same rank and seed.  Clique lists, per-subproblem
 * outputs and budgets are not offered here.
 *
 * All intermediate data lives in one library-owned device array of
 * MCE_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 * exit.  Graphs whose working data exceeds it (or with more than 4194303
 * vertices) are rejected with MCE_EINVAL and a message in mce_last_error().
 * The first call on a device looks up the array's address (with that device
 * current); make it before any stream capture.  Calls share the array: calls
 * that overlap on the GPU race and must be serialised by the caller. */
mce_status mce_enumerate_noalloc(const int32_t *row_ptr, const int32_t *col, int32_t n, int64_t nnz,
                                 const int32_t *rank, uint64_t hash_seed, void *stream, mce_result *res);

#ifdef __cplusplus
}
#endif

#endif /* MCE_GB300_H */
