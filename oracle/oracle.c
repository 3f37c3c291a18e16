/*
 * CPU oracle for maximal clique enumeration (MCE) and its incremental form.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code with
 * the CUDA path: it is a plain, slow, sequential restatement of the paper
 * (Das, Sanei-Mehri, Tirthapura, "Shared-Memory Parallel Maximal Clique
 * Enumeration from Static and Dynamic Graphs"):
 *
 *   - graph normalisation (Section 3 / Section 6.1),
 *   - vertex keys and ranks (Section 4.2: degree, triangle count, degeneracy),
 *   - TTT (Algorithm 1) with a pivot maximising |cand ∩ Γ(u)|,
 *   - ParMCE's per-vertex decomposition (Algorithm 5), run one subproblem at
 *     a time (optionally on several host threads, one subproblem per thread),
 *   - new cliques after an edge batch: Algorithm 6 with the sequential
 *     edge-excluding TTT of Algorithm 9 (Appendix A),
 *   - subsumed cliques: Algorithm 8,
 *   - the plain set differences C(G+H) \ C(G) and C(G) \ C(G+H),
 *   - edge deletions, by reduction to the incremental step (G = (G - H) + H):
 *     removed = Algorithm 6 on G, created = Algorithm 8's splits of the
 *     removed cliques that are maximal in G - H; and by the set differences.
 *
 * Sets are sorted int32 arrays.  Readings where the paper is silent:
 *   - rank(v) = position of (key(v), id(v)) in ascending lexicographic order;
 *   - pivot ties go to the smallest vertex id; ext is visited in ascending id;
 *   - "K_q ∩ E ≠ ∅" (Algorithms 7/9) means K_q contains both endpoints of an
 *     excluded edge; as K itself never contains one, only pairs (q, w), w ∈ K,
 *     are tested;
 *   - edge batches are canonicalised in arrival order: self-loops, pairs
 *     already in G and repeats inside the batch are dropped and counted.
 *   - Set hash: h(v) = splitmix64(v xor seed); H(K) = fmix(sum h(v) +
 *     |K| * 0x9E3779B97F4A7C15); Hash(C) = sum over cliques of H(K) mod 2^64.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAX_HIST 4096

/* ------------------------------------------------------------------ */
/* hashing of cliques (order independent)                              */
/* ------------------------------------------------------------------ */

static const uint64_t GOLDEN = 0x9E3779B97F4A7C15ULL;

static uint64_t fmix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static uint64_t vertex_hash(int32_t v, uint64_t seed) {
    return fmix(((uint64_t)(uint32_t)v ^ seed) + GOLDEN);
}

static uint64_t clique_hash(const int32_t *k, int32_t len, uint64_t seed) {
    uint64_t s = 0;
    for (int32_t i = 0; i < len; ++i) s += vertex_hash(k[i], seed);
    return fmix(s + (uint64_t)len * GOLDEN);
}

uint64_t or_clique_hash(const int32_t *k, int32_t len, uint64_t seed) { return clique_hash(k, len, seed); }

/* ------------------------------------------------------------------ */
/* graph                                                               */
/* ------------------------------------------------------------------ */

typedef struct {
    int32_t n;
    int64_t nnz;       /* 2m */
    int64_t *row_ptr;  /* n+1 */
    int32_t *col;      /* sorted per row */
} or_graph;

static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

/* Simple undirected graph from raw pairs: drop self loops, ignore direction,
 * merge parallel edges.  Returns NULL on an id outside [0, n). */
or_graph *or_graph_from_pairs(int32_t n, const int32_t *u, const int32_t *v, int64_t m) {
    uint64_t *dir = (uint64_t *)malloc((size_t)(2 * m + 1) * sizeof(uint64_t));
    if (!dir) return NULL;
    int64_t k = 0;
    for (int64_t i = 0; i < m; ++i) {
        if (u[i] < 0 || u[i] >= n || v[i] < 0 || v[i] >= n) { free(dir); return NULL; }
        if (u[i] == v[i]) continue;
        dir[k++] = ((uint64_t)(uint32_t)u[i] << 32) | (uint32_t)v[i];
        dir[k++] = ((uint64_t)(uint32_t)v[i] << 32) | (uint32_t)u[i];
    }
    qsort(dir, (size_t)k, sizeof(uint64_t), cmp_u64);
    int64_t w = 0;
    for (int64_t i = 0; i < k; ++i)
        if (w == 0 || dir[i] != dir[w - 1]) dir[w++] = dir[i];
    or_graph *g = (or_graph *)calloc(1, sizeof(or_graph));
    g->n = n;
    g->nnz = w;
    g->row_ptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->col = (int32_t *)malloc((size_t)(w + 1) * sizeof(int32_t));
    for (int64_t i = 0; i < w; ++i) {
        g->row_ptr[(dir[i] >> 32) + 1]++;
        g->col[i] = (int32_t)(dir[i] & 0xffffffffu);
    }
    for (int32_t i = 0; i < n; ++i) g->row_ptr[i + 1] += g->row_ptr[i];
    free(dir);
    return g;
}

void or_graph_free(or_graph *g) {
    if (!g) return;
    free(g->row_ptr);
    free(g->col);
    free(g);
}

int64_t or_graph_nnz(const or_graph *g) { return g->nnz; }
int32_t or_graph_n(const or_graph *g) { return g->n; }

void or_graph_export(const or_graph *g, int64_t *row_ptr, int32_t *col) {
    memcpy(row_ptr, g->row_ptr, ((size_t)g->n + 1) * sizeof(int64_t));
    memcpy(col, g->col, (size_t)g->nnz * sizeof(int32_t));
}

static inline const int32_t *nbr(const or_graph *g, int32_t v) { return g->col + g->row_ptr[v]; }
static inline int32_t deg(const or_graph *g, int32_t v) { return (int32_t)(g->row_ptr[v + 1] - g->row_ptr[v]); }

static int has_edge(const or_graph *g, int32_t a, int32_t b) {
    const int32_t *r = nbr(g, a);
    int32_t lo = 0, hi = deg(g, a);
    while (lo < hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (r[mid] < b) lo = mid + 1; else hi = mid;
    }
    return lo < deg(g, a) && r[lo] == b;
}

/* ------------------------------------------------------------------ */
/* sorted-set primitives                                               */
/* ------------------------------------------------------------------ */

static int32_t lower_bound(const int32_t *a, int32_t n, int32_t x) {
    int32_t lo = 0, hi = n;
    while (lo < hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

static int contains(const int32_t *a, int32_t n, int32_t x) {
    int32_t p = lower_bound(a, n, x);
    return p < n && a[p] == x;
}

/* |a ∩ b|: search the smaller set in the larger one (the method of the
 * proof of Lemma 1) when their sizes differ a lot, else merge. */
static int32_t isect_count(const int32_t *a, int32_t na, const int32_t *b, int32_t nb) {
    if (na > nb) { const int32_t *t = a; a = b; b = t; int32_t tn = na; na = nb; nb = tn; }
    int32_t c = 0;
    if ((int64_t)na * 16 < nb) {
        for (int32_t i = 0; i < na; ++i) c += contains(b, nb, a[i]);
        return c;
    }
    int32_t i = 0, j = 0;
    while (i < na && j < nb) {
        if (a[i] < b[j]) ++i;
        else if (a[i] > b[j]) ++j;
        else { ++c; ++i; ++j; }
    }
    return c;
}

/* out = a ∩ b (sorted); returns |out| */
static int32_t isect(const int32_t *a, int32_t na, const int32_t *b, int32_t nb, int32_t *out) {
    int32_t c = 0;
    if ((int64_t)na * 16 < nb) {
        for (int32_t i = 0; i < na; ++i) if (contains(b, nb, a[i])) out[c++] = a[i];
        return c;
    }
    if ((int64_t)nb * 16 < na) {
        for (int32_t j = 0; j < nb; ++j) if (contains(a, na, b[j])) out[c++] = b[j];
        return c;
    }
    int32_t i = 0, j = 0;
    while (i < na && j < nb) {
        if (a[i] < b[j]) ++i;
        else if (a[i] > b[j]) ++j;
        else { out[c++] = a[i]; ++i; ++j; }
    }
    return c;
}

/* out = a \ b (sorted); returns |out| */
static int32_t setminus(const int32_t *a, int32_t na, const int32_t *b, int32_t nb, int32_t *out) {
    int32_t c = 0;
    for (int32_t i = 0; i < na; ++i) if (!contains(b, nb, a[i])) out[c++] = a[i];
    return c;
}

/* remove x from sorted a (present); returns new size */
static int32_t erase_sorted(int32_t *a, int32_t n, int32_t x) {
    int32_t p = lower_bound(a, n, x);
    if (p < n && a[p] == x) { memmove(a + p, a + p + 1, (size_t)(n - p - 1) * sizeof(int32_t)); return n - 1; }
    return n;
}

/* insert x into sorted a (absent); capacity assumed; returns new size */
static int32_t insert_sorted(int32_t *a, int32_t n, int32_t x) {
    int32_t p = lower_bound(a, n, x);
    memmove(a + p + 1, a + p, (size_t)(n - p) * sizeof(int32_t));
    a[p] = x;
    return n + 1;
}

/* ------------------------------------------------------------------ */
/* output accumulator                                                  */
/* ------------------------------------------------------------------ */

typedef struct {
    uint64_t count, hash, nodes;
    uint64_t hist[OR_MAX_HIST];
    int32_t max_size;
    uint64_t seed;
    int want_list;
    int64_t n_cl, cap_cl, nnz, cap_nnz;
    int64_t *off;   /* n_cl + 1 */
    int32_t *vtx;
    int overflow;   /* clique larger than OR_MAX_HIST-1 */
} or_out;

or_out *or_out_new(int want_list, uint64_t seed) {
    or_out *o = (or_out *)calloc(1, sizeof(or_out));
    o->want_list = want_list;
    o->seed = seed;
    o->cap_cl = 1024;
    o->cap_nnz = 4096;
    if (want_list) {
        o->off = (int64_t *)malloc((size_t)(o->cap_cl + 1) * sizeof(int64_t));
        o->vtx = (int32_t *)malloc((size_t)o->cap_nnz * sizeof(int32_t));
        o->off[0] = 0;
    }
    return o;
}

void or_out_free(or_out *o) {
    if (!o) return;
    free(o->off);
    free(o->vtx);
    free(o);
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* record one maximal clique K (any order) */
static void emit(or_out *o, const int32_t *k, int32_t len) {
    o->count++;
    o->hash += clique_hash(k, len, o->seed);
    if (len < OR_MAX_HIST) o->hist[len]++; else o->overflow = 1;
    if (len > o->max_size) o->max_size = len;
    if (!o->want_list) return;
    if (o->n_cl == o->cap_cl) {
        o->cap_cl *= 2;
        o->off = (int64_t *)realloc(o->off, (size_t)(o->cap_cl + 1) * sizeof(int64_t));
    }
    while (o->nnz + len > o->cap_nnz) {
        o->cap_nnz *= 2;
        o->vtx = (int32_t *)realloc(o->vtx, (size_t)o->cap_nnz * sizeof(int32_t));
    }
    memcpy(o->vtx + o->nnz, k, (size_t)len * sizeof(int32_t));
    qsort(o->vtx + o->nnz, (size_t)len, sizeof(int32_t), cmp_i32);
    o->nnz += len;
    o->n_cl++;
    o->off[o->n_cl] = o->nnz;
}

static void out_merge(or_out *dst, const or_out *src) {
    dst->count += src->count;
    dst->hash += src->hash;
    dst->nodes += src->nodes;
    for (int i = 0; i <= src->max_size && i < OR_MAX_HIST; ++i) dst->hist[i] += src->hist[i];
    if (src->max_size > dst->max_size) dst->max_size = src->max_size;
    dst->overflow |= src->overflow;
    if (!(dst->want_list && src->want_list)) return;
    for (int64_t c = 0; c < src->n_cl; ++c) {
        int32_t len = (int32_t)(src->off[c + 1] - src->off[c]);
        if (dst->n_cl == dst->cap_cl) {
            dst->cap_cl *= 2;
            dst->off = (int64_t *)realloc(dst->off, (size_t)(dst->cap_cl + 1) * sizeof(int64_t));
        }
        while (dst->nnz + len > dst->cap_nnz) {
            dst->cap_nnz *= 2;
            dst->vtx = (int32_t *)realloc(dst->vtx, (size_t)dst->cap_nnz * sizeof(int32_t));
        }
        memcpy(dst->vtx + dst->nnz, src->vtx + src->off[c], (size_t)len * sizeof(int32_t));
        dst->nnz += len;
        dst->n_cl++;
        dst->off[dst->n_cl] = dst->nnz;
    }
}

/* empty the accumulator, keeping its buffers */
static void out_reset(or_out *o) {
    for (int i = 0; i <= o->max_size && i < OR_MAX_HIST; ++i) o->hist[i] = 0;
    o->count = o->hash = o->nodes = 0;
    o->max_size = 0;
    o->overflow = 0;
    o->n_cl = o->nnz = 0;
}

uint64_t or_out_count(const or_out *o) { return o->count; }
uint64_t or_out_hash(const or_out *o) { return o->hash; }
uint64_t or_out_nodes(const or_out *o) { return o->nodes; }
int32_t or_out_overflow(const or_out *o) { return o->overflow; }
int32_t or_out_hist_len(const or_out *o) { return o->count ? o->max_size + 1 : 0; }
void or_out_hist(const or_out *o, uint64_t *dst) {
    for (int32_t i = 0; i < or_out_hist_len(o); ++i) dst[i] = o->hist[i];
}
int64_t or_out_list_len(const or_out *o) { return o->n_cl; }
int64_t or_out_list_nnz(const or_out *o) { return o->nnz; }
void or_out_list_copy(const or_out *o, int64_t *off, int32_t *vtx) {
    memcpy(off, o->off, (size_t)(o->n_cl + 1) * sizeof(int64_t));
    memcpy(vtx, o->vtx, (size_t)o->nnz * sizeof(int32_t));
}

/* ------------------------------------------------------------------ */
/* vertex keys and ranks (Section 4.2)                                 */
/* ------------------------------------------------------------------ */

void or_degree(const or_graph *g, int64_t *out) {
    for (int32_t v = 0; v < g->n; ++v) out[v] = deg(g, v);
}

/* Core number by peeling: v has core number k when it lies in the k-core but
 * not in the (k+1)-core.  For k = 0, 1, 2, ... all vertices whose remaining
 * degree is at most k are removed repeatedly; those removed while k is the
 * current level have core number k. */
void or_core_numbers(const or_graph *g, int32_t *core) {
    int32_t n = g->n;
    int32_t *d = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    char *gone = (char *)calloc((size_t)n, 1);
    int32_t *queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t removed = 0;
    for (int32_t v = 0; v < n; ++v) d[v] = deg(g, v);
    for (int32_t k = 0; removed < n; ++k) {
        int32_t qh = 0, qt = 0;
        for (int32_t v = 0; v < n; ++v)
            if (!gone[v] && d[v] <= k) { gone[v] = 1; queue[qt++] = v; }
        while (qh < qt) {
            int32_t v = queue[qh++];
            core[v] = k;
            removed++;
            for (int64_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; ++e) {
                int32_t w = g->col[e];
                if (gone[w]) continue;
                if (--d[w] <= k) { gone[w] = 1; queue[qt++] = w; }
            }
        }
    }
    free(d);
    free(gone);
    free(queue);
}

/* t(v) = number of triangles containing v = number of edges among Γ(v).
 * For each edge {a, b} the common neighbours are the third corners of the
 * triangles through that edge; summing over the edges at v counts each of
 * v's triangles twice. */
void or_triangles(const or_graph *g, int64_t *t) {
    for (int32_t v = 0; v < g->n; ++v) t[v] = 0;
    for (int32_t a = 0; a < g->n; ++a)
        for (int64_t e = g->row_ptr[a]; e < g->row_ptr[a + 1]; ++e) {
            int32_t b = g->col[e];
            if (b <= a) continue;
            int32_t c = isect_count(nbr(g, a), deg(g, a), nbr(g, b), deg(g, b));
            t[a] += c;
            t[b] += c;
        }
    for (int32_t v = 0; v < g->n; ++v) t[v] /= 2;
}

typedef struct { double key; int32_t id; } keyed;

static int cmp_keyed(const void *a, const void *b) {
    const keyed *x = (const keyed *)a, *y = (const keyed *)b;
    if (x->key != y->key) return (x->key > y->key) - (x->key < y->key);
    return (x->id > y->id) - (x->id < y->id);
}

/* rank[v] = position of (key[v], v) in ascending lexicographic order. */
void or_rank_from_key(int32_t n, const double *key, int32_t *rank) {
    keyed *a = (keyed *)malloc((size_t)n * sizeof(keyed));
    for (int32_t v = 0; v < n; ++v) { a[v].key = key[v]; a[v].id = v; }
    qsort(a, (size_t)n, sizeof(keyed), cmp_keyed);
    for (int32_t i = 0; i < n; ++i) rank[a[i].id] = i;
    free(a);
}

/* ------------------------------------------------------------------ */
/* TTT (Algorithm 1) and its edge-excluding form (Algorithm 9)         */
/* ------------------------------------------------------------------ */

/* Excluded edges E = {e_1 .. e_{limit}} of a batch, looked up by key. */
typedef struct {
    const uint64_t *keys;  /* sorted canonical keys of the batch edges */
    const int64_t *index;  /* arrival index of keys[i] */
    int64_t n;
    int64_t limit;         /* edges with index < limit are excluded */
} excl_set;

static int excluded(const excl_set *x, int32_t a, int32_t b) {
    if (!x) return 0;
    uint64_t key = a < b ? ((uint64_t)(uint32_t)a << 32) | (uint32_t)b : ((uint64_t)(uint32_t)b << 32) | (uint32_t)a;
    int64_t lo = 0, hi = x->n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (x->keys[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo < x->n && x->keys[lo] == key && x->index[lo] < x->limit;
}

typedef struct {
    const or_graph *g;
    or_out *out;
    int32_t *K;          /* current clique, K[0..klen) */
    const excl_set *ex;  /* NULL for plain TTT */
    uint64_t stop_after; /* abandon once out->nodes passes this (0 = never) */
    int abandoned;
} ttt_ctx;

/* TTT(G, K, cand, fini) of Algorithm 1 (Algorithm 9 when ctx->ex is set).
 * cand and fini are owned by this call and modified in place, as the
 * pseudocode does.  Neighbourhoods are those of the whole graph: every set in
 * the recursion lies inside the subgraph being enumerated, so intersecting
 * with Γ_G(u) equals intersecting with the induced subgraph's Γ(u). */
static void ttt(ttt_ctx *c, int32_t klen, int32_t *cand, int32_t nc, int32_t *fini, int32_t nf) {
    const or_graph *g = c->g;
    c->out->nodes++;
    if (c->stop_after && c->out->nodes > c->stop_after) {   /* node cap: give the search up */
        c->abandoned = 1;
        return;
    }
    if (nc == 0 && nf == 0) {           /* K is maximal */
        emit(c->out, c->K, klen);
        return;
    }
    /* pivot u in cand ∪ fini maximising |cand ∩ Γ(u)|; ties: smallest id */
    int32_t best = -1, piv = -1;
    for (int32_t s = 0; s < 2; ++s) {
        const int32_t *set = s == 0 ? cand : fini;
        int32_t ns = s == 0 ? nc : nf;
        for (int32_t i = 0; i < ns; ++i) {
            int32_t u = set[i];
            int32_t t = isect_count(cand, nc, nbr(g, u), deg(g, u));
            if (t > best || (t == best && u < piv)) { best = t; piv = u; }
        }
    }
    /* ext = cand \ Γ(pivot), ascending */
    int32_t *ext = (int32_t *)malloc((size_t)(nc + 1) * sizeof(int32_t));
    int32_t ne = setminus(cand, nc, nbr(g, piv), deg(g, piv), ext);
    /* fini grows by one vertex per iteration */
    int32_t *fin = (int32_t *)malloc((size_t)(nf + ne + 1) * sizeof(int32_t));
    memcpy(fin, fini, (size_t)nf * sizeof(int32_t));
    int32_t *cq = (int32_t *)malloc((size_t)(nc + 1) * sizeof(int32_t));
    int32_t *fq = (int32_t *)malloc((size_t)(nf + ne + 1) * sizeof(int32_t));
    for (int32_t i = 0; i < ne; ++i) {
        int32_t q = ext[i];
        if (c->ex) {   /* Algorithm 9: K_q containing an excluded edge */
            int bad = 0;
            for (int32_t j = 0; j < klen && !bad; ++j) bad = excluded(c->ex, q, c->K[j]);
            if (bad) {
                nc = erase_sorted(cand, nc, q);
                nf = insert_sorted(fin, nf, q);
                continue;
            }
        }
        int32_t ncq = isect(cand, nc, nbr(g, q), deg(g, q), cq);
        int32_t nfq = isect(fin, nf, nbr(g, q), deg(g, q), fq);
        c->K[klen] = q;
        ttt(c, klen + 1, cq, ncq, fq, nfq);
        if (c->abandoned) break;
        nc = erase_sorted(cand, nc, q);
        nf = insert_sorted(fin, nf, q);
    }
    free(ext);
    free(fin);
    free(cq);
    free(fq);
}

/* Whole-graph TTT: K = ∅, cand = V, fini = ∅. */
void or_ttt_whole(const or_graph *g, or_out *out) {
    int32_t *cand = (int32_t *)malloc(((size_t)g->n + 1) * sizeof(int32_t));
    int32_t *K = (int32_t *)malloc(((size_t)g->n + 1) * sizeof(int32_t));
    for (int32_t v = 0; v < g->n; ++v) cand[v] = v;
    ttt_ctx c = {g, out, K, NULL, 0, 0};
    if (g->n > 0) ttt(&c, 0, cand, g->n, NULL, 0);
    free(cand);
    free(K);
}

/* ------------------------------------------------------------------ */
/* ParMCE decomposition (Algorithm 5)                                  */
/* ------------------------------------------------------------------ */

/* Subproblem of v: K = {v}, cand = higher-ranked neighbours, fini = the
 * lower-ranked ones, then TTT on G_v. */
static int parmce_one(const or_graph *g, const int32_t *rank, int32_t v, or_out *out, int32_t *K,
                      uint64_t node_cap) {
    int32_t d = deg(g, v);
    const int32_t *nv = nbr(g, v);
    int32_t *cand = (int32_t *)malloc((size_t)(d + 1) * sizeof(int32_t));
    int32_t *fini = (int32_t *)malloc((size_t)(d + 1) * sizeof(int32_t));
    int32_t nc = 0, nf = 0;
    for (int32_t i = 0; i < d; ++i) {
        int32_t w = nv[i];
        if (rank[w] > rank[v]) cand[nc++] = w; else fini[nf++] = w;
    }
    K[0] = v;
    ttt_ctx c = {g, out, K, NULL, node_cap ? out->nodes + node_cap : 0, 0};
    ttt(&c, 1, cand, nc, fini, nf);
    free(cand);
    free(fini);
    return c.abandoned;
}

typedef struct {
    const or_graph *g;
    const int32_t *rank;
    const int32_t *subset;   /* NULL: all vertices */
    int64_t nsub;
    int64_t next;            /* shared work counter */
    or_out *outs;            /* per thread (array of or_out*) */
    or_out **thread_out;
    uint64_t *pv_count, *pv_hash, *pv_nodes;
    uint64_t node_cap;       /* abandon a subproblem whose tree passes this many nodes (0 = never) */
    uint8_t *over;           /* per subset index: 1 = abandoned */
} pm_shared;

static void *pm_worker(void *arg) {
    void **a = (void **)arg;
    pm_shared *s = (pm_shared *)a[0];
    or_out *out = (or_out *)a[1];
    int32_t *K = (int32_t *)malloc(((size_t)s->g->n + 2) * sizeof(int32_t));
    /* with a node cap each subproblem runs into its own accumulator, merged
     * only when it finished within the cap */
    or_out *one = s->node_cap ? or_out_new(out->want_list, out->seed) : NULL;
    for (;;) {
        int64_t i = __atomic_fetch_add(&s->next, 1, __ATOMIC_RELAXED);
        if (i >= s->nsub) break;
        int32_t v = s->subset ? s->subset[i] : (int32_t)i;
        or_out *dst = one ? one : out;
        if (one) out_reset(one);
        uint64_t c0 = dst->count, h0 = dst->hash, n0 = dst->nodes;
        int ab = parmce_one(s->g, s->rank, v, dst, K, s->node_cap);
        if (s->pv_count) s->pv_count[i] = dst->count - c0;
        if (s->pv_hash) s->pv_hash[i] = dst->hash - h0;
        if (s->pv_nodes) s->pv_nodes[i] = dst->nodes - n0;
        if (s->over) s->over[i] = (uint8_t)ab;
        if (one && !ab) out_merge(out, one);
    }
    or_out_free(one);
    free(K);
    return NULL;
}

/* Run the subproblems of `subset` (all vertices when NULL) on `threads`
 * host threads, one whole subproblem per thread at a time.  Per-subproblem
 * count/hash/tree-node arrays (indexed like subset) are optional.  With
 * node_cap > 0 a subproblem is given up at its (node_cap + 1)-th tree node:
 * it is flagged in `over` (optional), its per-subproblem entries hold what it
 * reached, and it adds nothing to `out`. */
int32_t or_parmce(const or_graph *g, const int32_t *rank, const int32_t *subset, int64_t nsub,
                  int32_t threads, or_out *out, uint64_t *pv_count, uint64_t *pv_hash, uint64_t *pv_nodes,
                  uint64_t node_cap, uint8_t *over) {
    pm_shared s;
    memset(&s, 0, sizeof(s));
    s.g = g;
    s.rank = rank;
    s.subset = subset;
    s.nsub = subset ? nsub : g->n;
    s.pv_count = pv_count;
    s.pv_hash = pv_hash;
    s.pv_nodes = pv_nodes;
    s.node_cap = node_cap;
    s.over = over;
    if (threads < 1) threads = 1;
    if (threads == 1) {
        void *a[2] = {&s, out};
        pm_worker(a);
        return 1;
    }
    pthread_t *th = (pthread_t *)malloc((size_t)threads * sizeof(pthread_t));
    or_out **outs = (or_out **)malloc((size_t)threads * sizeof(or_out *));
    void **args = (void **)malloc((size_t)threads * 2 * sizeof(void *));
    for (int32_t t = 0; t < threads; ++t) {
        outs[t] = or_out_new(out->want_list, out->seed);
        args[2 * t] = &s;
        args[2 * t + 1] = outs[t];
        pthread_create(&th[t], NULL, pm_worker, &args[2 * t]);
    }
    for (int32_t t = 0; t < threads; ++t) {
        pthread_join(th[t], NULL);
        out_merge(out, outs[t]);
        or_out_free(outs[t]);
    }
    free(th);
    free(outs);
    free(args);
    return threads;
}

/* ------------------------------------------------------------------ */
/* incremental maintenance (Section 5)                                 */
/* ------------------------------------------------------------------ */

/* Canonical batch: (min, max) pairs in arrival order with self loops, pairs
 * already in G and repeats removed.  Returns the number kept, or -1 on an id
 * outside [0, n). */
int64_t or_canonical_batch(const or_graph *g, const int32_t *u, const int32_t *v, int64_t k,
                           int32_t *hu, int32_t *hv) {
    uint64_t cap = 16;
    while (cap < (uint64_t)k * 2 + 16) cap <<= 1;
    uint64_t *seen = (uint64_t *)malloc(cap * sizeof(uint64_t));   /* open addressing, UINT64_MAX = empty */
    memset(seen, 0xff, cap * sizeof(uint64_t));
    int64_t kept = 0;
    for (int64_t i = 0; i < k; ++i) {
        if (u[i] < 0 || u[i] >= g->n || v[i] < 0 || v[i] >= g->n) { free(seen); return -1; }
        if (u[i] == v[i]) continue;
        int32_t a = u[i] < v[i] ? u[i] : v[i], b = u[i] < v[i] ? v[i] : u[i];
        if (has_edge(g, a, b)) continue;
        uint64_t key = ((uint64_t)(uint32_t)a << 32) | (uint32_t)b;
        uint64_t h = fmix(key) & (cap - 1);
        int dup = 0;
        while (seen[h] != UINT64_MAX) {
            if (seen[h] == key) { dup = 1; break; }
            h = (h + 1) & (cap - 1);
        }
        if (dup) continue;
        seen[h] = key;
        hu[kept] = a;
        hv[kept] = b;
        kept++;
    }
    free(seen);
    return kept;
}

static or_graph *graph_plus(const or_graph *g, const int32_t *hu, const int32_t *hv, int64_t rho) {
    int64_t m0 = g->nnz;
    int32_t *u = (int32_t *)malloc((size_t)(m0 + rho + 1) * sizeof(int32_t));
    int32_t *v = (int32_t *)malloc((size_t)(m0 + rho + 1) * sizeof(int32_t));
    int64_t k = 0;
    for (int32_t a = 0; a < g->n; ++a)
        for (int64_t e = g->row_ptr[a]; e < g->row_ptr[a + 1]; ++e) { u[k] = a; v[k] = g->col[e]; k++; }
    for (int64_t i = 0; i < rho; ++i) { u[k] = hu[i]; v[k] = hv[i]; k++; }
    or_graph *gp = or_graph_from_pairs(g->n, u, v, k);
    free(u);
    free(v);
    return gp;
}

/* Algorithm 6 with Algorithm 9 as the enumerator: for each new edge
 * e_i = (u, v) in arrival order, enumerate the maximal cliques of G+H that
 * contain e_i and no earlier new edge e_1..e_{i-1}. */
static void imce_new(const or_graph *gp, const int32_t *hu, const int32_t *hv, int64_t rho, or_out *out) {
    /* sorted (key, arrival index) table of the batch */
    uint64_t *pairs = (uint64_t *)malloc((size_t)(rho + 1) * 2 * sizeof(uint64_t));
    for (int64_t i = 0; i < rho; ++i) {
        pairs[2 * i] = ((uint64_t)(uint32_t)hu[i] << 32) | (uint32_t)hv[i];
        pairs[2 * i + 1] = (uint64_t)i;
    }
    qsort(pairs, (size_t)rho, 2 * sizeof(uint64_t), cmp_u64);   /* keys are distinct */
    uint64_t *keys = (uint64_t *)malloc((size_t)(rho + 1) * sizeof(uint64_t));
    int64_t *idx = (int64_t *)malloc((size_t)(rho + 1) * sizeof(int64_t));
    for (int64_t i = 0; i < rho; ++i) { keys[i] = pairs[2 * i]; idx[i] = (int64_t)pairs[2 * i + 1]; }
    free(pairs);
    int32_t *K = (int32_t *)malloc(((size_t)gp->n + 2) * sizeof(int32_t));
    for (int64_t i = 0; i < rho; ++i) {
        int32_t u = hu[i], v = hv[i];
        int32_t du = deg(gp, u), dv = deg(gp, v);
        int32_t *cand = (int32_t *)malloc((size_t)((du < dv ? du : dv) + 1) * sizeof(int32_t));
        int32_t nc = isect(nbr(gp, u), du, nbr(gp, v), dv, cand);   /* V_e \ {u, v} */
        excl_set ex = {keys, idx, rho, i};
        K[0] = u;
        K[1] = v;
        ttt_ctx c = {gp, out, K, &ex, 0, 0};
        ttt(&c, 2, cand, nc, NULL, 0);
        free(cand);
    }
    free(K);
    free(keys);
    free(idx);
}

/* ---- a set of cliques (sorted vertex lists), for C and for S ---- */

typedef struct {
    int64_t *off;     /* clique c is vtx[off[c] .. off[c+1]) */
    int32_t *vtx;
    int64_t n, cap, nnz, cap_nnz;
    int64_t *slot;    /* open addressing over clique indices, -1 = empty */
    char *dead;       /* removed from the set */
    uint64_t mask;
} clset;

static uint64_t list_key(const int32_t *k, int32_t len) {
    uint64_t h = 1469598103934665603ULL;
    for (int32_t i = 0; i < len; ++i) h = (h ^ (uint32_t)k[i]) * 1099511628211ULL;
    return fmix(h);
}

static void cs_init(clset *s, int64_t expect) {
    memset(s, 0, sizeof(*s));
    s->cap = 16;
    s->cap_nnz = 64;
    s->off = (int64_t *)malloc((size_t)(s->cap + 1) * sizeof(int64_t));
    s->vtx = (int32_t *)malloc((size_t)s->cap_nnz * sizeof(int32_t));
    s->dead = (char *)calloc((size_t)s->cap, 1);
    s->off[0] = 0;
    uint64_t tcap = 64;
    while (tcap < (uint64_t)expect * 2 + 64) tcap <<= 1;
    s->slot = (int64_t *)malloc(tcap * sizeof(int64_t));
    memset(s->slot, 0xff, tcap * sizeof(int64_t));
    s->mask = tcap - 1;
}

static void cs_free(clset *s) {
    free(s->off);
    free(s->vtx);
    free(s->slot);
    free(s->dead);
}

static int64_t cs_find(const clset *s, const int32_t *k, int32_t len) {
    uint64_t i = list_key(k, len) & s->mask;
    for (;;) {
        int64_t c = s->slot[i];
        if (c < 0) return -1;
        int32_t l = (int32_t)(s->off[c + 1] - s->off[c]);
        if (l == len && memcmp(s->vtx + s->off[c], k, (size_t)len * sizeof(int32_t)) == 0) return c;
        i = (i + 1) & s->mask;
    }
}

static void cs_rehash(clset *s) {
    uint64_t tcap = (s->mask + 1) * 2;
    free(s->slot);
    s->slot = (int64_t *)malloc(tcap * sizeof(int64_t));
    memset(s->slot, 0xff, tcap * sizeof(int64_t));
    s->mask = tcap - 1;
    for (int64_t c = 0; c < s->n; ++c) {
        uint64_t i = list_key(s->vtx + s->off[c], (int32_t)(s->off[c + 1] - s->off[c])) & s->mask;
        while (s->slot[i] >= 0) i = (i + 1) & s->mask;
        s->slot[i] = c;
    }
}

/* insert sorted list k if absent; returns its index */
static int64_t cs_insert(clset *s, const int32_t *k, int32_t len) {
    int64_t f = cs_find(s, k, len);
    if (f >= 0) return f;
    if ((uint64_t)(s->n + 1) * 2 > s->mask + 1) cs_rehash(s);
    if (s->n == s->cap) {
        s->cap *= 2;
        s->off = (int64_t *)realloc(s->off, (size_t)(s->cap + 1) * sizeof(int64_t));
        s->dead = (char *)realloc(s->dead, (size_t)s->cap);
    }
    while (s->nnz + len > s->cap_nnz) {
        s->cap_nnz *= 2;
        s->vtx = (int32_t *)realloc(s->vtx, (size_t)s->cap_nnz * sizeof(int32_t));
    }
    memcpy(s->vtx + s->nnz, k, (size_t)len * sizeof(int32_t));
    s->nnz += len;
    s->dead[s->n] = 0;
    s->n++;
    s->off[s->n] = s->nnz;
    uint64_t i = list_key(k, len) & s->mask;
    while (s->slot[i] >= 0) i = (i + 1) & s->mask;
    s->slot[i] = s->n - 1;
    return s->n - 1;
}

static void cs_from_out(clset *s, const or_out *o) {
    cs_init(s, o->n_cl);
    for (int64_t c = 0; c < o->n_cl; ++c)
        cs_insert(s, o->vtx + o->off[c], (int32_t)(o->off[c + 1] - o->off[c]));
}

/* Algorithm 8: for every new clique c, split on each new edge inside c;
 * every resulting candidate that is an old maximal clique is reported once
 * and removed from C. */
static void imce_sub(const int32_t *hu, const int32_t *hv, int64_t rho, clset *C, const or_out *lnew, or_out *out) {
    uint64_t *keys = (uint64_t *)malloc((size_t)(rho + 1) * sizeof(uint64_t));
    for (int64_t i = 0; i < rho; ++i) keys[i] = ((uint64_t)(uint32_t)hu[i] << 32) | (uint32_t)hv[i];
    qsort(keys, (size_t)rho, sizeof(uint64_t), cmp_u64);
    int32_t *buf = NULL;
    int32_t bufcap = 0;
    for (int64_t c = 0; c < lnew->n_cl; ++c) {
        const int32_t *cv = lnew->vtx + lnew->off[c];
        int32_t len = (int32_t)(lnew->off[c + 1] - lnew->off[c]);
        if (len + 1 > bufcap) { bufcap = len + 1; buf = (int32_t *)realloc(buf, (size_t)bufcap * sizeof(int32_t)); }
        clset S;
        cs_init(&S, 4);
        cs_insert(&S, cv, len);
        for (int32_t a = 0; a < len; ++a)
            for (int32_t b = a + 1; b < len; ++b) {
                uint64_t key = ((uint64_t)(uint32_t)cv[a] << 32) | (uint32_t)cv[b];   /* cv sorted: cv[a] < cv[b] */
                int64_t lo = 0, hi = rho;
                while (lo < hi) { int64_t mid = lo + (hi - lo) / 2; if (keys[mid] < key) lo = mid + 1; else hi = mid; }
                if (!(lo < rho && keys[lo] == key)) continue;   /* e = (cv[a], cv[b]) ∈ E(c) ∩ H */
                clset S2;
                cs_init(&S2, S.n * 2);
                for (int64_t s = 0; s < S.n; ++s) {
                    const int32_t *sv = S.vtx + S.off[s];
                    int32_t sl = (int32_t)(S.off[s + 1] - S.off[s]);
                    if (contains(sv, sl, cv[a]) && contains(sv, sl, cv[b])) {
                        int32_t n1 = 0, n2 = 0;
                        for (int32_t t = 0; t < sl; ++t) if (sv[t] != cv[a]) buf[n1++] = sv[t];
                        cs_insert(&S2, buf, n1);       /* c' \ {u} */
                        for (int32_t t = 0; t < sl; ++t) if (sv[t] != cv[b]) buf[n2++] = sv[t];
                        cs_insert(&S2, buf, n2);       /* c' \ {v} */
                    } else {
                        cs_insert(&S2, sv, sl);
                    }
                }
                cs_free(&S);
                S = S2;
            }
        for (int64_t s = 0; s < S.n; ++s) {
            const int32_t *sv = S.vtx + S.off[s];
            int32_t sl = (int32_t)(S.off[s + 1] - S.off[s]);
            int64_t f = cs_find(C, sv, sl);
            if (f >= 0 && !C->dead[f]) {
                C->dead[f] = 1;
                emit(out, sv, sl);
            }
        }
        cs_free(&S);
    }
    free(buf);
    free(keys);
}

/* Mode B (the paper's algorithms) with the old cliques kept between
 * batches: the state holds G and C = C(G).  One batch: canonicalise H,
 * Λnew by Algorithms 6 + 9 on G+H, Λdel by Algorithm 8 against C, then
 * G := G+H and C := C \ Λdel ∪ Λnew. */
typedef struct {
    or_graph *g;
    clset C;
    int64_t alive;
    uint64_t seed;
} or_imce;

or_imce *or_imce_open(const or_graph *g0, uint64_t seed, int32_t threads) {
    or_imce *s = (or_imce *)calloc(1, sizeof(or_imce));
    s->seed = seed;
    /* private copy of G */
    int32_t *u = (int32_t *)malloc((size_t)(g0->nnz + 1) * sizeof(int32_t));
    int32_t *v = (int32_t *)malloc((size_t)(g0->nnz + 1) * sizeof(int32_t));
    int64_t k = 0;
    for (int32_t a = 0; a < g0->n; ++a)
        for (int64_t e = g0->row_ptr[a]; e < g0->row_ptr[a + 1]; ++e) { u[k] = a; v[k] = g0->col[e]; k++; }
    s->g = or_graph_from_pairs(g0->n, u, v, k);
    free(u);
    free(v);
    /* C(G) through the per-vertex decomposition (any rank gives C(G)); degree rank */
    double *key = (double *)malloc(((size_t)g0->n + 1) * sizeof(double));
    int32_t *rank = (int32_t *)malloc(((size_t)g0->n + 1) * sizeof(int32_t));
    for (int32_t a = 0; a < g0->n; ++a) key[a] = (double)deg(g0, a);
    or_rank_from_key(g0->n, key, rank);
    or_out *all = or_out_new(1, seed);
    or_parmce(s->g, rank, NULL, 0, threads, all, NULL, NULL, NULL, 0, NULL);
    cs_from_out(&s->C, all);
    s->alive = all->n_cl;
    or_out_free(all);
    free(key);
    free(rank);
    return s;
}

void or_imce_close(or_imce *s) {
    if (!s) return;
    or_graph_free(s->g);
    cs_free(&s->C);
    free(s);
}

const or_graph *or_imce_graph(const or_imce *s) { return s->g; }
int64_t or_imce_alive(const or_imce *s) { return s->alive; }

/* Returns the number of edges applied (ρ), or -1 on an invalid vertex id
 * (nothing is changed then). */
int64_t or_imce_add(or_imce *s, const int32_t *u, const int32_t *v, int64_t k, or_out *new_out, or_out *del_out) {
    int32_t *hu = (int32_t *)malloc((size_t)(k + 1) * sizeof(int32_t));
    int32_t *hv = (int32_t *)malloc((size_t)(k + 1) * sizeof(int32_t));
    int64_t rho = or_canonical_batch(s->g, u, v, k, hu, hv);
    if (rho < 0) { free(hu); free(hv); return -1; }
    or_graph *gp = graph_plus(s->g, hu, hv, rho);
    or_out *lnew = or_out_new(1, s->seed);
    imce_new(gp, hu, hv, rho, lnew);
    or_out *ldel = or_out_new(1, s->seed);
    imce_sub(hu, hv, rho, &s->C, lnew, ldel);
    for (int64_t c = 0; c < lnew->n_cl; ++c) {
        int64_t id = cs_insert(&s->C, lnew->vtx + lnew->off[c], (int32_t)(lnew->off[c + 1] - lnew->off[c]));
        s->C.dead[id] = 0;
    }
    s->alive += lnew->n_cl - ldel->n_cl;
    out_merge(new_out, lnew);
    out_merge(del_out, ldel);
    or_out_free(lnew);
    or_out_free(ldel);
    or_graph_free(s->g);
    s->g = gp;
    free(hu);
    free(hv);
    return rho;
}

/* One-shot mode B with C(G) from whole-graph TTT (Algorithm 1); hu/hv must
 * already be a canonical batch (or_canonical_batch). */
void or_imce_alg(const or_graph *g, const int32_t *hu, const int32_t *hv, int64_t rho,
                 or_out *new_out, or_out *del_out) {
    or_graph *gp = graph_plus(g, hu, hv, rho);
    or_out *lnew = or_out_new(1, new_out->seed);
    imce_new(gp, hu, hv, rho, lnew);
    out_merge(new_out, lnew);
    or_out *old = or_out_new(1, new_out->seed);
    or_ttt_whole(g, old);
    clset C;
    cs_from_out(&C, old);
    imce_sub(hu, hv, rho, &C, lnew, del_out);
    cs_free(&C);
    or_out_free(old);
    or_out_free(lnew);
    or_graph_free(gp);
}

/* Alive cliques of the state (sorted lists) into an accumulator. */
void or_imce_cliques(const or_imce *s, or_out *out) {
    for (int64_t c = 0; c < s->C.n; ++c)
        if (!s->C.dead[c]) emit(out, s->C.vtx + s->C.off[c], (int32_t)(s->C.off[c + 1] - s->C.off[c]));
}

/* Mode A (plain definition): Λnew = C(G+H) \ C(G), Λdel = C(G) \ C(G+H). */
void or_imce_diff(const or_graph *g, const int32_t *hu, const int32_t *hv, int64_t rho,
                  or_out *new_out, or_out *del_out) {
    or_graph *gp = graph_plus(g, hu, hv, rho);
    or_out *a = or_out_new(1, new_out->seed), *b = or_out_new(1, new_out->seed);
    or_ttt_whole(g, a);
    or_ttt_whole(gp, b);
    clset A, B;
    cs_from_out(&A, a);
    cs_from_out(&B, b);
    for (int64_t c = 0; c < b->n_cl; ++c) {
        const int32_t *k = b->vtx + b->off[c];
        int32_t len = (int32_t)(b->off[c + 1] - b->off[c]);
        if (cs_find(&A, k, len) < 0) emit(new_out, k, len);
    }
    for (int64_t c = 0; c < a->n_cl; ++c) {
        const int32_t *k = a->vtx + a->off[c];
        int32_t len = (int32_t)(a->off[c + 1] - a->off[c]);
        if (cs_find(&B, k, len) < 0) emit(del_out, k, len);
    }
    cs_free(&A);
    cs_free(&B);
    or_out_free(a);
    or_out_free(b);
    or_graph_free(gp);
}

/* G+H as a new graph (for chaining batches in tests). */
or_graph *or_graph_plus(const or_graph *g, const int32_t *hu, const int32_t *hv, int64_t rho) {
    return graph_plus(g, hu, hv, rho);
}

/* ------------------------------------------------------------------ */
/* decremental maintenance: edge deletions by reduction to additions   */
/* ------------------------------------------------------------------ */
/*
 * Deleting a batch H from G gives G' = G - H, and G = G' + H.  By Section 5
 * applied to (G', H): C(G) = C(G') \ Λdel ∪ Λnew, with Λnew the maximal
 * cliques of G containing an edge of H and Λdel the cliques of C(G') that are
 * not maximal in G.  Hence the deletion removes Λnew and creates Λdel:
 *   removed = Algorithm 6 (with Algorithm 9) run on G and H;
 *   created = Algorithm 8's splits of every removed clique on its H edges,
 *             keeping each split that is a maximal clique of G' (Algorithm 8
 *             tests membership in C(G'); the reduction does not hold C(G'),
 *             and for a clique of G' membership is maximality).
 * Deletion batches keep pairs that are edges of G, in arrival order; self
 * loops, non-edges and repeats are dropped.
 */

int64_t or_canonical_deletion(const or_graph *g, const int32_t *u, const int32_t *v, int64_t k,
                              int32_t *hu, int32_t *hv) {
    uint64_t cap = 16;
    while (cap < (uint64_t)k * 2 + 16) cap <<= 1;
    uint64_t *seen = (uint64_t *)malloc(cap * sizeof(uint64_t));
    memset(seen, 0xff, cap * sizeof(uint64_t));
    int64_t kept = 0;
    for (int64_t i = 0; i < k; ++i) {
        if (u[i] < 0 || u[i] >= g->n || v[i] < 0 || v[i] >= g->n) { free(seen); return -1; }
        if (u[i] == v[i]) continue;
        int32_t a = u[i] < v[i] ? u[i] : v[i], b = u[i] < v[i] ? v[i] : u[i];
        if (!has_edge(g, a, b)) continue;
        uint64_t key = ((uint64_t)(uint32_t)a << 32) | (uint32_t)b;
        uint64_t h = fmix(key) & (cap - 1);
        int dup = 0;
        while (seen[h] != UINT64_MAX) {
            if (seen[h] == key) { dup = 1; break; }
            h = (h + 1) & (cap - 1);
        }
        if (dup) continue;
        seen[h] = key;
        hu[kept] = a;
        hv[kept] = b;
        kept++;
    }
    free(seen);
    return kept;
}

static or_graph *graph_minus(const or_graph *g, const int32_t *hu, const int32_t *hv, int64_t rho) {
    uint64_t *keys = (uint64_t *)malloc((size_t)(rho + 1) * sizeof(uint64_t));
    for (int64_t i = 0; i < rho; ++i) keys[i] = ((uint64_t)(uint32_t)hu[i] << 32) | (uint32_t)hv[i];
    qsort(keys, (size_t)rho, sizeof(uint64_t), cmp_u64);
    int32_t *u = (int32_t *)malloc((size_t)(g->nnz + 1) * sizeof(int32_t));
    int32_t *v = (int32_t *)malloc((size_t)(g->nnz + 1) * sizeof(int32_t));
    int64_t k = 0;
    for (int32_t a = 0; a < g->n; ++a)
        for (int64_t e = g->row_ptr[a]; e < g->row_ptr[a + 1]; ++e) {
            int32_t b = g->col[e];
            int32_t x = a < b ? a : b, y = a < b ? b : a;
            uint64_t key = ((uint64_t)(uint32_t)x << 32) | (uint32_t)y;
            int64_t lo = 0, hi = rho;
            while (lo < hi) { int64_t mid = lo + (hi - lo) / 2; if (keys[mid] < key) lo = mid + 1; else hi = mid; }
            if (lo < rho && keys[lo] == key) continue;
            u[k] = a;
            v[k] = b;
            k++;
        }
    or_graph *gm = or_graph_from_pairs(g->n, u, v, k);
    free(u);
    free(v);
    free(keys);
    return gm;
}

/* K (sorted, a clique of g) is maximal iff no vertex outside K is adjacent
 * to all of K */
static int is_maximal(const or_graph *g, const int32_t *k, int32_t len) {
    int32_t best = 0;
    for (int32_t i = 1; i < len; ++i) if (deg(g, k[i]) < deg(g, k[best])) best = i;
    const int32_t *nb = nbr(g, k[best]);
    int32_t d = deg(g, k[best]);
    for (int32_t t = 0; t < d; ++t) {
        int32_t w = nb[t];
        if (contains(k, len, w)) continue;
        int all = 1;
        for (int32_t i = 0; i < len && all; ++i)
            if (i != best && !has_edge(g, w, k[i])) all = 0;
        if (all) return 0;
    }
    return 1;
}

/* Algorithm 8's splits of every removed clique on its H edges; the splits
 * that are maximal in G' are the created cliques (each reported once). */
static void dmce_created(const int32_t *hu, const int32_t *hv, int64_t rho, const or_graph *gm,
                         const or_out *removed, or_out *out) {
    uint64_t *keys = (uint64_t *)malloc((size_t)(rho + 1) * sizeof(uint64_t));
    for (int64_t i = 0; i < rho; ++i) keys[i] = ((uint64_t)(uint32_t)hu[i] << 32) | (uint32_t)hv[i];
    qsort(keys, (size_t)rho, sizeof(uint64_t), cmp_u64);
    clset done;
    cs_init(&done, removed->n_cl * 2 + 4);
    int32_t *buf = NULL;
    int32_t bufcap = 0;
    for (int64_t c = 0; c < removed->n_cl; ++c) {
        const int32_t *cv = removed->vtx + removed->off[c];
        int32_t len = (int32_t)(removed->off[c + 1] - removed->off[c]);
        if (len + 1 > bufcap) { bufcap = len + 1; buf = (int32_t *)realloc(buf, (size_t)bufcap * sizeof(int32_t)); }
        clset S;
        cs_init(&S, 4);
        cs_insert(&S, cv, len);
        for (int32_t a = 0; a < len; ++a)
            for (int32_t b = a + 1; b < len; ++b) {
                uint64_t key = ((uint64_t)(uint32_t)cv[a] << 32) | (uint32_t)cv[b];
                int64_t lo = 0, hi = rho;
                while (lo < hi) { int64_t mid = lo + (hi - lo) / 2; if (keys[mid] < key) lo = mid + 1; else hi = mid; }
                if (!(lo < rho && keys[lo] == key)) continue;   /* (cv[a], cv[b]) is a deleted edge */
                clset S2;
                cs_init(&S2, S.n * 2);
                for (int64_t t = 0; t < S.n; ++t) {
                    const int32_t *sv = S.vtx + S.off[t];
                    int32_t sl = (int32_t)(S.off[t + 1] - S.off[t]);
                    if (contains(sv, sl, cv[a]) && contains(sv, sl, cv[b])) {
                        int32_t n1 = 0, n2 = 0;
                        for (int32_t x = 0; x < sl; ++x) if (sv[x] != cv[a]) buf[n1++] = sv[x];
                        cs_insert(&S2, buf, n1);
                        for (int32_t x = 0; x < sl; ++x) if (sv[x] != cv[b]) buf[n2++] = sv[x];
                        cs_insert(&S2, buf, n2);
                    } else {
                        cs_insert(&S2, sv, sl);
                    }
                }
                cs_free(&S);
                S = S2;
            }
        for (int64_t t = 0; t < S.n; ++t) {
            const int32_t *sv = S.vtx + S.off[t];
            int32_t sl = (int32_t)(S.off[t + 1] - S.off[t]);
            if (sl == 0 || cs_find(&done, sv, sl) >= 0) continue;
            cs_insert(&done, sv, sl);
            if (is_maximal(gm, sv, sl)) emit(out, sv, sl);
        }
        cs_free(&S);
    }
    cs_free(&done);
    free(buf);
    free(keys);
}

/* One-shot, algorithmic: (removed, created) for a canonical deletion batch. */
void or_dmce_alg(const or_graph *g, const int32_t *hu, const int32_t *hv, int64_t rho,
                 or_out *removed_out, or_out *created_out) {
    or_out *rem = or_out_new(1, removed_out->seed);
    imce_new(g, hu, hv, rho, rem);   /* maximal cliques of G = G' + H through an edge of H */
    or_graph *gm = graph_minus(g, hu, hv, rho);
    dmce_created(hu, hv, rho, gm, rem, created_out);
    out_merge(removed_out, rem);
    or_out_free(rem);
    or_graph_free(gm);
}

/* One-shot, plain definition: removed = C(G) \ C(G - H), created = C(G - H) \ C(G). */
void or_dmce_diff(const or_graph *g, const int32_t *hu, const int32_t *hv, int64_t rho,
                  or_out *removed_out, or_out *created_out) {
    or_graph *gm = graph_minus(g, hu, hv, rho);
    or_out *a = or_out_new(1, removed_out->seed), *b = or_out_new(1, removed_out->seed);
    or_ttt_whole(g, a);
    or_ttt_whole(gm, b);
    clset A, B;
    cs_from_out(&A, a);
    cs_from_out(&B, b);
    for (int64_t c = 0; c < a->n_cl; ++c) {
        const int32_t *k = a->vtx + a->off[c];
        int32_t len = (int32_t)(a->off[c + 1] - a->off[c]);
        if (cs_find(&B, k, len) < 0) emit(removed_out, k, len);
    }
    for (int64_t c = 0; c < b->n_cl; ++c) {
        const int32_t *k = b->vtx + b->off[c];
        int32_t len = (int32_t)(b->off[c + 1] - b->off[c]);
        if (cs_find(&A, k, len) < 0) emit(created_out, k, len);
    }
    cs_free(&A);
    cs_free(&B);
    or_out_free(a);
    or_out_free(b);
    or_graph_free(gm);
}

/* Stateful deletion batch on the incremental state (C = C(G) kept): returns
 * the number of edges deleted, or -1 on an invalid id (nothing changed). */
int64_t or_imce_remove(or_imce *s, const int32_t *u, const int32_t *v, int64_t k, or_out *removed_out,
                       or_out *created_out) {
    int32_t *hu = (int32_t *)malloc((size_t)(k + 1) * sizeof(int32_t));
    int32_t *hv = (int32_t *)malloc((size_t)(k + 1) * sizeof(int32_t));
    int64_t rho = or_canonical_deletion(s->g, u, v, k, hu, hv);
    if (rho < 0) { free(hu); free(hv); return -1; }
    or_out *rem = or_out_new(1, s->seed);
    imce_new(s->g, hu, hv, rho, rem);
    or_graph *gm = graph_minus(s->g, hu, hv, rho);
    or_out *cre = or_out_new(1, s->seed);
    dmce_created(hu, hv, rho, gm, rem, cre);
    for (int64_t c = 0; c < rem->n_cl; ++c) {
        int64_t f = cs_find(&s->C, rem->vtx + rem->off[c], (int32_t)(rem->off[c + 1] - rem->off[c]));
        if (f >= 0) s->C.dead[f] = 1;
    }
    for (int64_t c = 0; c < cre->n_cl; ++c) {
        int64_t id = cs_insert(&s->C, cre->vtx + cre->off[c], (int32_t)(cre->off[c + 1] - cre->off[c]));
        s->C.dead[id] = 0;
    }
    s->alive += cre->n_cl - rem->n_cl;
    out_merge(removed_out, rem);
    out_merge(created_out, cre);
    or_out_free(rem);
    or_out_free(cre);
    or_graph_free(s->g);
    s->g = gm;
    free(hu);
    free(hv);
    return rho;
}

/* G - H as a new graph (for chaining batches in tests). */
or_graph *or_graph_minus(const or_graph *g, const int32_t *hu, const int32_t *hv, int64_t rho) {
    return graph_minus(g, hu, hv, rho);
}
