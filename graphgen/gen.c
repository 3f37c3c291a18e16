/*
 * Seeded synthetic graph generators.
 *
 * This module only draws random inputs: raw edge samples (which may contain
 * self-loops and repeated pairs), planted cliques and edge streams.  It holds
 * none of the enumeration arithmetic; turning samples into a simple undirected
 * graph is done separately by each consumer (Section 3 of the paper: a simple
 * undirected graph without self loops or multiple edges; Section 6.1: inputs
 * are normalised by dropping self loops, weights, parallel edges and
 * directions).
 *
 * Random numbers: splitmix64 (for seeding) and xoshiro256** (for streams), both
 * as published by S. Vigna (prng.di.unimi.it).  Uniform doubles are
 * (x >> 11) * 2^-53, so a Bernoulli(p) test "u < p" is exact on every host.
 * Generators that take logarithms or powers (log-uniform sizes, Chung-Lu skip
 * sampling) use the host's libm; the library is compiled with
 * -ffp-contract=off so that x86-64 and aarch64 agree except in the rare case
 * where libm itself differs in the last bit.
 *
 * All functions return malloc'd arrays that the caller releases with gg_free.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------- random number generation ---------------- */

static uint64_t splitmix64_next(uint64_t *state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

typedef struct { uint64_t s[4]; } xoshiro;

static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t xo_next(xoshiro *r) {
    uint64_t *s = r->s;
    const uint64_t result = rotl(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl(s[3], 45);
    return result;
}

static void xo_seed(xoshiro *r, uint64_t seed) {
    uint64_t st = seed;
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64_next(&st);
}

/* uniform double in [0, 1) with 53 random bits */
static double xo_unif(xoshiro *r) { return (double)(xo_next(r) >> 11) * 0x1.0p-53; }

/* uniform integer in [0, k) by rejection (unbiased) */
static uint64_t xo_below(xoshiro *r, uint64_t k) {
    uint64_t lim = UINT64_MAX - (UINT64_MAX % k);
    uint64_t x;
    do { x = xo_next(r); } while (x >= lim);
    return x % k;
}

/* seed of sub-stream k derived from a base seed */
uint64_t gg_substream_seed(uint64_t base, uint64_t k) {
    uint64_t st = base ^ (k * 0xD1B54A32D192ED03ULL);
    return splitmix64_next(&st);
}

/* ---------------- growable edge buffer ---------------- */

typedef struct { int32_t *u, *v; int64_t m, cap; } ebuf;

static int eb_push(ebuf *b, int32_t u, int32_t v) {
    if (b->m == b->cap) {
        int64_t nc = b->cap ? b->cap * 2 : 1024;
        int32_t *nu = (int32_t *)realloc(b->u, (size_t)nc * sizeof(int32_t));
        if (!nu) return -1;
        b->u = nu;
        int32_t *nv = (int32_t *)realloc(b->v, (size_t)nc * sizeof(int32_t));
        if (!nv) return -1;
        b->v = nv;
        b->cap = nc;
    }
    b->u[b->m] = u;
    b->v[b->m] = v;
    b->m++;
    return 0;
}

void gg_free(void *p) { free(p); }

/* ---------------- Erdos-Renyi G(n, p) ----------------
 * One draw per unordered pair (i, j), i < j, in lexicographic order; the pair
 * is an edge iff the draw is below p.  Output pairs have i < j. */
int64_t gg_er(int32_t n, double p, uint64_t seed, int32_t **u_out, int32_t **v_out) {
    xoshiro r;
    xo_seed(&r, seed);
    ebuf b = {0};
    for (int32_t i = 0; i < n; ++i)
        for (int32_t j = i + 1; j < n; ++j)
            if (xo_unif(&r) < p && eb_push(&b, i, j)) return -1;
    *u_out = b.u;
    *v_out = b.v;
    return b.m;
}

/* ---------------- R-MAT ----------------
 * `samples` edge samples over 2^scale vertices; each sample descends `scale`
 * levels, choosing quadrant (0,0),(0,1),(1,0),(1,1) with probabilities
 * a, b, c, 1-a-b-c from one uniform draw per level.  No noise, no vertex
 * permutation.  Samples may be self-loops or repeats. */
int64_t gg_rmat(int32_t scale, int64_t samples, double a, double b, double c, uint64_t seed,
                int32_t **u_out, int32_t **v_out) {
    xoshiro r;
    xo_seed(&r, seed);
    int32_t *u = (int32_t *)malloc((size_t)samples * sizeof(int32_t));
    int32_t *v = (int32_t *)malloc((size_t)samples * sizeof(int32_t));
    if (!u || !v) { free(u); free(v); return -1; }
    const double ab = a + b, abc = a + b + c;
    for (int64_t s = 0; s < samples; ++s) {
        int32_t x = 0, y = 0;
        for (int32_t l = 0; l < scale; ++l) {
            double d = xo_unif(&r);
            int bx, by;
            if (d < a) { bx = 0; by = 0; }
            else if (d < ab) { bx = 0; by = 1; }
            else if (d < abc) { bx = 1; by = 0; }
            else { bx = 1; by = 1; }
            x = (x << 1) | bx;
            y = (y << 1) | by;
        }
        u[s] = x;
        v[s] = y;
    }
    *u_out = u;
    *v_out = v;
    return samples;
}

/* ---------------- Chung-Lu expected-degree graphs ----------------
 * Weights w_i = wmax * ((i + i0) / i0)^(-1/(gamma-1)), i = 0..n-1 (decreasing),
 * with i0 > 0 chosen by bisection so that sum_i w_i = 2 * m_target.
 * Pair (i, j), i < j, is an edge with probability min(1, w_i w_j / S),
 * S = sum w, sampled with the skip method of Miller and Hagberg (2011,
 * "Efficient generation of networks with given expected degrees"). */
static double cl_weight(double wmax, double beta, double i0, int64_t i) {
    return wmax * pow(((double)i + i0) / i0, -beta);
}

static double cl_sum(int32_t n, double wmax, double beta, double i0) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += cl_weight(wmax, beta, i0, i);
    return s;
}

double gg_chung_lu_i0(int32_t n, double gamma, double wmax, double m_target) {
    const double beta = 1.0 / (gamma - 1.0);
    double lo = 1e-6, hi = (double)n;
    const double want = 2.0 * m_target;
    for (int it = 0; it < 64; ++it) {   /* sum grows with i0 */
        double mid = 0.5 * (lo + hi);
        if (cl_sum(n, wmax, beta, mid) < want) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

int64_t gg_chung_lu(int32_t n, double gamma, double wmax, double m_target, uint64_t seed,
                    int32_t **u_out, int32_t **v_out, double **w_out) {
    const double beta = 1.0 / (gamma - 1.0);
    const double i0 = gg_chung_lu_i0(n, gamma, wmax, m_target);
    double *w = (double *)malloc((size_t)n * sizeof(double));
    if (!w) return -1;
    double S = 0.0;
    for (int64_t i = 0; i < n; ++i) { w[i] = cl_weight(wmax, beta, i0, i); S += w[i]; }
    xoshiro r;
    xo_seed(&r, seed);
    ebuf b = {0};
    for (int32_t i = 0; i + 1 < n; ++i) {
        int64_t j = i + 1;
        double p = w[i] * w[j] / S;
        if (p > 1.0) p = 1.0;
        while (j < n && p > 0.0) {
            if (p != 1.0) {
                double rr = xo_unif(&r);
                double skip = floor(log1p(-rr) / log1p(-p));
                if (skip >= (double)(n - j)) break;
                j += (int64_t)skip;
            }
            if (j >= n) break;
            double q = w[i] * w[j] / S;
            if (q > 1.0) q = 1.0;
            if (xo_unif(&r) < q / p && eb_push(&b, i, (int32_t)j)) { free(w); return -1; }
            p = q;
            j += 1;
        }
    }
    *u_out = b.u;
    *v_out = b.v;
    if (w_out) *w_out = w; else free(w);
    return b.m;
}

/* ---------------- planted cliques ----------------
 * `count` cliques, size uniform in [kmin, kmax], vertices drawn uniformly
 * without replacement from [0, n); all pairs (a, b), a < b, are emitted. */
int64_t gg_planted_cliques(int32_t n, int32_t count, int32_t kmin, int32_t kmax, uint64_t seed,
                           int32_t **u_out, int32_t **v_out) {
    xoshiro r;
    xo_seed(&r, seed);
    ebuf b = {0};
    int32_t *members = (int32_t *)malloc((size_t)(kmax > 0 ? kmax : 1) * sizeof(int32_t));
    if (!members) return -1;
    for (int32_t t = 0; t < count; ++t) {
        int32_t k = kmin + (int32_t)xo_below(&r, (uint64_t)(kmax - kmin + 1));
        int32_t got = 0;
        while (got < k) {   /* rejection keeps the draw without replacement */
            int32_t x = (int32_t)xo_below(&r, (uint64_t)n);
            int dup = 0;
            for (int32_t s = 0; s < got; ++s) dup |= (members[s] == x);
            if (!dup) members[got++] = x;
        }
        for (int32_t s = 0; s < k; ++s)
            for (int32_t q = s + 1; q < k; ++q) {
                int32_t a = members[s] < members[q] ? members[s] : members[q];
                int32_t c = members[s] < members[q] ? members[q] : members[s];
                if (eb_push(&b, a, c)) { free(members); return -1; }
            }
    }
    free(members);
    *u_out = b.u;
    *v_out = b.v;
    return b.m;
}

/* ---------------- many independent G(n, p) ----------------
 * Graph g uses its own stream seeded by gg_substream_seed(seed, g).  From that
 * stream: n_g = round(exp(U[ln nmin, ln nmax])), p_g = pmin + (pmax-pmin) U,
 * then one draw per pair as in gg_er.  Vertex ids are offset so the graphs
 * are disjoint; graph_ptr[g] is the first vertex of graph g (k+1 entries). */
int64_t gg_batched_er(int32_t k, int32_t nmin, int32_t nmax, double pmin, double pmax, uint64_t seed,
                      int32_t *graph_ptr, double *p_out, int32_t **u_out, int32_t **v_out) {
    ebuf b = {0};
    int32_t base = 0;
    const double lmin = log((double)nmin), lmax = log((double)nmax);
    for (int32_t g = 0; g < k; ++g) {
        xoshiro r;
        xo_seed(&r, gg_substream_seed(seed, (uint64_t)g));
        int32_t ng = (int32_t)floor(exp(lmin + (lmax - lmin) * xo_unif(&r)) + 0.5);
        if (ng < nmin) ng = nmin;
        if (ng > nmax) ng = nmax;
        double pg = pmin + (pmax - pmin) * xo_unif(&r);
        graph_ptr[g] = base;
        if (p_out) p_out[g] = pg;
        for (int32_t i = 0; i < ng; ++i)
            for (int32_t j = i + 1; j < ng; ++j)
                if (xo_unif(&r) < pg && eb_push(&b, base + i, base + j)) return -1;
        base += ng;
    }
    graph_ptr[k] = base;
    *u_out = b.u;
    *v_out = b.v;
    return b.m;
}

/* ---------------- edge stream for the dynamic workload ----------------
 * `count` new edges with endpoints drawn independently with probability
 * proportional to weight w (inverse-CDF by binary search on prefix sums);
 * self-loops, pairs present in the base graph (given as sorted canonical
 * 64-bit keys a<<32|b, a<b) and repeats within the stream are rejected and
 * redrawn.  Output pairs are canonical (u < v) in arrival order. */
static int key_in_sorted(const uint64_t *keys, int64_t n, uint64_t key) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (keys[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo < n && keys[lo] == key;
}

typedef struct { uint64_t *slot; uint64_t mask; } kset;

static int kset_insert(kset *s, uint64_t key) {   /* 1 if newly inserted */
    uint64_t h = key * 0x9E3779B97F4A7C15ULL;
    uint64_t i = (h ^ (h >> 29)) & s->mask;
    for (;;) {
        if (s->slot[i] == UINT64_MAX) { s->slot[i] = key; return 1; }
        if (s->slot[i] == key) return 0;
        i = (i + 1) & s->mask;
    }
}

int64_t gg_edge_stream(int32_t n, const double *w, const uint64_t *base_keys, int64_t n_base,
                       int64_t count, uint64_t seed, int32_t **u_out, int32_t **v_out) {
    double *cdf = (double *)malloc((size_t)n * sizeof(double));
    int32_t *u = (int32_t *)malloc((size_t)count * sizeof(int32_t));
    int32_t *v = (int32_t *)malloc((size_t)count * sizeof(int32_t));
    uint64_t cap = 1;
    while (cap < (uint64_t)count * 2 + 2) cap <<= 1;
    kset seen = {(uint64_t *)malloc(cap * sizeof(uint64_t)), cap - 1};
    if (!cdf || !u || !v || !seen.slot) { free(cdf); free(u); free(v); free(seen.slot); return -1; }
    memset(seen.slot, 0xff, cap * sizeof(uint64_t));
    double acc = 0.0;
    for (int32_t i = 0; i < n; ++i) { acc += w[i]; cdf[i] = acc; }
    xoshiro r;
    xo_seed(&r, seed);
    int64_t got = 0;
    while (got < count) {
        int32_t e[2];
        for (int t = 0; t < 2; ++t) {
            double x = xo_unif(&r) * acc;
            int32_t lo = 0, hi = n - 1;
            while (lo < hi) {
                int32_t mid = lo + (hi - lo) / 2;
                if (cdf[mid] <= x) lo = mid + 1; else hi = mid;
            }
            e[t] = lo;
        }
        if (e[0] == e[1]) continue;
        int32_t a = e[0] < e[1] ? e[0] : e[1], c = e[0] < e[1] ? e[1] : e[0];
        uint64_t key = ((uint64_t)(uint32_t)a << 32) | (uint32_t)c;
        if (key_in_sorted(base_keys, n_base, key)) continue;
        if (!kset_insert(&seen, key)) continue;
        u[got] = a;
        v[got] = c;
        got++;
    }
    free(cdf);
    free(seen.slot);
    *u_out = u;
    *v_out = v;
    return got;
}

/* ---------------- batch sizes and arrival gaps ----------------
 * sizes[i] = round(exp(U[ln lo, ln hi])) until their sum reaches `total`
 * (the last batch is truncated); gaps[i] ~ Exp(1) (unit-rate Poisson process
 * inter-arrival times; the caller scales by 1/lambda).  Returns #batches. */
int64_t gg_batch_schedule(int64_t total, double lo, double hi, uint64_t seed,
                          int64_t **sizes_out, double **gaps_out) {
    xoshiro r;
    xo_seed(&r, seed);
    int64_t cap = 64, nb = 0, sum = 0;
    int64_t *sizes = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
    double *gaps = (double *)malloc((size_t)cap * sizeof(double));
    if (!sizes || !gaps) { free(sizes); free(gaps); return -1; }
    const double llo = log(lo), lhi = log(hi);
    while (sum < total) {
        if (nb == cap) {
            cap *= 2;
            int64_t *ns = (int64_t *)realloc(sizes, (size_t)cap * sizeof(int64_t));
            double *ng = (double *)realloc(gaps, (size_t)cap * sizeof(double));
            if (!ns || !ng) { free(ns ? ns : sizes); free(ng ? ng : gaps); return -1; }
            sizes = ns;
            gaps = ng;
        }
        int64_t s = (int64_t)floor(exp(llo + (lhi - llo) * xo_unif(&r)) + 0.5);
        if (s < 1) s = 1;
        if (sum + s > total) s = total - sum;
        sizes[nb] = s;
        gaps[nb] = -log1p(-xo_unif(&r));
        sum += s;
        nb++;
    }
    *sizes_out = sizes;
    *gaps_out = gaps;
    return nb;
}
