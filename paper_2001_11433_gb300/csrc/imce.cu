// Incremental maximal cliques for edge additions (Section 5).
//
// imce_state keeps G and C(G) on the device.  C(G) lives in a clique index:
// a pool of sorted vertex lists (pool[off] = size, the vertices follow), an
// alive flag per clique, and an open-addressing hash table from H(K) to the
// clique id (Theorem 1's concurrent hash table; lookups verify the list).
//
// imce_add_edges, one batch H:
//   1. canonicalise (arrival order e_1..e_ρ; self loops, edges of G and
//      repeats dropped)                                     k_batch_keys ...
//   2. G' = G + H by a per-row merge                         k_merge_rows
//   3. Λnew: Algorithm 6, one search per new edge with the exclusion of
//      Algorithm 7, on the persistent engine (bk.cu, BK_IMCE)
//   4. Λdel: Algorithm 8 per new clique — split on its new edges, probe the
//      index, claim alive old cliques once (CAS)             k_imce_sub
//   5. index := index \ Λdel ∪ Λnew, G := G'.
// Steps 1-4 leave the state untouched until everything succeeded; a failure
// restores the alive flags claimed in step 4.
//
// imce_remove_edges, one deletion batch H (edges of G), by the paper's
// reduction to additions (G = (G - H) + H):
//   removed = C(G) \ C(G - H): the cliques of G through an edge of H, step 3
//             run on G itself;
//   created = C(G - H) \ C(G): Algorithm 8's splits of the removed cliques
//             that are maximal in G - H, each once           k_dmce_created
// then the removed cliques leave the index, the created ones enter it, and
// G := G - H, all or nothing.
#include <string.h>

#include <vector>

#include "mce_host.h"

namespace mce {

struct CliqueIndex {
    int32_t *pool = nullptr;   // [size, v1..vs] per clique
    int64_t pool_words = 0, pool_cap = 0;
    int64_t *off = nullptr;    // per clique id
    int32_t *alive = nullptr;  // per clique id
    int64_t n_ids = 0, ids_cap = 0;
    unsigned long long *tkey = nullptr;   // table: key
    int32_t *tid = nullptr;               // table: id + 1 (0 = empty)
    int64_t tcap = 0;                     // power of two
    int64_t n_alive = 0;
};

}  // namespace mce

struct imce_state {
    mce_graph *g = nullptr;
    mce::CliqueIndex idx;
    uint64_t seed = 0;
    mce_opts opts{};
    cudaStream_t s = nullptr;
};

namespace mce {

namespace {

constexpr uint32_t FULL = 0xffffffffu;
constexpr int kSubMaxWords = 4;          // Algorithm 8 masks: up to 256 endpoints of new edges in a clique
constexpr int kSubCap = 4096;            // candidates per new clique

__device__ __forceinline__ int lower_bound_i32(const int32_t *a, int n, int32_t x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// ------------------------------------------------------------------ canonical batch

__global__ void k_batch_keys(const int32_t *u, const int32_t *v, int64_t k, int32_t n, const int32_t *row_ptr,
                             const int32_t *col, int32_t B, int32_t IB, int32_t present, uint64_t *keys, int32_t *bad) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a0 = u[i], b0 = v[i];
        uint64_t key = ~0ULL;
        if (a0 < 0 || a0 >= n || b0 < 0 || b0 >= n) {
            atomicOr(bad, 1);
        } else if (a0 != b0) {
            const int32_t a = min(a0, b0), b = max(a0, b0);
            const int32_t r0 = row_ptr[a], d = row_ptr[a + 1] - r0;
            const int p = lower_bound_i32(col + r0, d, b);
            const bool in_g = p < d && col[r0 + p] == b;
            if (in_g == (present != 0)) key = ((((uint64_t)a << B) | (uint64_t)b) << IB) | (uint64_t)i;
        }
        keys[i] = key;
    }
}

// keep[i] = 1 for the first arrival of each new pair
__global__ void k_first_arrival(const uint64_t *keys, int64_t k, int32_t IB, int32_t *keep) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = keys[j];
        if (key == ~0ULL) continue;
        if (j == 0 || (keys[j - 1] >> IB) != (key >> IB)) keep[key & ((1ULL << IB) - 1)] = 1;
    }
}

__global__ void k_emit_batch(const int32_t *u, const int32_t *v, const int32_t *keep_scan, int64_t k, int32_t *eu,
                             int32_t *ev) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
        if (keep_scan[i + 1] != keep_scan[i]) {
            const int32_t a = min(u[i], v[i]), b = max(u[i], v[i]);
            eu[keep_scan[i]] = a;
            ev[keep_scan[i]] = b;
        }
    }
}

// directed new pairs (x, y, index) as keys for the batch adjacency
__global__ void k_h_keys(const int32_t *eu, const int32_t *ev, int32_t rho, int32_t B, int32_t IB, uint64_t *keys,
                         int32_t *hdeg) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rho; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t a = (uint64_t)eu[i], b = (uint64_t)ev[i];
        keys[2 * i] = (((a << B) | b) << IB) | (uint64_t)i;
        keys[2 * i + 1] = (((b << B) | a) << IB) | (uint64_t)i;
        atomicAdd(&hdeg[a], 1);
        atomicAdd(&hdeg[b], 1);
    }
}

__global__ void k_h_fill(const uint64_t *keys, int64_t k2, int32_t B, int32_t IB, int32_t *h_adj, int32_t *h_idx) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k2; j += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = keys[j];
        h_idx[j] = (int32_t)(key & ((1ULL << IB) - 1));
        h_adj[j] = (int32_t)((key >> IB) & ((1ULL << B) - 1));
    }
}

__global__ void k_add_deg(const int32_t *row_ptr, const int32_t *hdeg, int32_t n, int32_t *deg2) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
        deg2[x] = row_ptr[x + 1] - row_ptr[x] + hdeg[x];
}

// Row x of G' = merge of the old row and the new neighbours (disjoint, sorted).
__global__ void k_merge_rows(const int32_t *row_ptr, const int32_t *col, const int32_t *h_ptr, const int32_t *h_adj,
                             const int32_t *row_ptr2, int32_t n, int32_t *col2) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = warp; x < n; x += nw) {
        const int32_t o0 = row_ptr[x], od = row_ptr[x + 1] - o0;
        const int32_t n0 = h_ptr[x], nd = h_ptr[x + 1] - n0;
        const int32_t dst = row_ptr2[x];
        for (int i = lane; i < od; i += 32) {
            const int32_t val = col[o0 + i];
            col2[dst + i + (nd ? lower_bound_i32(h_adj + n0, nd, val) : 0)] = val;
        }
        for (int j = lane; j < nd; j += 32) {
            const int32_t val = h_adj[n0 + j];
            col2[dst + j + lower_bound_i32(col + o0, od, val)] = val;
        }
    }
}

__global__ void k_edge_order_keys(const int32_t *row_ptr2, const int32_t *eu, const int32_t *ev, int32_t rho,
                                  int32_t IB, uint64_t *keys, unsigned long long *req) {
    unsigned long long r = 0, cm = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rho; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t du = row_ptr2[eu[i] + 1] - row_ptr2[eu[i]];
        const int32_t dv = row_ptr2[ev[i] + 1] - row_ptr2[ev[i]];
        const int32_t c = min(du, dv);
        r = max(r, (unsigned long long)bk_ws_words(c, c, BK_IMCE));
        cm = max(cm, (unsigned long long)c);
        keys[i] = ((uint64_t)((1u << 30) - 1 - (uint32_t)c) << IB) | (uint64_t)i;
    }
    for (int o = 16; o; o >>= 1) {
        r = max(r, __shfl_xor_sync(FULL, r, o));
        cm = max(cm, __shfl_xor_sync(FULL, cm, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(req, r);
        atomicMax(req + 1, cm);
    }
}

__global__ void k_keys_low(const uint64_t *keys, int32_t m, int32_t IB, int32_t *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int32_t)(keys[i] & ((1ULL << IB) - 1));
}

// ------------------------------------------------------------------ clique lists

// sort the vertices of every listed clique (one thread per clique)
__global__ void k_sort_cliques(const int64_t *off, int64_t nc, int32_t *vtx) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
        int32_t *p = vtx + off[c];
        const int32_t s = p[0];
        for (int i = 2; i <= s; ++i) {
            const int32_t x = p[i];
            int j = i - 1;
            while (j >= 1 && p[j] > x) {
                p[j + 1] = p[j];
                --j;
            }
            p[j + 1] = x;
        }
    }
}

__device__ __forceinline__ uint64_t list_hash(const int32_t *vs, int32_t s, uint64_t seed) {
    uint64_t h = 0;
    for (int i = 0; i < s; ++i) h += vertex_hash(vs[i], seed);
    return clique_hash_from_sum(h, (uint32_t)s);
}

// append listed cliques to the pool (ids base_id..) and the table
__global__ void k_index_insert(const int64_t *loff, const int32_t *lvtx, int64_t nc, int64_t base_id, int64_t pool_base,
                               const int64_t *woff, int32_t *pool, int64_t *off, int32_t *alive,
                               unsigned long long *tkey, int32_t *tid, int64_t tmask, uint64_t seed) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
        const int32_t *src = lvtx + loff[c];
        const int32_t s = src[0];
        const int64_t dst = pool_base + woff[c];
        for (int i = 0; i <= s; ++i) pool[dst + i] = src[i];
        const int64_t id = base_id + c;
        off[id] = dst;
        alive[id] = 1;
        const uint64_t h = list_hash(src + 1, s, seed);
        int64_t slot = (int64_t)(h & (uint64_t)tmask);
        for (;;) {
            if (atomicCAS(&tid[slot], 0, (int32_t)(id + 1)) == 0) {
                tkey[slot] = h;
                break;
            }
            slot = (slot + 1) & tmask;
        }
    }
}

__global__ void k_list_sizes(const int64_t *loff, const int32_t *lvtx, int64_t nc, int64_t *words) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x)
        words[c] = lvtx[loff[c]] + 1;
}

// re-insert every id into a fresh table (after growing it)
__global__ void k_index_rehash(const int32_t *pool, const int64_t *off, int64_t n_ids, unsigned long long *tkey,
                               int32_t *tid, int64_t tmask, uint64_t seed) {
    for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < n_ids;
         id += (int64_t)gridDim.x * blockDim.x) {
        const int32_t *p = pool + off[id];
        const uint64_t h = list_hash(p + 1, p[0], seed);
        int64_t slot = (int64_t)(h & (uint64_t)tmask);
        for (;;) {
            if (atomicCAS(&tid[slot], 0, (int32_t)(id + 1)) == 0) {
                tkey[slot] = h;
                break;
            }
            slot = (slot + 1) & tmask;
        }
    }
}

// ------------------------------------------------------------------ Algorithm 8

constexpr int kEpBits = MCE_HIST_CAP;   // cliques up to this size take the split loop
constexpr int kSubMaxEdges = 512;       // batch edges inside one clique taken by the split loop

// Batch edges inside the clique cv[0..s) (sorted, s <= kEpBits), one warp:
// edges[] gets them as position pairs (i < j, lexicographic order; the first
// kSubMaxEdges are kept) and ep[] the bitmap of their endpoints' positions.
// Returns the number of such edges.
__device__ int clique_batch_edges(const int32_t *cv, int32_t s, const int32_t *h_ptr, const int32_t *h_adj,
                                  int32_t *edges, uint32_t *ep, int lane) {
    const int sw = (s + 31) >> 5;
    for (int k = lane; k < sw; k += 32) ep[k] = 0u;
    __syncwarp();
    int ne = 0;
    for (int i = 0; i < s; ++i) {
        const int32_t a = cv[i];
        const int32_t h0 = h_ptr[a], hd = h_ptr[a + 1] - h0;
        for (int t0 = 0; t0 < hd; t0 += 32) {
            int j = -1;
            if (t0 + lane < hd) {
                const int32_t y = h_adj[h0 + t0 + lane];
                if (y > a) {
                    const int p = lower_bound_i32(cv, s, y);
                    if (p < s && cv[p] == y) j = p;
                }
            }
            const uint32_t b = __ballot_sync(FULL, j >= 0);
            // h_adj rows are sorted, so positions j come out ascending
            if (j >= 0) {
                const int slot = ne + __popc(b & lanemask_lt());
                if (slot < kSubMaxEdges) {
                    edges[2 * slot] = i;
                    edges[2 * slot + 1] = j;
                }
                atomicOr(&ep[i >> 5], 1u << (i & 31));
                atomicOr(&ep[j >> 5], 1u << (j & 31));
            }
            ne += __popc(b);
        }
    }
    __syncwarp();
    return ne;
}

// number of endpoints (set bits of ep over s positions), one warp
__device__ __forceinline__ int count_endpoints(const uint32_t *ep, int32_t s, int lane) {
    int nr = 0;
    for (int k = lane; k < ((s + 31) >> 5); k += 32) nr += __popc(ep[k]);
    return __reduce_add_sync(FULL, nr);
}

// R index (rank among the endpoints) of endpoint position p
__device__ __forceinline__ int endpoint_index(const uint32_t *ep, int p) {
    int r = 0;
    for (int k = 0; k < (p >> 5); ++k) r += __popc(ep[k]);
    return r + __popc(ep[p >> 5] & ((1u << (p & 31)) - 1u));
}

// Sum of h(v) over the core (positions that are no endpoint), one warp
__device__ __forceinline__ uint64_t core_hash_sum(const int32_t *cv, int32_t s, const uint32_t *ep, uint64_t seed,
                                                  int lane) {
    uint64_t h = 0;
    for (int p = lane; p < s; p += 32)
        if (!((ep[p >> 5] >> (p & 31)) & 1u)) h += vertex_hash(cv[p], seed);
    for (int o = 16; o; o >>= 1) h += __shfl_xor_sync(FULL, h, o);
    return h;
}

// Algorithm 8's split set over the endpoints' R indices, one warp: S starts
// as {c} (all nr endpoints); each edge (ei, ej) in turn replaces every member
// holding both ends by that member without ei and that member without ej,
// and S keeps the first occurrence of each set.  edges[] holds R indices.
// Returns |S| (masks of kSubMaxWords words in S), or -1 when S would pass
// kSubCap members.
__device__ int split_set(const int32_t *edges, int ne, int nr, unsigned long long *S, unsigned long long *S2,
                         int lane) {
    constexpr int MW = kSubMaxWords;
    int ns = 1;
    if (lane < MW) {
        const int lo = lane * 64;
        const int nb = nr - lo;
        S[lane] = nb >= 64 ? ~0ULL : (nb > 0 ? ((1ULL << nb) - 1) : 0ULL);
    }
    __syncwarp();
    for (int e = 0; e < ne; ++e) {
        const int ei = edges[2 * e], ej = edges[2 * e + 1];
        const int wi = ei >> 6, wj = ej >> 6;
        const unsigned long long bi = 1ULL << (ei & 63), bj = 1ULL << (ej & 63);
        int n2 = 0;
        for (int t0 = 0; t0 < ns; t0 += 32) {
            const int t = t0 + lane;
            bool both = false, valid = t < ns;
            unsigned long long m[MW];
            if (valid) {
#pragma unroll
                for (int w = 0; w < MW; ++w) m[w] = S[(int64_t)t * MW + w];
                both = (m[wi] & bi) && (m[wj] & bj);
            }
            const uint32_t bb = __ballot_sync(FULL, valid && both);
            const uint32_t bv = __ballot_sync(FULL, valid);
            // outputs: 2 for split ones, 1 otherwise
            const int before = 2 * __popc(bb & lanemask_lt()) + __popc(bv & ~bb & lanemask_lt());
            const int total = 2 * __popc(bb) + __popc(bv & ~bb);
            if (n2 + total > kSubCap) return -1;
            if (valid) {
                unsigned long long *d0 = S2 + (int64_t)(n2 + before) * MW;
                if (both) {
#pragma unroll
                    for (int w = 0; w < MW; ++w) {
                        d0[w] = m[w] & ~(w == wi ? bi : 0ULL);
                        d0[MW + w] = m[w] & ~(w == wj ? bj : 0ULL);
                    }
                } else {
#pragma unroll
                    for (int w = 0; w < MW; ++w) d0[w] = m[w];
                }
            }
            n2 += total;
        }
        __syncwarp();
        // S = set of S2 (drop repeats, keep first occurrences)
        ns = 0;
        for (int t = 0; t < n2; ++t) {
            const unsigned long long *cand = S2 + (int64_t)t * MW;
            bool dup = false;
            for (int q0 = 0; q0 < ns && !dup; q0 += 32) {
                const int q = q0 + lane;
                bool eq = false;
                if (q < ns) {
                    eq = true;
#pragma unroll
                    for (int w = 0; w < MW; ++w) eq &= S[(int64_t)q * MW + w] == cand[w];
                }
                dup = __any_sync(FULL, eq);
            }
            if (!dup) {
                if (lane < MW) S[(int64_t)ns * MW + lane] = cand[lane];
                ++ns;
                __syncwarp();
            }
        }
        __syncwarp();
    }
    return ns;
}

// Hash and size of split candidate m: the core's (hcore, s - nr) plus its endpoints
__device__ __forceinline__ uint64_t split_cand_hash(const int32_t *cv, int32_t s, const uint32_t *ep, int nr,
                                                   const unsigned long long *m, uint64_t hcore, uint64_t seed,
                                                   int32_t &size) {
    uint64_t hs = hcore;
    size = s - nr;
    int r = 0;
    for (int p = 0; p < s; ++p) {
        if (!((ep[p >> 5] >> (p & 31)) & 1u)) continue;
        if ((m[r >> 6] >> (r & 63)) & 1ULL) {
            hs += vertex_hash(cv[p], seed);
            ++size;
        }
        ++r;
    }
    return clique_hash_from_sum(hs, (uint32_t)size);
}

// Members of a split candidate: every position of c that is no endpoint (the
// core), and the endpoints whose R index is set in the mask m.
struct SplitMembers {
    const int32_t *cv;
    int32_t s;
    const uint32_t *ep;
    const unsigned long long *m;
    // f(v) for each member v in ascending order while f returns true
    template <class F> __device__ bool each(F f) const {
        int r = 0;
        for (int p = 0; p < s; ++p) {
            if ((ep[p >> 5] >> (p & 31)) & 1u) {
                const bool in = (m[r >> 6] >> (r & 63)) & 1ULL;
                ++r;
                if (!in) continue;
            }
            if (!f(cv[p])) return false;
        }
        return true;
    }
    __device__ bool has_pos(int p) const {
        if (!((ep[p >> 5] >> (p & 31)) & 1u)) return true;
        const int r = endpoint_index(ep, p);
        return (m[r >> 6] >> (r & 63)) & 1ULL;
    }
};

// Members core ∪ {cv[rpos[r]] : r ∈ K}, rpos = the endpoints' positions, ascending
struct RposMembers {
    const int32_t *cv;
    int32_t s;
    const int32_t *rpos;
    int32_t nr;
    const unsigned long long *K;
    template <class F> __device__ bool each(F f) const {
        int r = 0;
        for (int p = 0; p < s; ++p) {
            if (r < nr && rpos[r] == p) {
                const bool in = (K[r >> 6] >> (r & 63)) & 1ULL;
                ++r;
                if (!in) continue;
            }
            if (!f(cv[p])) return false;
        }
        return true;
    }
    __device__ bool has_pos(int p) const {
        int lo = 0, hi = nr;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (rpos[mid] < p) lo = mid + 1; else hi = mid;
        }
        if (lo == nr || rpos[lo] != p) return true;
        return (K[lo >> 6] >> (lo & 63)) & 1ULL;
    }
};

// are the members, ascending, the sorted list a (of their number of entries)?
template <class M> __device__ __forceinline__ bool members_equal(const M &mem, const int32_t *a) {
    int k = 0;
    return mem.each([&](int32_t v) { return a[k++] == v; });
}

struct SubParams {
    const int64_t *noff;      // new cliques (sorted lists)
    const int32_t *nvtx;
    int64_t n_new;
    const int32_t *h_ptr, *h_adj;
    const int32_t *pool;
    const int64_t *off;
    int32_t *alive;
    const unsigned long long *tkey;
    const int32_t *tid;
    int64_t tmask;
    uint64_t seed;
    unsigned long long *scratch;   // per warp: 2 * kSubCap masks of kSubMaxWords words
    unsigned long long *out;       // OUT block for Λdel
    int64_t *claimed;              // ids claimed (for rollback and the index update)
    unsigned long long *n_claimed;
    int64_t claimed_cap;
    int64_t *list_off;             // optional Λdel list
    int32_t *list_vtx;
    int64_t list_max_cliques, list_max_words;
    int32_t *status;               // 1 = more than 256 endpoints of new edges inside one clique
    int64_t *big;                  // new cliques left to the enumerating fallback
    unsigned long long *n_big;
    unsigned long long *bk_scratch;   // fallback: per thread kBkWords words
};

// Probe the index for the candidate (hash h, size) and claim it if alive;
// the index keeps dead entries (a clique that died and was created again
// after an edge deletion has a later alive copy).  Reports a claim.
template <class Members>
__device__ void sub_probe_claim(const SubParams &P, uint64_t h, int32_t size, const Members &mem) {
    int64_t slot = (int64_t)(h & (uint64_t)P.tmask), found = -1;
    for (int64_t probe = 0; probe <= P.tmask; ++probe) {
        const int32_t id1 = P.tid[slot];
        if (id1 == 0) break;
        if (P.tkey[slot] == h) {
            const int32_t *pl = P.pool + P.off[id1 - 1];
            bool eq = pl[0] == size;
            if (eq) eq = members_equal(mem, pl + 1);
            if (eq && atomicCAS(&P.alive[id1 - 1], 1, 0) == 1) {
                found = id1 - 1;
                break;
            }
        }
        slot = (slot + 1) & P.tmask;
    }
    if (found < 0) return;
    const unsigned long long k = atomicAdd(P.n_claimed, 1ULL);
    if ((int64_t)k < P.claimed_cap) P.claimed[k] = found;
    atomicAdd(&P.out[OUT_COUNT], 1ULL);
    atomicAdd(&P.out[OUT_HASH], h);
    if (size < MCE_HIST_CAP) atomicAdd(&P.out[OUT_HIST + size], 1ULL);
    atomicMax(&P.out[OUT_MAXSIZE], (unsigned long long)size);
    if (P.list_off) {
        const unsigned long long li = atomicAdd(&P.out[OUT_LIST_CLIQUES], 1ULL);
        const unsigned long long lp = atomicAdd(&P.out[OUT_LIST_WORDS], (unsigned long long)size + 1);
        if ((int64_t)li < P.list_max_cliques && (int64_t)(lp + size + 1) <= P.list_max_words) {
            P.list_off[li] = (int64_t)lp;
            const int32_t *pl = P.pool + P.off[found];
            for (int q = 0; q <= size; ++q) P.list_vtx[lp + q] = pl[q];
        } else {
            atomicOr(&P.out[OUT_FLAGS], 1ULL);
        }
    }
}

// One warp per new clique c: E(c) ∩ H in lexicographic order, then S is
// refined edge by edge (c' containing both endpoints is replaced by c' \ {u}
// and c' \ {v}); S stays a set.  Every c' ∈ S found alive in the index is
// claimed once and reported (Algorithm 8).  Vertices of c that are no
// endpoint of a new edge inside c belong to every candidate, so the masks run
// over the endpoints only (at most 256).  A clique larger than kEpBits, with
// more than kSubMaxEdges new edges inside, or whose S outgrows kSubCap goes
// to k_imce_sub_bk.
__global__ void __launch_bounds__(256) k_imce_sub(SubParams P) {
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    constexpr int MW = kSubMaxWords;
    unsigned long long *S = P.scratch + gw * (int64_t)2 * kSubCap * MW;
    unsigned long long *S2 = S + (int64_t)kSubCap * MW;
    __shared__ int32_t edges_s[8][2 * kSubMaxEdges];
    __shared__ uint32_t ep_s[8][kEpBits / 32];
    int32_t *edges = edges_s[wib];
    uint32_t *ep = ep_s[wib];
    for (int64_t c = gw; c < P.n_new; c += nw) {
        const int32_t *cv = P.nvtx + P.noff[c] + 1;
        const int32_t s = cv[-1];
        if (s > kEpBits) {
            if (lane == 0) P.big[atomicAdd(P.n_big, 1ULL)] = c;
            continue;
        }
        const int ne = clique_batch_edges(cv, s, P.h_ptr, P.h_adj, edges, ep, lane);
        const int nr = count_endpoints(ep, s, lane);
        if (nr > 64 * MW) {
            if (lane == 0) atomicOr(P.status, 1);
            continue;
        }
        if (ne > kSubMaxEdges) {
            if (lane == 0) P.big[atomicAdd(P.n_big, 1ULL)] = c;
            continue;
        }
        // endpoint positions -> R indices
        for (int e = lane; e < 2 * ne; e += 32) edges[e] = endpoint_index(ep, edges[e]);
        const uint64_t hcore = core_hash_sum(cv, s, ep, P.seed, lane);
        __syncwarp();
        const int ns = split_set(edges, ne, nr, S, S2, lane);
        if (ns < 0) {
            if (lane == 0) P.big[atomicAdd(P.n_big, 1ULL)] = c;
            continue;
        }
        // probe the index for each candidate
        for (int t0 = 0; t0 < ns; t0 += 32) {
            const int t = t0 + lane;
            if (t < ns) {
                const unsigned long long *m = S + (int64_t)t * MW;
                int32_t size;
                const uint64_t h = split_cand_hash(cv, s, ep, nr, m, hcore, P.seed, size);
                sub_probe_claim(P, h, size, SplitMembers{cv, s, ep, m});
            }
        }
        __syncwarp();
    }
}

// Enumerating fallback of Algorithm 8, one thread per clique c: the split
// candidates that can be maximal cliques (of the old graph for additions, of
// G - H for deletions) are exactly the maximal cliques of c without its batch
// edges, i.e. the core of c plus a maximal clique of the graph on the
// endpoints R whose edges are the pairs that are no batch edge.  Those are
// enumerated with Bron-Kerbosch (Tomita pivot) on 256-bit sets, and act(h,
// size, members) is called for each.  Returns false when R has more than 256
// vertices.
constexpr int kBkWords = 256 * 4 + 258 * 12;   // rows of the graph on R, then frames (cand, fini, ext)

template <class Act>
__device__ bool split_bk(const int32_t *cv, int32_t s, const int32_t *h_ptr, const int32_t *h_adj, uint64_t seed,
                         unsigned long long *adj, unsigned long long *fr, int32_t *rpos, int32_t *qd, Act act) {
    // endpoints of batch edges inside c, ascending position
    int nr = 0;
    for (int p = 0; p < s; ++p) {
        const int32_t a = cv[p];
        bool hit = false;
        for (int32_t e = h_ptr[a]; e < h_ptr[a + 1] && !hit; ++e) {
            const int q = lower_bound_i32(cv, s, h_adj[e]);
            hit = q < s && cv[q] == h_adj[e];
        }
        if (hit) {
            if (nr == 256) return false;
            rpos[nr++] = p;
        }
    }
    // rows of the graph on R: every other endpoint not joined by a batch edge
    for (int r = 0; r < nr; ++r) {
        unsigned long long *row = adj + r * 4;
        for (int w = 0; w < 4; ++w) {
            const int lo = w * 64, nb = nr - lo;
            row[w] = nb >= 64 ? ~0ULL : (nb > 0 ? ((1ULL << nb) - 1) : 0ULL);
        }
        row[r >> 6] &= ~(1ULL << (r & 63));
        const int32_t a = cv[rpos[r]];
        for (int32_t e = h_ptr[a]; e < h_ptr[a + 1]; ++e) {
            const int q = lower_bound_i32(cv, s, h_adj[e]);
            if (!(q < s && cv[q] == h_adj[e])) continue;
            int lo = 0, hi = nr;   // R index of position q
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (rpos[mid] < q) lo = mid + 1; else hi = mid;
            }
            row[lo >> 6] &= ~(1ULL << (lo & 63));
        }
    }
    uint64_t hcore = 0;
    {
        int r = 0;
        for (int p = 0; p < s; ++p) {
            if (r < nr && rpos[r] == p) {
                ++r;
                continue;
            }
            hcore += vertex_hash(cv[p], seed);
        }
    }
    // Bron-Kerbosch over R: frame d = (cand, fini, ext) at depth d; K = chosen
    unsigned long long K[4] = {0, 0, 0, 0};
    int d = 0;
    unsigned long long *f0 = fr;
    for (int w = 0; w < 4; ++w) {
        const int lo = w * 64, nb = nr - lo;
        f0[w] = nb >= 64 ? ~0ULL : (nb > 0 ? ((1ULL << nb) - 1) : 0ULL);
        f0[4 + w] = 0ULL;
    }
    bool enter = true;
    for (;;) {
        unsigned long long *f = fr + (int64_t)d * 12;
        if (enter) {
            bool any_c = false, any_f = false;
            for (int w = 0; w < 4; ++w) {
                any_c |= f[w] != 0ULL;
                any_f |= f[4 + w] != 0ULL;
            }
            if (!any_c) {
                if (!any_f) {
                    uint64_t hs = hcore;
                    int32_t size = s - nr;
                    for (int w = 0; w < 4; ++w)
                        for (unsigned long long x = K[w]; x; x &= x - 1) {
                            hs += vertex_hash(cv[rpos[w * 64 + __ffsll((long long)x) - 1]], seed);
                            ++size;
                        }
                    act(clique_hash_from_sum(hs, (uint32_t)size), size, RposMembers{cv, s, rpos, nr, K});
                }
                goto pop;
            }
            // pivot: the member of cand ∪ fini with most candidate neighbours
            int best = -1, bc = -1;
            for (int w = 0; w < 4; ++w)
                for (unsigned long long x = f[w] | f[4 + w]; x; x &= x - 1) {
                    const int u = w * 64 + __ffsll((long long)x) - 1;
                    int cnt = 0;
                    for (int v = 0; v < 4; ++v) cnt += __popcll(f[v] & adj[u * 4 + v]);
                    if (cnt > bc) {
                        bc = cnt;
                        best = u;
                    }
                }
            for (int w = 0; w < 4; ++w) f[8 + w] = f[w] & ~adj[best * 4 + w];
            enter = false;
        }
        {
            int q = -1;
            for (int w = 0; w < 4 && q < 0; ++w)
                if (f[8 + w]) q = w * 64 + __ffsll((long long)f[8 + w]) - 1;
            if (q < 0) goto pop;
            const unsigned long long qb = 1ULL << (q & 63);
            f[8 + (q >> 6)] &= ~qb;
            unsigned long long *g = f + 12;
            for (int w = 0; w < 4; ++w) {
                g[w] = f[w] & adj[q * 4 + w];
                g[4 + w] = f[4 + w] & adj[q * 4 + w];
            }
            f[q >> 6] &= ~qb;
            f[4 + (q >> 6)] |= qb;
            K[q >> 6] |= qb;
            qd[d] = q;
            ++d;
            enter = true;
            continue;
        }
    pop:
        if (d == 0) break;
        --d;
        K[qd[d] >> 6] &= ~(1ULL << (qd[d] & 63));
        enter = false;
    }
    return true;
}

__global__ void k_imce_sub_bk(SubParams P, int64_t n_big) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    unsigned long long *adj = P.bk_scratch + tid * (int64_t)kBkWords;   // 256 rows of 4 words
    unsigned long long *fr = adj + 256 * 4;                                // frames of 12 words
    int32_t rpos[256];
    int32_t qd[258];
    for (int64_t bi = tid; bi < n_big; bi += nth) {
        const int64_t c = P.big[bi];
        const int32_t *cv = P.nvtx + P.noff[c] + 1;
        const int32_t s = cv[-1];
        const bool ok = split_bk(cv, s, P.h_ptr, P.h_adj, P.seed, adj, fr, rpos, qd,
                                 [&](uint64_t h, int32_t size, const RposMembers &mm) { sub_probe_claim(P, h, size, mm); });
        if (!ok) atomicOr(P.status, 1);
    }
}

// ------------------------------------------------------------------ edge deletions

__global__ void k_sub_deg(const int32_t *row_ptr, const int32_t *hdeg, int32_t n, int32_t *deg2) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
        deg2[x] = row_ptr[x + 1] - row_ptr[x] - hdeg[x];
}

// Row x of G - H: the old row without the deleted neighbours (a sorted
// subset of it), each kept entry moved down by the deleted ones before it.
__global__ void k_minus_rows(const int32_t *row_ptr, const int32_t *col, const int32_t *h_ptr, const int32_t *h_adj,
                             const int32_t *row_ptr2, int32_t n, int32_t *col2) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = warp; x < n; x += nw) {
        const int32_t o0 = row_ptr[x], od = row_ptr[x + 1] - o0;
        const int32_t n0 = h_ptr[x], nd = h_ptr[x + 1] - n0;
        const int32_t dst = row_ptr2[x];
        for (int i = lane; i < od; i += 32) {
            const int32_t val = col[o0 + i];
            const int p = nd ? lower_bound_i32(h_adj + n0, nd, val) : 0;
            if (p < nd && h_adj[n0 + p] == val) continue;
            col2[dst + i - p] = val;
        }
    }
}

__device__ __forceinline__ bool has_edge_csr(const int32_t *row_ptr, const int32_t *col, int32_t a, int32_t b) {
    const int32_t r0 = row_ptr[a], d = row_ptr[a + 1] - r0;
    const int p = lower_bound_i32(col + r0, d, b);
    return p < d && col[r0 + p] == b;
}

// Do the members (a subset of the clique cv[0..s)) form a maximal clique of
// the graph (row_ptr, col)?  They are a clique there; it is maximal iff no
// neighbour y of its member of least degree, outside it, is adjacent to all
// of them.
template <class M>
__device__ bool is_maximal_in(const int32_t *row_ptr, const int32_t *col, const int32_t *cv, int32_t s,
                              const M &mem) {
    int32_t best = -1, bd = 0x7fffffff;
    mem.each([&](int32_t v) {
        const int32_t dv = row_ptr[v + 1] - row_ptr[v];
        if (dv < bd) {
            bd = dv;
            best = v;
        }
        return true;
    });
    if (best < 0) return false;
    for (int32_t e = row_ptr[best]; e < row_ptr[best + 1]; ++e) {
        const int32_t y = col[e];
        const int p = lower_bound_i32(cv, s, y);
        if (p < s && cv[p] == y && mem.has_pos(p)) continue;   // a member
        const bool all = mem.each([&](int32_t v) { return v == best || has_edge_csr(row_ptr, col, y, v); });
        if (all) return false;
    }
    return true;
}

struct DelParams {
    const int64_t *roff;      // removed cliques (sorted lists)
    const int32_t *rvtx;
    int64_t n_rem;
    const int32_t *h_ptr, *h_adj;
    const int32_t *row_ptr, *col;   // G - H
    uint64_t seed;
    unsigned long long *scratch;   // per warp: 2 * kSubCap masks of kSubMaxWords words
    // created cliques, each once: records (H(K), member list [size, ids] in
    // rec_pool) and a table of record + 1 that keeps one record per clique
    unsigned long long *rec_h;
    int64_t *rec_off;
    int32_t *rec_pool;
    int32_t *rec_win;              // 1 = the record that stands for its clique
    unsigned long long *n_rec, *n_words;
    int64_t rec_cap, pool_cap;
    int32_t *tid;
    int64_t tmask;
    unsigned long long *out;       // OUT block of the created cliques
    int32_t *status;               // 1 = more than 256 endpoints of deleted edges in a clique, 4 = record space full
    int64_t *big;                  // removed cliques left to the enumerating fallback
    unsigned long long *n_big;
    unsigned long long *bk_scratch;   // fallback: per thread kBkWords words
};

// Is record b's list (written by another thread: read through L2) the list a?
__device__ bool same_list(const DelParams &P, const int32_t *a, int64_t b) {
    const int32_t *lb = P.rec_pool + __ldcg(P.rec_off + b);
    const int32_t n = __ldcg(lb);
    if (n != a[0]) return false;
    for (int i = 1; i <= n; ++i)
        if (__ldcg(lb + i) != a[i]) return false;
    return true;
}

// A created clique (hash h, size, members), recorded once however many
// removed cliques split into it: the first record to take a table slot for
// its members stands for it and is counted.
template <class M>
__device__ void record_created(const DelParams &P, uint64_t h, int32_t size, const M &mem) {
    const unsigned long long r = atomicAdd(P.n_rec, 1ULL);
    const unsigned long long w = atomicAdd(P.n_words, (unsigned long long)size + 1);
    if ((int64_t)r >= P.rec_cap || (int64_t)(w + size + 1) > P.pool_cap) {
        atomicOr(P.status, 4);
        return;
    }
    int32_t *dst = P.rec_pool + w;
    dst[0] = size;
    int k = 1;
    mem.each([&](int32_t v) {
        dst[k++] = v;
        return true;
    });
    P.rec_off[r] = (int64_t)w;
    P.rec_h[r] = h;
    __threadfence();   // the record is complete before its slot is published
    int64_t slot = (int64_t)(h & (uint64_t)P.tmask);
    bool fresh = false;
    for (int64_t probe = 0; probe <= P.tmask; ++probe) {
        const int32_t prev = atomicCAS(&P.tid[slot], 0, (int32_t)(r + 1));
        if (prev == 0) {
            fresh = true;
            break;
        }
        const int64_t o = prev - 1;
        if (__ldcg(P.rec_h + o) == h && same_list(P, dst, o)) break;   // already there
        slot = (slot + 1) & P.tmask;
    }
    if (!fresh) return;
    P.rec_win[r] = 1;
    atomicAdd(&P.out[OUT_COUNT], 1ULL);
    atomicAdd(&P.out[OUT_HASH], h);
    if (size < MCE_HIST_CAP) atomicAdd(&P.out[OUT_HIST + size], 1ULL);
    atomicMax(&P.out[OUT_MAXSIZE], (unsigned long long)size);
}

// Edge deletions by reduction to additions: G = (G - H) + H, so the cliques
// that the deletion creates are Algorithm 8's splits of the removed cliques
// (those of G through an edge of H) that are maximal in G - H.  One warp per
// removed clique splits it as k_imce_sub does (masks over the endpoints of
// deleted edges inside it); each split that is maximal in G - H is recorded
// once.  A clique larger than kEpBits, with more than kSubMaxEdges deleted
// edges inside, or whose S outgrows kSubCap goes to k_dmce_created_bk.
__global__ void __launch_bounds__(256) k_dmce_created(DelParams P) {
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    constexpr int MW = kSubMaxWords;
    unsigned long long *S = P.scratch + gw * (int64_t)2 * kSubCap * MW;
    unsigned long long *S2 = S + (int64_t)kSubCap * MW;
    __shared__ int32_t edges_s[8][2 * kSubMaxEdges];
    __shared__ uint32_t ep_s[8][kEpBits / 32];
    int32_t *edges = edges_s[wib];
    uint32_t *ep = ep_s[wib];
    for (int64_t c = gw; c < P.n_rem; c += nw) {
        const int32_t *cv = P.rvtx + P.roff[c] + 1;
        const int32_t s = cv[-1];
        if (s > kEpBits) {
            if (lane == 0) P.big[atomicAdd(P.n_big, 1ULL)] = c;
            continue;
        }
        const int ne = clique_batch_edges(cv, s, P.h_ptr, P.h_adj, edges, ep, lane);
        const int nr = count_endpoints(ep, s, lane);
        if (nr > 64 * MW) {
            if (lane == 0) atomicOr(P.status, 1);
            continue;
        }
        if (ne > kSubMaxEdges) {
            if (lane == 0) P.big[atomicAdd(P.n_big, 1ULL)] = c;
            continue;
        }
        for (int e = lane; e < 2 * ne; e += 32) edges[e] = endpoint_index(ep, edges[e]);
        const uint64_t hcore = core_hash_sum(cv, s, ep, P.seed, lane);
        __syncwarp();
        const int ns = split_set(edges, ne, nr, S, S2, lane);
        if (ns < 0) {
            if (lane == 0) P.big[atomicAdd(P.n_big, 1ULL)] = c;
            continue;
        }
        // every split maximal in G - H, recorded once
        for (int t0 = 0; t0 < ns; t0 += 32) {
            const int t = t0 + lane;
            if (t >= ns) continue;
            const unsigned long long *m = S + (int64_t)t * MW;
            int32_t size;
            const uint64_t h = split_cand_hash(cv, s, ep, nr, m, hcore, P.seed, size);
            const SplitMembers mm{cv, s, ep, m};
            if (size > 0 && is_maximal_in(P.row_ptr, P.col, cv, s, mm)) record_created(P, h, size, mm);
        }
        __syncwarp();
    }
}

// Enumerating fallback of the created cliques (see split_bk), one thread per
// removed clique.
__global__ void k_dmce_created_bk(DelParams P, int64_t n_big) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    unsigned long long *adj = P.bk_scratch + tid * (int64_t)kBkWords;
    unsigned long long *fr = adj + 256 * 4;
    int32_t rpos[256];
    int32_t qd[258];
    for (int64_t bi = tid; bi < n_big; bi += nth) {
        const int64_t c = P.big[bi];
        const int32_t *cv = P.rvtx + P.roff[c] + 1;
        const int32_t s = cv[-1];
        const bool ok = split_bk(cv, s, P.h_ptr, P.h_adj, P.seed, adj, fr, rpos, qd,
                                 [&](uint64_t h, int32_t size, const RposMembers &mm) {
                                     if (size > 0 && is_maximal_in(P.row_ptr, P.col, cv, s, mm))
                                         record_created(P, h, size, mm);
                                 });
        if (!ok) atomicOr(P.status, 1);
    }
}

__global__ void k_rec_words(const int32_t *win, const int64_t *rec_off, const int32_t *rec_pool, int64_t n,
                            int32_t *flag, int64_t *words) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        flag[r] = win[r];
        words[r] = win[r] ? (int64_t)rec_pool[rec_off[r]] + 1 : 0;
    }
}

// winning record r -> list entry flag_scan[r] at word offset wpos[r]: size, then the members ascending
__global__ void k_rec_lists(const int32_t *flag_scan, const int64_t *wpos, const int64_t *rec_off,
                            const int32_t *rec_pool, int64_t n, int64_t *loff, int32_t *lvtx) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        if (flag_scan[r + 1] == flag_scan[r]) continue;
        const int32_t *src = rec_pool + rec_off[r];
        const int64_t p = wpos[r];
        loff[flag_scan[r]] = p;
        for (int32_t q = 0; q <= src[0]; ++q) lvtx[p + q] = src[q];
    }
}

// Claim (alive 1 -> 0) the index entry of every listed clique; a clique not
// found alive sets *missing.
__global__ void k_index_claim(const int64_t *loff, const int32_t *lvtx, int64_t nc, const int32_t *pool,
                              const int64_t *off, int32_t *alive, const unsigned long long *tkey, const int32_t *tid,
                              int64_t tmask, uint64_t seed, int64_t *claimed, unsigned long long *n_claimed,
                              int32_t *missing) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
        const int32_t *src = lvtx + loff[c];
        const int32_t sz = src[0];
        const uint64_t h = list_hash(src + 1, sz, seed);
        int64_t slot = (int64_t)(h & (uint64_t)tmask), found = -1;
        for (int64_t probe = 0; probe <= tmask; ++probe) {
            const int32_t id1 = tid[slot];
            if (id1 == 0) break;
            if (tkey[slot] == h) {
                const int32_t *pl = pool + off[id1 - 1];
                bool eq = pl[0] == sz;
                for (int q = 1; q <= sz && eq; ++q) eq = pl[q] == src[q];
                if (eq && alive[id1 - 1]) {
                    found = id1 - 1;
                    break;
                }
            }
            slot = (slot + 1) & tmask;
        }
        if (found >= 0 && atomicCAS(&alive[found], 1, 0) == 1) {
            claimed[atomicAdd(n_claimed, 1ULL)] = found;
        } else {
            atomicOr(missing, 1);
        }
    }
}

__global__ void k_restore_alive(const int64_t *claimed, int64_t n, int32_t *alive) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        alive[claimed[i]] = 1;
}

__global__ void k_alive_flags(const int32_t *alive, int64_t n, int32_t *flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = alive[i];
}

__global__ void k_export_alive(const int32_t *alive, const int32_t *pos, const int64_t *wpos, const int32_t *pool,
                               const int64_t *off, int64_t n, int64_t *loff, int32_t *lvtx) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (!alive[i]) continue;
        const int32_t *p = pool + off[i];
        const int64_t dst = wpos[i];
        loff[pos[i]] = dst;
        for (int q = 0; q <= p[0]; ++q) lvtx[dst + q] = p[q];
    }
}

__global__ void k_alive_words(const int32_t *alive, const int32_t *pool, const int64_t *off, int64_t n, int64_t *w) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        w[i] = alive[i] ? (int64_t)pool[off[i]] + 1 : 0;
}

// ------------------------------------------------------------------ host helpers

template <class T> mce_status grow(T *&p, int64_t &cap, int64_t need, int64_t used, cudaStream_t s) {
    if (need <= cap) return MCE_OK;
    int64_t nc = cap ? cap : 1024;
    while (nc < need) nc *= 2;
    T *q = nullptr;
    MCE_TRY(dev_alloc((void **)&q, (size_t)nc * sizeof(T), s, "index grow"));
    if (p && used) MCE_CUDA(cudaMemcpyAsync(q, p, (size_t)used * sizeof(T), cudaMemcpyDeviceToDevice, s));
    if (p) MCE_CUDA(cudaFreeAsync(p, s));
    p = q;
    cap = nc;
    return MCE_OK;
}

mce_status index_reserve_table(CliqueIndex &I, int64_t n_ids_after, cudaStream_t s, uint64_t seed) {
    if (I.tcap >= 2 * n_ids_after && I.tcap > 0) return MCE_OK;
    int64_t nc = 1024;
    while (nc < 2 * n_ids_after) nc *= 2;
    // the new table is allocated before the old one is freed, so a failed
    // allocation leaves the index as it was
    unsigned long long *tkey = nullptr;
    int32_t *tid = nullptr;
    MCE_TRY(dev_alloc((void **)&tkey, (size_t)nc * 8, s, "index table"));
    const mce_status st = dev_alloc((void **)&tid, (size_t)nc * 4, s, "index table");
    if (st != MCE_OK) {
        cudaFreeAsync(tkey, s);
        return st;
    }
    if (I.tkey) MCE_CUDA(cudaFreeAsync(I.tkey, s));
    if (I.tid) MCE_CUDA(cudaFreeAsync(I.tid, s));
    I.tkey = tkey;
    I.tid = tid;
    MCE_CUDA(cudaMemsetAsync(I.tid, 0, (size_t)nc * 4, s));
    I.tcap = nc;
    if (I.n_ids)
        MCE_LAUNCH(k_index_rehash, grid_for(I.n_ids, 256), 256, 0, s, I.pool, I.off, I.n_ids, I.tkey, I.tid, nc - 1,
                   seed);
    return MCE_OK;
}

// Append nc listed cliques (sorted lists) to the index.
mce_status index_append(CliqueIndex &I, const int64_t *loff, const int32_t *lvtx, int64_t nc, cudaStream_t s,
                        uint64_t seed) {
    if (nc == 0) return MCE_OK;
    DevBuf words;
    MCE_TRY(words.alloc((size_t)(nc + 1) * 8, s));
    MCE_LAUNCH(k_list_sizes, grid_for(nc, 256), 256, 0, s, loff, lvtx, nc, words.as<int64_t>());
    MCE_TRY(exclusive_scan_i64(words.as<int64_t>(), words.as<int64_t>(), nc, s));
    int64_t tot = 0;
    MCE_CUDA(cudaMemcpyAsync(&tot, words.as<int64_t>() + nc, 8, cudaMemcpyDeviceToHost, s));
    MCE_CUDA(cudaStreamSynchronize(s));
    MCE_TRY(grow(I.pool, I.pool_cap, I.pool_words + tot, I.pool_words, s));
    int64_t cap2 = I.ids_cap;
    MCE_TRY(grow(I.off, cap2, I.n_ids + nc, I.n_ids, s));
    int64_t cap3 = I.ids_cap;
    MCE_TRY(grow(I.alive, cap3, I.n_ids + nc, I.n_ids, s));
    I.ids_cap = cap2;
    MCE_TRY(index_reserve_table(I, I.n_ids + nc, s, seed));
    MCE_LAUNCH(k_index_insert, grid_for(nc, 256), 256, 0, s, loff, lvtx, nc, I.n_ids, I.pool_words,
               words.as<int64_t>(), I.pool, I.off, I.alive, I.tkey, I.tid, I.tcap - 1, seed);
    I.n_ids += nc;
    I.pool_words += tot;
    I.n_alive += nc;
    return MCE_OK;
}

// Enumerate with a clique list, growing the list buffers until it fits.
mce_status enumerate_list(const mce_graph *g, const mce_opts *o0, mce_result *res, DevBuf &loff, DevBuf &lvtx) {
    mce_opts o = *o0;
    cudaStream_t s = (cudaStream_t)o.stream;
    int64_t mc = 1 << 16, mw = 1 << 20;
    for (int attempt = 0; attempt < 8; ++attempt) {
        MCE_TRY(loff.alloc((size_t)mc * 8, s));
        MCE_TRY(lvtx.alloc((size_t)mw * 4, s));
        o.list_off = loff.as<int64_t>();
        o.list_vtx = lvtx.as<int32_t>();
        o.list_max_cliques = mc;
        o.list_max_words = mw;
        memset(res, 0, sizeof(*res));
        mce_status st = enumerate(g, &o, res, nullptr, nullptr, 0, nullptr, nullptr);
        if (st != MCE_EOVERFLOW) return st;
        mc = res->list_cliques + 16;
        mw = res->list_words + 64;
    }
    return MCE_EOVERFLOW;
}

void free_index(CliqueIndex &I) {
    cudaFree(I.pool);
    cudaFree(I.off);
    cudaFree(I.alive);
    cudaFree(I.tkey);
    cudaFree(I.tid);
    I = CliqueIndex();
}

mce_status copy_graph(const mce_graph *src, cudaStream_t s, mce_graph **out) {
    mce_graph *g = new mce_graph();
    g->n = src->n;
    g->nnz = src->nnz;
    g->id_bits = src->id_bits;
    mce_status st = dev_alloc((void **)&g->row_ptr, ((size_t)src->n + 1) * 4, s, "alloc");
    if (st == MCE_OK) st = dev_alloc((void **)&g->col, ((size_t)src->nnz + 4) * 4, s, "alloc");
    if (st == MCE_OK)
        st = cuda_status(cudaMemcpyAsync(g->row_ptr, src->row_ptr, ((size_t)src->n + 1) * 4, cudaMemcpyDeviceToDevice, s),
                         "copy");
    if (st == MCE_OK && src->nnz)
        st = cuda_status(cudaMemcpyAsync(g->col, src->col, (size_t)src->nnz * 4, cudaMemcpyDeviceToDevice, s), "copy");
    if (st != MCE_OK) {
        cudaFree(g->row_ptr);
        cudaFree(g->col);
        delete g;
        return st;
    }
    *out = g;
    return MCE_OK;
}

void fill_hist(const unsigned long long *h, int32_t *len, uint64_t *hist) {
    *len = (int32_t)(h[OUT_MAXSIZE] ? h[OUT_MAXSIZE] + 1 : 0);
    if (*len > MCE_HIST_CAP) *len = MCE_HIST_CAP;
    for (int i = 0; i < MCE_HIST_CAP; ++i) hist[i] = i < *len ? h[OUT_HIST + i] : 0;
}

// A canonical batch: e_1..e_rho in arrival order (Algorithm 6 line 2) and
// its adjacency (both directions, sorted by neighbour, with edge indices).
struct Batch {
    DevBuf eu, ev, hdeg, h_ptr, h_adj, h_idx;   // hdeg: batch edges at each vertex; h_ptr: their offsets
    int32_t rho = 0;
};

// Canonicalise k raw pairs against G: additions keep the pairs that are not
// edges of G, deletions those that are; self loops and repeats are dropped
// and the first arrival of a pair kept.
mce_status canonical_batch(imce_state *S, const int32_t *u, const int32_t *v, int64_t k, bool deletion,
                           const char *who, Batch &bt) {
    cudaStream_t s = S->s;
    const mce_graph *g = S->g;
    const int32_t n = g->n, B = g->id_bits;
    const int32_t IB = bits_for((uint64_t)(k > 0 ? k : 1));
    if (2 * B + IB > 63) {
        g_last_error = std::string(who) + ": batch too large for this graph";
        return MCE_EINVAL;
    }
    DevBuf keys, tmp, keep, bad;
    const int64_t kk = k > 0 ? k : 1;
    MCE_TRY(keys.alloc((size_t)kk * 8, s));
    MCE_TRY(tmp.alloc((size_t)kk * 8, s));
    MCE_TRY(keep.alloc((size_t)(kk + 1) * 4, s));
    MCE_TRY(bad.alloc(4, s));
    MCE_CUDA(cudaMemsetAsync(bad.p, 0, 4, s));
    MCE_CUDA(cudaMemsetAsync(keep.p, 0, (size_t)(kk + 1) * 4, s));
    bt.rho = 0;
    if (k > 0) {
        MCE_LAUNCH(k_batch_keys, grid_for(k, 256), 256, 0, s, u, v, k, n, g->row_ptr, g->col, B, IB,
                   (int32_t)deletion, keys.as<uint64_t>(), bad.as<int32_t>());
        MCE_TRY(radix_sort_u64(keys.as<uint64_t>(), tmp.as<uint64_t>(), k, 64, s));
        MCE_LAUNCH(k_first_arrival, grid_for(k, 256), 256, 0, s, keys.as<uint64_t>(), k, IB, keep.as<int32_t>());
        MCE_TRY(exclusive_scan_i32(keep.as<int32_t>(), keep.as<int32_t>(), k, s));
        int32_t hb = 0;
        MCE_CUDA(cudaMemcpyAsync(&hb, bad.p, 4, cudaMemcpyDeviceToHost, s));
        MCE_CUDA(cudaMemcpyAsync(&bt.rho, keep.as<int32_t>() + k, 4, cudaMemcpyDeviceToHost, s));
        MCE_CUDA(cudaStreamSynchronize(s));
        if (hb) {
            g_last_error = std::string(who) + ": vertex id outside [0, n)";
            return MCE_EINVAL;
        }
    }
    const int32_t rho = bt.rho;
    if (rho == 0) return MCE_OK;
    MCE_TRY(bt.eu.alloc((size_t)rho * 4, s));
    MCE_TRY(bt.ev.alloc((size_t)rho * 4, s));
    MCE_LAUNCH(k_emit_batch, grid_for(k, 256), 256, 0, s, u, v, keep.as<int32_t>(), k, bt.eu.as<int32_t>(),
               bt.ev.as<int32_t>());
    const int32_t IBr = bits_for((uint64_t)rho);
    DevBuf hkeys, htmp;
    MCE_TRY(hkeys.alloc((size_t)2 * rho * 8, s));
    MCE_TRY(htmp.alloc((size_t)2 * rho * 8, s));
    MCE_TRY(bt.hdeg.alloc(((size_t)n + 1) * 4, s));
    MCE_TRY(bt.h_ptr.alloc(((size_t)n + 1) * 4, s));
    MCE_TRY(bt.h_adj.alloc((size_t)2 * rho * 4, s));
    MCE_TRY(bt.h_idx.alloc((size_t)2 * rho * 4, s));
    MCE_CUDA(cudaMemsetAsync(bt.hdeg.p, 0, ((size_t)n + 1) * 4, s));
    MCE_LAUNCH(k_h_keys, grid_for(rho, 256), 256, 0, s, bt.eu.as<int32_t>(), bt.ev.as<int32_t>(), rho, B, IBr,
               hkeys.as<uint64_t>(), bt.hdeg.as<int32_t>());
    MCE_TRY(radix_sort_u64(hkeys.as<uint64_t>(), htmp.as<uint64_t>(), 2 * (int64_t)rho, 2 * B + IBr, s));
    MCE_LAUNCH(k_h_fill, grid_for(2 * (int64_t)rho, 256), 256, 0, s, hkeys.as<uint64_t>(), 2 * (int64_t)rho, B, IBr,
               bt.h_adj.as<int32_t>(), bt.h_idx.as<int32_t>());
    MCE_TRY(exclusive_scan_i32(bt.hdeg.as<int32_t>(), bt.h_ptr.as<int32_t>(), n, s));
    return MCE_OK;
}

struct GraphGuard {
    mce_graph *g = nullptr;
    ~GraphGuard() {
        if (g) {
            cudaFree(g->row_ptr);
            cudaFree(g->col);
            delete g;
        }
    }
};

// G + H (add) or G - H (every batch edge an edge of G).
mce_status combine_graph(const mce_graph *g, Batch &bt, bool add, cudaStream_t s, GraphGuard &out) {
    const int32_t n = g->n;
    DevBuf deg2;
    MCE_TRY(deg2.alloc(((size_t)n + 1) * 4, s));
    if (add) MCE_LAUNCH(k_add_deg, grid_for(n, 256), 256, 0, s, g->row_ptr, bt.hdeg.as<int32_t>(), n, deg2.as<int32_t>());
    else MCE_LAUNCH(k_sub_deg, grid_for(n, 256), 256, 0, s, g->row_ptr, bt.hdeg.as<int32_t>(), n, deg2.as<int32_t>());
    mce_graph *g2 = new mce_graph();
    out.g = g2;
    g2->n = n;
    g2->id_bits = g->id_bits;
    g2->nnz = g->nnz + (add ? 2 : -2) * (int64_t)bt.rho;
    MCE_TRY(dev_alloc((void **)&g2->row_ptr, ((size_t)n + 1) * 4, s, "alloc G'"));
    MCE_TRY(dev_alloc((void **)&g2->col, ((size_t)g2->nnz + 4) * 4, s, "alloc G'"));
    MCE_TRY(exclusive_scan_i32(deg2.as<int32_t>(), g2->row_ptr, n, s));
    if (add)
        MCE_LAUNCH(k_merge_rows, grid_for((int64_t)n * 32, 256), 256, 0, s, g->row_ptr, g->col, bt.h_ptr.as<int32_t>(),
                   bt.h_adj.as<int32_t>(), g2->row_ptr, n, g2->col);
    else
        MCE_LAUNCH(k_minus_rows, grid_for((int64_t)n * 32, 256), 256, 0, s, g->row_ptr, g->col, bt.h_ptr.as<int32_t>(),
                   bt.h_adj.as<int32_t>(), g2->row_ptr, n, g2->col);
    return MCE_OK;
}

// The maximal cliques of gp (a graph holding every batch edge) through an edge
// of the batch, each found once: Algorithm 6 with the exclusion of Algorithm
// 7/9, on the persistent engine.  Sorted lists in (loff, lvtx), summary in h.
mce_status batch_cliques(imce_state *S, const mce_graph *gp, Batch &bt, DevBuf &loff, DevBuf &lvtx,
                         unsigned long long *h) {
    cudaStream_t s = S->s;
    const int32_t n = gp->n, rho = bt.rho;
    const int32_t IBr = bits_for((uint64_t)rho);
    // degree-oriented Γ'+ lists
    DevBuf dkey, drank, up_ptr, up_col;
    MCE_TRY(dkey.alloc((size_t)n * 8, s));
    MCE_TRY(drank.alloc((size_t)n * 4, s));
    MCE_TRY(vertex_key(gp, MCE_RANK_DEGREE, s, dkey.as<int64_t>()));
    MCE_TRY(rank_from_key_i64(dkey.as<int64_t>(), n, gp->id_bits, s, drank.as<int32_t>()));
    int64_t up_nnz = 0;
    MCE_TRY(build_up_lists(gp, drank.as<int32_t>(), s, up_ptr, up_col, &up_nnz));
    DevBuf okeys, otmp, order, reqb, nout;
    MCE_TRY(okeys.alloc((size_t)rho * 8, s));
    MCE_TRY(otmp.alloc((size_t)rho * 8, s));
    MCE_TRY(order.alloc((size_t)rho * 4, s));
    MCE_TRY(reqb.alloc(16, s));
    MCE_CUDA(cudaMemsetAsync(reqb.p, 0, 16, s));
    MCE_LAUNCH(k_edge_order_keys, grid_for(rho, 256), 256, 0, s, gp->row_ptr, bt.eu.as<int32_t>(), bt.ev.as<int32_t>(),
               rho, IBr, okeys.as<uint64_t>(), reqb.as<unsigned long long>());
    MCE_TRY(radix_sort_u64(okeys.as<uint64_t>(), otmp.as<uint64_t>(), rho, 30 + IBr, s));
    MCE_LAUNCH(k_keys_low, grid_for(rho, 256), 256, 0, s, okeys.as<uint64_t>(), rho, IBr, order.as<int32_t>());
    unsigned long long reqc[2] = {0, 0};
    MCE_CUDA(cudaMemcpyAsync(reqc, reqb.p, 16, cudaMemcpyDeviceToHost, s));
    MCE_CUDA(cudaStreamSynchronize(s));
    MCE_TRY(nout.alloc(OUT_WORDS * 8, s));
    int64_t mc = 1 << 14, mw = 1 << 18;
    for (int attempt = 0;; ++attempt) {
        MCE_TRY(loff.alloc((size_t)mc * 8, s));
        MCE_TRY(lvtx.alloc((size_t)mw * 4, s));
        MCE_CUDA(cudaMemsetAsync(nout.p, 0, OUT_WORDS * 8, s));
        BkParams P{};
        P.mode = BK_IMCE;
        P.row_ptr = gp->row_ptr;
        P.col = gp->col;
        P.up_ptr = up_ptr.as<int32_t>();
        P.up_col = up_col.as<int32_t>();
        P.order = order.as<int32_t>();
        P.n_sub = rho;
        P.eu = bt.eu.as<int32_t>();
        P.ev = bt.ev.as<int32_t>();
        P.h_ptr = bt.h_ptr.as<int32_t>();
        P.h_adj = bt.h_adj.as<int32_t>();
        P.h_idx = bt.h_idx.as<int32_t>();
        P.seed = S->seed;
        P.out = nout.as<unsigned long long>();
        P.list_off = loff.as<int64_t>();
        P.list_vtx = lvtx.as<int32_t>();
        P.list_max_cliques = mc;
        P.list_max_words = mw;
        P.split = S->opts.split;
        BkBuffers bb;
        // incremental searches start wide (|Γ'(u) ∩ Γ'(v)| candidates) and spend
        // more of their time in the register-heavy wide search: two resident
        // blocks per SM (128 registers) measured faster than three
        mce_opts shape = S->opts;
        if (shape.blocks_per_sm <= 0) shape.blocks_per_sm = 2;
        const LaunchShape ls = launch_shape(&shape);
        MCE_TRY(run_bk(P, ls, (int64_t)reqc[0], (int64_t)reqc[1], s, bb));
        unsigned long long c[CTL_WORDS];
        MCE_CUDA(cudaMemcpyAsync(h, nout.p, OUT_WORDS * 8, cudaMemcpyDeviceToHost, s));
        MCE_CUDA(cudaMemcpyAsync(c, bb.ctl.p, sizeof(c), cudaMemcpyDeviceToHost, s));
        MCE_CUDA(cudaStreamSynchronize(s));
        if (c[CTL_ABORT] & 2ULL) {
            g_last_error = "imce: a bounded device wait gave up";
            return MCE_ETIMEOUT;
        }
        if (c[CTL_ABORT] & 4ULL) {
            g_last_error = "imce: search workspace smaller than a subproblem";
            return MCE_ESTATE;
        }
        if (!(h[OUT_FLAGS] & 1ULL)) break;
        if (attempt >= 6) return MCE_EOVERFLOW;
        mc = (int64_t)h[OUT_LIST_CLIQUES] + 16;
        mw = (int64_t)h[OUT_LIST_WORDS] + 64;
    }
    if (h[OUT_FLAGS] & 2ULL) {
        g_last_error = "imce: clique larger than the histogram";
        return MCE_EOVERFLOW;
    }
    const int64_t nl = (int64_t)h[OUT_LIST_CLIQUES];
    if (nl) MCE_LAUNCH(k_sort_cliques, grid_for(nl, 128), 128, 0, s, loff.as<int64_t>(), nl, lvtx.as<int32_t>());
    return MCE_OK;
}

struct EvTimer {
    cudaEvent_t a = nullptr, b = nullptr;
    ~EvTimer() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

mce_status add_edges(imce_state *S, const int32_t *u, const int32_t *v, int64_t k, imce_delta *out) {
    cudaStream_t s = S->s;
    mce_graph *g = S->g;
    EvTimer ev;
    MCE_CUDA(cudaEventCreate(&ev.a));
    MCE_CUDA(cudaEventCreate(&ev.b));
    MCE_CUDA(cudaEventRecord(ev.a, s));
    // ---- 1. canonical batch
    Batch bt;
    MCE_TRY(canonical_batch(S, u, v, k, false, "imce_add_edges", bt));
    const int32_t rho = bt.rho;
    memset(out, 0, sizeof(*out));
    out->applied = rho;
    out->dropped = k - rho;
    if (rho == 0) {
        out->alive = (uint64_t)S->idx.n_alive;
        MCE_CUDA(cudaEventRecord(ev.b, s));
        MCE_CUDA(cudaEventSynchronize(ev.b));
        cudaEventElapsedTime(&out->ms, ev.a, ev.b);
        return MCE_OK;
    }
    // ---- 2. G' = G + H
    GraphGuard gg;
    MCE_TRY(combine_graph(g, bt, true, s, gg));
    // ---- 3. Λnew
    DevBuf nloff, nlvtx;
    unsigned long long hn[OUT_WORDS];
    MCE_TRY(batch_cliques(S, gg.g, bt, nloff, nlvtx, hn));
    const int64_t n_new = (int64_t)hn[OUT_LIST_CLIQUES];
    // ---- 4. Λdel (Algorithm 8)
    DevBuf sout, scratch, claimed, nclaimed, sstat, big, nbig, bkscr;
    MCE_TRY(sout.alloc(OUT_WORDS * 8, s));
    MCE_CUDA(cudaMemsetAsync(sout.p, 0, OUT_WORDS * 8, s));
    const unsigned sub_blocks = (unsigned)num_sms() * 2;
    const int64_t sub_warps = (int64_t)sub_blocks * 8;
    MCE_TRY(scratch.alloc((size_t)sub_warps * 2 * kSubCap * kSubMaxWords * 8, s));
    // every claim takes an alive clique of the index, each at most once
    const int64_t claimed_cap = S->idx.n_alive + 16;
    MCE_TRY(claimed.alloc((size_t)claimed_cap * 8, s));
    MCE_TRY(nclaimed.alloc(8, s));
    MCE_TRY(sstat.alloc(4, s));
    MCE_TRY(big.alloc((size_t)(n_new + 1) * 8, s));
    MCE_TRY(nbig.alloc(8, s));
    MCE_CUDA(cudaMemsetAsync(nclaimed.p, 0, 8, s));
    MCE_CUDA(cudaMemsetAsync(sstat.p, 0, 4, s));
    MCE_CUDA(cudaMemsetAsync(nbig.p, 0, 8, s));
    unsigned long long hs[OUT_WORDS];
    memset(hs, 0, sizeof(hs));
    unsigned long long ncl = 0;
    int32_t hst = 0;
    if (n_new && S->idx.n_ids) {
        SubParams Q{};
        Q.noff = nloff.as<int64_t>();
        Q.nvtx = nlvtx.as<int32_t>();
        Q.n_new = n_new;
        Q.h_ptr = bt.h_ptr.as<int32_t>();
        Q.h_adj = bt.h_adj.as<int32_t>();
        Q.pool = S->idx.pool;
        Q.off = S->idx.off;
        Q.alive = S->idx.alive;
        Q.tkey = S->idx.tkey;
        Q.tid = S->idx.tid;
        Q.tmask = S->idx.tcap - 1;
        Q.seed = S->seed;
        Q.scratch = scratch.as<unsigned long long>();
        Q.out = sout.as<unsigned long long>();
        Q.claimed = claimed.as<int64_t>();
        Q.n_claimed = nclaimed.as<unsigned long long>();
        Q.claimed_cap = claimed_cap;
        Q.status = sstat.as<int32_t>();
        Q.big = big.as<int64_t>();
        Q.n_big = nbig.as<unsigned long long>();
        MCE_LAUNCH(k_imce_sub, sub_blocks, 256, 0, s, Q);
        // new cliques whose split set outgrew the warp's buffer: enumerating fallback
        unsigned long long hbig = 0;
        MCE_CUDA(cudaMemcpyAsync(&hbig, nbig.p, 8, cudaMemcpyDeviceToHost, s));
        MCE_CUDA(cudaStreamSynchronize(s));
        if (hbig) {
            const int64_t threads = (int64_t)hbig < 4096 ? (int64_t)hbig : 4096;
            MCE_TRY(bkscr.alloc((size_t)threads * kBkWords * 8, s));
            Q.bk_scratch = bkscr.as<unsigned long long>();
            MCE_LAUNCH(k_imce_sub_bk, (unsigned)((threads + 63) / 64), 64, 0, s, Q, (int64_t)hbig);
        }
        MCE_CUDA(cudaMemcpyAsync(hs, sout.p, sizeof(hs), cudaMemcpyDeviceToHost, s));
        MCE_CUDA(cudaMemcpyAsync(&ncl, nclaimed.p, 8, cudaMemcpyDeviceToHost, s));
        MCE_CUDA(cudaMemcpyAsync(&hst, sstat.p, 4, cudaMemcpyDeviceToHost, s));
        MCE_CUDA(cudaStreamSynchronize(s));
        if (hst || (int64_t)ncl > claimed_cap) {
            const int64_t nr = (int64_t)ncl < claimed_cap ? (int64_t)ncl : claimed_cap;
            if (nr) MCE_LAUNCH(k_restore_alive, grid_for(nr, 256), 256, 0, s, claimed.as<int64_t>(), nr, S->idx.alive);
            MCE_CUDA(cudaStreamSynchronize(s));
            g_last_error = hst & 1 ? "imce: more than 256 endpoints of new edges inside one new clique"
                                   : "imce: more subsumed cliques than the claim buffer holds";
            return MCE_ESTATE;
        }
    }
    // ---- 5. commit: index and graph
    mce_status st = index_append(S->idx, nloff.as<int64_t>(), nlvtx.as<int32_t>(), n_new, s, S->seed);
    if (st != MCE_OK) {
        if (ncl) MCE_LAUNCH(k_restore_alive, grid_for((int64_t)ncl, 256), 256, 0, s, claimed.as<int64_t>(),
                            (int64_t)ncl, S->idx.alive);
        return st;
    }
    S->idx.n_alive -= (int64_t)ncl;
    cudaFreeAsync(g->row_ptr, s);
    cudaFreeAsync(g->col, s);
    delete g;
    S->g = gg.g;
    gg.g = nullptr;
    MCE_CUDA(cudaEventRecord(ev.b, s));
    MCE_CUDA(cudaEventSynchronize(ev.b));
    cudaEventElapsedTime(&out->ms, ev.a, ev.b);
    out->new_count = hn[OUT_COUNT];
    out->new_hash = hn[OUT_HASH];
    fill_hist(hn, &out->new_hist_len, out->new_hist);
    out->sub_count = hs[OUT_COUNT];
    out->sub_hash = hs[OUT_HASH];
    fill_hist(hs, &out->sub_hist_len, out->sub_hist);
    out->alive = (uint64_t)S->idx.n_alive;
    return MCE_OK;
}

// Edge deletions (the paper reduces them to additions: G = (G - H) + H):
//   removed = the cliques of G through an edge of H = Λnew of adding H to
//             G - H, found on G by Algorithm 6 with Algorithm 7/9;
//   created = Algorithm 8's splits of the removed cliques that are maximal
//             in G - H (= Λdel of adding H to G - H).
mce_status remove_edges(imce_state *S, const int32_t *u, const int32_t *v, int64_t k, imce_delta *out) {
    cudaStream_t s = S->s;
    mce_graph *g = S->g;
    EvTimer ev;
    MCE_CUDA(cudaEventCreate(&ev.a));
    MCE_CUDA(cudaEventCreate(&ev.b));
    MCE_CUDA(cudaEventRecord(ev.a, s));
    Batch bt;
    MCE_TRY(canonical_batch(S, u, v, k, true, "imce_remove_edges", bt));
    const int32_t rho = bt.rho;
    memset(out, 0, sizeof(*out));
    out->applied = rho;
    out->dropped = k - rho;
    if (rho == 0) {
        out->alive = (uint64_t)S->idx.n_alive;
        MCE_CUDA(cudaEventRecord(ev.b, s));
        MCE_CUDA(cudaEventSynchronize(ev.b));
        cudaEventElapsedTime(&out->ms, ev.a, ev.b);
        return MCE_OK;
    }
    // ---- removed cliques, on G (which holds every batch edge)
    DevBuf rloff, rlvtx;
    unsigned long long hr[OUT_WORDS];
    MCE_TRY(batch_cliques(S, g, bt, rloff, rlvtx, hr));
    const int64_t n_rem = (int64_t)hr[OUT_LIST_CLIQUES];
    // ---- G - H
    GraphGuard gm;
    MCE_TRY(combine_graph(g, bt, false, s, gm));
    // ---- created cliques
    DevBuf cout_, scratch, roffr, rh, rpool, rw, nrec, nwords, tid, sstat, big, nbig, bkscr;
    MCE_TRY(cout_.alloc(OUT_WORDS * 8, s));
    MCE_CUDA(cudaMemsetAsync(cout_.p, 0, OUT_WORDS * 8, s));
    unsigned long long hc[OUT_WORDS];
    memset(hc, 0, sizeof(hc));
    DevBuf cloff, clvtx;
    int64_t n_cre = 0;
    if (n_rem) {
        const unsigned blocks = (unsigned)num_sms() * 2;
        const int64_t warps = (int64_t)blocks * 8;
        MCE_TRY(scratch.alloc((size_t)warps * 2 * kSubCap * kSubMaxWords * 8, s));
        int64_t cap = 8 * n_rem + 4096;
        int64_t pool_cap = 8 * (int64_t)hr[OUT_LIST_WORDS] + 65536;
        MCE_TRY(sstat.alloc(4, s));
        MCE_TRY(nrec.alloc(8, s));
        MCE_TRY(nwords.alloc(8, s));
        MCE_TRY(big.alloc((size_t)(n_rem + 1) * 8, s));
        MCE_TRY(nbig.alloc(8, s));
        unsigned long long nr = 0, nw = 0;
        int32_t hst = 0;
        int64_t bk_threads = 0;
        for (int attempt = 0;; ++attempt) {
            int64_t tcap = 1024;
            while (tcap < 2 * cap) tcap *= 2;
            MCE_TRY(roffr.alloc((size_t)cap * 8, s));
            MCE_TRY(rh.alloc((size_t)cap * 8, s));
            MCE_TRY(rpool.alloc((size_t)pool_cap * 4, s));
            MCE_TRY(rw.alloc((size_t)(cap + 1) * 4, s));
            MCE_TRY(tid.alloc((size_t)tcap * 4, s));
            MCE_CUDA(cudaMemsetAsync(rw.p, 0, (size_t)(cap + 1) * 4, s));
            MCE_CUDA(cudaMemsetAsync(tid.p, 0, (size_t)tcap * 4, s));
            MCE_CUDA(cudaMemsetAsync(nrec.p, 0, 8, s));
            MCE_CUDA(cudaMemsetAsync(nwords.p, 0, 8, s));
            MCE_CUDA(cudaMemsetAsync(sstat.p, 0, 4, s));
            MCE_CUDA(cudaMemsetAsync(nbig.p, 0, 8, s));
            MCE_CUDA(cudaMemsetAsync(cout_.p, 0, OUT_WORDS * 8, s));
            DelParams Q{};
            Q.roff = rloff.as<int64_t>();
            Q.rvtx = rlvtx.as<int32_t>();
            Q.n_rem = n_rem;
            Q.h_ptr = bt.h_ptr.as<int32_t>();
            Q.h_adj = bt.h_adj.as<int32_t>();
            Q.row_ptr = gm.g->row_ptr;
            Q.col = gm.g->col;
            Q.seed = S->seed;
            Q.scratch = scratch.as<unsigned long long>();
            Q.rec_h = rh.as<unsigned long long>();
            Q.rec_off = roffr.as<int64_t>();
            Q.rec_pool = rpool.as<int32_t>();
            Q.rec_win = rw.as<int32_t>();
            Q.n_rec = nrec.as<unsigned long long>();
            Q.n_words = nwords.as<unsigned long long>();
            Q.rec_cap = cap;
            Q.pool_cap = pool_cap;
            Q.tid = tid.as<int32_t>();
            Q.tmask = tcap - 1;
            Q.out = cout_.as<unsigned long long>();
            Q.status = sstat.as<int32_t>();
            Q.big = big.as<int64_t>();
            Q.n_big = nbig.as<unsigned long long>();
            MCE_LAUNCH(k_dmce_created, blocks, 256, 0, s, Q);
            // removed cliques that the split loop left: enumerating fallback
            unsigned long long hbig = 0;
            MCE_CUDA(cudaMemcpyAsync(&hbig, nbig.p, 8, cudaMemcpyDeviceToHost, s));
            MCE_CUDA(cudaStreamSynchronize(s));
            if (hbig) {
                const int64_t threads = (int64_t)hbig < 4096 ? (int64_t)hbig : 4096;
                if (threads > bk_threads) {
                    MCE_TRY(bkscr.alloc((size_t)threads * kBkWords * 8, s));
                    bk_threads = threads;
                }
                Q.bk_scratch = bkscr.as<unsigned long long>();
                MCE_LAUNCH(k_dmce_created_bk, (unsigned)((threads + 63) / 64), 64, 0, s, Q, (int64_t)hbig);
            }
            MCE_CUDA(cudaMemcpyAsync(&nr, nrec.p, 8, cudaMemcpyDeviceToHost, s));
            MCE_CUDA(cudaMemcpyAsync(&nw, nwords.p, 8, cudaMemcpyDeviceToHost, s));
            MCE_CUDA(cudaMemcpyAsync(&hst, sstat.p, 4, cudaMemcpyDeviceToHost, s));
            MCE_CUDA(cudaMemcpyAsync(hc, cout_.p, sizeof(hc), cudaMemcpyDeviceToHost, s));
            MCE_CUDA(cudaStreamSynchronize(s));
            if (hst & 1) {
                g_last_error = "imce: more than 256 endpoints of deleted edges inside one removed clique";
                return MCE_ESTATE;
            }
            if (!(hst & 4)) break;
            if (attempt >= 4) return MCE_EOVERFLOW;
            // room for every record of the last try
            cap = (int64_t)nr + 1024;
            pool_cap = (int64_t)nw + 65536;
        }
        // winning records -> sorted lists
        const int64_t nrec_all = (int64_t)nr;
        DevBuf flag, words;
        MCE_TRY(flag.alloc((size_t)(nrec_all + 1) * 4, s));
        MCE_TRY(words.alloc((size_t)(nrec_all + 1) * 8, s));
        if (nrec_all)
            MCE_LAUNCH(k_rec_words, grid_for(nrec_all, 256), 256, 0, s, rw.as<int32_t>(), roffr.as<int64_t>(),
                       rpool.as<int32_t>(), nrec_all, flag.as<int32_t>(), words.as<int64_t>());
        MCE_TRY(exclusive_scan_i32(flag.as<int32_t>(), flag.as<int32_t>(), nrec_all, s));
        MCE_TRY(exclusive_scan_i64(words.as<int64_t>(), words.as<int64_t>(), nrec_all, s));
        int32_t ncr = 0;
        int64_t nwd = 0;
        MCE_CUDA(cudaMemcpyAsync(&ncr, flag.as<int32_t>() + nrec_all, 4, cudaMemcpyDeviceToHost, s));
        MCE_CUDA(cudaMemcpyAsync(&nwd, words.as<int64_t>() + nrec_all, 8, cudaMemcpyDeviceToHost, s));
        MCE_CUDA(cudaStreamSynchronize(s));
        n_cre = ncr;
        MCE_TRY(cloff.alloc((size_t)(n_cre + 1) * 8, s));
        MCE_TRY(clvtx.alloc((size_t)(nwd + 1) * 4, s));
        if (nrec_all)
            MCE_LAUNCH(k_rec_lists, grid_for(nrec_all, 256), 256, 0, s, flag.as<int32_t>(), words.as<int64_t>(),
                       roffr.as<int64_t>(), rpool.as<int32_t>(), nrec_all, cloff.as<int64_t>(), clvtx.as<int32_t>());
    }
    // ---- commit: removed cliques leave the index, created ones enter it, G := G - H
    DevBuf claimed, nclaimed, missing;
    MCE_TRY(claimed.alloc((size_t)(n_rem + 1) * 8, s));
    MCE_TRY(nclaimed.alloc(8, s));
    MCE_TRY(missing.alloc(4, s));
    MCE_CUDA(cudaMemsetAsync(nclaimed.p, 0, 8, s));
    MCE_CUDA(cudaMemsetAsync(missing.p, 0, 4, s));
    unsigned long long ncl = 0;
    if (n_rem) {
        int32_t hm = 0;
        MCE_LAUNCH(k_index_claim, grid_for(n_rem, 256), 256, 0, s, rloff.as<int64_t>(), rlvtx.as<int32_t>(), n_rem,
                   S->idx.pool, S->idx.off, S->idx.alive, S->idx.tkey, S->idx.tid, S->idx.tcap - 1, S->seed,
                   claimed.as<int64_t>(), nclaimed.as<unsigned long long>(), missing.as<int32_t>());
        MCE_CUDA(cudaMemcpyAsync(&ncl, nclaimed.p, 8, cudaMemcpyDeviceToHost, s));
        MCE_CUDA(cudaMemcpyAsync(&hm, missing.p, 4, cudaMemcpyDeviceToHost, s));
        MCE_CUDA(cudaStreamSynchronize(s));
        if (hm) {
            if (ncl) MCE_LAUNCH(k_restore_alive, grid_for((int64_t)ncl, 256), 256, 0, s, claimed.as<int64_t>(),
                                (int64_t)ncl, S->idx.alive);
            MCE_CUDA(cudaStreamSynchronize(s));
            g_last_error = "imce_remove_edges: a removed clique is not in the index";
            return MCE_ESTATE;
        }
    }
    mce_status st = MCE_OK;
    if (n_cre) st = index_append(S->idx, cloff.as<int64_t>(), clvtx.as<int32_t>(), n_cre, s, S->seed);
    if (st != MCE_OK) {
        if (ncl) MCE_LAUNCH(k_restore_alive, grid_for((int64_t)ncl, 256), 256, 0, s, claimed.as<int64_t>(),
                            (int64_t)ncl, S->idx.alive);
        return st;
    }
    S->idx.n_alive -= (int64_t)ncl;
    cudaFreeAsync(g->row_ptr, s);
    cudaFreeAsync(g->col, s);
    delete g;
    S->g = gm.g;
    gm.g = nullptr;
    MCE_CUDA(cudaEventRecord(ev.b, s));
    MCE_CUDA(cudaEventSynchronize(ev.b));
    cudaEventElapsedTime(&out->ms, ev.a, ev.b);
    out->new_count = hc[OUT_COUNT];
    out->new_hash = hc[OUT_HASH];
    fill_hist(hc, &out->new_hist_len, out->new_hist);
    out->sub_count = hr[OUT_COUNT];
    out->sub_hash = hr[OUT_HASH];
    fill_hist(hr, &out->sub_hist_len, out->sub_hist);
    out->alive = (uint64_t)S->idx.n_alive;
    return MCE_OK;
}

}  // namespace

void imce_set_stream(imce_state *S, cudaStream_t s) { S->s = s; }

}  // namespace mce

using namespace mce;

extern "C" {

mce_status imce_open(const mce_graph *g, const mce_opts *opts, imce_state **out) {
    if (!g || !opts || !out) {
        g_last_error = "imce_open: bad arguments";
        return MCE_EINVAL;
    }
    imce_state *S = new imce_state();
    S->opts = *opts;
    S->opts.list_off = nullptr;
    S->opts.list_vtx = nullptr;
    S->opts.pv_count = S->opts.pv_hash = S->opts.pv_nodes = nullptr;
    S->opts.node_budget = 0;
    S->seed = opts->hash_seed;
    S->s = (cudaStream_t)opts->stream;
    mce_status st = copy_graph(g, S->s, &S->g);
    if (st == MCE_OK) {
        DevBuf loff, lvtx;
        mce_result r;
        st = enumerate_list(S->g, &S->opts, &r, loff, lvtx);
        if (st == MCE_OK && r.list_cliques) {
            MCE_LAUNCH(k_sort_cliques, grid_for(r.list_cliques, 128), 128, 0, S->s, loff.as<int64_t>(), r.list_cliques,
                       lvtx.as<int32_t>());
            st = index_append(S->idx, loff.as<int64_t>(), lvtx.as<int32_t>(), r.list_cliques, S->s, S->seed);
        }
        if (st == MCE_OK) st = cuda_status(cudaStreamSynchronize(S->s), "imce_open");
    }
    if (st != MCE_OK) {
        imce_close(S);
        return st;
    }
    *out = S;
    return MCE_OK;
}

mce_status imce_add_edges(imce_state *S, const int32_t *u, const int32_t *v, int64_t k, int32_t on_device,
                          imce_delta *out) {
    if (!S || !out || k < 0 || (k > 0 && (!u || !v))) {
        g_last_error = "imce_add_edges: bad arguments";
        return MCE_EINVAL;
    }
    if (k >= (int64_t)1 << 30) {
        g_last_error = "imce_add_edges: batch too large";
        return MCE_EINVAL;
    }
    DevBuf du, dv;
    const int32_t *pu = u, *pv = v;
    if (!on_device && k > 0) {
        MCE_TRY(du.alloc((size_t)k * 4, S->s));
        MCE_TRY(dv.alloc((size_t)k * 4, S->s));
        MCE_CUDA(cudaMemcpyAsync(du.p, u, (size_t)k * 4, cudaMemcpyHostToDevice, S->s));
        MCE_CUDA(cudaMemcpyAsync(dv.p, v, (size_t)k * 4, cudaMemcpyHostToDevice, S->s));
        pu = du.as<int32_t>();
        pv = dv.as<int32_t>();
    }
    return add_edges(S, pu, pv, k, out);
}

mce_status imce_remove_edges(imce_state *S, const int32_t *u, const int32_t *v, int64_t k, int32_t on_device,
                             imce_delta *out) {
    if (!S || !out || k < 0 || (k > 0 && (!u || !v))) {
        g_last_error = "imce_remove_edges: bad arguments";
        return MCE_EINVAL;
    }
    if (k >= (int64_t)1 << 30) {
        g_last_error = "imce_remove_edges: batch too large";
        return MCE_EINVAL;
    }
    DevBuf du, dv;
    const int32_t *pu = u, *pv = v;
    if (!on_device && k > 0) {
        MCE_TRY(du.alloc((size_t)k * 4, S->s));
        MCE_TRY(dv.alloc((size_t)k * 4, S->s));
        MCE_CUDA(cudaMemcpyAsync(du.p, u, (size_t)k * 4, cudaMemcpyHostToDevice, S->s));
        MCE_CUDA(cudaMemcpyAsync(dv.p, v, (size_t)k * 4, cudaMemcpyHostToDevice, S->s));
        pu = du.as<int32_t>();
        pv = dv.as<int32_t>();
    }
    return remove_edges(S, pu, pv, k, out);
}

const mce_graph *imce_graph(const imce_state *S) { return S ? S->g : nullptr; }

mce_status imce_cliques(const imce_state *S, int64_t *list_off, int32_t *list_vtx, int64_t max_cliques,
                        int64_t max_words, int64_t *n_cliques, int64_t *n_words) {
    if (!S || !n_cliques || !n_words) return MCE_EINVAL;
    cudaStream_t s = S->s;
    const CliqueIndex &I = S->idx;
    const int64_t n = I.n_ids;
    *n_cliques = 0;
    *n_words = 0;
    if (n == 0) return MCE_OK;
    DevBuf flag, words;
    MCE_TRY(flag.alloc((size_t)(n + 1) * 4, s));
    MCE_TRY(words.alloc((size_t)(n + 1) * 8, s));
    MCE_LAUNCH(k_alive_flags, grid_for(n, 256), 256, 0, s, I.alive, n, flag.as<int32_t>());
    MCE_TRY(exclusive_scan_i32(flag.as<int32_t>(), flag.as<int32_t>(), n, s));
    MCE_LAUNCH(k_alive_words, grid_for(n, 256), 256, 0, s, I.alive, I.pool, I.off, n, words.as<int64_t>());
    MCE_TRY(exclusive_scan_i64(words.as<int64_t>(), words.as<int64_t>(), n, s));
    int32_t nc = 0;
    int64_t nw = 0;
    MCE_CUDA(cudaMemcpyAsync(&nc, flag.as<int32_t>() + n, 4, cudaMemcpyDeviceToHost, s));
    MCE_CUDA(cudaMemcpyAsync(&nw, words.as<int64_t>() + n, 8, cudaMemcpyDeviceToHost, s));
    MCE_CUDA(cudaStreamSynchronize(s));
    *n_cliques = nc;
    *n_words = nw;
    if (nc > max_cliques || nw > max_words || !list_off || !list_vtx) return MCE_EOVERFLOW;
    MCE_LAUNCH(k_export_alive, grid_for(n, 256), 256, 0, s, I.alive, flag.as<int32_t>(), words.as<int64_t>(), I.pool,
               I.off, n, list_off, list_vtx);
    MCE_CUDA(cudaStreamSynchronize(s));
    return MCE_OK;
}

void imce_close(imce_state *S) {
    if (!S) return;
    cudaDeviceSynchronize();
    free_index(S->idx);
    if (S->g) {
        cudaFree(S->g->row_ptr);
        cudaFree(S->g->col);
        delete S->g;
    }
    delete S;
}

}  // extern "C"
