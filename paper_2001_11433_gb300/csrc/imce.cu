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
constexpr int kSubMaxWords = 4;          // cliques up to 256 vertices in Algorithm 8
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
                             const int32_t *col, int32_t B, int32_t IB, uint64_t *keys, int32_t *bad) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a0 = u[i], b0 = v[i];
        uint64_t key = ~0ULL;
        if (a0 < 0 || a0 >= n || b0 < 0 || b0 >= n) {
            atomicOr(bad, 1);
        } else if (a0 != b0) {
            const int32_t a = min(a0, b0), b = max(a0, b0);
            const int32_t r0 = row_ptr[a], d = row_ptr[a + 1] - r0;
            const int p = lower_bound_i32(col + r0, d, b);
            if (!(p < d && col[r0 + p] == b)) key = ((((uint64_t)a << B) | (uint64_t)b) << IB) | (uint64_t)i;
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
    int32_t *status;               // 1 = a clique too large, 2 = too many candidates
};

// One warp per new clique c: E(c) ∩ H in lexicographic order, then S is
// refined edge by edge (c' containing both endpoints is replaced by c' \ {u}
// and c' \ {v}); S stays a set.  Every c' ∈ S found alive in the index is
// claimed once and reported (Algorithm 8, lines 13-16).
__global__ void __launch_bounds__(256) k_imce_sub(SubParams P) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    constexpr int MW = kSubMaxWords;
    unsigned long long *S = P.scratch + gw * (int64_t)2 * kSubCap * MW;
    unsigned long long *S2 = S + (int64_t)kSubCap * MW;
    __shared__ int32_t edges_s[8][2 * 512];
    int32_t *edges = edges_s[threadIdx.x >> 5];
    for (int64_t c = gw; c < P.n_new; c += nw) {
        const int32_t *cv = P.nvtx + P.noff[c] + 1;
        const int32_t s = cv[-1];
        if (s > 64 * MW) {
            if (lane == 0) atomicOr(P.status, 1);
            continue;
        }
        // new edges inside c: (i, j) positions, i < j, lexicographic
        int ne = 0;
        for (int i = 0; i < s; ++i) {
            const int32_t a = cv[i];
            const int32_t h0 = P.h_ptr[a], hd = P.h_ptr[a + 1] - h0;
            for (int t0 = 0; t0 < hd; t0 += 32) {
                int j = -1;
                if (t0 + lane < hd) {
                    const int32_t y = P.h_adj[h0 + t0 + lane];
                    if (y > a) {
                        const int p = lower_bound_i32(cv, s, y);
                        if (p < s && cv[p] == y) j = p;
                    }
                }
                const uint32_t b = __ballot_sync(FULL, j >= 0);
                // h_adj rows are sorted, so positions j come out ascending
                if (j >= 0) {
                    const int slot = ne + __popc(b & lanemask_lt());
                    if (slot < 512) {
                        edges[2 * slot] = i;
                        edges[2 * slot + 1] = j;
                    }
                }
                ne += __popc(b);
            }
        }
        __syncwarp();
        if (ne > 512) {
            if (lane == 0) atomicOr(P.status, 2);
            continue;
        }
        // S = {c}
        int ns = 1;
        if (lane < MW) {
            const int lo = lane * 64;
            const int nb = s - lo;
            S[lane] = nb >= 64 ? ~0ULL : (nb > 0 ? ((1ULL << nb) - 1) : 0ULL);
        }
        __syncwarp();
        bool overflow = false;
        for (int e = 0; e < ne && !overflow; ++e) {
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
                if (n2 + total > kSubCap) {
                    overflow = true;
                    break;
                }
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
            if (overflow) break;
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
        if (overflow) {
            if (lane == 0) atomicOr(P.status, 2);
            continue;
        }
        // probe the index for each candidate
        for (int t0 = 0; t0 < ns; t0 += 32) {
            const int t = t0 + lane;
            int64_t found = -1;
            int32_t size = 0;
            uint64_t h = 0;
            if (t < ns) {
                unsigned long long m[MW];
#pragma unroll
                for (int w = 0; w < MW; ++w) m[w] = S[(int64_t)t * MW + w];
                uint64_t hs = 0;
                for (int w = 0; w < MW; ++w) {
                    unsigned long long x = m[w];
                    while (x) {
                        const int b = __ffsll((long long)x) - 1;
                        x &= x - 1;
                        hs += vertex_hash(cv[w * 64 + b], P.seed);
                        ++size;
                    }
                }
                h = clique_hash_from_sum(hs, (uint32_t)size);
                int64_t slot = (int64_t)(h & (uint64_t)P.tmask);
                for (;;) {
                    const int32_t id1 = P.tid[slot];
                    if (id1 == 0) break;
                    if (P.tkey[slot] == h) {
                        const int32_t *pl = P.pool + P.off[id1 - 1];
                        bool eq = pl[0] == size;
                        if (eq) {
                            int k = 1;
                            for (int w = 0; w < MW && eq; ++w) {
                                unsigned long long x = m[w];
                                while (x && eq) {
                                    const int b = __ffsll((long long)x) - 1;
                                    x &= x - 1;
                                    eq = pl[k++] == cv[w * 64 + b];
                                }
                            }
                        }
                        if (eq) {
                            found = id1 - 1;
                            break;
                        }
                    }
                    slot = (slot + 1) & P.tmask;
                }
                if (found >= 0 && atomicCAS(&P.alive[found], 1, 0) == 1) {
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
            }
        }
        __syncwarp();
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

mce_status add_edges(imce_state *S, const int32_t *u, const int32_t *v, int64_t k, imce_delta *out) {
    cudaStream_t s = S->s;
    mce_graph *g = S->g;
    const int32_t n = g->n, B = g->id_bits;
    const int32_t IB = bits_for((uint64_t)(k > 0 ? k : 1));
    if (2 * B + IB > 63) {
        g_last_error = "imce_add_edges: batch too large for this graph";
        return MCE_EINVAL;
    }
    cudaEvent_t e0, e1;
    MCE_CUDA(cudaEventCreate(&e0));
    MCE_CUDA(cudaEventCreate(&e1));
    struct EvG {
        cudaEvent_t a, b;
        ~EvG() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } evg{e0, e1};
    MCE_CUDA(cudaEventRecord(e0, s));
    // ---- 1. canonical batch
    DevBuf keys, tmp, keep, bad, eu, ev;
    const int64_t kk = k > 0 ? k : 1;
    MCE_TRY(keys.alloc((size_t)kk * 8, s));
    MCE_TRY(tmp.alloc((size_t)kk * 8, s));
    MCE_TRY(keep.alloc((size_t)(kk + 1) * 4, s));
    MCE_TRY(bad.alloc(4, s));
    MCE_CUDA(cudaMemsetAsync(bad.p, 0, 4, s));
    MCE_CUDA(cudaMemsetAsync(keep.p, 0, (size_t)(kk + 1) * 4, s));
    int32_t rho = 0;
    if (k > 0) {
        MCE_LAUNCH(k_batch_keys, grid_for(k, 256), 256, 0, s, u, v, k, n, g->row_ptr, g->col, B, IB,
                   keys.as<uint64_t>(), bad.as<int32_t>());
        MCE_TRY(radix_sort_u64(keys.as<uint64_t>(), tmp.as<uint64_t>(), k, 64, s));
        MCE_LAUNCH(k_first_arrival, grid_for(k, 256), 256, 0, s, keys.as<uint64_t>(), k, IB, keep.as<int32_t>());
        MCE_TRY(exclusive_scan_i32(keep.as<int32_t>(), keep.as<int32_t>(), k, s));
        int32_t hb = 0;
        MCE_CUDA(cudaMemcpyAsync(&hb, bad.p, 4, cudaMemcpyDeviceToHost, s));
        MCE_CUDA(cudaMemcpyAsync(&rho, keep.as<int32_t>() + k, 4, cudaMemcpyDeviceToHost, s));
        MCE_CUDA(cudaStreamSynchronize(s));
        if (hb) {
            g_last_error = "imce_add_edges: vertex id outside [0, n)";
            return MCE_EINVAL;
        }
    }
    memset(out, 0, sizeof(*out));
    out->applied = rho;
    out->dropped = k - rho;
    if (rho == 0) {
        out->alive = (uint64_t)S->idx.n_alive;
        MCE_CUDA(cudaEventRecord(e1, s));
        MCE_CUDA(cudaEventSynchronize(e1));
        cudaEventElapsedTime(&out->ms, e0, e1);
        return MCE_OK;
    }
    MCE_TRY(eu.alloc((size_t)rho * 4, s));
    MCE_TRY(ev.alloc((size_t)rho * 4, s));
    MCE_LAUNCH(k_emit_batch, grid_for(k, 256), 256, 0, s, u, v, keep.as<int32_t>(), k, eu.as<int32_t>(),
               ev.as<int32_t>());
    // ---- batch adjacency (both directions, sorted by neighbour, with edge index)
    const int32_t IBr = bits_for((uint64_t)rho);
    DevBuf hkeys, htmp, h_ptr, h_adj, h_idx;
    MCE_TRY(hkeys.alloc((size_t)2 * rho * 8, s));
    MCE_TRY(htmp.alloc((size_t)2 * rho * 8, s));
    MCE_TRY(h_ptr.alloc(((size_t)n + 1) * 4, s));
    MCE_TRY(h_adj.alloc((size_t)2 * rho * 4, s));
    MCE_TRY(h_idx.alloc((size_t)2 * rho * 4, s));
    MCE_CUDA(cudaMemsetAsync(h_ptr.p, 0, ((size_t)n + 1) * 4, s));
    MCE_LAUNCH(k_h_keys, grid_for(rho, 256), 256, 0, s, eu.as<int32_t>(), ev.as<int32_t>(), rho, B, IBr,
               hkeys.as<uint64_t>(), h_ptr.as<int32_t>());
    MCE_TRY(radix_sort_u64(hkeys.as<uint64_t>(), htmp.as<uint64_t>(), 2 * (int64_t)rho, 2 * B + IBr, s));
    MCE_LAUNCH(k_h_fill, grid_for(2 * (int64_t)rho, 256), 256, 0, s, hkeys.as<uint64_t>(), 2 * (int64_t)rho, B, IBr,
               h_adj.as<int32_t>(), h_idx.as<int32_t>());
    // ---- 2. G' = G + H
    DevBuf deg2;
    MCE_TRY(deg2.alloc(((size_t)n + 1) * 4, s));
    MCE_LAUNCH(k_add_deg, grid_for(n, 256), 256, 0, s, g->row_ptr, h_ptr.as<int32_t>(), n, deg2.as<int32_t>());
    MCE_TRY(exclusive_scan_i32(h_ptr.as<int32_t>(), h_ptr.as<int32_t>(), n, s));
    mce_graph *g2 = new mce_graph();
    struct GGuard {
        mce_graph *&g;
        bool keep = false;
        ~GGuard() {
            if (!keep && g) {
                cudaFree(g->row_ptr);
                cudaFree(g->col);
                delete g;
            }
        }
    } gg{g2};
    g2->n = n;
    g2->id_bits = B;
    g2->nnz = g->nnz + 2 * (int64_t)rho;
    MCE_TRY(dev_alloc((void **)&g2->row_ptr, ((size_t)n + 1) * 4, s, "alloc G'"));
    MCE_TRY(dev_alloc((void **)&g2->col, ((size_t)g2->nnz + 4) * 4, s, "alloc G'"));
    MCE_TRY(exclusive_scan_i32(deg2.as<int32_t>(), g2->row_ptr, n, s));
    MCE_LAUNCH(k_merge_rows, grid_for((int64_t)n * 32, 256), 256, 0, s, g->row_ptr, g->col, h_ptr.as<int32_t>(),
               h_adj.as<int32_t>(), g2->row_ptr, n, g2->col);
    // degree-oriented Γ'+ lists
    DevBuf dkey, drank, up_ptr, up_col;
    MCE_TRY(dkey.alloc((size_t)n * 8, s));
    MCE_TRY(drank.alloc((size_t)n * 4, s));
    MCE_TRY(vertex_key(g2, MCE_RANK_DEGREE, s, dkey.as<int64_t>()));
    MCE_TRY(rank_from_key_i64(dkey.as<int64_t>(), n, B, s, drank.as<int32_t>()));
    int64_t up_nnz = 0;
    MCE_TRY(build_up_lists(g2, drank.as<int32_t>(), s, up_ptr, up_col, &up_nnz));
    // ---- 3. Λnew
    DevBuf okeys, otmp, order, reqb, nout;
    MCE_TRY(okeys.alloc((size_t)rho * 8, s));
    MCE_TRY(otmp.alloc((size_t)rho * 8, s));
    MCE_TRY(order.alloc((size_t)rho * 4, s));
    MCE_TRY(reqb.alloc(16, s));
    MCE_CUDA(cudaMemsetAsync(reqb.p, 0, 16, s));
    MCE_LAUNCH(k_edge_order_keys, grid_for(rho, 256), 256, 0, s, g2->row_ptr, eu.as<int32_t>(), ev.as<int32_t>(), rho,
               IBr, okeys.as<uint64_t>(), reqb.as<unsigned long long>());
    MCE_TRY(radix_sort_u64(okeys.as<uint64_t>(), otmp.as<uint64_t>(), rho, 30 + IBr, s));
    MCE_LAUNCH(k_keys_low, grid_for(rho, 256), 256, 0, s, okeys.as<uint64_t>(), rho, IBr, order.as<int32_t>());
    unsigned long long reqc[2] = {0, 0};
    MCE_CUDA(cudaMemcpyAsync(reqc, reqb.p, 16, cudaMemcpyDeviceToHost, s));
    MCE_CUDA(cudaStreamSynchronize(s));
    MCE_TRY(nout.alloc(OUT_WORDS * 8, s));
    DevBuf nloff, nlvtx;
    int64_t mc = 1 << 14, mw = 1 << 18;
    unsigned long long hn[OUT_WORDS];
    for (int attempt = 0;; ++attempt) {
        MCE_TRY(nloff.alloc((size_t)mc * 8, s));
        MCE_TRY(nlvtx.alloc((size_t)mw * 4, s));
        MCE_CUDA(cudaMemsetAsync(nout.p, 0, OUT_WORDS * 8, s));
        BkParams P{};
        P.mode = BK_IMCE;
        P.row_ptr = g2->row_ptr;
        P.col = g2->col;
        P.up_ptr = up_ptr.as<int32_t>();
        P.up_col = up_col.as<int32_t>();
        P.order = order.as<int32_t>();
        P.n_sub = rho;
        P.eu = eu.as<int32_t>();
        P.ev = ev.as<int32_t>();
        P.h_ptr = h_ptr.as<int32_t>();
        P.h_adj = h_adj.as<int32_t>();
        P.h_idx = h_idx.as<int32_t>();
        P.seed = S->seed;
        P.out = nout.as<unsigned long long>();
        P.list_off = nloff.as<int64_t>();
        P.list_vtx = nlvtx.as<int32_t>();
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
        MCE_CUDA(cudaMemcpyAsync(hn, nout.p, sizeof(hn), cudaMemcpyDeviceToHost, s));
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
        if (!(hn[OUT_FLAGS] & 1ULL)) break;
        if (attempt >= 6) return MCE_EOVERFLOW;
        mc = (int64_t)hn[OUT_LIST_CLIQUES] + 16;
        mw = (int64_t)hn[OUT_LIST_WORDS] + 64;
    }
    if (hn[OUT_FLAGS] & 2ULL) {
        g_last_error = "imce: clique larger than the histogram";
        return MCE_EOVERFLOW;
    }
    const int64_t n_new = (int64_t)hn[OUT_LIST_CLIQUES];
    if (n_new) MCE_LAUNCH(k_sort_cliques, grid_for(n_new, 128), 128, 0, s, nloff.as<int64_t>(), n_new, nlvtx.as<int32_t>());
    // ---- 4. Λdel (Algorithm 8)
    DevBuf sout, scratch, claimed, nclaimed, sstat;
    MCE_TRY(sout.alloc(OUT_WORDS * 8, s));
    MCE_CUDA(cudaMemsetAsync(sout.p, 0, OUT_WORDS * 8, s));
    const unsigned sub_blocks = (unsigned)num_sms() * 2;
    const int64_t sub_warps = (int64_t)sub_blocks * 8;
    MCE_TRY(scratch.alloc((size_t)sub_warps * 2 * kSubCap * kSubMaxWords * 8, s));
    const int64_t claimed_cap = n_new * 4 + 1024;
    MCE_TRY(claimed.alloc((size_t)claimed_cap * 8, s));
    MCE_TRY(nclaimed.alloc(8, s));
    MCE_TRY(sstat.alloc(4, s));
    MCE_CUDA(cudaMemsetAsync(nclaimed.p, 0, 8, s));
    MCE_CUDA(cudaMemsetAsync(sstat.p, 0, 4, s));
    unsigned long long hs[OUT_WORDS];
    memset(hs, 0, sizeof(hs));
    unsigned long long ncl = 0;
    int32_t hst = 0;
    if (n_new && S->idx.n_ids) {
        SubParams Q{};
        Q.noff = nloff.as<int64_t>();
        Q.nvtx = nlvtx.as<int32_t>();
        Q.n_new = n_new;
        Q.h_ptr = h_ptr.as<int32_t>();
        Q.h_adj = h_adj.as<int32_t>();
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
        MCE_LAUNCH(k_imce_sub, sub_blocks, 256, 0, s, Q);
        MCE_CUDA(cudaMemcpyAsync(hs, sout.p, sizeof(hs), cudaMemcpyDeviceToHost, s));
        MCE_CUDA(cudaMemcpyAsync(&ncl, nclaimed.p, 8, cudaMemcpyDeviceToHost, s));
        MCE_CUDA(cudaMemcpyAsync(&hst, sstat.p, 4, cudaMemcpyDeviceToHost, s));
        MCE_CUDA(cudaStreamSynchronize(s));
        if (hst || (int64_t)ncl > claimed_cap) {
            const int64_t nr = (int64_t)ncl < claimed_cap ? (int64_t)ncl : claimed_cap;
            if (nr) MCE_LAUNCH(k_restore_alive, grid_for(nr, 256), 256, 0, s, claimed.as<int64_t>(), nr, S->idx.alive);
            MCE_CUDA(cudaStreamSynchronize(s));
            g_last_error = hst & 1 ? "imce: new clique larger than 256 vertices" : "imce: too many subsumed candidates";
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
    gg.keep = true;
    cudaFreeAsync(g->row_ptr, s);
    cudaFreeAsync(g->col, s);
    delete g;
    S->g = g2;
    MCE_CUDA(cudaEventRecord(e1, s));
    MCE_CUDA(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&out->ms, e0, e1);
    out->new_count = hn[OUT_COUNT];
    out->new_hash = hn[OUT_HASH];
    fill_hist(hn, &out->new_hist_len, out->new_hist);
    out->sub_count = hs[OUT_COUNT];
    out->sub_hash = hs[OUT_HASH];
    fill_hist(hs, &out->sub_hist_len, out->sub_hist);
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
