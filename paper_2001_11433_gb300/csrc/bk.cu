#include <atomic>
// Persistent warp-cooperative Bron-Kerbosch (TTT) engine.
//
// One warp runs one search at a time.  A search is either a whole
// subproblem (ParMCE, Algorithm 5: K = {v}, cand = Γ+(v), fini = the
// lower-ranked neighbours; or ParIMCENew, Algorithm 6: K = {u, v},
// cand = Γ(u) ∩ Γ(v), fini = ∅) or a piece of one handed over by another
// warp.  The search is Algorithm 1 (TTT) on an explicit stack:
//
//   node:   if cand = fini = ∅ emit K; else pivot p ∈ cand ∪ fini maximising
//           |cand ∩ Γ(p)| (ties: smallest vertex id), ext = cand \ Γ(p);
//   child:  for q ∈ ext in ascending id: (K+q, cand ∩ Γ(q), fini ∩ Γ(q)),
//           then cand -= q, fini += q.
//
// Subproblem layout (per warp, shared memory when it fits, else a private
// global workspace): local vertices [0, c) are the candidates (ascending id),
// [c, W) the lower-ranked neighbours that touch a candidate.  Row A[x] is the
// bitset of candidates adjacent to local x (⌈c/32⌉ words, odd stride so
// that lanes reading different rows hit different banks).  cand and the
// candidates moved to fini ("finic") are bitsets over candidate columns; the
// lower-ranked part of fini is an index list F that each child partitions in
// place (vertices adjacent to q first), so a frame only stores its length.
// A fini vertex with no candidate neighbour can never block or pivot below
// the current node, so the pivot step drops it from F.
//
// Splitting (ParTTT, Algorithm 3): the children of a node only depend on the
// ext vertices before them, so a warp that sees idle warps hands the upper
// half of the remaining ext of its shallowest open frame to a device queue as
// (K, cand \ ext_lo, fini ∪ ext_lo, ext_hi).  Thieves rebuild the subproblem
// (deterministic layout) and continue from that frame.
//
// Incremental mode (Algorithm 7): X[x] = local vertices joined to x by an
// earlier new edge e_j, j < i.  conf = ∪_{w ∈ K} X[w] is kept per frame; at
// node entry cand ∩ conf moves to fini.  Such a q can lie in no output clique
// (K+q would contain an excluded edge) yet still blocks non-maximal ones, the
// effect of Algorithm 9's "cand -= q; fini += q; continue".
#include "bk.cuh"

namespace mce {

namespace {

constexpr uint32_t FULL = 0xffffffffu;

struct Ws {
    int32_t w, c, W, f, wc, S;   // local vertices, candidates, kept vertices, kept fini, words, stride
    int32_t *gid;
    int32_t *bnd;                 // popc(A[x]): bound on |cand ∩ Γ(x)| at every node
    int32_t *F0;                  // kept lower-ranked vertices sorted by bnd, descending
    uint32_t *Cb;                 // per candidate q: bitset over F0 positions adjacent to q
    int32_t Wf0;                  // words of one Cb row
    uint32_t *A;
    uint32_t *X;                  // IMCE exclusion rows
    int32_t *F, *Fs;
    uint32_t *fr;                 // frames
    int32_t *kpath;               // K path of the current task (local ids)
    int32_t frw;                  // words per frame
    int32_t dcap;                 // frames available
    uint32_t *piv;                // this warp's pivot scratch in shared memory
    // lane-parallel small search: this warp's region in shared memory (root
    // table, then the arena of relabelled universes), roots and arena words in use
    uint32_t *lp;
    int32_t lp_n, lp_top;
};

__device__ __forceinline__ uint32_t *fr_cand(const Ws &s, int d) { return s.fr + (int64_t)d * s.frw; }
__device__ __forceinline__ uint32_t *fr_finic(const Ws &s, int d) { return s.fr + (int64_t)d * s.frw + s.wc; }
__device__ __forceinline__ uint32_t *fr_ext(const Ws &s, int d) { return s.fr + (int64_t)d * s.frw + 2 * s.wc; }
__device__ __forceinline__ uint32_t *fr_conf(const Ws &s, int d) { return s.fr + (int64_t)d * s.frw + 3 * s.wc; }
__device__ __forceinline__ uint32_t *fr_meta(const Ws &s, int d) { return s.fr + (int64_t)d * s.frw + 4 * s.wc; }
// meta: [0] F length, [1] q (local id added at this frame, -1 at the task root), [2..3] hash sum

__device__ __forceinline__ uint64_t meta_hsum(const uint32_t *m) { return (uint64_t)m[2] | ((uint64_t)m[3] << 32); }
__device__ __forceinline__ void meta_set_hsum(uint32_t *m, uint64_t h) {
    m[2] = (uint32_t)h;
    m[3] = (uint32_t)(h >> 32);
}

__device__ __forceinline__ void ws_layout(Ws &s, uint32_t *base, int32_t w, int32_t c, int32_t mode) {
    s.w = w;
    s.c = c;
    s.wc = (c + 31) >> 5;
    s.S = (int32_t)bk_row_stride(s.wc);
    s.frw = 4 * s.wc + 4;
    uint32_t *p = base;
    s.gid = reinterpret_cast<int32_t *>(p);
    p += w;
    s.bnd = reinterpret_cast<int32_t *>(p);
    p = base + bk_align4(2 * (int64_t)w);
    s.A = p;
    p += (int64_t)w * s.S;
    s.F0 = reinterpret_cast<int32_t *>(p);
    p += (w - c);
    s.F = reinterpret_cast<int32_t *>(p);
    p += (w - c);
    s.Fs = reinterpret_cast<int32_t *>(p);
    p += (w - c);
    s.fr = p;
    s.dcap = (int32_t)bk_depth_cap(c);
    p += (int64_t)s.dcap * s.frw;
    s.kpath = reinterpret_cast<int32_t *>(p);
    p += (c + 2);
    s.X = (mode == BK_IMCE) ? p : nullptr;
    s.Cb = nullptr;
    s.Wf0 = 0;
}

// MCE layout split in a read-only part (possibly shared through the build
// cache) and the warp's private search state.
__device__ __forceinline__ void ws_layout_split(Ws &s, uint32_t *shared, uint32_t *priv, int32_t w, int32_t c) {
    s.w = w;
    s.c = c;
    s.wc = (c + 31) >> 5;
    s.S = (int32_t)bk_row_stride(s.wc);
    s.frw = 4 * s.wc + 4;
    uint32_t *p = shared + 32;
    s.gid = reinterpret_cast<int32_t *>(p);
    p += w;
    s.bnd = reinterpret_cast<int32_t *>(p);
    p = shared + bk_align4(32 + 2 * (int64_t)w);
    s.A = p;
    p += (int64_t)w * s.S;
    s.F0 = reinterpret_cast<int32_t *>(p);
    p += (w - c);
    s.Wf0 = (w - c + 31) >> 5;
    s.Cb = p;
    p = priv;
    s.F = reinterpret_cast<int32_t *>(p);
    p += (w - c);
    s.Fs = reinterpret_cast<int32_t *>(p);
    p += (w - c);
    s.fr = p;
    s.dcap = (int32_t)bk_depth_cap(c);
    p += (int64_t)s.dcap * s.frw;
    s.kpath = reinterpret_cast<int32_t *>(p);
    s.X = nullptr;
}

// warp: true if any of the n words is non-zero
__device__ __forceinline__ bool warp_any(const uint32_t *a, int n, int lane) {
    bool nz = false;
    for (int k = lane; k < n; k += 32) nz |= a[k] != 0;
    return __any_sync(FULL, nz);
}

// warp: position of the lowest set bit of a[0..n), or -1
__device__ __forceinline__ int warp_first_bit(const uint32_t *a, int n, int lane) {
    for (int k0 = 0; k0 < n; k0 += 32) {
        const int k = k0 + lane;
        const uint32_t x = k < n ? a[k] : 0u;
        const uint32_t b = __ballot_sync(FULL, x != 0);
        if (b) {
            const int src = __ffs(b) - 1;
            const uint32_t xs = __shfl_sync(FULL, x, src);
            return ((k0 + src) << 5) + (__ffs(xs) - 1);
        }
    }
    return -1;
}

// warp: number of set bits of a[0..n)
__device__ __forceinline__ int warp_popc(const uint32_t *a, int n, int lane) {
    int c = 0;
    for (int k = lane; k < n; k += 32) c += __popc(a[k]);
    return __reduce_add_sync(FULL, c);
}

// binary search of y in sorted g[0..c); -1 if absent
__device__ __forceinline__ int bsearch_i32(const int32_t *g, int c, int32_t y) {
    int lo = 0, hi = c;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (g[mid] < y) lo = mid + 1; else hi = mid;
    }
    return (lo < c && g[lo] == y) ? lo : -1;
}

// Partition F[0..len) so that the entries with pred true come first; the
// others follow (both kept).  Returns the number with pred true.  Each chunk
// is read into registers before any lane writes, and writes to the front only
// reach positions already read.
template <class Pred>
__device__ int partition_F(const Ws &s, int len, int lane, Pred pred) {
    int wpos = 0, spos = 0;
    for (int b0 = 0; b0 < len; b0 += 32) {
        const int i = b0 + lane;
        const bool valid = i < len;
        const int32_t u = valid ? s.F[i] : 0;
        const bool pr = valid && pred(u);
        const uint32_t bp = __ballot_sync(FULL, pr);
        const uint32_t bn = __ballot_sync(FULL, valid && !pr);
        __syncwarp();
        if (pr) s.F[wpos + __popc(bp & lanemask_lt())] = u;
        if (valid && !pr) s.Fs[spos + __popc(bn & lanemask_lt())] = u;
        wpos += __popc(bp);
        spos += __popc(bn);
        __syncwarp();
    }
    for (int i = lane; i < spos; i += 32) s.F[wpos + i] = s.Fs[i];
    __syncwarp();
    return wpos;
}

// F[0..a) and F[a..len) are each sorted by bnd (descending); merge them
// stably (the first run wins ties) through the scratch array.  Output
// positions come from ranks in the other run (merge path), so lanes write
// disjoint slots.
__device__ void merge_F(const Ws &s, int a, int len, int lane) {
    const int b = len - a;
    if (a == 0 || b == 0) return;
    for (int i = lane; i < a; i += 32) {
        const int32_t x = s.F[i];
        const int32_t key = s.bnd[x];
        int lo = 0, hi = b;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (s.bnd[s.F[a + mid]] > key) lo = mid + 1; else hi = mid;
        }
        s.Fs[i + lo] = x;
    }
    for (int j = lane; j < b; j += 32) {
        const int32_t x = s.F[a + j];
        const int32_t key = s.bnd[x];
        int lo = 0, hi = a;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (s.bnd[s.F[mid]] >= key) lo = mid + 1; else hi = mid;
        }
        s.Fs[j + lo] = x;
    }
    __syncwarp();
    for (int i = lane; i < len; i += 32) s.F[i] = s.Fs[i];
    __syncwarp();
}

// bnd[x] = popc(A[x]) for every kept local vertex, and F0 = the kept
// lower-ranked vertices [c, W) ordered by bnd descending (counting sort; the
// frames area serves as the histogram before any frame exists).
__device__ void sort_F0(const Ws &s, int lane) {
    for (int x = lane; x < s.W; x += 32) {
        const uint32_t *row = s.A + (int64_t)x * s.S;
        int b = 0;
        for (int k = 0; k < s.wc; ++k) b += __popc(row[k]);
        s.bnd[x] = b;
    }
    if (s.f == 0) {
        __syncwarp();
        return;
    }
    int32_t *hist = reinterpret_cast<int32_t *>(s.fr);
    for (int b = lane; b <= s.c; b += 32) hist[b] = 0;
    __syncwarp();
    for (int x = s.c + lane; x < s.W; x += 32) atomicAdd(&hist[s.bnd[x]], 1);
    __syncwarp();
    // start[b] = number of kept vertices with a larger bound
    int run = 0;
    for (int top = s.c; top >= 0; top -= 32) {
        const int b = top - lane;
        const int h = b >= 0 ? hist[b] : 0;
        int incl = h;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
        }
        if (b >= 0) hist[b] = run + incl - h;
        run += __shfl_sync(FULL, incl, 31);
    }
    __syncwarp();
    for (int x = s.c + lane; x < s.W; x += 32) s.F0[atomicAdd(&hist[s.bnd[x]], 1)] = x;
    __syncwarp();
}

// ------------------------------------------------------------------ subproblem build

// ParMCE subproblem of v (Algorithm 5).  Local order: Γ+(v) (the candidates,
// ascending id), then the lower-ranked neighbours (ascending id).  Row A[x]
// marks the candidates adjacent to x.  Every candidate y adjacent to x has
// rank(y) > rank(v) > rank(x) when x is lower ranked, so y ∈ Γ+(x); for two
// candidates the edge lies in Γ+ of the lower-ranked one.  Scanning Γ+(x) for
// every local x therefore finds each needed adjacency exactly once.
// Γ+(x) longer than this many times |C| is searched for the candidates (a
// galloping search through the long list) instead of looking up each of its
// elements in C (binary searches in the short, L1-resident list).  Measured
// on GB300: 2 keeps the R-MAT 18 search as it was and halves the build-bound
// Chung-Lu searches (hubs with long Γ+ lists).
constexpr int BK_BUILD_REVERSE = 2;

__device__ void build_mce(const BkParams &P, Ws &s, int32_t v, int lane) {
    const int32_t r0 = P.row_ptr[v], w = P.row_ptr[v + 1] - r0;
    const int32_t u0 = P.up_ptr[v], c = P.up_ptr[v + 1] - u0;
    for (int i = lane; i < c; i += 32) s.gid[i] = P.up_col[u0 + i];
    {
        const int32_t rv = P.rank[v];
        int out = c;
        for (int e0 = 0; e0 < w; e0 += 32) {
            const int e = e0 + lane;
            int32_t x = 0;
            bool low = false;
            if (e < w) {
                x = P.col[r0 + e];
                low = P.rank[x] < rv;
            }
            const uint32_t b = __ballot_sync(FULL, low);
            if (low) s.gid[out + __popc(b & lanemask_lt())] = x;
            out += __popc(b);
        }
    }
    const int64_t awords = (int64_t)w * s.S;
    for (int64_t k = lane; k < awords; k += 32) s.A[k] = 0u;
    __syncwarp();
    // Γ+(x) ∩ C for every local x (Γ+ lists and C are sorted by id): each
    // element of Γ+(x) is looked up in C, unless Γ+(x) is much longer than C
    // (hubs), whose lists have the candidates searched in them instead
    for (int x = lane; x < w; x += 32) {
        const int32_t gx = s.gid[x];
        const int32_t e0 = P.up_ptr[gx], d = P.up_ptr[gx + 1] - e0;
        const int32_t *gl = P.up_col + e0;
        auto found = [&](int j) {
            atomicOr(&s.A[(int64_t)x * s.S + (j >> 5)], 1u << (j & 31));
            if (x < c) atomicOr(&s.A[(int64_t)j * s.S + (x >> 5)], 1u << (x & 31));
        };
        if (d > BK_BUILD_REVERSE * c) {
            // galloping search: the candidates ascend, so each search starts
            // where the previous one ended
            int32_t pos = 0;
            for (int j = 0; j < c && pos < d; ++j) {
                const int32_t y = s.gid[j];
                int32_t step = 1, lo = pos;
                while (pos + step < d && gl[pos + step] < y) {
                    lo = pos + step;
                    step <<= 1;
                }
                int32_t hi = pos + step < d ? pos + step + 1 : d;
                while (lo < hi) {
                    const int32_t mid = (lo + hi) >> 1;
                    if (gl[mid] < y) lo = mid + 1; else hi = mid;
                }
                pos = lo;
                if (pos < d && gl[pos] == y) found(j);
            }
        } else {
            for (int32_t e = 0; e < d; ++e) {
                const int j = bsearch_i32(s.gid, c, gl[e]);
                if (j >= 0) found(j);
            }
        }
    }
    __syncwarp();
    // keep the lower-ranked neighbours that touch a candidate; rows only move down
    int f = 0;
    for (int b0 = c; b0 < w; b0 += 32) {
        const int x = b0 + lane;
        bool nz = false;
        if (x < w)
            for (int k = 0; k < s.wc; ++k) nz |= s.A[(int64_t)x * s.S + k] != 0u;
        uint32_t keep = __ballot_sync(FULL, nz);
        while (keep) {
            const int l = __ffs(keep) - 1;
            keep &= keep - 1;
            const int src = b0 + l, dst = c + f;
            if (src != dst) {
                for (int k = lane; k < s.S; k += 32) s.A[(int64_t)dst * s.S + k] = s.A[(int64_t)src * s.S + k];
                if (lane == 0) s.gid[dst] = s.gid[src];
            }
            ++f;
            __syncwarp();
        }
    }
    s.f = f;
    s.W = c + f;
    __syncwarp();
    sort_F0(s, lane);
    // Cb[q] = F0 positions whose vertex is adjacent to candidate q
    const int64_t cbw = (int64_t)c * s.Wf0;
    for (int64_t k = lane; k < cbw; k += 32) s.Cb[k] = 0u;
    __syncwarp();
    for (int pos = lane; pos < f; pos += 32) {
        const uint32_t *row = s.A + (int64_t)s.F0[pos] * s.S;
        for (int k = 0; k < s.wc; ++k) {
            uint32_t m = row[k];
            while (m) {
                const int q = (k << 5) + __ffs(m) - 1;
                m &= m - 1;
                atomicOr(&s.Cb[(int64_t)q * s.Wf0 + (pos >> 5)], 1u << (pos & 31));
            }
        }
    }
    __syncwarp();
}

// F for a child of the root (or the first step of a handed-over path):
// F0 ∩ Γ(q) in F0 order, read off q's column bitset.  Returns its length.
__device__ int compact_cb(const Ws &s, int q, int lane) {
    const uint32_t *cb = s.Cb + (int64_t)q * s.Wf0;
    int out = 0;
    for (int w0 = 0; w0 < s.Wf0; w0 += 32) {
        const int k = w0 + lane;
        uint32_t m = k < s.Wf0 ? cb[k] : 0u;
        const int pc = __popc(m);
        int incl = pc;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
        }
        int j = out + incl - pc;
        while (m) {
            s.F[j++] = s.F0[(k << 5) + __ffs(m) - 1];
            m &= m - 1;
        }
        out += __shfl_sync(FULL, incl, 31);
    }
    __syncwarp();
    return out;
}

// ParIMCENew subproblem of new edge i = (u, v) (Algorithm 6): local vertices
// are V_e \ {u, v} = Γ'(u) ∩ Γ'(v), all candidates; fini is empty.
// Adjacency within V_e comes from the degree-oriented Γ'+ lists; X rows and
// the root conflict set from the batch adjacency restricted to indices < i.
__device__ void build_imce(const BkParams &P, Ws &s, int32_t i, int lane) {
    const int32_t u = P.eu[i], v = P.ev[i];
    int32_t a = u, b = v;
    if (P.row_ptr[a + 1] - P.row_ptr[a] > P.row_ptr[b + 1] - P.row_ptr[b]) {
        a = v;
        b = u;
    }
    const int32_t a0 = P.row_ptr[a], la = P.row_ptr[a + 1] - a0;
    const int32_t b0 = P.row_ptr[b], lb = P.row_ptr[b + 1] - b0;
    int c = 0;
    for (int e0 = 0; e0 < la; e0 += 32) {
        const int e = e0 + lane;
        int32_t x = 0;
        bool hit = false;
        if (e < la) {
            x = P.col[a0 + e];
            hit = bsearch_i32(P.col + b0, lb, x) >= 0;
        }
        const uint32_t bl = __ballot_sync(FULL, hit);
        if (hit) s.gid[c + __popc(bl & lanemask_lt())] = x;
        c += __popc(bl);
    }
    __syncwarp();
    // the layout was sized for the bound min(deg); re-derive it for the actual c
    s.c = c;
    s.wc = (c + 31) >> 5;
    s.S = (int32_t)bk_row_stride(s.wc);
    s.frw = 4 * s.wc + 4;
    s.w = c;
    s.W = c;
    s.f = 0;
    {
        uint32_t *p = reinterpret_cast<uint32_t *>(s.gid) + c;
        s.bnd = reinterpret_cast<int32_t *>(p);
        p = reinterpret_cast<uint32_t *>(s.gid) + bk_align4(2 * (int64_t)c);
        s.A = p;
        p += (int64_t)c * s.S;
        s.F0 = reinterpret_cast<int32_t *>(p);
        s.F = s.F0;
        s.Fs = s.F;
        s.fr = p;
        s.dcap = (int32_t)bk_depth_cap(c);
        p += (int64_t)s.dcap * s.frw;
        s.kpath = reinterpret_cast<int32_t *>(p);
        p += (c + 2);
        s.X = p;
    }
    uint32_t *root_conf = fr_conf(s, 0);
    const int64_t rows = (int64_t)c * s.S;
    for (int64_t k = lane; k < rows; k += 32) {
        s.A[k] = 0u;
        s.X[k] = 0u;
    }
    for (int k = lane; k < s.wc; k += 32) root_conf[k] = 0u;
    __syncwarp();
    for (int x = lane; x < c; x += 32) {
        const int32_t gx = s.gid[x];
        for (int32_t e = P.up_ptr[gx]; e < P.up_ptr[gx + 1]; ++e) {
            const int j = bsearch_i32(s.gid, c, P.up_col[e]);
            if (j >= 0) {
                atomicOr(&s.A[(int64_t)x * s.S + (j >> 5)], 1u << (j & 31));
                atomicOr(&s.A[(int64_t)j * s.S + (x >> 5)], 1u << (x & 31));
            }
        }
        for (int32_t e = P.h_ptr[gx]; e < P.h_ptr[gx + 1]; ++e) {
            if (P.h_idx[e] >= i) continue;
            const int j = bsearch_i32(s.gid, c, P.h_adj[e]);
            if (j >= 0) atomicOr(&s.X[(int64_t)x * s.S + (j >> 5)], 1u << (j & 31));
        }
    }
    for (int t = 0; t < 2; ++t) {
        const int32_t z = t == 0 ? u : v;
        for (int32_t e = P.h_ptr[z] + lane; e < P.h_ptr[z + 1]; e += 32) {
            if (P.h_idx[e] >= i) continue;
            const int j = bsearch_i32(s.gid, c, P.h_adj[e]);
            if (j >= 0) atomicOr(&root_conf[j >> 5], 1u << (j & 31));
        }
    }
    __syncwarp();
    for (int x = lane; x < c; x += 32) {
        const uint32_t *row = s.A + (int64_t)x * s.S;
        int b = 0;
        for (int k = 0; k < s.wc; ++k) b += __popc(row[k]);
        s.bnd[x] = b;
    }
    __syncwarp();
}

// ------------------------------------------------------------------ output

// Counters touched a few times per task live in shared memory, one set per
// warp (lane 0 updates them), to keep registers for the search.
struct AccCold {
    unsigned long long build_ns, idle_ns, builds, pieces, max_busy, maxsize;
    unsigned long long count, hash, nodes;   // whole launch
    unsigned long long t_rep;                // this task's nodes already credited to sub_nodes / graph_nodes
    unsigned long long t_split;              // this task's nodes at its last hand-over
};
__shared__ AccCold g_cold[8];   // warps of one search block
__device__ __forceinline__ AccCold &cold() { return g_cold[threadIdx.x >> 5]; }

struct Acc {
    unsigned long long wops;                 // per lane: algorithmic word operations
    unsigned long long t_count, t_hash, t_nodes;   // per task
    int tick;                                      // nodes between checks (shorter in the endgame)
    int give;                                      // hand-overs per check at most
    int lp_hold;                                   // warps wait for work: small subtrees stay with the whole warp
};

// Algorithmic word operations of one tree node with |cand| = cn and |fini| =
// fn, `next` of whose children are searched: the pivot counts (cn + fn)
// members against ⌈cn/32⌉ words, and each child intersects cand and fini
// (2⌈(cn + fn)/32⌉ words).  Counted once per node, on lane 0.
__device__ __forceinline__ void count_node_wops(Acc &acc, int lane, int cn, int fn, int next) {
    if (lane == 0)
        acc.wops += (unsigned long long)(cn + fn) * (unsigned long long)((cn + 31) >> 5) +
                    2ull * (unsigned long long)next * (unsigned long long)((cn + fn + 31) >> 5);
}

__device__ void emit(const BkParams &P, const Ws &s, int32_t root, int32_t k0, int d, uint64_t hsum, Acc &acc,
                     unsigned long long *shist, int lane) {
    const uint32_t size = (uint32_t)(k0 + d);
    if (lane == 0) acc.wops += size;   // |K| additions of the clique hash
    const uint64_t h = clique_hash_from_sum(hsum, size);
    acc.t_count++;
    acc.t_hash += h;
    if (lane == 0) {
        if (size < 256) atomicAdd(&shist[size], 1ULL);
        else if (size < MCE_HIST_CAP) atomicAdd(&P.out[OUT_HIST + size], 1ULL);
        else atomicOr(&P.out[OUT_FLAGS], 2ULL);
    }
    if (lane == 0 && size > cold().maxsize) cold().maxsize = size;
    if (P.list_off) {
        unsigned long long pos = 0, idx = 0;
        if (lane == 0) {
            pos = atomicAdd(&P.out[OUT_LIST_WORDS], (unsigned long long)(size + 1));
            idx = atomicAdd(&P.out[OUT_LIST_CLIQUES], 1ULL);
        }
        pos = __shfl_sync(FULL, pos, 0);
        idx = __shfl_sync(FULL, idx, 0);
        if (idx >= (unsigned long long)P.list_max_cliques || pos + size + 1 > (unsigned long long)P.list_max_words) {
            if (lane == 0) atomicOr(&P.out[OUT_FLAGS], 1ULL);
            return;
        }
        // K = seed vertices, the task's path, then the q of frames 1..d
        int32_t *dst = P.list_vtx + pos;
        if (lane == 0) {
            dst[0] = (int32_t)size;
            P.list_off[idx] = (int64_t)pos;
        }
        int nseed;
        if (P.mode == BK_MCE) {
            nseed = 1;
            if (lane == 0) dst[1] = root;
        } else {
            nseed = 2;
            if (lane == 0) {
                dst[1] = P.eu[root];
                dst[2] = P.ev[root];
            }
        }
        const int npath = k0 - nseed;
        for (int j = lane; j < npath + d; j += 32) {
            const int32_t loc = j < npath ? s.kpath[j] : (int32_t)fr_meta(s, j - npath + 1)[1];
            dst[1 + nseed + j] = s.gid[loc];
        }
    }
}

// ------------------------------------------------------------------ task queue

// Bounded multi-producer multi-consumer ring (sequence numbers per slot, as
// in D. Vyukov's bounded MPMC queue).  Slot i holds one record of
// P.slot_words words at P.arena + i * slot_words.  qseq[i] == pos means free
// for the pusher holding ticket pos; == pos + 1 means published for the
// popper holding ticket pos; the popper sets it to pos + qcap when done.
// Neither side ever waits: a full ring refuses the push, an empty ring the pop.
__device__ int64_t queue_claim_push(const BkParams &P) {
    unsigned long long pos = *(volatile unsigned long long *)&P.ctl[CTL_QTAIL];
    for (int tries = 0; tries < 64; ++tries) {
        const unsigned long long seq = *(volatile unsigned long long *)&P.qseq[pos % (unsigned long long)P.qcap];
        const long long dif = (long long)seq - (long long)pos;
        if (dif == 0) {
            const unsigned long long prev = atomicCAS(&P.ctl[CTL_QTAIL], pos, pos + 1);
            if (prev == pos) return (int64_t)pos;
            pos = prev;
        } else if (dif < 0) {
            return -1;
        } else {
            pos = *(volatile unsigned long long *)&P.ctl[CTL_QTAIL];
        }
    }
    return -1;
}

__device__ void queue_publish(const BkParams &P, int64_t pos) {
    atomicAdd(&P.ctl[CTL_PENDING], 1ULL);
    __threadfence();
    atomicExch(&P.qseq[(unsigned long long)pos % (unsigned long long)P.qcap], (unsigned long long)pos + 1ULL);
}

__device__ int64_t queue_claim_pop(const BkParams &P) {
    unsigned long long pos = *(volatile unsigned long long *)&P.ctl[CTL_QHEAD];
    for (int tries = 0; tries < 64; ++tries) {
        const unsigned long long seq = *(volatile unsigned long long *)&P.qseq[pos % (unsigned long long)P.qcap];
        const long long dif = (long long)seq - (long long)(pos + 1);
        if (dif == 0) {
            const unsigned long long prev = atomicCAS(&P.ctl[CTL_QHEAD], pos, pos + 1);
            if (prev == pos) {
                __threadfence();
                return (int64_t)pos;
            }
            pos = prev;
        } else if (dif < 0) {
            return -1;
        } else {
            pos = *(volatile unsigned long long *)&P.ctl[CTL_QHEAD];
        }
    }
    return -1;
}

__device__ void queue_release(const BkParams &P, int64_t pos) {
    __threadfence();
    atomicExch(&P.qseq[(unsigned long long)pos % (unsigned long long)P.qcap],
               (unsigned long long)pos + (unsigned long long)P.qcap);
}

// ------------------------------------------------------------------ the search

struct Task {
    int32_t root;        // vertex (MCE) or edge index (IMCE)
    int32_t kdepth;      // vertices of K beyond the seeds
    int64_t rec;         // arena offset of a handed-over frame, -1 for a whole subproblem
};

// Budget, abort and splitting checks, made every 64 nodes with the current
// frame written back to memory.  Returns 0 = go on, 1 = stop the launch,
// 2 = drop this task (its graph or subproblem is over budget).
// Lane 0 reads the control words and credits node counts; the result is
// broadcast: returns 1 = stop the launch, 2 = drop this task, 0 = go on with
// `hungry` = the number of hand-overs wanted (0 = none).
__device__ int poll(const BkParams &P, Acc &acc, int lane, int32_t root, uint64_t t_start,
                    unsigned long long &hungry_out) {
    unsigned long long ab = 0, hungry = 0;
    int lph = 0;
    if (lane == 0) {
        if (globaltimer_ns() - t_start > P.max_run_ns) atomicOr(&P.ctl[CTL_ABORT], 2ULL);
        ab = *(volatile unsigned long long *)&P.ctl[CTL_ABORT];
        if (P.node_budget) {
            const unsigned long long tot = atomicAdd(&P.ctl[CTL_NODES], 64ULL) + 64ULL;
            if (tot > P.node_budget) {
                atomicOr(&P.ctl[CTL_ABORT], 1ULL);
                ab |= 1ULL;
            }
        }
        // exact node counts per subproblem and per graph: the task's nodes
        // since the last report (the rest is credited when the task ends), so
        // "over budget" holds exactly when the whole tree exceeds the budget
        const unsigned long long delta = acc.t_nodes - cold().t_rep;
        cold().t_rep = acc.t_nodes;
        if (P.sub_nodes) {
            const unsigned long long tot = atomicAdd(&P.sub_nodes[root], delta) + delta;
            if (tot > P.sub_budget) ab |= 16ULL;
        }
        if (P.graph_nodes) {
            const int32_t gg = P.graph_of[P.mode == BK_MCE ? root : P.eu[root]];
            const unsigned long long tot = atomicAdd(&P.graph_nodes[gg], delta) + delta;
            if (P.graph_budget && tot > P.graph_budget) ab |= 16ULL;
        }
        if (P.split) {
            hungry = *(volatile unsigned long long *)&P.ctl[CTL_HUNGRY];
            const unsigned long long qh = *(volatile unsigned long long *)&P.ctl[CTL_QHEAD];
            const unsigned long long qt = *(volatile unsigned long long *)&P.ctl[CTL_QTAIL];
            const unsigned long long qlen = qt > qh ? qt - qh : 0ULL;
            // while warps wait for work, small subtrees are searched by the whole
            // warp, whose frames can be handed over
            lph = P.lp_hold_waiting && hungry > qlen && hungry - qlen >= (unsigned long long)P.lp_hold_waiting;
            if (qlen >= hungry) hungry = 0;
            // a subproblem predicted heavy spreads its subtree from the start
            const bool heavy = P.heavy && P.heavy[P.mode == BK_MCE ? root : 0];
            const unsigned long long every = heavy ? P.heavy_split_nodes : P.split_nodes;
            // a task hands over again only after 2048 more nodes of its own
            // (fewer for a heavy one): pieces cut too small cost their receivers
            // more than they hold
            if (acc.t_nodes - cold().t_split < (heavy && every < 2048ULL ? every : 2048ULL)) hungry = 0;
            // a long-running task spreads its subtree before anybody waits
            if (!hungry && every && acc.t_nodes - cold().t_split >= every &&
                qlen < (unsigned long long)P.qcap / 2) hungry = 1;
        }
    }
    // endgame: every subproblem has been taken and warps wait for pieces; the
    // busy warps check four times as often and hand over up to 8 per check
    {
        bool endgame = false;
        if (lane == 0 && P.split)
            endgame = *(volatile unsigned long long *)&P.ctl[CTL_NEXT] >= (unsigned long long)P.n_sub &&
                      *(volatile unsigned long long *)&P.ctl[CTL_HUNGRY] > 0ULL;
        endgame = __shfl_sync(FULL, endgame, 0);
        acc.tick = endgame ? 16 : 64;
        acc.give = endgame ? 8 : 4;
    }
    ab = __shfl_sync(FULL, ab, 0);
    hungry = __shfl_sync(FULL, hungry, 0);
    acc.lp_hold = __shfl_sync(FULL, lph, 0);
    hungry_out = hungry;
    if (ab & 3ULL) return 1;
    if (ab & 16ULL) return 2;
    if (hungry && lane == 0) cold().t_split = acc.t_nodes;
    return 0;
}

// Hand over pending children of the memory frames 0..dmax (shallowest
// first): at most `budget` records.  Below frame `dcur` a single pending
// sibling is a whole subtree worth handing over (this warp stays busy in the
// child it is in); at frame dcur itself at least one child stays here.
__device__ void donate_mem(const BkParams &P, Ws &s, const Task &T, int lane, int dmax, int dcur, int32_t root,
                           int &budget) {
    for (int dd = 0; dd <= dmax && budget > 0; ++dd) {
        const uint32_t *ext = fr_ext(s, dd);
        const int rem = warp_popc(ext, s.wc, lane);
        if (rem < (dd < dcur ? 1 : 2)) continue;
        const int kd = T.kdepth + dd;
        int64_t pos = -1;
        if (lane == 0) pos = queue_claim_push(P);
        pos = __shfl_sync(FULL, pos, 0);
        if (pos < 0) break;
        // lower half stays here, upper half goes (all of it when one sibling remains below)
        const int keep = rem / 2;
        uint32_t *rec = P.arena + (int64_t)((unsigned long long)pos % (unsigned long long)P.qcap) * P.slot_words;
        if (lane == 0) {
            rec[0] = (uint32_t)root;
            rec[1] = (uint32_t)kd;
        }
        for (int j = lane; j < kd; j += 32)
            rec[2 + j] = (uint32_t)(j < T.kdepth ? s.kpath[j] : (int32_t)fr_meta(s, j - T.kdepth + 1)[1]);
        uint32_t *rb = rec + 2 + kd;
        uint32_t *cand = fr_cand(s, dd), *finic = fr_finic(s, dd), *ext2 = fr_ext(s, dd);
        const uint32_t *conf = fr_conf(s, dd);
        int seen = 0;
        for (int k0w = 0; k0w < s.wc; k0w += 32) {
            const int k = k0w + lane;
            const uint32_t e = k < s.wc ? ext2[k] : 0u;
            const int pc = __popc(e);
            int incl = pc;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += y;
            }
            const int before = seen + incl - pc;
            uint32_t lo = 0u;
            if (k < s.wc) {
                if (before + pc <= keep) lo = e;
                else if (before < keep) {
                    uint32_t x = e;
                    for (int t = 0; t < keep - before; ++t) {
                        const uint32_t bit = x & (0u - x);
                        lo |= bit;
                        x ^= bit;
                    }
                }
                rb[k] = cand[k] & ~lo;               // cand \ ext_lo
                rb[s.wc + k] = finic[k] | lo;        // fini ∪ ext_lo
                rb[2 * s.wc + k] = e & ~lo;          // ext_hi
                rb[3 * s.wc + k] = P.mode == BK_IMCE ? conf[k] : 0u;
                ext2[k] = lo;
            }
            seen += __shfl_sync(FULL, incl, 31);
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) {
            queue_publish(P, pos);
            atomicAdd(&P.out[OUT_SPLITS], 1ULL);
        }
        --budget;
        --dd;   // the same frame may still hold two or more children
    }
    __syncwarp();
}

// Checks made every 64 nodes with the current frame written back to memory.
// Returns 0 = go on, 1 = stop the launch, 2 = drop this task.
__device__ int periodic(const BkParams &P, Ws &s, const Task &T, Acc &acc, int lane, int d, int32_t root,
                        uint64_t t_start) {
    unsigned long long hungry = 0;
    const int code = poll(P, acc, lane, root, t_start, hungry);
    if (code || !hungry) return code;
    // up to four hand-overs per check when many warps wait
    int budget = hungry > (unsigned long long)acc.give ? acc.give : (int)hungry;
    donate_mem(P, s, T, lane, d, d, root, budget);
    return 0;
}

// word k of a set lives in register k / 32 of lane k % 32
// ------------------------------------------------------------------ small universe in registers
//
// Below a node whose candidates number at most 32 and whose fini (finic plus
// the F list) at most 32, the whole subtree runs on 32-bit masks (the same
// TTT steps on a relabelled universe):
//   C = the node's candidates, ascending local id (so ascending global id);
//   X = its fini vertices (finic members, then the F list).
// Lane l holds adjC = {k : C_l ~ C_k}, adjX = {k : X_l ~ C_k}, and in
// incremental mode exclC = {k : (C_l, C_k) is an excluded earlier edge}.
// A frame is (cand, finc ⊆ C, ext, xs ⊆ X, conf); the stack of saved frames
// lives in the warp's shared scratch.
// Hand-overs turn a mask frame back into a task record over the
// subproblem's columns (the receiver rebuilds F from the path).

struct SmallU {
    uint32_t adjC, adjX, exclC;
    uint32_t tC, tX;         // 127 - (position of the global id among C ∪ X): pivot tie keys
    int cn, xn;
};

// tables of the small search in the warp's shared scratch (read by broadcast)
__device__ __forceinline__ uint64_t *small_h(const Ws &s) { return reinterpret_cast<uint64_t *>(s.piv); }
__device__ __forceinline__ int32_t *small_gid(const Ws &s) { return reinterpret_cast<int32_t *>(s.piv + 320); }
__device__ __forceinline__ int32_t *small_cidc(const Ws &s) { return reinterpret_cast<int32_t *>(s.piv + 352); }
__device__ __forceinline__ int32_t *small_cidx(const Ws &s) { return reinterpret_cast<int32_t *>(s.piv + 384); }

// Stack frame j of the small search: 8 words in the warp's shared scratch,
// [cand, finc, ext, xs, conf, q (C index that created frame j), hsum lo, hi].
// Every lane stores the same words, so every lane reads back its own store.
constexpr int SMALL_FRAME = 8;
// small frames with fewer candidates than this are not handed over
constexpr int SMALL_DONATE_MIN_CAND = 8;

// C-index mask -> the lane's words of a bitset over the subproblem's
// candidate columns (or-ed into w); X members that are columns go to wf
template <int NR>
__device__ __forceinline__ void small_to_words(const Ws &s, uint32_t m, int lane, uint32_t (&w)[NR]) {
    const int32_t *cidc = small_cidc(s);
    while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1;
        const int32_t cid = cidc[b];
#pragma unroll
        for (int r = 0; r < NR; ++r)
            if (lane + 32 * r == (cid >> 5)) w[r] |= 1u << (cid & 31);
    }
}

// record of small frame fd (its masks given) with ext split: ext_lo stays
template <int NR>
__device__ bool small_donate(const BkParams &P, const Ws &s, const Task &T, const SmallU &u, int lane, int d,
                             int fd, int ds, const uint32_t *stk, int32_t qcur, uint32_t mc, uint32_t mf,
                             uint32_t mx, uint32_t mk, uint32_t ext, uint32_t &ext_lo, int32_t root) {
    const int rem = __popc(ext);
    const int keep = rem / 2;
    uint32_t lo = 0u, x = ext;
    for (int t = 0; t < keep; ++t) {
        const uint32_t bit = x & (0u - x);
        lo |= bit;
        x ^= bit;
    }
    const int kd = T.kdepth + d + fd;
    int64_t pos = -1;
    if (lane == 0) pos = queue_claim_push(P);
    pos = __shfl_sync(FULL, pos, 0);
    if (pos < 0) return false;
    uint32_t *rec = P.arena + (int64_t)((unsigned long long)pos % (unsigned long long)P.qcap) * P.slot_words;
    if (lane == 0) {
        rec[0] = (uint32_t)root;
        rec[1] = (uint32_t)kd;
    }
    const int k_out = T.kdepth + d;
    for (int j0 = 0; j0 < kd; j0 += 32) {
        const int j = j0 + lane;
        // small frame m = j - k_out + 1 was created by C index q_m
        const int m = j - k_out + 1;
        const int32_t qm = (m == ds) ? qcur : (int32_t)stk[(m > 0 && m < 32 ? m : 0) * SMALL_FRAME + 5];
        const int32_t loc_small = small_cidc(s)[(qm >= 0 ? qm : 0) & 31];
        if (j < kd) {
            int32_t loc;
            if (j < T.kdepth) loc = s.kpath[j];
            else if (j < k_out) loc = (int32_t)fr_meta(s, j - T.kdepth + 1)[1];
            else loc = loc_small;
            rec[2 + j] = (uint32_t)loc;
        }
    }
    uint32_t wcand[NR], wfin[NR], wext[NR], wconf[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) wcand[r] = wfin[r] = wext[r] = wconf[r] = 0u;
    small_to_words<NR>(s, mc & ~lo, lane, wcand);
    small_to_words<NR>(s, mf | lo, lane, wfin);
    small_to_words<NR>(s, ext & ~lo, lane, wext);
    if (P.mode == BK_IMCE) small_to_words<NR>(s, mk, lane, wconf);
    // X members that are candidate columns (finic of the small root) stay fini
    uint32_t xm = mx;
    while (xm) {
        const int b = __ffs(xm) - 1;
        xm &= xm - 1;
        const int32_t cid = small_cidx(s)[b];
        if (cid < s.c) {
#pragma unroll
            for (int r = 0; r < NR; ++r)
                if (lane + 32 * r == (cid >> 5)) wfin[r] |= 1u << (cid & 31);
        }
    }
    uint32_t *rb = rec + 2 + kd;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int k = lane + 32 * r;
        if (k < s.wc) {
            rb[k] = wcand[r];
            rb[s.wc + k] = wfin[r];
            rb[2 * s.wc + k] = wext[r];
            rb[3 * s.wc + k] = wconf[r];
        }
    }
    __threadfence();
    __syncwarp();
    if (lane == 0) {
        queue_publish(P, pos);
        atomicAdd(&P.out[OUT_SPLITS], 1ULL);
    }
    ext_lo = lo;
    return true;
}

// Relabel the node (cand rc, finic rf, F list Fd[0..flen)) as a small
// universe: u gets lane l's rows and tie keys, gC / cidC the global and local
// id of C_l, cidX the local id of X_l.  The C and X lists pass through the
// pivot scratch, which is free again on return.
template <int NR>
__device__ __forceinline__ void small_relabel(const BkParams &P, const Ws &s, int lane, const uint32_t (&rc)[NR],
                                              const uint32_t (&rf)[NR], const int32_t *Fd, int flen, SmallU &u,
                                              int32_t &gC, int32_t &cidC, int32_t &cidX) {
    const bool imce = P.mode == BK_IMCE;
    int32_t *Cl = reinterpret_cast<int32_t *>(s.piv + 64);
    int32_t *Xl = Cl + 32;
    {
        int base_c = 0, base_f = 0;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const uint32_t wcw = rc[r], wfw = rf[r];
            const int pc = __popc(wcw), pf = __popc(wfw);
            int ic = pc, jf = pf;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(FULL, ic, o);
                const int z = __shfl_up_sync(FULL, jf, o);
                if (lane >= o) {
                    ic += y;
                    jf += z;
                }
            }
            int pcs = base_c + ic - pc, pfs = base_f + jf - pf;
            uint32_t m = wcw;
            while (m) {
                Cl[pcs++] = ((lane + 32 * r) << 5) + __ffs(m) - 1;
                m &= m - 1;
            }
            m = wfw;
            while (m) {
                Xl[pfs++] = ((lane + 32 * r) << 5) + __ffs(m) - 1;
                m &= m - 1;
            }
            base_c += __shfl_sync(FULL, ic, 31);
            base_f += __shfl_sync(FULL, jf, 31);
        }
        u.cn = base_c;
        u.xn = base_f + flen;
        if (lane < flen) Xl[base_f + lane] = Fd[lane];
    }
    __syncwarp();
    cidC = lane < u.cn ? Cl[lane] : 0;
    cidX = lane < u.xn ? Xl[lane] : 0;
    u.adjC = u.adjX = u.exclC = 0u;
    {
        // C_k is the k-th candidate column in ascending order, so lane l's
        // rows restricted to C are read word by word over the non-empty words
        // of cand: one load per word and row, then a bit per candidate
        const uint32_t *rowC = s.A + (int64_t)cidC * s.S;
        const uint32_t *rowX = s.A + (int64_t)cidX * s.S;
        const uint32_t *xrow = imce ? s.X + (int64_t)cidC * s.S : nullptr;
        int k = 0;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            for (uint32_t nz = __ballot_sync(FULL, rc[r] != 0u); nz; nz &= nz - 1u) {
                const int j = __ffs(nz) - 1;
                const int w = j + 32 * r;
                uint32_t cw = __shfl_sync(FULL, rc[r], j);
                const uint32_t a = lane < u.cn ? rowC[w] : 0u;
                const uint32_t x = lane < u.xn ? rowX[w] : 0u;
                const uint32_t e = (imce && lane < u.cn) ? xrow[w] : 0u;
                for (; cw; cw &= cw - 1u, ++k) {
                    const int b = __ffs(cw) - 1;
                    u.adjC |= ((a >> b) & 1u) << k;
                    u.adjX |= ((x >> b) & 1u) << k;
                    u.exclC |= ((e >> b) & 1u) << k;
                }
            }
        }
    }
    {
        gC = lane < u.cn ? s.gid[cidC] : 0x7fffffff;
        const int32_t gX = lane < u.xn ? s.gid[cidX] : 0x7fffffff;
        // C is in increasing global id, so C_l has l smaller ids in C
        int oc = lane, ox = 0;
        for (int k = 0; k < u.xn; ++k) {
            const int32_t gk = __shfl_sync(FULL, gX, k);
            oc += gk < gC;
            ox += gk < gX;
        }
        for (int k = 0; k < u.cn; ++k) ox += __shfl_sync(FULL, gC, k) < gX;
        u.tC = 127u - (uint32_t)oc;
        u.tX = 127u - (uint32_t)ox;
    }
    __syncwarp();   // Cl / Xl are scratch again after this point
}

// The subtree of the node at memory depth d (its cand/finic in rc/rf, conf
// in rx, F list Fd[0..flen)), already counted, with cand not empty.
// Frames 0..d-1 are in memory.  Returns as search<NR>.
template <int NR>
__device__ int search_small(const BkParams &P, Ws &s, const Task &T, Acc &acc, unsigned long long *shist, int lane,
                            int &node_tick, uint64_t t_start, int32_t root, int k0, int d, uint64_t hsum,
                            const uint32_t (&rc)[NR], const uint32_t (&rf)[NR], const uint32_t (&rx)[NR],
                            const int32_t *Fd, int flen) {
    const bool imce = P.mode == BK_IMCE;
    SmallU u;
    int32_t gC, cidC, cidX;
    small_relabel<NR>(P, s, lane, rc, rf, Fd, flen, u, gC, cidC, cidX);
    // the tables live where the wide pivot keeps its cand and after the stack
    // (the relabel lists, read by now, sit inside the stack area)
    if (lane < u.cn) {
        small_h(s)[lane] = vertex_hash(gC, P.seed);
        small_gid(s)[lane] = gC;
        small_cidc(s)[lane] = cidC;
    }
    if (lane < u.xn) small_cidx(s)[lane] = cidX;
    uint32_t conf = 0u;
    if (imce) {
        const int wd = cidC >> 5;
        uint32_t wv = __shfl_sync(FULL, rx[0], wd & 31);
        if (NR > 1) {
            const uint32_t w1 = __shfl_sync(FULL, rx[NR - 1], wd & 31);
            if (wd >= 32) wv = w1;
        }
        conf = __ballot_sync(FULL, lane < u.cn && ((wv >> (cidC & 31)) & 1u));
    }
    __syncwarp();   // the tables are read by every lane below
    // ---- the search
    uint32_t cand = u.cn == 32 ? FULL : ((1u << u.cn) - 1u);
    uint32_t finc = 0u, ext = 0u;
    uint32_t xs = u.xn == 32 ? FULL : ((1u << u.xn) - 1u);
    int32_t qcur = -1;
    uint64_t hs = 0;
    int ds = 0;
    uint32_t *stk = s.piv + 64;   // 32 frames; the relabel lists there are dead now
    // nodes and word-ops since the last flush into acc (32-bit, warp-uniform)
    uint32_t n32 = 0, w32 = 0, smax = 0;
    auto flush = [&]() {
        acc.t_nodes += n32;
        if (lane == 0) {
            acc.wops += w32;
            if (smax > cold().maxsize) cold().maxsize = smax;
        }
        n32 = w32 = 0;
    };
    // emit K = seeds + task path + memory path + small frames 1..ds + qa + qb
    auto small_emit = [&](uint32_t size, uint64_t hsm, int qa, int qb) {
        const uint64_t h = clique_hash_from_sum(hsum + hsm, size);
        w32 += size;
        acc.t_count++;
        acc.t_hash += h;
        if (lane == 0) {
            if (size < 256) atomicAdd(&shist[size], 1ULL);
            else if (size < MCE_HIST_CAP) atomicAdd(&P.out[OUT_HIST + size], 1ULL);
            else atomicOr(&P.out[OUT_FLAGS], 2ULL);
        }
        if (size > smax) smax = size;
        if (P.list_off) {
            unsigned long long pos = 0, idx = 0;
            if (lane == 0) {
                pos = atomicAdd(&P.out[OUT_LIST_WORDS], (unsigned long long)(size + 1));
                idx = atomicAdd(&P.out[OUT_LIST_CLIQUES], 1ULL);
            }
            pos = __shfl_sync(FULL, pos, 0);
            idx = __shfl_sync(FULL, idx, 0);
            if (idx >= (unsigned long long)P.list_max_cliques || pos + size + 1 > (unsigned long long)P.list_max_words) {
                if (lane == 0) atomicOr(&P.out[OUT_FLAGS], 1ULL);
                return;
            }
            int32_t *dst = P.list_vtx + pos;
            const int nseed = P.mode == BK_MCE ? 1 : 2;
            if (lane == 0) {
                dst[0] = (int32_t)size;
                P.list_off[idx] = (int64_t)pos;
                if (P.mode == BK_MCE) {
                    dst[1] = root;
                } else {
                    dst[1] = P.eu[root];
                    dst[2] = P.ev[root];
                }
            }
            const int npath = k0 - nseed;
            for (int j = lane; j < npath + d; j += 32) {
                const int32_t loc = j < npath ? s.kpath[j] : (int32_t)fr_meta(s, j - npath + 1)[1];
                dst[1 + nseed + j] = s.gid[loc];
            }
            // small frame fj (1..ds, up to 32) was created by C index q_fj; lane fj-1 writes it
            const int fj = lane + 1;
            const int32_t qj = (fj == ds) ? qcur : (int32_t)stk[(fj & 31) * SMALL_FRAME + 5];
            const int32_t gq = small_gid(s)[(qj >= 0 ? qj : 0) & 31];
            if (fj <= ds) dst[nseed + npath + d + fj] = gq;
            const int32_t ga = small_gid(s)[(qa >= 0 ? qa : 0) & 31];
            const int32_t gb = small_gid(s)[(qb >= 0 ? qb : 0) & 31];
            if (lane == 0) {
                if (qa >= 0) dst[nseed + npath + d + ds + 1] = ga;
                if (qb >= 0) dst[nseed + npath + d + ds + 2] = gb;
            }
        }
    };
    bool enter = true;
    for (;;) {
        if (enter) {
            // (children arrive with the incremental-mode conflict move applied)
            if (cand == 0u) {
                if (finc == 0u && xs == 0u) small_emit((uint32_t)(k0 + d + ds), hs, -1, -1);
                goto pop;
            }
            // ---- pivot over cand ∪ finc (C) and xs (X), ties to the smallest global id
            {
                // key = (count + 1, tie key): distinct for every member, so one
                // reduction finds the pivot (largest count, then smallest id)
                const uint32_t cf = cand | finc;
                const uint32_t kc = ((cf >> lane) & 1u) ? ((__popc(cand & u.adjC) + 1u) << 7) | u.tC : 0u;
                const uint32_t kx = ((xs >> lane) & 1u) ? ((__popc(cand & u.adjX) + 1u) << 7) | u.tX : 0u;
                const uint32_t key = kx > kc ? kx : kc;
                const uint32_t mx = __reduce_max_sync(FULL, key);
                const uint32_t who = __ballot_sync(FULL, key == mx);
                const uint32_t adjp = __shfl_sync(FULL, kx == mx ? u.adjX : u.adjC, __ffs(who) - 1);
                ext = cand & ~adjp;
                const uint32_t t = (uint32_t)(__popc(cf) + __popc(xs));
                w32 += t + 2u * (uint32_t)__popc(ext) * ((t + 31u) >> 5);
            }
            enter = false;
            if (++node_tick >= acc.tick) {
                node_tick = 0;
                flush();
                unsigned long long hungry = 0;
                const int code = poll(P, acc, lane, root, t_start, hungry);
                if (code) return code;
                if (hungry) {
                    int budget = hungry > (unsigned long long)acc.give ? acc.give : (int)hungry;
                    // memory frames above the small root first, then small frames
                    if (d > 0) donate_mem(P, s, T, lane, d - 1, d, root, budget);
                    for (int fd = 0; fd <= ds && budget > 0; ++fd) {
                        const uint32_t *fr = stk + fd * SMALL_FRAME;
                        const uint32_t fe = fd < ds ? fr[2] : ext;
                        if (__popc(fe) < (fd < ds ? 1 : 2)) continue;
                        const uint32_t fc = fd < ds ? fr[0] : cand;
                        // a piece costs its receiver a rebuild of F along the path and
                        // a relabel; frames with few candidates hold too little work
                        if (__popc(fc) < SMALL_DONATE_MIN_CAND) break;
                        const uint32_t ff = fd < ds ? fr[1] : finc;
                        const uint32_t fx = fd < ds ? fr[3] : xs;
                        const uint32_t fk = fd < ds ? fr[4] : conf;
                        uint32_t lo = fe;
                        if (!small_donate<NR>(P, s, T, u, lane, d, fd, ds, stk, qcur, fc, ff, fx, fk, fe, lo, root))
                            break;
                        if (fd < ds) {
                            stk[fd * SMALL_FRAME + 2] = lo;
                        } else {
                            ext = lo;
                        }
                        --budget;
                        --fd;   // the same frame may still hold pending children
                    }
                }
            }
        }
        // ---- next child of the current frame
        {
            if (ext == 0u) goto pop;
            const int q = __ffs(ext) - 1;
            const uint32_t qb = 1u << q;
            ext &= ~qb;
            cand &= ~qb;
            finc |= qb;
            const uint32_t aq = __shfl_sync(FULL, u.adjC, q);
            const uint32_t xq = __ballot_sync(FULL, (u.adjX >> q) & 1u);
            const uint64_t hq = small_h(s)[q];
            uint32_t cc = cand & aq, cf = finc & aq, cx = xs & xq, ck = conf;
            if (imce) {
                // Algorithm 7: a candidate joined to K + q by an earlier new edge moves to fini
                ck |= __shfl_sync(FULL, u.exclC, q);
                const uint32_t mv = cc & ck;
                cf |= mv;
                cc &= ~mv;
            }
            if (cc == 0u) {
                // the child is a leaf: a maximal clique unless fini is left
                ++n32;
                ++node_tick;
                if (cf == 0u && cx == 0u) small_emit((uint32_t)(k0 + d + ds + 1), hs + hq, q, -1);
                continue;
            }
            if ((cc & (cc - 1u)) == 0u) {
                // one candidate c: every pivot count is 0 or 1, so the child has one
                // child of its own ({c}, a maximal clique) unless a fini vertex is
                // adjacent to c, in which case that vertex is the pivot and there is none
                const int c = __ffs(cc) - 1;
                const uint32_t ac = __shfl_sync(FULL, u.adjC, c);
                const uint32_t xc = __ballot_sync(FULL, (u.adjX >> c) & 1u);
                const uint32_t t = 1u + (uint32_t)(__popc(cf) + __popc(cx));
                if ((cf & ac) != 0u || (cx & xc) != 0u) {
                    ++n32;
                    ++node_tick;
                    w32 += t;
                } else {
                    n32 += 2;
                    node_tick += 2;
                    w32 += t + 2u * ((t + 31u) >> 5);
                    small_emit((uint32_t)(k0 + d + ds + 2), hs + hq + small_h(s)[c], q, c);
                }
                continue;
            }
            if (ds >= 32) {   // cannot happen: every frame adds a distinct member of C
                if (lane == 0) atomicOr(&P.ctl[CTL_ABORT], 4ULL);
                flush();
                return 1;
            }
            {
                uint4 *fp = reinterpret_cast<uint4 *>(stk + ds * SMALL_FRAME);
                fp[0] = make_uint4(cand, finc, ext, xs);
                fp[1] = make_uint4(conf, (uint32_t)qcur, (uint32_t)hs, (uint32_t)(hs >> 32));
            }
            cand = cc;
            finc = cf;
            xs = cx;
            conf = ck;
            hs += hq;
            qcur = q;
            ++ds;
            ++n32;
            enter = true;
            continue;
        }
    pop:
        if (ds == 0) {
            flush();
            return 0;
        }
        --ds;
        {
            const uint4 *fp = reinterpret_cast<const uint4 *>(stk + ds * SMALL_FRAME);
            const uint4 a = fp[0], b = fp[1];
            cand = a.x;
            finc = a.y;
            ext = a.z;
            xs = a.w;
            conf = b.x;
            qcur = (int32_t)b.y;
            hs = (uint64_t)b.z | ((uint64_t)b.w << 32);
        }
        enter = false;
    }
}

// ------------------------------------------------------------------ lane-parallel small search
//
// In static MCE without clique lists the small nodes are not searched by the
// whole warp one node at a time.  The warp relabels each small node it
// reaches (small_relabel) into a universe in its shared-memory arena and goes
// on with the wide search; when the arena or the root table is full, or the
// task ends, the lanes search the buffered subtrees (lp_run): the TTT step of
// search_small on 32-bit masks, one node per lane at a time, the nodes taken
// 32 at a time from a stack of entered nodes that the lanes share, so that
// the heavy-tailed subtree sizes spread over the lanes node by node.  Trees,
// node counts, word operations and cliques are those of search_small.
//
// Universe of a small node with cn candidates and xn fini vertices (arena
// words): h(C_k) as uint64 [2 cn]; per C member its row adjC and tie key
// [2 cn]; per X member its row adjX and tie key [2 xn] (a row and its key are
// read together as one 8-byte word); the columns of adjX (adjXT[k] =
// {x : X_x ~ C_k}) [cn].  Root record (4 words): arena offset,
// cn | xn << 8 | (clique size at the node) << 16, hash sum at the node.

__device__ __forceinline__ int lp_universe_words(int cn, int xn) { return (5 * cn + 2 * xn + 1) & ~1; }

struct LpSums {
    unsigned long long hash, wops;
    uint32_t count, nodes, smax;
};

// A small-subtree node for one lane: its universe and its state.
struct LpNode {
    const uint64_t *hC;
    const uint2 *akC, *akX;   // (row, tie key) per C / X member
    const uint32_t *adjXT;
    int cn;
    uint32_t base;     // clique size at the universe's root
    uint32_t cand, finc, xs;
    uint64_t hs;
    int depth;         // below the universe's root
};

__device__ __forceinline__ void lp_emit(const BkParams &P, unsigned long long *shist, LpSums &o, uint32_t size,
                                        uint64_t hsum) {
    o.count++;
    o.hash += clique_hash_from_sum(hsum, size);
    o.wops += size;
    if (size < 256) atomicAdd(&shist[size], 1ULL);
    else if (size < MCE_HIST_CAP) atomicAdd(&P.out[OUT_HIST + size], 1ULL);
    else atomicOr(&P.out[OUT_FLAGS], 2ULL);
    if (size > o.smax) o.smax = size;
}

// Pivot of an entered node (cand not empty): ext = cand minus the pivot's
// neighbours, with the pivot the largest (count + 1, tie key) over cand ∪
// finc and xs (the order of search_small).
__device__ __forceinline__ uint32_t lp_pivot_ext(const LpNode &u, LpSums &o) {
    const uint32_t cf = u.cand | u.finc;
    uint32_t best = 0u, badj = 0u;
    for (uint32_t m = cf; m; m &= m - 1u) {
        const uint2 ak = u.akC[__ffs(m) - 1];
        const uint32_t kk = ((uint32_t)(__popc(u.cand & ak.x) + 1) << 7) | ak.y;
        if (kk > best) {
            best = kk;
            badj = ak.x;
        }
    }
    for (uint32_t m = u.xs; m; m &= m - 1u) {
        const uint2 ak = u.akX[__ffs(m) - 1];
        const uint32_t kk = ((uint32_t)(__popc(u.cand & ak.x) + 1) << 7) | ak.y;
        if (kk > best) {
            best = kk;
            badj = ak.x;
        }
    }
    const uint32_t ext = u.cand & ~badj;
    const uint32_t t = (uint32_t)(__popc(cf) + __popc(u.xs));
    o.wops += t + 2u * (uint32_t)__popc(ext) * ((t + 31u) >> 5);
    return ext;
}

// Child N = K + q with two candidates a < b (fini cf, cx), settled in closed
// form with the node counts, word operations and cliques of the search:
//   - a fini vertex adjacent to both is the pivot (count 2): N has no child;
//   - a ~ b: the pivot has count 1 and N has one child, whose one candidate
//     gives the clique N + a + b (two more nodes);
//   - a !~ b and a fini vertex adjacent to one of them: it is the pivot, and
//     N's one child (the other candidate) is a leaf, a clique unless a fini
//     vertex is adjacent to it;
//   - otherwise every count is 0: both candidates are leaf children and both
//     N + a and N + b are cliques.
__device__ __forceinline__ void lp_two(const BkParams &P, unsigned long long *shist, const LpNode &u, int q, LpSums &o,
                                       uint32_t cc, uint32_t cf, uint32_t cx, uint64_t hq) {
    const int a = __ffs(cc) - 1, b = __ffs(cc & (cc - 1u)) - 1;
    const uint2 ka = u.akC[a], kb = u.akC[b];
    const uint32_t xa = u.adjXT[a], xb = u.adjXT[b];
    const uint32_t t = 2u + (uint32_t)(__popc(cf) + __popc(cx));
    const uint32_t sz = u.base + (uint32_t)u.depth + 1u;   // |N|
    const uint64_t hn = u.hs + hq;                         // hash sum of N
    ++o.nodes;                                             // N
    if ((cf & ka.x & kb.x) != 0u || (cx & xa & xb) != 0u) {
        o.wops += t;
        return;
    }
    const uint32_t wt = 2u * ((t + 31u) >> 5);
    const uint32_t f1c = cf & (ka.x ^ kb.x), f1x = cx & (xa ^ xb);   // fini adjacent to exactly one
    // the fini member of f1 with the highest tie key, and whether it touches a
    uint32_t fk = 0u;
    bool f_on_a = false;
    for (uint32_t m = f1c; m; m &= m - 1u) {
        const int k = __ffs(m) - 1;
        const uint32_t kk = u.akC[k].y;
        if (kk >= fk) {
            fk = kk + 1u;
            f_on_a = (ka.x >> k) & 1u;
        }
    }
    for (uint32_t m = f1x; m; m &= m - 1u) {
        const int x = __ffs(m) - 1;
        const uint32_t kk = u.akX[x].y;
        if (kk >= fk) {
            fk = kk + 1u;
            f_on_a = (xa >> x) & 1u;
        }
    }
    if ((ka.x >> b) & 1u) {
        // a ~ b: pivot among a, b and f1 by tie key; the child is a if the pivot is
        // a or a fini vertex on b only, else b
        const uint32_t best = max(max(ka.y, kb.y) + 1u, fk);
        int qq;
        if (best == ka.y + 1u) qq = a;
        else if (best == kb.y + 1u) qq = b;
        else qq = f_on_a ? b : a;
        const uint32_t rq = qq == a ? ka.x : kb.x, xq = qq == a ? xa : xb;
        o.wops += t + wt;
        const uint32_t tg = 1u + (uint32_t)(__popc(cf & rq) + __popc(cx & xq));
        o.nodes += 2;
        o.wops += tg + 2u * ((tg + 31u) >> 5);
        lp_emit(P, shist, o, sz + 2u, hn + u.hC[a] + u.hC[b]);
        return;
    }
    if (fk) {
        // a !~ b: the pivot is the fini vertex; its other candidate is the child
        const int qq = f_on_a ? b : a;
        const uint32_t rq = qq == a ? ka.x : kb.x, xq = qq == a ? xa : xb;
        o.wops += t + wt;
        ++o.nodes;
        if ((cf & rq) == 0u && (cx & xq) == 0u) lp_emit(P, shist, o, sz + 1u, hn + u.hC[qq]);
        return;
    }
    // all counts 0: both candidates are children, both leaves and cliques
    o.wops += t + 2u * wt;
    o.nodes += 2;
    lp_emit(P, shist, o, sz + 1u, hn + u.hC[a]);
    lp_emit(P, shist, o, sz + 1u, hn + u.hC[b]);
}

// Child q of a node whose cand / finc already exclude / include q: leaves
// and one-candidate children are settled here (returns false); otherwise the
// child's sets are returned for a push (returns true).  Node counts and word
// operations follow search_small.
__device__ __forceinline__ bool lp_child(const BkParams &P, unsigned long long *shist, const LpNode &u, int q,
                                         LpSums &o, uint32_t &cc, uint32_t &cf, uint32_t &cx, uint64_t &hq) {
    const uint32_t aq = u.akC[q].x;
    cc = u.cand & aq;
    cf = u.finc & aq;
    cx = u.xs & u.adjXT[q];
    hq = u.hC[q];
    if (cc == 0u) {
        // a leaf: a maximal clique unless fini is left
        ++o.nodes;
        if ((cf | cx) == 0u) lp_emit(P, shist, o, u.base + (uint32_t)u.depth + 1u, u.hs + hq);
        return false;
    }
    if ((cc & (cc - 1u)) == 0u) {
        // one candidate c: one more node and the clique K + q + c, unless a fini
        // vertex adjacent to c is the pivot (then no child)
        const int c = __ffs(cc) - 1;
        const uint32_t t = 1u + (uint32_t)(__popc(cf) + __popc(cx));
        if ((cf & u.akC[c].x) != 0u || (cx & u.adjXT[c]) != 0u) {
            ++o.nodes;
            o.wops += t;
        } else {
            o.nodes += 2;
            o.wops += t + 2u * ((t + 31u) >> 5);
            lp_emit(P, shist, o, u.base + (uint32_t)u.depth + 2u, u.hs + hq + u.hC[c]);
        }
        return false;
    }
    if (__popc(cc) == 2) {
        lp_two(P, shist, u, q, o, cc, cf, cx, hq);
        return false;
    }
    ++o.nodes;
    return true;
}

// The whole subtree below an entered-but-not-yet-pivoted node, depth first.
__device__ void lp_dfs(const BkParams &P, unsigned long long *shist, LpNode u, LpSums &o) {
    uint32_t stk[32 * 5];   // frames: cand, finc, xs, ext, q (a frame adds a distinct candidate: depth < 31)
    const int d0 = u.depth;
    uint32_t ext = 0u;
    bool enter = true;
    for (;;) {
        if (enter) {
            if (u.cand == 0u) {
                if ((u.finc | u.xs) == 0u) lp_emit(P, shist, o, u.base + (uint32_t)u.depth, u.hs);
                goto lpop;
            }
            ext = lp_pivot_ext(u, o);
            enter = false;
        }
        if (ext == 0u) goto lpop;
        {
            const int q = __ffs(ext) - 1;
            const uint32_t qb = 1u << q;
            ext &= ~qb;
            u.cand &= ~qb;
            u.finc |= qb;
            uint32_t cc, cf, cx;
            uint64_t hq;
            if (!lp_child(P, shist, u, q, o, cc, cf, cx, hq)) continue;
            uint32_t *f = stk + 5 * (u.depth - d0);
            f[0] = u.cand;
            f[1] = u.finc;
            f[2] = u.xs;
            f[3] = ext;
            f[4] = (uint32_t)q;
            ++u.depth;
            u.cand = cc;
            u.finc = cf;
            u.xs = cx;
            u.hs += hq;
            enter = true;
            continue;
        }
    lpop:
        if (u.depth == d0) break;
        --u.depth;
        {
            const uint32_t *f = stk + 5 * (u.depth - d0);
            u.cand = f[0];
            u.finc = f[1];
            u.xs = f[2];
            ext = f[3];
            u.hs -= u.hC[f[4]];
        }
    }
}

__device__ __forceinline__ LpNode lp_root_node(const uint32_t *lp, int r) {
    const uint32_t *rec = lp + 4 * r;
    const uint32_t meta = rec[1];
    LpNode u;
    u.cn = (int)(meta & 0xffu);
    const int xn = (int)((meta >> 8) & 0xffu);
    u.base = meta >> 16;
    const uint32_t *uni = lp + BK_LP_TABLE_WORDS + rec[0];
    u.hC = reinterpret_cast<const uint64_t *>(uni);
    u.akC = reinterpret_cast<const uint2 *>(uni + 2 * u.cn);
    u.akX = reinterpret_cast<const uint2 *>(uni + 4 * u.cn);
    u.adjXT = uni + 4 * u.cn + 2 * xn;
    u.cand = u.cn == 32 ? FULL : ((1u << u.cn) - 1u);
    u.xs = xn == 32 ? FULL : ((1u << xn) - 1u);
    u.finc = 0u;
    u.hs = (uint64_t)rec[2] | ((uint64_t)rec[3] << 32);
    u.depth = 0;
    return u;
}

__device__ __forceinline__ void lp_task_put(uint32_t *t, int r, const LpNode &u) {
    t[0] = (uint32_t)r | ((uint32_t)u.depth << 8);
    t[1] = u.cand;
    t[2] = u.finc;
    t[3] = u.xs;
    t[4] = (uint32_t)u.hs;
    t[5] = (uint32_t)(u.hs >> 32);
}

__device__ __forceinline__ LpNode lp_task_get(const uint32_t *lp, const uint32_t *t) {
    LpNode u = lp_root_node(lp, (int)(t[0] & 0xffu));
    u.depth = (int)(t[0] >> 8);
    u.cand = t[1];
    u.finc = t[2];
    u.xs = t[3];
    u.hs = (uint64_t)t[4] | ((uint64_t)t[5] << 32);
    return u;
}

// Enter node u and put its non-trivial children into the list `dst` (leaves
// and one-candidate children are settled at once); a child that finds the
// list full is searched here instead.
__device__ void lp_expand(const BkParams &P, unsigned long long *shist, LpNode u, int r, LpSums &o, uint32_t *dst,
                          uint32_t *dst_n, uint32_t cap) {
    if (u.cand == 0u) {
        if ((u.finc | u.xs) == 0u) lp_emit(P, shist, o, u.base + (uint32_t)u.depth, u.hs);
        return;
    }
    uint32_t ext = lp_pivot_ext(u, o);
    while (ext) {
        const int q = __ffs(ext) - 1;
        const uint32_t qb = 1u << q;
        ext &= ~qb;
        u.cand &= ~qb;
        u.finc |= qb;
        uint32_t cc, cf, cx;
        uint64_t hq;
        if (!lp_child(P, shist, u, q, o, cc, cf, cx, hq)) continue;
        LpNode c = u;
        c.cand = cc;
        c.finc = cf;
        c.xs = cx;
        c.hs = u.hs + hq;
        c.depth = u.depth + 1;
        const uint32_t slot = atomicAdd(dst_n, 1u);
        if (slot < cap) lp_task_put(dst + (int64_t)slot * BK_LP_TASK_WORDS, r, c);
        else lp_dfs(P, shist, c, o);
    }
}

// The buffered small subtrees, searched from one stack of nodes (entered,
// not yet pivoted) shared by the warp's lanes: each round the lanes take up
// to 32 nodes off the top together and push the children that are not
// settled at once; a child that finds the stack full is searched depth
// first by its lane.
__device__ __noinline__ LpSums lp_run(const BkParams &P, uint32_t *lp, int nroots, unsigned long long *shist,
                                      uint32_t *tasks, int lane) {
    LpSums o = {0ULL, 0ULL, 0u, 0u, 0u};
    uint32_t *ctr = lp + BK_LP_MAX_ROOTS * 4;   // [0] stack top
    const uint32_t cap = (uint32_t)P.lp_task_cap;
    for (int r = lane; r < nroots; r += 32) lp_task_put(tasks + (int64_t)r * BK_LP_TASK_WORDS, r, lp_root_node(lp, r));
    if (lane == 0) ctr[0] = (uint32_t)nroots;
    __syncwarp();
    for (;;) {
        const uint32_t top = min(ctr[0], cap);
        if (top == 0u) break;
        const uint32_t take = min(top, 32u), base = top - take;
        LpNode u;
        int r = -1;
        if ((uint32_t)lane < take) {
            const uint32_t *t = tasks + (int64_t)(base + (uint32_t)lane) * BK_LP_TASK_WORDS;
            r = (int)(t[0] & 0xffu);
            u = lp_task_get(lp, t);
        }
        __syncwarp();   // every taken record is read before pushes reuse its slot
        if (lane == 0) ctr[0] = base;
        __syncwarp();
        if (r >= 0) lp_expand(P, shist, u, r, o, tasks, &ctr[0], cap);
        __syncwarp();
    }
    return o;
}

// Run the buffered small subtrees and fold their sums into the task.
__device__ void lp_flush(const BkParams &P, Ws &s, Acc &acc, unsigned long long *shist, int lane, int &node_tick) {
    if (s.lp_n == 0) return;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const LpSums r = lp_run(P, s.lp, s.lp_n, shist, P.lp_tasks + gwarp * (int64_t)P.lp_task_cap * BK_LP_TASK_WORDS,
                            lane);
    unsigned long long cnt = r.count, nodes = r.nodes, hsh = r.hash, wops = r.wops;
    uint32_t smax = r.smax;
    for (int o = 16; o; o >>= 1) {
        cnt += __shfl_xor_sync(FULL, cnt, o);
        nodes += __shfl_xor_sync(FULL, nodes, o);
        hsh += __shfl_xor_sync(FULL, hsh, o);
        wops += __shfl_xor_sync(FULL, wops, o);
        smax = max(smax, __shfl_xor_sync(FULL, smax, o));
    }
    acc.t_count += cnt;
    acc.t_hash += hsh;
    acc.t_nodes += nodes;
    if (lane == 0) {
        acc.wops += wops;
        if (smax > cold().maxsize) cold().maxsize = smax;
    }
    node_tick += nodes > 4096ULL ? 4096 : (int)nodes;
    s.lp_n = 0;
    s.lp_top = 0;
}

// Relabel the small node (as search_small does) into the arena; the search
// of its subtree is left to the next lp_flush.
template <int NR>
__device__ void lp_enqueue(const BkParams &P, Ws &s, Acc &acc, unsigned long long *shist, int lane, int &node_tick,
                           int k0, int d, uint64_t hsum, const uint32_t (&rc)[NR], const uint32_t (&rf)[NR],
                           const int32_t *Fd, int flen) {
    SmallU u;
    int32_t gC, cidC, cidX;
    small_relabel<NR>(P, s, lane, rc, rf, Fd, flen, u, gC, cidC, cidX);
    const int need = lp_universe_words(u.cn, u.xn);
    if (s.lp_n == BK_LP_MAX_ROOTS || s.lp_top + need > P.lp_words - BK_LP_TABLE_WORDS)
        lp_flush(P, s, acc, shist, lane, node_tick);
    // column k of adjX to lane k
    uint32_t adjXT = 0u;
    for (int k = 0; k < u.cn; ++k) {
        const uint32_t b = __ballot_sync(FULL, (u.adjX >> k) & 1u);
        if (lane == k) adjXT = b;
    }
    uint32_t *uni = s.lp + BK_LP_TABLE_WORDS + s.lp_top;
    if (lane < u.cn) {
        reinterpret_cast<uint64_t *>(uni)[lane] = vertex_hash(gC, P.seed);
        reinterpret_cast<uint2 *>(uni + 2 * u.cn)[lane] = make_uint2(u.adjC, u.tC);
        uni[4 * u.cn + 2 * u.xn + lane] = adjXT;
    }
    if (lane < u.xn) reinterpret_cast<uint2 *>(uni + 4 * u.cn)[lane] = make_uint2(u.adjX, u.tX);
    if (lane == 0) {
        uint32_t *rec = s.lp + 4 * s.lp_n;
        rec[0] = (uint32_t)s.lp_top;
        rec[1] = (uint32_t)u.cn | ((uint32_t)u.xn << 8) | ((uint32_t)(k0 + d) << 16);
        rec[2] = (uint32_t)hsum;
        rec[3] = (uint32_t)(hsum >> 32);
    }
    s.lp_n++;
    s.lp_top += need;
    __syncwarp();
}

template <int NR>
__device__ __forceinline__ uint32_t bcast(const uint32_t (&r)[NR], int k) {
    return __shfl_sync(FULL, (NR == 1 || k < 32) ? r[0] : r[NR - 1], k & 31);
}

// conf is only live in incremental mode (always empty in static MCE)
template <int NR>
__device__ __forceinline__ void frame_store(const Ws &s, int d, int lane, const uint32_t (&rc)[NR],
                                            const uint32_t (&rf)[NR], const uint32_t (&re)[NR],
                                            const uint32_t (&rx)[NR], bool with_conf) {
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int k = lane + 32 * r;
        if (k < s.wc) {
            fr_cand(s, d)[k] = rc[r];
            fr_finic(s, d)[k] = rf[r];
            fr_ext(s, d)[k] = re[r];
            if (with_conf) fr_conf(s, d)[k] = rx[r];
        }
    }
}

template <int NR>
__device__ __forceinline__ void frame_load(const Ws &s, int d, int lane, uint32_t (&rc)[NR], uint32_t (&rf)[NR],
                                           uint32_t (&re)[NR], uint32_t (&rx)[NR], bool with_conf) {
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int k = lane + 32 * r;
        const bool in = k < s.wc;
        rc[r] = in ? fr_cand(s, d)[k] : 0u;
        rf[r] = in ? fr_finic(s, d)[k] : 0u;
        re[r] = in ? fr_ext(s, d)[k] : 0u;
        rx[r] = (in && with_conf) ? fr_conf(s, d)[k] : 0u;
    }
}

// The search proper (Algorithm 1 on an explicit stack).  The words of the
// current frame (cand, finic, ext, conf) stay in registers, one word per
// lane per register; candidate words reach other lanes by warp shuffles.
// Frames are written to memory only when a child is pushed, and read back
// when it is popped.  Returns 0 = done, 1 = stop the launch, 2 = dropped.
template <int NR>
__device__ int search(const BkParams &P, Ws &s, const Task &T, Acc &acc, unsigned long long *shist, int lane,
                      int &node_tick, uint64_t t_start, int32_t root, int k0, bool enter) {
    const int wc = s.wc;
    const bool imce = P.mode == BK_IMCE;
    uint32_t rc[NR], rf[NR], re[NR], rx[NR];
    int d = 0;
    frame_load<NR>(s, 0, lane, rc, rf, re, rx, imce);
    uint32_t flen = fr_meta(s, 0)[0];
    uint64_t hsum = meta_hsum(fr_meta(s, 0));
    for (;;) {
        if (enter) {
            acc.t_nodes++;
            if (P.mode == BK_IMCE) {
                // Algorithm 7: a candidate joined to K by an earlier new edge cannot extend K
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const uint32_t x = rc[r] & rx[r];
                    rf[r] |= x;
                    rc[r] &= ~x;
                }
            }
            bool anyc = false, anyf = false;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                anyc |= rc[r] != 0u;
                anyf |= rf[r] != 0u;
            }
            if (!__any_sync(FULL, anyc)) {
                if (!__any_sync(FULL, anyf) && flen == 0u) emit(P, s, root, k0, d, hsum, acc, shist, lane);
                goto pop;
            }
            // ---- at most 32 candidates and 32 fini vertices: the whole subtree in registers
            int node_cn, node_fn;
            {
                int cn = 0, fcn = 0;
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    cn += __popc(rc[r]);
                    fcn += __popc(rf[r]);
                }
                cn = __reduce_add_sync(FULL, cn);
                fcn = __reduce_add_sync(FULL, fcn);
                node_cn = cn;
                node_fn = fcn + (int)flen;
                if (cn <= 32 && fcn + (int)flen <= 32) {
                    const int32_t *Fd = (T.kdepth == 0 && d == 0) ? s.F0 : s.F;
                    if (P.lp_words && P.mode == BK_MCE && !P.list_off && !acc.lp_hold) {
                        lp_enqueue<NR>(P, s, acc, shist, lane, node_tick, k0, d, hsum, rc, rf, Fd, (int)flen);
                        goto pop;
                    }
                    const int code = search_small<NR>(P, s, T, acc, shist, lane, node_tick, t_start, root, k0, d,
                                                      hsum, rc, rf, rx, Fd, (int)flen);
                    if (code) return code;
                    goto pop;
                }
            }
            // ---- pivot: argmax over cand ∪ finic ∪ F of |cand ∩ A[u]|, ties to the smallest id
            {
                uint32_t best_cnt = 0;
                int32_t best_gid = 0x7fffffff, best_loc = -1;
                // cand to this warp's shared scratch, read back as 16-byte vectors
                // beside the 16-byte aligned rows (words wc..S-1 are zero)
                uint32_t *scand = s.piv;
                uint16_t *ul = reinterpret_cast<uint16_t *>(s.piv + 64);
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const int k = lane + 32 * r;
                    if (k < s.S) scand[k] = k < wc ? rc[r] : 0u;
                }
                const int S4 = s.S >> 2;
                const uint4 *cv = reinterpret_cast<const uint4 *>(scand);
                __syncwarp();
                // members of cand ∪ finic in increasing local id, listed 16 words
                // (512 vertices) at a time and counted one member per lane
                for (int ch = 0; ch < ((wc + 15) >> 4); ++ch) {
                    const int wi = (ch << 4) + (lane & 15);
                    const uint32_t src = (NR == 1 || ch < 2) ? (rc[0] | rf[0]) : (rc[NR - 1] | rf[NR - 1]);
                    uint32_t word = __shfl_sync(FULL, src, wi & 31);
                    if (lane >= 16 || wi >= wc) word = 0u;
                    const int pc = __popc(word);
                    int incl = pc;
#pragma unroll
                    for (int o = 1; o < 16; o <<= 1) {
                        const int y = __shfl_up_sync(FULL, incl, o);
                        if (lane >= o) incl += y;
                    }
                    const int tot = __shfl_sync(FULL, incl, 15);
                    if (tot == 0) continue;
                    int pos = incl - pc;
                    while (word) {
                        ul[pos++] = (uint16_t)((wi << 5) + __ffs(word) - 1);
                        word &= word - 1;
                    }
                    __syncwarp();
                    for (int i = lane; i < tot; i += 32) {
                        const int u = ul[i];
                        const uint4 *row = reinterpret_cast<const uint4 *>(s.A + (int64_t)u * s.S);
                        uint32_t cnt = 0;
                        for (int g = 0; g < S4; ++g) {
                            const uint4 x = row[g], y = cv[g];
                            cnt += __popc(x.x & y.x) + __popc(x.y & y.y) + __popc(x.z & y.z) + __popc(x.w & y.w);
                        }
                        // local ids below c follow the global ids, and a lane meets its
                        // members in increasing local id: a tie never replaces the best
                        if (best_loc < 0 || cnt > best_cnt) {
                            best_cnt = cnt;
                            best_loc = u;
                        }
                    }
                    __syncwarp();
                }
                if (best_loc >= 0) best_gid = s.gid[best_loc];
                // F is ordered by bnd = popc(A[u]) >= |cand ∩ A[u]|; once the bound
                // of the next entries drops below the best count none of them can
                // win (a tie needs count == best), so the scan stops there.
                if (flen) {
                    const int32_t *Fd = (T.kdepth == 0 && d == 0) ? s.F0 : s.F;
                    uint32_t thr = __reduce_max_sync(FULL, best_loc >= 0 ? best_cnt + 1u : 0u);
                    for (int b0 = 0; b0 < (int)flen; b0 += 32) {
                        const int i = b0 + lane;
                        int u = 0;
                        bool take = false;
                        if (i < (int)flen) {
                            u = Fd[i];
                            take = (uint32_t)s.bnd[u] + 1u >= thr;
                        }
                        if (__any_sync(FULL, take)) {
                            uint32_t cnt = 0;
                            if (take) {
                                const uint4 *row = reinterpret_cast<const uint4 *>(s.A + (int64_t)u * s.S);
                                for (int g = 0; g < S4; ++g) {
                                    const uint4 x = row[g], y = cv[g];
                                    cnt += __popc(x.x & y.x) + __popc(x.y & y.y) + __popc(x.z & y.z) +
                                           __popc(x.w & y.w);
                                }
                            }
                            if (take) {
                                const int32_t g = s.gid[u];
                                if (best_loc < 0 || cnt > best_cnt || (cnt == best_cnt && g < best_gid)) {
                                    best_cnt = cnt;
                                    best_gid = g;
                                    best_loc = u;
                                }
                            }
                        }
                        thr = __reduce_max_sync(FULL, best_loc >= 0 ? best_cnt + 1u : 0u);
                        if (b0 + 32 < (int)flen && (uint32_t)s.bnd[Fd[b0 + 32]] + 1u < thr) break;
                    }
                }
                // warp argmax (lanes without a candidate hold best_loc = -1)
                const uint32_t key_cnt = best_loc >= 0 ? best_cnt + 1u : 0u;
                const uint32_t mx = __reduce_max_sync(FULL, key_cnt);
                const uint32_t gkey = (key_cnt == mx) ? (uint32_t)best_gid : 0xffffffffu;
                const uint32_t mg = __reduce_min_sync(FULL, gkey);
                const uint32_t who = __ballot_sync(FULL, key_cnt == mx && (uint32_t)best_gid == mg);
                const int p = __shfl_sync(FULL, best_loc, __ffs(who) - 1);
                const uint32_t *prow = s.A + (int64_t)p * s.S;
                int ne = 0;
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const int k = lane + 32 * r;
                    re[r] = k < wc ? (rc[r] & ~prow[k]) : 0u;
                    ne += __popc(re[r]);
                }
                count_node_wops(acc, lane, node_cn, node_fn, __reduce_add_sync(FULL, ne));
            }
            enter = false;
            if (++node_tick >= acc.tick) {
                node_tick = 0;
                frame_store<NR>(s, d, lane, rc, rf, re, rx, imce);
                __syncwarp();
                const int act = periodic(P, s, T, acc, lane, d, root, t_start);
                if (act) return act;
#pragma unroll
                for (int r = 0; r < NR; ++r) {   // a hand-over may have shrunk this frame's ext
                    const int k = lane + 32 * r;
                    re[r] = k < wc ? fr_ext(s, d)[k] : 0u;
                }
            }
        }
        // ---- next child of frame d
        {
            int q = -1;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                if (q >= 0) break;
                const uint32_t b = __ballot_sync(FULL, re[r] != 0u);
                if (b) {
                    const int src = __ffs(b) - 1;
                    const uint32_t xs = __shfl_sync(FULL, re[r], src);
                    q = ((src + 32 * r) << 5) + (__ffs(xs) - 1);
                }
            }
            if (q < 0) goto pop;
            const int32_t gq = s.gid[q];   // its latency overlaps the child build
            const int qw = q >> 5;
            const uint32_t qb = 1u << (q & 31);
            const uint32_t *qrow = s.A + (int64_t)q * s.S;
            uint32_t nc[NR], nf[NR], nx[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int k = lane + 32 * r;
                const uint32_t a = k < wc ? qrow[k] : 0u;
                nc[r] = rc[r] & a;
                nf[r] = rf[r] & a;
                nx[r] = rx[r];
                if (P.mode == BK_IMCE && k < wc) nx[r] |= s.X[(int64_t)q * s.S + k];
                if (k == qw) {
                    re[r] &= ~qb;
                    rc[r] &= ~qb;
                    rf[r] |= qb;
                }
            }
            int nfl = 0;
            if (flen) {
                if (T.kdepth == 0 && d == 0) {
                    nfl = compact_cb(s, q, lane);   // F0 stays untouched at the root
                } else {
                    nfl = partition_F(s, (int)flen, lane, [&](int32_t x) {
                        return (s.A[(int64_t)x * s.S + qw] & qb) != 0u;
                    });
                }
            }
            if (d + 2 > s.dcap) {   // deeper than the frame stack: stop with an error
                if (lane == 0) atomicOr(&P.ctl[CTL_ABORT], 4ULL);
                return 1;
            }
            // parent frame to memory (its meta is unchanged), child meta
            frame_store<NR>(s, d, lane, rc, rf, re, rx, imce);
            const uint64_t nh = hsum + vertex_hash(gq, P.seed);
            if (lane == 0) {
                uint32_t *nm = fr_meta(s, d + 1);
                nm[0] = (uint32_t)nfl;
                nm[1] = (uint32_t)q;
                meta_set_hsum(nm, nh);
            }
            __syncwarp();
            ++d;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                rc[r] = nc[r];
                rf[r] = nf[r];
                rx[r] = nx[r];
                re[r] = 0u;
            }
            flen = (uint32_t)nfl;
            hsum = nh;
            enter = true;
            continue;
        }
    pop:
        if (d == 0) {
            lp_flush(P, s, acc, shist, lane, node_tick);
            return 0;
        }
        if (P.mode == BK_MCE && !(T.kdepth == 0 && d == 1)) {
            // put frame d-1's F back in bnd order (the child split it into adjacent | rest);
            // the root frame reads F0, which no child touches
            const int a = (int)flen, len = (int)fr_meta(s, d - 1)[0];
            if (a > 0 && a < len) merge_F(s, a, len, lane);
        }
        --d;
        frame_load<NR>(s, d, lane, rc, rf, re, rx, imce);
        flen = fr_meta(s, d)[0];
        hsum = meta_hsum(fr_meta(s, d));
        enter = false;
    }
}

// The same search for candidate sets wider than 32 words (more than 1024
// candidates, which some ranks produce for hubs): frames stay in memory and
// every set operation loops over its words.  Returns as search<NR>.
__device__ int search_mem(const BkParams &P, Ws &s, const Task &T, Acc &acc, unsigned long long *shist, int lane,
                          int &node_tick, uint64_t t_start, int32_t root, int k0, bool enter) {
    const int wc = s.wc;
    int d = 0;
    for (;;) {
        uint32_t *cand = fr_cand(s, d), *finic = fr_finic(s, d), *ext = fr_ext(s, d);
        uint32_t *meta = fr_meta(s, d);
        if (enter) {
            acc.t_nodes++;
            if (P.mode == BK_IMCE) {
                const uint32_t *conf = fr_conf(s, d);
                for (int k = lane; k < wc; k += 32) {
                    const uint32_t x = cand[k] & conf[k];
                    finic[k] |= x;
                    cand[k] &= ~x;
                }
                __syncwarp();
            }
            if (!warp_any(cand, wc, lane)) {
                const bool fin = warp_any(finic, wc, lane) || meta[0] != 0u;
                if (!fin) emit(P, s, root, k0, d, meta_hsum(meta), acc, shist, lane);
                goto pop;
            }
            {
                uint32_t best_cnt = 0;
                int32_t best_gid = 0x7fffffff, best_loc = -1;
                for (int k = 0; k < wc; ++k) {
                    const uint32_t mword = cand[k] | finic[k];
                    if ((mword >> lane) & 1u) {
                        const int u = (k << 5) + lane;
                        const uint32_t *row = s.A + (int64_t)u * s.S;
                        uint32_t cnt = 0;
                        for (int t = 0; t < wc; ++t) cnt += __popc(cand[t] & row[t]);
                        const int32_t g = s.gid[u];
                        if (best_loc < 0 || cnt > best_cnt || (cnt == best_cnt && g < best_gid)) {
                            best_cnt = cnt;
                            best_gid = g;
                            best_loc = u;
                        }
                    }
                }
                const int flen = (int)meta[0];
                if (flen) {
                    const int32_t *Fd = (T.kdepth == 0 && d == 0) ? s.F0 : s.F;
                    uint32_t thr = __reduce_max_sync(FULL, best_loc >= 0 ? best_cnt + 1u : 0u);
                    for (int b0 = 0; b0 < flen; b0 += 32) {
                        const int i = b0 + lane;
                        if (i < flen) {
                            const int u = Fd[i];
                            if ((uint32_t)s.bnd[u] + 1u >= thr) {
                                const uint32_t *row = s.A + (int64_t)u * s.S;
                                uint32_t cnt = 0;
                                for (int t = 0; t < wc; ++t) cnt += __popc(cand[t] & row[t]);
                                const int32_t g = s.gid[u];
                                if (best_loc < 0 || cnt > best_cnt || (cnt == best_cnt && g < best_gid)) {
                                    best_cnt = cnt;
                                    best_gid = g;
                                    best_loc = u;
                                }
                            }
                        }
                        thr = __reduce_max_sync(FULL, best_loc >= 0 ? best_cnt + 1u : 0u);
                        if (b0 + 32 < flen && (uint32_t)s.bnd[Fd[b0 + 32]] + 1u < thr) break;
                    }
                }
                const uint32_t key_cnt = best_loc >= 0 ? best_cnt + 1u : 0u;
                const uint32_t mx = __reduce_max_sync(FULL, key_cnt);
                const uint32_t gkey = (key_cnt == mx) ? (uint32_t)best_gid : 0xffffffffu;
                const uint32_t mg = __reduce_min_sync(FULL, gkey);
                const uint32_t who = __ballot_sync(FULL, key_cnt == mx && (uint32_t)best_gid == mg);
                const int p = __shfl_sync(FULL, best_loc, __ffs(who) - 1);
                const uint32_t *prow = s.A + (int64_t)p * s.S;
                for (int k = lane; k < wc; k += 32) ext[k] = cand[k] & ~prow[k];
                __syncwarp();
                count_node_wops(acc, lane, warp_popc(cand, wc, lane), warp_popc(finic, wc, lane) + flen,
                                warp_popc(ext, wc, lane));
            }
            enter = false;
            if (++node_tick >= acc.tick) {
                node_tick = 0;
                const int act = periodic(P, s, T, acc, lane, d, root, t_start);
                if (act) return act;
            }
        }
        {
            const int q = warp_first_bit(ext, wc, lane);
            if (q < 0) goto pop;
            const int qw = q >> 5;
            const uint32_t qb = 1u << (q & 31);
            if (d + 2 > s.dcap) {
                if (lane == 0) atomicOr(&P.ctl[CTL_ABORT], 4ULL);
                return 1;
            }
            const uint32_t *qrow = s.A + (int64_t)q * s.S;
            uint32_t *ncand = fr_cand(s, d + 1), *nfinic = fr_finic(s, d + 1);
            for (int k = lane; k < wc; k += 32) {
                ncand[k] = cand[k] & qrow[k];
                nfinic[k] = finic[k] & qrow[k];
                fr_ext(s, d + 1)[k] = 0u;
                fr_conf(s, d + 1)[k] = fr_conf(s, d)[k] | (P.mode == BK_IMCE ? s.X[(int64_t)q * s.S + k] : 0u);
            }
            int nfl = 0;
            const int flen = (int)meta[0];
            if (flen) {
                if (T.kdepth == 0 && d == 0) {
                    nfl = compact_cb(s, q, lane);
                } else {
                    nfl = partition_F(s, flen, lane, [&](int32_t x) {
                        return (s.A[(int64_t)x * s.S + qw] & qb) != 0u;
                    });
                }
            }
            __syncwarp();
            if (lane == 0) {
                ext[qw] &= ~qb;
                cand[qw] &= ~qb;
                finic[qw] |= qb;
                uint32_t *nm = fr_meta(s, d + 1);
                nm[0] = (uint32_t)nfl;
                nm[1] = (uint32_t)q;
                meta_set_hsum(nm, meta_hsum(meta) + vertex_hash(s.gid[q], P.seed));
            }
            __syncwarp();
            ++d;
            enter = true;
            continue;
        }
    pop:
        if (d == 0) return 0;
        if (P.mode == BK_MCE && !(T.kdepth == 0 && d == 1)) {
            const int a = (int)fr_meta(s, d)[0], len = (int)fr_meta(s, d - 1)[0];
            if (a > 0 && a < len) merge_F(s, a, len, lane);
        }
        --d;
        enter = false;
    }
}

// Run one task to completion.  Returns false when the launch must stop.
__device__ bool run_task(const BkParams &P, Ws &s, const Task &T, Acc &acc, unsigned long long *shist,
                         uint32_t *ws_smem, uint32_t *ws_glob, const uint32_t *taskbuf, int lane,
                         int32_t &built, int &node_tick, uint64_t t_start) {
    const int32_t root = T.root;
    s.lp_n = s.lp_top = 0;   // nothing buffered survives a dropped task
    // ---- build (or reuse) the subproblem
    int32_t w, c;
    if (P.mode == BK_MCE) {
        w = P.row_ptr[root + 1] - P.row_ptr[root];
        c = P.up_ptr[root + 1] - P.up_ptr[root];
    } else {
        const int32_t du = P.row_ptr[P.eu[root] + 1] - P.row_ptr[P.eu[root]];
        const int32_t dv = P.row_ptr[P.ev[root] + 1] - P.row_ptr[P.ev[root]];
        c = du < dv ? du : dv;
        w = c;
    }
    const int64_t need = bk_ws_words(w, c, P.mode);
    uint32_t *base = (need <= P.smem_words) ? ws_smem : ws_glob;
    if (bk_private_words(w, c, P.mode) > P.gws_words && base == ws_glob) {
        if (lane == 0) atomicOr(&P.ctl[CTL_ABORT], 4ULL);
        return false;
    }
    const int k0 = (P.mode == BK_MCE ? 1 : 2) + T.kdepth;
    const uint64_t tb = globaltimer_ns();
    bool ready = false;
    if (P.mode == BK_MCE && P.cache) {
        const int64_t sw = bk_shared_words(w, c);
        long long off = -1;
        if (lane == 0) {
            if (T.rec < 0) {
                const unsigned long long o = atomicAdd(&P.ctl[CTL_CACHE_TOP], (unsigned long long)sw);
                off = ((int64_t)o + sw <= P.cache_words) ? (long long)o : -1;
            } else {
                off = __ldcg(P.cache_off + root);
            }
        }
        off = __shfl_sync(FULL, off, 0);
        if (off >= 0) {
            uint32_t *sh = P.cache + off;
            ws_layout_split(s, sh, base, w, c);
            if (T.rec < 0) {
                // open the subproblem: build it into the cache and publish it
                build_mce(P, s, root, lane);
                if (lane == 0) {
                    sh[0] = (uint32_t)s.W;
                    sh[1] = (uint32_t)s.f;
                }
                __threadfence();
                __syncwarp();
                if (lane == 0) atomicExch(reinterpret_cast<unsigned long long *>(P.cache_off + root),
                                          (unsigned long long)off);
                if (lane == 0) {
                    cold().builds++;
                    cold().build_ns += globaltimer_ns() - tb;
                }
            } else {
                s.W = (int32_t)__ldcg(sh);
                s.f = (int32_t)__ldcg(sh + 1);
            }
            built = -1;   // the private region no longer holds a private build
            ready = true;
        }
    }
    if (!ready) {
        if (need > P.gws_words && base == ws_glob) {   // no cache room and no room for a private build
            if (lane == 0) atomicOr(&P.ctl[CTL_ABORT], 4ULL);
            return false;
        }
        if (P.mode == BK_MCE) ws_layout_split(s, base, base + bk_shared_words(w, c), w, c);
        else ws_layout(s, base, w, c, P.mode);
        if (built != root || P.mode == BK_IMCE) {   // same pointers as the last build of `root`: f and W kept
            if (P.mode == BK_MCE) {
                build_mce(P, s, root, lane);
            } else {
                build_imce(P, s, root, lane);
            }
            built = root;
            if (lane == 0) {
                cold().builds++;
                cold().build_ns += globaltimer_ns() - tb;
            }
        }
    }
    // ---- frame 0
    uint64_t hs0 = P.mode == BK_MCE ? vertex_hash(root, P.seed)
                                    : vertex_hash(P.eu[root], P.seed) + vertex_hash(P.ev[root], P.seed);
    bool enter;
    uint32_t *m0 = fr_meta(s, 0);
    if (T.rec < 0) {
        uint32_t *cand = fr_cand(s, 0), *finic = fr_finic(s, 0);
        for (int k = lane; k < s.wc; k += 32) {
            const int lo = k << 5;
            const int nb = s.c - lo;
            cand[k] = nb >= 32 ? FULL : ((1u << nb) - 1u);
            finic[k] = 0u;
            if (P.mode == BK_MCE) fr_conf(s, 0)[k] = 0u;
        }
        if (lane == 0) {
            m0[0] = (uint32_t)s.f;   // the root frame reads F0 itself
            m0[1] = 0xffffffffu;
        }
        enter = true;
    } else {
        // handed-over frame (copied to this warp's task buffer): path, cand, finic, ext, conf
        const uint32_t *r = taskbuf;
        const int kd = T.kdepth;
        for (int j = lane; j < kd; j += 32) s.kpath[j] = (int32_t)r[2 + j];
        const uint32_t *rb = r + 2 + kd;
        for (int k = lane; k < s.wc; k += 32) {
            fr_cand(s, 0)[k] = rb[k];
            fr_finic(s, 0)[k] = rb[s.wc + k];
            fr_ext(s, 0)[k] = rb[2 * s.wc + k];
            fr_conf(s, 0)[k] = rb[3 * s.wc + k];
        }
        __syncwarp();
        for (int j = 0; j < kd; ++j) hs0 += vertex_hash(s.gid[s.kpath[j]], P.seed);
        int flen = 0;
        if (P.mode == BK_MCE) {
            // F at this frame: the kept lower-ranked vertices adjacent to the whole path,
            // in F0 order (the partition is stable).  A root piece reads F0 itself.
            if (kd == 0) {
                flen = s.f;
            } else {
                flen = compact_cb(s, s.kpath[0], lane);
            }
            for (int j = 1; j < kd; ++j) {
                const int q = s.kpath[j];
                flen = partition_F(s, flen, lane, [&](int32_t x) {
                    return (s.A[(int64_t)x * s.S + (q >> 5)] >> (q & 31)) & 1u;
                });
            }
        }
        if (lane == 0) {
            m0[0] = (uint32_t)flen;
            m0[1] = 0xffffffffu;
        }
        enter = false;
    }
    meta_set_hsum(m0, hs0);
    __syncwarp();

    __syncwarp();
    // candidate sets of up to 1024 columns keep the frame in registers; wider
    // ones (hubs under some ranks) run with frames in memory.  A second
    // register width was measured slower overall on GB300: the larger kernel
    // costs instruction-fetch stalls on every node.
    const int code = s.wc <= 32 ? search<1>(P, s, T, acc, shist, lane, node_tick, t_start, root, k0, enter)
                                : search_mem(P, s, T, acc, shist, lane, node_tick, t_start, root, k0, enter);
    return code != 1;
}

__global__ void k_init_seq(unsigned long long *seq, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        seq[i] = (unsigned long long)i;
}

template <int MINB>
__global__ void __launch_bounds__(256, MINB) k_bk(BkParams P) {
    if (P.sm_limit > 0) {
        // scaling measurements: the whole grid is resident and only the blocks
        // placed on the first sm_limit SMs take work (a smaller grid would be
        // spread over all SMs, one block each)
        uint32_t smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        if ((int32_t)smid >= P.sm_limit) return;
    }
    extern __shared__ __align__(16) uint32_t smem[];
    unsigned long long *shist = reinterpret_cast<unsigned long long *>(smem);   // 256 bins
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nw_block = blockDim.x >> 5;
    for (int i = threadIdx.x; i < 256; i += blockDim.x) shist[i] = 0ULL;
    __syncthreads();
    uint32_t *ws_smem = smem + 512 + (int64_t)nw_block * BK_PIV_WORDS + (int64_t)wib * P.smem_words;
    uint32_t *lp_smem = smem + 512 + (int64_t)nw_block * (BK_PIV_WORDS + P.smem_words) + (int64_t)wib * P.lp_words;
    const int64_t gwarp = (int64_t)blockIdx.x * nw_block + wib;
    uint32_t *ws_glob = P.gws + gwarp * P.gws_words;
    uint32_t *taskbuf = P.taskbuf + gwarp * P.slot_words;
    Acc acc = {0, 0, 0, 0, 64, 4, 0};
    if (lane == 0) cold() = AccCold{0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    Ws s;
    s.piv = smem + 512 + (int64_t)wib * BK_PIV_WORDS;
    s.lp = lp_smem;
    s.lp_n = s.lp_top = 0;
    int32_t built = -1;
    int node_tick = 0;
    bool hungry = false;
    uint64_t idle_since = 0;
    unsigned backoff = 500;   // ns between tries while waiting (doubles to 16 us)
    const uint64_t t_start = globaltimer_ns();
    for (;;) {
        // ---- acquire work: queued pieces first, then the next subproblem
        Task T;
        T.root = -1;
        T.kdepth = 0;
        T.rec = -1;
        int kind = 0;   // 0 none, 1 subproblem, 2 piece, 3 stop
        int64_t qpos = -1;
        if (lane == 0) {
            if (*(volatile unsigned long long *)&P.ctl[CTL_ABORT] & 3ULL) {
                kind = 3;
            } else {
                qpos = queue_claim_pop(P);
                if (qpos >= 0) {
                    kind = 2;
                } else if (*(volatile unsigned long long *)&P.ctl[CTL_NEXT] < (unsigned long long)P.n_sub) {
                    const unsigned long long i = atomicAdd(&P.ctl[CTL_NEXT], 1ULL);
                    if (i < (unsigned long long)P.n_sub) {
                        kind = 1;
                        T.root = P.order[i];
                        if (i + 1 == (unsigned long long)P.n_sub) P.ctl[CTL_T_LAST] = globaltimer_ns();
                    }
                }
                if (kind == 0 && *(volatile unsigned long long *)&P.ctl[CTL_PENDING] == 0ULL) kind = 3;
            }
        }
        kind = __shfl_sync(FULL, kind, 0);
        if (kind == 3) break;
        if (kind == 2) {
            // copy the record out of the ring and free its slot at once; its
            // length follows from the depth and the root's candidate count
            qpos = __shfl_sync(FULL, qpos, 0);
            const uint32_t *src = P.arena + (int64_t)((unsigned long long)qpos % (unsigned long long)P.qcap) *
                                                P.slot_words;
            const int32_t r0 = (int32_t)__ldcg(src), kd0 = (int32_t)__ldcg(src + 1);
            int32_t cr;
            if (P.mode == BK_MCE) {
                cr = P.up_ptr[r0 + 1] - P.up_ptr[r0];
            } else {
                const int32_t du = P.row_ptr[P.eu[r0] + 1] - P.row_ptr[P.eu[r0]];
                const int32_t dv = P.row_ptr[P.ev[r0] + 1] - P.row_ptr[P.ev[r0]];
                cr = du < dv ? du : dv;
            }
            int64_t words = 2 + (int64_t)kd0 + 4 * (int64_t)((cr + 31) >> 5);
            if (words > P.slot_words) words = P.slot_words;
            for (int64_t k = lane; k < words; k += 32) taskbuf[k] = __ldcg(src + k);
            __syncwarp();
            if (lane == 0) {
                T.root = (int32_t)taskbuf[0];
                T.kdepth = (int32_t)taskbuf[1];
                T.rec = 1;
                queue_release(P, qpos);
            }
        }
        if (kind == 0) {
            // Waiting is legitimate while other warps still work; only the
            // launch-wide time bound ends it.
            const uint64_t now = globaltimer_ns();
            if (!hungry) {
                hungry = true;
                idle_since = now;
                if (lane == 0) atomicAdd(&P.ctl[CTL_HUNGRY], 1ULL);
            } else if (now - t_start > P.max_run_ns + P.timeout_ns) {
                if (lane == 0) atomicOr(&P.ctl[CTL_ABORT], 2ULL);
                if (lane == 0) cold().idle_ns += now - idle_since;
                hungry = false;
                if (lane == 0) atomicAdd(&P.ctl[CTL_HUNGRY], ~0ULL);
                break;
            }
            __nanosleep(backoff);
            if (backoff < 16000u) backoff <<= 1;
            continue;
        }
        backoff = 500;
        if (hungry) {
            hungry = false;
            if (lane == 0) {
                cold().idle_ns += globaltimer_ns() - idle_since;
                atomicAdd(&P.ctl[CTL_HUNGRY], ~0ULL);
            }
        }
        if (kind == 2 && lane == 0) cold().pieces++;
        T.root = __shfl_sync(FULL, T.root, 0);
        T.kdepth = __shfl_sync(FULL, T.kdepth, 0);
        T.rec = __shfl_sync(FULL, T.rec, 0);
        acc.t_count = acc.t_hash = acc.t_nodes = 0;
        if (lane == 0) cold().t_rep = cold().t_split = 0;
        const uint64_t t0 = globaltimer_ns();
        const bool go_on = run_task(P, s, T, acc, shist, ws_smem, ws_glob, taskbuf, lane, built, node_tick, t_start);
        if (lane == 0) cold().max_busy += globaltimer_ns() - t0;
        if (lane == 0) {
            AccCold &c = cold();
            c.count += acc.t_count;
            c.hash += acc.t_hash;
            c.nodes += acc.t_nodes;
            if (P.sub_nodes && acc.t_nodes > c.t_rep) atomicAdd(&P.sub_nodes[T.root], acc.t_nodes - c.t_rep);
            if (P.graph_nodes && acc.t_nodes > c.t_rep)
                atomicAdd(&P.graph_nodes[P.graph_of[P.mode == BK_MCE ? T.root : P.eu[T.root]]], acc.t_nodes - c.t_rep);
            if (P.pv_count && P.mode == BK_MCE) {
                atomicAdd(&P.pv_count[T.root], acc.t_count);
                atomicAdd(&P.pv_hash[T.root], acc.t_hash);
                atomicAdd(&P.pv_nodes[T.root], acc.t_nodes);
            }
            if (P.g_count) {
                const int32_t gg = P.graph_of[P.mode == BK_MCE ? T.root : P.eu[T.root]];
                atomicAdd(&P.g_count[gg], acc.t_count);
                atomicAdd(&P.g_hash[gg], acc.t_hash);
            }
            __threadfence();
            atomicAdd(&P.ctl[CTL_PENDING], ~0ULL);
        }
        if (!go_on) break;
    }
    if (hungry) {
        if (lane == 0) {
            cold().idle_ns += globaltimer_ns() - idle_since;
            atomicAdd(&P.ctl[CTL_HUNGRY], ~0ULL);
        }
    }
    if (lane == 0) {
        atomicMax(&P.ctl[CTL_T_END], (unsigned long long)globaltimer_ns());
        const AccCold &c = cold();
        atomicAdd(&P.out[OUT_BUILD_NS], c.build_ns);
        atomicAdd(&P.out[OUT_SEARCH_NS], c.max_busy - c.build_ns);
        atomicAdd(&P.out[OUT_IDLE_NS], c.idle_ns);
        atomicAdd(&P.out[OUT_BUILDS], c.builds);
        atomicAdd(&P.out[OUT_PIECES], c.pieces);
        atomicMax(&P.out[OUT_MAXBUSY_NS], c.max_busy);
        atomicAdd(&P.out[OUT_NWARPS], 1ULL);
    }
    {
        unsigned long long w = acc.wops;
        for (int o = 16; o; o >>= 1) w += __shfl_xor_sync(FULL, w, o);
        if (lane == 0) atomicAdd(&P.out[OUT_WORDOPS], w);
    }
    if (lane == 0) {
        if (cold().maxsize) atomicMax(&P.out[OUT_MAXSIZE], cold().maxsize);
        atomicAdd(&P.out[OUT_COUNT], cold().count);
        atomicAdd(&P.out[OUT_HASH], cold().hash);
        atomicAdd(&P.out[OUT_NODES], cold().nodes);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        if (shist[i]) atomicAdd(&P.out[OUT_HIST + i], shist[i]);
}

}  // namespace

mce_status init_queue_seq(unsigned long long *seq, int64_t n, cudaStream_t s) {
    MCE_LAUNCH(k_init_seq, grid_for(n, 256), 256, 0, s, seq, n);
    return MCE_OK;
}

mce_status bk_prepare(int32_t blocks_per_sm, int64_t smem_bytes) {
    // dynamic shared memory above the 48 KB default must be opted into once
    // per kernel, outside any stream capture
    static std::atomic<int> granted[3] = {48 * 1024, 48 * 1024, 48 * 1024};
    const int smem = (int)smem_bytes;
    const int t = blocks_per_sm >= 4 ? 2 : (blocks_per_sm == 3 ? 1 : 0);
    if (smem <= granted[t].load()) return MCE_OK;
    if (t == 2) MCE_CUDA(cudaFuncSetAttribute(k_bk<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    else if (t == 1) MCE_CUDA(cudaFuncSetAttribute(k_bk<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    else MCE_CUDA(cudaFuncSetAttribute(k_bk<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int cur = granted[t].load();
    while (smem > cur && !granted[t].compare_exchange_weak(cur, smem)) {
    }
    return MCE_OK;
}

namespace {
int resident_blocks(int32_t blocks_per_sm, int32_t threads, size_t smem) {
    int active = 0;
    if (blocks_per_sm >= 4) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&active, k_bk<4>, threads, smem);
    else if (blocks_per_sm == 3) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&active, k_bk<3>, threads, smem);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&active, k_bk<2>, threads, smem);
    return active;
}
}  // namespace

mce_status launch_bk(const BkParams &p0, int32_t warps_per_block, int32_t blocks_per_sm, cudaStream_t s) {
    // a persistent grid must be resident at once: shrink the lane-parallel
    // regions until blocks_per_sm blocks fit on an SM
    BkParams p = p0;
    size_t smem = (size_t)bk_block_smem_bytes(warps_per_block, p.smem_words, p.lp_words);
    MCE_TRY(bk_prepare(blocks_per_sm, (int64_t)smem));   // the grant covers every smaller size below
    while (p.lp_words > 0 && resident_blocks(blocks_per_sm, warps_per_block * 32, smem) < blocks_per_sm) {
        p.lp_words = p.lp_words - 128 >= 512 ? p.lp_words - 128 : 0;
        smem = (size_t)bk_block_smem_bytes(warps_per_block, p.smem_words, p.lp_words);
    }
    const unsigned blocks = (unsigned)(num_sms() * blocks_per_sm);
    // 4 resident blocks of 256 threads leave 64 registers a thread; fewer
    // blocks let the compiler keep the search state in more registers
    if (blocks_per_sm >= 4) MCE_LAUNCH(k_bk<4>, blocks, warps_per_block * 32, smem, s, p);
    else if (blocks_per_sm == 3) MCE_LAUNCH(k_bk<3>, blocks, warps_per_block * 32, smem, s, p);
    else MCE_LAUNCH(k_bk<2>, blocks, warps_per_block * 32, smem, s, p);
    return MCE_OK;
}

}  // namespace mce
