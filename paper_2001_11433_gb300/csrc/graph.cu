#include <string>
// Graph ingest and vertex ranking kernels.
//
//   build_csr       simple undirected graph from raw pairs (Section 3; inputs
//                   normalised as in Section 6.1): drop self loops, symmetrise,
//                   radix sort, deduplicate, row offsets by scan.
//   vertex_key      Section 4.2 keys: degree, core number ("degeneracy" of a
//                   vertex: in the k-core but not the (k+1)-core) by parallel
//                   peeling, triangle count by oriented intersection.
//   rank_from_key   rank(v) = position of (key(v), id(v)) in ascending order.
//   build_up_lists  Γ+(v) = neighbours of higher rank (the cand set of v's
//                   subproblem in Algorithm 5), sorted by id.
#include <cooperative_groups.h>

#include "internal.cuh"

namespace cg = cooperative_groups;

namespace mce {

namespace {

// ------------------------------------------------------------------ CSR build

__global__ void k_make_keys(const int32_t *u, const int32_t *v, int64_t m, int32_t n, int32_t B, uint64_t *keys,
                            int32_t *bad) {
    const uint64_t sentinel = (B >= 32) ? ~0ULL : ((1ULL << (2 * B)) - 1);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = u[i], b = v[i];
        uint64_t k0 = sentinel, k1 = sentinel;
        if (a < 0 || a >= n || b < 0 || b >= n) {
            atomicOr(bad, 1);
        } else if (a != b) {
            k0 = ((uint64_t)a << B) | (uint64_t)b;
            k1 = ((uint64_t)b << B) | (uint64_t)a;
        }
        keys[2 * i] = k0;
        keys[2 * i + 1] = k1;
    }
}

__global__ void k_flag_unique(const uint64_t *keys, int64_t k, uint64_t sentinel, int32_t *flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = keys[i] != sentinel && (i == 0 || keys[i] != keys[i - 1]);
}

__global__ void k_compact_csr(const uint64_t *keys, const int32_t *pos, int64_t k, int32_t B, int32_t *col,
                              int32_t *deg) {
    const uint64_t mask = (1ULL << B) - 1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
        if (pos[i + 1] != pos[i]) {
            const uint64_t key = keys[i];
            col[pos[i]] = (int32_t)(key & mask);
            atomicAdd(&deg[key >> B], 1);
        }
    }
}

// ------------------------------------------------------------------ keys

__global__ void k_degree_key(const int32_t *row_ptr, int32_t n, int64_t *key) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        key[v] = row_ptr[v + 1] - row_ptr[v];
}

__global__ void k_degree_i32(const int32_t *row_ptr, int32_t n, int32_t *d) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        d[v] = row_ptr[v + 1] - row_ptr[v];
}

// Core numbers by level-synchronous peeling on a cooperative grid.  Level k:
// every alive vertex whose remaining degree is <= k is removed with core
// number k; removing a vertex decrements its alive neighbours, and those that
// fall to <= k are removed at the same level (claimed once by CAS).
// The seeding scan of a level visits only the vertices still alive after the
// previous one (a compacted list), so a level costs its alive count, not n.
// The removal cascade gives each removed vertex a warp (hubs leave at the
// high levels, where the frontier is short).  Levels that would remove
// nothing are skipped: the next level is the smallest remaining degree.
// ctl[0] = removed so far, ctl[1], ctl[2] = lengths of the two frontiers,
// ctl[3], ctl[4] = lengths of the two alive lists, ctl[5], ctl[6] = smallest
// remaining degree (one slot per level parity).
// Every read of a control word is followed by a grid barrier before any
// thread may change that word, so all threads take the same branches.
__global__ void k_core_peel(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col, int32_t n,
                            int32_t *d, int32_t *core, int32_t *fa, int32_t *fb, int32_t *la, int32_t *lb,
                            int32_t *ctl) {
    cg::grid_group grid = cg::this_grid();
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const int64_t wid = tid >> 5, nwarp = nth >> 5;
    int32_t *cur = fa, *nxt = fb, *alive = la, *alive2 = lb;
    int ci = 1, ni = 2, ai = 3, bi = 4;
    int par = 0;
    for (int32_t k = 0; k <= n;) {   // a core number never exceeds n - 1
        grid.sync();
        const int32_t removed = *(volatile int32_t *)&ctl[0];
        const int32_t na = *(volatile int32_t *)&ctl[ai];
        grid.sync();
        if (removed >= n) break;
        const int mi = 5 + par;
        if (tid == 0) ctl[5 + (1 - par)] = 0x7fffffff;   // slot of the next level, untouched in this one
        int32_t lmin = 0x7fffffff;
        for (int64_t i = tid; i < na; i += nth) {
            const int32_t v = alive[i];
            if (*(volatile int32_t *)&core[v] >= 0) continue;   // removed at an earlier level
            const int32_t dv = d[v];
            if (dv <= k) {
                core[v] = k;
                cur[atomicAdd(&ctl[ci], 1)] = v;
            } else {
                alive2[atomicAdd(&ctl[bi], 1)] = v;
                lmin = dv < lmin ? dv : lmin;
            }
        }
        lmin = __reduce_min_sync(0xffffffffu, lmin);
        if (lane == 0 && lmin != 0x7fffffff) atomicMin(&ctl[mi], lmin);
        grid.sync();
        if (tid == 0) ctl[ai] = 0;   // read by everyone before the last barrier
        {
            int32_t *t = alive;
            alive = alive2;
            alive2 = t;
            const int ti = ai;
            ai = bi;
            bi = ti;
        }
        for (;;) {
            const int32_t len = *(volatile int32_t *)&ctl[ci];
            grid.sync();
            if (len == 0) break;
            int32_t cmin = 0x7fffffff;
            for (int64_t i = wid; i < len; i += nwarp) {
                const int32_t x = cur[i];
                const int32_t e1 = row_ptr[x + 1];
                for (int32_t e = row_ptr[x] + lane; e < e1; e += 32) {
                    const int32_t w = col[e];
                    if (*(volatile int32_t *)&core[w] >= 0) continue;
                    const int32_t nd = atomicSub(&d[w], 1) - 1;
                    if (nd <= k) {
                        if (atomicCAS(&core[w], -1, k) == -1) nxt[atomicAdd(&ctl[ni], 1)] = w;
                    } else {
                        cmin = nd < cmin ? nd : cmin;
                    }
                }
            }
            cmin = __reduce_min_sync(0xffffffffu, cmin);
            if (lane == 0 && cmin != 0x7fffffff) atomicMin(&ctl[mi], cmin);
            if (tid == 0) {
                atomicAdd(&ctl[0], len);
                ctl[ci] = 0;   // nobody reads ctl[ci] again before the next barrier
            }
            int32_t *t = cur;
            cur = nxt;
            nxt = t;
            int ti = ci;
            ci = ni;
            ni = ti;
            grid.sync();
        }
        // every survivor now has a remaining degree > k; the smallest is the
        // next level that removes anything (slot mi is not written again
        // before everyone has read it: the next level uses the other slot)
        const int32_t mn = *(volatile int32_t *)&ctl[mi];
        k = mn > k + 1 ? mn : k + 1;
        par ^= 1;
    }
}

__global__ void k_iota(int32_t *a, int32_t n) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        a[v] = (int32_t)v;
}

__global__ void k_i32_to_i64(const int32_t *a, int32_t n, int64_t *b) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        b[v] = a[v];
}

// Triangles: with Γ+ oriented by degree rank, each triangle {a, b, x} with
// rank a < b < x is found once as x ∈ Γ+(a) ∩ Γ+(b) while visiting the
// oriented edge (a, b); all three corners are credited.  One warp per a.
__global__ void k_triangles(const int32_t *__restrict__ up_ptr, const int32_t *__restrict__ up_col, int32_t n,
                            unsigned long long *t) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t a = warp; a < n; a += nwarps) {
        const int32_t a0 = up_ptr[a], la = up_ptr[a + 1] - a0;
        if (la < 2) continue;
        const int32_t *A = up_col + a0;
        unsigned long long ta = 0;
        for (int32_t j = 0; j < la; ++j) {
            const int32_t b = A[j];
            const int32_t b0 = up_ptr[b], lb = up_ptr[b + 1] - b0;
            unsigned long long cnt = 0;
            for (int32_t s = 0; s < lb; s += 32) {
                bool hit = false;
                int32_t x = -1;
                if (s + lane < lb) {
                    x = up_col[b0 + s + lane];
                    int32_t lo = 0, hi = la;
                    while (lo < hi) {
                        const int32_t mid = (lo + hi) >> 1;
                        if (A[mid] < x) lo = mid + 1; else hi = mid;
                    }
                    hit = lo < la && A[lo] == x;
                }
                if (hit) atomicAdd(&t[x], 1ULL);
                cnt += __popc(__ballot_sync(0xffffffffu, hit));
            }
            if (lane == 0 && cnt) atomicAdd(&t[b], cnt);
            ta += cnt;
        }
        if (lane == 0 && ta) atomicAdd(&t[a], ta);
    }
}

// ------------------------------------------------------------------ ranks

__global__ void k_rank_keys_i64(const int64_t *key, int32_t n, int32_t idb, uint64_t *out) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        out[v] = ((uint64_t)key[v] << idb) | (uint64_t)v;
}

__global__ void k_rank_keys_f32(const float *key, int32_t n, int32_t idb, uint64_t *out) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        uint32_t b = __float_as_uint(key[v]);
        b ^= (b >> 31) ? 0xffffffffu : 0x80000000u;   // order-preserving map of floats to uint32
        out[v] = ((uint64_t)b << idb) | (uint64_t)v;
    }
}

__global__ void k_scatter_rank(const uint64_t *sorted, int32_t n, int32_t idb, int32_t *rank) {
    const uint64_t mask = (1ULL << idb) - 1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        rank[sorted[i] & mask] = (int32_t)i;
}

__global__ void k_max_i64(const int64_t *a, int32_t n, unsigned long long *mx) {
    unsigned long long m = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (unsigned long long)max(a[v], (int64_t)0));
    for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(mx, m);
}

// ------------------------------------------------------------------ Γ+ lists

__global__ void k_up_count(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                           const int32_t *__restrict__ rank, int32_t n, int32_t *cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < n; v += nwarps) {
        const int32_t rv = rank[v];
        int32_t c = 0;
        for (int32_t e = row_ptr[v] + lane; e < row_ptr[v + 1]; e += 32) c += rank[col[e]] > rv;
        c = __reduce_add_sync(0xffffffffu, c);
        if (lane == 0) cnt[v] = c;
    }
}

__global__ void k_up_fill(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                          const int32_t *__restrict__ rank, int32_t n, const int32_t *__restrict__ up_ptr,
                          int32_t *up_col) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < n; v += nwarps) {
        const int32_t rv = rank[v];
        int32_t out = up_ptr[v];
        const int32_t e1 = row_ptr[v + 1];
        for (int32_t e0 = row_ptr[v]; e0 < e1; e0 += 32) {
            const int32_t e = e0 + lane;
            int32_t w = 0;
            bool up = false;
            if (e < e1) {
                w = col[e];
                up = rank[w] > rv;
            }
            const uint32_t b = __ballot_sync(0xffffffffu, up);
            if (up) up_col[out + __popc(b & lanemask_lt())] = w;
            out += __popc(b);
        }
    }
}

}  // namespace

// ------------------------------------------------------------------ host side

namespace {

// Validation of a caller CSR (simple undirected graph): bit 1 row offsets,
// 2 row not strictly increasing, 4 id outside [0, n), 8 self loop, 16 an
// entry (x, y) without (y, x).
__global__ void k_check_csr(const int32_t *row_ptr, const int32_t *col, int32_t n, int64_t nnz, int32_t *bad) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t0 == 0 && (row_ptr[0] != 0 || (int64_t)row_ptr[n] != nnz)) atomicOr(bad, 1);
    for (int64_t x = t0; x < n; x += stride) {
        const int32_t r0 = row_ptr[x], r1 = row_ptr[x + 1];
        if (r0 < 0 || r1 < r0 || (int64_t)r1 > nnz) {
            atomicOr(bad, 1);
            continue;
        }
        for (int32_t e = r0; e < r1; ++e) {
            const int32_t y = col[e];
            if (y < 0 || y >= n) {
                atomicOr(bad, 4);
                continue;
            }
            if (y == x) atomicOr(bad, 8);
            if (e > r0 && col[e - 1] >= y) atomicOr(bad, 2);
            const int32_t q0 = row_ptr[y], q1 = row_ptr[y + 1];
            if (q0 < 0 || q1 < q0 || (int64_t)q1 > nnz) continue;   // row y is reported itself
            int32_t lo = q0, hi = q1;
            while (lo < hi) {
                const int32_t mid = lo + ((hi - lo) >> 1);
                if (col[mid] < (int32_t)x) lo = mid + 1; else hi = mid;
            }
            if (!(lo < q1 && col[lo] == (int32_t)x)) atomicOr(bad, 16);
        }
    }
}

}  // namespace

mce_status check_csr(const mce_graph *g, cudaStream_t s) {
    DevBuf bad;
    MCE_TRY(bad.alloc(4, s));
    MCE_CUDA(cudaMemsetAsync(bad.p, 0, 4, s));
    MCE_LAUNCH(k_check_csr, grid_for(g->n > 0 ? g->n : 1, 256), 256, 0, s, g->row_ptr, g->col, g->n, g->nnz,
               bad.as<int32_t>());
    int32_t hb = 0;
    MCE_CUDA(cudaMemcpyAsync(&hb, bad.p, 4, cudaMemcpyDeviceToHost, s));
    MCE_CUDA(cudaStreamSynchronize(s));
    if (hb) {
        g_last_error = std::string("mce_graph_from_csr: not a simple undirected CSR:") +
                       ((hb & 1) ? " row offsets" : "") + ((hb & 2) ? " row not strictly increasing" : "") +
                       ((hb & 4) ? " id outside [0, n)" : "") + ((hb & 8) ? " self loop" : "") +
                       ((hb & 16) ? " not symmetric" : "");
        return MCE_EINVAL;
    }
    return MCE_OK;
}

mce_status build_csr(const int32_t *u, const int32_t *v, int64_t m, int32_t n, cudaStream_t s, mce_graph *g) {
    g->n = n;
    g->id_bits = bits_for(n > 0 ? (uint64_t)(n - 1) : 0);
    MCE_TRY(dev_alloc((void **)&g->row_ptr, ((size_t)n + 1) * sizeof(int32_t), s, "cudaMallocAsync"));
    if (m == 0 || n == 0) {
        MCE_CUDA(cudaMemsetAsync(g->row_ptr, 0, ((size_t)n + 1) * sizeof(int32_t), s));
        MCE_TRY(dev_alloc((void **)&g->col, 16, s, "cudaMallocAsync"));
        g->nnz = 0;
        return MCE_OK;
    }
    const int32_t B = g->id_bits;
    const int64_t k = 2 * m;
    if (k >= ((int64_t)1 << 31) - 1) {
        g_last_error = "mce_graph_create: too many pairs";
        return MCE_EINVAL;
    }
    DevBuf keys, tmp, flag, bad;
    MCE_TRY(keys.alloc((size_t)k * sizeof(uint64_t), s));
    MCE_TRY(tmp.alloc((size_t)k * sizeof(uint64_t), s));
    MCE_TRY(flag.alloc(((size_t)k + 1) * sizeof(int32_t), s));
    MCE_TRY(bad.alloc(sizeof(int32_t), s));
    MCE_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int32_t), s));
    MCE_LAUNCH(k_make_keys, grid_for(m, 256), 256, 0, s, u, v, m, n, B, keys.as<uint64_t>(), bad.as<int32_t>());
    int32_t hbad = 0;
    MCE_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    MCE_CUDA(cudaStreamSynchronize(s));
    if (hbad) {
        g_last_error = "mce_graph_create: vertex id outside [0, n)";
        return MCE_EINVAL;
    }
    MCE_TRY(radix_sort_u64(keys.as<uint64_t>(), tmp.as<uint64_t>(), k, 2 * B, s));
    const uint64_t sentinel = (B >= 32) ? ~0ULL : ((1ULL << (2 * B)) - 1);
    MCE_LAUNCH(k_flag_unique, grid_for(k, 256), 256, 0, s, keys.as<uint64_t>(), k, sentinel, flag.as<int32_t>());
    MCE_TRY(exclusive_scan_i32(flag.as<int32_t>(), flag.as<int32_t>(), k, s));
    int32_t nnz = 0;
    MCE_CUDA(cudaMemcpyAsync(&nnz, flag.as<int32_t>() + k, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    MCE_CUDA(cudaStreamSynchronize(s));
    g->nnz = nnz;
    MCE_TRY(dev_alloc((void **)&g->col, ((size_t)nnz + 4) * sizeof(int32_t), s, "cudaMallocAsync"));
    MCE_CUDA(cudaMemsetAsync(g->row_ptr, 0, ((size_t)n + 1) * sizeof(int32_t), s));
    MCE_LAUNCH(k_compact_csr, grid_for(k, 256), 256, 0, s, keys.as<uint64_t>(), flag.as<int32_t>(), k, B, g->col,
               g->row_ptr);
    MCE_TRY(exclusive_scan_i32(g->row_ptr, g->row_ptr, n, s));
    return MCE_OK;
}

static mce_status core_numbers(const mce_graph *g, cudaStream_t s, int64_t *key) {
    const int32_t n = g->n;
    DevBuf d, core, fa, fb, la, lb, ctl;
    MCE_TRY(d.alloc((size_t)n * sizeof(int32_t), s));
    MCE_TRY(core.alloc((size_t)n * sizeof(int32_t), s));
    MCE_TRY(fa.alloc((size_t)n * sizeof(int32_t), s));
    MCE_TRY(fb.alloc((size_t)n * sizeof(int32_t), s));
    MCE_TRY(la.alloc((size_t)n * sizeof(int32_t), s));
    MCE_TRY(lb.alloc((size_t)n * sizeof(int32_t), s));
    MCE_TRY(ctl.alloc(8 * sizeof(int32_t), s));
    MCE_LAUNCH(k_degree_i32, grid_for(n, 256), 256, 0, s, g->row_ptr, n, d.as<int32_t>());
    MCE_LAUNCH(k_iota, grid_for(n, 256), 256, 0, s, la.as<int32_t>(), n);
    MCE_CUDA(cudaMemsetAsync(core.p, 0xff, (size_t)n * sizeof(int32_t), s));
    // ctl[3] = n alive, ctl[5] = no remaining degree seen yet
    const int32_t ctl0[8] = {0, 0, 0, n, 0, 0x7fffffff, 0x7fffffff, 0};
    MCE_CUDA(cudaMemcpyAsync(ctl.p, ctl0, sizeof(ctl0), cudaMemcpyHostToDevice, s));
    int dev = 0, per_sm = 0;
    MCE_CUDA(cudaGetDevice(&dev));
    MCE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_core_peel, 256, 0));
    if (per_sm < 1) {
        g_last_error = "core_numbers: cooperative kernel does not fit";
        return MCE_ECUDA;
    }
    // few blocks: the many grid barriers cost in proportion to the blocks
    unsigned blocks = (unsigned)(num_sms() * (per_sm < 2 ? per_sm : 2));
    const int32_t *rp = g->row_ptr, *cl = g->col;
    int32_t *pd = d.as<int32_t>(), *pc = core.as<int32_t>(), *pa = fa.as<int32_t>(), *pb = fb.as<int32_t>(),
            *pla = la.as<int32_t>(), *plb = lb.as<int32_t>(), *pt = ctl.as<int32_t>();
    int32_t nn = n;
    void *args[] = {(void *)&rp, (void *)&cl, (void *)&nn, (void *)&pd, (void *)&pc, (void *)&pa, (void *)&pb,
                    (void *)&pla, (void *)&plb, (void *)&pt};
    g_launches.fetch_add(1, std::memory_order_relaxed);
    MCE_CUDA(cudaLaunchCooperativeKernel((const void *)k_core_peel, dim3(blocks), dim3(256), args, 0, s));
    MCE_LAUNCH(k_i32_to_i64, grid_for(n, 256), 256, 0, s, core.as<int32_t>(), n, key);
    return MCE_OK;
}

static mce_status triangle_counts(const mce_graph *g, cudaStream_t s, int64_t *key) {
    const int32_t n = g->n;
    DevBuf deg, rank, up_ptr, up_col;
    MCE_TRY(deg.alloc((size_t)n * sizeof(int64_t), s));
    MCE_TRY(rank.alloc((size_t)n * sizeof(int32_t), s));
    MCE_LAUNCH(k_degree_key, grid_for(n, 256), 256, 0, s, g->row_ptr, n, deg.as<int64_t>());
    MCE_TRY(rank_from_key_i64(deg.as<int64_t>(), n, g->id_bits, s, rank.as<int32_t>()));
    int64_t up_nnz = 0;
    MCE_TRY(build_up_lists(g, rank.as<int32_t>(), s, up_ptr, up_col, &up_nnz));
    MCE_CUDA(cudaMemsetAsync(key, 0, (size_t)n * sizeof(int64_t), s));
    MCE_LAUNCH(k_triangles, grid_for((int64_t)n * 32, 256), 256, 0, s, up_ptr.as<int32_t>(), up_col.as<int32_t>(), n,
               reinterpret_cast<unsigned long long *>(key));
    return MCE_OK;
}

mce_status vertex_key(const mce_graph *g, int32_t kind, cudaStream_t s, int64_t *key) {
    if (g->n == 0) return MCE_OK;
    switch (kind) {
        case MCE_RANK_DEGREE:
            MCE_LAUNCH(k_degree_key, grid_for(g->n, 256), 256, 0, s, g->row_ptr, g->n, key);
            return MCE_OK;
        case MCE_RANK_DEGEN:
            return core_numbers(g, s, key);
        case MCE_RANK_TRIANGLE:
            return triangle_counts(g, s, key);
        default:
            g_last_error = "vertex_key: unknown kind";
            return MCE_EINVAL;
    }
}

mce_status rank_from_key_i64(const int64_t *key, int32_t n, int32_t id_bits, cudaStream_t s, int32_t *rank) {
    if (n == 0) return MCE_OK;
    DevBuf keys, tmp, mx;
    MCE_TRY(keys.alloc((size_t)n * sizeof(uint64_t), s));
    MCE_TRY(tmp.alloc((size_t)n * sizeof(uint64_t), s));
    MCE_TRY(mx.alloc(sizeof(unsigned long long), s));
    MCE_CUDA(cudaMemsetAsync(mx.p, 0, sizeof(unsigned long long), s));
    MCE_LAUNCH(k_max_i64, grid_for(n, 256), 256, 0, s, key, n, mx.as<unsigned long long>());
    unsigned long long hmx = 0;
    MCE_CUDA(cudaMemcpyAsync(&hmx, mx.p, sizeof(hmx), cudaMemcpyDeviceToHost, s));
    MCE_CUDA(cudaStreamSynchronize(s));
    const int32_t bits = bits_for(hmx) + id_bits;
    if (bits > 64) {
        g_last_error = "rank_from_key: key too large";
        return MCE_EINVAL;
    }
    MCE_LAUNCH(k_rank_keys_i64, grid_for(n, 256), 256, 0, s, key, n, id_bits, keys.as<uint64_t>());
    MCE_TRY(radix_sort_u64(keys.as<uint64_t>(), tmp.as<uint64_t>(), n, bits, s));
    MCE_LAUNCH(k_scatter_rank, grid_for(n, 256), 256, 0, s, keys.as<uint64_t>(), n, id_bits, rank);
    return MCE_OK;
}

mce_status rank_from_key_f32(const float *key, int32_t n, int32_t id_bits, cudaStream_t s, int32_t *rank) {
    if (n == 0) return MCE_OK;
    DevBuf keys, tmp;
    MCE_TRY(keys.alloc((size_t)n * sizeof(uint64_t), s));
    MCE_TRY(tmp.alloc((size_t)n * sizeof(uint64_t), s));
    MCE_LAUNCH(k_rank_keys_f32, grid_for(n, 256), 256, 0, s, key, n, id_bits, keys.as<uint64_t>());
    MCE_TRY(radix_sort_u64(keys.as<uint64_t>(), tmp.as<uint64_t>(), n, 32 + id_bits, s));
    MCE_LAUNCH(k_scatter_rank, grid_for(n, 256), 256, 0, s, keys.as<uint64_t>(), n, id_bits, rank);
    return MCE_OK;
}

mce_status build_up_lists(const mce_graph *g, const int32_t *rank, cudaStream_t s, DevBuf &up_ptr, DevBuf &up_col,
                          int64_t *up_nnz) {
    const int32_t n = g->n;
    MCE_TRY(up_ptr.alloc(((size_t)n + 1) * sizeof(int32_t), s));
    if (n == 0) {
        MCE_CUDA(cudaMemsetAsync(up_ptr.p, 0, sizeof(int32_t), s));
        MCE_TRY(up_col.alloc(16, s));
        *up_nnz = 0;
        return MCE_OK;
    }
    MCE_LAUNCH(k_up_count, grid_for((int64_t)n * 32, 256), 256, 0, s, g->row_ptr, g->col, rank, n,
               up_ptr.as<int32_t>());
    MCE_TRY(exclusive_scan_i32(up_ptr.as<int32_t>(), up_ptr.as<int32_t>(), n, s));
    int32_t tot = 0;
    MCE_CUDA(cudaMemcpyAsync(&tot, up_ptr.as<int32_t>() + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    MCE_CUDA(cudaStreamSynchronize(s));
    *up_nnz = tot;
    MCE_TRY(up_col.alloc(((size_t)tot + 4) * sizeof(int32_t), s));
    MCE_LAUNCH(k_up_fill, grid_for((int64_t)n * 32, 256), 256, 0, s, g->row_ptr, g->col, rank, n,
               up_ptr.as<int32_t>(), up_col.as<int32_t>());
    return MCE_OK;
}

}  // namespace mce
