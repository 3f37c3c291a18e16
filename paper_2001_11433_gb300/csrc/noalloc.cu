// mce_enumerate_noalloc: static maximal clique enumeration that allocates no
// memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the
// point where they want to enumerate: code running inside a memory-pool
// owner that forbids foreign allocations, long-running services that must
// not grow their footprint after start-up, or hosts that pre-reserve all
// device memory.  For them this entry point takes the graph (CSR) and a
// vertex rank that the caller already holds on the device, and keeps all of
// its intermediate data in one file-scope device array of fixed size
// (MCE_NOALLOC_SCRATCH_BYTES).  That array is part of the loaded library, so
// every GPU that loads the library holds it until the process exits.
//
// The host cannot use the array's name as a device address; the first call
// on each device (with that device current) looks the address up with
// cudaGetSymbolAddress and caches it.  Make that first call before any stream
// capture.  All calls share the array and it keeps the last call's contents;
// everything that must start at zero is cleared by the call itself.  Calls
// that overlap on the GPU (different streams, or several host threads) race
// on the array and must be serialised by the caller.
#include <mutex>

#include "mce_host.h"

namespace mce {
namespace {

constexpr size_t kScratchBytes = MCE_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {};

constexpr int kTile = 2048;          // scan tile (256 threads x 8 items)
constexpr int64_t kMaxScan = (int64_t)kTile * kTile;

// ---- small kernels of this entry point (their own copies; nothing allocates)

__global__ void k_na_up_count(const int32_t *row_ptr, const int32_t *col, const int32_t *rank, int32_t n,
                              int32_t *cnt) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = 0;
        const int32_t rv = rank[v];
        for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) c += rank[col[e]] > rv;
        cnt[v] = c;
    }
}

__global__ void k_na_up_fill(const int32_t *row_ptr, const int32_t *col, const int32_t *rank, int32_t n,
                             const int32_t *up_ptr, int32_t *up_col, int64_t up_cap) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        int32_t o = up_ptr[v];
        const int32_t rv = rank[v];
        for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e)
            if (rank[col[e]] > rv && o < up_cap) up_col[o++] = col[e];
    }
}

// Input checks, in two passes so that no pass reads through a value that an
// earlier pass has not checked.  Bits of *bad:
//   1 row_ptr[0] != 0 or row_ptr[n] != nnz     2 row_ptr decreases
//   4 rank value outside [0, n)                8 col id outside [0, n)
//  16 self loop                               32 row not strictly increasing
//  64 (x, y) present without (y, x)          128 two vertices with one rank value
__global__ void k_na_check_ptr(const int32_t *row_ptr, const int32_t *rank, int32_t n, int64_t nnz, int32_t *bad) {
    int32_t b = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        if (row_ptr[v] > row_ptr[v + 1]) b |= 2;
        if (rank[v] < 0 || rank[v] >= n) b |= 4;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && (row_ptr[0] != 0 || (int64_t)row_ptr[n] != nnz)) b |= 1;
    if (b) atomicOr(bad, b);
}

// seen: int32[n], zero on entry
__global__ void k_na_check_adj(const int32_t *row_ptr, const int32_t *col, const int32_t *rank, int32_t n,
                               int32_t *seen, int32_t *bad) {
    int32_t b = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        if (atomicExch(&seen[rank[v]], 1) != 0) b |= 128;
        const int32_t e0 = row_ptr[v], e1 = row_ptr[v + 1];
        for (int32_t e = e0; e < e1; ++e) {
            const int32_t x = col[e];
            if (x < 0 || x >= n) {
                b |= 8;
                continue;
            }
            if (x == v) b |= 16;
            if (e > e0 && col[e - 1] >= x) b |= 32;
            // (v, x) needs (x, v): binary search of v in x's row (sorted if the row checks pass)
            int32_t lo = row_ptr[x], hi = row_ptr[x + 1];
            while (lo < hi) {
                const int32_t mid = lo + ((hi - lo) >> 1);
                if (col[mid] < (int32_t)v) lo = mid + 1; else hi = mid;
            }
            if (lo >= row_ptr[x + 1] || col[lo] != (int32_t)v) b |= 64;
        }
    }
    if (b) atomicOr(bad, b);
}

const char *na_check_text(int32_t b) {
    if (b & 1) return "mce_enumerate_noalloc: row_ptr[0] must be 0 and row_ptr[n] must equal nnz";
    if (b & 2) return "mce_enumerate_noalloc: row_ptr decreases";
    if (b & 4) return "mce_enumerate_noalloc: a rank value lies outside [0, n)";
    if (b & 8) return "mce_enumerate_noalloc: a column id lies outside [0, n)";
    if (b & 16) return "mce_enumerate_noalloc: self loop in the CSR";
    if (b & 32) return "mce_enumerate_noalloc: a row is not strictly increasing (unsorted or repeated ids)";
    if (b & 64) return "mce_enumerate_noalloc: the CSR is not symmetric ((x, y) without (y, x))";
    return "mce_enumerate_noalloc: rank is not a permutation (two vertices share a value)";
}

// per-tile sums
__global__ void k_na_tile_sum(const int32_t *in, int64_t n, int32_t *sums) {
    __shared__ int32_t red[256];
    const int64_t base = (int64_t)blockIdx.x * kTile;
    int32_t s = 0;
    for (int i = threadIdx.x; i < kTile; i += 256)
        if (base + i < n) s += in[base + i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = red[0];
}

// exclusive scan of one tile of at most kTile values by one block, in place;
// writes the total to *total
__device__ void na_block_scan(int32_t *a, int64_t n, int32_t offset, int32_t *total) {
    __shared__ int32_t part[256];
    const int64_t base = (int64_t)threadIdx.x * 8;
    int32_t v[8], s = 0;
    for (int i = 0; i < 8; ++i) {
        v[i] = base + i < n ? a[base + i] : 0;
        s += v[i];
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < 256; o <<= 1) {   // Hillis-Steele over the 256 partial sums
        const int32_t y = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += y;
        __syncthreads();
    }
    int32_t run = part[threadIdx.x] - s + offset;
    for (int i = 0; i < 8; ++i) {
        if (base + i < n) a[base + i] = run;
        run += v[i];
    }
    if (threadIdx.x == 255 && total) *total = part[255] + offset;
}

__global__ void k_na_scan_sums(int32_t *sums, int64_t tiles) { na_block_scan(sums, tiles, 0, nullptr); }

// in[0..n) -> exclusive scan in out[0..n], out[n] = total; one block per tile
__global__ void k_na_scan_apply(const int32_t *in, int32_t *out, int64_t n, const int32_t *tile_off) {
    const int64_t base = (int64_t)blockIdx.x * kTile;
    const int64_t len = n - base < kTile ? n - base : kTile;
    int32_t *seg = out + base;
    for (int i = threadIdx.x; i < len; i += 256) seg[i] = in[base + i];
    __syncthreads();
    int32_t *tot = (blockIdx.x == gridDim.x - 1) ? out + n : nullptr;
    na_block_scan(seg, len, tile_off[blockIdx.x], tot);
}

__global__ void k_na_prepass(const int32_t *row_ptr, const int32_t *up_ptr, int32_t n, uint64_t seed,
                             unsigned long long *out, int32_t *flag, unsigned long long *reqc) {
    unsigned long long cnt = 0, hsh = 0, nodes = 0, req = 0, cm = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t w = row_ptr[v + 1] - row_ptr[v], c = up_ptr[v + 1] - up_ptr[v];
        int32_t f = 0;
        if (w == 0) {
            cnt++;
            hsh += clique_hash_from_sum(vertex_hash((int32_t)v, seed), 1);
            nodes++;
        } else if (c == 0) {
            nodes++;
        } else {
            f = 1;
            req = max(req, (unsigned long long)bk_ws_words(w, c, BK_MCE));
            cm = max(cm, (unsigned long long)c);
        }
        flag[v] = f;
    }
    if (cnt) {
        atomicAdd(&out[OUT_COUNT], cnt);
        atomicAdd(&out[OUT_HASH], hsh);
        atomicAdd(&out[OUT_HIST + 1], cnt);
        atomicMax(&out[OUT_MAXSIZE], 1ULL);
    }
    if (nodes) atomicAdd(&out[OUT_NODES], nodes);
    if (req) atomicMax(&reqc[0], req);
    if (cm) atomicMax(&reqc[1], cm);
}

__global__ void k_na_compact(const int32_t *flag_scan, int32_t n, int32_t *order) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        if (flag_scan[v + 1] != flag_scan[v]) order[flag_scan[v]] = (int32_t)v;
}

__global__ void k_na_seq(unsigned long long *seq, int64_t n, unsigned long long *ctl, unsigned long long pending) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        seq[i] = (unsigned long long)i;
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl[CTL_PENDING] = pending;
}

// bump allocator over the static array
struct Carve {
    unsigned char *base;
    size_t used = 0;
    bool ok = true;
    template <class T> T *take(size_t count) {
        const size_t bytes = ((count * sizeof(T)) + 255) & ~size_t(255);
        if (used + bytes > kScratchBytes) {
            ok = false;
            return nullptr;
        }
        T *p = reinterpret_cast<T *>(base + used);
        used += bytes;
        return p;
    }
};

mce_status scratch_address(void **out) {
    int dev = 0;
    MCE_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        g_last_error = "mce_enumerate_noalloc: device index out of range";
        return MCE_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return MCE_OK;
}

}  // namespace
}  // namespace mce

using namespace mce;

extern "C" mce_status mce_enumerate_noalloc(const int32_t *row_ptr, const int32_t *col, int32_t n, int64_t nnz,
                                            const int32_t *rank, uint64_t hash_seed, void *stream,
                                            mce_result *res) {
    if (!res || n < 0 || nnz < 0 || (n > 0 && (!row_ptr || !rank)) || (nnz > 0 && !col)) {
        g_last_error = "mce_enumerate_noalloc: bad arguments";
        return MCE_EINVAL;
    }
    if (n == 0 && nnz != 0) {
        g_last_error = "mce_enumerate_noalloc: nnz must be 0 when n is 0";
        return MCE_EINVAL;
    }
    if ((int64_t)n + 1 > kMaxScan) {
        g_last_error = "mce_enumerate_noalloc: more vertices than this entry point handles (4194303)";
        return MCE_EINVAL;
    }
    memset(res, 0, sizeof(*res));
    cudaStream_t s = (cudaStream_t)stream;
    void *sp = nullptr;
    MCE_TRY(scratch_address(&sp));
    Carve cv{reinterpret_cast<unsigned char *>(sp)};
    unsigned long long *out = cv.take<unsigned long long>(OUT_WORDS);
    unsigned long long *ctl = cv.take<unsigned long long>(CTL_WORDS);
    unsigned long long *reqc = cv.take<unsigned long long>(2);
    int32_t *up_ptr = cv.take<int32_t>((size_t)n + 1);
    int32_t *up_col = cv.take<int32_t>((size_t)nnz / 2 + 16);
    int32_t *flag = cv.take<int32_t>((size_t)n + 1);
    int32_t *sums = cv.take<int32_t>(kTile + 1);
    int32_t *order = cv.take<int32_t>((size_t)n + 1);
    int32_t *bad = cv.take<int32_t>(1);
    if (!cv.ok) {
        g_last_error = "mce_enumerate_noalloc: graph needs more than the MCE_NOALLOC_SCRATCH_BYTES scratch";
        return MCE_EINVAL;
    }
    MCE_CUDA(cudaMemsetAsync(out, 0, OUT_WORDS * 8, s));
    MCE_CUDA(cudaMemsetAsync(ctl, 0, CTL_WORDS * 8, s));
    MCE_CUDA(cudaMemsetAsync(reqc, 0, 16, s));
    const int64_t tiles = ((int64_t)n + kTile - 1) / kTile;
    int32_t n_act = 0;
    unsigned long long hreq[2] = {0, 0};
    if (n > 0) {
        // the caller's CSR and rank, checked before anything reads through them
        int32_t hbad = 0;
        MCE_CUDA(cudaMemsetAsync(bad, 0, 4, s));
        MCE_LAUNCH(k_na_check_ptr, grid_for(n, 256), 256, 0, s, row_ptr, rank, n, nnz, bad);
        MCE_CUDA(cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, s));
        MCE_CUDA(cudaStreamSynchronize(s));
        if (hbad == 0) {
            MCE_CUDA(cudaMemsetAsync(order, 0, (size_t)n * 4, s));   // `order` serves as the rank-seen flags
            MCE_LAUNCH(k_na_check_adj, grid_for(n, 256), 256, 0, s, row_ptr, col, rank, n, order, bad);
            MCE_CUDA(cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, s));
            MCE_CUDA(cudaStreamSynchronize(s));
        }
        if (hbad) {
            g_last_error = na_check_text(hbad);
            return MCE_EINVAL;
        }
        // Γ+ lists by the caller's rank
        MCE_LAUNCH(k_na_up_count, grid_for(n, 256), 256, 0, s, row_ptr, col, rank, n, flag);
        MCE_LAUNCH(k_na_tile_sum, (unsigned)tiles, 256, 0, s, flag, (int64_t)n, sums);
        MCE_LAUNCH(k_na_scan_sums, 1, 256, 0, s, sums, tiles);
        MCE_LAUNCH(k_na_scan_apply, (unsigned)tiles, 256, 0, s, flag, up_ptr, (int64_t)n, sums);
        MCE_LAUNCH(k_na_up_fill, grid_for(n, 256), 256, 0, s, row_ptr, col, rank, n, up_ptr, up_col,
                   (int64_t)(nnz / 2 + 16));
        // trivial subproblems, sizes, and the list of non-trivial ones (vertex order)
        MCE_LAUNCH(k_na_prepass, grid_for(n, 256), 256, 0, s, row_ptr, up_ptr, n, hash_seed, out, flag, reqc);
        MCE_LAUNCH(k_na_tile_sum, (unsigned)tiles, 256, 0, s, flag, (int64_t)n, sums);
        MCE_LAUNCH(k_na_scan_sums, 1, 256, 0, s, sums, tiles);
        MCE_LAUNCH(k_na_scan_apply, (unsigned)tiles, 256, 0, s, flag, flag, (int64_t)n, sums);
        MCE_LAUNCH(k_na_compact, grid_for(n, 256), 256, 0, s, flag, n, order);
        MCE_CUDA(cudaMemcpyAsync(&n_act, flag + n, 4, cudaMemcpyDeviceToHost, s));
        MCE_CUDA(cudaMemcpyAsync(hreq, reqc, 16, cudaMemcpyDeviceToHost, s));
        MCE_CUDA(cudaStreamSynchronize(s));
    }
    res->subproblems = n_act;
    if (n_act > 0) {
        // two blocks of eight warps per SM: fewer per-warp workspaces in the fixed scratch
        mce_opts shape;
        mce_opts_init(&shape);
        shape.blocks_per_sm = 2;
        const LaunchShape ls = launch_shape(&shape);
        const int64_t nwarps = (int64_t)num_sms() * ls.blocks_per_sm * ls.warps_per_block;
        BkParams P{};
        P.mode = BK_MCE;
        P.row_ptr = row_ptr;
        P.col = col;
        P.up_ptr = up_ptr;
        P.up_col = up_col;
        P.rank = rank;
        P.order = order;
        P.n_sub = n_act;
        P.seed = hash_seed;
        P.out = out;
        P.ctl = ctl;
        P.split = 1;
        P.split_nodes = 4096;
        P.smem_words = ls.smem_words;
        P.gws_words = (int64_t)hreq[0] > ls.smem_words ? (int64_t)hreq[0] : 16;
        const int64_t cmax = (int64_t)hreq[1];
        P.slot_words = (2 + cmax + 4 * ((cmax + 31) / 32) + 3) & ~int64_t(3);
        P.qcap = 1024;
        P.gws = cv.take<uint32_t>((size_t)nwarps * P.gws_words);
        P.arena = cv.take<uint32_t>((size_t)P.qcap * P.slot_words);
        P.qseq = cv.take<unsigned long long>((size_t)P.qcap);
        P.taskbuf = cv.take<uint32_t>((size_t)nwarps * P.slot_words);
        if (!cv.ok) {
            g_last_error = "mce_enumerate_noalloc: the search needs more than the MCE_NOALLOC_SCRATCH_BYTES scratch";
            return MCE_EINVAL;
        }
        P.timeout_ns = 60ULL * 1000000000ULL;
        P.max_run_ns = 600ULL * 1000000000ULL;
        MCE_LAUNCH(k_na_seq, grid_for(P.qcap, 256), 256, 0, s, P.qseq, P.qcap, ctl, (unsigned long long)n_act);
        MCE_TRY(launch_bk(P, ls.warps_per_block, ls.blocks_per_sm, s));
    }
    unsigned long long h[OUT_WORDS];
    unsigned long long c[CTL_WORDS];
    MCE_CUDA(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, s));
    MCE_CUDA(cudaMemcpyAsync(c, ctl, sizeof(c), cudaMemcpyDeviceToHost, s));
    MCE_CUDA(cudaStreamSynchronize(s));
    res->count = h[OUT_COUNT];
    res->hash = h[OUT_HASH];
    res->tree_nodes = h[OUT_NODES];
    res->hist_len = (int32_t)(h[OUT_MAXSIZE] ? h[OUT_MAXSIZE] + 1 : 0);
    if (res->hist_len > MCE_HIST_CAP) res->hist_len = MCE_HIST_CAP;
    for (int i = 0; i < res->hist_len; ++i) res->hist[i] = h[OUT_HIST + i];
    res->tasks_split = h[OUT_SPLITS];
    res->word_ops = h[OUT_WORDOPS];
    res->complete = (c[CTL_ABORT] & 3ULL) ? 0 : 1;
    if (c[CTL_ABORT] & 4ULL) {
        g_last_error = "mce_enumerate_noalloc: search workspace smaller than a subproblem";
        return MCE_ESTATE;
    }
    if (c[CTL_ABORT] & 2ULL) {
        g_last_error = "mce_enumerate_noalloc: a bounded device wait gave up";
        return MCE_ETIMEOUT;
    }
    if (h[OUT_FLAGS] & 2ULL) {
        g_last_error = "clique larger than the histogram";
        return MCE_EOVERFLOW;
    }
    return MCE_OK;
}
