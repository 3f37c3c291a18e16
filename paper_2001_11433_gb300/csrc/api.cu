// extern "C" entry points of libmce_gb300 (declared in include/mce.h).
#include <string.h>

#include "mce_host.h"

namespace mce {
thread_local std::string g_last_error;
std::atomic<uint64_t> g_launches{0};

// Allocation-failure injection (mce_debug_fail_alloc): the allocation that
// finds the counter at 0 fails; negative = off.
static std::atomic<int64_t> g_fail_alloc_after{-1};

mce_status dev_alloc(void **p, size_t bytes, cudaStream_t s, const char *what) {
    int64_t k = g_fail_alloc_after.load();
    while (k >= 0 && !g_fail_alloc_after.compare_exchange_weak(k, k - 1)) {
    }
    if (k == 0) {
        *p = nullptr;
        g_last_error = std::string(what) + ": injected allocation failure";
        return MCE_ENOMEM;
    }
    return cuda_status(cudaMallocAsync(p, bytes, s), what);
}

// Keep freed stream-ordered memory in the pool so that repeated calls do not
// return it to the driver and allocate it again.
static void init_pool_once() {
    static bool done = false;
    if (done) return;
    done = true;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return;
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
}
}  // namespace mce

using namespace mce;

extern "C" {

const char *mce_strerror(mce_status s) {
    switch (s) {
        case MCE_OK: return "ok";
        case MCE_EINVAL: return "invalid argument";
        case MCE_ENOMEM: return "out of device memory";
        case MCE_EOVERFLOW: return "output buffer too small (summary exact)";
        case MCE_EBUDGET: return "node budget exhausted (result incomplete)";
        case MCE_ETIMEOUT: return "bounded device wait gave up (result incomplete)";
        case MCE_ECUDA: return "CUDA error";
        case MCE_ESTATE: return "object in an unusable state";
        default: return "unknown status";
    }
}

const char *mce_last_error(void) { return g_last_error.c_str(); }

void mce_opts_init(mce_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->rank_kind = MCE_RANK_DEGEN;
    o->split = 1;
}

uint64_t mce_kernel_launches(void) { return g_launches.load(); }

void mce_debug_fail_alloc(int64_t after) { g_fail_alloc_after.store(after < 0 ? -1 : after); }

mce_status mce_graph_create(const int32_t *u, const int32_t *v, int64_t m, int32_t n, int32_t on_device, void *stream,
                            mce_graph **g) {
    if (!g || m < 0 || n < 0 || n >= (1 << 30) || (m > 0 && (!u || !v))) {
        g_last_error = "mce_graph_create: bad arguments";
        return MCE_EINVAL;
    }
    init_pool_once();
    cudaStream_t s = (cudaStream_t)stream;
    mce_graph *gr = new mce_graph();
    DevBuf du, dv;
    const int32_t *pu = u, *pv = v;
    mce_status st = MCE_OK;
    if (!on_device && m > 0) {
        st = du.alloc((size_t)m * 4, s);
        if (st == MCE_OK) st = dv.alloc((size_t)m * 4, s);
        if (st == MCE_OK) st = cuda_status(cudaMemcpyAsync(du.p, u, (size_t)m * 4, cudaMemcpyHostToDevice, s), "H2D u");
        if (st == MCE_OK) st = cuda_status(cudaMemcpyAsync(dv.p, v, (size_t)m * 4, cudaMemcpyHostToDevice, s), "H2D v");
        pu = du.as<int32_t>();
        pv = dv.as<int32_t>();
    }
    if (st == MCE_OK) st = build_csr(pu, pv, m, n, s, gr);
    if (st == MCE_OK) st = cuda_status(cudaStreamSynchronize(s), "mce_graph_create");
    if (st != MCE_OK) {
        mce_graph_free(gr);
        return st;
    }
    *g = gr;
    return MCE_OK;
}

mce_status mce_graph_from_csr(const int32_t *row_ptr, const int32_t *col, int32_t n, int64_t nnz, int32_t on_device,
                              void *stream, mce_graph **g) {
    if (!g || !row_ptr || n < 0 || n >= (1 << 30) || nnz < 0 || nnz >= ((int64_t)1 << 31) - 1 || (nnz > 0 && !col)) {
        g_last_error = "mce_graph_from_csr: bad arguments";
        return MCE_EINVAL;
    }
    init_pool_once();
    cudaStream_t s = (cudaStream_t)stream;
    mce_graph *gr = new mce_graph();
    gr->n = n;
    gr->nnz = nnz;
    gr->id_bits = bits_for(n > 0 ? (uint64_t)(n - 1) : 0);
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    mce_status st = dev_alloc((void **)&gr->row_ptr, ((size_t)n + 1) * 4, s, "cudaMallocAsync");
    if (st == MCE_OK) st = dev_alloc((void **)&gr->col, ((size_t)nnz + 4) * 4, s, "cudaMallocAsync");
    if (st == MCE_OK)
        st = cuda_status(cudaMemcpyAsync(gr->row_ptr, row_ptr, ((size_t)n + 1) * 4, kind, s), "copy row_ptr");
    if (st == MCE_OK && nnz > 0)
        st = cuda_status(cudaMemcpyAsync(gr->col, col, (size_t)nnz * 4, kind, s), "copy col");
    if (st == MCE_OK) st = check_csr(gr, s);
    if (st != MCE_OK) {
        mce_graph_free(gr);
        return st;
    }
    *g = gr;
    return MCE_OK;
}

mce_status mce_graph_csr(const mce_graph *g, int32_t *n, int64_t *nnz, const int32_t **row_ptr, const int32_t **col) {
    if (!g) return MCE_EINVAL;
    if (n) *n = g->n;
    if (nnz) *nnz = g->nnz;
    if (row_ptr) *row_ptr = g->row_ptr;
    if (col) *col = g->col;
    return MCE_OK;
}

mce_status mce_graph_copy_csr(const mce_graph *g, int32_t *row_ptr, int32_t *col, int32_t to_host, void *stream) {
    if (!g || !row_ptr || (!col && g->nnz)) {
        g_last_error = "mce_graph_copy_csr: bad arguments";
        return MCE_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const cudaMemcpyKind kind = to_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    MCE_CUDA(cudaMemcpyAsync(row_ptr, g->row_ptr, ((size_t)g->n + 1) * 4, kind, s));
    if (g->nnz) MCE_CUDA(cudaMemcpyAsync(col, g->col, (size_t)g->nnz * 4, kind, s));
    MCE_CUDA(cudaStreamSynchronize(s));
    return MCE_OK;
}

void mce_graph_free(mce_graph *g) {
    if (!g) return;
    cudaDeviceSynchronize();
    if (g->row_ptr) cudaFree(g->row_ptr);
    if (g->col) cudaFree(g->col);
    delete g;
}

mce_status mce_vertex_key(const mce_graph *g, int32_t kind, void *stream, int64_t *key) {
    if (!g || !key || kind < MCE_RANK_DEGREE || kind > MCE_RANK_TRIANGLE) {
        g_last_error = "mce_vertex_key: bad arguments";
        return MCE_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    MCE_TRY(vertex_key(g, kind, s, key));
    MCE_CUDA(cudaStreamSynchronize(s));
    return MCE_OK;
}

mce_status mce_rank(const mce_graph *g, const mce_opts *opts, int32_t *rank_out) {
    if (!g || !opts || !rank_out) {
        g_last_error = "mce_rank: bad arguments";
        return MCE_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)opts->stream;
    MCE_TRY(compute_rank(g, opts, s, rank_out));
    MCE_CUDA(cudaStreamSynchronize(s));
    return MCE_OK;
}

mce_status mce_enumerate(const mce_graph *g, const mce_opts *opts, mce_result *res) {
    if (!g || !opts || !res) {
        g_last_error = "mce_enumerate: bad arguments";
        return MCE_EINVAL;
    }
    if ((opts->list_off != nullptr) != (opts->list_vtx != nullptr) ||
        ((opts->pv_count != nullptr) != (opts->pv_hash != nullptr)) ||
        ((opts->pv_count != nullptr) != (opts->pv_nodes != nullptr))) {
        g_last_error = "mce_enumerate: list or per-vertex buffers incomplete";
        return MCE_EINVAL;
    }
    init_pool_once();
    memset(res, 0, sizeof(*res));
    return enumerate(g, opts, res, nullptr, nullptr, 0, nullptr, nullptr);
}

}  // extern "C"
