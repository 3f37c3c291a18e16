// Internal declarations shared by the translation units of libmce_gb300.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include "../../include/mce.h"

namespace mce {

// ------------------------------------------------------------------ errors

extern thread_local std::string g_last_error;
extern std::atomic<uint64_t> g_launches;

inline mce_status cuda_status(cudaError_t e, const char *where) {
    if (e == cudaSuccess) return MCE_OK;
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? MCE_ENOMEM : MCE_ECUDA;
}

#define MCE_TRY(expr)                              \
    do {                                           \
        mce_status _s = (expr);                    \
        if (_s != MCE_OK) return _s;               \
    } while (0)

#define MCE_CUDA(expr) MCE_TRY(::mce::cuda_status((expr), #expr))

// Every kernel launch goes through this macro so that launches are counted
// and launch errors are caught.
#define MCE_LAUNCH(kernel, grid, block, smem, stream, ...)                         \
    do {                                                                           \
        ::mce::g_launches.fetch_add(1, std::memory_order_relaxed);                 \
        kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);                \
        MCE_CUDA(cudaGetLastError());                                              \
    } while (0)

// ------------------------------------------------------------------ scratch

// Every device allocation of the library goes through this call, so that a
// host-side test hook (mce_debug_fail_alloc) can make one of them fail.
mce_status dev_alloc(void **p, size_t bytes, cudaStream_t s, const char *what);

// Stream-ordered device buffer freed at scope exit.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaStream_t s = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFreeAsync(p, s);
        p = nullptr;
        bytes = 0;
    }
    mce_status alloc(size_t nbytes, cudaStream_t stream) {
        release();
        s = stream;
        bytes = nbytes;
        if (nbytes == 0) nbytes = 16;
        return dev_alloc(&p, nbytes, stream, "cudaMallocAsync");
    }
    template <class T> T *as() const { return reinterpret_cast<T *>(p); }
};

// ------------------------------------------------------------------ graph

}  // namespace mce

struct mce_graph {
    int32_t n = 0;
    int64_t nnz = 0;
    int32_t *row_ptr = nullptr;  // int32[n+1], device
    int32_t *col = nullptr;      // int32[nnz], device, sorted per row
    int32_t id_bits = 1;         // bits needed for a vertex id
};

namespace mce {

// bits needed to represent values in [0, x]
inline int32_t bits_for(uint64_t x) {
    int32_t b = 1;
    while (b < 64 && (x >> b) != 0) ++b;
    return b;
}

inline int32_t num_sms() {
    static int32_t cached = -1;
    if (cached < 0) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached = v > 0 ? v : 1;
    }
    return cached;
}

inline unsigned grid_for(int64_t work, int32_t per_block) {
    int64_t g = (work + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > (int64_t)num_sms() * 64) g = (int64_t)num_sms() * 64;
    return (unsigned)g;
}

// ------------------------------------------------------------------ primitives (prims.cu)

// Exclusive prefix sum of in[0..n) into out[0..n]; out[n] = total.  In-place
// (in == out) is allowed.
mce_status exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s);
mce_status exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s);
// Ascending LSD radix sort of uint64 keys on their low `bits` bits (higher
// bits must be zero).  keys is sorted in place; tmp has n entries.
mce_status radix_sort_u64(uint64_t *keys, uint64_t *tmp, int64_t n, int32_t bits, cudaStream_t s);

// ------------------------------------------------------------------ graph kernels (graph.cu)

// CSR of the simple graph behind m pairs (device arrays).
mce_status build_csr(const int32_t *u, const int32_t *v, int64_t m, int32_t n, cudaStream_t s, mce_graph *g);
// Per-vertex keys (int64[n]).
mce_status vertex_key(const mce_graph *g, int32_t kind, cudaStream_t s, int64_t *key);
// rank[v] = position of (key[v], v); key values < 2^(64 - id_bits).
mce_status rank_from_key_i64(const int64_t *key, int32_t n, int32_t id_bits, cudaStream_t s, int32_t *rank);
// Same for float keys (higher float = higher rank; NaN not allowed).
mce_status rank_from_key_f32(const float *key, int32_t n, int32_t id_bits, cudaStream_t s, int32_t *rank);
// Higher-ranked neighbour lists: up_ptr int32[n+1], up_col int32[...] (sorted by id).
mce_status build_up_lists(const mce_graph *g, const int32_t *rank, cudaStream_t s, DevBuf &up_ptr, DevBuf &up_col,
                          int64_t *up_nnz);
// Features (mce_features).
mce_status features(const mce_graph *g, int32_t kind, cudaStream_t s, float *feat);
int32_t model_feature_kind(const mce_model *m);

// ------------------------------------------------------------------ device helpers

__device__ __forceinline__ uint64_t fmix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ULL;

// h(v) = splitmix64(v xor seed)
__device__ __forceinline__ uint64_t vertex_hash(int32_t v, uint64_t seed) {
    return fmix64(((uint64_t)(uint32_t)v ^ seed) + kGolden);
}

// H(K) from sum_{v in K} h(v) and |K|
__device__ __forceinline__ uint64_t clique_hash_from_sum(uint64_t hsum, uint32_t size) {
    return fmix64(hsum + (uint64_t)size * kGolden);
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

}  // namespace mce
