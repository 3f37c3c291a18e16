// Device primitives: exclusive prefix sums and a stable LSD radix sort.
#include "internal.cuh"

namespace mce {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// Block-wide exclusive scan of one value per thread; returns the block total.
template <class T>
__device__ T block_exclusive_scan(T x, T *warp_sums, T &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        T ws = lane < (kScanThreads / 32) ? warp_sums[lane] : T(0);
        T wi = ws;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < (kScanThreads / 32)) warp_sums[lane] = wi - ws;
        if (lane == (kScanThreads / 32) - 1) warp_sums[kScanThreads / 32] = wi;
    }
    __syncthreads();
    T r = warp_sums[warp] + incl - x;
    total = warp_sums[kScanThreads / 32];
    __syncthreads();
    return r;
}

template <class T>
__global__ void k_scan_reduce(const T *in, int64_t n, T *block_sums) {
    __shared__ T ws[kScanThreads / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) s += in[base + i];
    T total;
    block_exclusive_scan<T>(s, ws, total);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

template <class T>
__global__ void k_scan_apply(const T *in, T *out, int64_t n, const T *block_offsets) {
    __shared__ T ws[kScanThreads / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T v[kScanItems];
    T s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? in[base + i] : T(0);
        s += v[i];
    }
    T total;
    T run = block_exclusive_scan<T>(s, ws, total) + (block_offsets ? block_offsets[blockIdx.x] : T(0));
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanThreads - 1) out[n] = run;
}

template <class T>
mce_status exclusive_scan(const T *in, T *out, int64_t n, cudaStream_t s) {
    if (n <= 0) {
        return cuda_status(cudaMemsetAsync(out, 0, sizeof(T), s), "scan memset");
    }
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 1) {
        MCE_LAUNCH(k_scan_apply<T>, 1, kScanThreads, 0, s, in, out, n, (const T *)nullptr);
        return MCE_OK;
    }
    DevBuf sums;
    MCE_TRY(sums.alloc((size_t)(tiles + 1) * sizeof(T), s));
    MCE_LAUNCH(k_scan_reduce<T>, (unsigned)tiles, kScanThreads, 0, s, in, n, sums.as<T>());
    MCE_TRY(exclusive_scan<T>(sums.as<T>(), sums.as<T>(), tiles, s));
    MCE_LAUNCH(k_scan_apply<T>, (unsigned)tiles, kScanThreads, 0, s, in, out, n, (const T *)sums.as<T>());
    return MCE_OK;
}

// ------------------------------------------------------------------ radix sort

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kRadix = 256;

// counts[d * tiles + t] = keys of tile t whose digit is d
__global__ void k_radix_hist(const uint64_t *keys, int64_t n, int shift, int32_t *counts, int32_t tiles) {
    __shared__ int32_t h[kRadix];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll 4
    for (int r = 0; r < kSortItems; ++r) {
        int64_t i = base + (int64_t)r * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & (kRadix - 1)], 1);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter.  Items of a tile are visited in index order: round r covers
// [r*256, r*256+256), and inside a round warps then lanes go in order.  A
// digit's position = tile offset (from the scanned histogram) + items of the
// same digit in earlier rounds + in earlier warps of this round + in earlier
// lanes of this warp (match_any gives the lanes holding the same digit).
__global__ void k_radix_scatter(const uint64_t *in, uint64_t *out, int64_t n, int shift, const int32_t *offsets,
                                int32_t tiles) {
    constexpr int W = kSortThreads / 32;
    __shared__ int32_t base[kRadix];
    __shared__ int32_t wcnt[W][kRadix];
    const int tid = threadIdx.x, warp = tid >> 5;
    base[tid] = offsets[(int64_t)tid * tiles + blockIdx.x];
    const int64_t tile0 = (int64_t)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortItems; ++r) {
#pragma unroll
        for (int j = 0; j < W; ++j) wcnt[j][tid] = 0;
        __syncthreads();
        const int64_t i = tile0 + (int64_t)r * kSortThreads + tid;
        const bool valid = i < n;
        const uint64_t key = valid ? in[i] : 0;
        const uint32_t digit = valid ? (uint32_t)((key >> shift) & (kRadix - 1)) : kRadix;
        const uint32_t peers = __match_any_sync(0xffffffffu, digit);
        const int rank = __popc(peers & lanemask_lt());
        if (valid && rank == 0) wcnt[warp][digit] = __popc(peers);
        __syncthreads();
        {
            int32_t run = base[tid];
#pragma unroll
            for (int j = 0; j < W; ++j) {
                int32_t c = wcnt[j][tid];
                wcnt[j][tid] = run;
                run += c;
            }
            base[tid] = run;
        }
        __syncthreads();
        if (valid) out[wcnt[warp][digit] + rank] = key;
        __syncthreads();
    }
}

}  // namespace

mce_status exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s) {
    return exclusive_scan<int32_t>(in, out, n, s);
}

mce_status exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s) {
    return exclusive_scan<int64_t>(in, out, n, s);
}

mce_status radix_sort_u64(uint64_t *keys, uint64_t *tmp, int64_t n, int32_t bits, cudaStream_t s) {
    if (n <= 1) return MCE_OK;
    if (n >= (int64_t)1 << 31) {
        g_last_error = "radix_sort_u64: too many keys";
        return MCE_EINVAL;
    }
    const int32_t tiles = (int32_t)((n + kSortTile - 1) / kSortTile);
    DevBuf counts;
    MCE_TRY(counts.alloc((size_t)kRadix * tiles * sizeof(int32_t) + sizeof(int32_t), s));
    uint64_t *src = keys, *dst = tmp;
    int passes = 0;
    for (int shift = 0; shift < bits; shift += 8, ++passes) {
        MCE_LAUNCH(k_radix_hist, tiles, kSortThreads, 0, s, src, n, shift, counts.as<int32_t>(), tiles);
        MCE_TRY(exclusive_scan_i32(counts.as<int32_t>(), counts.as<int32_t>(), (int64_t)kRadix * tiles, s));
        MCE_LAUNCH(k_radix_scatter, tiles, kSortThreads, 0, s, src, dst, n, shift, counts.as<int32_t>(), tiles);
        uint64_t *t = src;
        src = dst;
        dst = t;
    }
    if (src != keys) MCE_CUDA(cudaMemcpyAsync(keys, src, (size_t)n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    return MCE_OK;
}

}  // namespace mce
