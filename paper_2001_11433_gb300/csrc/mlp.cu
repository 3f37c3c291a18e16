// Learned cost model for the vertex rank.
//
// Section 4.2 ranks vertices by a cheap estimate of the cost of their
// subproblem, giving costlier subproblems a higher rank so that they keep a
// smaller share of the cliques (the load-balancing idea taken from PECO).
// Here the estimate is learned: an MLP 8 -> H -> H -> 1 (ReLU) over
// per-vertex features predicts log(1 + search-tree nodes) of the vertex's
// subproblem, trained on node counts recorded by the search itself.
//
//   k_features    per-vertex features (warp per vertex)
//   k_mlp_fwd     inference, FP32 or BF16 weights/activations (FP32 accumulate)
//   k_mlp_grad    forward + backward of the MSE loss over a tile of rows;
//                 weight gradients reduced over the tile in shared memory
//   k_adam        Adam update
#include <cuda_bf16.h>
#include <string.h>

#include <vector>

#include "mce_host.h"

struct mce_model {
    int32_t H = 64;
    int32_t feature_kind = 0;   // MCE_FEATURES_* the model reads
    int64_t np = 0;
    float *w = nullptr;       // parameters, device
    float *m = nullptr;       // Adam first moment
    float *v = nullptr;       // Adam second moment
    float *g = nullptr;       // gradient
    int64_t step = 0;
};

namespace mce {

namespace {

constexpr int kFeat = 8;
constexpr int kMaxH = 64;
constexpr int kRowsPerBlock = 128;

struct Off {
    int64_t W1, b1, W2, b2, w3, b3, n;
};

__host__ __device__ inline Off offsets(int H) {
    Off o;
    o.W1 = 0;
    o.b1 = o.W1 + (int64_t)H * kFeat;
    o.W2 = o.b1 + H;
    o.b2 = o.W2 + (int64_t)H * H;
    o.w3 = o.b2 + H;
    o.b3 = o.w3 + H;
    o.n = o.b3 + 1;
    return o;
}

// ------------------------------------------------------------------ features

__global__ void k_features(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                           const int64_t *__restrict__ core, const int64_t *__restrict__ tri,
                           const int32_t *__restrict__ up_ptr, int32_t n, float *feat) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < n; v += nwarps) {
        const int32_t e0 = row_ptr[v], e1 = row_ptr[v + 1], d = e1 - e0;
        float s = 0.f, s2 = 0.f, mx = 0.f;
        for (int32_t e = e0 + lane; e < e1; e += 32) {
            const int32_t w = col[e];
            const float x = log1pf((float)(row_ptr[w + 1] - row_ptr[w]));
            s += x;
            s2 += x * x;
            mx = fmaxf(mx, x);
        }
        for (int o = 16; o; o >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        if (lane == 0) {
            float *f = feat + v * kFeat;
            const float mean = d ? s / d : 0.f;
            const float var = d ? fmaxf(s2 / d - mean * mean, 0.f) : 0.f;
            f[0] = log1pf((float)d);
            f[1] = (float)core[v];
            f[2] = log1pf((float)tri[v]);
            f[3] = mean;
            f[4] = sqrtf(var);
            f[5] = mx;
            f[6] = log1pf((float)(up_ptr[v + 1] - up_ptr[v]));
            f[7] = d >= 2 ? (float)(2.0 * (double)tri[v] / ((double)d * (d - 1))) : 0.f;
        }
    }
}

// One-pass features (MCE_FEATURES_LIGHT): degrees of the vertex and its
// neighbours only.  A neighbour w ranks higher than v by degree when
// (d(w), w) > (d(v), v).
__global__ void k_features_light(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col, int32_t n,
                                 float *feat) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < n; v += nwarps) {
        const int32_t e0 = row_ptr[v], e1 = row_ptr[v + 1], d = e1 - e0;
        float s = 0.f, s2 = 0.f, mx = 0.f, mins = 0.f, dsum = 0.f;
        int hi = 0;
        for (int32_t e = e0 + lane; e < e1; e += 32) {
            const int32_t w = col[e];
            const int32_t dw = row_ptr[w + 1] - row_ptr[w];
            const float x = log1pf((float)dw);
            s += x;
            s2 += x * x;
            mx = fmaxf(mx, x);
            mins += (float)min(dw, d);
            dsum += (float)dw;
            hi += (dw > d || (dw == d && w > (int32_t)v)) ? 1 : 0;
        }
        for (int o = 16; o; o >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            mins += __shfl_xor_sync(0xffffffffu, mins, o);
            dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
            hi += __shfl_xor_sync(0xffffffffu, hi, o);
        }
        if (lane == 0) {
            float *f = feat + v * kFeat;
            const float mean = d ? s / d : 0.f;
            const float var = d ? fmaxf(s2 / d - mean * mean, 0.f) : 0.f;
            f[0] = log1pf((float)d);
            f[1] = mean;
            f[2] = sqrtf(var);
            f[3] = mx;
            f[4] = log1pf((float)hi);
            f[5] = log1pf(mins * 0.5f);
            f[6] = d ? (float)hi / (float)d : 0.f;
            f[7] = log1pf(dsum);
        }
    }
}

// ------------------------------------------------------------------ MLP

// One thread per row.  HC > 0 fixes the hidden width at compile time, so
// that the hidden activations stay in registers and the weight rows are read
// from shared memory four at a time (same operations in the same order as
// the generic path, HC = 0).
template <bool BF16, int HC>
__global__ void k_mlp_fwd(const float *__restrict__ wts, int H_rt, const float *__restrict__ feat, int32_t rows,
                          float *out) {
    extern __shared__ __align__(16) float sw[];
    const int H = HC > 0 ? HC : H_rt;
    const Off o = offsets(H);
    for (int64_t i = threadIdx.x; i < o.n; i += blockDim.x) {
        float w = wts[i];
        if (BF16) w = __bfloat162float(__float2bfloat16(w));
        sw[i] = w;
    }
    __syncthreads();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
        float x[kFeat];
#pragma unroll
        for (int k = 0; k < kFeat; ++k) {
            float t = feat[r * kFeat + k];
            if (BF16) t = __bfloat162float(__float2bfloat16(t));
            x[k] = t;
        }
        float h1[kMaxH];
        float y = sw[o.b3];
        if constexpr (HC > 0) {
            static_assert(HC % 4 == 0 && HC <= kMaxH, "fixed hidden width");
            // weights are read per row, not held in registers across rows
            asm volatile("" ::: "memory");
#pragma unroll
            for (int j = 0; j < HC; ++j) {
                float a = sw[o.b1 + j];
#pragma unroll
                for (int k = 0; k < kFeat; ++k) a = fmaf(sw[o.W1 + j * kFeat + k], x[k], a);
                a = fmaxf(a, 0.f);
                if (BF16) a = __bfloat162float(__float2bfloat16(a));
                h1[j] = a;
            }
#pragma unroll 1
            for (int j = 0; j < HC; ++j) {
                float a = sw[o.b2 + j];
                const float4 *wr = reinterpret_cast<const float4 *>(sw + o.W2 + j * HC);
#pragma unroll
                for (int i = 0; i < HC / 4; ++i) {
                    const float4 w = wr[i];
                    a = fmaf(w.x, h1[4 * i], a);
                    a = fmaf(w.y, h1[4 * i + 1], a);
                    a = fmaf(w.z, h1[4 * i + 2], a);
                    a = fmaf(w.w, h1[4 * i + 3], a);
                }
                a = fmaxf(a, 0.f);
                if (BF16) a = __bfloat162float(__float2bfloat16(a));
                y = fmaf(sw[o.w3 + j], a, y);
            }
        } else {
#pragma unroll 4
            for (int j = 0; j < H; ++j) {
                float a = sw[o.b1 + j];
#pragma unroll
                for (int k = 0; k < kFeat; ++k) a = fmaf(sw[o.W1 + j * kFeat + k], x[k], a);
                a = fmaxf(a, 0.f);
                if (BF16) a = __bfloat162float(__float2bfloat16(a));
                h1[j] = a;
            }
            for (int j = 0; j < H; ++j) {
                float a = sw[o.b2 + j];
                const float *wr = sw + o.W2 + (int64_t)j * H;
#pragma unroll 8
                for (int i = 0; i < H; ++i) a = fmaf(wr[i], h1[i], a);
                a = fmaxf(a, 0.f);
                if (BF16) a = __bfloat162float(__float2bfloat16(a));
                y = fmaf(sw[o.w3 + j], a, y);
            }
        }
        out[r] = y;
    }
}

// Forward + backward over rows idx[r0 .. r0 + cnt) (or r0.. when idx is null),
// loss = (1/N) sum (y - t)^2.  One thread per row, kRowsPerBlock rows per block.
__global__ void __launch_bounds__(kRowsPerBlock) k_mlp_grad(const float *__restrict__ wts, int H,
                                                            const float *__restrict__ feat,
                                                            const float *__restrict__ label,
                                                            const int32_t *__restrict__ idx, int64_t r0, int64_t cnt,
                                                            float inv_n, float *grad, float *loss) {
    extern __shared__ float sm[];
    const Off o = offsets(H);
    float *sw = sm;                                // weights
    float *sx = sw + ((o.n + 3) & ~3LL);           // x   [rows][8]
    float *sh1 = sx + kRowsPerBlock * kFeat;       // h1  [rows][H]
    float *sd2 = sh1 + kRowsPerBlock * H;          // dh2 [rows][H]
    float *sd1 = sd2 + kRowsPerBlock * H;          // dh1 [rows][H]
    for (int64_t i = threadIdx.x; i < o.n; i += blockDim.x) sw[i] = wts[i];
    const int t = threadIdx.x;
    const int64_t rr = (int64_t)blockIdx.x * kRowsPerBlock + t;
    const bool valid = rr < cnt;
    const int64_t row = valid ? (idx ? idx[r0 + rr] : r0 + rr) : 0;
    for (int k = 0; k < kFeat; ++k) sx[t * kFeat + k] = valid ? feat[row * kFeat + k] : 0.f;
    __syncthreads();
    // forward
    for (int j = 0; j < H; ++j) {
        float a = sw[o.b1 + j];
        for (int k = 0; k < kFeat; ++k) a = fmaf(sw[o.W1 + j * kFeat + k], sx[t * kFeat + k], a);
        sh1[t * H + j] = fmaxf(a, 0.f);
    }
    float y = sw[o.b3];
    for (int j = 0; j < H; ++j) {
        float a = sw[o.b2 + j];
        for (int i = 0; i < H; ++i) a = fmaf(sw[o.W2 + (int64_t)j * H + i], sh1[t * H + i], a);
        const float h2 = fmaxf(a, 0.f);
        sd2[t * H + j] = h2;   // h2 for now; replaced by dh2 below
        y = fmaf(sw[o.w3 + j], h2, y);
    }
    const float err = valid ? (y - label[row]) : 0.f;
    const float dy = 2.f * err * inv_n;
    // loss
    {
        float l = err * err * inv_n;
        for (int of = 16; of; of >>= 1) l += __shfl_xor_sync(0xffffffffu, l, of);
        if ((t & 31) == 0 && l != 0.f) atomicAdd(loss, l);
    }
    // dh2 (and w3/b3 gradients need h2: accumulate per thread into shared later)
    __syncthreads();
    // dw3[j] = sum_r dy_r h2_r[j]; each thread j < H sums over rows
    __shared__ float sdy[kRowsPerBlock];
    sdy[t] = dy;
    __syncthreads();
    for (int j = t; j < H; j += blockDim.x) {
        float a = 0.f;
        for (int r = 0; r < kRowsPerBlock; ++r) a = fmaf(sdy[r], sd2[r * H + j], a);
        atomicAdd(&grad[o.w3 + j], a);
    }
    if (t == 0) {
        float a = 0.f;
        for (int r = 0; r < kRowsPerBlock; ++r) a += sdy[r];
        atomicAdd(&grad[o.b3], a);
    }
    __syncthreads();
    for (int j = 0; j < H; ++j) {
        const float h2 = sd2[t * H + j];
        sd2[t * H + j] = h2 > 0.f ? dy * sw[o.w3 + j] : 0.f;
    }
    // dh1[i] = sum_j W2[j][i] dh2[j], masked by h1 > 0
    for (int i = 0; i < H; ++i) {
        float a = 0.f;
        for (int j = 0; j < H; ++j) a = fmaf(sw[o.W2 + (int64_t)j * H + i], sd2[t * H + j], a);
        sd1[t * H + i] = sh1[t * H + i] > 0.f ? a : 0.f;
    }
    __syncthreads();
    // dW2[j][i] = sum_r dh2[r][j] h1[r][i]; db2[j] = sum_r dh2[r][j]
    for (int64_t e = t; e < (int64_t)H * H; e += blockDim.x) {
        const int j = (int)(e / H), i = (int)(e % H);
        float a = 0.f;
        for (int r = 0; r < kRowsPerBlock; ++r) a = fmaf(sd2[r * H + j], sh1[r * H + i], a);
        atomicAdd(&grad[o.W2 + e], a);
    }
    // dW1[i][k] = sum_r dh1[r][i] x[r][k]; db1, db2
    for (int64_t e = t; e < (int64_t)H * kFeat; e += blockDim.x) {
        const int i = (int)(e / kFeat), k = (int)(e % kFeat);
        float a = 0.f;
        for (int r = 0; r < kRowsPerBlock; ++r) a = fmaf(sd1[r * H + i], sx[r * kFeat + k], a);
        atomicAdd(&grad[o.W1 + e], a);
    }
    for (int j = t; j < H; j += blockDim.x) {
        float a = 0.f, b = 0.f;
        for (int r = 0; r < kRowsPerBlock; ++r) {
            a += sd1[r * H + j];
            b += sd2[r * H + j];
        }
        atomicAdd(&grad[o.b1 + j], a);
        atomicAdd(&grad[o.b2 + j], b);
    }
}

__global__ void k_adam(float *w, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// permutation keys: hash of (seed, i) in the high bits, i in the low bits
__global__ void k_perm_keys(int32_t n, uint64_t seed, int32_t idb, uint64_t *keys) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = ((fmix64(seed ^ ((uint64_t)i * kGolden)) >> idb) << idb) | (uint64_t)i;
}

__global__ void k_keys_to_idx(const uint64_t *keys, int32_t n, int32_t idb, int32_t *idx) {
    const uint64_t mask = (1ULL << idb) - 1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        idx[i] = (int32_t)(keys[i] & mask);
}

size_t grad_smem(int H) {
    const Off o = offsets(H);
    return (size_t)(((o.n + 3) & ~3LL) + kRowsPerBlock * kFeat + 3 * kRowsPerBlock * H) * 4;
}

}  // namespace

int32_t model_feature_kind(const mce_model *m) { return m ? m->feature_kind : 0; }

mce_status features(const mce_graph *g, int32_t kind, cudaStream_t s, float *feat) {
    const int32_t n = g->n;
    if (n == 0) return MCE_OK;
    if (kind == MCE_FEATURES_LIGHT) {
        MCE_LAUNCH(k_features_light, grid_for((int64_t)n * 32, 256), 256, 0, s, g->row_ptr, g->col, n, feat);
        return MCE_OK;
    }
    DevBuf core, tri, deg, drank, up_ptr, up_col;
    MCE_TRY(core.alloc((size_t)n * 8, s));
    MCE_TRY(tri.alloc((size_t)n * 8, s));
    MCE_TRY(deg.alloc((size_t)n * 8, s));
    MCE_TRY(drank.alloc((size_t)n * 4, s));
    MCE_TRY(vertex_key(g, MCE_RANK_DEGEN, s, core.as<int64_t>()));
    MCE_TRY(vertex_key(g, MCE_RANK_TRIANGLE, s, tri.as<int64_t>()));
    MCE_TRY(vertex_key(g, MCE_RANK_DEGREE, s, deg.as<int64_t>()));
    MCE_TRY(rank_from_key_i64(deg.as<int64_t>(), n, g->id_bits, s, drank.as<int32_t>()));
    int64_t nnz = 0;
    MCE_TRY(build_up_lists(g, drank.as<int32_t>(), s, up_ptr, up_col, &nnz));
    MCE_LAUNCH(k_features, grid_for((int64_t)n * 32, 256), 256, 0, s, g->row_ptr, g->col, core.as<int64_t>(),
               tri.as<int64_t>(), up_ptr.as<int32_t>(), n, feat);
    return MCE_OK;
}

mce_status model_predict(const mce_model *m, const float *feat, int32_t rows, int32_t bf16, cudaStream_t s,
                         float *out) {
    if (rows <= 0) return MCE_OK;
    const size_t smem = (size_t)offsets(m->H).n * 4;
    // the default width has its own compiled kernel
    void (*kf)(const float *, int, const float *, int32_t, float *) =
        m->H == kMaxH ? (bf16 ? k_mlp_fwd<true, kMaxH> : k_mlp_fwd<false, kMaxH>)
                      : (bf16 ? k_mlp_fwd<true, 0> : k_mlp_fwd<false, 0>);
    MCE_CUDA(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    MCE_LAUNCH(kf, grid_for(rows, 128), 128, smem, s, m->w, m->H, feat, rows, out);
    return MCE_OK;
}

static mce_status grad_launch(const mce_model *m, const float *feat, const float *label, const int32_t *idx,
                              int64_t r0, int64_t cnt, float inv_n, float *loss, cudaStream_t s) {
    const size_t smem = grad_smem(m->H);
    MCE_CUDA(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const unsigned blocks = (unsigned)((cnt + kRowsPerBlock - 1) / kRowsPerBlock);
    MCE_LAUNCH(k_mlp_grad, blocks, kRowsPerBlock, smem, s, m->w, m->H, feat, label, idx, r0, cnt, inv_n, m->g, loss);
    return MCE_OK;
}

}  // namespace mce

using namespace mce;

extern "C" {

mce_status mce_features(const mce_graph *g, void *stream, float *feat) {
    return mce_features_kind(g, MCE_FEATURES_FULL, stream, feat);
}

mce_status mce_features_kind(const mce_graph *g, int32_t kind, void *stream, float *feat) {
    if (!g || !feat || (kind != MCE_FEATURES_FULL && kind != MCE_FEATURES_LIGHT)) {
        g_last_error = "mce_features_kind: bad arguments";
        return MCE_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    MCE_TRY(features(g, kind, s, feat));
    MCE_CUDA(cudaStreamSynchronize(s));
    return MCE_OK;
}

mce_status mce_model_set_features(mce_model *m, int32_t kind) {
    if (!m || (kind != MCE_FEATURES_FULL && kind != MCE_FEATURES_LIGHT)) {
        g_last_error = "mce_model_set_features: bad arguments";
        return MCE_EINVAL;
    }
    m->feature_kind = kind;
    return MCE_OK;
}

mce_status mce_model_create(int32_t hidden, uint64_t seed, mce_model **out) {
    if (!out || hidden < 1 || hidden > kMaxH) {
        g_last_error = "mce_model_create: hidden must be in [1, 64]";
        return MCE_EINVAL;
    }
    mce_model *m = new mce_model();
    m->H = hidden;
    const Off o = offsets(hidden);
    m->np = o.n;
    std::vector<float> h((size_t)o.n, 0.f);
    // He-style uniform initialisation from a splitmix64 stream
    uint64_t st = seed;
    auto next = [&]() {
        uint64_t z = (st += 0x9E3779B97F4A7C15ULL);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        z ^= z >> 31;
        return (double)(z >> 11) * 0x1.0p-53 * 2.0 - 1.0;
    };
    for (int64_t i = 0; i < (int64_t)hidden * kFeat; ++i) h[o.W1 + i] = (float)(next() * sqrt(6.0 / kFeat));
    for (int64_t i = 0; i < (int64_t)hidden * hidden; ++i) h[o.W2 + i] = (float)(next() * sqrt(6.0 / hidden));
    for (int64_t i = 0; i < hidden; ++i) h[o.w3 + i] = (float)(next() * sqrt(3.0 / hidden));
    for (int64_t i = 0; i < hidden; ++i) {
        h[o.b1 + i] = 0.01f;
        h[o.b2 + i] = 0.01f;
    }
    mce_status st2 = MCE_OK;
    const size_t bytes = (size_t)o.n * 4;
    st2 = cuda_status(cudaMalloc(&m->w, bytes), "model alloc");
    if (st2 == MCE_OK) st2 = cuda_status(cudaMalloc(&m->m, bytes), "model alloc");
    if (st2 == MCE_OK) st2 = cuda_status(cudaMalloc(&m->v, bytes), "model alloc");
    if (st2 == MCE_OK) st2 = cuda_status(cudaMalloc(&m->g, bytes), "model alloc");
    if (st2 == MCE_OK) st2 = cuda_status(cudaMemcpy(m->w, h.data(), bytes, cudaMemcpyHostToDevice), "model init");
    if (st2 == MCE_OK) st2 = cuda_status(cudaMemset(m->m, 0, bytes), "model init");
    if (st2 == MCE_OK) st2 = cuda_status(cudaMemset(m->v, 0, bytes), "model init");
    if (st2 != MCE_OK) {
        mce_model_free(m);
        return st2;
    }
    *out = m;
    return MCE_OK;
}

void mce_model_free(mce_model *m) {
    if (!m) return;
    cudaDeviceSynchronize();
    cudaFree(m->w);
    cudaFree(m->m);
    cudaFree(m->v);
    cudaFree(m->g);
    delete m;
}

int64_t mce_model_num_params(const mce_model *m) { return m ? m->np : 0; }

mce_status mce_model_get(const mce_model *m, float *host) {
    if (!m || !host) return MCE_EINVAL;
    MCE_CUDA(cudaMemcpy(host, m->w, (size_t)m->np * 4, cudaMemcpyDeviceToHost));
    return MCE_OK;
}

mce_status mce_model_set(mce_model *m, const float *host) {
    if (!m || !host) return MCE_EINVAL;
    MCE_CUDA(cudaMemcpy(m->w, host, (size_t)m->np * 4, cudaMemcpyHostToDevice));
    return MCE_OK;
}

mce_status mce_model_loss_grad(const mce_model *m, const float *feat, const float *label, int32_t rows, void *stream,
                               float *loss, float *host_grad) {
    if (!m || !feat || !label || rows <= 0) return MCE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    DevBuf dl;
    MCE_TRY(dl.alloc(4, s));
    MCE_CUDA(cudaMemsetAsync(dl.p, 0, 4, s));
    MCE_CUDA(cudaMemsetAsync(m->g, 0, (size_t)m->np * 4, s));
    MCE_TRY(grad_launch(m, feat, label, nullptr, 0, rows, 1.f / rows, dl.as<float>(), s));
    if (loss) MCE_CUDA(cudaMemcpyAsync(loss, dl.p, 4, cudaMemcpyDeviceToHost, s));
    if (host_grad) MCE_CUDA(cudaMemcpyAsync(host_grad, m->g, (size_t)m->np * 4, cudaMemcpyDeviceToHost, s));
    MCE_CUDA(cudaStreamSynchronize(s));
    return MCE_OK;
}

mce_status mce_model_train(mce_model *m, const float *feat, const float *label, int32_t rows, int32_t epochs,
                           int32_t batch, float lr, uint64_t seed, void *stream, float *loss_out) {
    if (!m || !feat || !label || rows <= 0 || epochs < 0 || batch <= 0) return MCE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t idb = bits_for((uint64_t)rows);
    DevBuf keys, tmp, idx, dl;
    MCE_TRY(keys.alloc((size_t)rows * 8, s));
    MCE_TRY(tmp.alloc((size_t)rows * 8, s));
    MCE_TRY(idx.alloc((size_t)rows * 4, s));
    MCE_TRY(dl.alloc((size_t)(epochs + 1) * 4, s));
    MCE_CUDA(cudaMemsetAsync(dl.p, 0, (size_t)(epochs + 1) * 4, s));
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int32_t ep = 0; ep < epochs; ++ep) {
        MCE_LAUNCH(k_perm_keys, grid_for(rows, 256), 256, 0, s, rows, seed + (uint64_t)ep * 7919, idb,
                   keys.as<uint64_t>());
        MCE_TRY(radix_sort_u64(keys.as<uint64_t>(), tmp.as<uint64_t>(), rows, 64, s));
        MCE_LAUNCH(k_keys_to_idx, grid_for(rows, 256), 256, 0, s, keys.as<uint64_t>(), rows, idb, idx.as<int32_t>());
        for (int64_t r0 = 0; r0 < rows; r0 += batch) {
            const int64_t cnt = (r0 + batch <= rows) ? batch : rows - r0;
            MCE_CUDA(cudaMemsetAsync(m->g, 0, (size_t)m->np * 4, s));
            // per-batch mean for the gradient; the epoch loss is the mean over rows
            MCE_TRY(grad_launch(m, feat, label, idx.as<int32_t>(), r0, cnt, 1.f / (float)cnt,
                                dl.as<float>() + ep, s));
            m->step++;
            const float c1 = 1.f - powf(b1, (float)m->step), c2 = 1.f - powf(b2, (float)m->step);
            MCE_LAUNCH(k_adam, grid_for(m->np, 256), 256, 0, s, m->w, m->g, m->m, m->v, m->np, lr, b1, b2, eps, c1,
                       c2);
        }
    }
    std::vector<float> hl((size_t)epochs + 1);
    MCE_CUDA(cudaMemcpyAsync(hl.data(), dl.p, (size_t)(epochs + 1) * 4, cudaMemcpyDeviceToHost, s));
    MCE_CUDA(cudaStreamSynchronize(s));
    if (loss_out && epochs > 0) {
        // each batch added (mean batch loss); divide by the number of batches
        const int64_t nb = (rows + batch - 1) / batch;
        *loss_out = hl[epochs - 1] / (float)nb;
    }
    return MCE_OK;
}

mce_status mce_model_predict(const mce_model *m, const float *feat, int32_t rows, int32_t bf16, void *stream,
                             float *out) {
    if (!m || !feat || !out || rows < 0) return MCE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    MCE_TRY(model_predict(m, feat, rows, bf16, s, out));
    MCE_CUDA(cudaStreamSynchronize(s));
    return MCE_OK;
}

}  // extern "C"
