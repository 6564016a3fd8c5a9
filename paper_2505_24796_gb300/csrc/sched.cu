// sched.cu -- the learned tile-cost model that orders the batched renderer's work queue.
//
// Not part of the paper: TC-GS accelerates each tile's alpha-blending; a multi-view batch still
// finishes with its most expensive tiles, whose cost (list entries walked until every pixel has
// terminated) is not the list length.  A small MLP (8 -> 32 -> 32 -> 1, FP16 weights and
// activations, FP32 accumulation) predicts log(tile cost) from cheap per-tile statistics; the
// queue is ordered longest-predicted first.  Its training data are the per-tile costs the
// renderer itself records (tile_stats).
//
// Kernels: per-tile features (one warp per tile), feature normaliser, MLP forward, MLP backward
// (mean squared error), Adam.  The ordering sort lives with the radix sort in binsort.cu.
#include "common.cuh"

namespace tcgs {
namespace {

constexpr int kIn = TCGS_MLP_IN, kHid = TCGS_MLP_HIDDEN;
// parameter layout (float32 masters): W1[kHid][kIn], b1[kHid], W2[kHid][kHid], b2[kHid], W3[kHid], b3
constexpr int kW1 = 0, kB1 = kW1 + kHid * kIn, kW2 = kB1 + kHid, kB2 = kW2 + kHid * kHid, kW3 = kB2 + kHid,
              kB3 = kW3 + kHid, kParams = kB3 + 1;
static_assert(kParams == TCGS_MLP_PARAMS, "parameter layout");

__device__ __forceinline__ float h16(float x) { return __half2float(__float2half_rn(x)); }

// ---------------------------------------------------------------- features

__global__ void __launch_bounds__(256) k_tile_features(DevCamera cam, const uint32_t* __restrict__ ranges,
                                                       const uint32_t* __restrict__ ids,
                                                       const float* __restrict__ mean2d,
                                                       const float* __restrict__ conic,
                                                       const float* __restrict__ opacity,
                                                       const float* __restrict__ depth,
                                                       const int32_t* __restrict__ radius, float* __restrict__ feat) {
    const int tiles = cam.grid_w * cam.grid_h;
    const int tile = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (tile >= tiles) return;
    const int tx = tile % cam.grid_w, ty = tile / cam.grid_w;
    const float x0 = (float)(kTile * tx), y0 = (float)(kTile * ty);
    const uint32_t start = ranges[2 * tile], end = ranges[2 * tile + 1];
    float so = 0.f, mo = 0.f, dmin = 3.0e38f, dmax = -3.0e38f, sdet = 0.f, cov = 0.f;
    for (uint32_t i = start + lane; i < end; i += 32) {
        const uint32_t g = ids[i];
        const float o = opacity[g];
        so += o;
        mo = fmaxf(mo, o);
        const float d = depth[g];
        dmin = fminf(dmin, d);
        dmax = fmaxf(dmax, d);
        const float a = conic[3 * g], b = conic[3 * g + 1], c = conic[3 * g + 2];
        sdet += __logf(fmaxf(a * c - b * b, 1e-30f));
        const float2 m = reinterpret_cast<const float2*>(mean2d)[g];
        const float r = (float)radius[g];
        const float ox = fmaxf(0.f, fminf(m.x + r, x0 + kTile) - fmaxf(m.x - r, x0));
        const float oy = fmaxf(0.f, fminf(m.y + r, y0 + kTile) - fmaxf(m.y - r, y0));
        cov += ox * oy * (1.f / (kTile * kTile));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        so += __shfl_xor_sync(0xffffffffu, so, o);
        mo = fmaxf(mo, __shfl_xor_sync(0xffffffffu, mo, o));
        dmin = fminf(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
        dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        sdet += __shfl_xor_sync(0xffffffffu, sdet, o);
        cov += __shfl_xor_sync(0xffffffffu, cov, o);
    }
    if (lane == 0) {
        const float n = (float)(end - start);
        const float inv = n > 0.f ? 1.f / n : 0.f;
        const int w_in = min(kTile, cam.width - kTile * tx), h_in = min(kTile, cam.height - kTile * ty);
        float* f = feat + (size_t)tile * kIn;
        f[0] = log1pf(n);
        f[1] = so * inv;
        f[2] = mo;
        f[3] = n > 0.f ? log1pf(dmax - dmin) : 0.f;
        f[4] = sdet * inv;
        f[5] = log1pf(cov);
        f[6] = logf((float)cam.width * (float)cam.height);
        f[7] = (float)(w_in * h_in) * (1.f / (kTile * kTile));
    }
}

// norm[0..7] = mean, norm[8..15] = 1 / max(std, 1e-6) of each feature column (FP64 sums)
__global__ void __launch_bounds__(1024) k_feature_norm(const float* __restrict__ x, int n, float* __restrict__ norm) {
    __shared__ double s1[kIn][32], s2[kIn][32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    double a[kIn], b[kIn];
#pragma unroll
    for (int k = 0; k < kIn; ++k) a[k] = b[k] = 0.0;
    for (int i = t; i < n; i += blockDim.x)
#pragma unroll
        for (int k = 0; k < kIn; ++k) {
            const double v = x[(size_t)i * kIn + k];
            a[k] += v;
            b[k] += v * v;
        }
#pragma unroll
    for (int k = 0; k < kIn; ++k) {
        for (int o = 16; o > 0; o >>= 1) {
            a[k] += __shfl_xor_sync(0xffffffffu, a[k], o);
            b[k] += __shfl_xor_sync(0xffffffffu, b[k], o);
        }
        if (lane == 0) { s1[k][warp] = a[k]; s2[k][warp] = b[k]; }
    }
    __syncthreads();
    if (t < kIn) {
        double A = 0.0, B = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) { A += s1[t][w]; B += s2[t][w]; }
        const double mean = n > 0 ? A / n : 0.0;
        const double var = n > 0 ? B / n - mean * mean : 0.0;
        const double sd = var > 1e-12 ? sqrt(var) : 1e-6;
        norm[t] = (float)mean;
        norm[kIn + t] = (float)(1.0 / sd);
    }
}

// ---------------------------------------------------------------- MLP

// weights rounded to FP16 into shared memory (as float), plus the normaliser
__device__ __forceinline__ void load_weights(const float* __restrict__ params, const float* __restrict__ norm,
                                             float* w, float* nm) {
    for (int i = threadIdx.x; i < kParams; i += blockDim.x) w[i] = h16(params[i]);
    for (int i = threadIdx.x; i < 2 * kIn; i += blockDim.x) nm[i] = norm[i];
}

// forward of one item; keeps the FP16-rounded input and hidden activations
__device__ __forceinline__ float mlp_forward(const float* w, const float* nm, const float* __restrict__ xi, float* xh,
                                             float* h1, float* h2) {
#pragma unroll
    for (int k = 0; k < kIn; ++k) xh[k] = h16((xi[k] - nm[k]) * nm[kIn + k]);
#pragma unroll
    for (int j = 0; j < kHid; ++j) {
        float acc = w[kB1 + j];
#pragma unroll
        for (int k = 0; k < kIn; ++k) acc = fmaf(w[kW1 + j * kIn + k], xh[k], acc);
        h1[j] = h16(fmaxf(acc, 0.f));
    }
#pragma unroll
    for (int j = 0; j < kHid; ++j) {
        float acc = w[kB2 + j];
#pragma unroll
        for (int k = 0; k < kHid; ++k) acc = fmaf(w[kW2 + j * kHid + k], h1[k], acc);
        h2[j] = h16(fmaxf(acc, 0.f));
    }
    float y = w[kB3];
#pragma unroll
    for (int k = 0; k < kHid; ++k) y = fmaf(w[kW3 + k], h2[k], y);
    return y;
}

__global__ void __launch_bounds__(128) k_mlp_fwd(const float* __restrict__ params, const float* __restrict__ norm,
                                                 const float* __restrict__ x, int n, float* __restrict__ y) {
    __shared__ float w[kParams], nm[2 * kIn];
    load_weights(params, norm, w, nm);
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float xh[kIn], h1[kHid], h2[kHid];
        y[i] = mlp_forward(w, nm, x + (size_t)i * kIn, xh, h1, h2);
    }
}

// Backward of L = (1/n) sum (y - t)^2 for a block of kBwdItems items: per item the deltas are
// formed in registers and kept in shared memory; the block then sums every parameter's gradient
// over its items (a small matrix product per layer) and adds it to `grad` with one atomic each.
constexpr int kBwdItems = 64;

__global__ void __launch_bounds__(kBwdItems) k_mlp_bwd(const float* __restrict__ params, const float* __restrict__ norm,
                                                       const float* __restrict__ x, const float* __restrict__ target,
                                                       int n, float* __restrict__ grad, float* __restrict__ loss) {
    __shared__ float w[kParams], nm[2 * kIn];
    __shared__ float s_xh[kBwdItems][kIn + 1], s_h1[kBwdItems][kHid + 1], s_h2[kBwdItems][kHid + 1];
    __shared__ float s_d1[kBwdItems][kHid + 1], s_d2[kBwdItems][kHid + 1], s_dy[kBwdItems];
    load_weights(params, norm, w, nm);
    __syncthreads();
    const int t = threadIdx.x;
    const int i = blockIdx.x * kBwdItems + t;
    float se = 0.f;
    if (i < n) {
        float xh[kIn], h1[kHid], h2[kHid];
        const float y = mlp_forward(w, nm, x + (size_t)i * kIn, xh, h1, h2);
        const float e = y - target[i];
        se = e * e;
        const float dy = 2.f * e / (float)n;
        float d2[kHid];
#pragma unroll
        for (int k = 0; k < kHid; ++k) d2[k] = h2[k] > 0.f ? dy * w[kW3 + k] : 0.f;
#pragma unroll
        for (int k = 0; k < kHid; ++k) {
            float acc = 0.f;
#pragma unroll
            for (int j = 0; j < kHid; ++j) acc = fmaf(w[kW2 + j * kHid + k], d2[j], acc);
            s_d1[t][k] = h1[k] > 0.f ? acc : 0.f;
        }
#pragma unroll
        for (int k = 0; k < kIn; ++k) s_xh[t][k] = xh[k];
#pragma unroll
        for (int k = 0; k < kHid; ++k) { s_h1[t][k] = h1[k]; s_h2[t][k] = h2[k]; s_d2[t][k] = d2[k]; }
        s_dy[t] = dy;
    } else {
#pragma unroll
        for (int k = 0; k < kIn; ++k) s_xh[t][k] = 0.f;
#pragma unroll
        for (int k = 0; k < kHid; ++k) { s_h1[t][k] = s_h2[t][k] = s_d1[t][k] = s_d2[t][k] = 0.f; }
        s_dy[t] = 0.f;
    }
    __syncthreads();
    const int items = min(kBwdItems, n - (int)blockIdx.x * kBwdItems);
    for (int q = t; q < kParams; q += kBwdItems) {
        float g = 0.f;
        if (q < kB1) {                 // W1[j][k] += d1[j] xh[k]
            const int j = (q - kW1) / kIn, k = (q - kW1) % kIn;
            for (int it = 0; it < items; ++it) g = fmaf(s_d1[it][j], s_xh[it][k], g);
        } else if (q < kW2) {          // b1[j] += d1[j]
            const int j = q - kB1;
            for (int it = 0; it < items; ++it) g += s_d1[it][j];
        } else if (q < kB2) {          // W2[j][k] += d2[j] h1[k]
            const int j = (q - kW2) / kHid, k = (q - kW2) % kHid;
            for (int it = 0; it < items; ++it) g = fmaf(s_d2[it][j], s_h1[it][k], g);
        } else if (q < kW3) {          // b2[j] += d2[j]
            const int j = q - kB2;
            for (int it = 0; it < items; ++it) g += s_d2[it][j];
        } else if (q < kB3) {          // W3[k] += dy h2[k]
            const int k = q - kW3;
            for (int it = 0; it < items; ++it) g = fmaf(s_dy[it], s_h2[it][k], g);
        } else {                       // b3 += dy
            for (int it = 0; it < items; ++it) g += s_dy[it];
        }
        atomicAdd(&grad[q], g);
    }
    if (loss) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
        if ((t & 31) == 0) atomicAdd(loss, se / (float)n);
    }
}

__global__ void k_adam(float* __restrict__ params, float* __restrict__ m, float* __restrict__ v,
                       float* __restrict__ grad, int n, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = grad[i];
    grad[i] = 0.f;   // consumed: the next backward accumulates into a zeroed buffer
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    params[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace
}  // namespace tcgs

extern "C" tcgs_status tcgs_tile_features(const tcgs_camera* cam, const uint32_t* tile_ranges,
                                          const uint32_t* ids_sorted, const float* mean2d, const float* conic,
                                          const float* opacity, const float* depth, const int32_t* radius,
                                          float* features, tcgs_stream stream) {
    using namespace tcgs;
    if (!valid_camera(cam) || !tile_ranges || !ids_sorted || !mean2d || !conic || !opacity || !depth || !radius ||
        !features || (reinterpret_cast<uintptr_t>(mean2d) & 7))
        return TCGS_ERR_INVALID;
    const DevCamera dc = make_dev_camera(*cam);
    const int tiles = dc.grid_w * dc.grid_h;
    k_tile_features<<<(tiles * 32 + 255) / 256, 256, 0, (cudaStream_t)stream>>>(dc, tile_ranges, ids_sorted, mean2d,
                                                                              conic, opacity, depth, radius, features);
    count_launches(1);
    TCGS_CHECK_LAUNCH();
    return TCGS_OK;
}

extern "C" tcgs_status tcgs_feature_norm(const float* x, int32_t n, float* norm, tcgs_stream stream) {
    using namespace tcgs;
    if (n < 0 || !norm || (n > 0 && !x)) return TCGS_ERR_INVALID;
    k_feature_norm<<<1, 1024, 0, (cudaStream_t)stream>>>(x, n, norm);
    count_launches(1);
    TCGS_CHECK_LAUNCH();
    return TCGS_OK;
}

extern "C" tcgs_status tcgs_mlp_fwd(const float* params, const float* norm, const float* x, int32_t n, float* y,
                                    tcgs_stream stream) {
    using namespace tcgs;
    if (n < 0 || !params || !norm || (n > 0 && (!x || !y))) return TCGS_ERR_INVALID;
    if (n == 0) return TCGS_OK;
    int blocks = (n + 127) / 128;
    if (blocks > 4096) blocks = 4096;
    k_mlp_fwd<<<blocks, 128, 0, (cudaStream_t)stream>>>(params, norm, x, n, y);
    count_launches(1);
    TCGS_CHECK_LAUNCH();
    return TCGS_OK;
}

extern "C" tcgs_status tcgs_mlp_bwd(const float* params, const float* norm, const float* x, const float* target,
                                    int32_t n, float* grad, float* loss, tcgs_stream stream) {
    using namespace tcgs;
    if (n < 0 || !params || !norm || !grad || (n > 0 && (!x || !target))) return TCGS_ERR_INVALID;
    if (n == 0) return TCGS_OK;
    k_mlp_bwd<<<(n + kBwdItems - 1) / kBwdItems, kBwdItems, 0, (cudaStream_t)stream>>>(params, norm, x, target, n,
                                                                                      grad, loss);
    count_launches(1);
    TCGS_CHECK_LAUNCH();
    return TCGS_OK;
}

extern "C" tcgs_status tcgs_adam_step(float* params, float* m, float* v, float* grad, int32_t n_params,
                                      float lr, float beta1, float beta2, float eps, int32_t step,
                                      tcgs_stream stream) {
    using namespace tcgs;
    if (n_params < 0 || step < 1 || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) ||
        (n_params > 0 && (!params || !m || !v || !grad)))
        return TCGS_ERR_INVALID;
    if (n_params == 0) return TCGS_OK;
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    k_adam<<<(n_params + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, m, v, grad, n_params, lr, beta1, beta2,
                                                                    eps, c1, c2);
    count_launches(1);
    TCGS_CHECK_LAUNCH();
    return TCGS_OK;
}
