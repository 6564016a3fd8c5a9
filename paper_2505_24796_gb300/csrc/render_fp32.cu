// render_fp32.cu -- conditional alpha-blending on CUDA cores (Algorithm 1, Eq. 4-6): the
// FP32 baseline the tensor-core path is measured against, and the backward replay.
//
// Forward: one CTA of 256 threads per 16 x 16 tile, one thread per pixel.  The tile's sorted
// list is walked in batches of 256 Gaussians staged in shared memory (one coalesced-by-id
// gather per thread); each thread runs Algorithm 1 on the batch; a block-wide count of
// finished pixels ends the walk early.
#include "common.cuh"

namespace tcgs {
namespace {

constexpr int kFwdThreads = 256;

struct FwdParams {
    DevCamera cam;
    const uint32_t* ranges;
    const uint32_t* ids;
    const float* mean2d;
    const float* conic;
    const float* opacity;
    const float* rgb;
    float bg[3];
    float alpha_max;
    int early_cull;
    float* img;
    float* T_final;
    uint32_t* n_contrib;
    uint32_t* stats;
};

__global__ void __launch_bounds__(kFwdThreads) k_render_fp32(FwdParams p) {
    __shared__ float2 s_xy[kFwdThreads];
    __shared__ float4 s_co[kFwdThreads];   // sigma11, sigma12, sigma22, opacity
    __shared__ float4 s_rgb[kFwdThreads];  // r, g, b, ln(opacity)
    const int tile = blockIdx.x;
    const int tx = tile % p.cam.grid_w, ty = tile / p.cam.grid_w;
    const int t = threadIdx.x;
    const int px_i = tx * kTile + (t & 15), py_i = ty * kTile + (t >> 4);
    const bool inside = px_i < p.cam.width && py_i < p.cam.height;
    const float px = px_i + 0.5f, py = py_i + 0.5f;
    const uint32_t start = p.ranges[2 * tile], end = p.ranges[2 * tile + 1];

    const long long t_start = clock64();
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    uint32_t last = 0, n_eval = end - start, n_blend = 0;
    bool done = !inside;
    uint32_t walked = 0;
    for (uint32_t b0 = start; b0 < end; b0 += kFwdThreads) {
        if (__syncthreads_count(done) == kFwdThreads) break;
        uint32_t idx = b0 + t;
        if (idx < end) {
            uint32_t g = p.ids[idx];
            float2 m = reinterpret_cast<const float2*>(p.mean2d)[g];
            float o = p.opacity[g];
            s_xy[t] = m;
            s_co[t] = make_float4(p.conic[3 * g], p.conic[3 * g + 1], p.conic[3 * g + 2], o);
            s_rgb[t] = make_float4(p.rgb[3 * g], p.rgb[3 * g + 1], p.rgb[3 * g + 2], p.early_cull ? __logf(o) : 0.f);
        }
        __syncthreads();
        uint32_t nb = end - b0 < (uint32_t)kFwdThreads ? end - b0 : (uint32_t)kFwdThreads;
        walked += nb;
        for (uint32_t j = 0; j < nb && !done; ++j) {
            float2 m = s_xy[j];
            float4 co = s_co[j];
            float dx = m.x - px, dy = m.y - py;
            float power = -0.5f * (co.x * dx * dx + co.z * dy * dy) - co.y * dx * dy;
            if (p.early_cull && power + s_rgb[j].w < kBetaCull) continue;   // Sec. 4.1
            float alpha = fminf(p.alpha_max, co.w * expf(power));
            if (alpha < kCullAlpha) continue;                                  // Eq. (5)
            float Tn = fmaf(-alpha, T, T);                                     // T - alpha T
            if (Tn < kTmin) {                                                  // Algorithm 1: terminate
                done = true;
                n_eval = b0 + j + 1 - start;
                break;
            }
            float4 c = s_rgb[j];
            float w = alpha * T;
            C0 += c.x * w; C1 += c.y * w; C2 += c.z * w;
            T = Tn;
            last = b0 + j + 1 - start;
            ++n_blend;
        }
    }
    if (inside) {
        size_t pix = (size_t)py_i * p.cam.width + px_i;
        size_t plane = (size_t)p.cam.width * p.cam.height;
        p.img[pix] = C0 + T * p.bg[0];
        p.img[plane + pix] = C1 + T * p.bg[1];
        p.img[2 * plane + pix] = C2 + T * p.bg[2];
        p.T_final[pix] = T;
        p.n_contrib[pix] = last;
    }
    if (p.stats) {
        __shared__ unsigned long long s_acc[3];
        if (t < 3) s_acc[t] = 0ull;
        __syncthreads();
        if (inside) {
            atomicAdd(&s_acc[0], (unsigned long long)n_blend);
            atomicAdd(&s_acc[1], (unsigned long long)(n_eval - n_blend));
        }
        __syncthreads();
        if (t == 0) {
            uint32_t* st = p.stats + 8 * tile;
            atomicAdd(&st[0], (uint32_t)s_acc[0]);
            atomicAdd(&st[1], (uint32_t)s_acc[1]);
            atomicAdd(&st[2], walked * (uint32_t)kFwdThreads);
            atomicAdd(&st[3], end - start);
            atomicAdd(&st[4], walked);
            atomicAdd(&st[5], (uint32_t)((clock64() - t_start) >> 6));
        }
    }
}

// ---------------------------------------------------------------- backward
//
// One CTA of 128 threads per tile, two pixels a thread; each warp owns an 8 x 8 pixel block.  Each pixel replays
// its fragments 0 .. n_contrib-1 front to back with the forward's FP32 alpha arithmetic, so T_j
// matches the forward bit for bit; the colour blended after fragment j is img - bg T_final -
// (prefix up to j).  A warp replays only the fragments that can reach alpha >= 1/255 somewhere in
// its block (the exact minimum of the conic form over the block's pixel centres against the reach
// limit, as the tensor-core forward marks them): the others contribute to no pixel of the block.
// Per Gaussian, the 9 gradient terms of a warp's pixels are summed with shuffles before the block
// issues the atomics.

struct BwdParams {
    DevCamera cam;
    const uint32_t* ranges;
    const uint32_t* ids;
    const float* mean2d;
    const float* conic;
    const float* opacity;
    const float* rgb;
    float bg[3];
    float alpha_max;
    int early_cull;
    const float* img;
    const float* T_final;
    const uint32_t* n_contrib;
    const float* dL_dimg;
    float* dmean2d;
    float* dconic;
    float* dopacity;
    float* drgb;
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sums v[0..8] over the warp and stores the 9 totals in part[0..8].  v[0..7] take a transposing
// butterfly: at each of the first three levels a lane keeps half of its values and sends the other
// half to its partner, so that after them lane l holds a partial sum of one value,
// 4 bit4(l) + 2 bit3(l) + bit2(l), which two more levels complete (9 shuffles for the 8 values
// instead of 40); v[8] takes the plain 5-level sum.
__device__ __forceinline__ void warp_sum9_store(const float (&v)[9], float* part) {
    const int lane = threadIdx.x & 31;
    const bool u16 = lane & 16, u8 = lane & 8, u4 = lane & 4;
    float w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float send = u16 ? v[i] : v[i + 4], keep = u16 ? v[i + 4] : v[i];
        w[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    float x[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float send = u8 ? w[i] : w[i + 2], keep = u8 ? w[i + 2] : w[i];
        x[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    float y;
    {
        const float send = u4 ? x[0] : x[1], keep = u4 ? x[1] : x[0];
        y = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    y += __shfl_xor_sync(0xffffffffu, y, 2);
    y += __shfl_xor_sync(0xffffffffu, y, 1);
    const float z = warp_sum(v[8]);
    if ((lane & 3) == 0) part[(u16 ? 4 : 0) + (u8 ? 2 : 0) + (u4 ? 1 : 0)] = y;
    if (lane == 0) part[8] = z;
}

// Gradient partial sums of a fragment: each warp parks its 9 sums in shared memory (slots of
// fragments it does not replay, or to which none of its pixels contributes, stay zero); every
// kBwdChunk fragments the block adds the warps' sums, clears the slots, and issues one global atomic
// per nonzero (fragment, parameter).
constexpr int kBwdChunk = 32;
constexpr int kBwdPix = 2;                     // pixels a thread
constexpr int kBwdThreads = 256 / kBwdPix;     // one 16 x 16 tile
constexpr int kBwdWarps = kBwdThreads / 32;
// a warp's pixel block: 8 x 8 for two pixels a thread (2 x 2 warps), 16 x 8 for four (1 x 2 warps)
constexpr int kBwdBlockW = kBwdPix == 2 ? 8 : 16, kBwdBlockH = 8;
static_assert(kBwdPix == 2 || kBwdPix == 4, "two or four pixels a thread");
constexpr int kBwdBatch = 256;                 // fragments staged in shared memory at a time
constexpr int kBwdParams = 9;   // dmean2d (2), dconic (3), dopacity, drgb (3)

// Lane l of warp w replays kBwdPix pixels of the warp's block, one column, rows dyk apart (two
// pixels: (8 (w & 1) + l % 8, 8 (w >> 1) + l / 8) and the one 4 rows below), so that one warp
// reduction per fragment covers 32 kBwdPix pixels and the fragment's loads and block mark serve all
// of them.
__global__ void __launch_bounds__(kBwdThreads) k_render_bwd(BwdParams p) {
    __shared__ float2 s_xy[kBwdBatch];
    __shared__ float4 s_co[kBwdBatch];    // sigma11, sigma12, sigma22, opacity
    __shared__ float4 s_rgb[kBwdBatch];   // r, g, b, reach limit
    __shared__ float4 s_inv[kBwdBatch];   // 1 / sigma11, 1 / sigma22, ln(opacity)
    __shared__ uint32_t s_id[kBwdBatch];
    __shared__ uint32_t s_max;
    __shared__ float s_part[kBwdChunk][kBwdWarps][kBwdParams];
    const int warp = threadIdx.x >> 5;
    const int tile = blockIdx.x;
    const int tx = tile % p.cam.grid_w, ty = tile / p.cam.grid_w;
    const int t = threadIdx.x, lane = t & 31;
    const int bx = kBwdPix == 2 ? warp & 1 : 0, by = kBwdPix == 2 ? warp >> 1 : warp;
    const int lx = kBwdBlockW * bx + (lane & (kBwdBlockW - 1));
    const int ly = kBwdBlockH * by + lane / kBwdBlockW;   // first of the thread's rows; the others follow
    const int dyk = 32 / kBwdBlockW;                       // rows between a thread's pixels
    // the warp's pixel-centre rectangle relative to the tile centre
    const float cx = (float)(tx * kTile + kTile / 2), cy = (float)(ty * kTile + kTile / 2);
    const float bx0 = (float)(kBwdBlockW * bx) - 7.5f, bx1 = bx0 + (float)(kBwdBlockW - 1);
    const float by0 = (float)(kBwdBlockH * by) - 7.5f, by1 = by0 + (float)(kBwdBlockH - 1);
    const uint32_t start = p.ranges[2 * tile], end = p.ranges[2 * tile + 1];
    const float bg0 = p.bg[0], bg1 = p.bg[1], bg2 = p.bg[2];

    // per pixel k: n_contrib, dL/dimg, the colour still to come, T_final, the replayed T
    float px[kBwdPix], py[kBwdPix], g0[kBwdPix], g1[kBwdPix], g2[kBwdPix], R0[kBwdPix], R1[kBwdPix],
        R2[kBwdPix], Tf[kBwdPix], T[kBwdPix];
    uint32_t nc[kBwdPix];
#pragma unroll
    for (int k = 0; k < kBwdPix; ++k) {
        const int px_i = tx * kTile + lx, py_i = ty * kTile + ly + dyk * k;
        px[k] = px_i + 0.5f;
        py[k] = py_i + 0.5f;
        nc[k] = 0;
        g0[k] = g1[k] = g2[k] = R0[k] = R1[k] = R2[k] = 0.f;
        Tf[k] = T[k] = 1.f;
        if (px_i < p.cam.width && py_i < p.cam.height) {
            const size_t pix = (size_t)py_i * p.cam.width + px_i;
            const size_t plane = (size_t)p.cam.width * p.cam.height;
            nc[k] = p.n_contrib[pix];
            Tf[k] = p.T_final[pix];
            g0[k] = p.dL_dimg[pix]; g1[k] = p.dL_dimg[plane + pix]; g2[k] = p.dL_dimg[2 * plane + pix];
            // colour still to come after the current fragment, initially everything blended
            R0[k] = p.img[pix] - Tf[k] * bg0;
            R1[k] = p.img[plane + pix] - Tf[k] * bg1;
            R2[k] = p.img[2 * plane + pix] - Tf[k] * bg2;
        }
    }
    uint32_t nc_max = 0;
#pragma unroll
    for (int k = 0; k < kBwdPix; ++k) nc_max = nc[k] > nc_max ? nc[k] : nc_max;
    const uint32_t warp_nc = __reduce_max_sync(0xffffffffu, nc_max);
    if (t == 0) s_max = 0;
    for (int q = t; q < kBwdChunk * kBwdWarps * kBwdParams; q += kBwdThreads) (&s_part[0][0][0])[q] = 0.f;
    __syncthreads();
    if (lane == 0) atomicMax(&s_max, warp_nc);
    __syncthreads();
    const uint32_t span = s_max;
    for (uint32_t b0 = 0; b0 < span; b0 += kBwdBatch) {
        __syncthreads();
        for (int u = t; u < kBwdBatch; u += kBwdThreads) {
            const uint32_t idx = start + b0 + (uint32_t)u;
            if (idx < end) {
                const uint32_t g = p.ids[idx];
                const float o = p.opacity[g];
                const float a = p.conic[3 * g], c = p.conic[3 * g + 2];
                s_id[u] = g;
                s_xy[u] = reinterpret_cast<const float2*>(p.mean2d)[g];
                s_co[u] = make_float4(a, p.conic[3 * g + 1], c, o);
                const float lno = __logf(o);
                s_rgb[u] = make_float4(p.rgb[3 * g], p.rgb[3 * g + 1], p.rgb[3 * g + 2], reach_limit(lno));
                s_inv[u] = make_float4(__fdividef(1.f, a), __fdividef(1.f, c), lno, 0.f);
            }
        }
        __syncthreads();
        const uint32_t nb = span - b0 < (uint32_t)kBwdBatch ? span - b0 : (uint32_t)kBwdBatch;
        for (uint32_t c0 = 0; c0 < nb; c0 += kBwdChunk) {
            // this warp's fragments of the chunk: in some pixel's replay range and able to reach the block
            const uint32_t jl = c0 + (uint32_t)lane;
            bool mk = jl < nb && b0 + jl < warp_nc;
            if (mk) {
                const float2 m = s_xy[jl];
                const float4 co = s_co[jl];
                const float4 inv = s_inv[jl];
                const float lim = s_rgb[jl].w;
                mk = lim >= 0.f &&
                     min_q_box_facing(m.x - cx, m.y - cy, co.x, co.y, co.z, inv.x, inv.y, bx0, bx1, by0, by1) <= lim;
            }
            uint32_t marks = __ballot_sync(0xffffffffu, mk);
            while (marks) {
                const uint32_t j = c0 + (uint32_t)(__ffs(marks) - 1);
                marks &= marks - 1;
                const float2 m = s_xy[j];
                const float4 co = s_co[j];
                const float4 c = s_rgb[j];
                const float lno = s_inv[j].z;
                float v[kBwdParams] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                bool contrib = false;
#pragma unroll
                for (int k = 0; k < kBwdPix; ++k) {
                    if (b0 + j < nc[k]) {
                        const float dx = m.x - px[k], dy = m.y - py[k];
                        const float power = -0.5f * (co.x * dx * dx + co.z * dy * dy) - co.y * dx * dy;
                        const float G = expf(power);
                        const float raw = co.w * G;
                        const float alpha = fminf(p.alpha_max, raw);
                        const bool early = p.early_cull && power + lno < kBetaCull;   // same test as the forward
                        if (!early && alpha >= kCullAlpha) {
                            contrib = true;
                            const float w = alpha * T[k];
                            v[6] += w * g0[k]; v[7] += w * g1[k]; v[8] += w * g2[k];
                            R0[k] -= c.x * w; R1[k] -= c.y * w; R2[k] -= c.z * w;
                            const float ia = __frcp_rn(1.f - alpha);   // = 1 / (1 - alpha), correctly rounded
                            const float dL_da = g0[k] * (c.x * T[k] - (R0[k] + Tf[k] * bg0) * ia) +
                                                g1[k] * (c.y * T[k] - (R1[k] + Tf[k] * bg1) * ia) +
                                                g2[k] * (c.z * T[k] - (R2[k] + Tf[k] * bg2) * ia);
                            if (raw <= p.alpha_max) {
                                const float dL_dp = dL_da * alpha;
                                v[5] += dL_da * G;
                                v[0] += -dL_dp * (co.x * dx + co.y * dy);
                                v[1] += -dL_dp * (co.y * dx + co.z * dy);
                                v[2] += -0.5f * dL_dp * dx * dx;
                                v[3] += -dL_dp * dx * dy;
                                v[4] += -0.5f * dL_dp * dy * dy;
                            }
                            T[k] = fmaf(-alpha, T[k], T[k]);
                        }
                    }
                }
                if (__any_sync(0xffffffffu, contrib)) warp_sum9_store(v, s_part[j - c0][warp]);
            }
            // the block adds the warps' sums of the chunk's fragments: one atomic per value
            __syncthreads();
            const uint32_t nf = nb - c0 < (uint32_t)kBwdChunk ? nb - c0 : (uint32_t)kBwdChunk;
            for (uint32_t q = threadIdx.x; q < nf * kBwdParams; q += kBwdThreads) {
                const uint32_t f = q / kBwdParams, k = q - f * kBwdParams;
                float sum = 0.f;
#pragma unroll
                for (int w = 0; w < kBwdWarps; ++w) {
                    sum += s_part[f][w][k];
                    s_part[f][w][k] = 0.f;
                }
                if (sum != 0.f) {
                    const uint32_t g = s_id[c0 + f];
                    float* dst = k < 2 ? &p.dmean2d[2 * g + k]
                                       : (k < 5 ? &p.dconic[3 * g + (k - 2)]
                                                : (k == 5 ? &p.dopacity[g] : &p.drgb[3 * g + (k - 6)]));
                    atomicAdd(dst, sum);
                }
            }
            __syncthreads();
        }
    }
}

}  // namespace
}  // namespace tcgs

namespace tcgs {
tcgs_status launch_render_fp32(const tcgs_camera* cam, const tcgs_render_opts* opts, const uint32_t* tile_ranges,
                               const uint32_t* ids_sorted, const float* mean2d, const float* conic,
                               const float* opacity, const float* rgb, const float* bg3, float* img, float* T_final,
                               uint32_t* n_contrib, cudaStream_t s) {
    FwdParams p;
    p.cam = make_dev_camera(*cam);
    p.ranges = tile_ranges; p.ids = ids_sorted; p.mean2d = mean2d; p.conic = conic; p.opacity = opacity;
    p.rgb = rgb;
    for (int i = 0; i < 3; ++i) p.bg[i] = bg3 ? bg3[i] : 0.f;
    p.alpha_max = opts->alpha_max;
    p.early_cull = opts->early_cull;
    p.img = img; p.T_final = T_final; p.n_contrib = n_contrib; p.stats = opts->tile_stats;
    int tiles = p.cam.grid_w * p.cam.grid_h;
    k_render_fp32<<<tiles, kFwdThreads, 0, s>>>(p);
    count_launches(1);
    TCGS_CHECK_LAUNCH();
    return TCGS_OK;
}
}  // namespace tcgs

extern "C" tcgs_status tcgs_render_bwd(const tcgs_camera* cam, const tcgs_render_opts* opts,
                                       const uint32_t* tile_ranges, const uint32_t* ids_sorted, const float* mean2d,
                                       const float* conic, const float* opacity, const float* rgb, const float* bg3,
                                       const float* img, const float* T_final, const uint32_t* n_contrib,
                                       const float* dL_dimg, float* dmean2d, float* dconic, float* dopacity,
                                       float* drgb, tcgs_stream stream) {
    using namespace tcgs;
    if (!valid_camera(cam) || !opts || !tile_ranges || !ids_sorted || !mean2d || !conic || !opacity || !rgb ||
        !img || !T_final || !n_contrib || !dL_dimg || !dmean2d || !dconic || !dopacity || !drgb)
        return TCGS_ERR_INVALID;
    if (!(opts->alpha_max > 0.f && opts->alpha_max <= 1.f)) return TCGS_ERR_INVALID;
    if (opts->alpha_max >= 1.f) return TCGS_ERR_INVALID;  // 1 / (1 - alpha) must stay finite
    if (reinterpret_cast<uintptr_t>(mean2d) & 7) return TCGS_ERR_INVALID;
    BwdParams p;
    p.cam = make_dev_camera(*cam);
    p.ranges = tile_ranges; p.ids = ids_sorted; p.mean2d = mean2d; p.conic = conic; p.opacity = opacity;
    p.rgb = rgb;
    for (int i = 0; i < 3; ++i) p.bg[i] = bg3 ? bg3[i] : 0.f;
    p.alpha_max = opts->alpha_max;
    p.early_cull = opts->early_cull;
    p.img = img; p.T_final = T_final; p.n_contrib = n_contrib; p.dL_dimg = dL_dimg;
    p.dmean2d = dmean2d; p.dconic = dconic; p.dopacity = dopacity; p.drgb = drgb;
    int tiles = p.cam.grid_w * p.cam.grid_h;
    k_render_bwd<<<tiles, kBwdThreads, 0, (cudaStream_t)stream>>>(p);
    count_launches(1);
    TCGS_CHECK_LAUNCH();
    return TCGS_OK;
}
