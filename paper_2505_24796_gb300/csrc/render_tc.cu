// render_tc.cu -- conditional alpha-blending with the exponent on 5th-generation tensor cores:
// EarlyCull (Sec. 4.1) + Frag2Mat (Sec. 4.2, Eq. 18) + G2L (Sec. 4.3).
//
// Mapping on sm_103a.  One CTA of 128 threads renders one half tile (16 x 8 pixels) and
// walks its tile's sorted list in batches of 64 Gaussians:
//   - U (128 pixels x K, f16) is built once in shared memory: the tile-local pixel vectors
//     u = [1, dx, dy, dx^2, dx dy, dy^2] with dx, dy in {+-0.5, ..., +-7.5}, exact in FP16;
//   - per batch, 64 threads build V (64 Gaussians x K, f16) in shared memory from the
//     Gaussians' tile-local v = [ln o - 1/2 dmu^T Q dmu, (Q dmu)_x, (Q dmu)_y, -1/2 s11, -s12,
//     -1/2 s22] (Eq. 12 in G2L coordinates), scaled by log2(e) so the MMA yields log2(alpha);
//   - one elected thread issues a single tcgen05.mma (M = 128, N = 64, K = 16, FP32 accumulator
//     in TMEM) and commits it to an mbarrier;
//   - each warp reads its 32 TMEM lanes with tcgen05.ld.32x32b: thread i receives pixel i's 64
//     exponents, in list order, in registers, which is exactly the layout the front-to-back
//     blend needs (no transpose, no cross-lane scan);
//   - EarlyCull compares log2(alpha) with -log2(255) before ex2; survivors are blended in FP32.
// Two precisions share the kernel:
//   TC_FP16        the paper's K = 8 layout (v0 / 3 in three slots, u's 1 in three slots),
//   TC_FP16_SPLIT  v = v_hi + v_lo (both FP16) with u duplicated: 12 of the 16 K slots,
//                  same single MMA, about 22-bit accuracy of v.
// Every mbarrier wait is bounded; on a timeout the CTA records TCGS_ERR_TIMEOUT, stops, and still
// releases its TMEM.
#include "common.cuh"

namespace tcgs {
namespace {

constexpr int kTcThreads = 128;
constexpr int kTcN = 64;
constexpr uint32_t kTmemCols = 64;
constexpr int kSmemA = 0;          // U: 128 x 16 f16 = 4096 B
constexpr int kSmemB = 4096;       // V: 64 x 16 f16 = 2048 B
constexpr int kSmemC = 6144;       // colours: 64 x float4 = 1024 B
constexpr int kSmemUsed = 7168;
constexpr int kSmemDyn = 30 * 1024;  // keeps <= 7 CTAs per SM, so 7 x 64 TMEM columns always fit
constexpr float kMaxDp = 10.606601717798213f;   // largest |pixel - tile centre| = 7.5 sqrt(2)
constexpr float kCulledV = -30000.f;             // FP16-finite exponent of a batch slot that cannot pass

// Byte offset of element (row, k) of a K-major f16 operand in the canonical no-swizzle layout:
// 8-row x 16-byte core matrices, K-direction core matrices 128 B apart (LBO), 8-row groups 256 B
// apart (SBO).
__device__ __forceinline__ uint32_t canon_off(int row, int kchunk) {
    return (uint32_t)((row >> 3) * 256 + kchunk * 128 + (row & 7) * 16);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor: start >> 4 [0,14), LBO >> 4 [16,30), SBO >> 4
// [32,46), version 1 at [46,48), base offset 0, no swizzle.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)(128u >> 4) << 16;
    d |= (uint64_t)(256u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor, kind::f16: D = F32 (bit 4), A = B = F16 (0), both K-major,
// N >> 3 at [17,23), M >> 4 at [24,29).
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
    for (uint32_t i = 0; i < (1u << 22); ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(addr), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

__device__ __forceinline__ uint32_t pack2(__half a, __half b) {
    return (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
}

struct TcParams {
    DevCamera cam;
    const uint32_t* ranges;
    const uint32_t* ids;
    const float* mean2d;
    const float* conic;
    const float* opacity;
    const float* rgb;
    float bg[3];
    float alpha_max;
    int split;
    float* img;
    float* T_final;
    uint32_t* n_contrib;
    uint32_t* stats;
    int32_t* status;
    const int32_t* dbg_tiles;   // frag2mat inspection mode
    int dbg_max_n;
    float* dbg_beta;
};

template <bool kInspect>
__global__ void __launch_bounds__(kTcThreads) k_render_tc(TcParams p) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ uint32_t s_tmem;
    __shared__ unsigned long long s_acc[2];

    const int t = threadIdx.x, warp = t >> 5;
    int tile = kInspect ? p.dbg_tiles[blockIdx.x >> 1] : (int)(blockIdx.x >> 1);
    bool tile_ok = true;
    if (kInspect && (tile < 0 || tile >= p.cam.grid_w * p.cam.grid_h)) {   // never index past the grid
        if (t == 0) set_status(p.status, TCGS_ERR_INVALID);
        tile = 0;
        tile_ok = false;
    }
    const int half = blockIdx.x & 1;
    const int tx = tile % p.cam.grid_w, ty = tile / p.cam.grid_w;
    const int lx = t & 15, ly = half * 8 + (t >> 4);
    const int px_i = tx * kTile + lx, py_i = ty * kTile + ly;
    const bool inside = px_i < p.cam.width && py_i < p.cam.height;
    const float cx = (float)(tx * kTile + kTile / 2), cy = (float)(ty * kTile + kTile / 2);   // p(T)
    uint8_t* sA = smem + kSmemA;
    uint8_t* sB = smem + kSmemB;
    float4* sC = reinterpret_cast<float4*>(smem + kSmemC);
    const uint32_t mbar = smem_u32(&s_mbar);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) {
        mbar_init(mbar, 1);
        s_acc[0] = s_acc[1] = 0ull;
    }
    {
        // U row of this pixel (G2L: dp = p - p(T))
        const float dx = (float)lx + 0.5f - kTile / 2, dy = (float)ly + 0.5f - kTile / 2;
        __half u[16];
        const __half one = __float2half_rn(1.f), zero = __float2half_rn(0.f);
        const __half hx = __float2half_rn(dx), hy = __float2half_rn(dy);
        const __half hxx = __float2half_rn(dx * dx), hxy = __float2half_rn(dx * dy), hyy = __float2half_rn(dy * dy);
        if (p.split) {
            u[0] = one; u[1] = hx; u[2] = hy; u[3] = hxx; u[4] = hxy; u[5] = hyy;
            u[6] = one; u[7] = hx; u[8] = hy; u[9] = hxx; u[10] = hxy; u[11] = hyy;
            u[12] = zero; u[13] = zero; u[14] = zero; u[15] = zero;
        } else {
            u[0] = one; u[1] = one; u[2] = one; u[3] = hx; u[4] = hy; u[5] = hxx; u[6] = hxy; u[7] = hyy;
#pragma unroll
            for (int k = 8; k < 16; ++k) u[k] = zero;
        }
        uint4 c0 = make_uint4(pack2(u[0], u[1]), pack2(u[2], u[3]), pack2(u[4], u[5]), pack2(u[6], u[7]));
        uint4 c1 = make_uint4(pack2(u[8], u[9]), pack2(u[10], u[11]), pack2(u[12], u[13]), pack2(u[14], u[15]));
        *reinterpret_cast<uint4*>(sA + canon_off(t, 0)) = c0;
        *reinterpret_cast<uint4*>(sA + canon_off(t, 1)) = c1;
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint64_t descA = make_desc(smem_u32(sA));
    const uint64_t descB = make_desc(smem_u32(sB));
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);

    const uint32_t start = p.ranges[2 * tile], end = p.ranges[2 * tile + 1];
    uint32_t stop = end;
    if (kInspect) {
        uint32_t lim = start + (uint32_t)p.dbg_max_n;
        stop = !tile_ok ? start : (lim < end ? lim : end);
    }
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    uint32_t last = 0, n_eval = end - start, n_blend = 0, walked = 0, phase = 0;
    bool done = !inside;
    float thr = done ? __int_as_float(0x7f800000) : kBeta2Cull;

    for (uint32_t b0 = start; b0 < stop; b0 += kTcN) {
        if (t < kTcN) {
            // V row of Gaussian b0 + t (FP32 arithmetic, then FP16)
            uint32_t idx = b0 + t;
            float v[6] = {kCulledV, 0.f, 0.f, 0.f, 0.f, 0.f};
            float4 col = make_float4(0.f, 0.f, 0.f, 0.f);
            if (idx < stop) {
                uint32_t g = p.ids[idx];
                float2 m = reinterpret_cast<const float2*>(p.mean2d)[g];
                float s11 = p.conic[3 * g], s12 = p.conic[3 * g + 1], s22 = p.conic[3 * g + 2];
                float o = p.opacity[g];
                if (!kInspect) col = make_float4(p.rgb[3 * g], p.rgb[3 * g + 1], p.rgb[3 * g + 2], 0.f);
                float mx = m.x - cx, my = m.y - cy;   // G2L mean
                float qx = s11 * mx + s12 * my, qy = s12 * mx + s22 * my;
                float q0 = mx * qx + my * qy;
                float lno = __logf(o);
                // conservative whole-tile cull: ||dmu - dp||_Q >= sqrt(q0) - |dp| sqrt(lambda_max(Q))
                float lam = 0.5f * (s11 + s22) + sqrtf(0.25f * (s11 - s22) * (s11 - s22) + s12 * s12);
                float reach = sqrtf(fmaxf(q0, 0.f)) - kMaxDp * sqrtf(fmaxf(lam, 0.f));
                float need = 2.f * (lno - kBetaCull);
                bool hopeless = need <= 0.f || (reach > 0.f && reach * reach > 1.001f * need + 1e-3f);
                if (!hopeless) {
                    v[0] = (lno - 0.5f * q0) * kLog2e;
                    v[1] = qx * kLog2e;
                    v[2] = qy * kLog2e;
                    v[3] = -0.5f * s11 * kLog2e;
                    v[4] = -s12 * kLog2e;
                    v[5] = -0.5f * s22 * kLog2e;
                }
            }
            __half h[16];
#pragma unroll
            for (int k = 0; k < 6; ++k) v[k] = fminf(65504.f, fmaxf(-65504.f, v[k]));   // FP16-finite
            if (p.split) {
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    __half hi = __float2half_rn(v[k]);
                    h[k] = hi;
                    h[6 + k] = __float2half_rn(v[k] - __half2float(hi));
                }
                h[12] = h[13] = h[14] = h[15] = __float2half_rn(0.f);
            } else {
                __half third = __float2half_rn(v[0] * (1.f / 3.f));
                h[0] = h[1] = h[2] = third;
#pragma unroll
                for (int k = 1; k < 6; ++k) h[2 + k] = __float2half_rn(v[k]);
#pragma unroll
                for (int k = 8; k < 16; ++k) h[k] = __float2half_rn(0.f);
            }
            uint4 c0 = make_uint4(pack2(h[0], h[1]), pack2(h[2], h[3]), pack2(h[4], h[5]), pack2(h[6], h[7]));
            uint4 c1 = make_uint4(pack2(h[8], h[9]), pack2(h[10], h[11]), pack2(h[12], h[13]), pack2(h[14], h[15]));
            *reinterpret_cast<uint4*>(sB + canon_off(t, 0)) = c0;
            *reinterpret_cast<uint4*>(sB + canon_off(t, 1)) = c1;
            sC[t] = col;
            fence_async_smem();
        }
        tc_fence_before();
        __syncthreads();
        if (t == 0) {
            tc_fence_after();
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                "l"(descA), "l"(descB), "r"(kIdesc), "r"(0u)
                : "memory");
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                         : "memory");
        }
        bool ok = mbar_wait(mbar, phase);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            if (t == 0) set_status(p.status, TCGS_ERR_TIMEOUT);
            break;
        }
        tc_fence_after();
        uint32_t r[2 * 32];
        tmem_ld32(taddr, r);
        tmem_ld32(taddr + 32, r + 32);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const uint32_t nb = stop - b0 < (uint32_t)kTcN ? stop - b0 : (uint32_t)kTcN;
        walked += nb;
        if (kInspect) {
            const int pix = half * 128 + t;
            float* out = p.dbg_beta + ((size_t)(blockIdx.x >> 1) * 256 + pix) * p.dbg_max_n;
            for (uint32_t j = 0; j < nb; ++j) out[b0 - start + j] = __uint_as_float(r[j]) * 0.6931471805599453f;
        } else {
#pragma unroll
            for (int j = 0; j < kTcN; ++j) {
                const float b2 = __uint_as_float(r[j]);
                if (b2 >= thr) {   // EarlyCull: log2(alpha) against -log2(255) before ex2
                    const float a = fminf(p.alpha_max, ex2_approx(b2));
                    const float Tn = fmaf(-a, T, T);
                    if (Tn < kTmin) {
                        thr = __int_as_float(0x7f800000);
                        done = true;
                        n_eval = b0 + j + 1 - start;
                    } else {
                        const float4 c = sC[j];
                        const float w = a * T;
                        C0 = fmaf(c.x, w, C0);
                        C1 = fmaf(c.y, w, C1);
                        C2 = fmaf(c.z, w, C2);
                        T = Tn;
                        last = b0 + j + 1 - start;
                        ++n_blend;
                    }
                }
            }
        }
        tc_fence_before();
        if (!kInspect) {
            if (!__syncthreads_or(!done)) break;
        } else {
            __syncthreads();
        }
    }

    if (kInspect) {
        const int pix = half * 128 + t;
        float* out = p.dbg_beta + ((size_t)(blockIdx.x >> 1) * 256 + pix) * p.dbg_max_n;
        for (int j = (int)(stop - start); j < p.dbg_max_n; ++j) out[j] = -__int_as_float(0x7f800000);
    } else {
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
            if (inside) {
                atomicAdd(&s_acc[0], (unsigned long long)n_blend);
                atomicAdd(&s_acc[1], (unsigned long long)(n_eval - n_blend));
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (!kInspect && p.stats && t == 0) {
        atomicAdd(&p.stats[4 * tile + 0], (uint32_t)s_acc[0]);
        atomicAdd(&p.stats[4 * tile + 1], (uint32_t)s_acc[1]);
        atomicAdd(&p.stats[4 * tile + 2], walked * (uint32_t)kTcThreads);
        if (half == 0) atomicAdd(&p.stats[4 * tile + 3], end - start);
    }
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

int g_checked_device = -1;
bool g_device_ok = false;

bool device_is_sm103() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (dev == g_checked_device) return g_device_ok;
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    g_checked_device = dev;
    g_device_ok = (major == 10 && minor == 3);
    return g_device_ok;
}

bool g_attr_set[2] = {false, false};

template <bool kInspect>
tcgs_status launch_tc(const TcParams& p, int blocks, cudaStream_t s) {
    if (!g_attr_set[kInspect]) {
        if (cudaFuncSetAttribute(k_render_tc<kInspect>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemDyn) !=
            cudaSuccess)
            return TCGS_ERR_CUDA;
        g_attr_set[kInspect] = true;
    }
    k_render_tc<kInspect><<<blocks, kTcThreads, kSmemDyn, s>>>(p);
    count_launches(1);
    TCGS_CHECK_LAUNCH();
    return TCGS_OK;
}

TcParams base_params(const tcgs_camera* cam, int precision, const uint32_t* tile_ranges, const uint32_t* ids,
                     const float* mean2d, const float* conic, const float* opacity) {
    TcParams p = {};
    p.cam = make_dev_camera(*cam);
    p.ranges = tile_ranges; p.ids = ids; p.mean2d = mean2d; p.conic = conic; p.opacity = opacity;
    p.split = precision == TCGS_TC_FP16_SPLIT;
    p.alpha_max = 0.99f;
    return p;
}

}  // namespace

static_assert(kSmemUsed <= kSmemDyn, "shared memory layout");

tcgs_status launch_render_tc(const tcgs_camera* cam, const tcgs_render_opts* opts, const uint32_t* tile_ranges,
                             const uint32_t* ids_sorted, const float* mean2d, const float* conic,
                             const float* opacity, const float* rgb, const float* bg3, float* img, float* T_final,
                             uint32_t* n_contrib, cudaStream_t s) {
    if (!device_is_sm103()) return TCGS_ERR_UNSUPPORTED;
    TcParams p = base_params(cam, opts->precision, tile_ranges, ids_sorted, mean2d, conic, opacity);
    p.rgb = rgb;
    for (int i = 0; i < 3; ++i) p.bg[i] = bg3 ? bg3[i] : 0.f;
    p.alpha_max = opts->alpha_max;
    p.img = img; p.T_final = T_final; p.n_contrib = n_contrib;
    p.stats = opts->tile_stats; p.status = opts->device_status;
    int tiles = p.cam.grid_w * p.cam.grid_h;
    return launch_tc<false>(p, 2 * tiles, s);
}

}  // namespace tcgs

namespace tcgs {
tcgs_status launch_render_fp32(const tcgs_camera* cam, const tcgs_render_opts* opts, const uint32_t* tile_ranges,
                               const uint32_t* ids_sorted, const float* mean2d, const float* conic,
                               const float* opacity, const float* rgb, const float* bg3, float* img, float* T_final,
                               uint32_t* n_contrib, cudaStream_t s);
}

extern "C" tcgs_status tcgs_render_fwd(const tcgs_camera* cam, const tcgs_render_opts* opts,
                                       const uint32_t* tile_ranges, const uint32_t* ids_sorted, const float* mean2d,
                                       const float* conic, const float* opacity, const float* rgb, const float* bg3,
                                       float* img, float* T_final, uint32_t* n_contrib, tcgs_stream stream) {
    using namespace tcgs;
    if (!valid_camera(cam) || !opts || !tile_ranges || !ids_sorted || !mean2d || !conic || !opacity || !rgb ||
        !img || !T_final || !n_contrib)
        return TCGS_ERR_INVALID;
    if (!(opts->alpha_max > 0.f && opts->alpha_max <= 1.f)) return TCGS_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(mean2d) & 7) return TCGS_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    switch (opts->precision) {
        case TCGS_FP32:
            return launch_render_fp32(cam, opts, tile_ranges, ids_sorted, mean2d, conic, opacity, rgb, bg3, img,
                                      T_final, n_contrib, s);
        case TCGS_TC_FP16:
        case TCGS_TC_FP16_SPLIT:
            return launch_render_tc(cam, opts, tile_ranges, ids_sorted, mean2d, conic, opacity, rgb, bg3, img,
                                    T_final, n_contrib, s);
        default:
            return TCGS_ERR_INVALID;
    }
}

extern "C" tcgs_status tcgs_frag2mat_beta(const tcgs_camera* cam, int32_t precision, const uint32_t* tile_ranges,
                                          const uint32_t* ids_sorted, const float* mean2d, const float* conic,
                                          const float* opacity, int32_t n_tiles, const int32_t* tiles,
                                          int32_t max_n, float* beta_out, int32_t* device_status,
                                          tcgs_stream stream) {
    using namespace tcgs;
    if (!valid_camera(cam) || !tile_ranges || !ids_sorted || !mean2d || !conic || !opacity || n_tiles < 0 ||
        max_n < 0 || (n_tiles > 0 && (!tiles || !beta_out)))
        return TCGS_ERR_INVALID;
    if (precision != TCGS_TC_FP16 && precision != TCGS_TC_FP16_SPLIT) return TCGS_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(mean2d) & 7) return TCGS_ERR_INVALID;
    if (n_tiles == 0 || max_n == 0) return TCGS_OK;
    if (!device_is_sm103()) return TCGS_ERR_UNSUPPORTED;
    TcParams p = base_params(cam, precision, tile_ranges, ids_sorted, mean2d, conic, opacity);
    p.status = device_status;
    p.dbg_tiles = tiles; p.dbg_max_n = max_n; p.dbg_beta = beta_out;
    return launch_tc<true>(p, 2 * n_tiles, (cudaStream_t)stream);
}
