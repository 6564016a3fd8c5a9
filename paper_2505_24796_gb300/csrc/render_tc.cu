// render_tc.cu -- conditional alpha-blending with the exponent on 5th-generation tensor cores:
// EarlyCull (Sec. 4.1) + Frag2Mat (Sec. 4.2, Eq. 18) + G2L (Sec. 4.3).
//
// Mapping on sm_103a.  One CTA of 256 threads renders one 16 x 16 tile; each of its 8 warps owns an
// 8 x 4 pixel block.  The tile's sorted list is walked in batches of kN = 32 Gaussians:
//   - U (256 pixels x 16, f16) is built once in shared memory: the tile-local pixel vectors
//     u = [1, dx, dy, dx^2, dx dy, dy^2] with dx, dy in {+-0.5, ..., +-7.5}, exact in FP16;
//   - a loader warp gathers each batch's Gaussians one batch ahead (registers), and stages their
//     tile-local parameters, colours and V (32 Gaussians x 16, f16) in shared memory, V from the
//     tile-local v = [ln o - 1/2 dmu^T Q dmu, (Q dmu)_x, (Q dmu)_y, -1/2 s11, -s12, -1/2 s22]
//     (Eq. 12 in G2L coordinates) scaled by log2(e), so the MMA yields log2(alpha);
//   - one elected thread issues two tcgen05.mma (M = 128 rows each, N = 32, K = 16, FP32
//     accumulators in TMEM) against the same V and commits them to an mbarrier;
//   - each warp marks, one batch ahead, the Gaussians that can reach alpha >= 1/255 anywhere in its
//     block (exact minimum of the conic form over the block), then walks only its marked columns
//     (a warp-uniform loop), reading each with tcgen05.ld.32x32b.x1: every thread receives its own
//     pixel's exponent, in list order, which is the layout the front-to-back blend needs (no
//     transpose, no cross-lane scan);
//   - EarlyCull compares log2(alpha) with -log2(255) before ex2; survivors are blended in FP32,
//     branch-free (selects), so a warp never diverges inside the walk.
// Every precision uses 32-byte operand rows (one MMA of K = 32 bytes per half tile):
//   TC_FP16        kind::f16, the paper's K = 8 layout (v0 / 3 in three slots, u's 1 in three slots),
//   TC_FP16_SPLIT  kind::f16, v = v_hi + v_lo (both FP16) with u duplicated: 12 of the 16 K slots,
//                  same single MMA, about 22-bit accuracy of v,
//   TC_TF32        kind::tf32, K = 8: u and v rounded to TF32 (round to nearest, ties away),
//   TC_FP8         kind::f8f6f4, K = 32, e4m3: u = u_hi + u_lo (exact) and v = v_hi + v_lo + v_lo2,
//                  with power-of-two column scales that keep every part inside the e4m3 range;
//                  five groups of six products, u_hi (v_hi + v_lo + v_lo2) + u_lo (v_hi + v_lo),
//   TC_FP16_GLOBAL / TC_TF32_GLOBAL  the ablation of Table 5: Frag2Mat without G2L, u and v in
//                  global pixel coordinates (FP16 overflows past 256 px, as the paper observes);
//                  these walk every list entry of the tile (no FP32 reach test, no block marks).
// The block marks only skip list entries that Algorithm 1 would cull at every pixel of the block
// (the minimum over the block's pixel-centre rectangle bounds every pixel), so the image is that of
// Algorithm 1; with tile_cull = 0 every entry is walked.
// Every mbarrier wait is bounded; on a timeout the CTA records TCGS_ERR_TIMEOUT, stops, and still
// releases its TMEM; an MMA issued for a batch that is not walked is waited for before release.
// Two accumulator buffers let the MMAs of batch k+1 run while batch k is walked; only thread 0 polls
// the mbarrier, the others wait in a hardware barrier.
#include <cuda_fp8.h>

#include <cstring>
#include <mutex>

#include "common.cuh"

namespace tcgs {
namespace {

constexpr int kConsumerWarps = 8;      // 8 warps of 8 x 4 pixels = one 16 x 16 tile, one thread per pixel
constexpr int kN = 32;                 // Gaussians per MMA batch (UMMA N; slot = producer lane)
constexpr uint32_t kTmemCols = 4 * kN; // 2 accumulator buffers x 2 row halves
constexpr int kVBytes = kN * 32;       // one V buffer: 32 x 16 f16
constexpr int kPBytes = kN * 48;       // one parameter buffer: 3 float4 per slot
constexpr int kSmemA = 0;              // U: 256 x 16 f16 = 8192 B (two 128-row halves)
constexpr int kSmemB = 8192;           // V: 3 buffers
constexpr int kSmemP = kSmemB + 3 * kVBytes;   // slot parameters and colours: 3 buffers
constexpr int kSmemVf = kSmemP + 3 * kPBytes;  // CUDA-core product: FP32 v of each slot, 3 buffers of kN x 32 B
// 46 KB of dynamic shared memory caps residency at 4 CTAs per SM (4 x 47 KB <= 228 KB < 5 x 47 KB),
// so 4 x 128 TMEM columns always fit in the 512 available and tcgen05.alloc never waits; the
// launch bound (56 registers a thread) lets all 4 be resident
constexpr int kSmemDyn = 46 * 1024;
constexpr int kTcCtasPerSm = 4;
constexpr float kCulledV = -30000.f;   // FP16-finite exponent of a slot that no pixel can use

// Byte offset of the 16-byte chunk kchunk (K elements 8 kchunk .. 8 kchunk + 7) of row `row` of a
// K-major f16 operand in the canonical no-swizzle layout: 8-row x 16-byte core matrices,
// K-direction core matrices 128 B apart (LBO), 8-row groups 256 B apart (SBO).
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

// Instruction descriptors: D = F32 (bit 4), A and B types at [7,10) and [10,13), both K-major,
// N >> 3 at [17,23), M >> 4 at [24,29).  kind::f16 with F16 = 0; kind::tf32 with TF32 = 2;
// kind::f8f6f4 with E4M3 = 0.
constexpr uint32_t kIdescShape = (1u << 4) | ((uint32_t)(kN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
constexpr uint32_t kIdescF16 = kIdescShape;
constexpr uint32_t kIdescTf32 = kIdescShape | (2u << 7) | (2u << 10);
constexpr uint32_t kIdescE4m3 = kIdescShape;

// Operand encodings of a 32-byte K row (see the file comment).
enum : int { kEncF16Split = 0, kEncF16Pad = 1, kEncTf32 = 2, kEncFp8 = 3 };

__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity, uint32_t polls = 1u << 22) {
    for (uint32_t i = 0; i < polls; ++i) {
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
// tcgen05.wait::ld with the registers of the loads it completes as operands, so that no use of them
// can be scheduled above the wait.
__device__ __forceinline__ void tmem_wait_ld1(uint32_t& a) {
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(a)::"memory");
}
__device__ __forceinline__ void tmem_wait_ld2(uint32_t& a, uint32_t& b) {
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(a), "+r"(b)::"memory");
}
__device__ __forceinline__ void tmem_wait_ld32(uint32_t* r) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31])::"memory");
}

__device__ __forceinline__ uint32_t tmem_ld1(uint32_t taddr) {
    uint32_t r;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr));
    return r;
}

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

__device__ __forceinline__ uint32_t tf32_bits(float x) {   // round to TF32 (10 fraction bits)
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ uint32_t e4m3_bits(float x) {   // round to nearest e4m3, saturating at +-448
    return (uint32_t)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
}

__device__ __forceinline__ float e4m3_value(uint32_t b) {
    return __half2float(__half(__nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)b, __NV_E4M3)));
}

// FP8 column scales 2^-a_i of u (and 2^a_i of v), a = {0, 2, 2, 6, 6, 6}: the scaled tile-local
// u parts stay exact e4m3 numbers (at least 2^-8) and the scaled v of any Gaussian that can reach
// the tile stays below 448 (|v0| <= 371, |v1|, |v2| <= 60, |v3|, |v5| <= 2.4, |v4| <= 4.8 in log2
// units, from the reach test and lambda_max(Q) <= 1 / 0.3).
__device__ __forceinline__ float fp8_uscale(int i) { return i == 0 ? 1.f : (i < 3 ? 0.25f : 0.015625f); }

// One 32-byte K row of U (kV = false, c = u) or V (kV = true, c = v) in encoding `enc`, as eight
// 32-bit words in K order.
template <bool kV>
__device__ __forceinline__ void encode_row(int enc, const float c[6], uint32_t w[8]) {
    if (enc == kEncTf32) {
#pragma unroll
        for (int k = 0; k < 6; ++k) w[k] = tf32_bits(c[k]);
        w[6] = w[7] = 0u;
    } else if (enc == kEncFp8) {
        uint32_t b[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) b[k] = 0u;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float sc = kV ? 1.f / fp8_uscale(k) : fp8_uscale(k);
            const float x = c[k] * sc;
            const uint32_t hi = e4m3_bits(x);
            const float r1 = x - e4m3_value(hi);
            const uint32_t lo = e4m3_bits(r1);
            if (kV) {   // [v_hi | v_lo | v_lo2 | v_hi | v_lo]
                const uint32_t lo2 = e4m3_bits(r1 - e4m3_value(lo));
                b[k] = hi; b[6 + k] = lo; b[12 + k] = lo2; b[18 + k] = hi; b[24 + k] = lo;
            } else {    // [u_hi | u_hi | u_hi | u_lo | u_lo]
                b[k] = hi; b[6 + k] = hi; b[12 + k] = hi; b[18 + k] = lo; b[24 + k] = lo;
            }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) w[q] = b[4 * q] | (b[4 * q + 1] << 8) | (b[4 * q + 2] << 16) | (b[4 * q + 3] << 24);
    } else {
        __half h[16];
        const __half zero = __float2half_rn(0.f);
#pragma unroll
        for (int k = 0; k < 16; ++k) h[k] = zero;
        if (enc == kEncF16Split) {
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const __half hi = __float2half_rn(c[k]);
                h[k] = hi;
                h[6 + k] = kV ? __float2half_rn(c[k] - __half2float(hi)) : hi;
            }
        } else {   // paper padding: [v0/3 x 3, v1..v5] and [1 x 3, u1..u5]
            const __half c0 = __float2half_rn(kV ? c[0] * (1.f / 3.f) : c[0]);
            h[0] = h[1] = h[2] = c0;
#pragma unroll
            for (int k = 1; k < 6; ++k) h[2 + k] = __float2half_rn(c[k]);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) w[q] = pack2(h[2 * q], h[2 * q + 1]);
    }
}

__device__ __forceinline__ void store_row(uint8_t* base, int row, const uint32_t w[8]) {
    *reinterpret_cast<uint4*>(base + canon_off(row, 0)) = make_uint4(w[0], w[1], w[2], w[3]);
    *reinterpret_cast<uint4*>(base + canon_off(row, 1)) = make_uint4(w[4], w[5], w[6], w[7]);
}

// Per-view inputs and outputs (the batched renderer walks (view, tile) items of up to
// TCGS_MAX_VIEWS views; the single-view call uses entry 0).
struct ViewData {
    DevCamera cam;
    const uint32_t* ranges;
    const uint32_t* ids;
    const float* mean2d;
    const float* conic;
    const float* rgb;
    float* img;
    float* T_final;
    uint32_t* n_contrib;
    uint32_t* stats;
};

struct TcParams {
    ViewData v[TCGS_MAX_VIEWS];
    const float* opacity;
    float bg[3];
    float alpha_max;
    int enc;                    // operand encoding (kEnc*)
    int global;                 // 1: Frag2Mat in global pixel coordinates (ablation, no G2L)
    int cuda_core;              // 1: the product u^T v on CUDA cores in FP32 (TCGS_FP32_FRAG2MAT)
    int tile_cull;
    int early_cull;             // selects the kernel instance (kEarly)
    int ppt;                    // pixels per consumer thread (kPPT instance; 2 only for the EarlyCull
                                // split-FP16 and CUDA-core paths, anything else renders with 1)
    int32_t* status;
    int n_views;
    const uint32_t* queue;      // queue mode: items (view << 16 | tile) in the order to render
    int queue_tiles;            // queue mode, one view: the items are plain tile indices
    uint32_t n_items;
    uint32_t* counter;          // queue mode: next item to take (zeroed before the launch)
    const int32_t* dbg_tiles;   // frag2mat inspection mode
    int dbg_max_n;
    float* dbg_beta;
};

// Gaussian data of one batch slot, held in the producer's registers one batch ahead of its use.
struct Slot {
    float mx, my, s11, s12, s22, o, r, g, b;
    bool valid;
};

__device__ __forceinline__ Slot load_slot(const ViewData& vd, const float* opacity, uint32_t g, bool valid,
                                          bool colour) {
    Slot d;
    d.valid = valid;
    if (valid) {
        const float2 m = reinterpret_cast<const float2*>(vd.mean2d)[g];
        d.mx = m.x; d.my = m.y;
        d.s11 = vd.conic[3 * g]; d.s12 = vd.conic[3 * g + 1]; d.s22 = vd.conic[3 * g + 2];
        d.o = opacity[g];
        if (colour) { d.r = vd.rgb[3 * g]; d.g = vd.rgb[3 * g + 1]; d.b = vd.rgb[3 * g + 2]; }
        else { d.r = d.g = d.b = 0.f; }
    } else {
        d.mx = d.my = d.s11 = d.s12 = d.s22 = d.r = d.g = d.b = 0.f;
        d.o = 1.f;
    }
    return d;
}

// Product paths: the tensor cores with the encoding and frame taken from p (kPathGeneric), the tensor
// cores with the default encoding fixed at compile time (TC_FP16_SPLIT with G2L), or the same product
// u^T v on CUDA cores in FP32 (TCGS_FP32_FRAG2MAT: no TMEM, no MMA; everything else identical).
enum : int { kPathGeneric = 0, kPathSplit = 1, kPathCudaCore = 2 };

// Consumer warps and threads of a CTA with kPPT pixels per consumer thread: 8 warps of 8 x 4 pixels
// (one each), or 4 warps of 8 x 8 pixels (two each, four rows apart: one in each MMA half, at the
// same TMEM lane), plus the producer warp.
template <int kPPT>
constexpr int consumer_warps() { return kPPT == 2 ? 4 : kConsumerWarps; }
template <int kPPT>
constexpr int tc_threads() { return 32 * (consumer_warps<kPPT>() + 1); }

// kEarly: EarlyCull form of the cull test; kPath: how the exponents are produced (above); kPPT:
// pixels per consumer thread (2: coarser 8 x 8 block marks and two blend chains per walked column,
// which pays off for views of large footprints, whose batches mark most entries anyway).
template <bool kInspect, bool kStats, bool kQueue, bool kEarly, int kPath, int kPPT>
__global__ void __launch_bounds__(tc_threads<kPPT>(), kTcCtasPerSm) k_render_tc(TcParams p) {
    constexpr bool kSplit = kPath == kPathSplit;
    constexpr bool kCC = kPath == kPathCudaCore;
    constexpr bool k2 = kPPT == 2;
    constexpr int kCW = consumer_warps<kPPT>();
    static_assert(kPPT == 1 || (kPPT == 2 && !kInspect), "two pixels a thread: rendering only");
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t s_mbar[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_timeout;
    __shared__ uint32_t s_item;
    __shared__ unsigned long long s_acc[3];

    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const bool producer = warp == kCW;
    // consumer warp block of a tile, and this thread's pixel in it.  One pixel a thread: 8 x 4 blocks,
    // warps 0-3 cover rows 0-7 (MMA half 0, U rows 0-127), warps 4-7 rows 8-15 (half 1, U rows
    // 128-255).  Two: 8 x 8 blocks, warp w rows 8 (w >> 1) .. + 7; pixel (lx, ly) in half 0 (U row
    // 32 w + lane) and (lx, ly + 4) in half 1 (U row 128 + 32 w + lane), both at TMEM lane 32 w + lane.
    const int half = k2 ? 0 : (warp >> 2) & 1;
    const int bx = warp & 1, by = k2 ? (warp >> 1) & 1 : (warp >> 1) & 3;
    const int lx = 8 * bx + (lane & 7), ly = (k2 ? 8 : 4) * by + (lane >> 3);
    // this warp's pixel-centre rectangle, tile-local
    const float bx0 = 8.f * bx - 7.5f, bx1 = bx0 + 7.f;
    const float by0 = (k2 ? 8.f : 4.f) * by - 7.5f, by1 = by0 + (k2 ? 7.f : 3.f);
    uint8_t* sA = smem + kSmemA;
    const uint32_t mbar0 = smem_u32(&s_mbar[0]);
    const int enc = kSplit ? (int)kEncF16Split : p.enc;
    const bool global = (kSplit || kCC) ? false : p.global != 0;
    // CUDA-core product: this thread's tile-local pixel vector (u1..u5; u0 = 1) in registers
    const float ux = (float)lx + 0.5f - kTile / 2, uy = (float)ly + 0.5f - kTile / 2;
    const float uxx = ux * ux, uxy = ux * uy, uyy = uy * uy;
    const float uyB = uy + 4.f;   // the second pixel (two a thread)
    const float uxyB = ux * uyB, uyyB = uyB * uyB;

    if (producer) {
        if (!kCC) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(&s_tmem)),
                         "r"(kTmemCols)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
        if (lane == 0) {
            mbar_init(mbar0, 1);
            mbar_init(mbar0 + 8, 1);
            s_timeout = 0;
        }
    } else if (!kCC) {
        // U row t = this thread's pixel, tile-local (G2L: dp = p - p(T)); the same for every tile.
        // Without G2L (one tile per CTA) it is the global pixel centre of the CTA's tile.
        float dx = (float)lx + 0.5f - kTile / 2, dy = (float)ly + 0.5f - kTile / 2;
        if (global && !kQueue) {
            int tile0 = kInspect ? p.dbg_tiles[blockIdx.x] : (int)blockIdx.x;
            const int ntiles = p.v[0].cam.grid_w * p.v[0].cam.grid_h;
            tile0 = tile0 < 0 || tile0 >= ntiles ? 0 : tile0;   // an invalid tile is reported below
            dx += (float)((tile0 % p.v[0].cam.grid_w) * kTile + kTile / 2);
            dy += (float)((tile0 / p.v[0].cam.grid_w) * kTile + kTile / 2);
        }
        const float u[6] = {1.f, dx, dy, dx * dx, dx * dy, dy * dy};
        uint32_t w[8];
        encode_row<false>(enc, u, w);
        store_row(sA, t, w);
        if (k2) {   // U row 128 + t: the thread's second pixel, four rows below
            const float dyB = dy + 4.f;
            const float uB[6] = {1.f, dx, dyB, dx * dx, dx * dyB, dyB * dyB};
            encode_row<false>(enc, uB, w);
            store_row(sA, 128 + t, w);
        }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();   // U visible to the tensor core, TMEM address and mbarriers published
    tc_fence_after();
    pdl_wait();        // the set-up above touches no global memory; the tiles below do
    const uint32_t tmem = kCC ? 0u : s_tmem;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    const float kInf = __int_as_float(0x7f800000);
    uint32_t phase_bits = 0;   // producer lane 0: completed-phase parity of the two mbarriers
    bool stopped = false;

    for (uint32_t round = 0;; ++round) {
        // ---------------- which tile of which view
        int view = 0, tile;
        bool tile_ok = true;
        if (kQueue) {
            if (t == 0) s_item = atomicAdd(p.counter, 1u);
            __syncthreads();
            const uint32_t item = s_item;
            if (item >= p.n_items) break;
            const uint32_t it = p.queue[item];
            view = p.queue_tiles ? 0 : (int)(it >> 16);
            tile = p.queue_tiles ? (int)it : (int)(it & 0xFFFFu);
        } else {
            if (round > 0) break;
            tile = kInspect ? p.dbg_tiles[blockIdx.x] : (int)blockIdx.x;
        }
        if (view >= p.n_views) {   // never index past the view table
            if (t == 0) set_status(p.status, TCGS_ERR_INVALID);
            view = 0;
            tile_ok = false;
        }
        const ViewData& vd = p.v[view];
        if (tile < 0 || tile >= vd.cam.grid_w * vd.cam.grid_h) {   // never index past the grid
            if (t == 0) set_status(p.status, TCGS_ERR_INVALID);
            tile = 0;
            tile_ok = false;
        }
        const long long t_start = clock64();
        const int tx = tile % vd.cam.grid_w, ty = tile / vd.cam.grid_w;
        const int px_i = tx * kTile + lx, py_i = ty * kTile + ly;
        const bool inside = !producer && tile_ok && px_i < vd.cam.width && py_i < vd.cam.height;
        const bool insideB = k2 && !producer && tile_ok && px_i < vd.cam.width && py_i + 4 < vd.cam.height;
        const float cx = (float)(tx * kTile + kTile / 2), cy = (float)(ty * kTile + kTile / 2);   // p(T)
        const uint32_t start = vd.ranges[2 * tile], end = vd.ranges[2 * tile + 1];
        uint32_t stop = tile_ok ? end : start;
        if (kInspect) {
            uint32_t lim = start + (uint32_t)p.dbg_max_n;
            stop = !tile_ok ? start : (lim < end ? lim : end);
        }
        const uint32_t nbat = (stop - start + kN - 1) / kN;
        if (kStats && t == 0) s_acc[0] = s_acc[1] = s_acc[2] = 0ull;

        // Producer: stage batch slot `lane` into buffer `buf`: tile-local parameters (with the
        // reciprocals the block tests need) and colour, and the V row of the MMA.
        auto stage = [&](const Slot& d, int buf) {
            float4* sP = reinterpret_cast<float4*>(smem + kSmemP + buf * kPBytes);
            float v[6] = {kCulledV, 0.f, 0.f, 0.f, 0.f, 0.f};
            float mx = 0.f, my = 0.f, lim = -1.f, ia = 0.f, ic = 0.f;
            if (d.valid && global) {
                // ablation without G2L: Eq. 12 in global coordinates for every listed Gaussian
                mx = d.mx; my = d.my;
                const float lno = __logf(d.o);
                const float qx = d.s11 * mx + d.s12 * my, qy = d.s12 * mx + d.s22 * my;
                v[0] = (lno - 0.5f * (mx * qx + my * qy)) * kLog2e;
                v[1] = qx * kLog2e;
                v[2] = qy * kLog2e;
                v[3] = -0.5f * d.s11 * kLog2e;
                v[4] = -d.s12 * kLog2e;
                v[5] = -0.5f * d.s22 * kLog2e;
                lim = 3.0e38f;
            } else if (d.valid) {
                mx = d.mx - cx; my = d.my - cy;   // G2L mean
                const float lno = __logf(d.o);
                lim = reach_limit(lno);
                if (lim >= 0.f) {
                    // V only for Gaussians that can reach the tile: ||dmu - dp||_Q >= sqrt(q0) -
                    // |dp| sqrt(lambda_max(Q)), |dp| <= 7.5 sqrt(2); their tile-local coefficients
                    // are then bounded and FP16 never overflows
                    const float qx = d.s11 * mx + d.s12 * my, qy = d.s12 * mx + d.s22 * my;
                    const float q0 = fmaxf(mx * qx + my * qy, 0.f);
                    const float dd = 0.25f * (d.s11 - d.s22) * (d.s11 - d.s22) + d.s12 * d.s12;
                    const float lam = fmaxf(0.5f * (d.s11 + d.s22) + dd * rsqrtf(fmaxf(dd, 1e-30f)), 0.f);
                    const float gap = q0 * rsqrtf(fmaxf(q0, 1e-30f)) -
                                      10.606601717798213f * lam * rsqrtf(fmaxf(lam, 1e-30f));
                    if (!(gap > 0.f && gap * gap > 1.01f * lim + 1e-2f)) {   // looser than any block test
                        v[0] = (lno - 0.5f * q0) * kLog2e;
                        v[1] = qx * kLog2e;
                        v[2] = qy * kLog2e;
                        v[3] = -0.5f * d.s11 * kLog2e;
                        v[4] = -d.s12 * kLog2e;
                        v[5] = -0.5f * d.s22 * kLog2e;
                        ia = __fdividef(1.f, d.s11);
                        ic = __fdividef(1.f, d.s22);
                    } else {
                        lim = -1.f;   // cannot reach the tile: no block test passes
                    }
                }
            }
            sP[3 * lane] = make_float4(mx, my, d.s11, d.s12);
            sP[3 * lane + 1] = make_float4(d.s22, lim, ia, ic);
            sP[3 * lane + 2] = make_float4(d.r, d.g, d.b, 0.f);
            if (kCC) {   // FP32 coefficients for the CUDA-core product; no FP16 operand
                float4* sV = reinterpret_cast<float4*>(smem + kSmemVf + buf * (kN * 32));
                sV[2 * lane] = make_float4(v[0], v[1], v[2], v[3]);
                sV[2 * lane + 1] = make_float4(v[4], v[5], 0.f, 0.f);
                return;
            }
            if (!global) {
#pragma unroll
                for (int k = 0; k < 6; ++k) v[k] = fminf(65504.f, fmaxf(-65504.f, v[k]));   // FP16-finite
            }
            uint32_t w[8];
            encode_row<true>(enc, v, w);
            store_row(smem + kSmemB + buf * kVBytes, lane, w);
            fence_async_smem();
        };
        // Consumer warps: which slots of buffer `buf` can reach alpha >= 1/255 somewhere in this
        // warp's 8 x 4 block (exact minimum of the conic form over the block's pixel centres).
        auto block_mask = [&](int buf) -> uint32_t {
            const float4* sP = reinterpret_cast<const float4*>(smem + kSmemP + buf * kPBytes);
            const float4 a = sP[3 * lane], b = sP[3 * lane + 1];
            bool act = b.y >= 0.f;
            if (act && p.tile_cull) act = min_q_box_facing(a.x, a.y, a.z, a.w, b.x, b.z, b.w, bx0, bx1, by0, by1) <= b.y;
            return __ballot_sync(0xffffffffu, act);
        };
        // Producer lane 0: both 128-row halves of U against the same V, committed to one mbarrier.
        auto issue_mma = [&](uint32_t k) {
            if (kCC) return;
            tc_fence_after();
            const int vb = (int)(k % 3u), tb = (int)(k & 1u);
            const uint64_t descB = make_desc(smem_u32(smem + kSmemB + vb * kVBytes));
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint64_t descA = make_desc(smem_u32(sA + h * 4096));
                const uint32_t dt = tmem + (uint32_t)(tb * 2 * kN + h * kN);
                if (enc == kEncTf32)
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dt),
                        "l"(descA), "l"(descB), "r"(kIdescTf32), "r"(0u)
                        : "memory");
                else if (enc == kEncFp8)
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(dt),
                        "l"(descA), "l"(descB), "r"(kIdescE4m3), "r"(0u)
                        : "memory");
                else
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dt),
                        "l"(descA), "l"(descB), "r"(kIdescF16), "r"(0u)
                        : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             mbar0 + 8u * (uint32_t)tb)
                         : "memory");
        };
        auto wait_mma = [&](uint32_t k) -> bool {   // producer lane 0, batches in order
            if (kCC) return true;
            const uint32_t tb = k & 1u;
            const bool ok = mbar_wait(mbar0 + 8u * tb, (phase_bits >> tb) & 1u);
            phase_bits ^= 1u << tb;
            return ok;
        };

        // producer registers: `nxt` holds the data of the batch to stage next, `nid` the ids after that
        Slot nxt;
        uint32_t nid = 0;
        auto prefetch = [&](uint32_t kb) {   // data of batch kb (ids already in nid), ids of batch kb + 1
            const uint32_t i = start + kb * kN + lane;
            nxt = load_slot(vd, p.opacity, nid, i < stop, !kInspect);
            const uint32_t i2 = i + kN;
            if (i2 < stop) nid = vd.ids[i2];
        };
        if (producer) {
            if (start + lane < stop) nid = vd.ids[start + lane];
            prefetch(0);
        }

        float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
        uint32_t last = 0, n_eval = end - start, n_blend = 0, cols = 0, walked = 0;
        // the second pixel (two a thread)
        float TB = 1.f, D0 = 0.f, D1 = 0.f, D2 = 0.f;
        uint32_t lastB = 0, n_evalB = end - start, n_blendB = 0;
        float thrB = insideB ? kBeta2Cull : kInf;
        bool done = !inside && !insideB;
        float thr = (k2 ? !inside : done) ? kInf : kBeta2Cull;
        uint32_t mask_cur = 0;

        // prologue: batches 0 and 1 staged, MMA 0 complete, MMA 1 issued, masks of batch 0 known
        if (nbat > 0) {
            if (producer) {
                stage(nxt, 0);
                if (nbat > 1) prefetch(1);
            }
            tc_fence_before();
            __syncthreads();
            if (producer) {
                if (lane == 0) issue_mma(0);
                if (nbat > 1) {
                    stage(nxt, 1);
                    if (nbat > 2) prefetch(2);
                }
                if (lane == 0 && !wait_mma(0)) s_timeout = 1;
            } else {
                mask_cur = block_mask(0);
            }
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            if (producer && lane == 0 && nbat > 1 && !s_timeout) issue_mma(1);
        }
        bool timed_out = nbat > 0 && s_timeout;
        for (uint32_t k = 0; k < nbat && !timed_out; ++k) {
            // window: consumers walk batch k while the producer stages batch k + 2 and waits for
            // MMA k + 1
            if (producer) {
                if (k + 2 < nbat) {
                    stage(nxt, (int)((k + 2) % 3u));
                    if (k + 3 < nbat) prefetch(k + 3);
                }
                if (lane == 0 && k + 1 < nbat && !wait_mma(k + 1)) s_timeout = 1;
            } else if (kInspect) {
                const uint32_t taddr = tmem + lane_base + (uint32_t)((k & 1u) * 2 * kN + half * kN);
                uint32_t r[32];
                tmem_ld32(taddr, r);
                tmem_wait_ld32(r);
                const uint32_t b0 = start + k * kN;
                const uint32_t nb = stop - b0 < (uint32_t)kN ? stop - b0 : (uint32_t)kN;
                const int pix = ly * kTile + lx;
                float* out = p.dbg_beta + ((size_t)blockIdx.x * 256 + pix) * p.dbg_max_n + (b0 - start);
#pragma unroll
                for (int j = 0; j < kN; ++j)
                    if ((uint32_t)j < nb) out[j] = __uint_as_float(r[j]) * 0.6931471805599453f;
            } else {
                // walk this warp's marked list entries, in list order
                const uint32_t b0 = start + k * kN;
                const uint32_t taddr = tmem + lane_base + (uint32_t)((k & 1u) * 2 * kN + half * kN);
                const float4* sP = reinterpret_cast<const float4*>(smem + kSmemP + (k % 3u) * kPBytes);
                uint32_t m = __all_sync(0xffffffffu, done) ? 0u : mask_cur;
                if (kStats) cols += __popc(m);
                const uint32_t pbase = b0 + 1u - start;   // 1 + list index of column 0
                while (m) {
                    const int j = __clz(__brev(m));   // lowest marked column
                    m &= m - 1;
                    float b2, b2B = 0.f;
                    if (kCC) {   // u^T v on CUDA cores, FP32 (broadcast shared-memory reads)
                        const float4* sV = reinterpret_cast<const float4*>(smem + kSmemVf + (k % 3u) * (kN * 32));
                        const float4 va = sV[2 * j], vb = sV[2 * j + 1];
                        b2 = fmaf(vb.y, uyy, fmaf(vb.x, uxy, fmaf(va.w, uxx, fmaf(va.z, uy, fmaf(va.y, ux, va.x)))));
                        if (k2)
                            b2B = fmaf(vb.y, uyyB, fmaf(vb.x, uxyB, fmaf(va.w, uxx, fmaf(va.z, uyB, fmaf(va.y, ux, va.x)))));
                    } else if (k2) {   // both halves' accumulators, one wait
                        uint32_t r = tmem_ld1(taddr + (uint32_t)j), rB = tmem_ld1(taddr + (uint32_t)(kN + j));
                        tmem_wait_ld2(r, rB);
                        b2 = __uint_as_float(r);
                        b2B = __uint_as_float(rB);
                    } else {
                        uint32_t r = tmem_ld1(taddr + (uint32_t)j);
                        tmem_wait_ld1(r);
                        b2 = __uint_as_float(r);
                    }
                    const float e = ex2_approx(b2);
                    // EarlyCull compares log2(alpha) with -log2(255); without it alpha itself is
                    // compared with 1/255 (thr is infinite once the pixel has terminated)
                    const bool pass = kEarly ? b2 >= thr : (e >= kCullAlpha && thr < kInf);
                    const float a = fminf(p.alpha_max, e);
                    const float Tn = fmaf(-a, T, T);
                    const bool term = pass && (Tn < kTmin);           // Algorithm 1: terminate, unblended
                    const bool blend = pass && !term;
                    const float4 c = sP[3 * j + 2];
                    // weight alpha T as the drop in transmittance (the weights then telescope to 1 - T)
                    const float Tb = blend ? Tn : T;
                    const float w = T - Tb;
                    C0 = fmaf(c.x, w, C0);
                    C1 = fmaf(c.y, w, C1);
                    C2 = fmaf(c.z, w, C2);
                    T = Tb;
                    const uint32_t pos = pbase + (uint32_t)j;
                    last = blend ? pos : last;
                    if (kStats) {
                        n_eval = term ? pos : n_eval;
                        n_blend += blend ? 1u : 0u;
                    }
                    thr = term ? kInf : thr;
                    if (k2) {   // the second pixel: the same steps
                        const float eB = ex2_approx(b2B);
                        const bool passB = kEarly ? b2B >= thrB : (eB >= kCullAlpha && thrB < kInf);
                        const float aB = fminf(p.alpha_max, eB);
                        const float TnB = fmaf(-aB, TB, TB);
                        const bool termB = passB && (TnB < kTmin);
                        const bool blendB = passB && !termB;
                        const float TbB = blendB ? TnB : TB;
                        const float wB = TB - TbB;
                        D0 = fmaf(c.x, wB, D0);
                        D1 = fmaf(c.y, wB, D1);
                        D2 = fmaf(c.z, wB, D2);
                        TB = TbB;
                        lastB = blendB ? pos : lastB;
                        if (kStats) {
                            n_evalB = termB ? pos : n_evalB;
                            n_blendB += blendB ? 1u : 0u;
                        }
                        thrB = termB ? kInf : thrB;
                    }
                }
                // terminated (thr starts infinite for pixels outside the image)
                done = k2 ? thr == kInf && thrB == kInf : thr == kInf;
                // marks of batch k + 1 (staged in the previous window, so stable during this one) before
                // the barrier: warps that finish early take this cost while the slowest one walks
                if (k + 1 < nbat)
                    mask_cur = __all_sync(0xffffffffu, done) ? 0u : block_mask((int)((k + 1) % 3u));
            }
            walked = (k + 1) * kN;
            tc_fence_before();
            const bool more = __syncthreads_or(!done);   // batch k walked, batch k+2 staged, MMA k+1 done
            tc_fence_after();
            if (s_timeout) {
                timed_out = true;
                break;
            }
            if (!kInspect && !more) break;
            if (producer && lane == 0 && k + 2 < nbat) issue_mma(k + 2);
        }
        // every MMA issued has been waited for (MMA k + 2 is only issued after the walk of batch k
        // continues, and is waited for in the next window), so TMEM is idle between tiles

        if (!kInspect) {
            if (inside) {
                size_t pix = (size_t)py_i * vd.cam.width + px_i;
                size_t plane = (size_t)vd.cam.width * vd.cam.height;
                vd.img[pix] = C0 + T * p.bg[0];
                vd.img[plane + pix] = C1 + T * p.bg[1];
                vd.img[2 * plane + pix] = C2 + T * p.bg[2];
                vd.T_final[pix] = T;
                vd.n_contrib[pix] = last;
            }
            if (insideB) {
                size_t pix = (size_t)(py_i + 4) * vd.cam.width + px_i;
                size_t plane = (size_t)vd.cam.width * vd.cam.height;
                vd.img[pix] = D0 + TB * p.bg[0];
                vd.img[plane + pix] = D1 + TB * p.bg[1];
                vd.img[2 * plane + pix] = D2 + TB * p.bg[2];
                vd.T_final[pix] = TB;
                vd.n_contrib[pix] = lastB;
            }
            if (kStats) {
                if (inside) {
                    atomicAdd(&s_acc[0], (unsigned long long)n_blend);
                    atomicAdd(&s_acc[1], (unsigned long long)(n_eval - n_blend));
                }
                if (insideB) {
                    atomicAdd(&s_acc[0], (unsigned long long)n_blendB);
                    atomicAdd(&s_acc[1], (unsigned long long)(n_evalB - n_blendB));
                }
                if (lane == 0 && !producer) atomicAdd(&s_acc[2], (unsigned long long)cols * (32ull * kPPT));
            }
        } else if (!producer) {
            const int pix = ly * kTile + lx;
            float* out = p.dbg_beta + ((size_t)blockIdx.x * 256 + pix) * p.dbg_max_n;
            for (int j = (int)(stop - start); j < p.dbg_max_n; ++j) out[j] = -kInf;
        }
        tc_fence_before();
        __syncthreads();
        if (kStats && t == 0 && tile_ok && vd.stats) {
            uint32_t* st = vd.stats + 8 * tile;
            atomicAdd(&st[0], (uint32_t)s_acc[0]);
            atomicAdd(&st[1], (uint32_t)s_acc[1]);
            atomicAdd(&st[2], (uint32_t)s_acc[2]);
            atomicAdd(&st[3], end - start);
            atomicAdd(&st[4], walked < end - start ? walked : end - start);
            atomicAdd(&st[5], (uint32_t)((clock64() - t_start) >> 6));
        }
        if (timed_out) {
            if (t == 0) set_status(p.status, TCGS_ERR_TIMEOUT);
            stopped = true;
            break;
        }
    }
    (void)stopped;
    tc_fence_before();
    __syncthreads();
    if (producer && !kCC) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// The work-queue counter is zeroed by a one-thread kernel rather than a memset, so that the
// launches on either side of it stay programmatic (a memset between two kernels would serialise them).
__global__ void k_zero_counter(uint32_t* c) {
    pdl_wait();
    *c = 0u;
}

void zero_counter(uint32_t* c, cudaStream_t s) {
    launch_pdl(k_zero_counter, 1, 1, 0, s, c);
    count_launches(1);
}

// The renderer's bounded mbarrier wait on a barrier that nothing completes: it must give up after
// `polls` polls and report TCGS_ERR_TIMEOUT, leaving the context usable.
__global__ void k_wait_selftest(int32_t* status, uint32_t polls) {
    __shared__ __align__(8) uint64_t bar;
    const uint32_t a = smem_u32(&bar);
    if (threadIdx.x == 0) mbar_init(a, 1);
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait(a, 0u, polls)) set_status(status, TCGS_ERR_TIMEOUT);
}

// The current device when it is an sm_103 part (sms = its SM count), else false.
bool device_is_sm103(int* sms = nullptr) {
    DeviceInfo d;
    if (!current_device_info(&d) || !d.sm103) return false;
    if (sms) *sms = d.sms;
    return true;
}

// Whether the dynamic shared memory size has been raised for an instance on a device (a flag per
// instance and device; function attributes are per device).
std::mutex g_attr_mutex;

template <bool kInspect, bool kStats, bool kQueue, bool kEarly, int kPath, int kPPT>
tcgs_status launch_tc_t(const TcParams& p, int blocks, cudaStream_t s) {
    static bool attr_set[kMaxDevices] = {};
    auto kern = k_render_tc<kInspect, kStats, kQueue, kEarly, kPath, kPPT>;
    DeviceInfo d;
    if (!current_device_info(&d)) return TCGS_ERR_CUDA;
    {
        std::lock_guard<std::mutex> lock(g_attr_mutex);
        if (!attr_set[d.device]) {
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemDyn) != cudaSuccess)
                return TCGS_ERR_CUDA;
            attr_set[d.device] = true;
        }
    }
    launch_pdl(kern, blocks, tc_threads<kPPT>(), kSmemDyn, s, p);
    count_launches(1);
    TCGS_CHECK_LAUNCH();
    return TCGS_OK;
}

// The cull test and the operand encoding sit in the per-fragment and per-batch paths, so the
// default configuration (EarlyCull, split encoding, G2L) is an instance of its own; the other
// encodings and the alpha-form cull test share generic instances.  The CUDA-core product has
// instances of its own, with and without EarlyCull.
template <bool kInspect, bool kStats, bool kQueue>
tcgs_status launch_tc(const TcParams& p, int blocks, cudaStream_t s) {
    if constexpr (kInspect) {
        return launch_tc_t<kInspect, kStats, kQueue, true, kPathGeneric, 1>(p, blocks, s);
    } else {
        const bool two = p.ppt == 2 && p.early_cull;
        if (p.cuda_core) {
            if (two) return launch_tc_t<kInspect, kStats, kQueue, true, kPathCudaCore, 2>(p, blocks, s);
            return p.early_cull ? launch_tc_t<kInspect, kStats, kQueue, true, kPathCudaCore, 1>(p, blocks, s)
                                : launch_tc_t<kInspect, kStats, kQueue, false, kPathCudaCore, 1>(p, blocks, s);
        }
        const bool split = p.enc == kEncF16Split && !p.global;
        if (!p.early_cull) return launch_tc_t<kInspect, kStats, kQueue, false, kPathGeneric, 1>(p, blocks, s);
        if (split)
            return two ? launch_tc_t<kInspect, kStats, kQueue, true, kPathSplit, 2>(p, blocks, s)
                       : launch_tc_t<kInspect, kStats, kQueue, true, kPathSplit, 1>(p, blocks, s);
        return launch_tc_t<kInspect, kStats, kQueue, true, kPathGeneric, 1>(p, blocks, s);
    }
}

ViewData make_view(const tcgs_camera* cam, const uint32_t* tile_ranges, const uint32_t* ids, const float* mean2d,
                   const float* conic, const float* rgb, float* img, float* T_final, uint32_t* n_contrib,
                   uint32_t* stats) {
    ViewData v;
    v.cam = make_dev_camera(*cam);
    v.ranges = tile_ranges; v.ids = ids; v.mean2d = mean2d; v.conic = conic; v.rgb = rgb;
    v.img = img; v.T_final = T_final; v.n_contrib = n_contrib; v.stats = stats;
    return v;
}

bool is_tc_precision(int precision) {
    return precision == TCGS_TC_FP16 || precision == TCGS_TC_FP16_SPLIT || precision == TCGS_TC_FP8 ||
           precision == TCGS_TC_TF32 || precision == TCGS_TC_FP16_GLOBAL || precision == TCGS_TC_TF32_GLOBAL;
}

// Precisions rendered by k_render_tc (per view or batched): the tensor-core ones and the same
// kernel with the product on CUDA cores.
bool uses_tile_kernel(int precision) { return is_tc_precision(precision) || precision == TCGS_FP32_FRAG2MAT; }

bool is_global_precision(int precision) {
    return precision == TCGS_TC_FP16_GLOBAL || precision == TCGS_TC_TF32_GLOBAL;
}

TcParams base_params(int precision, const float* opacity) {
    TcParams p;
    memset(&p, 0, sizeof(p));
    p.opacity = opacity;
    switch (precision) {
        case TCGS_TC_FP16_SPLIT: p.enc = kEncF16Split; break;
        case TCGS_TC_TF32:
        case TCGS_TC_TF32_GLOBAL: p.enc = kEncTf32; break;
        case TCGS_TC_FP8: p.enc = kEncFp8; break;
        default: p.enc = kEncF16Pad; break;   // TC_FP16, TC_FP16_GLOBAL
    }
    p.global = is_global_precision(precision) ? 1 : 0;
    p.cuda_core = precision == TCGS_FP32_FRAG2MAT ? 1 : 0;
    p.alpha_max = 0.99f;
    p.tile_cull = 1;
    p.early_cull = 1;
    return p;
}

}  // namespace

tcgs_status launch_render_tc(const tcgs_camera* cam, const tcgs_render_opts* opts, const uint32_t* tile_ranges,
                             const uint32_t* ids_sorted, const float* mean2d, const float* conic,
                             const float* opacity, const float* rgb, const float* bg3, float* img, float* T_final,
                             uint32_t* n_contrib, cudaStream_t s) {
    int sms = 0;
    if (!device_is_sm103(&sms)) return TCGS_ERR_UNSUPPORTED;
    TcParams p = base_params(opts->precision, opacity);
    p.v[0] = make_view(cam, tile_ranges, ids_sorted, mean2d, conic, rgb, img, T_final, n_contrib, opts->tile_stats);
    p.n_views = 1;
    for (int i = 0; i < 3; ++i) p.bg[i] = bg3 ? bg3[i] : 0.f;
    p.alpha_max = opts->alpha_max;
    p.status = opts->device_status;
    p.tile_cull = p.global ? 0 : opts->tile_cull;   // the ablation walks every entry
    p.early_cull = opts->early_cull;
    if (opts->pixels_per_thread < 0 || opts->pixels_per_thread > 2) return TCGS_ERR_INVALID;
    p.ppt = opts->pixels_per_thread == 2 ? 2 : 1;
    const int tiles = p.v[0].cam.grid_w * p.v[0].cam.grid_h;
    if (opts->tile_order && !opts->work_counter) return TCGS_ERR_INVALID;
    if (opts->tile_order && !p.global && tiles > sms * kTcCtasPerSm) {
        // persistent grid over the tiles in the given order: each CTA allocates TMEM and builds U
        // once, and the longest lists start first (with at most one wave of tiles every tile starts
        // at once, so the plain grid below runs without the counter's reset)
        p.queue = opts->tile_order;
        p.queue_tiles = 1;
        p.n_items = (uint32_t)tiles;
        p.counter = opts->work_counter;
        zero_counter(opts->work_counter, s);
        int ctas = sms * kTcCtasPerSm;
        if (ctas > tiles) ctas = tiles;
        return opts->tile_stats ? launch_tc<false, true, true>(p, ctas, s) : launch_tc<false, false, true>(p, ctas, s);
    }
    return opts->tile_stats ? launch_tc<false, true, false>(p, tiles, s) : launch_tc<false, false, false>(p, tiles, s);
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
        case TCGS_TC_FP8:
        case TCGS_TC_TF32:
        case TCGS_TC_FP16_GLOBAL:
        case TCGS_TC_TF32_GLOBAL:
        case TCGS_FP32_FRAG2MAT:
            return launch_render_tc(cam, opts, tile_ranges, ids_sorted, mean2d, conic, opacity, rgb, bg3, img,
                                    T_final, n_contrib, s);
        default:
            return TCGS_ERR_INVALID;
    }
}

extern "C" tcgs_status tcgs_render_fwd_batched(int32_t n_views, const tcgs_view* views, const tcgs_render_opts* opts,
                                               const float* opacity, const float* bg3, const uint32_t* queue,
                                               int32_t n_items, uint32_t* work_counter, int32_t max_ctas,
                                               tcgs_stream stream) {
    using namespace tcgs;
    if (n_views < 1 || n_views > TCGS_MAX_VIEWS || !views || !opts || !opacity || n_items < 0 ||
        (n_items > 0 && (!queue || !work_counter)))
        return TCGS_ERR_INVALID;
    if (!uses_tile_kernel(opts->precision) || is_global_precision(opts->precision)) return TCGS_ERR_INVALID;
    if (!(opts->alpha_max > 0.f && opts->alpha_max <= 1.f)) return TCGS_ERR_INVALID;
    TcParams p = base_params(opts->precision, opacity);
    for (int v = 0; v < n_views; ++v) {
        const tcgs_view& w = views[v];
        if (!valid_camera(&w.cam) || !w.tile_ranges || !w.ids_sorted || !w.mean2d || !w.conic || !w.rgb || !w.img ||
            !w.T_final || !w.n_contrib || (reinterpret_cast<uintptr_t>(w.mean2d) & 7))
            return TCGS_ERR_INVALID;
        const int gw = (w.cam.width + kTile - 1) / kTile, gh = (w.cam.height + kTile - 1) / kTile;
        if (gw * gh > 65536) return TCGS_ERR_INVALID;   // items carry the tile in 16 bits
        p.v[v] = make_view(&w.cam, w.tile_ranges, w.ids_sorted, w.mean2d, w.conic, w.rgb, w.img, w.T_final,
                           w.n_contrib, w.tile_stats);
    }
    p.n_views = n_views;
    if (n_items == 0) return TCGS_OK;
    int sms = 0;
    if (!device_is_sm103(&sms)) return TCGS_ERR_UNSUPPORTED;
    for (int i = 0; i < 3; ++i) p.bg[i] = bg3 ? bg3[i] : 0.f;
    p.alpha_max = opts->alpha_max;
    p.status = opts->device_status;
    p.tile_cull = opts->tile_cull;
    p.early_cull = opts->early_cull;
    p.queue = queue;
    p.n_items = (uint32_t)n_items;
    p.counter = work_counter;
    cudaStream_t s = (cudaStream_t)stream;
    zero_counter(work_counter, s);
    bool any_stats = false;
    for (int v = 0; v < n_views; ++v) any_stats = any_stats || views[v].tile_stats;
    // persistent grid: at most the CTAs that are resident at once (4 per SM for this kernel)
    int ctas = sms * kTcCtasPerSm;
    if (max_ctas > 0 && max_ctas < ctas) ctas = max_ctas;
    if (ctas > n_items) ctas = n_items;
    return any_stats ? launch_tc<false, true, true>(p, ctas, s) : launch_tc<false, false, true>(p, ctas, s);
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
    if (!is_tc_precision(precision)) return TCGS_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(mean2d) & 7) return TCGS_ERR_INVALID;
    if (n_tiles == 0 || max_n == 0) return TCGS_OK;
    if (!device_is_sm103()) return TCGS_ERR_UNSUPPORTED;
    TcParams p = base_params(precision, opacity);
    p.v[0] = make_view(cam, tile_ranges, ids_sorted, mean2d, conic, nullptr, nullptr, nullptr, nullptr, nullptr);
    p.n_views = 1;
    p.status = device_status;
    p.dbg_tiles = tiles; p.dbg_max_n = max_n; p.dbg_beta = beta_out;
    return launch_tc<true, false, false>(p, n_tiles, (cudaStream_t)stream);
}

extern "C" int32_t tcgs_tc_wave_tiles(void) {
    using namespace tcgs;
    int sms = 0;
    return device_is_sm103(&sms) ? sms * kTcCtasPerSm : 0;
}

extern "C" tcgs_status tcgs_selftest_bounded_wait(int32_t* device_status, uint32_t polls, tcgs_stream stream) {
    using namespace tcgs;
    if (!device_status || polls == 0 || polls > (1u << 22)) return TCGS_ERR_INVALID;
    if (!device_is_sm103()) return TCGS_ERR_UNSUPPORTED;
    k_wait_selftest<<<1, 32, 0, (cudaStream_t)stream>>>(device_status, polls);
    count_launches(1);
    TCGS_CHECK_LAUNCH();
    return TCGS_OK;
}
