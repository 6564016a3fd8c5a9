// common.cuh -- shared device helpers of libtcgs (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "tcgs.h"

namespace tcgs {

constexpr int kTile = 16;            // tile edge in pixels (Sec. 4.3: 16 x 16 tiles)
constexpr float kCullAlpha = 1.0f / 255.0f;   // Eq. (5)
constexpr float kTmin = 1e-4f;       // termination threshold of Algorithm 1
constexpr float kLog2e = 1.4426950408889634f;
// -ln(255) (EarlyCull, Sec. 4.1) and the same threshold in log2 units
constexpr float kBetaCull = -5.541263545158426f;
constexpr float kBeta2Cull = -7.994353436858858f;   // -log2(255)

struct DevCamera {
    int width, height, grid_w, grid_h;
    float fx, fy, cx, cy;
    float R[9], t[3];
    float campos[3];
    float near_z, limx, limy;
};

inline DevCamera make_dev_camera(const tcgs_camera& c) {
    DevCamera d;
    d.width = c.width;
    d.height = c.height;
    d.grid_w = (c.width + kTile - 1) / kTile;
    d.grid_h = (c.height + kTile - 1) / kTile;
    d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy;
    for (int i = 0; i < 3; ++i) {
        for (int k = 0; k < 3; ++k) d.R[3 * i + k] = c.viewmat[4 * i + k];
        d.t[i] = c.viewmat[4 * i + 3];
        d.campos[i] = c.campos[i];
    }
    d.near_z = c.near_z;
    float tx = c.tan_fovx > 0.f ? c.tan_fovx : 0.5f * (float)c.width / c.fx;
    float ty = c.tan_fovy > 0.f ? c.tan_fovy : 0.5f * (float)c.height / c.fy;
    d.limx = 1.3f * tx;
    d.limy = 1.3f * ty;
    return d;
}

inline bool valid_camera(const tcgs_camera* c) {
    return c && c->width > 0 && c->height > 0 && c->fx > 0.f && c->fy > 0.f && c->width <= (1 << 20) &&
           c->height <= (1 << 20);
}

// Tile rectangle of a projected Gaussian, exact for any finite float mean and integer radius:
// x tiles [floor((mx - r) / 16), floor((mx + r) / 16)] clipped to the grid.  floor(mx) is exact
// in float, so floor((mx -+ r) / 16) = floor_div(floor(mx) -+ r, 16) in 64-bit integers.
struct Rect { int x0, x1, y0, y1; };   // inclusive bounds; empty when x1 < x0 or y1 < y0

__device__ __forceinline__ long long floor_div16(long long v) { return v >= 0 ? v / 16 : -((-v + 15) / 16); }

__device__ __forceinline__ Rect tile_rect(float mx, float my, int r, int gw, int gh) {
    Rect o;
    const float lim = 4.0e18f;
    if (!(fabsf(mx) < lim) || !(fabsf(my) < lim) || r <= 0) { o.x0 = o.y0 = 0; o.x1 = o.y1 = -1; return o; }
    long long fx = (long long)floorf(mx), fy = (long long)floorf(my);
    long long lx = floor_div16(fx - r), hx = floor_div16(fx + r);
    long long ly = floor_div16(fy - r), hy = floor_div16(fy + r);
    lx = lx < 0 ? 0 : lx; ly = ly < 0 ? 0 : ly;
    hx = hx > gw - 1 ? gw - 1 : hx; hy = hy > gh - 1 ? gh - 1 : hy;
    if (hx < lx || hy < ly) { o.x0 = o.y0 = 0; o.x1 = o.y1 = -1; return o; }
    o.x0 = (int)lx; o.x1 = (int)hx; o.y0 = (int)ly; o.y1 = (int)hy;
    return o;
}

__device__ __forceinline__ uint32_t rect_count(const Rect& r) {
    if (r.x1 < r.x0 || r.y1 < r.y0) return 0u;
    return (uint32_t)(r.x1 - r.x0 + 1) * (uint32_t)(r.y1 - r.y0 + 1);
}

// Smallest value of q(p) = (m - p)^T Q (m - p) over the rectangle [x0, x1] x [y0, y1] of pixel
// centres, Q = [[a, b], [b, c]] positive definite, with ia = 1/a and ic = 1/c precomputed: 0 when m
// is inside; otherwise it lies on an edge facing m -- a vertical edge when m is left or right of the
// rectangle, a horizontal one when m is above or below (the edges facing away cannot hold the
// minimum of a convex form whose minimiser lies beyond the opposite side) -- where the form is a 1-D
// convex quadratic minimised at its clamped stationary point.
__device__ __forceinline__ float min_q_box_facing(float mx, float my, float a, float b, float c, float ia, float ic,
                                                  float x0, float x1, float y0, float y1) {
    const bool lx = mx < x0, hx = mx > x1, ly = my < y0, hy = my > y1;
    if (!(lx || hx || ly || hy)) return 0.f;
    float best = __int_as_float(0x7f800000);
    if (lx || hx) {
        const float X = lx ? x0 : x1;
        const float dx = mx - X;
        const float y = fminf(y1, fmaxf(y0, my + b * dx * ic));
        const float dy = my - y;
        best = fminf(best, a * dx * dx + 2.f * b * dx * dy + c * dy * dy);
    }
    if (ly || hy) {
        const float Y = ly ? y0 : y1;
        const float ey = my - Y;
        const float x = fminf(x1, fmaxf(x0, mx + b * ey * ia));
        const float ex = mx - x;
        best = fminf(best, a * ex * ex + 2.f * b * ex * ey + c * ey * ey);
    }
    return best;
}

// Reach limit of a Gaussian with ln-opacity lno: alpha = o exp(-q/2) >= 1/255 (Eq. 5) needs
// q <= 2 (ln o + ln 255).  The relative and absolute margins keep every test built on it (the TC
// renderer's block marks, the exact tile coverage of the sorting stage) conservative under FP32
// rounding; -1 when no q qualifies.
__device__ __forceinline__ float reach_limit(float lno) {
    const float reach = 2.f * (lno - kBetaCull);
    return reach > -1e-3f ? reach * 1.0001f + 1e-3f : -1.f;
}

// 2^x on the SFU (PTX ex2.approx.ftz.f32).
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Programmatic dependent launch: a kernel started with launch_pdl may be scheduled while the kernel
// before it in the stream drains; it calls pdl_wait() before its first global memory access, which
// returns once that kernel has completed and its writes are visible (at once after a plain launch).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Lets the next kernel in the stream be scheduled now rather than when this block exits (for
// kernels whose blocks all fit on the GPU at once, so early arrivals take no slot they need).
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

__device__ __forceinline__ void set_status(int32_t* st, int code) {
    if (st) atomicCAS(st, 0, code);
}

}  // namespace tcgs

namespace tcgs {
// host-side count of kernel launches (tcgs_kernel_launches)
void count_launches(unsigned n);

// Properties of the current device, looked up once per device (thread-safe).  Returns false when no
// device is current or its index is beyond kMaxDevices.
constexpr int kMaxDevices = 64;
struct DeviceInfo {
    int device;   // index of the current device
    int sms;      // streaming multiprocessors
    bool sm103;   // compute capability 10.3 (the tensor-core paths need sm_103a)
};
bool current_device_info(DeviceInfo* out);
}

#define TCGS_CHECK_LAUNCH()                                  \
    do {                                                     \
        cudaError_t e_ = cudaGetLastError();                 \
        if (e_ != cudaSuccess) return TCGS_ERR_CUDA;         \
    } while (0)
