// project.cu -- preprocess stage (Sec. 3.1, Eq. 2): EWA projection of 3D Gaussians.
//
// One thread per Gaussian; the stage is HBM bound (read ~40 B + the SH coefficients,
// write 44 B per Gaussian).  SH degree-3 coefficients (192 B per Gaussian) are staged per warp:
// the warp's 32 rows (6 KB, contiguous) are loaded with coalesced 16-byte loads into shared memory,
// then each thread reads its own row.
#include "common.cuh"

namespace tcgs {
namespace {

// Real SH normalisation constants sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) times Legendre factors.
constexpr float kY00 = 0.28209479177387814f;   // 1/2 sqrt(1/pi)
constexpr float kY1 = 0.4886025119029199f;     // sqrt(3/(4 pi))
constexpr float kY2a = 1.0925484305920792f;    // 1/2 sqrt(15/pi)
constexpr float kY20 = 0.31539156525252005f;   // 1/4 sqrt(5/pi)
constexpr float kY22 = 0.5462742152960396f;    // 1/4 sqrt(15/pi)
constexpr float kY33 = 0.5900435899266435f;    // 1/4 sqrt(35/(2 pi))
constexpr float kY32 = 2.890611442640554f;     // 1/2 sqrt(105/pi)
constexpr float kY31 = 0.4570457994644658f;    // 1/4 sqrt(21/(2 pi))
constexpr float kY30 = 0.3731763325901154f;    // 1/4 sqrt(7/pi)
constexpr float kY32b = 1.445305721320277f;    // 1/4 sqrt(105/pi)

__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float* Y) {
    Y[0] = kY00;
    if (deg < 1) return;
    Y[1] = -kY1 * y; Y[2] = kY1 * z; Y[3] = -kY1 * x;
    if (deg < 2) return;
    float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = kY2a * x * y; Y[5] = -kY2a * y * z; Y[6] = kY20 * (2.f * zz - xx - yy);
    Y[7] = -kY2a * x * z; Y[8] = kY22 * (xx - yy);
    if (deg < 3) return;
    Y[9] = -kY33 * y * (3.f * xx - yy);
    Y[10] = kY32 * x * y * z;
    Y[11] = -kY31 * y * (4.f * zz - xx - yy);
    Y[12] = kY30 * z * (2.f * zz - 3.f * xx - 3.f * yy);
    Y[13] = -kY31 * x * (4.f * zz - xx - yy);
    Y[14] = kY32b * z * (xx - yy);
    Y[15] = -kY33 * x * (xx - 3.f * yy);
}

constexpr int kProjThreads = 128;
constexpr int kShRow4 = 13;   // float4 slots per staged SH row: 12 used; the odd stride keeps a row's
                              // 16-byte reads by 8 consecutive threads in distinct bank groups

template <bool kStageSh>
__global__ void __launch_bounds__(kProjThreads) k_project(DevCamera cam, int P, int deg,
                                                          const float* __restrict__ means3,
                                                          const float* __restrict__ scales,
                                                          const float* __restrict__ quats,
                                                          const float* __restrict__ sh,
                                                          const float* __restrict__ opacity,
                                                          float* __restrict__ mean2d,
                                                          float* __restrict__ conic, float* __restrict__ depth,
                                                          int32_t* __restrict__ radius, float* __restrict__ rgb,
                                                          uint32_t* __restrict__ tiles_touched) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    __shared__ float4 s_sh[kStageSh ? kProjThreads / 32 : 1][kStageSh ? 32 * kShRow4 : 1];
    if (kStageSh) {
        // the warp's degree-3 rows, coalesced, copied asynchronously (no registers held): float4 i
        // of the warp's block goes to row i / 12
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int g0 = g - lane;
        const int rows = P - g0 < 32 ? P - g0 : 32;
        if (rows > 0) {
            const float4* src = reinterpret_cast<const float4*>(sh) + (size_t)g0 * 12;
#pragma unroll
            for (int m = 0; m < 12; ++m) {
                const int i = lane + 32 * m;
                if (i < 12 * rows) {
                    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&s_sh[warp][(i / 12) * kShRow4 + i % 12]);
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src + i) : "memory");
                }
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    // every other input of this Gaussian is requested before the staged rows are waited for
    float m0 = 0.f, m1 = 0.f, m2 = 0.f, s0 = 0.f, s1 = 0.f, s2 = 0.f, op = 1.f;
    float4 q = make_float4(1.f, 0.f, 0.f, 0.f);
    if (g < P) {
        m0 = means3[3 * g]; m1 = means3[3 * g + 1]; m2 = means3[3 * g + 2];
        q = *reinterpret_cast<const float4*>(quats + 4 * (size_t)g);
        s0 = scales[3 * g]; s1 = scales[3 * g + 1]; s2 = scales[3 * g + 2];
        if (opacity) op = opacity[g];
    }
    if (kStageSh) {
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncwarp();
    }
    if (g >= P) return;
    // camera-space mean t = W mu
    float tx = cam.R[0] * m0 + cam.R[1] * m1 + cam.R[2] * m2 + cam.t[0];
    float ty = cam.R[3] * m0 + cam.R[4] * m1 + cam.R[5] * m2 + cam.t[1];
    float tz = cam.R[6] * m0 + cam.R[7] * m1 + cam.R[8] * m2 + cam.t[2];

    float o_mx = 0.f, o_my = 0.f, o_c0 = 0.f, o_c1 = 0.f, o_c2 = 0.f, o_z = 0.f;
    float o_r = 0.f, o_g = 0.f, o_b = 0.f;
    int32_t o_rad = 0;
    uint32_t o_tiles = 0;

    if (tz > cam.near_z) {
        // Sigma = M M^T with M = R(q) diag(s)
        float qn = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
        float w = q.x * qn, x = q.y * qn, y = q.z * qn, z = q.w * qn;
        float Rq[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                       2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                       2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
        float M[9];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            M[3 * i] = Rq[3 * i] * s0;
            M[3 * i + 1] = Rq[3 * i + 1] * s1;
            M[3 * i + 2] = Rq[3 * i + 2] * s2;
        }
        // Jacobian rows at the frustum-clamped mean; T = J W (2x3)
        float xc = fminf(cam.limx, fmaxf(-cam.limx, tx / tz)) * tz;
        float yc = fminf(cam.limy, fmaxf(-cam.limy, ty / tz)) * tz;
        float iz = 1.f / tz;
        float j00 = cam.fx * iz, j02 = -cam.fx * xc * iz * iz;
        float j11 = cam.fy * iz, j12 = -cam.fy * yc * iz * iz;
        float T0[3], T1[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            T0[k] = j00 * cam.R[k] + j02 * cam.R[6 + k];
            T1[k] = j11 * cam.R[3 + k] + j12 * cam.R[6 + k];
        }
        // A = T M (2x3); Sigma' = A A^T
        float A0[3], A1[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            A0[k] = T0[0] * M[k] + T0[1] * M[3 + k] + T0[2] * M[6 + k];
            A1[k] = T1[0] * M[k] + T1[1] * M[3 + k] + T1[2] * M[6 + k];
        }
        float a = A0[0] * A0[0] + A0[1] * A0[1] + A0[2] * A0[2] + 0.3f;
        float b = A0[0] * A1[0] + A0[1] * A1[1] + A0[2] * A1[2];
        float c = A1[0] * A1[0] + A1[1] * A1[1] + A1[2] * A1[2] + 0.3f;
        float det = a * c - b * b;
        // squared reach in units of sigma: 9 for the 3-sigma square, 2 ln(255 o) for the square
        // bounding the ellipse where alpha >= 1/255 (Eq. 5); o <= 1/255 reaches no pixel
        const float reach2 = opacity ? 2.f * logf(255.f * op) : 9.f;
        if (det > 0.f && reach2 > 0.f) {
            float mid = 0.5f * (a + c);
            float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - det));
            float rf = ceilf(sqrtf(reach2 * lam));
            int32_t r = rf < 1.0e9f ? (int32_t)rf : 1000000000;
            float mx = cam.fx * tx * iz + cam.cx;
            float my = cam.fy * ty * iz + cam.cy;
            Rect rc = tile_rect(mx, my, r, cam.grid_w, cam.grid_h);
            uint32_t nt = rect_count(rc);
            if (nt > 0) {
                float idet = 1.f / det;
                o_mx = mx; o_my = my;
                o_c0 = c * idet; o_c1 = -b * idet; o_c2 = a * idet;
                o_z = tz; o_rad = r; o_tiles = nt;
                // colour from SH at the view direction
                float dx = m0 - cam.campos[0], dy = m1 - cam.campos[1], dz = m2 - cam.campos[2];
                float dn = rsqrtf(dx * dx + dy * dy + dz * dz);
                float Y[16];
                sh_basis(kStageSh ? 3 : deg, dx * dn, dy * dn, dz * dn, Y);   // staged rows are degree 3
                int K = (deg + 1) * (deg + 1);
                float cr = 0.5f, cg = 0.5f, cb = 0.5f;
                const float* s = sh + (size_t)g * K * 3;
                if (kStageSh || deg == 3) {
                    const float4* s4 = kStageSh ? &s_sh[threadIdx.x >> 5][(threadIdx.x & 31) * kShRow4]
                                                : reinterpret_cast<const float4*>(s);
                    float v[48];
#pragma unroll
                    for (int i = 0; i < 12; ++i) {
                        float4 t4 = s4[i];
                        v[4 * i] = t4.x; v[4 * i + 1] = t4.y; v[4 * i + 2] = t4.z; v[4 * i + 3] = t4.w;
                    }
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        cr += Y[k] * v[3 * k]; cg += Y[k] * v[3 * k + 1]; cb += Y[k] * v[3 * k + 2];
                    }
                } else {
                    for (int k = 0; k < K; ++k) {
                        cr += Y[k] * s[3 * k]; cg += Y[k] * s[3 * k + 1]; cb += Y[k] * s[3 * k + 2];
                    }
                }
                o_r = fmaxf(cr, 0.f); o_g = fmaxf(cg, 0.f); o_b = fmaxf(cb, 0.f);
            }
        }
    }
    reinterpret_cast<float2*>(mean2d)[g] = make_float2(o_mx, o_my);
    conic[3 * g] = o_c0; conic[3 * g + 1] = o_c1; conic[3 * g + 2] = o_c2;
    depth[g] = o_z;
    radius[g] = o_rad;
    rgb[3 * g] = o_r; rgb[3 * g + 1] = o_g; rgb[3 * g + 2] = o_b;
    tiles_touched[g] = o_tiles;
}

// d Y_k / d(x, y, z) of sh_basis at a unit direction (the polynomials above differentiated).
__device__ __forceinline__ void sh_basis_grad(int deg, float x, float y, float z, float (*dY)[3]) {
#pragma unroll
    for (int k = 0; k < 16; ++k) dY[k][0] = dY[k][1] = dY[k][2] = 0.f;
    if (deg < 1) return;
    dY[1][1] = -kY1; dY[2][2] = kY1; dY[3][0] = -kY1;
    if (deg < 2) return;
    dY[4][0] = kY2a * y;        dY[4][1] = kY2a * x;
    dY[5][1] = -kY2a * z;       dY[5][2] = -kY2a * y;
    dY[6][0] = -2.f * kY20 * x; dY[6][1] = -2.f * kY20 * y; dY[6][2] = 4.f * kY20 * z;
    dY[7][0] = -kY2a * z;       dY[7][2] = -kY2a * x;
    dY[8][0] = 2.f * kY22 * x;  dY[8][1] = -2.f * kY22 * y;
    if (deg < 3) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    dY[9][0] = -6.f * kY33 * x * y;       dY[9][1] = -3.f * kY33 * (xx - yy);
    dY[10][0] = kY32 * y * z;             dY[10][1] = kY32 * x * z;       dY[10][2] = kY32 * x * y;
    dY[11][0] = 2.f * kY31 * x * y;       dY[11][1] = -kY31 * (4.f * zz - xx - 3.f * yy);
    dY[11][2] = -8.f * kY31 * y * z;
    dY[12][0] = -6.f * kY30 * x * z;      dY[12][1] = -6.f * kY30 * y * z;
    dY[12][2] = kY30 * (6.f * zz - 3.f * xx - 3.f * yy);
    dY[13][0] = -kY31 * (4.f * zz - 3.f * xx - yy);   dY[13][1] = 2.f * kY31 * x * y;
    dY[13][2] = -8.f * kY31 * x * z;
    dY[14][0] = 2.f * kY32b * x * z;      dY[14][1] = -2.f * kY32b * y * z;   dY[14][2] = kY32b * (xx - yy);
    dY[15][0] = -3.f * kY33 * (xx - yy);  dY[15][1] = 6.f * kY33 * x * y;
}

// Backward of k_project for one Gaussian per thread: the forward's steps recomputed and
// differentiated in reverse (conic inverse, Sigma' = T Sigma T^T, T = J W, J and mean2d of the
// camera-space mean with the frustum clamp, Sigma = M M^T, M = R(q/|q|) diag(s), the SH colour and
// its view direction).  Gradients are accumulated (+=).  The SH degree is a template parameter so
// that the basis and its gradient stay in registers.
template <int kDeg>
__global__ void __launch_bounds__(256) k_project_bwd(DevCamera cam, int P, const float* __restrict__ means3,
                                                     const float* __restrict__ scales,
                                                     const float* __restrict__ quats, const float* __restrict__ sh,
                                                     const int32_t* __restrict__ radius,
                                                     const float* __restrict__ dmean2d,
                                                     const float* __restrict__ dconic,
                                                     const float* __restrict__ drgb, float* __restrict__ dmeans3,
                                                     float* __restrict__ dscales, float* __restrict__ dquats,
                                                     float* __restrict__ dsh) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= P || radius[g] <= 0) return;
    const float m0 = means3[3 * g], m1 = means3[3 * g + 1], m2 = means3[3 * g + 2];
    const float tx = cam.R[0] * m0 + cam.R[1] * m1 + cam.R[2] * m2 + cam.t[0];
    const float ty = cam.R[3] * m0 + cam.R[4] * m1 + cam.R[5] * m2 + cam.t[1];
    const float tz = cam.R[6] * m0 + cam.R[7] * m1 + cam.R[8] * m2 + cam.t[2];
    const float4 q = *reinterpret_cast<const float4*>(quats + 4 * (size_t)g);
    const float qn2 = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
    const float iqn = rsqrtf(qn2);
    const float w = q.x * iqn, x = q.y * iqn, y = q.z * iqn, z = q.w * iqn;
    const float s[3] = {scales[3 * g], scales[3 * g + 1], scales[3 * g + 2]};
    const float Rq[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                         2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                         2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
    float M[9], S3[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) M[3 * i + k] = Rq[3 * i + k] * s[k];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) S3[3 * i + k] = M[3 * i] * M[3 * k] + M[3 * i + 1] * M[3 * k + 1] + M[3 * i + 2] * M[3 * k + 2];
    const float iz = 1.f / tz;
    const float u = tx * iz, v = ty * iz;
    const float cu = fminf(cam.limx, fmaxf(-cam.limx, u)), cv = fminf(cam.limy, fmaxf(-cam.limy, v));
    const float du = (u > -cam.limx && u < cam.limx) ? 1.f : 0.f, dv = (v > -cam.limy && v < cam.limy) ? 1.f : 0.f;
    const float J[6] = {cam.fx * iz, 0.f, -cam.fx * cu * iz, 0.f, cam.fy * iz, -cam.fy * cv * iz};
    float T[6];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) T[3 * i + k] = J[3 * i] * cam.R[k] + J[3 * i + 1] * cam.R[3 + k] + J[3 * i + 2] * cam.R[6 + k];
    float TS[6];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) TS[3 * i + k] = T[3 * i] * S3[k] + T[3 * i + 1] * S3[3 + k] + T[3 * i + 2] * S3[6 + k];
    const float A = TS[0] * T[0] + TS[1] * T[1] + TS[2] * T[2] + 0.3f;
    const float B = TS[0] * T[3] + TS[1] * T[4] + TS[2] * T[5];
    const float C = TS[3] * T[3] + TS[4] * T[4] + TS[5] * T[5] + 0.3f;
    const float idet = 1.f / (A * C - B * B);
    const float Q[4] = {C * idet, -B * idet, -B * idet, A * idet};

    // conic -> Sigma': H = dL/dSigma' = -Q G Q, G the symmetric matrix of dconic
    const float G[4] = {dconic[3 * g], 0.5f * dconic[3 * g + 1], 0.5f * dconic[3 * g + 1], dconic[3 * g + 2]};
    float QG[4], H[4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int k = 0; k < 2; ++k) QG[2 * i + k] = Q[2 * i] * G[k] + Q[2 * i + 1] * G[2 + k];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int k = 0; k < 2; ++k) H[2 * i + k] = -(QG[2 * i] * Q[k] + QG[2 * i + 1] * Q[2 + k]);
    // Sigma' = T Sigma T^T: dL/dT = 2 H T Sigma, dL/dSigma = T^T H T
    float dT[6], dS[9];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) dT[3 * i + k] = 2.f * (H[2 * i] * TS[k] + H[2 * i + 1] * TS[3 + k]);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            dS[3 * i + k] = T[i] * (H[0] * T[k] + H[1] * T[3 + k]) + T[3 + i] * (H[2] * T[k] + H[3] * T[3 + k]);
    // T = J W: dL/dJ = dL/dT W^T
    float dJ[6];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            dJ[3 * i + k] = dT[3 * i] * cam.R[3 * k] + dT[3 * i + 1] * cam.R[3 * k + 1] + dT[3 * i + 2] * cam.R[3 * k + 2];
    // J(t) and mean2d(t) -> dL/dt -> dL/dmu = W^T dL/dt
    const float dmx = dmean2d[2 * g], dmy = dmean2d[2 * g + 1];
    const float iz2 = iz * iz, iz3 = iz2 * iz;
    const float dtx = cam.fx * iz * dmx - dJ[2] * cam.fx * du * iz2;
    const float dty = cam.fy * iz * dmy - dJ[5] * cam.fy * dv * iz2;
    const float dtz = -cam.fx * tx * iz2 * dmx - cam.fy * ty * iz2 * dmy - dJ[0] * cam.fx * iz2 - dJ[4] * cam.fy * iz2 +
                      dJ[2] * cam.fx * (du * tx * iz3 + cu * iz2) + dJ[5] * cam.fy * (dv * ty * iz3 + cv * iz2);
    float dmu[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) dmu[k] = cam.R[k] * dtx + cam.R[3 + k] * dty + cam.R[6 + k] * dtz;
    // Sigma = M M^T: dL/dM = (dS + dS^T) M; M = R diag(s)
    float dR[9], ds[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float acc = 0.f;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            float dm = 0.f;
#pragma unroll
            for (int l = 0; l < 3; ++l) dm += (dS[3 * i + l] + dS[3 * l + i]) * M[3 * l + k];
            acc += dm * Rq[3 * i + k];
            dR[3 * i + k] = dm * s[k];
        }
        ds[k] = acc;
    }
    // R of the unit quaternion (w, x, y, z), then the normalisation q / |q|
    float dqn[4];
    dqn[0] = 2.f * (-dR[1] * z + dR[2] * y + dR[3] * z - dR[5] * x - dR[6] * y + dR[7] * x);
    dqn[1] = 2.f * (dR[1] * y + dR[2] * z + dR[3] * y - 2.f * dR[4] * x - dR[5] * w + dR[6] * z + dR[7] * w -
                    2.f * dR[8] * x);
    dqn[2] = 2.f * (-2.f * dR[0] * y + dR[1] * x + dR[2] * w + dR[3] * x + dR[5] * z - dR[6] * w + dR[7] * z -
                    2.f * dR[8] * y);
    dqn[3] = 2.f * (-2.f * dR[0] * z - dR[1] * w + dR[2] * x + dR[3] * w - 2.f * dR[4] * z + dR[5] * y + dR[6] * x +
                    dR[7] * y);
    const float dot = w * dqn[0] + x * dqn[1] + y * dqn[2] + z * dqn[3];
    const float qh[4] = {w, x, y, z};
    // colour: rgb = max(0, sum_k Y_k(dir) sh_k + 1/2)
    const float dx = m0 - cam.campos[0], dy = m1 - cam.campos[1], dz = m2 - cam.campos[2];
    const float idn = rsqrtf(dx * dx + dy * dy + dz * dz);
    const float ex = dx * idn, ey = dy * idn, ez = dz * idn;
    constexpr int K = (kDeg + 1) * (kDeg + 1);
    float Y[16], dY[16][3];
    sh_basis(kDeg, ex, ey, ez, Y);
    sh_basis_grad(kDeg, ex, ey, ez, dY);
    const float* shg = sh + (size_t)g * K * 3;
    float* dshg = dsh + (size_t)g * K * 3;
    float gc[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        float a = 0.5f;
#pragma unroll
        for (int k = 0; k < K; ++k) a += Y[k] * shg[3 * k + ch];
        gc[ch] = a < 0.f ? 0.f : drgb[3 * g + ch];
    }
    float ddir[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < K; ++k) {
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const float c = shg[3 * k + ch];
            dshg[3 * k + ch] += Y[k] * gc[ch];
            ddir[0] += gc[ch] * c * dY[k][0];
            ddir[1] += gc[ch] * c * dY[k][1];
            ddir[2] += gc[ch] * c * dY[k][2];
        }
    }
    const float dd = ex * ddir[0] + ey * ddir[1] + ez * ddir[2];
    dmu[0] += (ddir[0] - ex * dd) * idn;
    dmu[1] += (ddir[1] - ey * dd) * idn;
    dmu[2] += (ddir[2] - ez * dd) * idn;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        dmeans3[3 * g + k] += dmu[k];
        dscales[3 * g + k] += ds[k];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) dquats[4 * (size_t)g + i] += (dqn[i] - qh[i] * dot) * iqn;
}

}  // namespace
}  // namespace tcgs

extern "C" tcgs_status tcgs_project(const tcgs_camera* cam, int32_t P, int32_t sh_degree, const float* means3,
                                    const float* scales, const float* quats, const float* sh,
                                    const float* opacity, float* mean2d,
                                    float* conic, float* depth, int32_t* radius, float* rgb,
                                    uint32_t* tiles_touched, tcgs_stream stream) {
    using namespace tcgs;
    if (!valid_camera(cam) || P < 0 || sh_degree < 0 || sh_degree > 3) return TCGS_ERR_INVALID;
    if (P == 0) return TCGS_OK;
    if (!means3 || !scales || !quats || !sh || !mean2d || !conic || !depth || !radius || !rgb || !tiles_touched)
        return TCGS_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(quats) & 15) || (reinterpret_cast<uintptr_t>(mean2d) & 7) ||
        (sh_degree == 3 && (reinterpret_cast<uintptr_t>(sh) & 15)))
        return TCGS_ERR_INVALID;
    DevCamera dc = make_dev_camera(*cam);
    const int blocks = (P + kProjThreads - 1) / kProjThreads;
    if (sh_degree == 3)
        k_project<true><<<blocks, kProjThreads, 0, (cudaStream_t)stream>>>(dc, P, sh_degree, means3, scales, quats, sh,
                                                                          opacity, mean2d, conic, depth, radius, rgb,
                                                                          tiles_touched);
    else
        k_project<false><<<blocks, kProjThreads, 0, (cudaStream_t)stream>>>(dc, P, sh_degree, means3, scales, quats,
                                                                           sh, opacity, mean2d, conic, depth, radius,
                                                                           rgb, tiles_touched);
    count_launches(1);
    TCGS_CHECK_LAUNCH();
    return TCGS_OK;
}

extern "C" tcgs_status tcgs_project_bwd(const tcgs_camera* cam, int32_t P, int32_t sh_degree, const float* means3,
                                        const float* scales, const float* quats, const float* sh,
                                        const int32_t* radius, const float* dmean2d, const float* dconic,
                                        const float* drgb, float* dmeans3, float* dscales, float* dquats,
                                        float* dsh, tcgs_stream stream) {
    using namespace tcgs;
    if (!valid_camera(cam) || P < 0 || sh_degree < 0 || sh_degree > 3) return TCGS_ERR_INVALID;
    if (P == 0) return TCGS_OK;
    if (!means3 || !scales || !quats || !sh || !radius || !dmean2d || !dconic || !drgb || !dmeans3 || !dscales ||
        !dquats || !dsh)
        return TCGS_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(quats) & 15) return TCGS_ERR_INVALID;
    DevCamera dc = make_dev_camera(*cam);
    const int threads = 256;
    const int blocks = (P + threads - 1) / threads;
    cudaStream_t s = (cudaStream_t)stream;
    switch (sh_degree) {
        case 0: k_project_bwd<0><<<blocks, threads, 0, s>>>(dc, P, means3, scales, quats, sh, radius, dmean2d, dconic,
                                                            drgb, dmeans3, dscales, dquats, dsh); break;
        case 1: k_project_bwd<1><<<blocks, threads, 0, s>>>(dc, P, means3, scales, quats, sh, radius, dmean2d, dconic,
                                                            drgb, dmeans3, dscales, dquats, dsh); break;
        case 2: k_project_bwd<2><<<blocks, threads, 0, s>>>(dc, P, means3, scales, quats, sh, radius, dmean2d, dconic,
                                                            drgb, dmeans3, dscales, dquats, dsh); break;
        default: k_project_bwd<3><<<blocks, threads, 0, s>>>(dc, P, means3, scales, quats, sh, radius, dmean2d, dconic,
                                                             drgb, dmeans3, dscales, dquats, dsh); break;
    }
    count_launches(1);
    TCGS_CHECK_LAUNCH();
    return TCGS_OK;
}
