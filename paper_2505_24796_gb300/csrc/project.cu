// project.cu -- preprocess stage (Sec. 3.1, Eq. 2): EWA projection of 3D Gaussians.
//
// One thread per Gaussian; the stage is HBM bound (read ~40 B + the SH coefficients,
// write 44 B per Gaussian).  SH degree-3 coefficients (192 B per Gaussian) are read as
// twelve 16-byte vectors.
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

__global__ void __launch_bounds__(256) k_project(DevCamera cam, int P, int deg, const float* __restrict__ means3,
                                                 const float* __restrict__ scales, const float* __restrict__ quats,
                                                 const float* __restrict__ sh, const float* __restrict__ opacity,
                                                 float* __restrict__ mean2d,
                                                 float* __restrict__ conic, float* __restrict__ depth,
                                                 int32_t* __restrict__ radius, float* __restrict__ rgb,
                                                 uint32_t* __restrict__ tiles_touched) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= P) return;
    float m0 = means3[3 * g], m1 = means3[3 * g + 1], m2 = means3[3 * g + 2];
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
        float4 q = *reinterpret_cast<const float4*>(quats + 4 * (size_t)g);
        float qn = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
        float w = q.x * qn, x = q.y * qn, y = q.z * qn, z = q.w * qn;
        float s0 = scales[3 * g], s1 = scales[3 * g + 1], s2 = scales[3 * g + 2];
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
        const float reach2 = opacity ? 2.f * logf(255.f * opacity[g]) : 9.f;
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
                sh_basis(deg, dx * dn, dy * dn, dz * dn, Y);
                int K = (deg + 1) * (deg + 1);
                float cr = 0.5f, cg = 0.5f, cb = 0.5f;
                const float* s = sh + (size_t)g * K * 3;
                if (deg == 3) {
                    const float4* s4 = reinterpret_cast<const float4*>(s);
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
    int threads = 256;
    int blocks = (P + threads - 1) / threads;
    k_project<<<blocks, threads, 0, (cudaStream_t)stream>>>(dc, P, sh_degree, means3, scales, quats, sh, opacity, mean2d,
                                                           conic, depth, radius, rgb, tiles_touched);
    count_launches(1);
    TCGS_CHECK_LAUNCH();
    return TCGS_OK;
}
