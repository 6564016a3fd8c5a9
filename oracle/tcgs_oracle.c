/*
 * tcgs_oracle.c -- plain, slow FP64 CPU oracle of the TC-GS rasterizer hot path
 * (TC-GS: "A Faster Gaussian Splatting Module Utilizing Tensor Cores").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file.  Its users are the tests, the smoke check and the CPU
 * baseline leg of the benchmark.  It shares no code, header, table or
 * constant with the CUDA library; it is written from the paper's equations.
 *
 * Every routine works in double precision on plain host arrays and uses the
 * most direct loop that states the definition.  No blocking, fusion or
 * reordering beyond what the definition itself implies.
 *
 * Conventions the paper leaves open (each one is a "reading"):
 *   - pixel (i, j) is sampled at (i + 0.5, j + 0.5); tiles are 16 x 16 pixels;
 *   - mean2d = (fx * X / Z + cx, fy * Y / Z + cy) in camera coordinates;
 *   - a Gaussian covers tile (tx, ty) iff the axis-aligned square
 *     [mx - r, mx + r] x [my - r, my + r] meets the tile's pixel square
 *     [16 tx, 16 tx + 16) x [16 ty, 16 ty + 16); with exact coverage it must
 *     also reach alpha >= 1/255 (Eq. 5) somewhere on the tile's box of pixel
 *     centres, with the margins stated at tile_reached();
 *   - alpha is clamped to alpha_max (0.99 in the official 3DGS renderer that
 *     the paper builds on; alpha_max = 1 reproduces Algorithm 1 literally);
 *   - the termination test of Algorithm 1 is T - alpha * T < 1e-4, evaluated
 *     before blending (a terminating fragment is not blended);
 *   - the low-pass dilation adds 0.3 px^2 to the diagonal of Sigma', the
 *     Jacobian uses x/z, y/z clamped to +-1.3 tan(fov/2), near plane culls.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TILE 16

typedef struct {
    int32_t width, height;
    double fx, fy, cx, cy;
    double viewmat[12];  /* row-major 3x4 world -> camera [R | t] */
    double campos[3];    /* camera centre in world coordinates */
    double near_z;       /* Gaussians with camera z <= near_z are culled */
    double tan_fovx, tan_fovy;
} orc_camera;

static int grid_w(const orc_camera* c) { return (c->width + ORC_TILE - 1) / ORC_TILE; }
static int grid_h(const orc_camera* c) { return (c->height + ORC_TILE - 1) / ORC_TILE; }

/* ------------------------------------------------------------------------ */
/* Real spherical harmonics up to degree 3 (colour model of the 3DGS scenes  */
/* the paper renders, Sec. 3.1; coefficients ordered l = 0..3, m = -l..l,    */
/* Condon-Shortley phase).  Constants are the real-SH normalisation          */
/* sqrt((2l+1)/(4 pi) * (l-|m|)!/(l+|m|)!) times the Legendre factors,        */
/* written out as closed forms.                                               */
/* ------------------------------------------------------------------------ */
void orc_sh_basis(int degree, const double dir[3], double* out)
{
    const double pi = 3.14159265358979323846;
    double x = dir[0], y = dir[1], z = dir[2];
    out[0] = 0.5 * sqrt(1.0 / pi);
    if (degree < 1) return;
    double k1 = sqrt(3.0 / (4.0 * pi));
    out[1] = -k1 * y;
    out[2] = k1 * z;
    out[3] = -k1 * x;
    if (degree < 2) return;
    double k2a = 0.5 * sqrt(15.0 / pi);
    double k20 = 0.25 * sqrt(5.0 / pi);
    double k22 = 0.25 * sqrt(15.0 / pi);
    out[4] = k2a * x * y;
    out[5] = -k2a * y * z;
    out[6] = k20 * (2.0 * z * z - x * x - y * y);
    out[7] = -k2a * x * z;
    out[8] = k22 * (x * x - y * y);
    if (degree < 3) return;
    double k33 = 0.25 * sqrt(35.0 / (2.0 * pi));
    double k32 = 0.5 * sqrt(105.0 / pi);
    double k31 = 0.25 * sqrt(21.0 / (2.0 * pi));
    double k30 = 0.25 * sqrt(7.0 / pi);
    double k32b = 0.25 * sqrt(105.0 / pi);
    out[9] = -k33 * y * (3.0 * x * x - y * y);
    out[10] = k32 * x * y * z;
    out[11] = -k31 * y * (4.0 * z * z - x * x - y * y);
    out[12] = k30 * z * (2.0 * z * z - 3.0 * x * x - 3.0 * y * y);
    out[13] = -k31 * x * (4.0 * z * z - x * x - y * y);
    out[14] = k32b * z * (x * x - y * y);
    out[15] = -k33 * x * (x * x - 3.0 * y * y);
}

/* Rotation matrix (row-major) of the unit quaternion q / |q|, q = (w, x, y, z). */
void orc_quat_to_rot(const double q_in[4], double R[9])
{
    double n = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
    double w = q_in[0] / n, x = q_in[1] / n, y = q_in[2] / n, z = q_in[3] / n;
    R[0] = 1.0 - 2.0 * (y * y + z * z); R[1] = 2.0 * (x * y - w * z);       R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);       R[4] = 1.0 - 2.0 * (x * x + z * z); R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);       R[7] = 2.0 * (y * z + w * x);       R[8] = 1.0 - 2.0 * (x * x + y * y);
}

/* Tile rectangle covered by a projected Gaussian (reading above).
 * Writes inclusive bounds; returns the number of tiles (0 when empty). */
static int64_t tile_rect(const orc_camera* cam, double mx, double my, int32_t r,
                         int* x0, int* x1, int* y0, int* y1)
{
    int gw = grid_w(cam), gh = grid_h(cam);
    double lx = floor((mx - r) / ORC_TILE), hx = floor((mx + r) / ORC_TILE);
    double ly = floor((my - r) / ORC_TILE), hy = floor((my + r) / ORC_TILE);
    if (lx < 0) lx = 0;
    if (ly < 0) ly = 0;
    if (hx > gw - 1) hx = gw - 1;
    if (hy > gh - 1) hy = gh - 1;
    if (hx < lx || hy < ly) { *x0 = *y0 = 0; *x1 = *y1 = -1; return 0; }
    *x0 = (int)lx; *x1 = (int)hx; *y0 = (int)ly; *y1 = (int)hy;
    return (int64_t)(*x1 - *x0 + 1) * (int64_t)(*y1 - *y0 + 1);
}

/* ------------------------------------------------------------------------ */
/* Preprocess (Sec. 3.1, Eq. 2): mu' = W mu, Sigma' = J W Sigma W^T J^T.     */
/* Sigma = R S S^T R^T with S = diag(scale); conic = (Sigma')^{-1} stored as  */
/* (sigma11, sigma12, sigma22) in the notation of Sec. 4.2.                   */
/* cov2d_out (nullable) receives (a, b, c) of Sigma' after dilation.          */
/* Coverage radius: tight_radius = 0 gives the 3-sigma square of official    */
/* 3DGS, r = ceil(3 sqrt(lambda_max)); tight_radius = 1 the square bounding  */
/* the ellipse where alpha >= 1/255 (Eq. 5): o exp(-q/2) >= 1/255 iff        */
/* q <= 2 ln(255 o), so r = ceil(sqrt(2 ln(255 o) lambda_max)); a Gaussian   */
/* with o <= 1/255 reaches no pixel and is culled.                            */
/* ------------------------------------------------------------------------ */
void orc_project(const orc_camera* cam, int P, int sh_degree,
                 const double* means3, const double* scales, const double* quats,
                 const double* opacity, const double* sh, int tight_radius,
                 double* mean2d, double* conic, double* depth, int32_t* radius,
                 double* rgb, int32_t* tiles_touched, double* cov2d_out)
{
    const double* V = cam->viewmat;
    int K = (sh_degree + 1) * (sh_degree + 1);
    for (int g = 0; g < P; ++g) {
        const double* m = means3 + 3 * g;
        mean2d[2 * g] = mean2d[2 * g + 1] = 0.0;
        conic[3 * g] = conic[3 * g + 1] = conic[3 * g + 2] = 0.0;
        depth[g] = 0.0;
        radius[g] = 0;
        tiles_touched[g] = 0;
        rgb[3 * g] = rgb[3 * g + 1] = rgb[3 * g + 2] = 0.0;
        if (cov2d_out) cov2d_out[3 * g] = cov2d_out[3 * g + 1] = cov2d_out[3 * g + 2] = 0.0;

        /* camera-space mean t = W mu */
        double t[3];
        for (int i = 0; i < 3; ++i)
            t[i] = V[4 * i] * m[0] + V[4 * i + 1] * m[1] + V[4 * i + 2] * m[2] + V[4 * i + 3];
        if (t[2] <= cam->near_z) continue;

        /* 3D covariance Sigma = R S S^T R^T */
        double R[9];
        orc_quat_to_rot(quats + 4 * g, R);
        double M[9];  /* M = R S */
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) M[3 * i + k] = R[3 * i + k] * scales[3 * g + k];
        double S3[9];
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) {
                double s = 0.0;
                for (int l = 0; l < 3; ++l) s += M[3 * i + l] * M[3 * k + l];
                S3[3 * i + k] = s;
            }

        /* Jacobian of the pinhole projection at the (frustum-clamped) mean */
        double limx = 1.3 * cam->tan_fovx, limy = 1.3 * cam->tan_fovy;
        double txtz = t[0] / t[2], tytz = t[1] / t[2];
        double tx = fmin(limx, fmax(-limx, txtz)) * t[2];
        double ty = fmin(limy, fmax(-limy, tytz)) * t[2];
        double J[6] = {cam->fx / t[2], 0.0, -cam->fx * tx / (t[2] * t[2]),
                       0.0, cam->fy / t[2], -cam->fy * ty / (t[2] * t[2])};
        /* T = J W (2x3) */
        double T[6];
        for (int i = 0; i < 2; ++i)
            for (int k = 0; k < 3; ++k)
                T[3 * i + k] = J[3 * i] * V[k] + J[3 * i + 1] * V[4 + k] + J[3 * i + 2] * V[8 + k];
        /* Sigma' = T Sigma T^T */
        double C2[4];
        for (int i = 0; i < 2; ++i)
            for (int k = 0; k < 2; ++k) {
                double s = 0.0;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) s += T[3 * i + a] * S3[3 * a + b] * T[3 * k + b];
                C2[2 * i + k] = s;
            }
        double a = C2[0] + 0.3, b = C2[1], c = C2[3] + 0.3;
        double det = a * c - b * b;
        if (!(det > 0.0)) continue;

        double mid = 0.5 * (a + c);
        double lam1 = mid + sqrt(fmax(0.1, mid * mid - det));
        double lam2 = mid - sqrt(fmax(0.1, mid * mid - det));
        double reach2 = 9.0;   /* squared reach in units of sigma */
        if (tight_radius) {
            reach2 = 2.0 * log(255.0 * opacity[g]);
            if (!(reach2 > 0.0)) continue;
        }
        int32_t r = (int32_t)ceil(sqrt(reach2 * fmax(lam1, lam2)));
        double mx = cam->fx * t[0] / t[2] + cam->cx;
        double my = cam->fy * t[1] / t[2] + cam->cy;
        int x0, x1, y0, y1;
        int64_t nt = tile_rect(cam, mx, my, r, &x0, &x1, &y0, &y1);
        if (nt == 0) continue;

        mean2d[2 * g] = mx;
        mean2d[2 * g + 1] = my;
        conic[3 * g] = c / det;
        conic[3 * g + 1] = -b / det;
        conic[3 * g + 2] = a / det;
        depth[g] = t[2];
        radius[g] = r;
        tiles_touched[g] = (int32_t)nt;
        if (cov2d_out) { cov2d_out[3 * g] = a; cov2d_out[3 * g + 1] = b; cov2d_out[3 * g + 2] = c; }

        /* colour from SH at the viewing direction (mu - campos) / |mu - campos| */
        double d[3] = {m[0] - cam->campos[0], m[1] - cam->campos[1], m[2] - cam->campos[2]};
        double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        d[0] /= dn; d[1] /= dn; d[2] /= dn;
        double Y[16];
        orc_sh_basis(sh_degree, d, Y);
        for (int ch = 0; ch < 3; ++ch) {
            double s = 0.0;
            for (int k = 0; k < K; ++k) s += Y[k] * sh[(size_t)g * K * 3 + 3 * k + ch];
            s += 0.5;
            rgb[3 * g + ch] = s < 0.0 ? 0.0 : s;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Sorting stage (Sec. 3.1, Eq. 3): splats (tile, Gaussian), each tile's     */
/* list in increasing depth; ties by Gaussian index.                          */
/* ------------------------------------------------------------------------ */
typedef struct { int32_t tile; double depth; int32_t id; } orc_splat;

static int cmp_splat(const void* pa, const void* pb)
{
    const orc_splat* a = (const orc_splat*)pa;
    const orc_splat* b = (const orc_splat*)pb;
    if (a->tile != b->tile) return a->tile < b->tile ? -1 : 1;
    if (a->depth != b->depth) return a->depth < b->depth ? -1 : 1;
    if (a->id != b->id) return a->id < b->id ? -1 : 1;
    return 0;
}

/* Least value of q(x, y) = a (x - mx)^2 + 2 b (x - mx)(y - my) + c (y - my)^2 (Q = [[a, b], [b, c]]
 * positive definite) over the box [x0, x1] x [y0, y1].  The unconstrained minimiser is (mx, my);
 * when it lies outside the box the minimum is on the boundary, and on each edge q is a parabola in
 * the free coordinate: on x = X it is least at y = my - b (X - mx) / c, on y = Y at
 * x = mx - b (Y - my) / a, each clamped to the edge. */
double orc_box_min_q(double mx, double my, double a, double b, double c, double x0, double x1, double y0, double y1)
{
    if (mx >= x0 && mx <= x1 && my >= y0 && my <= y1) return 0.0;
    double best = INFINITY;
    const double xs[2] = {x0, x1}, ys[2] = {y0, y1};
    for (int e = 0; e < 2; ++e) {
        double X = xs[e];
        double y = my - b * (X - mx) / c;
        if (y < y0) y = y0;
        if (y > y1) y = y1;
        double dx = X - mx, dy = y - my;
        double q = a * dx * dx + 2.0 * b * dx * dy + c * dy * dy;
        if (q < best) best = q;
        double Y = ys[e];
        double x = mx - b * (Y - my) / a;
        if (x < x0) x = x0;
        if (x > x1) x = x1;
        dx = x - mx; dy = Y - my;
        q = a * dx * dx + 2.0 * b * dx * dy + c * dy * dy;
        if (q < best) best = q;
    }
    return best;
}

/* Exact coverage: alpha = o exp(-q / 2) >= 1/255 (Eq. 5) needs q <= 2 (ln o + ln 255); the limit
 * adds a relative margin of 1e-4 and an absolute one of 1e-3 (so that no splat that some FP32
 * evaluation could keep is dropped), and no tile qualifies when 2 (ln o + ln 255) <= -1e-3. */
static double reach_limit(double o)
{
    double reach = 2.0 * (log(o) + log(255.0));
    return reach > -1e-3 ? reach * 1.0001 + 1e-3 : -1.0;
}

static int tile_reached(int tx, int ty, double mx, double my, const double* q, double o)
{
    double lim = reach_limit(o);
    if (lim < 0.0) return 0;
    double x0 = ORC_TILE * tx + 0.5, y0 = ORC_TILE * ty + 0.5;
    return orc_box_min_q(mx, my, q[0], q[1], q[2], x0, x0 + ORC_TILE - 1, y0, y0 + ORC_TILE - 1) <= lim;
}

/* Splats of Gaussian g: its rectangle's tiles, or with conic and opacity given (exact coverage)
 * those of them it reaches.  tiles (nullable) receives the tile ids in row-major order. */
static int64_t gaussian_tiles(const orc_camera* cam, int g, const double* mean2d, const int32_t* radius,
                              const double* conic, const double* opacity, int32_t* tiles)
{
    if (radius[g] <= 0) return 0;
    int x0, x1, y0, y1, gw = grid_w(cam);
    if (tile_rect(cam, mean2d[2 * g], mean2d[2 * g + 1], radius[g], &x0, &x1, &y0, &y1) == 0) return 0;
    int64_t n = 0;
    for (int ty = y0; ty <= y1; ++ty)
        for (int tx = x0; tx <= x1; ++tx) {
            if (conic && !tile_reached(tx, ty, mean2d[2 * g], mean2d[2 * g + 1], conic + 3 * g, opacity[g]))
                continue;
            if (tiles) tiles[n] = ty * gw + tx;
            ++n;
        }
    return n;
}

int64_t orc_count_splats(const orc_camera* cam, int P, const double* mean2d, const int32_t* radius,
                         const double* conic, const double* opacity)
{
    int64_t n = 0;
    for (int g = 0; g < P; ++g) n += gaussian_tiles(cam, g, mean2d, radius, conic, opacity, NULL);
    return n;
}

/* ids_sorted[N], tile_of[N] (nullable), ranges[2 * num_tiles] = [start, end). */
int64_t orc_bin_sort(const orc_camera* cam, int P, const double* mean2d, const int32_t* radius,
                     const double* conic, const double* opacity, const double* depth, int64_t capacity,
                     int32_t* ids_sorted, int32_t* tile_of, int32_t* ranges)
{
    int gw = grid_w(cam), gh = grid_h(cam);
    int64_t n = orc_count_splats(cam, P, mean2d, radius, conic, opacity);
    for (int t = 0; t < 2 * gw * gh; ++t) ranges[t] = 0;
    if (n > capacity) return -n;
    orc_splat* sp = (orc_splat*)malloc(sizeof(orc_splat) * (size_t)(n > 0 ? n : 1));
    int32_t* tl = (int32_t*)malloc(sizeof(int32_t) * (size_t)gw * (size_t)gh);
    int64_t k = 0;
    for (int g = 0; g < P; ++g) {
        int64_t m = gaussian_tiles(cam, g, mean2d, radius, conic, opacity, tl);
        for (int64_t j = 0; j < m; ++j) {
            sp[k].tile = tl[j];
            sp[k].depth = depth[g];
            sp[k].id = g;
            ++k;
        }
    }
    free(tl);
    qsort(sp, (size_t)n, sizeof(orc_splat), cmp_splat);
    for (int64_t s = 0; s < n; ++s) {
        ids_sorted[s] = sp[s].id;
        if (tile_of) tile_of[s] = sp[s].tile;
        if (s == 0 || sp[s - 1].tile != sp[s].tile) ranges[2 * sp[s].tile] = (int32_t)s;
        if (s == n - 1 || sp[s + 1].tile != sp[s].tile) ranges[2 * sp[s].tile + 1] = (int32_t)(s + 1);
    }
    free(sp);
    return n;
}

/* ------------------------------------------------------------------------ */
/* Conditional alpha-blending, Algorithm 1, per pixel, alpha from Eq. (4).    */
/* ------------------------------------------------------------------------ */
typedef struct {
    double alpha_max;
    double cull_threshold;   /* 1/255, Eq. (5) */
    double t_min;            /* 1e-4, termination test of Algorithm 1 */
} orc_params;

/* One pixel at sample point (px, py) over the Gaussian list ids[0..n).
 * Returns the composited colour (without background) in C[3], T in *T_out,
 * the count of list entries up to and including the last blended one in
 * *n_contrib, the count of list entries evaluated (up to the terminating one,
 * or the whole list) in *n_eval, and the counts of blended / culled
 * fragments.  cull_margin receives min |beta - (-ln 255)| over evaluated
 * fragments; term_margin the min |ln(T - alpha T) - ln(1e-4)| over fragments
 * that reached the termination test. */
static void render_pixel(const orc_params* prm, double px, double py, const int32_t* ids, int64_t n,
                         const double* mean2d, const double* conic, const double* opacity, const double* rgb,
                         double C[3], double* T_out, int64_t* n_contrib, int64_t* n_eval,
                         int64_t* f_blend, int64_t* f_cull, double* cull_margin, double* term_margin)
{
    double T = 1.0;
    C[0] = C[1] = C[2] = 0.0;
    int64_t last = 0, evaluated = n, nb = 0, nc = 0;
    double cm = INFINITY, tm = INFINITY;
    const double ln255 = log(255.0);
    for (int64_t k = 0; k < n; ++k) {
        int32_t g = ids[k];
        double dx = mean2d[2 * g] - px, dy = mean2d[2 * g + 1] - py;
        double s11 = conic[3 * g], s12 = conic[3 * g + 1], s22 = conic[3 * g + 2];
        double q = s11 * dx * dx + 2.0 * s12 * dx * dy + s22 * dy * dy;
        double o = opacity[g];
        double alpha = o * exp(-0.5 * q);
        double beta = log(o) - 0.5 * q;
        double m = fabs(beta + ln255);
        if (m < cm) cm = m;
        if (alpha > prm->alpha_max) alpha = prm->alpha_max;
        if (alpha < prm->cull_threshold) { ++nc; continue; }
        double Tn = T - alpha * T;
        double tmar = fabs(log(Tn) - log(prm->t_min));
        if (tmar < tm) tm = tmar;
        if (Tn < prm->t_min) { evaluated = k + 1; ++nc; break; }
        C[0] += rgb[3 * g] * alpha * T;
        C[1] += rgb[3 * g + 1] * alpha * T;
        C[2] += rgb[3 * g + 2] * alpha * T;
        T = Tn;
        last = k + 1;
        ++nb;
    }
    *T_out = T;
    *n_contrib = last;
    *n_eval = evaluated;
    *f_blend = nb;
    *f_cull = nc;
    if (cull_margin) *cull_margin = cm;
    if (term_margin) *term_margin = tm;
}

/* Tiled renderer: every pixel walks its tile's sorted list (Algorithm 1).
 * img [3, H, W]; T_final, n_contrib, n_eval, cull_margin, term_margin [H, W]
 * (the last four nullable).  counts (nullable) += {f_blend, f_cull, sum n_eval}.
 * tile_subset (nullable) restricts the work to n_subset tiles; other pixels
 * are left untouched. */
void orc_render(const orc_camera* cam, double alpha_max, const int32_t* ranges, const int32_t* ids_sorted,
                const double* mean2d, const double* conic, const double* opacity, const double* rgb,
                const double* bg3, double* img, double* T_final, int32_t* n_contrib, int32_t* n_eval,
                double* cull_margin, double* term_margin, int64_t* counts,
                const int32_t* tile_subset, int n_subset)
{
    orc_params prm = {alpha_max, 1.0 / 255.0, 1e-4};
    int W = cam->width, H = cam->height, gw = grid_w(cam), gh = grid_h(cam);
    int ntiles = tile_subset ? n_subset : gw * gh;
    for (int ti = 0; ti < ntiles; ++ti) {
        int t = tile_subset ? tile_subset[ti] : ti;
        int tx = t % gw, ty = t / gw;
        const int32_t* ids = ids_sorted + ranges[2 * t];
        int64_t n = ranges[2 * t + 1] - ranges[2 * t];
        for (int j = ty * ORC_TILE; j < (ty + 1) * ORC_TILE && j < H; ++j)
            for (int i = tx * ORC_TILE; i < (tx + 1) * ORC_TILE && i < W; ++i) {
                double C[3], T, cm, tm;
                int64_t nct, nev, nb, nc;
                render_pixel(&prm, i + 0.5, j + 0.5, ids, n, mean2d, conic, opacity, rgb,
                             C, &T, &nct, &nev, &nb, &nc, &cm, &tm);
                size_t p = (size_t)j * W + i;
                for (int ch = 0; ch < 3; ++ch) img[(size_t)ch * W * H + p] = C[ch] + T * bg3[ch];
                if (T_final) T_final[p] = T;
                if (n_contrib) n_contrib[p] = (int32_t)nct;
                if (n_eval) n_eval[p] = (int32_t)nev;
                if (cull_margin) cull_margin[p] = cm;
                if (term_margin) term_margin[p] = tm;
                if (counts) { counts[0] += nb; counts[1] += nc; counts[2] += nev; }
            }
    }
}

/* Untiled brute force: every pixel walks ALL Gaussians in global (depth, id)
 * order and keeps Gaussian g iff the pixel's tile lies in g's rectangle.
 * Membership is decided by the interval test of the reading above, written
 * independently of tile_rect(). */
typedef struct { double depth; int32_t id; } orc_dep;
static int cmp_dep(const void* pa, const void* pb)
{
    const orc_dep* a = (const orc_dep*)pa;
    const orc_dep* b = (const orc_dep*)pb;
    if (a->depth != b->depth) return a->depth < b->depth ? -1 : 1;
    return a->id < b->id ? -1 : (a->id > b->id);
}

void orc_render_bruteforce(const orc_camera* cam, double alpha_max, int P, const double* mean2d,
                           const int32_t* radius, const double* depth, const double* conic,
                           const double* opacity, const double* rgb, const double* bg3,
                           double* img, double* T_final, int32_t* n_contrib)
{
    orc_params prm = {alpha_max, 1.0 / 255.0, 1e-4};
    int W = cam->width, H = cam->height;
    orc_dep* order = (orc_dep*)malloc(sizeof(orc_dep) * (size_t)(P > 0 ? P : 1));
    int nv = 0;
    for (int g = 0; g < P; ++g)
        if (radius[g] > 0) { order[nv].depth = depth[g]; order[nv].id = g; ++nv; }
    qsort(order, (size_t)nv, sizeof(orc_dep), cmp_dep);
    int32_t* list = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nv > 0 ? nv : 1));
    for (int j = 0; j < H; ++j)
        for (int i = 0; i < W; ++i) {
            int tx = i / ORC_TILE, ty = j / ORC_TILE;
            double lo_x = ORC_TILE * tx, lo_y = ORC_TILE * ty;
            int64_t n = 0;
            for (int k = 0; k < nv; ++k) {
                int32_t g = order[k].id;
                double mx = mean2d[2 * g], my = mean2d[2 * g + 1], r = radius[g];
                int in_x = (mx - r < lo_x + ORC_TILE) && (mx + r >= lo_x);
                int in_y = (my - r < lo_y + ORC_TILE) && (my + r >= lo_y);
                if (in_x && in_y) list[n++] = g;
            }
            double C[3], T;
            int64_t nct, nev, nb, nc;
            render_pixel(&prm, i + 0.5, j + 0.5, list, n, mean2d, conic, opacity, rgb,
                         C, &T, &nct, &nev, &nb, &nc, NULL, NULL);
            size_t p = (size_t)j * W + i;
            for (int ch = 0; ch < 3; ++ch) img[(size_t)ch * W * H + p] = C[ch] + T * bg3[ch];
            if (T_final) T_final[p] = T;
            if (n_contrib) n_contrib[p] = (int32_t)nct;
        }
    free(list);
    free(order);
}

/* ------------------------------------------------------------------------ */
/* Backward of Algorithm 1 with respect to mean2d, conic, opacity and colour. */
/* C = sum_j c_j a_j T_j + bg T_final, T_j = prod_{k<j} (1 - a_k) (Eq. 6).    */
/* dC/dc_j = a_j T_j;  dC/da_j = c_j T_j - S_j / (1 - a_j) with S_j the       */
/* colour blended after j plus bg T_final;  a = min(alpha_max, o exp(p)),     */
/* p = -1/2 d^T Q d, d = mu' - pixel, Q = (sigma11, sigma12; sigma12, sigma22)*/
/* The clamp has zero derivative where it is active.  Gradients accumulate.   */
/* ------------------------------------------------------------------------ */
void orc_render_bwd(const orc_camera* cam, double alpha_max, const int32_t* ranges, const int32_t* ids_sorted,
                    const double* mean2d, const double* conic, const double* opacity, const double* rgb,
                    const double* bg3, const double* dL_dimg,
                    double* dmean2d, double* dconic, double* dopacity, double* drgb)
{
    int W = cam->width, H = cam->height, gw = grid_w(cam), gh = grid_h(cam);
    const double thr = 1.0 / 255.0, t_min = 1e-4;
    int maxn = 0;
    for (int t = 0; t < gw * gh; ++t)
        if (ranges[2 * t + 1] - ranges[2 * t] > maxn) maxn = ranges[2 * t + 1] - ranges[2 * t];
    int32_t* bj = (int32_t*)malloc(sizeof(int32_t) * (size_t)(maxn + 1));
    double* ba = (double*)malloc(sizeof(double) * (size_t)(maxn + 1));
    double* bT = (double*)malloc(sizeof(double) * (size_t)(maxn + 1));
    int* bclamped = (int*)malloc(sizeof(int) * (size_t)(maxn + 1));
    for (int t = 0; t < gw * gh; ++t) {
        int tx = t % gw, ty = t / gw;
        const int32_t* ids = ids_sorted + ranges[2 * t];
        int n = ranges[2 * t + 1] - ranges[2 * t];
        for (int j = ty * ORC_TILE; j < (ty + 1) * ORC_TILE && j < H; ++j)
            for (int i = tx * ORC_TILE; i < (tx + 1) * ORC_TILE && i < W; ++i) {
                double px = i + 0.5, py = j + 0.5;
                /* forward replay, recording the blended fragments */
                double T = 1.0;
                int nb = 0;
                for (int k = 0; k < n; ++k) {
                    int32_t g = ids[k];
                    double dx = mean2d[2 * g] - px, dy = mean2d[2 * g + 1] - py;
                    double q = conic[3 * g] * dx * dx + 2.0 * conic[3 * g + 1] * dx * dy + conic[3 * g + 2] * dy * dy;
                    double a = opacity[g] * exp(-0.5 * q);
                    int clamped = a > alpha_max;
                    if (clamped) a = alpha_max;
                    if (a < thr) continue;
                    double Tn = T - a * T;
                    if (Tn < t_min) break;
                    bj[nb] = g; ba[nb] = a; bT[nb] = T; bclamped[nb] = clamped; ++nb;
                    T = Tn;
                }
                size_t p = (size_t)j * W + i;
                double gch[3] = {dL_dimg[p], dL_dimg[(size_t)W * H + p], dL_dimg[(size_t)2 * W * H + p]};
                /* suffix colour S, walking back from the last blended fragment */
                double S[3] = {bg3[0] * T, bg3[1] * T, bg3[2] * T};
                for (int k = nb - 1; k >= 0; --k) {
                    int32_t g = bj[k];
                    double a = ba[k], Tk = bT[k];
                    double dL_da = 0.0;
                    for (int ch = 0; ch < 3; ++ch) {
                        drgb[3 * g + ch] += a * Tk * gch[ch];
                        dL_da += gch[ch] * (rgb[3 * g + ch] * Tk - S[ch] / (1.0 - a));
                    }
                    for (int ch = 0; ch < 3; ++ch) S[ch] += rgb[3 * g + ch] * a * Tk;
                    if (bclamped[k]) continue;
                    double dx = mean2d[2 * g] - px, dy = mean2d[2 * g + 1] - py;
                    double s11 = conic[3 * g], s12 = conic[3 * g + 1], s22 = conic[3 * g + 2];
                    double dL_dp = dL_da * a;  /* da/dp = a when unclamped */
                    dopacity[g] += dL_da * a / opacity[g];
                    dmean2d[2 * g] += dL_dp * -(s11 * dx + s12 * dy);
                    dmean2d[2 * g + 1] += dL_dp * -(s12 * dx + s22 * dy);
                    dconic[3 * g] += dL_dp * -0.5 * dx * dx;
                    dconic[3 * g + 1] += dL_dp * -dx * dy;
                    dconic[3 * g + 2] += dL_dp * -0.5 * dy * dy;
                }
            }
    }
    free(bj); free(ba); free(bT); free(bclamped);
}

/* ------------------------------------------------------------------------ */
/* Backward of the preprocess (Sec. 3.1, Eq. 2): given dL/d(mean2d, conic,   */
/* rgb) of each Gaussian, dL/d(means3, scales, quats, sh), written.  The      */
/* forward is recomputed step by step and every step is differentiated in    */
/* reverse: conic = Sigma'^-1, Sigma' = T Sigma T^T + 0.3 I, T = J W,         */
/* Sigma = M M^T, M = R(q/|q|) diag(s), J from the frustum-clamped mean,      */
/* mean2d = (fx tx / tz + cx, fy ty / tz + cy), t = W mu + t0, and           */
/* rgb = max(0, sum_k Y_k(dir) sh_k + 1/2), dir = (mu - campos) / |.|.       */
/* conic holds (s11, s12, s22); dconic[1] is the derivative with respect to  */
/* the one parameter s12 that fills both off-diagonal entries.  Gaussians    */
/* with radius 0 (culled) get zero gradients.                                 */
/* ------------------------------------------------------------------------ */

/* d Y_k / d(x, y, z) of the basis of orc_sh_basis at a unit direction. */
static void sh_basis_grad(int degree, const double dir[3], double dY[16][3])
{
    const double pi = 3.14159265358979323846;
    double x = dir[0], y = dir[1], z = dir[2];
    for (int k = 0; k < 16; ++k) dY[k][0] = dY[k][1] = dY[k][2] = 0.0;
    if (degree < 1) return;
    double k1 = sqrt(3.0 / (4.0 * pi));
    dY[1][1] = -k1;
    dY[2][2] = k1;
    dY[3][0] = -k1;
    if (degree < 2) return;
    double k2a = 0.5 * sqrt(15.0 / pi), k20 = 0.25 * sqrt(5.0 / pi), k22 = 0.25 * sqrt(15.0 / pi);
    dY[4][0] = k2a * y;          dY[4][1] = k2a * x;
    dY[5][1] = -k2a * z;         dY[5][2] = -k2a * y;
    dY[6][0] = -2.0 * k20 * x;   dY[6][1] = -2.0 * k20 * y;   dY[6][2] = 4.0 * k20 * z;
    dY[7][0] = -k2a * z;         dY[7][2] = -k2a * x;
    dY[8][0] = 2.0 * k22 * x;    dY[8][1] = -2.0 * k22 * y;
    if (degree < 3) return;
    double k33 = 0.25 * sqrt(35.0 / (2.0 * pi)), k32 = 0.5 * sqrt(105.0 / pi);
    double k31 = 0.25 * sqrt(21.0 / (2.0 * pi)), k30 = 0.25 * sqrt(7.0 / pi), k32b = 0.25 * sqrt(105.0 / pi);
    /* Y9 = -k33 (3 x^2 y - y^3) */
    dY[9][0] = -6.0 * k33 * x * y;           dY[9][1] = -k33 * (3.0 * x * x - 3.0 * y * y);
    /* Y10 = k32 x y z */
    dY[10][0] = k32 * y * z;                 dY[10][1] = k32 * x * z;   dY[10][2] = k32 * x * y;
    /* Y11 = -k31 (4 y z^2 - x^2 y - y^3) */
    dY[11][0] = 2.0 * k31 * x * y;           dY[11][1] = -k31 * (4.0 * z * z - x * x - 3.0 * y * y);
    dY[11][2] = -8.0 * k31 * y * z;
    /* Y12 = k30 (2 z^3 - 3 x^2 z - 3 y^2 z) */
    dY[12][0] = -6.0 * k30 * x * z;          dY[12][1] = -6.0 * k30 * y * z;
    dY[12][2] = k30 * (6.0 * z * z - 3.0 * x * x - 3.0 * y * y);
    /* Y13 = -k31 (4 x z^2 - x^3 - x y^2) */
    dY[13][0] = -k31 * (4.0 * z * z - 3.0 * x * x - y * y);   dY[13][1] = 2.0 * k31 * x * y;
    dY[13][2] = -8.0 * k31 * x * z;
    /* Y14 = k32b (x^2 z - y^2 z) */
    dY[14][0] = 2.0 * k32b * x * z;          dY[14][1] = -2.0 * k32b * y * z;   dY[14][2] = k32b * (x * x - y * y);
    /* Y15 = -k33 (x^3 - 3 x y^2) */
    dY[15][0] = -k33 * (3.0 * x * x - 3.0 * y * y);   dY[15][1] = 6.0 * k33 * x * y;
}

void orc_project_bwd(const orc_camera* cam, int P, int sh_degree,
                     const double* means3, const double* scales, const double* quats, const double* sh,
                     const int32_t* radius, const double* dmean2d, const double* dconic, const double* drgb,
                     double* dmeans3, double* dscales, double* dquats, double* dsh)
{
    const double* V = cam->viewmat;
    int K = (sh_degree + 1) * (sh_degree + 1);
    for (int g = 0; g < P; ++g) {
        for (int i = 0; i < 3; ++i) dmeans3[3 * g + i] = dscales[3 * g + i] = 0.0;
        for (int i = 0; i < 4; ++i) dquats[4 * g + i] = 0.0;
        for (int i = 0; i < K * 3; ++i) dsh[(size_t)g * K * 3 + i] = 0.0;
        if (radius[g] <= 0) continue;
        const double* m = means3 + 3 * g;
        const double* s = scales + 3 * g;
        const double* q = quats + 4 * g;

        /* ---- forward recomputation */
        double t[3];
        for (int i = 0; i < 3; ++i)
            t[i] = V[4 * i] * m[0] + V[4 * i + 1] * m[1] + V[4 * i + 2] * m[2] + V[4 * i + 3];
        double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        double w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
        double R[9];
        orc_quat_to_rot(q, R);
        double M[9], S3[9];
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) M[3 * i + k] = R[3 * i + k] * s[k];
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) {
                double a = 0.0;
                for (int l = 0; l < 3; ++l) a += M[3 * i + l] * M[3 * k + l];
                S3[3 * i + k] = a;
            }
        double limx = 1.3 * cam->tan_fovx, limy = 1.3 * cam->tan_fovy;
        double u = t[0] / t[2], v = t[1] / t[2];
        double cu = fmin(limx, fmax(-limx, u)), cv = fmin(limy, fmax(-limy, v));
        double du = (u > -limx && u < limx) ? 1.0 : 0.0, dv = (v > -limy && v < limy) ? 1.0 : 0.0;
        double tz = t[2];
        double J[6] = {cam->fx / tz, 0.0, -cam->fx * cu / tz, 0.0, cam->fy / tz, -cam->fy * cv / tz};
        double T[6];
        for (int i = 0; i < 2; ++i)
            for (int k = 0; k < 3; ++k)
                T[3 * i + k] = J[3 * i] * V[k] + J[3 * i + 1] * V[4 + k] + J[3 * i + 2] * V[8 + k];
        double C2[4];
        for (int i = 0; i < 2; ++i)
            for (int k = 0; k < 2; ++k) {
                double a = 0.0;
                for (int aa = 0; aa < 3; ++aa)
                    for (int bb = 0; bb < 3; ++bb) a += T[3 * i + aa] * S3[3 * aa + bb] * T[3 * k + bb];
                C2[2 * i + k] = a;
            }
        double A = C2[0] + 0.3, B = C2[1], C = C2[3] + 0.3;
        double det = A * C - B * B;
        double Q[4] = {C / det, -B / det, -B / det, A / det};

        /* ---- conic -> Sigma':  dL/dSigma' = -Q G Q, G the symmetric matrix of dconic */
        const double* dc = dconic + 3 * g;
        double G[4] = {dc[0], 0.5 * dc[1], 0.5 * dc[1], dc[2]};
        double QG[4], H[4];
        for (int i = 0; i < 2; ++i)
            for (int k = 0; k < 2; ++k) QG[2 * i + k] = Q[2 * i] * G[k] + Q[2 * i + 1] * G[2 + k];
        for (int i = 0; i < 2; ++i)
            for (int k = 0; k < 2; ++k) H[2 * i + k] = -(QG[2 * i] * Q[k] + QG[2 * i + 1] * Q[2 + k]);

        /* ---- Sigma' = T Sigma T^T:  dL/dT = 2 H T Sigma, dL/dSigma = T^T H T */
        double TS[6], dT[6], dS[9];
        for (int i = 0; i < 2; ++i)
            for (int k = 0; k < 3; ++k) {
                double a = 0.0;
                for (int l = 0; l < 3; ++l) a += T[3 * i + l] * S3[3 * l + k];
                TS[3 * i + k] = a;
            }
        for (int i = 0; i < 2; ++i)
            for (int k = 0; k < 3; ++k) dT[3 * i + k] = 2.0 * (H[2 * i] * TS[k] + H[2 * i + 1] * TS[3 + k]);
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) {
                double a = 0.0;
                for (int aa = 0; aa < 2; ++aa)
                    for (int bb = 0; bb < 2; ++bb) a += T[3 * aa + i] * H[2 * aa + bb] * T[3 * bb + k];
                dS[3 * i + k] = a;
            }

        /* ---- T = J W:  dL/dJ = dL/dT W^T (W the rotation part of the view matrix) */
        double dJ[6];
        for (int i = 0; i < 2; ++i)
            for (int k = 0; k < 3; ++k)
                dJ[3 * i + k] = dT[3 * i] * V[4 * k] + dT[3 * i + 1] * V[4 * k + 1] + dT[3 * i + 2] * V[4 * k + 2];

        /* ---- J(t) and mean2d(t) -> dL/dt */
        const double* dm2 = dmean2d + 2 * g;
        double dt[3];
        dt[0] = cam->fx / tz * dm2[0] + dJ[2] * (-cam->fx * du / (tz * tz));
        dt[1] = cam->fy / tz * dm2[1] + dJ[5] * (-cam->fy * dv / (tz * tz));
        dt[2] = -cam->fx * t[0] / (tz * tz) * dm2[0] - cam->fy * t[1] / (tz * tz) * dm2[1]
                + dJ[0] * (-cam->fx / (tz * tz)) + dJ[4] * (-cam->fy / (tz * tz))
                + dJ[2] * cam->fx * (du * t[0] / (tz * tz * tz) + cu / (tz * tz))
                + dJ[5] * cam->fy * (dv * t[1] / (tz * tz * tz) + cv / (tz * tz));
        double* dmu = dmeans3 + 3 * g;
        for (int k = 0; k < 3; ++k) dmu[k] = V[k] * dt[0] + V[4 + k] * dt[1] + V[8 + k] * dt[2];

        /* ---- Sigma = M M^T:  dL/dM = 2 dS M;  M = R diag(s) */
        double dM[9];
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) {
                double a = 0.0;
                for (int l = 0; l < 3; ++l) a += (dS[3 * i + l] + dS[3 * l + i]) * M[3 * l + k];
                dM[3 * i + k] = a;
            }
        double dR[9];
        for (int k = 0; k < 3; ++k) {
            double a = 0.0;
            for (int i = 0; i < 3; ++i) {
                a += dM[3 * i + k] * R[3 * i + k];
                dR[3 * i + k] = dM[3 * i + k] * s[k];
            }
            dscales[3 * g + k] = a;
        }
        /* ---- R(w, x, y, z) of the unit quaternion, then the normalisation q / |q| */
        double dqn[4];
        dqn[0] = dR[1] * (-2 * z) + dR[2] * (2 * y) + dR[3] * (2 * z) + dR[5] * (-2 * x) + dR[6] * (-2 * y)
                 + dR[7] * (2 * x);
        dqn[1] = dR[1] * (2 * y) + dR[2] * (2 * z) + dR[3] * (2 * y) + dR[4] * (-4 * x) + dR[5] * (-2 * w)
                 + dR[6] * (2 * z) + dR[7] * (2 * w) + dR[8] * (-4 * x);
        dqn[2] = dR[0] * (-4 * y) + dR[1] * (2 * x) + dR[2] * (2 * w) + dR[3] * (2 * x) + dR[5] * (2 * z)
                 + dR[6] * (-2 * w) + dR[7] * (2 * z) + dR[8] * (-4 * y);
        dqn[3] = dR[0] * (-4 * z) + dR[1] * (-2 * w) + dR[2] * (2 * x) + dR[3] * (2 * w) + dR[4] * (-4 * z)
                 + dR[5] * (2 * y) + dR[6] * (2 * x) + dR[7] * (2 * y);
        double qh[4] = {w, x, y, z};
        double dot = qh[0] * dqn[0] + qh[1] * dqn[1] + qh[2] * dqn[2] + qh[3] * dqn[3];
        for (int i = 0; i < 4; ++i) dquats[4 * g + i] = (dqn[i] - qh[i] * dot) / qn;

        /* ---- colour: rgb = max(0, sum_k Y_k(dir) sh_k + 1/2) */
        double d[3] = {m[0] - cam->campos[0], m[1] - cam->campos[1], m[2] - cam->campos[2]};
        double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double dir[3] = {d[0] / dn, d[1] / dn, d[2] / dn};
        double Y[16], dY[16][3];
        orc_sh_basis(sh_degree, dir, Y);
        sh_basis_grad(sh_degree, dir, dY);
        const double* shg = sh + (size_t)g * K * 3;
        double* dshg = dsh + (size_t)g * K * 3;
        double ddir[3] = {0.0, 0.0, 0.0};
        for (int ch = 0; ch < 3; ++ch) {
            double a = 0.5;
            for (int k = 0; k < K; ++k) a += Y[k] * shg[3 * k + ch];
            double gc = a < 0.0 ? 0.0 : drgb[3 * g + ch];
            for (int k = 0; k < K; ++k) {
                dshg[3 * k + ch] = Y[k] * gc;
                for (int j = 0; j < 3; ++j) ddir[j] += gc * shg[3 * k + ch] * dY[k][j];
            }
        }
        double dd = dir[0] * ddir[0] + dir[1] * ddir[1] + dir[2] * ddir[2];
        for (int j = 0; j < 3; ++j) dmu[j] += (ddir[j] - dir[j] * dd) / dn;
    }
}
