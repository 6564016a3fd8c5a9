/*
 * tcgs.h -- C ABI of the GB300 (sm_103a) TC-GS rasterizer library (libtcgs.so).
 *
 * TC-GS ("A Faster Gaussian Splatting Module Utilizing Tensor Cores") renders
 * 3D Gaussian Splatting scenes in three stages (Sec. 3.1): preprocess
 * (projection), sorting (tile binning + depth sort) and conditional
 * alpha-blending (Algorithm 1).  Its contribution is the third stage:
 * EarlyCull (Sec. 4.1), Frag2Mat (Sec. 4.2, the exponent of every
 * pixel-Gaussian pair as one matrix product B = U^T V on tensor cores) and
 * G2L (Sec. 4.3, tile-local coordinates so the quadratic pixel terms survive
 * half precision).
 *
 * General rules for every call:
 *   - All array arguments are DEVICE pointers owned by the caller, unless the
 *     argument's comment says "host".  The library never allocates, frees or
 *     keeps a pointer after the call returns.
 *   - Every call only enqueues work on `stream` (NULL = the legacy default
 *     stream) and returns without synchronising.  Argument errors are detected
 *     on the host and returned at once (TCGS_ERR_INVALID, nothing enqueued).
 *     A launch failure returns TCGS_ERR_CUDA.  Errors found on the device
 *     (capacity overflow, a timed-out wait) are written to a caller-provided
 *     device status word, readable after the stream is synchronised.
 *   - Arrays are dense, row-major, float32 unless stated otherwise.
 *   - Pixel (i, j) is sampled at (i + 0.5, j + 0.5).  Tiles are 16 x 16
 *     pixels, numbered row-major: tile = ty * ceil(W / 16) + tx.
 *   - Gradient outputs are ACCUMULATED (+=): the caller zeroes them.
 */
#ifndef TCGS_H
#define TCGS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TCGS_API __attribute__((visibility("default")))
#else
#define TCGS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t (CUstream); NULL selects the legacy default stream. */
typedef struct CUstream_st* tcgs_stream;

typedef enum {
    TCGS_OK = 0,
    TCGS_ERR_INVALID = 1,     /* bad argument (null pointer, negative size, unsupported option) */
    TCGS_ERR_CUDA = 2,        /* a CUDA runtime call or kernel launch failed */
    TCGS_ERR_CAPACITY = 3,    /* more splats than the caller's capacity (device status word) */
    TCGS_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up (device status word) */
    TCGS_ERR_UNSUPPORTED = 5, /* the current device cannot run this call (not sm_103a) */
    TCGS_ERR_SCRATCH_LIMIT = 6 /* the request needs more scratch than the built-in array holds */
} tcgs_status;

/* How the exponent beta = ln(o) - 1/2 d^T Sigma'^-1 d of Eq. (9) is evaluated. */
typedef enum {
    TCGS_FP32 = 0,          /* CUDA cores, FP32, Eq. (4) per fragment: the 3DGS baseline */
    TCGS_TC_FP16 = 1,       /* Frag2Mat + G2L on tensor cores, FP16 inputs, FP32 accumulate, with
                               the paper's K = 8 padding (v0 / 3 in three slots, Sec. 5.1) */
    TCGS_TC_FP16_SPLIT = 2, /* as TC_FP16 but v = v_hi + v_lo in FP16 over K = 16 (u duplicated) */
    TCGS_TC_FP8 = 3,        /* trial: Frag2Mat + G2L on FP8 e4m3 inputs (K = 32 per MMA): u = u_hi + u_lo
                               exactly, v = v_hi + v_lo + v_lo2, power-of-two column scales; FP32
                               accumulate (accuracy reported; not a faster path) */
    TCGS_TC_TF32 = 4,       /* Frag2Mat + G2L on TF32 inputs (K = 8 per MMA), FP32 accumulate */
    TCGS_TC_FP16_GLOBAL = 5,/* ablation of Table 5: Frag2Mat WITHOUT G2L, u and v in global pixel
                               coordinates, FP16 inputs in the TC_FP16 layout (overflows to inf past
                               256 px; non-finite exponents are culled).  Every list entry is walked
                               (tile_cull ignored).  tcgs_render_fwd and tcgs_frag2mat_beta only */
    TCGS_TC_TF32_GLOBAL = 6,/* ablation of Table 5: as TC_FP16_GLOBAL with TF32 inputs */
    TCGS_FP32_FRAG2MAT = 7  /* the tensor-core renderer with its product u^T v (Eq. 18, G2L coefficients
                               of Eq. 12) evaluated on CUDA cores in FP32: the same persistent schedule,
                               staging, per-block skip (tile_cull) and EarlyCull, no tensor core.  The
                               ablation arm that isolates what the tensor-core product buys (Table 4) */
} tcgs_precision;

/* Pinhole camera.  mean2d = (fx X / Z + cx, fy Y / Z + cy) for camera-space (X, Y, Z). */
typedef struct {
    int32_t width, height;     /* image size in pixels (>= 1) */
    float fx, fy, cx, cy;      /* focal lengths and principal point, pixels */
    float viewmat[12];         /* row-major 3x4 world -> camera [R | t] */
    float campos[3];           /* camera centre in world coordinates (SH view direction) */
    float near_z;              /* Gaussians with camera Z <= near_z are culled */
    float tan_fovx, tan_fovy;  /* frustum clamp of the Jacobian at 1.3 tan; <= 0: W / (2 fx), H / (2 fy) */
} tcgs_camera;

/* Options of the alpha-blending calls. */
typedef struct {
    int32_t precision;       /* tcgs_precision */
    float alpha_max;         /* alpha clamp (0.99 as in the official 3DGS renderer; 1 = Algorithm 1 literally) */
    int32_t early_cull;      /* 1 = EarlyCull (Sec. 4.1): cull on beta < -ln 255, tested before the exponential;
                                0 = cull on alpha < 1/255 after it (Eq. 5, the 3DGS baseline).  On the TC paths
                                the walk is branch-free and evaluates ex2 for every walked fragment either way:
                                the option changes the test, not the work */
    int32_t tile_cull;       /* TC paths: 1 = skip, per 8x4 pixel block, list entries whose Gaussian cannot
                                reach alpha >= 1/255 at any pixel of the block (exact minimum of the conic
                                form over the block; the image is unchanged); 0 = walk every entry */
    uint32_t* tile_stats;    /* nullable device [num_tiles * 8], accumulated (+=) per tile:
                                [0] blended fragments, [1] evaluated but not blended fragments
                                (culled, plus the fragment that triggers termination),
                                [2] fragment slots the kernel executed (pixels x list entries walked),
                                [3] list length n(T), [4] list entries the tile's CTA walked before all
                                its pixels terminated, [5] the tile's CTA time in SM clock cycles / 64,
                                [6], [7] reserved (0) */
    int32_t* device_status;  /* nullable device int32: set to a tcgs_status on a device-side error */
    const uint32_t* tile_order; /* nullable device [num_tiles]: TC precisions in tile-local coordinates
                                and TCGS_FP32_FRAG2MAT render with a persistent grid (4 CTAs per SM) that takes the tiles in this
                                order, a permutation of all tiles such as tcgs_tile_order's (the order
                                changes the schedule, never the image); NULL: one CTA per tile.  A view
                                of at most tcgs_tc_wave_tiles() tiles is rendered one CTA per tile even
                                when an order is given: every tile then starts in the first wave */
    uint32_t* work_counter;  /* device uint32, required with tile_order: the grid's next-tile counter,
                                zeroed by the call */
    int32_t pixels_per_thread; /* 0 or 1: the tensor-core renderer's consumer threads blend one pixel
                                each, its warps own 8x4 blocks (the default); 2: two pixels each, four
                                rows apart (one in each MMA half, the same TMEM lane), warps owning 8x8
                                blocks, so every walked list entry serves 64 pixels at the cost of coarser
                                block marks: faster for views of large footprints, whose batches mark most
                                entries anyway, slower for views of small ones.  Honoured by
                                TCGS_TC_FP16_SPLIT and TCGS_FP32_FRAG2MAT with early_cull = 1 in
                                tcgs_render_fwd; the other configurations, and tcgs_render_fwd_batched,
                                render with one.  The image is the same either way */
} tcgs_render_opts;

/* Human-readable name of a status code (static string). */
TCGS_API const char* tcgs_status_string(int status);

/* Library version, 100 * major + minor. */
TCGS_API int tcgs_version(void);

/* Number of CUDA kernels this library has launched in this process so far (a host-side counter,
 * incremented once per kernel launch; no device work, no synchronisation). */
TCGS_API uint64_t tcgs_kernel_launches(void);

/*
 * Preprocess (Sec. 3.1, Eq. 2): EWA projection of P 3D Gaussians.
 *   Sigma = R(q) diag(s)^2 R(q)^T, t = W mu, J = d(mean2d)/d(t) at t with x/z, y/z
 *   clamped to +-1.3 tan_fov, Sigma' = J W Sigma W^T J^T + 0.3 I (low-pass dilation),
 *   conic = Sigma'^-1 = (sigma11, sigma12, sigma22), radius = half-width of the coverage square
 *   (below), lambda_max = m + sqrt(max(0.1, m^2 - det)), m = (a + c) / 2.
 *   Colour = sum_k sh[k] Y_k(dir) + 0.5 clamped at 0, dir = (mu - campos) / |mu - campos|,
 *   real SH up to degree 3 (3DGS convention).
 * Coverage square: with opacity == NULL, the 3-sigma square of official 3DGS,
 *   radius = ceil(3 sqrt(lambda_max)); with opacity [P] (post-sigmoid), the opacity-aware square
 *   that bounds the ellipse where alpha = o exp(-q/2) >= 1/255 (Eq. 5),
 *   radius = ceil(sqrt(2 ln(255 o) lambda_max)), and Gaussians with o <= 1/255 are culled.
 * In:  means3 [P,3]; scales [P,3] (standard deviations, > 0); quats [P,4] (w,x,y,z, any
 *      non-zero norm); sh [P, (sh_degree+1)^2, 3]; 0 <= sh_degree <= 3; opacity [P] or NULL.
 * Out: mean2d [P,2]; conic [P,3]; depth [P] (camera Z); radius [P] int32 (0 = culled: behind the
 *      near plane, degenerate, or touching no tile); rgb [P,3]; tiles_touched [P] uint32.
 *      Culled Gaussians get zeros in every output.
 * P = 0 is valid (nothing is launched).
 */
TCGS_API tcgs_status tcgs_project(const tcgs_camera* cam /* host */, int32_t P, int32_t sh_degree,
                         const float* means3, const float* scales, const float* quats, const float* sh,
                         const float* opacity /* nullable */, float* mean2d, float* conic, float* depth, int32_t* radius, float* rgb,
                         uint32_t* tiles_touched, tcgs_stream stream);

/*
 * Backward of tcgs_project (Sec. 3.1, Eq. 2): given dL/d(mean2d, conic, rgb) of every Gaussian,
 * accumulates (+=) dL/d(means3, scales, quats, sh).  conic is (sigma11, sigma12, sigma22) and
 * dconic[1] is the derivative with respect to the one parameter sigma12 that fills both
 * off-diagonal entries, as tcgs_render_bwd produces it.  Per Gaussian the forward is recomputed
 * and differentiated step by step: conic = Sigma'^-1, Sigma' = J W Sigma W^T J^T + 0.3 I (J at the
 * frustum-clamped mean: a clamped coordinate passes no gradient through J), Sigma = M M^T with
 * M = R(q / |q|) diag(s), mean2d of the camera-space mean, and the SH colour including its
 * view-direction term (a colour channel clamped at 0 passes none).  Depth, radius and the
 * culling decisions are not differentiable; Gaussians with radius[g] <= 0 are skipped.
 * In:  as tcgs_project (without opacity), radius [P] int32 from the forward, dmean2d [P,2],
 *      dconic [P,3], drgb [P,3].
 * Out: dmeans3 [P,3], dscales [P,3], dquats [P,4], dsh [P, (sh_degree+1)^2, 3], accumulated.
 */
TCGS_API tcgs_status tcgs_project_bwd(const tcgs_camera* cam /* host */, int32_t P, int32_t sh_degree,
                             const float* means3, const float* scales, const float* quats, const float* sh,
                             const int32_t* radius, const float* dmean2d, const float* dconic,
                             const float* drgb, float* dmeans3, float* dscales, float* dquats, float* dsh,
                             tcgs_stream stream);

/* Bytes of device workspace tcgs_bin_sort needs (a pure host function). */
TCGS_API size_t tcgs_bin_sort_workspace_size(int32_t P, int64_t splat_capacity, int32_t num_tiles);

/*
 * Sorting stage (Sec. 3.1, Eq. 3): build the splats (tile, Gaussian), order every tile's
 * list by increasing depth (ties: increasing Gaussian index) and find each tile's range.
 * Gaussian g covers tile (tx, ty) iff [mx - r, mx + r] x [my - r, my + r] meets the tile's
 * pixel square [16 tx, 16 tx + 16) x [16 ty, 16 ty + 16), r = radius[g] > 0.
 * The order is the (tile, depth-bits) key order of the paper's radix sort; it is produced by
 * an LSD radix sort whose depth digits run before duplication (on P keys) and whose tile
 * digits run after it (on N keys).  A small view (at most 256 tiles, P <= 8192 and
 * splat_capacity <= 32768) runs the same passes in two single-CTA kernels (4 launches in all,
 * against about 20), with the same result.  With two tile passes and splat_capacity >= 2^23, the
 * first tile pass packs (tile >> 8, Gaussian id) into one word when they fit 32 bits, and the second
 * writes the ranges from per-tile counts: again the same result.  Empty tiles get [0, 0).
 * In:  mean2d [P,2], radius [P], depth [P] (> 0 where radius > 0).
 * Out: ids_sorted [splat_capacity] uint32 (first N entries valid), tile_ranges [num_tiles, 2]
 *      uint32 [start, end), n_splats: device int64 = N, status: device int32 (TCGS_OK, or
 *      TCGS_ERR_CAPACITY when N > splat_capacity; then ids_sorted is untouched and every range
 *      is empty).
 * workspace: device, ws_bytes >= tcgs_bin_sort_workspace_size(P, splat_capacity, num_tiles),
 *      256-byte aligned; contents are scratch.  splat_capacity <= 2^32 - 1.
 */
TCGS_API tcgs_status tcgs_bin_sort(const tcgs_camera* cam /* host */, int32_t P, const float* mean2d,
                          const int32_t* radius, const float* depth, int64_t splat_capacity,
                          void* workspace, size_t ws_bytes, uint32_t* ids_sorted, uint32_t* tile_ranges,
                          int64_t* n_splats, int32_t* status, tcgs_stream stream);

/*
 * tcgs_bin_sort with exact tile coverage.  The paper leaves the Gaussian-tile coverage test to the
 * implementation (Sec. 3.1: it "depends on the specific algorithm"; Sec. 2 cites methods that cut
 * the Gaussian-tile pairs).  Here splat (g, t) is made only when t lies in g's rectangle (as for
 * tcgs_bin_sort) AND g can reach alpha >= 1/255 (Eq. 5) at some pixel centre of t:
 *   min over the pixel-centre box of t of (m - p)^T Q (m - p)  <=  L(o),
 *   L(o) = 2 (ln o + ln 255) (1 + 1e-4) + 1e-3   (no tile when 2 (ln o + ln 255) <= -1e-3),
 * with m = mean2d[g], Q = the conic of g, o = opacity[g], evaluated in FP32 (the minimum over the
 * box in tile-local coordinates, in closed form: 0 when m is inside, else the least of the four edge
 * minima).  A dropped splat is culled at every pixel of its tile by Algorithm 1, and the margins make
 * that hold for the FP32 and tensor-core renderers' own arithmetic too, so every image rendered from
 * these lists equals the image rendered from tcgs_bin_sort's (only list positions, and so
 * n_contrib, differ).  Order, ranges, outputs, workspace and status as tcgs_bin_sort.
 * When splat_capacity >= 32 P (wide footprints), Gaussians whose rectangle is at least 6 tiles wide
 * are covered row by row: in a tile row the reached tiles form one run (the region q <= L is
 * convex), found from the ellipse's extent with its end tiles settled by the test above, so the
 * lists are the same; this needs Q positive definite, as tcgs_project makes it.
 * In:  conic [P,3], opacity [P] (post-sigmoid) as given to the renderer; both non-null when P > 0.
 */
TCGS_API tcgs_status tcgs_bin_sort_exact(const tcgs_camera* cam /* host */, int32_t P, const float* mean2d,
                                         const int32_t* radius, const float* depth, const float* conic,
                                         const float* opacity, int64_t splat_capacity, void* workspace,
                                         size_t ws_bytes, uint32_t* ids_sorted, uint32_t* tile_ranges,
                                         int64_t* n_splats, int32_t* status, tcgs_stream stream);

/* Size of the scratch array built into the library for tcgs_bin_sort_noalloc (64 MiB). */
#define TCGS_BIN_SORT_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)

/*
 * tcgs_bin_sort for callers that cannot allocate device memory.  The paper has no counterpart.
 * Some callers have no way to obtain a scratch buffer: code that runs while another component owns
 * every allocation (a host application's memory manager, a framework allocator that only hands
 * out its own tensors), code on a real-time or latency-critical path where cudaMalloc would
 * synchronise the device, or thin C callers with no CUDA memory management of their own.  They
 * still pass the inputs and outputs exactly as for tcgs_bin_sort; only `workspace` is replaced by
 * a static device array of TCGS_BIN_SORT_NOALLOC_SCRATCH_BYTES inside libtcgs.so, which every GPU
 * that loads the library holds until the process exits.
 *   - Requests whose tcgs_bin_sort_workspace_size(P, splat_capacity, num_tiles) exceeds the array
 *     return TCGS_ERR_SCRATCH_LIMIT at once (nothing enqueued).  64 MiB holds, for example,
 *     P = 1,000 Gaussians with 5.4 million splats, or P = 500,000 with 4.5 million.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress with
 *     that device current) and caches it with the device's current CUDA context; make that first
 *     call before any stream capture.  A call that finds another context current on the device
 *     (after cudaDeviceReset, or after the primary context was released and created again) looks
 *     the address up again, so it too should come before any capture.
 *   - The call allocates nothing (no cudaMalloc, cudaFree or allocating library routine).
 *   - All calls share the one array and it keeps whatever the previous call left there; the
 *     kernels initialise every scratch word they read, so no clearing is needed between calls.
 *     Calls that overlap on the GPU (two streams, or two host threads) race on the array and
 *     produce garbage: serialise them.
 * Arguments, outputs and device status as tcgs_bin_sort.
 */
TCGS_API tcgs_status tcgs_bin_sort_noalloc(const tcgs_camera* cam /* host */, int32_t P, const float* mean2d,
                                           const int32_t* radius, const float* depth, int64_t splat_capacity,
                                           uint32_t* ids_sorted, uint32_t* tile_ranges, int64_t* n_splats,
                                           int32_t* status, tcgs_stream stream);

/*
 * Conditional alpha-blending (Algorithm 1), front to back per pixel over its tile's list:
 *   alpha = min(alpha_max, o exp(beta)), beta from Eq. (9);  cull if alpha < 1/255 (Eq. 5; the
 *   TC paths test beta < -ln 255 first, Sec. 4.1);  break (without blending) if
 *   T - alpha T < 1e-4;  C += c alpha T;  T -= alpha T.  Final colour C + T bg.
 * TC precisions compute every beta of a 128-pixel half tile and a batch of Gaussians as one
 * tcgen05 MMA (Eq. 18) in tile-local coordinates (Sec. 4.3) and need sm_103a.
 * In:  tile_ranges, ids_sorted from tcgs_bin_sort; mean2d [P,2]; conic [P,3]; opacity [P] in
 *      (0, 1]; rgb [P,3]; bg3: host float[3] background.
 * Out: img [3,H,W]; T_final [H,W]; n_contrib [H,W] uint32 = 1 + (list index of the last blended
 *      fragment), 0 if none.
 * TC preconditions: the largest eigenvalue of the conic is at most 1000 px^-2 (the projection's
 *      0.3 px^2 dilation keeps it below 3.34); otherwise FP16 saturates and the result is
 *      unspecified (finite).
 */
TCGS_API tcgs_status tcgs_render_fwd(const tcgs_camera* cam /* host */, const tcgs_render_opts* opts /* host */,
                            const uint32_t* tile_ranges, const uint32_t* ids_sorted, const float* mean2d,
                            const float* conic, const float* opacity, const float* rgb,
                            const float* bg3 /* host */, float* img, float* T_final, uint32_t* n_contrib,
                            tcgs_stream stream);

/*
 * Longest-first order of a view's tiles for the persistent renderer (tcgs_render_opts.tile_order):
 * every tile once, grouped by floor(log2(list length)) from the longest group to the empty tiles,
 * in tile order inside a group (neighbouring tiles share Gaussians).  The order decides only which
 * CTA renders a tile, and when.  The paper has no counterpart: its blending launches one thread
 * block per tile.
 * In:  tile_ranges [num_tiles, 2] from the sorting stage.  Out: tile_order [num_tiles] (device).
 */
TCGS_API tcgs_status tcgs_tile_order(const tcgs_camera* cam /* host */, const uint32_t* tile_ranges,
                                     uint32_t* tile_order, tcgs_stream stream);

/*
 * Tiles the tensor-core renderer keeps resident at once on the current device (4 CTAs per SM; 608 on
 * a 152-SM GB300), or 0 when the device is not sm_103.  A view with at most this many tiles starts
 * every tile in the first wave, where no order can shorten the schedule: tcgs_render_fwd then ignores
 * tile_order (and leaves work_counter alone), so a caller may skip tcgs_tile_order for such views.
 */
TCGS_API int32_t tcgs_tc_wave_tiles(void);

/* Largest number of views one batched launch can render. */
#define TCGS_MAX_VIEWS 16

/* One view of a batched render: its camera, its projection and sort outputs, and its outputs
 * (all device pointers as in tcgs_render_fwd; tile_stats nullable, [num_tiles * 8]). */
typedef struct {
    tcgs_camera cam;
    const uint32_t* tile_ranges;
    const uint32_t* ids_sorted;
    const float* mean2d;
    const float* conic;
    const float* rgb;
    float* img;
    float* T_final;
    uint32_t* n_contrib;
    uint32_t* tile_stats;
} tcgs_view;

/*
 * Batched multi-view conditional alpha-blending with a persistent scheduler: a grid of resident
 * CTAs (at most max_ctas when > 0) repeatedly takes the next work item from `queue` with an atomic
 * counter and renders that tile exactly as tcgs_render_fwd does (same per-tile body, so every image
 * is identical to a per-view launch whatever the queue order).  An item is (view << 16) | tile.
 * The order of `queue` decides the schedule only: a longest-predicted-first order shortens the
 * makespan when tile costs are uneven.  TC precisions with G2L (not the *_GLOBAL ablations) and
 * TCGS_FP32_FRAG2MAT (the same kernel with the product on CUDA cores).
 * In:  n_views in [1, TCGS_MAX_VIEWS] views (host array of tcgs_view), opacity [P] shared by all
 *      views, bg3 host float[3], queue: device [n_items] uint32.
 * work_counter: device uint32, scratch (reset by the call on `stream`).
 */
TCGS_API tcgs_status tcgs_render_fwd_batched(int32_t n_views, const tcgs_view* views /* host */,
                                             const tcgs_render_opts* opts /* host */, const float* opacity,
                                             const float* bg3 /* host */, const uint32_t* queue, int32_t n_items,
                                             uint32_t* work_counter, int32_t max_ctas, tcgs_stream stream);

/* ---------------------------------------------------------------------------------------------
 * Learned tile-cost model for the batched renderer's queue (not part of the paper).  The paper has
 * no counterpart: it is the scheduling layer a batched multi-view pipeline needs once each tile's
 * alpha-blending is fast.  An MLP 8 -> 32 -> 32 -> 1 (ReLU, FP16 weights and activations, FP32
 * accumulation) predicts log(tile cost) from per-tile statistics.
 * Parameters (float32 masters, TCGS_MLP_PARAMS values): W1[32][8], b1[32], W2[32][32], b2[32],
 * W3[32], b3.  The forward rounds every weight, the normalised input and both hidden activations
 * to FP16; products and sums are FP32.
 * ------------------------------------------------------------------------------------------- */
#define TCGS_MLP_IN 8
#define TCGS_MLP_HIDDEN 32
#define TCGS_MLP_PARAMS 1377

/* Per-tile features of one view, [num_tiles, 8] float32:
 *   0 log(1 + n(T)), 1 mean opacity, 2 max opacity, 3 log(1 + depth span), 4 mean log det(conic),
 *   5 log(1 + coverage) with coverage = sum over the list of |3-sigma square ∩ tile| / 256,
 *   6 log(W H), 7 fraction of the tile's pixels inside the image (empty list: 0, 0, 0, 0, 0, 0, .). */
TCGS_API tcgs_status tcgs_tile_features(const tcgs_camera* cam /* host */, const uint32_t* tile_ranges,
                                        const uint32_t* ids_sorted, const float* mean2d, const float* conic,
                                        const float* opacity, const float* depth, const int32_t* radius,
                                        float* features, tcgs_stream stream);

/* Feature normaliser of n rows of x [n, 8]: norm[0..7] = column means, norm[8..15] = 1 / std. */
TCGS_API tcgs_status tcgs_feature_norm(const float* x, int32_t n, float* norm, tcgs_stream stream);

/* y[i] = MLP((x[i] - norm[0..7]) * norm[8..15]) for n rows of x [n, 8]. */
TCGS_API tcgs_status tcgs_mlp_fwd(const float* params, const float* norm, const float* x, int32_t n, float* y,
                                  tcgs_stream stream);

/* Gradient of L = (1/n) sum_i (MLP(x_i) - target_i)^2, accumulated (+=) into grad [TCGS_MLP_PARAMS];
 * loss (nullable, device float) accumulates L.  The backward uses the forward's FP16-rounded values
 * and passes through the rounding unchanged. */
TCGS_API tcgs_status tcgs_mlp_bwd(const float* params, const float* norm, const float* x, const float* target,
                                  int32_t n, float* grad, float* loss, tcgs_stream stream);

/* One Adam step (bias-corrected, step >= 1) on n_params parameters; grad is consumed (set to 0). */
TCGS_API tcgs_status tcgs_adam_step(float* params, float* m, float* v, float* grad, int32_t n_params, float lr,
                                    float beta1, float beta2, float eps, int32_t step, tcgs_stream stream);

/* Bytes of device workspace tcgs_sched_order needs for n items (host function). */
TCGS_API size_t tcgs_sched_order_workspace_size(int32_t n);

/* queue_out = items ordered by decreasing cost (ties keep their input order): a stable LSD radix
 * sort of the cost's order-preserving bits, 4 passes of 8 bits. */
TCGS_API tcgs_status tcgs_sched_order(const float* cost, const uint32_t* items, int32_t n, uint32_t* queue_out,
                                      void* workspace, size_t ws_bytes, tcgs_stream stream);

/*
 * Backward of Algorithm 1 (C = sum_j c_j a_j T_j + bg T_final, Eq. 6) w.r.t. mean2d, conic,
 * opacity and rgb, replaying each pixel's fragments 0 .. n_contrib-1 front to back with the
 * FP32 forward's alpha arithmetic:
 *   dL/dc_j = a_j T_j g;  dL/da_j = g . (c_j T_j - S_j / (1 - a_j)), S_j = colour blended after j
 *   plus bg T_final;  through a = o exp(p) when unclamped: dL/do = dL/da a / o,
 *   dL/dp = dL/da a, dp/dmean = -Q d, dp/dsigma11 = -d_x^2 / 2, dp/dsigma12 = -d_x d_y,
 *   dp/dsigma22 = -d_y^2 / 2 (d = mean2d - pixel).  Clamped fragments pass no gradient to p, o.
 * In:  as tcgs_render_fwd plus its outputs img, T_final, n_contrib, and dL_dimg [3,H,W].
 * Out (accumulated): dmean2d [P,2], dconic [P,3], dopacity [P], drgb [P,3].
 * opts->precision is ignored (the replay is FP32); opts->alpha_max must match the forward.
 */
TCGS_API tcgs_status tcgs_render_bwd(const tcgs_camera* cam /* host */, const tcgs_render_opts* opts /* host */,
                            const uint32_t* tile_ranges, const uint32_t* ids_sorted, const float* mean2d,
                            const float* conic, const float* opacity, const float* rgb,
                            const float* bg3 /* host */, const float* img, const float* T_final,
                            const uint32_t* n_contrib, const float* dL_dimg, float* dmean2d, float* dconic,
                            float* dopacity, float* drgb, tcgs_stream stream);

/*
 * Frag2Mat exponents as the tensor cores compute them (Eq. 18; in the G2L frame of Sec. 4.3, or
 * in global pixel coordinates for the *_GLOBAL ablations), for inspection against the error bound
 * of Appendix A.  For each of n_tiles tiles (device
 * tiles[n_tiles] int32) and each of the first min(max_n, n(T)) list entries, writes
 * beta_hat in natural-log units to beta_out [n_tiles, 256, max_n] (pixel-major within the tile,
 * row-major pixels; entries past the list end are set to -INFINITY).
 * precision: any TC precision (TC_FP16, TC_FP16_SPLIT, TC_FP8, TC_TF32, TC_FP16_GLOBAL, TC_TF32_GLOBAL).
 */
TCGS_API tcgs_status tcgs_frag2mat_beta(const tcgs_camera* cam /* host */, int32_t precision, const uint32_t* tile_ranges,
                               const uint32_t* ids_sorted, const float* mean2d, const float* conic,
                               const float* opacity, int32_t n_tiles, const int32_t* tiles, int32_t max_n,
                               float* beta_out, int32_t* device_status, tcgs_stream stream);

/*
 * Self-test of the device-side failure reporting: one kernel waits, with the bounded mbarrier wait
 * that the tensor-core renderer uses, on a barrier that nothing completes.  After `polls` polls
 * (1 .. 2^22; the renderer uses 2^22) the wait gives up and TCGS_ERR_TIMEOUT is written to
 * device_status (device int32, first error wins); the context stays usable.
 */
TCGS_API tcgs_status tcgs_selftest_bounded_wait(int32_t* device_status, uint32_t polls, tcgs_stream stream);

/*
 * Microbenchmark of the special-function unit: `blocks` blocks of 256 threads, each thread running 8
 * independent chains of `iters` base-2 exponentials (ex2.approx.ftz.f32, the one transcendental
 * the tensor-core renderer evaluates per walked slot), so blocks x 256 x 8 x iters exponentials in
 * all; out: device float [blocks x 256] (a checksum).  Timed by the caller (CUDA events).
 */
TCGS_API tcgs_status tcgs_microbench_ex2(float* out, int32_t blocks, int32_t iters, tcgs_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* TCGS_H */
