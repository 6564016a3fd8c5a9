"""Seeded synthetic inputs shaped like the scenes TC-GS renders.

This module only draws random numbers and builds cameras; it contains none
of the rasterizer's arithmetic (no projection, no SH evaluation, no
compositing).  It feeds both the CUDA path and the FP64 oracle.

Every generator uses numpy's PCG64 with a fixed seed and returns float32
arrays (the precision the library consumes):

  means3  [P, 3]   world-space means
  scales  [P, 3]   per-axis standard deviations (exp of the log-scales)
  quats   [P, 4]   (w, x, y, z), not necessarily normalised
  opacity [P]      post-sigmoid opacity in (0, 1)
  sh      [P, K, 3] SH coefficients, K = (degree + 1)^2
  sh_degree int

A camera is a plain dict: width, height, fx, fy, cx, cy, viewmat (3x4
row-major world -> camera), campos, near_z.
"""
from __future__ import annotations

import numpy as np

SQRT_PI = float(np.sqrt(np.pi))  # DC coefficient range that maps to colours in [0, 1]


def pinhole(width: int, height: int, fx: float, fy: float | None = None, viewmat=None, campos=None,
            near_z: float = 0.2) -> dict:
    """Camera with the principal point at the image centre."""
    fy = fx if fy is None else fy
    vm = np.hstack([np.eye(3), np.zeros((3, 1))]) if viewmat is None else np.asarray(viewmat, np.float64)
    return dict(width=int(width), height=int(height), fx=float(fx), fy=float(fy), cx=width / 2.0,
                cy=height / 2.0, viewmat=vm.astype(np.float32).astype(np.float64),
                campos=np.zeros(3) if campos is None else np.asarray(campos, np.float64), near_z=float(near_z))


def look_at(eye, target, width: int, height: int, fx: float) -> dict:
    """Camera at ``eye`` looking at ``target``; image y points along world +y
    (x right, y down, z forward as for the identity camera)."""
    eye = np.asarray(eye, np.float64); target = np.asarray(target, np.float64)
    z = target - eye
    z /= np.linalg.norm(z)
    x = np.cross(np.array([0.0, 1.0, 0.0]), z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z])
    vm = np.hstack([R, (-R @ eye)[:, None]])
    return pinhole(width, height, fx, viewmat=vm, campos=eye)


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _quats(rng, P):
    return rng.standard_normal((P, 4))


def _sh(rng, P, degree, high_std):
    K = (degree + 1) ** 2
    sh = np.zeros((P, K, 3))
    sh[:, 0, :] = rng.uniform(-SQRT_PI, SQRT_PI, (P, 3))  # colour uniform in [0, 1]
    if K > 1:
        sh[:, 1:, :] = rng.normal(0.0, high_std, (P, K - 1, 3))
    return sh


def _pack(means3, scales, quats, opacity, sh, degree) -> dict:
    f = np.float32
    return dict(means3=np.ascontiguousarray(means3, f), scales=np.ascontiguousarray(scales, f),
                quats=np.ascontiguousarray(quats, f), opacity=np.ascontiguousarray(opacity, f),
                sh=np.ascontiguousarray(sh, f), sh_degree=int(degree))


def uniform_box(rng, P, xy=2.0, z=(2.0, 10.0), log_scale=(-3.0, 0.5), sh_degree=0, sh_high_std=0.05) -> dict:
    """Means uniform in [-xy, xy]^2 x [z0, z1]; log-scales N(mu, sd) per axis;
    uniform random rotations; opacity sigmoid(N(0, 1)); colour uniform."""
    means = np.stack([rng.uniform(-xy, xy, P), rng.uniform(-xy, xy, P), rng.uniform(z[0], z[1], P)], axis=1)
    scales = np.exp(rng.normal(log_scale[0], log_scale[1], (P, 3)))
    quats = _quats(rng, P)
    opacity = _sigmoid(rng.standard_normal(P))
    return _pack(means, scales, quats, opacity, _sh(rng, P, sh_degree, sh_high_std), sh_degree)


def clustered(rng, P, n_clusters, cam, z_range=(1.0, 50.0), log_scale=(-4.5, 1.0), bimodal_opacity=True,
              sh_degree=3, sh_high_std=0.05, box=None) -> dict:
    """Means from an anisotropic Gaussian mixture inside the camera frustum
    (or inside ``box`` = (xy, z0, z1) when given); z clipped to z_range."""
    if box is None:
        zc = rng.uniform(z_range[0] + 3.0, 0.8 * z_range[1], n_clusters)
        xc = zc * rng.uniform(-0.75, 0.75, n_clusters) * (cam["width"] / 2.0) / cam["fx"]
        yc = zc * rng.uniform(-0.75, 0.75, n_clusters) * (cam["height"] / 2.0) / cam["fy"]
        spread = zc[:, None] * rng.uniform(0.01, 0.08, (n_clusters, 3))
    else:
        xy, z0, z1 = box
        zc = rng.uniform(z0, z1, n_clusters)
        xc = rng.uniform(-xy, xy, n_clusters)
        yc = rng.uniform(-xy, xy, n_clusters)
        spread = rng.uniform(0.02, 0.3, (n_clusters, 3))
    centres = np.stack([xc, yc, zc], axis=1)
    axes = np.linalg.qr(rng.standard_normal((n_clusters, 3, 3)))[0]  # random orthonormal frames
    labels = rng.integers(0, n_clusters, P)
    local = rng.standard_normal((P, 3)) * spread[labels]
    means = centres[labels] + np.einsum("pij,pj->pi", axes[labels], local)
    if box is None:
        means[:, 2] = np.clip(means[:, 2], z_range[0], z_range[1])
    else:
        means[:, 0] = np.clip(means[:, 0], -box[0], box[0])
        means[:, 1] = np.clip(means[:, 1], -box[0], box[0])
        means[:, 2] = np.clip(means[:, 2], box[1], box[2])
    scales = np.exp(rng.normal(log_scale[0], log_scale[1], (P, 3)))
    quats = _quats(rng, P)
    if bimodal_opacity:
        hi = rng.random(P) < 0.7
        opacity = np.where(hi, _sigmoid(rng.normal(3.0, 1.0, P)), _sigmoid(rng.normal(-3.0, 1.0, P)))
    else:
        opacity = _sigmoid(rng.standard_normal(P))
    return _pack(means, scales, quats, opacity, _sh(rng, P, sh_degree, sh_high_std), sh_degree)


# --------------------------------------------------------------------------
# The five workloads (seed = workload number).
# --------------------------------------------------------------------------

def plain_forward(P=1000, width=128, height=128, seed=1):
    """Plain forward: 1 view 128x128, fx = fy = 128, 1,000 Gaussians, SH degree 0."""
    rng = np.random.default_rng(seed)
    cam = pinhole(width, height, fx=128.0 * width / 128.0)
    return cam, uniform_box(rng, P)


def precision(P=1_000_000, width=1920, height=1080, seed=2):
    """Precision: 1 view 1920x1080, fx = fy = 1100, 1M Gaussians, 64 clusters, SH degree 3."""
    rng = np.random.default_rng(seed)
    cam = pinhole(width, height, fx=1100.0 * width / 1920.0)
    return cam, clustered(rng, P, 64, cam)


def differentiation(P=500_000, width=1280, height=720, seed=3):
    """Differentiation: 1 view 1280x720, fx = fy = 1280, 500k Gaussians drawn as in the plain
    workload, plus a seeded target image in [0, 1]."""
    rng = np.random.default_rng(seed)
    cam = pinhole(width, height, fx=float(width))
    scene = uniform_box(rng, P)
    target = rng.random((3, height, width)).astype(np.float32)
    return cam, scene, target


def wide_field(P=3000, width=160, height=96, seed=17):
    """Parity case for the frustum clamp: a 160x96 view (fx = fy = 128) of Gaussians whose means
    spread to about three times the half field of view (x, y in [-6, 6], z in [2, 10]), with
    log-scales N(-1.5, 0.5) so that many of those outside the frustum still reach the image."""
    rng = np.random.default_rng(seed)
    cam = pinhole(width, height, fx=128.0)
    return cam, uniform_box(rng, P, xy=6.0, log_scale=(-1.5, 0.5))


RESOLUTIONS = [(640, 480), (800, 600), (1024, 768), (1280, 720), (1600, 900), (1920, 1080)]
SCENE_CENTRE = np.array([0.0, 0.0, 6.0])


def multiview_cameras(n_views, seed, radius=20.0):
    """Cameras on a sphere of the given radius around the scene centre, looking at it,
    each with a resolution drawn from RESOLUTIONS and fx = fy = width."""
    rng = np.random.default_rng(seed)
    cams = []
    while len(cams) < n_views:
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        if abs(d[1]) > 0.9:
            continue
        w, h = RESOLUTIONS[rng.integers(0, len(RESOLUTIONS))]
        cams.append(look_at(SCENE_CENTRE + radius * d, SCENE_CENTRE, w, h, float(w)))
    return cams


def occluded_volume(n_faint=200_000, n_blobs=60, per_blob=3000, seed=6, radius=6.0, blob_radius=2.0):
    """Scheduler workload where list length mispredicts tile cost: a faint volume (means uniform in a
    ball of the given radius around the scene centre, opacity sigmoid(N(-3, 0.5)): long lists that
    rarely terminate) with n_blobs opaque clusters inside it (per_blob Gaussians each, normal with
    standard deviation blob_radius / 2 around centres uniform in a cube of half-width 0.7 radius,
    opacity sigmoid(N(4, 1)): they lengthen the lists of the tiles they cover but end those tiles'
    blending early).  Log-scales N(-2.3, 0.3) per axis, uniform rotations, SH degree 0."""
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((n_faint, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    mf = SCENE_CENTRE + u * (radius * rng.random(n_faint) ** (1.0 / 3.0))[:, None]
    centres = SCENE_CENTRE + rng.uniform(-0.7 * radius, 0.7 * radius, (n_blobs, 3))
    labels = rng.integers(0, n_blobs, n_blobs * per_blob)
    mb = centres[labels] + rng.standard_normal((n_blobs * per_blob, 3)) * (blob_radius / 2.0)
    means = np.r_[mf, mb]
    P = len(means)
    scales = np.exp(rng.normal(-2.3, 0.3, (P, 3)))
    quats = _quats(rng, P)
    opacity = np.r_[_sigmoid(rng.normal(-3.0, 0.5, n_faint)), _sigmoid(rng.normal(4.0, 1.0, n_blobs * per_blob))]
    return _pack(means, scales, quats, opacity, _sh(rng, P, 0, 0.0), 0)


def low_res_cameras(n_views, seed, width=320, height=240, radius=20.0):
    """Cameras as multiview_cameras (on a sphere around the scene centre, looking at it) at one fixed
    low resolution, fx = fy = width."""
    cams = multiview_cameras(n_views, seed, radius)
    for c in cams:
        vm = c["viewmat"]
        c.update(pinhole(width, height, float(width), viewmat=vm, campos=c["campos"]))
    return cams


def learned_scheduler_occluded(n_views=16, seed=6):
    """Scheduler workload with few, uneven items per resident CTA: 16 views at 320x240 (4,800 tiles) of
    the occluded volume (380k Gaussians)."""
    return low_res_cameras(n_views, seed + 1000), occluded_volume(seed=seed)


def learned_scheduler(P=3_000_000, n_views=16, seed=4):
    """Learned scheduler: 16 views of one 3M-Gaussian scene (plain-workload distributions)."""
    rng = np.random.default_rng(seed)
    scene = uniform_box(rng, P)
    return multiview_cameras(n_views, seed + 1000), scene


def large(P=6_000_000, width=3840, height=2160, seed=5):
    """Large: 1 view 3840x2160, fx = fy = 2200, 6M Gaussians in 256 clusters, SH degree 3."""
    rng = np.random.default_rng(seed)
    cam = pinhole(width, height, fx=2200.0 * width / 3840.0)
    return cam, clustered(rng, P, 256, cam, log_scale=(-3.0, 0.5), bimodal_opacity=False,
                          box=(2.0, 2.0, 10.0))
