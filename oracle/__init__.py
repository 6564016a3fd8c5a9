"""FP64 CPU oracle of the TC-GS rasterizer hot path.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only users.  The product path (the CUDA
library and its Python binding) never imports this package, and this package
never imports the product.  The C part (``tcgs_oracle.c``) is compiled with
gcc on first use; the numpy parts live in ``frag2mat.py``, ``mlp.py`` and
``features.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tcgs_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

TILE = 16


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/liboracle.so`` (plain gcc, -O2)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class Camera(ctypes.Structure):
    _fields_ = [
        ("width", ctypes.c_int32), ("height", ctypes.c_int32),
        ("fx", ctypes.c_double), ("fy", ctypes.c_double), ("cx", ctypes.c_double), ("cy", ctypes.c_double),
        ("viewmat", ctypes.c_double * 12), ("campos", ctypes.c_double * 3), ("near_z", ctypes.c_double),
        ("tan_fovx", ctypes.c_double), ("tan_fovy", ctypes.c_double),
    ]


def camera(cam: dict) -> Camera:
    """Build the oracle camera from the plain-dict camera of the input generators."""
    c = Camera()
    c.width, c.height = int(cam["width"]), int(cam["height"])
    c.fx, c.fy, c.cx, c.cy = (float(cam[k]) for k in ("fx", "fy", "cx", "cy"))
    c.viewmat[:] = [float(v) for v in np.asarray(cam["viewmat"], dtype=np.float64).reshape(12)]
    c.campos[:] = [float(v) for v in np.asarray(cam["campos"], dtype=np.float64).reshape(3)]
    c.near_z = float(cam.get("near_z", 0.2))
    c.tan_fovx = float(cam.get("tan_fovx", 0.5 * cam["width"] / cam["fx"]))
    c.tan_fovy = float(cam.get("tan_fovy", 0.5 * cam["height"] / cam["fy"]))
    return c


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            d, i32, i64 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64
            cam = P(Camera)
            lib.orc_sh_basis.argtypes = [ctypes.c_int, P(d), P(d)]
            lib.orc_quat_to_rot.argtypes = [P(d), P(d)]
            lib.orc_project.argtypes = [cam, ctypes.c_int, ctypes.c_int] + [P(d)] * 5 + [ctypes.c_int] + \
                [P(d), P(d), P(d), P(i32), P(d), P(i32), P(d)]
            lib.orc_count_splats.argtypes = [cam, ctypes.c_int, P(d), P(i32), P(d), P(d)]
            lib.orc_count_splats.restype = i64
            lib.orc_bin_sort.argtypes = [cam, ctypes.c_int, P(d), P(i32), P(d), P(d), P(d), i64, P(i32), P(i32),
                                         P(i32)]
            lib.orc_bin_sort.restype = i64
            lib.orc_box_min_q.argtypes = [ctypes.c_double] * 9
            lib.orc_box_min_q.restype = ctypes.c_double
            lib.orc_render.argtypes = [cam, d, P(i32), P(i32), P(d), P(d), P(d), P(d), P(d),
                                       P(d), P(d), P(i32), P(i32), P(d), P(d), P(i64), P(i32), ctypes.c_int]
            lib.orc_render_bruteforce.argtypes = [cam, d, ctypes.c_int, P(d), P(i32), P(d), P(d), P(d), P(d),
                                                  P(d), P(d), P(d), P(i32)]
            lib.orc_render_bwd.argtypes = [cam, d, P(i32), P(i32), P(d), P(d), P(d), P(d), P(d), P(d),
                                           P(d), P(d), P(d), P(d)]
            lib.orc_project_bwd.argtypes = [cam, ctypes.c_int, ctypes.c_int, P(d), P(d), P(d), P(d), P(i32),
                                            P(d), P(d), P(d), P(d), P(d), P(d), P(d)]
            _lib = lib
    return _lib


def _p(a, ct):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def sh_basis(degree: int, direction) -> np.ndarray:
    out = np.zeros(16, np.float64)
    _L().orc_sh_basis(degree, _p(_f64(direction), ctypes.c_double), _p(out, ctypes.c_double))
    return out[: (degree + 1) ** 2]


def quat_to_rot(q) -> np.ndarray:
    R = np.zeros(9, np.float64)
    _L().orc_quat_to_rot(_p(_f64(q), ctypes.c_double), _p(R, ctypes.c_double))
    return R.reshape(3, 3)


def project(cam: dict, scene: dict, tight_radius: bool = False) -> dict:
    """Preprocess stage in FP64 (Sec. 3.1, Eq. 2).  tight_radius: the coverage square bounds the
    ellipse where alpha >= 1/255 (opacity-aware) instead of the 3-sigma square."""
    c = camera(cam)
    means3 = _f64(scene["means3"]); P = means3.shape[0]
    deg = int(scene["sh_degree"])
    out = dict(mean2d=np.zeros((P, 2)), conic=np.zeros((P, 3)), depth=np.zeros(P),
               radius=np.zeros(P, np.int32), rgb=np.zeros((P, 3)), tiles_touched=np.zeros(P, np.int32),
               cov2d=np.zeros((P, 3)))
    d = ctypes.c_double
    _L().orc_project(ctypes.byref(c), P, deg, _p(means3, d), _p(_f64(scene["scales"]), d),
                     _p(_f64(scene["quats"]), d), _p(_f64(scene["opacity"]), d), _p(_f64(scene["sh"]), d),
                     int(bool(tight_radius)), _p(out["mean2d"], d), _p(out["conic"], d), _p(out["depth"], d),
                     _p(out["radius"], ctypes.c_int32), _p(out["rgb"], d),
                     _p(out["tiles_touched"], ctypes.c_int32), _p(out["cov2d"], d))
    return out


def grid(cam: dict):
    return (int(cam["width"]) + TILE - 1) // TILE, (int(cam["height"]) + TILE - 1) // TILE


def bin_sort(cam: dict, mean2d, radius, depth, conic=None, opacity=None) -> dict:
    """Splats, per-tile depth order and tile ranges (Sec. 3.1, Eq. 3).  With conic and opacity,
    exact coverage: a rectangle tile is kept only when the Gaussian reaches alpha >= 1/255 on the
    tile's box of pixel centres (limit with margins, see tile_reached in the C oracle)."""
    c = camera(cam)
    mean2d = _f64(mean2d); radius = _i32(radius); depth = _f64(depth)
    d = ctypes.c_double
    cq = None if conic is None else _f64(conic)
    op = None if conic is None else _f64(opacity)
    P = radius.shape[0]
    gw, gh = grid(cam)
    n = _L().orc_count_splats(ctypes.byref(c), P, _p(mean2d, d), _p(radius, ctypes.c_int32), _p(cq, d), _p(op, d))
    ids = np.zeros(max(n, 1), np.int32)
    tiles = np.zeros(max(n, 1), np.int32)
    ranges = np.zeros(2 * gw * gh, np.int32)
    got = _L().orc_bin_sort(ctypes.byref(c), P, _p(mean2d, d), _p(radius, ctypes.c_int32), _p(cq, d), _p(op, d),
                            _p(depth, d), n, _p(ids, ctypes.c_int32), _p(tiles, ctypes.c_int32),
                            _p(ranges, ctypes.c_int32))
    assert got == n
    return dict(n=int(n), ids=ids[:n], tile_of=tiles[:n], ranges=ranges.reshape(-1, 2))


def box_min_q(mx, my, a, b, c, x0, x1, y0, y1) -> float:
    """Least value of the conic form (x - m)^T Q (x - m) over a box (the exact-coverage test)."""
    return float(_L().orc_box_min_q(mx, my, a, b, c, x0, x1, y0, y1))


def render(cam: dict, binned: dict, mean2d, conic, opacity, rgb, bg=(0.0, 0.0, 0.0), alpha_max=0.99,
           tiles=None, margins=True) -> dict:
    """Algorithm 1 per pixel over each tile's sorted list, FP64."""
    c = camera(cam)
    W, H = int(cam["width"]), int(cam["height"])
    out = dict(img=np.zeros((3, H, W)), T=np.zeros((H, W)), n_contrib=np.zeros((H, W), np.int32),
               n_eval=np.zeros((H, W), np.int32), counts=np.zeros(3, np.int64))
    if margins:
        out["cull_margin"] = np.full((H, W), np.inf)
        out["term_margin"] = np.full((H, W), np.inf)
    d = ctypes.c_double
    sub = None if tiles is None else _i32(tiles)
    _L().orc_render(ctypes.byref(c), float(alpha_max), _p(_i32(binned["ranges"]), ctypes.c_int32),
                    _p(_i32(binned["ids"]), ctypes.c_int32), _p(_f64(mean2d), d), _p(_f64(conic), d),
                    _p(_f64(opacity), d), _p(_f64(rgb), d), _p(_f64(bg), d), _p(out["img"], d), _p(out["T"], d),
                    _p(out["n_contrib"], ctypes.c_int32), _p(out["n_eval"], ctypes.c_int32),
                    _p(out.get("cull_margin"), d), _p(out.get("term_margin"), d),
                    _p(out["counts"], ctypes.c_int64), _p(sub, ctypes.c_int32), 0 if sub is None else len(sub))
    out["f_blend"], out["f_cull"], out["alpha_evals"] = (int(v) for v in out["counts"])
    return out


def render_bruteforce(cam: dict, mean2d, radius, depth, conic, opacity, rgb, bg=(0.0, 0.0, 0.0),
                      alpha_max=0.99) -> dict:
    """Untiled renderer: every pixel walks all Gaussians in global depth order."""
    c = camera(cam)
    W, H = int(cam["width"]), int(cam["height"])
    out = dict(img=np.zeros((3, H, W)), T=np.zeros((H, W)), n_contrib=np.zeros((H, W), np.int32))
    d = ctypes.c_double
    radius = _i32(radius)
    _L().orc_render_bruteforce(ctypes.byref(c), float(alpha_max), radius.shape[0], _p(_f64(mean2d), d),
                               _p(radius, ctypes.c_int32), _p(_f64(depth), d), _p(_f64(conic), d),
                               _p(_f64(opacity), d), _p(_f64(rgb), d), _p(_f64(bg), d), _p(out["img"], d),
                               _p(out["T"], d), _p(out["n_contrib"], ctypes.c_int32))
    return out


def render_bwd(cam: dict, binned: dict, mean2d, conic, opacity, rgb, dL_dimg, bg=(0.0, 0.0, 0.0),
               alpha_max=0.99) -> dict:
    """Analytic gradient of Algorithm 1's image w.r.t. mean2d, conic, opacity, colour."""
    c = camera(cam)
    P = np.asarray(opacity).shape[0]
    out = dict(dmean2d=np.zeros((P, 2)), dconic=np.zeros((P, 3)), dopacity=np.zeros(P), drgb=np.zeros((P, 3)))
    d = ctypes.c_double
    _L().orc_render_bwd(ctypes.byref(c), float(alpha_max), _p(_i32(binned["ranges"]), ctypes.c_int32),
                        _p(_i32(binned["ids"]), ctypes.c_int32), _p(_f64(mean2d), d), _p(_f64(conic), d),
                        _p(_f64(opacity), d), _p(_f64(rgb), d), _p(_f64(bg), d), _p(_f64(dL_dimg), d),
                        _p(out["dmean2d"], d), _p(out["dconic"], d), _p(out["dopacity"], d), _p(out["drgb"], d))
    return out


def project_bwd(cam: dict, scene: dict, radius, dmean2d, dconic, drgb) -> dict:
    """Analytic gradient of the preprocess (Sec. 3.1, Eq. 2) w.r.t. means3, scales, quats and sh,
    given the gradients of mean2d, conic and rgb; Gaussians with radius 0 get zeros."""
    c = camera(cam)
    means3 = _f64(scene["means3"]); P = means3.shape[0]
    deg = int(scene["sh_degree"])
    K = (deg + 1) ** 2
    out = dict(dmeans3=np.zeros((P, 3)), dscales=np.zeros((P, 3)), dquats=np.zeros((P, 4)),
               dsh=np.zeros((P, K, 3)))
    d = ctypes.c_double
    _L().orc_project_bwd(ctypes.byref(c), P, deg, _p(means3, d), _p(_f64(scene["scales"]), d),
                         _p(_f64(scene["quats"]), d), _p(_f64(scene["sh"]), d), _p(_i32(radius), ctypes.c_int32),
                         _p(_f64(dmean2d), d), _p(_f64(dconic), d), _p(_f64(drgb), d), _p(out["dmeans3"], d),
                         _p(out["dscales"], d), _p(out["dquats"], d), _p(out["dsh"], d))
    return out
