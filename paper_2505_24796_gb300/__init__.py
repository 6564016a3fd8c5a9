"""GB300 (sm_103a) TC-GS rasterizer: PyTorch-facing binding of libtcgs.so.

The functions named ``tcgs_*`` mirror the C ABI in ``include/tcgs.h`` one to
one; they only check tensors, allocate outputs with PyTorch when the caller
does not pass them, and hand raw device pointers and the current CUDA stream to
the library.  Every step of the rasterizer runs in the library's CUDA kernels;
nothing here computes on the CPU and there is no fallback path.

``Renderer`` owns preallocated buffers for one camera and scene size and runs a
whole frame (project -> bin_sort -> render_fwd) without host synchronisation.
``rasterize`` is the differentiable alpha-blending stage (torch.autograd).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import (PRECISIONS, TCGS_FP32, TCGS_TC_FP16, TCGS_TC_FP16_GLOBAL, TCGS_TC_FP16_SPLIT, TCGS_TC_FP8,
                   TCGS_TC_TF32, TCGS_TC_TF32_GLOBAL, TcgsError, check,
                   tcgs_camera, tcgs_render_opts)

TILE = 16

__all__ = ["tcgs_project", "tcgs_project_bwd", "tcgs_bin_sort", "tcgs_bin_sort_workspace_size", "tcgs_bin_sort_noalloc",
           "tcgs_bin_sort_exact", "tcgs_tile_order", "tcgs_tc_wave_tiles", "tcgs_selftest_bounded_wait", "tcgs_microbench_ex2",
           "tcgs_render_fwd", "tcgs_render_bwd", "tcgs_render_fwd_batched", "tcgs_tile_features", "tcgs_feature_norm",
           "tcgs_mlp_fwd", "tcgs_mlp_bwd", "tcgs_adam_step", "tcgs_sched_order", "tcgs_frag2mat_beta", "make_camera", "render_opts", "Renderer", "rasterize", "render_gaussians", "TcgsError", "PRECISIONS", "FramePipeline",
           "TCGS_FP32", "TCGS_TC_FP16", "TCGS_TC_FP16_SPLIT", "TCGS_TC_FP8", "TCGS_TC_TF32", "TCGS_TC_FP16_GLOBAL",
           "TCGS_TC_TF32_GLOBAL"]


def _L():
    return _lib.load()


def _stream(stream=None) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t: torch.Tensor | None, dtype=None, name="tensor") -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (no CPU path exists)")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    return t.data_ptr()


def make_camera(cam: dict) -> tcgs_camera:
    """C camera struct from the plain-dict camera of ``scenes``."""
    c = tcgs_camera()
    c.width, c.height = int(cam["width"]), int(cam["height"])
    c.fx, c.fy, c.cx, c.cy = (float(cam[k]) for k in ("fx", "fy", "cx", "cy"))
    c.viewmat[:] = [float(v) for v in np.asarray(cam["viewmat"], dtype=np.float64).reshape(12)]
    c.campos[:] = [float(v) for v in np.asarray(cam["campos"], dtype=np.float64).reshape(3)]
    c.near_z = float(cam.get("near_z", 0.2))
    c.tan_fovx = float(cam.get("tan_fovx", 0.0))
    c.tan_fovy = float(cam.get("tan_fovy", 0.0))
    return c


def grid(cam) -> tuple[int, int]:
    w, h = (cam.width, cam.height) if isinstance(cam, tcgs_camera) else (int(cam["width"]), int(cam["height"]))
    return (w + TILE - 1) // TILE, (h + TILE - 1) // TILE


def _cam(cam) -> tcgs_camera:
    return cam if isinstance(cam, tcgs_camera) else make_camera(cam)


def render_opts(precision="tc_fp16_split", alpha_max=0.99, early_cull=None, tile_stats=None,
                device_status=None, tile_cull=True, tile_order=None, work_counter=None,
                pixels_per_thread=1) -> tcgs_render_opts:
    """early_cull None: the path's default (off on the FP32 path, the 3DGS baseline; on for the
    tensor-core paths, as the paper's renderer).  tile_order / work_counter: the persistent TC
    renderer's tile order (tcgs_tile_order) and its counter.  pixels_per_thread: 1, or 2 for views of
    large footprints (tcgs_render_opts.pixels_per_thread)."""
    o = tcgs_render_opts()
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.alpha_max = float(alpha_max)
    o.early_cull = int(o.precision != TCGS_FP32) if early_cull is None else int(bool(early_cull))
    o.tile_cull = int(bool(tile_cull))
    o.tile_stats = _ptr(tile_stats, torch.int32, "tile_stats") if tile_stats is not None else None
    o.device_status = _ptr(device_status, torch.int32, "device_status") if device_status is not None else None
    o.tile_order = _ptr(tile_order, torch.int32, "tile_order") if tile_order is not None else None
    o.work_counter = _ptr(work_counter, torch.int32, "work_counter") if work_counter is not None else None
    o.pixels_per_thread = int(pixels_per_thread)
    return o


# ---------------------------------------------------------------- one-to-one C ABI wrappers

def tcgs_project(cam, means3, scales, quats, sh, sh_degree, out=None, stream=None, opacity=None) -> dict:
    """opacity: None for the 3-sigma coverage square, or the opacities for the opacity-aware one."""
    c = _cam(cam)
    P = means3.shape[0]
    dev = means3.device
    if out is None:
        out = dict(mean2d=torch.empty(P, 2, device=dev), conic=torch.empty(P, 3, device=dev),
                   depth=torch.empty(P, device=dev), radius=torch.empty(P, dtype=torch.int32, device=dev),
                   rgb=torch.empty(P, 3, device=dev), tiles_touched=torch.empty(P, dtype=torch.int32, device=dev))
    f = torch.float32
    check("tcgs_project", _L().tcgs_project(
        ctypes.byref(c), P, int(sh_degree), _ptr(means3, f, "means3"), _ptr(scales, f, "scales"),
        _ptr(quats, f, "quats"), _ptr(sh, f, "sh"), _ptr(opacity, f, "opacity") if opacity is not None else None,
        _ptr(out["mean2d"], f), _ptr(out["conic"], f),
        _ptr(out["depth"], f), _ptr(out["radius"], torch.int32), _ptr(out["rgb"], f),
        _ptr(out["tiles_touched"], torch.int32), _stream(stream)))
    return out


def tcgs_project_bwd(cam, means3, scales, quats, sh, sh_degree, radius, dmean2d, dconic, drgb, grads=None,
                     stream=None) -> dict:
    """Accumulates dL/d(means3, scales, quats, sh) into ``grads`` (zeros when None) and returns it."""
    c = _cam(cam)
    P = means3.shape[0]
    if grads is None:
        grads = dict(dmeans3=torch.zeros_like(means3), dscales=torch.zeros_like(scales),
                     dquats=torch.zeros_like(quats), dsh=torch.zeros_like(sh))
    f = torch.float32
    check("tcgs_project_bwd", _L().tcgs_project_bwd(
        ctypes.byref(c), P, int(sh_degree), _ptr(means3, f, "means3"), _ptr(scales, f, "scales"),
        _ptr(quats, f, "quats"), _ptr(sh, f, "sh"), _ptr(radius, torch.int32, "radius"),
        _ptr(dmean2d, f, "dmean2d"), _ptr(dconic, f, "dconic"), _ptr(drgb, f, "drgb"),
        _ptr(grads["dmeans3"], f), _ptr(grads["dscales"], f), _ptr(grads["dquats"], f), _ptr(grads["dsh"], f),
        _stream(stream)))
    return grads


def tcgs_bin_sort_workspace_size(P: int, capacity: int, num_tiles: int) -> int:
    return int(_L().tcgs_bin_sort_workspace_size(int(P), int(capacity), int(num_tiles)))


def tcgs_bin_sort(cam, mean2d, radius, depth, capacity: int, workspace=None, out=None, stream=None, conic=None,
                  opacity=None) -> dict:
    """Sorting stage.  With conic and opacity given, tcgs_bin_sort_exact (exact tile coverage)."""
    c = _cam(cam)
    P = mean2d.shape[0]
    dev = mean2d.device
    gw, gh = grid(c)
    nt = gw * gh
    ws_bytes = tcgs_bin_sort_workspace_size(P, capacity, nt)
    if workspace is None:
        workspace = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    if out is None:
        out = dict(ids_sorted=torch.empty(max(int(capacity), 1), dtype=torch.int32, device=dev),
                   tile_ranges=torch.empty(nt, 2, dtype=torch.int32, device=dev),
                   n_splats=torch.empty(1, dtype=torch.int64, device=dev),
                   status=torch.empty(1, dtype=torch.int32, device=dev))
    tail = (int(capacity), _ptr(workspace, None, "workspace"), workspace.numel() * workspace.element_size(),
            _ptr(out["ids_sorted"], torch.int32), _ptr(out["tile_ranges"], torch.int32),
            _ptr(out["n_splats"], torch.int64), _ptr(out["status"], torch.int32), _stream(stream))
    head = (ctypes.byref(c), P, _ptr(mean2d, torch.float32, "mean2d"), _ptr(radius, torch.int32, "radius"),
            _ptr(depth, torch.float32, "depth"))
    if conic is None:
        check("tcgs_bin_sort", _L().tcgs_bin_sort(*head, *tail))
    else:
        check("tcgs_bin_sort_exact", _L().tcgs_bin_sort_exact(*head, _ptr(conic, torch.float32, "conic"),
                                                              _ptr(opacity, torch.float32, "opacity"), *tail))
    return out


def tcgs_bin_sort_exact(cam, mean2d, radius, depth, conic, opacity, capacity: int, workspace=None, out=None,
                        stream=None) -> dict:
    """tcgs_bin_sort_exact: splats only for the tiles each Gaussian reaches with alpha >= 1/255."""
    return tcgs_bin_sort(cam, mean2d, radius, depth, capacity, workspace, out, stream, conic=conic, opacity=opacity)


def tcgs_selftest_bounded_wait(device_status, polls: int = 4096, stream=None) -> None:
    """The renderer's bounded mbarrier wait on a barrier nothing completes: gives up after `polls`
    polls and writes TCGS_ERR_TIMEOUT to device_status (device int32)."""
    check("tcgs_selftest_bounded_wait", _L().tcgs_selftest_bounded_wait(
        _ptr(device_status, torch.int32, "device_status"), int(polls), _stream(stream)))


def tcgs_microbench_ex2(out: torch.Tensor, blocks: int, iters: int, stream=None) -> int:
    """Enqueues blocks x 256 x 8 x iters ex2.approx evaluations (out: device float [blocks x 256]);
    returns that count for the caller's timing."""
    if out.numel() < blocks * 256:
        raise ValueError("out needs blocks x 256 floats")
    check("tcgs_microbench_ex2", _L().tcgs_microbench_ex2(_ptr(out, torch.float32, "out"), int(blocks), int(iters),
                                                          _stream(stream)))
    return blocks * 256 * 8 * iters


def tcgs_tc_wave_tiles() -> int:
    """Tiles the tensor-core renderer keeps resident at once on the current device (0 when it is not
    sm_103): views with no more tiles than this render one CTA per tile, without a tile order."""
    return int(_L().tcgs_tc_wave_tiles())


def tcgs_tile_order(cam, tile_ranges, out=None, stream=None) -> torch.Tensor:
    """Longest-first order of the view's tiles for the persistent renderer."""
    c = _cam(cam)
    nt = grid(c)[0] * grid(c)[1]
    if out is None:
        out = torch.empty(nt, dtype=torch.int32, device=tile_ranges.device)
    check("tcgs_tile_order", _L().tcgs_tile_order(ctypes.byref(c), _ptr(tile_ranges, torch.int32, "tile_ranges"),
                                                  _ptr(out, torch.int32, "tile_order"), _stream(stream)))
    return out


def tcgs_bin_sort_noalloc(cam, mean2d, radius, depth, capacity: int, out=None, stream=None) -> dict:
    """tcgs_bin_sort working in the library's built-in scratch array instead of a workspace
    (for callers that cannot allocate device memory; see include/tcgs.h for the size limit and
    the rule that calls must not overlap on the GPU)."""
    c = _cam(cam)
    dev = mean2d.device
    nt = grid(c)[0] * grid(c)[1]
    if out is None:
        out = dict(ids_sorted=torch.empty(max(int(capacity), 1), dtype=torch.int32, device=dev),
                   tile_ranges=torch.empty(nt, 2, dtype=torch.int32, device=dev),
                   n_splats=torch.empty(1, dtype=torch.int64, device=dev),
                   status=torch.empty(1, dtype=torch.int32, device=dev))
    check("tcgs_bin_sort_noalloc", _L().tcgs_bin_sort_noalloc(
        ctypes.byref(c), mean2d.shape[0], _ptr(mean2d, torch.float32, "mean2d"), _ptr(radius, torch.int32, "radius"),
        _ptr(depth, torch.float32, "depth"), int(capacity), _ptr(out["ids_sorted"], torch.int32),
        _ptr(out["tile_ranges"], torch.int32), _ptr(out["n_splats"], torch.int64), _ptr(out["status"], torch.int32),
        _stream(stream)))
    return out


def tcgs_render_fwd(cam, opts, tile_ranges, ids_sorted, mean2d, conic, opacity, rgb, bg=(0.0, 0.0, 0.0), out=None,
                    stream=None) -> dict:
    c = _cam(cam)
    if not isinstance(opts, tcgs_render_opts):
        opts = render_opts(**opts)
    dev = mean2d.device
    H, W = c.height, c.width
    if out is None:
        out = dict(img=torch.empty(3, H, W, device=dev), T_final=torch.empty(H, W, device=dev),
                   n_contrib=torch.empty(H, W, dtype=torch.int32, device=dev))
    bg3 = (ctypes.c_float * 3)(*[float(b) for b in bg])
    f = torch.float32
    check("tcgs_render_fwd", _L().tcgs_render_fwd(
        ctypes.byref(c), ctypes.byref(opts), _ptr(tile_ranges, torch.int32, "tile_ranges"),
        _ptr(ids_sorted, torch.int32, "ids_sorted"), _ptr(mean2d, f, "mean2d"), _ptr(conic, f, "conic"),
        _ptr(opacity, f, "opacity"), _ptr(rgb, f, "rgb"), ctypes.cast(bg3, ctypes.c_void_p),
        _ptr(out["img"], f), _ptr(out["T_final"], f), _ptr(out["n_contrib"], torch.int32), _stream(stream)))
    return out


def tcgs_render_bwd(cam, opts, tile_ranges, ids_sorted, mean2d, conic, opacity, rgb, img, T_final, n_contrib,
                    dL_dimg, bg=(0.0, 0.0, 0.0), grads=None, stream=None) -> dict:
    c = _cam(cam)
    if not isinstance(opts, tcgs_render_opts):
        opts = render_opts(**opts)
    P = mean2d.shape[0]
    dev = mean2d.device
    if grads is None:
        grads = dict(dmean2d=torch.zeros(P, 2, device=dev), dconic=torch.zeros(P, 3, device=dev),
                     dopacity=torch.zeros(P, device=dev), drgb=torch.zeros(P, 3, device=dev))
    bg3 = (ctypes.c_float * 3)(*[float(b) for b in bg])
    f = torch.float32
    check("tcgs_render_bwd", _L().tcgs_render_bwd(
        ctypes.byref(c), ctypes.byref(opts), _ptr(tile_ranges, torch.int32, "tile_ranges"),
        _ptr(ids_sorted, torch.int32, "ids_sorted"), _ptr(mean2d, f, "mean2d"), _ptr(conic, f, "conic"),
        _ptr(opacity, f, "opacity"), _ptr(rgb, f, "rgb"), ctypes.cast(bg3, ctypes.c_void_p), _ptr(img, f, "img"),
        _ptr(T_final, f, "T_final"), _ptr(n_contrib, torch.int32, "n_contrib"), _ptr(dL_dimg, f, "dL_dimg"),
        _ptr(grads["dmean2d"], f), _ptr(grads["dconic"], f), _ptr(grads["dopacity"], f), _ptr(grads["drgb"], f),
        _stream(stream)))
    return grads


def tcgs_render_fwd_batched(views, opts, opacity, queue, bg=(0.0, 0.0, 0.0), counter=None, max_ctas=0,
                            stream=None):
    """Persistent multi-view render of the (view << 16 | tile) items of ``queue`` in that order.
    ``views``: list of dicts with cam, tile_ranges, ids_sorted, mean2d, conic, rgb, img, T_final,
    n_contrib and optional tile_stats (device tensors)."""
    if not isinstance(opts, tcgs_render_opts):
        opts = render_opts(**opts)
    arr = (_lib.tcgs_view * len(views))()
    for i, v in enumerate(views):
        w = arr[i]
        w.cam = _cam(v["cam"])
        w.tile_ranges = _ptr(v["tile_ranges"], torch.int32, "tile_ranges")
        w.ids_sorted = _ptr(v["ids_sorted"], torch.int32, "ids_sorted")
        w.mean2d = _ptr(v["mean2d"], torch.float32, "mean2d")
        w.conic = _ptr(v["conic"], torch.float32, "conic")
        w.rgb = _ptr(v["rgb"], torch.float32, "rgb")
        w.img = _ptr(v["img"], torch.float32, "img")
        w.T_final = _ptr(v["T_final"], torch.float32, "T_final")
        w.n_contrib = _ptr(v["n_contrib"], torch.int32, "n_contrib")
        w.tile_stats = _ptr(v["tile_stats"], torch.int32, "tile_stats") if v.get("tile_stats") is not None else None
    if counter is None:
        counter = torch.zeros(1, dtype=torch.int32, device=opacity.device)
    bg3 = (ctypes.c_float * 3)(*[float(b) for b in bg])
    check("tcgs_render_fwd_batched", _L().tcgs_render_fwd_batched(
        len(views), arr, ctypes.byref(opts), _ptr(opacity, torch.float32, "opacity"), ctypes.cast(bg3, ctypes.c_void_p),
        _ptr(queue, torch.int32, "queue"), queue.numel(), _ptr(counter, torch.int32, "counter"), int(max_ctas),
        _stream(stream)))
    return views


def tcgs_tile_features(cam, tile_ranges, ids_sorted, mean2d, conic, opacity, depth, radius, out=None,
                       stream=None) -> torch.Tensor:
    c = _cam(cam)
    nt = grid(c)[0] * grid(c)[1]
    if out is None:
        out = torch.empty(nt, _lib.TCGS_MLP_IN, device=mean2d.device)
    f = torch.float32
    check("tcgs_tile_features", _L().tcgs_tile_features(
        ctypes.byref(c), _ptr(tile_ranges, torch.int32), _ptr(ids_sorted, torch.int32), _ptr(mean2d, f),
        _ptr(conic, f), _ptr(opacity, f), _ptr(depth, f), _ptr(radius, torch.int32), _ptr(out, f), _stream(stream)))
    return out


def tcgs_feature_norm(x, out=None, stream=None) -> torch.Tensor:
    if out is None:
        out = torch.empty(2 * _lib.TCGS_MLP_IN, device=x.device)
    check("tcgs_feature_norm", _L().tcgs_feature_norm(_ptr(x, torch.float32, "x"), x.shape[0],
                                                       _ptr(out, torch.float32), _stream(stream)))
    return out


def tcgs_mlp_fwd(params, norm, x, out=None, stream=None) -> torch.Tensor:
    if out is None:
        out = torch.empty(x.shape[0], device=x.device)
    f = torch.float32
    check("tcgs_mlp_fwd", _L().tcgs_mlp_fwd(_ptr(params, f, "params"), _ptr(norm, f, "norm"), _ptr(x, f, "x"),
                                             x.shape[0], _ptr(out, f), _stream(stream)))
    return out


def tcgs_mlp_bwd(params, norm, x, target, grad=None, loss=None, stream=None):
    f = torch.float32
    if grad is None:
        grad = torch.zeros(_lib.TCGS_MLP_PARAMS, device=x.device)
    check("tcgs_mlp_bwd", _L().tcgs_mlp_bwd(_ptr(params, f, "params"), _ptr(norm, f, "norm"), _ptr(x, f, "x"),
                                             _ptr(target, f, "target"), x.shape[0], _ptr(grad, f, "grad"),
                                             _ptr(loss, f, "loss") if loss is not None else None, _stream(stream)))
    return grad, loss


def tcgs_adam_step(params, m, v, grad, lr, beta1=0.9, beta2=0.999, eps=1e-8, step=1, stream=None):
    f = torch.float32
    check("tcgs_adam_step", _L().tcgs_adam_step(_ptr(params, f), _ptr(m, f), _ptr(v, f), _ptr(grad, f),
                                                 params.numel(), float(lr), float(beta1), float(beta2), float(eps),
                                                 int(step), _stream(stream)))


def tcgs_sched_order(cost, items, workspace=None, out=None, stream=None) -> torch.Tensor:
    n = cost.numel()
    ws_bytes = int(_L().tcgs_sched_order_workspace_size(n))
    if workspace is None:
        workspace = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=cost.device)
    if out is None:
        out = torch.empty(n, dtype=torch.int32, device=cost.device)
    check("tcgs_sched_order", _L().tcgs_sched_order(
        _ptr(cost, torch.float32, "cost"), _ptr(items, torch.int32, "items"), n, _ptr(out, torch.int32),
        _ptr(workspace, None, "workspace"), workspace.numel(), _stream(stream)))
    return out


def tcgs_frag2mat_beta(cam, precision, tile_ranges, ids_sorted, mean2d, conic, opacity, tiles, max_n,
                       device_status=None, stream=None) -> torch.Tensor:
    c = _cam(cam)
    tiles = torch.as_tensor(tiles, dtype=torch.int32, device=mean2d.device).contiguous()
    out = torch.empty(tiles.numel(), 256, int(max_n), device=mean2d.device)
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    f = torch.float32
    check("tcgs_frag2mat_beta", _L().tcgs_frag2mat_beta(
        ctypes.byref(c), prec, _ptr(tile_ranges, torch.int32), _ptr(ids_sorted, torch.int32), _ptr(mean2d, f),
        _ptr(conic, f), _ptr(opacity, f), tiles.numel(), _ptr(tiles, torch.int32), int(max_n), _ptr(out, f),
        _ptr(device_status, torch.int32) if device_status is not None else None, _stream(stream)))
    return out


# ---------------------------------------------------------------- frame pipeline

def scene_to_device(scene: dict, device="cuda") -> dict:
    """Copy a ``scenes`` dict of numpy arrays to device tensors (float32)."""
    out = {k: torch.from_numpy(np.ascontiguousarray(v)).to(device) for k, v in scene.items()
           if isinstance(v, np.ndarray)}
    out["sh_degree"] = int(scene["sh_degree"])
    return out


_PERSISTENT_PRECISIONS = ("tc_fp16_split", "tc_fp16", "tc_tf32", "tc_fp8", "fp32_frag2mat")
# A Renderer whose capacity allows at least this many splats per Gaussian renders two pixels a thread
# (the footprints are large, so the coarser block marks cost little).
DENSE_SPLATS_PER_GAUSSIAN = 16


class Renderer:
    """Preallocated buffers for one camera, scene size and splat capacity; ``frame`` runs
    project -> bin_sort -> render_fwd on the current stream with no host synchronisation."""

    def __init__(self, cam, P: int, capacity: int, device="cuda", stats: bool = False, tight_radius: bool = False,
                 exact_tiles: bool = True, persistent: bool = True, pixels_per_thread=None):
        """tight_radius: bin with the opacity-aware coverage square instead of the 3-sigma one.
        exact_tiles (default): keep only the tiles each Gaussian reaches with alpha >= 1/255
        (tcgs_bin_sort_exact: the same images as the rectangle's tiles, shorter lists); False bins
        every tile of the rectangle (tcgs_bin_sort).  persistent (default): the tensor-core renders
        take the tiles longest list first on a persistent grid (tcgs_tile_order) when the view has
        more tiles than one wave of CTAs holds (tcgs_tc_wave_tiles); the image is the same as with
        one CTA per tile.  pixels_per_thread (tcgs_render_opts.pixels_per_thread): None picks 2 for views
        of large footprints, where the capacity allows at least DENSE_SPLATS_PER_GAUSSIAN splats per
        Gaussian, else 1; the image is the same either way."""
        self.cam = _cam(cam)
        self.tight_radius = bool(tight_radius)
        self.exact_tiles = bool(exact_tiles)
        self.opacity = None
        self.P, self.capacity = int(P), int(capacity)
        if pixels_per_thread is None:
            pixels_per_thread = 2 if self.capacity >= DENSE_SPLATS_PER_GAUSSIAN * max(self.P, 1) else 1
        self.pixels_per_thread = int(pixels_per_thread)
        dev = torch.device(device)
        gw, gh = grid(self.cam)
        self.num_tiles = gw * gh
        H, W = self.cam.height, self.cam.width
        self.proj = dict(mean2d=torch.empty(P, 2, device=dev), conic=torch.empty(P, 3, device=dev),
                         depth=torch.empty(P, device=dev), radius=torch.empty(P, dtype=torch.int32, device=dev),
                         rgb=torch.empty(P, 3, device=dev), tiles_touched=torch.empty(P, dtype=torch.int32, device=dev))
        self.ws = torch.empty(tcgs_bin_sort_workspace_size(P, capacity, self.num_tiles), dtype=torch.uint8,
                              device=dev)
        self.bins = dict(ids_sorted=torch.empty(max(capacity, 1), dtype=torch.int32, device=dev),
                         tile_ranges=torch.empty(self.num_tiles, 2, dtype=torch.int32, device=dev),
                         n_splats=torch.zeros(1, dtype=torch.int64, device=dev),
                         status=torch.zeros(1, dtype=torch.int32, device=dev))
        self.out = dict(img=torch.empty(3, H, W, device=dev), T_final=torch.empty(H, W, device=dev),
                        n_contrib=torch.empty(H, W, dtype=torch.int32, device=dev))
        self.stats = (torch.zeros(self.num_tiles, _lib.TILE_STATS_WORDS, dtype=torch.int32, device=dev)
                      if stats else None)
        self.device_status = torch.zeros(1, dtype=torch.int32, device=dev)
        self.persistent = bool(persistent)
        self._wave_tiles = None
        self.tile_order = torch.empty(self.num_tiles, dtype=torch.int32, device=dev)
        self.work_counter = torch.zeros(1, dtype=torch.int32, device=dev)

    def project(self, scene: dict, stream=None):
        self.opacity = scene["opacity"]
        return tcgs_project(self.cam, scene["means3"], scene["scales"], scene["quats"], scene["sh"],
                            scene["sh_degree"], out=self.proj, stream=stream,
                            opacity=scene["opacity"] if self.tight_radius else None)

    def bin_sort(self, stream=None, opacity=None):
        """opacity: the scene's (exact_tiles only; default the one the last project() saw)."""
        exact = self.exact_tiles
        op = (opacity if opacity is not None else self.opacity) if exact else None
        if exact and op is None:
            raise ValueError("exact_tiles binning needs the opacities: call project() first or pass opacity")
        return tcgs_bin_sort(self.cam, self.proj["mean2d"], self.proj["radius"], self.proj["depth"], self.capacity,
                             workspace=self.ws, out=self.bins, stream=stream,
                             conic=self.proj["conic"] if exact else None, opacity=op)

    def render(self, opacity, precision="tc_fp16_split", alpha_max=0.99, early_cull=None, bg=(0, 0, 0),
               stream=None, tile_cull=True):
        order = None
        if self.persistent and precision in _PERSISTENT_PRECISIONS and self._wave_tiles is None:
            self._wave_tiles = tcgs_tc_wave_tiles()
        if self.persistent and precision in _PERSISTENT_PRECISIONS and self.num_tiles > self._wave_tiles:
            order = tcgs_tile_order(self.cam, self.bins["tile_ranges"], out=self.tile_order, stream=stream)
        opts = render_opts(precision, alpha_max, early_cull, self.stats, self.device_status, tile_cull,
                           tile_order=order, work_counter=self.work_counter if order is not None else None,
                           pixels_per_thread=self.pixels_per_thread)
        return tcgs_render_fwd(self.cam, opts, self.bins["tile_ranges"], self.bins["ids_sorted"],
                               self.proj["mean2d"], self.proj["conic"], opacity, self.proj["rgb"], bg=bg,
                               out=self.out, stream=stream)

    def frame(self, scene: dict, precision="tc_fp16_split", stream=None, **kw):
        self.project(scene, stream)
        self.bin_sort(stream)
        return self.render(scene["opacity"], precision, stream=stream, **kw)


class FramePipeline:
    """Frames whose scene arrays start in pinned host memory and whose image ends there.

    The host->device copy of a frame's scene runs on a copy stream into one of two device scene
    buffers while the previous frame renders on the compute stream, and each image returns on a
    third stream, so a stream of frames runs at the pace of the slowest of the three (on GB300 the
    host link).  Every frame's copies are issued by ``submit``; ``synchronize`` waits for all.

      pipe = FramePipeline(renderer, precision="tc_fp16_split")
      host_scene = FramePipeline.pinned_scene(scene)   # the arrays in one pinned buffer
      pipe.submit(host_scene, host_img)                # returns at once
      pipe.synchronize()

    A scene from ``pinned_scene`` goes up in one copy (its arrays are views of one pinned buffer, laid
    out as the device slot); any other dict of pinned tensors goes up array by array.
    """

    _ALIGN = 256

    @staticmethod
    def _layout(arrays: dict):
        """Byte offsets of the arrays in one buffer (each 256-byte aligned) and the total size."""
        offs, off = {}, 0
        for k, v in arrays.items():
            offs[k] = off
            off += (v.numel() * v.element_size() + FramePipeline._ALIGN - 1) // FramePipeline._ALIGN * FramePipeline._ALIGN
        return offs, off

    @staticmethod
    def _views(buf: torch.Tensor, like: dict, offs: dict) -> dict:
        out = {}
        for k, v in like.items():
            n = v.numel() * v.element_size()
            out[k] = buf[offs[k]:offs[k] + n].view(v.dtype).view(v.shape)
        return out

    @staticmethod
    def pinned_scene(scene: dict) -> dict:
        """The scene's arrays (numpy or torch) copied into views of one pinned host buffer, which
        ``submit`` uploads in one copy; non-array entries (sh_degree) are kept."""
        arrays = {k: (torch.from_numpy(np.ascontiguousarray(v)) if isinstance(v, np.ndarray) else v.contiguous().cpu())
                  for k, v in scene.items() if isinstance(v, (np.ndarray, torch.Tensor))}
        offs, total = FramePipeline._layout(arrays)
        buf = torch.empty(total, dtype=torch.uint8).pin_memory()
        out = FramePipeline._views(buf, arrays, offs)
        for k, v in arrays.items():
            out[k].copy_(v)
        out["_buffer"] = buf
        for k, v in scene.items():
            if not isinstance(v, (np.ndarray, torch.Tensor)):
                out[k] = v
        return out

    def __init__(self, renderer: "Renderer", precision="tc_fp16_split", **render_kw):
        self.r = renderer
        self.precision = precision
        self.render_kw = render_kw
        dev = renderer.out["img"].device
        self.device = dev
        self.copy_stream = torch.cuda.Stream(device=dev)
        self.d2h_stream = torch.cuda.Stream(device=dev)
        self.compute_stream = torch.cuda.current_stream(dev)
        self.scenes = [None, None]
        self.outs = [renderer.out, {k: torch.empty_like(v) for k, v in renderer.out.items()}]
        self.scene_free = [None, None]   # compute finished reading the slot's scene
        self.out_free = [None, None]     # the slot's image has reached the host
        self.n = 0

    def _slot_scene(self, slot, host_scene):
        arrays = {k: v for k, v in host_scene.items() if isinstance(v, torch.Tensor) and k != "_buffer"}
        if self.scenes[slot] is None:
            offs, total = self._layout(arrays)
            buf = torch.empty(total, dtype=torch.uint8, device=self.device)
            self.scenes[slot] = self._views(buf, arrays, offs)
            self.scenes[slot]["_buffer"] = buf
            self.scenes[slot]["sh_degree"] = int(host_scene["sh_degree"])
        return self.scenes[slot]

    def submit(self, host_scene: dict, host_img: torch.Tensor):
        slot = self.n & 1
        dsc = self._slot_scene(slot, host_scene)
        hbuf = host_scene.get("_buffer")
        with torch.cuda.stream(self.copy_stream):
            if self.scene_free[slot] is not None:
                self.copy_stream.wait_event(self.scene_free[slot])
            if hbuf is not None and hbuf.numel() == dsc["_buffer"].numel():
                dsc["_buffer"].copy_(hbuf, non_blocking=True)   # one copy: same layout on both sides
            else:
                for k, v in host_scene.items():
                    if isinstance(v, torch.Tensor) and k != "_buffer":
                        dsc[k].copy_(v, non_blocking=True)
            copied = self.copy_stream.record_event()
        cs = self.compute_stream
        cs.wait_event(copied)
        if self.out_free[slot] is not None:
            cs.wait_event(self.out_free[slot])
        self.r.out = self.outs[slot]
        out = self.r.frame(dsc, precision=self.precision, stream=None, **self.render_kw)
        self.scene_free[slot] = cs.record_event()
        with torch.cuda.stream(self.d2h_stream):
            self.d2h_stream.wait_event(self.scene_free[slot])
            host_img.copy_(out["img"], non_blocking=True)
            self.out_free[slot] = self.d2h_stream.record_event()
        self.n += 1
        return out

    def synchronize(self):
        for s in (self.copy_stream, self.d2h_stream, self.compute_stream):
            s.synchronize()


# ---------------------------------------------------------------- autograd

class _Rasterize(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mean2d, conic, opacity, rgb, cam, tile_ranges, ids_sorted, precision, alpha_max, bg):
        out = tcgs_render_fwd(cam, render_opts(precision, alpha_max), tile_ranges, ids_sorted, mean2d, conic,
                              opacity, rgb, bg=bg)
        ctx.cam, ctx.alpha_max, ctx.bg = cam, alpha_max, bg
        ctx.save_for_backward(mean2d, conic, opacity, rgb, tile_ranges, ids_sorted, out["img"], out["T_final"],
                              out["n_contrib"])
        ctx.mark_non_differentiable(out["T_final"])
        return out["img"], out["T_final"]

    @staticmethod
    def backward(ctx, g_img, g_T):
        mean2d, conic, opacity, rgb, ranges, ids, img, T_final, n_contrib = ctx.saved_tensors
        g = tcgs_render_bwd(ctx.cam, render_opts("fp32", ctx.alpha_max), ranges, ids, mean2d, conic, opacity, rgb,
                            img, T_final, n_contrib, g_img.contiguous(), bg=ctx.bg)
        return g["dmean2d"], g["dconic"], g["dopacity"], g["drgb"], None, None, None, None, None, None


def rasterize(mean2d, conic, opacity, rgb, cam, tile_ranges, ids_sorted, precision="fp32", alpha_max=0.99,
              bg=(0.0, 0.0, 0.0)):
    """Differentiable alpha-blending stage: returns (img [3,H,W], T_final [H,W]); gradients flow
    to mean2d, conic, opacity and rgb through the library's backward kernel."""
    return _Rasterize.apply(mean2d, conic, opacity, rgb, _cam(cam), tile_ranges, ids_sorted, precision, alpha_max,
                            tuple(bg))


class _Project(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means3, scales, quats, sh, cam, sh_degree, radius_opacity):
        out = tcgs_project(cam, means3, scales, quats, sh, sh_degree, opacity=radius_opacity)
        ctx.cam, ctx.sh_degree = cam, sh_degree
        ctx.save_for_backward(means3, scales, quats, sh, out["radius"])
        ctx.mark_non_differentiable(out["depth"], out["radius"], out["tiles_touched"])
        return out["mean2d"], out["conic"], out["rgb"], out["depth"], out["radius"], out["tiles_touched"]

    @staticmethod
    def backward(ctx, g_mean2d, g_conic, g_rgb, g_depth, g_radius, g_tiles):
        means3, scales, quats, sh, radius = ctx.saved_tensors
        zeros = lambda t, g: g.contiguous() if g is not None else torch.zeros_like(t)
        P = means3.shape[0]
        dev = means3.device
        g = tcgs_project_bwd(ctx.cam, means3, scales, quats, sh, ctx.sh_degree, radius,
                             zeros(torch.empty(P, 2, device=dev), g_mean2d), zeros(torch.empty(P, 3, device=dev), g_conic),
                             zeros(torch.empty(P, 3, device=dev), g_rgb))
        return g["dmeans3"], g["dscales"], g["dquats"], g["dsh"], None, None, None


def render_gaussians(cam, means3, scales, quats, opacity, sh, sh_degree, precision="tc_fp16_split", alpha_max=0.99,
                     bg=(0.0, 0.0, 0.0), tight_radius=False, capacity=None, exact_tiles=True):
    """Differentiable frame from 3D Gaussians: project -> bin_sort -> render.  Gradients flow to
    means3, scales, quats, opacity and sh through tcgs_render_bwd and tcgs_project_bwd (binning is
    piecewise constant).  Returns (img [3,H,W], T_final [H,W]).  capacity None sizes the splat
    buffer from the projection (one host synchronisation)."""
    c = _cam(cam)
    mean2d, conic, rgb, depth, radius, tiles = _Project.apply(means3, scales, quats, sh, c, int(sh_degree),
                                                              opacity.detach() if tight_radius else None)
    if capacity is None:
        capacity = int(tiles.to(torch.int64).sum().item()) + 1
    bins = tcgs_bin_sort(c, mean2d.detach(), radius, depth, capacity,
                         conic=conic.detach() if exact_tiles else None,
                         opacity=opacity.detach() if exact_tiles else None)
    return rasterize(mean2d, conic, opacity, rgb, c, bins["tile_ranges"], bins["ids_sorted"], precision, alpha_max,
                     bg)
