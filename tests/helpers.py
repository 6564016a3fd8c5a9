"""Shared helpers of the GPU parity tests: oracle runs on seeded inputs, GPU runs through the
C ABI, and the comparison statistics.  The oracle never sees a value the GPU produced."""
from __future__ import annotations

import math

import numpy as np

import oracle

F32 = np.float32


def f32(a):
    return np.asarray(a, np.float64).astype(F32)


def scene64(sc):
    return {k: (v.astype(np.float64) if isinstance(v, np.ndarray) else v) for k, v in sc.items()}


def oracle_frame(cam, sc, alpha_max=0.99, bg=(0, 0, 0), render=True):
    """Oracle projection in FP64, then its outputs rounded to FP32: these FP32 values are the
    common inputs of both sides for the binning and blending stages (and the oracle image unless
    render is False)."""
    pr = oracle.project(cam, scene64(sc))
    inp = dict(mean2d=f32(pr["mean2d"]), conic=f32(pr["conic"]), depth=f32(pr["depth"]), radius=pr["radius"],
               rgb=f32(pr["rgb"]), opacity=f32(sc["opacity"]))
    b = oracle.bin_sort(cam, inp["mean2d"], inp["radius"], inp["depth"])
    out = (oracle.render(cam, b, inp["mean2d"], inp["conic"], inp["opacity"], inp["rgb"], bg=bg, alpha_max=alpha_max)
           if render else None)
    return pr, inp, b, out


def psnr(a, b):
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return math.inf if mse == 0 else 10.0 * math.log10(1.0 / mse)


def to_torch(a, dev, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(dev)


def margin_mask(o, cull_tol=1e-5, term_tol=1e-4):
    """Pixels whose cull or termination decision lies near its threshold in the oracle's arithmetic,
    where FP32 may decide it the other way: |beta + ln 255| < cull_tol (the FP32 exponent carries an
    error of about 1e-6 here) or |ln(T - alpha T) - ln 1e-4| < term_tol (T is a product over up to
    thousands of blends, each adding about 6e-8 of relative error)."""
    return (o["cull_margin"] < cull_tol) | (o["term_margin"] < term_tol)


def gaussians_at_pixels(b, cam, pixels, n_eval, n_contrib_gpu):
    """Boolean mask over Gaussians: those a pixel of `pixels` (boolean [H, W]) evaluates on either
    side, i.e. its tile's list up to one past the later of the oracle's evaluation count and the
    GPU's last blended index.  A flipped decision at such a pixel changes the transmittance of every
    later fragment there and the colour blended behind every earlier one."""
    gw = (int(cam["width"]) + 15) // 16
    P = int(b["ids"].max()) + 1 if b["n"] > 0 else 0
    out = np.zeros(P, bool)
    for py, px in zip(*np.nonzero(pixels)):
        t = (py // 16) * gw + px // 16
        s, e = b["ranges"][t]
        k = min(e - s, max(int(n_eval[py, px]), int(n_contrib_gpu[py, px]) + 1) + 1)
        out[b["ids"][s:s + k]] = True
    return out
