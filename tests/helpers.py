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
