"""Frag2Mat and G2L in FP64 (Sec. 4.2 and 4.3) plus the tensor-core error
bound of Appendix A (Proposition "dot product"), and the input roundings of the
tensor-core encodings it is checked against (FP16, TF32, FP8 e4m3), with the
error bound of the FP8 split encoding derived from them.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

beta = ln(o) - 1/2 (mu' - p)^T Q (mu' - p) is written as u^T v with
  u = [1, px, py, px^2, px py, py^2]                       (Eq. 14)
  v = [ln o - 1/2 mu'^T Q mu',  s11 mux + s12 muy,  s12 mux + s22 muy,
       -1/2 s11,  -s12,  -1/2 s22]                          (Eq. 12)
with Q = [[s11, s12], [s12, s22]] = Sigma'^-1.  G2L (Sec. 4.3) applies the
same formulas to p - p(T) and mu' - p(T), p(T) the tile centre.
"""
from __future__ import annotations

import numpy as np

EPS_H = 2.0 ** -10      # Table "floating points": FP16 / TF32 machine epsilon (9.77e-4)
EPS_F = 2.0 ** -23      # FP32 machine epsilon (1.19e-7)
TILE = 16
# FP8 encoding: column i of u is scaled by 2^-a_i and of v by 2^a_i before the split
FP8_COLUMN_EXP = (0, 2, 2, 6, 6, 6)
E4M3_MAX = 448.0


def tile_centre(tx: int, ty: int):
    """p(T): centre of the 16 x 16 tile (tx, ty) in pixel units (appendix A, local coordinates)."""
    return np.array([TILE * tx + TILE / 2.0, TILE * ty + TILE / 2.0])


def pixel_vectors(px, py) -> np.ndarray:
    """Rows u_i for pixel sample points (px, py): shape [m, 6] (Eq. 14)."""
    px = np.asarray(px, np.float64); py = np.asarray(py, np.float64)
    return np.stack([np.ones_like(px), px, py, px * px, px * py, py * py], axis=-1)


def gaussian_vectors(mean2d, conic, opacity) -> np.ndarray:
    """Rows v_j for projected Gaussians: shape [n, 6] (Eq. 12)."""
    mean2d = np.asarray(mean2d, np.float64); conic = np.asarray(conic, np.float64)
    o = np.asarray(opacity, np.float64)
    mx, my = mean2d[:, 0], mean2d[:, 1]
    s11, s12, s22 = conic[:, 0], conic[:, 1], conic[:, 2]
    v0 = np.log(o) - 0.5 * (s11 * mx * mx + 2.0 * s12 * mx * my + s22 * my * my)
    return np.stack([v0, s11 * mx + s12 * my, s12 * mx + s22 * my, -0.5 * s11, -s12, -0.5 * s22], axis=-1)


def beta_direct(px, py, mean2d, conic, opacity) -> np.ndarray:
    """beta_{i,j} of Eq. (9) evaluated directly: shape [m, n]."""
    px = np.asarray(px, np.float64)[:, None]; py = np.asarray(py, np.float64)[:, None]
    mean2d = np.asarray(mean2d, np.float64); conic = np.asarray(conic, np.float64)
    dx = mean2d[None, :, 0] - px; dy = mean2d[None, :, 1] - py
    q = conic[None, :, 0] * dx * dx + 2.0 * conic[None, :, 1] * dx * dy + conic[None, :, 2] * dy * dy
    return np.log(np.asarray(opacity, np.float64))[None, :] - 0.5 * q


def tile_pixels_local(half: int | None = None):
    """G2L pixel offsets Delta p of the 256 pixel centres of a tile, row-major
    (or the 128 of the upper / lower half when half is 0 / 1)."""
    j, i = np.meshgrid(np.arange(TILE), np.arange(TILE), indexing="ij")
    dx = (i + 0.5 - TILE / 2.0).reshape(-1); dy = (j + 0.5 - TILE / 2.0).reshape(-1)
    if half is not None:
        sl = slice(half * 128, (half + 1) * 128)
        dx, dy = dx[sl], dy[sl]
    return dx, dy


def local_products(tx: int, ty: int, mean2d, conic, opacity, half: int | None = None):
    """U, V in the G2L frame of tile (tx, ty), exact beta = U V^T, and the
    per-fragment Appendix-A bound 2 eps_H sum_i |u_i v_i|."""
    c = tile_centre(tx, ty)
    dx, dy = tile_pixels_local(half)
    U = pixel_vectors(dx, dy)
    V = gaussian_vectors(np.asarray(mean2d, np.float64) - c[None, :], conic, opacity)
    beta = U @ V.T
    absum = np.abs(U) @ np.abs(V).T
    return U, V, beta, absum


def paper_bound(absum) -> np.ndarray:
    """|beta_hat - beta| <= 2 eps_H sum |u_i v_i| (+ O(eps_H^2 + eps_F)) (Appendix A)."""
    return 2.0 * EPS_H * absum


def round_f16(a) -> np.ndarray:
    return np.asarray(a, np.float64).astype(np.float16).astype(np.float64)


def global_products(tx: int, ty: int, mean2d, conic, opacity, half: int | None = None):
    """U, V in global pixel coordinates for the pixels of tile (tx, ty) (Frag2Mat without G2L, the
    ablation of Table 5), exact beta = U V^T and sum |u_i v_i|."""
    c = tile_centre(tx, ty)
    dx, dy = tile_pixels_local(half)
    U = pixel_vectors(dx + c[0], dy + c[1])
    V = gaussian_vectors(mean2d, conic, opacity)
    return U, V, U @ V.T, np.abs(U) @ np.abs(V).T


def round_tf32(a) -> np.ndarray:
    """Round to TF32 (1 + 10 fraction bits, FP32 exponent range), to nearest with ties away from
    zero."""
    a = np.asarray(a, np.float64)
    m, e = np.frexp(a)                      # a = m 2^e, 0.5 <= |m| < 1
    q = np.sign(m) * np.floor(np.abs(m) * 2.0 ** 11 + 0.5)
    return np.ldexp(q / 2.0 ** 11, e)


def round_e4m3(a) -> np.ndarray:
    """Round to the FP8 e4m3 format (4 exponent bits, bias 7, 3 fraction bits; largest finite value
    448, smallest subnormal 2^-9), to nearest even, saturating at +-448."""
    a = np.asarray(a, np.float64)
    x = np.abs(a)
    e = np.maximum(np.floor(np.log2(np.maximum(x, 2.0 ** -9))), -6.0)   # subnormals share 2^-6's spacing
    q = 2.0 ** (e - 3)
    return np.sign(a) * np.minimum(np.round(x / q) * q, E4M3_MAX)


def fp8_split(U, V):
    """The FP8 split encoding: column-scaled u' = u 2^-a = u_hi + u_lo and v' = v 2^a ~ v_hi + v_lo +
    v_lo2, each part an e4m3 number; returns the exponent that the five groups of products
    u_hi (v_hi + v_lo + v_lo2) + u_lo (v_hi + v_lo) evaluate to, in FP64."""
    s = 2.0 ** -np.asarray(FP8_COLUMN_EXP, np.float64)
    u = np.asarray(U, np.float64) * s
    v = np.asarray(V, np.float64) / s
    uh = round_e4m3(u); ul = round_e4m3(u - uh)
    vh = round_e4m3(v); r1 = v - vh
    vl = round_e4m3(r1); vl2 = round_e4m3(r1 - vl)
    return uh @ (vh + vl + vl2).T + ul @ (vh + vl).T


def fp8_split_bound(U, V, log2_scale: bool = False) -> np.ndarray:
    """|beta_hat - beta| of the FP8 split encoding, before accumulation rounding, when u' splits
    exactly and |v'| <= 448.  Each e4m3 rounding errs by at most max(2^-4 |x|, 2^-10), so the v
    residuals after one and after three parts obey |r2| <= max(2^-8 |v'|, 2^-10) and
    |r3| <= max(2^-12 |v'|, 2^-10); the products evaluate u' v' - u_hi r3 - u_lo r2 with
    |u_hi| <= (1 + 2^-4) |u'| and |u_lo| <= 2^-4 |u'|.  The 2^-10 floor applies to v in the units
    the kernel encodes (log2 units): with log2_scale = False, V is in natural-log units and the
    floor is converted."""
    s = 2.0 ** -np.asarray(FP8_COLUMN_EXP, np.float64)
    aU, aV = np.abs(np.asarray(U, np.float64)), np.abs(np.asarray(V, np.float64))
    rel = ((1 + 2.0 ** -4) * 2.0 ** -12 + 2.0 ** -4 * 2.0 ** -8) * (aU @ aV.T)
    floor = (1 + 2.0 ** -4 + 2.0 ** -4) * 2.0 ** -10 * (aU @ s)
    if not log2_scale:
        floor = floor * np.log(2.0)
    return rel + floor[:, None]
