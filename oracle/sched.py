"""FP64 oracle of the learned tile-cost model (features, MLP, Adam, queue order).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Plain numpy, written from the
definitions stated in include/tcgs.h for these calls: the paper has no counterpart, so these are
the definitions the scheduler layer is built to.
"""
from __future__ import annotations

import numpy as np

IN, HID = 8, 32
# parameter layout: W1[HID][IN], b1[HID], W2[HID][HID], b2[HID], W3[HID], b3
SIZES = [("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)), ("W3", (HID,)), ("b3", (1,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SIZES)
TILE = 16


def unpack(params):
    params = np.asarray(params, np.float64)
    out, off = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = params[off:off + n].reshape(shape)
        off += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], np.float64).reshape(-1) for name, _ in SIZES])


def _r16(a, fp16):
    return np.asarray(a, np.float64).astype(np.float16).astype(np.float64) if fp16 else np.asarray(a, np.float64)


def mlp_forward(params, norm, X, fp16=True):
    """y = W3 h2 + b3, h2 = relu(W2 h1 + b2), h1 = relu(W1 xh + b1), xh = (x - mu) / sigma; with
    fp16 every weight, xh, h1 and h2 are rounded to FP16 (sums exact here)."""
    P = {k: _r16(v, fp16) for k, v in unpack(params).items()}
    norm = np.asarray(norm, np.float64)
    X = np.asarray(X, np.float64)
    xh = _r16((X - norm[:IN]) * norm[IN:], fp16)
    a1 = xh @ P["W1"].T + P["b1"]
    h1 = _r16(np.maximum(a1, 0.0), fp16)
    a2 = h1 @ P["W2"].T + P["b2"]
    h2 = _r16(np.maximum(a2, 0.0), fp16)
    y = h2 @ P["W3"] + P["b3"][0]
    return y, dict(xh=xh, a1=a1, h1=h1, a2=a2, h2=h2, P=P)


def mlp_backward(params, norm, X, target, fp16=True):
    """Gradient of L = (1/n) sum (y - t)^2; rounding passes gradients through unchanged."""
    y, c = mlp_forward(params, norm, X, fp16)
    n = len(y)
    e = y - np.asarray(target, np.float64)
    loss = float(np.mean(e * e))
    dy = 2.0 * e / n
    P = c["P"]
    d2 = (dy[:, None] * P["W3"][None, :]) * (c["h2"] > 0)
    d1 = (d2 @ P["W2"]) * (c["h1"] > 0)
    g = dict(W3=dy @ c["h2"], b3=np.array([dy.sum()]), W2=d2.T @ c["h1"], b2=d2.sum(0), W1=d1.T @ c["xh"],
             b1=d1.sum(0))
    return pack(g), loss


def adam_step(params, m, v, grad, lr, b1, b2, eps, step):
    m = b1 * np.asarray(m, np.float64) + (1 - b1) * grad
    v = b2 * np.asarray(v, np.float64) + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return np.asarray(params, np.float64) - lr * mh / (np.sqrt(vh) + eps), m, v


def order(cost, items):
    """Items by decreasing cost, ties in input order."""
    idx = np.argsort(-np.asarray(cost, np.float64), kind="stable")
    return np.asarray(items)[idx]


def tile_features(cam, binned, mean2d, conic, opacity, depth, radius):
    """Per-tile features (see tcgs_tile_features): [tiles, 8]."""
    W, H = int(cam["width"]), int(cam["height"])
    gw, gh = (W + TILE - 1) // TILE, (H + TILE - 1) // TILE
    out = np.zeros((gw * gh, IN))
    mean2d = np.asarray(mean2d, np.float64); conic = np.asarray(conic, np.float64)
    for t in range(gw * gh):
        tx, ty = t % gw, t // gw
        s, e = binned["ranges"][t]
        ids = np.asarray(binned["ids"][s:e])
        n = len(ids)
        x0, y0 = TILE * tx, TILE * ty
        f = out[t]
        f[0] = np.log1p(n)
        if n:
            o = np.asarray(opacity, np.float64)[ids]
            d = np.asarray(depth, np.float64)[ids]
            a, b, c = conic[ids, 0], conic[ids, 1], conic[ids, 2]
            r = np.asarray(radius, np.float64)[ids]
            mx, my = mean2d[ids, 0], mean2d[ids, 1]
            ox = np.maximum(0.0, np.minimum(mx + r, x0 + TILE) - np.maximum(mx - r, x0))
            oy = np.maximum(0.0, np.minimum(my + r, y0 + TILE) - np.maximum(my - r, y0))
            f[1] = o.mean()
            f[2] = o.max()
            f[3] = np.log1p(d.max() - d.min())
            f[4] = np.mean(np.log(np.maximum(a * c - b * b, 1e-30)))
            f[5] = np.log1p(np.sum(ox * oy) / (TILE * TILE))
        f[6] = np.log(float(W) * float(H))
        f[7] = min(TILE, W - x0) * min(TILE, H - y0) / (TILE * TILE)
    return out


def lpt_makespan(costs, workers):
    """Greedy list scheduling: each item (in the given order) goes to the earliest-free worker."""
    import heapq
    heap = [0.0] * workers
    heapq.heapify(heap)
    for c in costs:
        heapq.heappush(heap, heapq.heappop(heap) + float(c))
    return max(heap)
