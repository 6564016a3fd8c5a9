"""Pins of the scheduler oracle (features, MLP, Adam, ordering) against closed forms, finite
differences and library routines.  CPU only."""
import math

import numpy as np
import pytest

from oracle import sched as osc
from paper_2505_24796_gb300 import scenes


def _params(seed):
    rng = np.random.default_rng(seed)
    P = osc.unpack(rng.normal(0, 0.3, osc.NPARAMS))
    P["b1"] = np.abs(P["b1"]) + 0.1   # keep most units active
    P["b2"] = np.abs(P["b2"]) + 0.1
    return osc.pack(P)


def test_parameter_count():
    assert osc.NPARAMS == 1377


def test_mlp_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    params = _params(1)
    X = rng.normal(0, 1, (40, 8))
    t = rng.normal(0, 1, 40)
    norm = np.r_[rng.normal(0, 0.1, 8), rng.uniform(0.5, 2, 8)]
    g, _ = osc.mlp_backward(params, norm, X, t, fp16=False)
    h = 1e-6
    for q in rng.choice(osc.NPARAMS, 60, replace=False):
        pp, pm = params.copy(), params.copy()
        pp[q] += h
        pm[q] -= h
        lp = np.mean((osc.mlp_forward(pp, norm, X, False)[0] - t) ** 2)
        lm = np.mean((osc.mlp_forward(pm, norm, X, False)[0] - t) ** 2)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[q]) <= 1e-6 * max(1.0, abs(g[q])), (q, fd, g[q])


def test_mlp_forward_matches_torch_reference():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    params = _params(3)
    X = rng.normal(0, 1, (25, 8))
    norm = np.r_[np.zeros(8), np.ones(8)]
    P = osc.unpack(params)
    net = torch.nn.Sequential(torch.nn.Linear(8, 32), torch.nn.ReLU(), torch.nn.Linear(32, 32), torch.nn.ReLU(),
                              torch.nn.Linear(32, 1)).double()
    with torch.no_grad():
        net[0].weight.copy_(torch.from_numpy(P["W1"])); net[0].bias.copy_(torch.from_numpy(P["b1"]))
        net[2].weight.copy_(torch.from_numpy(P["W2"])); net[2].bias.copy_(torch.from_numpy(P["b2"]))
        net[4].weight.copy_(torch.from_numpy(P["W3"][None, :])); net[4].bias.copy_(torch.from_numpy(P["b3"]))
        ref = net(torch.from_numpy(X)).numpy()[:, 0]
    np.testing.assert_allclose(osc.mlp_forward(params, norm, X, fp16=False)[0], ref, rtol=1e-12, atol=1e-12)


def test_fp16_rounding_changes_little():
    rng = np.random.default_rng(4)
    params = _params(5)
    X = rng.normal(0, 1, (100, 8))
    norm = np.r_[np.zeros(8), np.ones(8)]
    y16 = osc.mlp_forward(params, norm, X, fp16=True)[0]
    y64 = osc.mlp_forward(params, norm, X, fp16=False)[0]
    assert np.abs(y16 - y64).max() < 0.05 * (1 + np.abs(y64).max())
    assert not np.array_equal(y16, y64)


def test_adam_matches_torch_optimizer():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(6)
    p0 = rng.normal(0, 1, 50)
    grads = [rng.normal(0, 1, 50) for _ in range(5)]
    w = torch.tensor(p0.copy(), requires_grad=True)
    opt = torch.optim.Adam([w], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for k, g in enumerate(grads, 1):
        opt.zero_grad()
        w.grad = torch.tensor(g.copy())
        opt.step()
        p, m, v = osc.adam_step(p, m, v, g, 1e-2, 0.9, 0.999, 1e-8, k)
    np.testing.assert_allclose(p, w.detach().numpy(), rtol=1e-10, atol=1e-12)


def test_order_is_stable_descending():
    cost = np.array([1.0, 3.0, 3.0, -2.0, 0.5, 3.0])
    items = np.array([10, 11, 12, 13, 14, 15])
    assert list(osc.order(cost, items)) == [11, 12, 15, 10, 14, 13]


def test_tile_features_closed_forms():
    cam = scenes.pinhole(40, 24, fx=40.0)    # 3 x 2 tiles, the right column 8 px wide, bottom row 8 px high
    mean2d = np.array([[8.0, 8.0], [24.0, 8.0]])
    radius = np.array([4, 100])
    conic = np.array([[0.5, 0.1, 0.25], [0.02, 0.0, 0.02]])
    opacity = np.array([0.4, 0.8])
    depth = np.array([2.0, 5.0])
    # tile 0 holds both (Gaussian 1 covers every tile), tile 1 only Gaussian 1
    binned = dict(ranges=np.array([[0, 2], [2, 3], [3, 4], [4, 5], [5, 6], [6, 7]]),
                  ids=np.array([0, 1, 1, 1, 1, 1, 1]))
    f = osc.tile_features(cam, binned, mean2d, conic, opacity, depth, radius)
    assert f[0, 0] == pytest.approx(math.log(3))
    assert f[0, 1] == pytest.approx(0.6) and f[0, 2] == pytest.approx(0.8)
    assert f[0, 3] == pytest.approx(math.log(4))
    det0, det1 = 0.5 * 0.25 - 0.01, 0.02 * 0.02
    assert f[0, 4] == pytest.approx(0.5 * (math.log(det0) + math.log(det1)))
    # Gaussian 0's 8 x 8 square lies inside tile 0 (coverage 1/4); Gaussian 1 covers the whole tile
    assert f[0, 5] == pytest.approx(math.log1p(0.25 + 1.0))
    assert f[1, 5] == pytest.approx(math.log1p(1.0))
    assert f[0, 6] == pytest.approx(math.log(40 * 24))
    assert f[0, 7] == 1.0 and f[2, 7] == pytest.approx(8 * 16 / 256) and f[5, 7] == pytest.approx(8 * 8 / 256)


def test_lpt_makespan_small_cases():
    assert osc.lpt_makespan([5, 3, 3, 2, 2], 2) == 8
    assert osc.lpt_makespan([1] * 10, 5) == 2
