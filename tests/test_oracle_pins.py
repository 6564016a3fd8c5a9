"""Pins of the FP64 oracle against facts other than itself: closed forms,
library routines, Monte-Carlo and brute force.  CPU only."""
import json
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation
from scipy.special import sph_harm_y

import oracle
from oracle import frag2mat as f2m
from paper_2505_24796_gb300 import scenes

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def scene_arrays(sc):
    return {k: (v.astype(np.float64) if isinstance(v, np.ndarray) else v) for k, v in sc.items()}


def make_scene(means3, scales, quats, opacity, rgb):
    """Degree-0 scene whose colours are exactly ``rgb`` (DC coefficient (rgb - 0.5) / Y00)."""
    means3 = np.atleast_2d(np.asarray(means3, np.float64))
    P = means3.shape[0]
    y00 = 0.5 / math.sqrt(math.pi)
    sh = ((np.asarray(rgb, np.float64).reshape(P, 3) - 0.5) / y00).reshape(P, 1, 3)
    return dict(means3=means3, scales=np.asarray(scales, np.float64).reshape(P, 3),
                quats=np.asarray(quats, np.float64).reshape(P, 4), opacity=np.asarray(opacity, np.float64).reshape(P),
                sh=sh, sh_degree=0)


# ---------------------------------------------------------------- projection

def test_quaternion_matches_scipy():
    rng = np.random.default_rng(0)
    for _ in range(50):
        q = rng.standard_normal(4) * rng.uniform(0.1, 5.0)  # unnormalised on purpose
        R = oracle.quat_to_rot(q)
        ref = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()  # scipy is (x, y, z, w)
        np.testing.assert_allclose(R, ref, atol=1e-13)


def _real_sh_3dgs(l, m, d):
    """Real SH from scipy's complex SH (Condon-Shortley phase included), in the
    sign convention of the 3DGS colour model: (-1)^m times the usual real form."""
    x, y, z = d
    theta = math.acos(max(-1.0, min(1.0, z)))
    phi = math.atan2(y, x)
    if m == 0:
        val = sph_harm_y(l, 0, theta, phi).real
    elif m > 0:
        val = math.sqrt(2.0) * (-1) ** m * sph_harm_y(l, m, theta, phi).real
    else:
        val = math.sqrt(2.0) * (-1) ** m * sph_harm_y(l, -m, theta, phi).imag
    return (-1) ** abs(m) * val


def test_sh_basis_matches_scipy():
    rng = np.random.default_rng(1)
    for _ in range(40):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        got = oracle.sh_basis(3, d)
        ref = [_real_sh_3dgs(l, m, d) for l in range(4) for m in range(-l, l + 1)]
        np.testing.assert_allclose(got, ref, atol=1e-12)


def test_sh_basis_orthonormal():
    # Gauss-Legendre in cos(theta) x uniform phi: exact for these polynomial degrees
    ct, w = np.polynomial.legendre.leggauss(24)
    phis = np.linspace(0, 2 * np.pi, 48, endpoint=False)
    G = np.zeros((16, 16))
    for c, wc in zip(ct, w):
        s = math.sqrt(1 - c * c)
        for ph in phis:
            Y = oracle.sh_basis(3, [s * math.cos(ph), s * math.sin(ph), c])
            G += wc * (2 * np.pi / len(phis)) * np.outer(Y, Y)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_isotropic_on_axis_closed_form():
    f, z, s = 300.0, 5.0, 0.04
    cam = scenes.pinhole(320, 240, fx=f)
    sc = make_scene([0, 0, z], [s, s, s], [0.3, -0.2, 0.5, 0.7], [0.5], [[0.2, 0.4, 0.6]])
    pr = oracle.project(cam, sc)
    var = (f * s / z) ** 2 + 0.3
    np.testing.assert_allclose(pr["mean2d"][0], [160.0, 120.0], atol=1e-12)
    np.testing.assert_allclose(pr["cov2d"][0], [var, 0.0, var], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(pr["conic"][0], [1 / var, 0.0, 1 / var], rtol=1e-12, atol=1e-15)
    # isotropic: the eigen-gap term is floored at 0.1 (radius reading)
    assert pr["radius"][0] == math.ceil(3 * math.sqrt(var + math.sqrt(0.1)))
    assert pr["depth"][0] == z
    np.testing.assert_allclose(pr["rgb"][0], [0.2, 0.4, 0.6], atol=1e-12)


def _random_view(rng):
    R = Rotation.from_rotvec(rng.normal(0, 0.3, 3)).as_matrix()
    t = rng.normal(0, 0.5, 3)
    return np.hstack([R, t[:, None]])


def test_projection_matches_monte_carlo():
    """EWA (Eq. 2) is the linearisation of the pinhole map: for a small Gaussian the
    covariance of projected samples must match Sigma' - 0.3 I."""
    rng = np.random.default_rng(2)
    vm = _random_view(rng)
    cam = scenes.pinhole(640, 480, fx=500.0, fy=450.0, viewmat=vm)
    cam["viewmat"] = vm
    R3, t3 = vm[:, :3], vm[:, 3]
    target_cam = np.array([0.3, -0.2, 6.0])
    mu = np.linalg.solve(R3, target_cam - t3)
    scales = np.array([0.03, 0.012, 0.02])
    q = np.array([0.8, 0.3, -0.4, 0.2])
    sc = make_scene(mu, scales, q, [0.9], [[0.5, 0.5, 0.5]])
    pr = oracle.project(cam, sc)
    Rg = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    n = 400_000
    pts = mu[None, :] + (rng.standard_normal((n, 3)) * scales[None, :]) @ Rg.T
    pc = pts @ R3.T + t3[None, :]
    u = cam["fx"] * pc[:, 0] / pc[:, 2] + cam["cx"]
    v = cam["fy"] * pc[:, 1] / pc[:, 2] + cam["cy"]
    emp = np.cov(np.stack([u, v]))
    a, b, c = pr["cov2d"][0]
    ewa = np.array([[a - 0.3, b], [b, c - 0.3]])
    np.testing.assert_allclose(emp, ewa, rtol=0.02, atol=0.02 * np.abs(ewa).max())
    np.testing.assert_allclose(pr["mean2d"][0], [u.mean(), v.mean()], atol=0.02)


def test_projection_numeric_jacobian():
    """Sigma' equals J_num Sigma_world J_num^T + 0.3 I with J_num the finite-difference
    Jacobian of the pinhole map of world points (no frustum clamp active)."""
    rng = np.random.default_rng(3)
    vm = _random_view(rng)
    cam = scenes.pinhole(800, 600, fx=700.0, fy=650.0, viewmat=vm)
    cam["viewmat"] = vm
    R3, t3 = vm[:, :3], vm[:, 3]
    for _ in range(20):
        mu = np.linalg.solve(R3, np.array([rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(3, 8)]) - t3)
        scales = np.exp(rng.normal(-3, 0.5, 3))
        q = rng.standard_normal(4)
        sc = make_scene(mu, scales, q, [0.5], [[0.5, 0.5, 0.5]])
        pr = oracle.project(cam, sc)

        def proj(p):
            pc = R3 @ p + t3
            return np.array([cam["fx"] * pc[0] / pc[2] + cam["cx"], cam["fy"] * pc[1] / pc[2] + cam["cy"]])

        h = 1e-6
        J = np.stack([(proj(mu + h * e) - proj(mu - h * e)) / (2 * h) for e in np.eye(3)], axis=1)
        Rg = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        Sw = Rg @ np.diag(scales ** 2) @ Rg.T
        ref = J @ Sw @ J.T + 0.3 * np.eye(2)
        a, b, c = pr["cov2d"][0]
        np.testing.assert_allclose([a, b, c], [ref[0, 0], ref[0, 1], ref[1, 1]], rtol=1e-6, atol=1e-9)
        lam = np.linalg.eigvalsh(ref)
        mid, det = 0.5 * (a + c), a * c - b * b
        lam1 = mid + math.sqrt(max(0.1, mid * mid - det))
        assert lam1 >= lam.max() * (1 - 1e-6)


def _pinhole_cam_jacobian(cam, pc):
    """Central-difference Jacobian (2 x 3) of the pinhole map (X, Y, Z) -> (fx X / Z + cx, fy Y / Z + cy)
    at the camera-space point pc."""
    def proj(p):
        return np.array([cam["fx"] * p[0] / p[2] + cam["cx"], cam["fy"] * p[1] / p[2] + cam["cy"]])
    h = 1e-6 * max(1.0, float(np.abs(pc).max()))
    return np.stack([(proj(pc + h * e) - proj(pc - h * e)) / (2 * h) for e in np.eye(3)], axis=1)


@pytest.mark.parametrize("view", ["identity", "rotated"])
def test_projection_frustum_clamp_of_the_jacobian(view):
    """Gaussians beyond the frustum: x/z and y/z are clamped to +-1.3 tan(fov / 2) where J is built
    (3DGS convention), so Sigma' must equal J_num Sigma_cam J_num^T + 0.3 I with J_num the numerical
    Jacobian of the pinhole map taken at the point of the same depth on the clamped ray, while mean2d
    keeps the unclamped projection.  Cases: x beyond the right edge, y beyond the top, both beyond
    on the negative side, and one inside (no clamp); width != height and fx != fy, so a limit taken
    from the wrong axis, a missing 1.3, a clamp of X instead of X / Z or a clamped mean all fail."""
    rng = np.random.default_rng(5)
    vm = np.hstack([np.eye(3), np.zeros((3, 1))]) if view == "identity" else _random_view(rng)
    cam = scenes.pinhole(640, 360, fx=500.0, fy=420.0, viewmat=vm)
    cam["viewmat"] = vm
    R3, t3 = vm[:, :3], vm[:, 3]
    limx, limy = 1.3 * 320 / 500.0, 1.3 * 180 / 420.0
    z = 4.0
    cases = [(1.25 * limx, 0.1), (0.2, -1.3 * limy), (-1.2 * limx, -1.4 * limy), (0.5 * limx, 0.5 * limy)]
    for (rx, ry) in cases:
        pc = np.array([rx * z, ry * z, z])
        mu = np.linalg.solve(R3, pc - t3)
        scales = np.array([0.9, 0.5, 0.7])   # wide enough to reach the image from outside the frustum
        q = rng.standard_normal(4)
        sc = make_scene(mu, scales, q, [0.9], [[0.5, 0.5, 0.5]])
        pr = oracle.project(cam, sc)
        assert pr["radius"][0] > 0, (rx, ry)
        pcl = np.array([np.clip(rx, -limx, limx) * z, np.clip(ry, -limy, limy) * z, z])
        J = _pinhole_cam_jacobian(cam, pcl)
        Rg = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        S_cam = R3 @ (Rg @ np.diag(scales ** 2) @ Rg.T) @ R3.T
        ref = J @ S_cam @ J.T + 0.3 * np.eye(2)
        a, b, c = pr["cov2d"][0]
        np.testing.assert_allclose([a, b, c], [ref[0, 0], ref[0, 1], ref[1, 1]], rtol=1e-6, atol=1e-9)
        np.testing.assert_allclose(pr["mean2d"][0], [500.0 * rx + 320.0, 420.0 * ry + 180.0], rtol=1e-12)


def test_projection_frustum_clamp_isotropic_closed_form():
    """Isotropic Gaussian (Sigma = s^2 I, identity view) at camera point (X, Y, Z) with X / Z past the
    limit: with xc = 1.3 tan(fov_x / 2) Z (the clamped abscissa) and Y inside,
    Sigma' = s^2 J J^T + 0.3 I, J = [[fx / Z, 0, -fx xc / Z^2], [0, fy / Z, -fy Y / Z^2]], so
    a = s^2 fx^2 (1 + (xc / Z)^2) / Z^2 + 0.3, b = s^2 fx fy xc Y / Z^4, c = s^2 fy^2 (1 + (Y / Z)^2) / Z^2 + 0.3."""
    fx, fy, W, H = 600.0, 500.0, 800, 400
    cam = scenes.pinhole(W, H, fx=fx, fy=fy)
    s, Z, X, Y = 1.0, 5.0, 5.0, 0.7
    sc = make_scene([X, Y, Z], [s, s, s], [0.4, 0.1, -0.7, 0.2], [0.9], [[0.5, 0.5, 0.5]])
    pr = oracle.project(cam, sc)
    xc = 1.3 * (W / 2 / fx) * Z
    assert X > xc and pr["radius"][0] > 0
    a = s * s * fx * fx * (1 + (xc / Z) ** 2) / Z ** 2 + 0.3
    b = s * s * fx * fy * xc * Y / Z ** 4
    c = s * s * fy * fy * (1 + (Y / Z) ** 2) / Z ** 2 + 0.3
    np.testing.assert_allclose(pr["cov2d"][0], [a, b, c], rtol=1e-12)


def test_projection_culls_behind_near_plane():
    cam = scenes.pinhole(64, 64, fx=64.0)
    sc = make_scene([[0, 0, 0.1], [0, 0, -3], [0, 0, 2]], np.full((3, 3), 0.05), np.tile([1, 0, 0, 0], (3, 1)),
                    [0.5, 0.5, 0.5], np.full((3, 3), 0.5))
    pr = oracle.project(cam, sc)
    assert list(pr["radius"][:2]) == [0, 0] and pr["radius"][2] > 0
    assert list(pr["tiles_touched"][:2]) == [0, 0]


def test_sh_colour_clamped_at_zero():
    cam = scenes.pinhole(64, 64, fx=64.0)
    sc = make_scene([0, 0, 3], [0.05] * 3, [1, 0, 0, 0], [0.5], [[-0.3, 0.2, 1.4]])
    pr = oracle.project(cam, sc)
    np.testing.assert_allclose(pr["rgb"][0], [0.0, 0.2, 1.4], atol=1e-12)


def test_degree3_colour_uses_view_direction():
    rng = np.random.default_rng(4)
    cam = scenes.pinhole(256, 256, fx=200.0, campos=[0.1, -0.2, -0.5])
    cam["campos"] = np.array([0.1, -0.2, -0.5])
    mu = np.array([0.2, 0.1, 4.0])
    sh = rng.normal(0, 0.3, (1, 16, 3))
    sc = dict(means3=mu[None], scales=np.full((1, 3), 0.05), quats=np.array([[1.0, 0, 0, 0]]),
              opacity=np.array([0.5]), sh=sh, sh_degree=3)
    pr = oracle.project(cam, sc)
    d = mu - cam["campos"]
    d /= np.linalg.norm(d)
    Y = np.array([_real_sh_3dgs(l, m, d) for l in range(4) for m in range(-l, l + 1)])
    np.testing.assert_allclose(pr["rgb"][0], np.maximum(Y @ sh[0] + 0.5, 0.0), atol=1e-12)


# ---------------------------------------------------------------- binning

def _brute_splats(cam, mean2d, radius, depth):
    gw, gh = oracle.grid(cam)
    out = []
    for g in range(len(radius)):
        r = radius[g]
        if r <= 0:
            continue
        for ty in range(gh):
            for tx in range(gw):
                inx = mean2d[g, 0] - r < 16 * tx + 16 and mean2d[g, 0] + r >= 16 * tx
                iny = mean2d[g, 1] - r < 16 * ty + 16 and mean2d[g, 1] + r >= 16 * ty
                if inx and iny:
                    out.append((ty * gw + tx, depth[g], g))
    return sorted(out)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_binning_matches_brute_force(seed):
    cam, sc = scenes.plain_forward(P=150, width=72, height=56, seed=seed)
    pr = oracle.project(cam, sc)
    b = oracle.bin_sort(cam, pr["mean2d"], pr["radius"], pr["depth"])
    ref = _brute_splats(cam, pr["mean2d"], pr["radius"], pr["depth"])
    assert b["n"] == len(ref) == int(pr["tiles_touched"].sum())
    assert list(b["tile_of"]) == [t for t, _, _ in ref]
    assert list(b["ids"]) == [g for _, _, g in ref]
    gw, gh = oracle.grid(cam)
    for t in range(gw * gh):
        members = [i for i, (tt, _, _) in enumerate(ref) if tt == t]
        if members:
            assert tuple(b["ranges"][t]) == (members[0], members[-1] + 1)
        else:
            assert b["ranges"][t, 0] == b["ranges"][t, 1]


def test_binning_depth_ties_ordered_by_index():
    cam = scenes.pinhole(32, 32, fx=32.0)
    mean2d = np.array([[10.0, 10.0], [12.0, 9.0], [11.0, 11.0]])
    radius = np.array([3, 3, 3], np.int32)
    depth = np.array([2.0, 1.0, 2.0])
    b = oracle.bin_sort(cam, mean2d, radius, depth)
    assert list(b["ids"]) == [1, 0, 2]


# ---------------------------------------------------------------- exact tile coverage

def test_box_min_matches_dense_sampling_and_bounded_optimiser():
    """The closed-form least value of the conic form over a box against the minimum over a
    dense grid of the box and against a bounded quasi-Newton solve."""
    from scipy.optimize import minimize
    rng = np.random.default_rng(5)
    for _ in range(60):
        A = rng.standard_normal((2, 2))
        Q = A @ A.T + rng.uniform(0.01, 0.5) * np.eye(2)
        a, b, c = Q[0, 0], Q[0, 1], Q[1, 1]
        x0, y0 = rng.uniform(-20, 20, 2)
        x1, y1 = x0 + rng.uniform(0.5, 15), y0 + rng.uniform(0.5, 15)
        m = rng.uniform(-40, 40, 2)
        got = oracle.box_min_q(m[0], m[1], a, b, c, x0, x1, y0, y1)
        xs, ys = np.meshgrid(np.linspace(x0, x1, 801), np.linspace(y0, y1, 801))
        dx, dy = xs - m[0], ys - m[1]
        grid_min = float((a * dx * dx + 2 * b * dx * dy + c * dy * dy).min())
        assert got <= grid_min + 1e-9 * (1 + grid_min)
        f = lambda p: float(Q[0, 0] * (p[0] - m[0]) ** 2 + 2 * Q[0, 1] * (p[0] - m[0]) * (p[1] - m[1])
                            + Q[1, 1] * (p[1] - m[1]) ** 2)
        best = min(minimize(f, np.array(s0), bounds=[(x0, x1), (y0, y1)], method="L-BFGS-B",
                            options=dict(ftol=1e-15, gtol=1e-12)).fun
                   for s0 in [(x0, y0), (x1, y1), ((x0 + x1) / 2, (y0 + y1) / 2)])
        assert abs(got - best) <= 1e-6 * (1 + best)


def _exact_case(seed, P=400, width=96, height=80):
    cam, sc = scenes.plain_forward(P=P, width=width, height=height, seed=seed)
    pr = oracle.project(cam, sc)
    op = np.asarray(sc["opacity"], np.float64)
    rect = oracle.bin_sort(cam, pr["mean2d"], pr["radius"], pr["depth"])
    exact = oracle.bin_sort(cam, pr["mean2d"], pr["radius"], pr["depth"], conic=pr["conic"], opacity=op)
    return cam, sc, pr, op, rect, exact


def _tile_lists(b):
    return [list(b["ids"][s:e]) for s, e in b["ranges"]]


def _max_alpha_on_tile(cam, pr, op, g, t):
    gw, _ = oracle.grid(cam)
    tx, ty = t % gw, t // gw
    ys, xs = np.meshgrid(16 * ty + np.arange(16) + 0.5, 16 * tx + np.arange(16) + 0.5, indexing="ij")
    dx, dy = xs - pr["mean2d"][g, 0], ys - pr["mean2d"][g, 1]
    s11, s12, s22 = pr["conic"][g]
    return float((op[g] * np.exp(-0.5 * (s11 * dx * dx + 2 * s12 * dx * dy + s22 * dy * dy))).max())


@pytest.mark.parametrize("seed", [0, 1])
def test_exact_coverage_drops_only_splats_culled_at_every_pixel(seed):
    """Each tile's exact list is its 3-sigma list minus entries whose alpha is below 1/255 at all
    256 pixel centres (brute force), in the same order; an entry that reaches 1/255 anywhere stays."""
    cam, sc, pr, op, rect, exact = _exact_case(seed)
    assert 0 < exact["n"] < rect["n"]
    for t, (lr, le) in enumerate(zip(_tile_lists(rect), _tile_lists(exact))):
        assert le == [g for g in lr if g in set(le)]          # a subsequence: order kept
        for g in set(lr) - set(le):
            assert _max_alpha_on_tile(cam, pr, op, g, t) < 1.0 / 255.0
        for g in le:
            if _max_alpha_on_tile(cam, pr, op, g, t) >= 1.0 / 255.0:
                continue
            # kept without reaching 1/255 at a pixel centre: only inside the box and margin slack
            gw, _ = oracle.grid(cam)
            tx, ty = t % gw, t // gw
            s11, s12, s22 = pr["conic"][g]
            qmin = oracle.box_min_q(pr["mean2d"][g, 0], pr["mean2d"][g, 1], s11, s12, s22, 16 * tx + 0.5,
                                    16 * tx + 15.5, 16 * ty + 0.5, 16 * ty + 15.5)
            assert qmin <= 2 * (math.log(op[g]) + math.log(255.0)) * 1.0001 + 1e-3


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_exact_coverage_rows_are_runs(seed):
    """In every row of tiles, the tiles a Gaussian's exact list entries fall in form one run of
    consecutive tiles: the reach region {q <= L} is convex and each tile's pixel-centre box spans the
    same band of rows, so a box meets the region exactly when its x-range meets the region's shadow
    on the band (an interval).  This is what lets wide Gaussians be covered row by row."""
    cam, sc, pr, op, rect, exact = _exact_case(seed, P=600, width=256, height=160)
    gw, gh = oracle.grid(cam)
    rows = {}
    for t, lst in enumerate(_tile_lists(exact)):
        for g in lst:
            rows.setdefault((g, t // gw), []).append(t % gw)
    wide = 0
    for (g, ty), txs in rows.items():
        txs = sorted(txs)
        assert txs == list(range(txs[0], txs[-1] + 1)), (g, ty, txs)
        wide += len(txs) >= 3
    assert wide > 20   # the scenes have Gaussians several tiles wide


@pytest.mark.parametrize("seed", [0, 1])
def test_exact_coverage_renders_the_same_image(seed):
    """Algorithm 1 over the exact lists gives the image and final transmittance of the 3-sigma
    lists bit for bit; n_contrib counts the same last blended Gaussian in the shorter list."""
    cam, sc, pr, op, rect, exact = _exact_case(seed)
    o_r = oracle.render(cam, rect, pr["mean2d"], pr["conic"], op, pr["rgb"])
    o_e = oracle.render(cam, exact, pr["mean2d"], pr["conic"], op, pr["rgb"])
    np.testing.assert_array_equal(o_r["img"], o_e["img"])
    np.testing.assert_array_equal(o_r["T"], o_e["T"])
    gw, _ = oracle.grid(cam)
    lr, le = _tile_lists(rect), _tile_lists(exact)
    H, W = o_r["T"].shape
    for y in range(H):
        for x in range(W):
            t = (y // 16) * gw + x // 16
            nr, ne = o_r["n_contrib"][y, x], o_e["n_contrib"][y, x]
            if nr == 0:
                assert ne == 0
            else:
                assert le[t][ne - 1] == lr[t][nr - 1]
    assert o_e["alpha_evals"] < o_r["alpha_evals"] and o_e["f_blend"] == o_r["f_blend"]


# ---------------------------------------------------------------- rendering

def _render_scene(cam, sc, alpha_max=0.99, bg=(0, 0, 0)):
    pr = oracle.project(cam, sc)
    b = oracle.bin_sort(cam, pr["mean2d"], pr["radius"], pr["depth"])
    op = np.asarray(sc["opacity"], np.float64)
    out = oracle.render(cam, b, pr["mean2d"], pr["conic"], op, pr["rgb"], bg=bg, alpha_max=alpha_max)
    return pr, b, out


def test_single_gaussian_closed_form():
    cam = scenes.pinhole(48, 40, fx=60.0)
    sc = make_scene([0.05, -0.03, 3.0], [0.08, 0.05, 0.06], [0.9, 0.1, 0.3, -0.2], [0.8], [[0.9, 0.3, 0.1]])
    pr, b, out = _render_scene(cam, sc)
    a_, b_, c_ = pr["cov2d"][0]
    Q = np.linalg.inv(np.array([[a_, b_], [b_, c_]]))  # conic from the covariance, independently
    m, (s11, s12, s22) = pr["mean2d"][0], (Q[0, 0], Q[0, 1], Q[1, 1])
    j, i = np.meshgrid(np.arange(40) + 0.5, np.arange(48) + 0.5, indexing="ij")
    dx, dy = m[0] - i, m[1] - j
    a = np.minimum(0.99, 0.8 * np.exp(-0.5 * (s11 * dx * dx + 2 * s12 * dx * dy + s22 * dy * dy)))
    # only pixels of covered tiles see the Gaussian
    gw, _ = oracle.grid(cam)
    tile = (j.astype(int) // 16) * gw + (i.astype(int) // 16)
    covered = np.isin(tile, b["tile_of"])
    a = np.where((a >= 1 / 255) & covered, a, 0.0)
    for ch, c in enumerate([0.9, 0.3, 0.1]):
        np.testing.assert_allclose(out["img"][ch], c * a, atol=1e-12)
    np.testing.assert_allclose(out["T"], 1 - a, atol=1e-12)


def test_two_colocated_gaussians_closed_form():
    cam = scenes.pinhole(32, 32, fx=40.0)
    sc = make_scene([[0, 0, 2.0], [0, 0, 3.0]], [[0.1] * 3, [0.15] * 3], [[1, 0, 0, 0]] * 2, [0.6, 0.7],
                    [[1, 0, 0], [0, 1, 0]])
    pr, b, out = _render_scene(cam, sc)
    p = (16, 16)  # pixel centre (16.5, 16.5); mean at (16, 16)
    a = []
    for g in range(2):
        d = pr["mean2d"][g] - np.array([16.5, 16.5])
        s11, s12, s22 = pr["conic"][g]
        a.append(min(0.99, sc["opacity"][g] * math.exp(-0.5 * (s11 * d[0] ** 2 + 2 * s12 * d[0] * d[1] + s22 * d[1] ** 2))))
    assert abs(out["img"][0][p] - a[0]) < 1e-13
    assert abs(out["img"][1][p] - a[1] * (1 - a[0])) < 1e-13
    assert abs(out["T"][p] - (1 - a[0]) * (1 - a[1])) < 1e-13


def test_termination_index():
    """Five co-located Gaussians with alpha 0.95 at the centre: T runs 1, .05, .0025,
    1.25e-4; the fourth would give 6.25e-6 < 1e-4, so it breaks there unblended."""
    cam = scenes.pinhole(17, 17, fx=17.0)  # cx = 8.5: pixel (8, 8) samples the mean exactly
    P = 5
    sc = make_scene(np.tile([0.0, 0.0, 0.0], (P, 1)) + np.array([[0, 0, 2.0 + 0.1 * k] for k in range(P)]),
                    np.full((P, 3), 1.0), np.tile([1, 0, 0, 0], (P, 1)), np.full(P, 0.95), np.full((P, 3), 1.0))
    pr, b, out = _render_scene(cam, sc, alpha_max=1.0)
    p = (8, 8)
    d = pr["mean2d"][0] - np.array([8.5, 8.5])
    assert np.abs(d).max() < 1e-12
    assert out["n_contrib"][p] == 3 and out["n_eval"][p] == 4
    assert abs(out["T"][p] - 0.05 ** 3) < 1e-15


def test_alg1_literal_opaque_gaussian_breaks_unblended():
    """With alpha_max = 1 (no clamp) an alpha = 1 fragment fails T - aT >= 1e-4 at once
    and Algorithm 1 breaks without blending it; the 0.99 clamp keeps it."""
    cam = scenes.pinhole(17, 17, fx=17.0)
    sc = make_scene([0, 0, 2.0], [1.0, 1.0, 1.0], [1, 0, 0, 0], [1.0], [[1, 1, 1]])
    _, _, lit = _render_scene(cam, sc, alpha_max=1.0)
    _, _, clamped = _render_scene(cam, sc, alpha_max=0.99)
    assert lit["img"][0, 8, 8] == 0.0 and lit["T"][8, 8] == 1.0
    assert abs(clamped["img"][0, 8, 8] - 0.99) < 1e-15


def test_cull_threshold():
    cam = scenes.pinhole(17, 17, fx=17.0)
    for o, seen in [(1 / 255 * 0.999, False), (1 / 255 * 1.001, True)]:
        sc = make_scene([0, 0, 2.0], [1.0, 1.0, 1.0], [1, 0, 0, 0], [o], [[1, 1, 1]])
        _, _, out = _render_scene(cam, sc)
        assert (out["img"][0, 8, 8] > 0) == seen


def test_white_composite_equals_one_minus_T_and_T_monotone():
    cam, sc = scenes.plain_forward(P=300, width=64, height=48, seed=7)
    sc["sh"][:] = 0.5 / (0.5 / math.sqrt(math.pi))  # colour exactly 1
    pr, b, out = _render_scene(cam, scene_arrays(sc))
    np.testing.assert_allclose(out["img"][0], 1 - out["T"], atol=1e-12)
    assert (out["T"] > 0).all() and (out["T"] <= 1).all()
    # T along each pixel's list never increases: check with growing list prefixes
    b2 = dict(b)
    prev = np.ones_like(out["T"])
    for cut in [1, 2, 4, 8, 16, 10 ** 9]:
        r = b["ranges"].copy()
        r[:, 1] = np.minimum(r[:, 1], r[:, 0] + cut)
        b2["ranges"] = r
        o2 = oracle.render(cam, b2, pr["mean2d"], pr["conic"], sc["opacity"], pr["rgb"])
        assert (o2["T"] <= prev + 1e-15).all()
        prev = o2["T"]


@pytest.mark.parametrize("seed,bg", [(0, (0, 0, 0)), (1, (0.2, 0.5, 0.9))])
def test_tiled_equals_untiled_bruteforce(seed, bg):
    cam, sc = scenes.plain_forward(P=200, width=56, height=40, seed=seed)
    sc = scene_arrays(sc)
    pr, b, out = _render_scene(cam, sc, bg=bg)
    bf = oracle.render_bruteforce(cam, pr["mean2d"], pr["radius"], pr["depth"], pr["conic"], sc["opacity"],
                                  pr["rgb"], bg=bg)
    assert np.array_equal(out["img"], bf["img"])
    assert np.array_equal(out["T"], bf["T"])
    assert np.array_equal(out["n_contrib"], bf["n_contrib"])


def test_tight_radius_closed_form_and_opacity_cull():
    f, z, s = 300.0, 5.0, 0.04
    cam = scenes.pinhole(320, 240, fx=f)
    var = (f * s / z) ** 2 + 0.3
    for o in [0.9, 0.05, 1.5 / 255]:
        sc = make_scene([0, 0, z], [s, s, s], [1, 0, 0, 0], [o], [[0.2, 0.4, 0.6]])
        pr = oracle.project(cam, sc, tight_radius=True)
        assert pr["radius"][0] == math.ceil(math.sqrt(2 * math.log(255 * o) * (var + math.sqrt(0.1))))
    sc = make_scene([0, 0, z], [s, s, s], [1, 0, 0, 0], [0.999 / 255], [[0.2, 0.4, 0.6]])
    assert oracle.project(cam, sc, tight_radius=True)["radius"][0] == 0      # reaches no pixel
    assert oracle.project(cam, sc)["radius"][0] > 0                           # the 3-sigma square keeps it


@pytest.mark.parametrize("seed", [3, 4])
def test_tight_radius_tiled_equals_untiled_without_membership(seed):
    """With the opacity-aware square, every pixel where alpha >= 1/255 lies in a covered tile, so
    the tiled render equals Algorithm 1 over all Gaussians at every pixel; the 3-sigma square cuts
    opaque Gaussians off (o exp(-9/2) > 1/255 when o > 0.36) and does not."""
    cam, sc = scenes.plain_forward(P=200, width=56, height=40, seed=seed)
    sc = scene_arrays(sc)
    sc["opacity"] = np.where(np.arange(200) % 2 == 0, 0.97, sc["opacity"])   # many opaque Gaussians
    sc["scales"] = sc["scales"] * 4                                          # splats of several pixels
    op = sc["opacity"]
    proj = {tight: oracle.project(cam, sc, tight_radius=tight) for tight in (True, False)}
    # every Gaussian either square keeps, each at every pixel (one left out by both has alpha < 1/255
    # at every pixel, or fails the near-plane or determinant test)
    kept_t = proj[True]["radius"] > 0
    src = {k: np.where(kept_t.reshape(-1, *[1] * (proj[True][k].ndim - 1)), proj[True][k], proj[False][k])
           for k in ("mean2d", "conic", "depth", "rgb")}
    everywhere = np.where(kept_t | (proj[False]["radius"] > 0), 10 ** 6, 0).astype(np.int32)
    bf = oracle.render_bruteforce(cam, src["mean2d"], everywhere, src["depth"], src["conic"], op, src["rgb"])
    err = {}
    for tight, pr in proj.items():
        b = oracle.bin_sort(cam, pr["mean2d"], pr["radius"], pr["depth"])
        out = oracle.render(cam, b, pr["mean2d"], pr["conic"], op, pr["rgb"])
        err[tight] = (np.abs(out["img"] - bf["img"]).max(), np.abs(out["T"] - bf["T"]).max())
    assert err[True][0] <= 1e-12 and err[True][1] <= 1e-12
    assert err[False][0] > 1e-4


def test_fragment_counts_consistent():
    cam, sc = scenes.plain_forward(P=300, width=64, height=64, seed=5)
    pr, b, out = _render_scene(cam, scene_arrays(sc))
    assert out["f_blend"] + out["f_cull"] == out["alpha_evals"] == int(out["n_eval"].sum())
    assert (out["n_contrib"] <= out["n_eval"]).all()


# ---------------------------------------------------------------- Frag2Mat / G2L

def test_frag2mat_identity_global_and_local():
    rng = np.random.default_rng(8)
    n = 64
    mean2d = rng.uniform(0, 200, (n, 2))
    L = rng.normal(0, 0.5, (n, 2, 2))
    Q = np.einsum("nij,nkj->nik", L, L) + 0.05 * np.eye(2)
    conic = np.stack([Q[:, 0, 0], Q[:, 0, 1], Q[:, 1, 1]], 1)
    o = rng.uniform(0.01, 1, n)
    px, py = rng.uniform(0, 200, 100), rng.uniform(0, 200, 100)
    ref = f2m.beta_direct(px, py, mean2d, conic, o)
    got = f2m.pixel_vectors(px, py) @ f2m.gaussian_vectors(mean2d, conic, o).T
    np.testing.assert_allclose(got, ref, atol=1e-9 * np.abs(ref).max())
    # G2L: shifting pixels and means by the same tile centre leaves beta unchanged
    c = f2m.tile_centre(3, 5)
    got_l = f2m.pixel_vectors(px - c[0], py - c[1]) @ f2m.gaussian_vectors(mean2d - c, conic, o).T
    np.testing.assert_allclose(got_l, ref, atol=1e-9 * np.abs(ref).max())


def test_g2l_pixel_vectors_small_and_exact_in_fp16():
    dx, dy = f2m.tile_pixels_local()
    U = f2m.pixel_vectors(dx, dy)
    assert np.abs(U).max() <= GOLD["local_max_u"]["value"]
    assert np.abs(np.stack([dx, dy])).max() <= GOLD["local_range"]["value"]
    assert np.array_equal(f2m.round_f16(U), U)


def _emulate_tc(U, V, dtype=np.float16):
    """Tensor-core dot products: inputs rounded to ``dtype``, exact products, FP32
    accumulation left to right (Appendix A's model)."""
    Ur = U.astype(dtype).astype(np.float64)
    Vr = V.astype(dtype).astype(np.float64)
    acc = np.zeros((U.shape[0], V.shape[0]), np.float32)
    for k in range(U.shape[1]):
        acc = (acc.astype(np.float64) + np.outer(Ur[:, k], Vr[:, k])).astype(np.float32)
    return acc.astype(np.float64)


def test_appendix_bound_holds_for_emulated_fp16_local():
    cam, sc = scenes.plain_forward(P=400, width=96, height=96, seed=9)
    pr = oracle.project(cam, scene_arrays(sc))
    b = oracle.bin_sort(cam, pr["mean2d"], pr["radius"], pr["depth"])
    gw, gh = oracle.grid(cam)
    checked = 0
    for t in range(gw * gh):
        s, e = b["ranges"][t]
        ids = b["ids"][s:e]
        if len(ids) == 0:
            continue
        U, V, beta, absum = f2m.local_products(t % gw, t // gw, pr["mean2d"][ids], pr["conic"][ids],
                                               sc["opacity"][ids])
        bh = _emulate_tc(U, V)
        keep = beta >= -math.log(255.0)  # the bound is stated for fragments that are not culled
        err = np.abs(bh - beta)
        assert (err[keep] <= f2m.paper_bound(absum)[keep] + 1e-5).all()
        checked += keep.sum()
    assert checked > 1000


def test_global_fp16_overflows_at_1920px():
    """Sec. 4.3: global pixel coordinates make u's quadratic terms overflow FP16."""
    U = f2m.pixel_vectors(np.array([1919.5]), np.array([1079.5]))
    assert np.isinf(U.astype(np.float16)).any()


def _format_values(exp_bits, frac_bits, bias, max_exp_field):
    """Every finite non-negative value of a binary float format, built from its bit fields."""
    vals = [0.0]
    for f in range(1, 2 ** frac_bits):   # subnormals: 0.f x 2^(1 - bias)
        vals.append(f / 2 ** frac_bits * 2.0 ** (1 - bias))
    for e in range(1, max_exp_field + 1):
        for f in range(2 ** frac_bits):
            vals.append((1 + f / 2 ** frac_bits) * 2.0 ** (e - bias))
    return np.array(sorted(vals))


def test_e4m3_rounding_against_the_format_definition():
    # e4m3: exponent field 1..15 normal except the all-ones pattern 1111.111 (NaN), so the
    # largest finite value is 1.110 x 2^8 = 448
    vals = _format_values(4, 3, 7, 15)[:-1]
    assert vals[-1] == 448.0 and vals[1] == 2.0 ** -9 and len(vals) == 127
    assert np.array_equal(f2m.round_e4m3(vals), vals)
    assert np.array_equal(f2m.round_e4m3(-vals), -vals)
    mids = 0.5 * (vals[1:] + vals[:-1])
    r = f2m.round_e4m3(mids)
    # a midpoint goes to the neighbour whose last fraction bit is 0 (ties to even)
    lo, hi = vals[:-1], vals[1:]
    even_lo = np.array([(round(v / 2.0 ** (max(math.floor(math.log2(v)), -6) - 3)) % 2 == 0) if v > 0 else True
                        for v in lo])
    assert np.array_equal(r, np.where(even_lo, lo, hi))
    rng = np.random.default_rng(30)
    x = rng.uniform(0, 460, 20000) * 2.0 ** rng.integers(-12, 1, 20000)
    r = f2m.round_e4m3(x)
    nearest = vals[np.abs(x[:, None] - vals[None, :]).argmin(1)]
    ok = np.abs(r - x) <= np.abs(nearest - x) + 0.0
    assert ok.all()
    assert f2m.round_e4m3(1e6) == 448.0   # saturation


def test_tf32_rounding_against_the_format_definition():
    rng = np.random.default_rng(31)
    x = rng.uniform(1, 2, 20000)
    r = f2m.round_tf32(x)
    grid = 1 + np.arange(2 ** 10 + 1) / 2 ** 10   # TF32 values in [1, 2]
    idx = np.abs(x[:, None] - grid[None, :]).argmin(1)
    assert np.array_equal(r, grid[idx])
    assert f2m.round_tf32(1 + 2.0 ** -11) == 1 + 2.0 ** -10      # ties away from zero
    assert f2m.round_tf32(-(1 + 2.0 ** -11)) == -(1 + 2.0 ** -10)
    assert np.array_equal(f2m.round_tf32(x * 2.0 ** 40), r * 2.0 ** 40)


def test_fp8_split_of_tile_pixel_vectors_is_exact():
    """Every G2L pixel vector, column-scaled, is the sum of two e4m3 numbers: u is carried
    exactly by the FP8 encoding, so all of its error comes from v."""
    dx, dy = f2m.tile_pixels_local()
    U = f2m.pixel_vectors(dx, dy) * 2.0 ** -np.array(f2m.FP8_COLUMN_EXP)
    hi = f2m.round_e4m3(U)
    lo = f2m.round_e4m3(U - hi)
    assert np.array_equal(hi + lo, U)
    assert np.abs(U).min() >= 2.0 ** -8   # (dx, dy never 0) every part at or above the subnormal grid


def _reachable_gaussians(rng, n):
    """Tile-local Gaussians that can reach alpha >= 1/255 in a tile: Q with eigenvalues in
    [1e-4, 1 / 0.3] (the 0.3 px^2 dilation), opacity in [1/255, 1], and Q-distance of the local
    mean at most sqrt(2 ln(255 o)) + 7.5 sqrt(2) sqrt(lambda_max(Q)) (the reach of the tile), with
    a share of samples on the extremes."""
    lam = np.exp(rng.uniform(np.log(1e-4), np.log(1 / 0.3), (n, 2)))
    lam[: n // 4, :] = 1 / 0.3
    th = rng.uniform(0, np.pi, n)
    c, s = np.cos(th), np.sin(th)
    Q11 = lam[:, 0] * c * c + lam[:, 1] * s * s
    Q22 = lam[:, 0] * s * s + lam[:, 1] * c * c
    Q12 = (lam[:, 0] - lam[:, 1]) * c * s
    o = np.exp(rng.uniform(np.log(1 / 255), 0, n))
    o[: n // 4] = 1.0
    lmax = lam.max(1)
    reach = np.sqrt(2 * np.log(255 * o)) + 7.5 * np.sqrt(2) * np.sqrt(lmax)
    # a point at Q-distance `reach` in a random direction: mu = reach * L^-T w, |w| = 1
    phi = rng.uniform(0, 2 * np.pi, n)
    w = np.stack([np.cos(phi), np.sin(phi)], 1)
    frac = np.where(np.arange(n) < n // 2, 1.0, rng.uniform(0, 1, n))
    mu = np.empty((n, 2))
    for i in range(n):
        Q = np.array([[Q11[i], Q12[i]], [Q12[i], Q22[i]]])
        Lc = np.linalg.cholesky(Q)
        mu[i] = np.linalg.solve(Lc.T, w[i]) * reach[i] * frac[i]
    return mu, np.stack([Q11, Q12, Q22], 1), o


def test_fp8_column_scales_keep_reachable_v_in_range():
    rng = np.random.default_rng(32)
    mu, conic, o = _reachable_gaussians(rng, 4000)
    V = f2m.gaussian_vectors(mu, conic, o) / math.log(2.0)        # log2 units, as encoded
    Vs = V * 2.0 ** np.array(f2m.FP8_COLUMN_EXP)
    assert np.abs(Vs).max() < f2m.E4M3_MAX


def test_fp8_split_bound_holds_by_emulation():
    rng = np.random.default_rng(33)
    mu, conic, o = _reachable_gaussians(rng, 3000)
    dx, dy = f2m.tile_pixels_local()
    U = f2m.pixel_vectors(dx, dy)
    V = f2m.gaussian_vectors(mu, conic, o) / math.log(2.0)
    exact = U @ V.T
    got = f2m.fp8_split(U, V)
    bound = f2m.fp8_split_bound(U, V, log2_scale=True)
    err = np.abs(got - exact)
    assert (err <= bound).all(), float((err - bound).max())
    # the bound is not vacuous (some fragment comes within a factor 5 of it), and the split is far
    # better than a single e4m3 rounding of v
    assert (err / bound).max() > 0.2
    sc = 2.0 ** np.array(f2m.FP8_COLUMN_EXP)
    one_term = (U / sc) @ f2m.round_e4m3(V * sc).T
    assert np.abs(one_term - exact).max() > 100 * err.max()


def test_appendix_bound_holds_for_tf32_in_global_coordinates():
    """Frag2Mat without G2L on TF32 inputs (Table 5): the Appendix A bound still holds, but in
    global coordinates sum |u_i v_i| is orders of magnitude larger than |beta|."""
    rng = np.random.default_rng(34)
    n = 200
    mean2d = np.c_[rng.uniform(1700, 1800, n), rng.uniform(900, 1000, n)]
    mu, conic, o = _reachable_gaussians(rng, n)
    tx, ty = 1750 // 16, 950 // 16
    U, V, beta, absum = f2m.global_products(tx, ty, f2m.tile_centre(tx, ty)[None, :] + mu, conic, o)
    got = f2m.round_tf32(U) @ f2m.round_tf32(V).T
    assert (np.abs(got - beta) <= f2m.paper_bound(absum)).all()
    # same Gaussians in the tile's local frame: the bound shrinks by orders of magnitude
    _, _, beta_l, absum_l = f2m.local_products(tx, ty, f2m.tile_centre(tx, ty)[None, :] + mu, conic, o)
    np.testing.assert_allclose(beta_l, beta, atol=1e-6 * np.abs(absum).max())
    assert np.median(absum / absum_l) > 1e3


def test_global_fp16_overflow_culls():
    """Past 256 px, u's quadratic terms overflow FP16 to +inf; with sigma11, sigma22 > 0 the
    exponent is then -inf or NaN, which the EarlyCull comparison rejects: the fragment is dropped."""
    rng = np.random.default_rng(35)
    mu, conic, o = _reachable_gaussians(rng, 200)
    tx, ty = 40, 20
    c = f2m.tile_centre(tx, ty)
    U, V, beta, _ = f2m.global_products(tx, ty, c[None, :] + mu, conic, o)
    # the paper's K = 8 layout of both operands
    Up = np.c_[U[:, :1], U[:, :1], U[:, :1], U[:, 1:]].astype(np.float16).astype(np.float64)
    Vp = np.c_[V[:, :1] / 3, V[:, :1] / 3, V[:, :1] / 3, V[:, 1:]].astype(np.float16).astype(np.float64)
    assert np.isinf(Up).any(axis=1).all()
    with np.errstate(invalid="ignore", over="ignore"):
        bh = Up @ Vp.T
    assert not (bh >= -math.log(255.0)).any()
    assert (np.isnan(bh) | (bh == -np.inf)).all()


def test_constants_match_paper():
    assert abs(f2m.EPS_H - GOLD["eps_H"]["value"]) < 5e-7
    assert abs(f2m.EPS_F - GOLD["eps_F"]["value"]) < 5e-10
    assert abs(-math.log(255.0) - GOLD["early_cull_beta"]["value"]) < 1e-12
    assert abs(1 / 255 - GOLD["cull_alpha"]["value"]) < 1e-15


# ---------------------------------------------------------------- backward

def _fd_setup(seed=11):
    cam, sc = scenes.plain_forward(P=200, width=64, height=64, seed=seed)
    pr = oracle.project(cam, scene_arrays(sc))
    b = oracle.bin_sort(cam, pr["mean2d"], pr["radius"], pr["depth"])
    rng = np.random.default_rng(seed)
    gimg = rng.standard_normal((3, 64, 64))
    return cam, sc, pr, b, gimg


def test_backward_matches_finite_differences():
    cam, sc, pr, b, gimg = _fd_setup()
    op = np.asarray(sc["opacity"], np.float64)
    base = dict(mean2d=pr["mean2d"].copy(), conic=pr["conic"].copy(), opacity=op.copy(), rgb=pr["rgb"].copy())
    g = oracle.render_bwd(cam, b, base["mean2d"], base["conic"], base["opacity"], base["rgb"], gimg)
    grads = dict(mean2d=g["dmean2d"], conic=g["dconic"], opacity=g["dopacity"], rgb=g["drgb"])
    ref = oracle.render(cam, b, **base)

    def loss(p):
        o = oracle.render(cam, b, p["mean2d"], p["conic"], p["opacity"], p["rgb"])
        stable = (np.array_equal(o["n_contrib"], ref["n_contrib"]) and np.array_equal(o["n_eval"], ref["n_eval"]))
        return float((o["img"] * gimg).sum()), stable

    rng = np.random.default_rng(0)
    visible = np.nonzero(pr["radius"] > 0)[0]
    # pick Gaussians with non-negligible gradient
    mag = np.abs(g["dopacity"][visible])
    cand = visible[np.argsort(-mag)[:40]]
    n_checked = 0
    for name, h in [("mean2d", 1e-5), ("conic", 1e-7), ("opacity", 1e-7), ("rgb", 1e-6)]:
        for gid in rng.choice(cand, 6, replace=False):
            for k in range(base[name].reshape(len(op), -1).shape[1]):
                p_plus = {kk: vv.copy() for kk, vv in base.items()}
                p_minus = {kk: vv.copy() for kk, vv in base.items()}
                p_plus[name].reshape(len(op), -1)[gid, k] += h
                p_minus[name].reshape(len(op), -1)[gid, k] -= h
                lp, s1 = loss(p_plus)
                lm, s2 = loss(p_minus)
                if not (s1 and s2):
                    continue  # a cull / termination decision flipped: not differentiable here
                fd = (lp - lm) / (2 * h)
                an = grads[name].reshape(len(op), -1)[gid, k]
                assert abs(fd - an) <= 1e-5 * max(1.0, abs(an)), (name, gid, k, fd, an)
                n_checked += 1
    assert n_checked > 40


def test_backward_clamped_alpha_finite_differences():
    """Fragments whose alpha hits the 0.99 clamp carry no gradient through the
    exponent; a near-opaque Gaussian over several pixels exercises that branch."""
    cam = scenes.pinhole(32, 32, fx=32.0)
    sc = make_scene([[0.02, -0.01, 2.0], [0.1, 0.05, 3.0], [-0.2, 0.1, 2.5]],
                    [[0.5, 0.45, 0.4], [0.2, 0.15, 0.1], [0.1, 0.3, 0.1]],
                    [[1, 0, 0, 0], [0.9, 0.2, 0.1, 0.3], [0.7, -0.3, 0.2, 0.1]],
                    [0.9995, 0.6, 0.8], [[0.9, 0.2, 0.3], [0.1, 0.8, 0.3], [0.4, 0.4, 0.9]])
    pr = oracle.project(cam, sc)
    b = oracle.bin_sort(cam, pr["mean2d"], pr["radius"], pr["depth"])
    base = dict(mean2d=pr["mean2d"].copy(), conic=pr["conic"].copy(), opacity=sc["opacity"].copy(),
                rgb=pr["rgb"].copy())
    ref = oracle.render(cam, b, **base)
    d = ref["img"]  # sanity: the clamp is active at some pixel
    q = base["conic"][0]
    j, i = np.meshgrid(np.arange(32) + 0.5, np.arange(32) + 0.5, indexing="ij")
    dx, dy = base["mean2d"][0, 0] - i, base["mean2d"][0, 1] - j
    raw = 0.9995 * np.exp(-0.5 * (q[0] * dx * dx + 2 * q[1] * dx * dy + q[2] * dy * dy))
    assert (raw > 0.99).sum() >= 2 and d.max() > 0
    gimg = np.random.default_rng(5).standard_normal((3, 32, 32))
    g = oracle.render_bwd(cam, b, base["mean2d"], base["conic"], base["opacity"], base["rgb"], gimg)
    grads = dict(mean2d=g["dmean2d"], conic=g["dconic"], opacity=g["dopacity"], rgb=g["drgb"])
    for name, h in [("mean2d", 1e-6), ("conic", 1e-8), ("opacity", 1e-8)]:
        arr = base[name].reshape(3, -1)
        for k in range(arr.shape[1]):
            pp = {kk: vv.copy() for kk, vv in base.items()}
            pm = {kk: vv.copy() for kk, vv in base.items()}
            pp[name].reshape(3, -1)[0, k] += h
            pm[name].reshape(3, -1)[0, k] -= h
            op_, om_ = oracle.render(cam, b, **pp), oracle.render(cam, b, **pm)
            assert np.array_equal(op_["n_contrib"], ref["n_contrib"])
            fd = ((op_["img"] * gimg).sum() - (om_["img"] * gimg).sum()) / (2 * h)
            an = grads[name].reshape(3, -1)[0, k]
            assert abs(fd - an) <= 2e-5 * max(1.0, abs(an)), (name, k, fd, an)


# ---------------------------------------------------------------- projection backward

def _project_fd_case(seed, deg=3, clamp=False):
    rng = np.random.default_rng(seed)
    P = 12
    cam = scenes.pinhole(160, 120, fx=150.0)
    R = Rotation.from_rotvec(rng.normal(0, 0.2, 3)).as_matrix()
    cam["viewmat"] = np.hstack([R, rng.normal(0, 0.3, (3, 1))]).reshape(-1).tolist()
    cam["campos"] = (-R.T @ np.asarray(cam["viewmat"]).reshape(3, 4)[:, 3]).tolist()
    means3 = np.c_[rng.uniform(-1, 1, P), rng.uniform(-0.8, 0.8, P), rng.uniform(3, 6, P)]
    means3 = (R.T @ (means3.T - np.asarray(cam["viewmat"]).reshape(3, 4)[:, 3:])).T   # in front of the camera
    scales = np.exp(rng.normal(-2.5, 0.4, (P, 3)))
    if clamp:   # far outside the frustum in x, large enough to still touch the image
        t = np.asarray(cam["viewmat"]).reshape(3, 4)
        cm = np.c_[np.full(P, 3.5), rng.uniform(-0.5, 0.5, P), np.full(P, 2.0)]
        means3 = (R.T @ (cm.T - t[:, 3:])).T
        scales = np.full((P, 3), 1.5)
    sc = dict(means3=means3, scales=scales, quats=rng.normal(0, 1, (P, 4)) * 2.0, opacity=np.full(P, 0.5),
              sh=rng.normal(0, 0.3, (P, (deg + 1) ** 2, 3)), sh_degree=deg)
    sc["sh"][:, 0, :] = 1.0   # colours away from the clamp at 0
    return cam, sc


@pytest.mark.parametrize("seed,deg,clamp", [(40, 3, False), (41, 1, False), (42, 3, True)])
def test_project_backward_matches_finite_differences(seed, deg, clamp):
    cam, sc = _project_fd_case(seed, deg, clamp)
    rng = np.random.default_rng(seed + 100)
    pr = oracle.project(cam, sc)
    vis = pr["radius"] > 0
    assert vis.sum() >= 6
    P = len(vis)
    wm, wc, wr = rng.normal(size=(P, 2)), rng.normal(size=(P, 3)), rng.normal(size=(P, 3))
    if clamp:
        txtz = np.array([(np.asarray(cam["viewmat"]).reshape(3, 4) @ np.r_[m, 1.0]) for m in sc["means3"]])
        assert (txtz[:, 0] / txtz[:, 2] > 1.3 * cam["width"] / (2 * cam["fx"]))[vis].all()   # clamped Jacobian

    def loss(s):
        o = oracle.project(cam, s)
        return float((o["mean2d"] * wm).sum() + (o["conic"] * wc).sum() + (o["rgb"] * wr).sum())

    g = oracle.project_bwd(cam, sc, pr["radius"], wm, wc, wr)
    grads = dict(means3=g["dmeans3"], scales=g["dscales"], quats=g["dquats"], sh=g["dsh"])
    for name, h in [("means3", 1e-6), ("scales", 1e-7), ("quats", 1e-6), ("sh", 1e-6)]:
        base = sc[name]
        for gid in np.nonzero(vis)[0][:6]:
            for k in range(base[gid].size):
                sp = {kk: (vv.copy() if isinstance(vv, np.ndarray) else vv) for kk, vv in sc.items()}
                sm = {kk: (vv.copy() if isinstance(vv, np.ndarray) else vv) for kk, vv in sc.items()}
                sp[name][gid].reshape(-1)[k] += h
                sm[name][gid].reshape(-1)[k] -= h
                fd = (loss(sp) - loss(sm)) / (2 * h)
                an = grads[name][gid].reshape(-1)[k]
                assert abs(fd - an) <= 2e-5 * max(1.0, abs(an)), (name, gid, k, fd, an)
    # culled Gaussians get zero gradients
    assert (g["dmeans3"][~vis] == 0).all()


def test_end_to_end_gradient_chain_matches_finite_differences():
    """dL/d(3D parameters) of L = sum(img * G) through Algorithm 1 and the preprocess: the
    oracle's render backward followed by its projection backward (the conic convention of the
    two must agree) against central differences of the whole oracle forward."""
    cam, sc = scenes.plain_forward(P=120, width=48, height=48, seed=7)
    sc = scene_arrays(sc)
    sc["scales"] = sc["scales"] * 3.0
    op = sc["opacity"]
    rng = np.random.default_rng(8)
    G = rng.standard_normal((3, 48, 48))
    pr = oracle.project(cam, sc)
    b = oracle.bin_sort(cam, pr["mean2d"], pr["radius"], pr["depth"])
    ref = oracle.render(cam, b, pr["mean2d"], pr["conic"], op, pr["rgb"])
    rb = oracle.render_bwd(cam, b, pr["mean2d"], pr["conic"], op, pr["rgb"], G)
    g = oracle.project_bwd(cam, sc, pr["radius"], rb["dmean2d"], rb["dconic"], rb["drgb"])

    def loss(s):
        p2 = oracle.project(cam, s)
        if not np.array_equal(p2["radius"], pr["radius"]):
            return None, False
        b2 = oracle.bin_sort(cam, p2["mean2d"], p2["radius"], p2["depth"])
        o = oracle.render(cam, b2, p2["mean2d"], p2["conic"], op, p2["rgb"])
        same = np.array_equal(b2["ids"], b["ids"]) and np.array_equal(o["n_eval"], ref["n_eval"]) and \
            np.array_equal(o["n_contrib"], ref["n_contrib"])
        return float((o["img"] * G).sum()), same

    vis = np.nonzero(pr["radius"] > 0)[0]
    cand = vis[np.argsort(-np.abs(rb["dopacity"][vis]))[:8]]
    checked = 0
    for name, h, key in [("means3", 1e-6, "dmeans3"), ("scales", 1e-7, "dscales"), ("quats", 1e-6, "dquats"),
                         ("sh", 1e-6, "dsh")]:
        for gid in cand[:5]:
            for k in range(sc[name][gid].size):
                sp = {kk: (vv.copy() if isinstance(vv, np.ndarray) else vv) for kk, vv in sc.items()}
                sm = {kk: (vv.copy() if isinstance(vv, np.ndarray) else vv) for kk, vv in sc.items()}
                sp[name][gid].reshape(-1)[k] += h
                sm[name][gid].reshape(-1)[k] -= h
                lp, s1 = loss(sp)
                lm, s2 = loss(sm)
                if not (s1 and s2):
                    continue   # a discrete decision moved: not differentiable here
                fd = (lp - lm) / (2 * h)
                an = g[key][gid].reshape(-1)[k]
                assert abs(fd - an) <= 1e-4 * max(1.0, abs(an)), (name, gid, k, fd, an)
                checked += 1
    assert checked >= 60
