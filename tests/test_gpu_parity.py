"""GPU parity of every stage against the FP64 oracle, through the C ABI.

Bars (stated per test): bit-exact for binning/sort (integer work); FP32 render max |RGB| <= 1e-5
outside decision-margin pixels (counted, expected << 0.1%); TC render PSNR >= 50 dB and >= 99.9% of
pixels within 2e-3; Frag2Mat exponents within the Appendix-A bound; backward within 1e-4 relative
of the oracle's analytic gradient (itself pinned by finite differences)."""
import math

import numpy as np
import pytest

import oracle
from oracle import frag2mat as f2m
from paper_2505_24796_gb300 import scenes

from .helpers import f32, gaussians_at_pixels, oracle_frame, psnr, scene64, to_torch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.fixture(scope="module")
def tc():
    import paper_2505_24796_gb300 as m
    m._lib.load()
    return m


def gpu_inputs(inp, b):
    return dict(mean2d=to_torch(inp["mean2d"], DEV), conic=to_torch(inp["conic"], DEV),
                depth=to_torch(inp["depth"], DEV), radius=to_torch(inp["radius"].astype(np.int32), DEV),
                rgb=to_torch(inp["rgb"], DEV), opacity=to_torch(inp["opacity"], DEV),
                ranges=to_torch(b["ranges"].astype(np.int32), DEV),
                ids=to_torch(b["ids"].astype(np.int32) if b["n"] > 0 else np.zeros(1, np.int32), DEV))


# workloads: (name, factory kwargs) -- small enough for the oracle, several tiles, ragged edges
SMALL = [
    ("plain_128", lambda: scenes.plain_forward()),
    ("plain_ragged_200x136", lambda: scenes.plain_forward(P=1500, width=200, height=136, seed=11)),
    ("precision_crop_240x120", lambda: scenes.precision(P=30_000, width=240, height=120, seed=12)),
]


# ------------------------------------------------------------------ projection

# projection cases: the small workloads plus a view whose Gaussians reach the image from up to three
# half-fields outside it, so the frustum clamp of the Jacobian is active for many of them
PROJ = SMALL + [("wide_field_160x96", lambda: scenes.wide_field())]


@pytest.mark.parametrize("name,make", PROJ)
@pytest.mark.parametrize("tight", [False, True])
def test_project_matches_oracle(tc, name, make, tight):
    """Projection against the FP64 oracle.  The conic is the inverse of Sigma', whose FP32 entries
    carry a few ulps of relative error; inverting a 2 x 2 matrix multiplies that by its condition
    number kappa, so each Gaussian's conic must be within 128 ulps x kappa of the oracle's, relative
    to its largest entry (measured: below 16 ulps x kappa)."""
    cam, sc = make()
    pr = oracle.project(cam, scene64(sc), tight_radius=tight)
    dsc = {k: to_torch(v, DEV) for k, v in sc.items() if isinstance(v, np.ndarray)}
    out = tc.tcgs_project(cam, dsc["means3"], dsc["scales"], dsc["quats"], dsc["sh"], sc["sh_degree"],
                          opacity=dsc["opacity"] if tight else None)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in out.items()}
    vis_o = pr["radius"] > 0
    vis_g = g["radius"] > 0
    # visibility may only differ where the decision is on a rounding edge (radius ceil or tile edge)
    diff = vis_o != vis_g
    assert diff.mean() < 1e-3, (name, diff.sum())
    both = vis_o & vis_g
    # FP32 rounding of fx X / Z + cx: a few ulps of the coordinate (measured at most 1.5e-5 px)
    np.testing.assert_allclose(g["mean2d"][both], pr["mean2d"][both], rtol=2e-6, atol=5e-5)
    np.testing.assert_allclose(g["depth"][both], pr["depth"][both], rtol=1e-6)
    scale = np.abs(pr["conic"][both]).max(axis=1)
    cerr = np.abs(g["conic"][both] - pr["conic"][both]).max(axis=1) / scale
    a, b, c = pr["cov2d"][both].T
    half_gap = np.sqrt(0.25 * (a - c) ** 2 + b * b)
    kappa = (0.5 * (a + c) + half_gap) / (0.5 * (a + c) - half_gap)
    ulps = cerr / (2.0 ** -24 * kappa)
    if name.startswith("wide_field"):
        m = sc["means3"].astype(np.float64)
        lim = 1.3 * np.array([cam["width"] / (2 * cam["fx"]), cam["height"] / (2 * cam["fy"])])
        clamped = ((np.abs(m[:, :2] / m[:, 2:]) > lim).any(axis=1))[both]
        assert clamped.sum() >= 100, clamped.sum()   # the clamp is exercised
    print(f"\n[project] {name}: max rel conic err {cerr.max():.3g} ({ulps.max():.1f} ulps x kappa, kappa <= "
          f"{kappa.max():.1f}), mean2d err {np.abs(g['mean2d'][both] - pr['mean2d'][both]).max():.3g}")
    assert ulps.max() <= 128, ulps.max()
    np.testing.assert_allclose(g["rgb"][both], pr["rgb"][both], atol=2e-6)
    rad_diff = g["radius"][both] != pr["radius"][both]
    assert rad_diff.mean() < 1e-3
    assert (np.abs(g["radius"][both] - pr["radius"][both]) <= 1).all()


def test_tight_radius_render_matches_oracle(tc):
    """Opacity-aware coverage: GPU project -> bin_sort -> TC render against the oracle on the
    same (FP32-rounded) projection, and fewer splats than the 3-sigma square where opacities are low."""
    cam, sc = scenes.precision(P=30_000, width=240, height=120, seed=12)
    dsc = tc.scene_to_device(sc, DEV)
    pr = oracle.project(cam, scene64(sc), tight_radius=True)
    inp = dict(mean2d=f32(pr["mean2d"]), conic=f32(pr["conic"]), depth=f32(pr["depth"]), radius=pr["radius"],
               rgb=f32(pr["rgb"]), opacity=f32(sc["opacity"]))
    b = oracle.bin_sort(cam, inp["mean2d"], inp["radius"], inp["depth"])
    o = oracle.render(cam, b, inp["mean2d"], inp["conic"], inp["opacity"], inp["rgb"])
    g = gpu_inputs(inp, b)
    out = tc.tcgs_render_fwd(cam, tc.render_opts("tc_fp16_split"), g["ranges"], g["ids"], g["mean2d"], g["conic"],
                             g["opacity"], g["rgb"])
    torch.cuda.synchronize()
    img = out["img"].cpu().numpy()
    assert psnr(img, o["img"]) >= 50.0
    assert (np.abs(img - o["img"]).max(axis=0) <= 2e-3).mean() >= 0.999
    # the GPU's own projection bins to the oracle's splat count up to radius rounding edges
    r = tc.Renderer(cam, len(sc["opacity"]), b["n"] + 4096, tight_radius=True, exact_tiles=False)
    r.project(dsc)
    r.bin_sort()
    torch.cuda.synchronize()
    n_gpu = int(r.bins["n_splats"].item())
    assert abs(n_gpu - b["n"]) <= max(20, 1e-3 * b["n"])
    p3 = oracle.project(cam, scene64(sc))
    wide = oracle.bin_sort(cam, f32(p3["mean2d"]), p3["radius"], f32(p3["depth"]))
    print(f"\n[tight radius] splats {b['n']} (3-sigma square: {wide['n']})")


# ------------------------------------------------------------------ binning (bit exact)

@pytest.mark.parametrize("name,make", SMALL + [("diff_crop_320x180", lambda: scenes.differentiation(
    P=20_000, width=320, height=180, seed=13)[:2])])
def test_bin_sort_bit_exact(tc, name, make):
    cam, sc = make()
    pr = oracle.project(cam, scene64(sc))
    inp = dict(mean2d=f32(pr["mean2d"]), radius=pr["radius"], depth=f32(pr["depth"]))
    b = oracle.bin_sort(cam, inp["mean2d"], inp["radius"], inp["depth"])
    m = to_torch(inp["mean2d"], DEV); r = to_torch(inp["radius"].astype(np.int32), DEV)
    d = to_torch(inp["depth"], DEV)
    out = tc.tcgs_bin_sort(cam, m, r, d, capacity=b["n"] + 17)
    torch.cuda.synchronize()
    assert int(out["status"].item()) == 0
    assert int(out["n_splats"].item()) == b["n"]
    np.testing.assert_array_equal(out["ids_sorted"].cpu().numpy()[: b["n"]], b["ids"])
    np.testing.assert_array_equal(out["tile_ranges"].cpu().numpy(), b["ranges"])


SMALL_VIEW_SCENES = [
    ("plain_128", lambda: scenes.plain_forward()),
    ("plain_ragged_200x136", lambda: scenes.plain_forward(P=1500, width=200, height=136, seed=11)),
    ("plain_8192_128x128", lambda: scenes.plain_forward(P=8192, width=128, height=128, seed=16)),
]


@pytest.mark.parametrize("exact", [False, True])
@pytest.mark.parametrize("name,make", SMALL_VIEW_SCENES)
def test_bin_sort_small_view_path_matches_multi_block_path(tc, name, make, exact):
    """A view of at most 256 tiles with P <= 8192 sorts in two single-CTA kernels when the capacity
    is at most 32768, and in the multi-block passes above it: the same N, lists and ranges either
    way (with the row path too, at 32 P), and the oracle's lists for the rectangle coverage."""
    cam, sc = make()
    pr = oracle.project(cam, scene64(sc))
    inp = dict(mean2d=f32(pr["mean2d"]), radius=pr["radius"], depth=f32(pr["depth"]), conic=f32(pr["conic"]))
    P = len(sc["opacity"])
    b = oracle.bin_sort(cam, inp["mean2d"], inp["radius"], inp["depth"])
    m = to_torch(inp["mean2d"], DEV); r = to_torch(inp["radius"].astype(np.int32), DEV)
    d = to_torch(inp["depth"], DEV)
    kw = dict(conic=to_torch(inp["conic"], DEV), opacity=to_torch(sc["opacity"], DEV)) if exact else {}
    caps = [b["n"] + 17] + ([32 * P + 5] if 32 * P + 5 <= 32768 else []) + [40_000]
    assert caps[0] <= 32768 and caps[-1] > 32768
    res = []
    for cap in caps:
        out = tc.tcgs_bin_sort(cam, m, r, d, capacity=cap, **kw)
        torch.cuda.synchronize()
        assert int(out["status"].item()) == 0
        n = int(out["n_splats"].item())
        res.append((n, out["ids_sorted"].cpu().numpy()[:n], out["tile_ranges"].cpu().numpy()))
    for n, ids, ranges in res[1:]:
        assert n == res[0][0]
        np.testing.assert_array_equal(ids, res[0][1])
        np.testing.assert_array_equal(ranges, res[0][2])
    if not exact:
        assert res[0][0] == b["n"]
        np.testing.assert_array_equal(res[0][1], b["ids"])
        np.testing.assert_array_equal(res[0][2], b["ranges"])


# the capacity from which two tile passes run on packed (tile >> 8, id) words (binsort.cu)
PACKED_TILE_SORT_CAPACITY = 1 << 23


@pytest.mark.parametrize("exact", [False, True])
@pytest.mark.parametrize("name,make", [
    ("large_crop_960x540", lambda: scenes.large(P=20_000, width=960, height=540, seed=14)),
    ("precision_crop_1024x512", lambda: scenes.precision(P=100_000, width=1024, height=512, seed=13))])
def test_packed_tile_sort_matches_key_value_passes(tc, name, make, exact):
    """Views of more than 256 tiles sort their splats in two tile passes: as key-value pairs followed by
    a ranges pass below a capacity of 2^23 splats, and from 2^23 on as packed (tile >> 8, id) words
    whose second pass takes the ranges from per-tile counts.  Both give the same N, lists and ranges
    (empty tiles [0, 0)); with the rectangle coverage both equal the oracle's lists."""
    cam, sc = make()
    pr = oracle.project(cam, scene64(sc))
    inp = dict(mean2d=f32(pr["mean2d"]), radius=pr["radius"], depth=f32(pr["depth"]), conic=f32(pr["conic"]))
    b = oracle.bin_sort(cam, inp["mean2d"], inp["radius"], inp["depth"])
    gw, gh = oracle.grid(cam)
    assert gw * gh > 256 and b["n"] + 17 < PACKED_TILE_SORT_CAPACITY
    m = to_torch(inp["mean2d"], DEV); r = to_torch(inp["radius"].astype(np.int32), DEV)
    d = to_torch(inp["depth"], DEV)
    kw = dict(conic=to_torch(inp["conic"], DEV), opacity=to_torch(sc["opacity"], DEV)) if exact else {}
    res = []
    for cap in (b["n"] + 17, PACKED_TILE_SORT_CAPACITY):
        out = tc.tcgs_bin_sort(cam, m, r, d, capacity=cap, **kw)
        torch.cuda.synchronize()
        assert int(out["status"].item()) == 0
        n = int(out["n_splats"].item())
        res.append((n, out["ids_sorted"].cpu().numpy()[:n], out["tile_ranges"].cpu().numpy()))
    assert res[1][0] == res[0][0]
    np.testing.assert_array_equal(res[1][1], res[0][1])
    np.testing.assert_array_equal(res[1][2], res[0][2])
    if not exact:
        assert res[1][0] == b["n"]
        np.testing.assert_array_equal(res[1][1], b["ids"])
        np.testing.assert_array_equal(res[1][2], b["ranges"])


def test_bin_sort_capacity_overflow_reports_status(tc):
    cam, sc = scenes.plain_forward()
    pr = oracle.project(cam, scene64(sc))
    n = int(pr["tiles_touched"].sum())
    m = to_torch(f32(pr["mean2d"]), DEV); r = to_torch(pr["radius"].astype(np.int32), DEV)
    d = to_torch(f32(pr["depth"]), DEV)
    for cap in (n - 1, 1, 0):   # N is still counted (by the duplication's last block) when nothing fits
        out = tc.tcgs_bin_sort(cam, m, r, d, capacity=cap)
        torch.cuda.synchronize()
        assert int(out["status"].item()) == 3 and int(out["n_splats"].item()) == n
        assert (out["tile_ranges"][:, 0] == out["tile_ranges"][:, 1]).all()


def test_bin_sort_empty_and_all_culled(tc):
    cam = scenes.pinhole(40, 24, fx=40.0)
    for P in [0, 5]:
        m = torch.zeros(P, 2, device=DEV); r = torch.zeros(P, dtype=torch.int32, device=DEV)
        d = torch.ones(P, device=DEV)
        out = tc.tcgs_bin_sort(cam, m, r, d, capacity=8)
        torch.cuda.synchronize()
        assert int(out["n_splats"].item()) == 0 and int(out["status"].item()) == 0
        assert (out["tile_ranges"] == 0).all()


def test_bin_sort_depth_ties_and_huge_gaussian(tc):
    cam = scenes.pinhole(100, 70, fx=100.0)
    rng = np.random.default_rng(3)
    P = 400
    mean2d = f32(np.c_[rng.uniform(-30, 130, P), rng.uniform(-30, 100, P)])
    radius = rng.integers(0, 40, P).astype(np.int32)
    radius[7] = 100000         # covers every tile
    mean2d[9] = [-1e9, 5.0]    # far off-screen
    depth = f32(rng.choice([1.0, 2.0, 3.0], P))   # many exact ties
    b = oracle.bin_sort(cam, mean2d, radius, depth)
    out = tc.tcgs_bin_sort(cam, to_torch(mean2d, DEV), to_torch(radius, DEV), to_torch(depth, DEV), capacity=b["n"])
    torch.cuda.synchronize()
    assert int(out["n_splats"].item()) == b["n"]
    np.testing.assert_array_equal(out["ids_sorted"].cpu().numpy()[: b["n"]], b["ids"])
    np.testing.assert_array_equal(out["tile_ranges"].cpu().numpy(), b["ranges"])


@pytest.mark.parametrize("depths", ["distinct", "short_ties", "three_levels", "all_equal"])
def test_bin_sort_long_lists(tc, depths):
    """Tiles with lists far longer than the shared-memory sort (thousands of splats per tile), so
    each tile's depth sort runs in chunked passes through global memory; depth ties from none to
    every splat of a tile being equal."""
    cam = scenes.pinhole(100, 70, fx=100.0)
    rng = np.random.default_rng(17)
    P = 20_000
    mean2d = f32(np.c_[rng.uniform(-10, 110, P), rng.uniform(-10, 80, P)])
    radius = rng.integers(0, 48, P).astype(np.int32)
    depth = f32(rng.uniform(0.5, 40.0, P))
    if depths == "short_ties":
        depth[::5] = depth[1::5]
    elif depths == "three_levels":
        depth = f32(rng.choice([1.0, 2.0, 3.0], P))
    elif depths == "all_equal":
        depth = np.full(P, 4.0, np.float32)
    b = oracle.bin_sort(cam, mean2d, radius, depth)
    lens = np.diff(b["ranges"], axis=1).ravel()
    assert lens.min() > 2048 and lens.max() > 3 * 2048
    out = tc.tcgs_bin_sort(cam, to_torch(mean2d, DEV), to_torch(radius, DEV), to_torch(depth, DEV), capacity=b["n"])
    torch.cuda.synchronize()
    assert int(out["status"].item()) == 0 and int(out["n_splats"].item()) == b["n"]
    np.testing.assert_array_equal(out["ids_sorted"].cpu().numpy()[: b["n"]], b["ids"])
    np.testing.assert_array_equal(out["tile_ranges"].cpu().numpy(), b["ranges"])


def _borderline(cam, inp, g, t, rel=1e-4, absol=2e-3):
    """Splat (g, t) whose exact-coverage decision sits within FP32 rounding of the limit."""
    gw, _ = oracle.grid(cam)
    tx, ty = t % gw, t // gw
    m = inp["mean2d"][g].astype(np.float64)
    s11, s12, s22 = inp["conic"][g].astype(np.float64)
    o = float(inp["opacity"][g])
    qmin = oracle.box_min_q(m[0], m[1], s11, s12, s22, 16 * tx + 0.5, 16 * tx + 15.5, 16 * ty + 0.5, 16 * ty + 15.5)
    lim = 2 * (math.log(o) + math.log(255.0)) * 1.0001 + 1e-3
    return abs(qmin - lim) <= rel * (abs(lim) + qmin) + absol


EXACT_SCENES = SMALL + [("diff_crop_320x180", lambda: scenes.differentiation(P=20_000, width=320, height=180,
                                                                              seed=13)[:2]),
                        ("large_crop_960x540", lambda: scenes.large(P=20_000, width=960, height=540, seed=14))]


def _capacity(n_rect, P, rows):
    """A capacity of at least 32 splats per Gaussian selects the row path of exact coverage."""
    return max(n_rect + 5, 32 * P + 5) if rows else n_rect + 5


@pytest.mark.parametrize("rows", [False, True])
@pytest.mark.parametrize("name,make", EXACT_SCENES)
def test_bin_sort_exact_matches_oracle(tc, name, make, rows):
    """Exact tile coverage, tile by tile or (rows) by rows for the wide Gaussians: per tile, the GPU
    list equals the oracle's on the same FP32 inputs except for splats whose decision lies within
    FP32 rounding of the limit (each checked, and rare)."""
    cam, sc = make()
    _, inp, b_rect, _ = oracle_frame(cam, sc, render=False)
    b = oracle.bin_sort(cam, inp["mean2d"], inp["radius"], inp["depth"], conic=inp["conic"],
                        opacity=inp["opacity"])
    g = gpu_inputs(inp, b)
    out = tc.tcgs_bin_sort(cam, g["mean2d"], g["radius"], g["depth"],
                           capacity=_capacity(b_rect["n"], len(inp["opacity"]), rows), conic=g["conic"],
                           opacity=g["opacity"])
    torch.cuda.synchronize()
    assert int(out["status"].item()) == 0
    n = int(out["n_splats"].item())
    ids, ranges = out["ids_sorted"].cpu().numpy()[:n], out["tile_ranges"].cpu().numpy()
    mism = 0
    for t, ((s0, e0), (s1, e1)) in enumerate(zip(b["ranges"], ranges)):
        lo, lg = list(b["ids"][s0:e0]), list(ids[s1:e1])
        if lo == lg:
            continue
        diff = set(lo) ^ set(lg)
        mism += len(diff)
        assert all(_borderline(cam, inp, gg, t) for gg in diff), (name, t, diff)
        keep = lambda l: [x for x in l if x not in diff]
        assert keep(lo) == keep(lg), (name, t)
    print(f"\n[exact bins] {name} rows={rows}: {n} splats (3-sigma: {b_rect['n']}), {mism} borderline differences")
    assert mism <= max(2, 1e-4 * b["n"])
    assert n < b_rect["n"]


@pytest.mark.parametrize("precision", ["tc_fp16_split", "fp32"])
def test_exact_tiles_render_the_same_image(tc, precision):
    """Rendering from the exact lists gives the image and final transmittance of the 3-sigma lists
    bit for bit (the dropped splats are culled at every pixel by the renderers' own arithmetic);
    n_contrib names the same last blended Gaussian."""
    cam, sc = scenes.precision(P=30_000, width=240, height=120, seed=12)
    dsc = {k: to_torch(v, DEV) if isinstance(v, np.ndarray) else v for k, v in sc.items()}
    pr_g = tc.tcgs_project(cam, dsc["means3"], dsc["scales"], dsc["quats"], dsc["sh"], sc["sh_degree"])
    cap = int(pr_g["tiles_touched"].to(torch.int64).sum().item()) + 1
    res = {}
    for exact in (False, True):
        b = tc.tcgs_bin_sort(cam, pr_g["mean2d"], pr_g["radius"], pr_g["depth"], cap,
                             conic=pr_g["conic"] if exact else None, opacity=dsc["opacity"] if exact else None)
        o = tc.tcgs_render_fwd(cam, tc.render_opts(precision), b["tile_ranges"], b["ids_sorted"], pr_g["mean2d"],
                               pr_g["conic"], dsc["opacity"], pr_g["rgb"])
        torch.cuda.synchronize()
        n = int(b["n_splats"].item())
        res[exact] = dict(img=o["img"].cpu().numpy(), T=o["T_final"].cpu().numpy(),
                          nc=o["n_contrib"].cpu().numpy(), ids=b["ids_sorted"].cpu().numpy()[:n],
                          ranges=b["tile_ranges"].cpu().numpy(), n=n)
    r, e = res[False], res[True]
    assert e["n"] < r["n"]
    np.testing.assert_array_equal(r["img"], e["img"])
    np.testing.assert_array_equal(r["T"], e["T"])
    gw, _ = oracle.grid(cam)
    H, W = r["T"].shape
    ys, xs = np.nonzero(r["nc"] > 0)
    assert ((r["nc"] > 0) == (e["nc"] > 0)).all()
    t = (ys // 16) * gw + xs // 16
    last_r = r["ids"][r["ranges"][t, 0] + r["nc"][ys, xs] - 1]
    last_e = e["ids"][e["ranges"][t, 0] + e["nc"][ys, xs] - 1]
    np.testing.assert_array_equal(last_r, last_e)
    print(f"\n[exact tiles] {precision}: splats {r['n']} -> {e['n']}")


@pytest.mark.parametrize("rows", [False, True])
def test_bin_sort_exact_long_lists_and_ties(tc, rows):
    """Exact coverage on tiles with thousands of candidate splats and exact depth ties, tile by tile
    or by rows for the wide Gaussians."""
    cam = scenes.pinhole(100, 70, fx=100.0)
    rng = np.random.default_rng(23)
    P = 20_000
    mean2d = f32(np.c_[rng.uniform(-10, 110, P), rng.uniform(-10, 80, P)])
    radius = rng.integers(1, 48, P).astype(np.int32)
    A = rng.standard_normal((P, 2, 2)) * (radius[:, None, None] / 3.0)
    cov = A @ A.transpose(0, 2, 1) + 0.3 * np.eye(2)
    inv = np.linalg.inv(cov)
    conic = f32(np.c_[inv[:, 0, 0], inv[:, 0, 1], inv[:, 1, 1]])
    opacity = f32(rng.uniform(0.002, 1.0, P))
    depth = f32(rng.choice([1.0, 2.0, 3.0, 4.0], P))
    inp = dict(mean2d=mean2d, conic=conic, opacity=opacity)
    b = oracle.bin_sort(cam, mean2d, radius, depth, conic=conic, opacity=opacity)
    out = tc.tcgs_bin_sort(cam, to_torch(mean2d, DEV), to_torch(radius, DEV), to_torch(depth, DEV),
                           capacity=max(b["n"] + 64, 32 * P + 64) if rows else b["n"] + 64,
                           conic=to_torch(conic, DEV), opacity=to_torch(opacity, DEV))
    torch.cuda.synchronize()
    n = int(out["n_splats"].item())
    ids, ranges = out["ids_sorted"].cpu().numpy()[:n], out["tile_ranges"].cpu().numpy()
    assert np.diff(b["ranges"], axis=1).max() > 2048
    for t, ((s0, e0), (s1, e1)) in enumerate(zip(b["ranges"], ranges)):
        lo, lg = list(b["ids"][s0:e0]), list(ids[s1:e1])
        if lo != lg:
            diff = set(lo) ^ set(lg)
            assert all(_borderline(cam, inp, gg, t) for gg in diff), (t, diff)
            assert [x for x in lo if x not in diff] == [x for x in lg if x not in diff]


@pytest.mark.parametrize("name,make", EXACT_SCENES[-2:])
def test_bin_sort_exact_rows_equal_tiles(tc, name, make):
    """The row path of exact coverage (wide Gaussians: each row's reached tiles from the ellipse's
    shadow, the end tiles settled by the per-tile test) makes the lists of the tile-by-tile path."""
    cam, sc = make()
    dsc = {k: to_torch(v, DEV) if isinstance(v, np.ndarray) else v for k, v in sc.items()}
    pr = tc.tcgs_project(cam, dsc["means3"], dsc["scales"], dsc["quats"], dsc["sh"], sc["sh_degree"])
    n_rect = int(pr["tiles_touched"].to(torch.int64).sum().item())
    P = len(sc["opacity"])
    res = []
    for rows in (False, True):
        b = tc.tcgs_bin_sort(cam, pr["mean2d"], pr["radius"], pr["depth"], _capacity(n_rect, P, rows),
                             conic=pr["conic"], opacity=dsc["opacity"])
        torch.cuda.synchronize()
        n = int(b["n_splats"].item())
        res.append((n, b["ids_sorted"][:n].cpu().numpy(), b["tile_ranges"].cpu().numpy()))
    assert res[0][0] == res[1][0] and res[0][0] > 0
    np.testing.assert_array_equal(res[0][1], res[1][1])
    np.testing.assert_array_equal(res[0][2], res[1][2])
    print(f"\n[rows = tiles] {name}: {res[0][0]} splats of {n_rect} rectangle tiles")


def test_frame_pipeline_matches_direct_frames(tc):
    """FramePipeline (scene uploaded from pinned host memory while the previous frame renders, image
    returned to the host) gives every frame's image bit for bit as a direct frame of that scene."""
    cam, sc = scenes.plain_forward(P=1500, width=200, height=136, seed=11)
    P = len(sc["opacity"])
    cap = 4 * int(oracle.project(cam, scene64(sc))["tiles_touched"].sum()) + 64
    variants = []
    for i, f in enumerate((1.0, 0.4, 0.8, 0.25, 1.0)):
        s2 = dict(sc, opacity=(np.asarray(sc["opacity"]) * f).astype(np.float32))
        if i % 2:   # arrays in one pinned buffer: one copy a frame
            v = tc.FramePipeline.pinned_scene(s2)
        else:       # separate pinned arrays: a copy per array
            v = {k: (torch.from_numpy(np.ascontiguousarray(x)).pin_memory() if isinstance(x, np.ndarray) else x)
                 for k, x in s2.items()}
        variants.append(v)
    r = tc.Renderer(cam, P, cap, device=DEV)
    pipe = tc.FramePipeline(r)
    host = [torch.empty(3, cam["height"], cam["width"]).pin_memory() for _ in variants]
    for v, h in zip(variants, host):
        pipe.submit(v, h)
    pipe.synchronize()
    r2 = tc.Renderer(cam, P, cap, device=DEV)
    for v, h in zip(variants, host):
        d = {k: (x.to(DEV) if isinstance(x, torch.Tensor) else x) for k, x in v.items() if k != "_buffer"}
        out = r2.frame(d)
        torch.cuda.synchronize()
        assert torch.equal(out["img"].cpu(), h)
    assert not torch.equal(host[0], host[1])


PERSISTENT_SCENES = SMALL[1:] + [
    ("precision_crop_640x400", lambda: scenes.precision(P=40_000, width=640, height=400, seed=15)),
    ("large_crop_960x540", lambda: scenes.large(P=20_000, width=960, height=540, seed=14)),
]


@pytest.mark.parametrize("name,make", PERSISTENT_SCENES)
def test_persistent_render_matches_one_cta_per_tile(tc, name, make):
    """With a tile order (tcgs_tile_order), the TC renderer gives the image, T and n_contrib of one
    CTA per tile bit for bit, for every tile-local encoding.  Views of more tiles than one wave of CTAs
    (tcgs_tc_wave_tiles) run the persistent grid, which pops the work counter; smaller views run one
    CTA per tile and leave the counter alone.  The order is a permutation of the tiles with
    non-increasing list-length groups."""
    cam, sc = make()
    dsc = {k: to_torch(v, DEV) if isinstance(v, np.ndarray) else v for k, v in sc.items()}
    P = len(sc["opacity"])
    cap = int(oracle.project(cam, scene64(sc))["tiles_touched"].sum()) + 64
    wave = tc.tcgs_tc_wave_tiles()
    assert wave == 4 * torch.cuda.get_device_properties(0).multi_processor_count
    r = tc.Renderer(cam, P, cap, device=DEV, persistent=False)
    r.project(dsc)
    r.bin_sort()
    torch.cuda.synchronize()
    n_tiles = r.num_tiles
    order = tc.tcgs_tile_order(r.cam, r.bins["tile_ranges"])
    sentinel = 0x5A5A5A5A
    counter = torch.full((1,), sentinel, dtype=torch.int32, device=DEV)
    for prec in ("tc_fp16_split", "tc_fp16", "tc_tf32", "tc_fp8", "fp32_frag2mat"):
        a = {k: v.clone() for k, v in r.render(dsc["opacity"], prec).items()}
        counter.fill_(sentinel)
        opts = tc.render_opts(prec, tile_order=order, work_counter=counter)
        b = tc.tcgs_render_fwd(r.cam, opts, r.bins["tile_ranges"], r.bins["ids_sorted"], r.proj["mean2d"],
                               r.proj["conic"], dsc["opacity"], r.proj["rgb"])
        torch.cuda.synchronize()
        for k in ("img", "T_final", "n_contrib"):
            assert torch.equal(a[k], b[k]), (prec, k)
        popped = int(counter.item()) != sentinel
        assert popped == (n_tiles > wave), (prec, n_tiles, wave)
        if n_tiles > wave:   # every tile popped once, plus one failed pop per CTA
            assert int(counter.item()) == n_tiles + wave
    rp = tc.Renderer(cam, P, cap, device=DEV)   # the default Renderer picks the same path itself
    rp.project(dsc)
    rp.bin_sort()
    o = rp.render(dsc["opacity"], "tc_fp16_split")
    torch.cuda.synchronize()
    assert torch.equal(o["img"], r.render(dsc["opacity"], "tc_fp16_split")["img"])
    order = order.cpu().numpy()
    lens = np.diff(r.bins["tile_ranges"].cpu().numpy(), axis=1).ravel().astype(np.int64)
    np.testing.assert_array_equal(np.sort(order), np.arange(len(lens)))
    groups = np.where(lens[order] > 0, np.floor(np.log2(np.maximum(lens[order], 1))) + 1, 0)
    assert (np.diff(groups) <= 0).all()
    same = np.diff(groups) == 0
    assert (np.diff(order)[same] > 0).all()   # tile order inside a group


@pytest.mark.parametrize("name,make", [
    ("diff_crop_320x180", lambda: scenes.differentiation(P=20_000, width=320, height=180, seed=13)[:2]),
    ("plain_ragged_200x134", lambda: scenes.plain_forward(P=1500, width=200, height=134, seed=11)),
    ("large_crop_960x540", lambda: scenes.large(P=20_000, width=960, height=540, seed=14))])
def test_two_pixels_a_thread_render_the_same_image(tc, name, make):
    """The renderer instance with two pixels a consumer thread (8 x 8 warp blocks, one pixel in each
    MMA half) gives the image, T and n_contrib of the one-pixel instance bit for bit, with the tensor-
    core and the CUDA-core product, one CTA per tile and persistent, and the same blended and evaluated
    fragment counts (only the executed slots differ: coarser block marks).  The ragged view's last
    tile row is 6 pixels high, so some threads have only their first pixel inside the image."""
    cam, sc = make()
    dsc = {k: to_torch(v, DEV) if isinstance(v, np.ndarray) else v for k, v in sc.items()}
    P = len(sc["opacity"])
    cap = int(oracle.project(cam, scene64(sc))["tiles_touched"].sum()) + 64
    r = tc.Renderer(cam, P, cap, device=DEV, stats=True, persistent=False, pixels_per_thread=1)
    r.project(dsc)
    r.bin_sort()
    torch.cuda.synchronize()
    order = tc.tcgs_tile_order(r.cam, r.bins["tile_ranges"])
    counter = torch.zeros(1, dtype=torch.int32, device=DEV)
    for prec in ("tc_fp16_split", "fp32_frag2mat"):
        res = {}
        for ppt in (1, 2):
            for persistent in (False, True):
                r.stats.zero_()
                opts = tc.render_opts(prec, tile_stats=r.stats, pixels_per_thread=ppt,
                                      tile_order=order if persistent else None,
                                      work_counter=counter if persistent else None)
                o = tc.tcgs_render_fwd(r.cam, opts, r.bins["tile_ranges"], r.bins["ids_sorted"], r.proj["mean2d"],
                                       r.proj["conic"], dsc["opacity"], r.proj["rgb"])
                torch.cuda.synchronize()
                res[(ppt, persistent)] = ({k: v.clone() for k, v in o.items()}, r.stats.clone())
        base_img, base_st = res[(1, False)]
        assert base_img["n_contrib"].max() > 0
        for key, (img, st) in res.items():
            for k in ("img", "T_final", "n_contrib"):
                assert torch.equal(img[k], base_img[k]), (name, prec, key, k)
            assert torch.equal(st[:, :2], base_st[:, :2]), (name, prec, key)   # blended, evaluated
            assert torch.equal(st[:, 3], base_st[:, 3]), (name, prec, key)     # list lengths
    assert tc.Renderer(cam, P, 16 * P, device=DEV).pixels_per_thread == 2
    assert tc.Renderer(cam, P, 16 * P - 1, device=DEV).pixels_per_thread == 1


@pytest.mark.parametrize("width,height", [(40, 24), (1920, 1080), (4160, 2176)])
def test_tile_order_is_the_stable_longest_first_sort(tc, width, height):
    """tcgs_tile_order on synthetic list lengths spanning every length group (empty lists up to
    2^32 - 1 entries), on grids from 6 tiles to one past the kernel's shared-memory cache of 32768
    tiles: the order is the stable sort of the tiles by descending floor(log2(length)) + 1."""
    cam = scenes.pinhole(width, height, 1000.0)
    nt = ((width + 15) // 16) * ((height + 15) // 16)
    rng = np.random.default_rng(nt)
    g = rng.integers(0, 33, nt)
    lo = np.where(g > 0, np.left_shift(np.ones(nt, np.uint64), np.maximum(g, 1).astype(np.uint64) - 1), 0)
    lens = lo + (rng.random(nt) * lo).astype(np.uint64)          # inside [2^(g-1), 2^g)
    starts = rng.integers(0, 2**32, nt, dtype=np.uint64)
    ranges = np.stack([starts, (starts + lens) % 2**32], axis=1).astype(np.uint32)
    out = tc.tcgs_tile_order(cam, torch.from_numpy(ranges.view(np.int32)).to(DEV))
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint32)
    lens32 = (ranges[:, 1] - ranges[:, 0]).astype(np.int64)
    assert (lens32 == lens.astype(np.int64)).all()
    groups = np.where(lens32 > 0, np.floor(np.log2(np.maximum(lens32, 1))).astype(np.int64) + 1, 0)
    np.testing.assert_array_equal(groups, g)
    np.testing.assert_array_equal(got, np.argsort(-groups, kind="stable"))


def test_bounded_wait_reports_timeout_and_context_stays_usable(tc):
    """A device-side wait that nothing ends gives up after its poll limit and reports
    TCGS_ERR_TIMEOUT in the status word; the next launches run normally."""
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    for polls in (1, 4096):
        status.zero_()
        tc.tcgs_selftest_bounded_wait(status, polls)
        torch.cuda.synchronize()
        assert int(status.item()) == 4   # TCGS_ERR_TIMEOUT
    cam, sc = SMALL[0][1]()
    _, inp, b, o = oracle_frame(cam, sc)
    g = gpu_inputs(inp, b)
    out = tc.tcgs_render_fwd(cam, tc.render_opts("tc_fp16_split", device_status=status.zero_()), g["ranges"],
                             g["ids"], g["mean2d"], g["conic"], g["opacity"], g["rgb"])
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert psnr(out["img"].cpu().numpy(), o["img"]) > 50


def _tile_mask(cam, tiles):
    H, W = cam["height"], cam["width"]
    gw, _ = oracle.grid(cam)
    m = np.zeros((H, W), bool)
    for t in tiles:
        tx, ty = t % gw, t // gw
        m[16 * ty:16 * ty + 16, 16 * tx:16 * tx + 16] = True
    return m


def test_full_size_frame_matches_oracle_on_sampled_tiles(tc):
    """The bench's workload (1920x1080, 1M Gaussians, SH3) in the bench's launch configuration (exact
    tile coverage, persistent TC renderer in longest-list order), checked on 96 random tiles the
    oracle renders one by one.  (1) On the oracle's FP32-rounded projection: the tile lists match the
    oracle's (up to splats within FP32 rounding of the coverage limit), the FP32 renderer within 1e-5
    away from cull and termination margins, the TC renderer at PSNR >= 50 dB with >= 99.9% of pixels
    within 2e-3.  (2) The whole GPU frame from the scene (GPU projection) against the FP64 oracle
    frame: the TC criteria again."""
    cam, sc = scenes.precision()
    P = len(sc["opacity"])
    pr, inp, b_rect, _ = oracle_frame(cam, sc, render=False)
    b = oracle.bin_sort(cam, inp["mean2d"], inp["radius"], inp["depth"], conic=inp["conic"], opacity=inp["opacity"])
    gw, gh = oracle.grid(cam)
    tiles = np.sort(np.random.default_rng(7).choice(gw * gh, 96, replace=False)).astype(np.int32)
    o = oracle.render(cam, b, inp["mean2d"], inp["conic"], inp["opacity"], inp["rgb"], tiles=tiles)
    mask = _tile_mask(cam, tiles)

    # (1) binning and both renderers on the oracle's FP32 inputs
    g = gpu_inputs(inp, b)
    out_b = tc.tcgs_bin_sort(cam, g["mean2d"], g["radius"], g["depth"], capacity=b_rect["n"] + 1024,
                             conic=g["conic"], opacity=g["opacity"])
    torch.cuda.synchronize()
    assert int(out_b["status"].item()) == 0
    n = int(out_b["n_splats"].item())
    ids, ranges = out_b["ids_sorted"].cpu().numpy()[:n], out_b["tile_ranges"].cpu().numpy()
    mism = 0
    for t in tiles:
        (s0, e0), (s1, e1) = b["ranges"][t], ranges[t]
        lo, lg = list(b["ids"][s0:e0]), list(ids[s1:e1])
        if lo != lg:
            diff = set(lo) ^ set(lg)
            mism += len(diff)
            assert all(_borderline(cam, inp, gg, int(t)) for gg in diff), (t, diff)
            assert [x for x in lo if x not in diff] == [x for x in lg if x not in diff]
    assert abs(n - b["n"]) <= max(16, 1e-5 * b["n"])
    order = tc.tcgs_tile_order(cam, out_b["tile_ranges"])
    counter = torch.zeros(1, dtype=torch.int32, device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    imgs = {}
    for prec in ("fp32", "tc_fp16_split", "tc_fp16", "fp32_frag2mat"):
        opts = tc.render_opts(prec, device_status=status,
                              tile_order=order if prec != "fp32" else None,
                              work_counter=counter if prec != "fp32" else None)
        out = tc.tcgs_render_fwd(cam, opts, out_b["tile_ranges"], out_b["ids_sorted"], g["mean2d"], g["conic"],
                                 g["opacity"], g["rgb"])
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        imgs[prec] = (out["img"].cpu().numpy(), out["T_final"].cpu().numpy())
    img32, T32 = imgs["fp32"]
    keep = mask & ~margin_mask(o, 1e-4, 1e-4)
    assert keep.sum() > 0.99 * mask.sum()
    assert np.abs(img32 - o["img"]).max(axis=0)[keep].max() <= 1e-5
    assert np.abs(T32 - o["T"])[keep].max() <= 1e-5
    imgtc = imgs["tc_fp16_split"][0]
    assert psnr(imgtc[:, mask], o["img"][:, mask]) >= 50.0
    assert (np.abs(imgtc - o["img"]).max(axis=0)[mask] <= 2e-3).mean() >= 0.999
    # the paper's K = 8 layout (v0 / 3 in three FP16 slots, Sec. 5.1) is recorded, not held to the TC bar:
    # about 55 dB, but only about 86% of pixels within 2e-3 on this frame, so it fails the 99.9% criterion
    # (its exponent error reaches ~0.1 where |v0| is large; the split layout is the shipped default)
    img16 = imgs["tc_fp16"][0]
    p16 = psnr(img16[:, mask], o["img"][:, mask])
    w16 = float((np.abs(img16 - o["img"]).max(axis=0)[mask] <= 2e-3).mean())
    assert 50.0 <= p16 <= 60.0 and 0.75 <= w16 <= 0.95, (p16, w16)
    # the same kernel with the product on CUDA cores: the TC criteria, and within 1e-4 off the margins
    imgcc = imgs["fp32_frag2mat"][0]
    assert psnr(imgcc[:, mask], o["img"][:, mask]) >= 50.0
    assert np.abs(imgcc - o["img"]).max(axis=0)[keep].max() <= 1e-4

    # (2) the whole frame from the scene, as the bench renders it
    d = tc.scene_to_device(sc, DEV)
    r = tc.Renderer(cam, P, b_rect["n"] + 1024, device=DEV)
    img = r.frame(d)["img"].cpu().numpy()
    o64 = oracle.render(cam, oracle.bin_sort(cam, pr["mean2d"], pr["radius"], pr["depth"], conic=pr["conic"],
                                             opacity=scene64(sc)["opacity"]),
                        pr["mean2d"], pr["conic"], scene64(sc)["opacity"], pr["rgb"], tiles=tiles, margins=False)
    assert psnr(img[:, mask], o64["img"][:, mask]) >= 50.0
    assert (np.abs(img - o64["img"]).max(axis=0)[mask] <= 2e-3).mean() >= 0.999
    print(f"\n[full size] {n} splats, {mism} borderline list differences on {len(tiles)} tiles, "
          f"TC PSNR {psnr(imgtc[:, mask], o['img'][:, mask]):.1f} dB (FP32 inputs), paper K = 8 layout {p16:.1f} dB "
          f"with {100 * w16:.1f}% within 2e-3, "
          f"{psnr(img[:, mask], o64['img'][:, mask]):.1f} dB (whole frame)")


def test_ex2_microbenchmark_runs_its_chains(tc):
    """tcgs_microbench_ex2: every thread's 8 chains x <- -2^x settle at the fixed point of
    x = -2^x (about -0.6412), so each checksum is about 8 times it."""
    out = torch.full((2 * 256,), float("nan"), device=DEV)
    n = tc.tcgs_microbench_ex2(out, 2, 64)
    torch.cuda.synchronize()
    assert n == 2 * 256 * 8 * 64
    v = out.cpu().numpy()
    x = -0.5
    for _ in range(200):
        x = -2.0 ** x
    np.testing.assert_allclose(v, 8 * x, rtol=1e-4)


# ------------------------------------------------------------------ alpha blending

def margin_mask(o, cull_tol, term_tol):
    return (o["cull_margin"] < cull_tol) | (o["term_margin"] < term_tol)


@pytest.mark.parametrize("name,make", SMALL)
@pytest.mark.parametrize("alpha_max,bg", [(0.99, (0, 0, 0)), (1.0, (0.25, 0.5, 0.75))])
def test_render_fp32_matches_oracle(tc, name, make, alpha_max, bg):
    cam, sc = make()
    _, inp, b, o = oracle_frame(cam, sc, alpha_max=alpha_max, bg=bg)
    g = gpu_inputs(inp, b)
    stats = torch.zeros(b["ranges"].shape[0], 8, dtype=torch.int32, device=DEV)
    out = tc.tcgs_render_fwd(cam, tc.render_opts("fp32", alpha_max, tile_stats=stats), g["ranges"], g["ids"],
                             g["mean2d"], g["conic"], g["opacity"], g["rgb"], bg=bg)
    torch.cuda.synchronize()
    img, T, nc = (out[k].cpu().numpy() for k in ("img", "T_final", "n_contrib"))
    excl = margin_mask(o, 1e-4, 1e-4)
    assert excl.mean() < 1e-3
    keep = ~excl
    err = np.abs(img - o["img"]).max(axis=0)
    assert err[keep].max() <= 1e-5, err[keep].max()
    assert np.abs(T - o["T"])[keep].max() <= 1e-5
    assert (nc[keep] == o["n_contrib"][keep]).all()
    s = stats.cpu().numpy().astype(np.int64)
    # fragment classes agree with the oracle's counts up to margin pixels
    assert abs(s[:, 0].sum() - o["f_blend"]) <= max(10, 1e-4 * o["f_blend"])
    assert abs(s[:, 0].sum() + s[:, 1].sum() - o["alpha_evals"]) <= max(10, 1e-3 * o["alpha_evals"])
    np.testing.assert_array_equal(s[:, 3], b["ranges"][:, 1] - b["ranges"][:, 0])


@pytest.mark.parametrize("name,make", SMALL)
def test_render_fp32_early_cull_same_image(tc, name, make):
    cam, sc = make()
    _, inp, b, o = oracle_frame(cam, sc)
    g = gpu_inputs(inp, b)
    a = tc.tcgs_render_fwd(cam, tc.render_opts("fp32", early_cull=False), g["ranges"], g["ids"], g["mean2d"],
                           g["conic"], g["opacity"], g["rgb"])["img"]
    c = tc.tcgs_render_fwd(cam, tc.render_opts("fp32", early_cull=True), g["ranges"], g["ids"], g["mean2d"],
                           g["conic"], g["opacity"], g["rgb"])["img"]
    torch.cuda.synchronize()
    diff = (a - c).abs().amax(dim=0).cpu().numpy()
    assert (diff > 1e-6).mean() < 1e-3   # only cull-margin fragments can differ


@pytest.mark.parametrize("name,make", SMALL)
@pytest.mark.parametrize("alpha_max", [0.99, 1.0])
def test_render_tc_split_matches_oracle(tc, name, make, alpha_max):
    cam, sc = make()
    _, inp, b, o = oracle_frame(cam, sc, alpha_max=alpha_max)
    g = gpu_inputs(inp, b)
    stats = torch.zeros(b["ranges"].shape[0], 8, dtype=torch.int32, device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    out = tc.tcgs_render_fwd(cam, tc.render_opts("tc_fp16_split", alpha_max, tile_stats=stats, device_status=status),
                             g["ranges"], g["ids"], g["mean2d"], g["conic"], g["opacity"], g["rgb"])
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    img = out["img"].cpu().numpy()
    err = np.abs(img - o["img"]).max(axis=0)
    p = psnr(img, o["img"])
    within = (err <= 2e-3).mean()
    assert p >= 50.0, p
    assert within >= 0.999, within
    s = stats.cpu().numpy().astype(np.int64)
    assert abs(s[:, 0].sum() - o["f_blend"]) <= max(20, 1e-3 * o["f_blend"])
    np.testing.assert_array_equal(s[:, 3], b["ranges"][:, 1] - b["ranges"][:, 0])


@pytest.mark.parametrize("name,make", SMALL)
@pytest.mark.parametrize("alpha_max", [0.99, 1.0])
def test_render_fp32_frag2mat_matches_oracle(tc, name, make, alpha_max):
    """TCGS_FP32_FRAG2MAT, the tensor-core renderer with its product u^T v on CUDA cores in FP32 (the
    ablation arm that differs from the TC path only in the product).  Its exponent carries FP32
    rounding of the tile-local coefficients, a few ulps of sum |u_i v_i|, below the split encoding's
    error, so it meets the TC criteria (PSNR >= 50 dB, >= 99.9% of pixels within 2e-3) and, away
    from margin pixels, max |RGB| <= 1e-4 (recorded: about 1e-6); block marks change nothing."""
    cam, sc = make()
    _, inp, b, o = oracle_frame(cam, sc, alpha_max=alpha_max)
    g = gpu_inputs(inp, b)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    imgs = []
    for cull in (True, False):
        out = tc.tcgs_render_fwd(cam, tc.render_opts("fp32_frag2mat", alpha_max, device_status=status, tile_cull=cull),
                                 g["ranges"], g["ids"], g["mean2d"], g["conic"], g["opacity"], g["rgb"])
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        imgs.append({k: v.cpu().numpy() for k, v in out.items()})
    for k in ("img", "T_final", "n_contrib"):
        np.testing.assert_array_equal(imgs[0][k], imgs[1][k])
    img = imgs[0]["img"]
    err = np.abs(img - o["img"]).max(axis=0)
    keep = ~margin_mask(o, 1e-4, 1e-4)
    print(f"\n[fp32_frag2mat] {name} alpha_max={alpha_max}: PSNR {psnr(img, o['img']):.1f} dB, max abs outside "
          f"margins {err[keep].max():.2e}")
    assert psnr(img, o["img"]) >= 50.0
    assert (err <= 2e-3).mean() >= 0.999
    assert err[keep].max() <= 1e-4


# Measured accuracy of the encodings that do not meet the TC criteria (PSNR >= 50 dB and >= 99.9% of
# pixels within 2e-3 of the FP64 oracle): (PSNR dB, fraction of pixels within 2e-3) per workload.  The
# paper's K = 8 layout (v0 / 3 in three FP16 slots, Sec. 5.1) and TF32 carry about 11 bits of v, so the
# exponents of Gaussians far from the tile centre (|v0| up to ~300) are off by up to ~0.1 and the
# precision crop (small splats, long lists) falls below even 50 dB; the FP8 split keeps ~16 bits.
RECORDED_ENCODINGS = {
    ("tc_fp16", "plain_128"): (62.2, 0.949), ("tc_fp16", "plain_ragged_200x136"): (66.1, 0.983),
    ("tc_fp16", "precision_crop_240x120"): (45.4, 0.568),
    ("tc_tf32", "plain_128"): (62.4, 0.956), ("tc_tf32", "plain_ragged_200x136"): (66.8, 0.983),
    ("tc_tf32", "precision_crop_240x120"): (45.4, 0.567),
    ("tc_fp8", "plain_128"): (77.3, 0.9996), ("tc_fp8", "plain_ragged_200x136"): (77.3, 0.9998),
    ("tc_fp8", "precision_crop_240x120"): (67.2, 0.981),
}


@pytest.mark.parametrize("name,make", SMALL)
@pytest.mark.parametrize("precision", ["tc_fp16", "tc_tf32", "tc_fp8"])
def test_render_tc_other_encodings_recorded_error(tc, name, make, precision):
    """The paper's K = 8 layout, TF32 and the FP8 split, against the FP64 oracle: their measured
    accuracy (RECORDED_ENCODINGS) is reproduced to within 1 dB and 1% of pixels, and each falls short
    of the TC criteria on the precision crop (the split FP16 layout, the default, meets them)."""
    cam, sc = make()
    _, inp, b, o = oracle_frame(cam, sc)
    g = gpu_inputs(inp, b)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    out = tc.tcgs_render_fwd(cam, tc.render_opts(precision, device_status=status), g["ranges"], g["ids"],
                             g["mean2d"], g["conic"], g["opacity"], g["rgb"])
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    img = out["img"].cpu().numpy()
    p = psnr(img, o["img"])
    within = float((np.abs(img - o["img"]).max(axis=0) <= 2e-3).mean())
    print(f"\n[{precision}] {name}: PSNR {p:.2f} dB, within 2e-3: {within:.5f}")
    rp, rw = RECORDED_ENCODINGS[(precision, name)]
    assert abs(p - rp) <= 1.0 and abs(within - rw) <= 0.01, (p, within)
    if name.startswith("precision"):
        assert not (p >= 50.0 and within >= 0.999)


def test_render_outputs_empty_tiles_background(tc):
    cam = scenes.pinhole(33, 17, fx=33.0)
    nt = 3 * 2
    ranges = torch.zeros(nt, 2, dtype=torch.int32, device=DEV)
    ids = torch.zeros(1, dtype=torch.int32, device=DEV)
    z = torch.zeros(1, 2, device=DEV)
    for prec in ["fp32", "tc_fp16_split", "tc_fp16"]:
        out = tc.tcgs_render_fwd(cam, tc.render_opts(prec), ranges, ids, z, torch.zeros(1, 3, device=DEV),
                                 torch.ones(1, device=DEV), torch.zeros(1, 3, device=DEV), bg=(0.1, 0.2, 0.3))
        torch.cuda.synchronize()
        img = out["img"].cpu().numpy()
        np.testing.assert_allclose(img[:, 0, 0], [0.1, 0.2, 0.3], rtol=1e-6)
        assert (out["T_final"] == 1).all() and (out["n_contrib"] == 0).all()


# ------------------------------------------------------------------ Frag2Mat error bound (Appendix A)

F16_MAX = 65504.0
LOG2E = 1.0 / math.log(2.0)


def _fp16_inputs_overflow(U, V):
    """Per fragment: does the paper's K = 8 layout of u or v (log2 units, v0 / 3 in three slots)
    leave the FP16 range (True), stay clearly inside it (False), or sit within 0.1 % of the edge
    (None, not checked)?"""
    Vp = np.abs(np.c_[V[:, :1] / 3, V[:, 1:]]) * LOG2E
    Up = np.abs(U)
    edge = 65520.0   # values from here up round to inf
    over = (Up > edge).any(1)[:, None] | (Vp > edge).any(1)[None, :]
    near = ((np.abs(Up - edge) < 1e-3 * edge).any(1)[:, None] | (np.abs(Vp - edge) < 1e-3 * edge).any(1)[None, :])
    return over, near


# precision -> (frame of u and v, bound on |beta_hat - beta| before the FP32 slack)
F2M_MODES = {
    "tc_fp16": ("local", lambda U, V, absum: f2m.paper_bound(absum)),
    "tc_fp16_split": ("local", lambda U, V, absum: 2.0 ** -10 * f2m.paper_bound(absum)),
    "tc_tf32": ("local", lambda U, V, absum: f2m.paper_bound(absum)),
    "tc_fp8": ("local", lambda U, V, absum: f2m.fp8_split_bound(U, V)),
    "tc_tf32_global": ("global", lambda U, V, absum: f2m.paper_bound(absum)),
    "tc_fp16_global": ("global", lambda U, V, absum: f2m.paper_bound(absum)),
}


@pytest.mark.parametrize("precision", list(F2M_MODES))
def test_frag2mat_exponents_within_appendix_bound(tc, precision):
    frame, bound_of = F2M_MODES[precision]
    cam, sc = scenes.precision(P=30_000, width=240, height=120, seed=12)
    _, inp, b, _ = oracle_frame(cam, sc, render=False)
    g = gpu_inputs(inp, b)
    gw, gh = oracle.grid(cam)
    lens = b["ranges"][:, 1] - b["ranges"][:, 0]
    nz = np.nonzero(lens > 0)[0]
    tiles = nz[np.linspace(0, len(nz) - 1, 24).astype(int)]   # spread over the image
    max_n = int(lens[tiles].max())
    beta = tc.tcgs_frag2mat_beta(cam, precision, g["ranges"], g["ids"], g["mean2d"], g["conic"], g["opacity"],
                                 tiles, max_n).cpu().numpy()
    checked = culled_overflow = 0
    for k, t in enumerate(tiles):
        s, e = b["ranges"][t]
        ids = b["ids"][s:e]
        prod = f2m.local_products if frame == "local" else f2m.global_products
        U, V, bex, absum = prod(t % gw, t // gw, inp["mean2d"][ids], inp["conic"][ids], inp["opacity"][ids])
        keep = bex >= -math.log(255.0)
        bh = beta[k, :, : e - s]
        if precision == "tc_fp16_global":
            over, near = _fp16_inputs_overflow(U, V)
            # an input past the FP16 range gives -inf or NaN: the fragment is culled
            ov = keep & over & ~near
            assert not (bh[ov] >= -math.log(255.0)).any()
            culled_overflow += int(ov.sum())
            keep = keep & ~over & ~near
        # FP32 v-construction and accumulation slack (v is built from FP32 inputs in FP32)
        bound = bound_of(U, V, absum) + 8 * 2.0 ** -24 * (absum + 8 * np.abs(bex)) + 1e-6
        if precision == "tc_fp8":
            bound = bound + 32 * 2.0 ** -24 * absum   # 30 products accumulated
        err = np.abs(bh - bex)
        assert (err[keep] <= bound[keep]).all(), (precision, t, float((err - bound)[keep].max()))
        checked += int(keep.sum())
    print(f"\n[frag2mat {precision}] fragments checked {checked}, culled by FP16 overflow {culled_overflow}")
    assert checked > 1000


def test_global_coordinates_collapse_in_fp16(tc):
    """Table 5: Frag2Mat without G2L.  Past 256 px FP16 overflows and the image collapses; TF32
    stays finite but loses accuracy; G2L in FP16 is what keeps the image."""
    cam, sc = scenes.precision(P=100_000, width=1024, height=512, seed=13)
    _, inp, b, _ = oracle_frame(cam, sc, render=False)
    g = gpu_inputs(inp, b)
    imgs = {}
    for prec in ["tc_fp16_split", "tc_fp16", "tc_fp16_global", "tc_tf32_global"]:
        imgs[prec] = tc.tcgs_render_fwd(cam, tc.render_opts(prec), g["ranges"], g["ids"], g["mean2d"], g["conic"],
                                        g["opacity"], g["rgb"])["img"].cpu().numpy()
    ref = imgs["tc_fp16_split"]
    p = {k: psnr(v, ref) for k, v in imgs.items() if k != "tc_fp16_split"}
    print("\n[ablation, PSNR vs TC split] " + ", ".join(f"{k} {v:.2f} dB" for k, v in p.items()))
    assert all(np.isfinite(v).all() for v in imgs.values())
    assert p["tc_fp16_global"] < 20.0
    assert p["tc_fp16"] > p["tc_tf32_global"] + 10.0


# ------------------------------------------------------------------ backward

@pytest.mark.parametrize("name,make", SMALL[:2])
def test_backward_matches_oracle_gradient(tc, name, make):
    """Backward kernel against the oracle's analytic gradient (pinned by FP64 finite differences).
    Every Gaussian that no counted margin pixel evaluates is checked: per Gaussian and gradient
    array, |gpu - oracle| <= 1e-4 x (its largest oracle component + 1e-3 x the array's largest);
    the excluded ones are exactly those evaluated at a margin pixel (helpers.gaussians_at_pixels)."""
    cam, sc = make()
    _, inp, b, o = oracle_frame(cam, sc)
    g = gpu_inputs(inp, b)
    rng = np.random.default_rng(21)
    gimg = f32(rng.standard_normal((3, cam["height"], cam["width"])))
    ref = oracle.render_bwd(cam, b, inp["mean2d"], inp["conic"], inp["opacity"], inp["rgb"], gimg)
    fwd = tc.tcgs_render_fwd(cam, tc.render_opts("fp32"), g["ranges"], g["ids"], g["mean2d"], g["conic"],
                             g["opacity"], g["rgb"])
    grads = tc.tcgs_render_bwd(cam, tc.render_opts("fp32"), g["ranges"], g["ids"], g["mean2d"], g["conic"],
                               g["opacity"], g["rgb"], fwd["img"], fwd["T_final"], fwd["n_contrib"],
                               to_torch(gimg, DEV))
    torch.cuda.synchronize()
    P = len(inp["opacity"])
    margin = margin_mask(o, 1e-4, 1e-4)
    assert margin.mean() < 1e-3
    excl = np.zeros(P, bool)
    ex = gaussians_at_pixels(b, cam, margin, o["n_eval"], fwd["n_contrib"].cpu().numpy())
    excl[:len(ex)] = ex
    print(f"\n[backward] {name}: {int(margin.sum())} margin pixels, {int(excl.sum())} of {P} Gaussians excluded")
    for key in ("dmean2d", "dconic", "dopacity", "drgb"):
        a = grads[key].cpu().numpy().reshape(P, -1)
        r = ref[key].reshape(P, -1)
        scale = np.abs(r).max(axis=1) + 1e-3 * np.abs(r).max()
        rel = (np.abs(a - r).max(axis=1) / scale)[~excl]
        print(f"  {key}: rel err 99.9% {np.quantile(rel, 0.999):.2e}, max {rel.max():.2e}")
        assert rel.max() <= 1e-4, (key, int((rel > 1e-4).sum()), float(rel.max()))


def test_autograd_function_matches_backward(tc):
    cam, sc = scenes.plain_forward(P=300, width=64, height=64, seed=31)
    _, inp, b, o = oracle_frame(cam, sc)
    g = gpu_inputs(inp, b)
    params = [g[k].clone().requires_grad_(True) for k in ("mean2d", "conic", "opacity", "rgb")]
    target = torch.rand(3, 64, 64, device=DEV, generator=torch.Generator(DEV).manual_seed(0))
    img, T = tc.rasterize(*params, cam, g["ranges"], g["ids"], precision="fp32")
    loss = (img - target).abs().sum()
    loss.backward()
    gimg = torch.sign(img.detach() - target).cpu().numpy().astype(np.float32)
    ref = oracle.render_bwd(cam, b, inp["mean2d"], inp["conic"], inp["opacity"], inp["rgb"], gimg)
    for p, k in zip(params, ("dmean2d", "dconic", "dopacity", "drgb")):
        a = p.grad.cpu().numpy().reshape(ref[k].shape)
        np.testing.assert_allclose(a, ref[k], rtol=1e-3, atol=1e-4 * np.abs(ref[k]).max())


@pytest.mark.parametrize("name,make", SMALL)
@pytest.mark.parametrize("precision", ["tc_fp16_split", "tc_fp16"])
def test_tc_block_culling_changes_nothing(tc, name, make, precision):
    """The per-block skip only drops list entries whose exact exponent is below -ln 255 (with a margin
    of about 5e-4) at every pixel of the block.  For the split layout (exponent error ~1e-5) the image
    is therefore bit-identical with and without the skip; the paper's K = 8 layout has exponent errors
    up to ~0.1, which can lift such an entry over the threshold when it is not skipped, so there only
    a handful of pixels may differ.  Fewer entries are executed either way."""
    cam, sc = make()
    _, inp, b, o = oracle_frame(cam, sc)
    g = gpu_inputs(inp, b)
    nt = b["ranges"].shape[0]
    res = {}
    for cull in (False, True):
        stats = torch.zeros(nt, 8, dtype=torch.int32, device=DEV)
        out = tc.tcgs_render_fwd(cam, tc.render_opts(precision, tile_stats=stats, tile_cull=cull), g["ranges"],
                                 g["ids"], g["mean2d"], g["conic"], g["opacity"], g["rgb"])
        torch.cuda.synchronize()
        res[cull] = ({k: v.cpu().numpy() for k, v in out.items()}, stats.cpu().numpy().astype(np.int64))
    if precision == "tc_fp16_split":
        for k in ("img", "T_final", "n_contrib"):
            np.testing.assert_array_equal(res[True][0][k], res[False][0][k])
        np.testing.assert_array_equal(res[True][1][:, :2], res[False][1][:, :2])
    else:
        diff = (res[True][0]["img"] != res[False][0]["img"]).any(axis=0)
        assert diff.mean() < 1e-2
        # skipping only removes entries that are culled in exact arithmetic: never further from the oracle
        assert psnr(res[True][0]["img"], o["img"]) >= psnr(res[False][0]["img"], o["img"]) - 0.05
    assert res[True][1][:, 2].sum() < res[False][1][:, 2].sum()


# ------------------------------------------------------------------ projection backward

def _rel_err_per_gaussian(got, ref):
    got = got.reshape(len(got), -1).astype(np.float64)
    ref = ref.reshape(len(ref), -1)
    scale = np.abs(ref).max(axis=1) + 1e-6 * (np.abs(ref).max() + 1e-30)
    return np.abs(got - ref).max(axis=1) / scale


@pytest.mark.parametrize("name,make", SMALL)
def test_project_backward_matches_oracle(tc, name, make):
    cam, sc = make()
    pr = oracle.project(cam, scene64(sc))
    P = len(sc["opacity"])
    rng = np.random.default_rng(31)
    wm, wc, wr = f32(rng.normal(size=(P, 2))), f32(rng.normal(size=(P, 3))), f32(rng.normal(size=(P, 3)))
    ref = oracle.project_bwd(cam, scene64(sc), pr["radius"], wm, wc, wr)
    dsc = tc.scene_to_device(sc, DEV)
    g = tc.tcgs_project_bwd(cam, dsc["means3"], dsc["scales"], dsc["quats"], dsc["sh"], sc["sh_degree"],
                            to_torch(pr["radius"].astype(np.int32), DEV), to_torch(wm, DEV), to_torch(wc, DEV),
                            to_torch(wr, DEV))
    torch.cuda.synchronize()
    vis = pr["radius"] > 0
    for key in ("dmeans3", "dscales", "dquats", "dsh"):
        got = g[key].cpu().numpy()
        assert (got[~vis] == 0).all()
        e = _rel_err_per_gaussian(got[vis], ref[key][vis])
        print(f"\n[project bwd] {name} {key}: median rel err {np.median(e):.2e}, 99.9% {np.quantile(e, 0.999):.2e}, "
              f"max {e.max():.2e}")
        assert np.quantile(e, 0.999) <= 1e-4 and e.max() <= 2e-3, (key, e.max())


@pytest.mark.parametrize("precision", ["fp32", "tc_fp16_split"])
def test_render_gaussians_gradients_match_oracle_chain(tc, precision):
    """End to end: autograd through the library's render and projection backward kernels against
    the oracle's render backward followed by its projection backward."""
    cam, sc = scenes.plain_forward(P=400, width=96, height=64, seed=21)
    sc = dict(sc)
    sc["scales"] = f32(sc["scales"] * 2.0)
    s64 = scene64(sc)
    rng = np.random.default_rng(22)
    G = f32(rng.standard_normal((3, 64, 96)))
    pr = oracle.project(cam, s64)
    b = oracle.bin_sort(cam, pr["mean2d"], pr["radius"], pr["depth"])
    rb = oracle.render_bwd(cam, b, pr["mean2d"], pr["conic"], s64["opacity"], pr["rgb"], G)
    ref = oracle.project_bwd(cam, s64, pr["radius"], rb["dmean2d"], rb["dconic"], rb["drgb"])
    ref["dopacity"] = rb["dopacity"]
    leaves = {k: to_torch(sc[k], DEV).requires_grad_(True) for k in ("means3", "scales", "quats", "opacity", "sh")}
    img, _ = tc.render_gaussians(cam, leaves["means3"], leaves["scales"], leaves["quats"], leaves["opacity"],
                                 leaves["sh"], sc["sh_degree"], precision=precision)
    (img * to_torch(G, DEV)).sum().backward()
    torch.cuda.synchronize()
    vis = pr["radius"] > 0
    for key, leaf in [("dmeans3", "means3"), ("dscales", "scales"), ("dquats", "quats"), ("dopacity", "opacity"),
                      ("dsh", "sh")]:
        got = leaves[leaf].grad.cpu().numpy()
        e = _rel_err_per_gaussian(got[vis], ref[key][vis])
        print(f"\n[end to end {precision}] {key}: median rel err {np.median(e):.2e}, 99% {np.quantile(e, 0.99):.2e}")
        assert np.quantile(e, 0.99) <= 1e-3, (key, np.quantile(e, 0.99))
