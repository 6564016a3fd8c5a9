"""GPU parity at the workloads' full sizes, through the C ABI, on tiles the FP64 oracle computes one
by one: the backward of the differentiation workload (1280x720, 500k Gaussians) and the forward of
the large workload (3840x2160, 6M Gaussians), each in the launch configuration the benchmark times.

Common inputs: the oracle's FP64 projection rounded to FP32 feeds both sides of the binning and
blending stages.  Decision-margin pixels (a cull test within 1e-5 or a termination test within 1e-4 of
its threshold in the oracle's arithmetic; helpers.margin_mask) are counted and excluded from the element-wise bounds, and so are the
Gaussians evaluated at such pixels in the backward (a flipped decision changes the transmittance of
every later fragment and the blended colour behind every earlier one)."""
import math

import numpy as np
import pytest

import oracle
from paper_2505_24796_gb300 import scenes

from .helpers import f32, gaussians_at_pixels, margin_mask, psnr, scene64, to_torch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.fixture(scope="module")
def tc():
    import paper_2505_24796_gb300 as m
    m._lib.load()
    return m


def _fp32_inputs(pr, sc):
    return dict(mean2d=f32(pr["mean2d"]), conic=f32(pr["conic"]), depth=f32(pr["depth"]), radius=pr["radius"],
                rgb=f32(pr["rgb"]), opacity=f32(sc["opacity"]))


def _on_device(inp):
    return {k: to_torch(v.astype(np.int32) if k == "radius" else v, DEV) for k, v in inp.items()}


def _restrict(b, tiles):
    """The binned lists with every tile outside `tiles` emptied (both sides then work on the
    sampled tiles only)."""
    ranges = np.zeros_like(b["ranges"])
    ranges[tiles] = b["ranges"][tiles]
    return dict(n=b["n"], ids=b["ids"], ranges=ranges)


def _tile_mask(cam, tiles):
    gw, _ = oracle.grid(cam)
    m = np.zeros((cam["height"], cam["width"]), bool)
    for t in tiles:
        tx, ty = int(t) % gw, int(t) // gw
        m[16 * ty:16 * ty + 16, 16 * tx:16 * tx + 16] = True
    return m


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


def test_backward_full_size_matches_oracle_on_sampled_tiles(tc):
    """Differentiation workload at full size (1280x720, 500k Gaussians, exact tile coverage, L1 loss to
    the seeded target): the FP32 forward and the backward kernel on 48 sampled tiles (all other tiles'
    lists emptied on both sides) against the oracle's analytic gradient (itself pinned by FP64 finite
    differences).  dL/dimg = sign(oracle image - target), the same input on both sides.  Every
    Gaussian that is not evaluated at a counted margin pixel is checked: per Gaussian and gradient
    array, |gpu - oracle| <= 2e-4 x (its largest oracle component + 1e-3 x the array's largest)."""
    cam, sc, target = scenes.differentiation()
    P = len(sc["opacity"])
    pr = oracle.project(cam, scene64(sc))
    inp = _fp32_inputs(pr, sc)
    b_full = oracle.bin_sort(cam, inp["mean2d"], inp["radius"], inp["depth"], conic=inp["conic"],
                             opacity=inp["opacity"])
    gw, gh = oracle.grid(cam)
    lens = b_full["ranges"][:, 1] - b_full["ranges"][:, 0]
    tiles = np.sort(np.random.default_rng(23).choice(np.nonzero(lens > 0)[0], 48, replace=False))
    b = _restrict(b_full, tiles)
    o = oracle.render(cam, b, inp["mean2d"], inp["conic"], inp["opacity"], inp["rgb"], tiles=tiles)
    gimg = f32(np.sign(o["img"] - target))
    ref = oracle.render_bwd(cam, b, inp["mean2d"], inp["conic"], inp["opacity"], inp["rgb"], gimg)

    g = _on_device(inp)
    ranges = to_torch(b["ranges"].astype(np.int32), DEV)
    ids = to_torch(b["ids"].astype(np.int32), DEV)
    opts = tc.render_opts("fp32")
    fwd = tc.tcgs_render_fwd(cam, opts, ranges, ids, g["mean2d"], g["conic"], g["opacity"], g["rgb"])
    grads = tc.tcgs_render_bwd(cam, opts, ranges, ids, g["mean2d"], g["conic"], g["opacity"], g["rgb"], fwd["img"],
                               fwd["T_final"], fwd["n_contrib"], to_torch(gimg, DEV))
    torch.cuda.synchronize()
    nc = fwd["n_contrib"].cpu().numpy()

    mask = _tile_mask(cam, tiles)
    margin = margin_mask(o) & mask
    excluded = np.zeros(P, bool)
    ex = gaussians_at_pixels(b, cam, margin, o["n_eval"], nc)
    excluded[:len(ex)] = ex
    in_lists = np.zeros(P, bool)
    for t in tiles:
        s, e = b["ranges"][t]
        in_lists[b["ids"][s:e]] = True
    checked = in_lists & ~excluded
    print(f"\n[backward full size] {len(tiles)} tiles, {int(mask.sum())} pixels, {int(margin.sum())} margin pixels, "
          f"{int(in_lists.sum())} Gaussians in the lists, {int(excluded.sum())} excluded")
    assert margin.sum() <= 5e-3 * mask.sum()   # long lists: more fragments per pixel near a threshold
    assert checked.sum() >= 0.9 * in_lists.sum()
    for key in ("dmean2d", "dconic", "dopacity", "drgb"):
        a = grads[key].cpu().numpy().reshape(P, -1).astype(np.float64)
        r = ref[key].reshape(P, -1)
        assert (a[~in_lists] == 0).all(), key
        scale = np.abs(r).max(axis=1) + 1e-3 * np.abs(r[checked]).max()
        rel = (np.abs(a - r).max(axis=1) / scale)[checked]
        print(f"  {key}: rel err median {np.median(rel):.2e}, 99.9% {np.quantile(rel, 0.999):.2e}, "
              f"max {rel.max():.2e}")
        assert rel.max() <= 2e-4, (key, float(rel.max()), int((rel > 2e-4).sum()))


def _gaussians_near_tiles(inp, tiles, gw):
    """Indices (ascending) of the Gaussians whose tile rectangle can meet one of `tiles`: a superset
    (one tile of slack) of those the sorting stage lists there, so the oracle bins only these."""
    m = inp["mean2d"].astype(np.float64)
    r = inp["radius"].astype(np.float64)
    vis = r > 0
    keep = np.zeros(len(r), bool)
    for t in tiles:
        x0, y0 = 16.0 * (int(t) % gw), 16.0 * (int(t) // gw)
        keep |= vis & (m[:, 0] + r + 16 >= x0) & (m[:, 0] - r - 16 <= x0 + 16) & \
            (m[:, 1] + r + 16 >= y0) & (m[:, 1] - r - 16 <= y0 + 16)
    return np.nonzero(keep)[0]


def _subset(inp, S):
    return {k: v[S] for k, v in inp.items()}


def test_large_frame_full_size_matches_oracle_on_sampled_tiles(tc):
    """Large workload at full size (3840x2160, 6M Gaussians in 256 clusters, SH3, exact tile coverage,
    about 605M splats) in the benchmark's launch configuration (persistent TC renderer in longest-list
    order), on 48 random tiles.  The oracle bins only the Gaussians whose rectangle can reach those
    tiles (ids kept in ascending order, so its depth ties resolve as on the whole scene).
    (1) On the oracle's FP32-rounded projection: the GPU's lists of the sampled tiles equal the
    oracle's up to splats within FP32 rounding of the coverage limit; FP32 renderer within 1e-5 away
    from margin pixels; TC renderer PSNR >= 50 dB with >= 99.9% of pixels within 2e-3.  (2) The whole
    GPU frame from the scene against the FP64 oracle: the TC criteria."""
    cam, sc = scenes.large()
    P = len(sc["opacity"])
    s64 = scene64(sc)
    pr = oracle.project(cam, s64)
    inp = _fp32_inputs(pr, sc)
    n_rect = int(pr["tiles_touched"].astype(np.int64).sum())
    gw, gh = oracle.grid(cam)
    tiles = np.sort(np.random.default_rng(29).choice(gw * gh, 48, replace=False)).astype(np.int32)
    mask = _tile_mask(cam, tiles)

    S = _gaussians_near_tiles(inp, tiles, gw)
    sub = _subset(inp, S)
    b = oracle.bin_sort(cam, sub["mean2d"], sub["radius"], sub["depth"], conic=sub["conic"], opacity=sub["opacity"])
    o = oracle.render(cam, b, sub["mean2d"], sub["conic"], sub["opacity"], sub["rgb"], tiles=tiles)

    g = _on_device(inp)
    out_b = tc.tcgs_bin_sort(cam, g["mean2d"], g["radius"], g["depth"], capacity=n_rect + 1024, conic=g["conic"],
                             opacity=g["opacity"])
    torch.cuda.synchronize()
    assert int(out_b["status"].item()) == 0
    n = int(out_b["n_splats"].item())
    ranges = out_b["tile_ranges"].cpu().numpy().astype(np.int64)
    mism = 0
    for t in tiles:
        s0, e0 = b["ranges"][t]
        lo = list(S[b["ids"][s0:e0]])
        s1, e1 = ranges[t]
        lg = list(out_b["ids_sorted"][s1:e1].cpu().numpy().astype(np.int64))
        if lo != lg:
            diff = set(lo) ^ set(lg)
            mism += len(diff)
            assert all(_borderline(cam, inp, int(gg), int(t)) for gg in diff), (t, diff)
            assert [x for x in lo if x not in diff] == [x for x in lg if x not in diff]
    order = tc.tcgs_tile_order(cam, out_b["tile_ranges"])
    counter = torch.zeros(1, dtype=torch.int32, device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    imgs = {}
    for prec in ("fp32", "tc_fp16_split", "fp32_frag2mat"):
        opts = tc.render_opts(prec, device_status=status, tile_order=order if prec != "fp32" else None,
                              work_counter=counter if prec != "fp32" else None)
        out = tc.tcgs_render_fwd(cam, opts, out_b["tile_ranges"], out_b["ids_sorted"], g["mean2d"], g["conic"],
                                 g["opacity"], g["rgb"])
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        imgs[prec] = (out["img"].cpu().numpy(), out["T_final"].cpu().numpy())
    del out_b, g
    torch.cuda.empty_cache()
    img32, T32 = imgs["fp32"]
    keep = mask & ~margin_mask(o)
    print(f"\n[large full size] {int((mask & ~keep).sum())} margin pixels of {int(mask.sum())}")
    assert keep.sum() >= 0.995 * mask.sum()   # long lists: more fragments per pixel near a threshold
    assert np.abs(img32 - o["img"]).max(axis=0)[keep].max() <= 1e-5
    assert np.abs(T32 - o["T"])[keep].max() <= 1e-5
    imgtc = imgs["tc_fp16_split"][0]
    p_tc = psnr(imgtc[:, mask], o["img"][:, mask])
    assert p_tc >= 50.0
    assert (np.abs(imgtc - o["img"]).max(axis=0)[mask] <= 2e-3).mean() >= 0.999
    # the same kernel with the product on CUDA cores: the TC criteria, and within 1e-4 off the margins
    imgcc = imgs["fp32_frag2mat"][0]
    assert psnr(imgcc[:, mask], o["img"][:, mask]) >= 50.0
    assert np.abs(imgcc - o["img"]).max(axis=0)[keep].max() <= 1e-4

    # (2) the whole frame from the scene, as the benchmark renders it
    d = tc.scene_to_device(sc, DEV)
    r = tc.Renderer(cam, P, n_rect + 1024, device=DEV)
    img = r.frame(d)["img"].cpu().numpy()
    del r, d
    torch.cuda.empty_cache()
    pr64 = {k: pr[k] for k in ("mean2d", "conic", "depth", "radius", "rgb")}
    pr64["opacity"] = s64["opacity"]
    S64 = _gaussians_near_tiles(pr64, tiles, gw)
    sub64 = _subset(pr64, S64)
    b64 = oracle.bin_sort(cam, sub64["mean2d"], sub64["radius"], sub64["depth"], conic=sub64["conic"],
                          opacity=sub64["opacity"])
    o64 = oracle.render(cam, b64, sub64["mean2d"], sub64["conic"], sub64["opacity"], sub64["rgb"], tiles=tiles,
                        margins=False)
    p_frame = psnr(img[:, mask], o64["img"][:, mask])
    assert p_frame >= 50.0
    assert (np.abs(img - o64["img"]).max(axis=0)[mask] <= 2e-3).mean() >= 0.999
    print(f"\n[large full size] {n} splats, {len(S)} Gaussians near the {len(tiles)} tiles, {mism} borderline list "
          f"differences, TC PSNR {p_tc:.1f} dB (FP32 inputs), {p_frame:.1f} dB (whole frame)")
