"""Benchmark of the TC-GS rasterizer hot path on one GB300 (or N replicas under torchrun).

One step = one frame of the precision workload (1920x1080, fx = fy = 1100, 1M Gaussians in
64 clusters, SH degree 3): project -> bin_sort (exact tile coverage) -> render_fwd with the
Frag2Mat tensor-core path (FP16 hi/lo split, G2L).  Inputs are resident in HBM; L2 is flushed between steps
(outside the timed events).  The same frame on the FP32 CUDA-core path is timed beside it.

Prints ONE JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle instead, on a
bounded sample of the same workload per step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl tcgs|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "frames/s & alpha-evals/s, TC-FP16 vs FP32 path, 1 GB300, PSNR>=50dB vs FP64 oracle"
WORKLOAD = ("precision: 1 view 1920x1080, fx=fy=1100, 1M Gaussians from a 64-cluster anisotropic mixture, "
            "z in [1,50], log-scales N(-4.5,1), bimodal opacity, SH degree 3, seed 2")
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
SM_COUNT, SM_LANES, SM_MAX_MHZ = 152, 128, 2070.0
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) and executed warp
# instructions (smsp__inst_executed.sum) of the render kernel on this workload, from one
# `ncu --set full` capture of this command's kernel.  They are reported only while the kernel's
# sources hash to the value they had when the counters were taken.
NCU_TRAFFIC = {
    "k_render_tc": {"bytes": 44007168 + 9517312, "warp_instructions": 193418978,
                    "sha256": "bcb4542d41fbf2d80dfaeace567d8d180428e0f0e0086258c3603ec35c278bc6",
                    "sources": ["paper_2505_24796_gb300/csrc/render_tc.cu", "paper_2505_24796_gb300/csrc/common.cuh"]},
}


def sources_sha256(paths):
    import hashlib
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def ncu_traffic(kernel, scale=1.0, key="bytes"):
    """A per-launch counter (DRAM bytes by default) from the recorded capture, or None when there is
    none for this source and workload."""
    ent = NCU_TRAFFIC.get(kernel)
    if not ent or ent.get(key) is None or scale != 1.0:
        return None
    return ent[key] if sources_sha256(ent["sources"]) == ent["sha256"] else None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="tcgs", choices=["tcgs", "reference"])
    ap.add_argument("--precision", default="tc_fp16_split", choices=["tc_fp16_split", "tc_fp16"])
    ap.add_argument("--no-graph", action="store_true", help="launch kernels eagerly instead of a CUDA graph")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--scale", type=float, default=1.0, help="fraction of the 1M Gaussians (profiling runs)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the plain, differentiation, scheduler and large workloads (reported beside the headline)")
    ap.add_argument("--sched-train-views", type=int, default=200)
    ap.add_argument("--large-frames", type=int, default=0, metavar="P",
                    help="profiling run: two frames of the large workload's distribution with P Gaussians, "
                         "stage times per frame (no headline line)")
    ap.add_argument("--diff-frames", action="store_true",
                    help="profiling run: two forward + backward frames of the differentiation workload, stage "
                         "times per frame (no headline line)")
    ap.add_argument("--render-arms", action="store_true",
                    help="profiling run: the headline frame binned once, then rendered twice by each renderer arm "
                         "(TC split, the same kernel with the product on CUDA cores, the 3DGS-style FP32 kernel); "
                         "render times per arm (no headline line)")
    ap.add_argument("--arms-workload", default="precision", choices=["precision", "differentiation"],
                    help="workload of --render-arms")
    ap.add_argument("--coverage", default="exact", choices=["exact", "square"],
                    help="tile coverage of the headline binning: the 3-sigma square of the paper's pipeline, or "
                         "exact (tcgs_bin_sort_exact); the other one is timed beside it")
    return ap.parse_args()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return PEAKS_FALLBACK, "fallback"


def workload(scale=1.0):
    from paper_2505_24796_gb300 import scenes
    return scenes.precision(P=int(round(1_000_000 * scale)))


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.25)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ CPU oracle timing

def _scene64(sc):
    return {k: (v.astype(np.float64) if isinstance(v, np.ndarray) else v) for k, v in sc.items()}


def oracle_frame_single(cam, s64):
    """One whole frame of the FP64 oracle on one host thread: projection and binning of the whole
    scene, Algorithm 1 on every tile.  Returns (seconds, info with the image)."""
    import oracle
    t0 = time.perf_counter()
    pr = oracle.project(cam, s64)
    t1 = time.perf_counter()
    b = oracle.bin_sort(cam, pr["mean2d"], pr["radius"], pr["depth"])
    t2 = time.perf_counter()
    o = oracle.render(cam, b, pr["mean2d"], pr["conic"], s64["opacity"], pr["rgb"], margins=False)
    t3 = time.perf_counter()
    gw, gh = oracle.grid(cam)
    return t3 - t0, dict(project_s=t1 - t0, bin_s=t2 - t1, render_s=t3 - t2, tiles=gw * gh, img=o["img"])


def oracle_frame_all_cores(cam, s64, threads=None):
    """The FP64 oracle on one whole frame with every host core: projection and binning as they stand
    (single-threaded), then Algorithm 1 on the tiles dealt round-robin to one thread per core (the C
    renderer keeps no global state, and ctypes releases the GIL for the call); the threads' images
    cover disjoint tiles on a black background, so their sum is the frame.  Returns (seconds, threads,
    image)."""
    import concurrent.futures as cf
    import oracle
    threads = threads or len(os.sched_getaffinity(0))
    t0 = time.perf_counter()
    pr = oracle.project(cam, s64)
    b = oracle.bin_sort(cam, pr["mean2d"], pr["radius"], pr["depth"])
    gw, gh = oracle.grid(cam)
    parts = [np.arange(i, gw * gh, threads, dtype=np.int32) for i in range(threads)]

    def part(tiles):
        return oracle.render(cam, b, pr["mean2d"], pr["conic"], s64["opacity"], pr["rgb"], tiles=tiles,
                             margins=False)["img"]
    with cf.ThreadPoolExecutor(threads) as ex:
        imgs = list(ex.map(part, parts))
    t1 = time.perf_counter()
    return t1 - t0, threads, np.sum(imgs, axis=0)


def run_reference(args):
    """Reference arm: the FP64 CPU oracle, as it stands, on the host cores.  Every step, warm-up
    included, is one whole frame of the bench workload (projection and binning single-threaded,
    Algorithm 1 on all tiles dealt to one thread per core); the line reports the mean of the timed
    frames, measured, not extrapolated.  Under torchrun only rank 0 runs it."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cam, sc = workload(args.scale)
    s64 = _scene64(sc)
    times, n_thr = [], 1
    for i in range(args.warmup + args.steps):
        t, n_thr, _ = oracle_frame_all_cores(cam, s64)
        if i >= args.warmup:
            times.append(t)
    t = statistics.mean(times)
    v = 1.0 / t
    gw, gh = (cam["width"] + 15) // 16, (cam["height"] + 15) // 16
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "frames/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "P": len(sc["opacity"]), "coverage": "square (3-sigma)"},
        "cpu_baseline": {"value": v, "unit": "frames/s", "cores": n_thr, "kind": "oracle",
                         "sample": f"every step one whole frame: FP64 projection + binning of the whole scene "
                                   f"(one thread) and Algorithm 1 on all {gw * gh} tiles dealt to {n_thr} threads; "
                                   f"mean of {args.steps} timed frames after {args.warmup} warm-up frames"},
        "e2e": {"value": v, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ------------------------------------------------------------------ other workloads (same run)

def _events_ms(fn, reps, warmup, flush=None):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def bench_plain(dev, flush, stream, steps=50, warmup=5):
    """128x128, 1,000 Gaussians, SH0: whole frames of both renderers, each replayed as one CUDA graph
    with the L2 flushed before every frame (at this size a frame is bound by launch latency)."""
    import torch
    import paper_2505_24796_gb300 as tc
    from paper_2505_24796_gb300 import scenes
    cam, sc = scenes.plain_forward()
    d = tc.scene_to_device(sc, dev)
    pr = tc.tcgs_project(cam, d["means3"], d["scales"], d["quats"], d["sh"], d["sh_degree"])
    n = int(pr["tiles_touched"].to(torch.int64).sum().item())
    r = tc.Renderer(cam, len(sc["opacity"]), n + 1024, device=dev, stats=True)
    r.frame(d, precision="fp32")
    torch.cuda.synchronize()
    st = r.stats.to(torch.int64).sum(0).tolist()
    img32 = r.out["img"].clone()
    r.stats = None
    out = {"workload": "plain: 128x128, fx=fy=128, 1,000 Gaussians, SH0; exact tile coverage",
           "splats": int(r.bins["n_splats"].item()), "alpha_evals": st[0] + st[1]}
    for prec in ("tc_fp16_split", "fp32", "fp32_frag2mat"):
        tot, stg = time_frames(r, d, prec, steps, warmup, True, flush, stream)
        ms = statistics.median(tot)
        out[prec] = {"frames_per_s": 1000.0 / ms, "frame_ms": ms,
                     "stages_ms": dict(zip(["project", "bin_sort", "render_fwd"],
                                           [statistics.median(x) for x in stg]))}
    out["speedup_frame"] = out["fp32"]["frame_ms"] / out["tc_fp16_split"]["frame_ms"]
    out["speedup_render"] = (out["fp32"]["stages_ms"]["render_fwd"] /
                             out["tc_fp16_split"]["stages_ms"]["render_fwd"])
    out["speedup_render_vs_fp32_same_skip"] = (out["fp32_frag2mat"]["stages_ms"]["render_fwd"] /
                                               out["tc_fp16_split"]["stages_ms"]["render_fwd"])
    r.frame(d, precision="tc_fp16_split")
    torch.cuda.synchronize()
    diff = (r.out["img"] - img32).abs().max().item()
    out["max_abs_tc_vs_fp32"] = diff
    return out


def bench_differentiation(dev, flush):
    """1280x720, 500k Gaussians: forward and backward of the alpha-blending stage (L1 loss to a seeded
    target); the loss gradient itself is user code and is formed outside the timed events."""
    import torch
    import paper_2505_24796_gb300 as tc
    from paper_2505_24796_gb300 import scenes
    cam, sc, target = scenes.differentiation()
    d = tc.scene_to_device(sc, dev)
    pr = tc.tcgs_project(cam, d["means3"], d["scales"], d["quats"], d["sh"], d["sh_degree"])
    n = int(pr["tiles_touched"].to(torch.int64).sum().item())
    r = tc.Renderer(cam, len(sc["opacity"]), n + 1024, device=dev, stats=True)
    r.frame(d, precision="fp32")
    torch.cuda.synchronize()
    st = r.stats.to(torch.int64).sum(0).tolist()
    n_exact = int(r.bins["n_splats"].item())
    r.stats = None
    square = _coverage_render(cam, d, n + 1024, dev, flush, exact=False)
    tgt = torch.from_numpy(target).to(dev)
    gimg = torch.sign(r.out["img"] - tgt).contiguous()
    P = len(sc["opacity"])
    grads = dict(dmean2d=torch.zeros(P, 2, device=dev), dconic=torch.zeros(P, 3, device=dev),
                 dopacity=torch.zeros(P, device=dev), drgb=torch.zeros(P, 3, device=dev))
    opts = tc.render_opts("fp32")

    def bwd():
        tc.tcgs_render_bwd(r.cam, opts, r.bins["tile_ranges"], r.bins["ids_sorted"], r.proj["mean2d"], r.proj["conic"],
                           d["opacity"], r.proj["rgb"], r.out["img"], r.out["T_final"], r.out["n_contrib"], gimg,
                           grads=grads)
    fwd32 = _events_ms(lambda: r.render(d["opacity"], "fp32"), 10, 3, flush)
    fwdtc = _events_ms(lambda: r.render(d["opacity"], "tc_fp16_split"), 10, 3, flush)
    fwdcc = _events_ms(lambda: r.render(d["opacity"], "fp32_frag2mat"), 10, 3, flush)
    one = _one_pixel_a_thread(r, d, flush, 10, 3)
    r.render(d["opacity"], "fp32")
    bwd_ms = _events_ms(bwd, 10, 3, flush)
    proj_ms = _events_ms(lambda: r.project(d), 10, 3, flush)
    bin_ms = _events_ms(lambda: r.bin_sort(), 10, 3, flush)
    g3 = dict(dmeans3=torch.zeros_like(d["means3"]), dscales=torch.zeros_like(d["scales"]),
              dquats=torch.zeros_like(d["quats"]), dsh=torch.zeros_like(d["sh"]))
    pbwd_ms = _events_ms(lambda: tc.tcgs_project_bwd(r.cam, d["means3"], d["scales"], d["quats"], d["sh"],
                                                     d["sh_degree"], r.proj["radius"], grads["dmean2d"],
                                                     grads["dconic"], grads["drgb"], grads=g3), 10, 3, flush)
    return {"workload": "differentiation: 1280x720, fx=fy=1280, 500k Gaussians (plain distributions), L1 to a "
                        "seeded target; backward replays the FP32 forward; exact tile coverage",
            "splats": n_exact, "square_coverage": square,
            "alpha_evals": st[0] + st[1], "f_blend": st[0],
            "ms": {"project": proj_ms, "bin_sort": bin_ms, "render_fwd_fp32": fwd32,
                   "render_fwd_tc": fwdtc, "render_fwd_fp32_same_skip": fwdcc, "render_bwd": bwd_ms,
                   "project_bwd": pbwd_ms},
            "pixels_per_thread": r.pixels_per_thread, "render_fwd_one_pixel_a_thread_ms": one,
            "speedup_render": {"vs_fp32": fwd32 / fwdtc, "vs_fp32_same_skip": fwdcc / fwdtc},
            "frames_per_s_fwd": {"tc_fp16_split": 1000.0 / (proj_ms + bin_ms + fwdtc),
                                 "fp32": 1000.0 / (proj_ms + bin_ms + fwd32)},
            "train_step_ms_fp32": proj_ms + bin_ms + fwd32 + bwd_ms + pbwd_ms,
            "train_step_ms_tc_fwd": proj_ms + bin_ms + fwdtc + bwd_ms + pbwd_ms,
            "train_step_note": "forward and backward to the 3D parameters (means, scales, quaternions, opacity, "
                               "SH); per-stage CUDA events with L2 flushed before each stage",
            "bwd_alpha_evals_per_s": (st[0] + st[1]) / (bwd_ms * 1e-3)}


def _sched_run(dev, eval_cams, scene, train_cams, label, chunk=16):
    """Train the tile-cost MLP on the tile costs recorded by renders of train_cams, then time the
    batched render of eval_cams in natural, list-length and MLP order; also the FP32 arms of the same
    batch: the batched renderer with its product on CUDA cores (list-length order) and the 3DGS-style
    FP32 kernel launched view by view."""
    import torch
    import paper_2505_24796_gb300 as tc
    from oracle import sched as osc
    from paper_2505_24796_gb300.sched import MultiView, TileCostModel
    d = tc.scene_to_device(scene, dev)
    t0 = time.perf_counter()
    Xs, ys = [], []
    for i in range(0, len(train_cams), chunk):
        mv = MultiView(d, train_cams[i:i + chunk], device=dev)
        X, y = mv.training_data()
        Xs.append(X); ys.append(y)
        del mv
    X, y = torch.cat(Xs).contiguous(), torch.cat(ys).contiguous()
    collect_s = time.perf_counter() - t0
    model = TileCostModel(device=dev, seed=0)
    t1 = time.perf_counter()
    loss = model.fit(X, y, steps=800)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t1
    mv = MultiView(d, eval_cams, device=dev)
    Xt, yt = mv.training_data()
    walked, cycles = mv.tile_costs()
    pred = model.predict(Xt)
    torch.cuda.synchronize()
    ytn, pn = yt.cpu().numpy().astype(np.float64), pred.cpu().numpy().astype(np.float64)
    nlen = torch.cat([(r.bins["tile_ranges"][:, 1] - r.bins["tile_ranges"][:, 0]) for r in mv.views]).cpu().numpy()
    A = np.c_[np.log1p(nlen), np.ones_like(ytn)]
    base = A @ np.linalg.lstsq(A, ytn, rcond=None)[0]
    res = {"workload": label, "tiles": int(Xt.shape[0]), "train_items": int(X.shape[0]), "train_loss": loss,
           "collect_s": collect_s, "train_s": train_s,
           "heldout_mse_log_cost": {"mlp": float(np.mean((pn - ytn) ** 2)),
                                    "list_length_fit": float(np.mean((base - ytn) ** 2))}}
    items = mv.items().cpu().numpy()
    cyc = dict(zip(items.tolist(), cycles.cpu().numpy().tolist()))
    workers = tc.tcgs_tc_wave_tiles()   # resident CTAs of the persistent renderer
    times, sim, imgs = {}, {}, {}
    for policy in ("natural", "length", "mlp"):
        q = mv.queue(policy, model)
        times[policy] = mv.time_render(q, reps=15, warmup=3)
        sim[policy] = osc.lpt_makespan([cyc[i] for i in q.cpu().numpy().tolist()], workers)
        torch.cuda.synchronize()
        imgs[policy] = [r.out["img"].clone() for r in mv.views]
    res["batched_render_ms"] = times
    res["simulated_makespan_cycles"] = sim
    cyc_all = np.asarray(list(cyc.values()), dtype=np.float64)
    # no order of whole tiles can finish before the heaviest tile, nor before the work spread evenly
    res["makespan_lower_bound_cycles"] = {"heaviest_tile": float(cyc_all.max()),
                                          "even_spread": float(cyc_all.sum() / workers)}
    res["resident_ctas"] = workers
    res["gain_vs_length"] = times["length"] / times["mlp"]
    res["gain_vs_natural"] = times["natural"] / times["mlp"]
    res["simulated_gain_vs_length"] = sim["length"] / sim["mlp"]
    res["images_equal_across_orders"] = all(torch.equal(a, b) for p in ("natural", "length")
                                            for a, b in zip(imgs[p], imgs["mlp"]))
    # FP32 arms of the same batch
    q_len = mv.queue("length")
    mv_cc = MultiView(d, eval_cams, precision="fp32_frag2mat", device=dev)
    t_cc = mv_cc.time_render(q_len, reps=15, warmup=3)
    del mv_cc

    opts32 = tc.render_opts("fp32")

    def per_view_fp32():
        for r in mv.views:
            tc.tcgs_render_fwd(r.cam, opts32, r.bins["tile_ranges"], r.bins["ids_sorted"], r.proj["mean2d"],
                               r.proj["conic"], d["opacity"], r.proj["rgb"], out=r.out)
    t_fp32 = _events_ms(per_view_fp32, 15, 3)
    res["fp32_arms_ms"] = {"batched_same_skip_length_order": t_cc, "fp32_3dgs_kernel_view_by_view": t_fp32}
    res["speedup_tc_mlp_vs_fp32"] = {"vs_same_skip_batched": t_cc / times["mlp"], "vs_fp32_view_by_view": t_fp32 / times["mlp"]}
    return res


def bench_scheduler(dev, train_views=200):
    """Config 4: 16 views of one 3M-Gaussian scene at uneven resolutions; the MLP is trained on the tile
    costs recorded by train_views renders of other views, then orders the batched renderer's queue."""
    from paper_2505_24796_gb300 import scenes
    eval_cams, scene = scenes.learned_scheduler()
    return _sched_run(dev, eval_cams, scene, scenes.multiview_cameras(train_views, 77),
                      "learned scheduler: 16 views (640x480..1920x1080, cameras on a sphere of radius 20) of a "
                      "3M-Gaussian scene; MLP 8->32->32->1 trained on tile costs of %d other renders" % train_views)


def bench_scheduler_occluded(dev, train_views=200):
    """16 views at 320x240 (about 8 tiles per resident CTA) of a faint volume with opaque clusters, where
    list length mispredicts tile cost; the MLP is trained on train_views other renders."""
    from paper_2505_24796_gb300 import scenes
    eval_cams, scene = scenes.learned_scheduler_occluded()
    return _sched_run(dev, eval_cams, scene, scenes.low_res_cameras(train_views, 77),
                      "learned scheduler, occluded volume: 16 views at 320x240 of a faint volume (200k Gaussians) "
                      "with 60 opaque clusters (180k); MLP trained on tile costs of %d other renders" % train_views)


def bench_large(dev, flush, steps=5, warmup=2):
    """3840x2160, 6M Gaussians in 256 clusters, SH3: TC forward frame vs FP32 frame, plus backward."""
    import torch
    import paper_2505_24796_gb300 as tc
    from paper_2505_24796_gb300 import scenes
    cam, sc = scenes.large()
    d = tc.scene_to_device(sc, dev)
    pr = tc.tcgs_project(cam, d["means3"], d["scales"], d["quats"], d["sh"], d["sh_degree"])
    n = int(pr["tiles_touched"].to(torch.int64).sum().item())
    del pr
    r = tc.Renderer(cam, len(sc["opacity"]), n + 1024, device=dev, stats=True)
    r.frame(d, precision="fp32")
    torch.cuda.synchronize()
    st = r.stats.to(torch.int64).sum(0).tolist()
    r.stats = None
    out = {"workload": "large: 3840x2160, fx=fy=2200, 6M Gaussians (256 clusters, plain distributions), SH3; "
                       "exact tile coverage",
           "splats": int(r.bins["n_splats"].item()), "alpha_evals": st[0] + st[1]}
    # project and bin_sort are the same kernels on the same inputs for both renderers: timed once, so
    # that the sort's run-to-run spread (about 1 ms on 605M splats) does not decide the comparison
    shared = [_events_ms(lambda: r.project(d), steps, warmup, flush),
              _events_ms(lambda: r.bin_sort(), steps, warmup, flush)]
    out["shared_stages_note"] = "project and bin_sort timed once (identical for both renderers)"
    for prec in ("tc_fp16_split", "fp32", "fp32_frag2mat"):
        stg = shared + [_events_ms(lambda: r.render(d["opacity"], prec), steps, warmup, flush)]
        out[prec] = {"stages_ms": dict(zip(["project", "bin_sort", "render_fwd"], stg)), "frame_ms": sum(stg),
                     "frames_per_s": 1000.0 / sum(stg)}
    out["speedup_render"] = out["fp32"]["stages_ms"]["render_fwd"] / out["tc_fp16_split"]["stages_ms"]["render_fwd"]
    out["speedup_render_vs_fp32_same_skip"] = (out["fp32_frag2mat"]["stages_ms"]["render_fwd"] /
                                               out["tc_fp16_split"]["stages_ms"]["render_fwd"])
    out["speedup_frame"] = out["fp32"]["frame_ms"] / out["tc_fp16_split"]["frame_ms"]
    out["pixels_per_thread"] = r.pixels_per_thread
    out["render_fwd_one_pixel_a_thread_ms"] = _one_pixel_a_thread(r, d, flush, steps, warmup)
    r.render(d["opacity"], "fp32")
    gimg = torch.ones_like(r.out["img"])
    P = len(sc["opacity"])
    grads = dict(dmean2d=torch.zeros(P, 2, device=dev), dconic=torch.zeros(P, 3, device=dev),
                 dopacity=torch.zeros(P, device=dev), drgb=torch.zeros(P, 3, device=dev))
    opts = tc.render_opts("fp32")
    out["render_bwd_ms"] = _events_ms(lambda: tc.tcgs_render_bwd(
        r.cam, opts, r.bins["tile_ranges"], r.bins["ids_sorted"], r.proj["mean2d"], r.proj["conic"], d["opacity"],
        r.proj["rgb"], r.out["img"], r.out["T_final"], r.out["n_contrib"], gimg, grads=grads), 3, 1, flush)
    del r
    torch.cuda.empty_cache()
    out["square_coverage"] = _coverage_render(cam, d, n + 1024, dev, flush, exact=False, steps=steps, warmup=warmup)
    return out


def _one_pixel_a_thread(r, d, flush, steps, warmup):
    """Render times of the tile kernel with one pixel a consumer thread (8 x 4 warp blocks), beside the
    Renderer's own choice (two pixels a thread for views of large footprints); same image."""
    keep = r.pixels_per_thread
    r.pixels_per_thread = 1
    out = {prec: _events_ms(lambda: r.render(d["opacity"], prec), steps, warmup, flush)
           for prec in ("tc_fp16_split", "fp32_frag2mat")}
    r.pixels_per_thread = keep
    return out


def _coverage_render(cam, d, capacity, dev, flush, exact, steps=10, warmup=3):
    """The same view binned with the given coverage rule: splats, bin_sort and both renderers' times."""
    import torch
    import paper_2505_24796_gb300 as tc
    r = tc.Renderer(cam, d["means3"].shape[0], capacity, device=dev, exact_tiles=exact)
    r.frame(d, precision="fp32")
    torch.cuda.synchronize()
    out = {"splats": int(r.bins["n_splats"].item()),
           "ms": {"bin_sort": _events_ms(lambda: r.bin_sort(), steps, warmup, flush),
                  "render_fwd_tc": _events_ms(lambda: r.render(d["opacity"], "tc_fp16_split"), steps, warmup, flush),
                  "render_fwd_fp32": _events_ms(lambda: r.render(d["opacity"], "fp32"), steps, warmup, flush)}}
    del r
    torch.cuda.empty_cache()
    return out


ABLATION = [
    # (label, precision, early_cull, tile_cull): Table 4 (EarlyCull x Frag2Mat with G2L) ...
    ("fp32", "fp32", False, True),
    ("fp32+earlycull", "fp32", True, True),
    # the tensor-core renderer with its product u^T v on CUDA cores in FP32: the same schedule, staging,
    # block marks and EarlyCull, so against the rows below only the tensor-core product differs
    ("fp32_frag2mat_g2l+earlycull", "fp32_frag2mat", True, False),
    ("fp32_frag2mat_g2l+earlycull+block_marks", "fp32_frag2mat", True, True),
    ("frag2mat_g2l_fp16", "tc_fp16", False, False),
    ("frag2mat_g2l_fp16+earlycull", "tc_fp16", True, False),
    ("frag2mat_g2l_fp16+earlycull+block_marks", "tc_fp16", True, True),
    # ... Table 5 (Frag2Mat without G2L) and the other encodings of this renderer
    ("frag2mat_global_fp16", "tc_fp16_global", True, False),
    ("frag2mat_global_tf32", "tc_tf32_global", True, False),
    ("frag2mat_g2l_tf32", "tc_tf32", True, True),
    ("frag2mat_g2l_fp8_split", "tc_fp8", True, True),
    ("frag2mat_g2l_fp16_split", "tc_fp16_split", True, True),
]


def bench_ablation(r, dsc, flush, img32, oracle_img=None, mask=None, reps=10, warmup=3):
    """Render-stage time and accuracy of each configuration of ABLATION on one frame's bins."""
    import torch
    out = {}
    ref32 = img32.cpu().numpy().astype(np.float64)
    for label, prec, ec, tcull in ABLATION:
        fn = lambda: r.render(dsc["opacity"], prec, early_cull=ec, tile_cull=tcull)
        ms = _events_ms(fn, reps, warmup, flush)
        fn()
        torch.cuda.synchronize()
        im = r.out["img"].cpu().numpy().astype(np.float64)
        row = {"precision": prec, "early_cull": ec,
               "block_marks": tcull and prec != "fp32" and not prec.endswith("_global"),
               "render_ms": ms, "finite": bool(np.isfinite(im).all())}
        mse = float(np.mean((im - ref32) ** 2))
        row["psnr_vs_fp32_db"] = 10 * math.log10(1 / mse) if mse > 0 else None
        if oracle_img is not None:
            d = (im - oracle_img)[:, mask]
            mse = float(np.mean(d ** 2))
            row["psnr_vs_oracle_db"] = 10 * math.log10(1 / mse) if mse > 0 else None
            row["within_2e-3_vs_oracle"] = float((np.abs(d).max(axis=0) <= 2e-3).mean())
        out[label] = row
    base = out["fp32"]["render_ms"]
    for row in out.values():
        row["speedup_vs_fp32"] = base / row["render_ms"]
    return out


def time_frames(r, dsc, precision, steps, warmup, use_graph, flush, stream):
    """Frames of renderer r (project -> bin_sort -> render); L2 flushed before every timed frame,
    outside the events.  With graphs, the frame time comes from one CUDA graph holding the whole
    frame (as a renderer would replay it), and the stage times from a second set of steps with one
    graph per stage and events between them.  Returns the frame times and the per-stage times (ms)."""
    import torch
    fns = [lambda: r.project(dsc), lambda: r.bin_sort(), lambda: r.render(dsc["opacity"], precision)]
    frame = None
    if use_graph:
        for f in fns:
            f()
        torch.cuda.synchronize()
        graphs = []
        for f in fns:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                f()
            graphs.append(g)
        run = [g.replay for g in graphs]
        gf = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gf):
            for f in fns:
                f()
        frame = gf.replay
    else:
        run = fns
    for _ in range(warmup):
        for f in run:
            f()
        if frame is not None:
            frame()
    torch.cuda.synchronize()
    per_stage = [[] for _ in run]
    total = []
    for _ in range(steps):
        flush.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(run) + 1)]
        ev[0].record(stream)
        for i, f in enumerate(run):
            f()
            ev[i + 1].record(stream)
        ev[-1].synchronize()
        for i in range(len(run)):
            per_stage[i].append(ev[i].elapsed_time(ev[i + 1]))
        total.append(ev[0].elapsed_time(ev[-1]))
    if frame is not None:
        total = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            frame()
            e1.record(stream)
            e1.synchronize()
            total.append(e0.elapsed_time(e1))
    return total, per_stage


def time_frames_two_in_flight(renderers, dsc, precision, frames, warmup, flush):
    """Throughput of a stream of independent frames with two in flight: renderer i (own buffers) replays
    its whole-frame CUDA graph on its own stream, frames alternating between the two, so one frame's
    sort can overlap the other's render.  L2 flushed once before the timed frames.  Returns ms per frame."""
    import torch
    streams = [torch.cuda.Stream() for _ in renderers]
    graphs = []
    for r, st in zip(renderers, streams):
        with torch.cuda.stream(st):
            r.frame(dsc, precision=precision)
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=st):
                r.frame(dsc, precision=precision)
        graphs.append(g)
    torch.cuda.synchronize()

    def run(n):
        for i in range(n):
            k = i % len(graphs)
            with torch.cuda.stream(streams[k]):
                graphs[k].replay()
    run(warmup)
    torch.cuda.synchronize()
    flush.zero_()
    start = torch.cuda.Event(enable_timing=True)
    start.record()
    for st in streams:
        st.wait_event(start)
    run(frames)
    ends = []
    for st in streams:
        e = torch.cuda.Event(enable_timing=True)
        e.record(st)
        ends.append(e)
    torch.cuda.synchronize()
    return max(start.elapsed_time(e) for e in ends) / frames


def bench_tight_radius(cam, sc, dsc, dev, flush, with_oracle=True, reps=20, warmup=5):
    """The same frame binned with the opacity-aware coverage square (Gaussians cover only the
    tiles where alpha >= 1/255 is possible): splats and stage times, and the image against the
    oracle run with the same coverage on a sample of tiles."""
    import torch
    import paper_2505_24796_gb300 as tc
    P = len(sc["opacity"])
    pr = tc.tcgs_project(cam, dsc["means3"], dsc["scales"], dsc["quats"], dsc["sh"], dsc["sh_degree"],
                         opacity=dsc["opacity"])
    n = int(pr["tiles_touched"].to(torch.int64).sum().item())
    del pr
    r = tc.Renderer(cam, P, n + 1024, device=dev, tight_radius=True, exact_tiles=False)
    tot, stg = time_frames(r, dsc, "tc_fp16_split", reps, warmup, True, flush, torch.cuda.current_stream(dev))
    ms = dict(zip(["project", "bin_sort", "render_fwd"], [statistics.mean(x) for x in stg]))
    r.frame(dsc, precision="tc_fp16_split")
    torch.cuda.synchronize()
    out = {"splats": n, "stages_ms": ms, "frame_ms": statistics.mean(tot),
           "frames_per_s": 1000.0 / statistics.mean(tot)}
    if with_oracle:
        import oracle
        s64 = {k: (v.astype(np.float64) if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
        po = oracle.project(cam, s64, tight_radius=True)
        b = oracle.bin_sort(cam, po["mean2d"], po["radius"], po["depth"])
        gw, gh = oracle.grid(cam)
        tiles = np.random.default_rng(7).choice(gw * gh, (gw * gh) // 8, replace=False)
        o = oracle.render(cam, b, po["mean2d"], po["conic"], s64["opacity"], po["rgb"], tiles=tiles, margins=False)
        H, W = cam["height"], cam["width"]
        mask = np.zeros((H, W), bool)
        for t in tiles:
            ty, tx = divmod(int(t), gw)
            mask[16 * ty:16 * ty + 16, 16 * tx:16 * tx + 16] = True
        d = (r.out["img"].cpu().numpy().astype(np.float64) - o["img"])[:, mask]
        mse = float(np.mean(d ** 2))
        out["oracle_splats"] = int(b["n"])
        out["psnr_vs_oracle_db"] = 10 * math.log10(1 / mse) if mse > 0 else None
        out["within_2e-3_vs_oracle"] = float((np.abs(d).max(axis=0) <= 2e-3).mean())
        out["oracle_pixels_compared"] = int(mask.sum())
    del r
    return out


# ------------------------------------------------------------------ ranks

def max_over_ranks(x: float, device=None) -> float:
    """The largest x over the ranks of the default process group (x itself without one): the step
    time of the slowest replica."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(ms_slowest: float, world: int) -> float:
    """Whole-job frames/s: every replica renders one frame per step, so world frames per step of
    the slowest replica."""
    return world * 1000.0 / ms_slowest


def barrier_if_distributed():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


# ------------------------------------------------------------------ GPU arm

def run_tcgs(args):
    import torch
    import torch.distributed as dist

    import paper_2505_24796_gb300 as tc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lib = tc._lib.load()

    cam, sc = workload(args.scale)
    P = len(sc["opacity"])
    dsc = tc.scene_to_device(sc, dev)
    H, W = cam["height"], cam["width"]

    # --- setup (untimed): splat count and capacity, fragment classes from the FP32 counters
    probe = tc.tcgs_project(cam, dsc["means3"], dsc["scales"], dsc["quats"], dsc["sh"], dsc["sh_degree"])
    n_splats = int(probe["tiles_touched"].to(torch.int64).sum().item())
    capacity = n_splats + 1024
    exact = args.coverage == "exact"
    r = tc.Renderer(cam, P, capacity, device=dev, stats=True, exact_tiles=exact)
    r.frame(dsc, precision="fp32")
    torch.cuda.synchronize()
    n_binned = int(r.bins["n_splats"].item())
    st = r.stats.to(torch.int64).sum(dim=0).tolist()
    f_blend, f_cull, slots_fp32 = st[0], st[1], st[2]
    alpha_evals = f_blend + f_cull
    img_fp32 = r.out["img"].clone()
    r.stats.zero_()
    r.frame(dsc, precision=args.precision)
    torch.cuda.synchronize()
    st_tc = r.stats.to(torch.int64).sum(dim=0).tolist()
    img_tc = r.out["img"].clone()
    status = (int(r.bins["status"].item()), int(r.device_status.item()))
    r.stats = None  # no counters in the timed region

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (126 MB)
    stream = torch.cuda.current_stream(dev)

    use_graph = not args.no_graph
    # --- FP32 comparison paths: the 3DGS baseline kernel, and the tensor-core renderer with its product on
    # CUDA cores (same schedule, block marks and EarlyCull: only the tensor-core product differs)
    tot32, st32 = time_frames(r, dsc, "fp32", args.steps, args.warmup, use_graph, flush, stream)
    totcc, stcc = time_frames(r, dsc, "fp32_frag2mat", args.steps, args.warmup, use_graph, flush, stream)
    # --- headline path, with clocks sampled during the timed region; a barrier and a device
    # synchronisation on both sides of it
    barrier_if_distributed()
    torch.cuda.synchronize()
    l0 = lib.tcgs_kernel_launches()
    with ClockSampler(local) as clk:
        tot, stg = time_frames(r, dsc, args.precision, args.steps, args.warmup, use_graph, flush, stream)
    launches_total = lib.tcgs_kernel_launches() - l0
    torch.cuda.synchronize()
    barrier_if_distributed()
    # launches per frame, counted by the library on one eager frame (graphs replay the same kernels)
    l1 = lib.tcgs_kernel_launches()
    r.frame(dsc, precision=args.precision)
    torch.cuda.synchronize()
    launches_per_frame = lib.tcgs_kernel_launches() - l1
    ms = max_over_ranks(statistics.mean(tot), dev)
    fps = job_rate(ms, world)
    ms32 = statistics.mean(tot32)
    render_ms = statistics.mean(stg[2])
    render32_ms = statistics.mean(st32[2])

    # --- two independent frames in flight on two streams (a serving loop's throughput), beside the
    # per-frame figure above
    r2 = tc.Renderer(cam, P, capacity, device=dev, exact_tiles=exact)
    two_ms = {prec: time_frames_two_in_flight([r, r2], dsc, prec, 4 * args.steps, args.warmup, flush)
              for prec in (args.precision, "fp32")}
    del r2

    # --- end to end through the public API with host buffers: every frame's scene goes host -> device
    # from pinned memory and its image device -> host, in the timed region; FramePipeline overlaps
    # frame i + 1's upload with frame i's render (the scene, 236 MB, exceeds L2, so no flush is needed)
    pinned = tc.FramePipeline.pinned_scene(sc)   # the scene's arrays in one pinned buffer: one copy a frame
    host_imgs = [torch.empty(3, H, W, dtype=torch.float32).pin_memory() for _ in range(2)]
    h2d = pinned["_buffer"].numel()
    d2h = host_imgs[0].numel() * 4
    pipe = tc.FramePipeline(r, precision=args.precision)
    for i in range(args.warmup):
        pipe.submit(pinned, host_imgs[i & 1])
    pipe.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(pipe.compute_stream)
    pipe.copy_stream.wait_event(e0)
    pipe.d2h_stream.wait_event(e0)
    for i in range(args.steps):
        pipe.submit(pinned, host_imgs[i & 1])
    pipe.compute_stream.wait_stream(pipe.d2h_stream)
    e1.record(pipe.compute_stream)
    e1.synchronize()
    e2e_ms = [e0.elapsed_time(e1) / args.steps]
    e2e_img_ok = bool(torch.equal(host_imgs[(args.steps - 1) & 1], img_tc.cpu()))
    e2e_fps = job_rate(max_over_ranks(statistics.mean(e2e_ms), dev), world)

    if world > 1:
        dist.barrier()
    if rank != 0:
        dist.destroy_process_group()
        return

    # --- accuracy of this frame: TC vs FP32 on the GPU, and vs the FP64 oracle on the sampled tiles
    oimg, mask = None, None
    img_tc_np = img_tc.cpu().numpy().astype(np.float64)
    img32_np = img_fp32.cpu().numpy().astype(np.float64)
    mse_tc_fp32 = float(np.mean((img_tc_np - img32_np) ** 2))
    cpu_baseline = cpu_all = None
    acc = {"psnr_tc_vs_fp32_db": (10 * math.log10(1 / mse_tc_fp32) if mse_tc_fp32 > 0 else None)}
    if not args.no_cpu_baseline and world == 1:   # the host-core baseline is taken at N = 1 only
        s64 = _scene64(sc)
        t1, info = oracle_frame_single(cam, s64)
        t2, _ = oracle_frame_single(cam, s64)
        est = 0.5 * (t1 + t2)
        cpu_baseline = {"value": 1.0 / est, "unit": "frames/s", "cores": 1, "kind": "oracle",
                        "sample": f"two whole frames: FP64 projection + binning of the whole scene and "
                                  f"Algorithm 1 on all {info['tiles']} tiles, mean of the two; "
                                  f"{t1 + t2:.1f} s of CPU work"}
        mask = np.ones((H, W), bool)
        oimg = info["img"]
        for name, im in (("tc", img_tc_np), ("fp32", img32_np)):
            d = (im - oimg)[:, mask]
            mse = float(np.mean(d ** 2))
            acc[f"psnr_{name}_vs_oracle_db"] = 10 * math.log10(1 / mse) if mse > 0 else None
            acc[f"within_2e-3_{name}"] = float((np.abs(d).max(axis=0) <= 2e-3).mean())
            acc[f"max_abs_{name}"] = float(np.abs(d).max())
        acc["oracle_pixels_compared"] = int(mask.sum())
        try:   # the same oracle on every host core, reported beside the single-thread baseline
            t_all, n_thr, img_all = oracle_frame_all_cores(cam, s64)
            cpu_all = {"value": 1.0 / t_all, "unit": "frames/s", "cores": n_thr, "kind": "oracle",
                       "sample": f"one whole frame: FP64 projection + binning (single-threaded, as the oracle "
                                 f"stands) and Algorithm 1 on all {info['tiles']} tiles dealt to {n_thr} threads",
                       "image_equals_single_thread_frame": bool(np.array_equal(img_all, oimg))}
        except Exception as e:   # report, do not hide: the headline line is still printed
            cpu_all = {"error": f"{type(e).__name__}: {e}"}
    ablation = tight = other = None
    if not args.no_extras:
        # the same frame binned with the other coverage rule, both renderers; the ablation of Tables 4
        # and 5 runs on the paper's lists (3-sigma squares)
        r_o = tc.Renderer(cam, P, capacity, device=dev, exact_tiles=not exact)
        r_o.frame(dsc, precision="fp32")
        torch.cuda.synchronize()
        other = {"coverage": "square" if exact else "exact", "splats": int(r_o.bins["n_splats"].item())}
        img_o32 = r_o.out["img"].clone()
        for prec in (args.precision, "fp32"):
            tq, sq = time_frames(r_o, dsc, prec, args.steps, args.warmup, use_graph, flush, stream)
            other[prec] = {"frames_per_s": 1000.0 / statistics.mean(tq),
                           "stages_ms": dict(zip(["project", "bin_sort", "render_fwd"],
                                                 [statistics.mean(x) for x in sq]))}
        r_o.frame(dsc, precision=args.precision)
        torch.cuda.synchronize()
        other["images_equal_headline"] = {args.precision: bool(torch.equal(r_o.out["img"], img_tc)),
                                          "fp32": bool(torch.equal(img_o32, img_fp32))}
        r_sq = r_o if exact else r
        r_sq.frame(dsc, precision="fp32")
        ablation = bench_ablation(r_sq, dsc, flush, r_sq.out["img"].clone(), oimg, mask)
        del r_o, r_sq
        tight = bench_tight_radius(cam, sc, dsc, dev, flush, with_oracle=not args.no_cpu_baseline)

    # --- roofline of the dominant kernel
    peaks, peak_src = load_peaks()
    stage_names = ["project", "bin_sort", "render_fwd"]
    stage_ms = [statistics.mean(s) for s in stg]
    # the dominant kernel: k_render_tc is the longest single launch of the frame (bin_sort is a stage
    # of 17 launches, the longest of them a tenth of the render in the ncu launch list)
    dominant = "render_fwd"
    ops = alpha_evals * 1 + f_blend * 8   # EarlyCull compare per evaluated fragment + 8 FP32 ops per blend
    alu_peak = SM_COUNT * SM_LANES * SM_MAX_MHZ * 1e6 / 1e12   # thread-ops/s at max clock, TOP/s
    rl_render = {"bound": "alu", "achieved": ops / (render_ms * 1e-3) / 1e12, "peak": alu_peak, "unit": "TOP/s",
                 "traffic": ncu_traffic("k_render_tc", args.scale), "kernel": "k_render_tc",
                 "tensor_tflops": 12 * alpha_evals / (render_ms * 1e-3) / 1e12,
                 # a 0.23 ms kernel inside a 0.5 ms frame: the burst peak (a kernel timed alone)
                 "tensor_peak_tflops": peaks.get("bf16_tflops"),
                 "peak_source": f"alu: {SM_COUNT} SMs x {SM_LANES} lanes x {SM_MAX_MHZ:.0f} MHz; tensor: {peak_src}"}
    rl_render["frac"] = rl_render["achieved"] / rl_render["peak"]
    rl_render["tensor_frac"] = rl_render["tensor_tflops"] / rl_render["tensor_peak_tflops"]
    # what bounds it: instruction issue (warp instructions from the capture over the live time, against
    # 4 issue slots per SM per clock)
    # the special-function unit: one ex2 per walked (pixel, Gaussian) slot, against its throughput
    # measured here (tcgs_microbench_ex2: 8 blocks of 256 threads per SM, 8 independent chains each)
    ex2_out = torch.empty(SM_COUNT * 8 * 256, dtype=torch.float32, device=dev)
    tc.tcgs_microbench_ex2(ex2_out, SM_COUNT * 8, 256)
    torch.cuda.synchronize()
    ex2_rate = 0.0
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        n_ex2 = tc.tcgs_microbench_ex2(ex2_out, SM_COUNT * 8, 2048)
        e1.record()
        e1.synchronize()
        ex2_rate = max(ex2_rate, n_ex2 / (e0.elapsed_time(e1) * 1e-3) / 1e9)
    walked_slots = st_tc[2]
    rl_render["sfu"] = {"achieved": walked_slots / (render_ms * 1e-3) / 1e9, "peak": ex2_rate, "unit": "G ex2/s",
                        "frac": walked_slots / (render_ms * 1e-3) / 1e9 / ex2_rate,
                        "source": "one ex2 per walked slot (the TC path's executed fragment slots); peak measured "
                                  "in this run by tcgs_microbench_ex2"}
    n_inst = ncu_traffic("k_render_tc", args.scale, key="warp_instructions")
    if n_inst is not None:
        issue_peak = SM_COUNT * 4 * SM_MAX_MHZ * 1e6 / 1e9
        rl_render["issue"] = {"achieved": n_inst / (render_ms * 1e-3) / 1e9, "peak": issue_peak,
                              "unit": "G warp-instr/s", "frac": n_inst / (render_ms * 1e-3) / 1e9 / issue_peak,
                              "source": "smsp__inst_executed.sum of the capture; 152 SMs x 4 schedulers x max clock"}
    tile_bits = max(1, math.ceil(math.log2(r.num_tiles)))
    tpasses = 1 if tile_bits <= 8 else (2 if tile_bits <= 16 else 3)
    bin_bytes = P * (4 * 20 + 8 + 24) + n_binned * (8 + tpasses * 20 + 8)
    rl_bin = {"bound": "hbm", "achieved": bin_bytes / (stage_ms[1] * 1e-3) / 1e9, "peak": peaks["hbm_gbs"],
              "unit": "GB/s", "traffic": None, "kernel": "tcgs_bin_sort (whole stage)",
              "peak_source": peak_src}
    rl_bin["frac"] = rl_bin["achieved"] / rl_bin["peak"]
    proj_bytes = P * (12 + 12 + 16 + 192 + 44)
    rl_proj = {"bound": "hbm", "achieved": proj_bytes / (stage_ms[0] * 1e-3) / 1e9, "peak": peaks["hbm_gbs"],
               "unit": "GB/s", "traffic": None, "kernel": "k_project", "peak_source": peak_src}
    rl_proj["frac"] = rl_proj["achieved"] / rl_proj["peak"]
    roof = {"project": rl_proj, "bin_sort": rl_bin, "render_fwd": rl_render}[dominant]

    extras = {}
    if not args.no_extras:
        del r
        torch.cuda.empty_cache()
        for name, fn in (("plain", lambda: bench_plain(dev, flush, stream)),
                         ("differentiation", lambda: bench_differentiation(dev, flush)),
                         ("scheduler", lambda: bench_scheduler(dev, args.sched_train_views)),
                         ("scheduler_occluded", lambda: bench_scheduler_occluded(dev, args.sched_train_views)),
                         ("large", lambda: bench_large(dev, flush))):
            try:
                extras[name] = fn()
            except Exception as e:   # report, do not hide: the headline line is still printed
                extras[name] = {"error": f"{type(e).__name__}: {e}"}
            torch.cuda.empty_cache()

    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f16 tensor-core exponent, f32 accumulate and blend", "data": "synthetic",
        "config": {"workload": WORKLOAD, "P": P, "splats": n_binned, "splats_3sigma_square": n_splats,
                   "coverage": args.coverage, "precision": args.precision,
                   "l2": "flushed (256 MB write) between timed steps, outside the events",
                   "cuda_graph": "one graph per frame; stage times from one graph per stage" if use_graph else False, "parallelism": "replicas" if world > 1 else "single GPU"},
        "alpha_evals_per_frame": alpha_evals, "f_blend": f_blend, "f_cull": f_cull,
        "alpha_evals_per_s": alpha_evals / (render_ms * 1e-3),
        "stages_ms": dict(zip(stage_names, stage_ms)),
        "fp32": {"frames_per_s": 1000.0 / ms32, "ms_per_step": ms32,
                 "stages_ms": dict(zip(stage_names, [statistics.mean(s) for s in st32])),
                 "alpha_evals_per_s": alpha_evals / (render32_ms * 1e-3)},
        "fp32_same_skip": {"frames_per_s": 1000.0 / statistics.mean(totcc), "ms_per_step": statistics.mean(totcc),
                           "stages_ms": dict(zip(stage_names, [statistics.mean(s) for s in stcc])),
                           "kernel": "k_render_tc with the product u^T v on CUDA cores (TCGS_FP32_FRAG2MAT)"},
        "two_frames_in_flight": {"frames_per_s": {k: 1000.0 / v for k, v in two_ms.items()},
                                 "note": "independent frames alternating between two renderers and two streams, "
                                         "each frame one CUDA graph; the headline value is one frame at a time"},
        "speedup_vs_fp32": {"frame": ms32 / ms, "render": render32_ms / render_ms,
                            "render_vs_same_skip": statistics.mean(stcc[2]) / render_ms},
        "accuracy": acc, "status": {"bin_sort": status[0], "render": status[1]},
        "executed_fragment_slots": {"fp32": slots_fp32, "tc": st_tc[2]},
        "roofline": roof, "roofline_all": {"project": rl_proj, "bin_sort": rl_bin, "render_fwd": rl_render},
        "cpu_baseline": cpu_baseline, "cpu_baseline_all_cores": cpu_all,
        "e2e": {"value": e2e_fps, "unit": "frames/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "pipelined": "FramePipeline: frame i+1's host->device upload (one copy of the scene's pinned "
                             "buffer) overlaps frame i's render",
                "image_matches_device_frame": e2e_img_ok},
        "gpu_launches": int(launches_per_frame * args.steps), "gpu_launches_per_frame": int(launches_per_frame),
        "gpu_launches_counted_in_capture": int(launches_total),
        "clocks": clocks,
        "workloads": extras,
        "ablation": ablation,
        "tight_radius": tight,
        "other_coverage": other,
    }
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def run_large_frames(args):
    """Two frames (project, bin_sort, TC render, FP32 render) of the 3840x2160 large-workload
    distribution with args.large_frames Gaussians: the small case for ncu captures of that workload."""
    import torch
    import paper_2505_24796_gb300 as tc
    from paper_2505_24796_gb300 import scenes
    cam, sc = scenes.large(P=args.large_frames)
    d = tc.scene_to_device(sc, "cuda")
    pr = tc.tcgs_project(cam, d["means3"], d["scales"], d["quats"], d["sh"], d["sh_degree"])
    n = int(pr["tiles_touched"].to(torch.int64).sum().item())
    del pr
    r = tc.Renderer(cam, len(sc["opacity"]), n + 1024, device="cuda")
    steps = [("project", lambda: r.project(d)), ("bin_sort", lambda: r.bin_sort()),
             ("render_tc", lambda: r.render(d["opacity"], "tc_fp16_split")),
             ("render_fp32", lambda: r.render(d["opacity"], "fp32"))]
    for frame in range(2):
        ms = {}
        for name, fn in steps:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            ms[name] = e0.elapsed_time(e1)
        print(json.dumps({"large_frames": args.large_frames, "frame": frame, "rect_tiles": n,
                          "splats": int(r.bins["n_splats"].item()), "ms": ms}), flush=True)


def run_diff_frames(args):
    """Two frames of the differentiation workload (1280x720, 500k Gaussians): project, bin_sort, FP32
    render, render backward (L1 loss to the seeded target), projection backward: the small case for
    ncu captures of the backward."""
    import torch
    import paper_2505_24796_gb300 as tc
    from paper_2505_24796_gb300 import scenes
    cam, sc, target = scenes.differentiation()
    d = tc.scene_to_device(sc, "cuda")
    pr = tc.tcgs_project(cam, d["means3"], d["scales"], d["quats"], d["sh"], d["sh_degree"])
    n = int(pr["tiles_touched"].to(torch.int64).sum().item())
    del pr
    P = len(sc["opacity"])
    r = tc.Renderer(cam, P, n + 1024, device="cuda")
    tgt = torch.from_numpy(target).to("cuda")
    grads = dict(dmean2d=torch.zeros(P, 2, device="cuda"), dconic=torch.zeros(P, 3, device="cuda"),
                 dopacity=torch.zeros(P, device="cuda"), drgb=torch.zeros(P, 3, device="cuda"))
    g3 = dict(dmeans3=torch.zeros_like(d["means3"]), dscales=torch.zeros_like(d["scales"]),
              dquats=torch.zeros_like(d["quats"]), dsh=torch.zeros_like(d["sh"]))
    opts = tc.render_opts("fp32")
    gimg = {}

    def render_bwd():
        gimg["g"] = torch.sign(r.out["img"] - tgt).contiguous()
        tc.tcgs_render_bwd(r.cam, opts, r.bins["tile_ranges"], r.bins["ids_sorted"], r.proj["mean2d"],
                           r.proj["conic"], d["opacity"], r.proj["rgb"], r.out["img"], r.out["T_final"],
                           r.out["n_contrib"], gimg["g"], grads=grads)

    steps = [("project", lambda: r.project(d)), ("bin_sort", lambda: r.bin_sort()),
             ("render_fp32", lambda: r.render(d["opacity"], "fp32")), ("render_bwd", render_bwd),
             ("project_bwd", lambda: tc.tcgs_project_bwd(r.cam, d["means3"], d["scales"], d["quats"], d["sh"],
                                                         d["sh_degree"], r.proj["radius"], grads["dmean2d"],
                                                         grads["dconic"], grads["drgb"], grads=g3))]
    for frame in range(2):
        ms = {}
        for name, fn in steps:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            ms[name] = e0.elapsed_time(e1)
        print(json.dumps({"diff_frames": P, "frame": frame, "splats": int(r.bins["n_splats"].item()), "ms": ms}),
              flush=True)


def run_render_arms(args):
    """The headline frame (or the differentiation frame, --arms-workload), projected and binned once,
    then rendered twice by each renderer arm in turn: the small case for ncu captures comparing the
    arms' kernels."""
    import torch
    import paper_2505_24796_gb300 as tc
    from paper_2505_24796_gb300 import scenes
    cam, sc = workload(args.scale) if args.arms_workload == "precision" else scenes.differentiation()[:2]
    d = tc.scene_to_device(sc, "cuda")
    pr = tc.tcgs_project(cam, d["means3"], d["scales"], d["quats"], d["sh"], d["sh_degree"])
    n = int(pr["tiles_touched"].to(torch.int64).sum().item())
    del pr
    r = tc.Renderer(cam, len(sc["opacity"]), n + 1024, device="cuda", exact_tiles=args.coverage == "exact")
    r.project(d)
    r.bin_sort()
    torch.cuda.synchronize()
    for rep in range(2):
        ms = {}
        for prec in ("tc_fp16_split", "fp32_frag2mat", "fp32"):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            r.render(d["opacity"], prec)
            e1.record()
            e1.synchronize()
            ms[prec] = e0.elapsed_time(e1)
        print(json.dumps({"render_arms": rep, "splats": int(r.bins["n_splats"].item()), "ms": ms}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.large_frames > 0:
        run_large_frames(args)
    elif args.diff_frames:
        run_diff_frames(args)
    elif args.render_arms:
        run_render_arms(args)
    else:
        run_tcgs(args)


if __name__ == "__main__":
    main()
