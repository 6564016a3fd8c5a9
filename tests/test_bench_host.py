"""Host-side parts of bench.py that need no GPU: the oracle timed on every host core renders the
frame the single-thread oracle renders, bit for bit."""
import numpy as np

import bench
import oracle
from paper_2505_24796_gb300 import scenes


def test_oracle_on_all_cores_renders_the_single_thread_frame():
    cam, sc = scenes.plain_forward(P=1500, width=200, height=136, seed=11)   # 117 tiles, ragged edges
    s64 = {k: (v.astype(np.float64) if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    t, threads, img = bench.oracle_frame_all_cores(cam, s64, threads=3)
    assert threads == 3 and t > 0
    pr = oracle.project(cam, s64)
    b = oracle.bin_sort(cam, pr["mean2d"], pr["radius"], pr["depth"])
    ref = oracle.render(cam, b, pr["mean2d"], pr["conic"], s64["opacity"], pr["rgb"], margins=False)["img"]
    assert np.array_equal(img, ref)
    assert ref.max() > 0


def test_single_thread_oracle_frame_renders_every_tile():
    cam, sc = scenes.plain_forward(P=500, width=96, height=80, seed=12)
    s64 = bench._scene64(sc)
    t, info = bench.oracle_frame_single(cam, s64)
    _, _, img = bench.oracle_frame_all_cores(cam, s64, threads=2)
    assert t > 0 and info["tiles"] == 6 * 5
    assert np.array_equal(info["img"], img)
