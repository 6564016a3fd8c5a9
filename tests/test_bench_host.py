"""Host-side parts of bench.py that need no GPU: the oracle timed on every host core renders the
frame the single-thread oracle renders, bit for bit."""
import numpy as np

import bench
import oracle
from paper_2505_24796_gb300 import scenes


def test_oracle_on_all_cores_renders_the_single_thread_frame():
    cam, sc = scenes.plain_forward(P=1500, width=200, height=136, seed=11)   # 117 tiles, ragged edges
    t, threads, img = bench.oracle_frame_all_cores(cam, sc, threads=3)
    assert threads == 3 and t > 0
    s64 = {k: (v.astype(np.float64) if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    pr = oracle.project(cam, s64)
    b = oracle.bin_sort(cam, pr["mean2d"], pr["radius"], pr["depth"])
    ref = oracle.render(cam, b, pr["mean2d"], pr["conic"], s64["opacity"], pr["rgb"], margins=False)["img"]
    assert np.array_equal(img, ref)
    assert ref.max() > 0
