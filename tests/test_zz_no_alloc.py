"""tcgs_bin_sort_noalloc: the bin/sort stage for callers that cannot allocate device memory.

Such callers (a host application that owns every allocation, a latency-critical loop where
cudaMalloc would synchronise the device, a plain C caller without a CUDA allocator) pass only
inputs and outputs; the library works in a static scratch array of its own.  These tests call the
entry point through the C ABI several times in a row, on different inputs, and check each result
against the ordinary tcgs_bin_sort with a caller workspace.  Binning is integer work, so the
comparison is exact.  The cases cover both code paths of the sort: the single-CTA passes of small
views (at most 256 tiles, P <= 8192, capacity <= 32768) and the multi-block radix passes, the
larger multi-block case first so that the next call starts from the scratch words it left behind.
The file is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda"


def _inputs(seed, P, width, height, rmax=24):
    from paper_2505_24796_gb300 import scenes
    rng = np.random.default_rng(seed)
    cam = scenes.pinhole(width, height, fx=float(width))
    mean2d = np.c_[rng.uniform(-20, width + 20, P), rng.uniform(-20, height + 20, P)].astype(np.float32)
    radius = rng.integers(0, rmax, P).astype(np.int32)
    depth = rng.uniform(0.5, 30.0, P).astype(np.float32)
    depth[::7] = depth[0]   # exact depth ties
    return cam, (torch.from_numpy(mean2d).to(DEV), torch.from_numpy(radius).to(DEV), torch.from_numpy(depth).to(DEV))


def _noalloc(tc, lib, c, P, m, r, d, cap):
    nt = tc.grid(c)[0] * tc.grid(c)[1]
    ids = torch.full((cap,), -7, dtype=torch.int32, device=DEV)
    ranges = torch.full((nt, 2), -7, dtype=torch.int32, device=DEV)
    n_dev = torch.full((1,), -7, dtype=torch.int64, device=DEV)
    st = torch.full((1,), -7, dtype=torch.int32, device=DEV)
    code = lib.tcgs_bin_sort_noalloc(ctypes.byref(c), P, m.data_ptr(), r.data_ptr(), d.data_ptr(), cap,
                                     ids.data_ptr(), ranges.data_ptr(), n_dev.data_ptr(), st.data_ptr(),
                                     torch.cuda.current_stream().cuda_stream)
    return code, ids, ranges, n_dev, st


# (seed, P, width, height, max radius): multi-block path (640x480 = 1200 tiles; 30,000 Gaussians),
# a smaller multi-block case after it, then two single-CTA cases
CASES = [(104, 30_000, 640, 480, 40), (105, 9000, 400, 300, 24), (101, 6000, 333, 190, 24),
         (102, 1500, 128, 128, 24)]


def test_noalloc_matches_bin_sort_on_consecutive_calls():
    import paper_2505_24796_gb300 as tc
    lib = tc._lib.load()
    for seed, P, w, h, rmax in CASES:
        cam, (m, r, d) = _inputs(seed, P, w, h, rmax)
        c = tc.make_camera(cam)
        # reference: the existing entry point with a caller-allocated workspace
        probe = tc.tcgs_bin_sort(c, m, r, d, capacity=0)
        torch.cuda.synchronize()
        n = int(probe["n_splats"].item())
        cap = n + 5
        nt = tc.grid(c)[0] * tc.grid(c)[1]
        small = nt <= 256 and P <= 8192 and cap <= 32768
        assert small == (seed in (101, 102)), (seed, nt, P, cap)   # both sort paths are covered
        ref = tc.tcgs_bin_sort(c, m, r, d, capacity=cap)
        code, ids, ranges, n_dev, st = _noalloc(tc, lib, c, P, m, r, d, cap)
        assert code == tc._lib.TCGS_OK, lib.tcgs_status_string(code)
        torch.cuda.synchronize()
        assert int(st.item()) == int(ref["status"].item()) == 0
        assert int(n_dev.item()) == int(ref["n_splats"].item()) == n
        assert torch.equal(ids[:n], ref["ids_sorted"][:n])
        assert torch.equal(ranges, ref["tile_ranges"])
        assert int(ids[n:].eq(-7).sum().item()) == cap - n   # nothing written past N


def test_noalloc_allocates_no_device_memory():
    """After a first call (which loads the module and looks up the scratch address), further calls
    change neither the device's free memory nor torch's allocated bytes."""
    import paper_2505_24796_gb300 as tc
    lib = tc._lib.load()
    seed, P, w, h, rmax = CASES[0]
    cam, (m, r, d) = _inputs(seed, P, w, h, rmax)
    c = tc.make_camera(cam)
    cap = 1_000_000
    nt = tc.grid(c)[0] * tc.grid(c)[1]
    ids = torch.empty(cap, dtype=torch.int32, device=DEV)
    ranges = torch.empty(nt, 2, dtype=torch.int32, device=DEV)
    n_dev = torch.empty(1, dtype=torch.int64, device=DEV)
    st = torch.empty(1, dtype=torch.int32, device=DEV)
    stream = torch.cuda.current_stream().cuda_stream

    def call():
        return lib.tcgs_bin_sort_noalloc(ctypes.byref(c), P, m.data_ptr(), r.data_ptr(), d.data_ptr(), cap,
                                         ids.data_ptr(), ranges.data_ptr(), n_dev.data_ptr(), st.data_ptr(), stream)
    assert call() == tc._lib.TCGS_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        assert call() == tc._lib.TCGS_OK
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0


def test_noalloc_rejects_requests_beyond_the_scratch_array():
    import paper_2505_24796_gb300 as tc
    lib = tc._lib.load()
    cam, (m, r, d) = _inputs(103, 100, 64, 64)
    c = tc.make_camera(cam)
    too_many = tc._lib.TCGS_BIN_SORT_NOALLOC_SCRATCH_BYTES // 12 + 1   # 12 scratch bytes per splat
    code = lib.tcgs_bin_sort_noalloc(ctypes.byref(c), 100, m.data_ptr(), r.data_ptr(), d.data_ptr(), too_many,
                                     None, None, None, None, None)
    assert code == tc._lib.TCGS_ERR_SCRATCH_LIMIT
    assert b"scratch" in lib.tcgs_status_string(code)
