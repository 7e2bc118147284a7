"""integral_images_u32_noalloc(): the variant for callers that cannot
allocate device memory when they need the integral images (applications
that hand out all device memory from their own pool or budget, loops that
cannot afford the synchronisation an allocation may imply).  It must give
exactly what the context-based integral_images_u32() gives, call after call,
although its scratch is one fixed array shared by every call, and it must
allocate nothing.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""

import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu]


@pytest.fixture(scope="module")
def dc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_06513_gb300 import build as dc_build
    dc_build.build()
    from paper_2408_06513_gb300 import declutter
    declutter.load_library()
    return declutter


def _reference(dc, grid_dev, k):
    """The existing, context-based entry point."""
    N = 1 << k
    ctx = dc.declutter_create(k, kernel_r=0)
    try:
        a = torch.empty(N * N, dtype=torch.int64, device="cuda:0")
        at = torch.empty(N * N, dtype=torch.int64, device="cuda:0")
        dc.integral_images_u32(ctx, grid_dev, a, at)
        dc.declutter_sync(ctx)
    finally:
        dc.declutter_destroy(ctx)
    return a.cpu(), at.cpu()


@pytest.mark.parametrize("k", [4, 7, 9, 10])
def test_noalloc_matches_context_path_on_consecutive_calls(dc, k):
    N = 1 << k
    lib = dc.load_library()
    grids = [synth.sat_grid(k, seed=s) for s in (0, 1)]
    for g in grids:
        g_dev = torch.from_numpy(g.view(np.int32)).to("cuda:0")
        ref_a, ref_at = _reference(dc, g_dev, k)
        # two calls in a row through the C ABI: the shared scratch keeps the
        # previous call's contents, which must not leak into the result
        for _ in range(2):
            a = torch.full((N * N,), -1, dtype=torch.int64, device="cuda:0")
            at = torch.full((N * N,), -1, dtype=torch.int64, device="cuda:0")
            st = lib.integral_images_u32_noalloc(ctypes.c_void_p(g_dev.data_ptr()), k,
                                                 ctypes.c_void_p(a.data_ptr()),
                                                 ctypes.c_void_p(at.data_ptr()), None)
            assert st == 0, dc.declutter_last_error()
            torch.cuda.synchronize()
            assert torch.equal(a.cpu(), ref_a)
            assert torch.equal(at.cpu(), ref_at)


def test_noalloc_binding_and_limit(dc):
    k = 8
    N = 1 << k
    g = torch.from_numpy(synth.sat_grid(k).view(np.int32)).to("cuda:0")
    ref_a, ref_at = _reference(dc, g, k)
    a = torch.empty(N * N, dtype=torch.int64, device="cuda:0")
    at = torch.empty(N * N, dtype=torch.int64, device="cuda:0")
    dc.integral_images_u32_noalloc(g, k, a, at)
    torch.cuda.synchronize()
    assert torch.equal(a.cpu(), ref_a) and torch.equal(at.cpu(), ref_at)
    # grids beyond the fixed scratch are refused with a clear message
    lib = dc.load_library()
    big = torch.zeros(1 << 22, dtype=torch.int32, device="cuda:0")
    st = lib.integral_images_u32_noalloc(ctypes.c_void_p(big.data_ptr()), 11, None, None, None)
    assert st == 1
    assert "no-allocation limit" in dc.declutter_last_error()


def test_noalloc_allocates_nothing(dc):
    # after a first call (which looks up the array's address and loads the
    # kernels), calls change neither torch's allocations nor the device's
    # free memory as cudaMemGetInfo reports it
    k = 10
    N = 1 << k
    g = torch.from_numpy(synth.sat_grid(k, seed=3).view(np.int32)).to("cuda:0")
    a = torch.empty(N * N, dtype=torch.int64, device="cuda:0")
    at = torch.empty(N * N, dtype=torch.int64, device="cuda:0")
    dc.integral_images_u32_noalloc(g, k, a, at)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(0)
    used0 = torch.cuda.memory_allocated(0)
    for _ in range(3):
        dc.integral_images_u32_noalloc(g, k, a, at)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(0)
    assert torch.cuda.memory_allocated(0) == used0
    assert free1 == free0, (free0, free1)


def test_noalloc_rejects_memory_of_another_kind_before_launching(dc):
    # the kernels run on the current device: a grid or output that is not
    # device memory of that device is refused before anything is launched
    k = 6
    N = 1 << k
    lib = dc.load_library()
    host = np.zeros(N * N, np.uint32)
    st = lib.integral_images_u32_noalloc(ctypes.c_void_p(host.ctypes.data), k, None, None, None)
    assert st == 1
    assert "not device memory" in dc.declutter_last_error()
    pinned = torch.zeros(N * N, dtype=torch.int64).pin_memory()
    g = torch.zeros(N * N, dtype=torch.int32, device="cuda:0")
    st = lib.integral_images_u32_noalloc(ctypes.c_void_p(g.data_ptr()), k, ctypes.c_void_p(pinned.data_ptr()),
                                         None, None)
    assert st == 1
    assert "alpha_out" in dc.declutter_last_error()
    with pytest.raises((TypeError, ValueError)):
        dc.integral_images_u32_noalloc(g, k, torch.zeros(N * N, dtype=torch.int64))
