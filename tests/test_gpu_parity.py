"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Bars (written here, derived in the design notes):
  * counts and integer integral images: bit-exact;
  * float displacement: max abs error <= 1e-4 pixel per iteration against the
    FP64 oracle on the same float32 inputs;
  * exact-mode displacement: within half an ulp of float32 (relative 2^-24)
    plus 1e-12 of the FP64 value;
  * positions: the displacement bound plus one float32 ulp of storage rounding.
Multi-iteration runs are teacher-forced: every GPU iteration starts from the
oracle's float32 positions of the previous iteration.
"""

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu]

DISP_TOL_PX = 1e-4


@pytest.fixture(scope="module")
def dc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_06513_gb300 import build as dc_build
    dc_build.build()
    from paper_2408_06513_gb300 import declutter
    declutter.load_library()
    return declutter


DEV = "cuda:0"


def to_dev(z):
    return torch.from_numpy(np.ascontiguousarray(z, dtype=np.float32)).to(DEV)


def u32(t, N):
    return t.cpu().numpy().view(np.uint32).reshape(N, N)


def u64(t, N):
    return t.cpu().numpy().view(np.uint64).reshape(N, N)


def gpu_step(dc, ctx, z, want_inims=False):
    """One GPU iteration step by step; returns dict of intermediates."""
    N = ctx.N
    pos = to_dev(z)
    counts = torch.empty(N * N, dtype=torch.int32, device=DEV)
    dens = torch.empty(N * N, dtype=torch.float32, device=DEV) if ctx.params.kernel_r != 0 else None
    disp = torch.empty(2 * N * N, dtype=torch.float32, device=DEV)
    dc.splat_density(ctx, pos, counts_out=counts, density_out=dens)
    out = {}
    if want_inims:
        if ctx.params.kernel_r == 0:
            a = torch.empty(N * N, dtype=torch.int64, device=DEV)
            at = torch.empty(N * N, dtype=torch.int64, device=DEV)
        else:
            a = torch.empty(N * N, dtype=torch.float32, device=DEV)
            at = torch.empty(N * N, dtype=torch.float32, device=DEV)
        dc.integral_images(ctx, a, at)
        out["alpha"], out["alpha_t"] = a, at
    dc.displacement_field(ctx, disp)
    dc.advect_samples(ctx, pos)
    dc.declutter_sync(ctx)
    out["counts"] = u32(counts, N).astype(np.uint64)
    out["density"] = None if dens is None else dens.cpu().numpy().reshape(N, N).astype(np.float64)
    out["D"] = disp.cpu().numpy().reshape(N, N, 2).astype(np.float64)
    out["pos"] = pos.cpu().numpy()
    return out


def pos_tol_px(N):
    return DISP_TOL_PX + N * float(np.spacing(np.float32(1.0)))


def check_iteration(dc, ctx, z, p, exact_disp=False, disp_tol_px=DISP_TOL_PX):
    N = ctx.N
    ref_new, aux = oracle.iterate(z, p, keep=True)
    g = gpu_step(dc, ctx, z)
    assert np.array_equal(g["counts"], aux["counts"])
    if g["density"] is not None:
        scale = max(1.0, float(aux["d_r"].max()))
        assert np.max(np.abs(g["density"] - aux["d_r"])) <= 2e-6 * scale
    err = np.abs(g["D"] - aux["D"])
    if exact_disp:
        assert np.all(err <= 6e-8 * np.abs(aux["D"]) + 1e-12), float(err.max() * N)
    else:
        assert float(err.max()) * N <= disp_tol_px, float(err.max()) * N
    perr = float(np.max(np.abs(g["pos"].astype(np.float64) - ref_new))) * N
    assert perr <= pos_tol_px(N), perr
    return float(err.max()) * N


# --------------------------------------------------------------------------
# Step by step on the 128x128 workload, exact and smoothed
# --------------------------------------------------------------------------

@pytest.mark.parametrize("r", [0, 2])
def test_tiny_teacher_forced_iterations(dc, r):
    z, _ = synth.tiny_mixture()
    p = oracle.Params(log2_res=7, kernel_r=r)
    traj = oracle.regularize(z, p, 4)
    ctx = dc.declutter_create(7, kernel_r=r)
    try:
        for k in range(4):
            check_iteration(dc, ctx, traj[k], p, exact_disp=(r == 0))
    finally:
        dc.declutter_destroy(ctx)


@pytest.mark.parametrize("k,r,band_rows", [(4, 0, 0), (4, 2, 1), (5, 0, 2), (6, 3, 4), (7, 0, 8),
                                           (8, 2, 16), (9, 0, 64), (9, 4, 1),
                                           # heights that do not divide N: a shorter last band
                                           (7, 0, 3), (8, 2, 5), (11, 4, 0), (11, 0, 13)])
def test_sizes_and_band_heights(dc, k, r, band_rows):
    z, _ = synth.tiny_mixture(5003, seed=k + r)
    p = oracle.Params(log2_res=k, kernel_r=r)
    ctx = dc.declutter_create(k, kernel_r=r, band_rows=band_rows)
    try:
        check_iteration(dc, ctx, z, p, exact_disp=(r == 0))
    finally:
        dc.declutter_destroy(ctx)


@pytest.mark.parametrize("r", [0, 2])
def test_integral_images_match_oracle(dc, r):
    k = 7
    N = 1 << k
    z, _ = synth.tiny_mixture(20_000, seed=4)
    ctx = dc.declutter_create(k, kernel_r=r)
    try:
        g = gpu_step(dc, ctx, z, want_inims=True)
    finally:
        dc.declutter_destroy(ctx)
    p = oracle.Params(log2_res=k, kernel_r=r)
    c, d_r = oracle.density(z, p)
    if r == 0:
        a_ref, at_ref = oracle.sat_u64(c.astype(np.uint32))
        assert np.array_equal(u64(g["alpha"], N), a_ref)
        assert np.array_equal(u64(g["alpha_t"], N), at_ref)
    else:
        ims = oracle.inims(d_r)
        C = d_r.sum()
        a = g["alpha"].cpu().numpy().reshape(N, N)
        at = g["alpha_t"].cpu().numpy().reshape(N, N)
        assert np.max(np.abs(a - ims["alpha"])) <= 2e-6 * C
        assert np.max(np.abs(at - ims["alpha_t"])) <= 2e-6 * C


@pytest.mark.parametrize("k", [4, 8, 9, 10, 11])
def test_integral_images_u32_sweep_exact(dc, k):
    N = 1 << k
    grid = synth.sat_grid(k)
    a_ref, at_ref = oracle.sat_u64(grid)
    ctx = dc.declutter_create(k, kernel_r=0)
    try:
        g = torch.from_numpy(grid.view(np.int32)).to(DEV)
        a = torch.empty(N * N, dtype=torch.int64, device=DEV)
        at = torch.empty(N * N, dtype=torch.int64, device=DEV)
        dc.integral_images_u32(ctx, g, a, at)
        dc.declutter_sync(ctx)
    finally:
        dc.declutter_destroy(ctx)
    assert np.array_equal(u64(a, N), a_ref)
    assert np.array_equal(u64(at, N), at_ref)


@pytest.mark.parametrize("k", [12, 13])
def test_integral_images_u32_large_exact(dc, k):
    # the largest grids of the sweep: full comparison, values beyond 2^32
    N = 1 << k
    grid = synth.sat_grid(k)
    a_ref, at_ref = oracle.sat_u64(grid)
    if k == 13:
        assert int(a_ref[-1, -1]) > 2**32
    ctx = dc.declutter_create(k, kernel_r=0)
    try:
        g = torch.from_numpy(grid.view(np.int32)).to(DEV)
        a = torch.empty(N * N, dtype=torch.int64, device=DEV)
        at = torch.empty(N * N, dtype=torch.int64, device=DEV)
        dc.integral_images_u32(ctx, g, a, at)
        dc.declutter_sync(ctx)
        assert np.array_equal(u64(a, N), a_ref)
        assert np.array_equal(u64(at, N), at_ref)
    finally:
        dc.declutter_destroy(ctx)


@pytest.mark.parametrize("k,T", [(7, 1), (7, 64), (8, 2), (9, 5), (10, 7), (11, 64), (11, 14), (12, 1), (12, 16),
                                 (12, 27), (13, 8), (13, 54), (13, 0)])
def test_integral_images_u32_band_heights(dc, k, T):
    # every column layout of the band kernels (4, 8 and 16 columns a thread)
    # and band heights from one row to 64, including heights that do not
    # divide N (a shorter last band) and the automatic height (T = 0)
    N = 1 << k
    grid = synth.sat_grid(k, seed=T)
    a_ref, at_ref = oracle.sat_u64(grid)
    ctx = dc.declutter_create(k, kernel_r=0, band_rows=T)
    try:
        g = torch.from_numpy(grid.view(np.int32)).to(DEV)
        a = torch.empty(N * N, dtype=torch.int64, device=DEV)
        at = torch.empty(N * N, dtype=torch.int64, device=DEV)
        dc.integral_images_u32(ctx, g, a, at)
        dc.declutter_sync(ctx)
        assert np.array_equal(u64(a, N), a_ref)
        assert np.array_equal(u64(at, N), at_ref)
    finally:
        dc.declutter_destroy(ctx)


@pytest.mark.parametrize("k,T", [(7, 4), (9, 64), (12, 32), (13, 64)])
def test_integral_images_u32_wide_bands(dc, k, T):
    # Bands whose sums reach 2^32 take the 64-bit path; the others keep
    # band-local sums in 32 bits while max(grid) * T * N < 2^32.  Bands cycle
    # through: values in [2^31, 2^32); every value at that bound (32-bit path,
    # sums up to 2^32 - 1); the bound plus one pixel one above it (64-bit path).
    N = 1 << k
    rng = np.random.default_rng(100 * k + T)
    grid = synth.sat_grid(k).copy()
    lim = (2**32 - 1) // (T * N)
    for band in range(N // T):
        rows = slice(band * T, (band + 1) * T)
        kind = band % 3
        if kind == 0:
            grid[rows] = rng.integers(2**31, 2**32, size=(T, N), dtype=np.uint64).astype(np.uint32)
        elif kind == 1:
            grid[rows] = lim
        else:
            grid[rows] = lim
            grid[band * T + int(rng.integers(T)), int(rng.integers(N))] = lim + 1
    a_ref, at_ref = oracle.sat_u64(grid)
    ctx = dc.declutter_create(k, kernel_r=0, band_rows=T)
    try:
        g = torch.from_numpy(grid.view(np.int32)).to(DEV)
        a = torch.empty(N * N, dtype=torch.int64, device=DEV)
        at = torch.empty(N * N, dtype=torch.int64, device=DEV)
        dc.integral_images_u32(ctx, g, a, at)
        dc.declutter_sync(ctx)
        assert np.array_equal(u64(a, N), a_ref)
        assert np.array_equal(u64(at, N), at_ref)
    finally:
        dc.declutter_destroy(ctx)


# --------------------------------------------------------------------------
# Options and edge cases
# --------------------------------------------------------------------------

@pytest.mark.parametrize("opts", [
    dict(pixel_center=True),
    dict(clamp_positions=False),
    dict(d0=0.25),
    dict(sigma=1.1),
    dict(carry_mode=1),
])
@pytest.mark.parametrize("r", [0, 3])
def test_options(dc, opts, r):
    if r == 0 and ("sigma" in opts or "carry_mode" in opts):
        pytest.skip("smoothing option")
    k = 7
    z, _ = synth.tiny_mixture(8000, seed=21)
    p = oracle.Params(log2_res=k, kernel_r=r, sigma=opts.get("sigma", 0.0), d0=opts.get("d0", -1.0),
                      pixel_center=opts.get("pixel_center", False),
                      clamp_positions=opts.get("clamp_positions", True))
    ctx = dc.declutter_create(k, kernel_r=r, **opts)
    try:
        check_iteration(dc, ctx, z, p, exact_disp=(r == 0))
    finally:
        dc.declutter_destroy(ctx)


@pytest.mark.parametrize("case", ["empty", "one", "one_pixel", "borders", "ragged"])
@pytest.mark.parametrize("r", [0, 2])
def test_edge_cases(dc, case, r):
    k = 6
    rng = np.random.default_rng(3)
    if case == "empty":
        z = np.zeros((0, 2), np.float32)
    elif case == "one":
        z = np.array([[0.3, 0.7]], np.float32)
    elif case == "one_pixel":
        z = np.full((100_000, 2), 0.41, np.float32)
    elif case == "borders":
        z = np.array([[0, 0], [1, 1], [1, 0], [0, 1], [-0.2, 0.5], [0.5, 1.7], [0.999999, 0.5]] * 50,
                     np.float32)
    else:
        z = rng.uniform(0, 1, size=(10_007, 2)).astype(np.float32)
    p = oracle.Params(log2_res=k, kernel_r=r)
    ctx = dc.declutter_create(k, kernel_r=r)
    try:
        if case == "empty":
            g = gpu_step(dc, ctx, z)
            assert g["counts"].sum() == 0 and np.all(g["D"] == 0)
        else:
            check_iteration(dc, ctx, z, p, exact_disp=(r == 0))
    finally:
        dc.declutter_destroy(ctx)


@pytest.mark.parametrize("pixel_center", [False, True])
def test_even_layout_is_exact_fixed_point(dc, pixel_center):
    # Sec. 4.2: the defect-corrected mapping is the identity for an even
    # layout; the exact path gives exactly zero displacement.
    k = 6
    z = synth.uniform_grid_samples(k, per_pixel=3, pixel_center=pixel_center)
    ctx = dc.declutter_create(k, kernel_r=0, pixel_center=pixel_center)
    try:
        g = gpu_step(dc, ctx, z)
        assert np.all(g["D"] == 0.0)
        assert np.array_equal(g["pos"], z)
    finally:
        dc.declutter_destroy(ctx)
    ctx = dc.declutter_create(k, kernel_r=2, pixel_center=pixel_center)
    try:
        g = gpu_step(dc, ctx, z)
        assert float(np.max(np.abs(g["D"]))) * (1 << k) <= 1e-6
    finally:
        dc.declutter_destroy(ctx)


# --------------------------------------------------------------------------
# regularize(): graph path, determinism, host path, metrics
# --------------------------------------------------------------------------

@pytest.mark.parametrize("r", [0, 2])
def test_regularize_graph_teacher_forced(dc, r):
    z, _ = synth.tiny_mixture()
    k = 7
    N = 1 << k
    p = oracle.Params(log2_res=k, kernel_r=r)
    traj = oracle.regularize(z, p, 4)
    ctx = dc.declutter_create(k, kernel_r=r)
    try:
        pos = to_dev(z)
        for it in range(4):
            pos.copy_(to_dev(traj[it]))
            dc.regularize(ctx, pos, 1)
            dc.declutter_sync(ctx)
            err = float(np.max(np.abs(pos.cpu().numpy().astype(np.float64) - traj[it + 1]))) * N
            assert err <= pos_tol_px(N), (it, err)
    finally:
        dc.declutter_destroy(ctx)


@pytest.mark.parametrize("r", [0, 2])
def test_regularize_free_running_and_metrics(dc, r):
    z, _ = synth.tiny_mixture()
    k = 7
    N = 1 << k
    p = oracle.Params(log2_res=k, kernel_r=r)
    traj = oracle.regularize(z, p, 4)
    ref_u = [oracle.quality(oracle.splat(t, k))["bin_std"] for t in traj[1:]]
    ctx = dc.declutter_create(k, kernel_r=r)
    try:
        pos = to_dev(z)
        u = dc.regularize(ctx, pos, 4, uniformity=True)
        q = dc.quality_metrics(ctx)
    finally:
        dc.declutter_destroy(ctx)
    assert all(a > b for a, b in zip(u, u[1:])), u
    assert np.allclose(u, ref_u, rtol=0.02), (u, ref_u)
    d = np.abs(pos.cpu().numpy().astype(np.float64) - traj[-1]) * N
    assert np.median(d) < 1e-3 and np.percentile(d, 99) < 0.1, (np.median(d), np.percentile(d, 99))
    qo = oracle.quality(oracle.splat(pos.cpu().numpy(), k))
    assert abs(q["bin_std"] - qo["bin_std"]) <= 1e-9 * max(1.0, qo["bin_std"])
    assert abs(q["overplot"] - qo["overplot"]) <= 1e-12


@pytest.mark.parametrize("r", [0, 2])
def test_regularize_split_is_bitwise_identical(dc, r):
    # resume: regularize(4) == regularize(1) + regularize(3), bit for bit
    z, _ = synth.tiny_mixture()
    ctx = dc.declutter_create(7, kernel_r=r)
    try:
        a = to_dev(z)
        b = to_dev(z)
        dc.regularize(ctx, a, 4)
        dc.regularize(ctx, b, 1)
        dc.regularize(ctx, b, 3)
        dc.declutter_sync(ctx)
        assert torch.equal(a, b)
        c = to_dev(z)
        dc.regularize(ctx, c, 4)
        dc.declutter_sync(ctx)
        assert torch.equal(a, c)
    finally:
        dc.declutter_destroy(ctx)


@pytest.mark.parametrize("r", [0, 2])
def test_reordering_does_not_change_results(dc, r):
    # iterating on samples sorted by pixel gives the same bits as iterating
    # in the caller's order
    z, _ = synth.gmm20(200_000, seed=5)
    out = []
    for keep in (False, True):
        ctx = dc.declutter_create(9, kernel_r=r, keep_order=keep)
        try:
            pos = to_dev(z)
            u = dc.regularize(ctx, pos, 3, uniformity=True)
            out.append((pos.cpu(), u))
        finally:
            dc.declutter_destroy(ctx)
    assert torch.equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]


@pytest.mark.parametrize("memory,direct", [("pinned", True), ("pinned", False), ("pageable", True)])
def test_regularize_host_matches_device(dc, memory, direct):
    # pinned host memory is used in place over the host link (or staged with
    # the DC_OPT_STAGE_HOST option); pageable memory is always staged
    z, _ = synth.tiny_mixture()
    ctx = dc.declutter_create(7, kernel_r=2, options=0 if direct else dc.DC_OPT_STAGE_HOST)
    try:
        a = to_dev(z)
        ua = dc.regularize(ctx, a, 3, uniformity=True)
        dc.declutter_sync(ctx)
        h = torch.from_numpy(z.copy())
        if memory == "pinned":
            h = h.pin_memory()
        for _ in range(2):  # the second call replays the cached graph
            h.copy_(torch.from_numpy(z))
            uh = dc.regularize_host(ctx, h, 3, uniformity=True)
            assert torch.equal(a.cpu(), h)
            assert ua == uh
    finally:
        dc.declutter_destroy(ctx)


@pytest.mark.parametrize("fused,fused_smooth", [("1", "1"), ("0", "1"), ("0", "0")])
def test_profile_counts_launches(dc, fused, fused_smooth):
    # the three band phases run as one cooperative launch on small grids
    # (DC_OPT_FUSED_BANDS) or as three launches; the smoothing runs inside
    # the aggregate pass unless DC_OPT_SEPARATE_SMOOTH
    opts = (dc.DC_OPT_FUSED_BANDS if fused == "1" else 0) | (dc.DC_OPT_SEPARATE_SMOOTH if fused_smooth == "0" else 0)
    z, _ = synth.tiny_mixture()
    ctx = dc.declutter_create(7, kernel_r=2, options=opts)
    try:
        pos = to_dev(z)
        src = to_dev(z)
        prof = dc.declutter_profile_regularize(ctx, pos, 3, reps=3, reset_src=src)
    finally:
        dc.declutter_destroy(ctx)
    k = prof["kernels"]
    assert prof["step_ms"] > 0
    assert k["splat"]["launches"] == 1
    if k["band_fused"]["launches"]:
        names = ("smooth", "band_fused")
    elif fused_smooth == "1":
        names = ("smooth_aggregate", "band_carry", "band_final")
    else:
        names = ("smooth", "band_aggregate", "band_carry", "band_final")
    if fused == "0":
        assert "band_fused" not in names
    for name in ("advect",) + names:
        assert k[name]["launches"] == 3 and k[name]["ms"] >= 0
    for name in set(k) - set(names) - {"advect", "splat", "reorder", "quality"}:
        assert k[name]["launches"] == 0, name


@pytest.mark.parametrize("log2,r,band_rows,fused", [(7, 2, 0, 1), (8, 2, 0, 1), (8, 5, 3, 1), (9, 4, 0, 1),
                                                     (9, 4, 5, 1), (9, 12, 7, 1), (10, 8, 0, 1), (10, 3, 16, 1),
                                                     (7, 40, 0, 1), (10, 16, 0, 1), (10, 40, 0, 0)])
def test_fused_smoothing_matches_separate_launches(dc, log2, r, band_rows, fused):
    # bitwise: smoothing inside the aggregate pass (windows of 4 or 8 rows,
    # ragged last bands, radii up to the shared-memory limit) against the
    # smoothing kernel plus the aggregate pass; r = 40 at 1024^2 does not fit
    # and keeps the separate launches
    rng = np.random.default_rng(log2 * 100 + r)
    z = rng.beta(2.0, 5.0, size=(60_000, 2)).astype(np.float32)
    outs, us = [], []
    for fs in ("1", "0"):
        ctx = dc.declutter_create(log2, kernel_r=r, band_rows=band_rows,
                                  options=0 if fs == "1" else dc.DC_OPT_SEPARATE_SMOOTH)
        try:
            pos = to_dev(z)
            us.append(dc.regularize(ctx, pos, 3, uniformity=True))
            dc.declutter_sync(ctx)
            if fs == "1":
                prof = dc.declutter_profile_regularize(ctx, to_dev(z), 1, reps=1)
                assert prof["kernels"]["smooth_aggregate"]["launches"] == fused
                assert prof["kernels"]["smooth"]["launches"] == 1 - fused
            outs.append(pos.cpu())
        finally:
            dc.declutter_destroy(ctx)
    assert torch.equal(outs[0], outs[1])
    assert us[0] == us[1]


@pytest.mark.parametrize("r", [0, 2])
def test_fused_and_separate_band_launches_agree(dc, r):
    # bitwise: the fused launch runs the same code as the three launches
    z, _ = synth.tiny_mixture()
    outs = []
    for fused in ("1", "0"):
        ctx = dc.declutter_create(9, kernel_r=r, options=dc.DC_OPT_FUSED_BANDS if fused == "1" else 0)
        try:
            pos = to_dev(z)
            dc.regularize(ctx, pos, 4)
            dc.declutter_sync(ctx)
            outs.append(pos.cpu())
        finally:
            dc.declutter_destroy(ctx)
    assert torch.equal(outs[0], outs[1])


@pytest.mark.parametrize("r", [0, 2])
def test_grid_barrier_timeout_is_reported_and_recovers(dc, r):
    # The one wait between CTAs (the grid barrier of the cooperative band
    # launch) is bounded.  A test option makes it wait for one CTA more than
    # the grid holds, so that every wait runs to its limit (2 ms here): the
    # kernel ends, the status says DC_ERR_TIMEOUT, and the context stays
    # usable.  A fresh context with the default limit then gives the
    # oracle's result and the bits of the three separate launches.
    z, _ = synth.tiny_mixture()
    k = 9
    N = 1 << k
    bad = dc.declutter_create(k, kernel_r=r, options=dc.DC_OPT_FUSED_BANDS | dc.DC_OPT_TEST_UNREACHED_BARRIER,
                              wait_limit_us=2000)
    try:
        pos = to_dev(z)
        dc.regularize(bad, pos, 2)
        with pytest.raises(dc.DeclutterError) as ei:
            dc.declutter_sync(bad)
        assert ei.value.status == 5
        dc.declutter_sync(bad)  # cleared: the context is usable again
        assert declutter_info_ok(dc, bad)
    finally:
        dc.declutter_destroy(bad)
    p = oracle.Params(log2_res=k, kernel_r=r)
    ref = oracle.iterate(z, p)
    outs = []
    for opts in (dc.DC_OPT_FUSED_BANDS, 0):
        ctx = dc.declutter_create(k, kernel_r=r, options=opts)
        try:
            pos = to_dev(z)
            dc.regularize(ctx, pos, 1)
            dc.declutter_sync(ctx)
            outs.append(pos.cpu())
            if opts:
                prof = dc.declutter_profile_regularize(ctx, to_dev(z), 1, reps=1)
                assert prof["kernels"]["band_fused"]["launches"] == 1
        finally:
            dc.declutter_destroy(ctx)
    assert torch.equal(outs[0], outs[1])
    err = float(np.max(np.abs(outs[0].numpy().astype(np.float64) - ref))) * N
    assert err <= pos_tol_px(N), err


def declutter_info_ok(dc, ctx):
    info = dc.declutter_get_info(ctx)
    return info.N == ctx.N


def test_options_and_limits_are_validated(dc):
    for kw in ({"options": 1 << 20}, {"wait_limit_us": -1}, {"wait_limit_us": 10_000_001}):
        with pytest.raises(dc.DeclutterError):
            dc.declutter_create(7, kernel_r=2, **kw)


def test_bad_arguments_are_rejected(dc):
    ctx = dc.declutter_create(6, kernel_r=0)
    try:
        pos = torch.zeros(10, 2, device=DEV)
        with pytest.raises(dc.DeclutterError):
            dc.advect_samples(ctx, pos)          # before any displacement
        with pytest.raises(dc.DeclutterError):
            dc.displacement_field(ctx)           # before any splat
        lib = dc.load_library()
        import ctypes
        mis = ctypes.c_void_p(pos.data_ptr() + 4)
        assert lib.splat_density(ctx.handle, mis, 4, None, None) == 1
        assert lib.splat_density(ctx.handle, ctypes.c_void_p(pos.data_ptr()), -1, None, None) == 1
    finally:
        dc.declutter_destroy(ctx)


# --------------------------------------------------------------------------
# Full-size workloads
# --------------------------------------------------------------------------

def test_gmm20_512_full_size_one_iteration(dc):
    # 1M samples, 512x512, r = 4: the launch configuration the benchmark times
    z, _ = synth.gmm20()
    p = oracle.Params(log2_res=9, kernel_r=4)
    ctx = dc.declutter_create(9, kernel_r=4)
    try:
        check_iteration(dc, ctx, z, p)
        traj = oracle.regularize(z, p, 2)
        pos = to_dev(traj[1])
        dc.regularize(ctx, pos, 1)
        dc.declutter_sync(ctx)
        err = float(np.max(np.abs(pos.cpu().numpy().astype(np.float64) - traj[2]))) * 512
        assert err <= pos_tol_px(512), err
    finally:
        dc.declutter_destroy(ctx)


@pytest.mark.parametrize("carry_mode", [0, 1])
def test_student_t_2048_full_size_one_iteration(dc, carry_mode):
    # 16M heavy-tailed samples, 2048x2048, r = 16
    z, _ = synth.student_t_clusters()
    p = oracle.Params(log2_res=11, kernel_r=16)
    ctx = dc.declutter_create(11, kernel_r=16, carry_mode=carry_mode)
    try:
        err = check_iteration(dc, ctx, z, p)
        print(f"2048^2 carry_mode={carry_mode}: max |D - D_fp64| = {err:.3e} px")
    finally:
        dc.declutter_destroy(ctx)


def test_largest_grid_8192_one_iteration(dc):
    # the largest resolution (8192 x 8192) in exact mode: counts bit-exact,
    # the field and the moved samples against the oracle
    z, _ = synth.student_t_clusters(2_000_000, seed=5)
    p = oracle.Params(log2_res=13, kernel_r=0)
    ctx = dc.declutter_create(13, kernel_r=0)
    try:
        err = check_iteration(dc, ctx, z, p, exact_disp=True)
        print(f"8192^2 exact: max |D - D_fp64| = {err:.3e} px")
    finally:
        dc.declutter_destroy(ctx)


@pytest.mark.parametrize("k", [12, 13])
def test_float_mode_above_2048_is_refused(dc, k):
    # float (smoothed) mode holds the 1e-4 px bound up to 2048^2; above, the
    # FP32 region sums alone err by about 2^-24 N / 2 px, so contexts and
    # the lens refuse it (exact mode runs at every size)
    with pytest.raises(dc.DeclutterError) as ei:
        dc.declutter_create(k, kernel_r=8)
    assert ei.value.status == 1 and "kernel_r = 0" in dc.declutter_last_error()
    with pytest.raises(dc.DeclutterError):
        dc.declutter_create(k)  # the automatic radius N / 128
    ctx = dc.declutter_create(k, kernel_r=0)
    try:
        N = 1 << k
        with pytest.raises(dc.DeclutterError):
            dc.lens_field(ctx, torch.ones(N * N, dtype=torch.float32, device=DEV), 1.0)
    finally:
        dc.declutter_destroy(ctx)


# --------------------------------------------------------------------------
# The splat fused into the advection inside regularize() (Sec. 4.3 step 1 of
# every iteration after the first), compared with the oracle's splat
# --------------------------------------------------------------------------

FUSED_CASES = {
    # name: (generator, log2 N, r)
    "gmm20_512": (lambda: synth.gmm20()[0], 9, 4),
    "student_t_2048": (lambda: synth.student_t_clusters()[0], 11, 16),
    # an odd sample count: the last sample is moved and splatted outside the
    # pairs of the warp-wide run aggregation
    "tiny_odd": (lambda: synth.tiny_mixture(20_001, seed=3)[0], 7, 2),
}


@pytest.mark.parametrize("case,keep_order,k", [("gmm20_512", False, 2), ("gmm20_512", False, 3),
                                               ("gmm20_512", True, 2), ("student_t_2048", False, 2),
                                               ("student_t_2048", False, 3), ("tiny_odd", False, 3),
                                               ("tiny_odd", True, 3)])
def test_fused_splat_inside_regularize_matches_oracle(dc, case, keep_order, k):
    # Inside regularize(k) the advection of iteration m splats the moved
    # samples into the count grid of iteration m + 1 (atomics aggregated over
    # runs of equal pixels on pixel-ordered samples, __match_any_sync in the
    # caller's order).  Three checks:
    #  (1) regularize(k) without metrics leaves the input grid of its last
    #      iteration, i.e. the in-graph splat of the positions after k - 1
    #      iterations (regularize(k - 1) on a copy gives those bits):
    #      bit-exact against oracle.splat;
    #  (2) regularize(k) with metrics also splats the final positions:
    #      bit-exact against oracle.splat of the returned positions;
    #  (3) the last in-graph iteration, which ran on those counts, against
    #      oracle.iterate of the positions it started from (teacher-forced).
    gen, log2, r = FUSED_CASES[case]
    z = gen()
    N = 1 << log2
    p = oracle.Params(log2_res=log2, kernel_r=r)
    ctx = dc.declutter_create(log2, kernel_r=r, keep_order=keep_order)
    try:
        prev = to_dev(z)
        dc.regularize(ctx, prev, k - 1)
        dc.declutter_sync(ctx)
        prev_np = prev.cpu().numpy()
        del prev
        counts = torch.empty(N * N, dtype=torch.int32, device=DEV)
        pos = to_dev(z)
        dc.regularize(ctx, pos, k)
        dc.declutter_counts(ctx, counts)
        dc.declutter_sync(ctx)
        c_in = u32(counts, N).astype(np.uint64)
        assert np.array_equal(c_in, oracle.splat(prev_np, log2)), "in-graph splat of the input of iteration k"
        got = pos.cpu().numpy()
        ref = oracle.iterate(prev_np, p)
        perr = float(np.max(np.abs(got.astype(np.float64) - ref))) * N
        assert perr <= pos_tol_px(N), perr
        pos.copy_(to_dev(z))
        u = dc.regularize(ctx, pos, k, uniformity=True)
        dc.declutter_counts(ctx, counts)
        dc.declutter_sync(ctx)
        fin = pos.cpu().numpy()
        assert np.array_equal(fin, got), "metrics must not change the positions"
        c_out = u32(counts, N).astype(np.uint64)
        ref_c = oracle.splat(fin, log2)
        assert np.array_equal(c_out, ref_c), "in-graph splat of the final positions"
        assert abs(u[-1] - oracle.quality(ref_c)["bin_std"]) <= 1e-9 * max(1.0, u[-1])
        print(f"{case} keep_order={keep_order} k={k}: counts bit-exact, last iteration {perr:.3e} px")
    finally:
        dc.declutter_destroy(ctx)


@pytest.mark.parametrize("keep_order", [False, True])
def test_fused_splat_with_unaligned_samples(dc, keep_order):
    # samples starting 8 bytes past a 16-byte boundary and an odd count: in
    # the caller's order the first and the last sample fall outside the
    # aligned pairs of the advection; counts of the in-graph splat bit-exact
    log2, r, k = 7, 2, 3
    z, _ = synth.tiny_mixture(20_001, seed=8)
    N = 1 << log2
    ctx = dc.declutter_create(log2, kernel_r=r, keep_order=keep_order)
    try:
        buf = torch.zeros(z.shape[0] + 1, 2, dtype=torch.float32, device=DEV)
        pos = buf[1:]
        assert pos.data_ptr() % 16 == 8
        pos.copy_(to_dev(z))
        dc.regularize(ctx, pos, k - 1)
        dc.declutter_sync(ctx)
        prev_np = pos.cpu().numpy()
        pos.copy_(to_dev(z))
        counts = torch.empty(N * N, dtype=torch.int32, device=DEV)
        dc.regularize(ctx, pos, k, uniformity=True)
        dc.declutter_counts(ctx, counts)
        dc.declutter_sync(ctx)
        fin = pos.cpu().numpy()
        assert np.array_equal(u32(counts, N).astype(np.uint64), oracle.splat(fin, log2))
        ref = oracle.iterate(prev_np, oracle.Params(log2_res=log2, kernel_r=r))
        perr = float(np.max(np.abs(fin.astype(np.float64) - ref))) * N
        assert perr <= pos_tol_px(N), perr
        assert float(buf[0].abs().sum()) == 0.0, "the slot before the samples must stay untouched"
    finally:
        dc.declutter_destroy(ctx)


def test_declutter_counts_state_and_arguments(dc):
    ctx = dc.declutter_create(6, kernel_r=0)
    try:
        out = torch.empty(64 * 64, dtype=torch.int32, device=DEV)
        with pytest.raises(dc.DeclutterError):
            dc.declutter_counts(ctx, out)         # before any splat
        z, _ = synth.tiny_mixture(3000, seed=9)
        dc.splat_density(ctx, to_dev(z))
        dc.declutter_counts(ctx, out)
        dc.declutter_sync(ctx)
        assert np.array_equal(u32(out, 64).astype(np.uint64), oracle.splat(z, 6))
        lib = dc.load_library()
        import ctypes
        assert lib.declutter_counts(ctx.handle, None) == 1
        assert lib.declutter_counts(ctx.handle, ctypes.c_void_p(out.data_ptr() + 2)) == 1
    finally:
        dc.declutter_destroy(ctx)


# --------------------------------------------------------------------------
# Virtual lens (end of Sec. 3.2): eq. (map) without the defect
# --------------------------------------------------------------------------

def painted_density(N, seed):
    # constant outside, a few painted rectangles of other constant values
    rng = np.random.default_rng(seed)
    d = np.ones((N, N), np.float32)
    for _ in range(3):
        i0, j0 = rng.integers(0, N - N // 4, size=2)
        w, h = rng.integers(N // 16, N // 4, size=2)
        d[j0:j0 + h, i0:i0 + w] = float(rng.choice([0.25, 2.0, 4.0, 8.0]))
    return d


def lens_tol_px(N, hint="zero"):
    # With the density's mean as the hint the pixel position cancels in
    # exact integers before any rounding (t - x from excess sums), so the
    # displacement bound holds.  With hint 0 the sums are not centred and
    # t(x, y; d) is formed as an O(1) float32 value before the position is
    # taken off: a few float32 roundings of 1, i.e. of 2^-24 N pixel, on
    # top of the displacement bound.
    if hint == "mean":
        return DISP_TOL_PX
    return DISP_TOL_PX + 6 * N * 2.0 ** -24


@pytest.mark.parametrize("k,r,pixel_center,hint", [(4, 2, 0, "mean"), (6, 2, 0, "mean"), (9, 0, 0, "mean"),
                                                   (9, 4, 1, "zero"), (11, 16, 0, "mean"), (11, 16, 1, "zero")])
def test_lens_field_matches_oracle(dc, k, r, pixel_center, hint):
    N = 1 << k
    d = painted_density(N, seed=k * 10 + pixel_center)
    ref = oracle.lens_displacement(d.astype(np.float64), pixel_center=bool(pixel_center))
    ctx = dc.declutter_create(k, kernel_r=r, pixel_center=pixel_center)
    try:
        dg = torch.from_numpy(d).to(DEV)
        out = torch.empty(2 * N * N, dtype=torch.float32, device=DEV)
        dc.lens_field(ctx, dg, float(d.mean()) if hint == "mean" else 0.0, out)
        # samples on pixel positions move to the mapped positions
        off = 0.5 if pixel_center else 0.0
        jj, ii = np.meshgrid(np.arange(0, N, 7), np.arange(0, N, 5), indexing="ij")
        z = np.stack([(ii.ravel() + off) / N, (jj.ravel() + off) / N], 1).astype(np.float32)
        pos = to_dev(z)
        dc.advect_samples(ctx, pos)
        dc.declutter_sync(ctx)
        assert torch.equal(dg, torch.from_numpy(d).to(DEV))  # the density is not modified
    finally:
        dc.declutter_destroy(ctx)
    err = float(np.max(np.abs(out.cpu().numpy().reshape(N, N, 2).astype(np.float64) - ref))) * N
    print(f"lens {N}^2 pc={pixel_center} hint={hint}: max error {err:.2e} px")
    assert err <= lens_tol_px(N, hint), err
    want = z.astype(np.float64) + ref[jj.ravel(), ii.ravel()]
    perr = float(np.max(np.abs(pos.cpu().numpy().astype(np.float64) - want))) * N
    assert perr <= lens_tol_px(N, hint) + N * float(np.spacing(np.float32(1.0))), perr


@pytest.mark.parametrize("k", [7, 11])
def test_lens_field_without_mass_writes_zero_and_reports(dc, k):
    # eq. (map) divides by the total mass: for an all-zero density the lens
    # writes a zero field and the status reports an invalid argument
    N = 1 << k
    ctx = dc.declutter_create(k, kernel_r=2)
    try:
        out = torch.full((2 * N * N,), 7.0, dtype=torch.float32, device=DEV)
        dc.lens_field(ctx, torch.zeros(N * N, dtype=torch.float32, device=DEV), 0.0, out)
        with pytest.raises(dc.DeclutterError) as ei:
            dc.declutter_sync(ctx)
        assert ei.value.status == 1
        assert bool(torch.all(out == 0))
        dc.declutter_sync(ctx)  # the status was cleared
    finally:
        dc.declutter_destroy(ctx)


def test_lens_field_rejects_bad_arguments(dc):
    ctx = dc.declutter_create(7, kernel_r=2)
    try:
        d = torch.ones(128 * 128, dtype=torch.float32, device=DEV)
        with pytest.raises(dc.DeclutterError):
            dc.lens_field(ctx, d, -1.0)
        with pytest.raises(dc.DeclutterError):
            dc.lens_field(ctx, d, float("nan"))
        with pytest.raises(dc.DeclutterError):  # not 16-byte aligned
            dc.lens_field(ctx, torch.ones(128 * 128 + 1, dtype=torch.float32, device=DEV)[1:], 1.0)
    finally:
        dc.declutter_destroy(ctx)


# --------------------------------------------------------------------------
# Deformed grid (Sec. 5): pixel nodes as massless tracers
# --------------------------------------------------------------------------

@pytest.mark.parametrize("r", [0, 2])
def test_regularize_tracers_moves_nodes_by_the_field(dc, r):
    z, _ = synth.tiny_mixture()
    N = 128
    p = oracle.Params(log2_res=7, kernel_r=r)
    jj, ii = np.meshgrid(np.arange(0, N, 4), np.arange(0, N, 4), indexing="ij")
    nodes = np.stack([ii.ravel() / N, jj.ravel() / N], 1).astype(np.float32)
    # one iteration: every node moves by the oracle's field at that node
    _, aux = oracle.iterate(z, p, keep=True)
    want = oracle.advect(nodes.astype(np.float64), aux["D"])
    ctx = dc.declutter_create(7, kernel_r=r)
    try:
        pos, tr = to_dev(z), to_dev(nodes)
        dc.regularize_tracers(ctx, pos, tr, 1)
        dc.declutter_sync(ctx)
        err = float(np.max(np.abs(tr.cpu().numpy().astype(np.float64) - want))) * N
        assert err <= pos_tol_px(N), err
        moved = np.abs(tr.cpu().numpy() - nodes).max() * N
        assert moved > 1e-3  # the field is not trivial here
        # three iterations: the samples are those of regularize(), bit for bit
        # (tracers are moved, never splatted)
        pos3, tr3 = to_dev(z), to_dev(nodes)
        dc.regularize_tracers(ctx, pos3, tr3, 3)
        ref3 = to_dev(z)
        dc.regularize(ctx, ref3, 3)
        dc.declutter_sync(ctx)
        assert torch.equal(pos3, ref3)
        assert bool(torch.all(torch.isfinite(tr3))) and float(tr3.min()) >= 0.0 and float(tr3.max()) <= 1.0
    finally:
        dc.declutter_destroy(ctx)


# --------------------------------------------------------------------------
# Contour lines (Sec. 5): marching squares
# --------------------------------------------------------------------------

CONTOUR_TOL = 2.0 ** -20  # domain units: a few float32 roundings of the interpolated vertex


def smooth_field(N, seed):
    rng = np.random.default_rng(seed)
    jj, ii = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    f = np.zeros((N, N))
    for _ in range(12):
        ci, cj = rng.uniform(0, N, size=2)
        s = rng.uniform(N / 30, N / 6)
        f += rng.uniform(0.5, 2.0) * np.exp(-((ii - ci) ** 2 + (jj - cj) ** 2) / (2 * s * s))
    return f.astype(np.float32)


def check_contour_cells(out, f, level, cells, pixel_center):
    N = f.shape[0]
    M = N - 1
    slots = out.reshape(M * M, 2, 4)
    for c in cells:
        j, i = divmod(int(c), M)
        want = sorted(tuple(sorted(s)) for s in oracle.contour_cell(f, level, i, j, bool(pixel_center)))
        got_slots = [s for s in slots[c] if not np.isnan(s[0])]
        assert all(np.isnan(s).all() for s in slots[c] if np.isnan(s[0])), (i, j)
        got = sorted(tuple(sorted([(float(s[0]), float(s[1])), (float(s[2]), float(s[3]))])) for s in got_slots)
        assert len(got) == len(want), (i, j, got, want)
        for g, w in zip(got, want):
            assert np.max(np.abs(np.array(g) - np.array(w))) <= CONTOUR_TOL, (i, j, g, w)


@pytest.mark.parametrize("k,kind,pixel_center", [(4, "smooth", 0), (7, "smooth", 0), (7, "ties", 0),
                                                  (7, "smooth", 1), (11, "smooth", 0), (13, "smooth", 0)])
def test_contour_segments_match_oracle(dc, k, kind, pixel_center):
    N = 1 << k
    if kind == "smooth":
        f = smooth_field(N, seed=k)
        levels = [float(np.float32(np.quantile(f, q))) for q in (0.3, 0.6, 0.9)]
    else:  # integer values: corners and saddle centres equal to the level
        jj, ii = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
        f = ((ii * 7 + jj * 13) % 5).astype(np.float32) * 2.0
        levels = [4.0, 5.0]
    M = N - 1
    rng = np.random.default_rng(k)
    cells = np.arange(M * M) if N <= 128 else np.unique(np.concatenate([
        rng.integers(0, M * M, size=4000), np.arange(M * 700, M * 702), np.arange(M * M - 2 * M, M * M)]))
    ctx = dc.declutter_create(k, kernel_r=0, pixel_center=pixel_center)
    try:
        fg = torch.from_numpy(f).to(DEV)
        for lv in levels:
            out = torch.empty(8 * M * M, dtype=torch.float32, device=DEV)
            dc.contour_segments(ctx, fg, lv, out)
            dc.declutter_sync(ctx)
            check_contour_cells(out.cpu().numpy(), f, lv, cells, pixel_center)
    finally:
        dc.declutter_destroy(ctx)
