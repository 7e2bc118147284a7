"""GPU parity of the layout-level rows through the C ABI against
oracle/layout.py: the transition blend (Sec. 1), the layout measures of
Sec. 6.2 (trustworthiness, orthogonal ordering) and the stopping criteria
of Sec. 4.3 step 4 (regularize_adaptive).

Bars: the blend and every integer term of the measures are bit-exact; the
stopping iteration is the oracle's (criteria placed between two
iterations' measures); positions after an adaptive run are those of
regularize() with the same number of iterations, bit for bit.
"""

import numpy as np
import pytest

import oracle
import synth
from oracle import layout as L

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu]

DEV = "cuda:0"


@pytest.fixture(scope="module")
def dc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_06513_gb300 import build as dc_build
    dc_build.build()
    from paper_2408_06513_gb300 import declutter
    declutter.load_library()
    return declutter


def to_dev(z):
    return torch.from_numpy(np.ascontiguousarray(z, dtype=np.float32)).to(DEV)


# --------------------------------------------------------------------------
# transition
# --------------------------------------------------------------------------

@pytest.mark.parametrize("s", [0.0, 0.25, 0.5, 0.8, 1.0])
@pytest.mark.parametrize("offset", [0, 1])
def test_transition_bit_exact(dc, s, offset):
    # offset 1: 8-byte (not 16-byte) aligned arrays take the scalar path
    rng = np.random.default_rng(11)
    n = 100_003
    a = rng.random((n + 1, 2)).astype(np.float32)
    b = rng.random((n + 1, 2)).astype(np.float32)
    ctx = dc.declutter_create(6, kernel_r=0)
    try:
        ad, bd = to_dev(a), to_dev(b)
        out = torch.empty_like(ad)
        dc.transition_positions(ctx, ad[offset:offset + n], bd[offset:offset + n], s, out[offset:offset + n])
        dc.declutter_sync(ctx)
        got = out[offset:offset + n].cpu().numpy()
    finally:
        dc.declutter_destroy(ctx)
    ref = L.transition(a[offset:offset + n], b[offset:offset + n], s)
    assert np.array_equal(got, ref)


def test_transition_of_a_regularised_plot_and_bad_s(dc):
    z, _ = synth.gmm20(200_000, seed=3)
    ctx = dc.declutter_create(9, kernel_r=4)
    try:
        a = to_dev(z)
        b = to_dev(z)
        dc.regularize(ctx, b, 4)
        out = torch.empty_like(a)
        dc.transition_positions(ctx, a, b, 0.3, out)
        dc.declutter_sync(ctx)
        assert np.array_equal(out.cpu().numpy(), L.transition(z, b.cpu().numpy(), 0.3))
        with pytest.raises(dc.DeclutterError):
            dc.transition_positions(ctx, a, b, 1.5, out)
    finally:
        dc.declutter_destroy(ctx)


# --------------------------------------------------------------------------
# trustworthiness and orthogonal ordering
# --------------------------------------------------------------------------

@pytest.mark.parametrize("k", [1, 7, 10, 32])
def test_layout_metrics_all_queries_bit_exact(dc, k):
    z, _ = synth.tiny_mixture(3000, seed=k)
    ctx = dc.declutter_create(7, kernel_r=2)
    try:
        a, b = to_dev(z), to_dev(z)
        dc.regularize(ctx, b, 4)
        got = dc.layout_metrics(ctx, a, b, k, want_terms=True)
        reg = b.cpu().numpy()
    finally:
        dc.declutter_destroy(ctx)
    ref = L.layout_metrics(z, reg, k)
    assert np.array_equal(got["terms"][:, 0], ref["t_terms"])
    assert np.array_equal(got["terms"][:, 1], ref["o_terms"])
    assert abs(got["trustworthiness"] - ref["trustworthiness"]) <= 1e-12
    assert abs(got["ordering"] - ref["ordering"]) <= 1e-12
    assert 0.5 < got["trustworthiness"] <= 1.0 and 0.5 < got["ordering"] <= 1.0
    print(f"k={k}: T={got['trustworthiness']:.4f} O={got['ordering']:.4f}")


def test_layout_metrics_full_size_sampled_queries(dc):
    # 1M samples, 512^2, r = 4, 8 iterations (the benchmark workload): the
    # per-query terms of 48 random queries against the oracle, bit for bit
    z, _ = synth.gmm20()
    ctx = dc.declutter_create(9, kernel_r=4)
    try:
        a, b = to_dev(z), to_dev(z)
        dc.regularize(ctx, b, 8)
        q = np.random.default_rng(2).choice(z.shape[0], size=48, replace=False).astype(np.int32)
        got = dc.layout_metrics(ctx, a, b, 10, queries=torch.from_numpy(q).to(DEV), want_terms=True)
        reg = b.cpu().numpy()
    finally:
        dc.declutter_destroy(ctx)
    ref = L.layout_metrics(z, reg, 10, queries=q)
    assert np.array_equal(got["terms"][:, 0], ref["t_terms"])
    assert np.array_equal(got["terms"][:, 1], ref["o_terms"])
    assert abs(got["trustworthiness"] - ref["trustworthiness"]) <= 1e-12
    print(f"1M samples, 48 queries: T={got['trustworthiness']:.4f} O={got['ordering']:.4f}")


def test_layout_metrics_identity_and_errors(dc):
    z, _ = synth.tiny_mixture(1000, seed=1)
    ctx = dc.declutter_create(6, kernel_r=0)
    try:
        a = to_dev(z)
        m = dc.layout_metrics(ctx, a, a, 5)
        assert m["trustworthiness"] == 1.0 and m["ordering"] == 1.0
        with pytest.raises(dc.DeclutterError) as ei:
            dc.layout_metrics(ctx, a, a, 5, queries=torch.tensor([3, 1000], dtype=torch.int32, device=DEV))
        assert ei.value.status == 6  # DC_ERR_RANGE
        with pytest.raises(dc.DeclutterError):
            dc.layout_metrics(ctx, a, a, 33)
        with pytest.raises(dc.DeclutterError):
            dc.layout_metrics(ctx, a[:10], a[:10], 5)  # k >= n / 2
    finally:
        dc.declutter_destroy(ctx)


# --------------------------------------------------------------------------
# stopping criteria (one graph launch, conditional iterations)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("r,keep_order", [(2, False), (0, False), (2, True)])
def test_adaptive_matches_fixed_iterations(dc, r, keep_order):
    z, _ = synth.tiny_mixture()
    k = 7
    ctx = dc.declutter_create(k, kernel_r=r, keep_order=keep_order)
    try:
        full = to_dev(z)
        res = dc.regularize_adaptive(ctx, full, 6)
        assert res["iters"] == 6
        ref = to_dev(z)
        u = dc.regularize(ctx, ref, 6, uniformity=True)
        dc.declutter_sync(ctx)
        assert torch.equal(full, ref)
        mean = z.shape[0] / ((1 << k) // 4) ** 2  # samples per 4x4 bin
        assert np.allclose(np.array(res["cv"]) * mean, u, rtol=1e-12, atol=0)
        cv, mv = res["cv"], res["move_px"]
        assert all(a > b for a, b in zip(cv, cv[1:])), cv
        # the first iteration whose measure reaches the target ends the run:
        # a target between the measures after iterations stop - 1 and stop
        for stop in (1, 3, 5):
            tgt = 1.05 * cv[0] if stop == 1 else 0.5 * (cv[stop - 2] + cv[stop - 1])
            pos = to_dev(z)
            got = dc.regularize_adaptive(ctx, pos, 6, target_cv=tgt)
            assert got["iters"] == stop, (stop, got)
            # the context's counts are those of the returned positions
            counts = torch.empty(128 * 128, dtype=torch.int32, device=DEV)
            dc.declutter_counts(ctx, counts)
            dc.declutter_sync(ctx)
            c = counts.cpu().numpy().view(np.uint32).reshape(128, 128).astype(np.uint64)
            assert np.array_equal(c, oracle.splat(pos.cpu().numpy(), k))
            want = to_dev(z)
            dc.regularize(ctx, want, stop)
            dc.declutter_sync(ctx)
            assert torch.equal(pos, want)
        # the largest move of an iteration
        got = dc.regularize_adaptive(ctx, to_dev(z), 6, min_move_px=0.5 * (mv[1] + mv[2]))
        assert got["iters"] == 3
        # a time budget already spent after the first iteration
        got = dc.regularize_adaptive(ctx, to_dev(z), 6, max_ms=1e-6)
        assert got["iters"] == 1
    finally:
        dc.declutter_destroy(ctx)


def test_adaptive_stop_iteration_matches_oracle(dc):
    # criteria placed half-way (geometrically) between two iterations of the
    # oracle's own run: the GPU stops at the same iteration, and its
    # measures and moves agree with the oracle's
    z, _ = synth.tiny_mixture()
    p = oracle.Params(log2_res=7, kernel_r=2)
    full = L.regularize_until(z, p, 6)
    cv, mv = full["cv"], full["move_px"]
    ctx = dc.declutter_create(7, kernel_r=2)
    try:
        g = dc.regularize_adaptive(ctx, to_dev(z), 6)
        assert np.allclose(g["cv"], cv, rtol=0.02)
        assert np.allclose(g["move_px"], mv, rtol=0.02)
        for stop in (2, 4):
            tgt = float(np.sqrt(cv[stop - 2] * cv[stop - 1]))
            r = L.regularize_until(z, p, 6, target_cv=tgt)
            got = dc.regularize_adaptive(ctx, to_dev(z), 6, target_cv=tgt)
            assert got["iters"] == r["iters"] == stop
            mtol = float(np.sqrt(mv[stop - 2] * mv[stop - 1]))
            r = L.regularize_until(z, p, 6, min_move_px=mtol)
            got = dc.regularize_adaptive(ctx, to_dev(z), 6, min_move_px=mtol)
            assert got["iters"] == r["iters"]
    finally:
        dc.declutter_destroy(ctx)


def test_adaptive_full_size_2048(dc):
    # 16M samples, 2048^2, r = 16: a run stopped by the measure equals the
    # fixed-iteration run of the same length
    z, _ = synth.student_t_clusters()
    ctx = dc.declutter_create(11, kernel_r=16)
    try:
        pos = to_dev(z)
        full = dc.regularize_adaptive(ctx, pos, 5)
        cv = full["cv"]
        del pos
        tgt = 0.5 * (cv[1] + cv[2])  # reached after the third iteration
        pos = to_dev(z)
        got = dc.regularize_adaptive(ctx, pos, 5, target_cv=tgt)
        assert got["iters"] == 3
        want = to_dev(z)
        dc.regularize(ctx, want, 3)
        dc.declutter_sync(ctx)
        assert torch.equal(pos, want)
    finally:
        dc.declutter_destroy(ctx)


def test_adaptive_rejects_bad_arguments(dc):
    ctx = dc.declutter_create(6, kernel_r=0)
    try:
        z = to_dev(np.random.default_rng(0).random((100, 2)))
        for kw in ({"max_iters": 0}, {"max_iters": 2000}, {"max_iters": 3, "target_cv": -1.0},
                   {"max_iters": 3, "max_ms": float("inf")}):
            with pytest.raises(dc.DeclutterError):
                dc.regularize_adaptive(ctx, z, **kw)
    finally:
        dc.declutter_destroy(ctx)


# --------------------------------------------------------------------------
# density texture on the deformed mesh, transfer function (Sec. 5)
# --------------------------------------------------------------------------

def _smooth_nodes(N):
    nodes = L.identity_nodes(N).astype(np.float64)
    x, y = nodes[..., 0] * N / (N - 1), nodes[..., 1] * N / (N - 1)
    nodes[..., 0] += 0.05 * np.sin(np.pi * x) * np.sin(2 * np.pi * y) * (N - 1) / N
    nodes[..., 1] += 0.04 * np.sin(2 * np.pi * x) * np.sin(np.pi * y) * (N - 1) / N
    return nodes.astype(np.float32)


def _warp_gpu(dc, ctx, nodes, tex, log2M, mass):
    M = 1 << log2M
    out = torch.empty(M * M, dtype=torch.float32, device=DEV)
    tri = torch.empty(M * M, dtype=torch.int32, device=DEV)
    dc.warp_texture(ctx, to_dev(nodes.reshape(-1, 2)), to_dev(tex.reshape(-1)), log2M, out, mass=mass, tri_out=tri)
    dc.declutter_sync(ctx)
    return out.cpu().numpy().reshape(M, M), tri.cpu().numpy().reshape(M, M).astype(np.int64)


@pytest.mark.parametrize("log2M,mass", [(5, False), (6, True), (4, False)])
def test_warp_texture_smooth_mesh(dc, log2M, mass):
    N = 32
    jj, ii = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    tex = (1.0 + np.exp(-((ii - 9.0) ** 2 + (jj - 20.0) ** 2) / 40.0) * 4.0).astype(np.float32)
    nodes = _smooth_nodes(N)
    ctx = dc.declutter_create(5, kernel_r=2)
    try:
        got, tri = _warp_gpu(dc, ctx, nodes, tex, log2M, mass)
    finally:
        dc.declutter_destroy(ctx)
    ref, cov = L.warp_texture(nodes, tex, log2M, mass=mass)
    assert np.array_equal(tri, cov)
    assert np.max(np.abs(got - ref)) <= 2e-5 * float(np.abs(ref).max())


@pytest.mark.parametrize("r", [0, 2])
def test_warp_texture_of_regularised_nodes(dc, r):
    # the pixel nodes moved by 8 iterations as tracers (the deformed grid of
    # Sec. 5), the smoothed density drawn on them: coverage bit-exact,
    # values within float32 rounding, and the push-forward of the density
    # keeps its mass and is much more even than the density itself (the
    # method equalises density)
    k = 6
    N = 1 << k
    z, _ = synth.tiny_mixture(20_000, seed=4)
    ctx = dc.declutter_create(k, kernel_r=r)
    try:
        pos = to_dev(z)
        nodes0 = L.identity_nodes(N)
        tr = to_dev(nodes0.reshape(-1, 2))
        dc.regularize_tracers(ctx, pos, tr, 8)
        if r > 0:  # the smoothed density d_r
            dens = torch.empty(N * N, dtype=torch.float32, device=DEV)
            dc.splat_density(ctx, to_dev(z), density_out=dens)
        else:      # the counts
            cnt = torch.empty(N * N, dtype=torch.int32, device=DEV)
            dc.splat_density(ctx, to_dev(z), counts_out=cnt)
            dens = cnt.float()
        dc.declutter_sync(ctx)
        nodes = tr.cpu().numpy().reshape(N, N, 2)
        tex = dens.cpu().numpy().reshape(N, N)
        log2M = k + 1
        got, tri = _warp_gpu(dc, ctx, nodes, tex, log2M, True)
        gid, _ = _warp_gpu(dc, ctx, nodes0, tex, log2M, True)
    finally:
        dc.declutter_destroy(ctx)
    ref, cov = L.warp_texture(nodes, tex, log2M, mass=True)
    assert np.array_equal(tri, cov)
    assert np.max(np.abs(got - ref)) <= 1e-4 * float(np.abs(ref).max())
    assert abs(got.sum() / gid.sum() - 1.0) < 0.03
    inside = cov >= 0
    cv_push = got[inside].std() / got[inside].mean()
    cv_orig = gid[gid > 0].std() / gid[gid > 0].mean()
    print(f"r={r}: push-forward CV {cv_push:.3f} against {cv_orig:.3f} for the density itself")
    assert cv_push < 0.5 * cv_orig


def test_transfer_function_bit_exact(dc):
    rng = np.random.default_rng(9)
    v = np.concatenate([rng.normal(0.5, 0.6, 100_000), [np.nan, -np.inf, np.inf]]).astype(np.float32)
    lut = (rng.integers(0, 2 ** 32, size=256, dtype=np.uint64)).astype(np.uint32)
    ctx = dc.declutter_create(6, kernel_r=0)
    try:
        out = torch.empty(v.size, dtype=torch.int32, device=DEV)
        dc.transfer_function(ctx, to_dev(v), -0.25, 1.3, torch.from_numpy(lut.view(np.int32)).to(DEV), out)
        dc.declutter_sync(ctx)
        got = out.cpu().numpy().view(np.uint32)
        with pytest.raises(dc.DeclutterError):
            dc.transfer_function(ctx, to_dev(v), 1.0, 1.0, torch.from_numpy(lut.view(np.int32)).to(DEV), out)
    finally:
        dc.declutter_destroy(ctx)
    assert np.array_equal(got, L.transfer(v, -0.25, 1.3, lut))


@pytest.mark.parametrize("opts", ["fused", "separate_smooth", "pixel_center"])
def test_adaptive_with_launch_options(dc, opts):
    # the conditional graph holds whatever the context launches: the
    # cooperative band kernel, the separate smoothing, other conventions
    z, _ = synth.tiny_mixture()
    kw = {"fused": {"options": dc.DC_OPT_FUSED_BANDS}, "separate_smooth": {"options": dc.DC_OPT_SEPARATE_SMOOTH},
          "pixel_center": {"pixel_center": True}}[opts]
    ctx = dc.declutter_create(7, kernel_r=2, **kw)
    try:
        a = to_dev(z)
        res = dc.regularize_adaptive(ctx, a, 5)
        b = to_dev(z)
        dc.regularize(ctx, b, res["iters"])
        dc.declutter_sync(ctx)
        assert res["iters"] == 5 and torch.equal(a, b)
        tgt = 0.5 * (res["cv"][1] + res["cv"][2])
        c = to_dev(z)
        assert dc.regularize_adaptive(ctx, c, 5, target_cv=tgt)["iters"] == 3
    finally:
        dc.declutter_destroy(ctx)
