"""Batched regularisation of scatterplot-matrix panels (one CUDA graph for all
panels) against each panel regularised on its own, and the band-height
autotuner."""

import numpy as np
import pytest

import oracle
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


@pytest.fixture(scope="module")
def panels():
    # 5 dimensions -> 10 panels of 256^2 / 512^2 / 1024^2, uneven sizes
    return synth.splom(rows=30_000, dims=5, comps=4, seed=8)


@pytest.mark.parametrize("r,launches", [(0, "1"), (-1, "1"), (-1, "0"), (0, "0")])
def test_batch_matches_panels_alone(dc, panels, r, launches):
    # batched launches per resolution class ("1") or one branch per panel
    # ("0"): bit-identical to every panel regularised on its own
    iters = 3
    pos_b = [torch.from_numpy(z).cuda() for z, _ in panels]
    batch = dc.declutter_batch_create([k for _, k in panels], [z.shape[0] for z, _ in panels], kernel_r=r,
                                      options=dc.DC_OPT_BATCHED_LAUNCHES if launches == "1" else 0)
    try:
        u_b = dc.declutter_batch_regularize(batch, pos_b, iters, uniformity=True)
        # second call replays the cached graph
        pos_b2 = [torch.from_numpy(z).cuda() for z, _ in panels]
        dc.declutter_batch_regularize(batch, pos_b2, iters)
        dc.declutter_batch_sync(batch)
    finally:
        dc.declutter_batch_destroy(batch)
    for k, (z, log2) in enumerate(panels):
        ctx = dc.declutter_create(log2, kernel_r=r)
        try:
            pos = torch.from_numpy(z).cuda()
            u = dc.regularize(ctx, pos, iters, uniformity=True)
        finally:
            dc.declutter_destroy(ctx)
        assert torch.equal(pos, pos_b[k]), k
        assert torch.equal(pos, pos_b2[k]), k
        assert u == u_b[k], k


def test_batch_panel_against_oracle(dc, panels):
    # one panel of the batch, one teacher-forced iteration, against the oracle
    z, log2 = panels[1]
    p = oracle.Params(log2_res=log2, kernel_r=-1)
    ref = oracle.iterate(z, p)
    pos = [torch.from_numpy(zz).cuda() for zz, _ in panels]
    batch = dc.declutter_batch_create([k for _, k in panels], [zz.shape[0] for zz, _ in panels])
    try:
        dc.declutter_batch_regularize(batch, pos, 1)
        dc.declutter_batch_sync(batch)
    finally:
        dc.declutter_batch_destroy(batch)
    N = 1 << log2
    err = float(np.max(np.abs(pos[1].cpu().numpy().astype(np.float64) - ref))) * N
    assert err <= 1e-4 + N * float(np.spacing(np.float32(1.0))), err


def test_autotune_band_rows(dc, panels):
    z, log2 = panels[2]
    pos = torch.from_numpy(z).cuda()
    before = pos.clone()
    T, ms = dc.declutter_autotune_band_rows(pos, 2, log2, kernel_r=0)
    N = 1 << log2
    # a power of two or the automatic one-band-per-SM height, at most 1024 bands
    assert 1 <= T <= 64 and T <= N and (N + T - 1) // T <= 1024
    assert ms > 0
    assert torch.equal(pos, before)              # samples untouched
    T2, ms2 = dc.declutter_autotune_band_rows(pos, 2, log2, kernel_r=0)
    assert T2 == T and ms2 == -1.0               # cached answer
    # exact mode: every band height gives the same bits
    outs = []
    for bt in (0, T):
        ctx = dc.declutter_create(log2, kernel_r=0, band_rows=bt)
        try:
            q = torch.from_numpy(z).cuda()
            dc.regularize(ctx, q, 2)
            dc.declutter_sync(ctx)
            outs.append(q)
        finally:
            dc.declutter_destroy(ctx)
    assert torch.equal(outs[0], outs[1])


@pytest.mark.parametrize("r", [2, 0])
def test_autotune_options_and_cache_file(dc, panels, tmp_path, r):
    # band heights x launch sequences: the tuned settings give the bits of
    # the default ones; the cache survives a save, clear and load
    z, log2 = panels[1]
    pos = torch.from_numpy(z).cuda()
    before = pos.clone()
    dc.declutter_autotune_clear()
    T, opts, ms = dc.declutter_autotune(pos, 2, log2, kernel_r=r)
    assert ms > 0 and torch.equal(pos, before)
    assert opts & ~(dc.DC_OPT_FUSED_BANDS | dc.DC_OPT_SEPARATE_SMOOTH) == 0
    path = tmp_path / "tune.txt"
    dc.declutter_autotune_save(str(path))
    dc.declutter_autotune_clear()
    dc.declutter_autotune_load(str(path))
    T2, opts2, ms2 = dc.declutter_autotune(pos, 2, log2, kernel_r=r)
    assert (T2, opts2, ms2) == (T, opts, -1.0)
    outs = []
    for bt, o in ((0, 0), (T, opts)):
        ctx = dc.declutter_create(log2, kernel_r=r, band_rows=bt, options=o)
        try:
            q = torch.from_numpy(z).cuda()
            dc.regularize(ctx, q, 1)
            dc.declutter_sync(ctx)
            outs.append(q)
        finally:
            dc.declutter_destroy(ctx)
    if r == 0:  # exact mode: every band height gives the same bits
        assert torch.equal(outs[0], outs[1])
    else:  # float mode: the band height changes the order of the float
        # sums; both fields are within 1e-4 px of FP64
        assert float((outs[0] - outs[1]).abs().max()) * (1 << log2) <= 2e-4 + 2 * (1 << log2) * 2.0 ** -23
    print(f"r={r}: band rows {T}, options {opts}, {ms:.3f} ms")


def test_batch_autotune_keeps_results(dc, panels):
    pos_a = [torch.from_numpy(z).cuda() for z, _ in panels]
    pos_b = [torch.from_numpy(z).cuda() for z, _ in panels]
    batch = dc.declutter_batch_create([k for _, k in panels], [z.shape[0] for z, _ in panels], kernel_r=0)
    try:
        dc.declutter_batch_regularize(batch, pos_a, 2)
        rows = dc.declutter_batch_autotune(batch, pos_b, 2)
        assert len(rows) == len(panels)
        dc.declutter_batch_regularize(batch, pos_b, 2)
        dc.declutter_batch_sync(batch)
    finally:
        dc.declutter_batch_destroy(batch)
    for a, b in zip(pos_a, pos_b):
        assert torch.equal(a, b)


@pytest.mark.parametrize("launches", ["0", "1"])
def test_batch_with_empty_and_tiny_panels(dc, launches):
    # a class with an empty panel, a one-sample panel and a full one
    rng = np.random.default_rng(3)
    zs = [np.zeros((0, 2), np.float32), rng.random((1, 2)).astype(np.float32),
          rng.random((5000, 2)).astype(np.float32), rng.random((700, 2)).astype(np.float32)]
    log2s = [8, 8, 8, 9]
    pos_b = [torch.from_numpy(z).cuda() for z in zs]
    batch = dc.declutter_batch_create(log2s, [max(1, z.shape[0]) for z in zs],
                                      options=dc.DC_OPT_BATCHED_LAUNCHES if launches == "1" else 0)
    try:
        u_b = dc.declutter_batch_regularize(batch, pos_b, 2, uniformity=True)
        dc.declutter_batch_sync(batch)
    finally:
        dc.declutter_batch_destroy(batch)
    for k, (z, log2) in enumerate(zip(zs, log2s)):
        ctx = dc.declutter_create(log2)
        try:
            pos = torch.from_numpy(z).cuda()
            u = dc.regularize(ctx, pos, 2, uniformity=True) if z.shape[0] else None
        finally:
            dc.declutter_destroy(ctx)
        assert torch.equal(pos, pos_b[k]), k
        if u is not None:
            assert u == u_b[k], k
