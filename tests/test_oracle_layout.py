"""Pins of oracle/layout.py (CPU only): the transition blend (Sec. 1), the
layout metrics of Sec. 6.2 (trustworthiness, orthogonal ordering), the
stopping criteria of Sec. 4.3 step 4 and the warped density texture of
Sec. 5, each against something other than itself: a library routine,
closed forms, brute force on tiny inputs, exact rational arithmetic."""

from fractions import Fraction
from math import comb

import numpy as np
import pytest

import oracle
import synth
from oracle import layout as L


# --------------------------------------------------------------------------
# transition
# --------------------------------------------------------------------------

def test_transition_endpoints_exact_and_rounding():
    rng = np.random.default_rng(0)
    a = rng.random((500, 2)).astype(np.float32)
    b = rng.random((500, 2)).astype(np.float32)
    assert np.array_equal(L.transition(a, b, 0.0), a)
    assert np.array_equal(L.transition(a, b, 1.0), b)
    for s in (0.25, 0.5, 0.7):
        got = L.transition(a, b, s)
        s32 = Fraction(float(np.float32(s)))
        for k in range(0, 500, 37):
            for c in range(2):
                exact = (1 - s32) * Fraction(float(a[k, c])) + s32 * Fraction(float(b[k, c]))
                # three float32 roundings of values below 1: within 2^-23
                assert abs(Fraction(float(got[k, c])) - exact) <= Fraction(1, 2 ** 23)


# --------------------------------------------------------------------------
# trustworthiness and orthogonal ordering
# --------------------------------------------------------------------------

def test_quantise_lattice():
    z = np.array([[0.0, 1.0], [0.5, np.nan], [-1.0, 2.0], [1.0 / 65535, 65534 / 65535]], np.float32)
    q = L.quantise(z)
    assert q.tolist() == [[0, 65535], [32768, 0], [0, 65535], [1, 65534]]


def _lattice_layout(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.choice(65536, size=(n, 2), replace=True)
    return X, (X / 65535.0).astype(np.float32)


def _tie_free(X):
    # no two samples at the same distance from any sample
    for i in range(X.shape[0]):
        d = ((X - X[i]) ** 2).sum(1)
        if np.unique(d).size != d.size:
            return False
    return True


def test_trustworthiness_matches_sklearn():
    manifold = pytest.importorskip("sklearn.manifold")
    for seed in range(20):
        Xo, zo = _lattice_layout(120, seed)
        Xn, zn = _lattice_layout(120, seed + 1000)
        # a layout that keeps some structure: half-way towards the original
        Xn = (Xo + Xn) // 2
        zn = (Xn / 65535.0).astype(np.float32)
        if _tie_free(Xo) and _tie_free(Xn):
            break
    assert np.array_equal(L.quantise(zo), Xo) and np.array_equal(L.quantise(zn), Xn)
    for k in (1, 5, 12):
        ref = manifold.trustworthiness(Xo.astype(np.float64), Xn.astype(np.float64), n_neighbors=k)
        got = L.layout_metrics(zo, zn, k)["trustworthiness"]
        assert abs(got - ref) <= 1e-12, (k, got, ref)


def test_metrics_of_identity_mirror_and_shuffle():
    Xo, zo = _lattice_layout(300, 7)
    m = L.layout_metrics(zo, zo, 8)
    assert m["trustworthiness"] == 1.0 and m["ordering"] == 1.0
    # the mirror x -> 1 - x keeps every distance, and reverses the x order of
    # every pair with distinct x
    Xm = Xo.copy()
    Xm[:, 0] = 65535 - Xm[:, 0]
    zm = (Xm / 65535.0).astype(np.float32)
    assert np.array_equal(L.quantise(zm), Xm)
    m = L.layout_metrics(zo, zm, 8)
    assert m["trustworthiness"] == 1.0
    n = Xo.shape[0]
    _, cnt = np.unique(Xo[:, 0], return_counts=True)
    flipped = comb(n, 2) - sum(comb(int(c), 2) for c in cnt)
    assert abs(m["ordering"] - (1.0 - flipped / comb(n, 2))) <= 1e-15
    # a random assignment of positions keeps nothing: T near 1/2
    perm = np.random.default_rng(1).permutation(n)
    m = L.layout_metrics(zo, zo[perm], 5)
    assert 0.35 < m["trustworthiness"] < 0.65, m["trustworthiness"]


def test_ordering_brute_force_and_query_subsets():
    rng = np.random.default_rng(3)
    zo = rng.random((60, 2)).astype(np.float32)
    zn = (zo + rng.normal(0, 0.05, zo.shape)).clip(0, 1).astype(np.float32)
    Xo, Xn = L.quantise(zo), L.quantise(zn)
    bad = 0
    for i in range(60):
        for j in range(i + 1, 60):
            keep_x = np.sign(Xo[i, 0] - Xo[j, 0]) == np.sign(Xn[i, 0] - Xn[j, 0])
            keep_y = np.sign(Xo[i, 1] - Xo[j, 1]) == np.sign(Xn[i, 1] - Xn[j, 1])
            bad += not (keep_x and keep_y)
    m = L.layout_metrics(zo, zn, 4)
    assert abs(m["ordering"] - (1.0 - bad / comb(60, 2))) <= 1e-15
    # the estimate over a subset of queries sums the same per-query terms
    q = np.array([3, 17, 59])
    sub = L.layout_metrics(zo, zn, 4, queries=q)
    assert np.array_equal(sub["o_terms"], m["o_terms"][q])
    assert np.array_equal(sub["t_terms"], m["t_terms"][q])


def test_trustworthiness_brute_force_ranks():
    # ranks by an explicit sort of (distance, index) pairs
    rng = np.random.default_rng(5)
    zo = rng.random((40, 2)).astype(np.float32)
    zn = rng.random((40, 2)).astype(np.float32)
    Xo, Xn = L.quantise(zo), L.quantise(zn)
    k = 3
    total = 0
    for i in range(40):
        oo = sorted((int(((Xo[j] - Xo[i]) ** 2).sum()), j) for j in range(40) if j != i)
        on = sorted((int(((Xn[j] - Xn[i]) ** 2).sum()), j) for j in range(40) if j != i)
        rank = {j: r + 1 for r, (_, j) in enumerate(oo)}
        nn_o = {j for _, j in oo[:k]}
        total += sum(rank[j] - k for _, j in on[:k] if j not in nn_o)
    T = 1.0 - 2.0 / (40 * k * (2 * 40 - 3 * k - 1)) * total
    assert abs(L.layout_metrics(zo, zn, k)["trustworthiness"] - T) <= 1e-15


# --------------------------------------------------------------------------
# stopping criteria
# --------------------------------------------------------------------------

def test_regularize_until_criteria():
    z, _ = synth.tiny_mixture(6000, seed=2)
    p = oracle.Params(log2_res=6, kernel_r=2)
    full = L.regularize_until(z, p, 5)
    assert full["iters"] == 5
    assert np.array_equal(full["pos"], oracle.regularize(z, p, 5)[-1])
    cv = full["cv"]
    assert all(a > b for a, b in zip(cv, cv[1:])), cv
    # the first iteration whose measure reaches the target ends the run
    tgt = 0.5 * (cv[2] + cv[3])
    r = L.regularize_until(z, p, 5, target_cv=tgt)
    assert r["iters"] == 4 and np.array_equal(r["pos"], oracle.regularize(z, p, 4)[-1])
    assert L.regularize_until(z, p, 5, target_cv=10.0)["iters"] == 1
    mv = full["move_px"]
    r = L.regularize_until(z, p, 5, min_move_px=0.5 * (mv[1] + mv[2]))
    assert r["iters"] == 3
    # the move is the largest sample displacement of the iteration
    t = oracle.regularize(z, p, 2)
    d = np.abs(t[2].astype(np.float64) - t[1].astype(np.float64))
    assert abs(mv[1] - np.sqrt((d ** 2).sum(1)).max() * 64) <= 1e-12


# --------------------------------------------------------------------------
# warped density texture
# --------------------------------------------------------------------------

def _containing(nodes, log2M, p, q):
    # brute force: triangles whose closed region holds the pixel centre,
    # and whether it lies on an edge or a vertex of one
    N = nodes.shape[0]
    V = L._fixed(nodes, log2M)
    cx, cy = (p << L.SUB) + (1 << (L.SUB - 1)), (q << L.SUB) + (1 << (L.SUB - 1))
    hits = []
    for t, tri in enumerate(L._tri_vertices(N)):
        pts = [(int(V[j, i, 0]), int(V[j, i, 1])) for i, j in tri]
        e = []
        for a in range(3):
            (ux, uy), (vx, vy) = pts[a], pts[(a + 1) % 3]
            e.append((vx - ux) * (cy - uy) - (vy - uy) * (cx - ux))
        if all(x >= 0 for x in e) or all(x <= 0 for x in e):
            hits.append(t)
    return hits


@pytest.mark.parametrize("pixel_center", [False, True])
def test_coverage_is_watertight(pixel_center):
    # a smoothly deformed 12 x 12 mesh on a 32 x 32 raster: every pixel
    # centre strictly inside one triangle is covered by it, and every centre
    # on shared edges or vertices by exactly one of the triangles holding it
    N, log2M = 12, 5
    nodes = L.identity_nodes(N, pixel_center).astype(np.float64)
    x, y = nodes[..., 0], nodes[..., 1]
    nodes[..., 0] = x + 0.04 * np.sin(np.pi * x) * np.sin(2 * np.pi * y)
    nodes[..., 1] = y + 0.04 * np.sin(2 * np.pi * x) * np.sin(np.pi * y)
    nodes = nodes.astype(np.float32)
    cov = L.coverage(nodes, log2M)
    M = 1 << log2M
    for q in range(M):
        for p in range(M):
            hits = _containing(nodes, log2M, p, q)
            if not hits:
                assert cov[q, p] == -1
            else:
                assert cov[q, p] in hits, (p, q, hits, cov[q, p])


def test_identity_mesh_reproduces_the_texture():
    rng = np.random.default_rng(4)
    N = 16
    tex = rng.random((N, N))
    # pixel centres on the nodes: every covered pixel is its node's value
    out, cov = L.warp_texture(L.identity_nodes(N, True), tex, 4, pixel_center=True)
    inner = cov[:-1, :-1] >= 0
    assert inner.all()
    assert np.max(np.abs(out[:-1, :-1] - tex[:-1, :-1])) <= 1e-12
    # literal pixel positions: the centre of cell (p, q) is the mean of its corners
    out, cov = L.warp_texture(L.identity_nodes(N, False), tex, 4)
    mean4 = 0.25 * (tex[:-1, :-1] + tex[:-1, 1:] + tex[1:, :-1] + tex[1:, 1:])
    assert np.max(np.abs(out[:-1, :-1] - mean4)) <= 1e-12
    assert np.all(cov[-1, :] == -1) and np.all(cov[:, -1] == -1)


def test_scaled_mesh_and_mass_factor():
    # nodes scaled by 1/2 about the origin: pixel (p, q) samples node
    # (2p + 1, 2q + 1); the push-forward multiplies by the area ratio 4
    rng = np.random.default_rng(6)
    N = 16
    tex = rng.random((N, N))
    nodes = (L.identity_nodes(N) * np.float32(0.5)).astype(np.float32)
    out, _ = L.warp_texture(nodes, tex, 4)
    outm, _ = L.warp_texture(nodes, tex, 4, mass=True)
    for q in range(7):
        for p in range(7):
            assert abs(out[q, p] - tex[2 * q + 1, 2 * p + 1]) <= 1e-12
            assert abs(outm[q, p] - 4.0 * tex[2 * q + 1, 2 * p + 1]) <= 1e-11


def test_push_forward_keeps_the_mass():
    N, log2M = 32, 6
    jj, ii = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    tex = 1.0 + np.exp(-((ii - 10.0) ** 2 + (jj - 20.0) ** 2) / 30.0) * 5.0
    nodes = L.identity_nodes(N).astype(np.float64)
    x, y = nodes[..., 0] * N / (N - 1), nodes[..., 1] * N / (N - 1)  # [0, 1] on the mesh
    nodes[..., 0] += 0.05 * np.sin(np.pi * x) * np.sin(np.pi * y) * (N - 1) / N
    nodes[..., 1] += 0.03 * np.sin(2 * np.pi * x) * np.sin(np.pi * y) * (N - 1) / N
    nodes = nodes.astype(np.float32)
    ident, _ = L.warp_texture(L.identity_nodes(N), tex, log2M, mass=True)
    warped, _ = L.warp_texture(nodes, tex, log2M, mass=True)
    assert abs(warped.sum() / ident.sum() - 1.0) < 0.01


def test_transfer_closed_form():
    lut = np.arange(256, dtype=np.uint32) * 3 + 7
    v = np.array([0.0, 1.0, 0.5, -3.0, 9.0, np.nan, 0.25, 1.0 / 255.0], np.float32)
    got = L.transfer(v, 0.0, 1.0, lut)
    # rint(127.5) = 128 (ties to even), rint(63.75) = 64
    assert got.tolist() == [7, 7 + 3 * 255, 7 + 3 * 128, 7, 7 + 3 * 255, 7, 7 + 3 * 64, 7 + 3]
    g2 = L.transfer(np.array([2.0, 6.0], np.float32), 2.0, 6.0, lut)
    assert g2.tolist() == [7, 7 + 3 * 255]
