"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test checks one oracle function against brute force from the paper's
definitions, a closed form, a library routine, or a geometric fact about the
printed formulas, chosen so that a dropped term, a wrong sign or index, or a
transposed operand in the oracle fails at least one of them.
"""

import itertools
import math
import os

import numpy as np
import pytest
import scipy.ndimage as ndi
from scipy.interpolate import RegularGridInterpolator

import oracle
import synth

pytestmark = pytest.mark.usefixtures("oracle_lib")


# --------------------------------------------------------------------------
# Sec. 4.1: single-pixel accumulation
# --------------------------------------------------------------------------

def test_splat_matches_histogram2d():
    z, _ = synth.tiny_mixture(20_000, seed=7)
    for k in (4, 5, 7):
        N = 1 << k
        c = oracle.splat(z, k)
        # np.histogram2d: bins [m/N, (m+1)/N), last bin closed -- the floor rule
        h, _, _ = np.histogram2d(z[:, 1].astype(np.float64), z[:, 0].astype(np.float64),
                                 bins=N, range=[[0, 1], [0, 1]])
        assert c.sum() == z.shape[0]
        assert np.array_equal(c, h.astype(np.uint64))


def test_splat_clamps_out_of_range_and_edges():
    z = np.array([[-0.5, 0.2], [1.0, 1.0], [2.0, -3.0], [0.999999, 0.0], [np.nan, 0.5]], np.float32)
    c = oracle.splat(z, 4)
    assert c[int(0.2 * 16), 0] == 1        # x < 0 -> column 0
    assert c[15, 15] == 1                   # (1, 1) -> last pixel
    assert c[0, 15] == 2                    # (2, -3) -> (15, 0); (0.999999, 0) -> (15, 0)
    assert c[8, 0] == 1                     # NaN x -> column 0
    assert c.sum() == 5


# --------------------------------------------------------------------------
# Sec. 4.1 / 4.4: Gaussian smoothing
# --------------------------------------------------------------------------

@pytest.mark.parametrize("r,sigma", [(2, 0.0), (4, 0.0), (8, 2.5)])
def test_gauss_weights(r, sigma):
    g = oracle.gauss_weights(r, sigma)
    s = sigma if sigma > 0 else r / 3.0
    assert abs(g.sum() - 1.0) < 1e-15
    assert np.allclose(g, g[::-1], rtol=0, atol=1e-18)
    # ratio of neighbouring taps is exp(-(2k+1)/(2 s^2)) for a Gaussian
    for k in range(r):
        assert math.isclose(g[r + k + 1] / g[r + k], math.exp(-(2 * k + 1) / (2 * s * s)), rel_tol=1e-12)


@pytest.mark.parametrize("r", [1, 3, 6])
def test_smooth_matches_scipy_reflect(r):
    rng = np.random.default_rng(r)
    a = rng.integers(0, 50, size=(32, 32)).astype(np.float64)
    g = oracle.gauss_weights(r)
    ref = ndi.correlate1d(ndi.correlate1d(a, g, axis=1, mode="reflect"), g, axis=0, mode="reflect")
    out = oracle.smooth(a, r)
    assert np.max(np.abs(out - ref)) < 1e-11


def test_smooth_preserves_mass_constants_and_impulse():
    r = 4
    a = np.zeros((32, 32))
    a[16, 10] = 7.0
    out = oracle.smooth(a, r)
    g = oracle.gauss_weights(r)
    assert abs(out.sum() - 7.0) < 1e-12
    assert np.allclose(out[16 - r:16 + r + 1, 10 - r:10 + r + 1], 7.0 * np.outer(g, g), atol=1e-14)
    # mass also preserved for an impulse at the border (reflection)
    b = np.zeros((16, 16))
    b[0, 0] = 3.0
    b[15, 7] = 2.0
    assert abs(oracle.smooth(b, 5).sum() - 5.0) < 1e-12
    c = np.full((16, 16), 2.5)
    assert np.max(np.abs(oracle.smooth(c, 5) - 2.5)) < 1e-13


# --------------------------------------------------------------------------
# Sec. 3.1: integral images
# --------------------------------------------------------------------------

def brute_inims(d):
    """The Sec. 3.1 definitions summed term by term."""
    N = d.shape[0]
    out = {k: np.zeros((N, N)) for k in oracle.INIM_NAMES}
    for j, i in itertools.product(range(N), range(N)):
        u, v = i + j, i - j
        for jp, ip in itertools.product(range(N), range(N)):
            w = d[jp, ip]
            up, vp = ip + jp, ip - jp
            if ip <= i and jp <= j:
                out["alpha"][j, i] += w
            if ip <= i and jp > j:
                out["beta"][j, i] += w
            if ip > i and jp > j:
                out["gamma"][j, i] += w
            if ip > i and jp <= j:
                out["delta"][j, i] += w
            if up <= u and vp >= v:
                out["alpha_t"][j, i] += w
            if up <= u and vp < v:
                out["beta_t"][j, i] += w
            if up > u and vp < v:
                out["gamma_t"][j, i] += w
            if up > u and vp >= v:
                out["delta_t"][j, i] += w
    return out


@pytest.mark.parametrize("N", [4, 7, 8])
def test_inims_brute_force(N):
    rng = np.random.default_rng(N)
    d = rng.random((N, N))
    got = oracle.inims(d)
    ref = brute_inims(d)
    for k in oracle.INIM_NAMES:
        assert np.max(np.abs(got[k] - ref[k])) < 1e-12, k


def test_inims_partition_and_cumsum():
    rng = np.random.default_rng(3)
    d = rng.random((32, 32))
    ims = oracle.inims(d)
    C = d.sum()
    assert np.max(np.abs(ims["alpha"] + ims["beta"] + ims["gamma"] + ims["delta"] - C)) < 1e-10
    assert np.max(np.abs(ims["alpha_t"] + ims["beta_t"] + ims["gamma_t"] + ims["delta_t"] - C)) < 1e-10
    assert np.max(np.abs(ims["alpha"] - np.cumsum(np.cumsum(d, axis=0), axis=1))) < 1e-10
    # monotone: alpha non-decreasing in i and j, alpha_t in j (Sec. 5)
    assert np.all(np.diff(ims["alpha"], axis=0) >= -1e-12)
    assert np.all(np.diff(ims["alpha"], axis=1) >= -1e-12)
    assert np.all(np.diff(ims["alpha_t"], axis=0) >= -1e-12)


def lattice_alpha_t(i, j, N):
    """Pixels of the clipped upward cone, a closed form."""
    def tri(m):
        return m * (m + 1) // 2 if m > 0 else 0
    return (j + 1) ** 2 - tri(j - (N - 1 - i)) - tri(j - i)


@pytest.mark.parametrize("N", [8, 16])
def test_inims_constant_closed_form(N):
    ims = oracle.inims(np.ones((N, N)))
    jj, ii = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    assert np.array_equal(ims["alpha"], (ii + 1) * (jj + 1))
    assert np.array_equal(ims["gamma"], (N - 1 - ii) * (N - 1 - jj))
    at = np.vectorize(lambda i, j: lattice_alpha_t(i, j, N))(ii, jj)
    assert np.array_equal(ims["alpha_t"], at)


def test_inims_single_pixel_delta():
    N, m = 16, 5.0
    for (i0, j0) in [(0, 0), (3, 9), (15, 2), (7, 15)]:
        d = np.zeros((N, N))
        d[j0, i0] = m
        ims = oracle.inims(d)
        jj, ii = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
        assert np.array_equal(ims["alpha"], m * ((ii >= i0) & (jj >= j0)))
        cone = (jj >= j0) & (np.abs(i0 - ii) <= jj - j0)
        assert np.array_equal(ims["alpha_t"], m * cone)


def test_sat_u64_exact():
    rng = np.random.default_rng(5)
    g = rng.integers(0, 256, size=(8, 8)).astype(np.uint32)
    a, at = oracle.sat_u64(g)
    ref = brute_inims(g.astype(np.float64))
    assert np.array_equal(a, ref["alpha"].astype(np.uint64))
    assert np.array_equal(at, ref["alpha_t"].astype(np.uint64))
    # values beyond 2^32: compare with Python integers
    big = np.full((16, 16), 0xFFFFFFFF, dtype=np.uint32)
    a, at = oracle.sat_u64(big)
    M = 0xFFFFFFFF
    for (i, j) in [(15, 15), (3, 12), (0, 15), (15, 0)]:
        assert int(a[j, i]) == M * (i + 1) * (j + 1)
        assert int(at[j, i]) == M * lattice_alpha_t(i, j, 16)
    g = synth.sat_grid(8)
    a, at = oracle.sat_u64(g)
    assert np.array_equal(a, np.cumsum(np.cumsum(g.astype(np.uint64), axis=0), axis=1))
    ims = oracle.inims(g.astype(np.float64))
    assert np.array_equal(at, ims["alpha_t"].astype(np.uint64))


# --------------------------------------------------------------------------
# Sec. 3.2: eq. (map) and its anchors, pinned by geometry
# --------------------------------------------------------------------------

def ray_hit(x, y, dx, dy):
    """Point where the ray (x, y) + s (dx, dy), s >= 0, leaves [0, 1]^2."""
    s = math.inf
    if dx > 0:
        s = min(s, (1 - x) / dx)
    if dx < 0:
        s = min(s, x / -dx)
    if dy > 0:
        s = min(s, (1 - y) / dy)
    if dy < 0:
        s = min(s, y / -dy)
    return x + s * dx, y + s * dy


def point_mass_map(N, ip, jp, i, j, off=0.0):
    """Mapping of pixel (i, j) under a unit mass at (ip, jp), from geometry.

    A mass in one of the four axis quadrants pushes the pixel along the
    diagonal pointing away from that quadrant until it meets the border; a
    mass in one of the four tilted wedges pushes it along the axis pointing
    away from that wedge.  The mapping is the mean of the two border points
    (weights C + C over 2C).  Quadrant and wedge membership follow the
    inequalities of Sec. 3.1.
    """
    x, y = (i + off) / N, (j + off) / N
    if ip <= i and jp <= j:
        diag = (1, 1)
    elif ip <= i and jp > j:
        diag = (1, -1)
    elif ip > i and jp > j:
        diag = (-1, -1)
    else:
        diag = (-1, 1)
    u, v, up, vp = i + j, i - j, ip + jp, ip - jp
    if up <= u and vp >= v:
        ax = (0, 1)      # mass above: push down
    elif up <= u and vp < v:
        ax = (1, 0)      # mass to the left: push right
    elif up > u and vp < v:
        ax = (0, -1)     # mass below: push up
    else:
        ax = (-1, 0)     # mass to the right: push left
    h1 = ray_hit(x, y, *diag)
    h2 = ray_hit(x, y, *ax)
    return (h1[0] + h2[0]) / 2, (h1[1] + h2[1]) / 2


@pytest.mark.parametrize("pixel_center", [False, True])
def test_mapping_point_masses_geometry(pixel_center):
    N = 8
    off = 0.5 if pixel_center else 0.0
    for ip, jp in itertools.product(range(N), range(N)):
        d = np.zeros((N, N))
        d[jp, ip] = 1.0
        t = oracle.mapping(d, pixel_center)
        for i, j in itertools.product(range(N), range(N)):
            ex = point_mass_map(N, ip, jp, i, j, off)
            assert abs(t[j, i, 0] - ex[0]) < 1e-14 and abs(t[j, i, 1] - ex[1]) < 1e-14, (ip, jp, i, j)


@pytest.mark.parametrize("N,pixel_center", [(8, False), (16, False), (8, True)])
def test_mapping_is_mass_weighted_mean_of_point_maps(N, pixel_center):
    # X(d) is linear in d and C is its total, so t(.; d) is the d/C-weighted
    # mean of the point-mass mappings.
    rng = np.random.default_rng(N + pixel_center)
    d = rng.random((N, N)) ** 3
    off = 0.5 if pixel_center else 0.0
    t = oracle.mapping(d, pixel_center)
    C = d.sum()
    for i, j in [(0, 0), (N - 1, N - 1), (2, 5), (5, 2), (N - 1, 0), (0, N - 1), (3, 3), (N // 2, N // 2 - 1)]:
        ex = np.zeros(2)
        for ip, jp in itertools.product(range(N), range(N)):
            ex += d[jp, ip] / C * np.array(point_mass_map(N, ip, jp, i, j, off))
        assert np.max(np.abs(t[j, i] - ex)) < 1e-13


def test_mapping_properties():
    N = 32
    rng = np.random.default_rng(9)
    d = ndi.gaussian_filter(rng.random((N, N)) ** 4, 2) + 1e-3
    t = oracle.mapping(d)
    assert t.min() >= 0.0 and t.max() <= 1.0
    # the mapping of a constant texture is not the identity (Sec. 3.2) ...
    t1 = oracle.mapping(np.ones((N, N)))
    jj, ii = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    ident = np.stack([ii / N, jj / N], axis=-1)
    assert np.max(np.abs(t1 - ident)) > 1e-2
    # ... but it does not depend on the constant's value
    assert np.max(np.abs(oracle.mapping(np.full((N, N), 7.25)) - t1)) < 1e-14
    # and the mapping is homogeneous of degree 0 in d
    assert np.max(np.abs(oracle.mapping(3.0 * d) - t)) < 1e-14


# --------------------------------------------------------------------------
# Sec. 4.2: eq. (map_res)
# --------------------------------------------------------------------------

def test_unit_mass_worked_example():
    # hand-derived worked example (tests/golden/unit_mass_4x4.txt, Sec. 3.1,
    # eq. (map), Sec. 4.1-4.2): one sample at pixel (1, 2) of a 4x4 grid;
    # the constant texture's numerator X(1), t(.; c + d0) and D at four
    # pixels, all exact binary fractions
    path = os.path.join(os.path.dirname(__file__), "golden", "unit_mass_4x4.txt")
    rows = np.loadtxt(path, comments="#")
    N = 4
    c = np.zeros((N, N))
    c[2, 1] = 1.0  # [j][i]
    d0 = 1.0 / 16
    t1 = oracle.mapping(np.ones((N, N)))
    td = oracle.mapping(c + d0)
    D = oracle.displacement(c, d0)
    assert rows.shape == (4, 8)
    for i, j, x1x, x1y, tdx, tdy, dx, dy in rows:
        i, j = int(i), int(j)
        assert np.array_equal(t1[j, i] * (2 * N * N), [x1x, x1y]), (i, j)
        assert np.array_equal(td[j, i], [tdx, tdy]), (i, j)
        assert np.array_equal(D[j, i], [dx, dy]), (i, j)


def test_lens_of_constant_density_from_worked_example():
    # end of Sec. 3.2: eq. (map) is not the identity for a constant texture;
    # its lens displacement is t(1) - p = X(1) / (2 N^2) - p, with X(1) from
    # the hand-derived fixture (tests/golden/unit_mass_4x4.txt)
    rows = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "unit_mass_4x4.txt"), comments="#")
    N = 4
    L = oracle.lens_displacement(np.full((N, N), 3.0))
    for i, j, x1x, x1y, *_ in rows:
        i, j = int(i), int(j)
        want = [x1x / (2 * N * N) - i / N, x1y / (2 * N * N) - j / N]
        assert np.array_equal(L[j, i], want), (i, j)
        assert np.any(L[j, i] != 0.0)


def test_lens_magnifies_the_selected_area():
    # end of Sec. 3.2: the density is constant inside and outside the
    # selected area, and a larger value inside magnifies the area more
    N = 32
    spans = []
    for inside in (1.0, 2.0, 4.0, 8.0):
        d = np.ones((N, N))
        d[12:20, 12:20] = inside
        L = oracle.lens_displacement(d)
        xs = (np.arange(N) / N)[None, :] + L[:, :, 0]
        ys = (np.arange(N) / N)[:, None] + L[:, :, 1]
        spans.append((xs[12:20, 12:20].max() - xs[12:20, 12:20].min(), ys[12:20, 12:20].max() - ys[12:20, 12:20].min()))
        assert np.all(xs >= 0.0) and np.all(xs <= 1.0) and np.all(ys >= 0.0) and np.all(ys <= 1.0)
    for a, b in zip(spans, spans[1:]):
        assert b[0] > a[0] and b[1] > a[1], spans


def _segset(segs):
    return sorted(tuple(sorted(seg)) for seg in segs)


def test_contour_saddle_cells_by_hand():
    # Sec. 5 contour lines (marching squares): a 2x2 checkerboard, nodes at
    # 0 and 1/2; the saddle follows the cell centre (mean 0.5)
    f = np.array([[1.0, 0.0], [0.0, 1.0]], np.float32)
    # level 0.5: centre inside, the outside corners (1/2, 0) and (0, 1/2) are cut off
    assert _segset(oracle.contour_cell(f, 0.5, 0, 0)) == _segset(
        [((0.25, 0.0), (0.5, 0.25)), ((0.25, 0.5), (0.0, 0.25))])
    # level 0.625: centre outside, the inside corners (0, 0) and (1/2, 1/2) are cut off
    assert _segset(oracle.contour_cell(f, 0.625, 0, 0)) == _segset(
        [((0.1875, 0.0), (0.0, 0.1875)), ((0.5, 0.3125), (0.3125, 0.5))])


def test_contour_of_a_ramp_is_straight():
    # f(i, j) = i: the level 10.5 crosses only the cells of column 10, at
    # x = 10.5 / N, each from row j to row j + 1
    N = 32
    f = np.tile(np.arange(N, dtype=np.float32), (N, 1))
    cells = oracle.contour_segments(f, 10.5)
    for c, segs in enumerate(cells):
        j, i = divmod(c, N - 1)
        if i == 10:
            assert _segset(segs) == _segset([((10.5 / N, j / N), (10.5 / N, (j + 1) / N))])
        else:
            assert segs == []


def test_contour_of_a_distance_field_is_a_closed_circle():
    # f = distance (pixels) to the centre: the level R contour lies on the
    # circle up to the chord error of linear interpolation (< 1 / (8 R) px),
    # its length is 2 pi R within 1 %, and every vertex ends two segments
    N, R = 64, 20.0
    jj, ii = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    f = np.sqrt((ii - 31.3) ** 2 + (jj - 30.6) ** 2).astype(np.float32)
    segs = [s for cell in oracle.contour_segments(f, R) for s in cell]
    pts = np.array([p for s in segs for p in s]) * N
    d = np.hypot(pts[:, 0] - 31.3, pts[:, 1] - 30.6)
    assert np.all(np.abs(d - R) < 1.0 / (8 * R) + 1e-5)
    length = sum(np.hypot((b[0] - a[0]) * N, (b[1] - a[1]) * N) for a, b in segs)
    assert abs(length - 2 * np.pi * R) < 0.01 * 2 * np.pi * R
    ends = {}
    for s in segs:
        for p in s:
            k = (round(p[0], 9), round(p[1], 9))
            ends[k] = ends.get(k, 0) + 1
    assert set(ends.values()) == {2}


def test_displacement_uniform_is_zero_and_identities():
    N = 32
    D = oracle.displacement(np.full((N, N), 4.0), d0=4.0 / 1.0)
    assert np.max(np.abs(D)) < 1e-14
    rng = np.random.default_rng(2)
    d_r = ndi.gaussian_filter(rng.random((N, N)) ** 4 * 10, 1.5)
    n = d_r.sum()
    d0 = n / N**2
    D = oracle.displacement(d_r, d0)
    # homogeneity: scaling d_r and d0 together leaves D unchanged
    assert np.max(np.abs(oracle.displacement(5 * d_r, 5 * d0) - D)) < 1e-14
    # D = lam * (t(d_r) - t(1)) with lam = C_r / (C_r + d0 N^2)
    lam = n / (n + d0 * N * N)
    D2 = lam * (oracle.mapping(d_r) - oracle.mapping(np.ones((N, N))))
    assert np.max(np.abs(D - D2)) < 1e-14
    # no mass -> no displacement
    assert np.max(np.abs(oracle.displacement(np.zeros((N, N)), 0.0))) == 0.0


def test_displacement_pushes_away_from_cluster():
    N = 32
    d_r = np.zeros((N, N))
    d_r[8:12, 8:12] = 100.0          # cluster in the upper-left part
    D = oracle.displacement(d_r, d_r.sum() / N**2)
    # a pixel to the lower right of the cluster moves further down-right
    assert D[20, 20, 0] > 0 and D[20, 20, 1] > 0
    # a pixel to the upper left of it moves further up-left
    assert D[4, 4, 0] < 0 and D[4, 4, 1] < 0


# --------------------------------------------------------------------------
# Sec. 4.2: bilinear sample update
# --------------------------------------------------------------------------

def test_advect_nodes_linear_field_and_scipy():
    N = 16
    rng = np.random.default_rng(4)
    D = rng.normal(scale=0.01, size=(N, N, 2))
    jj, ii = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    nodes = np.stack([ii.ravel() / N, jj.ravel() / N], axis=1).astype(np.float32)
    out = oracle.advect(nodes, D, clamp=False)
    ex = (nodes.astype(np.float64) + D.reshape(-1, 2)).astype(np.float32)
    assert np.array_equal(out, ex)
    # a field linear in the pixel indices is reproduced exactly inside the grid
    L = np.stack([0.001 * ii + 0.002 * jj, -0.003 * ii + 0.0005 * jj], axis=-1)
    z = rng.uniform(0, (N - 1) / N, size=(500, 2)).astype(np.float32)
    out = oracle.advect(z, L, clamp=False)
    px = z.astype(np.float64) * N
    ex = z.astype(np.float64) + np.stack([0.001 * px[:, 0] + 0.002 * px[:, 1],
                                          -0.003 * px[:, 0] + 0.0005 * px[:, 1]], axis=1)
    assert np.max(np.abs(out - ex.astype(np.float32))) <= 1e-7
    # general field: scipy's linear grid interpolator on the pixel positions
    gx = np.arange(N) / N
    fx = RegularGridInterpolator((gx, gx), D[..., 0])   # axes (y, x)
    fy = RegularGridInterpolator((gx, gx), D[..., 1])
    out = oracle.advect(z, D, clamp=False)
    pts = np.stack([z[:, 1], z[:, 0]], axis=1).astype(np.float64)
    ex = z.astype(np.float64) + np.stack([fx(pts), fy(pts)], axis=1)
    assert np.max(np.abs(out - ex.astype(np.float32))) <= 1e-7


def test_advect_border_and_clamp():
    N = 8
    D = np.zeros((N, N, 2))
    D[..., 0] = 0.5
    D[..., 1] = -0.5
    z = np.array([[1.0, 1.0], [0.99, 0.01], [0.0, 0.0]], np.float32)
    out = oracle.advect(z, D, clamp=True)
    assert np.all((out >= 0) & (out <= 1))
    assert out[0, 0] == 1.0 and out[0, 1] == np.float32(0.5)
    out = oracle.advect(z, D, clamp=False)
    assert out[1, 0] == np.float32(0.99 + 0.5) or abs(out[1, 0] - 1.49) < 1e-6


# --------------------------------------------------------------------------
# Sec. 6.2: quality measures
# --------------------------------------------------------------------------

def test_quality_definitions():
    N = 16
    c = np.ones((N, N), dtype=np.uint64)
    q = oracle.quality(c)
    assert q["bin_std"] == 0.0 and q["overplot"] == 0.0
    c = np.zeros((N, N), dtype=np.uint64)
    c[3, 5] = 100
    q = oracle.quality(c)
    nb = (N // 4) ** 2
    mean = 100 / nb
    sd = math.sqrt(((100 - mean) ** 2 + (nb - 1) * mean**2) / nb)
    assert math.isclose(q["bin_std"], sd, rel_tol=1e-12)
    assert math.isclose(q["overplot"], 99 / 100, rel_tol=1e-12)
    rng = np.random.default_rng(1)
    c = rng.integers(0, 4, size=(N, N)).astype(np.uint64)
    b = c.reshape(N // 4, 4, N // 4, 4).sum(axis=(1, 3)).astype(np.float64)
    q = oracle.quality(c)
    assert math.isclose(q["bin_std"], b.std(), rel_tol=1e-12)
    assert math.isclose(q["overplot"], (c.sum() - np.count_nonzero(c)) / c.sum(), rel_tol=1e-12)


# --------------------------------------------------------------------------
# Sec. 4.3 / 6.2: iteration-level properties
# --------------------------------------------------------------------------

@pytest.mark.parametrize("pixel_center", [False, True])
def test_even_layout_is_fixed_point(pixel_center):
    k = 5
    z = synth.uniform_grid_samples(k, per_pixel=2, pixel_center=pixel_center)
    for r in (0, 2):
        p = oracle.Params(log2_res=k, kernel_r=r, pixel_center=pixel_center)
        new, aux = oracle.iterate(z, p, keep=True)
        assert np.max(np.abs(aux["D"])) < 1e-14
        assert np.array_equal(new, z)


def test_bin_std_and_overplot_decrease():
    z, _ = synth.tiny_mixture()
    p = oracle.Params(log2_res=7, kernel_r=2)
    traj = oracle.regularize(z, p, 4)
    qs = [oracle.quality(oracle.splat(t, 7)) for t in traj]
    stds = [q["bin_std"] for q in qs]
    ovp = [q["overplot"] for q in qs]
    assert all(a > b for a, b in zip(stds, stds[1:])), stds
    assert all(a > b for a, b in zip(ovp, ovp[1:])), ovp
    assert stds[-1] < 0.5 * stds[0]


def test_diagonal_band_spreads():
    # Fig. 3: samples along the diagonal have uniform marginals, yet the
    # method spreads them across the plot.
    z, _ = synth.diagonal_band(20_000)
    p = oracle.Params(log2_res=7, kernel_r=2)
    traj = oracle.regularize(z, p, 4)
    w0 = np.std(z[:, 0] - z[:, 1])
    w4 = np.std(traj[-1][:, 0] - traj[-1][:, 1])
    assert w4 > 2.0 * w0


def test_pixel_mapping_does_not_fold():
    # Sec. 5: no twisting; the deformed pixel grid stays ordered along rows
    # and columns for a smooth density.
    N = 64
    z, _ = synth.tiny_mixture(20_000, seed=3)
    p = oracle.Params(log2_res=6, kernel_r=2)
    _, aux = oracle.iterate(z, p, keep=True)
    jj, ii = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    mx = ii / N + aux["D"][..., 0]
    my = jj / N + aux["D"][..., 1]
    assert np.all(np.diff(mx, axis=1) > 0)
    assert np.all(np.diff(my, axis=0) > 0)
