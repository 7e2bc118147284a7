"""CPU oracle for the layout-level parts around the iteration (test
infrastructure only; same rules as the package ``oracle``: only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use
it, and it shares no code with the CUDA library).

* :func:`transition`        -- Sec. 1, continuous transition between the
  original and the regularised scatterplot (reading: a per-sample linear
  blend of the two positions)
* :func:`quantise`          -- the 2^16 lattice the layout metrics work on
* :func:`layout_metrics`    -- Sec. 6.2 (comparison with Hagrid):
  trustworthiness (Venna and Kaski) and orthogonal ordering (Misue et al.)
  of the regularised layout against the original one
* :func:`regularize_until`  -- Sec. 4.3 step 4, the stopping criteria
* :func:`warp_texture`      -- Sec. 5, the density background texture
  deformed by the mesh mapping, and its push-forward (mass) variant
* :func:`transfer`          -- Sec. 5, the transfer function to colours

Plain numpy; slow on purpose.  Every function is pinned in
``tests/test_oracle_layout.py``.
"""

from __future__ import annotations

import numpy as np

from . import iterate, quality, splat

# ---------------------------------------------------------------------------
# Sec. 1: continuous transition between the two views
# ---------------------------------------------------------------------------


def transition(orig: np.ndarray, reg: np.ndarray, s: float) -> np.ndarray:
    """Positions at blend parameter s in [0, 1]: (1 - s) orig + s reg, every
    operation rounded to float32 in this order: a = (1 - s), b = a * orig,
    c = s * reg, b + c.  s = 0 gives orig and s = 1 gives reg exactly."""
    o = np.ascontiguousarray(orig, dtype=np.float32)
    r = np.ascontiguousarray(reg, dtype=np.float32)
    s32 = np.float32(s)
    a = np.float32(np.float32(1.0) - s32)
    return (a * o).astype(np.float32) + (s32 * r).astype(np.float32)


# ---------------------------------------------------------------------------
# Sec. 6.2: trustworthiness and orthogonal ordering
# ---------------------------------------------------------------------------

QUANT = 65535  # lattice of the metrics: X = rint(x * 65535) for x in [0, 1]


def quantise(xy: np.ndarray) -> np.ndarray:
    """Integer lattice coordinates (int64 [n, 2]) of float32 positions:
    rint(float32(x * 65535)) after clamping x to [0, 1] (NaN -> 0); the
    product is rounded to float32 first, as the device does."""
    z = np.ascontiguousarray(xy, dtype=np.float32).reshape(-1, 2)
    z = np.where(np.isnan(z), np.float32(0.0), z)
    z = np.clip(z, np.float32(0.0), np.float32(1.0))
    return np.rint(z * np.float32(QUANT)).astype(np.int64)


def _keys(q: np.ndarray, i: int) -> np.ndarray:
    """Ordering keys of every sample seen from sample i: squared lattice
    distance, ties broken by the sample index (key = d2 * 2^31 + index as an
    unsigned 64-bit integer, n < 2^31; the sample itself gets the largest key
    so that it is never a neighbour)."""
    d = q - q[i]
    d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]).astype(np.uint64)  # < 2^33
    key = d2 * np.uint64(1 << 31) + np.arange(q.shape[0], dtype=np.uint64)  # < 2^64
    key[i] = np.iinfo(np.uint64).max
    return key


def trustworthiness_terms(orig: np.ndarray, new: np.ndarray, k: int, queries) -> np.ndarray:
    """Per query i: sum over j in U_k(i) of (r(i, j) - k), where U_k(i) holds
    the k nearest neighbours of i in the new layout that are not among its k
    nearest in the original layout, and r(i, j) is the rank of j by distance
    from i in the original layout (the nearest has rank 1).  Distances on the
    lattice of :func:`quantise`, ties broken by index."""
    qo, qn = quantise(orig), quantise(new)
    out = np.zeros(len(queries), dtype=np.int64)
    for a, i in enumerate(queries):
        ko = _keys(qo, int(i))
        kn = _keys(qn, int(i))
        order_o = np.argsort(ko, kind="stable")
        rank_o = np.empty_like(order_o)
        rank_o[order_o] = np.arange(1, order_o.size + 1)
        nn_o = set(order_o[:k].tolist())
        nn_n = np.argsort(kn, kind="stable")[:k]
        out[a] = sum(int(rank_o[j]) - k for j in nn_n if int(j) not in nn_o)
    return out


def ordering_terms(orig: np.ndarray, new: np.ndarray, queries) -> np.ndarray:
    """Per query i: the number of samples j != i whose orthogonal order
    relative to i is not kept: sign(X_i - X_j) or sign(Y_i - Y_j) differs
    between the original and the new layout (lattice coordinates)."""
    qo, qn = quantise(orig), quantise(new)
    out = np.zeros(len(queries), dtype=np.int64)
    for a, i in enumerate(queries):
        so = np.sign(qo[int(i)] - qo)
        sn = np.sign(qn[int(i)] - qn)
        bad = np.any(so != sn, axis=1)
        out[a] = int(np.count_nonzero(bad))
    return out


def layout_metrics(orig: np.ndarray, new: np.ndarray, k: int, queries=None) -> dict:
    """Trustworthiness T(k) of Venna and Kaski and the orthogonal ordering of
    Misue et al., estimated over the query samples (all samples when
    ``queries`` is None, which gives the exact values):

      T = 1 - 2 / (m k (2n - 3k - 1)) * sum_i sum_{j in U_k(i)} (r(i, j) - k)
      O = 1 - (sum_i #pairs (i, j) whose orthogonal order changed) / (m (n - 1))

    with m the number of queries (k < n / 2)."""
    n = np.asarray(orig).reshape(-1, 2).shape[0]
    if queries is None:
        queries = np.arange(n)
    queries = np.asarray(queries, dtype=np.int64)
    m = queries.size
    t = trustworthiness_terms(orig, new, k, queries)
    o = ordering_terms(orig, new, queries)
    T = 1.0 - 2.0 / (m * k * (2.0 * n - 3.0 * k - 1.0)) * float(t.sum())
    O = 1.0 - float(o.sum()) / (m * (n - 1.0))
    return {"trustworthiness": T, "ordering": O, "t_terms": t, "o_terms": o}


# ---------------------------------------------------------------------------
# Sec. 4.3 step 4: stopping criteria
# ---------------------------------------------------------------------------


def max_move_px(before: np.ndarray, after: np.ndarray, N: int) -> float:
    """Largest distance a sample moved in one iteration, in pixels."""
    d = after.astype(np.float64) - before.astype(np.float64)
    return float(np.sqrt((d * d).sum(axis=1)).max()) * N if d.size else 0.0


def regularize_until(xy: np.ndarray, p, max_iters: int, target_cv: float = 0.0,
                     min_move_px: float = 0.0) -> dict:
    """Iterations of Sec. 4.3 until a stopping criterion of step 4 holds:
    after an iteration, the Sec. 6.2 bin std over the mean bin count is at
    most target_cv (when > 0), or the largest move of a sample in that
    iteration is at most min_move_px (when > 0); at most max_iters.
    Returns the positions, the iterations done and the per-iteration
    measures."""
    z = np.ascontiguousarray(xy, dtype=np.float32).reshape(-1, 2)
    cvs, moves = [], []
    done = 0
    for _ in range(max_iters):
        new = iterate(z, p)
        q = quality(splat(new, p.log2_res))
        cvs.append(q["bin_cv"])
        moves.append(max_move_px(z, new, p.N))
        z = new
        done += 1
        if (target_cv > 0 and cvs[-1] <= target_cv) or (min_move_px > 0 and moves[-1] <= min_move_px):
            break
    return {"pos": z, "iters": done, "cv": cvs, "move_px": moves}


# ---------------------------------------------------------------------------
# Sec. 5: density background texture deformed by the mesh mapping
# ---------------------------------------------------------------------------

SUB = 8  # sub-pixel bits of the rasteriser's fixed-point vertices


def _tri_vertices(N: int):
    """The two triangles of cell (i, j) of the node mesh, as node index
    triples: triangle 2c: (i, j), (i+1, j), (i+1, j+1); triangle 2c + 1:
    (i, j), (i+1, j+1), (i, j+1); c = j (N - 1) + i."""
    tris = []
    for j in range(N - 1):
        for i in range(N - 1):
            tris.append(((i, j), (i + 1, j), (i + 1, j + 1)))
            tris.append(((i, j), (i + 1, j + 1), (i, j + 1)))
    return tris


def _fixed(xy: np.ndarray, log2M: int) -> np.ndarray:
    """Fixed-point vertex coordinates: rint(float32(x * 2^(log2M + SUB))) of
    x clamped to [-1, 2] (NaN -> -1); nodes are expected in [0, 1]."""
    z = np.asarray(xy, dtype=np.float32)
    z = np.clip(np.where(np.isnan(z), np.float32(-1.0), z), np.float32(-1.0), np.float32(2.0))
    return np.rint(z * np.float32(2.0 ** (log2M + SUB))).astype(np.int64)


def _top_left(ax, ay, bx, by) -> bool:
    """Fill rule for points exactly on the edge a -> b of a triangle of
    positive orientation: the edge owns them when it runs up (dy < 0) or,
    level, to the right (dx > 0); the opposite edge of a neighbour then does
    not, so every point of a tiling is covered once."""
    dy, dx = by - ay, bx - ax
    return dy < 0 or (dy == 0 and dx > 0)


def coverage(nodes_xy: np.ndarray, log2M: int) -> np.ndarray:
    """Winning triangle per output pixel of an M x M raster (int64 [M, M],
    -1 where no triangle covers the pixel centre): the lowest-numbered
    triangle of the deformed mesh whose interior, or owned edge, holds the
    centre ((p + 1/2) / M, (q + 1/2) / M).  Exact integer edge functions on
    the fixed-point vertices; degenerate triangles cover nothing."""
    N = nodes_xy.shape[0]
    M = 1 << log2M
    V = _fixed(nodes_xy.reshape(N, N, 2), log2M)
    half = 1 << (SUB - 1)
    out = np.full((M, M), -1, dtype=np.int64)
    for t, tri in enumerate(_tri_vertices(N)):
        pts = [V[j, i] for i, j in tri]
        (ax, ay), (bx, by), (cx, cy) = [(int(p[0]), int(p[1])) for p in pts]
        area = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax)
        if area == 0:
            continue
        if area < 0:  # orient positively
            (bx, by), (cx, cy) = (cx, cy), (bx, by)
        xs, ys = (ax, bx, cx), (ay, by, cy)
        p0 = max(0, (min(xs) - half + (1 << SUB) - 1) >> SUB)
        p1 = min(M - 1, (max(xs) - half) >> SUB)
        q0 = max(0, (min(ys) - half + (1 << SUB) - 1) >> SUB)
        q1 = min(M - 1, (max(ys) - half) >> SUB)
        if p1 < p0 or q1 < q0:
            continue
        P, Q = np.meshgrid(np.arange(p0, p1 + 1), np.arange(q0, q1 + 1))
        px = (P << SUB) + half
        py = (Q << SUB) + half
        inside = np.ones(P.shape, dtype=bool)
        for (ux, uy), (vx, vy) in (((ax, ay), (bx, by)), ((bx, by), (cx, cy)), ((cx, cy), (ax, ay))):
            e = (vx - ux) * (py - uy) - (vy - uy) * (px - ux)
            inside &= (e > 0) | ((e == 0) & _top_left(ux, uy, vx, vy))
        sel = inside & (out[Q, P] == -1)  # the lowest triangle index wins
        out[Q[sel], P[sel]] = t
    return out


def warp_texture(nodes_xy: np.ndarray, texture: np.ndarray, log2M: int, mass: bool = False,
                 pixel_center: bool = False):
    """The texture (values at the N x N pixel nodes) drawn on the mesh whose
    nodes moved to nodes_xy (domain units, [N, N, 2] or [N*N, 2]): every
    output pixel covered by a deformed triangle takes the texture at the
    source point with the same barycentric coordinates in the undeformed
    triangle (bilinear texture lookup between nodes); uncovered pixels are
    0.  mass: the value is multiplied by the undeformed over the deformed
    triangle area (the push-forward density, which keeps the mass).
    Returns (values float64 [M, M], coverage int64 [M, M])."""
    N = texture.shape[0]
    M = 1 << log2M
    nodes = np.asarray(nodes_xy, dtype=np.float32).reshape(N, N, 2)
    cov = coverage(nodes, log2M)
    V = _fixed(nodes, log2M).astype(np.float64)
    tex = np.asarray(texture, dtype=np.float64)
    tris = _tri_vertices(N)
    half = 1 << (SUB - 1)
    out = np.zeros((M, M), dtype=np.float64)
    # edge cross product (twice the area) of an undeformed triangle, fixed-point units
    cross0 = (float(M << SUB) / N) ** 2
    for q in range(M):
        for p in range(M):
            t = int(cov[q, p])
            if t < 0:
                continue
            (i0, j0), (i1, j1), (i2, j2) = tris[t]
            a, b, c = V[j0, i0], V[j1, i1], V[j2, i2]
            px, py = float((p << SUB) + half), float((q << SUB) + half)
            area = (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])
            # barycentric weights of the pixel centre (of b and c; a gets the rest)
            lb = ((px - a[0]) * (c[1] - a[1]) - (py - a[1]) * (c[0] - a[0])) / area
            lc = ((b[0] - a[0]) * (py - a[1]) - (b[1] - a[1]) * (px - a[0])) / area
            la = 1.0 - lb - lc
            si = la * i0 + lb * i1 + lc * i2
            sj = la * j0 + lb * j1 + lc * j2
            # bilinear texture lookup at node coordinates (si, sj), clamped
            si = min(max(si, 0.0), N - 1.0)
            sj = min(max(sj, 0.0), N - 1.0)
            x0, y0 = min(int(np.floor(si)), N - 2), min(int(np.floor(sj)), N - 2)
            fx, fy = si - x0, sj - y0
            v = ((1 - fy) * ((1 - fx) * tex[y0, x0] + fx * tex[y0, x0 + 1])
                 + fy * ((1 - fx) * tex[y0 + 1, x0] + fx * tex[y0 + 1, x0 + 1]))
            if mass:
                v *= cross0 / abs(area)
            out[q, p] = v
    return out, cov


def transfer(values: np.ndarray, lo: float, hi: float, lut: np.ndarray) -> np.ndarray:
    """Transfer function of the background texture (Sec. 5): lut[i] with
    i = rint((v - lo) * (255 / (hi - lo))) clamped to 0..255, in float32
    with each operation rounded in that order (NaN -> 0)."""
    v = np.asarray(values, dtype=np.float32)
    scale = np.float32(255.0) / (np.float32(hi) - np.float32(lo))
    x = ((v - np.float32(lo)).astype(np.float32) * scale).astype(np.float32)
    i = np.clip(np.rint(np.where(np.isnan(x), np.float32(0.0), x)), 0, 255).astype(np.int64)
    return np.asarray(lut, dtype=np.uint32)[i]


def identity_nodes(N: int, pixel_center: bool = False) -> np.ndarray:
    """Undeformed node positions ((i + o) / N, (j + o) / N), float32 [N, N, 2]."""
    o = 0.5 if pixel_center else 0.0
    jj, ii = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    return np.stack([(ii + o) / N, (jj + o) / N], -1).astype(np.float32)
