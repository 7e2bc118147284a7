"""CPU oracle for the de-cluttering iteration (test infrastructure only).

Rave, Molchanov and Linsen, "De-cluttering Scatterplots with Integral Images"
(arXiv 2408.06513).  Plain FP64 / exact-integer restatement of the method's
steps, written in C (``declutter_oracle.c``) and called through ctypes.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it, and
it never calls the CUDA library: the two share no code.

Every function cites the passage it follows:

* :func:`splat`         -- Sec. 4.1 / Sec. 4.3 step 1, single-pixel accumulation
* :func:`smooth`        -- Sec. 4.1 / Sec. 4.4, separable Gaussian smoothing
* :func:`inims`         -- Sec. 3.1, the eight (tilted) integral images
* :func:`sat_u64`       -- Sec. 3.1, exact alpha and alpha_t of a uint32 grid
* :func:`mapping`       -- Sec. 3.2, eq. (map) with anchors q1..q4
* :func:`displacement`  -- Sec. 4.1-4.2, eqs. (d0) and (map_res)
* :func:`lens_displacement` -- end of Sec. 3.2, eq. (map) as a virtual lens
* :func:`contour_cell`  -- Sec. 5, contour lines (marching squares)
* :func:`advect`        -- Sec. 4.2 / 4.3 step 3, bilinear sample update
* :func:`quality`       -- Sec. 6.2, 4x4-bin std and overplotting
* :func:`iterate`       -- Sec. 4.3, one full iteration

Parity status: every function above is pinned by ``tests/test_oracle_*.py``
against brute force, closed forms, library routines or geometric facts.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "declutter_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP) into ``oracle/_liboracle.so``."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    P = ctypes.c_void_p
    i64 = ctypes.c_int64
    ci = ctypes.c_int
    cd = ctypes.c_double
    lib.orc_max_threads.restype = ci
    lib.orc_set_threads.argtypes = [ci]
    lib.orc_splat.argtypes = [P, i64, ci, P]
    lib.orc_gauss_weights.argtypes = [ci, cd, P]
    lib.orc_smooth.argtypes = [P, ci, ci, cd, P]
    lib.orc_inims.argtypes = [P, ci, P]
    lib.orc_sat_u64.argtypes = [P, ci, P, P]
    lib.orc_mapping.argtypes = [P, ci, ci, P]
    lib.orc_displacement.argtypes = [P, ci, cd, ci, P]
    lib.orc_advect.argtypes = [P, i64, ci, P, ci, ci, P]
    lib.orc_quality.argtypes = [P, ci, P]
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _res(log2_res: int) -> int:
    return 1 << int(log2_res)


def max_threads() -> int:
    return int(_load().orc_max_threads())


def set_threads(t: int) -> None:
    _load().orc_set_threads(int(t))


def splat(xy: np.ndarray, log2_res: int) -> np.ndarray:
    """Counts per pixel (uint64 [N, N], row j, column i), Sec. 4.1."""
    xy = np.ascontiguousarray(xy, dtype=np.float32).reshape(-1, 2)
    N = _res(log2_res)
    out = np.empty((N, N), dtype=np.uint64)
    _load().orc_splat(_ptr(xy), xy.shape[0], N, _ptr(out))
    return out


def gauss_weights(r: int, sigma: float = 0.0) -> np.ndarray:
    """Normalised discrete Gaussian, taps -r..r (sigma <= 0 -> r/3)."""
    g = np.empty(2 * r + 1, dtype=np.float64)
    _load().orc_gauss_weights(int(r), float(sigma), _ptr(g))
    return g


def smooth(field: np.ndarray, r: int, sigma: float = 0.0) -> np.ndarray:
    """Separable Gaussian with reflect border, FP64 (Sec. 4.1, Sec. 4.4)."""
    a = np.ascontiguousarray(field, dtype=np.float64)
    N = a.shape[0]
    if r == 0:
        return a.copy()
    out = np.empty_like(a)
    _load().orc_smooth(_ptr(a), N, int(r), float(sigma), _ptr(out))
    return out


INIM_NAMES = ("alpha", "beta", "gamma", "delta", "alpha_t", "beta_t", "gamma_t", "delta_t")


def inims(d: np.ndarray) -> dict:
    """The eight integral images of texture ``d`` (Sec. 3.1), FP64."""
    a = np.ascontiguousarray(d, dtype=np.float64)
    N = a.shape[0]
    out = np.empty((8, N, N), dtype=np.float64)
    _load().orc_inims(_ptr(a), N, _ptr(out))
    return {k: out[q] for q, k in enumerate(INIM_NAMES)}


def sat_u64(grid: np.ndarray):
    """Exact (alpha, alpha_t) of a uint32 grid as uint64 (Sec. 3.1)."""
    g = np.ascontiguousarray(grid, dtype=np.uint32)
    N = g.shape[0]
    a = np.empty((N, N), dtype=np.uint64)
    at = np.empty((N, N), dtype=np.uint64)
    _load().orc_sat_u64(_ptr(g), N, _ptr(a), _ptr(at))
    return a, at


def mapping(d: np.ndarray, pixel_center: bool = False) -> np.ndarray:
    """t(x, y; d) of eq. (map) at every pixel, shape [N, N, 2] (x, y)."""
    ims = inims(d)
    N = d.shape[0]
    stack = np.ascontiguousarray(np.stack([ims[k] for k in INIM_NAMES]))
    out = np.empty((N, N, 2), dtype=np.float64)
    _load().orc_mapping(_ptr(stack), N, int(bool(pixel_center)), _ptr(out))
    return out


def lens_displacement(d: np.ndarray, pixel_center: bool = False) -> np.ndarray:
    """The virtual lens of Molchanov and Linsen (end of Sec. 3.2): eq. (map)
    applied once, without the defect of eq. (map_res); t(x, y; d) - (x, y)
    at every pixel, [N, N, 2], domain units."""
    N = d.shape[0]
    off = 0.5 if pixel_center else 0.0
    pos = (np.arange(N, dtype=np.float64) + off) / N
    out = mapping(d, pixel_center)
    out[:, :, 0] -= pos[None, :]
    out[:, :, 1] -= pos[:, None]
    return out


def contour_cell(f: np.ndarray, level: float, i: int, j: int, pixel_center: bool = False) -> list:
    """Contour segments of cell (i, j) of the float32 field f at ``level``
    (Sec. 5 contour lines; reading: marching squares over the pixel nodes).
    Corners f[j, i], f[j, i+1], f[j+1, i+1], f[j+1, i] at the node positions
    ((i + o) / N, (j + o) / N); a corner is inside when f >= level (compared
    in float32); each edge whose ends differ holds the linearly interpolated
    vertex.  Two crossed edges make one segment; four (a saddle) make two,
    around the two corners on the other side of the cell centre, the float32
    mean ((a + b) + (c + d)) / 4.  Returns [((x0, y0), (x1, y1)), ...] in
    domain units, FP64."""
    N = f.shape[0]
    o = 0.5 if pixel_center else 0.0
    lv = np.float32(level)
    # corners counter-clockwise in (i, j): (i, j), (i+1, j), (i+1, j+1), (i, j+1)
    ij = [(i, j), (i + 1, j), (i + 1, j + 1), (i, j + 1)]
    val = [np.float32(f[b, a]) for a, b in ij]
    ins = [v >= lv for v in val]

    def cross(p, q):  # vertex on the edge from corner p to corner q
        t = (float(lv) - float(val[p])) / (float(val[q]) - float(val[p]))
        (ap, bp), (aq, bq) = ij[p], ij[q]
        return ((ap + o + t * (aq - ap)) / N, (bp + o + t * (bq - bp)) / N)

    sides = [(0, 1), (1, 2), (2, 3), (3, 0)]  # the four edges as corner pairs
    hit = [s for s in sides if ins[s[0]] != ins[s[1]]]
    if not hit:
        return []
    if len(hit) == 2:
        return [(cross(*hit[0]), cross(*hit[1]))]
    centre = ((val[0] + val[1]) + (val[2] + val[3])) * np.float32(0.25)
    # the corners cut off: those whose side differs from the centre's
    cut = [k for k in range(4) if ins[k] != (centre >= lv)]
    segs = []
    for k in cut:
        a, b = (k + 3) % 4, (k + 1) % 4  # neighbours of corner k
        segs.append((cross(a, k), cross(k, b)))
    return segs


def contour_segments(f: np.ndarray, level: float, pixel_center: bool = False) -> list:
    """contour_cell of every cell, in cell order (j, then i); for small grids."""
    N = f.shape[0]
    return [contour_cell(f, level, i, j, pixel_center) for j in range(N - 1) for i in range(N - 1)]


def displacement(d_r: np.ndarray, d0: float, pixel_center: bool = False) -> np.ndarray:
    """D = t(.; d_r + d0) - t(.; d0), eqs. (d0), (map_res); [N, N, 2], domain units."""
    a = np.ascontiguousarray(d_r, dtype=np.float64)
    N = a.shape[0]
    out = np.empty((N, N, 2), dtype=np.float64)
    _load().orc_displacement(_ptr(a), N, float(d0), int(bool(pixel_center)), _ptr(out))
    return out


def advect(xy: np.ndarray, D: np.ndarray, pixel_center: bool = False, clamp: bool = True) -> np.ndarray:
    """New float32 positions z + bilinear(D)(z) (Sec. 4.2)."""
    xy = np.ascontiguousarray(xy, dtype=np.float32).reshape(-1, 2)
    Dd = np.ascontiguousarray(D, dtype=np.float64)
    N = Dd.shape[0]
    out = np.empty_like(xy)
    _load().orc_advect(_ptr(xy), xy.shape[0], N, _ptr(Dd), int(bool(pixel_center)), int(bool(clamp)),
                       _ptr(out))
    return out


def quality(counts: np.ndarray) -> dict:
    """Sec. 6.2: 4x4-bin std (and std/mean) and overplotting of a count grid."""
    c = np.ascontiguousarray(counts, dtype=np.uint64)
    out = np.empty(3, dtype=np.float64)
    _load().orc_quality(_ptr(c), c.shape[0], _ptr(out))
    return {"bin_std": float(out[0]), "bin_cv": float(out[1]), "overplot": float(out[2])}


@dataclass
class Params:
    """Method parameters (Sec. 4.1, 4.3): grid 2^k, radius r, sigma, d0."""
    log2_res: int
    kernel_r: int = -1        # < 0: N/128 (at least 2); 0: no smoothing
    sigma: float = 0.0        # <= 0: r/3
    d0: float = -1.0          # < 0: n / N^2
    pixel_center: bool = False
    clamp_positions: bool = True

    @property
    def N(self) -> int:
        return 1 << self.log2_res

    def radius(self) -> int:
        if self.kernel_r < 0:
            return max(2, self.N // 128)
        return int(self.kernel_r)

    def d0_for(self, n: int) -> float:
        return float(n) / float(self.N * self.N) if self.d0 < 0 else float(self.d0)


def density(xy: np.ndarray, p: Params):
    """Counts and the smoothed density d_r (Sec. 4.1)."""
    c = splat(xy, p.log2_res)
    r = p.radius()
    d_r = smooth(c.astype(np.float64), r, p.sigma) if r > 0 else c.astype(np.float64)
    return c, d_r


def iterate(xy: np.ndarray, p: Params, keep: bool = False):
    """One iteration of Sec. 4.3 (steps 1-3) from float32 positions ``xy``.

    Returns the new float32 positions, and, when ``keep`` is set, a dict of
    intermediates (counts, d_r, D, d0).
    """
    xy = np.ascontiguousarray(xy, dtype=np.float32).reshape(-1, 2)
    c, d_r = density(xy, p)
    d0 = p.d0_for(xy.shape[0])
    D = displacement(d_r, d0, p.pixel_center)
    new = advect(xy, D, p.pixel_center, p.clamp_positions)
    if keep:
        return new, {"counts": c, "d_r": d_r, "D": D, "d0": d0}
    return new


def regularize(xy: np.ndarray, p: Params, iters: int):
    """``iters`` iterations of :func:`iterate`; returns the trajectory list."""
    traj = [np.ascontiguousarray(xy, dtype=np.float32).reshape(-1, 2)]
    for _ in range(iters):
        traj.append(iterate(traj[-1], p))
    return traj


if __name__ == "__main__":  # pragma: no cover
    build(force="--force" in sys.argv)
    print(_LIB)
