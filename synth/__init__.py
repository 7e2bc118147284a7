"""Seeded synthetic inputs for the de-cluttering workloads.

This module only draws random numbers: it holds none of the method's
arithmetic (no splatting, smoothing, integral images, mapping or advection).
Both the CPU oracle tests and the CUDA tests / bench take their inputs from
here, so that the two sides always see identical float32 samples.

Workloads (sizes follow the configurations the method is measured on):

* ``tiny``      -- 10,000 samples, mixture of 3 anisotropic Gaussians
                   (weights 0.5/0.3/0.2, per-axis std U[0.02, 0.1], random
                   rotation, means U[0.2, 0.8]^2); used on a 128x128 grid.
* ``gmm20``     -- 1,000,000 samples, 20 Gaussians (means U[0.05, 0.95]^2,
                   per-axis std U[0.005, 0.05], random rotation, weights
                   proportional to U[0.5, 1.5]) plus 10% uniform background;
                   used on a 512x512 grid.
* ``student_t`` -- 16,000,000 samples from 8 Student-t (nu = 3) clusters with
                   heavy overlap (centres U[0.35, 0.65]^2, scale
                   U[0.03, 0.08]); used on a 2048x2048 grid.
* ``sat_grid``  -- uint32 grids with values U{0..255} for the standalone
                   integral-image sweep (256^2 .. 8192^2).
* ``splom``     -- scatterplot matrix: 200,000 rows of a 16-dimensional
                   12-component correlated Gaussian mixture (means U[-3,3]^16,
                   covariances A A^T with A ~ N(0, 0.3^2)); all 120 dimension
                   pairs, each min-max normalised; panel p keeps a seeded
                   fraction U[0.25, 1] of the rows and uses a grid of
                   256^2 / 512^2 / 1024^2 for p mod 3 = 0 / 1 / 2.

Samples drawn outside the unit square are rejected and redrawn; the reject
fraction is returned with the samples.  The paper's own statistics use random
Gaussian-cluster datasets (Section 6.2); its named datasets (MNIST, COIL, UCI)
are not available, and these generators stand in for them.
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "gaussian_mixture",
    "tiny_mixture",
    "gmm20",
    "student_t_clusters",
    "sat_grid",
    "uniform_grid_samples",
    "diagonal_band",
    "four_clusters",
    "WORKLOADS",
    "workload",
    "splom",
]


def _rotation(rng: np.random.Generator) -> np.ndarray:
    th = rng.uniform(0.0, np.pi)
    c, s = np.cos(th), np.sin(th)
    return np.array([[c, -s], [s, c]])


def _draw_until_inside(draw, n: int, rng: np.random.Generator):
    """Call ``draw(m)`` -> (m, 2) float64 until ``n`` samples lie in [0,1]^2."""
    out = np.empty((n, 2), dtype=np.float64)
    have = 0
    drawn = 0
    while have < n:
        m = max(1024, int((n - have) * 1.25))
        z = draw(m)
        drawn += m
        ok = np.all((z >= 0.0) & (z <= 1.0), axis=1)
        z = z[ok]
        take = min(n - have, z.shape[0])
        out[have:have + take] = z[:take]
        have += take
    return out, 1.0 - n / max(drawn, 1)


def gaussian_mixture(n: int, seed: int, n_comp: int, mean_lo: float, mean_hi: float,
                     std_lo: float, std_hi: float, weights=None, uniform_frac: float = 0.0):
    """Mixture of rotated anisotropic Gaussians (+ optional uniform share).

    Returns ``(samples float32 [n,2] C-contiguous, reject_fraction)``.
    """
    rng = np.random.default_rng(seed)
    means = rng.uniform(mean_lo, mean_hi, size=(n_comp, 2))
    stds = rng.uniform(std_lo, std_hi, size=(n_comp, 2))
    rots = np.stack([_rotation(rng) for _ in range(n_comp)])
    if weights is None:
        w = rng.uniform(0.5, 1.5, size=n_comp)
    else:
        w = np.asarray(weights, dtype=np.float64)
    w = w / w.sum()
    n_uni = int(round(n * uniform_frac))
    n_g = n - n_uni

    def draw(m):
        comp = rng.choice(n_comp, size=m, p=w)
        e = rng.standard_normal((m, 2)) * stds[comp]
        z = np.einsum("mij,mj->mi", rots[comp], e) + means[comp]
        return z

    zg, rej = _draw_until_inside(draw, n_g, rng) if n_g > 0 else (np.zeros((0, 2)), 0.0)
    zu = rng.uniform(0.0, 1.0, size=(n_uni, 2))
    z = np.concatenate([zg, zu], axis=0)
    perm = rng.permutation(n)
    z = z[perm]
    return np.ascontiguousarray(z.astype(np.float32)), rej


def tiny_mixture(n: int = 10_000, seed: int = 1):
    """3 anisotropic Gaussians, weights 0.5/0.3/0.2 (128x128 workload)."""
    return gaussian_mixture(n, seed, 3, 0.2, 0.8, 0.02, 0.1, weights=[0.5, 0.3, 0.2])


def gmm20(n: int = 1_000_000, seed: int = 2):
    """20 Gaussians + 10% uniform background (512x512 workload)."""
    return gaussian_mixture(n, seed, 20, 0.05, 0.95, 0.005, 0.05, uniform_frac=0.10)


def student_t_clusters(n: int = 16_000_000, seed: int = 3, nu: float = 3.0, n_comp: int = 8):
    """Heavy-tailed, heavily overlapping Student-t clusters (2048x2048 workload)."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.35, 0.65, size=(n_comp, 2))
    scales = rng.uniform(0.03, 0.08, size=(n_comp, 2))
    rots = np.stack([_rotation(rng) for _ in range(n_comp)])

    def draw(m):
        comp = rng.integers(0, n_comp, size=m)
        e = rng.standard_t(nu, size=(m, 2)) * scales[comp]
        return np.einsum("mij,mj->mi", rots[comp], e) + centres[comp]

    z, rej = _draw_until_inside(draw, n, rng)
    return np.ascontiguousarray(z.astype(np.float32)), rej


def sat_grid(log2_res: int, seed: int = 0) -> np.ndarray:
    """uint32 grid N x N with values U{0..255} (integral-image sweep input)."""
    n = 1 << log2_res
    rng = np.random.default_rng(1000 + seed + log2_res)
    return np.ascontiguousarray(rng.integers(0, 256, size=(n, n), dtype=np.uint32))


def uniform_grid_samples(log2_res: int, per_pixel: int = 1, pixel_center: bool = False):
    """Samples placed exactly on the pixel positions (a perfectly even layout).

    Pixel (i, j) sits at (i, j) / N, or at (i + 1/2, j + 1/2) / N when
    ``pixel_center`` is set.  Every pixel receives ``per_pixel`` samples.
    """
    n = 1 << log2_res
    off = 0.5 if pixel_center else 0.0
    jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    z = np.stack([(ii.ravel() + off) / n, (jj.ravel() + off) / n], axis=1)
    z = np.repeat(z, per_pixel, axis=0)
    return np.ascontiguousarray(z.astype(np.float32))


def diagonal_band(n: int, seed: int = 11, width: float = 0.03):
    """Samples spread along the main diagonal (uniform marginals, thin band)."""
    rng = np.random.default_rng(seed)

    def draw(m):
        s = rng.uniform(0.0, 1.0, size=m)
        e = rng.standard_normal(m) * width
        return np.stack([s + e / np.sqrt(2.0), s - e / np.sqrt(2.0)], axis=1)

    z, rej = _draw_until_inside(draw, n, rng)
    return np.ascontiguousarray(z.astype(np.float32)), rej


def four_clusters(n: int = 1_000_000, seed: int = 12, std: float = 0.04):
    """Four Gaussian clusters holding 40/30/20/10 % of the samples, with labels."""
    rng = np.random.default_rng(seed)
    centres = np.array([[0.3, 0.3], [0.7, 0.3], [0.3, 0.7], [0.7, 0.7]])
    counts = [int(n * f) for f in (0.4, 0.3, 0.2)]
    counts.append(n - sum(counts))
    zs, labels = [], []
    for k, (c, m) in enumerate(zip(centres, counts)):
        def draw(mm, c=c):
            return rng.standard_normal((mm, 2)) * std + c
        z, _ = _draw_until_inside(draw, m, rng)
        zs.append(z)
        labels.append(np.full(m, k, dtype=np.int32))
    z = np.concatenate(zs)
    lab = np.concatenate(labels)
    perm = rng.permutation(n)
    return np.ascontiguousarray(z[perm].astype(np.float32)), lab[perm]


# Named workloads: (generator, grid log2, iterations, smoothing radius r)
WORKLOADS = {
    "tiny": dict(gen=tiny_mixture, n=10_000, log2_res=7, iters=4, kernel_r=2),
    "tiny_exact": dict(gen=tiny_mixture, n=10_000, log2_res=7, iters=4, kernel_r=0),
    "gmm20_512": dict(gen=gmm20, n=1_000_000, log2_res=9, iters=8, kernel_r=4),
    "student_t_2048": dict(gen=student_t_clusters, n=16_000_000, log2_res=11, iters=8, kernel_r=16),
}


def workload(name: str, n: int | None = None):
    """Return ``(samples, spec)`` for a named workload (optionally resized)."""
    spec = dict(WORKLOADS[name])
    nn = spec["n"] if n is None else n
    z, _ = spec["gen"](nn)
    spec["n"] = nn
    return z, spec


def splom(rows: int = 200_000, dims: int = 16, comps: int = 12, seed: int = 4):
    """Panels of a scatterplot matrix: list of ``(samples float32 [n_p, 2],
    log2_res)`` for every pair i < j of the ``dims`` dimensions."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-3.0, 3.0, size=(comps, dims))
    A = rng.normal(0.0, 0.3, size=(comps, dims, dims))
    w = rng.uniform(0.5, 1.5, size=comps)
    w = w / w.sum()
    comp = rng.choice(comps, size=rows, p=w)
    e = rng.standard_normal((rows, dims))
    X = np.einsum("rij,rj->ri", A[comp], e) + means[comp]
    panels = []
    p = 0
    for i in range(dims):
        for j in range(i + 1, dims):
            frac = rng.uniform(0.25, 1.0)
            keep = rng.random(rows) < frac
            z = X[keep][:, [i, j]]
            lo, hi = z.min(axis=0), z.max(axis=0)
            z = (z - lo) / np.where(hi > lo, hi - lo, 1.0)
            panels.append((np.ascontiguousarray(z.astype(np.float32)), (8, 9, 10)[p % 3]))
            p += 1
    return panels
