"""Training data, training loop and evaluation of the learned surrogate.

Pairs come from the plain method on the GPU: for random Gaussian mixtures
(2-30 components, n log-uniform in [10k, 2M]) the input is the smoothed
density of the samples (``splat_density``) and the target is the displacement
field composed over ``iters`` plain iterations, obtained by moving the pixel
nodes as massless tracers through the same iterations
(``regularize_tracers``): target = (final - initial node positions) * N, in
pixels.  With a 3-channel network the input also holds the field of one
plain iteration (``displacement_field``, in pixels): the displacement is a
function of global integrals of the density, which a convolutional network
of limited receptive field cannot see, while one iteration's field carries
them; the network then learns the composed field as a skip kappa * field
(kappa fitted by least squares, ``fit_skip``) plus a correction.  Every step
of the method and of the network runs in the CUDA library; PyTorch only holds
device memory, draws the random samples and fits the one scalar kappa.
"""

from __future__ import annotations

import math
import time

import numpy as np

from . import declutter as dc


def gmm_samples(n: int, n_comp: int, rng: np.random.Generator, device):
    """Samples of a random rotated-Gaussian mixture inside the unit square."""
    import torch
    means = torch.tensor(rng.uniform(0.1, 0.9, (n_comp, 2)), dtype=torch.float32, device=device)
    stds = torch.tensor(rng.uniform(0.005, 0.08, (n_comp, 2)), dtype=torch.float32, device=device)
    th = rng.uniform(0, math.pi, n_comp)
    R = np.zeros((n_comp, 2, 2))
    R[:, 0, 0], R[:, 0, 1], R[:, 1, 0], R[:, 1, 1] = np.cos(th), -np.sin(th), np.sin(th), np.cos(th)
    rot = torch.tensor(R, dtype=torch.float32, device=device)
    w = torch.tensor(rng.uniform(0.5, 1.5, n_comp), dtype=torch.float32, device=device)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(rng.integers(0, 2**62)))
    out = []
    have = 0
    while have < n:
        m = int((n - have) * 1.3) + 1024
        comp = torch.multinomial(w, m, replacement=True, generator=gen)
        e = torch.randn(m, 2, device=device, generator=gen) * stds[comp]
        z = torch.einsum("mij,mj->mi", rot[comp], e) + means[comp]
        z = z[((z >= 0) & (z <= 1)).all(dim=1)]
        out.append(z[: n - have])
        have += out[-1].shape[0]
    return torch.cat(out).contiguous()


class PairGenerator:
    """Generates (density, scale, composed displacement) triples with the plain method."""

    def __init__(self, log2_res: int = 8, iters: int = 8, kernel_r: int = -1, device: int = 0):
        import torch
        self.log2_res, self.iters, self.device = log2_res, iters, device
        self.N = 1 << log2_res
        self.ctx = dc.declutter_create(log2_res, kernel_r=kernel_r, device=device)
        N = self.N
        jj, ii = torch.meshgrid(torch.arange(N, device=device), torch.arange(N, device=device), indexing="ij")
        self.nodes = torch.stack([ii.reshape(-1) / N, jj.reshape(-1) / N], dim=1).float().contiguous()

    def close(self):
        dc.declutter_destroy(self.ctx)

    def make(self, count: int, rng: np.random.Generator, n_range=(10_000, 2_000_000), comps=(2, 30)):
        """Returns (density [P,N,N], scales [P], field [P,N,N,2], target [P,N,N,2]):
        field = one plain iteration's displacement, target = the composed one (pixels)."""
        import torch
        N = self.N
        dens = torch.empty(count, N, N, device=self.device)
        field = torch.empty(count, N, N, 2, device=self.device)
        target = torch.empty(count, N, N, 2, device=self.device)
        scales = torch.empty(count, device=self.device)
        for k in range(count):
            n = int(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1]))))
            K = int(rng.integers(comps[0], comps[1] + 1))
            pos = gmm_samples(n, K, rng, self.device)
            dc.splat_density(self.ctx, pos, density_out=dens[k].view(-1))
            dc.displacement_field(self.ctx, field[k].view(-1))
            field[k] *= N
            tr = self.nodes.clone()
            dc.regularize_tracers(self.ctx, pos, tr, self.iters)
            target[k] = ((tr - self.nodes) * N).view(N, N, 2)
            scales[k] = float(N * N) / n
        dc.declutter_sync(self.ctx)
        return dens, scales, field, target


def fit_skip(field, target) -> float:
    """Least-squares kappa of target ~ kappa * field over all pairs."""
    f = field.double()
    return float((target.double() * f).sum() / (f * f).sum().clamp_min(1e-30))


def train(sg, dens, scales, target, steps: int, batch: int, lr: float, rng: np.random.Generator,
          time_budget_s: float | None = None, log_every: int = 0, field=None):
    """Adam on random mini-batches of the given pairs, cosine learning-rate
    decay over the steps or, with a time budget, over the budget."""
    import torch
    count = dens.shape[0]
    losses = []
    t0 = time.perf_counter()
    for s in range(steps):
        idx = torch.from_numpy(rng.choice(count, size=batch, replace=False)).to(dens.device)
        frac = s / max(steps, 1)
        if time_budget_s:
            frac = max(frac, (time.perf_counter() - t0) / time_budget_s)
        lr_s = lr * 0.5 * (1 + math.cos(math.pi * min(frac, 1.0)))
        want = log_every and (s % log_every == 0 or s == steps - 1)
        loss = dc.surrogate_train_step(sg, dens[idx].contiguous(), scales[idx].contiguous(),
                                       target[idx].contiguous(), lr_s, want_loss=bool(want),
                                       field=field[idx].contiguous() if field is not None else None)
        if want:
            losses.append((s, loss))
        if time_budget_s is not None and time.perf_counter() - t0 > time_budget_s:
            break
    return losses


def field_error(sg, dens, scales, target, batch: int = 8, field=None):
    """RMS and mean-abs error (pixels) of the predicted composed displacement."""
    import torch
    se, ae, cnt = 0.0, 0.0, 0
    out = torch.empty_like(target[:batch])
    for b0 in range(0, dens.shape[0], batch):
        b1 = min(dens.shape[0], b0 + batch)
        o = out[: b1 - b0]
        dc.surrogate_forward(sg, dens[b0:b1].contiguous(), scales[b0:b1].contiguous(), o,
                             field=field[b0:b1].contiguous() if field is not None else None)
        d = (o - target[b0:b1]).double()
        se += float((d * d).sum())
        ae += float(d.abs().sum())
        cnt += d.numel()
    ref = float((target.double() ** 2).mean().sqrt())
    return {"rms_px": math.sqrt(se / cnt), "mae_px": ae / cnt, "target_rms_px": ref}
