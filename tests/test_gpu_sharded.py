"""One plot split into sample shards on the GPU: splat_counts per shard, the
grids summed (the exchange of a multi-rank run, here an in-process sum),
density_from_counts, displacement_field and advect_samples per shard must
give the positions of regularize() on the whole plot, bit for bit
(integer counts are exact; every sample then moves by the same field)."""

import numpy as np
import pytest

import synth

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


@pytest.mark.parametrize("log2,r,shards", [(7, 2, 2), (7, 0, 3), (9, 4, 4)])
def test_sharded_steps_match_regularize(dc, log2, r, shards):
    from paper_2408_06513_gb300 import sharded
    z, _ = synth.gmm20(300_001, seed=7) if log2 == 9 else synth.tiny_mixture(20_001, seed=3)
    n = z.shape[0]
    N = 1 << log2
    iters = 3
    ctx = dc.declutter_create(log2, kernel_r=r)
    try:
        whole = to_dev(z)
        dc.regularize(ctx, whole, iters)
        dc.declutter_sync(ctx)
        parts = [to_dev(z[slice(*sharded.shard_bounds(n, shards, k))]) for k in range(shards)]
        grids = [torch.empty(N * N, dtype=torch.int32, device=DEV) for _ in range(shards)]
        for _ in range(iters):
            for part, g in zip(parts, grids):
                dc.splat_counts(ctx, part, g)
            total = torch.stack(grids).sum(0, dtype=torch.int64).to(torch.int32)  # the exchange
            dc.declutter_sync(ctx)
            dc.density_from_counts(ctx, total, n)
            dc.displacement_field(ctx)
            for part in parts:
                dc.advect_samples(ctx, part)
        dc.declutter_sync(ctx)
        joined = torch.cat(parts)
        assert torch.equal(joined, whole)
        # the exchanged grid of the last iteration is the oracle's splat of its input
        counts = torch.empty(N * N, dtype=torch.int32, device=DEV)
        dc.declutter_counts(ctx, counts)
        dc.declutter_sync(ctx)
        assert np.array_equal(counts.cpu().numpy(), total.cpu().numpy())
    finally:
        dc.declutter_destroy(ctx)


def test_sharded_driver_single_rank(dc):
    # the driver with a one-rank exchange equals regularize()
    from paper_2408_06513_gb300 import sharded
    z, _ = synth.tiny_mixture()
    ctx = dc.declutter_create(7, kernel_r=2)
    try:
        a, b = to_dev(z), to_dev(z)
        dc.regularize(ctx, a, 4)
        counts = sharded.regularize_sharded(ctx, b, 4, z.shape[0], reduce=lambda t: None)
        assert torch.equal(a, b)
        assert int(counts.cpu().numpy().view(np.uint32).sum()) == z.shape[0]
    finally:
        dc.declutter_destroy(ctx)
