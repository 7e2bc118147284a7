"""One scatterplot sharded over two ranks (gloo, world size 2, on the CPU):
the host logic of paper_2408_06513_gb300.sharded -- the partition of the
samples, the all-reduce of the uint32 count grid (int32 bit patterns that
wrap like unsigned sums) and the order of the steps -- with the CPU oracle
standing in for the CUDA kernels.  The shards moved by the two ranks,
joined, must be bit for bit the oracle's iterations of the whole plot."""

import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleOps:
    """splat_counts / density_from_counts / displacement_field /
    advect_samples of the binding, computed by the oracle on CPU tensors."""

    def __init__(self, p):
        import oracle
        self.o, self.p = oracle, p

    def splat_counts(self, ctx, pos, counts):
        c = self.o.splat(pos.numpy(), self.p.log2_res).astype(np.uint32)
        counts.copy_(torch.from_numpy(c.reshape(-1).view(np.int32)))

    def declutter_sync(self, ctx):
        pass

    def density_from_counts(self, ctx, counts, n):
        c = counts.numpy().view(np.uint32).reshape(ctx.N, ctx.N).astype(np.float64)
        r = self.p.radius()
        ctx.d_r = self.o.smooth(c, r, self.p.sigma) if r > 0 else c
        ctx.n = n

    def displacement_field(self, ctx):
        ctx.D = self.o.displacement(ctx.d_r, self.p.d0_for(ctx.n), self.p.pixel_center)

    def advect_samples(self, ctx, pos):
        pos.copy_(torch.from_numpy(self.o.advect(pos.numpy(), ctx.D, self.p.pixel_center, self.p.clamp_positions)))


class FakeCtx:
    def __init__(self, N):
        self.N = N


def _worker(rank, world, port, q, n, log2, r, iters):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as tdist

    import oracle
    import synth
    from paper_2408_06513_gb300 import sharded
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        z, _ = synth.tiny_mixture(n, seed=6)
        b, e = sharded.shard_bounds(n, world, rank)
        local = torch.from_numpy(z[b:e].copy())
        n_total = sharded.total_samples(e - b)
        p = oracle.Params(log2_res=log2, kernel_r=r)
        counts = sharded.regularize_sharded(FakeCtx(1 << log2), local, iters, n_total, ops=OracleOps(p))
        q.put((rank, b, e, n_total, local.numpy().copy(), counts.numpy().copy()))
    finally:
        tdist.destroy_process_group()


@pytest.mark.parametrize("r", [0, 2])
def test_sharded_plot_gloo_world2_matches_whole_plot(r):
    import torch.multiprocessing as mp

    import oracle
    import synth
    n, log2, iters = 4001, 6, 3
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(k, 2, port, q, n, log2, r, iters)) for k in range(2)]
    for pr in procs:
        pr.start()
    got = {}
    for _ in procs:
        rank, b, e, nt, pos, counts = q.get(timeout=300)
        got[rank] = (b, e, nt, pos, counts)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    assert got[0][0] == 0 and got[0][1] == got[1][0] and got[1][1] == n
    assert got[0][2] == got[1][2] == n
    joined = np.concatenate([got[0][3], got[1][3]])
    z, _ = synth.tiny_mixture(n, seed=6)
    p = oracle.Params(log2_res=log2, kernel_r=r)
    traj = oracle.regularize(z, p, iters)
    assert np.array_equal(joined, traj[-1])
    # the exchanged grid is the whole plot's grid of the last input
    want = oracle.splat(traj[-2], log2).astype(np.uint32).reshape(-1)
    for k in (0, 1):
        assert np.array_equal(got[k][4].view(np.uint32), want)


def test_shard_bounds_cover_every_sample_once():
    from paper_2408_06513_gb300 import sharded
    for n in (0, 1, 7, 1000, 1001):
        for world in (1, 2, 3, 8):
            spans = [sharded.shard_bounds(n, world, k) for k in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [e - b for b, e in spans]
            assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)
    with pytest.raises(ValueError):
        sharded.shard_bounds(10, 2, 2)


def test_uint32_sums_wrap_like_int32():
    # counts are exchanged as int32 bit patterns: sums past 2^31 come back
    # with the unsigned value's bits
    a = np.array([3_000_000_000, 5], np.uint32)
    b = np.array([1_000_000_000, 7], np.uint32)
    ta = torch.from_numpy(a.view(np.int32).copy())
    ta += torch.from_numpy(b.view(np.int32).copy())
    assert ta.numpy().view(np.uint32).tolist() == [4_000_000_000, 12]
