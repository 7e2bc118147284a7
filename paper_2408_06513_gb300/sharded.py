"""One scatterplot whose samples are split over several ranks (one GPU each).

Every rank holds a contiguous shard of the samples.  Per iteration of
Sec. 4.3 each rank splats its shard into a uint32 count grid, the ranks sum
the grids (one all-reduce of N*N uint32 values: the only exchange), and then
every rank smooths the summed grid, evaluates the integral images and the
displacement of eqs. (map), (map_res) on it and moves its own samples.
Integer sums are exact, so the summed grid is bit for bit the grid of all
samples and every rank moves its samples exactly as one GPU holding the whole
plot would (``regularize`` gives the same bits).

The exchange is a callable ``reduce(tensor)`` that sums an int32 tensor in
place over the ranks (uint32 bit patterns: two's-complement sums wrap like
unsigned ones); by default ``torch.distributed.all_reduce``.  Argument
marshalling and the exchange only: every step of the method runs in the
CUDA library.
"""

from __future__ import annotations

from . import declutter as dc


def shard_bounds(n: int, world: int, rank: int) -> tuple[int, int]:
    """Half-open sample range [begin, end) of ``rank``: contiguous shards
    whose sizes differ by at most one, the larger ones first."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError(f"n={n}, world={world}, rank={rank}")
    base, extra = divmod(n, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def _dist_sum(t, group=None):
    import torch.distributed as tdist
    tdist.all_reduce(t, op=tdist.ReduceOp.SUM, group=group)


def total_samples(n_local: int, reduce=None, device=None) -> int:
    """Samples of the whole plot: the shards' sizes summed over the ranks."""
    import torch
    t = torch.tensor([n_local], dtype=torch.int64, device=device)
    (reduce or _dist_sum)(t)
    return int(t.item())


def regularize_sharded(ctx, local_pos, iters: int, n_total: int, reduce=None, ops=dc, counts=None):
    """``iters`` iterations of Sec. 4.3 on this rank's shard ``local_pos``
    (float32 [n_local, 2], moved in place) of a plot of ``n_total`` samples.

    ``reduce``: sums an int32 tensor over the ranks in place (default: the
    default process group's all-reduce).  ``ops``: the module providing
    splat_counts / density_from_counts / displacement_field /
    advect_samples / declutter_sync (the CUDA binding).  ``counts``: an
    int32 tensor of N*N elements to use as the exchange buffer, or None.
    Returns the exchange buffer (the summed grid of the last iteration's
    input positions)."""
    import torch
    if n_total < 0 or n_total >= 1 << 32:
        raise ValueError(f"n_total = {n_total}")
    red = reduce or _dist_sum
    NN = ctx.N * ctx.N
    if counts is None:
        counts = torch.empty(NN, dtype=torch.int32, device=local_pos.device)
    for _ in range(int(iters)):
        ops.splat_counts(ctx, local_pos, counts)
        # the exchange reads the grid on another stream or on the host: the
        # splat must be complete
        ops.declutter_sync(ctx)
        red(counts)
        if counts.is_cuda:  # the library's stream reads what the reduction wrote
            torch.cuda.current_stream(counts.device).synchronize()
        ops.density_from_counts(ctx, counts, n_total)
        ops.displacement_field(ctx)
        ops.advect_samples(ctx, local_pos)
    ops.declutter_sync(ctx)
    return counts
