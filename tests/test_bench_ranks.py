"""The multi-rank path of bench.py on the CPU: gloo process groups of world
size 2.  Each rank regularises its own scatterplot (independent problems, no
collective in the data path); the only collectives are the barrier around the
timed region and the max over ranks of the step time.  The GPU steps
themselves need a GPU; what is checked here is the host logic around them:
rank discovery, the max-over-ranks reduction, the whole-job value, and that
under torchrun only rank 0 prints a bench line."""

import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    w, r, local, pg = bench.dist_init()
    try:
        assert pg is not None and (w, r, local) == (world, rank, rank)
        assert torch.distributed.get_backend() == "gloo"
        # rank-dependent timings: the slowest rank sets the job's time
        job = bench.combine_ranks(pg, w, 1000, 8, 10.0 + 5.0 * rank, 0.02 + 0.01 * rank)
        bench.barrier(pg)
        q.put((rank, job))
    finally:
        pg.destroy_process_group()


def test_combine_ranks_gloo_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    for _ in procs:
        rank, job = q.get(timeout=120)
        got[rank] = job
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(got) == [0, 1]
    for job in got.values():
        assert job["ms_per_step"] == 15.0
        assert job["value"] == pytest.approx(2 * 1000 * 8 / 15e-3 / 1e6)
        assert job["e2e_value"] == pytest.approx(2 * 1000 * 8 / 0.03 / 1e6)


def test_combine_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    job = bench.combine_ranks(None, 1, 1_000_000, 8, 0.25, 0.5)
    assert job["ms_per_step"] == 0.25
    assert job["value"] == pytest.approx(8e6 / 0.25e-3 / 1e6)
    assert job["e2e_value"] == pytest.approx(8e6 / 0.5 / 1e6)


def test_reference_arm_torchrun_world2():
    """Launched like the multi-GPU bench (torchrun, two ranks): rank 0 times
    the oracle on a bounded sample and prints the one bench line; rank 1
    exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "3", "--cpu-budget", "0.2"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["steps"] == 1 and d["warmup"] == 3
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    # the same work as the GPU arm: one plot per rank
    assert "each of 2 plot(s)" in d["cpu_baseline"]["sample"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0
