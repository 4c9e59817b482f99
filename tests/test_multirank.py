"""The multi-rank host logic of bench.py on CPU: two gloo ranks (world size 2), no GPU.

bench.py runs one process per GPU, each on its own catalog (weak scaling, no data-path
collective): the timed region is reduced with MAX over ranks and the work with SUM. These tests
exercise exactly those helpers over a real gloo process group, and launch the reference arm
under torchrun with two ranks (rank 0 measures and prints, rank 1 exits without work).
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [100.0, 150.0][rank]          # rank 1 is the slow one
        pairs = [1.0e9, 3.0e9][rank]       # each rank's own catalog
        mx = bench.reduce_over_ranks([ms], "max", dist)[0]
        tot = bench.reduce_over_ranks([pairs], "sum", dist)[0]
        value = bench.whole_job(tot, 5, mx / 1e3)
        q.put((rank, mx, tot, value, bench.rank_seed(7, rank)))
    finally:
        dist.destroy_process_group()


def test_reductions_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, mx, tot, value, seed in out:
        assert mx == 150.0                       # max over ranks
        assert tot == 4.0e9                      # sum over ranks
        assert value == pytest.approx(4.0e9 * 5 / 0.150)
    assert out[0][4] != out[1][4]                # distinct catalogs per rank


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks([3.0, 4.0], "max") == [3.0, 4.0]
    assert bench.whole_job(10.0, 2, 4.0) == 5.0


def test_reference_arm_under_torchrun_two_ranks():
    env = dict(os.environ, OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "0", "--workload", "uniform_noise_2k", "--ref-step-s", "0.3"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1  # rank 0 alone prints
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_oracle_thread_count_and_cpu_model():
    """The CPU baseline is timed on all host cores and on one core; the thread count is set on
    the oracle and restored, and the CPU model is reported."""
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    oracle.build_oracle()
    n = oracle.num_threads()
    assert oracle.set_num_threads(1) == 1 and oracle.num_threads() == 1
    assert oracle.set_num_threads(n) == n
    assert isinstance(bench.cpu_model(), str) and bench.cpu_model()
