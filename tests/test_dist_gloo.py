"""Multi-rank host logic of bench.py on CPU: two gloo ranks (127.0.0.1),
the job time is the slowest rank's (all-reduce MAX), the job value counts
every rank's replicas, and the reference arm does no work on ranks > 0."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    ms = [120.0, 250.0][rank]
    mx = bench.max_over_ranks(ms, dist, torch.device("cpu"))
    val = bench.job_gflops(1000, 500, 2, world, mx)
    # the reference arm: rank > 0 returns at once (rank 0 would time the oracle)
    os.environ["RANK"], os.environ["WORLD_SIZE"] = str(rank), str(world)
    sys.argv = ["bench.py", "--impl", "reference", "--gpus", str(world)]
    ref_rc = bench.run_reference(bench.parse()) if rank > 0 else None
    dist.barrier()
    q.put((rank, mx, val, ref_rc))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sys.path.insert(0, ROOT)
    import bench
    expect = bench.nominal_flops(1000, 500) * 2 * 2 / 0.250 / 1e9
    for rank, mx, val, ref_rc in out:
        assert mx == 250.0
        assert abs(val - expect) <= 1e-9 * expect
    assert out[1][3] == 0


def test_single_process_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5, None, None) == 7.5
    assert bench.job_gflops(100, 10, 1, 1, 1000.0) == pytest.approx(bench.nominal_flops(100, 10) / 1e9)
