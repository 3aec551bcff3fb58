"""The multi-rank path of bench.py on CPU: world_size-2 gloo ranks (replicas of
the workload, no collective on the data path; the whole-job value is the sum of
the ranks' units over the slowest rank's time)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import importlib.util
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    assert bench.dist_env()[:2] == (rank, world)
    # rank r refines (r+1) units in (1 + r) seconds
    value, slowest = bench.whole_job(float(rank + 1), float(1 + rank), dist, "cpu")
    dist.barrier()
    q.put((rank, value, slowest))
    dist.destroy_process_group()


def test_whole_job_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, slowest in got:
        assert slowest == 2.0                 # the slowest rank's time
        assert abs(value - 3.0 / 2.0) < 1e-12  # (1 + 2) units / 2 s


def test_whole_job_single_rank():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    assert bench.whole_job(10.0, 2.0) == (5.0, 2.0)
