"""The N > 1 path of bench.py is replicas only: every rank advances its own seeded instance and
the job's time is the slowest rank's.  Checked here with world_size 2 over gloo on the CPU: the
max-over-ranks reduction and the whole-job value."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = _bench()
    ms = [120.0, 150.0][rank]                    # rank 1 is the slow one
    m = b.max_over_ranks(ms, dist, device="cpu")
    out.put((rank, m, b.job_value(world, 1000, 10, m)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_job_value():
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [150.0, 150.0]                 # both see the slowest rank
    assert all(abs(r[2] - 2 * 1000 * 10 / 0.150) < 1e-6 for r in res)


def test_single_rank_passthrough():
    b = _bench()
    assert b.max_over_ranks(42.0, None) == 42.0
    assert b.job_value(1, 500, 4, 2000.0) == 1000.0
