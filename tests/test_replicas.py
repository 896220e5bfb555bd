"""The N > 1 replica path of the benchmark (one process per GPU, no data-path
collective): rendezvous, barrier and max-over-ranks timing, run here as two
gloo ranks on the CPU."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    b = _bench()
    r, w, local = b.dist_setup(False)
    b.barrier(w)
    slowest = b.max_over_ranks(1.5 * (rank + 1), w, torch.device("cpu"))
    # whole-job throughput: units of all ranks over the slowest rank's time
    value = 1000 * w / (slowest * 1e-3)
    out.put((r, w, local, slowest, value))
    b.barrier(w)
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    assert all(r[3] == 3.0 for r in res)          # both ranks see the slower rank's 3.0 ms
    assert all(abs(r[4] - 2000 / 3e-3) < 1e-6 for r in res)


def _reference_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    b = _bench()
    # ranks other than 0 leave the reference arm at once, before reading any argument
    out.put((rank, b.run_reference(None) is None))


def test_reference_arm_runs_on_rank_zero_only():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    p = ctx.Process(target=_reference_worker, args=(1, 2, port, q))
    p.start()
    rank, ok = q.get(timeout=120)
    p.join(timeout=60)
    assert p.exitcode == 0 and rank == 1 and ok
