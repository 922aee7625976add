"""The N > 1 path of bench.py on CPU: world_size-2 gloo process groups.

The setup path is not sharded (one level fits one GPU), so N GPUs run N
independent replicas; the only cross-rank work is the barrier around the timed
region and the maximum of the per-rank times.  These tests run that logic with
the gloo backend on the host: the maximum is taken over ranks, the whole-job
time per level divides it by the number of replicas, the reference arm runs
on rank 0 only, and a rank that fails is seen by the other rank as a
collective error instead of a hang.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, world, port):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)


def _max_worker(rank, world, port, q):
    _env(rank, world, port)
    import bench
    rep = bench.Replicas(backend="gloo", device="cpu")
    rep.barrier()
    local_ms = 100.0 + 50.0 * rank          # rank 1 is the slow replica
    ms = rep.max(local_ms)
    rep.barrier()
    q.put((rank, rep.world, ms, bench.per_level(ms, rep.world)))
    rep.close()


def test_max_over_ranks_and_per_level():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_max_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=5) for _ in range(world))
    for rank, w, ms, per in res:
        assert w == 2
        assert ms == 150.0                   # every rank sees the slowest replica
        assert per == pytest.approx(0.075)   # 2 levels in 150 ms


def _reference_worker(rank, world, port, q):
    _env(rank, world, port)
    import io
    import contextlib
    import bench
    args = type("A", (), {"steps": 1, "warmup": 0, "gpus": world})()
    out = io.StringIO()
    # a non-zero rank of the reference arm returns at once, before any work
    if rank != 0:
        with contextlib.redirect_stdout(out):
            r = bench.run_reference(args, bench.workload("32^3x64"))
        q.put((rank, r, out.getvalue()))
    else:
        q.put((rank, None, ""))


def test_reference_arm_runs_on_rank0_only():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_reference_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    res = dict((r, (v, o)) for r, v, o in (q.get(timeout=5) for _ in range(world)))
    assert res[1] == (None, "")


def _failing_worker(rank, world, port, q):
    _env(rank, world, port)
    import datetime
    import torch.distributed as dist
    dist.init_process_group("gloo", timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        # the replica fails between steps, before the timing collective
        dist.destroy_process_group()
        os._exit(3)
    try:
        t = torch.tensor([1.0], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        q.put((rank, "completed"))
    except Exception as e:  # noqa: BLE001 - any collective error is the expected outcome
        q.put((rank, "error:" + type(e).__name__))


def test_failed_replica_is_an_error_not_a_hang():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_failing_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert procs[1].exitcode == 3
    assert procs[0].exitcode == 0
    rank, outcome = q.get(timeout=5)
    assert rank == 0 and outcome.startswith("error:")


def test_step_stats():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    assert bench.step_stats([5.0]) == {"median": 5.0, "p90": 5.0, "min": 5.0, "max": 5.0}
    s = bench.step_stats([3.0, 1.0, 2.0, 4.0])
    assert s["median"] == 2.5 and s["p90"] == 4.0 and s["min"] == 1.0
    s = bench.step_stats(list(range(20, 0, -1)))
    assert s["median"] == 10.5 and s["p90"] == 18 and s["max"] == 20
