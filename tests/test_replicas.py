"""The multi-GPU path of bench.py is a job of independent replicas (frames
are independent units; there is no data-path exchange).  Its host logic runs
here on the CPU: two gloo ranks, spawned, agree on the slowest rank's step
time, and the job's value counts the units of every rank over that time; the
reference arm (the oracle) runs on rank 0 only."""
import io
import multiprocessing as mp
import os
import socket
import sys
from contextlib import redirect_stdout
from types import SimpleNamespace

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, step_ms, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, _ = bench.dist_info()
        slowest = bench.max_over_ranks(step_ms[r], w, "cpu")
        value = bench.job_value(2_000_000, w, slowest)
        dist.barrier()
        q.put((r, w, slowest, value))
    finally:
        dist.destroy_process_group()


def test_two_replicas_agree_on_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    step_ms = [12.5, 20.0]
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, step_ms, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=180) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[:2] for o in out] == [(0, 2), (1, 2)]
    assert all(o[2] == 20.0 for o in out)
    # 2 ranks x 2e6 units in 20 ms: 200 M units/s for the job
    assert all(abs(o[3] - 200.0) < 1e-9 for o in out)


def test_single_process_is_its_own_slowest_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.25, 1, "cpu") == 7.25
    assert abs(bench.job_value(1_000_000, 1, 10.0) - 100.0) < 1e-9


def test_reference_arm_runs_on_rank_0_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(SimpleNamespace(workload="iir_fir", steps=1, warmup=3))
    assert buf.getvalue() == ""
