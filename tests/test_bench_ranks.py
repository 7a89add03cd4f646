"""Host logic of the multi-rank bench (replicas, one rank per GPU) on CPU:
world_size-2 gloo ranks agree on the slowest rank's time, the job value counts
every rank's points, and the CPU reference arm runs on rank 0 only."""
import importlib.util
import io
import os
import socket
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        b = load_bench()
        t = b.max_over_ranks(10.0 + 5.0 * rank, ws, "cpu")
        out[rank] = (t, b.job_value(1_000_000, ws, t / 10))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_ranks_agree_on_the_slowest_time():
    ws = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(ws, free_port(), out), nprocs=ws, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    # 2 ranks x 1e6 points in 1.5 ms per step
    assert res[0][1] == pytest.approx(2e6 / 1.5e-3)


def test_single_rank_keeps_its_own_time():
    b = load_bench()
    assert b.max_over_ranks(7.5, 1, "cpu") == 7.5
    assert b.job_value(1000, 1, 2.0) == pytest.approx(5e5)


def test_reference_arm_runs_on_rank_zero_only():
    b = load_bench()
    buf = io.StringIO()
    with redirect_stdout(buf):
        rc = b.run_reference(None, 2, 1)
    assert rc == 0 and buf.getvalue() == ""
