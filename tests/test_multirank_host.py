"""The multi-rank host logic of bench.py on CPU: two gloo ranks (the
replicas-only path: no collective on the data path, only the timing
reduction), the rank setup from the launcher's environment, and the reference
arm's rule that ranks other than 0 exit without work."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    args = type("A", (), {"gpus": world})()
    w, r, loc = bench.dist_setup(args)
    per_rank_s = 1.0 + rank  # rank 1 is the slow one
    slowest = bench.max_over_ranks(per_rank_s, torch.device("cpu"))
    rate = bench.job_rate(100.0, w, slowest)
    out.put((r, w, loc, slowest, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [x[0] for x in res] == [0, 1] and all(x[1] == 2 for x in res)
    assert [x[2] for x in res] == [0, 1]
    for _, _, _, slowest, rate in res:
        assert slowest == 2.0               # every rank sees the slowest rank's time
        assert rate == pytest.approx(100.0)  # 2 ranks x 100 units / 2 s


def test_single_process_defaults(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_setup(None) == (1, 0, 0)
    assert bench.max_over_ranks(3.5, torch.device("cpu")) == 3.5
    assert bench.job_rate(10.0, 1, 2.0) == 5.0


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    args = type("A", (), {"gpus": 2, "steps": 1, "warmup": 0, "seed": 1})()
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
