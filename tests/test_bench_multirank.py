"""The multi-process path of bench.py on CPU: two gloo ranks (127.0.0.1)
combine their timings as the GPU run does (work summed, time = slowest rank),
and the reference arm runs on rank 0 only."""
import argparse
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    units, secs = bench.job_totals(100.0 * (rank + 1), 1.0 + 0.5 * rank, dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, units, secs))


def test_two_gloo_ranks_sum_work_and_take_the_slowest_time():
    ws = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(ws))
    for rank, units, secs in got:
        assert units == 300.0      # 100 + 200: every rank's own instance counts
        assert secs == 1.5         # the slowest rank's time


def test_single_process_totals_are_local():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_totals(7.0, 2.0) == (7.0, 2.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = argparse.Namespace(gpus=2, steps=1, warmup=0, ref_budget=1.0)
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
