"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the
whole-job aggregation (slowest rank's step time, bytes summed over ranks)
and the reference arm's rule that only rank 0 runs and prints."""
import importlib.util
import os
import socket
import sys

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


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        t_ms = [0.050, 0.080][rank]  # rank 1 is the slower one
        val, t = b.whole_job(torch, 241.44e6, t_ms, world, torch.device("cpu"))
        out[rank] = (val, t)
    finally:
        dist.destroy_process_group()


def test_whole_job_two_gloo_ranks():
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True,
                       start_method="spawn")
    assert set(out.keys()) == {0, 1}
    for r in range(world):
        val, t = out[r]
        assert t == pytest.approx(0.080)  # the slowest rank's step time
        assert val == pytest.approx(2 * 241.44e6 / 0.080 / 1e6)  # bytes of both ranks


def test_whole_job_single_rank_is_plain_ratio():
    b = _bench()
    val, t = b.whole_job(torch, 1e9, 0.5, 1, torch.device("cpu"))
    assert (val, t) == (pytest.approx(2000.0), 0.5)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun a rank other than 0 returns 0 at once, printing nothing."""
    b = _bench()
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    assert b.main() == 0
    assert capsys.readouterr().out == ""
