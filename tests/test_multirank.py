"""The N > 1 path of bench.py on the CPU: world_size-2 gloo ranks run the
max-over-ranks timing reduction (replicas: no collective on the data path, one
all-reduce of the timed total) and the reference arm's rank rule (rank 0 alone
works)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, totals, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, v = bench.reduce_timing(totals[rank], 2 * 3, world, "cpu")
    out[rank] = (t, v)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_timing_is_max_over_ranks():
    import torch.multiprocessing as mp
    world = 2
    totals = [1.25, 2.5]
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, totals, out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        t, v = out[r]
        assert t == max(totals)
        assert v == pytest.approx(2 * 3 * world / max(totals))


def test_single_rank_timing_has_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_timing(2.0, 6, 1, "cpu") == (2.0, 3.0)


def test_reference_arm_other_ranks_do_no_work(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"])
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    called = []
    monkeypatch.setattr(bench, "run_reference", lambda *a, **k: called.append(1) or {})
    bench.main()
    assert called == [] and capsys.readouterr().out == ""
