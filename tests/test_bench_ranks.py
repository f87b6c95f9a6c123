"""The replica path of bench.py on CPU: two gloo ranks (no GPU).

bench.py --gpus N runs N independent replicas.  Its whole-job throughput
divides the unknowns all ranks solved (sum) by the slowest rank's time
(max).  This is the only collective on the path.  The test runs it on two
spawned gloo processes, with a rendezvous on 127.0.0.1.  The reference arm
runs on rank 0 only; the other ranks return without work.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms, unknowns = 10.0 + 2.5 * rank, 1000 * (rank + 1)
        out[rank] = bench.aggregate_ranks(ms, unknowns, world, "cpu")
        assert bench.dist_env() == (rank, world, rank)
    finally:
        dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    world, port = 2, free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(rank_main, args=(world, port, out), nprocs=world, join=True)
        got = dict(out)
    # max of 10.0 and 12.5 ms, sum of 1000 and 2000 unknowns, on both ranks
    assert got == {0: (12.5, 3000.0), 1: (12.5, 3000.0)}


def test_single_rank_runs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert not dist.is_initialized()
    assert bench.aggregate_ranks(7.0, 42, 1, "cpu") == (7.0, 42.0)


def test_reference_arm_other_ranks_do_no_work(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(bench, "oracle_state", lambda n: pytest.fail("rank 1 ran the oracle"))
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference"])
    bench.reference_arm(bench.parse_args())
    assert capsys.readouterr().out == ""
