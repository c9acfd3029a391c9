"""bench.py's multi-rank host logic on CPU: two gloo ranks, each solving its
own sequence, reduce their times with a max and count the frames of all
ranks (weak scaling, replicas only). No GPU needed."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist, r, w, local = bench.dist_setup("gloo")
    assert (r, w, local) == (rank, world, rank)
    t_ms = 100.0 * (rank + 1)  # rank 1 is the slower one
    t_max = bench.max_over_ranks(dist, t_ms, "cpu")
    out[rank] = (t_max, bench.aggregate_rate(w, 30, t_max))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time_and_sum_the_frames():
    world, port = 2, _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    for rank in range(world):
        t_max, rate = out[rank]
        assert t_max == 200.0
        assert rate == pytest.approx(2 * 30 / 0.2)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")

    class Args:
        steps, warmup = 1, 3
    bench.run_reference(Args())
    assert capsys.readouterr().out == ""
