"""Host logic of the multi-rank benchmark path, run as gloo ranks on CPU.

Ranks fit independent images (no collective on the data path); the only
exchange is the max-over-ranks step time, and the job throughput counts the
steps of every rank."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, lr = bench.rank_env()
    ms = 1.0 + 0.5 * rank                      # rank 1 is the slowest
    m = bench.max_over_ranks(ms, dist, "cpu")
    seeds = [bench.rank_workload(bench.WORKLOAD, k)["seed"] for k in range(world)]
    out[rank] = (w, r, lr, m, bench.job_throughput(m, w), seeds)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_fit_distinct_images():
    world = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        w, r, lr, m, thr, seeds = res[rank]
        assert (w, r, lr) == (world, rank, rank)
        assert m == 1.5                        # max over ranks, seen by every rank
        assert abs(thr - world * 1000.0 / 1.5) < 1e-9
        assert len(set(seeds)) == world       # independent problems per rank


def test_reference_arm_is_silent_on_other_ranks(capsys, monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup = 1, 0
    bench.run_reference(A())
    assert capsys.readouterr().out == ""
