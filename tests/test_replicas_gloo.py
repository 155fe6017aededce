"""The N > 1 path of bench.py (independent replicas, one per rank): the timed
region's duration is the maximum over ranks and only rank 0 reports; checked
with world size 2 on the gloo backend (CPU)."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank          # the slower rank decides
    out[rank] = bench.max_over_ranks(ms, torch.device("cpu"))
    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_world_size_2():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    assert out[0] == 15.0 and out[1] == 15.0


def test_reference_arm_rank_1_does_no_work(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class A:
        steps, warmup = 1, 0
    bench.run_reference(A())
    assert capsys.readouterr().out == ""
