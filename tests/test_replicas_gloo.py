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


def test_reference_arm_prints_the_contract_line(capsys, monkeypatch):
    """At N = 1 the reference arm (the FP64 oracle on the host cores, a
    bounded sample of the headline workload) prints one JSON line with the
    keys of the benchmark contract, the same metric and unit as the GPU arm,
    and a positive rate."""
    import json

    import bench
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.delenv("RANK", raising=False)

    class A:
        steps, warmup = 1, 0
    bench.run_reference(A())
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and "workload" in d["config"]
