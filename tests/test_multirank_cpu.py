"""The benchmark's multi-rank path on CPU ranks (gloo, world size 2): the
slowest rank's time is the one every rank reports, the whole-job value counts
every rank's copy of the workload, and the reference arm runs on rank 0 only.
Each rank also compresses its own shard with the oracle, and the shards'
stream sizes gathered over the group add up to the whole job's."""
import json
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def worker(rank, world, port, out_dir):
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    import oracle
    from paper_1805_01844_gb300 import datagen

    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    # rank r pretends its timed region took 10 + r ms
    slowest = bench.max_over_ranks(10.0 + rank, dist, "cpu")
    value = bench.weak_scaling_value(world, 1_000_000, 5, slowest)
    # each rank's own copy of the workload, compressed by the oracle
    x = datagen.cherenkov_events(2, seed=rank).reshape(-1)
    size = len(oracle.compress(x, 0, 64, 1024))
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([size], dtype=torch.int64))
    dist.barrier()
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
        json.dump({"slowest": slowest, "value": value, "size": size,
                   "sizes": [int(t.item()) for t in sizes]}, f)
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp

    port = free_port()
    mp.start_processes(worker, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(2)]
    assert res[0]["slowest"] == res[1]["slowest"] == 11.0
    assert res[0]["value"] == pytest.approx(2 * 1_000_000 * 5 / 0.011 / 1e9)
    assert res[0]["sizes"] == res[1]["sizes"] == [res[0]["size"], res[1]["size"]]


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench

    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                                     "--cpu-events", "1"])
    bench.run_reference(bench.parse())
    assert capsys.readouterr().out == ""
    monkeypatch.setenv("RANK", "0")
    bench.run_reference(bench.parse())
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
