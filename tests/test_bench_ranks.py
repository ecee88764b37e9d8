"""The multi-rank host logic of bench.py on CPU (gloo, world size 2): the
replicas' timing is the slowest rank's and the throughput counts every
rank's particles; the reference arm runs on rank 0 only."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _combine(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        tmax, value = bench.combine_ranks(10.0 + 5.0 * rank, 1000, 4, world)
    finally:
        dist.destroy_process_group()
    with open(os.path.join(out, "r%d.json" % rank), "w") as f:
        json.dump({"tmax": tmax, "value": value}, f)


def test_replica_timing_is_the_slowest_rank(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    mp.spawn(_combine, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        d = json.load(open(tmp_path / ("r%d.json" % r)))
        assert d["tmax"] == 15.0
        assert abs(d["value"] - 2 * 1000 * 4 / 0.015) < 1e-6 * d["value"]


def _reference(rank, world, out):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    path = os.path.join(out, "ref%d.txt" % rank)
    with open(path, "w") as f:
        old = sys.stdout
        sys.stdout = f
        try:
            rc = bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0"])
        finally:
            sys.stdout = old
    assert rc == 0


def test_reference_arm_prints_on_rank_zero_only(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    mp.spawn(_reference, args=(2, str(tmp_path)), nprocs=2, join=True)
    line = open(tmp_path / "ref0.txt").read().strip().splitlines()
    assert len(line) == 1
    d = json.loads(line[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["n_gpus"] == 2
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert open(tmp_path / "ref1.txt").read() == ""
