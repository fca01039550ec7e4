"""Multi-GPU runs are independent replicas (no data-path collective): the
bench times each replica, takes the slowest over ranks and reports the
whole-job rate. The host side of that runs here as two gloo ranks on CPU."""
import json
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slowest = bench.max_over_ranks(10.0 + 5.0 * rank, dist)      # rank 1 is the slow one
        value = bench.replicas_value(1000, 4, slowest, world)
        # the reference arm: rank 0 alone works, the others leave with 0
        args = type("A", (), {"workload": "naca0012_10k", "shuffle": 0, "mach": 0.63, "aoa": 2.0, "order": 1,
                              "inner": 0, "limiter": 0.0, "scheme": "euler", "steps": 1, "warmup": 0})()
        rc = bench.run_reference(args, rank, world) if rank == 1 else None
        with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
            json.dump({"slowest": slowest, "value": value, "ref_rc": rc}, f)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replica_timing_takes_the_slowest_rank(tmp_path):
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(2)]
    for r in res:
        assert r["slowest"] == 15.0                                  # max over ranks, on every rank
        assert r["value"] == pytest.approx(2 * 1000 * 4 / 0.015)     # whole job: both replicas' work
    assert res[1]["ref_rc"] == 0                                     # non-zero ranks skip the reference arm
