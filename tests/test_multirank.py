"""The multi-GPU path of the bench on CPU: two gloo ranks.

The solve shards by drone: every rank solves its own batch (its own seeded
courses) with no collective on the data path; only the timing is reduced
(slowest rank's time, all ranks' rollout steps).
"""
import json
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    items = bench.workload(rank, 6)
    steps = float(sum(it.K * it.N for it in items))
    ms = 2.0 + rank  # rank 1 is the slow one
    value, ms_max, total = bench.aggregate(world, steps, ms)
    digest = [int(it.K) for it in items] + [round(float(it.track.gates[0, 0]), 6) for it in items]
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"steps": steps, "value": value, "ms_max": ms_max, "total": total, "digest": digest}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_drones_and_reduce_timing(tmp_path):
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r0 = json.load(open(tmp_path / "r0.json"))
    r1 = json.load(open(tmp_path / "r1.json"))
    assert r0["digest"] != r1["digest"]  # each rank has its own drones
    total = r0["steps"] + r1["steps"]
    for r in (r0, r1):
        assert r["ms_max"] == 3.0
        assert r["total"] == total
        assert abs(r["value"] - total / 3.0e-3) < 1e-6 * total
