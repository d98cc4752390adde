"""Host side of the multi-GPU path (replicas and ensemble sharding) with two
gloo ranks on the CPU: the cases are dealt out without overlap, the per-case
results come back in case order, and the job time is the slowest rank's."""
import json
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2207_09431_gb300 import inputs, replicas


def test_shard_and_unshard_round_trip():
    items = list(range(11))
    parts = [replicas.shard(items, r, 3) for r in range(3)]
    assert sorted(sum(parts, [])) == items
    assert replicas.unshard(parts) == items
    with pytest.raises(ValueError):
        replicas.shard(items, 3, 3)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_path):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cases = inputs.ensemble_cases(10, seed=3)
    mine = replicas.shard(cases, rank, world)
    # a per-case result computed on this rank only: the case's grid size and Eotvos number
    local = [[int(p["nx"]), int(p["ny"]), round(float(m["Eo"]), 9)] for p, _, m in mine]
    merged = replicas.gather_results(local, dist)
    t = replicas.job_time_ms(10.0 * (rank + 1), dist)
    if rank == 0:
        with open(out_path, "w") as f:
            json.dump([merged, t], f)
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    out = tmp_path / "result.txt"
    mp.start_processes(_worker, args=(2, _free_port(), str(out)), nprocs=2, join=True, start_method="spawn")
    merged, t = json.loads(out.read_text())
    want = [[int(p["nx"]), int(p["ny"]), round(float(m["Eo"]), 9)] for p, _, m in inputs.ensemble_cases(10, seed=3)]
    assert merged == want
    assert t == 20.0
