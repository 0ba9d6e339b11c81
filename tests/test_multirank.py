"""The N > 1 host logic of bench.py on two CPU ranks (gloo): every rank solves
its own system (independent replicas, no data-path collective), the timed
region is taken as the slowest rank's, and the whole-job value counts the work
of all ranks. The reference arm runs on rank 0 only."""
import json
import os
import socket
import sys
import types

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        elapsed = [10.0, 12.5][rank]                     # this rank's timed region (ms)
        dist.barrier()
        slowest = bench.max_over_ranks(elapsed, dist, "cpu")
        value = bench.whole_job_rate(8256, 3, world, slowest)
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.input_seed(rank))
        ref_rc = None
        if rank != 0:                                    # returns before any oracle work
            ref_rc = bench.run_reference(types.SimpleNamespace(steps=1, warmup=0))
        with open(os.path.join(outdir, f"{rank}.json"), "w") as f:
            json.dump({"slowest": slowest, "value": value, "seeds": seeds, "ref_rc": ref_rc}, f)
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas(tmp_path):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.loads((tmp_path / f"{r}.json").read_text()) for r in range(world)]
    for r in res:
        assert r["slowest"] == 12.5                      # max over ranks, on every rank
        assert r["value"] == pytest.approx(8256 * 3 * world / 12.5e-3)
        assert len(set(r["seeds"])) == world             # one independent system per rank
    assert res[1]["ref_rc"] == 0


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.0, None, "cpu") == 7.0
    assert bench.whole_job_rate(100, 4, 1, 2.0) == pytest.approx(100 * 4 / 2e-3)
