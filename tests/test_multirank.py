"""The benchmark's multi-GPU mode runs independent populations ("replicas
only": no collective on the data path).  Its host logic -- one seed per
rank, the slowest rank's time, whole-job throughput, one JSON line from rank
0 -- runs here as two gloo ranks on the CPU."""
import json
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seed = bench.rank_seed(12345, rank)
        elapsed = [2.0, 5.0][rank]          # seconds; rank 1 is the slow one
        units = 1000.0 * (rank + 1)          # per-rank work differs only to catch mixing
        slowest = bench.max_over_ranks(elapsed, dist)
        seeds = [None] * world
        dist.all_gather_object(seeds, seed)
        value = bench.job_throughput(1000.0, world, slowest)
        if rank == 0:
            with open(os.path.join(out_dir, "line.json"), "w") as f:
                f.write(json.dumps({"slowest": slowest, "seeds": seeds, "value": value,
                                    "units": units}))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_on_gloo(tmp_path):
    port = 29500 + (os.getpid() % 2000)
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    line = json.loads((tmp_path / "line.json").read_text())
    assert line["slowest"] == 5.0
    assert len(set(line["seeds"])) == 2              # independent populations
    assert line["value"] == pytest.approx(2 * 1000.0 / 5.0)
