"""The benchmark's multi-rank path on CPU: two gloo ranks (the replicas run
independent batches; the only collective is the max of their timed
seconds), whole-job rate = units of all ranks / that max."""
import json
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench._dist()
    seconds, rate = bench.whole_job(1.0 + rank, 100.0)
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"ws": ws, "rank": r, "seconds": seconds, "rate": rate}, f)


def test_two_gloo_ranks_take_the_slowest_rank(tmp_path):
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for r, d in enumerate(res):
        assert d["ws"] == 2 and d["rank"] == r
        assert d["seconds"] == pytest.approx(2.0)  # the slower rank's time
        assert d["rate"] == pytest.approx(2 * 100.0 / 2.0)  # units of both ranks


def test_single_rank_has_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job(2.0, 50.0) == (2.0, 25.0)
