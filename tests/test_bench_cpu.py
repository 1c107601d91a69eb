"""CPU checks of bench.py: the multi-rank aggregation under torch.distributed
(gloo, world size 2) and the reference arm's JSON line."""
import json
import os
import socket
import subprocess
import sys

import pytest

from _util import ROOT


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r did 100 units in (10 + 5 r) ms
    rate, tmax = bench.aggregate(100.0, 10.0 + 5.0 * rank, dist, "cpu")
    if rank == 0:
        with open(out_path, "w") as f:
            json.dump({"rate": rate, "tmax": tmax}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_is_total_units_over_slowest_rank(tmp_path):
    import torch.multiprocessing as mp
    out = tmp_path / "agg.json"
    mp.start_processes(_rank_main, args=(2, _free_port(), str(out)), nprocs=2, start_method="spawn")
    res = json.loads(out.read_text())
    assert res["tmax"] == 15.0
    assert res["rate"] == pytest.approx(200.0 / 15e-3)


def test_aggregate_single_process():
    sys.path.insert(0, ROOT)
    import bench
    rate, tmax = bench.aggregate(50.0, 20.0)
    assert tmax == 20.0 and rate == pytest.approx(2500.0)


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--shape", "8x8x6",
                        "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["higher_is_better"] is True


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--shape", "8x8x6",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True, timeout=300, cwd=ROOT,
                       env=env)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_shard_cases_partitions_every_case_once():
    sys.path.insert(0, ROOT)
    import bench
    for n in (0, 1, 5, 96, 97):
        for world in (1, 2, 3, 4, 8):
            shards = [bench.shard_cases(n, world, r) for r in range(world)]
            flat = [c for sh in shards for c in sh]
            assert flat == list(range(n))                        # contiguous, in order, each case once
            sizes = [len(sh) for sh in shards]
            assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)
    with pytest.raises(ValueError):
        bench.shard_cases(4, 2, 2)


def _sharded_rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # 7 cases over 2 ranks: rank 0 solves 4 in 40 ms, rank 1 solves 3 in 36 ms
    mine = bench.shard_cases(7, world, rank)
    rate, tmax, total = bench.aggregate_sharded(len(mine), 40.0 - 4.0 * rank, dist, "cpu")
    gathered = [None] * world
    dist.all_gather_object(gathered, {"cases": list(mine)})
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
        json.dump({"rate": rate, "tmax": tmax, "total": total, "cases": [g["cases"] for g in gathered]}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_aggregate_gloo_world_two(tmp_path):
    import torch.multiprocessing as mp
    mp.start_processes(_sharded_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, start_method="spawn")
    for r in range(2):
        res = json.loads((tmp_path / ("rank%d.json" % r)).read_text())
        assert res["total"] == 7.0 and res["tmax"] == 40.0
        assert res["rate"] == pytest.approx(7.0 / 40e-3)
        assert res["cases"] == [[0, 1, 2, 3], [4, 5, 6]]
