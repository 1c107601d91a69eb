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
