"""The N > 1 host path of bench.py on CPU: two gloo ranks (replicas only --
each rank runs the whole workload with its own seed, there is no data-path
collective; the only exchange is the max of the timed regions)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.dist_env()
    local_ms = 10.0 + 5.0 * rank                     # rank 1 is the slower one
    mx = bench.max_over_ranks(local_ms, w, "cpu")
    rate = bench.whole_job_rate(3.0e7, 4, w, mx)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
        json.dump({"rank": r, "world": w, "local_rank": lr, "max_ms": mx, "rate": rate}, f)


def test_two_gloo_ranks_reduce_to_the_slowest(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as tmp
    port = _free_port()
    tmp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(2)]
    for r, d in enumerate(res):
        assert (d["rank"], d["world"], d["local_rank"]) == (r, 2, r)
        assert d["max_ms"] == 15.0                    # both ranks see the slowest rank's time
        assert d["rate"] == pytest.approx(2 * 3.0e7 * 4 / 0.015)


def test_reference_arm_runs_on_rank0_only():
    """Under torchrun the oracle arm runs on rank 0 alone; another rank exits
    0 at once without printing."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_json_line_on_rank0():
    """The oracle arm at N = 1: one JSON line with the headline's metric and
    unit, impl "reference", a cpu_baseline describing the run, and an e2e
    object with no host-device bytes."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["steps"] == 1 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
