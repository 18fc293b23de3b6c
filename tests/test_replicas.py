"""Multi-GPU host logic (independent replicas) on CPU with gloo, world size 2.

The search path does not shard: each rank runs a replica of the whole path on
its own batch, and only the timing is combined (MAX over ranks) into one
whole-job throughput. These tests run that combination on two CPU ranks.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, elapsed, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2504_04018_gb300 import replicas as R
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    R.barrier()
    t = R.max_over_ranks(elapsed[rank], torch.device("cpu"))
    rate = R.job_rate(1000, world, 4, t)
    R.barrier()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"max_ms": t, "rate": rate}, f)
    dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_gloo(tmp_path):
    elapsed = [125.0, 250.0]
    mp.start_processes(_worker, args=(2, _free_port(), elapsed, str(tmp_path)), nprocs=2,
                       join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(2)]
    for r in res:
        assert r["max_ms"] == 250.0
        # 2 replicas x 1000 queries x 4 steps in 0.25 s
        assert r["rate"] == pytest.approx(2 * 1000 * 4 / 0.25)


def test_single_process_identity():
    from paper_2504_04018_gb300 import replicas as R
    assert R.max_over_ranks(3.5) == 3.5
    assert R.job_rate(10, 1, 2, 1000.0) == pytest.approx(20.0)
    with pytest.raises(ValueError):
        R.job_rate(10, 1, 2, 0.0)


def test_reference_arm_nonzero_rank_is_silent():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""


def test_reference_arm_json_line():
    """The reference arm (the oracle on the host cores) prints one JSON line
    with the keys the benchmark contract names."""
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "2", "--warmup", "1", "--n", "20000", "--nq", "64"],
                       env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e", "impl"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_roofline_traffic_only_for_unchanged_kernel(tmp_path, monkeypatch):
    """The bench reports the recorded DRAM traffic only for the captured
    variant and search parameters, and only while the kernel sources hash to
    the recorded value."""
    import importlib
    bench = importlib.import_module("bench")
    rec = json.load(open(os.path.join(ROOT, "profiles", "search_kernel_traffic.txt")))
    name, r = next(iter(rec.items()))
    params = dict(r["params"], max_expansions=0, rerank=1, warps_per_block=1, hash_slots=0,
                  lanes_per_row=4)
    assert bench.measured_traffic("scale:some-other-variant", params) is None
    assert bench.measured_traffic(name, dict(params, ef=params["ef"] + 1)) is None
    # a copy of the tree whose kernel source differs by one byte
    root = tmp_path / "tree"
    for rel in r["kernel_sources"] + ["profiles/search_kernel_traffic.txt"]:
        dst = root / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        dst.write_bytes(open(os.path.join(ROOT, rel), "rb").read())
    monkeypatch.setattr(bench, "ROOT", str(root))
    same = bench.measured_traffic(name, params)
    src = root / r["kernel_sources"][0]
    src.write_bytes(src.read_bytes() + b"\n")
    assert bench.measured_traffic(name, params) is None
    if same is not None:
        assert same == r["traffic_bytes_per_launch"]
