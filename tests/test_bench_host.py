"""Host-side pieces of bench.py that need no GPU: the replicas-only aggregation
across ranks (world size 2 over gloo) and the FP64 oracle reference arm."""
import json
import os
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    secs = [2.0, 3.0][rank]
    units = [100, 100][rank]
    q.put((rank, bench.replica_totals(secs, units, world)))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_totals_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29517
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        assert out[r] == (3.0, 200.0)


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    j = json.loads(lines[0])
    assert j["impl"] == "reference" and j["unit"] == "MLUPS" and j["value"] > 0
    assert j["cpu_baseline"]["kind"] == "oracle" and j["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_nonzero_rank_exits_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_profile_traffic_only_for_the_profiled_sources(tmp_path, monkeypatch):
    """roofline.traffic comes from the committed ncu summary only while its
    source_sha matches the current kernel sources; otherwise it is null."""
    sys.path.insert(0, ROOT)
    import bench

    h = bench.kernel_source_hash()
    good = tmp_path / "good.md"
    good.write_text(f"source_sha = {h}\ntraffic_bytes_per_launch[f32] = 1.25e9\n")
    monkeypatch.setattr(bench, "PROFILE", str(good))
    assert bench.profile_traffic("f32") == 1.25e9
    assert bench.profile_traffic("bf16") is None
    stale = tmp_path / "stale.md"
    stale.write_text("source_sha = 0123456789abcdef\ntraffic_bytes_per_launch[f32] = 1.25e9\n")
    monkeypatch.setattr(bench, "PROFILE", str(stale))
    assert bench.profile_traffic("f32") is None
