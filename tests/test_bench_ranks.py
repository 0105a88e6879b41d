"""bench.py's multi-rank launch on CPU: torchrun with two gloo ranks and the reference arm (the CPU
oracle on a small sample).  Rank 0 alone measures and prints one JSON line; rank 1 exits cleanly
without work; the replicas share no data-path collective."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_under_two_gloo_ranks():
    pytest.importorskip("torch.distributed")
    env = dict(os.environ, OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", "29533", "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--bodies", "4096"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["value"] > 0 and line["unit"] == "bodies/s"
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_bench_energy_report_matches_the_oracle_energy():
    """The bench's energy report uses its own numpy pair sum (the bench executes the oracle only
    for its CPU baseline); on the 4096-body Plummer state it agrees with the oracle's §2.3 energy
    to rounding."""
    sys.path.insert(0, ROOT)
    import bench
    import ics
    import oracle
    w = ics.WORKLOADS["plummer_4k"]
    pos, vel, mass = ics.plummer(w["n"], w["seed"])
    ref = oracle.energy(pos, vel, mass, 1.0, w["eps"])[2]
    assert abs(bench.plain_energy(pos, vel, mass, w["eps"]) - ref) <= 1e-12 * abs(ref)
