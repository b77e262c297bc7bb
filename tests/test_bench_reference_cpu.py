"""The benchmark's reference arm on CPU: `bench.py --impl reference` times the
oracle on a bounded sample of the workload and prints one JSON line with the
same metric, unit and direction as the GPU arm, a `cpu_baseline` describing
the run and an `e2e` entry with no host-device bytes; under several ranks only
rank 0 runs it.  Also the full-size oracle estimate the GPU arm reports beside
its own line."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr
    return p.stdout


def test_reference_arm_prints_one_contract_line():
    sys.path.insert(0, ROOT)
    import bench

    out = [l for l in _run({}).splitlines() if l.strip()]
    assert len(out) == 1
    line = json.loads(out[0])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == "GDOF/s"
    assert line["higher_is_better"] is True and line["scaling"] == "weak"
    assert line["steps"] == 1 and line["warmup"] == 0 and line["n_gpus"] == 1
    assert line["vs_baseline"] is None and line["data"] == "synthetic"
    assert line["config"]["workload"] == bench.WORKLOAD
    assert line["value"] > 0 and line["ms_per_step"] > 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["unit"] == "GDOF/s" and cb["cores"] >= 1
    assert cb["value"] == line["value"] and "12^3" in cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == "GDOF/s"
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    out = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert out.strip() == ""


def test_oracle_extrapolation_scales_by_elements_and_gpu_iterations():
    sys.path.insert(0, ROOT)
    import bench

    # 12 iterations in 1.2 s on 12^3: 0.1 s per iteration, x 64 at 48^3, x 7
    r = bench.oracle_extrapolated(1.2, 12, 12, 48, 7, 38272753)
    assert r["kind"] == "extrapolated" and r["iterations"] == 7
    assert abs(r["per_iteration_s"] - 6.4) < 1e-12
    assert abs(r["solve_s"] - 44.8) < 1e-12
    assert abs(r["gdofs"] - 38272753 / 44.8 / 1e9) < 1e-15
