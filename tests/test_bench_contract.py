"""The benchmark's CPU side: the reference arm (the FP64 oracle timed on the
host cores) prints the JSON line of the benchmark contract with the GPU arm's
metric, unit and workload, and ranks other than 0 print nothing."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _run(env_extra=None):
    env = dict(os.environ, **(env_extra or {}))
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert p.returncode == 0, p.stderr[-2000:]
    return [l for l in p.stdout.splitlines() if l.strip()]


@pytest.mark.timeout(900)
def test_reference_arm_prints_one_contract_line():
    lines = _run()
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert (d["metric"], d["unit"], d["config"]) == (bench.METRIC, bench.UNIT, dict(bench.WORKLOAD))
    assert d["higher_is_better"] is True and d["n_gpus"] == 1 and d["steps"] >= 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["e2e"] == {"value": d["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]


def test_reference_arm_is_silent_on_other_ranks():
    assert _run({"RANK": "1", "WORLD_SIZE": "2"}) == []


def test_compulsory_bytes_of_the_benchmark_workload():
    """The bytes model behind the roofline line, at the 256-structure workload
    (57,101 atoms, 2,679,524 radial and 474,686 angular pairs): every kernel's
    bytes grow with its units, and the c-gradient sweep's compulsory bytes are
    the 138.8 MB its profile summary compares the measured traffic with."""
    full = bench.algo_bytes(N=57101, PR=2679524, PA=474686)
    assert full["cgrad"] == pytest.approx(138.76e6, rel=1e-3)
    double = bench.algo_bytes(N=2 * 57101, PR=2 * 2679524, PA=2 * 474686)
    for k, v in full.items():
        assert v > 0 and double[k] == pytest.approx(2 * v), k


def test_work_model_of_the_benchmark_workload():
    """The FLOP model behind the roofline line at the 256-structure workload:
    the tangent sweep's angular part costs 4 N_q^A K + 270 + 4 N_q^A L =
    468 + 270 + 864 = 1,602 FLOP per angular pair plus 2 N_q^A L = 432 per
    atom, 0.785 GFLOP per launch; the network 12 N_des H per atom in all."""
    f = bench.work_model_flops(N=57101, PR=2679524, PA=474686)
    assert f["tangent_angular"] == 1602 * 474686 + 432 * 57101
    assert f["tangent_angular"] == pytest.approx(0.785e9, rel=1e-3)
    assert f["mlp_fwd"] + f["mlp_bwd"] == 12 * 54 * 50 * 57101
    assert f["desc_radial"] == (15 + 4 * 13 + 2 * 9 * 13) * 2679524
    double = bench.work_model_flops(N=2 * 57101, PR=2 * 2679524, PA=2 * 474686)
    for k, v in f.items():
        assert v > 0 and double[k] == 2 * v, k
