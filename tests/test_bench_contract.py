"""bench.py's reference arm (the CPU oracle on the host cores) keeps the JSON contract
of a bench line: one line from rank 0, the workload's metric and config, a
cpu_baseline describing the run and an e2e block with the line's own value; other
ranks exit 0 without work.  The GPU arm is exercised on a GB300 only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CMD = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "0",
       "--ref-pairs", "1e5"]


def _run(env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    return subprocess.run(CMD, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    sys.path.insert(0, ROOT)
    import bench
    p = _run({})
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "queries/s"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    # ms_per_step is the measured sample step; value is 1 / the estimated full query, which
    # adds the unsampled walk pairs' time
    assert 0 < d["ms_per_step"] <= 1000.0 / d["value"] * (1 + 1e-9)
    assert d["config"]["workload"] == "cl100k"
    assert d["config"]["n"] == 100_000 and d["config"]["m"] == 1_000_000 and d["config"]["eps"] == 1e-6
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    chk = cb["scaling_check"]  # a whole unsampled oracle query against its estimate from a tenth
    assert chk["pairs"] > 0 and chk["measured_full_s"] > 0 and chk["ratio"] > 0
    assert d["e2e"] == {"value": d["value"], "unit": "queries/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_without_work():
    p = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""
