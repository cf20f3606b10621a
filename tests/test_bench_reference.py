"""The oracle arm of bench.py (--impl reference) runs on the host CPU alone: its JSON line carries
the keys the benchmark contract asks for, describes its own CPU run, and prints nothing on a
rank other than 0.  CPU only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(extra_env=None, *args):
    env = dict(os.environ, **(extra_env or {}))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "2", "--warmup", "3", "--cpu-sample", "20", *args],
                       capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    return [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]


def test_reference_line_has_the_contract_keys():
    (line,) = run()
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 3
    assert line["value"] > 0 and line["higher_is_better"] is True
    cpu = line["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["value"] == line["value"]
    assert isinstance(cpu["cores"], int) and 1 <= cpu["cores"] <= (os.cpu_count() or 1) + 8
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == "transmon_cavity_d40" and line["config"]["sample_slices"] == 20
    assert "flushed" not in line["config"]["l2"]


def test_reference_line_only_on_rank_zero():
    assert run({"RANK": "1", "WORLD_SIZE": "2"}) == []
