"""The benchmark's host-side contract on the CPU: the reference arm (the CPU oracle) prints
one JSON line with the keys the driver reads, ranks other than 0 print nothing, and the
workload text follows the options."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(args, env_extra=None, timeout=300):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=timeout)


def test_reference_arm_prints_one_json_line():
    p = run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["unit"] == "cell-updates/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["steps"] == 1 and d["warmup"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] == 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["sample_cells"] == 6 * 12 ** 3 and d["dtype"] == "f64"


def test_reference_arm_other_ranks_print_nothing():
    p = run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0"],
                  {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""


def test_workload_text_follows_the_options():
    sys.path.insert(0, ROOT)
    import bench

    class A:
        inner, prec = 0, "fp64"
    plain = bench.workload_text(A)
    assert plain == bench.WORKLOAD and "FP64 plain method" in plain
    A.prec = "mixed"
    mixed = bench.workload_text(A)
    assert "mixed precision" in mixed and "FP32 inner CG" in mixed and "FP64 plain" not in mixed
    A.inner = 2
    mg = bench.workload_text(A)
    assert "2 multigrid V-cycles per outer step" in mg and "inner CG" not in mg


@pytest.mark.parametrize("opt", ["--prec", "--inner", "--transport-only"])
def test_bench_options_are_declared(opt):
    p = run_bench(["--help"], timeout=60)
    assert p.returncode == 0 and opt in p.stdout
