"""bench.py's JSON line keeps the keys its consumers read: the reference arm
(the FP64 oracle on the host, runnable without a GPU) and, on a GPU, the
native arm with its roofline, clocks, end-to-end leg and CPU baseline."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
COMMON = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
          "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"}


def _run(*args, timeout=600):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                         capture_output=True, text=True, timeout=timeout)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def test_reference_arm_line(orc):
    d = _run("--impl", "reference", "--envs", "300", "--steps", "3", "--warmup", "1")
    assert COMMON <= set(d)
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


@pytest.mark.gpu
def test_native_arm_line(vmas_lib):
    d = _run("--envs", "2000", "--steps", "5", "--warmup", "3", "--cpu-budget", "1")
    assert COMMON <= set(d)
    assert d["n_gpus"] == 1 and d["steps"] == 5 and d["value"] > 0
    r = d["roofline"]
    assert {"bound", "achieved", "peak", "unit", "frac", "traffic"} <= set(r)
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-9
    assert {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"} <= set(d["e2e"])
    assert d["e2e"]["h2d_bytes_per_step"] > 0 and d["e2e"]["d2h_bytes_per_step"] > 0
    assert d["gpu_launches"] == 5
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= set(d["clocks"])
    assert {"value", "unit", "cores", "kind", "sample"} <= set(d["cpu_baseline"])


def _bench_module():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench

    return bench


def test_kernel_digest_ignores_comments_and_layout():
    b = _bench_module()
    code = "int f(int x) {\n  return x + 1;  // one more\n}\n"
    same = "/* header */\nint f(int x) { return x + 1; }\n"
    other = "int f(int x) { return x + 2; }\n"
    assert b._code_text(code) == b._code_text(same)
    assert b._code_text(code) != b._code_text(other)


def test_step_kernel_profile_matches_the_code():
    """The committed ncu summary of the step kernel was taken on the current
    kernel code, so the bench reports its DRAM traffic (a changed kernel needs
    a new capture)."""
    traffic, figures = _bench_module()._recorded_profile()
    assert traffic is not None and traffic > 0
    assert figures["issue_active_pct"] > 0 and figures["warps_per_sm"] > 0
