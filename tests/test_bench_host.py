"""Host-side helpers of bench.py on CPU: the formulation switch applied to a
single case and to an ensemble, and the reference arm's JSON line on the
6,000-fluid-particle dam break (the oracle on this machine's cores)."""
import json
import os
import subprocess
import sys

import __graft_entry__  # noqa: F401
import bench
from paper_1210_1017_gb300 import cases

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_formulation_switch():
    c = bench.with_formulation(cases.c1_dam_break(), "paper")
    assert (c.kernel, c.integrator) == ("cubic", "verlet")
    assert c.params()["kernel"] == "cubic"
    d = bench.with_formulation(cases.c1_dam_break(), "default")
    assert (d.kernel, d.integrator) == ("wendland", "symplectic")
    e = bench.with_formulation(cases.dam_break_ensemble(3, t_end=1.0), "paper")
    assert e.params["integrator"] == "verlet"
    assert all(m.kernel == "cubic" for m in e.cases)
    assert bench.formulation_config("paper")["integrator"].startswith("Verlet")


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "dam_break_6k", "--formulation", "paper", "--steps", "1",
                          "--warmup", "3"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "pairs/s"
    assert d["config"]["formulation"] == "paper" and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
