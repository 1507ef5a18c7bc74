"""A short logged run through sph_rollout: one JSONL line per save boundary,
steps and time increasing, mass conserved to rounding, no status bits."""
import json

import pytest

import __graft_entry__  # noqa: F401
from paper_1210_1017_gb300 import cases, runlog
from paper_1210_1017_gb300 import sph as S

pytestmark = pytest.mark.gpu


def test_logged_run(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    case = cases.c1_dam_break()
    sim = S.Simulation.from_case(case)
    path = tmp_path / "run.jsonl"
    recs = runlog.run(sim, 60, 20, str(path), front_band=(0.0, 2 * case.dp))
    lines = [json.loads(x) for x in open(path)]
    assert lines == recs and len(lines) == 4
    assert [r["step"] for r in lines] == [0, 20, 40, 60]
    assert all(b["t"] > a["t"] for a, b in zip(lines, lines[1:]))
    assert all(abs(r["mass_drift"]) < 1e-12 and r["status"] == 0 for r in lines)
    assert all(r["steps_per_s"] > 0 and r["pairs_per_s"] > 0 for r in lines[1:])
    assert len(lines[-1]["front"]) == 1 and lines[-1]["front"][0] > 0.0
    sim.close()
