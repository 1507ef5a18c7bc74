"""The run log's line builder (host logic, no GPU): drifts against the first
record, rates against the previous one."""
import json

import pytest

import __graft_entry__  # noqa: F401
from paper_1210_1017_gb300 import runlog


def _diag(step, t, mass, kin, pot, inn, pairs, n_out=0):
    return dict(step=step, t=t, dt=1e-4, mass=mass, momentum=[0.0, 0.0, 0.0], kinetic=kin,
                potential=pot, internal=inn, pairs_total=pairs, n_out=n_out, status=0,
                amax=1.0, cmax=2.0, mumax=0.5)


def test_drift_and_rates():
    first = _diag(0, 0.0, 10.0, 1.0, -5.0, 2.0, 0)
    r0 = runlog.record(first, first, None, 0.0, None)
    assert r0["mass_drift"] == 0.0 and r0["energy_drift"] == 0.0 and "steps_per_s" not in r0
    later = _diag(100, 0.01, 10.0, 1.5, -5.0, 2.0, 4_000_000)
    r1 = runlog.record(later, first, first, 2.0, 0.0, front=[0.4, 0.5])
    assert r1["energy"] == pytest.approx(-1.5)
    assert r1["energy_drift"] == pytest.approx(0.5 / 2.0)      # (E - E0) / |E0|, E0 = -2
    assert r1["steps_per_s"] == pytest.approx(50.0)
    assert r1["pairs_per_s"] == pytest.approx(2e6)
    assert r1["sim_s_per_wall_s"] == pytest.approx(0.005)
    assert r1["front"] == [0.4, 0.5]
    json.dumps(r1)   # every field is JSON-serialisable
