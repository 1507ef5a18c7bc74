"""Programmatic dependent launch changes scheduling only: a run with it and a
run without it (SPH_PDL=0, decided once per process, so the second run is a
child process) give the same state bit for bit."""
import os
import subprocess
import sys

import numpy as np
import pytest

import __graft_entry__
from paper_1210_1017_gb300 import cases
from paper_1210_1017_gb300 import sph as S

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
import numpy as np
sys.path.insert(0, sys.argv[2])
from paper_1210_1017_gb300 import cases
from paper_1210_1017_gb300 import sph as S
sim = S.Simulation.from_case(cases.c1_dam_break())
sim.step(60)
sim.check()
st = sim.download()
np.savez(sys.argv[1], pdl=np.array(S.pdl_enabled()), **st)
"""


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()
    yield


def test_state_is_the_same_with_and_without_programmatic_launch(tmp_path):
    sim = S.Simulation.from_case(cases.c1_dam_break())
    sim.step(60)                                  # one device-side loop launch
    sim.check()
    mine = sim.download()
    on = S.pdl_enabled()
    print("programmatic dependent launch in this process:", on)
    out = tmp_path / "off.npz"
    env = dict(os.environ, SPH_PDL="0")
    r = subprocess.run([sys.executable, "-c", CHILD, str(out), ROOT], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    other = np.load(out)
    assert not bool(other["pdl"])                 # the child ran without it
    for k, v in mine.items():
        assert np.array_equal(v, other[k]), k
    sim.close()
