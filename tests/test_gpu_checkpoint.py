"""Checkpoint and resume through the C ABI: a run resumed from a checkpoint
file (state, member times and step counts) repeats the uninterrupted run bit
for bit, for a single dam break and for an ensemble whose members stop at
their end time."""
import numpy as np
import pytest

import __graft_entry__  # noqa: F401
from paper_1210_1017_gb300 import cases
from paper_1210_1017_gb300 import sph as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()
    yield


def _same(a, b):
    for key in ("ids", "pos", "vel", "rho"):
        assert np.array_equal(a[key], b[key]), key


def test_resumed_dam_break_repeats_the_run(tmp_path):
    path = tmp_path / "c1.npz"
    case = cases.c1_dam_break()
    a = S.Simulation.from_case(case)
    a.step(10)
    saved = a.instance_state()
    a.save_checkpoint(path)
    a.step(15)
    want, want_i = a.download(), a.instance_state()
    a.close()
    b = S.Simulation.load_checkpoint(path)
    got0 = b.instance_state()
    assert got0["t"][0] == saved["t"][0] and got0["steps"][0] == 10
    b.step(15)
    _same(b.download(), want)
    got_i = b.instance_state()
    assert got_i["t"][0] == want_i["t"][0] and got_i["steps"][0] == 25
    b.close()


def test_resumed_ensemble_keeps_members_that_finished(tmp_path):
    path = tmp_path / "ens.npz"
    members = [cases.ensemble_instance(s) for s in cases.ensemble_specs(2, seed=5)]
    ens = cases.ensemble(members, t_end=3e-3)    # about 10 and 11 steps
    a = S.Simulation.from_ensemble(ens)
    for _ in range(60):
        a.step(1)
        if a.instance_state()["done"].any():
            break
    ia = a.instance_state()
    assert ia["done"].any() and not ia["done"].all()     # one finished, one runs
    a.save_checkpoint(path)
    a.step(6)
    want, want_i = a.download(), a.instance_state()
    a.close()
    b = S.Simulation.load_checkpoint(path)
    assert np.array_equal(b.instance_state()["done"], ia["done"])
    b.step(6)
    _same(b.download(), want)
    got_i = b.instance_state()
    assert np.array_equal(got_i["t"], want_i["t"]) and np.array_equal(got_i["steps"], want_i["steps"])
    assert np.array_equal(got_i["done"], want_i["done"])
    b.close()
