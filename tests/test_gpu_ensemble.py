"""Batched ensemble (many independent dam breaks in one lockstep run) against
the same cases run alone, and against the FP64 oracle.

Batching changes neither the arithmetic of a member nor its neighbour order
(labels are offset per member, ids per member), so every member of an
ensemble must reproduce its stand-alone run bit for bit, with its own step
size, and stop at its own end time.
"""
import numpy as np
import pytest

import __graft_entry__  # noqa: F401
import oracle
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


def _members(n=3, seed=99):
    return [cases.ensemble_instance(s) for s in cases.ensemble_specs(n, seed=seed)]


def _by_id(st):
    k = np.argsort(st["ids"])
    return {key: st[key][k] for key in ("pos", "vel", "rho", "ids")}


def test_members_reproduce_their_standalone_runs_bit_for_bit():
    members = _members(3)
    ens = cases.ensemble(members)
    sim = S.Simulation.from_ensemble(ens)
    sim.step(20)
    st = _by_id(sim.download())
    ist = sim.instance_state()
    sim.close()
    assert np.all(ist["steps"] == 20)
    for q, case in enumerate(members):
        alone = S.Simulation.from_case(case)
        alone.step(20)
        a = _by_id(alone.download())
        d = alone.diagnostics()
        alone.close()
        sl = ens.member_slice(q)
        assert np.array_equal(st["pos"][sl], a["pos"])
        assert np.array_equal(st["vel"][sl], a["vel"])
        assert np.array_equal(st["rho"][sl], a["rho"])
        assert ist["t"][q] == d["t"]
    # members with different c0 take different steps
    assert len(set(np.round(ist["dt"], 12))) > 1


def test_members_stop_at_their_end_time_and_stay_frozen():
    members = _members(2, seed=5)
    ens = cases.ensemble(members, t_end=2e-3)
    sim = S.Simulation.from_ensemble(ens)
    for _ in range(40):
        sim.step(1)
        if sim.instance_state()["done"].all():
            break
    ist = sim.instance_state()
    assert ist["done"].all()
    assert np.all(ist["t"] >= 2e-3)
    a = sim.download()
    sim.step(3)
    b = sim.download()
    ist2 = sim.instance_state()
    assert np.array_equal(ist2["t"], ist["t"]) and np.array_equal(ist2["steps"], ist["steps"])
    assert np.array_equal(a["pos"], b["pos"]) and np.array_equal(a["rho"], b["rho"])
    sim.close()


def test_member_rates_match_the_oracle():
    members = _members(3, seed=7)
    ens = cases.ensemble(members)
    sim = S.Simulation.from_ensemble(ens)
    sim.step(5)
    sim.interact()
    ace = sim.read(S.SPH_ARRAY_ACE)
    st = sim.download()
    sim.close()
    for q in (0, 2):
        lo, hi = ens.id_base[q], ens.id_base[q + 1]
        sel = (st["ids"] >= lo) & (st["ids"] < hi)
        case = members[q]
        ost = oracle.State(st["pos"][sel], st["vel"][sel], st["rho"][sel],
                           (st["ids"][sel] - lo).astype(np.uint32))
        ref = oracle.Oracle(case.params()).interact(ost)
        fluid = ost.ids >= case.n_bound
        a = ace[sel]
        ea = np.linalg.norm(a[fluid, :3] - ref["a"][fluid], axis=1) / ref["sa"][fluid]
        ed = np.abs(a[:, 3] - ref["drho"]) / np.where(ref["sd"] > 0, ref["sd"], 1.0)
        print(f"member {q}: n={case.n} accel {ea.max():.2e} drho {ed.max():.2e}")
        assert ea.max() <= 2e-5 and ed.max() <= 2e-5


def test_device_step_loop_stops_once_every_member_is_done():
    """One sph_step call with far more steps than needed: the device loop
    ends as soon as every member has reached its end time, each member with
    the same step count as when stepping one step per call."""
    members = _members(2, seed=5)
    ens = cases.ensemble(members, t_end=2e-3)
    ref = S.Simulation.from_ensemble(ens)
    lock = 0
    while not ref.instance_state()["done"].all():
        ref.step(1)
        lock += 1
        assert lock < 100
    want = ref.instance_state()
    a = ref.download()
    pairs_ref = ref.diagnostics()["pairs_total"]
    ref.close()
    sim = S.Simulation.from_ensemble(ens)
    d0 = sim.diagnostics()
    sim.step(100000)
    got = sim.instance_state()
    d1 = sim.diagnostics()
    assert got["done"].all()
    assert np.array_equal(got["steps"], want["steps"]) and np.array_equal(got["t"], want["t"])
    b = sim.download()
    for key in ("ids", "pos", "vel", "rho"):
        assert np.array_equal(a[key], b[key])
    # only the lockstep steps up to the last member's end were evaluated
    assert d1["pairs_total"] - d0["pairs_total"] == pairs_ref
    sim.close()
