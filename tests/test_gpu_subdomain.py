"""Sub-domain selection of Sec. 4.2-4.3 on the GPU (labels, radix sort by
(label, id), copy of the labelled particles), through the C ABI, against the
oracle: counts, order and copied state bit for bit, including the worked
example of Sec. 4.3."""
import json
import os

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


def _check_against_oracle(case, sim, mode, xlo, xhi):
    got = sim.subdomain_select(mode, xlo, xhi)
    st = sim.download()
    O = oracle.Oracle(case.params())
    _, counts, sel = O.subdomain_select(st["pos"], st["ids"], mode, xlo, xhi)
    assert got["counts"].tolist() == counts.tolist()
    assert np.array_equal(got["ids"], st["ids"][sel])
    assert np.array_equal(got["pos"], st["pos"][sel])
    assert np.array_equal(got["vel"], st["vel"][sel])
    assert np.array_equal(got["rho"], st["rho"][sel])
    return got


def test_worked_example_of_the_paper(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "radix_sort_halo_example.json")))
    base = cases.random_block(64, seed=1)
    h = base.h
    xlo, xhi = 0.02, 0.02 + 5 * h
    xs = {0: 0.5 * (xlo + xhi), 1: xlo + 0.5 * h, 2: xhi - 0.5 * h}
    pos = np.array([[xs[v], 0.05 + 0.01 * k, 0.05] for k, v in enumerate(g["halo"])])
    n = pos.shape[0]
    case = cases.Case(name="example", pos=pos, vel=np.zeros((n, 3), np.float32),
                      rho=np.full(n, 1000.0, np.float32), ids=np.array(g["id"], np.uint32),
                      n_bound=0, dp=base.dp, h=h, rho0=1000.0, c0=20.0, alpha=0.01, cfl=0.2,
                      gravity=(0.0, 0.0, -9.81), dmin=(-0.1, -0.1, -0.1), dmax=(0.3, 0.3, 0.3),
                      fluid_height=0.0)
    sim = S.Simulation.from_case(case)
    sim.build_cells()
    got = sim.subdomain_select(S.SPH_SUBDOMAIN_EDGE, xlo, xhi)
    # the example's sorted ids are 1, 4, 6, 7 (label 0), then 2, 3, 5 (label
    # 1) and 8 (label 2): what the sub-domain sends is the labelled tail
    tail = [i for i, l in zip(g["sorted_id"], g["sorted_halo"]) if l != 0]
    assert got["ids"].tolist() == tail
    assert got["counts"].tolist() == [g["sorted_halo"].count(v) for v in range(3)]
    byid = {int(i): k for k, i in enumerate(g["id"])}
    assert np.array_equal(got["pos"], pos[[byid[i] for i in tail]])
    _check_against_oracle(case, sim, S.SPH_SUBDOMAIN_EDGE, xlo, xhi)
    sim.close()


@pytest.mark.parametrize("mode", [S.SPH_SUBDOMAIN_EDGE, S.SPH_SUBDOMAIN_MIGRATE])
def test_dam_break_slabs_match_the_oracle(mode):
    case = cases.c1_dam_break(shuffle_seed=5)
    sim = S.Simulation.from_case(case)
    sim.step(30)
    edges = np.linspace(0.0, 1.0, 5)           # four sub-domains along x
    total = 0
    for xlo, xhi in zip(edges[:-1], edges[1:]):
        got = _check_against_oracle(case, sim, mode, xlo, xhi)
        total += int(got["counts"][1] + got["counts"][2])
    assert total > 0
    sim.close()


def test_random_ids_and_large_selection():
    """Ids far above n (the sort by id runs over all 32 bits) and a
    selection of most particles (several sort tiles)."""
    case = cases.random_block(20000, seed=44, jitter=0.4)
    # an odd multiplier is a bijection modulo 2^32: distinct ids over 32 bits
    k = np.arange(case.n, dtype=np.uint64)
    case.ids = ((k * np.uint64(2654435761) + np.uint64(12345)) % (np.uint64(1) << np.uint64(32))
                ).astype(np.uint32)
    assert np.unique(case.ids).size == case.n and case.ids.max() > (1 << 31)
    case.n_bound = 0
    sim = S.Simulation.from_case(case)
    sim.build_cells()
    x = case.pos[:, 0]
    got = _check_against_oracle(case, sim, S.SPH_SUBDOMAIN_MIGRATE,
                                np.quantile(x, 0.45), np.quantile(x, 0.55))
    assert got["counts"][1] + got["counts"][2] > 15000
    sim.close()


def test_capacity_empty_selection_and_argument_checks():
    case = cases.random_block(3000, seed=12)
    sim = S.Simulation.from_case(case)
    sim.build_cells()
    x = case.pos[:, 0]
    xlo, xhi = x.min() + 0.01, x.max() - 0.01
    full = sim.subdomain_select(S.SPH_SUBDOMAIN_EDGE, xlo, xhi)
    m = int(full["counts"][1] + full["counts"][2])
    assert m > 0
    with pytest.raises(S.SphError, match="SPH_ERR_CAPACITY"):
        sim.subdomain_select(S.SPH_SUBDOMAIN_EDGE, xlo, xhi, capacity=m - 1)
    again = sim.subdomain_select(S.SPH_SUBDOMAIN_EDGE, xlo, xhi, capacity=m)
    assert np.array_equal(again["ids"], full["ids"])
    # a sub-domain holding everything: nothing migrates
    none = sim.subdomain_select(S.SPH_SUBDOMAIN_MIGRATE, x.min() - 1.0, x.max() + 1.0)
    assert none["counts"].tolist() == [case.n, 0, 0] and none["ids"].size == 0
    with pytest.raises(S.SphError, match="SPH_ERR_INVALID_ARG"):
        sim.subdomain_select(S.SPH_SUBDOMAIN_EDGE, 0.1, 0.1 + 3 * case.h)   # < 4h
    with pytest.raises(S.SphError, match="SPH_ERR_INVALID_ARG"):
        sim.subdomain_select(7, xlo, xhi)
    # after an integrator update the cells are stale until the next rebuild
    sim.interact()
    sim.predict()
    with pytest.raises(S.SphError, match="SPH_ERR_STATE"):
        sim.subdomain_select(S.SPH_SUBDOMAIN_EDGE, xlo, xhi)
    sim.check()
    sim.close()


def test_labels_at_exactly_2h_and_signed_zero():
    """Dyadic h = 1/4: every threshold is exact, so the strict and non-strict
    bounds decide; -0.0 and +0.0 are the same x."""
    h = 0.25
    xlo, xhi = 0.0, 2.0
    xs = [xlo - 2.0 ** -30, -0.0, xlo, xlo + 2 * h - 2.0 ** -40, xlo + 2 * h, 1.0,
          xhi - 2 * h - 2.0 ** -40, xhi - 2 * h, xhi - 2.0 ** -40, xhi]
    n = len(xs)
    pos = np.array([[v, 0.1 * k - 0.45, 0.0] for k, v in enumerate(xs)])
    case = cases.Case(name="thresholds", pos=pos, vel=np.zeros((n, 3), np.float32),
                      rho=np.full(n, 1000.0, np.float32), ids=np.arange(n, dtype=np.uint32),
                      n_bound=0, dp=0.2, h=h, rho0=1000.0, c0=20.0, alpha=0.01, cfl=0.2,
                      gravity=(0.0, 0.0, -9.81), dmin=(-1.0, -1.0, -1.0), dmax=(3.0, 1.0, 1.0),
                      fluid_height=0.0)
    sim = S.Simulation.from_case(case)
    sim.build_cells()
    edge = _check_against_oracle(case, sim, S.SPH_SUBDOMAIN_EDGE, xlo, xhi)
    assert sorted(edge["ids"].tolist()) == [1, 2, 3, 7, 8]
    mig = _check_against_oracle(case, sim, S.SPH_SUBDOMAIN_MIGRATE, xlo, xhi)
    assert mig["ids"].tolist() == [0, 9]
    sim.close()
