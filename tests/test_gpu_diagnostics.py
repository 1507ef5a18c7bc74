"""FP64 conservation sums and the free-surface front on the GPU (through the
C ABI) against the oracle and the front's definition.

sph_diagnostics sums FP64 values of the widened FP32 state (mass, fluid
momentum, kinetic and potential energy, internal energy of the Tait law);
or_diagnostics sums the same quantities of the same downloaded state in
another order (sequentially).  The bars follow from FP64 rounding: a
recursive sum of n terms is within (n - 1) u of the sum of their
magnitudes (u = 2^-53; about 1.9e-12 at n = 17,472), the device's tree
sum within less, so the two agree within 2 n u of it; the internal
energy's two closed forms (the device expands (rho/rho0)^6, the oracle
calls pow) cancel to about 1e-3 of their terms near rho0, so they agree
within 1e-9 of the sum of the magnitudes.
The front (the largest x of fluid particles within 2 dp of the floor) is a
maximum of FP64 positions and must equal the host's maximum bit for bit.
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


def _scales(case, st):
    m = case.params()["mass"]
    fluid = st["ids"] >= case.n_bound
    v = st["vel"].astype(np.float64)[fluid]
    g = np.array(case.gravity)
    mom = m * np.abs(v).sum(0)
    kin = 0.5 * m * (v * v).sum()
    pot = m * np.abs(st["pos"][fluid] @ g).sum()
    return mom, kin, pot


def test_conservation_sums_match_the_oracle_on_a_moving_state():
    case = cases.c1_dam_break()
    sim = S.Simulation.from_case(case)
    sim.step(120)
    d = sim.diagnostics()
    st = sim.download()
    O = oracle.Oracle(case.params())
    ref = O.diagnostics(oracle.State(st["pos"], st["vel"], st["rho"], st["ids"]))
    m = case.params()["mass"]
    mom_s, kin_s, pot_s = _scales(case, st)
    assert kin_s > 0                         # the dam has started to move
    tol = 2 * case.n * 2.0 ** -53
    assert d["mass"] == pytest.approx(ref["mass"], rel=tol)
    assert d["mass"] == pytest.approx(m * case.n, rel=tol)
    for a in range(3):
        assert abs(d["momentum"][a] - ref["momentum"][a]) <= tol * mom_s[a] + 1e-300
    assert abs(d["kinetic"] - ref["kinetic"]) <= tol * kin_s
    assert abs(d["potential"] - ref["potential"]) <= tol * pot_s
    e_terms = m * np.abs([O.internal_energy(r) for r in st["rho"].astype(np.float64)]).sum()
    assert abs(d["internal"] - ref["internal"]) <= 1e-9 * e_terms
    print("internal energy: device", d["internal"], "oracle", ref["internal"])
    assert d["n_out"] == ref["n_out"] == 0
    sim.check()
    sim.close()


def _front_ref(st, n_bound, z_lo, z_hi):
    fluid = st["ids"] >= n_bound
    z = st["pos"][:, 2]
    sel = fluid & (z >= z_lo) & (z < z_hi)
    return st["pos"][sel, 0].max() if sel.any() else -np.inf


def test_front_equals_the_host_maximum_bit_for_bit():
    case = cases.c1_dam_break()
    sim = S.Simulation.from_case(case)
    band = (0.0, 2 * case.dp)                # the tank floor is at z = 0
    with pytest.raises(S.SphError, match="SPH_ERR_STATE"):
        sim.front(*band)                     # the cells are not built yet
    sim.build_cells()
    f0 = sim.front(*band)
    assert f0.shape == (1,)
    st = sim.download()
    assert f0[0] == _front_ref(st, case.n_bound, *band)
    assert f0[0] < 0.4                        # the block's face at t = 0
    sim.step(300)
    f1 = sim.front(*band)
    st = sim.download()
    assert f1[0] == _front_ref(st, case.n_bound, *band)
    assert f1[0] > f0[0]                      # the surge has moved along x
    # a band with no fluid particle, and invalid bands
    assert sim.front(10.0, 11.0)[0] == -np.inf
    for bad in ((1.0, 1.0), (1.0, 0.5), (np.nan, 1.0)):
        with pytest.raises(S.SphError, match="INVALID_ARG"):
            sim.front(*bad)
    sim.close()


def test_front_per_member_of_an_ensemble():
    members = [cases.ensemble_instance(s) for s in cases.ensemble_specs(3, seed=5)]
    ens = cases.ensemble(members)
    sim = S.Simulation.from_ensemble(ens)
    sim.step(150)
    band = (0.0, 2 * ens.params["dp"])
    got = sim.front(*band)
    st = sim.download()
    for q, c in enumerate(members):
        lo, hi = int(ens.id_base[q]), int(ens.id_base[q + 1])
        mine = (st["ids"] >= lo) & (st["ids"] < hi)
        sub = {k: v[mine] for k, v in st.items()}
        sub["ids"] = sub["ids"] - lo
        assert got[q] == _front_ref(sub, c.n_bound, *band)
    sim.close()
