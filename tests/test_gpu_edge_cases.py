"""Degenerate inputs through the C ABI against the FP64 oracle: a single
particle, particles sitting exactly on cell faces and corners with pairs at
exactly the support radius 2h, a state of boundary particles only, and
particles whose whole neighbourhood is empty."""
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


def _case(pos, n_bound, dp, h, vel=None, below=0.0):
    """A case around given positions (dyadic values make every label and
    distance exact); `below` extends the domain downwards."""
    pos = np.asarray(pos, np.float64)
    n = pos.shape[0]
    cs = 2 * h
    dmin = tuple(float(v) for v in pos.min(0) - cs - np.array([0.0, 0.0, below]))
    dmax = tuple(float(v) for v in pos.max(0) + 2 * cs)
    vel = np.zeros((n, 3), np.float32) if vel is None else np.asarray(vel, np.float32)
    return cases.Case(name="edge", pos=pos, vel=vel, rho=np.full(n, 1000.0, np.float32),
                      ids=np.arange(n, dtype=np.uint32), n_bound=n_bound, dp=dp, h=h,
                      rho0=1000.0, c0=20.0, alpha=0.01, cfl=0.2, gravity=(0.0, 0.0, -9.81),
                      dmin=dmin, dmax=dmax, fluid_height=float(pos[:, 2].max()))


def _run(case, steps=0):
    sim = S.Simulation.from_case(case)
    sim.build_cells()
    sim.interact(counts=True)
    out = dict(ace=sim.read(S.SPH_ARRAY_ACE), nnb=sim.read(S.SPH_ARRAY_NNB),
               nnb64=sim.neighbour_counts_fp64(), keys=sim.read(S.SPH_ARRAY_KEY),
               off=sim.read(S.SPH_ARRAY_CELL_OFF), st=sim.download())
    if steps:
        sim.step(steps)
        out["after"] = sim.download()
        out["diag"] = sim.diagnostics()
    sim.check()
    sim.close()
    return out


def test_single_particle_falls_freely():
    case = _case([[0.5, 0.5, 2.0]], 0, 0.02, 0.026, below=2.0)
    r = _run(case, steps=200)
    assert r["nnb"][0] == 0 and r["nnb64"][0] == 0
    assert np.array_equal(r["ace"][0], np.float32([0.0, 0.0, -9.81, 0.0]))
    # symplectic midpoint under constant gravity: z = z0 - g t^2 / 2, up to
    # the FP32 rounding of the velocity (FP64 positions)
    t = r["diag"]["t"]
    assert r["diag"]["n_out"] == 0 and t > 0.04
    z = r["after"]["pos"][0, 2]
    assert abs(z - (2.0 - 0.5 * 9.81 * t * t)) < 1e-6
    assert r["after"]["pos"][0, 0] == 0.5 and r["after"]["pos"][0, 1] == 0.5


def test_lattice_on_cell_faces_and_exact_support_distance():
    """h = dp = 1/4: cells of 1/2, every lattice point on a cell face, edge or
    corner, and lattice neighbours two apart at exactly 2h (not neighbours)."""
    dp = 0.25
    g = np.stack(np.meshgrid(np.arange(6), np.arange(5), np.arange(4), indexing="ij"), -1)
    pos = 1.0 + dp * g.reshape(-1, 3).astype(np.float64)
    rng = np.random.default_rng(0)
    perm = rng.permutation(pos.shape[0])
    case = _case(pos[perm], 0, dp, dp, vel=rng.uniform(-0.1, 0.1, (pos.shape[0], 3)))
    case.ids = np.arange(pos.shape[0], dtype=np.uint32)
    r = _run(case)
    O = oracle.Oracle(case.params())
    ref = O.build_cells(case.pos, case.ids)
    assert np.array_equal(r["st"]["ids"], ref["sorted_ids"])
    assert np.array_equal(r["keys"], ref["sorted_key"])
    assert np.array_equal(r["off"], ref["cell_off"])
    # neighbours: lattice points at dp, sqrt(2) dp, sqrt(3) dp (< 2h = 2 dp);
    # the points exactly 2 dp away are not neighbours
    c64 = O.neighbour_counts(r["st"]["pos"], brute=True)
    assert np.array_equal(r["nnb64"], c64)
    assert np.array_equal(r["nnb"], c64)        # exact distances: FP32 agrees too
    d = np.sqrt(((r["st"]["pos"][:, None] - r["st"]["pos"][None]) ** 2).sum(-1))
    assert np.array_equal(c64, ((d > 0) & (d < 2 * dp)).sum(1))
    st = oracle.State(r["st"]["pos"], r["st"]["vel"], r["st"]["rho"], r["st"]["ids"])
    o = O.interact(st, brute=True)
    ea = np.linalg.norm(r["ace"][:, :3] - o["a"], axis=1) / np.maximum(o["sa"], 1e-300)
    ed = np.abs(r["ace"][:, 3] - o["drho"]) / np.where(o["sd"] > 0, o["sd"], 1.0)
    assert ea.max() <= 2e-5 and ed.max() <= 2e-5


def test_boundary_particles_only():
    c = cases.random_block(500, seed=3, bound_layers=100)      # every layer boundary
    assert c.n_bound == c.n
    r = _run(c, steps=3)
    g = np.float32(c.gravity)
    assert np.array_equal(r["ace"][:, :3], np.tile(g, (c.n, 1)))
    # boundary-boundary terms vanish (v_ij = 0): no density rates
    assert np.all(r["ace"][:, 3] == 0)
    o = np.argsort(r["st"]["ids"])
    oa = np.argsort(r["after"]["ids"])
    assert np.array_equal(r["after"]["pos"][oa], r["st"]["pos"][o])


def test_isolated_particles_have_no_neighbours():
    """Particles three cells apart: every 27-cell neighbourhood holds only the
    particle itself."""
    h = 0.25
    pos = np.array([[0.0, 0.0, 0.0], [1.6, 0.0, 0.0], [0.0, 1.6, 0.0], [0.0, 0.0, 1.6]]) + 2.0
    case = _case(pos, 1, h, h)
    r = _run(case)
    assert np.all(r["nnb"] == 0) and np.all(r["nnb64"] == 0)
    assert np.all(r["ace"][:, 3] == 0)
    assert np.array_equal(r["ace"][:, :3], np.tile(np.float32([0, 0, -9.81]), (4, 1)))
