"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these tests compares the oracle with itself: each one checks it
against a value printed in the paper, a library routine, a closed form, a
conservation law of the discrete equations, a symmetry, brute force, or a
convergence order.  A dropped term, a wrong sign or index, or a transposed
operand in the oracle fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_1210_1017_gb300 import cases


def _oracle(case, **over):
    p = case.params()
    p.update(over)
    return oracle.Oracle(p)


def _lattice_case(nx, ny, nz, dp=0.02, rho=1000.0, c0=20.0, alpha=0.0,
                  n_bound=0, jitter=0.0, seed=3):
    ii, jj, kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz),
                             indexing="ij")
    pos = np.stack([(ii.ravel() + 0.5) * dp, (jj.ravel() + 0.5) * dp,
                    (kk.ravel() + 0.5) * dp], axis=1)
    if jitter:
        pos += np.random.default_rng(seed).uniform(-jitter, jitter, pos.shape) * dp
    n = pos.shape[0]
    h = 1.3 * dp
    dmin, dmax = cases.domain_for(pos, h, float(pos[:, 2].max()), nz * dp)
    return cases.Case(name="lattice", pos=pos,
                      vel=np.zeros((n, 3), np.float32),
                      rho=np.full(n, rho, np.float32),
                      ids=np.arange(n, dtype=np.uint32), n_bound=n_bound,
                      dp=dp, h=h, rho0=1000.0, c0=c0, alpha=alpha, cfl=0.2,
                      gravity=(0.0, 0.0, -9.81), dmin=dmin, dmax=dmax,
                      fluid_height=nz * dp)


def _interior(pos, margin):
    lo = pos.min(axis=0) + margin
    hi = pos.max(axis=0) - margin
    return np.all((pos >= lo) & (pos <= hi), axis=1)


# --- Sec. 4.3 worked example and the sort -----------------------------------

def test_sort_reproduces_paper_worked_example(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "radix_sort_halo_example.json")))
    c = cases.random_block(8)
    O = _oracle(c)
    key = np.array(g["halo"], np.uint32)
    ids = np.array(g["id"], np.uint32)
    perm = O.sort_by_key_id(key, ids)
    assert key[perm].tolist() == g["sorted_halo"]
    assert ids[perm].tolist() == g["sorted_id"]


def test_sort_matches_numpy_lexsort():
    rng = np.random.default_rng(11)
    O = _oracle(cases.random_block(8))
    for n in (0, 1, 5, 1000, 50000):
        key = rng.integers(0, 300, n).astype(np.uint32)
        ids = rng.permutation(n).astype(np.uint32)
        perm = O.sort_by_key_id(key, ids)
        ref = np.lexsort((ids, key))
        assert np.array_equal(perm, ref)


def test_cell_offsets_are_lower_bounds():
    rng = np.random.default_rng(5)
    c = cases.random_block(200)
    O = _oracle(c)
    ncells = O.ncells
    skey = np.sort(rng.integers(0, ncells + 1, 3000).astype(np.uint32))
    off = O.cell_offsets(skey)
    ref = np.searchsorted(skey, np.arange(ncells + 2), side="left")
    assert np.array_equal(off, ref.astype(np.uint32))


# --- cell keys ---------------------------------------------------------------

def test_cell_keys_on_known_points():
    c = cases.random_block(100)
    O = _oracle(c)
    ncx, ncy, ncz = O.grid_dims()
    cs = 2.0 * c.h
    x0, y0, z0 = c.dmin
    pts, want = [], []
    for (ix, iy, iz) in [(0, 0, 0), (1, 2, 3), (ncx - 1, ncy - 1, ncz - 1),
                         (ncx // 2, 0, ncz - 1)]:
        pts.append((x0 + (ix + 0.5) * cs, y0 + (iy + 0.5) * cs, z0 + (iz + 0.5) * cs))
        want.append(ix + ncx * (iy + ncy * iz))
    # exactly on the domain's lower corner belongs to cell 0
    pts.append((x0, y0, z0))
    want.append(0)
    # labels follow floor((x - x0) * (1/(2h))) with 1/(2h) rounded once
    inv_cs = 1.0 / cs
    for f in (1.0, 2.0):
        x = x0 + f * cs
        pts.append((x, y0 + 0.5 * cs, z0 + 0.5 * cs))
        want.append(int(math.floor((x - x0) * inv_cs)))
    ncells = ncx * ncy * ncz
    for bad in [(x0 - 1e-9, y0 + cs, z0 + cs), (x0 + cs, y0 + cs, z0 + ncz * cs + 1e-6),
                (np.nan, y0, z0), (np.inf, y0, z0)]:
        pts.append(bad)
        want.append(ncells)
    key, nout = O.cell_keys(np.array(pts))
    assert key.tolist() == want
    assert nout == 4


def test_neighbours_lie_in_adjacent_cells():
    c = cases.random_block(1500, seed=21, jitter=0.45)
    O = _oracle(c)
    ncx, ncy, _ = O.grid_dims()
    key, _ = O.cell_keys(c.pos)
    cx = key % ncx
    cy = (key // ncx) % ncy
    cz = key // (ncx * ncy)
    d = c.pos[:, None, :] - c.pos[None, :, :]
    near = (d ** 2).sum(-1) < (2 * c.h) ** 2
    i, j = np.nonzero(near)
    assert np.all(np.abs(cx[i].astype(int) - cx[j].astype(int)) <= 1)
    assert np.all(np.abs(cy[i].astype(int) - cy[j].astype(int)) <= 1)
    assert np.all(np.abs(cz[i].astype(int) - cz[j].astype(int)) <= 1)


# --- neighbour search: grid == brute force ----------------------------------

@pytest.mark.parametrize("n,jitter,seed", [(64, 0.0, 1), (500, 0.25, 7),
                                           (2000, 0.45, 9)])
def test_grid_neighbours_equal_brute_force(n, jitter, seed):
    c = cases.random_block(n, seed=seed, jitter=jitter)
    O = _oracle(c)
    a = O.neighbour_counts(c.pos, brute=False)
    b = O.neighbour_counts(c.pos, brute=True)
    assert np.array_equal(a, b)
    # and brute force itself against numpy's all-pairs distances
    d2 = ((c.pos[:, None, :] - c.pos[None, :, :]) ** 2).sum(-1)
    ref = (d2 < (2 * c.h) ** 2).sum(1) - 1
    assert np.array_equal(b, ref.astype(np.uint32))


def test_grid_neighbours_on_cell_faces_and_corners():
    c = cases.random_block(300, seed=4)
    O = _oracle(c)
    cs = 2 * c.h
    x0 = np.array(c.dmin)
    rng = np.random.default_rng(2)
    base = rng.integers(1, 4, size=(400, 3)) * cs + x0
    # points exactly on cell corners, faces and 2h apart along an axis
    offs = rng.choice([0.0, 0.5 * cs, cs, 0.999999 * cs], size=(400, 3))
    pos = np.concatenate([base + offs, base + offs + [cs, 0, 0]])
    a = O.neighbour_counts(pos, brute=False)
    b = O.neighbour_counts(pos, brute=True)
    assert np.array_equal(a, b)


# --- kernel ------------------------------------------------------------------

def test_kernel_integrates_to_one_and_has_compact_support():
    c = cases.c1_dam_break()
    O = _oracle(c)
    h = c.h
    val, err = integrate.quad(lambda r: 4 * math.pi * r * r * O.w(r), 0.0, 2 * h,
                              epsabs=1e-14, epsrel=1e-13, limit=200)
    assert abs(val - 1.0) < 1e-12
    assert O.w(2 * h) == 0.0 and O.f(2 * h) == 0.0
    rs = np.linspace(0, 2 * h, 200)
    w = np.array([O.w(r) for r in rs])
    assert np.all(np.diff(w) <= 0) and np.all(w >= 0)


def test_kernel_gradient_is_derivative_of_kernel():
    c = cases.c1_dam_break()
    O = _oracle(c)
    h = c.h
    for q in np.linspace(0.05, 1.95, 39):
        r = q * h
        e = 1e-6 * h
        dw = (O.w(r + e) - O.w(r - e)) / (2 * e)
        assert O.f(r) == pytest.approx(dw / r, rel=1e-7, abs=1e-9 * abs(O.f(0.5 * h)))


def test_lattice_kernel_sum_close_to_one():
    """Particle approximation of f = 1 on a regular interior lattice (report:
    discretisation error at h = 1.3 dp)."""
    c = _lattice_case(9, 9, 9)
    O = _oracle(c)
    centre = c.pos[np.argmin(((c.pos - c.pos.mean(0)) ** 2).sum(1))]
    r = np.sqrt(((c.pos - centre) ** 2).sum(1))
    s = sum(O.w(v) for v in r) * c.dp ** 3
    assert abs(s - 1.0) < 2e-2   # about 0.95% at h = 1.3 dp


# --- equation of state -------------------------------------------------------

def test_tait_closed_form_properties():
    c = cases.c1_dam_break()
    O = _oracle(c)
    r0, c0 = c.rho0, c.c0
    assert O.pressure(r0) == 0.0
    assert O.sound_speed(r0) == pytest.approx(c0, rel=1e-15)
    for rho in (980.0, 1000.0, 1003.0, 1050.0):
        e = 1e-4
        dpdrho = (O.pressure(rho + e) - O.pressure(rho - e)) / (2 * e)
        assert O.sound_speed(rho) ** 2 == pytest.approx(dpdrho, rel=1e-7)
    # gamma = 7: doubling (rho/rho0 - 1) small -> p ~ c0^2 (rho - rho0)
    assert O.pressure(r0 * (1 + 1e-7)) == pytest.approx(c0 ** 2 * r0 * 1e-7, rel=1e-5)


def test_internal_energy_derivative_is_p_over_rho2():
    c = cases.c1_dam_break()
    O = _oracle(c)
    assert O.internal_energy(c.rho0) == 0.0
    for rho in (990.0, 1010.0, 1100.0):
        e = 1e-3
        de = (O.internal_energy(rho + e) - O.internal_energy(rho - e)) / (2 * e)
        assert de == pytest.approx(O.pressure(rho) / rho ** 2, rel=1e-6)


def test_hydrostatic_initial_density_inverts_the_eos():
    c = cases.c1_dam_break()
    O = _oracle(c)
    for z in (0.01, 0.15, 0.29):
        rho = cases.hydrostatic_density(z, c.fluid_height, c.rho0, c.c0)
        assert O.pressure(float(rho)) == pytest.approx(
            c.rho0 * 9.81 * (c.fluid_height - z), rel=1e-10)


# --- pair sums: conservation laws of Eqs. 7 and 9 ----------------------------

def _random_state(n=800, seed=13, alpha=0.05):
    c = cases.random_block(n, seed=seed, jitter=0.3, vel_range=1.0,
                           rho_range=(0.995, 1.02), alpha=alpha)
    return c, _oracle(c), oracle.State.from_case(c)


def test_linear_and_angular_momentum_of_internal_forces_vanish():
    c, O, st = _random_state()
    r = O.interact(st, brute=True)
    m = c.mass
    g = np.array(c.gravity)
    fint = m * (r["a"] - g)
    scale = m * r["sa"].sum()
    assert np.abs(fint.sum(0)).max() < 1e-13 * scale
    torque = np.cross(c.pos, fint).sum(0)
    assert np.abs(torque).max() < 1e-13 * scale * np.abs(c.pos).max()


@pytest.mark.parametrize("alpha", [0.0, 0.05])
def test_energy_rate_of_inviscid_equations_is_zero(alpha):
    """With P = p/rho^2 and the symmetric pair form, the semi-discrete
    equations conserve E = sum m (v^2/2 - g.r + e(rho)) exactly when
    alpha = 0, and the viscosity can only dissipate."""
    c, O, st = _random_state(alpha=alpha)
    r = O.interact(st, brute=True)
    m = c.mass
    g = np.array(c.gravity)
    v = st.vel()
    p_over_rho2 = np.array([O.pressure(x) / x ** 2 for x in st.rho])
    kin = m * np.einsum("ij,ij->i", v, r["a"] - g)
    intl = m * p_over_rho2 * r["drho"]
    dEdt = kin.sum() + intl.sum()
    scale = np.abs(kin).sum() + np.abs(intl).sum()
    if alpha == 0.0:
        assert abs(dEdt) < 1e-12 * scale
    else:
        assert dEdt < -1e-6 * scale


def test_galilean_invariance():
    c, O, st = _random_state()
    r0 = O.interact(st, brute=True)
    st2 = st.copy()
    st2.vx += 0.75
    st2.vy -= 0.5
    st2.vz += 0.25
    r1 = O.interact(st2, brute=True)
    assert np.abs(r1["a"] - r0["a"]).max() < 1e-12 * r0["sa"].max()
    assert np.abs(r1["drho"] - r0["drho"]).max() < 1e-12 * r0["sd"].max()


def test_translation_by_whole_cells_leaves_rates_unchanged():
    c, O, st = _random_state()
    r0 = O.interact(st)
    cs = 2 * c.h
    p = dict(c.params())
    shift = np.array([3 * cs, -2 * cs, cs])
    p["dmin"] = tuple(np.array(c.dmin) + shift)
    p["dmax"] = tuple(np.array(c.dmax) + shift)
    O2 = oracle.Oracle(p)
    st2 = oracle.State(st.pos() + shift, st.vel(), st.rho, st.ids)
    r1 = O2.interact(st2)
    assert np.array_equal(r0["nnb"], r1["nnb"])
    assert np.abs(r1["a"] - r0["a"]).max() < 1e-9 * r0["sa"].max()


@pytest.mark.parametrize("h_over_dp,rtol", [(1.3, 3e-2), (2.0, 5e-3)])
def test_continuity_recovers_minus_rho_div_v_on_a_lattice(h_over_dp, rtol):
    """Eq. 7 for a linear velocity field v = A r at an interior lattice
    particle approximates -rho tr(A) (Eq. 1); the lattice moment error
    (about 2% at h = 1.3 dp) shrinks as h/dp grows."""
    c = _lattice_case(13, 13, 13)
    p = c.params()
    p["h"] = h_over_dp * c.dp
    p["dmin"] = tuple(np.array(c.dmin) - 2 * p["h"])
    p["dmax"] = tuple(np.array(c.dmax) + 2 * p["h"])
    O = oracle.Oracle(p)
    A = np.array([[0.3, 0.1, -0.2], [0.05, -0.7, 0.4], [0.2, 0.1, 0.9]])
    st = oracle.State(c.pos, c.pos @ A.T, c.rho, c.ids)
    r = O.interact(st)
    inner = _interior(c.pos, 2.01 * p["h"])
    assert inner.sum() > 10
    want = -c.rho0 * np.trace(A)
    assert np.allclose(r["drho"][inner], want, rtol=rtol)


@pytest.mark.parametrize("h_over_dp,tol", [(1.3, 0.05), (2.0, 0.01)])
def test_hydrostatic_column_is_in_balance(h_over_dp, tol):
    """Eq. 9 on a lattice column with the hydrostatic density profile: the
    pressure gradient balances gravity away from the free surface, up to the
    same lattice moment error as the continuity pin (about 2% of g at
    h = 1.3 dp, falling as h/dp grows).  A large c0 keeps the compressibility
    error (of order 4 g (rho - rho0)/rho0) out of the way."""
    c = _lattice_case(12, 12, 20, c0=300.0)
    H = 20 * c.dp
    rho = cases.hydrostatic_density(c.pos[:, 2], H, c.rho0, c.c0).astype(np.float32)
    p = c.params()
    p["h"] = h_over_dp * c.dp
    p["dmin"] = tuple(np.array(c.dmin) - 2 * p["h"])
    p["dmax"] = tuple(np.array(c.dmax) + 2 * p["h"])
    O = oracle.Oracle(p)
    st = oracle.State(c.pos, np.zeros_like(c.pos), rho, c.ids)
    r = O.interact(st)
    inner = _interior(c.pos, 2.01 * p["h"])
    assert inner.sum() > 20
    assert np.abs(r["a"][inner][:, :2]).max() < 1e-9
    assert np.abs(r["a"][inner][:, 2]).max() < tol * 9.81


def test_viscosity_switch_linearity_and_scaling():
    c, _, st = _random_state(alpha=0.0)
    p = c.params()
    rs = {}
    for a in (0.0, 0.05, 0.1):
        p["alpha"] = a
        rs[a] = oracle.Oracle(p).interact(st, brute=True)
    scale = rs[0.0]["sa"].max()
    # linear in alpha
    d1 = rs[0.05]["a"] - rs[0.0]["a"]
    d2 = rs[0.1]["a"] - rs[0.05]["a"]
    assert np.abs(d1 - d2).max() < 1e-12 * scale
    assert np.abs(d1).max() > 1e-6 * scale
    # only approaching pairs: with all particles receding from the centre
    # (v = +r) viscosity does nothing
    st2 = oracle.State(st.pos(), st.pos() - st.pos().mean(0), st.rho, st.ids)
    p["alpha"] = 0.0
    a0 = oracle.Oracle(p).interact(st2, brute=True)["a"]
    p["alpha"] = 0.5
    a1 = oracle.Oracle(p).interact(st2, brute=True)["a"]
    assert np.array_equal(a0, a1)
    # rho = rho0 everywhere: no pressure force, viscous force ~ c0
    st3 = oracle.State(st.pos(), -(st.pos() - st.pos().mean(0)),
                       np.full(st.n, c.rho0), st.ids)
    p["alpha"] = 0.1
    p["c0"] = 20.0
    b1 = oracle.Oracle(p).interact(st3, brute=True)["a"] - np.array(c.gravity)
    p["c0"] = 40.0
    b2 = oracle.Oracle(p).interact(st3, brute=True)["a"] - np.array(c.gravity)
    assert np.abs(b1).max() > 0
    assert np.allclose(b2, 2 * b1, rtol=1e-12, atol=1e-12 * np.abs(b1).max())


# --- artificial viscosity and the viscous CFL term, worked by hand -----------
#
# Sec. 2.2 with the readings R2 (rho_ij = (rho_i + rho_j)/2), R3 (c_i =
# c0 (rho_i/rho0)^3) and R7 (dt = CFL min(sqrt(h/|a|), h/(c_max + mu_max)),
# mu_max = max over pairs of h |v_ij.r_ij| / (r_ij^2 + eta^2)).  Scale-free
# constants make every factor a small rational: h = 1, rho0 = 1000, c0 = 10,
# gamma = 7 (B = 10^5/7), alpha = 1/2, eta^2 = h^2/100, m = 1, no gravity.
# The kernel gradient F(r) cancels from the ratios used below, so these pins
# fix the viscosity and the pressure terms independently of the kernel.

def _hand_params(alpha=0.5):
    return dict(dp=0.5, h=1.0, rho0=1000.0, gamma=7.0, c0=10.0, alpha=alpha,
                eta2_coef=0.01, gravity=(0.0, 0.0, 0.0), cfl=0.2, mass=1.0,
                dmin=(-4.0, -4.0, -4.0), dmax=(4.0, 4.0, 4.0), n_bound=0)


def test_viscosity_of_an_approaching_pair_worked_by_hand():
    """Two fluid particles: i at the origin with v_i = (2, 0, 0) and rho_i =
    rho0; j at (3/2, 0, 0) with v_j = (-1, 0, 0) and rho_j = 2 rho0.

      r_ij = (-3/2, 0, 0), v_ij = (3, 0, 0), v_ij.r_ij = -9/2 (approaching)
      nu    = h v_ij.r_ij / (r^2 + eta^2) = -(9/2) / (9/4 + 1/100) = -225/113
      c_i = 10, c_j = 10 * 2^3 = 80: c_bar = 45;  rho_bar = 1500
      Pi_ij = -alpha c_bar nu / rho_bar = 27/904
      P_i = 0 (rho_i = rho0);  P_j = B (2^7 - 1) / rho_j^2 = 127/280
      a_i,x = -m (P_i + P_j + Pi_ij) F (-3/2),  drho_i/dt = m (-9/2) F
      => a_i,x / (drho_i/dt) = -(P_j + Pi_ij)/3 = -1912/11865
                              = -0.161146228402865571...
         (alpha = 0: -(127/280)/3 = -0.151190476190476190...)
      particle j: r_ji = -r_ij, same v.r, so its ratio is +1912/11865
      mu_max = 225/113 = 1.99115044247787610...;  c_max = 80
      dt = 0.2 / (80 + 225/113) = 0.00243928764166216945...
           (|a| is about 0.02 here, so sqrt(h/|a|) ~ 6.5 does not decide)

    Wrong readings give, for a_i,x / (drho_i/dt): eta^2 = 0.1 h^2 ->
    -0.16076494; rho_i for rho_bar -> -0.16612410; c0 (or c_i) for c_bar ->
    -0.15340287; and dt without mu_max would be 0.0025."""
    p = _hand_params()
    pos = np.array([[0.0, 0.0, 0.0], [1.5, 0.0, 0.0]])
    vel = np.array([[2.0, 0.0, 0.0], [-1.0, 0.0, 0.0]])
    st = oracle.State(pos, vel, np.array([1000.0, 2000.0]), np.array([0, 1], np.uint32))
    for brute in (True, False):
        r = oracle.Oracle(p).interact(st, brute=brute)
        assert r["pairs"] == 2
        ratio_i = r["a"][0, 0] / r["drho"][0]
        ratio_j = r["a"][1, 0] / r["drho"][1]
        assert ratio_i == pytest.approx(-1912 / 11865, rel=1e-13)
        assert ratio_j == pytest.approx(1912 / 11865, rel=1e-13)
        assert ratio_i == pytest.approx(-0.161146228402865571, rel=1e-13)
        assert np.all(r["a"][:, 1:] == 0.0)
        assert r["drho"][0] == r["drho"][1]          # v.r and F are symmetric
        assert r["terms"][2] == pytest.approx(225 / 113, rel=1e-14)
        assert r["terms"][1] == 80.0
        assert r["dt"] == pytest.approx(0.00243928764166216945, rel=1e-14)
    # without viscosity only the pressure term is left
    r0 = oracle.Oracle(_hand_params(alpha=0.0)).interact(st, brute=True)
    assert r0["a"][0, 0] / r0["drho"][0] == pytest.approx(-127 / 840, rel=1e-13)
    # the viscous part alone: Pi_ij = -3 (ratio(alpha) - ratio(0))
    pi = -3.0 * (ratio_i - r0["a"][0, 0] / r0["drho"][0])
    assert pi == pytest.approx(27 / 904, rel=1e-11)
    # the literal discriminates each wrong reading by far more than the tolerance
    for wrong in (-0.16076494427558257, -0.16612410450906026, -0.15340286557100716):
        assert abs(wrong - ratio_i) > 1e-3 * abs(ratio_i)


def test_viscous_cfl_term_from_a_receding_pair_worked_by_hand():
    """Three fluid particles: i and j as in the two-particle case, plus k at
    (0, 5/4, 0) with v_k = (0, 3, 0) and rho_k = rho0/2 (c_k = 10/8,
    P_k = B (2^-7 - 1) / 500^2 = -127/2240).  Pairs (all within 2h = 2):

      (i, j): |r|^2 = 9/4,   v.r = -9/2 (approaching), |nu| = 225/113
      (i, k): |r|^2 = 25/16, v.r = 15/4 (receding),    |nu| = 1500/629
      (j, k): |r|^2 = 61/16, v.r = 9/4  (receding),    |nu| = 0.5886...

    mu_max is set by the receding pair (i, k): 1500/629 = 2.38473767885532591;
    c_max = 80; dt = 0.2 / (80 + 1500/629) = 0.00242763411810111926.
    The receding pair adds no viscosity, and (i, j) acts along x and (i, k)
    along y only, so with P_i = 0 the kernel values follow from i's
    acceleration, F_ij = a_i,x / ((3/2)(P_j + Pi_ij)) and
    F_ik = a_i,y / ((5/4) P_k), and Eq. 7 must then give
    drho_i/dt = (-9/2) F_ij + (15/4) F_ik with Pi_ij = 27/904 from the
    two-particle case (a viscosity applied to the receding pair, or any
    other Pi_ij, breaks this identity)."""
    p = _hand_params()
    pos = np.array([[0.0, 0.0, 0.0], [1.5, 0.0, 0.0], [0.0, 1.25, 0.0]])
    vel = np.array([[2.0, 0.0, 0.0], [-1.0, 0.0, 0.0], [0.0, 3.0, 0.0]])
    rho = np.array([1000.0, 2000.0, 500.0])
    st = oracle.State(pos, vel, rho, np.array([0, 1, 2], np.uint32))
    r = oracle.Oracle(p).interact(st, brute=True)
    assert r["pairs"] == 6
    assert r["terms"][2] == pytest.approx(1500 / 629, rel=1e-14)
    assert r["terms"][1] == 80.0
    assert r["dt"] == pytest.approx(0.00242763411810111926, rel=1e-14)
    Pj, Pk, Pij = 127 / 280, -127 / 2240, 27 / 904
    F_ij = r["a"][0, 0] / (1.5 * (Pj + Pij))
    F_ik = r["a"][0, 1] / (1.25 * Pk)
    assert F_ij < 0 and F_ik < 0                       # the kernel decreases
    assert r["drho"][0] == pytest.approx(-4.5 * F_ij + 3.75 * F_ik, rel=1e-12)
    # the same identity with a viscosity on the receding pair would be off
    nu_ik = 1500 / 629
    Pik_wrong = -0.5 * (10 + 1.25) / 2 * nu_ik / 750
    F_ik_wrong = r["a"][0, 1] / (1.25 * (Pk + Pik_wrong))
    assert abs((-4.5 * F_ij + 3.75 * F_ik_wrong) - r["drho"][0]) > 1e-3 * abs(r["drho"][0])
    # a boundary particle never sets mu_max by itself: with k a boundary
    # particle (id below n_bound) mu_max comes from fluid i's pairs, which
    # still include (i, k)
    pb = dict(p, n_bound=1)
    st_b = oracle.State(pos[[2, 0, 1]], vel[[2, 0, 1]], rho[[2, 0, 1]],
                        np.array([0, 1, 2], np.uint32))
    rb = oracle.Oracle(pb).interact(st_b, brute=True)
    assert rb["terms"][2] == pytest.approx(1500 / 629, rel=1e-14)


# --- time step and integrator ------------------------------------------------

def _isolated(n=5, dp=0.02, v=None, n_bound=0):
    pos = np.array([[i * 1.0, 0.5, 0.5] for i in range(n)], dtype=np.float64)
    vel = np.zeros((n, 3), np.float32) if v is None else np.asarray(v, np.float32)
    h = 1.3 * dp
    dmin, dmax = (-1.0, -1.0, -1.0), (n + 1.0, 2.0, 2.0)
    return cases.Case(name="iso", pos=pos, vel=vel,
                      rho=np.full(n, 1000.0, np.float32),
                      ids=np.arange(n, dtype=np.uint32), n_bound=n_bound,
                      dp=dp, h=h, rho0=1000.0, c0=20.0, alpha=0.01, cfl=0.2,
                      gravity=(0.0, 0.0, -9.81), dmin=dmin, dmax=dmax,
                      fluid_height=0.0)


def test_cfl_step_for_isolated_particles():
    c = _isolated()
    O = _oracle(c)
    r = O.interact(oracle.State.from_case(c))
    assert r["pairs"] == 0
    h = c.h
    want = 0.2 * min(math.sqrt(h / 9.81), h / 20.0)
    assert r["dt"] == pytest.approx(want, rel=1e-15)


def test_free_particle_follows_the_parabola():
    v0 = np.array([[0.3, -0.2, 1.5]] * 3, np.float32)
    c = _isolated(3, v=v0)
    O = _oracle(c)
    st = oracle.State.from_case(c)
    x0 = st.pos().copy()
    t = 0.0
    for k in range(50):
        dt, _ = O.step(st, dt_fixed=1e-3 * (1 + 0.1 * (k % 3)))
        t += dt
    g = np.array(c.gravity)
    want = x0 + v0.astype(np.float64) * t + 0.5 * g * t * t
    assert np.abs(st.pos() - want).max() < 1e-13
    assert np.abs(st.vel() - (v0 + g * t)).max() < 1e-13
    assert np.all(st.rho == 1000.0)


def test_boundary_particles_never_move():
    c = cases.c1_dam_break()
    O = _oracle(c)
    st = oracle.State.from_case(c)
    b = st.ids < c.n_bound
    x0, v0, r0 = st.pos()[b].copy(), st.vel()[b].copy(), st.rho[b].copy()
    for _ in range(3):
        O.step(st)
    assert np.array_equal(st.pos()[b], x0)
    assert np.array_equal(st.vel()[b], v0)
    assert not np.array_equal(st.rho[b], r0)      # density does evolve


def test_integrator_is_second_order():
    c = cases.random_block(120, seed=31, jitter=0.2, vel_range=0.5)
    O = _oracle(c)

    def run(nsub):
        st = oracle.State.from_case(c)
        dt = 4e-4 / nsub
        for _ in range(8 * nsub):
            O.step(st, dt_fixed=dt)
        return np.concatenate([st.pos().ravel(), st.vel().ravel() * 1e-3,
                               st.rho * 1e-6])

    ref = run(16)
    e1 = np.abs(run(1) - ref).max()
    e2 = np.abs(run(2) - ref).max()
    e4 = np.abs(run(4) - ref).max()
    assert e1 > 0
    assert 3.0 < e1 / e2 < 5.5
    assert 3.0 < e2 / e4 < 5.5


def test_excluded_particles_are_frozen_and_do_not_interact():
    c = cases.random_block(300, seed=8)
    pos = c.pos.copy()
    pos[0] = np.array(c.dmax) + 1.0
    pos[1, 0] = np.nan
    c.pos = pos
    O = _oracle(c)
    st = oracle.State.from_case(c)
    r = O.interact(st)
    assert r["nnb"][0] == 0 and r["nnb"][1] == 0
    assert np.all(r["a"][:2] == 0)
    x0 = st.pos()[0].copy()
    O.step(st, dt_fixed=1e-4)
    assert np.array_equal(st.pos()[0], x0)
    assert O.diagnostics(st)["n_out"] == 2


def test_diagnostics_closed_forms():
    c = _isolated(4, v=[[1.0, 0, 0], [0, 2.0, 0], [0, 0, -1.0], [0, 0, 0]])
    O = _oracle(c)
    d = O.diagnostics(oracle.State.from_case(c))
    m = c.mass
    assert d["mass"] == pytest.approx(4 * m)
    assert np.allclose(d["momentum"], [m, 2 * m, -m])
    assert d["kinetic"] == pytest.approx(0.5 * m * (1 + 4 + 1))
    assert d["potential"] == pytest.approx(4 * m * 9.81 * 0.5)
    assert d["internal"] == 0.0


@pytest.mark.slow
def test_still_tank_stays_hydrostatic():
    """A tank filled to a level at rest (hydrostatic start) stays close to the
    hydrostatic pressure profile after 0.1 s (dynamic boundaries leave a
    near-wall gap, so this is a weak pin)."""
    c = cases.dam_break(tank=(0.2, 0.12, 0.3), fluid=(0.2, 0.12, 0.2),
                        dp=0.02, name="still_tank")
    O = _oracle(c)
    st = oracle.State.from_case(c)
    t = 0.0
    while t < 0.1:
        dt, _ = O.step(st)
        t += dt
    fl = st.ids >= c.n_bound
    z = st.z[fl]
    p = np.array([O.pressure(x) for x in st.rho[fl]])
    deep = (c.fluid_height - z) > 3 * c.dp
    want = c.rho0 * 9.81 * (c.fluid_height - z[deep])
    assert np.abs(p[deep].mean() / want.mean() - 1) < 0.1
    assert np.abs(st.vel()[fl]).max() < 0.5
