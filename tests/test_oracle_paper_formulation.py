"""Pins of the oracle's paper formulation: the cubic spline kernel (Sec. 2.2)
and the second-order Verlet integrator (Sec. 3.3).

As with the other pins, nothing here compares the oracle with itself: the
kernel is checked against its normalisation, its smoothness at the joint of
the two pieces and the finite-difference derivative of W; the pair sums
against the conservation laws of the discrete equations; the integrator
against closed-form motion and against convergence to the solution of the
same ordinary differential equations.
"""
import dataclasses
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_1210_1017_gb300 import cases


def _cubic(case):
    return dataclasses.replace(case, kernel="cubic")


def _oracle(case, **over):
    p = case.params()
    p.update(over)
    return oracle.Oracle(p)


# --- cubic spline (Sec. 2.2) -------------------------------------------------

def test_cubic_spline_integrates_to_one_with_compact_support():
    c = _cubic(cases.c1_dam_break())
    O = _oracle(c)
    h = c.h
    # the two polynomial pieces integrated separately (no kink inside)
    inner, _ = integrate.quad(lambda r: 4 * math.pi * r * r * O.w(r), 0.0, h,
                              epsabs=1e-14, epsrel=1e-13)
    outer, _ = integrate.quad(lambda r: 4 * math.pi * r * r * O.w(r), h, 2 * h,
                              epsabs=1e-14, epsrel=1e-13)
    assert abs(inner + outer - 1.0) < 1e-12
    assert O.w(2 * h) == 0.0 and O.f(2 * h) == 0.0
    assert O.w(2.5 * h) == 0.0 and O.f(2.5 * h) == 0.0
    rs = np.linspace(0, 2 * h, 401)
    w = np.array([O.w(r) for r in rs])
    assert np.all(np.diff(w) < 0) and np.all(w[:-1] > 0)
    # it differs from the Wendland kernel the other formulation uses
    Ow = _oracle(cases.c1_dam_break())
    assert abs(O.w(0.5 * h) - Ow.w(0.5 * h)) > 1e-3 * Ow.w(0.5 * h)


def test_cubic_spline_is_twice_differentiable_at_the_joint():
    """W, dW/dr and d2W/dr2 are continuous at q = 1, where the two pieces
    meet; a wrong coefficient in either piece breaks one of them."""
    c = _cubic(cases.c1_dam_break())
    O = _oracle(c)
    h = c.h
    e = 1e-7 * h
    w0 = O.w(h)
    assert O.w(h - e) == pytest.approx(w0, rel=1e-6)
    # first derivative dW/dr = F r from each side
    d_lo, d_hi = O.f(h - e) * (h - e), O.f(h + e) * (h + e)
    assert d_lo == pytest.approx(d_hi, rel=1e-6)
    # second derivative by one-sided differences of dW/dr
    s = 1e-4 * h
    g = lambda r: O.f(r) * r
    dd_lo = (g(h - s) - g(h - 2 * s)) / s
    dd_hi = (g(h + 2 * s) - g(h + s)) / s
    assert dd_lo == pytest.approx(dd_hi, rel=1e-3)
    # and the value at the joint is a quarter of the peak: W(h) = W(0)/4
    assert w0 == pytest.approx(0.25 * O.w(0.0), rel=1e-14)


def test_cubic_spline_gradient_is_derivative_of_kernel():
    c = _cubic(cases.c1_dam_break())
    O = _oracle(c)
    h = c.h
    for q in np.concatenate([np.linspace(0.05, 0.95, 19), np.linspace(1.05, 1.95, 19)]):
        r = q * h
        e = 1e-6 * h
        dw = (O.w(r + e) - O.w(r - e)) / (2 * e)
        assert O.f(r) == pytest.approx(dw / r, rel=1e-7, abs=1e-9 * abs(O.f(0.5 * h)))


def _random_state(alpha, seed=13):
    c = _cubic(cases.random_block(800, seed=seed, jitter=0.3, vel_range=1.0,
                                  rho_range=(0.995, 1.02), alpha=alpha))
    return c, _oracle(c), oracle.State.from_case(c)


def test_cubic_spline_pair_sums_conserve_momentum():
    c, O, st = _random_state(alpha=0.05)
    r = O.interact(st, brute=True)
    fint = c.mass * (r["a"] - np.array(c.gravity))
    scale = c.mass * r["sa"].sum()
    assert np.abs(fint.sum(0)).max() < 1e-13 * scale
    torque = np.cross(c.pos, fint).sum(0)
    assert np.abs(torque).max() < 1e-13 * scale * np.abs(c.pos).max()


@pytest.mark.parametrize("alpha", [0.0, 0.05])
def test_cubic_spline_energy_rate(alpha):
    """The energy identity of the semi-discrete equations holds for any
    kernel: dE/dt = 0 without viscosity and < 0 with it."""
    c, O, st = _random_state(alpha=alpha)
    r = O.interact(st, brute=True)
    m = c.mass
    v = st.vel()
    p_over_rho2 = np.array([O.pressure(x) / x ** 2 for x in st.rho])
    kin = m * np.einsum("ij,ij->i", v, r["a"] - np.array(c.gravity))
    intl = m * p_over_rho2 * r["drho"]
    dEdt = kin.sum() + intl.sum()
    scale = np.abs(kin).sum() + np.abs(intl).sum()
    if alpha == 0.0:
        assert abs(dEdt) < 1e-12 * scale
    else:
        assert dEdt < -1e-6 * scale


def test_cubic_spline_grid_neighbours_equal_brute_force():
    c, O, st = _random_state(alpha=0.01, seed=21)
    a = O.interact(st, brute=False)
    b = O.interact(st, brute=True)
    assert np.array_equal(a["nnb"], b["nnb"])
    assert np.abs(a["a"] - b["a"]).max() <= 1e-12 * a["sa"].max()


# --- Verlet integrator (Sec. 3.3) --------------------------------------------

def _isolated(n=3, v=None):
    dp = 0.02
    pos = np.array([[i * 1.0, 0.5, 0.5] for i in range(n)], dtype=np.float64)
    vel = np.asarray(v, np.float32)
    return cases.Case(name="iso", pos=pos, vel=vel,
                      rho=np.full(n, 1000.0, np.float32),
                      ids=np.arange(n, dtype=np.uint32), n_bound=0,
                      dp=dp, h=1.3 * dp, rho0=1000.0, c0=20.0, alpha=0.01, cfl=0.2,
                      gravity=(0.0, 0.0, -9.81), dmin=(-1.0, -1.0, -1.0),
                      dmax=(n + 1.0, 2.0, 2.0), fluid_height=0.0,
                      integrator="verlet")


@pytest.mark.parametrize("every", [1, 3, 40])
def test_verlet_free_fall_is_exact(every):
    """Under a constant acceleration both the leapfrog and the Euler steps
    reproduce r = r0 + v0 t + g t^2/2 and v = v0 + g t (constant dt)."""
    v0 = np.array([[0.3, -0.2, 1.5]] * 3, np.float32)
    c = _isolated(3, v=v0)
    O = _oracle(c)
    st = oracle.State.from_case(c)
    x0 = st.pos().copy()
    dts, _ = O.verlet_run(st, 60, every=every, dt_fixed=1e-3)
    t = sum(dts)
    g = np.array(c.gravity)
    assert np.abs(st.pos() - (x0 + v0.astype(np.float64) * t + 0.5 * g * t * t)).max() < 1e-13
    assert np.abs(st.vel() - (v0 + g * t)).max() < 1e-13
    assert np.all(st.rho == 1000.0)


def test_verlet_update_closed_forms():
    """The update on given rates: a constant density rate gives
    rho = rho0 + D t exactly; with zero rates the leapfrog step swaps the
    current and earlier velocities while the Euler step keeps the current
    one (which steps are Euler steps is the caller's choice)."""
    c = _isolated(2, v=[[1.0, 0.0, 0.0], [0.0, 2.0, 0.0]])
    O = _oracle(c)
    st = oracle.State.from_case(c)
    prev = st.copy()
    D = np.array([3.0, -1.5])
    a0 = np.zeros((2, 3))
    dt = 1e-3
    for k in range(7):
        O.verlet_update(st, prev, a0, D, dt, euler=(k % 3 == 0))
    assert np.allclose(st.rho, 1000.0 + D * 7 * dt, rtol=0, atol=1e-12)
    # an inconsistent history: earlier velocity 0, current v
    st = oracle.State.from_case(c)
    prev = st.copy()
    prev.vx[:] = 0.0
    prev.vy[:] = 0.0
    v = st.vel().copy()
    seen = []
    for euler in (False, False, True, False):
        O.verlet_update(st, prev, a0, np.zeros(2), dt, euler=euler)
        seen.append(st.vel().copy())
    assert np.array_equal(seen[0], np.zeros_like(v))   # leapfrog: v1 = v_-1
    assert np.array_equal(seen[1], v)                  # leapfrog: v2 = v0
    assert np.array_equal(seen[2], v)                  # Euler: v3 = v2
    assert np.array_equal(seen[3], v)                  # leapfrog: v4 = v2 = v3
    # positions move with the current velocity only
    assert np.allclose(st.pos() - c.pos, dt * (1 + 0 + 1 + 1) * v, rtol=0, atol=1e-15)


def test_verlet_boundary_particles_never_move():
    c = dataclasses.replace(cases.c1_dam_break(), integrator="verlet")
    O = _oracle(c)
    st = oracle.State.from_case(c)
    b = st.ids < c.n_bound
    x0, v0, r0 = st.pos()[b].copy(), st.vel()[b].copy(), st.rho[b].copy()
    O.verlet_run(st, 4, every=40)
    assert np.array_equal(st.pos()[b], x0)
    assert np.array_equal(st.vel()[b], v0)
    assert not np.array_equal(st.rho[b], r0)


def _conv_case():
    return cases.random_block(120, seed=31, jitter=0.2, vel_range=0.5)


def _flat(st):
    return np.concatenate([st.pos().ravel(), st.vel().ravel() * 1e-3, st.rho * 1e-6])


@pytest.mark.parametrize("kernel", ["wendland", "cubic"])
def test_verlet_converges_to_the_same_solution(kernel):
    """Verlet and the symplectic scheme integrate the same equations: with
    a single Euler start the leapfrog is second order and converges to the
    fine symplectic solution; with an Euler step every 40 steps it still
    converges (the Euler steps add a first-order term of size 1/40)."""
    c = dataclasses.replace(_conv_case(), kernel=kernel)
    O = _oracle(c)
    T = 4 * 8e-4

    st = oracle.State.from_case(c)
    for _ in range(64):
        O.step(st, dt_fixed=T / 64)
    ref = _flat(st)

    def verlet(nsteps, every):
        s = oracle.State.from_case(c)
        O.verlet_run(s, nsteps, every=every, dt_fixed=T / nsteps)
        return _flat(s)

    e = [np.abs(verlet(n, 10 ** 9) - ref).max() for n in (8, 16, 32)]
    assert e[0] > 0
    assert 3.0 < e[0] / e[1] < 5.5 and 3.0 < e[1] / e[2] < 5.5
    e40 = [np.abs(verlet(n, 40) - ref).max() for n in (40, 80, 160)]
    assert e40[0] / e40[1] > 1.8 and e40[1] / e40[2] > 1.8
    assert e40[2] < 0.1 * np.abs(_flat(oracle.State.from_case(c)) - ref).max()
