"""Seeded synthetic inputs for the weakly compressible SPH dam-break workloads.

This module is shared by the CUDA path's callers, the tests and the FP64
oracle.  It only places particles and sets their initial velocity and
density; it contains none of the per-step arithmetic of the method (no
kernel, no equation of state evaluation during a step, no neighbour search,
no integrator).  Everything is deterministic for a given seed.

Geometry conventions (the paper gives none; these are the readings used
throughout the project):

* Particles sit on a lattice of spacing ``dp`` at ``(i + 1/2) dp``.
* A tank of interior ``Lx x Ly x Lz`` spans ``[0, nx*dp] x [0, ny*dp] x
  [0, nz*dp]`` with ``n = round(L/dp)``.  Its floor and four side walls are
  two layers of boundary particles outside the interior, at ``-dp/2`` and
  ``-3dp/2`` from each wall; the top is open.  Dynamic boundary particles
  follow continuity and the equation of state but never move (Sec. 2.3).
* The fluid block starts at the tank's ``x = 0`` wall, spans
  ``floor(L/dp)`` lattice sites per axis (clamped to the tank), and is at
  rest with a hydrostatic density profile (the initial condition).
* Particle mass is ``rho0 * dp**3`` for every particle.
* Ids ``0 .. n_bound-1`` are boundary particles, ``n_bound .. N-1`` fluid.
* The cell-grid domain is the bounding box of the initial particles widened
  by one cell (``2h``) on every side, with the top raised to at least half a
  tank height above the tank rim, so splashes stay inside it.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1


def splitmix64_stream(seed: int):
    """The SplitMix64 generator (Steele, Lea and Flood, OOPSLA 2014), as a
    Python generator of 64-bit integers."""
    state = seed & MASK64
    while True:
        state = (state + 0x9E3779B97F4A7C15) & MASK64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        yield z ^ (z >> 31)


class SplitMix64:
    """Uniform doubles in [0, 1) from SplitMix64 (top 53 bits)."""

    def __init__(self, seed: int):
        self._it = splitmix64_stream(seed)

    def u01(self) -> float:
        return (next(self._it) >> 11) * (1.0 / (1 << 53))

    def uniform(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * self.u01()


@dataclass
class Case:
    """One particle set plus the physical constants the method needs.

    Arrays are in the generator's order (boundary first, then fluid) unless
    ``shuffle`` was requested.  ``pos`` is float64, ``vel`` and ``rho``
    float32 (the storage precision of the GPU path; the oracle widens them
    exactly), ``ids`` uint32.
    """

    name: str
    pos: np.ndarray          # (N, 3) float64
    vel: np.ndarray          # (N, 3) float32
    rho: np.ndarray          # (N,)   float32
    ids: np.ndarray          # (N,)   uint32
    n_bound: int
    dp: float
    h: float
    rho0: float
    c0: float
    alpha: float
    cfl: float
    gravity: tuple
    dmin: tuple
    dmax: tuple
    fluid_height: float
    eta2_coef: float = 0.01
    gamma: float = 7.0
    kernel: str = "wendland"          # or "cubic" (the paper's, Sec. 2.2)
    integrator: str = "symplectic"    # or "verlet" (the paper's, Sec. 3.3)
    verlet_every: int = 40            # Verlet: an Euler step every this many
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    @property
    def n_fluid(self) -> int:
        return self.n - self.n_bound

    @property
    def mass(self) -> float:
        return self.rho0 * self.dp ** 3

    def params(self) -> dict:
        """Scalar inputs handed to both the CUDA path and the oracle."""
        return dict(dp=self.dp, h=self.h, rho0=self.rho0, gamma=self.gamma,
                    c0=self.c0, alpha=self.alpha, eta2_coef=self.eta2_coef,
                    gravity=tuple(self.gravity), cfl=self.cfl, mass=self.mass,
                    dmin=tuple(self.dmin), dmax=tuple(self.dmax),
                    n_bound=int(self.n_bound), kernel=self.kernel,
                    integrator=self.integrator, verlet_every=int(self.verlet_every))


def _nsites(length: float, dp: float) -> int:
    """Lattice sites that fit in ``length`` (floor with a rounding guard)."""
    return int(math.floor(length / dp + 1e-6))


def _nround(length: float, dp: float) -> int:
    return int(round(length / dp))


def _lattice(ix, iy, iz, dp, origin=(0.0, 0.0, 0.0)):
    """Positions (i + 1/2) dp for integer index arrays."""
    p = np.empty((ix.size, 3), dtype=np.float64)
    p[:, 0] = origin[0] + (ix + 0.5) * dp
    p[:, 1] = origin[1] + (iy + 0.5) * dp
    p[:, 2] = origin[2] + (iz + 0.5) * dp
    return p


def tank_boundary(nxt: int, nyt: int, nzt: int, dp: float, layers: int = 2):
    """Two-layer open-top tank shell around the interior [0,nxt)x[0,nyt)x[0,nzt)."""
    ii = np.arange(-layers, nxt + layers)
    jj = np.arange(-layers, nyt + layers)
    gi, gj = np.meshgrid(ii, jj, indexing="ij")
    gi = gi.ravel()
    gj = gj.ravel()
    ring = ~((gi >= 0) & (gi < nxt) & (gj >= 0) & (gj < nyt))
    ri, rj = gi[ring], gj[ring]
    parts = []
    for k in range(-layers, nzt):
        if k < 0:
            parts.append(_lattice(gi, gj, np.full(gi.size, k), dp))
        else:
            parts.append(_lattice(ri, rj, np.full(ri.size, k), dp))
    return np.concatenate(parts, axis=0)


def obstacle_shell(i0: int, j0: int, nx: int, ny: int, nz: int, dp: float,
                   layers: int = 2):
    """Boundary particles filling the outer ``layers`` sites of a cuboid
    obstacle standing on the floor (sites [i0,i0+nx) x [j0,j0+ny) x [0,nz))."""
    ii, jj, kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz),
                             indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
    dist = np.minimum.reduce([ii, nx - 1 - ii, jj, ny - 1 - jj, nz - 1 - kk])
    keep = dist < layers
    return _lattice(ii[keep] + i0, jj[keep] + j0, kk[keep], dp)


def fluid_block(nfx: int, nfy: int, nfz: int, dp: float, i0: int = 0,
                j0: int = 0, exclude=None):
    ii, jj, kk = np.meshgrid(np.arange(nfx), np.arange(nfy), np.arange(nfz),
                             indexing="ij")
    # x fastest so that ids follow the lattice rows
    ii = ii.transpose(2, 1, 0).ravel() + i0
    jj = jj.transpose(2, 1, 0).ravel() + j0
    kk = kk.transpose(2, 1, 0).ravel()
    if exclude is not None:
        keep = np.ones(ii.size, dtype=bool)
        for (a0, b0, na, nb, nc) in exclude:
            keep &= ~((ii >= a0) & (ii < a0 + na) & (jj >= b0) & (jj < b0 + nb)
                      & (kk < nc))
        ii, jj, kk = ii[keep], jj[keep], kk[keep]
    return _lattice(ii, jj, kk, dp)


def hydrostatic_density(z, surface: float, rho0: float, c0: float,
                        g: float = 9.81, gamma: float = 7.0):
    """Initial density of a fluid column at rest: the Tait law inverted for
    p = rho0 * g * (surface - z) (rho0 above the surface).  This is the
    initial condition only; B = c0^2 rho0 / gamma as in Sec. 2.2."""
    B = c0 * c0 * rho0 / gamma
    depth = np.maximum(surface - np.asarray(z, dtype=np.float64), 0.0)
    return rho0 * np.power(1.0 + rho0 * g * depth / B, 1.0 / gamma)


def domain_for(pos: np.ndarray, h: float, tank_top: float, tank_height: float):
    cs = 2.0 * h
    lo = pos.min(axis=0) - cs
    hi = pos.max(axis=0)
    hi = hi.copy()
    hi[2] = max(hi[2], tank_top + 0.5 * tank_height)
    hi = hi + cs
    return tuple(float(v) for v in lo), tuple(float(v) for v in hi)


def dam_break(tank=(1.0, 0.4, 0.6), fluid=(0.4, 0.4, 0.3), dp=0.02,
              h_over_dp=1.3, rho0=1000.0, alpha=0.01, cfl=0.2, g=9.81,
              obstacles=0, obstacle_size=(0.1, 0.1, 0.2),
              obstacle_x=(1.4, 2.8), obstacle_y=(0.1, 0.9), seed=1210,
              shuffle_seed=None, name="dam_break") -> Case:
    """Dam break in an open-top tank, optionally with cuboid obstacles placed
    downstream at seeded, non-overlapping positions on the floor."""
    nxt, nyt, nzt = (_nround(L, dp) for L in tank)
    nfx = min(_nsites(fluid[0], dp), nxt)
    nfy = min(_nsites(fluid[1], dp), nyt)
    nfz = min(_nsites(fluid[2], dp), nzt)
    bparts = [tank_boundary(nxt, nyt, nzt, dp)]
    placed = []
    if obstacles:
        rng = SplitMix64(seed)
        onx, ony, onz = (_nround(L, dp) for L in obstacle_size)
        tries = 0
        while len(placed) < obstacles:
            tries += 1
            if tries > 10000:
                raise RuntimeError("could not place obstacles")
            x = rng.uniform(obstacle_x[0], obstacle_x[1] - obstacle_size[0])
            y = rng.uniform(obstacle_y[0], obstacle_y[1] - obstacle_size[1])
            i0, j0 = int(round(x / dp)), int(round(y / dp))
            ok = all(i0 + onx + 2 <= a or a + onx + 2 <= i0 or
                     j0 + ony + 2 <= b or b + ony + 2 <= j0
                     for (a, b, _, _, _) in placed)
            if ok and i0 + onx <= nxt and j0 + ony <= nyt:
                placed.append((i0, j0, onx, ony, onz))
        for (i0, j0, a, b, c) in placed:
            bparts.append(obstacle_shell(i0, j0, a, b, c, dp))
    bpos = np.concatenate(bparts, axis=0)
    fpos = fluid_block(nfx, nfy, nfz, dp,
                       exclude=placed if placed else None)
    H = nfz * dp
    c0 = 10.0 * math.sqrt(g * H)
    pos = np.concatenate([bpos, fpos], axis=0)
    n = pos.shape[0]
    nb = bpos.shape[0]
    rho = hydrostatic_density(pos[:, 2], H, rho0, c0, g).astype(np.float32)
    vel = np.zeros((n, 3), dtype=np.float32)
    ids = np.arange(n, dtype=np.uint32)
    dmin, dmax = domain_for(pos, h_over_dp * dp, nzt * dp, nzt * dp)
    case = Case(name=name, pos=pos, vel=vel, rho=rho, ids=ids, n_bound=nb,
                dp=dp, h=h_over_dp * dp, rho0=rho0, c0=c0, alpha=alpha,
                cfl=cfl, gravity=(0.0, 0.0, -g), dmin=dmin, dmax=dmax,
                fluid_height=H,
                meta=dict(tank_sites=(nxt, nyt, nzt),
                          fluid_sites=(nfx, nfy, nfz), obstacles=placed))
    if shuffle_seed is not None:
        shuffle(case, shuffle_seed)
    return case


def shuffle(case: Case, seed: int) -> Case:
    """Permute the particle order in place (ids travel with particles)."""
    perm = np.random.default_rng(seed).permutation(case.n)
    case.pos = np.ascontiguousarray(case.pos[perm])
    case.vel = np.ascontiguousarray(case.vel[perm])
    case.rho = np.ascontiguousarray(case.rho[perm])
    case.ids = np.ascontiguousarray(case.ids[perm])
    return case


# --- the workloads --------------------------------------------------------

def c1_dam_break(**kw) -> Case:
    """Tank 1.0x0.4x0.6 m, fluid 0.4x0.4x0.3 m, dp = 0.02 m: 6,000 fluid
    particles plus a two-layer open tank."""
    return dam_break(tank=(1.0, 0.4, 0.6), fluid=(0.4, 0.4, 0.3), dp=0.02,
                     name="dam_break_6k", **kw)


def c2_dam_break_obstacles(dp=0.00733, **kw) -> Case:
    """Tank 3.2x1.0x0.8 m, fluid block 0.8x1.0x0.5 m (about 1.0M fluid
    particles at dp = 7.33 mm), three 0.1x0.1x0.2 m obstacles downstream."""
    return dam_break(tank=(3.2, 1.0, 0.8), fluid=(0.8, 1.0, 0.5), dp=dp,
                     obstacles=3, seed=1210, name="dam_break_obstacles_1m",
                     **kw)


def c3_dam_break_32m(dp=0.00114, **kw) -> Case:
    """The 1.0x0.4x0.6 m dam break scaled to dp = 1.14 mm: 32.2M fluid plus
    3.2M boundary particles."""
    return dam_break(tank=(1.0, 0.4, 0.6), fluid=(0.4, 0.4, 0.3), dp=dp,
                     name="dam_break_32m", **kw)


def scaled_dam_break(n_fluid_target: int, **kw) -> Case:
    """The 1.0x0.4x0.6 m dam break at the dp that gives about
    ``n_fluid_target`` fluid particles (for smaller stand-ins of C3)."""
    dp = (0.4 * 0.4 * 0.3 / n_fluid_target) ** (1.0 / 3.0)
    return dam_break(tank=(1.0, 0.4, 0.6), fluid=(0.4, 0.4, 0.3), dp=dp,
                     name=f"dam_break_{n_fluid_target}", **kw)


def ensemble_specs(n_instances=256, seed=1017, lo=0.2, hi=0.6, dp=0.02):
    """Per-instance fluid block sizes (bx, by, bz) drawn uniformly from
    [lo, hi] m with SplitMix64."""
    rng = SplitMix64(seed)
    return [(rng.uniform(lo, hi), rng.uniform(lo, hi), rng.uniform(lo, hi))
            for _ in range(n_instances)]


def ensemble_instance(spec, dp=0.02, **kw) -> Case:
    """One member of the batched ensemble: a 1.0 x b_y x 0.8 m tank whose
    fluid block b_x x b_y x b_z spans the full tank width."""
    bx, by, bz = spec
    return dam_break(tank=(1.0, by, 0.8), fluid=(bx, by, bz), dp=dp,
                     name="ensemble_member", **kw)


def random_block(n: int, seed: int = 7, dp: float = 0.02, h_over_dp=1.3,
                 jitter: float = 0.25, bound_layers: int = 1,
                 vel_range: float = 1.0, rho_range=(0.99, 1.02),
                 rho0: float = 1000.0, c0: float = 20.0, alpha: float = 0.01,
                 cfl: float = 0.2, g: float = 9.81) -> Case:
    """Small parity case: about ``n`` particles on a jittered cubic lattice,
    the bottom ``bound_layers`` sites marked as (fixed) boundary particles,
    fluid velocities U[-v, v] m/s and densities rho0 * U[rho_range]."""
    rng = np.random.default_rng(seed)
    side = max(2, int(round(n ** (1.0 / 3.0))))
    nz = max(bound_layers + 1, int(math.ceil(n / (side * side))))
    ii, jj, kk = np.meshgrid(np.arange(side), np.arange(side), np.arange(nz),
                             indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
    order = np.lexsort((ii, jj, kk))[:n]
    ii, jj, kk = ii[order], jj[order], kk[order]
    pos = _lattice(ii, jj, kk, dp)
    isb = kk < bound_layers
    pos[~isb] += rng.uniform(-jitter, jitter, size=(int((~isb).sum()), 3)) * dp
    bpos, fpos = pos[isb], pos[~isb]
    pos = np.concatenate([bpos, fpos], axis=0)
    nb = bpos.shape[0]
    vel = np.zeros((pos.shape[0], 3), dtype=np.float32)
    vel[nb:] = rng.uniform(-vel_range, vel_range,
                           size=(pos.shape[0] - nb, 3)).astype(np.float32)
    rho = (rho0 * rng.uniform(rho_range[0], rho_range[1],
                              size=pos.shape[0])).astype(np.float32)
    h = h_over_dp * dp
    dmin, dmax = domain_for(pos, h, float(pos[:, 2].max()),
                            float(np.ptp(pos[:, 2]) + dp))
    case = Case(name=f"random_block_{n}", pos=pos, vel=vel, rho=rho,
                ids=np.arange(pos.shape[0], dtype=np.uint32), n_bound=nb,
                dp=dp, h=h, rho0=rho0, c0=c0, alpha=alpha, cfl=cfl,
                gravity=(0.0, 0.0, -g), dmin=dmin, dmax=dmax,
                fluid_height=float(pos[:, 2].max()))
    return shuffle(case, seed + 1)


@dataclass
class Ensemble:
    """Independent dam breaks concatenated for a lockstep (batched) run.

    Member q owns the global ids [id_base[q], id_base[q+1]) (its own ids
    shifted, boundary particles first).  ``members`` holds the per-member
    inputs of the C ABI (domain, c0, counts, end time); ``params`` the shared
    constants (taken from member 0, which must agree with all others on dp,
    h, rho0, alpha, cfl, gravity and mass).
    """
    cases: list
    pos: np.ndarray
    vel: np.ndarray
    rho: np.ndarray
    ids: np.ndarray
    id_base: np.ndarray
    members: list
    params: dict

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    def member_slice(self, q):
        return slice(int(self.id_base[q]), int(self.id_base[q + 1]))


def ensemble(case_list, t_end=float("inf")) -> Ensemble:
    """Concatenate cases (same dp, h and physical constants except c0)."""
    base = [0]
    for c in case_list:
        base.append(base[-1] + c.n)
    pos = np.concatenate([c.pos for c in case_list])
    vel = np.concatenate([c.vel for c in case_list])
    rho = np.concatenate([c.rho for c in case_list])
    ids = np.concatenate([c.ids.astype(np.uint64) + b for c, b in zip(case_list, base)]
                         ).astype(np.uint32)
    members = [dict(dmin=c.dmin, dmax=c.dmax, c0=c.c0, n_particles=c.n, n_bound=c.n_bound,
                    t_end=t_end) for c in case_list]
    p = case_list[0].params()
    for c in case_list[1:]:
        q = c.params()
        for k in ("dp", "h", "rho0", "alpha", "cfl", "mass", "gravity", "eta2_coef",
                  "kernel", "integrator", "verlet_every"):
            if q[k] != p[k]:
                raise ValueError(f"ensemble members disagree on {k}")
    return Ensemble(cases=list(case_list), pos=pos, vel=vel, rho=rho, ids=ids,
                    id_base=np.array(base, dtype=np.int64), members=members, params=p)


def dam_break_ensemble(n_instances=256, seed=1017, dp=0.02, t_end=1.0) -> Ensemble:
    """The batched workload: n dam breaks, fluid block b_x, b_y, b_z drawn
    from U[0.2, 0.6] m (SplitMix64 ``seed``) in a 1.0 x b_y x 0.8 m tank, each
    run to ``t_end`` seconds."""
    specs = ensemble_specs(n_instances, seed=seed, dp=dp)
    return ensemble([ensemble_instance(s, dp=dp) for s in specs], t_end=t_end)
