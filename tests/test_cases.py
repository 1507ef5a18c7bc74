"""The seeded input generator: particle counts of the dam-break workloads
(closed forms of the open two-layer tank), lattice placement, obstacle
placement, the ensemble's seeded block sizes, the grid-domain rule, and the
SplitMix64 stream against its published first outputs."""
import numpy as np
import pytest

from paper_1210_1017_gb300 import cases


def test_splitmix64_matches_its_published_outputs():
    # first outputs of SplitMix64 (Steele, Lea, Flood 2014) from state 0
    it = cases.splitmix64_stream(0)
    assert next(it) == 0xE220A8397B1DCDAF
    assert next(it) == 0x6E789E6AA1B965F4
    u = cases.SplitMix64(1017)
    xs = [u.u01() for _ in range(1000)]
    assert 0.0 <= min(xs) and max(xs) < 1.0 and abs(np.mean(xs) - 0.5) < 0.03


def _tank_count(nx, ny, nz, layers=2):
    """Open two-layer tank around nx x ny x nz interior sites: two full floor
    layers plus, for every interior height, the ring outside the walls."""
    full = (nx + 2 * layers) * (ny + 2 * layers)
    return layers * full + nz * (full - nx * ny)


def test_dam_break_6k_counts_and_lattice():
    c = cases.c1_dam_break()
    assert c.n_fluid == 20 * 20 * 15 == 6000
    assert c.n_bound == _tank_count(50, 20, 30) == 11472
    assert c.n == 17472
    assert np.array_equal(c.ids, np.arange(c.n))              # boundary first
    f, b = c.pos[c.n_bound:], c.pos[:c.n_bound]
    # fluid on the (i + 1/2) dp lattice inside the 0.4 x 0.4 x 0.3 m block
    site = f / c.dp - 0.5
    assert np.allclose(site, np.round(site), atol=1e-9)
    assert f.min() > 0 and f[:, 0].max() < 0.4 and f[:, 1].max() < 0.4 and f[:, 2].max() < 0.3
    # boundary particles outside the interior (floor below z = 0 or walls)
    inside = ((b[:, 0] > 0) & (b[:, 0] < 1.0) & (b[:, 1] > 0) & (b[:, 1] < 0.4) & (b[:, 2] > 0))
    assert not inside.any()
    assert np.isclose(b[:, 2].min(), -1.5 * c.dp) and np.isclose(b[:, 0].min(), -1.5 * c.dp)
    # at rest, with the mass of rho0 dp^3
    assert np.all(c.vel == 0) and c.mass == pytest.approx(1000.0 * 0.02 ** 3)
    assert c.c0 == pytest.approx(10 * np.sqrt(9.81 * 0.3))


def test_grid_domain_rule():
    c = cases.c1_dam_break()
    cs = 2 * c.h
    assert np.allclose(c.dmin, c.pos.min(0) - cs)
    top = max(c.pos[:, 2].max(), 0.6 + 0.3)                   # tank rim + half its height
    assert np.allclose(c.dmax, [c.pos[:, 0].max() + cs, c.pos[:, 1].max() + cs, top + cs])


def test_dam_break_with_obstacles_counts_and_placement():
    c = cases.c2_dam_break_obstacles()
    assert c.n_fluid == 1008032 and c.n_bound == 383428 and c.n == 1391460
    obs = c.meta["obstacles"]
    assert len(obs) == 3
    dp = c.dp
    for (i0, j0, nx, ny, nz) in obs:
        assert (nx, ny, nz) == (14, 14, 27)                    # 0.1 x 0.1 x 0.2 m at 7.33 mm
        assert 1.4 - dp <= i0 * dp and (i0 + nx) * dp <= 2.8 + dp
        assert 0.1 - dp <= j0 * dp and (j0 + ny) * dp <= 0.9 + dp
    for a in range(3):
        for b in range(a + 1, 3):
            (i0, j0, nx, ny, _), (i1, j1, _, _, _) = obs[a], obs[b]
            assert i0 + nx + 2 <= i1 or i1 + nx + 2 <= i0 or j0 + ny + 2 <= j1 or j1 + ny + 2 <= j0
    # the fluid block (x < 0.8 m) does not reach the obstacles: no fluid inside them
    f = c.pos[c.n_bound:]
    for (i0, j0, nx, ny, nz) in obs:
        inside = ((f[:, 0] > i0 * dp) & (f[:, 0] < (i0 + nx) * dp) & (f[:, 1] > j0 * dp)
                  & (f[:, 1] < (j0 + ny) * dp) & (f[:, 2] < nz * dp))
        assert not inside.any()
    # seeded: the same placement every time
    assert cases.c2_dam_break_obstacles().meta["obstacles"] == obs


def test_ensemble_sizes_from_the_seed():
    specs = cases.ensemble_specs(256, seed=1017)
    s = np.array(specs)
    assert s.shape == (256, 3) and s.min() >= 0.2 and s.max() < 0.6
    assert cases.ensemble_specs(256, seed=1017) == specs
    ens = cases.dam_break_ensemble(256, t_end=1.0)
    sizes = [m.n for m in ens.cases]
    assert ens.n == sum(sizes) == 5467022
    assert min(sizes) == 13052 and max(sizes) == 37296
    # members own consecutive id ranges, boundary particles first in each
    assert np.array_equal(np.sort(ens.ids), np.arange(ens.n))
    for q in (0, 100, 255):
        lo = ens.id_base[q]
        m = ens.cases[q]
        assert ens.members[q]["n_bound"] == m.n_bound and ens.members[q]["n_particles"] == m.n
        assert lo + m.n == ens.id_base[q + 1]


def test_dam_break_32m_counts():
    c = cases.c3_dam_break_32m()
    assert c.n_fluid == 350 * 350 * 263 == 32217500
    assert c.n_bound == _tank_count(877, 351, 526) == 3217638
    assert c.n == 35435138
    cells = np.prod([np.ceil((hi - lo) / (2 * c.h)) for lo, hi in zip(c.dmin, c.dmax)])
    assert cells == 341 * 139 * 307 and cells < 2 ** 24       # a 24-bit cell label


def test_shuffle_keeps_particles_with_their_ids():
    a = cases.c1_dam_break()
    b = cases.c1_dam_break(shuffle_seed=3)
    k = np.argsort(b.ids)
    assert np.array_equal(b.pos[k], a.pos) and np.array_equal(b.rho[k], a.rho)
    assert not np.array_equal(b.ids, a.ids)
