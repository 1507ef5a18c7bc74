"""The interaction's work units (Sec. 3.2: runs of sorted particles of one
row of cells) built in one launch (k_units_fused: row sums in shared memory,
a look-back over rows) equal the list built by row sums, counts, a scan and
the fill as separate launches (SPH_UNITS_FUSED=0 at context creation), bit
for bit, and both tile the particles of the cells exactly."""
import os

import numpy as np
import pytest

import __graft_entry__
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


def _pair(make):
    one = make()
    os.environ["SPH_UNITS_FUSED"] = "0"
    try:
        many = make()
    finally:
        del os.environ["SPH_UNITS_FUSED"]
    return one, many


def _check_tiling(sim, units, ncx=None):
    off = sim.read(S.SPH_ARRAY_CELL_OFF)
    n_in = int(off[-2])
    assert units.shape[0] > 0
    first, end = units[:, 0].astype(np.int64), units[:, 1].astype(np.int64)
    assert first[0] == 0 and end[-1] == n_in
    assert np.all(end > first)
    assert np.array_equal(end[:-1], first[1:])          # contiguous, in order
    assert np.all(end - first <= 128)                    # at most 4 warps of particles
    if ncx is not None:
        key = sim.read(S.SPH_ARRAY_KEY).astype(np.int64)
        assert np.array_equal(key[first] // ncx, key[end - 1] // ncx)   # one row each


def test_one_launch_unit_list_equals_the_multi_launch_list():
    case = cases.c1_dam_break()
    one, many = _pair(lambda: S.Simulation.from_case(case))
    # one launch instead of row sums, counts, scan (one block here) and fill
    assert one.kernels_per_step() + 2 * 3 == many.kernels_per_step()
    with pytest.raises(S.SphError, match="SPH_ERR_STATE"):
        one.units()                                      # no cells yet
    ncx = int(one.sizes.ncx)
    for steps in (0, 40, 160):
        for sim in (one, many):
            if steps:
                sim.step(steps)
            else:
                sim.build_cells()
            sim.check()
        u1, u2 = one.units(), many.units()
        assert np.array_equal(u1, u2), steps
        _check_tiling(one, u1, ncx)
        assert np.array_equal(one.download()["pos"], many.download()["pos"])
    # another block shape cuts other units; the two builders still agree
    for v in (0, S.sph_num_variants() - 1):
        one.set_variant(v)
        many.set_variant(v)
        u1, u2 = one.units(), many.units()
        assert np.array_equal(u1, u2), v
        _check_tiling(one, u1, ncx)
    one.close()
    many.close()


def test_one_launch_unit_list_of_an_ensemble():
    members = [cases.ensemble_instance(s) for s in cases.ensemble_specs(3, seed=11)]
    ens = cases.ensemble(members)
    one, many = _pair(lambda: S.Simulation.from_ensemble(ens))
    for sim in (one, many):
        sim.step(30)
        sim.check()
    u1, u2 = one.units(), many.units()
    assert np.array_equal(u1, u2)
    _check_tiling(one, u1)
    one.close()
    many.close()


def test_forked_unit_list_equals_the_serial_one():
    """Each rebuild builds the unit list on a second stream, beside the cell
    scatter and the reorder, and joins it before the interaction; a context
    created with SPH_FORK_UNITS=0 builds it in line.  Both give the same
    steps, bit for bit, in the device loop and call by call."""
    import os
    case = cases.c1_dam_break(shuffle_seed=12)
    forked = S.Simulation.from_case(case)
    os.environ["SPH_FORK_UNITS"] = "0"
    try:
        serial = S.Simulation.from_case(case)
    finally:
        del os.environ["SPH_FORK_UNITS"]
    for sim in (forked, serial):
        sim.step(20)
        sim.build_cells()
        sim.interact()
        sim.predict()
        sim.build_cells()
        sim.interact()
        sim.correct()
        sim.step(1)
        sim.check()
    a, b = forked.download(), serial.download()
    for key in ("ids", "pos", "vel", "rho"):
        assert np.array_equal(a[key], b[key])
    assert np.array_equal(forked.units(), serial.units())
    forked.close()
    serial.close()
