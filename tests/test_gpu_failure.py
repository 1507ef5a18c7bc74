"""Failure detection on the GPU without a fault: a bounded device wait (the
radix sort's decoupled look-back, or the unit list's look-back over rows)
runs against a predecessor that never publishes, gives up after a short poll
limit, and reports SPH_ERR_TIMEOUT through the context's status word; the
context then keeps working."""
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


def test_bounded_wait_gives_up_reports_timeout_and_the_context_recovers():
    case = cases.c1_dam_break()
    sim = S.Simulation.from_case(case)
    sim.step(3)
    before = sim.download()
    sim.check()
    S.sph_selftest_timeout(sim.ctx, 1000)
    with pytest.raises(S.SphError, match="SPH_ERR_TIMEOUT"):
        sim.check()
    assert sim.diagnostics()["status"] & 1
    after = sim.download()
    for key in ("ids", "pos", "vel", "rho"):
        assert np.array_equal(before[key], after[key])
    # the bit stays until cleared; then the run goes on as if nothing happened
    with pytest.raises(S.SphError, match="SPH_ERR_TIMEOUT"):
        sim.check()
    sim.clear_status()
    sim.check()
    sim.step(3)
    sim.check()
    got = sim.download()
    sim.close()
    ref = S.Simulation.from_case(case)
    ref.step(6)
    want = ref.download()
    ref.close()
    for key in ("ids", "pos", "vel", "rho"):
        assert np.array_equal(got[key], want[key])


def test_row_lookback_gives_up_reports_timeout_and_the_context_recovers():
    """The same for the one-launch unit list's bounded look-back over rows."""
    case = cases.c1_dam_break()
    sim = S.Simulation.from_case(case)
    sim.step(3)
    before = sim.download()
    units = sim.units()
    sim.check()
    S.sph_units_selftest_timeout(sim.ctx, 1000)
    with pytest.raises(S.SphError, match="SPH_ERR_TIMEOUT"):
        sim.check()
    after = sim.download()
    for key in ("ids", "pos", "vel", "rho"):
        assert np.array_equal(before[key], after[key])
    assert np.array_equal(units, sim.units())
    sim.clear_status()
    sim.step(3)
    sim.check()
    got = sim.download()
    sim.close()
    ref = S.Simulation.from_case(case)
    ref.step(6)
    want = ref.download()
    ref.close()
    for key in ("ids", "pos", "vel", "rho"):
        assert np.array_equal(got[key], want[key])
    for polls in (0, (1 << 20) + 1):
        s2 = S.Simulation.from_case(cases.random_block(200, seed=4))
        with pytest.raises(S.SphError, match="SPH_ERR_INVALID_ARG"):
            S.sph_units_selftest_timeout(s2.ctx, polls)
        s2.close()


def test_selftest_rejects_an_unbounded_poll_count():
    sim = S.Simulation.from_case(cases.random_block(200, seed=4))
    for polls in (0, (1 << 20) + 1):
        with pytest.raises(S.SphError, match="SPH_ERR_INVALID_ARG"):
            S.sph_selftest_timeout(sim.ctx, polls)
    sim.check()
    sim.close()


def test_standalone_sort_reports_a_lookback_that_gave_up():
    """sph_radix_sort_pairs keeps its look-back flag in the caller's scratch:
    sph_radix_sort_status reads it (OK after a good sort, SPH_ERR_TIMEOUT
    after the self-test made the bounded wait run out, OK again once the
    next sort has cleared it)."""
    import torch
    L = S.lib()
    n = 50000
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(3)
    keys = rng.integers(0, 1 << 16, n, dtype=np.uint64).astype(np.uint32)
    kin = torch.from_numpy(keys.view(np.int32)).cuda()
    kout, vout = torch.empty_like(kin), torch.empty_like(kin)
    nb = int(L.sph_radix_sort_scratch_bytes(n))
    scratch = torch.empty(nb, dtype=torch.uint8, device="cuda")
    S.sph_radix_sort_pairs(kin, None, kout, vout, n, 16, scratch, nb, stream.cuda_stream)
    S.sph_radix_sort_status(scratch, nb, n, stream.cuda_stream)
    S.sph_radix_sort_selftest_timeout(scratch, nb, n, 500, stream.cuda_stream)
    with pytest.raises(S.SphError, match="SPH_ERR_TIMEOUT"):
        S.sph_radix_sort_status(scratch, nb, n, stream.cuda_stream)
    S.sph_radix_sort_pairs(kin, None, kout, vout, n, 16, scratch, nb, stream.cuda_stream)
    S.sph_radix_sort_status(scratch, nb, n, stream.cuda_stream)
    stream.synchronize()
    order = np.argsort(keys, kind="stable").astype(np.uint32)
    assert np.array_equal(vout.cpu().numpy().view(np.uint32), order)


def test_rollout_stops_at_the_save_boundary_where_the_status_is_set():
    """A non-finite density makes the interaction flag SPH_STATUS_NONFINITE;
    sph_rollout reads the status word at its first save boundary and
    returns the error before calling the snapshot callback.  (The NaN
    spreads and pushes the particles out of the domain; once none is left
    the CFL step h / (c_max + mu_max) is infinite, as in the oracle, the
    member reaches its end time and stops counting steps.)"""
    case = cases.random_block(500, seed=21)
    sim = S.Simulation.from_case(case)
    rho = case.rho.copy()
    rho[17] = np.nan
    sim.upload(case.pos, case.vel, rho, case.ids)
    calls = []
    with pytest.raises(S.SphError, match="SPH_ERR_NONFINITE"):
        sim.rollout(10, save_every=5, cb=lambda s, t: calls.append(s))
    assert calls == []
    assert 1 <= sim.diagnostics()["step"] <= 5
    sim.clear_status()
    sim.close()
    # a clean rollout calls back at every boundary and returns normally
    sim = S.Simulation.from_case(case)
    calls = []
    sim.rollout(10, save_every=5, cb=lambda s, t: calls.append(s))
    assert calls == [5, 10]
    sim.close()
