"""Failure detection on the GPU without a fault: a bounded device wait (the
radix sort's decoupled look-back) runs against a predecessor that never
publishes, gives up after a short poll limit, and reports SPH_ERR_TIMEOUT
through the context's status word; the context then keeps working."""
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


def test_selftest_rejects_an_unbounded_poll_count():
    sim = S.Simulation.from_case(cases.random_block(200, seed=4))
    for polls in (0, (1 << 20) + 1):
        with pytest.raises(S.SphError, match="SPH_ERR_INVALID_ARG"):
            S.sph_selftest_timeout(sim.ctx, polls)
    sim.check()
    sim.close()
