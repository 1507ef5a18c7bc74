"""Pipelined host transfers (sph_upload_async / sph_download_async on the
context's two copy streams) against the synchronous sph_upload /
sph_download: the same states, bit for bit, and the id check resolved at the
sync point."""
import numpy as np
import pytest

import __graft_entry__  # noqa: F401
from paper_1210_1017_gb300 import cases
from paper_1210_1017_gb300 import sph as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()
    return t


def test_pipelined_rounds_equal_synchronous_rounds(torch):
    case = cases.c1_dam_break(shuffle_seed=3)
    n = case.n
    ref = S.Simulation.from_case(case)
    sim = S.Simulation.from_case(case)
    sim.enable_async_transfers()
    pin = dict(pos=torch.from_numpy(np.ascontiguousarray(case.pos)).pin_memory(),
               vel=torch.from_numpy(np.ascontiguousarray(case.vel)).pin_memory(),
               rho=torch.from_numpy(np.ascontiguousarray(case.rho)).pin_memory(),
               ids=torch.from_numpy(np.ascontiguousarray(case.ids).view(np.int32)).pin_memory())
    rounds = 4
    outs = [dict(pos=torch.empty((n, 3), dtype=torch.float64).pin_memory(),
                 vel=torch.empty((n, 3), dtype=torch.float32).pin_memory(),
                 rho=torch.empty(n, dtype=torch.float32).pin_memory(),
                 ids=torch.empty(n, dtype=torch.int32).pin_memory()) for _ in range(rounds)]
    # round k: the case's state again, k + 1 steps, the result back; nothing
    # waits in between, so uploads and downloads overlap the steps
    for k in range(rounds):
        S.sph_upload_async(sim.ctx, pin["pos"], pin["vel"], pin["rho"], pin["ids"])
        sim.step(k + 1)
        o = outs[k]
        S.sph_download_async(sim.ctx, o["pos"], o["vel"], o["rho"], o["ids"])
    S.sph_sync_transfers(sim.ctx)
    sim.check()
    for k in range(rounds):
        ref.upload(case.pos, case.vel, case.rho, case.ids)
        ref.step(k + 1)
        want = ref.download()
        o = outs[k]
        assert np.array_equal(o["ids"].numpy().view(np.uint32), want["ids"]), k
        for key in ("pos", "vel", "rho"):
            assert np.array_equal(o[key].numpy(), want[key]), (k, key)
    # the id check of the pipelined upload was read at the sync point
    got = []
    for s_ in (ref, sim):
        arrs = (np.empty((n, 3), np.float64), np.empty((n, 3), np.float32), np.empty(n, np.float32))
        s_.download_by_id(*arrs)
        got.append(arrs)
    for x, y in zip(*got):
        assert np.array_equal(x, y)
    ref.close()
    sim.close()


def test_pipelined_calls_need_the_staging_buffer(torch):
    case = cases.random_block(500, seed=9)
    sim = S.Simulation.from_case(case)
    pos = np.ascontiguousarray(case.pos)
    with pytest.raises(S.SphError, match="SPH_ERR_STATE"):
        S.sph_upload_async(sim.ctx, pos, case.vel, case.rho, case.ids)
    with pytest.raises(S.SphError, match="SPH_ERR_STATE"):
        S.sph_download_async(sim.ctx, pos)
    nb = S.sph_async_transfer_bytes(sim.ctx)
    assert nb >= 44 * case.n * 3
    small = torch.empty(nb - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(S.SphError, match="SPH_ERR_WORKSPACE"):
        S.sph_enable_async_transfers(sim.ctx, small, nb - 256)
    sim.close()
