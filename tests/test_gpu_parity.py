"""GPU path (through the C ABI) against the FP64 oracle, element by element.

Bars: bit-exact cell labels, (label, id) order, cell offsets and FP64-
predicate neighbour counts; per-particle density rates and accelerations
within a relative error of 2e-5 of the sum of the magnitudes of their pair
terms (the scale at which FP32 rounding of cancelling terms is judged, since
the plain relative error is undefined where the sum cancels, e.g. at the
free surface where p ~ 0); the step size and the integrator within bounds
derived from FP32 rounding of the increments.
"""
import json
import os

import numpy as np
import pytest

import __graft_entry__  # noqa: F401
import oracle
from paper_1210_1017_gb300 import cases
from paper_1210_1017_gb300 import sph as S

pytestmark = pytest.mark.gpu

REL_TOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()
    yield


def _case_list():
    return [
        ("random_64", lambda: cases.random_block(64, seed=7)),
        ("random_777", lambda: cases.random_block(777, seed=8, jitter=0.4)),
        ("random_2000", lambda: cases.random_block(2000, seed=9, jitter=0.3)),
        ("dam_break_6k", lambda: cases.c1_dam_break(shuffle_seed=3)),
        # h = 3 dp: ~200 particles per cell, so work units overflow the
        # shared-memory staging and take the global-memory path
        ("dense_h3dp", lambda: cases.random_block(3000, seed=5, h_over_dp=3.0, jitter=0.2)),
    ]


CASES = _case_list()


def _state(sim):
    st = sim.download()
    return st, oracle.State(st["pos"], st["vel"], st["rho"], st["ids"])


def _scaled(gpu, ref, scale):
    diff = np.abs(np.asarray(gpu, np.float64) - ref)
    if diff.ndim == 2:
        diff = np.linalg.norm(diff, axis=1)
    return diff / np.maximum(scale, 1e-300)


def _rates_ok(ace, ref, fluid):
    """Scaled errors: accelerations of fluid particles (boundary particles
    carry gravity only), density rates of all particles."""
    ea = _scaled(ace[fluid, :3], ref["a"][fluid], ref["sa"][fluid])
    ed = _scaled(ace[:, 3], ref["drho"], np.where(ref["sd"] > 0, ref["sd"], 1.0))
    gl_a = np.linalg.norm(ace[fluid, :3] - ref["a"][fluid]) / np.linalg.norm(ref["a"][fluid])
    return ea, ed, gl_a


# --- radix sort through the C ABI ------------------------------------------

def _gpu_sort(keys, vals, key_bits):
    import torch
    n = keys.size
    dev = torch.device("cuda", 0)
    kin = torch.from_numpy(keys.astype(np.uint32).view(np.int32)).to(dev)
    vin = None if vals is None else torch.from_numpy(vals.astype(np.uint32).view(np.int32)).to(dev)
    kout = torch.empty_like(kin)
    vout = torch.empty_like(kin)
    nb = int(S.lib().sph_radix_sort_scratch_bytes(n))
    scratch = torch.empty(nb, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    S.sph_radix_sort_pairs(kin, vin, kout, vout, n, key_bits, scratch, nb, stream.cuda_stream)
    stream.synchronize()
    return kout.cpu().numpy().view(np.uint32), vout.cpu().numpy().view(np.uint32)


def test_radix_sort_reproduces_paper_worked_example(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "radix_sort_halo_example.json")))
    k, v = _gpu_sort(np.array(g["halo"]), np.array(g["id"]), 2)
    assert k.tolist() == g["sorted_halo"]
    assert v.tolist() == g["sorted_id"]


@pytest.mark.parametrize("n,bits", [(1, 8), (4095, 12), (4097, 8), (100003, 17),
                                    (1 << 20, 24), (3000000, 32)])
def test_radix_sort_is_stable_and_matches_numpy(n, bits):
    rng = np.random.default_rng(n)
    keys = rng.integers(0, 1 << bits, n, dtype=np.uint64).astype(np.uint32)
    if n > 1000:
        keys[: n // 3] = np.sort(keys[: n // 3])       # long runs, as in the cell sort
    k, v = _gpu_sort(keys, None, bits)
    ref = np.argsort(keys, kind="stable")
    assert np.array_equal(v, ref.astype(np.uint32))
    assert np.array_equal(k, keys[ref])


# --- cell build: labels, order, offsets --------------------------------------

@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_cells_bit_exact(name, make):
    case = make()
    sim = S.Simulation.from_case(case)
    sim.build_cells()
    st = sim.download()
    keys = sim.read(S.SPH_ARRAY_KEY)
    off = sim.read(S.SPH_ARRAY_CELL_OFF)
    ref = oracle.Oracle(case.params()).build_cells(case.pos, case.ids)
    assert np.array_equal(st["ids"], ref["sorted_ids"])
    assert np.array_equal(keys, ref["sorted_key"])
    assert np.array_equal(off, ref["cell_off"])
    # the state moved with its particle
    assert np.array_equal(st["pos"], case.pos[ref["perm"]])
    assert np.array_equal(st["rho"], case.rho[ref["perm"]])
    sim.close()


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_neighbour_counts_fp64_bit_exact(name, make):
    case = make()
    sim = S.Simulation.from_case(case)
    sim.build_cells()
    got = sim.neighbour_counts_fp64()
    st = sim.download()
    ref = oracle.Oracle(case.params()).neighbour_counts(st["pos"], brute=case.n <= 2000)
    assert np.array_equal(got, ref)
    sim.close()


def test_fp32_counts_differ_only_at_the_support_edge():
    case = cases.random_block(2000, seed=12, jitter=0.45)
    sim = S.Simulation.from_case(case)
    sim.build_cells()
    sim.interact(counts=True)
    c32 = sim.read(S.SPH_ARRAY_NNB).astype(np.int64)
    st = sim.download()
    c64 = oracle.Oracle(case.params()).neighbour_counts(st["pos"], brute=True).astype(np.int64)
    d2 = ((st["pos"][:, None, :] - st["pos"][None, :, :]) ** 2).sum(-1)
    r2 = (2 * case.h) ** 2
    edge = (np.abs(d2 - r2) < 1e-6 * r2).sum(1)
    assert np.all(np.abs(c32 - c64) <= edge)
    sim.close()


# --- interaction -------------------------------------------------------------

@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_interaction_within_2e5(name, make):
    case = make()
    sim = S.Simulation.from_case(case)
    sim.build_cells()
    sim.interact()
    ace = sim.read(S.SPH_ARRAY_ACE)
    st, ost = _state(sim)
    ref = oracle.Oracle(case.params()).interact(ost, brute=case.n <= 2000)
    fluid = st["ids"] >= case.n_bound
    ea, ed, gl = _rates_ok(ace, ref, fluid)
    assert np.array_equal(ace[~fluid, :3], np.tile(np.float32(case.gravity), ((~fluid).sum(), 1)))
    print(f"{name}: max scaled |a| err {ea.max():.2e}, drho {ed.max():.2e}, global {gl:.2e}")
    assert ea.max() <= REL_TOL
    assert ed.max() <= REL_TOL
    assert gl <= REL_TOL
    # FP32 and FP64 predicates may disagree for pairs at |r_ij| = 2h
    # (their terms vanish there); the FP64 counts are compared bit for bit
    # in test_neighbour_counts_fp64_bit_exact
    d = sim.diagnostics()
    assert abs(d["pairs_last"] - int(ref["nnb"].sum())) <= 1e-4 * ref["nnb"].sum()
    assert abs(d["pairs_fluid_last"] - int(ref["nnb"][fluid].sum())) <= 1e-4 * ref["nnb"].sum()
    sim.close()


def test_interaction_with_moving_state_within_2e5():
    """A dam-break state after some steps (non-zero velocities, viscosity
    active), replayed into the oracle."""
    case = cases.c1_dam_break()
    sim = S.Simulation.from_case(case)
    sim.step(40)
    sim.interact()
    ace = sim.read(S.SPH_ARRAY_ACE)
    st, ost = _state(sim)
    ref = oracle.Oracle(case.params()).interact(ost)
    ea, ed, gl = _rates_ok(ace, ref, st["ids"] >= case.n_bound)
    print(f"moving: {ea.max():.2e} {ed.max():.2e} {gl:.2e}")
    assert ea.max() <= REL_TOL and ed.max() <= REL_TOL and gl <= REL_TOL
    sim.check()
    sim.close()


def test_step_size_matches_oracle():
    case = cases.c1_dam_break()
    sim = S.Simulation.from_case(case)
    sim.step(10)
    sim.interact()
    dt = sim.read(S.SPH_ARRAY_DT)[0]
    st, ost = _state(sim)
    ref = oracle.Oracle(case.params()).interact(ost)
    assert dt == pytest.approx(ref["dt"], rel=1e-5)
    d = sim.diagnostics()
    assert d["amax"] == pytest.approx(ref["terms"][0], rel=1e-5)
    assert d["cmax"] == pytest.approx(ref["terms"][1], rel=1e-6)
    assert d["mumax"] == pytest.approx(ref["terms"][2], rel=1e-5, abs=1e-9)
    sim.close()


# --- integrator --------------------------------------------------------------

def test_predictor_and_corrector_match_oracle():
    case = cases.random_block(1500, seed=21, jitter=0.3, vel_range=0.8)
    O = oracle.Oracle(case.params())
    sim = S.Simulation.from_case(case)
    sim.build_cells()
    sim.interact()
    s0, o0 = _state(sim)
    ace0 = sim.read(S.SPH_ARRAY_ACE).astype(np.float64)
    dt = float(sim.read(S.SPH_ARRAY_DT)[0])
    sim.predict()
    s1 = sim.download()
    oh = O.predict(o0.copy(), ace0[:, :3], ace0[:, 3], dt)
    disp = np.abs(oh.pos() - o0.pos()).max()
    print("predict errors", np.abs(s1["pos"] - oh.pos()).max() / disp,
          np.abs(s1["vel"] - oh.vel()).max(), np.abs(s1["rho"] - oh.rho).max())
    assert np.abs(s1["pos"] - oh.pos()).max() <= 1e-6 * disp + 1e-15
    assert np.abs(s1["vel"] - oh.vel()).max() <= 2e-7 * (np.abs(oh.vel()).max() + 1)
    assert np.abs(s1["rho"] - oh.rho).max() <= 1e-7 * oh.rho.max()
    sim.build_cells()
    sim.interact()
    h2, oh2 = _state(sim)
    ace1 = sim.read(S.SPH_ARRAY_ACE).astype(np.float64)
    # the start state, reordered like the half-step state
    pos0 = {int(i): k for k, i in enumerate(s0["ids"])}
    idx = np.array([pos0[int(i)] for i in h2["ids"]])
    pre = oracle.State(s0["pos"][idx], s0["vel"][idx], s0["rho"][idx], s0["ids"][idx])
    sim.correct()
    s2 = sim.download()
    assert float(sim.read(S.SPH_ARRAY_DT)[0]) == dt
    on = O.correct(pre, oh2.copy(), ace1[:, :3], ace1[:, 3], dt)
    disp = np.abs(on.pos() - pre.pos()).max()
    print("correct errors", np.abs(s2["pos"] - on.pos()).max() / disp,
          np.abs(s2["vel"] - on.vel()).max(), np.abs(s2["rho"] - on.rho).max())
    assert np.abs(s2["pos"] - on.pos()).max() <= 1e-6 * disp + 1e-15
    assert np.abs(s2["vel"] - on.vel()).max() <= 2e-7 * (np.abs(on.vel()).max() + 1)
    assert np.abs(s2["rho"] - on.rho).max() <= 2e-7 * on.rho.max()
    b = s2["ids"] < case.n_bound
    assert np.array_equal(s2["pos"][b], pre.pos()[b])
    sim.close()


def test_boundary_particles_never_move_and_mass_is_constant():
    case = cases.c1_dam_break()
    sim = S.Simulation.from_case(case)
    sim.step(30)
    st = sim.download()
    b = st["ids"] < case.n_bound
    ref = case.pos[st["ids"][b]]
    assert np.array_equal(st["pos"][b], ref)
    assert np.all(st["vel"][b] == 0)
    d = sim.diagnostics()
    assert d["mass"] == pytest.approx(case.n * case.mass, rel=1e-12)
    assert d["step"] == 30 and d["n_out"] == 0 and d["status"] == 0
    sim.close()


def test_excluded_particles_are_frozen_and_counted():
    case = cases.random_block(600, seed=30)
    pos = case.pos.copy()
    pos[5] = np.array(case.dmax) + 0.5
    pos[9, 2] = np.nan
    case.pos = pos
    sim = S.Simulation.from_case(case)
    sim.build_cells()
    off = sim.read(S.SPH_ARRAY_CELL_OFF)
    assert off[-2] == case.n - 2 and off[-1] == case.n
    sim.step(3)
    st = sim.download()
    k = {int(i): j for j, i in enumerate(st["ids"])}
    assert np.array_equal(st["pos"][k[int(case.ids[5])]], pos[5])
    assert sim.diagnostics()["n_out"] == 2
    sim.close()


# --- determinism and permutation invariance ----------------------------------

def test_two_runs_are_bit_identical_and_order_independent():
    a = cases.c1_dam_break(shuffle_seed=1)
    b = cases.c1_dam_break(shuffle_seed=2)
    out = []
    for case in (a, a, b):
        sim = S.Simulation.from_case(case)
        sim.step(25)
        st = sim.download()
        out.append((st, sim.read(S.SPH_ARRAY_ACE)))
        sim.close()
    for st, ace in out[1:]:
        assert np.array_equal(st["ids"], out[0][0]["ids"])
        assert np.array_equal(st["pos"], out[0][0]["pos"])
        assert np.array_equal(st["vel"], out[0][0]["vel"])
        assert np.array_equal(st["rho"], out[0][0]["rho"])
        assert np.array_equal(ace, out[0][1])


def test_graph_and_direct_launch_paths_agree():
    case = cases.c1_dam_break()
    import torch
    sims = [S.Simulation.from_case(case),
            S.Simulation.from_case(case, stream=torch.cuda.default_stream(0))]
    sts = []
    for sim in sims:
        sim.step(5)
        sts.append(sim.download())
        sim.close()
    assert np.array_equal(sts[0]["pos"], sts[1]["pos"])
    assert np.array_equal(sts[0]["rho"], sts[1]["rho"])


# --- trajectory report ---------------------------------------------------------

def test_dam_break_200_steps_tracks_the_oracle():
    """Free-running 200 steps of the 6,000-fluid-particle dam break, GPU
    versus FP64 oracle from the same start: the trajectories separate only
    by accumulated FP32 rounding (report; bar: RMS position difference below
    1e-3 dp and the same step sizes to 1e-4)."""
    case = cases.c1_dam_break()
    O = oracle.Oracle(case.params())
    ost = oracle.State.from_case(case)
    t_ref = 0.0
    for _ in range(200):
        dt, _ = O.step(ost)
        t_ref += dt
    sim = S.Simulation.from_case(case)
    sim.step(200)
    st = sim.download()
    d = sim.diagnostics()
    k = np.argsort(st["ids"])
    rms = np.sqrt(((st["pos"][k] - ost.pos()) ** 2).sum(1).mean())
    print(f"200 steps: t_gpu={d['t']:.6f} t_ref={t_ref:.6f} rms/dp={rms / case.dp:.3e}")
    assert d["t"] == pytest.approx(t_ref, rel=1e-4)
    assert rms < 1e-3 * case.dp
    sim.close()


def test_every_interaction_variant_is_within_2e5():
    case = cases.c1_dam_break(shuffle_seed=4)
    sim = S.Simulation.from_case(case)
    sim.step(10)
    st, ost = _state(sim)
    ref = oracle.Oracle(case.params()).interact(ost)
    fluid = st["ids"] >= case.n_bound
    results = []
    for v in range(S.sph_num_variants()):
        sim.set_variant(v)
        sim.interact()
        ace = sim.read(S.SPH_ARRAY_ACE)
        ea, ed, gl = _rates_ok(ace, ref, fluid)
        print(f"variant {v}: {ea.max():.2e} {ed.max():.2e} {gl:.2e}")
        assert ea.max() <= REL_TOL and ed.max() <= REL_TOL and gl <= REL_TOL
        results.append(ace)
    best, ms = S.sph_autotune(sim.ctx, 2)
    assert 0 <= best < S.sph_num_variants() and np.all(ms > 0)
    # the autotuner leaves the state alone
    st2 = sim.download()
    assert np.array_equal(st2["pos"], st["pos"])
    sim.close()


def test_device_step_loop_equals_single_step_graphs():
    """sph_step(n) runs its n steps in one launch (a CUDA graph whose
    conditional WHILE node repeats the step on the device); the result must
    be bit-identical to n launches of the single-step graph."""
    case = cases.c1_dam_break()
    a = S.Simulation.from_case(case)
    for _ in range(25):
        a.step(1)
    b = S.Simulation.from_case(case)
    b.step(25)
    sa, sb = a.download(), b.download()
    for key in ("ids", "pos", "vel", "rho"):
        assert np.array_equal(sa[key], sb[key])
    da, db = a.diagnostics(), b.diagnostics()
    assert da["step"] == db["step"] == 25 and da["t"] == db["t"]
    assert da["pairs_total"] == db["pairs_total"]
    # the loop graph is reused by the next call
    a.step(7)
    b.step(7)
    for key in ("pos", "vel", "rho"):
        assert np.array_equal(a.download()[key], b.download()[key])
    a.close()
    b.close()


def test_counter_scheduled_variants_equal_their_static_shapes():
    """The variants that take work units from a counter (and fetch the next
    unit's record and offsets during the current one) compute every unit as
    the round-robin variant of the same block shape does, so their rates are
    bit-identical.  Three launches in a row check that the last block rearms
    the counter (a stale counter would skip units)."""
    case = cases.c2_dam_break_obstacles(dp=0.012)     # ~330k particles: many units per block
    sim = S.Simulation.from_case(case)
    sim.step(20)
    nv = S.sph_num_variants()
    pairs = [(10, 13), (11, 14), (12, 15)]
    assert nv == 16
    for vs, vd in pairs:
        sim.set_variant(vs)
        sim.interact()
        ref = sim.read(S.SPH_ARRAY_ACE).copy()
        sim.set_variant(vd)
        for _ in range(3):
            sim.interact()
            sim.check()
            got = sim.read(S.SPH_ARRAY_ACE)
            assert np.array_equal(got, ref), (vs, vd)
    sim.close()


def test_upload_after_a_predict_or_correct_without_rebuild():
    """sph_predict / sph_correct count the new labels into the per-cell
    counts for the next rebuild.  When new state is uploaded instead, those
    counts must not carry over: the next step equals the same step on a
    fresh context, bit for bit (stale counts would double the cell sizes and
    misplace the scatter)."""
    case = cases.c1_dam_break(shuffle_seed=8)
    ref = S.Simulation.from_case(case)
    ref.step(3)
    want = ref.download()
    for stop in ("predict", "correct"):
        sim = S.Simulation.from_case(case)
        sim.step(2)
        sim.build_cells()
        sim.interact()
        sim.predict()
        if stop == "correct":
            sim.build_cells()
            sim.interact()
            sim.correct()
        sim.check()
        # the pending counts are dropped by the upload; the same for the
        # pipelined upload
        sim.upload(case.pos, case.vel, case.rho, case.ids)
        sim.step(3)
        sim.check()
        got = sim.download()
        for key in ("ids", "pos", "vel", "rho"):
            assert np.array_equal(got[key], want[key]), (stop, key)
        sim.enable_async_transfers()
        sim.build_cells()
        sim.interact()
        sim.predict()
        S.sph_upload_async(sim.ctx, np.ascontiguousarray(case.pos, np.float64),
                           np.ascontiguousarray(case.vel, np.float32),
                           np.ascontiguousarray(case.rho, np.float32),
                           np.ascontiguousarray(case.ids, np.uint32))
        S.sph_sync_transfers(sim.ctx)
        sim.step(3)
        sim.check()
        got = sim.download()
        for key in ("ids", "pos", "vel", "rho"):
            assert np.array_equal(got[key], want[key]), (stop, "async", key)
        sim.close()
    ref.close()
