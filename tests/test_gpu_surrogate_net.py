"""The surrogate network through the C ABI (graph, forward, backward, Adam,
integration step) against the FP64 reference of oracle/sur_oracle.py on the
same seeded particles and weights, with the reference rounding to bfloat16
wherever the GPU stores bfloat16."""
import numpy as np
import pytest

import __graft_entry__  # noqa: F401
from oracle import sur_oracle as so
from paper_1210_1017_gb300 import cases
from paper_1210_1017_gb300 import sph as S
from paper_1210_1017_gb300 import surrogate as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()
    return t


class Setup:
    """A jittered particle block on the GPU with a random velocity history,
    and the same data by particle id for the reference."""

    def __init__(self, torch, n, layers, seed=0, train=True, v_scale=0.5):
        self.case = c = cases.random_block(n, seed=seed + 21, jitter=0.3)
        self.layers = layers
        self.sim = S.Simulation.from_case(c)
        self.sim.build_cells()
        rng = np.random.default_rng(seed)
        self.n = c.n
        order = np.argsort(c.ids)
        self.pos = c.pos[order]                       # by id
        self.bnd = np.arange(c.n) < c.n_bound
        self.hist = rng.normal(0, 0.4, (c.n, 15)).astype(np.float32)
        self.hist[self.bnd] = 0
        self.target = rng.normal(0, 1.0, (c.n, 3)).astype(np.float32)
        self.d_hist = torch.tensor(self.hist, device="cuda")
        self.d_target = torch.tensor(self.target, device="cuda")
        self.v_scale = v_scale
        self.sur = U.Surrogate(self.sim, layers=layers, train=train, v_scale=v_scale)
        self.w = so.init_params(layers, seed=seed + 5)
        self.sur.set_params(self.w)
        self.src, self.dst = so.graph(self.pos, c.h)
        self.xn = so.node_features(self.hist, self.bnd, np.float32(v_scale))
        self.xe = so.edge_features(self.pos, c.h, self.src, self.dst)

    def gpu_forward(self, torch):
        acc = torch.zeros((self.n, 3), dtype=torch.float32, device="cuda")
        self.sur.forward(self.d_hist, acc)
        self.sim.synchronize()
        return acc.cpu().numpy().astype(np.float64)

    def ref(self, bf16=True):
        return so.forward_backward(self.w, self.layers, self.xn, self.xe, self.src, self.dst,
                                   self.target, ~self.bnd, bf16=bf16)


def _cos(a, b):
    a, b = a.ravel(), b.ravel()
    return float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("n,layers", [(700, 1), (2000, 2), (2000, 10)])
def test_graph_and_forward_match_reference(torch, n, layers):
    s = Setup(torch, n, layers, seed=n + layers)
    got = s.gpu_forward(torch)
    # the graph: the same FP64 predicate, so the same ordered pairs; the GPU's
    # CSR rows are in cell order, mapped to particle ids here
    assert s.sur.num_edges == len(s.src)
    rowptr, col = s.sur.read_graph()
    ids = s.sim.download()["ids"].astype(np.int64)
    g_src = ids[np.repeat(np.arange(s.n), np.diff(rowptr.astype(np.int64)))]
    g_dst = ids[col.astype(np.int64)]
    order = np.lexsort((g_dst, g_src))
    assert np.array_equal(g_src[order], s.src)
    assert np.array_equal(g_dst[order], s.dst)
    out, _, _ = s.ref(bf16=True)
    ref = out[:, :3]
    assert _cos(got, ref) >= 0.9999, _cos(got, ref)
    assert _rel(got, ref) <= 1e-2, _rel(got, ref)
    # element by element against a per-row scale: the row's largest
    # component, floored at the median of those over rows (rows whose
    # output nearly vanishes are judged at the typical output size).  The
    # reference rounds to bfloat16 at the same points, but an FP32 sum in
    # another order can round the other way (one bf16 step, 2^-8 relative)
    # and that difference propagates through the later layers.  Up to two
    # layers all but 0.1% of the elements are within 1e-2 of their row's
    # scale; at ten layers the flips compound (measured: 99.9% within
    # 1.7e-2, 99% within 1.3e-2), so the 99.9% bar there is 2.5e-2; no
    # element beyond 3e-2 at any depth
    row = np.abs(ref).max(axis=1)
    scale = np.maximum(row, np.median(row))
    e = (np.abs(got - ref) / scale[:, None]).ravel()
    print(f"n={n} layers={layers}: per-row scaled element error max {e.max():.2e}, "
          f"99.9% {np.quantile(e, 0.999):.2e}, 99% {np.quantile(e, 0.99):.2e}")
    assert np.quantile(e, 0.999) <= (1e-2 if layers <= 2 else 2.5e-2)
    assert e.max() <= 3e-2
    # the bf16 storage error itself, for the record (FP64 without rounding)
    out64, _, _ = s.ref(bf16=False)
    assert _rel(got, out64[:, :3]) <= 5e-2


@pytest.mark.parametrize("n,layers", [(1500, 1), (2000, 3), (2000, 10)])
def test_backward_matches_reference_gradients(torch, n, layers):
    s = Setup(torch, n, layers, seed=3 * n + layers)
    s.gpu_forward(torch)
    loss = s.sur.backward(s.d_target)
    g = s.sur.grads().astype(np.float64)
    _, lref, gref = s.ref(bf16=True)
    assert abs(loss - lref) <= 1e-2 * lref, (loss, lref)
    assert _cos(g, gref) >= 0.9999, _cos(g, gref)
    o = 0
    for name, ki, ko, has_b in so.layer_shapes(layers):
        for part, size in (("W", ki * ko), ("b", ko if has_b else 0)):
            if size == 0:
                continue
            a, b = g[o:o + size], gref[o:o + size]
            o += size
            if np.linalg.norm(b) < 1e-6 * np.linalg.norm(gref):
                continue
            assert _rel(a, b) <= 3e-2, (name, part, _rel(a, b))
    assert o == len(g)


def test_inference_context_gives_the_training_forward(torch):
    s = Setup(torch, 1800, 4, seed=9)
    a = s.gpu_forward(torch)
    inf = U.Surrogate(s.sim, layers=4, train=False, v_scale=s.v_scale)
    inf.set_params(s.w)
    acc = torch.zeros((s.n, 3), dtype=torch.float32, device="cuda")
    inf.forward(s.d_hist, acc)
    s.sim.synchronize()
    assert np.array_equal(acc.cpu().numpy().astype(np.float64), a)
    # and repeated calls are deterministic
    assert np.array_equal(s.gpu_forward(torch), a)


def test_adam_step_matches_reference(torch):
    s = Setup(torch, 900, 1, seed=4)
    s.gpu_forward(torch)
    s.sur.backward(s.d_target)
    g = s.sur.grads().astype(np.float64)
    w0 = s.sur.params().astype(np.float64)
    lr = 1e-3
    s.sur.adam(lr)
    w1 = s.sur.params().astype(np.float64)
    ref, m, v = so.adam(w0, g, np.zeros_like(g), np.zeros_like(g), 1, lr)
    assert np.abs(w1 - ref).max() <= 1e-5 * lr + 2e-7 * np.abs(w0).max()
    # second step with fresh gradients
    s.gpu_forward(torch)
    s.sur.backward(s.d_target)
    g2 = s.sur.grads().astype(np.float64)
    s.sur.adam(lr)
    w2 = s.sur.params().astype(np.float64)
    ref2, _, _ = so.adam(w1, g2, m, v, 2, lr)
    assert np.abs(w2 - ref2).max() <= 1e-5 * lr + 2e-7 * np.abs(w1).max()


def test_advance_is_semi_implicit_euler_and_shifts_history(torch):
    dt = 2e-3
    s = Setup(torch, 1200, 2, seed=6)
    sur = U.Surrogate(s.sim, layers=2, train=False, v_scale=s.v_scale,
                      a_mean=(0.1, -0.2, -9.81), a_std=(2.0, 3.0, 4.0), dt_s=dt)
    sur.set_params(s.w)
    acc = torch.zeros((s.n, 3), dtype=torch.float32, device="cuda")
    sur.forward(s.d_hist, acc)
    s.sim.synchronize()
    acc = acc.cpu().numpy()
    before = s.sim.download()
    hist = s.d_hist.clone()
    sur.advance(hist)
    after = s.sim.download()
    ob, oa = np.argsort(before["ids"]), np.argsort(after["ids"])
    pb, vb = before["pos"][ob], before["vel"][ob].astype(np.float64)
    pa, va = after["pos"][oa], after["vel"][oa].astype(np.float64)
    fluid = ~s.bnd
    # the denormalised output is out * a_std + a_mean of the plain forward
    out, _, _ = s.ref(bf16=True)
    want_acc = out[:, :3] * np.array([2.0, 3.0, 4.0]) + np.array([0.1, -0.2, -9.81])
    assert _rel(acc, want_acc) <= 1e-2
    pw, vw = so.euler_step(pb, vb, acc.astype(np.float64), fluid, dt)
    # the GPU keeps velocities in FP32 and positions in FP64: v is off by its
    # rounding, r by that rounding times dt
    ulp = 2.0 ** -23 * (np.abs(vw).max() + 1)
    np.testing.assert_allclose(va, vw, rtol=0, atol=2 * ulp)
    np.testing.assert_allclose(pa, pw, rtol=0, atol=2 * ulp * dt + 1e-12)
    assert np.all(np.abs((pa - pb)[fluid] - va[fluid] * dt) <= ulp * dt + 1e-12)
    assert np.array_equal(pa[s.bnd], pb[s.bnd]) and np.array_equal(va[s.bnd], vb[s.bnd])
    h = hist.cpu().numpy()
    assert np.array_equal(h[:, :12], s.hist[:, 3:])
    assert np.array_equal(h[fluid, 12:], after["vel"][oa][fluid])
    assert np.all(h[s.bnd, 12:] == 0)
    # the cells are stale until rebuilt; the next call needs them
    with pytest.raises(S.SphError):
        sur.forward(hist, None)
    s.sim.build_cells()
    sur.forward(hist, None)


def test_training_reduces_the_loss_on_a_learnable_target(torch):
    s = Setup(torch, 1500, 2, seed=8)
    # a smooth function of the inputs: the newest velocity, scaled
    tgt = (0.5 * s.hist[:, 12:15] / s.v_scale).astype(np.float32)
    d_t = torch.tensor(tgt, device="cuda")
    losses = []
    for _ in range(150):
        s.sur.forward(s.d_hist, None)
        losses.append(s.sur.backward(d_t))
        s.sur.adam(1e-3)
    assert np.isfinite(losses).all()
    assert losses[-1] < 0.1 * losses[0], (losses[0], losses[-1])


def test_errors_are_reported_not_faulted(torch):
    s = Setup(torch, 600, 1, seed=2, train=False)
    with pytest.raises(S.SphError, match="STATE"):
        s.sur.backward(s.d_target)          # inference context
    small = U.Surrogate(s.sim, layers=1, max_edges=100, v_scale=1.0)
    with pytest.raises(S.SphError, match="CAPACITY"):
        small.forward(s.d_hist, None)
    with pytest.raises(S.SphError, match="INVALID_ARG"):
        U.sur_set_params(s.sur.ctx, np.zeros(5, np.float32))


def _frames(s, rng, dt):
    """Seven frames by id: ballistic motion with a per-particle acceleration
    (boundary particles fixed)."""
    v0 = rng.normal(0, 0.3, (s.n, 3))
    a0 = rng.normal(0, 5.0, (s.n, 3))
    v0[s.bnd] = 0
    a0[s.bnd] = 0
    t = (np.arange(7) - 5) * dt
    return s.pos[None] + v0[None] * t[:, None, None] + 0.5 * a0[None] * t[:, None, None] ** 2


def test_make_sample_without_noise_is_the_finite_difference_definition(torch):
    dt = 1e-3
    s = Setup(torch, 1500, 1, seed=12)
    sur = U.Surrogate(s.sim, layers=1, train=False, v_scale=1.0, a_mean=(0.5, -1.0, 2.0),
                      a_std=(3.0, 2.0, 4.0), dt_s=dt, max_edges=1)
    fr = _frames(s, np.random.default_rng(1), dt)
    d_fr = torch.tensor(fr, device="cuda")
    pos = torch.empty((s.n, 3), dtype=torch.float64, device="cuda")
    vel = torch.empty((s.n, 3), dtype=torch.float32, device="cuda")
    hist = torch.empty((s.n, 15), dtype=torch.float32, device="cuda")
    tgt = torch.empty((s.n, 3), dtype=torch.float32, device="cuda")
    sur.make_sample(d_fr, 0.0, 7, pos, vel, hist, tgt)
    torch.cuda.synchronize()
    v = (fr[1:6] - fr[0:5]) / dt                       # v^{k-4} .. v^k
    a = (fr[6] - 2 * fr[5] + fr[4]) / dt ** 2
    want_t = (a - np.array([0.5, -1.0, 2.0])) / np.array([3.0, 2.0, 4.0])
    assert np.array_equal(pos.cpu().numpy(), fr[5])
    np.testing.assert_allclose(vel.cpu().numpy(), v[4], rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(hist.cpu().numpy(), v.transpose(1, 0, 2).reshape(s.n, 15),
                               rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(tgt.cpu().numpy(), want_t, rtol=1e-5, atol=1e-4)


def test_make_sample_noise_is_a_random_walk_of_the_stated_size(torch):
    dt, sigma = 1e-3, 3e-4
    s = Setup(torch, 6000, 1, seed=13)
    sur = U.Surrogate(s.sim, layers=1, train=False, v_scale=1.0, dt_s=dt, max_edges=1)
    fr = _frames(s, np.random.default_rng(2), dt)
    d_fr = torch.tensor(fr, device="cuda")
    outs = []
    for seed in (11, 11, 12):
        pos = torch.empty((s.n, 3), dtype=torch.float64, device="cuda")
        vel = torch.empty((s.n, 3), dtype=torch.float32, device="cuda")
        hist = torch.empty((s.n, 15), dtype=torch.float32, device="cuda")
        tgt = torch.empty((s.n, 3), dtype=torch.float32, device="cuda")
        sur.make_sample(d_fr, sigma, seed, pos, vel, hist, tgt)
        torch.cuda.synchronize()
        outs.append((pos.cpu().numpy(), hist.cpu().numpy().astype(np.float64),
                     tgt.cpu().numpy().astype(np.float64)))
    assert all(np.array_equal(a, b) for a, b in zip(outs[0], outs[1]))     # same seed
    assert not np.array_equal(outs[0][0], outs[2][0])                       # other seed
    pos, hist, tgt = outs[0]
    f = ~s.bnd
    nu = pos - fr[5]
    assert np.all(nu[s.bnd] == 0)
    assert abs(nu[f].std() / sigma - 1) < 0.05 and abs(nu[f].mean()) < 0.05 * sigma
    # velocity noise: increments of std sigma / sqrt(5) per frame, independent
    v_clean = ((fr[1:6] - fr[0:5]) / dt).transpose(1, 0, 2).reshape(s.n, 15)
    inc = (hist - v_clean)[f] * dt
    sd = inc.std(axis=0)
    assert np.all(np.abs(sd / (sigma / np.sqrt(5)) - 1) < 0.06), sd
    c = np.corrcoef(inc[:, 0], inc[:, 3])[0, 1]
    assert abs(c) < 0.05
    # the target lands the noisy x^k on the clean x^{k+1}: a dt^2 = x6 - 2 x~5 + x~4
    x4 = pos - hist[:, 12:15] * dt
    a = tgt                                       # a_mean 0, a_std 1
    np.testing.assert_allclose((a * dt * dt)[f], (fr[6] - 2 * pos + x4)[f], rtol=0, atol=1e-9)


def test_download_by_id_is_the_sorted_download_reordered(torch):
    s = Setup(torch, 900, 1, seed=14)
    d = s.sim.download()
    pos = torch.empty((s.n, 3), dtype=torch.float64, device="cuda")
    vel = torch.empty((s.n, 3), dtype=torch.float32, device="cuda")
    rho = np.empty(s.n, np.float32)
    s.sim.download_by_id(pos, vel, rho)
    o = np.argsort(d["ids"])
    assert np.array_equal(pos.cpu().numpy(), d["pos"][o])
    assert np.array_equal(vel.cpu().numpy(), d["vel"][o])
    assert np.array_equal(rho, d["rho"][o])


def test_rollout_equals_repeated_calls_and_reports_snapshots(torch):
    dt = 1e-3
    s = Setup(torch, 1000, 2, seed=15)
    sur = U.Surrogate(s.sim, layers=2, train=False, v_scale=s.v_scale, dt_s=dt)
    sur.set_params(s.w)
    before = s.sim.download()
    h1 = s.d_hist.clone()
    for _ in range(3):
        sur.advance(h1)
        s.sim.build_cells()
    a = s.sim.download()
    s.sim.upload(before["pos"], before["vel"], before["rho"], before["ids"])
    s.sim.build_cells()
    h2 = s.d_hist.clone()
    seen = []
    sur.rollout(h2, 3, save_every=2, cb=lambda k, t: seen.append((k, t)) and False)
    b = s.sim.download()
    oa, ob = np.argsort(a["ids"]), np.argsort(b["ids"])
    assert np.array_equal(a["pos"][oa], b["pos"][ob]) and np.array_equal(a["vel"][oa], b["vel"][ob])
    assert torch.equal(h1, h2)
    assert [k for k, _ in seen] == [2, 3] and abs(seen[-1][1] - 3 * dt) < 1e-9


def test_sparser_graph_keeps_the_pairs_within_its_radius(torch):
    """radius < 1: the edges are exactly the ordered pairs closer than
    radius * 2h (the reference graph at smoothing length radius * h), and
    the network still runs on them."""
    s = Setup(torch, 1500, 1, seed=31)
    for radius in (0.5, 0.75):
        sur = U.Surrogate(s.sim, layers=1, train=False, v_scale=s.v_scale, radius=radius)
        sur.set_params(s.w)
        acc = torch.zeros((s.n, 3), dtype=torch.float32, device="cuda")
        sur.forward(s.d_hist, acc)
        s.sim.synchronize()
        rowptr, col = sur.read_graph()
        ids = s.sim.download()["ids"].astype(np.int64)
        g_src = ids[np.repeat(np.arange(s.n), np.diff(rowptr.astype(np.int64)))]
        g_dst = ids[col.astype(np.int64)]
        order = np.lexsort((g_dst, g_src))
        ref_src, ref_dst = so.graph(s.pos, radius * s.case.h)
        assert np.array_equal(g_src[order], ref_src)
        assert np.array_equal(g_dst[order], ref_dst)
        assert 0 < len(ref_src) < len(s.src)
        assert np.isfinite(acc.cpu().numpy()).all()
        sur.close()
    with pytest.raises(S.SphError):
        U.Surrogate(s.sim, layers=1, v_scale=1.0, radius=1.5)


def test_graph_pairs_at_the_radius_follow_the_fp64_predicate(torch):
    """The graph builder decides most candidates in FP32 and defers to the
    FP64 predicate within 2^-12 of the radius: pairs placed at r (1 + delta),
    delta from -3e-4 to 3e-4 down to 1e-12 and exactly 0, come out exactly as
    the FP64 brute-force reference has them, for the full and a sparser
    radius."""
    rng = np.random.default_rng(77)
    h = 0.026
    cs = 2 * h
    g = np.stack(np.meshgrid(np.arange(7), np.arange(6), np.arange(5), indexing="ij"), -1)
    base = 0.5 + 3.0 * cs * g.reshape(-1, 3).astype(np.float64)
    deltas = np.array([0.0, 1e-12, -1e-12, 1e-9, -1e-9, 1e-6, -1e-6, 1e-4, -1e-4, 3e-4, -3e-4])
    for radius in (1.0, 0.5):
        d = deltas[np.arange(base.shape[0]) % len(deltas)]
        u = rng.normal(size=base.shape)
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        partner = base + (radius * cs * (1.0 + d))[:, None] * u
        pos = np.concatenate([base, partner])
        n = pos.shape[0]
        case = cases.Case(name="radius", pos=pos, vel=np.zeros((n, 3), np.float32),
                          rho=np.full(n, 1000.0, np.float32), ids=np.arange(n, dtype=np.uint32),
                          n_bound=0, dp=h / 1.3, h=h, rho0=1000.0, c0=20.0, alpha=0.01, cfl=0.2,
                          gravity=(0.0, 0.0, -9.81),
                          dmin=tuple(float(v) for v in pos.min(0) - cs),
                          dmax=tuple(float(v) for v in pos.max(0) + 2 * cs),
                          fluid_height=float(pos[:, 2].max()))
        sim = S.Simulation.from_case(case)
        sim.build_cells()
        sur = U.Surrogate(sim, layers=1, train=False, v_scale=1.0, radius=radius)
        sur.set_params(so.init_params(1, seed=3))
        hist = torch.zeros((n, 15), dtype=torch.float32, device="cuda")
        acc = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
        sur.forward(hist, acc)
        sim.synchronize()
        rowptr, col = sur.read_graph()
        ids = sim.download()["ids"].astype(np.int64)
        g_src = ids[np.repeat(np.arange(n), np.diff(rowptr.astype(np.int64)))]
        g_dst = ids[col.astype(np.int64)]
        order = np.lexsort((g_dst, g_src))
        ref_src, ref_dst = so.graph(pos, radius * h)
        assert np.array_equal(g_src[order], ref_src), radius
        assert np.array_equal(g_dst[order], ref_dst), radius
        # both sides of the radius occur
        inside = ((pos[:base.shape[0]] - partner) ** 2).sum(1) < (2 * radius * h) ** 2
        assert inside.any() and (~inside).any()
        sur.close()
        sim.close()
