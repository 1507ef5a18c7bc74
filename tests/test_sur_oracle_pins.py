"""Pins of the FP64 reference surrogate (oracle/sur_oracle.py) against what
mathematics fixes: brute-force neighbour pairs, central finite differences of
the forward map, closed forms for the aggregation, the optimiser and the
integration step, exact bfloat16 rounding of hand-worked values, and the
symmetries of the network (node relabelling, translation, which endpoint of
an edge each weight reads).  CPU only."""
import numpy as np
import pytest
import torch

import __graft_entry__  # noqa: F401  (puts the repo root on sys.path)
from oracle import sur_oracle as so
from paper_1210_1017_gb300 import cases


def _block(n=60, seed=3):
    c = cases.random_block(n, seed=seed, jitter=0.3)
    return c


def _inputs(c, seed=0, v_scale=1.0):
    rng = np.random.default_rng(seed)
    hist = rng.normal(0, 0.5, (c.n, 15)).astype(np.float32)
    bnd = c.ids < c.n_bound
    src, dst = so.graph(c.pos, c.h)
    xn = so.node_features(hist, bnd, v_scale)
    xe = so.edge_features(c.pos, c.h, src, dst)
    return hist, bnd, src, dst, xn, xe


def test_graph_matches_brute_force_including_exact_support_distance():
    c = _block(300, seed=11)
    s1, d1 = so.graph(c.pos, c.h)
    s0, d0 = so.graph_bruteforce(c.pos, c.h)
    assert len(s1) > 0
    assert set(zip(s1.tolist(), d1.tolist())) == set(zip(s0.tolist(), d0.tolist()))
    # a lattice whose spacing is exactly 2h: neighbours at distance 2h are out
    g = np.stack(np.meshgrid(np.arange(4.0), np.arange(3.0), np.arange(2.0),
                             indexing="ij"), -1).reshape(-1, 3)
    s, d = so.graph(g, 0.5)
    assert len(s) == 0
    s, d = so.graph(g, 0.5000001)
    # each site links to its 6-neighbourhood
    deg = np.bincount(s, minlength=len(g))
    want = sum(((g[:, a] > 0).astype(int) + (g[:, a] < g[:, a].max()).astype(int))
               for a in range(3))
    assert np.array_equal(deg, want)
    # rows are sorted by source then destination, and the graph is symmetric
    assert np.all(np.diff(s) >= 0)
    pairs = set(zip(s.tolist(), d.tolist()))
    assert all((j, i) in pairs for i, j in pairs)


def test_edge_features_are_antisymmetric_with_equal_distance():
    c = _block(80)
    s, d = so.graph(c.pos, c.h)
    f = so.edge_features(c.pos, c.h, s, d)
    fr = so.edge_features(c.pos, c.h, d, s)
    assert np.array_equal(f[:, :3], -fr[:, :3])
    assert np.array_equal(f[:, 3], fr[:, 3])
    assert np.all(f[:, 3] < 1.0) and np.all(f[:, 4:] == 0)


def test_gradient_matches_central_finite_differences():
    layers = 2
    c = _block(40, seed=5)
    hist, bnd, src, dst, xn, xe = _inputs(c)
    rng = np.random.default_rng(1)
    w = so.init_params(layers, seed=2).astype(np.float64)
    w += rng.normal(0, 0.02, w.shape)
    target = rng.normal(0, 1.0, (c.n, 3))
    fluid = ~bnd
    _, lo, g = so.forward_backward(w, layers, xn, xe, src, dst, target, fluid, bf16=False)
    assert lo > 0

    def f(wv):
        with torch.no_grad():
            out = so.forward(torch.tensor(wv), layers, torch.tensor(xn), torch.tensor(xe),
                             src, dst, bf16=False)
            return float(so.loss(out, target, fluid))

    # parameters from every block: weights and biases of each layer
    idx, o = [], 0
    for _, ki, ko, has_b in so.layer_shapes(layers):
        idx += list(o + rng.choice(ki * ko, 4, replace=False))
        o += ki * ko
        if has_b:
            idx += list(o + rng.choice(ko, 2, replace=False))
            o += ko
    eps = 1e-6
    scale = np.abs(g).max()
    for k in idx:
        wp, wm = w.copy(), w.copy()
        wp[k] += eps
        wm[k] -= eps
        fd = (f(wp) - f(wm)) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-6 * max(abs(g[k]), 1e-3 * scale) + 1e-9, (k, fd, g[k])


def test_aggregation_closed_form_degree_times_edge_bias():
    """Zero node encoder, constant edge latent b, one layer passing the sum
    through: out_i = deg_i * b (for b > 0)."""
    layers = 1
    c = _block(120, seed=9)
    hist, bnd, src, dst, xn, xe = _inputs(c)
    P = np.zeros(so.param_count(layers))
    views = so.unpack(torch.from_numpy(P), layers)
    b = np.linspace(0.1, 1.0, so.L)
    views["enc_e1"][1][:] = torch.from_numpy(b)
    W3 = views["mp0_w3"][0]
    W3[so.L:, :] = torch.eye(so.L, dtype=torch.float64)
    views["mp0_w4"][0][:] = torch.eye(so.L, dtype=torch.float64)
    views["dec0"][0][:] = torch.eye(so.L, dtype=torch.float64)
    views["dec1"][0][:] = torch.eye(so.L, dtype=torch.float64)[:, :so.KOUT]
    with torch.no_grad():
        out = so.forward(torch.from_numpy(P), layers, torch.tensor(xn), torch.tensor(xe),
                         src, dst, bf16=False).numpy()
    deg = np.bincount(src, minlength=c.n).astype(np.float64)
    assert deg.max() > 5
    np.testing.assert_allclose(out, deg[:, None] * b[None, :so.KOUT], rtol=1e-13, atol=0)


def test_w1a_reads_the_receiving_node_and_w1b_the_sender():
    """After one layer with W1b = 0, node i does not depend on a neighbour's
    node input; with W1a = 0 and W1b != 0 it does."""
    layers = 1
    c = _block(100, seed=4)
    hist, bnd, src, dst, xn, xe = _inputs(c)
    i = int(src[len(src) // 2])
    j = int(dst[len(src) // 2])
    xn2 = xn.copy()
    xn2[j, :15] += 0.7
    base = so.init_params(layers, seed=8).astype(np.float64)

    def out_i(P, x):
        with torch.no_grad():
            return so.forward(torch.from_numpy(P), layers, torch.tensor(x), torch.tensor(xe),
                              src, dst, bf16=False).numpy()[i]

    Pa = base.copy()
    so.unpack(torch.from_numpy(Pa), layers)["mp0_w1b"][0][:] = 0
    # only the aggregate half of W3 feeds node i, so h_j can enter only via W1b
    so.unpack(torch.from_numpy(Pa), layers)["mp0_w3"][0][:so.L] = 0
    so.unpack(torch.from_numpy(Pa), layers)["mp0_w4"][1][:] = 0
    d_a = np.abs(out_i(Pa, xn) - out_i(Pa, xn2)).max()
    Pb = base.copy()
    so.unpack(torch.from_numpy(Pb), layers)["mp0_w1a"][0][:] = 0
    so.unpack(torch.from_numpy(Pb), layers)["mp0_w3"][0][:so.L] = 0
    d_b = np.abs(out_i(Pb, xn) - out_i(Pb, xn2)).max()
    # with W1b = 0 the change of h_j reaches i only through i's own h_i
    # (unchanged, since j != i), so the output is identical
    assert d_a == 0.0
    assert d_b > 1e-6


def test_relabelling_and_translation_leave_outputs_unchanged():
    layers = 3
    c = _block(150, seed=12)
    hist, bnd, src, dst, xn, xe = _inputs(c)
    w = so.init_params(layers, seed=3)
    with torch.no_grad():
        out = so.forward(torch.tensor(w, dtype=torch.float64), layers, torch.tensor(xn),
                         torch.tensor(xe), src, dst, bf16=False).numpy()
    perm = np.random.default_rng(0).permutation(c.n)
    pos2 = c.pos[perm] + np.array([0.3, -1.25, 2.0])     # dyadic shift: exact
    s2, d2 = so.graph(pos2, c.h)
    xn2 = so.node_features(hist[perm], bnd[perm], 1.0)
    xe2 = so.edge_features(pos2, c.h, s2, d2)
    with torch.no_grad():
        out2 = so.forward(torch.tensor(w, dtype=torch.float64), layers, torch.tensor(xn2),
                          torch.tensor(xe2), s2, d2, bf16=False).numpy()
    np.testing.assert_allclose(out2, out[perm], rtol=1e-9, atol=1e-9)


def test_bf16_rounding_hand_worked_values():
    x = torch.tensor([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -8 + 2.0 ** -20,
                      -(2.0 + 2.0 ** -7), 3.0e38, 1.0 + 2.0 ** -7], dtype=torch.float64)
    want = [1.0, 1.0 + 2.0 ** -6, 1.0 + 2.0 ** -7, -2.0, 2.9993e38, 1.0 + 2.0 ** -7]
    got = so.bf16_round(x).tolist()
    assert got[0] == want[0]          # tie -> even (1.0)
    assert got[1] == want[1]          # tie -> even (upper)
    assert got[2] == want[2]          # above the tie -> up
    assert got[3] == want[3]          # tie at exponent 1 -> even (2.0)
    assert abs(got[4] - 3.0e38) / 3.0e38 < 2 ** -8
    assert got[5] == want[5]          # representable: unchanged


def test_loss_closed_form_counts_fluid_only():
    out = torch.zeros(4, so.KOUT, dtype=torch.float64)
    out[:, 0] = torch.tensor([1.0, 2.0, 3.0, 4.0])
    target = np.zeros((4, 3))
    fluid = np.array([False, True, True, False])
    assert float(so.loss(out, target, fluid)) == (4.0 + 9.0) / 2


def test_adam_first_step_is_signed_learning_rate():
    rng = np.random.default_rng(0)
    w = rng.normal(size=50)
    g = rng.normal(size=50)
    w1, m, v = so.adam(w, g, np.zeros(50), np.zeros(50), 1, lr=1e-3, eps=0.0)
    np.testing.assert_allclose(w1, w - 1e-3 * np.sign(g), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_euler_step_constant_acceleration_closed_form():
    pos = np.array([[0.0, 0.0, 1.0], [5.0, 5.0, 5.0]])
    vel = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    acc = np.array([[0.0, 0.0, -9.81], [1.0, 1.0, 1.0]])
    fluid = np.array([True, False])
    dt, k = 0.01, 25
    p, v = pos, vel
    for _ in range(k):
        p, v = so.euler_step(p, v, acc, fluid, dt)
    # semi-implicit Euler: x_k = x_0 + k v_0 dt + a dt^2 k (k + 1) / 2
    want = pos[0] + k * vel[0] * dt + acc[0] * dt * dt * k * (k + 1) / 2
    np.testing.assert_allclose(p[0], want, rtol=0, atol=1e-12)
    assert np.array_equal(p[1], pos[1]) and np.array_equal(v[1], vel[1])


@pytest.mark.parametrize("layers", [1, 10])
def test_param_count_matches_layer_list(layers):
    per_layer = 5 * so.L * so.L + 2 * so.L * so.L + 4 * so.L
    enc = 2 * (so.KIN * so.L + so.L + so.L * so.L + so.L)
    dec = so.L * so.L + so.L + so.L * so.KOUT + so.KOUT
    assert so.param_count(layers) == enc + layers * per_layer + dec
