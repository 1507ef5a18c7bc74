"""FP64 CPU reference of the message-passing surrogate (graph, encoder,
message-passing layers, decoder, loss, gradients, Adam, one integration
step).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product path never
imports this module, and it shares no code with the CUDA path.

The surrogate is not part of the paper.  It learns the particle update that
the paper's WCSPH method computes (Sec. 2-3): the graph is the paper's
neighbour relation (pairs closer than the kernel support 2h, Sec. 2.2 and
Sec. 3.1), and the network is the plain definition below, written with plain
PyTorch CPU ops in float64:

  node input   x_i  = [v_i^{k-4} .. v_i^k] / v_scale (15), boundary flag (1)
  edge input   x_ij = (r_i - r_j) / 2h (3), |r_i - r_j| / 2h (1), zeros (12)
  encoders     h_i = W1n relu(W0n x_i + b0n) + b1n,  e_ij likewise
  layer l      e'_ij = e_ij + W2 relu(W1a h_i + W1b h_j + W1c e_ij + b1) + b2
               h'_i  = h_i + W4 relu(W3 [h_i, sum_j e'_ij] + b3) + b4
  decoder      out_i = W6 relu(W5 h_i + b5) + b6  (16 outputs, first 3 used)
  loss         sum over fluid i of |out_i[0:3] - target_i|^2 / n_fluid

Row vectors times W (kin x kout).  With ``bf16=True`` every value that the
GPU stores in bfloat16 (inputs, weights, activations) is rounded to the
nearest bfloat16 (ties to even) at the same point, through a straight-through
rounding, so that autograd differentiates the unrounded map at the rounded
point.  Gradients come from torch autograd (a library primitive); the tests
pin them against central finite differences of ``forward``.
"""
from __future__ import annotations

import numpy as np
import torch

L = 128     # latent width
KIN = 16    # padded encoder input width
KOUT = 16   # padded decoder output width


# ------------------------------------------------------------------ graph --

def graph_bruteforce(pos: np.ndarray, h: float):
    """All ordered pairs (i, j), i != j, with d^2 < (2h)^2, d^2 evaluated as
    (dx dx + dy dy) + dz dz in FP64; O(N^2), for tiny inputs."""
    r2max = (2.0 * h) ** 2
    n = len(pos)
    src, dst = [], []
    for i in range(n):
        d = pos[i] - pos
        d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
        js = np.nonzero(d2 < r2max)[0]
        js = js[js != i]
        src.extend([i] * len(js))
        dst.extend(js.tolist())
    return np.asarray(src, np.int64), np.asarray(dst, np.int64)


def graph(pos: np.ndarray, h: float):
    """Same pairs as graph_bruteforce, candidates from a k-d tree with a
    slightly larger radius, then the exact FP64 predicate."""
    from scipy.spatial import cKDTree
    r2max = (2.0 * h) ** 2
    pairs = cKDTree(pos).query_pairs(2.0 * h * (1 + 1e-6), output_type="ndarray")
    i, j = pairs[:, 0].astype(np.int64), pairs[:, 1].astype(np.int64)
    d = pos[i] - pos[j]
    d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
    keep = d2 < r2max
    i, j = i[keep], j[keep]
    src = np.concatenate([i, j])
    dst = np.concatenate([j, i])
    order = np.lexsort((dst, src))
    return src[order], dst[order]


def edge_features(pos: np.ndarray, h: float, src, dst) -> np.ndarray:
    d = pos[src] - pos[dst]
    d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
    f = np.zeros((len(src), KIN))
    f[:, 0:3] = d / (2.0 * h)
    f[:, 3] = np.sqrt(d2) / (2.0 * h)
    return f


def node_features(hist: np.ndarray, boundary: np.ndarray, v_scale: float) -> np.ndarray:
    f = np.zeros((len(hist), KIN))
    f[:, 0:15] = hist.astype(np.float64) / v_scale
    f[:, 15] = boundary.astype(np.float64)
    return f


# ------------------------------------------------------------- parameters --

def layer_shapes(layers: int):
    """(name, kin, kout, has_bias) in the order of the flat parameter array
    (per layer: W as kin x kout row-major, then the bias)."""
    out = [("enc_n0", KIN, L, True), ("enc_n1", L, L, True),
           ("enc_e0", KIN, L, True), ("enc_e1", L, L, True)]
    for l in range(layers):
        out += [(f"mp{l}_w1a", L, L, False), (f"mp{l}_w1b", L, L, False),
                (f"mp{l}_w1c", L, L, True), (f"mp{l}_w2", L, L, True),
                (f"mp{l}_w3", 2 * L, L, True), (f"mp{l}_w4", L, L, True)]
    out += [("dec0", L, L, True), ("dec1", L, KOUT, True)]
    return out


def param_count(layers: int) -> int:
    return sum(ki * ko + (ko if b else 0) for _, ki, ko, b in layer_shapes(layers))


def unpack(flat, layers: int) -> dict:
    """name -> (W, b or None) views of a flat parameter vector (tensor)."""
    out, o = {}, 0
    for name, ki, ko, has_b in layer_shapes(layers):
        W = flat[o:o + ki * ko].reshape(ki, ko)
        o += ki * ko
        b = None
        if has_b:
            b = flat[o:o + ko]
            o += ko
        out[name] = (W, b)
    assert o == len(flat)
    return out


def init_params(layers: int, seed: int = 0, gain: float = 1.0) -> np.ndarray:
    """He-style random initialisation (float32 values), small random biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, ki, ko, has_b in layer_shapes(layers):
        std = gain * np.sqrt(2.0 / ki)
        if name.endswith(("w2", "w4")):
            std *= 0.5            # residual branches start small
        parts.append(rng.normal(0.0, std, ki * ko))
        if has_b:
            parts.append(rng.normal(0.0, 0.05, ko))
    return np.concatenate(parts).astype(np.float32)


# ---------------------------------------------------------------- forward --

def bf16_round(x: torch.Tensor) -> torch.Tensor:
    """Round float64 values to the nearest bfloat16 (ties to even) and back,
    with a straight-through gradient."""
    r = x.detach().to(torch.bfloat16).to(torch.float64)
    return x + (r - x.detach())


def forward(params, layers: int, xn, xe, src, dst, bf16: bool = True) -> torch.Tensor:
    """Network output (n x 16, float64) for node inputs xn (n x 16), edge
    inputs xe (E x 16) and edges (src[e] = i, dst[e] = j)."""
    q = bf16_round if bf16 else (lambda t: t)
    P = unpack(params, layers)
    n = xn.shape[0]
    src_t = torch.as_tensor(src, dtype=torch.long)
    dst_t = torch.as_tensor(dst, dtype=torch.long)

    def lin(x, name, bias=True):
        W, b = P[name]
        y = x @ q(W)
        if bias and b is not None:
            y = y + b
        return y

    relu = torch.relu
    h = q(lin(q(relu(lin(q(xn), "enc_n0"))), "enc_n1"))
    e = q(lin(q(relu(lin(q(xe), "enc_e0"))), "enc_e1"))
    for l in range(layers):
        Pn = q(lin(h, f"mp{l}_w1a"))
        Qn = q(lin(h, f"mp{l}_w1b"))
        z1 = q(relu(lin(e, f"mp{l}_w1c") + Pn[src_t] + Qn[dst_t]))
        e = q(e + lin(z1, f"mp{l}_w2"))
        agg = torch.zeros(n, L, dtype=e.dtype).index_add(0, src_t, e)
        y1 = q(relu(lin(torch.cat([h, q(agg)], dim=1), f"mp{l}_w3")))
        h = q(h + lin(y1, f"mp{l}_w4"))
    d1 = q(relu(lin(h, "dec0")))
    return lin(d1, "dec1")


def loss(out, target, fluid) -> torch.Tensor:
    """Sum over fluid nodes of |out[:, :3] - target|^2, divided by their count."""
    f = torch.as_tensor(fluid, dtype=torch.bool)
    r = out[f, :3] - torch.as_tensor(target, dtype=torch.float64)[f]
    return (r * r).sum() / max(int(f.sum()), 1)


def forward_backward(params_np, layers, xn, xe, src, dst, target, fluid, bf16=True):
    """(out, loss, dloss/dparams) in float64."""
    p = torch.tensor(np.asarray(params_np, np.float64), requires_grad=True)
    out = forward(p, layers, torch.as_tensor(xn, dtype=torch.float64),
                  torch.as_tensor(xe, dtype=torch.float64), src, dst, bf16)
    lo = loss(out, target, fluid)
    lo.backward()
    return out.detach().numpy(), float(lo.detach()), p.grad.numpy().copy()


# --------------------------------------------------------- optimiser, step --

def adam(w, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba, bias-corrected), float64; returns new
    (w, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def euler_step(pos, vel, acc, fluid, dt):
    """Semi-implicit Euler for fluid particles: v += a dt, r += v dt."""
    vel = vel.copy()
    pos = pos.copy()
    vel[fluid] += acc[fluid] * dt
    pos[fluid] += vel[fluid] * dt
    return pos, vel
