"""The interaction's FP16 candidate pre-filter never rejects a pair that the
FP32 neighbour test accepts.

The kernel first tests candidates two at a time in half precision on
positions scaled to cell units (cell size 2h = 1) and centred on the cell
(minus 1/2): with q for particle i and p for the candidate, the sign of
    (|p|^2 + (|q|^2 - thr)) - 2 q.p,    thr = 1 + 2^-6,
where |p|^2 is computed in FP32 from the rounded p and stored in half
precision, |q|^2 - thr likewise from the rounded q, and the rest is one
half-precision add and three fused multiply-adds (z, then y, then x).  The
exact FP32 test |r_ij|^2 < (2h)^2 is applied to the survivors.
This emulates the half-precision arithmetic with numpy (every operation
rounded once to the nearest float16; sums and fused multiply-adds exactly in
float64, then rounded once) on pairs placed near the support radius, checks
that no pair inside the support is rejected, and checks the worst-case
rounding bound the margin relies on.  CPU only."""
import numpy as np

THR = 1.0 + 2.0 ** -6


def h(x):
    return np.asarray(x, np.float64).astype(np.float16)


def hadd(a, b):
    return (a.astype(np.float64) + b.astype(np.float64)).astype(np.float16)


def hfma(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float16)


def centred(v, inv):
    """Cell units, centred on the cell, rounded to half precision (FP32
    scaling and offset first, as the kernel's fused multiply-add does)."""
    return h(np.float32(v) * np.float32(inv) - np.float32(0.5))


def sq32(v):
    """|v|^2 in FP32 from half-precision components."""
    f = v.astype(np.float32)
    return f[:, 0] * f[:, 0] + (f[:, 1] * f[:, 1] + f[:, 2] * f[:, 2])


def half_value(hq, hp):
    k = h(sq32(hp))                                   # stored with the candidate
    c = h(sq32(hq) - np.float32(THR))                 # per particle and cell
    m2q = h(-2.0 * hq.astype(np.float64))             # exact
    v = hadd(k, c)
    v = hfma(m2q[:, 2], hp[:, 2], v)
    v = hfma(m2q[:, 1], hp[:, 1], v)
    return hfma(m2q[:, 0], hp[:, 0], v)


def half_hit(hq, hp):
    """The kernel's test: a set sign bit (negative or -0) marks a candidate."""
    return np.signbit(half_value(hq, hp))


def fp32_d2(q, p):
    d = (q - p).astype(np.float32)
    return np.float32(d[:, 0] * d[:, 0] + np.float32(d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]))


def pairs(rng, n, cs, rmin, rmax):
    """Particle i at a cell-relative position plus its candidate cell's whole
    x offset (-1, 0 or +1 cells); the candidate at distance r in [rmin, rmax)
    cell sizes, kept where its own cell-relative x lies in [0, 1) and its y, z
    within one cell of i's row (the frame the kernel stages in)."""
    q = rng.uniform(0, 1, (n, 3)).astype(np.float32) * cs
    q[:, 0] += rng.integers(-1, 2, n).astype(np.float32) * cs
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    r = cs * rng.uniform(rmin, rmax, n)
    p = (q - u * r[:, None]).astype(np.float32)
    ok = (p[:, 0] >= 0) & (p[:, 0] < cs) & np.all((p[:, 1:] >= -cs) & (p[:, 1:] < 2 * cs), axis=1)
    return q[ok], p[ok]


def test_half_prefilter_keeps_every_fp32_neighbour():
    rng = np.random.default_rng(0)
    cs = np.float32(2 * 1.3 * 0.00114)          # the 32M case: 2h in metres
    inv = np.float32(1.0) / cs
    q, p = pairs(rng, 3_000_000, cs, 0.9, 1.0)  # inside, down to 10% below 2h
    d2 = fp32_d2(q, p)
    inside = d2 < np.float32(cs * cs)
    assert inside.sum() > 1_000_000
    hq, hp = centred(q, inv), centred(p, inv)
    # centred coordinates: |x| <= 1.5 for i (x in the candidate cell's frame),
    # |x| <= 1/2 for the candidate; y, z the other way round
    assert np.all(np.abs(hq.astype(np.float64)[:, 0]) <= 1.5)
    assert np.all(np.abs(hp.astype(np.float64)[:, 1:]) <= 1.5)
    keep = half_hit(hq, hp)
    assert np.all(keep[inside]), int((~keep[inside]).sum())
    # the margin: over pairs inside the support the half-precision value
    # stays below -(2^-6 - 1.04e-2), the worked bound of the rounding
    v = half_value(hq, hp).astype(np.float64)[inside]
    exact = (d2[inside].astype(np.float64) / np.float64(cs) ** 2) - THR
    assert np.max(v - exact) <= 1.04e-2
    # and it rejects most pairs well outside the support
    q2, p2 = pairs(rng, 3_000_000, cs, 1.05, 2.0)
    far = half_hit(centred(q2, inv), centred(p2, inv))
    assert far.mean() < 1e-3
