"""The interaction's FP16 candidate pre-filter never rejects a pair that the
FP32 neighbour test accepts.

The kernel first tests candidates two at a time in half precision on
positions scaled to cell units (cell size 2h = 1): the sign of
|r_ij|^2 - (1 + 2^-6), accumulated by fused multiply-adds; then it applies the
exact FP32 test |r_ij|^2 < (2h)^2 to the survivors.
This emulates the half-precision arithmetic with numpy (every operation
rounded once to the nearest float16; the fused multiply-adds exactly in
float64, then rounded once) on pairs placed near the support radius, and
checks the margin.  CPU only."""
import numpy as np

THR = np.float16(1.0 + 2.0 ** -6)


def h(x):
    return np.asarray(x, np.float64).astype(np.float16)


def hfma(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float16)


def half_hit(q, p):
    """The kernel's test: the sign of dx dx + (dy dy + (dz dz - THR)), each
    fused multiply-add rounded once to float16 (negative or -0: candidate)."""
    dx = (q[:, 0] - p[:, 0]).astype(np.float16)
    dy = (q[:, 1] - p[:, 1]).astype(np.float16)
    dz = (q[:, 2] - p[:, 2]).astype(np.float16)
    v = hfma(dx, dx, hfma(dy, dy, hfma(dz, dz, np.full_like(dz, -THR))))
    return np.signbit(v)


def fp32_d2(q, p):
    d = (q - p).astype(np.float32)
    return np.float32(d[:, 0] * d[:, 0] + np.float32(d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]))


def test_half_prefilter_keeps_every_fp32_neighbour():
    rng = np.random.default_rng(0)
    cs = np.float32(2 * 1.3 * 0.00114)          # the 32M case: 2h in metres
    inv = np.float32(1.0) / cs
    n = 2_000_000
    # own particle: cell-relative, plus the candidate cell's whole-cell offset
    # (x in [-1, 2] cells); candidate: cell-relative in its own cell, y and z
    # shifted by -1, 0 or +1 cells into the row frame
    q = rng.uniform(0, 1, (n, 3)).astype(np.float32) * cs
    q[:, 0] += rng.integers(-1, 2, n).astype(np.float32) * cs
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    r = cs * rng.uniform(0.9, 1.0, n)            # inside, down to 10% below 2h
    p = (q - u * r[:, None]).astype(np.float32)
    d2 = fp32_d2(q, p)
    inside = d2 < np.float32(cs * cs)
    assert inside.sum() > 0.9 * n
    hq, hp = h(q * inv), h(p * inv)
    assert np.all(np.abs(hq.astype(np.float64)) <= 3) and np.all(np.isfinite(hp.astype(np.float64)))
    keep = half_hit(hq, hp)
    assert np.all(keep[inside]), int((~keep[inside]).sum())
    # and it rejects most pairs well outside the support
    p2 = (q - u * (cs * rng.uniform(1.05, 2.0, n))[:, None]).astype(np.float32)
    far = half_hit(h(q * inv), h(p2 * inv))
    assert far.mean() < 1e-3
