"""Checkpoint files (no GPU): a state written and read back is identical,
and files of another format or with inconsistent sizes are refused."""
import json

import numpy as np
import pytest

from paper_1210_1017_gb300 import cases
from paper_1210_1017_gb300 import sph as S


def _payload(n=50, members=None, nm=1):
    c = cases.random_block(n, seed=2)
    rng = np.random.default_rng(0)
    state = dict(pos=c.pos, vel=c.vel, rho=c.rho, ids=rng.permutation(n).astype(np.uint32))
    inst = dict(t=np.linspace(0.1, 0.2, nm), dt=np.full(nm, 1e-4), steps=np.arange(nm) + 7,
                done=np.arange(nm) % 2 == 1)
    return c.params(), members, inst, state


def test_round_trip_is_exact(tmp_path):
    params, members, inst, state = _payload()
    params["dt_fixed"] = 0.0
    path = tmp_path / "a.npz"
    S.write_checkpoint(path, params, members, inst, state)
    p2, m2, i2, s2 = S.read_checkpoint(path)
    assert p2 == params and m2 is None
    for k in state:
        assert s2[k].dtype == np.asarray(state[k]).dtype
        assert np.array_equal(s2[k], state[k])
    for k in ("t", "dt", "steps"):
        assert np.array_equal(i2[k], inst[k])
    assert np.array_equal(i2["done"], inst["done"])


def test_ensemble_members_round_trip(tmp_path):
    members = [dict(dmin=[0, 0, 0], dmax=[1, 1, 1], c0=17.0, t_end=float("inf"),
                    n_particles=30, n_bound=5),
               dict(dmin=[2, 0, 0], dmax=[3, 1, 1], c0=15.0, t_end=1.0,
                    n_particles=20, n_bound=4)]
    params, _, inst, state = _payload(50, members, nm=2)
    path = tmp_path / "e.npz"
    S.write_checkpoint(path, params, members, inst, state)
    _, m2, i2, _ = S.read_checkpoint(path)
    assert m2 == members and i2["steps"].tolist() == [7, 8]


def test_other_formats_and_sizes_are_refused(tmp_path):
    params, members, inst, state = _payload()
    path = tmp_path / "b.npz"
    S.write_checkpoint(path, params, members, inst, state)
    with np.load(path) as z:
        parts = {k: z[k] for k in z.files}
    meta = json.loads(bytes(parts["meta"]).decode())
    bad = dict(meta, version=meta["version"] + 1)
    np.savez(tmp_path / "c.npz", **dict(parts, meta=np.frombuffer(json.dumps(bad).encode(),
                                                                  np.uint8)))
    with pytest.raises(ValueError, match="checkpoint"):
        S.read_checkpoint(tmp_path / "c.npz")
    np.savez(tmp_path / "d.npz", **dict(parts, rho=parts["rho"][:-1]))
    with pytest.raises(ValueError, match="do not match"):
        S.read_checkpoint(tmp_path / "d.npz")
