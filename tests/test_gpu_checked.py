"""The checked build (libsph_checked.so, compiled with -DSPH_CHECKED): its
kernels test every index they compute (staged and global candidate indexes,
gather and scatter slots, cell offsets, the unit list) and report an
out-of-range one as SPH_ERR_BOUNDS instead of following it.  The GPU test
runs a set of scenarios under it in a child process -- no index may be
reported -- and checks that the results equal the normal build's bit for
bit, so the checks change nothing else.  (A build of the checked library
also runs on the CPU, where only its symbols are compared.)"""
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def scenarios(out_path):
    """Every path the checks cover, through the C ABI; results saved by name."""
    import dataclasses

    from paper_1210_1017_gb300 import cases
    from paper_1210_1017_gb300 import sph as S
    res = {}
    # dam break: steps in the device loop, rates, FP32 counts, every variant
    case = cases.c1_dam_break(shuffle_seed=6)
    sim = S.Simulation.from_case(case)
    sim.step(30)
    sim.check()
    st = sim.download()
    for k in ("pos", "vel", "rho", "ids"):
        res[f"dam_{k}"] = st[k]
    sim.interact(counts=True)
    res["dam_nnb"] = sim.read(S.SPH_ARRAY_NNB)
    for v in range(S.sph_num_variants()):
        sim.set_variant(v)
        sim.interact()
        sim.check()
        res[f"dam_ace_v{v}"] = sim.read(S.SPH_ARRAY_ACE)
    sel = sim.subdomain_select(S.SPH_SUBDOMAIN_EDGE, 0.2, 0.6)
    res["sub_ids"] = sel["ids"]
    sim.check()
    sim.close()
    # dense block: the global-memory path of the interaction
    dense = cases.random_block(3000, seed=5, h_over_dp=3.0, jitter=0.2)
    sim = S.Simulation.from_case(dense)
    sim.build_cells()
    sim.interact()
    sim.check()
    res["dense_ace"] = sim.read(S.SPH_ARRAY_ACE)
    sim.close()
    # the paper's formulation
    pcase = dataclasses.replace(case, kernel="cubic", integrator="verlet")
    sim = S.Simulation.from_case(pcase)
    sim.step(11)
    sim.check()
    res["verlet_pos"] = sim.download()["pos"]
    sim.close()
    # an ensemble of three members
    members = [cases.ensemble_instance(s) for s in cases.ensemble_specs(3, seed=11)]
    sim = S.Simulation.from_ensemble(cases.ensemble(members))
    sim.step(20)
    sim.check()
    res["ens_pos"] = sim.download()["pos"]
    sim.close()
    np.savez(out_path, **res)


@pytest.mark.gpu
def test_checked_build_reports_nothing_and_changes_nothing(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    from paper_1210_1017_gb300 import _build
    __graft_entry__.build()
    _build.build(checked=True)
    env = dict(os.environ, SPH_CHECKED="1")
    got_path = tmp_path / "checked.npz"
    r = subprocess.run([sys.executable, os.path.abspath(__file__), str(got_path)], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    want_path = tmp_path / "normal.npz"
    scenarios(want_path)
    got, want = np.load(got_path), np.load(want_path)
    assert sorted(got.files) == sorted(want.files)
    for k in want.files:
        assert np.array_equal(got[k], want[k]), k


@pytest.mark.slow
def test_checked_build_compiles_and_exports_the_same_symbols():
    import re

    from paper_1210_1017_gb300 import _build
    libs = [_build.build(), _build.build(checked=True)]
    syms = []
    for lib in libs:
        out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True,
                             check=True).stdout
        syms.append(sorted(set(re.findall(r" T ((?:sph|sur)_[a-z0-9_]+)", out))))
    assert syms[0] == syms[1] and len(syms[0]) > 20


if __name__ == "__main__":
    from paper_1210_1017_gb300 import sph as _S
    assert _S.checked() and _S.library_path().endswith("libsph_checked.so")
    scenarios(sys.argv[1])
