"""The C ABI library builds, loads and exports what include/sph.h declares
(no compute calls: these run without a GPU)."""
import ctypes as C
import os
import re
import subprocess

import pytest

import __graft_entry__  # noqa: F401  (puts the repo root on sys.path)
from paper_1210_1017_gb300 import _build, cases
from paper_1210_1017_gb300 import sph as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in ("sph.h", "sur.h")]


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return S.lib()


def declared_functions():
    names = set()
    for h in HEADERS:
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b((?:sph|sur)_[a-z0-9_]+)\s*\(", src))
    return sorted(names - {"sph_snapshot_fn"})


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T ((?:sph|sur)_[a-z0-9_]+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)
    from paper_1210_1017_gb300 import surrogate as U
    assert sorted(S.EXPORTED + U.EXPORTED) == names


def test_struct_layouts_match_the_header(tmp_path):
    prog = tmp_path / "sz.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "sph.h"\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(sph_params),'
                    ' sizeof(sph_sizes), sizeof(sph_diag), offsetof(sph_params, dt_fixed),'
                    ' offsetof(sph_diag, n_out), offsetof(sph_params, scheme),'
                    ' offsetof(sph_params, verlet_every), sizeof(sph_instance));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = [C.sizeof(S.SphParams), C.sizeof(S.SphSizes), C.sizeof(S.SphDiag),
            S.SphParams.dt_fixed.offset, S.SphDiag.n_out.offset, S.SphParams.scheme.offset,
            S.SphParams.verlet_every.offset, C.sizeof(S.SphInstance)]
    assert got == want


def test_query_sizes_without_gpu(lib):
    case = cases.c1_dam_break()
    P = S.make_params(case.params())
    sz = S.sph_query_sizes(P, case.n)
    ncx = -(-(case.dmax[0] - case.dmin[0]) // (2 * case.h))
    assert sz.ncx == int(ncx)
    assert sz.ncells == sz.ncx * sz.ncy * sz.ncz
    assert sz.sort_passes == 1          # one counting-sort pass over the whole label
    # about 260 bytes per particle plus the cell arrays
    assert 200 * case.n < sz.workspace_bytes < 400 * case.n + 64 * sz.ncells + (1 << 20)


def test_invalid_arguments_are_rejected(lib):
    case = cases.c1_dam_break()
    p = case.params()
    bad = dict(p, gamma=5.0)
    with pytest.raises(S.SphError, match="INVALID_ARG"):
        S.sph_query_sizes(S.make_params(bad), case.n)
    with pytest.raises(S.SphError, match="INVALID_ARG"):
        S.sph_query_sizes(S.make_params(p), 0)
    with pytest.raises(S.SphError, match="INVALID_ARG"):
        S.sph_query_sizes(S.make_params(p), 1 << 26)
    flat = dict(p, dmax=(p["dmin"][0], p["dmax"][1], p["dmax"][2]))
    with pytest.raises(S.SphError, match="INVALID_ARG"):
        S.sph_query_sizes(S.make_params(flat), case.n)
    # init refuses a misaligned or short workspace before touching the GPU
    ctx = C.c_void_p()
    P = S.make_params(p)
    assert lib.sph_init(C.byref(P), case.n, 0x1001, 1 << 30, None, C.byref(ctx)) == -3
    assert lib.sph_init(C.byref(P), case.n, 0x1000, 16, None, C.byref(ctx)) == -3
    assert lib.sph_radix_sort_pairs(None, None, None, None, 8, 8, None, 0, None) == -1


def test_sort_scratch_size_grows_with_n(lib):
    a = lib.sph_radix_sort_scratch_bytes(1000)
    b = lib.sph_radix_sort_scratch_bytes(1000000)
    assert 8000 <= a < b
    assert b >= 8 * 1000000


def test_formulation_flags_and_their_validation(lib):
    """The scheme bits follow the case's kernel and integrator names; the
    library refuses unknown bits and a non-zero reserved field before any
    GPU work (query runs the same validation as init)."""
    case = cases.c1_dam_break()
    p = case.params()
    assert S.make_params(p).scheme == 0
    both = dict(p, kernel="cubic", integrator="verlet", verlet_every=25)
    P = S.make_params(both)
    assert P.scheme == S.SPH_SCHEME_CUBIC | S.SPH_SCHEME_VERLET and P.verlet_every == 25
    assert S.make_params(dict(p, integrator="verlet")).scheme == S.SPH_SCHEME_VERLET
    assert S.sph_query_sizes(P, case.n).workspace_bytes > 0
    with pytest.raises(ValueError):
        S.make_params(dict(p, kernel="gaussian"))
    bad = S.make_params(p)
    bad.scheme = 4
    with pytest.raises(S.SphError, match="INVALID_ARG"):
        S.sph_query_sizes(bad, case.n)
    bad = S.make_params(p)
    bad.reserved = 1
    with pytest.raises(S.SphError, match="INVALID_ARG"):
        S.sph_query_sizes(bad, case.n)


def test_entry_points_refuse_a_null_context(lib):
    """Every context call checks its context pointer first (no GPU needed)."""
    counts = (C.c_uint32 * 3)()
    assert lib.sph_verlet(None) == -1
    assert lib.sph_subdomain_select(None, 0, 0.0, 1.0, counts, 0, None, None, None, None) == -1
    assert lib.sph_selftest_timeout(None, 10) == -1
    assert lib.sph_units_selftest_timeout(None, 10) == -1
    assert lib.sph_clear_status(None) == -1
    t = (C.c_double * 1)(0.0)
    assert lib.sph_set_instance_state(None, t, None) == -1
    # pipelined transfers
    assert lib.sph_async_transfer_bytes(None) == 0
    assert lib.sph_enable_async_transfers(None, 0x1000, 1 << 20) == -1
    assert lib.sph_upload_async(None, 0x1000, 0x1000, 0x1000, 0x1000) == -1
    assert lib.sph_download_async(None, None, None, None, None) == -1
    assert lib.sph_sync_transfers(None) == -1


def test_new_entry_points_check_their_arguments_before_any_gpu_work(lib):
    assert lib.sph_front(None, 0.0, 1.0, None) == -1
    # standalone-sort status and self-test: scratch pointer, alignment and
    # size are checked first, then the poll limit
    assert lib.sph_radix_sort_status(None, 0, 8, None) == -1
    assert lib.sph_radix_sort_status(0x1001, 1 << 20, 8, None) == -3
    assert lib.sph_radix_sort_status(0x1000, 16, 1000, None) == -3
    assert lib.sph_radix_sort_status(0x1000, 1 << 20, 0, None) == -1
    need = int(lib.sph_radix_sort_scratch_bytes(1000))
    assert lib.sph_radix_sort_selftest_timeout(0x1000, need - 1, 1000, 10, None) == -3
    assert lib.sph_radix_sort_selftest_timeout(0x1000, need, 1000, 0, None) == -1
    assert lib.sph_radix_sort_selftest_timeout(0x1000, need, 1000, (1 << 20) + 1, None) == -1
    assert lib.sph_radix_sort_static_selftest_timeout(0, None) == -1


def test_static_sort_maximum_in_the_binding_matches_the_header():
    src = open(HEADERS[0]).read()
    m = re.search(r"#define\s+SPH_RADIX_SORT_STATIC_MAX_N\s+\(1u\s*<<\s*(\d+)\)", src)
    assert m, "SPH_RADIX_SORT_STATIC_MAX_N not found in sph.h"
    assert S.SPH_RADIX_SORT_STATIC_MAX_N == 1 << int(m.group(1))
