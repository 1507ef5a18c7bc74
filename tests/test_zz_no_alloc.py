"""sph_radix_sort_pairs_static -- the radix sort for callers that cannot give
the library device memory (no device allocator of their own, device memory
owned by another allocator's pool, or no cudaMalloc allowed in a
latency-critical loop) -- against the workspace version sph_radix_sort_pairs.

Both are integer sorts, so the bar is bit equality.  Two calls in a row with
different sizes and key widths check that nothing left in the shared fixed
scratch by the first call leaks into the second.  This file sorts last so
that a run stopping at the first failure has run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import __graft_entry__  # noqa: F401
from paper_1210_1017_gb300 import sph as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()
    return t


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def _host(t):
    return t.cpu().numpy().view(np.uint32)


def test_static_scratch_sort_matches_workspace_sort_on_two_calls(torch):
    L = S.lib()
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(20)
    for n, bits in ((S.SPH_RADIX_SORT_STATIC_MAX_N, 24), (70001, 13)):
        keys = rng.integers(0, 1 << bits, n, dtype=np.uint64).astype(np.uint32)
        keys[: n // 4] = np.sort(keys[: n // 4])
        vals = rng.permutation(n).astype(np.uint32)
        kin, vin = _dev(torch, keys), _dev(torch, vals)
        # reference: the entry point that takes caller scratch
        nb = int(L.sph_radix_sort_scratch_bytes(n))
        scratch = torch.empty(nb, dtype=torch.uint8, device="cuda")
        kref, vref = torch.empty_like(kin), torch.empty_like(kin)
        S.sph_radix_sort_pairs(kin, vin, kref, vref, n, bits, scratch, nb, stream.cuda_stream)
        # the fixed-scratch entry point, straight through the C ABI
        kout, vout = torch.empty_like(kin), torch.empty_like(kin)
        rc = L.sph_radix_sort_pairs_static(kin.data_ptr(), vin.data_ptr(), kout.data_ptr(),
                                           vout.data_ptr(), n, bits, stream.cuda_stream)
        assert rc == 0
        stream.synchronize()
        assert np.array_equal(_host(kout), _host(kref))
        assert np.array_equal(_host(vout), _host(vref))
        order = np.argsort(keys, kind="stable")
        assert np.array_equal(_host(vout), vals[order])


def test_static_scratch_sort_rejects_sizes_above_its_maximum(torch):
    L = S.lib()
    small = torch.zeros(16, dtype=torch.int32, device="cuda")
    p = small.data_ptr()
    n = S.SPH_RADIX_SORT_STATIC_MAX_N + 1
    assert L.sph_radix_sort_pairs_static(p, p, p, p, n, 8, None) == -8
    with pytest.raises(S.SphError, match="TOO_LARGE"):
        S.sph_radix_sort_pairs_static(small, small, small, small, n, 8, 0)


def test_static_scratch_sort_32_bit_keys_at_the_maximum_and_implicit_values(torch):
    """Four passes over the largest n (the status region sized for the
    maximum tiles and passes) and d_vals_in = NULL (values 0..n-1), each
    bit for bit against the workspace sort."""
    L = S.lib()
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(21)
    for n, bits, with_vals in ((S.SPH_RADIX_SORT_STATIC_MAX_N, 32, True), (70001, 32, False)):
        keys = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
        kin = _dev(torch, keys)
        vin = _dev(torch, rng.permutation(n).astype(np.uint32)) if with_vals else None
        nb = int(L.sph_radix_sort_scratch_bytes(n))
        scratch = torch.empty(nb, dtype=torch.uint8, device="cuda")
        kref, vref = torch.empty_like(kin), torch.empty_like(kin)
        S.sph_radix_sort_pairs(kin, vin, kref, vref, n, bits, scratch, nb, stream.cuda_stream)
        kout, vout = torch.empty_like(kin), torch.empty_like(kin)
        rc = L.sph_radix_sort_pairs_static(kin.data_ptr(), None if vin is None else vin.data_ptr(),
                                           kout.data_ptr(), vout.data_ptr(), n, bits,
                                           stream.cuda_stream)
        assert rc == 0
        assert L.sph_radix_sort_static_status(stream.cuda_stream) == 0
        assert np.array_equal(_host(kout), _host(kref))
        assert np.array_equal(_host(vout), _host(vref))
        if not with_vals:
            assert np.array_equal(_host(vout), np.argsort(keys, kind="stable").astype(np.uint32))


def test_static_scratch_sort_reports_a_lookback_that_gave_up(torch):
    L = S.lib()
    stream = torch.cuda.current_stream()
    assert L.sph_radix_sort_static_selftest_timeout(500, stream.cuda_stream) == 0
    assert L.sph_radix_sort_static_status(stream.cuda_stream) == -4
    keys = np.arange(1000, 0, -1, dtype=np.uint32)
    kin = _dev(torch, keys)
    kout, vout = torch.empty_like(kin), torch.empty_like(kin)
    S.sph_radix_sort_pairs_static(kin, None, kout, vout, 1000, 10, stream.cuda_stream)
    S.sph_radix_sort_static_status(stream.cuda_stream)      # cleared by the sort
    assert np.array_equal(_host(vout), np.arange(999, -1, -1, dtype=np.uint32))
