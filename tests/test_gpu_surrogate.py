"""The surrogate's tensor-core kernels through the C ABI against numpy on
the same bf16-rounded inputs (fp32 accumulation on both sides)."""
import numpy as np
import pytest

import __graft_entry__  # noqa: F401
from paper_1210_1017_gb300 import surrogate as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()
    return t


def _bf16(torch, a):
    # row-major device memory: the C ABI takes raw pointers
    return torch.tensor(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).contiguous().cuda()


def _np(t):
    return t.float().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("K,N", [(16, 128), (128, 128), (256, 128), (128, 16), (16, 16),
                                 (128, 256)])
@pytest.mark.parametrize("M", [1, 200, 1000, 70001])
def test_linear_matches_numpy(torch, K, N, M):
    rng = np.random.default_rng(K * 1000 + N + M)
    A = _bf16(torch, rng.normal(size=(M, K)))
    Bt = _bf16(torch, rng.normal(size=(N, K)) / np.sqrt(K))
    bias = torch.tensor(rng.normal(size=N).astype(np.float32)).cuda()
    out = torch.empty((M, N), dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()
    U.sur_linear(A, Bt, bias, M, K, N, U.SUR_EPI_NONE, None, None, out, st.cuda_stream)
    st.synchronize()
    a, b = _np(A), _np(Bt)
    ref = a @ b.T + bias.cpu().numpy()
    scale = np.abs(a) @ np.abs(b).T + 1.0
    err = np.abs(out.cpu().numpy() - ref) / scale
    assert err.max() < 1e-5, err.max()


def test_linear_epilogues(torch):
    rng = np.random.default_rng(3)
    M, K, N = 3000, 128, 128
    A = _bf16(torch, rng.normal(size=(M, K)))
    Bt = _bf16(torch, rng.normal(size=(N, K)) / 11.3)
    bias = torch.tensor(rng.normal(size=N).astype(np.float32)).cuda()
    res = _bf16(torch, rng.normal(size=(M, N)))
    st = torch.cuda.current_stream()
    a, b, r = _np(A), _np(Bt), _np(res)
    lin = a @ b.T
    for epi, want in ((U.SUR_EPI_RELU, np.maximum(lin + bias.cpu().numpy(), 0)),
                      (U.SUR_EPI_RESIDUAL, r + lin + bias.cpu().numpy()),
                      (U.SUR_EPI_RELU_MASK, np.where(r > 0, lin, 0.0))):
        out = torch.empty((M, N), dtype=torch.bfloat16, device="cuda")
        use_bias = None if epi == U.SUR_EPI_RELU_MASK else bias
        U.sur_linear(A, Bt, use_bias, M, K, N, epi, res, out, None, st.cuda_stream)
        st.synchronize()
        got = _np(out)
        assert np.allclose(got, want, rtol=1e-2, atol=2e-2), (epi, np.abs(got - want).max())


@pytest.mark.parametrize("N", [128, 16])
@pytest.mark.parametrize("M", [100, 5000, 100003])
def test_wgrad_matches_numpy(torch, N, M):
    rng = np.random.default_rng(N + M)
    P = _bf16(torch, rng.normal(size=(M, 128)))
    Q = _bf16(torch, rng.normal(size=(M, N)))
    dW = torch.empty((128, N), dtype=torch.float32, device="cuda")
    nb = U.sur_wgrad_scratch_bytes(N)
    scratch = torch.empty(nb, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()
    U.sur_wgrad(P, Q, M, N, 0.5, dW, scratch, nb, st.cuda_stream)
    st.synchronize()
    p, q = _np(P), _np(Q)
    ref = 0.5 * (p.T @ q)
    scale = 0.5 * (np.abs(p).T @ np.abs(q)) + 1.0
    err = np.abs(dW.cpu().numpy() - ref) / scale
    assert err.max() < 1e-5, err.max()
    # deterministic: a second call gives the same bits
    dW2 = torch.empty_like(dW)
    U.sur_wgrad(P, Q, M, N, 0.5, dW2, scratch, nb, st.cuda_stream)
    st.synchronize()
    assert torch.equal(dW, dW2)


@pytest.mark.parametrize("M", [1, 300, 5000, 70001, 600011])
def test_fused_edge_layer_matches_numpy(torch, M):
    """z = relu(E W1 + b1 + P[src] + Q[dst]) (bf16), E' = E + z W2 + b2 (bf16),
    against numpy in float64 on the same bf16 inputs; z within one bf16
    rounding of the reference, E' within its rounding plus the effect of z's.
    The sizes cover one tile, a grid smaller than the SMs with a half-block
    idle, a ragged last tile, and (600011 edges) many tiles per half-block,
    so the row indices loaded a tile ahead are used on every path."""
    rng = np.random.default_rng(M)
    nodes = max(2, M // 7)
    E = _bf16(torch, rng.normal(size=(M, 128)))
    W1 = rng.normal(size=(128, 128)) / 11.3
    W2 = rng.normal(size=(128, 128)) / 11.3
    W1t, W2t = _bf16(torch, W1.T), _bf16(torch, W2.T)
    b1 = torch.tensor(rng.normal(size=128).astype(np.float32)).cuda()
    b2 = torch.tensor(rng.normal(size=128).astype(np.float32)).cuda()
    P = _bf16(torch, rng.normal(size=(nodes, 128)))
    Q = _bf16(torch, rng.normal(size=(nodes, 128)))
    src = np.sort(rng.integers(0, nodes, M)).astype(np.uint32)
    dst = rng.integers(0, nodes, M).astype(np.uint32)
    d_src = torch.tensor(src.view(np.int32)).cuda()
    d_dst = torch.tensor(dst.view(np.int32)).cuda()
    Z = torch.empty((M, 128), dtype=torch.bfloat16, device="cuda")
    Eo = torch.empty((M, 128), dtype=torch.bfloat16, device="cuda")
    st = torch.cuda.current_stream()
    U.sur_edge_layer(E, W1t, W2t, b1, b2, P, Q, d_src, d_dst, M, Z, Eo, st.cuda_stream)
    st.synchronize()
    e, w1, w2 = _np(E), _np(W1t).T, _np(W2t).T
    pre = e @ w1 + b1.cpu().numpy() + _np(P)[src] + _np(Q)[dst]
    z_ref = np.maximum(pre, 0)
    z = _np(Z)
    scale1 = np.abs(e) @ np.abs(w1) + np.abs(b1.cpu().numpy()) + np.abs(_np(P)[src]) + np.abs(_np(Q)[dst])
    assert np.all(np.abs(z - z_ref) <= 2.0 ** -8 * np.abs(z_ref) + 1e-5 * scale1)
    # the second GEMM on the GPU's own z
    eo_ref = e + z @ w2 + b2.cpu().numpy()
    scale2 = np.abs(e) + np.abs(z) @ np.abs(w2) + np.abs(b2.cpu().numpy())
    assert np.all(np.abs(_np(Eo) - eo_ref) <= 2.0 ** -8 * np.abs(eo_ref) + 1e-5 * scale2)
    # without Z the update is the same
    Eo2 = torch.empty_like(Eo)
    U.sur_edge_layer(E, W1t, W2t, b1, b2, P, Q, d_src, d_dst, M, None, Eo2, st.cuda_stream)
    st.synchronize()
    assert torch.equal(Eo, Eo2)


@pytest.mark.parametrize("M", [1, 300, 5000, 100003, 600011])
def test_fused_edge_encoder_equals_two_linear_calls(torch, M):
    """The fused edge encoder, z = relu(X W1 + b1) (bf16), E0 = z W2 + b2
    (bf16), bit for bit against the same two layers as separate sur_linear
    calls (same MMA chains, same bf16 rounding of z), and E0 within its
    rounding of numpy in float64 on the GPU's own z."""
    rng = np.random.default_rng(M + 17)
    X = _bf16(torch, rng.normal(size=(M, 16)))
    W1 = rng.normal(size=(16, 128)) / 4.0
    W2 = rng.normal(size=(128, 128)) / 11.3
    W1t, W2t = _bf16(torch, W1.T), _bf16(torch, W2.T)
    b1 = torch.tensor(rng.normal(size=128).astype(np.float32)).cuda()
    b2 = torch.tensor(rng.normal(size=128).astype(np.float32)).cuda()
    st = torch.cuda.current_stream()
    Z = torch.empty((M, 128), dtype=torch.bfloat16, device="cuda")
    E0 = torch.empty((M, 128), dtype=torch.bfloat16, device="cuda")
    U.sur_edge_encoder(X, W1t, W2t, b1, b2, M, Z, E0, st.cuda_stream)
    Z_ref = torch.empty_like(Z)
    E0_ref = torch.empty_like(E0)
    U.sur_linear(X, W1t, b1, M, 16, 128, U.SUR_EPI_RELU, None, Z_ref, None, st.cuda_stream)
    U.sur_linear(Z_ref, W2t, b2, M, 128, 128, U.SUR_EPI_NONE, None, E0_ref, None, st.cuda_stream)
    E0b = torch.empty_like(E0)
    U.sur_edge_encoder(X, W1t, W2t, b1, b2, M, None, E0b, st.cuda_stream)
    st.synchronize()
    assert torch.equal(Z, Z_ref)
    assert torch.equal(E0, E0_ref)
    assert torch.equal(E0, E0b)
    z, w2 = _np(Z), _np(W2t).T
    ref = z @ w2 + b2.cpu().numpy()
    scale = np.abs(z) @ np.abs(w2) + np.abs(b2.cpu().numpy())
    assert np.all(np.abs(_np(E0) - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-5 * scale)
