"""Python binding of the surrogate's C ABI (include/sur.h), same names as
the C functions; argument marshalling only."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import sph as _sph


class SurConfig(C.Structure):
    _fields_ = [("layers", C.c_uint32), ("max_nodes", C.c_uint32), ("max_edges", C.c_uint32),
                ("train", C.c_uint32), ("v_scale", C.c_float), ("a_mean", C.c_float * 3),
                ("a_std", C.c_float * 3), ("dt_s", C.c_float), ("radius", C.c_float)]

EXPORTED = ["sur_linear", "sur_wgrad_scratch_bytes", "sur_wgrad", "sur_edge_layer",
            "sur_edge_encoder",
            "sur_param_count",
            "sur_query_bytes", "sur_init", "sur_set_params", "sur_get_params", "sur_get_grads",
            "sur_forward", "sur_backward", "sur_adam", "sur_advance", "sur_rollout", "sur_make_sample",
            "sur_num_edges", "sur_read_graph",
            "sur_last_error", "sur_destroy"]
SUR_EPI_NONE, SUR_EPI_RELU, SUR_EPI_RESIDUAL, SUR_EPI_RELU_MASK = 0, 1, 2, 4

_ready = False


def lib():
    global _ready
    L = _sph.lib()
    if not _ready:
        vp, u32, u64, i32 = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int
        L.sur_linear.argtypes = [vp, vp, vp, u32, u32, u32, i32, vp, vp, vp, vp]
        L.sur_wgrad_scratch_bytes.argtypes = [u32]
        L.sur_wgrad_scratch_bytes.restype = u64
        L.sur_wgrad.argtypes = [vp, vp, u32, u32, C.c_float, vp, vp, u64, vp]
        L.sur_edge_layer.argtypes = [vp] * 9 + [u32, vp, vp, vp]
        L.sur_edge_encoder.argtypes = [vp] * 5 + [u32, vp, vp, vp]
        PC = C.POINTER(SurConfig)
        f = C.c_float
        L.sur_param_count.argtypes = [PC]
        L.sur_param_count.restype = u64
        L.sur_query_bytes.argtypes = [PC]
        L.sur_query_bytes.restype = u64
        L.sur_init.argtypes = [PC, vp, u64, vp, C.POINTER(vp)]
        for name in ("sur_set_params", "sur_get_params", "sur_get_grads"):
            getattr(L, name).argtypes = [vp, vp, u64]
        L.sur_forward.argtypes = [vp, vp, vp, vp]
        L.sur_backward.argtypes = [vp, vp, vp, vp]
        L.sur_adam.argtypes = [vp, f, f, f, f]
        L.sur_advance.argtypes = [vp, vp, vp]
        L.sur_make_sample.argtypes = [vp, vp, vp, C.c_double, u64, vp, vp, vp, vp]
        L.sur_rollout.argtypes = [vp, vp, vp, u32, u32, _sph.SNAPSHOT_FN, vp]
        L.sur_num_edges.argtypes = [vp]
        L.sur_num_edges.restype = u32
        L.sur_read_graph.argtypes = [vp, vp, vp]
        L.sur_last_error.argtypes = [vp]
        L.sur_last_error.restype = C.c_char_p
        L.sur_destroy.argtypes = [vp]
        L.sur_destroy.restype = None
        _ready = True
    return L


def _p(t):
    return None if t is None else t.data_ptr()


def sur_linear(A, Bt, bias, M, K, N, epilogue, res, out_bf16, out_f32, stream):
    _sph._check(lib().sur_linear(_p(A), _p(Bt), _p(bias), M, K, N, epilogue, _p(res),
                                 _p(out_bf16), _p(out_f32), stream), what="sur_linear")


def sur_wgrad_scratch_bytes(N):
    return int(lib().sur_wgrad_scratch_bytes(N))


def sur_wgrad(P, Q, M, N, scale, dW, scratch, scratch_bytes, stream):
    _sph._check(lib().sur_wgrad(_p(P), _p(Q), M, N, scale, _p(dW), _p(scratch), scratch_bytes,
                                stream), what="sur_wgrad")


def sur_edge_layer(E, W1t, W2t, b1, b2, P, Q, src, dst, M, Z, Eout, stream):
    _sph._check(lib().sur_edge_layer(_p(E), _p(W1t), _p(W2t), _p(b1), _p(b2), _p(P), _p(Q),
                                     _p(src), _p(dst), M, _p(Z), _p(Eout), stream),
                what="sur_edge_layer")


def sur_edge_encoder(X, W1t, W2t, b1, b2, M, Z, Eout, stream):
    _sph._check(lib().sur_edge_encoder(_p(X), _p(W1t), _p(W2t), _p(b1), _p(b2), M, _p(Z),
                                       _p(Eout), stream), what="sur_edge_encoder")


def _chk(rc, ctx, what):
    if rc != 0:
        m = lib().sur_last_error(ctx) if ctx else b""
        raise _sph.SphError(f"{what}: {_sph.ERRORS.get(rc, rc)} {(m or b'').decode()}".strip())


def make_config(layers=10, max_nodes=0, max_edges=0, train=False, v_scale=1.0,
                a_mean=(0.0, 0.0, 0.0), a_std=(1.0, 1.0, 1.0), dt_s=0.0,
                radius=1.0) -> SurConfig:
    c = SurConfig()
    c.layers, c.max_nodes, c.max_edges, c.train = layers, max_nodes, max_edges, int(bool(train))
    c.v_scale, c.dt_s, c.radius = v_scale, dt_s, radius
    for a in range(3):
        c.a_mean[a], c.a_std[a] = a_mean[a], a_std[a]
    return c


def sur_param_count(cfg: SurConfig) -> int:
    return int(lib().sur_param_count(C.byref(cfg)))


def sur_query_bytes(cfg: SurConfig) -> int:
    return int(lib().sur_query_bytes(C.byref(cfg)))


def sur_init(cfg: SurConfig, d_workspace: int, nbytes: int, stream: int):
    ctx = C.c_void_p()
    _chk(lib().sur_init(C.byref(cfg), d_workspace, nbytes, stream, C.byref(ctx)), None, "sur_init")
    return ctx


def sur_set_params(ctx, host: np.ndarray):
    host = np.ascontiguousarray(host, np.float32)
    _chk(lib().sur_set_params(ctx, host.ctypes.data, host.size), ctx, "sur_set_params")


def sur_get_params(ctx, count: int) -> np.ndarray:
    out = np.empty(count, np.float32)
    _chk(lib().sur_get_params(ctx, out.ctypes.data, count), ctx, "sur_get_params")
    return out


def sur_get_grads(ctx, count: int) -> np.ndarray:
    out = np.empty(count, np.float32)
    _chk(lib().sur_get_grads(ctx, out.ctypes.data, count), ctx, "sur_get_grads")
    return out


def sur_forward(ctx, sph_ctx, d_hist, d_acc=None):
    _chk(lib().sur_forward(ctx, sph_ctx, _p(d_hist), _p(d_acc)), ctx, "sur_forward")


def sur_backward(ctx, sph_ctx, d_target) -> float:
    loss = C.c_float()
    _chk(lib().sur_backward(ctx, sph_ctx, _p(d_target), C.byref(loss)), ctx, "sur_backward")
    return float(loss.value)


def sur_adam(ctx, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    _chk(lib().sur_adam(ctx, lr, beta1, beta2, eps), ctx, "sur_adam")


def sur_advance(ctx, sph_ctx, d_hist):
    _chk(lib().sur_advance(ctx, sph_ctx, _p(d_hist)), ctx, "sur_advance")


def sur_rollout(ctx, sph_ctx, d_hist, ncalls, save_every=0, cb=None):
    """cb(call, t) -> truthy to stop; called every save_every calls."""
    fn = _sph.SNAPSHOT_FN(lambda user, k, t: int(bool(cb(int(k), float(t))))) if cb else \
        _sph.SNAPSHOT_FN(0)
    _chk(lib().sur_rollout(ctx, sph_ctx, _p(d_hist), ncalls, save_every, fn, None), ctx,
         "sur_rollout")


def sur_make_sample(ctx, sph_ctx, d_frames, sigma, seed, d_pos, d_vel, d_hist, d_target):
    _chk(lib().sur_make_sample(ctx, sph_ctx, _p(d_frames), sigma, seed, _p(d_pos), _p(d_vel),
                               _p(d_hist), _p(d_target)), ctx, "sur_make_sample")


def sur_num_edges(ctx) -> int:
    return int(lib().sur_num_edges(ctx))


def sur_last_error(ctx) -> str:
    m = lib().sur_last_error(ctx)
    return m.decode() if m else ""


def sur_destroy(ctx):
    lib().sur_destroy(ctx)


class Surrogate:
    """The message-passing surrogate on one GPU, bound to the particles of
    an :class:`sph.Simulation` (same stream).  ``hist`` is a device float32
    tensor (n, 15) by particle id: the last five velocities, oldest first."""

    def __init__(self, sim, layers=10, max_edges=None, train=False, v_scale=1.0,
                 a_mean=(0.0, 0.0, 0.0), a_std=(1.0, 1.0, 1.0), dt_s=0.0, edges_per_node=90,
                 max_nodes=None, radius=1.0):
        import torch
        self.sim = sim
        self.torch = torch
        max_nodes = int(max_nodes or sim.n)
        if max_edges is None:
            max_edges = max_nodes * edges_per_node
        self.cfg = make_config(layers, max_nodes, int(max_edges), train, v_scale, a_mean, a_std,
                               dt_s, radius)
        self.nparams = sur_param_count(self.cfg)
        nbytes = sur_query_bytes(self.cfg)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=sim.device)
        self.ctx = sur_init(self.cfg, self.workspace.data_ptr(), nbytes, sim.stream.cuda_stream)

    def bind(self, sim):
        """Work on the particles of another simulation on the same stream
        (at most max_nodes particles)."""
        assert sim.stream == self.sim.stream and sim.n <= self.cfg.max_nodes
        self.sim = sim

    def set_params(self, w):
        sur_set_params(self.ctx, w)

    def params(self):
        return sur_get_params(self.ctx, self.nparams)

    def grads(self):
        return sur_get_grads(self.ctx, self.nparams)

    # Tensors come from torch's current stream and the library works on the
    # simulation's stream: each call orders the two both ways.
    def _enter(self):
        self.sim.stream.wait_stream(self.torch.cuda.current_stream(self.sim.device))

    def _leave(self):
        self.torch.cuda.current_stream(self.sim.device).wait_stream(self.sim.stream)

    def forward(self, hist, acc=None):
        self._enter()
        sur_forward(self.ctx, self.sim.ctx, hist, acc)
        self._leave()

    def backward(self, target):
        self._enter()
        loss = sur_backward(self.ctx, self.sim.ctx, target)
        self._leave()
        return loss

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        sur_adam(self.ctx, lr, beta1, beta2, eps)

    def advance(self, hist):
        self._enter()
        sur_advance(self.ctx, self.sim.ctx, hist)
        self._leave()

    def rollout(self, hist, ncalls, save_every=0, cb=None):
        self._enter()
        sur_rollout(self.ctx, self.sim.ctx, hist, ncalls, save_every, cb)
        self._leave()

    def make_sample(self, frames, sigma, seed, pos, vel, hist, target):
        self._enter()
        sur_make_sample(self.ctx, self.sim.ctx, frames, sigma, seed, pos, vel, hist, target)
        self._leave()

    @property
    def num_edges(self):
        return sur_num_edges(self.ctx)

    def read_graph(self):
        """(rowptr, col) of the last forward's graph, in the SPH context's
        particle order at that call."""
        E = sur_num_edges(self.ctx)
        rowptr = np.zeros(self.sim.n + 1, np.uint32)
        col = np.zeros(max(E, 1), np.uint32)
        _chk(lib().sur_read_graph(self.ctx, rowptr.ctypes.data, col.ctypes.data), self.ctx,
             "sur_read_graph")
        return rowptr, col[:E]

    def close(self):
        if getattr(self, "ctx", None):
            self.sim.synchronize()
            sur_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
