"""Python binding of libsph.so (the C ABI in include/sph.h).

The functions below carry the C names and only marshal arguments; every
step of the hot path runs in the library's CUDA kernels.  PyTorch supplies
the device workspace (one ``torch.empty`` of the size the library asks for)
and the CUDA stream.  There is no CPU fallback: if the library is missing
or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

# Revision tag of the interaction kernel; DRAM-traffic figures captured with
# ncu are only quoted while they were taken on this revision.
KERNEL_REV = "interact-v4.14"

SPH_OK = 0
SPH_INTERACT_COUNTS = 1
SPH_ARRAY_KEY, SPH_ARRAY_CELL_OFF, SPH_ARRAY_ACE, SPH_ARRAY_NNB = 0, 1, 2, 3
SPH_ARRAY_NNB64, SPH_ARRAY_POSC, SPH_ARRAY_DT, SPH_ARRAY_PREV = 4, 5, 6, 7
SPH_ARRAY_UNITS = 8
SPH_SCHEME_CUBIC, SPH_SCHEME_VERLET = 1, 2
SPH_SUBDOMAIN_EDGE, SPH_SUBDOMAIN_MIGRATE = 0, 1
ERRORS = {-1: "SPH_ERR_INVALID_ARG", -2: "SPH_ERR_CUDA", -3: "SPH_ERR_WORKSPACE",
          -4: "SPH_ERR_TIMEOUT", -5: "SPH_ERR_NONFINITE", -6: "SPH_ERR_CAPACITY",
          -7: "SPH_ERR_STATE", -8: "SPH_ERR_TOO_LARGE", -9: "SPH_ERR_BOUNDS"}
SPH_RADIX_SORT_STATIC_MAX_N = 1 << 20

EXPORTED = ["sph_query_sizes", "sph_init", "sph_upload", "sph_build_cells", "sph_download_by_id",
            "sph_interact", "sph_predict", "sph_correct", "sph_verlet", "sph_step",
            "sph_rollout", "sph_download", "sph_array_bytes", "sph_read_array",
            "sph_neighbour_counts_fp64", "sph_diagnostics", "sph_check",
            "sph_kernels_per_step", "sph_last_error", "sph_destroy",
            "sph_radix_sort_scratch_bytes", "sph_radix_sort_pairs",
            "sph_radix_sort_pairs_static", "sph_query_sizes_batch", "sph_init_batch",
            "sph_instance_state", "sph_num_variants", "sph_set_variant", "sph_autotune",
            "sph_subdomain_select", "sph_clear_status", "sph_selftest_timeout",
            "sph_set_instance_state", "sph_front", "sph_radix_sort_status",
            "sph_radix_sort_selftest_timeout", "sph_radix_sort_static_status",
            "sph_radix_sort_static_selftest_timeout", "sph_fma_probe", "sph_pdl_enabled",
            "sph_units_selftest_timeout", "sph_async_transfer_bytes",
            "sph_enable_async_transfers", "sph_upload_async", "sph_download_async",
            "sph_sync_transfers"]


class SphParams(C.Structure):
    _fields_ = [("dp", C.c_double), ("h", C.c_double), ("rho0", C.c_double),
                ("gamma", C.c_double), ("c0", C.c_double), ("alpha", C.c_double),
                ("eta2_coef", C.c_double), ("gravity", C.c_double * 3),
                ("cfl", C.c_double), ("mass", C.c_double),
                ("dmin", C.c_double * 3), ("dmax", C.c_double * 3),
                ("n_bound", C.c_uint32), ("scheme", C.c_uint32),
                ("dt_fixed", C.c_double), ("verlet_every", C.c_uint32),
                ("reserved", C.c_uint32)]


class SphInstance(C.Structure):
    _fields_ = [("dmin", C.c_double * 3), ("dmax", C.c_double * 3), ("c0", C.c_double),
                ("t_end", C.c_double), ("n_particles", C.c_uint32), ("n_bound", C.c_uint32)]


class SphSizes(C.Structure):
    _fields_ = [("workspace_bytes", C.c_uint64), ("ncells", C.c_uint64),
                ("ncx", C.c_uint32), ("ncy", C.c_uint32), ("ncz", C.c_uint32),
                ("sort_passes", C.c_uint32)]


class SphDiag(C.Structure):
    _fields_ = [("t", C.c_double), ("dt", C.c_double), ("mass", C.c_double),
                ("momentum", C.c_double * 3), ("kinetic", C.c_double),
                ("potential", C.c_double), ("internal", C.c_double),
                ("step", C.c_uint64), ("pairs_total", C.c_uint64),
                ("candidates_total", C.c_uint64), ("pairs_last", C.c_uint64),
                ("candidates_last", C.c_uint64), ("pairs_fluid_last", C.c_uint64),
                ("pairs_boundary_last", C.c_uint64), ("pairs_fluid_total", C.c_uint64),
                ("pairs_boundary_total", C.c_uint64), ("n_out", C.c_uint32),
                ("status", C.c_uint32), ("amax", C.c_float), ("cmax", C.c_float),
                ("mumax", C.c_float)]

    def as_dict(self):
        return dict(t=self.t, dt=self.dt, mass=self.mass,
                    momentum=list(self.momentum), kinetic=self.kinetic,
                    potential=self.potential, internal=self.internal,
                    step=int(self.step), pairs_total=int(self.pairs_total),
                    candidates_total=int(self.candidates_total),
                    pairs_last=int(self.pairs_last),
                    candidates_last=int(self.candidates_last),
                    pairs_fluid_last=int(self.pairs_fluid_last),
                    pairs_boundary_last=int(self.pairs_boundary_last),
                    pairs_fluid_total=int(self.pairs_fluid_total),
                    pairs_boundary_total=int(self.pairs_boundary_total),
                    n_out=int(self.n_out), status=int(self.status),
                    amax=self.amax, cmax=self.cmax, mumax=self.mumax)


SNAPSHOT_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_uint64, C.c_double)

_lib = None


def checked() -> bool:
    """SPH_CHECKED=1 in the environment selects the checked build
    (libsph_checked.so: every kernel index tested, an out-of-range one
    reported as SPH_ERR_BOUNDS by sph_check)."""
    return os.environ.get("SPH_CHECKED", "0") == "1"


def library_path() -> str:
    return _build.LIB_CHECKED if checked() else _build.LIB


def lib(build: bool = False):
    """Load libsph.so, or libsph_checked.so under SPH_CHECKED=1 (building
    it first if asked).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build(checked=checked()) if build else library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libsph.so not built ({path}); run __graft_entry__.build()")
    L = C.CDLL(path)
    vp, u32, u64, i32 = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int
    P = C.POINTER(SphParams)
    L.sph_query_sizes.argtypes = [P, u32, C.POINTER(SphSizes)]
    L.sph_init.argtypes = [P, u32, vp, u64, vp, C.POINTER(vp)]
    L.sph_upload.argtypes = [vp, vp, vp, vp, vp]
    L.sph_build_cells.argtypes = [vp]
    L.sph_interact.argtypes = [vp, u32]
    L.sph_predict.argtypes = [vp]
    L.sph_correct.argtypes = [vp]
    L.sph_verlet.argtypes = [vp]
    L.sph_step.argtypes = [vp, u32]
    L.sph_rollout.argtypes = [vp, u32, u32, SNAPSHOT_FN, vp]
    L.sph_download.argtypes = [vp, vp, vp, vp, vp]
    L.sph_download_by_id.argtypes = [vp, vp, vp, vp]
    L.sph_async_transfer_bytes.argtypes = [vp]
    L.sph_async_transfer_bytes.restype = u64
    L.sph_enable_async_transfers.argtypes = [vp, vp, u64]
    L.sph_upload_async.argtypes = [vp, vp, vp, vp, vp]
    L.sph_download_async.argtypes = [vp, vp, vp, vp, vp]
    L.sph_sync_transfers.argtypes = [vp]
    L.sph_array_bytes.argtypes = [vp, i32]
    L.sph_array_bytes.restype = u64
    L.sph_read_array.argtypes = [vp, i32, vp, u64]
    L.sph_neighbour_counts_fp64.argtypes = [vp]
    L.sph_diagnostics.argtypes = [vp, C.POINTER(SphDiag)]
    L.sph_check.argtypes = [vp]
    L.sph_clear_status.argtypes = [vp]
    L.sph_selftest_timeout.argtypes = [vp, u32]
    L.sph_units_selftest_timeout.argtypes = [vp, u32]
    L.sph_kernels_per_step.argtypes = [vp]
    L.sph_kernels_per_step.restype = u32
    L.sph_last_error.argtypes = [vp]
    L.sph_last_error.restype = C.c_char_p
    L.sph_destroy.argtypes = [vp]
    L.sph_destroy.restype = None
    L.sph_radix_sort_scratch_bytes.argtypes = [u32]
    L.sph_radix_sort_scratch_bytes.restype = u64
    L.sph_radix_sort_pairs.argtypes = [vp, vp, vp, vp, u32, u32, vp, u64, vp]
    L.sph_radix_sort_pairs_static.argtypes = [vp, vp, vp, vp, u32, u32, vp]
    L.sph_radix_sort_status.argtypes = [vp, u64, u32, vp]
    L.sph_radix_sort_selftest_timeout.argtypes = [vp, u64, u32, u32, vp]
    L.sph_radix_sort_static_status.argtypes = [vp]
    L.sph_radix_sort_static_selftest_timeout.argtypes = [u32, vp]
    L.sph_front.argtypes = [vp, C.c_double, C.c_double, vp]
    L.sph_fma_probe.argtypes = [vp, u32, u32, vp]
    PI = C.POINTER(SphInstance)
    L.sph_query_sizes_batch.argtypes = [P, PI, u32, C.POINTER(SphSizes)]
    L.sph_init_batch.argtypes = [P, PI, u32, vp, u64, vp, C.POINTER(vp)]
    L.sph_instance_state.argtypes = [vp, vp, vp, vp, vp]
    L.sph_set_instance_state.argtypes = [vp, vp, vp]
    L.sph_num_variants.argtypes = []
    L.sph_num_variants.restype = u32
    L.sph_pdl_enabled.argtypes = []
    L.sph_pdl_enabled.restype = C.c_int
    L.sph_set_variant.argtypes = [vp, u32]
    L.sph_autotune.argtypes = [vp, u32, vp, vp]
    L.sph_subdomain_select.argtypes = [vp, i32, C.c_double, C.c_double, vp, u32, vp, vp, vp, vp]
    _lib = L
    return L


class SphError(RuntimeError):
    pass


def _check(rc, ctx=None, what=""):
    if rc != SPH_OK:
        msg = ""
        if ctx:
            m = lib().sph_last_error(ctx)
            msg = m.decode() if m else ""
        raise SphError(f"{what}: {ERRORS.get(rc, rc)} {msg}".strip())


def make_params(p: dict, dt_fixed: float = 0.0) -> SphParams:
    s = SphParams()
    s.dp, s.h, s.rho0, s.gamma = p["dp"], p["h"], p["rho0"], p["gamma"]
    s.c0, s.alpha, s.eta2_coef = p["c0"], p["alpha"], p["eta2_coef"]
    for a in range(3):
        s.gravity[a] = p["gravity"][a]
        s.dmin[a] = p["dmin"][a]
        s.dmax[a] = p["dmax"][a]
    s.cfl, s.mass = p["cfl"], p["mass"]
    s.n_bound = int(p["n_bound"])
    s.dt_fixed = float(p.get("dt_fixed", dt_fixed))
    kernel, integ = p.get("kernel", "wendland"), p.get("integrator", "symplectic")
    if kernel not in ("wendland", "cubic") or integ not in ("symplectic", "verlet"):
        raise ValueError(f"unknown formulation: kernel {kernel!r}, integrator {integ!r}")
    s.scheme = (SPH_SCHEME_CUBIC if kernel == "cubic" else 0) | \
        (SPH_SCHEME_VERLET if integ == "verlet" else 0)
    s.verlet_every = int(p.get("verlet_every", 40))
    return s


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    return a.data_ptr()      # torch tensor (host pinned or device)


# --- C-named wrappers -------------------------------------------------------

def sph_query_sizes(params: SphParams, n: int) -> SphSizes:
    out = SphSizes()
    _check(lib().sph_query_sizes(C.byref(params), n, C.byref(out)), what="sph_query_sizes")
    return out


def sph_init(params: SphParams, n: int, d_workspace: int, nbytes: int, stream: int):
    ctx = C.c_void_p()
    _check(lib().sph_init(C.byref(params), n, d_workspace, nbytes, stream, C.byref(ctx)),
           what="sph_init")
    return ctx


def make_instances(members) -> "C.Array":
    """members: sequence of dicts with dmin, dmax, c0, n_particles, n_bound
    and optionally t_end (default: never stops)."""
    arr = (SphInstance * len(members))()
    for k, m in enumerate(members):
        for a in range(3):
            arr[k].dmin[a] = m["dmin"][a]
            arr[k].dmax[a] = m["dmax"][a]
        arr[k].c0 = m["c0"]
        arr[k].t_end = float(m.get("t_end", float("inf")))
        arr[k].n_particles = int(m["n_particles"])
        arr[k].n_bound = int(m["n_bound"])
    return arr


def sph_query_sizes_batch(params: SphParams, inst) -> SphSizes:
    out = SphSizes()
    _check(lib().sph_query_sizes_batch(C.byref(params), inst, len(inst), C.byref(out)),
           what="sph_query_sizes_batch")
    return out


def sph_init_batch(params: SphParams, inst, d_workspace: int, nbytes: int, stream: int):
    ctx = C.c_void_p()
    _check(lib().sph_init_batch(C.byref(params), inst, len(inst), d_workspace, nbytes, stream,
                                C.byref(ctx)), what="sph_init_batch")
    return ctx


def sph_instance_state(ctx, n_inst: int):
    t = np.zeros(n_inst, np.float64)
    dt = np.zeros(n_inst, np.float64)
    done = np.zeros(n_inst, np.uint32)
    steps = np.zeros(n_inst, np.uint64)
    _check(lib().sph_instance_state(ctx, _ptr(t), _ptr(dt), _ptr(done), _ptr(steps)), ctx,
           "sph_instance_state")
    return dict(t=t, dt=dt, done=done.astype(bool), steps=steps)


def sph_set_instance_state(ctx, t, steps=None):
    t = np.ascontiguousarray(t, dtype=np.float64)
    steps = None if steps is None else np.ascontiguousarray(steps, dtype=np.uint64)
    _check(lib().sph_set_instance_state(ctx, _ptr(t), _ptr(steps)), ctx, "sph_set_instance_state")


# --- checkpoints ---------------------------------------------------------------
#
# A checkpoint is one .npz file: a format tag and version, the parameter
# dictionary and ensemble members as JSON, each member's time, step size,
# step count and end flag, and the particle state as structure-of-arrays
# (positions float64, velocities and densities float32, ids uint32, in the
# library's (cell, id) order).  Writing and reading need no GPU.

CHECKPOINT_FORMAT = "gb300-wcsph-checkpoint"
CHECKPOINT_VERSION = 1


def write_checkpoint(path, params: dict, members, inst: dict, state: dict):
    import json
    meta = dict(format=CHECKPOINT_FORMAT, version=CHECKPOINT_VERSION,
                params={k: (list(v) if isinstance(v, tuple) else v) for k, v in params.items()},
                members=members, n=int(state["ids"].shape[0]))
    with open(path, "wb") as f:
        np.savez(f, meta=np.frombuffer(json.dumps(meta).encode(), dtype=np.uint8),
                 t=np.asarray(inst["t"], np.float64), dt=np.asarray(inst["dt"], np.float64),
                 steps=np.asarray(inst["steps"], np.uint64),
                 done=np.asarray(inst["done"], np.uint8),
                 pos=np.ascontiguousarray(state["pos"], np.float64),
                 vel=np.ascontiguousarray(state["vel"], np.float32),
                 rho=np.ascontiguousarray(state["rho"], np.float32),
                 ids=np.ascontiguousarray(state["ids"], np.uint32))


def read_checkpoint(path):
    """Returns (params, members, member state, particle state); raises on a
    file of another format or version, or with inconsistent sizes."""
    import json
    with np.load(path) as z:
        meta = json.loads(bytes(z["meta"]).decode())
        if meta.get("format") != CHECKPOINT_FORMAT or meta.get("version") != CHECKPOINT_VERSION:
            raise ValueError(f"{path}: not a version-{CHECKPOINT_VERSION} checkpoint")
        inst = {k: z[k].copy() for k in ("t", "dt", "steps", "done")}
        state = {k: z[k].copy() for k in ("pos", "vel", "rho", "ids")}
    n = meta["n"]
    if any(state[k].shape[0] != n for k in state) or state["pos"].shape != (n, 3):
        raise ValueError(f"{path}: particle arrays do not match n = {n}")
    params = {k: (tuple(v) if isinstance(v, list) else v) for k, v in meta["params"].items()}
    members = meta["members"]
    nm = 1 if members is None else len(members)
    if any(inst[k].shape[0] != nm for k in inst):
        raise ValueError(f"{path}: member arrays do not match {nm} members")
    inst["done"] = inst["done"].astype(bool)
    return params, members, inst, state


def sph_num_variants() -> int:
    return int(lib().sph_num_variants())


def pdl_enabled() -> bool:
    """Whether the step's kernels use programmatic dependent launch (decided
    by the first context of the process; SPH_PDL=0 turns it off)."""
    return bool(lib().sph_pdl_enabled())


def sph_set_variant(ctx, v: int):
    _check(lib().sph_set_variant(ctx, v), ctx, "sph_set_variant")


def sph_autotune(ctx, reps: int = 3):
    """Times every interaction variant on the current cells and selects the
    fastest; returns (best, milliseconds per variant)."""
    ms = np.zeros(sph_num_variants(), np.float32)
    best = np.zeros(1, np.uint32)
    _check(lib().sph_autotune(ctx, reps, _ptr(ms), _ptr(best)), ctx, "sph_autotune")
    return int(best[0]), ms


def sph_upload(ctx, pos, vel, rho, ids):
    _check(lib().sph_upload(ctx, _ptr(pos), _ptr(vel), _ptr(rho), _ptr(ids)), ctx, "sph_upload")


def sph_build_cells(ctx):
    _check(lib().sph_build_cells(ctx), ctx, "sph_build_cells")


def sph_interact(ctx, flags: int = 0):
    _check(lib().sph_interact(ctx, flags), ctx, "sph_interact")


def sph_predict(ctx):
    _check(lib().sph_predict(ctx), ctx, "sph_predict")


def sph_correct(ctx):
    _check(lib().sph_correct(ctx), ctx, "sph_correct")


def sph_verlet(ctx):
    _check(lib().sph_verlet(ctx), ctx, "sph_verlet")


def sph_step(ctx, nsteps: int = 1):
    _check(lib().sph_step(ctx, nsteps), ctx, "sph_step")


def sph_rollout(ctx, nsteps: int, save_every: int = 0, cb=None):
    """cb(step, t) -> truthy to stop; may call sph_download."""
    fn = SNAPSHOT_FN(0) if cb is None else SNAPSHOT_FN(lambda u, s, t: int(bool(cb(s, t))))
    _check(lib().sph_rollout(ctx, nsteps, save_every, fn, None), ctx, "sph_rollout")


def sph_download(ctx, pos=None, vel=None, rho=None, ids=None):
    _check(lib().sph_download(ctx, _ptr(pos), _ptr(vel), _ptr(rho), _ptr(ids)), ctx,
           "sph_download")


def sph_async_transfer_bytes(ctx) -> int:
    return int(lib().sph_async_transfer_bytes(ctx))


def sph_enable_async_transfers(ctx, buf, nbytes):
    _check(lib().sph_enable_async_transfers(ctx, _ptr(buf), int(nbytes)), ctx,
           "sph_enable_async_transfers")


def sph_upload_async(ctx, pos, vel, rho, ids):
    _check(lib().sph_upload_async(ctx, _ptr(pos), _ptr(vel), _ptr(rho), _ptr(ids)), ctx,
           "sph_upload_async")


def sph_download_async(ctx, pos=None, vel=None, rho=None, ids=None):
    _check(lib().sph_download_async(ctx, _ptr(pos), _ptr(vel), _ptr(rho), _ptr(ids)), ctx,
           "sph_download_async")


def sph_sync_transfers(ctx):
    _check(lib().sph_sync_transfers(ctx), ctx, "sph_sync_transfers")


def sph_download_by_id(ctx, pos=None, vel=None, rho=None):
    _check(lib().sph_download_by_id(ctx, _ptr(pos), _ptr(vel), _ptr(rho)), ctx,
           "sph_download_by_id")


def sph_read_array(ctx, which: int, out: np.ndarray):
    nbytes = lib().sph_array_bytes(ctx, which)
    assert out.nbytes == nbytes, (out.nbytes, nbytes)
    _check(lib().sph_read_array(ctx, which, _ptr(out), nbytes), ctx, "sph_read_array")
    return out


def sph_subdomain_select(ctx, mode, xlo, xhi, capacity, pos=None, vel=None, rho=None,
                         ids=None):
    """Returns the per-label counts; fills the caller's arrays (host numpy
    or device tensors) with the selected particles' state."""
    counts = np.zeros(3, np.uint32)
    _check(lib().sph_subdomain_select(ctx, int(mode), float(xlo), float(xhi), _ptr(counts),
                                      int(capacity), _ptr(pos), _ptr(vel), _ptr(rho), _ptr(ids)),
           ctx, "sph_subdomain_select")
    return counts


def sph_neighbour_counts_fp64(ctx):
    _check(lib().sph_neighbour_counts_fp64(ctx), ctx, "sph_neighbour_counts_fp64")


def sph_diagnostics(ctx) -> dict:
    d = SphDiag()
    _check(lib().sph_diagnostics(ctx, C.byref(d)), ctx, "sph_diagnostics")
    return d.as_dict()


def sph_front(ctx, n_inst: int, z_lo: float, z_hi: float) -> np.ndarray:
    """Per member, the largest x of fluid particles with z_lo <= z < z_hi
    (-inf where none)."""
    out = np.zeros(n_inst, np.float64)
    _check(lib().sph_front(ctx, float(z_lo), float(z_hi), _ptr(out)), ctx, "sph_front")
    return out


FMA_PROBE_FLOP_PER_THREAD_ITER = 256


def fp32_peak_tflops(torch, device, reps=10, iters=2000, blocks_per_sm=8, sms=None):
    """Measured FP32 peak: sph_fma_probe over every SM (blocks_per_sm blocks
    of 256 threads each), timed with CUDA events on a private stream after
    one warm-up launch; returns (best, median) TFLOP/s over reps launches."""
    if sms is None:
        sms = torch.cuda.get_device_properties(device).multi_processor_count
    blocks = sms * blocks_per_sm
    out = torch.empty(blocks * 256, dtype=torch.float32, device=device)
    st = torch.cuda.Stream(device=device)
    flop = float(blocks) * 256 * iters * FMA_PROBE_FLOP_PER_THREAD_ITER
    L = lib()
    ms = []
    with torch.cuda.stream(st):
        _check(L.sph_fma_probe(_ptr(out), blocks, iters, st.cuda_stream), what="sph_fma_probe")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            _check(L.sph_fma_probe(_ptr(out), blocks, iters, st.cuda_stream),
                   what="sph_fma_probe")
            e1.record(st)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
    st.synchronize()
    tf = sorted(flop / (m * 1e-3) / 1e12 for m in ms)
    return tf[-1], tf[len(tf) // 2]


def sph_check(ctx):
    _check(lib().sph_check(ctx), ctx, "sph_check")


def sph_clear_status(ctx):
    _check(lib().sph_clear_status(ctx), ctx, "sph_clear_status")


def sph_selftest_timeout(ctx, polls: int):
    _check(lib().sph_selftest_timeout(ctx, polls), ctx, "sph_selftest_timeout")


def sph_units_selftest_timeout(ctx, polls: int):
    _check(lib().sph_units_selftest_timeout(ctx, polls), ctx, "sph_units_selftest_timeout")


def sph_kernels_per_step(ctx) -> int:
    return int(lib().sph_kernels_per_step(ctx))


def sph_destroy(ctx):
    lib().sph_destroy(ctx)


def sph_radix_sort_pairs(keys_in, vals_in, keys_out, vals_out, n, key_bits, scratch,
                         scratch_bytes, stream):
    _check(lib().sph_radix_sort_pairs(_ptr(keys_in), _ptr(vals_in), _ptr(keys_out),
                                      _ptr(vals_out), n, key_bits, _ptr(scratch),
                                      scratch_bytes, stream), what="sph_radix_sort_pairs")


def sph_radix_sort_status(scratch, scratch_bytes, n, stream):
    """Raises SphError (SPH_ERR_TIMEOUT) if the last sort on this scratch
    gave up a look-back wait."""
    _check(lib().sph_radix_sort_status(_ptr(scratch), scratch_bytes, n, stream),
           what="sph_radix_sort_status")


def sph_radix_sort_selftest_timeout(scratch, scratch_bytes, n, polls, stream):
    _check(lib().sph_radix_sort_selftest_timeout(_ptr(scratch), scratch_bytes, n, polls, stream),
           what="sph_radix_sort_selftest_timeout")


def sph_radix_sort_static_status(stream):
    _check(lib().sph_radix_sort_static_status(stream), what="sph_radix_sort_static_status")


def sph_radix_sort_static_selftest_timeout(polls, stream):
    _check(lib().sph_radix_sort_static_selftest_timeout(polls, stream),
           what="sph_radix_sort_static_selftest_timeout")


def sph_radix_sort_pairs_static(keys_in, vals_in, keys_out, vals_out, n, key_bits, stream):
    """The sort with the library's fixed scratch (no caller memory)."""
    _check(lib().sph_radix_sort_pairs_static(_ptr(keys_in), _ptr(vals_in), _ptr(keys_out),
                                             _ptr(vals_out), n, key_bits, stream),
           what="sph_radix_sort_pairs_static")


# --- autotuner cache ----------------------------------------------------------

def _cache_path():
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "paper_1210_1017_gb300", "autotune.json")


def autotune_cached(sim, reps=3):
    """Autotune once per (GPU, size bucket, member count) and reuse the choice."""
    import json
    import math
    name = sim.torch.cuda.get_device_name(sim.device)
    key = f"{name}|{KERNEL_REV}|n2^{int(math.log2(max(sim.n, 1)))}|m{sim.n_inst}"
    path = _cache_path()
    table = {}
    try:
        with open(path) as f:
            table = json.load(f)
    except (OSError, ValueError):
        table = {}
    if key in table:
        sim.set_variant(int(table[key]["variant"]))
        return int(table[key]["variant"]), np.array(table[key]["ms"], np.float32)
    best, ms = sph_autotune(sim.ctx, reps)
    table[key] = {"variant": best, "ms": [float(v) for v in ms]}
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path + ".tmp", "w") as f:
            json.dump(table, f, indent=1)
        os.replace(path + ".tmp", path)
    except OSError:
        pass
    return best, ms


# --- convenience object ------------------------------------------------------

class Simulation:
    """One simulation on one GPU: workspace, stream and context.

    ``params`` is the scalar dict of :meth:`cases.Case.params`.  Arrays go in
    and out in the library's (cell, id)-sorted order; ``ids`` says which
    particle is which.
    """

    def __init__(self, params: dict, n: int, device: int = 0, stream=None,
                 dt_fixed: float = 0.0, members=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the SPH hot path needs a CUDA GPU")
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.n = int(n)
        self.params = dict(params)
        self.P = make_params(params, dt_fixed)
        self.members = make_instances(members) if members is not None else None
        self.n_inst = len(members) if members is not None else 1
        if self.members is not None:
            self.sizes = sph_query_sizes_batch(self.P, self.members)
        else:
            self.sizes = sph_query_sizes(self.P, self.n)
        self.workspace = torch.empty(int(self.sizes.workspace_bytes), dtype=torch.uint8,
                                     device=self.device)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        if self.members is not None:
            self.ctx = sph_init_batch(self.P, self.members, self.workspace.data_ptr(),
                                      int(self.sizes.workspace_bytes), self.stream.cuda_stream)
        else:
            self.ctx = sph_init(self.P, self.n, self.workspace.data_ptr(),
                                int(self.sizes.workspace_bytes), self.stream.cuda_stream)

    @classmethod
    def from_case(cls, case, **kw):
        sim = cls(case.params(), case.n, **kw)
        sim.upload(case.pos, case.vel, case.rho, case.ids)
        return sim

    @classmethod
    def from_ensemble(cls, ens, **kw):
        """An ensemble built by cases.ensemble (members run in lockstep)."""
        sim = cls(ens.params, ens.n, members=ens.members, **kw)
        sim.upload(ens.pos, ens.vel, ens.rho, ens.ids)
        return sim

    def instance_state(self):
        return sph_instance_state(self.ctx, self.n_inst)

    def set_instance_state(self, t, steps=None):
        sph_set_instance_state(self.ctx, t, steps)

    def save_checkpoint(self, path):
        """Write the state and each member's time and step count (sync)."""
        members = None
        if self.members is not None:
            members = [dict(dmin=list(m.dmin), dmax=list(m.dmax), c0=m.c0, t_end=m.t_end,
                            n_particles=int(m.n_particles), n_bound=int(m.n_bound))
                       for m in self.members]
        params = dict(self.params)
        params["dt_fixed"] = float(self.P.dt_fixed)
        write_checkpoint(path, params, members, self.instance_state(), self.download())

    @classmethod
    def load_checkpoint(cls, path, **kw):
        """A new simulation resumed from a checkpoint: same parameters and
        members, the saved state uploaded, times and step counts restored."""
        params, members, inst, state = read_checkpoint(path)
        sim = cls(params, int(state["ids"].shape[0]), members=members, **kw)
        sim.upload(state["pos"], state["vel"], state["rho"], state["ids"])
        sim.set_instance_state(inst["t"], inst["steps"])
        return sim

    def autotune(self, reps=3, cache=True):
        """Pick the fastest interaction variant for this GPU and size (needs
        built cells).  With cache=True the choice is kept in the user cache
        directory per (GPU name, log2 particle count, member count)."""
        return autotune_cached(self, reps) if cache else sph_autotune(self.ctx, reps)

    def set_variant(self, v):
        sph_set_variant(self.ctx, v)

    def upload(self, pos, vel, rho, ids):
        pos = np.ascontiguousarray(pos, dtype=np.float64) if isinstance(pos, np.ndarray) else pos
        vel = np.ascontiguousarray(vel, dtype=np.float32) if isinstance(vel, np.ndarray) else vel
        rho = np.ascontiguousarray(rho, dtype=np.float32) if isinstance(rho, np.ndarray) else rho
        ids = np.ascontiguousarray(ids, dtype=np.uint32) if isinstance(ids, np.ndarray) else ids
        # device tensors come from torch's current stream
        self.stream.wait_stream(self.torch.cuda.current_stream(self.device))
        sph_upload(self.ctx, pos, vel, rho, ids)

    def build_cells(self):
        sph_build_cells(self.ctx)

    def interact(self, counts=False):
        sph_interact(self.ctx, SPH_INTERACT_COUNTS if counts else 0)

    def predict(self):
        sph_predict(self.ctx)

    def correct(self):
        sph_correct(self.ctx)

    def verlet(self):
        sph_verlet(self.ctx)

    def step(self, nsteps=1):
        sph_step(self.ctx, nsteps)

    def rollout(self, nsteps, save_every=0, cb=None):
        sph_rollout(self.ctx, nsteps, save_every, cb)

    def subdomain_select(self, mode, xlo, xhi, capacity=None):
        """Sec. 4.3 selection for the sub-domain [xlo, xhi) (needs built
        cells): counts per label and the labelled particles' state in
        (label, id) order, in host arrays."""
        cap = self.n if capacity is None else int(capacity)
        pos = np.empty((max(cap, 1), 3), np.float64)
        vel = np.empty((max(cap, 1), 3), np.float32)
        rho = np.empty(max(cap, 1), np.float32)
        ids = np.empty(max(cap, 1), np.uint32)
        counts = sph_subdomain_select(self.ctx, mode, xlo, xhi, cap, pos, vel, rho, ids)
        m = int(counts[1]) + int(counts[2])
        return dict(counts=counts.astype(np.int64), pos=pos[:m], vel=vel[:m], rho=rho[:m],
                    ids=ids[:m])

    def neighbour_counts_fp64(self):
        sph_neighbour_counts_fp64(self.ctx)
        return self.read(SPH_ARRAY_NNB64)

    def synchronize(self):
        self.stream.synchronize()

    def download(self):
        n = self.n
        pos = np.empty((n, 3), np.float64)
        vel = np.empty((n, 3), np.float32)
        rho = np.empty(n, np.float32)
        ids = np.empty(n, np.uint32)
        sph_download(self.ctx, pos, vel, rho, ids)
        return dict(pos=pos, vel=vel, rho=rho, ids=ids)

    def download_to(self, pos=None, vel=None, rho=None, ids=None):
        """Copy the state into caller-owned arrays or device tensors (sorted
        order; any may be None)."""
        self.stream.wait_stream(self.torch.cuda.current_stream(self.device))
        sph_download(self.ctx, pos, vel, rho, ids)
        self.torch.cuda.current_stream(self.device).wait_stream(self.stream)

    def enable_async_transfers(self):
        """Attach a device staging buffer (allocated here, owned by this
        object) for sph_upload_async / sph_download_async."""
        nb = sph_async_transfer_bytes(self.ctx)
        self._xfer = self.torch.empty(nb, dtype=self.torch.uint8, device=self.device)
        sph_enable_async_transfers(self.ctx, self._xfer, nb)

    def download_by_id(self, pos=None, vel=None, rho=None):
        """State indexed by particle id into caller-owned arrays or device
        tensors (any may be None)."""
        self.stream.wait_stream(self.torch.cuda.current_stream(self.device))
        sph_download_by_id(self.ctx, pos, vel, rho)
        self.torch.cuda.current_stream(self.device).wait_stream(self.stream)

    def read(self, which):
        n = self.n
        shapes = {SPH_ARRAY_KEY: ((n,), np.uint32),
                  SPH_ARRAY_CELL_OFF: ((int(self.sizes.ncells) + 2,), np.uint32),
                  SPH_ARRAY_ACE: ((n, 4), np.float32), SPH_ARRAY_NNB: ((n,), np.uint32),
                  SPH_ARRAY_NNB64: ((n,), np.uint32), SPH_ARRAY_POSC: ((n, 4), np.float32),
                  SPH_ARRAY_DT: ((self.n_inst,), np.float64),
                  SPH_ARRAY_PREV: ((n, 4), np.float32)}
        shape, dt = shapes[which]
        return sph_read_array(self.ctx, which, np.empty(shape, dt))

    def units(self):
        """The interaction's work units, uint32 (m, 2): first sorted index and
        end of each (SPH_ARRAY_UNITS)."""
        nbytes = int(lib().sph_array_bytes(self.ctx, SPH_ARRAY_UNITS))
        buf = sph_read_array(self.ctx, SPH_ARRAY_UNITS, np.empty(nbytes // 4, np.uint32))
        m = int(buf[0])
        return buf[1:1 + 2 * m].reshape(m, 2).copy()

    def diagnostics(self):
        return sph_diagnostics(self.ctx)

    def front(self, z_lo, z_hi):
        """Free-surface front per member (see sph_front)."""
        return sph_front(self.ctx, self.n_inst, z_lo, z_hi)

    def check(self):
        sph_check(self.ctx)

    def clear_status(self):
        sph_clear_status(self.ctx)

    def kernels_per_step(self):
        return sph_kernels_per_step(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            self.synchronize()
            sph_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
