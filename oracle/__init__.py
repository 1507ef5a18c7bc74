"""Python binding of the FP64 CPU oracle (``sph_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product path never
imports this package.  The oracle shares no code with the CUDA path; see the
header of ``sph_oracle.c`` for the equations and readings it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE doubles, no contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or \
            os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [("dp", C.c_double), ("h", C.c_double), ("rho0", C.c_double),
                ("gamma", C.c_double), ("c0", C.c_double),
                ("alpha", C.c_double), ("eta2_coef", C.c_double),
                ("g", C.c_double * 3), ("cfl", C.c_double),
                ("mass", C.c_double), ("dmin", C.c_double * 3),
                ("dmax", C.c_double * 3), ("n_bound", C.c_int64),
                ("kernel", C.c_int64)]

# Smoothing kernels the oracle knows (Sec. 2.2), by the name a case uses.
KERNELS = {"wendland": 0, "cubic": 1}


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        dp = C.POINTER(C.c_double)
        u32 = C.POINTER(C.c_uint32)
        i64 = C.POINTER(C.c_int64)
        P = C.POINTER(_Params)
        L = _lib
        L.or_grid_dims.argtypes = [P, i64]
        L.or_cell_keys.argtypes = [P, C.c_int64, dp, dp, dp, u32]
        L.or_cell_keys.restype = C.c_int64
        L.or_sort_by_key_id.argtypes = [C.c_int64, u32, u32, i64]
        L.or_cell_offsets.argtypes = [C.c_int64, C.c_int64, u32, u32]
        L.or_neighbour_counts.argtypes = [P, C.c_int64, dp, dp, dp, C.c_int, u32]
        L.or_kernel_w.argtypes = [P, C.c_double]
        L.or_kernel_w.restype = C.c_double
        L.or_kernel_f.argtypes = [P, C.c_double]
        L.or_kernel_f.restype = C.c_double
        L.or_pressure.argtypes = [P, C.c_double]
        L.or_pressure.restype = C.c_double
        L.or_sound_speed.argtypes = [P, C.c_double]
        L.or_sound_speed.restype = C.c_double
        L.or_internal_energy.argtypes = [P, C.c_double]
        L.or_internal_energy.restype = C.c_double
        L.or_interact.argtypes = [P, C.c_int64, dp, dp, dp, dp, dp, dp, dp,
                                  u32, C.c_int, C.c_int64, C.c_int64,
                                  dp, dp, dp, dp, u32, dp]
        L.or_interact.restype = C.c_int64
        L.or_dt.argtypes = [P, dp]
        L.or_dt.restype = C.c_double
        L.or_predict.argtypes = [P, C.c_int64, dp, dp, dp, dp, dp, dp, dp,
                                 u32, dp, dp, C.c_double]
        L.or_correct.argtypes = [P, C.c_int64] + [dp] * 14 + [u32, dp, dp,
                                                               C.c_double]
        L.or_step.argtypes = [P, C.c_int64, dp, dp, dp, dp, dp, dp, dp, u32,
                              C.c_double, C.c_int, i64]
        L.or_step.restype = C.c_double
        L.or_verlet_update.argtypes = [P, C.c_int64] + [dp] * 11 + [u32, dp, dp,
                                                                    C.c_double, C.c_int]
        L.or_verlet_step.argtypes = [P, C.c_int64] + [dp] * 11 + [u32, C.c_double,
                                                                  C.c_int, C.c_int, i64]
        L.or_verlet_step.restype = C.c_double
        L.or_subdomain_labels.argtypes = [P, C.c_int64, dp, dp, dp, C.c_int, C.c_double,
                                          C.c_double, u32]
        L.or_subdomain_labels.restype = C.c_int64
        L.or_diagnostics.argtypes = [P, C.c_int64, dp, dp, dp, dp, dp, dp, dp,
                                     u32, dp]
        L.or_num_threads.restype = C.c_int
        L.or_set_num_threads.argtypes = [C.c_int]
    return _lib


def params(p: dict) -> _Params:
    """Oracle parameter block from the scalar inputs of a case."""
    s = _Params()
    s.dp, s.h, s.rho0 = p["dp"], p["h"], p["rho0"]
    s.gamma, s.c0, s.alpha = p["gamma"], p["c0"], p["alpha"]
    s.eta2_coef = p["eta2_coef"]
    for a in range(3):
        s.g[a] = p["gravity"][a]
        s.dmin[a] = p["dmin"][a]
        s.dmax[a] = p["dmax"][a]
    s.cfl, s.mass = p["cfl"], p["mass"]
    s.n_bound = int(p["n_bound"])
    s.kernel = KERNELS[p.get("kernel", "wendland")]
    return s


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _u(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint32))


def _i(a):
    return a.ctypes.data_as(C.POINTER(C.c_int64))


class State:
    """FP64 particle state in structure-of-arrays form (the oracle's own)."""

    def __init__(self, pos, vel, rho, ids):
        pos = np.asarray(pos, dtype=np.float64)
        vel = np.asarray(vel, dtype=np.float64)
        self.x = np.ascontiguousarray(pos[:, 0])
        self.y = np.ascontiguousarray(pos[:, 1])
        self.z = np.ascontiguousarray(pos[:, 2])
        self.vx = np.ascontiguousarray(vel[:, 0])
        self.vy = np.ascontiguousarray(vel[:, 1])
        self.vz = np.ascontiguousarray(vel[:, 2])
        self.rho = np.ascontiguousarray(np.asarray(rho, dtype=np.float64))
        self.ids = np.ascontiguousarray(np.asarray(ids, dtype=np.uint32))

    @classmethod
    def from_case(cls, case):
        return cls(case.pos, case.vel, case.rho, case.ids)

    @property
    def n(self):
        return self.x.shape[0]

    def pos(self):
        return np.stack([self.x, self.y, self.z], axis=1)

    def vel(self):
        return np.stack([self.vx, self.vy, self.vz], axis=1)

    def copy(self):
        return State(self.pos(), self.vel(), self.rho.copy(), self.ids.copy())

    def arrays(self):
        return (_d(self.x), _d(self.y), _d(self.z), _d(self.vx), _d(self.vy),
                _d(self.vz), _d(self.rho))


class Oracle:
    """Thin object wrapper: one parameter block, many calls."""

    def __init__(self, p: dict):
        self.p = dict(p)
        self.P = params(p)
        self.L = lib()

    def grid_dims(self):
        nc = np.zeros(3, dtype=np.int64)
        self.L.or_grid_dims(C.byref(self.P), _i(nc))
        return tuple(int(v) for v in nc)

    @property
    def ncells(self):
        a, b, c = self.grid_dims()
        return a * b * c

    def cell_keys(self, pos):
        pos = np.asarray(pos, dtype=np.float64)
        x, y, z = (np.ascontiguousarray(pos[:, a]) for a in range(3))
        key = np.zeros(pos.shape[0], dtype=np.uint32)
        nout = self.L.or_cell_keys(C.byref(self.P), pos.shape[0], _d(x), _d(y),
                                   _d(z), _u(key))
        return key, int(nout)

    def sort_by_key_id(self, key, ids):
        key = np.ascontiguousarray(key, dtype=np.uint32)
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        perm = np.zeros(key.shape[0], dtype=np.int64)
        self.L.or_sort_by_key_id(key.shape[0], _u(key), _u(ids), _i(perm))
        return perm

    def cell_offsets(self, sorted_key):
        sorted_key = np.ascontiguousarray(sorted_key, dtype=np.uint32)
        off = np.zeros(self.ncells + 2, dtype=np.uint32)
        self.L.or_cell_offsets(self.ncells, sorted_key.shape[0], _u(sorted_key),
                               _u(off))
        return off

    def build_cells(self, pos, ids):
        """Keys, (key, id) permutation, sorted keys and cell offsets."""
        key, nout = self.cell_keys(pos)
        perm = self.sort_by_key_id(key, ids)
        skey = key[perm]
        return dict(key=key, perm=perm, sorted_key=skey,
                    sorted_ids=np.asarray(ids)[perm],
                    cell_off=self.cell_offsets(skey), n_out=nout)

    def neighbour_counts(self, pos, brute=False):
        pos = np.asarray(pos, dtype=np.float64)
        x, y, z = (np.ascontiguousarray(pos[:, a]) for a in range(3))
        cnt = np.zeros(pos.shape[0], dtype=np.uint32)
        self.L.or_neighbour_counts(C.byref(self.P), pos.shape[0], _d(x), _d(y),
                                   _d(z), int(brute), _u(cnt))
        return cnt

    def w(self, r):
        return self.L.or_kernel_w(C.byref(self.P), float(r))

    def f(self, r):
        return self.L.or_kernel_f(C.byref(self.P), float(r))

    def pressure(self, rho):
        return self.L.or_pressure(C.byref(self.P), float(rho))

    def sound_speed(self, rho):
        return self.L.or_sound_speed(C.byref(self.P), float(rho))

    def internal_energy(self, rho):
        return self.L.or_internal_energy(C.byref(self.P), float(rho))

    def interact(self, st: State, brute=False, i0=0, i1=None):
        n = st.n
        i1 = n if i1 is None else i1
        a = np.zeros((n, 3), dtype=np.float64)
        dr = np.zeros(n, dtype=np.float64)
        sa = np.zeros(n, dtype=np.float64)
        sd = np.zeros(n, dtype=np.float64)
        nn = np.zeros(n, dtype=np.uint32)
        terms = np.zeros(3, dtype=np.float64)
        pairs = self.L.or_interact(C.byref(self.P), n, *st.arrays(), _u(st.ids),
                                   int(brute), int(i0), int(i1), _d(a), _d(dr),
                                   _d(sa), _d(sd), _u(nn), _d(terms))
        return dict(a=a, drho=dr, sa=sa, sd=sd, nnb=nn, terms=terms,
                    pairs=int(pairs), dt=self.dt(terms))

    def dt(self, terms):
        terms = np.ascontiguousarray(terms, dtype=np.float64)
        return self.L.or_dt(C.byref(self.P), _d(terms))

    def predict(self, st: State, a, drho, dt):
        """Predictor half step, in place on ``st``."""
        a = np.ascontiguousarray(a, dtype=np.float64)
        drho = np.ascontiguousarray(drho, dtype=np.float64)
        self.L.or_predict(C.byref(self.P), st.n, *st.arrays(), _u(st.ids),
                          _d(a), _d(drho), float(dt))
        return st

    def correct(self, pre: State, st: State, a, drho, dt):
        """Corrector from the step's start state ``pre``, in place on ``st``
        (which holds the half-step state on entry)."""
        a = np.ascontiguousarray(a, dtype=np.float64)
        drho = np.ascontiguousarray(drho, dtype=np.float64)
        self.L.or_correct(C.byref(self.P), st.n, *pre.arrays(), *st.arrays(),
                          _u(st.ids), _d(a), _d(drho), float(dt))
        return st

    def step(self, st: State, dt_fixed=0.0, brute=False):
        """One full symplectic step in place; returns (dt, pairs)."""
        pairs = np.zeros(1, dtype=np.int64)
        dt = self.L.or_step(C.byref(self.P), st.n, *st.arrays(), _u(st.ids),
                            float(dt_fixed), int(brute), _i(pairs))
        return dt, int(pairs[0])

    def verlet_update(self, st: State, prev: State, a, drho, dt, euler):
        """Verlet update in place on ``st`` (S^n -> S^n+1) from the rates at
        S^n; ``prev`` holds the velocities and densities one step earlier and
        receives those of S^n."""
        a = np.ascontiguousarray(a, dtype=np.float64)
        drho = np.ascontiguousarray(drho, dtype=np.float64)
        self.L.or_verlet_update(C.byref(self.P), st.n, *st.arrays(),
                                _d(prev.vx), _d(prev.vy), _d(prev.vz), _d(prev.rho),
                                _u(st.ids), _d(a), _d(drho), float(dt), int(bool(euler)))
        return st

    def verlet_step(self, st: State, prev: State, euler, dt_fixed=0.0, brute=False):
        """One Verlet step in place (``prev`` as in verlet_update); returns
        (dt, pairs)."""
        pairs = np.zeros(1, dtype=np.int64)
        dt = self.L.or_verlet_step(C.byref(self.P), st.n, *st.arrays(),
                                   _d(prev.vx), _d(prev.vy), _d(prev.vz), _d(prev.rho),
                                   _u(st.ids), float(dt_fixed), int(bool(euler)),
                                   int(brute), _i(pairs))
        return dt, int(pairs[0])

    def verlet_run(self, st: State, nsteps, every=40, dt_fixed=0.0, prev=None, first=0):
        """``nsteps`` Verlet steps in place, counting steps from ``first``:
        step k is an Euler step when k is a multiple of ``every`` (so the
        first step of a run that starts at 0, which has no earlier state, is
        one).  Returns (step sizes, the earlier state for a further run)."""
        prev = st.copy() if prev is None else prev
        dts = []
        for k in range(first, first + nsteps):
            dt, _ = self.verlet_step(st, prev, k % every == 0, dt_fixed=dt_fixed)
            dts.append(dt)
        return dts, prev

    def subdomain_labels(self, pos, mode, xlo, xhi):
        """Sec. 4.2-4.3 labels (mode 0: edge, 1: migration) of a 1-D
        decomposition along x for the sub-domain [xlo, xhi)."""
        pos = np.asarray(pos, dtype=np.float64)
        x, y, z = (np.ascontiguousarray(pos[:, a]) for a in range(3))
        lab = np.zeros(pos.shape[0], dtype=np.uint32)
        self.L.or_subdomain_labels(C.byref(self.P), pos.shape[0], _d(x), _d(y), _d(z),
                                   int(mode), float(xlo), float(xhi), _u(lab))
        return lab

    def subdomain_select(self, pos, ids, mode, xlo, xhi):
        """Labels, then the paper's (label, id) order; returns the labels,
        the counts per label and the input indices of the particles labelled
        1 or 2 in that order (the data a sub-domain sends)."""
        lab = self.subdomain_labels(pos, mode, xlo, xhi)
        perm = self.sort_by_key_id(lab, ids)
        key, _ = self.cell_keys(pos)
        inside = key != self.ncells          # particles of the cell-grid domain
        counts = np.array([np.sum((lab == v) & inside) for v in range(3)], dtype=np.int64)
        sel = perm[lab[perm] != 0]
        return lab, counts, sel

    def diagnostics(self, st: State):
        out = np.zeros(8, dtype=np.float64)
        self.L.or_diagnostics(C.byref(self.P), st.n, *st.arrays(), _u(st.ids),
                              _d(out))
        return dict(mass=out[0], momentum=out[1:4].copy(), kinetic=out[4],
                    potential=out[5], internal=out[6], n_out=int(out[7]))


def num_threads() -> int:
    return int(lib().or_num_threads())


def set_num_threads(t: int) -> None:
    lib().or_set_num_threads(int(t))
