"""JSONL run log of a simulation: one JSON line per save boundary with the
step, the simulated time and step size, the throughput since the previous
line, the FP64 conservation sums and their drift since the first line, the
particles that left the domain and the device status word (the quantities
of Sec. 2 that a run is checked by; the paper reports its runs' timings per
phase, here the wall time between save boundaries).

The stepping is sph_rollout's: the stream is synchronised at each save
boundary, where the callback reads sph_diagnostics and, if asked, the
free-surface front of each member (sph_front)."""
from __future__ import annotations

import json
import time


def energy(d: dict) -> float:
    """Total energy of a diagnostics record (kinetic + potential + internal)."""
    return float(d["kinetic"] + d["potential"] + d["internal"])


def record(d: dict, first: dict, prev: dict | None, wall_s: float, prev_wall_s: float | None,
           front=None) -> dict:
    """One log line from a diagnostics record `d`, the run's first record and
    the previous one (None for the first line)."""
    e, e0 = energy(d), energy(first)
    out = {"step": int(d["step"]), "t": float(d["t"]), "dt": float(d["dt"]),
           "wall_s": round(wall_s, 6),
           "mass": float(d["mass"]), "momentum": [float(v) for v in d["momentum"]],
           "energy": e,
           "mass_drift": (float(d["mass"]) - float(first["mass"])) / abs(float(first["mass"]))
           if first["mass"] else 0.0,
           "energy_drift": (e - e0) / abs(e0) if e0 else 0.0,
           "n_out": int(d["n_out"]), "status": int(d["status"]),
           "amax": float(d["amax"]), "cmax": float(d["cmax"]), "mumax": float(d["mumax"])}
    if prev is not None and prev_wall_s is not None and wall_s > prev_wall_s:
        span = wall_s - prev_wall_s
        out["steps_per_s"] = (int(d["step"]) - int(prev["step"])) / span
        out["pairs_per_s"] = (int(d["pairs_total"]) - int(prev["pairs_total"])) / span
        out["sim_s_per_wall_s"] = (float(d["t"]) - float(prev["t"])) / span
    if front is not None:
        out["front"] = [float(v) for v in front]
    return out


def run(sim, nsteps: int, save_every: int, path: str, front_band=None) -> list:
    """Step `sim` (a sph.Simulation) nsteps steps, appending one line per
    save boundary (and one before the first step) to the JSONL file `path`;
    returns the records.  front_band = (z_lo, z_hi) adds each member's
    front."""
    recs = []
    state = {"first": None, "prev": None, "prev_wall": None}
    t0 = time.perf_counter()

    def log_now():
        d = sim.diagnostics()
        wall = time.perf_counter() - t0
        if state["first"] is None:
            state["first"] = d
        fr = sim.front(*front_band) if front_band is not None else None
        r = record(d, state["first"], state["prev"], wall, state["prev_wall"], fr)
        state["prev"], state["prev_wall"] = d, wall
        recs.append(r)
        with open(path, "a") as f:
            f.write(json.dumps(r) + "\n")

    sim.build_cells()   # the front reads the cell list; the first step would build it anyway
    log_now()
    sim.rollout(nsteps, save_every, lambda step, t: log_now() and False)
    return recs
