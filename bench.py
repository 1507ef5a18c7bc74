"""Throughput of the GB300 WCSPH hot path on the 32M-fluid-particle dam break.

One step = one full symplectic step of the method: two force evaluations,
each preceded by a cell rebuild (labels, radix sort, offsets, reorder), the
CFL reduction, predictor and corrector.  The metric is particle interactions
per second: ordered neighbour pairs (i, j) with |r_ij| < 2h evaluated by the
interaction kernel, both evaluations of each step counted.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--workload dam_break_32m|dam_break_obstacles_1m|dam_break_6k]
                [--formulation default|paper]

--formulation paper runs the paper's own kernel and integrator instead (cubic
spline of Sec. 2.2, second-order Verlet of Sec. 3.3: one force evaluation
and one rebuild per step).

Under torchrun (N > 1) every rank runs an independent replica (the path has
no exchange step on one GPU); value = pairs of all ranks / max rank time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-interactions/s"
UNIT = "pairs/s"
# Algorithmic FP32 flops per unit of interaction work (FMA = 2): the
# distance test of one 27-cell candidate, one pair with a fluid particle i
# (kernel gradient, continuity, viscosity, momentum), one pair with a
# boundary particle i (kernel gradient and continuity only).
FLOP_CANDIDATE, FLOP_FLUID_PAIR, FLOP_BOUNDARY_PAIR = 8, 50, 12
# FP32 (non-tensor) peak: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz.
SMS, FP32_LANES, MAX_CLOCK_GHZ = 152, 128, 2.07


WORKLOADS = ("dam_break_32m", "dam_break_obstacles_1m", "dam_break_6k", "dam_break_ensemble_256",
             "surrogate_obstacles_1m", "surrogate_block_50k", "surrogate_variant_1m")


def workload(name):
    from paper_1210_1017_gb300 import cases
    if name == "dam_break_32m":
        return cases.c3_dam_break_32m()
    if name == "dam_break_obstacles_1m":
        return cases.c2_dam_break_obstacles()
    if name == "dam_break_6k":
        return cases.c1_dam_break()
    if name == "dam_break_ensemble_256":
        return cases.dam_break_ensemble(256, t_end=1.0)
    raise SystemExit(f"unknown workload {name}")


def is_ensemble(w):
    return hasattr(w, "members")


FORMULATIONS = {"default": ("wendland", "symplectic"), "paper": ("cubic", "verlet")}


def with_formulation(w, name):
    """The workload with the chosen kernel and integrator."""
    import dataclasses
    kernel, integrator = FORMULATIONS[name]
    if is_ensemble(w):
        w.params.update(kernel=kernel, integrator=integrator)
        w.cases = [dataclasses.replace(c, kernel=kernel, integrator=integrator) for c in w.cases]
        return w
    return dataclasses.replace(w, kernel=kernel, integrator=integrator)


def formulation_config(name):
    if name == "paper":
        return {"kernel": "cubic spline, h=1.3dp", "integrator":
                "Verlet (Euler step every 40), 1 evaluation/step"}
    return {"kernel": "Wendland C2, h=1.3dp", "integrator": "symplectic, 2 evaluations/step"}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4)
                          if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_over_ranks(ms, count, dist=None, device="cpu"):
    """Whole-job figures of a replicated run: the slowest rank's timed
    milliseconds and the work summed over ranks (single process: as given)."""
    if dist is None:
        return float(ms), int(count)
    import torch
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(count)], device=device, dtype=torch.float64)
    dist.all_reduce(c)
    return float(t.item()), int(c.item())


def cpu_baseline(case, max_seconds=25.0):
    """The FP64 oracle as it stands, on this host's cores: one interaction
    evaluation (its own grid over all particles + the pair sums) for a
    contiguous block of particles sized to a bounded amount of CPU work."""
    import oracle
    O = oracle.Oracle(case.params())
    st = oracle.State.from_case(case)
    cores = oracle.num_threads()
    n = case.n
    # calibrate on a small block, then size the measured block
    i0 = case.n_bound
    t = time.perf_counter()
    r = O.interact(st, i0=i0, i1=i0 + min(200000, n - i0))
    t_small = time.perf_counter() - t
    per_pair = t_small / max(r["pairs"], 1)
    want_pairs = max_seconds * 0.6 / per_pair
    count = int(min(n - i0, max(200000, want_pairs / 76.0)))
    t = time.perf_counter()
    r = O.interact(st, i0=i0, i1=i0 + count)
    el = time.perf_counter() - t
    return {"value": r["pairs"] / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"one oracle interaction evaluation (its neighbour grid over all "
                       f"{n} particles plus the pair sums of {count} fluid particles, "
                       f"{r['pairs']} pairs) of the {case.name} initial state, "
                       f"{el:.1f} s wall")}


def cpu_baseline_ensemble(ens, max_seconds=15.0):
    """The oracle on the ensemble's members in turn (each member's own grid
    and the pair sums of its fluid particles) until about max_seconds."""
    import oracle
    cores = oracle.num_threads()
    pairs, el, used = 0, 0.0, 0
    for c in ens.cases:
        O = oracle.Oracle(c.params())
        st = oracle.State.from_case(c)
        t = time.perf_counter()
        r = O.interact(st, i0=c.n_bound, i1=c.n)
        el += time.perf_counter() - t
        pairs += r["pairs"]
        used += 1
        if el > max_seconds:
            break
    return {"value": pairs / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"one oracle interaction evaluation (own grid + fluid pair sums) of each of "
                       f"the first {used} of {len(ens.cases)} members, {pairs} pairs, "
                       f"{el:.1f} s wall")}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    case = with_formulation(workload(args.workload), args.formulation)
    if is_ensemble(case):
        case = case.cases[0]
    import oracle
    O = oracle.Oracle(case.params())
    st = oracle.State.from_case(case)
    cores = oracle.num_threads()
    i0 = case.n_bound
    count = min(case.n - i0, 400000)
    for _ in range(args.warmup):
        O.interact(st, i0=i0, i1=i0 + count // 8)
    pairs = 0
    t = time.perf_counter()
    for _ in range(args.steps):
        r = O.interact(st, i0=i0, i1=i0 + count)
        pairs += r["pairs"]
    el = time.perf_counter() - t
    value = pairs / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": case.name, "n_particles": case.n,
                       "n_fluid": case.n_fluid, "dp": case.dp,
                       "formulation": args.formulation},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": (f"each step: one oracle interaction evaluation (grid over "
                                        f"all {case.n} particles + pair sums of {count} fluid "
                                        f"particles)")},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def pinned_copy_gbs(torch, host, stream):
    """GB/s of one torch copy of a pinned host tensor to the device (best of
    3, CUDA events on `stream`): the host link the e2e transfers share."""
    dev = torch.empty(host.shape, dtype=host.dtype, device="cuda")
    best = 0.0
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            dev.copy_(host, non_blocking=True)
            e1.record(stream)
        e1.synchronize()
        best = max(best, host.numel() * host.element_size() / (e0.elapsed_time(e1) * 1e6))
    del dev
    return best


def phase_split(sim, torch, paper, reps=3):
    """Per-phase device time of one step (ms), the step issued call by call
    with CUDA events between the calls on the simulation's stream: the
    rebuilds (labels, counting sort, offsets, unit list, reorder), the
    force evaluations (interaction and CFL step) and the integrator.
    Median over reps steps."""
    stream = sim.stream
    seq = ([("rebuild", sim.build_cells), ("interact", sim.interact), ("verlet", sim.verlet)]
           if paper else
           [("rebuild", sim.build_cells), ("interact", sim.interact), ("predict", sim.predict),
            ("rebuild", sim.build_cells), ("interact", sim.interact), ("correct", sim.correct)])
    rows = []
    for _ in range(reps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(seq) + 1)]
        ev[0].record(stream)
        for k, (_, fn) in enumerate(seq):
            fn()
            ev[k + 1].record(stream)
        ev[-1].synchronize()
        row = {}
        for k, (name, _) in enumerate(seq):
            row[name] = row.get(name, 0.0) + ev[k].elapsed_time(ev[k + 1])
        rows.append(row)
    sim.check()
    return {name: round(float(np.median([r[name] for r in rows])), 4) for name in rows[0]}


def run_ours(args):
    import torch

    from paper_1210_1017_gb300 import sph as S

    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    S.lib(build=True)
    case = with_formulation(workload(args.workload), args.formulation)
    evals_per_step = 1 if args.formulation == "paper" else 2
    if is_ensemble(case):
        sim = S.Simulation.from_ensemble(case, device=local)
    else:
        sim = S.Simulation.from_case(case, device=local)
    stream = sim.stream
    sim.build_cells()
    variant, variant_ms = sim.autotune(reps=3, cache=False)
    for _ in range(args.warmup):
        sim.step(1)
    sim.synchronize()
    d0 = sim.diagnostics()

    # --- timed region: K steps, device time with CUDA events ---------------
    def barrier():
        if dist is not None:
            dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    sim.step(args.steps)
    ev1.record(stream)
    ev1.synchronize()
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    d1 = sim.diagnostics()
    sim.check()
    pairs = d1["pairs_total"] - d0["pairs_total"]
    pf = d1["pairs_fluid_total"] - d0["pairs_fluid_total"]
    pb = d1["pairs_boundary_total"] - d0["pairs_boundary_total"]
    cand = d1["candidates_total"] - d0["candidates_total"]
    t_max, pairs_all = reduce_over_ranks(ms, pairs, dist, device="cuda")
    value = pairs_all / (t_max * 1e-3)
    steps_per_s = args.steps / (t_max * 1e-3)

    # --- dominant kernel: the interaction, timed per launch with events ------
    nlaunch = evals_per_step * args.steps
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(2 * nlaunch)]
    dsum = 0.0
    kflop = 0.0
    for k in range(nlaunch):
        evs[2 * k].record(stream)
        sim.interact()
        evs[2 * k + 1].record(stream)
    sim.synchronize()
    dk = sim.diagnostics()
    for k in range(nlaunch):
        dsum += evs[2 * k].elapsed_time(evs[2 * k + 1])
    t_int = dsum / nlaunch * 1e-3
    flop = (FLOP_CANDIDATE * dk["candidates_last"] + FLOP_FLUID_PAIR * dk["pairs_fluid_last"]
            + FLOP_BOUNDARY_PAIR * dk["pairs_boundary_last"])
    peak_derived = SMS * FP32_LANES * 2 * MAX_CLOCK_GHZ / 1e3
    # measured FP32 peak: the FMA-loop probe over every SM, best of 10
    peak_tflops, peak_median = S.fp32_peak_tflops(torch, sim.device)
    achieved = flop / t_int / 1e12
    traffic = None
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(prof):
        with open(prof) as f:
            tr = json.load(f)
        # captured on the Wendland C2 build; the cubic-spline build has none
        if tr.get("kernel_rev") == S.KERNEL_REV and args.formulation == "default":
            traffic = tr.get("bytes_per_launch", {}).get(args.workload)
    roofline = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak_tflops, 2),
                "unit": "TFLOP/s", "frac": round(achieved / peak_tflops, 4), "traffic": traffic,
                "kernel": "k_interact", "ms_per_launch": round(t_int * 1e3, 4),
                "peak_source": ("measured: sph_fma_probe, 8 independent FMA chains per thread, "
                                "SMs x 8 blocks x 256 threads, best of 10 launches (CUDA events)"),
                "peak_median": round(peak_median, 2),
                "peak_derived": round(peak_derived, 2),
                "frac_of_derived": round(achieved / peak_derived, 4)}

    # --- per-phase split of one step (call by call, events between) ---------
    phases = phase_split(sim, torch, args.formulation == "paper")

    # --- end to end through the C ABI with pinned host buffers ---------------
    n = case.n
    if is_ensemble(case):
        st0 = sim.download()   # resume point: the e2e steps restart from here
        case_pos, case_vel, case_rho, case_ids = st0["pos"], st0["vel"], st0["rho"], st0["ids"]
    else:
        case_pos, case_vel, case_rho, case_ids = case.pos, case.vel, case.rho, case.ids
    pin = dict(pos=torch.from_numpy(np.ascontiguousarray(case_pos)).pin_memory(),
               vel=torch.from_numpy(np.ascontiguousarray(case_vel)).pin_memory(),
               rho=torch.from_numpy(np.ascontiguousarray(case_rho)).pin_memory(),
               ids=torch.from_numpy(np.ascontiguousarray(case_ids).view(np.int32)).pin_memory())
    out = dict(pos=torch.empty((n, 3), dtype=torch.float64).pin_memory(),
               vel=torch.empty((n, 3), dtype=torch.float32).pin_memory(),
               rho=torch.empty(n, dtype=torch.float32).pin_memory(),
               ids=torch.empty(n, dtype=torch.int32).pin_memory())
    e2e_steps = max(1, min(args.steps, 20))
    bytes_h2d = n * (24 + 12 + 4 + 4)
    # one untimed round trip first: it instantiates the step graph of the
    # buffer parity the uploads land in
    S.sph_upload(sim.ctx, pin["pos"], pin["vel"], pin["rho"], pin["ids"])
    S.sph_step(sim.ctx, 1)
    S.sph_download(sim.ctx, out["pos"], out["vel"], out["rho"], out["ids"])
    # the link itself: one plain copy of the pinned positions (torch, events)
    link = pinned_copy_gbs(torch, pin["pos"], stream)

    # (1) pipelined: every step uploads its inputs and downloads its result
    # through sph_upload_async / sph_download_async, which run on the
    # context's copy streams and overlap the neighbouring steps; one
    # sph_sync_transfers ends the timed region
    sim.enable_async_transfers()
    S.sph_upload_async(sim.ctx, pin["pos"], pin["vel"], pin["rho"], pin["ids"])
    S.sph_step(sim.ctx, 1)
    S.sph_download_async(sim.ctx, out["pos"], out["vel"], out["rho"], out["ids"])
    S.sph_sync_transfers(sim.ctx)
    de0 = sim.diagnostics()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        S.sph_upload_async(sim.ctx, pin["pos"], pin["vel"], pin["rho"], pin["ids"])
        S.sph_step(sim.ctx, 1)
        S.sph_download_async(sim.ctx, out["pos"], out["vel"], out["rho"], out["ids"])
    S.sph_sync_transfers(sim.ctx)
    t_e2e = time.perf_counter() - t0
    de1 = sim.diagnostics()
    barrier()
    e2e_pairs = de1["pairs_total"] - de0["pairs_total"]

    # (2) synchronous calls, for comparison: sph_upload, sph_step,
    # stream sync, sph_download, each waiting for the last
    ds0 = sim.diagnostics()
    ts0 = time.perf_counter()
    parts = np.zeros(3)
    each = []
    for _ in range(e2e_steps):
        ta = time.perf_counter()
        S.sph_upload(sim.ctx, pin["pos"], pin["vel"], pin["rho"], pin["ids"])
        tb = time.perf_counter()
        S.sph_step(sim.ctx, 1)
        sim.synchronize()
        tc = time.perf_counter()
        S.sph_download(sim.ctx, out["pos"], out["vel"], out["rho"], out["ids"])
        td = time.perf_counter()
        parts += (tb - ta, tc - tb, td - tc)
        each.append([round((tb - ta) * 1e3, 3), round((tc - tb) * 1e3, 3), round((td - tc) * 1e3, 3)])
    t_sync = time.perf_counter() - ts0
    ds1 = sim.diagnostics()
    sync_pairs = ds1["pairs_total"] - ds0["pairs_total"]
    e2e = {"value": e2e_pairs / t_e2e, "unit": UNIT, "h2d_bytes_per_step": bytes_h2d,
           "d2h_bytes_per_step": bytes_h2d, "steps": e2e_steps,
           "ms_per_step": round(t_e2e / e2e_steps * 1e3, 3),
           "pinned_copy_h2d_gbs": round(link, 1),
           "note": ("per step: sph_upload_async (pinned host) + sph_step(1) + sph_download_async "
                    "(pinned host); copies on the context's two copy streams overlap the "
                    "neighbouring steps; one sph_sync_transfers ends the timed region"),
           "synchronous": {"value": sync_pairs / t_sync, "ms_per_step": round(t_sync / e2e_steps * 1e3, 3),
                           "ms_upload_step_download": [round(v / e2e_steps * 1e3, 3) for v in parts],
                           "ms_each_step": each,
                           "note": "sph_upload + sph_step(1) + stream sync + sph_download, in turn"}}

    sub = subdomain_timing(sim, case, args.subdomains, S, torch) if args.subdomains else None

    kps = sim.kernels_per_step()
    # symplectic runs of two or more steps go through the device step loop
    loop = args.formulation == "default" and args.steps >= 2
    if is_ensemble(case):
        ist = sim.instance_state()
        cfg = {"workload": args.workload, "members": len(case.members), "n_particles": case.n,
               "member_sizes": [int(min(c.n for c in case.cases)), int(max(c.n for c in case.cases))],
               "dp": case.params["dp"], "t_end": 1.0,
               "members_done_after_run": int(ist["done"].sum())}
        base_case = case.cases[0]
    else:
        cfg = {"workload": case.name, "n_particles": case.n, "n_fluid": case.n_fluid,
               "n_boundary": case.n_bound, "dp": case.dp}
        base_case = case
    cfg.update(formulation_config(args.formulation))
    cfg.update({"formulation": args.formulation, "position_dtype": "f64", "l2": "inputs larger than L2",
                "parallelism": f"replicas x{ws}", "interaction_variant": variant,
                "variant_ms": [round(float(v), 3) for v in variant_ms],
                "programmatic_dependent_launch": S.pdl_enabled()})
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic", "config": cfg,
            "steps_per_s": steps_per_s, "pairs_per_step": pairs / args.steps,
            "fluid_pairs_per_step": pf / args.steps, "boundary_pairs_per_step": pb / args.steps,
            "candidates_per_step": cand / args.steps,
            "sim_time_per_step": (d1["t"] - d0["t"]) / args.steps,
            # time to solution: wall seconds per simulated second (member 0)
            "wall_s_per_simulated_s": ((t_max * 1e-3) / (d1["t"] - d0["t"])
                                       if d1["t"] > d0["t"] else None),
            "member_steps_per_s": steps_per_s * getattr(sim, "n_inst", 1),
            "roofline": roofline, "e2e": e2e, "phases_ms": phases,
            # the step kernels, one loop-control kernel per step and the loop's
            # arming kernel (sph_step with two or more steps is one graph launch)
            "gpu_launches": (kps * args.steps + (args.steps + 1 if loop else 0)),
            "clocks": clocks}
    if sub is not None:
        line["subdomain_select"] = sub
    pk, src = peaks()
    line["peaks_source"] = src
    if args.workload == "dam_break_32m" and args.formulation == "default" and not args.no_ensemble:
        sim.close()
        del sim
        torch.cuda.empty_cache()
        sim = None
        line["ensemble_256"] = ensemble_record(args, S, torch, local, args.steps)
        torch.cuda.empty_cache()
        line["surrogate_1m"] = surrogate_record(args, S, torch, local)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        if sim is not None:
            sim.close()
        del sim
        torch.cuda.empty_cache()
        line["cpu_baseline"] = (cpu_baseline_ensemble(case) if is_ensemble(case)
                                else cpu_baseline(base_case))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def surrogate_record(args, S, torch, device, calls=5):
    """The learned surrogate's speed against plain GPU SPH, as a nested record
    of the default line: the fastest variant (2 message-passing layers, 16
    SPH steps per call, edges only within 0.65 2h) on the 1.39M-particle dam
    break with obstacles, random initial weights (the speed does not depend
    on them).  Plain SPH steps and surrogate calls (graph, layers, Euler step,
    cell rebuild) are timed with CUDA events on the simulation's stream;
    both sides advance the same simulated time per SPH step.  Accuracy needs
    trained weights and comes from the training runs, not from here."""
    from paper_1210_1017_gb300 import cases
    from paper_1210_1017_gb300 import surrogate as U
    from paper_1210_1017_gb300 import surrogate_train as T
    layers, per_call, radius = 2, 16, 0.65
    case = cases.c2_dam_break_obstacles()
    st = torch.cuda.Stream(device)
    sim = S.Simulation.from_case(case, device=device, stream=st)
    sim.build_cells()
    sim.autotune(reps=2, cache=False)
    sim.step(args.warmup)
    sim.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    d0 = sim.diagnostics()
    e0.record(st)
    sim.step(per_call * calls)
    e1.record(st)
    e1.synchronize()
    d1 = sim.diagnostics()
    sph_s = e0.elapsed_time(e1) / 1e3
    dt = (d1["t"] - d0["t"]) / (per_call * calls)
    sur = U.Surrogate(sim, layers=layers, train=False, v_scale=1.0, dt_s=per_call * dt,
                      edges_per_node=30, radius=radius)
    sur.set_params(T.init_params(layers, 0))
    hist = torch.zeros((case.n, 15), dtype=torch.float32, device=sim.device)
    sim.build_cells()
    for _ in range(2):
        sur.advance(hist)
        sim.build_cells()
    sim.synchronize()
    e0.record(st)
    for _ in range(calls):
        sur.advance(hist)
        sim.build_cells()
    e1.record(st)
    e1.synchronize()
    sur_s = e0.elapsed_time(e1) / 1e3
    sph_rate = per_call * calls * dt / sph_s
    sur_rate = per_call * calls * dt / sur_s
    rec = {"workload": "dam_break_obstacles_1m", "n_particles": case.n, "layers": layers,
           "latent": 128, "sph_steps_per_call": per_call, "edge_radius_2h": radius,
           "edges": sur.num_edges, "calls": calls, "ms_per_call": round(sur_s / calls * 1e3, 3),
           "sph_ms_per_step": round(sph_s / (per_call * calls) * 1e3, 4),
           "sim_s_per_wall_s": sur_rate, "sph_sim_s_per_wall_s": sph_rate,
           "speedup_vs_sph": sur_rate / sph_rate, "weights": "random initialisation",
           "note": ("speed only; accuracy of the trained variant (RMSE / dp, front) is "
                    "measured by surrogate_train.py runs")}
    sur.close()
    sim.close()
    return rec


def ensemble_record(args, S, torch, device, steps):
    """The batched configuration as a nested record of the default line: the
    256-member ensemble of uneven dam breaks (fluid blocks drawn from
    U[0.2, 0.6] m, 5.47M particles), ``steps`` lockstep steps issued as one
    sph_step call (one launch of the step graph, whose conditional WHILE node
    repeats the step on the device), timed with CUDA events on the
    simulation's stream after a warm-up, with its own clock samples.
    ``device`` is this rank's CUDA device index."""
    from paper_1210_1017_gb300 import cases
    ens = cases.dam_break_ensemble(256, t_end=1.0)
    sim = S.Simulation.from_ensemble(ens, device=device)
    sim.build_cells()
    variant, _ = sim.autotune(reps=2, cache=False)
    sim.step(args.warmup)
    sim.synchronize()
    d0 = sim.diagnostics()
    i0 = sim.instance_state()
    sampler = ClockSampler(device)
    sampler.start()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(sim.stream)
    sim.step(steps)
    e1.record(sim.stream)
    e1.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    d1 = sim.diagnostics()
    i1 = sim.instance_state()
    sim.check()
    member_steps = int((i1["steps"] - i0["steps"]).sum())
    pairs = d1["pairs_total"] - d0["pairs_total"]
    rec = {"workload": "dam_break_ensemble_256", "members": len(ens.members),
           "n_particles": ens.n,
           "member_sizes": [int(min(c.n for c in ens.cases)), int(max(c.n for c in ens.cases))],
           "steps": steps, "ms_per_step": ms / steps, "steps_per_s": steps / (ms * 1e-3),
           "member_steps_per_s": member_steps / (ms * 1e-3),
           "pairs_per_s": pairs / (ms * 1e-3), "interaction_variant": variant,
           "gpu_launches": (sim.kernels_per_step() + 1) * steps + 1,
           "launch": "one sph_step call: one CUDA graph launch whose conditional WHILE node "
                     "runs the step body on the device",
           "clocks": clocks}
    sim.close()
    return rec


def subdomain_timing(sim, case, nsub, S, torch):
    """Sec. 4.3 selection on the current state for nsub equal slabs along
    x of the particles' range: per slab, the edge particles that would build
    the neighbours' halos (labels, (label, id) sort, copy into device
    buffers).  Wall time per call (the call synchronises; it includes the
    host read of the counts)."""
    if is_ensemble(case):
        return None
    sim.build_cells()
    st = sim.download()
    x0, x1 = float(st["pos"][:, 0].min()), float(st["pos"][:, 0].max()) * (1 + 1e-12) + 1e-9
    edges = np.linspace(x0, x1, nsub + 1)
    n = case.n
    dev = sim.device
    out = dict(pos=torch.empty((n, 3), dtype=torch.float64, device=dev),
               vel=torch.empty((n, 3), dtype=torch.float32, device=dev),
               rho=torch.empty(n, dtype=torch.float32, device=dev),
               ids=torch.empty(n, dtype=torch.int32, device=dev))
    ms, sel = [], []
    for lo, hi in zip(edges[:-1], edges[1:]):
        args = (sim.ctx, S.SPH_SUBDOMAIN_EDGE, lo, hi, n, out["pos"], out["vel"], out["rho"],
                out["ids"])
        S.sph_subdomain_select(*args)                       # warm
        reps = 5
        t = time.perf_counter()
        for _ in range(reps):
            c = S.sph_subdomain_select(*args)
        ms.append(round((time.perf_counter() - t) / reps * 1e3, 3))
        sel.append(int(c[1]) + int(c[2]))
    return {"slabs": nsub, "mode": "edge", "ms_per_call": ms, "selected": sel,
            "note": "labels of all particles, (label, id) radix sort of the selected, copy "
                    "into device buffers; wall time per synchronous call"}


def run_surrogate(args):
    """The learned surrogate on the 1.39M-particle dam break with obstacles:
    simulated seconds per wall second of surrogate calls (each advances 4 SPH
    steps: graph, 10 message-passing layers on the tensor cores, Euler step,
    cell rebuild) next to the plain GPU SPH on the same case.  Weights are
    the random initialisation: the speed does not depend on them."""
    import torch

    from paper_1210_1017_gb300 import cases
    from paper_1210_1017_gb300 import sph as S
    from paper_1210_1017_gb300 import surrogate as U
    from paper_1210_1017_gb300 import surrogate_train as T

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    S.lib(build=True)
    # surrogate_block_50k: a 50,000-particle jittered block (about 3.5M
    # edges, a few GB of workspace) for kernel captures; it skips the
    # standalone 16M-edge kernel timing below
    small = args.workload == "surrogate_block_50k"
    case = cases.random_block(50000, seed=41, jitter=0.3) if small else \
        cases.c2_dam_break_obstacles()
    st = torch.cuda.Stream()
    sim = S.Simulation.from_case(case, device=local, stream=st)
    sim.build_cells()
    sim.autotune(reps=3)
    for _ in range(args.warmup):
        sim.step(1)
    sim.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    d0 = sim.diagnostics()
    e0.record(st)
    sim.step(4 * args.steps)
    e1.record(st)
    e1.synchronize()
    d1 = sim.diagnostics()
    sph_s = e0.elapsed_time(e1) / 1e3
    sph_sim = d1["t"] - d0["t"]
    dt = sph_sim / (4 * args.steps)
    sur = U.Surrogate(sim, layers=10, train=False, v_scale=1.0, dt_s=4 * dt, edges_per_node=80)
    sur.set_params(T.init_params(10, 0))
    hist = torch.zeros((case.n, 15), dtype=torch.float32, device=sim.device)
    sim.build_cells()
    for _ in range(args.warmup):
        sur.advance(hist)
        sim.build_cells()
    sampler = ClockSampler(local)
    sampler.start()
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(args.steps):
        sur.advance(hist)
        sim.build_cells()
    e1.record(st)
    e1.synchronize()
    clocks = sampler.stop()
    sur_s = e0.elapsed_time(e1) / 1e3
    n_edges = sur.num_edges
    value = args.steps * 4 * dt / sur_s
    # dominant kernel: the fused edge update (two K = N = 128 GEMMs per tile),
    # run on its own over 16M edges with 2M-node tables (inputs larger than
    # L2); algorithmic bytes per edge: e read 256 + e' written 256 (the
    # gathered node rows are counted once per node)
    M, nodes = (1 << 24, 1 << 21) if not small else (1 << 20, 1 << 17)
    dev = sim.device
    E = torch.randn((M, 128), device=dev).to(torch.bfloat16)
    Eo = torch.empty((M, 128), dtype=torch.bfloat16, device=dev)
    Wt = (torch.randn((128, 128), device=dev) / 11.3).to(torch.bfloat16)
    bias = torch.zeros(128, device=dev)
    P = torch.randn((nodes, 128), device=dev).to(torch.bfloat16)
    src = torch.sort(torch.randint(0, nodes, (M,), device=dev, dtype=torch.int32)).values
    dst = torch.clamp(src + torch.randint(-64, 65, (M,), device=dev, dtype=torch.int32), 0,
                      nodes - 1)
    cs = torch.cuda.current_stream()
    for _ in range(3):
        U.sur_edge_layer(E, Wt, Wt, bias, bias, P, P, src, dst, M, None, Eo, cs.cuda_stream)
    e0.record(cs)
    for _ in range(10):
        U.sur_edge_layer(E, Wt, Wt, bias, bias, P, P, src, dst, M, None, Eo, cs.cuda_stream)
    e1.record(cs)
    e1.synchronize()
    t_gemm = e0.elapsed_time(e1) / 10 / 1e3
    pk, src_pk = peaks()
    gbs = (2 * 256 * M + 2 * 256 * nodes) / t_gemm / 1e9
    line = {"metric": "surrogate simulated s per wall s", "value": value, "unit": "sim-s/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sur_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": args.workload, "n_particles": case.n, "edges": n_edges,
                       "layers": 10, "latent": 128, "sph_steps_per_call": 4, "dt": dt,
                       "weights": "random initialisation"},
            "sph_sim_per_s": sph_sim / sph_s, "speedup_vs_sph": value / (sph_sim / sph_s),
            "edges_per_s": n_edges * args.steps / sur_s,
            "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": pk["hbm_gbs"],
                         "unit": "GB/s", "frac": round(gbs / pk["hbm_gbs"], 4), "traffic": None,
                         "kernel": (f"k_edge_pp (fused edge update of a layer), {M >> 20}M edges, "
                                    f"{nodes >> 10}k nodes"),
                         "ms_per_launch": round(t_gemm * 1e3, 4)},
            "gpu_launches": None, "clocks": clocks, "peaks_source": src_pk}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_surrogate_variant(args):
    """The fastest surrogate variant on its own line: the default line's nested
    surrogate_1m record (2 layers, 16 SPH steps per call, edges within
    0.65 2h, the 1.39M-particle dam break with obstacles) over --steps calls,
    with the clocks sampled around it."""
    import torch

    from paper_1210_1017_gb300 import sph as S
    torch.cuda.set_device(0)
    sampler = ClockSampler(0)
    sampler.start()
    rec = surrogate_record(args, S, torch, 0, calls=max(args.steps, 1))
    clocks = sampler.stop()
    keys = ("n_particles", "layers", "latent", "sph_steps_per_call", "edge_radius_2h", "edges",
            "weights")
    line = {"metric": "surrogate simulated s per wall s", "value": rec["sim_s_per_wall_s"],
            "unit": "sim-s/s", "n_gpus": 1, "steps": rec["calls"], "warmup": args.warmup,
            "ms_per_step": rec["ms_per_call"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": args.workload, **{k: rec[k] for k in keys}},
            "sph_sim_per_s": rec["sph_sim_s_per_wall_s"], "sph_ms_per_step": rec["sph_ms_per_step"],
            "speedup_vs_sph": rec["speedup_vs_sph"], "gpu_launches": None, "clocks": clocks,
            "note": rec["note"]}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dam_break_32m", choices=WORKLOADS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true",
                    help="skip the nested 256-member ensemble record of the default line")
    ap.add_argument("--formulation", default="default", choices=sorted(FORMULATIONS))
    ap.add_argument("--subdomains", type=int, default=0,
                    help="also time the Sec. 4.3 edge selection for this many slabs")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "surrogate_variant_1m":
        return run_surrogate_variant(args)
    if args.workload in ("surrogate_obstacles_1m", "surrogate_block_50k"):
        return run_surrogate(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
