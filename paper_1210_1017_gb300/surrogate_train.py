"""Training data, training loop and rollout evaluation of the learned
surrogate, all on one GPU through the C ABI (include/sph.h, include/sur.h).

* Data: groups of dam-break ensemble members run by the GPU SPH with a fixed
  step (the smallest adaptive step of a pilot run), positions saved by id
  every ``steps_per_frame`` steps into device memory (frames spaced dt_s).
* Samples: seven consecutive frames of a group -> noisy input state,
  velocity history and normalised target acceleration (sur_make_sample).
* Training: forward, backward and Adam on the tensor-core kernels of the
  library; a sample is one whole group (all its members at one time).
* Evaluation: surrogate rollouts against the SPH frames (position RMSE / dp,
  front position, kinetic + potential energy) and against constant-velocity
  extrapolation (the update without a learned acceleration).

PyTorch only holds device memory and streams here; the statistics of the
data (means, standard deviations) and the error metrics are plain tensor
reductions outside the hot path.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import cases
from . import sph as S
from . import surrogate as U


# ------------------------------------------------------------------- data --

@dataclass
class Group:
    """Ensemble members simulated together, with their saved frames."""
    ens: "cases.Ensemble"
    sim: "S.Simulation"
    frames: object = None           # torch float64 (F, n, 3) by id
    dt: float = 0.0                 # SPH step
    steps_per_frame: int = 4
    fluid: object = None            # torch bool (n,) by id

    @property
    def n(self):
        return self.ens.n

    @property
    def dt_s(self):
        return self.dt * self.steps_per_frame


def make_group(specs, dp=0.02, t_end=1.0, stream=None, dt_fixed=0.0):
    ens = cases.ensemble([cases.ensemble_instance(sp, dp=dp) for sp in specs], t_end=t_end)
    sim = S.Simulation(ens.params, ens.n, members=ens.members, stream=stream, dt_fixed=dt_fixed)
    sim.upload(ens.pos, ens.vel, ens.rho, ens.ids)
    return Group(ens=ens, sim=sim)


def pilot_dt(group: Group, t_end: float, chunk: int = 100) -> float:
    """Smallest adaptive CFL step over all members until t_end (the fixed
    step of the data runs)."""
    sim = group.sim
    sim.upload(group.ens.pos, group.ens.vel, group.ens.rho, group.ens.ids)
    dt_min = math.inf
    while True:
        sim.step(chunk)
        st = sim.instance_state()
        t, dt, done = st["t"], st["dt"], st["done"]
        live = dt > 0
        if live.any():
            dt_min = min(dt_min, float(dt[live].min()))
        if done.all() or float(t.min()) >= t_end:
            break
    return dt_min


def record(group: Group, dt: float, n_frames: int, steps_per_frame: int = 4):
    """Run the group with the fixed step dt from its initial state and keep
    n_frames position frames by id (device, float64), steps_per_frame steps
    apart."""
    import torch
    ens = group.ens
    sim = S.Simulation(ens.params, ens.n, members=ens.members, stream=group.sim.stream,
                       dt_fixed=dt)
    sim.upload(ens.pos, ens.vel, ens.rho, ens.ids)
    frames = torch.empty((n_frames, ens.n, 3), dtype=torch.float64, device=sim.device)
    for f in range(n_frames):
        if f:
            sim.step(steps_per_frame)
        sim.download_by_id(pos=frames[f])
    sim.check()
    group.sim.close()
    group.sim = sim
    group.frames = frames
    group.dt = dt
    group.steps_per_frame = steps_per_frame
    fluid = np.ones(ens.n, bool)
    for q, m in enumerate(ens.members):
        b = int(ens.id_base[q])
        fluid[b:b + int(m["n_bound"])] = False
    group.fluid = torch.tensor(fluid, device=sim.device)
    return group


def data_stats(groups):
    """Velocity scale and per-axis mean / std of the (clean) finite-difference
    accelerations over the fluid particles of all frames."""
    import torch
    vs, acc = [], []
    for g in groups:
        fr = g.frames[:, g.fluid]
        v = (fr[1:] - fr[:-1]) / g.dt_s
        a = (fr[2:] - 2 * fr[1:-1] + fr[:-2]) / g.dt_s ** 2
        vs.append(v.reshape(-1, 3))
        acc.append(a.reshape(-1, 3))
    v = torch.cat(vs)
    a = torch.cat(acc)
    v_scale = float(v.pow(2).mean().sqrt())
    a_mean = tuple(float(x) for x in a.mean(0))
    a_std = tuple(max(float(x), 1e-3) for x in a.std(0))
    return v_scale, a_mean, a_std


# ----------------------------------------------------------- parameters --

def layer_list(layers: int):
    """(name, kin, kout, has_bias) in the order of the flat parameter array
    of include/sur.h."""
    L, K = 128, 16
    out = [("enc_n0", K, L, True), ("enc_n1", L, L, True),
           ("enc_e0", K, L, True), ("enc_e1", L, L, True)]
    for l in range(layers):
        out += [(f"mp{l}_w1a", L, L, False), (f"mp{l}_w1b", L, L, False),
                (f"mp{l}_w1c", L, L, True), (f"mp{l}_w2", L, L, True),
                (f"mp{l}_w3", 2 * L, L, True), (f"mp{l}_w4", L, L, True)]
    out += [("dec0", L, L, True), ("dec1", L, K, True)]
    return out


def init_params(layers: int, seed: int = 0, mean_degree: float = 50.0,
                residual_gain: float = 0.1) -> np.ndarray:
    """Initial weights: He-normal for layers feeding a ReLU, 1/sqrt(kin)
    times ``residual_gain`` for the residual branches, the aggregate half of
    W3 scaled by 1/mean_degree (the sum runs over that many edges), a small
    last decoder layer and zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, ki, ko, has_b in layer_list(layers):
        if name.endswith(("w2", "w4")):
            W = rng.normal(0, residual_gain / math.sqrt(ki), (ki, ko))
        elif name in ("enc_n1", "enc_e1"):
            W = rng.normal(0, 1.0 / math.sqrt(ki), (ki, ko))
        elif name == "dec1":
            W = rng.normal(0, 0.01 / math.sqrt(ki), (ki, ko))
        else:
            W = rng.normal(0, math.sqrt(2.0 / ki), (ki, ko))
        if name.endswith("w3"):
            W[ki // 2:] /= mean_degree
        if name.endswith(("w1a", "w1b", "w1c")):
            W /= math.sqrt(3.0)          # three terms enter the same ReLU
        parts.append(W.ravel())
        if has_b:
            parts.append(np.zeros(ko))
    return np.concatenate(parts).astype(np.float32)


# --------------------------------------------------------------- training --

@dataclass
class TrainLog:
    step: list = field(default_factory=list)
    loss: list = field(default_factory=list)
    seconds: float = 0.0
    samples: int = 0
    nodes: int = 0
    edges: int = 0


class Trainer:
    """One surrogate context serving several groups (same stream)."""

    def __init__(self, groups, layers=10, sigma=3e-4, seed=0, edges_per_node=80, stats=None,
                 train=True, max_nodes=0, radius=1.0):
        import torch
        self.torch = torch
        self.groups = groups
        self.layers = layers
        self.radius = radius
        self.sigma = sigma
        self.rng = np.random.default_rng(seed)
        self.seed = seed
        self.dt_s = groups[0].dt_s
        for g in groups:
            assert abs(g.dt_s - self.dt_s) < 1e-15 * max(1.0, self.dt_s) + 1e-18
        self.v_scale, self.a_mean, self.a_std = stats or data_stats(groups)
        nmax = max(max(g.n for g in groups), int(max_nodes))
        dev = groups[0].sim.device
        self.sur = U.Surrogate(groups[0].sim, layers=layers, train=train, v_scale=self.v_scale,
                               a_mean=self.a_mean, a_std=self.a_std, dt_s=self.dt_s,
                               max_nodes=nmax, max_edges=nmax * edges_per_node, radius=radius)
        self.sur.set_params(init_params(layers, seed))
        f64, f32 = torch.float64, torch.float32
        self.pos = torch.empty((nmax, 3), dtype=f64, device=dev)
        self.vel = torch.empty((nmax, 3), dtype=f32, device=dev)
        self.hist = torch.empty((nmax, 15), dtype=f32, device=dev)
        self.tgt = torch.empty((nmax, 3), dtype=f32, device=dev)
        self.rho = torch.full((nmax,), float(groups[0].ens.params["rho0"]), dtype=f32,
                              device=dev)
        self.ids = torch.arange(nmax, dtype=torch.int32, device=dev)
        self.log = TrainLog()

    def load_sample(self, g: Group, k: int, sigma: float, seed: int):
        """Frames k-5 .. k+1 of group g -> the group's SPH state (noisy x^k,
        v^k, cells built), velocity history and target."""
        n = g.n
        self.sur.bind(g.sim)
        self.sur.make_sample(g.frames[k - 5], sigma, seed, self.pos, self.vel, self.hist,
                             self.tgt)
        g.sim.upload(self.pos[:n], self.vel[:n], self.rho[:n], self.ids[:n])
        g.sim.build_cells()

    def step(self, lr: float):
        g = self.groups[int(self.rng.integers(len(self.groups)))]
        k = int(self.rng.integers(5, g.frames.shape[0] - 1))
        self.load_sample(g, k, self.sigma, self.seed * 1000003 + self.log.samples)
        self.sur.forward(self.hist, None)
        loss = self.sur.backward(self.tgt)
        self.sur.adam(lr)
        self.log.samples += 1
        self.log.nodes += g.n
        self.log.edges += self.sur.num_edges
        return loss

    def train(self, steps: int, lr0=1e-4, lr1=1e-6, log_every=50, verbose=False):
        """Adam with the learning rate decaying exponentially from lr0 to lr1."""
        t0 = time.perf_counter()
        for i in range(steps):
            lr = lr0 * (lr1 / lr0) ** (i / max(steps - 1, 1))
            loss = self.step(lr)
            if not math.isfinite(loss):
                raise FloatingPointError(f"loss {loss} at step {i}")
            if i % log_every == 0 or i == steps - 1:
                self.log.step.append(i)
                self.log.loss.append(loss)
                if verbose:
                    print(f"step {i:6d}  loss {loss:.5f}  lr {lr:.2e}", flush=True)
        self.groups[0].sim.synchronize()
        self.log.seconds += time.perf_counter() - t0
        return self.log

    def one_step_loss(self, g: Group, ks, sigma=0.0):
        """Mean loss (normalised acceleration MSE) of the current weights on
        frames ks of group g, without training, and the same for a zero
        prediction (the constant-velocity update) for comparison."""
        torch = self.torch
        net, zero = [], []
        for k in ks:
            self.load_sample(g, int(k), sigma, 0)
            self.sur.forward(self.hist, None)
            net.append(self.sur.backward(self.tgt))      # loss only; no Adam step
            a = self.tgt[:g.n][g.fluid]
            # zero predicted acceleration: out = -a_mean / a_std
            am = torch.tensor(self.a_mean, device=a.device, dtype=a.dtype)
            sd = torch.tensor(self.a_std, device=a.device, dtype=a.dtype)
            zero.append(float(((-am / sd - a) ** 2).sum(1).mean()))
        return float(np.mean(net)), float(np.mean(zero))


# ------------------------------------------------------------- evaluation --

def member_of(ens):
    """Member index of every particle id (numpy)."""
    q = np.zeros(ens.n, np.int64)
    for m in range(len(ens.members)):
        q[int(ens.id_base[m]):int(ens.id_base[m + 1])] = m
    return q


def metrics(ens, pos, ref, fluid, dp, g=9.81, vel=None, mass=None):
    """Position RMSE / dp over fluid particles, mean |front difference| over
    members (front: largest x of fluid particles within 2 dp of the floor,
    the floor being each member's lowest fluid z at t = 0 minus dp / 2) and
    the per-member fronts.  pos, ref: (n, 3) by id (torch or numpy)."""
    pos = np.asarray(pos.cpu() if hasattr(pos, "cpu") else pos)
    ref = np.asarray(ref.cpu() if hasattr(ref, "cpu") else ref)
    fluid = np.asarray(fluid.cpu() if hasattr(fluid, "cpu") else fluid)
    d = pos[fluid] - ref[fluid]
    rmse = float(np.sqrt((d * d).sum(1).mean())) / dp
    q = member_of(ens)
    fronts = []
    for m in range(len(ens.members)):
        sel = fluid & (q == m)
        z0 = float(ens.pos[np.argsort(ens.ids)][sel][:, 2].min()) - 0.5 * dp
        lo = lambda p: p[sel][p[sel][:, 2] < z0 + 2 * dp]
        fa, fb = lo(pos), lo(ref)
        fronts.append((float(fa[:, 0].max()) if len(fa) else float("nan"),
                       float(fb[:, 0].max()) if len(fb) else float("nan")))
    fr = np.array(fronts)
    return dict(rmse_dp=rmse, front_err=float(np.nanmean(np.abs(fr[:, 0] - fr[:, 1]))),
                fronts=fronts)


def mechanical_energy(pos_prev, pos, dt_s, fluid, mass, g=9.81):
    """Kinetic (finite-difference velocity) plus potential energy of the
    fluid particles, in joules (float64 numpy)."""
    p0 = np.asarray(pos_prev.cpu() if hasattr(pos_prev, "cpu") else pos_prev)[fluid]
    p1 = np.asarray(pos.cpu() if hasattr(pos, "cpu") else pos)[fluid]
    v = (p1 - p0) / dt_s
    return float(mass * (0.5 * (v * v).sum() + g * p1[:, 2].sum()))


def rollout(trainer: Trainer, g: Group, k0: int, n_calls: int, every: int = 1):
    """Surrogate rollout of group g from frame k0 (history from frames
    k0-5..k0, no noise) for n_calls calls; returns [(call, pos by id)] every
    ``every`` calls and the seconds per call (advance + cell rebuild, timed
    on the stream)."""
    torch = trainer.torch
    sur = trainer.sur
    trainer.load_sample(g, k0, 0.0, 0)
    hist = trainer.hist[:g.n].clone()
    out = []
    st = g.sim.stream
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    secs = 0.0
    for c in range(1, n_calls + 1):
        ev0.record(st)
        sur.advance(hist)
        g.sim.build_cells()
        ev1.record(st)
        ev1.synchronize()
        secs += ev0.elapsed_time(ev1) / 1e3
        if c % every == 0 or c == n_calls:
            p = torch.empty((g.n, 3), dtype=torch.float64, device=g.sim.device)
            g.sim.download_by_id(pos=p)
            out.append((c, p))
    return out, secs / n_calls


def evaluate_group(trainer: Trainer, g: Group, k0: int, n_calls: int, every: int = 10):
    """Surrogate and constant-velocity rollouts against the group's SPH
    frames: per saved call, RMSE / dp and front error of both."""
    dp = float(g.ens.params["dp"])
    fluid = g.fluid.cpu().numpy()
    n_calls = min(n_calls, g.frames.shape[0] - 1 - k0)
    traj, spc = rollout(trainer, g, k0, n_calls, every)
    x0, xm = g.frames[k0], g.frames[k0 - 1]
    rows = []
    for c, p in traj:
        ref = g.frames[k0 + c]
        cv = x0 + c * (x0 - xm)             # constant-velocity extrapolation
        ms = metrics(g.ens, p, ref, fluid, dp)
        mc = metrics(g.ens, cv, ref, fluid, dp)
        rows.append(dict(call=c, t=c * g.dt_s, rmse_dp=ms["rmse_dp"], front_err=ms["front_err"],
                         cv_rmse_dp=mc["rmse_dp"], cv_front_err=mc["front_err"]))
    return rows, spc


def evaluate_case(trainer: Trainer, case, t_sim: float, every: int = 10, pilot_t: float = None,
                  edges_per_node: int = 80, sph_steps_timed: int = 200, steps_per_call: int = 4):
    """The trained network on a standalone case (its own resolution and
    step) against the GPU SPH on the same case: both start from rest, the
    SPH runs with the fixed step dt (smallest adaptive step of a pilot run)
    and the surrogate advances steps_per_call dt per call.  Returns per saved
    call the position RMSE / dp and front error, and the simulated seconds
    per wall second of both."""
    K = int(steps_per_call)
    import torch
    st = trainer.groups[0].sim.stream
    g = Group(ens=cases.ensemble([case]), sim=None)
    g.sim = S.Simulation(case.params(), case.n, stream=st)
    dt = pilot_dt(g, pilot_t if pilot_t is not None else min(t_sim, 0.2))
    n_calls = int(round(t_sim / (K * dt)))
    # SPH frames: 6 initial frames K steps apart, then every `every` calls
    sim = S.Simulation(case.params(), case.n, stream=st, dt_fixed=dt)
    sim.upload(case.pos, case.vel, case.rho, case.ids)
    dev = sim.device
    first = torch.empty((7, case.n, 3), dtype=torch.float64, device=dev)
    for f in range(7):
        if f:
            sim.step(K)
        sim.download_by_id(pos=first[f])
    ref = {}
    c = 1                      # frame 6 = call 1 after frame 5
    ref[1] = first[6].clone()
    while c < n_calls:
        k = min(every - (c % every) if c % every else every, n_calls - c)
        sim.step(K * k)
        c += k
        p = torch.empty((case.n, 3), dtype=torch.float64, device=dev)
        sim.download_by_id(pos=p)
        ref[c] = p
    # SPH speed: fixed-step steps timed on the stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sim.step(20)
    e0.record(st)
    sim.step(sph_steps_timed)
    e1.record(st)
    e1.synchronize()
    sph_sps = dt * sph_steps_timed / (e0.elapsed_time(e1) / 1e3)
    sim.close()
    # surrogate on the case, same weights and normalisation, this case's step
    g.frames, g.dt, g.steps_per_frame = first, dt, K
    g.fluid = torch.tensor(np.arange(case.n) >= case.n_bound, device=dev)   # by id
    sur = U.Surrogate(g.sim, layers=trainer.layers, train=False, v_scale=trainer.v_scale,
                      a_mean=trainer.a_mean, a_std=trainer.a_std, dt_s=K * dt,
                      max_nodes=case.n, max_edges=case.n * edges_per_node,
                      radius=getattr(trainer, "radius", 1.0))
    sur.set_params(trainer.sur.params())
    ev = Trainer.__new__(Trainer)
    ev.torch, ev.sur = torch, sur
    f64, f32 = torch.float64, torch.float32
    ev.pos = torch.empty((case.n, 3), dtype=f64, device=dev)
    ev.vel = torch.empty((case.n, 3), dtype=f32, device=dev)
    ev.hist = torch.empty((case.n, 15), dtype=f32, device=dev)
    ev.tgt = torch.empty((case.n, 3), dtype=f32, device=dev)
    ev.rho = torch.full((case.n,), float(case.rho0), dtype=f32, device=dev)
    ev.ids = torch.arange(case.n, dtype=torch.int32, device=dev)
    traj, spc = rollout(ev, g, 5, n_calls, every)
    dp = float(case.dp)
    fluid = g.fluid.cpu().numpy()
    rows = []
    for c, p in traj:
        if c not in ref:
            continue
        m = metrics(g.ens, p, ref[c], fluid, dp)
        rows.append(dict(call=c, t=c * K * dt, rmse_dp=m["rmse_dp"], front_err=m["front_err"]))
    sur_sps = K * dt / spc
    sur.close()
    g.sim.close()
    return dict(dt=dt, calls=n_calls, rows=rows, sur_seconds_per_call=spc, sur_sim_per_s=sur_sps,
                sph_sim_per_s=sph_sps, speedup=sur_sps / sph_sps, n=case.n)


def main(argv=None):
    """Train on dam-break ensemble members and evaluate (JSON report)."""
    import argparse
    import json
    import torch
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--out", required=True)
    ap.add_argument("--group-size", type=int, default=8)
    ap.add_argument("--train-groups", type=int, default=3)
    ap.add_argument("--t-end", type=float, default=1.0)
    ap.add_argument("--layers", type=int, default=10)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--lr0", type=float, default=3e-4)
    ap.add_argument("--lr1", type=float, default=1e-5)
    ap.add_argument("--sigma", type=float, default=3e-6)
    ap.add_argument("--eval-calls", type=int, default=1000)
    ap.add_argument("--case-seconds", type=float, default=0.1)
    ap.add_argument("--case", default="c2", choices=["c2", "none"])
    ap.add_argument("--save-params", default=None)
    ap.add_argument("--steps-per-call", type=int, default=4,
                    help="SPH steps one surrogate call advances (frames are this many apart)")
    ap.add_argument("--radius", type=float, default=1.0,
                    help="graph edge radius as a fraction of 2h (sparser graph below 1)")
    ap.add_argument("--case-every", type=int, default=10,
                    help="surrogate calls between the compared frames of the case")
    a = ap.parse_args(argv)
    report = dict(args=vars(a))
    t0 = time.perf_counter()
    st = torch.cuda.Stream()
    specs = cases.ensemble_specs(256, seed=1017)
    gs = a.group_size
    groups = [make_group(specs[i * gs:(i + 1) * gs], t_end=a.t_end, stream=st)
              for i in range(a.train_groups + 1)]
    dt = min(pilot_dt(g, a.t_end) for g in groups)
    K = a.steps_per_call
    n_frames = int(a.t_end / (K * dt)) + 1
    for g in groups:
        record(g, dt, n_frames, steps_per_frame=K)
    train, held = groups[:-1], groups[-1]
    report["data"] = dict(dt=dt, dt_s=K * dt, frames=n_frames,
                          train_particles=[g.n for g in train], held_particles=held.n,
                          seconds=time.perf_counter() - t0)
    print(json.dumps(report["data"]), flush=True)
    tr = Trainer(train, layers=a.layers, sigma=a.sigma, seed=0, max_nodes=held.n,
                 radius=a.radius)
    report["stats"] = dict(v_scale=tr.v_scale, a_mean=tr.a_mean, a_std=tr.a_std)
    ks = range(10, n_frames - 2, max(1, (n_frames - 12) // 8))
    report["untrained_held_one_step"], report["zero_held_one_step"] = tr.one_step_loss(held, ks)
    tr.sur.bind(train[0].sim)
    log = tr.train(a.steps, lr0=a.lr0, lr1=a.lr1, log_every=50, verbose=True)
    report["train"] = dict(steps=log.step, loss=log.loss, seconds=log.seconds,
                           samples=log.samples, nodes=log.nodes, edges=log.edges,
                           edges_per_s=log.edges / log.seconds)
    report["trained_held_one_step"], _ = tr.one_step_loss(held, ks)
    if a.save_params:
        np.save(a.save_params, tr.sur.params())
    tr.sur.bind(held.sim)
    rows, spc = evaluate_group(tr, held, 5, a.eval_calls, every=25)
    report["held_rollout"] = dict(rows=rows, seconds_per_call=spc)
    print(json.dumps(report["held_rollout"]["rows"][-1]), flush=True)
    if a.case == "c2":
        report["c2"] = evaluate_case(tr, cases.c2_dam_break_obstacles(), a.case_seconds,
                                     every=a.case_every, steps_per_call=K)
        print(json.dumps({k: v for k, v in report["c2"].items() if k != "rows"}), flush=True)
    report["seconds"] = time.perf_counter() - t0
    with open(a.out, "w") as f:
        json.dump(report, f, indent=1)


if __name__ == "__main__":
    main()
