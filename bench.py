#!/usr/bin/env python
"""Throughput of the batched position-based collocation rollout on B300.

Workload (default): 4096 independent 3D serial chains of 10 capsule links
with ball joints (exponential-map coordinates), link lengths U[0.5, 1.5],
masses lognormal(0, 0.3), dt = 0.033, three collocation stages, L-BFGS
history 8, 100 time steps in one persistent launch captured in a CUDA graph.
One bench step = one full 100-step rollout of the whole batch from the same
seeded initial state. Metric: link-steps/s = instances * links * time steps /
time.

Prints one JSON line (rank 0). See --help for the knobs.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "link-steps/s on 1 B300, batched vs plain; fwd+adjoint rollout ms; % FP64 peak"
UNIT = "link-steps/s"

# Algorithmic FP64 flops of one objective evaluation, per link and per stage
# (FMA = 2 flops), counted from the formulas of the residual pass (forward
# kinematics, seeds of Eq. HOC, wrench, joint contraction) and of the tangent
# pass (S >= 2); the stage coupling adds 24 S per pass. sincos calls are not
# counted as flops.
PRIMAL_FLOPS = {0: 347, 1: 540}    # hinge, ball
TANGENT_FLOPS = {0: 327, 1: 680}
ENERGY_FLOPS = 54                   # Eq. EQ energy terms (one stage only)
COUPLING_FLOPS = 24                 # per stage of the sum over stages, per pass

# DRAM bytes (read + write) per instance-evaluation of the rollout kernel,
# from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of the
# launch named by the key (mapping, stages, links), valid only for the kernel
# sources whose hash is stored with it: any change to the files the kernel's
# device code comes from (ROLLOUT_KERNEL_SOURCES) makes the roofline's
# traffic null until the kernel is captured again.
ROLLOUT_TRAFFIC = {
    # link mapping, 3 stages, 10 links: 4096 ball chains x 100 steps, five launches of
    # k_rollout_lp<3>: 50.58 MB read + 17.63 MB written over 5 x 56,195,050 evaluations
    (1, 3, 10): ("4ae377fb961b07f8b13c84a51632ba974a7080cb", 0.24274),
}


# the headers k_rollout_lp's device code is compiled from (its body, the
# per-lane passes, the launch arguments, the model layout, double-float)
ROLLOUT_KERNEL_SOURCES = ("pbad_device.cuh", "pbad_df64.cuh", "pbad_launch.cuh", "pbad_lp.cuh")


def csrc_hash(files=ROLLOUT_KERNEL_SOURCES) -> str:
    """SHA-1 of the named CUDA sources (the kernel the traffic figure
    describes)."""
    import hashlib
    h = hashlib.sha1()
    d = os.path.join(ROOT, "paper_1709_04145_b300", "csrc")
    for f in sorted(files):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()


def rollout_traffic(mapping, S, N, evals_total):
    """DRAM bytes of one rollout launch from the stored capture, or None."""
    rec = ROLLOUT_TRAFFIC.get((mapping, S, N))
    if rec is None or rec[0] != csrc_hash():
        return None
    return rec[1] * evals_total


def primal_flops_per_eval(jtypes, S):
    """Residual pass (and for one stage the energy terms) of one evaluation,
    all S stage lanes."""
    per_stage = 0
    for jt in jtypes:
        per_stage += PRIMAL_FLOPS[jt] + COUPLING_FLOPS * S
        if S == 1:
            per_stage += ENERGY_FLOPS
    return per_stage * S


def tangent_flops_per_eval(jtypes, S):
    """Tangent pass of the Eq. EQHOC gradient (S >= 2; for one stage the
    gradient is the residual itself)."""
    if S == 1:
        return 0
    return S * sum(TANGENT_FLOPS[jt] + COUPLING_FLOPS * S for jt in jtypes)


def rollout_flops(spec, S, m, evals, grads, iters):
    """Algorithmic flops of a rollout from its per-instance counters: every
    evaluation's residual pass, the tangent pass of the evaluations that
    formed the gradient, and the L-BFGS bookkeeping per iteration."""
    jt = spec.jtype.tolist()
    return (float(evals.sum()) * primal_flops_per_eval(jt, S) +
            float(grads.sum()) * tangent_flops_per_eval(jt, S) +
            float(iters.sum()) * lbfgs_flops_per_iter(spec.n_dof, S, m))


STATUS_NAMES = ("CONVERGED", "MAX_ITER", "LS_FAIL", "CHOL_FAIL", "NONFINITE", "STALLED")


def step_outcomes(out, sl=None):
    """Per-step outcome record of a rollout from its step logs: the fraction
    of instance-steps that ended in each status, the fraction solved
    (CONVERGED or STALLED) and the median / max |r|_2 at which the steps
    ended. sl selects a slice of instances (a bucket)."""
    import numpy as np
    st = out["step_status"].cpu().numpy()
    rn = out["step_rnorm"].cpu().numpy()
    if sl is not None:
        st, rn = st[:, sl], rn[:, sl]
    n = st.size
    frac = {nm: float((st == k).sum()) / n for k, nm in enumerate(STATUS_NAMES)}
    fin = np.isfinite(rn)
    return {"instance_steps": int(n),
            "fractions": {k: v for k, v in frac.items() if v > 0},
            "solved_fraction": frac["CONVERGED"] + frac["STALLED"],
            "exit_rnorm_median": float(np.median(rn[fin])) if fin.any() else None,
            "exit_rnorm_max": float(np.max(rn[fin])) if fin.any() else None,
            "exit_rnorm_nonfinite": int((~fin).sum())}


def lbfgs_flops_per_iter(n, S, m):
    """Two-loop recursion, preconditioner, dots and updates per iteration."""
    return S * n * (8 * m + 20 + 2 * 3 + 2 * S)


def parse():
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3, help="timed bench steps (rollouts)")
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--instances", type=int, default=4096)
    p.add_argument("--links", type=int, default=10)
    p.add_argument("--timesteps", type=int, default=100)
    p.add_argument("--max-iter", type=int, default=50, help="L-BFGS iteration cap per time step")
    p.add_argument("--tol", type=float, default=1e-8)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--e2e-steps", type=int, default=5,
                   help="steps of the end-to-end timing (at most --steps)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-clocks", action="store_true")
    p.add_argument("--cpu-sample-seconds", type=float, default=10.0)
    p.add_argument("--threads", type=int, default=0,
                   help="threads per block (0 = autotune the mapping and 32/64/128 threads on a "
                        "short rollout)")
    p.add_argument("--mapping", type=int, default=0,
                   help="instance-to-lane mapping when --threads is given: 0 one lane per stage, "
                        "1 one lane per stage and link")
    p.add_argument("--plain-instances", type=int, default=64,
                   help="instances timed in the plain form (one launch per instance-step)")
    p.add_argument("--plain-timesteps", type=int, default=2)
    p.add_argument("--throughput-instances", type=int, default=65536,
                   help="instances of the large-batch throughput point (0 = skip)")
    p.add_argument("--throughput-timesteps", type=int, default=20)
    p.add_argument("--uneven-steps", type=int, default=20,
                   help="steps of the uneven three-bucket batch (0 = skip)")
    p.add_argument("--max-iter-uneven", type=int, default=100)
    p.add_argument("--drag-steps", type=int, default=20,
                   help="steps of the swimmer-like drag workload (0 = skip)")
    p.add_argument("--f32-steps", type=int, default=20,
                   help="steps of the one-stage binary32-direction L-BFGS comparisons "
                        "(0 = skip the mixed-precision section)")
    p.add_argument("--dt-sweep", action="store_true",
                   help="add a step-size sweep of both solvers (ball and hinge chains, dt 0.001-0.128)")
    p.add_argument("--scaling-steps", type=int, default=50,
                   help="steps per rollout of the hinge-chain scaling study (0 = skip)")
    p.add_argument("--scaling-budget", type=float, default=60.0,
                   help="seconds per (links, solver) row of the scaling study: fewer steps are "
                        "run when a one-step probe says the requested ones would take longer")
    p.add_argument("--scaling-adjoint-budget", type=float, default=6.0,
                   help="seconds of forward work per row for its forward + adjoint timing")
    p.add_argument("--scaling-links", type=int, nargs="+", default=[25, 50, 100, 200])
    p.add_argument("--damped-links", type=int, default=200,
                   help="links of the damped-system (Gram + Cholesky) timing, S = 4; 0 skips it")
    p.add_argument("--max-iter-scaling", type=int, default=3,
                   help="iteration cap per step of the scaling study (a fixed budget: the study "
                        "compares the cost per iteration of the two solvers)")
    p.add_argument("--companion-steps-thin", type=int, default=20,
                   help="steps of the 0.05 m capsule variants")
    p.add_argument("--no-pendulum", dest="pendulum", action="store_false",
                   help="skip the plain-method pendulum (batch 1, 200 steps)")
    p.add_argument("--companion-steps", type=int, default=100,
                   help="steps of the headline batch solved by Newton and of the 0.05 m capsule "
                        "variants (0 = skip)")
    p.add_argument("--adjoint-steps", type=int, default=64,
                   help="steps of the differentiable humanoid rollout timed forward and forward+adjoint "
                        "(0 = skip; the workload defines 64)")
    return p.parse_args()


def workload(args, rank=0):
    from paper_1709_04145_b300 import inputs as I
    w = I.ball_chains(count=args.instances, n_links=args.links, seed_base=shard_seed_base(rank),
                      n_steps=args.timesteps)
    w["max_iter"] = args.max_iter
    w["tol"] = args.tol
    return w


# ------------------------------------------------------------- multi-rank
def shard_seed_base(rank: int) -> int:
    """Every rank integrates its own seeded batch (weak scaling: instances are
    independent, so the path shards with no data-path collective)."""
    return 2000 + 17 * rank


def max_over_ranks(x: float, dist, device) -> float:
    """The slowest rank's time (the job ends when the last rank ends)."""
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def job_throughput(units_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job units/s: all ranks' units over the slowest rank's time."""
    return units_per_rank * world / (ms_max / 1e3)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------- oracle
def _oracle_worker_init():
    """Pool initializer: imports the oracle and loads its library, so that the
    timed map runs no imports or builds."""
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    O.lib()


def _oracle_instance(job):
    """Runs the CPU oracle on one instance (spawned worker); returns its
    compute seconds, iterations and evaluations. fast: its L-BFGS evaluates
    with the O(N) path (Algorithm DERIV and its tangent) instead of the
    brute-force one."""
    import numpy as np
    from oracle import oracle as O
    spec, b, qp, qc, S, dt, m, tol, max_iter, n_steps, fast = job
    om = O.OracleModel.from_spec(spec, b)
    om.set_fast(fast)
    t0 = time.perf_counter()
    res = om.rollout(S, dt, qp, qc, np.zeros((n_steps, om.n_dof)), "lbfgs", m, tol, max_iter)
    return time.perf_counter() - t0, res["iters"], res["evals"]


def _cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_oracle_rate(w, n_inst, n_steps, budget_s, fast=False, counts=None):
    """Oracle link-steps/s on the host cores over a bounded sample: the first
    n_inst instances of the workload, one process per core (spawn; started,
    imported and warmed before the timed map). n_steps = 0 picks the number
    of time steps so that the timed map takes about budget_s seconds, from
    the warm-up's seconds per instance-step. Returns (rate, cores, sample
    description); `counts`, a dict, receives the sample's size and each
    instance's iterations and evaluations."""
    import multiprocessing as mp
    from oracle import oracle as O
    spec = w["spec"]
    S, dt = w["stages"], w["dt"]
    nodes, _ = O.colloc(S)
    qp = w["q0"] + nodes[0] * dt * w["qd0"]
    n_inst = min(n_inst, spec.count)
    procs = min(os.cpu_count() or 1, n_inst)

    def job(b, steps):
        return (spec.select([b]), 0, qp[b], w["q0"][b], S, dt, w["history"], w["tol"],
                w["max_iter"], steps, fast)

    ctx = mp.get_context("spawn")
    with ctx.Pool(procs, initializer=_oracle_worker_init) as pool:
        warm = pool.map(_oracle_instance, [job(b, 1) for b in range(procs)], chunksize=1)
        per_step = max(sum(r[0] for r in warm) / len(warm), 1e-6)
        if n_steps <= 0:
            n_steps = int(budget_s * procs / (n_inst * per_step))
            n_steps = max(1, min(n_steps, w["n_steps"]))
        t0 = time.perf_counter()
        res = pool.map(_oracle_instance, [job(b, n_steps) for b in range(n_inst)], chunksize=1)
        wall = time.perf_counter() - t0
    if counts is not None:
        counts.update(n_inst=n_inst, n_steps=n_steps, iters=[int(r[1]) for r in res],
                      evals=[int(r[2]) for r in res])
    link_steps = n_inst * spec.n_links * n_steps
    sample = (f"{n_inst} of {spec.count} instances x the first {n_steps} of {w['n_steps']} time "
              f"steps, same solver settings, {'O(N)' if fast else 'brute-force O(N^2)'} "
              f"evaluations; {wall:.1f} s wall on {procs} processes "
              f"({sum(r[0] for r in res):.1f} s of oracle compute), {_cpu_model()}, "
              f"nproc {os.cpu_count()}")
    return link_steps / wall, procs, sample


# --------------------------------------------------------------------- ours
def autotune(P, batch, args, w):
    """Picks the instance-to-lane mapping (one lane per stage, or one per
    stage and link) and the threads per block with the shortest 2-step
    rollout of this workload. Returns (mapping, threads, trials)."""
    import torch
    from paper_1709_04145_b300.tuning import autotune_mapping
    S, dt, m = w["stages"], w["dt"], w["history"]
    nodes, _ = P.colloc(S)
    dev = torch.device("cuda", torch.cuda.current_device())
    qc = torch.tensor(w["q0"].reshape(-1), device=dev)
    qp = torch.tensor((w["q0"] + nodes[0] * dt * w["qd0"]).reshape(-1), device=dev)
    probe = lambda: P.rollout(batch, qp, qc, None, 2, dt, S, P.LBFGS, m, w["tol"],
                              min(w["max_iter"], 20), want_traj=False, want_step_log=False)
    return autotune_mapping(batch, probe, mappings=(P.MAP_STAGE, P.MAP_LINK))


def measure_throughput_point(P, args, dev, threads, mapping):
    """The same rollout on a large batch (65536 ten-link ball chains, 20
    steps): every FP64 sub-partition busy. Returns link-steps/s and the FP64
    roofline fraction."""
    import numpy as np
    import torch
    from paper_1709_04145_b300 import inputs as I
    w = I.ball_chains(count=args.throughput_instances, n_links=args.links, seed_base=2500,
                      n_steps=args.throughput_timesteps)
    w["max_iter"], w["tol"] = args.max_iter, args.tol
    spec = w["spec"]
    S, dt, m = w["stages"], w["dt"], w["history"]
    nodes, _ = P.colloc(S)
    batch = P.Batch([P.Model.from_spec(spec, device=dev.index)], max_stages=S, max_history=m)
    batch.set_threads(threads)
    batch.set_mapping(mapping)
    qp = torch.tensor((w["q0"] + nodes[0] * dt * w["qd0"]).reshape(-1), device=dev)
    qc = torch.tensor(w["q0"].reshape(-1), device=dev)
    T = w["n_steps"]
    P.rollout(batch, qp, qc, None, 1, dt, S, P.LBFGS, m, w["tol"], w["max_iter"], want_traj=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    out = P.rollout(batch, qp, qc, None, T, dt, S, P.LBFGS, m, w["tol"], w["max_iter"], want_traj=False)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ev = out["evals"].cpu().numpy()
    it = out["iters"].cpu().numpy()
    flops = rollout_flops(spec, S, m, ev, out["grads"].cpu().numpy(), it)
    return {"value": spec.count * spec.n_links * T / (ms / 1e3), "unit": UNIT, "ms": ms,
            "instances": spec.count, "timesteps": T, "achieved_tflops": flops / (ms / 1e3) / 1e12,
            "evals_per_step": float(ev.mean() / T), "step_outcomes": step_outcomes(out)}


def measure_plain(P, w, args, dev):
    """Plain form: the same kernels with one instance per launch and one launch
    per instance-step (pbad_step on a batch of one), no graph; returns
    link-steps/s over the first instances of the workload."""
    import torch
    spec = w["spec"]
    S, dt, m = w["stages"], w["dt"], w["history"]
    nodes, _ = P.colloc(S)
    n_inst = min(args.plain_instances, spec.count)
    T = args.plain_timesteps
    jobs = []
    for b in range(n_inst):
        model = P.Model.from_spec(spec.select([b]), device=dev.index)
        batch = P.Batch([model], max_stages=S, max_history=m)
        qp = torch.tensor((w["q0"][b] + nodes[0] * dt * w["qd0"][b]), device=dev)
        qc = torch.tensor(w["q0"][b], device=dev)
        jobs.append((model, batch, qp, qc))
    for model, batch, qp, qc in jobs[:1]:  # warm-up
        P.step(batch, qp, qc, None, dt, S, P.LBFGS, m, w["tol"], w["max_iter"])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for model, batch, qp, qc in jobs:
        for _ in range(T):
            out = P.step(batch, qp, qc, None, dt, S, P.LBFGS, m, w["tol"], w["max_iter"])
            qp, qc = out["q_prev"], out["q_cur"]
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    return {"value": n_inst * spec.n_links * T / (ms / 1e3), "unit": UNIT, "ms": ms,
            "sample": f"{n_inst} instances x {T} time steps, one pbad_step launch per "
                      "instance-step, no graph"}


def measure_pendulum(P, args, dev):
    """The plain method, batch 1: the 3-link rod pendulum (dt = 0.01, one
    stage, L-BFGS m = 5, |r| < 1e-10, 200 steps) as one persistent rollout
    launch under each mapping, and as 200 pbad_step launches (one per
    step, no graph)."""
    import torch
    from paper_1709_04145_b300 import inputs as I
    w = I.pendulum3()
    spec, T = w["spec"], w["n_steps"]
    batch = P.Batch([P.Model.from_spec(spec, device=dev.index)], max_stages=1,
                    max_history=w["history"])
    q0 = torch.tensor(w["q0"].reshape(-1), device=dev)
    out = {"instances": 1, "links": spec.n_links, "timesteps": T, "dt": w["dt"], "stages": 1,
           "history": w["history"], "tol": w["tol"]}
    for name, mp in (("rollout_stage_mapping", P.MAP_STAGE), ("rollout_link_mapping", P.MAP_LINK)):
        batch.set_mapping(mp)
        run = lambda: P.rollout(batch, q0, q0, None, T, w["dt"], 1, P.LBFGS, w["history"], w["tol"],
                                1000, want_traj=False)
        run()
        ms, res = _timed(run)
        out[name] = {"ms": ms, "value": spec.n_links * T / (ms / 1e3), "unit": UNIT,
                     "iters_per_step": float(res["iters"].float().mean().item() / T),
                     "step_outcomes": step_outcomes(res)}
    batch.set_mapping(P.MAP_STAGE)

    def per_step():
        qp, qc = q0, q0
        for _ in range(T):
            o = P.step(batch, qp, qc, None, w["dt"], 1, P.LBFGS, w["history"], w["tol"], 1000)
            qp, qc = o["q_prev"], o["q_cur"]
        return qc
    per_step()
    ms, _ = _timed(per_step)
    out["per_step_launches"] = {"ms": ms, "value": spec.n_links * T / (ms / 1e3), "unit": UNIT,
                                "launches": T}
    return out


def measure_companions(P, args, dev):
    """The headline batch (4096 ten-link ball chains, dt = 0.033, three
    stages, 100 steps) solved by Newton (LM) instead of L-BFGS, and both
    solvers on the same chains with the 0.05 m capsule radius first proposed
    for them; one timed rollout each after a warm-up rollout, with the
    per-step outcomes."""
    import torch
    from paper_1709_04145_b300 import inputs as I
    rows = {}
    for radius in (0.15, 0.05):
        T = args.companion_steps if radius == 0.15 else args.companion_steps_thin
        w = I.ball_chains(count=args.instances, n_links=args.links, n_steps=T, radius=radius)
        spec, S, dt, m = w["spec"], w["stages"], w["dt"], w["history"]
        batch = P.Batch([P.Model.from_spec(spec, device=dev.index)], max_stages=S, max_history=m,
                        newton=True)
        qp, qc = _state_tensors(P, [(w["q0"], w["qd0"])], S, dt, dev)
        for name, sv, mi in (("newton", P.NEWTON, 100), ("lbfgs", P.LBFGS, args.max_iter)):
            if radius == 0.15 and sv == P.LBFGS:
                continue  # the headline itself
            run = lambda T_: P.rollout(batch, qp, qc, None, T_, dt, S, sv, m, args.tol, mi,
                                       want_traj=False)
            cta = None
            if sv == P.NEWTON:  # one warp or one CTA per instance, by a two-step probe
                from paper_1709_04145_b300.tuning import autotune_newton_cta
                cta = autotune_newton_cta(batch, lambda: run(2), S)
            run(2)
            ms, out = _timed(lambda: run(T))
            it = out["iters"].float().mean().item() / T
            rows[f"{name}_radius{radius}"] = {
                "solver": name, "capsule_radius_m": radius, "instances": spec.count,
                "links": spec.n_links, "timesteps": T, "dt": dt, "stages": S, "tol": args.tol,
                "max_iter_per_step": mi, "ms": ms,
                "value": spec.count * spec.n_links * T / (ms / 1e3), "unit": UNIT,
                "iters_per_step": it, "step_outcomes": step_outcomes(out)}
            row = rows[f"{name}_radius{radius}"]
            # the same rate counting only the solved instance-steps
            row["solved_value"] = row["value"] * row["step_outcomes"]["solved_fraction"]
            if cta is not None:
                rows[f"{name}_radius{radius}"]["newton_cta_min"] = {
                    "chosen": cta[0], "two_step_ms": {str(k): v for k, v in cta[1].items()},
                    "rule": "S n >= threshold: one CTA of four warps per instance; 4097: "
                            "one warp per instance"}
        del batch
        torch.cuda.empty_cache()
    return rows


def measure_adjoint(P, args, dev):
    """Forward and forward+adjoint wall time (CUDA events) of the differentiable
    humanoid rollout: 1024 humanoids, dt = 0.033, two stages, Newton,
    checkpoint every 8 steps, end-effector loss at the last step."""
    import numpy as np
    import torch
    from paper_1709_04145_b300 import inputs as I
    from paper_1709_04145_b300.autograd import points_differentiable, rollout_differentiable
    steps = args.adjoint_steps
    w = I.humanoid_adjoint(n_steps=steps)
    spec = w["spec"]
    S = w["stages"]
    batch = P.Batch([P.Model.from_spec(spec, device=dev.index)], max_stages=S, max_history=8,
                    newton=True)
    t = lambda a: torch.tensor(np.ascontiguousarray(a), device=dev)
    x0 = t(w["q0"].reshape(-1)).requires_grad_()
    v0 = t(w["qd0"].reshape(-1)).requires_grad_()
    tt = t(w["tau"].reshape(steps, -1)).requires_grad_()
    tip = t(w["ee_point"])
    target = t(np.random.default_rng(w["target_seed"]).normal(0, 0.3, (spec.count, 3)))
    kw = dict(dt=w["dt"], stages=S, solver=P.NEWTON, tol=w["tol"], max_iter=100,
              checkpoint_every=w["checkpoint_every"])
    # one warp or one CTA per instance for the forward solves, by a one-step probe
    from paper_1709_04145_b300.tuning import autotune_newton_cta
    qp1, qc1 = _state_tensors(P, [(w["q0"], w["qd0"])], S, w["dt"], dev)
    tau1 = tt[:1].detach().reshape(-1).contiguous()
    cta = autotune_newton_cta(batch, lambda: P.rollout(batch, qp1, qc1, tau1, 1, w["dt"], S, P.NEWTON,
                                                       8, w["tol"], 100, want_traj=False), S)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    # warm-up: the first forward and adjoint launches in a process load their
    # kernels and the allocator's blocks (several seconds, once)
    qw, _, _ = rollout_differentiable(batch, x0, v0, tt[:2], **kw)
    ((points_differentiable(batch, qw, [w["ee_link"]], tip) - target) ** 2).sum().backward()
    x0.grad = v0.grad = tt.grad = None
    torch.cuda.synchronize()
    a, b = ev(), ev()
    a.record()
    with torch.no_grad():
        _, _, st = rollout_differentiable(batch, x0, v0, tt, **kw)
    b.record()
    torch.cuda.synchronize()
    fwd = a.elapsed_time(b)
    adj = torch.empty(spec.count, dtype=torch.int32, device=dev)
    a, b = ev(), ev()
    a.record()
    qc, _, st = rollout_differentiable(batch, x0, v0, tt, adjoint_status=adj, **kw)
    loss = ((points_differentiable(batch, qc, [w["ee_link"]], tip) - target) ** 2).sum()
    loss.backward()
    b.record()
    torch.cuda.synchronize()
    fwd_adj = a.elapsed_time(b)
    g_ckpt = [g.detach().clone() for g in (x0.grad, v0.grad, tt.grad)]
    stc = st.cpu().numpy()
    adjc = adj.cpu().numpy()
    # the same pass keeping every step's stages in the forward launches
    # (S n doubles per instance-step) instead of recomputing each segment
    x0.grad = v0.grad = tt.grad = None
    a, b = ev(), ev()
    a.record()
    qc, _, _ = rollout_differentiable(batch, x0, v0, tt, keep_stages=True, **kw)
    loss = ((points_differentiable(batch, qc, [w["ee_link"]], tip) - target) ** 2).sum()
    loss.backward()
    b.record()
    torch.cuda.synchronize()
    kept_ms = a.elapsed_time(b)
    same = all(torch.equal(torch.nan_to_num(g1, nan=7.0), torch.nan_to_num(g2, nan=7.0))
               for g1, g2 in zip(g_ckpt, (x0.grad, v0.grad, tt.grad)))
    stage_mb = steps * S * batch.D * 8 / 1e6
    # gradients over the first checkpoint segment alone (loss at its end)
    k = min(w["checkpoint_every"], steps)
    adj1 = torch.empty(spec.count, dtype=torch.int32, device=dev)
    x0.grad = v0.grad = tt.grad = None
    qc, _, _ = rollout_differentiable(batch, x0, v0, tt[:k], adjoint_status=adj1, keep_stages=True,
                                      **kw)
    ((points_differentiable(batch, qc, [w["ee_link"]], tip) - target) ** 2).sum().backward()
    x0.grad = v0.grad = tt.grad = None
    return {"fwd_ms": fwd, "fwd_adjoint_ms": fwd_adj, "steps": steps,
            "workload_steps": 64, "instances": spec.count,
            "newton_cta_min": {"chosen": cta[0], "one_step_ms": {str(k): v for k, v in cta[1].items()}},
            "all_steps_converged_fraction": float((stc == 0).mean()),
            "gradient_valid_fraction": float(np.isin(adjc, [0, 5]).mean()),
            "kept_stages": {"fwd_adjoint_ms": kept_ms, "stage_bytes_mb": stage_mb,
                            "gradients_bitwise_equal_to_checkpointed": bool(same),
                            "note": "forward launches keep every step's stages; the backward "
                                    "pass runs only the segment adjoint launches"},
            "first_segment": {"steps": k, "gradient_valid_fraction":
                              float(np.isin(adj1.cpu().numpy(), [0, 5]).mean())},
            "note": "gradients of instances with an unsolved step (or a singular adjoint "
                    "system) are NaN (the implicit-function theorem needs r = 0)"}


def _state_tensors(P, spec_states, S, dt, dev):
    """DOF-packed (q_prev0, q_cur0) device tensors of several buckets."""
    import numpy as np
    import torch
    nodes, _ = P.colloc(S)
    qc = np.concatenate([q0.reshape(-1) for q0, _ in spec_states])
    qp = np.concatenate([(q0 + nodes[0] * dt * qd0).reshape(-1) for q0, qd0 in spec_states])
    return torch.tensor(qp, device=dev), torch.tensor(qc, device=dev)


def _timed(fn):
    import torch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    r = fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), r


def measure_uneven(P, args, dev):
    """Uneven batch in one persistent launch: 1024 humanoid trees (Newton),
    1024 chains of 50 hinge rods and 2048 chains of 5 (L-BFGS m = 8), dt =
    0.05, two stages, torques N(0, 0.1^2). Threads per block autotuned over
    32/64/128 on one step (near-ties to the smaller block: tuning.pick_threads)
    and the mapping per bucket; then one rollout of args.uneven_steps steps."""
    import numpy as np
    import torch
    from paper_1709_04145_b300 import inputs as I
    T = args.uneven_steps
    u = I.uneven_batch(n_steps=T)
    S, dt, m = u["stages"], u["dt"], u["history"]
    batch = P.Batch([P.Model.from_spec(s, device=dev.index) for s in u["specs"]], max_stages=S,
                    max_history=m, newton=True)
    qp, qc = _state_tensors(P, u["states"], S, dt, dev)
    tau = torch.tensor(np.concatenate([t.reshape(T, -1) for t in u["taus"]], axis=1), device=dev)
    solvers = [P.NEWTON if sv == "newton" else P.LBFGS for sv in u["solvers"]]
    run = lambda steps: P.rollout(batch, qp, qc, tau[:steps].reshape(-1).contiguous(), steps, dt, S,
                                  solvers, m, u["tol"], args.max_iter_uneven, want_traj=False)
    tuned = {}
    for threads in (32, 64, 128):
        batch.set_threads(threads)
        tuned[threads] = _timed(lambda: run(1))[0]
    from paper_1709_04145_b300.tuning import autotune_bucket_mapping, pick_threads
    best = pick_threads(tuned)
    batch.set_threads(best)
    mapping_names = {P.MAP_STAGE: "stage", P.MAP_LINK: "link"}
    bmap, btrials = autotune_bucket_mapping(batch, lambda: run(1))
    ms, out = _timed(lambda: run(T))
    st = out["status"].cpu().numpy()
    it = out["iters"].cpu().numpy()
    evl = out["evals"].cpu().numpy()
    buckets = []
    link_steps = 0
    for k, spec in enumerate(u["specs"]):
        a, b = int(batch.inst_off[k]), int(batch.inst_off[k + 1])
        link_steps += spec.count * spec.n_links * T
        buckets.append({"model": spec.name, "instances": spec.count, "links": spec.n_links,
                        "dofs": spec.n_dof, "solver": u["solvers"][k],
                        "converged_fraction": float((st[a:b] == 0).mean()),
                        "iters_per_step": float(it[a:b].mean() / T),
                        "evals_per_step": float(evl[a:b].mean() / T),
                        "step_outcomes": step_outcomes(out, slice(a, b))})
    res = {"value": link_steps / (ms / 1e3), "unit": UNIT, "ms": ms, "timesteps": T,
           "launches": 1, "threads_per_block": best,
           "autotune_ms_per_step": {str(k): v for k, v in tuned.items()},
           "bucket_mapping": {"chosen": [mapping_names[x] for x in bmap],
                              "rule": "greedy per bucket: link-map bucket k if a one-step "
                                      "launch gets faster (refused where not a chain, S N > 32 "
                                      "or Newton)",
                              "one_step_ms_stage_then_link": btrials},
           "max_iter_per_step": args.max_iter_uneven, "tol": u["tol"], "buckets": buckets}
    # per-bucket solver choice from one-step probes, then the same rollout
    from paper_1709_04145_b300.tuning import choose_solvers
    batch.set_bucket_mapping(None)
    t0 = time.perf_counter()
    chosen, report = choose_solvers(batch, qp, qc, tau, dt, S, probe_steps=1, history=m,
                                    tol=u["tol"], max_iter={P.LBFGS: args.max_iter_uneven,
                                                            P.NEWTON: args.max_iter_uneven},
                                    threads=best)
    probe_s = time.perf_counter() - t0
    run_c = lambda steps: P.rollout(batch, qp, qc, tau[:steps].reshape(-1).contiguous(), steps, dt,
                                    S, chosen, m, u["tol"], args.max_iter_uneven, want_traj=False)
    bmap_c, _ = autotune_bucket_mapping(batch, lambda: run_c(1))
    cta_c = None
    if P.NEWTON in chosen:
        from paper_1709_04145_b300.tuning import autotune_newton_cta
        cta_c = autotune_newton_cta(batch, lambda: run_c(1), S)
    ms_c, out_c = _timed(lambda: run_c(T))
    st_c = out_c["status"].cpu().numpy()
    names = {P.LBFGS: "lbfgs", P.NEWTON: "newton"}
    res["solver_choice"] = {
        "rule": "per bucket, the solver with the least device time per converged instance-step "
                "over a one-step probe of the bucket alone",
        "probe_wall_s": probe_s,
        "chosen": [names[c] for c in chosen],
        "bucket_mapping": [mapping_names[x] for x in bmap_c],
        "newton_cta_min": None if cta_c is None else
        {"chosen": cta_c[0], "one_step_ms": {str(k): v for k, v in cta_c[1].items()}},
        "value": link_steps / (ms_c / 1e3), "ms": ms_c,
        "buckets": [{"model": spec.name,
                     "probe": {names[r.solver]: {"ms": r.ms, "converged_fraction": r.converged / r.total}
                               for r in report[k]},
                     "converged_fraction": float((st_c[int(batch.inst_off[k]):int(batch.inst_off[k + 1])] == 0).mean()),
                     "step_outcomes": step_outcomes(out_c, slice(int(batch.inst_off[k]),
                                                                 int(batch.inst_off[k + 1])))}
                    for k, spec in enumerate(u["specs"])]}
    return res


def measure_drag(P, args, dev):
    """Drag potential (Section 6.2): swimmer-like chains (4096 x 4 hinge rods,
    no gravity, c = 0.5, dt = 0.05, one stage, L-BFGS) and the swimmer body
    on a free 6-DOF root (4096 x 4 links, 9 DOFs) over args.drag_steps
    steps, and the main ball-chain batch with c = 0.5 against the same batch
    without drag over 5 steps (the drag only changes seed weights there)."""
    import torch
    from paper_1709_04145_b300 import inputs as I
    out = {}
    w = I.swimmers(n_steps=args.drag_steps)
    spec, S, dt, m = w["spec"], w["stages"], w["dt"], w["history"]
    batch = P.Batch([P.Model.from_spec(spec, device=dev.index, drag=w["drag"])], max_stages=S,
                    max_history=m)
    qp, qc = _state_tensors(P, [(w["q0"], w["qd0"])], S, dt, dev)
    T = w["n_steps"]
    run = lambda: P.rollout(batch, qp, qc, None, T, dt, S, P.LBFGS, m, w["tol"], 200, want_traj=False)
    run()
    ms, res = _timed(run)
    st = res["status"].cpu().numpy()
    out["swimmers"] = {"value": spec.count * spec.n_links * T / (ms / 1e3), "unit": UNIT, "ms": ms,
                       "instances": spec.count, "links": spec.n_links, "timesteps": T, "dt": dt,
                       "stages": S, "drag": w["drag"], "tol": w["tol"],
                       "converged_fraction": float((st == 0).mean()),
                       "iters_per_step": float(res["iters"].float().mean().item() / T),
                       "step_outcomes": step_outcomes(res)}
    # Section 6.2's swimmer body: 4 links on a free 6-DOF root (9 DOFs)
    w = I.swimmers_free(n_steps=args.drag_steps)
    spec, S, dt, m = w["spec"], w["stages"], w["dt"], w["history"]
    batch = P.Batch([P.Model.from_spec(spec, device=dev.index, drag=w["drag"])], max_stages=S,
                    max_history=m)
    qp, qc = _state_tensors(P, [(w["q0"], w["qd0"])], S, dt, dev)
    T = w["n_steps"]
    run = lambda: P.rollout(batch, qp, qc, None, T, dt, S, P.LBFGS, m, w["tol"], 200, want_traj=False)
    run()
    ms, res = _timed(run)
    st = res["status"].cpu().numpy()
    bodies = spec.n_links - 1  # the root's massless carrier link is not a body
    out["swimmers_free_root"] = {"value": spec.count * bodies * T / (ms / 1e3), "unit": UNIT,
                                 "ms": ms, "instances": spec.count, "links": bodies,
                                 "dofs": spec.n_dof, "timesteps": T, "dt": dt, "stages": S,
                                 "drag": w["drag"], "tol": w["tol"],
                                 "converged_fraction": float((st == 0).mean()),
                                 "iters_per_step": float(res["iters"].float().mean().item() / T),
                                 "step_outcomes": step_outcomes(res)}
    # Section 6.2's spider on the ground (free root, 4 legs, 22 DOFs, six
    # contact points of Eq. FRI), one stage, both solvers
    w = I.spiders(n_steps=args.drag_steps)
    spec, S, dt, m = w["spec"], w["stages"], w["dt"], w["history"]
    batch = P.Batch([P.Model.from_spec(spec, device=dev.index, drag=w["drag"], contact=w["contact"])],
                    max_stages=S, max_history=m, newton=True)
    qp, qc = _state_tensors(P, [(w["q0"], w["qd0"])], S, dt, dev)
    T = w["n_steps"]
    bodies = spec.n_links - 1
    for name, sv, mi in (("lbfgs", P.LBFGS, 500), ("newton", P.NEWTON, 100)):
        run = lambda: P.rollout(batch, qp, qc, None, T, dt, S, sv, m, w["tol"], mi, want_traj=False)
        run()
        ms, res = _timed(run)
        st = res["status"].cpu().numpy()
        out[f"spiders_contact_{name}"] = {
            "value": spec.count * bodies * T / (ms / 1e3), "unit": UNIT, "ms": ms,
            "instances": spec.count, "links": bodies, "dofs": spec.n_dof, "timesteps": T, "dt": dt,
            "stages": S, "contact_points": len(w["contact"]["link"]), "tol": w["tol"],
            "max_iter_per_step": mi, "worst_status_converged_fraction": float((st == 0).mean()),
            "iters_per_step": float(res["iters"].float().mean().item() / T),
            "step_outcomes": step_outcomes(res)}
    wb = I.ball_chains(count=args.instances, n_links=args.links, n_steps=5)
    spec = wb["spec"]
    S, dt, m = wb["stages"], wb["dt"], wb["history"]
    qp, qc = _state_tensors(P, [(wb["q0"], wb["qd0"])], S, dt, dev)
    row = {}
    for c in (0.0, 0.5):
        bt = P.Batch([P.Model.from_spec(spec, device=dev.index, drag=c)], max_stages=S, max_history=m)
        run = lambda: P.rollout(bt, qp, qc, None, 5, dt, S, P.LBFGS, m, args.tol, args.max_iter,
                                want_traj=False)
        run()
        ms, res = _timed(run)
        row[f"c={c}"] = {"ms": ms, "value": spec.count * spec.n_links * 5 / (ms / 1e3),
                         "evals_per_step": float(res["evals"].float().mean().item() / 5),
                         "step_outcomes": step_outcomes(res)}
    out["ball_chains_5_steps"] = row
    return out


def measure_mixed_precision(P, args, dev):
    """L-BFGS with the binary32 two-loop recursion (binary64 line search and
    evaluations) against binary64 L-BFGS on the same batches: the main
    ball-chain workload (all its steps), and one-stage swimmer-like chains
    and humanoids, where L-BFGS converges, over args.f32_steps steps."""
    import numpy as np
    from paper_1709_04145_b300 import inputs as I
    out = {}

    def pair(name, batch, qp, qc, T, S, dt, m, tol, max_iter, units, warm=True):
        row = {}
        for label, sv in (("f64", P.LBFGS), ("f32_direction", P.LBFGS_F32)):
            run = lambda: P.rollout(batch, qp, qc, None, T, dt, S, sv, m, tol, max_iter,
                                    want_traj=False)
            if warm:
                run()
            ms, res = _timed(run)
            st = res["status"].cpu().numpy()
            row[label] = {"ms": ms, "value": units * T / (ms / 1e3), "unit": UNIT,
                          "iters_per_step": float(res["iters"].float().mean().item() / T),
                          "evals_per_step": float(res["evals"].float().mean().item() / T),
                          "status_counts": np.bincount(st, minlength=6).tolist(),
                          "step_outcomes": step_outcomes(res)}
        row["speedup"] = row["f64"]["ms"] / row["f32_direction"]["ms"]
        row.update({"timesteps": T, "stages": S, "dt": dt, "tol": tol, "max_iter": max_iter})
        out[name] = row

    # the main workload at its full length: one run of each (the kernels are
    # loaded and warm from the timed bench)
    T = args.timesteps
    wb = I.ball_chains(count=args.instances, n_links=args.links, n_steps=T)
    spec, S, dt, m = wb["spec"], wb["stages"], wb["dt"], wb["history"]
    batch = P.Batch([P.Model.from_spec(spec, device=dev.index)], max_stages=S, max_history=m)
    qp, qc = _state_tensors(P, [(wb["q0"], wb["qd0"])], S, dt, dev)
    pair(f"ball_chains_{spec.count}x{spec.n_links}", batch, qp, qc, T, S, dt, m, args.tol,
         args.max_iter, spec.count * spec.n_links, warm=False)
    T = args.f32_steps
    w = I.swimmers(n_steps=T)
    spec, S, dt, m = w["spec"], w["stages"], w["dt"], w["history"]
    batch = P.Batch([P.Model.from_spec(spec, device=dev.index, drag=w["drag"])], max_stages=S,
                    max_history=m)
    qp, qc = _state_tensors(P, [(w["q0"], w["qd0"])], S, dt, dev)
    pair("swimmers_one_stage", batch, qp, qc, T, S, dt, m, w["tol"], 200, spec.count * spec.n_links)
    spec = I.humanoid(1024, seed=5)
    q0, qd0 = I.random_state(spec, 6, pose_scale=0.3, vel_sigma=0.3)
    batch = P.Batch([P.Model.from_spec(spec, device=dev.index)], max_stages=1, max_history=8)
    qp, qc = _state_tensors(P, [(q0, qd0)], 1, 0.033, dev)
    pair("humanoids_one_stage", batch, qp, qc, T, 1, 0.033, 8, 1e-8, 1000, spec.count * spec.n_links)
    return out


def measure_df64(P, args, dev):
    """Double-float residual pass against the binary64 one on the batched
    workload's 4096 ten-link ball chains (three stages, link mapping): time
    per evaluation launch (E, r and the binary64 gradient tangent pass) at
    the steps' initial guesses, and the difference of the residuals at
    solved steps (Newton to |r| < 1e-8) against the tolerance."""
    import numpy as np
    import torch
    from paper_1709_04145_b300 import inputs as I
    w = I.ball_chains(count=args.instances, n_links=args.links, n_steps=1)
    spec, S, dt = w["spec"], w["stages"], w["dt"]
    nodes, _ = P.colloc(S)
    t = lambda a: torch.tensor(np.ascontiguousarray(a).reshape(-1), device=dev)
    qp, qc = t(w["q0"] + nodes[0] * dt * w["qd0"]), t(w["q0"])
    batch = P.Batch([P.Model.from_spec(spec, device=dev.index)], max_stages=S, max_history=8,
                    newton=True)
    step = P.step(batch, qp, qc, None, dt, S, P.NEWTON, 8, 1e-8, 100)
    solved = step["status"].cpu().numpy() == 0
    guess = torch.cat([qc.view(spec.count, 1, -1) + (nodes[2 + i] / (0 - nodes[0])) *
                       (qc - qp).view(spec.count, 1, -1) for i in range(S)], dim=1).reshape(-1)
    out = {"instances": spec.count, "stages": S, "launches_timed": 50}
    res = {}
    batch.set_mapping(P.MAP_LINK)
    for name, prec in (("f64", P.PRECISION_F64), ("df64", P.PRECISION_DF64)):
        batch.set_precision(prec)
        run = lambda: [P.eval_objective_grad(batch, guess, qp, qc, None, dt, S) for _ in range(50)]
        run()
        ms, _ = _timed(run)
        out[f"{name}_ms_per_eval"] = ms / 50
        _, _, r = P.eval_objective_grad(batch, step["q_stages"], qp, qc, None, dt, S)
        res[name] = r.cpu().numpy().reshape(spec.count, -1)
    batch.set_precision(P.PRECISION_F64)
    out["df64_speedup"] = out["f64_ms_per_eval"] / out["df64_ms_per_eval"]
    d = np.linalg.norm(res["df64"] - res["f64"], axis=1)[solved]
    out["solved_steps"] = int(solved.sum())
    out["residual_difference_at_solved_steps"] = {
        "median": float(np.median(d)), "max": float(np.max(d)), "tol": 1e-8,
        "fraction_above_tol": float((d > 1e-8).mean())}
    return out


def measure_dt_sweep(P, args, dev):
    """Step-size sweep of both solvers on two bodies: 512 ten-link ball chains
    (three stages) and 512 five-link hinge-rod chains (two stages), two
    steps per size from the seeded initial states, zero torques."""
    import torch
    from paper_1709_04145_b300 import inputs as I
    from paper_1709_04145_b300.tuning import dt_sweep
    dts = [0.001 * 2 ** k for k in range(8)]
    out = {}
    for name, spec, S in (("ball_chain10", I.ball_chain(512, 10, 2601, radius=0.15), 3),
                          ("rod_chain5", I.rod_chain(512, 5, name="rod_chain5"), 2)):
        q0, qd0 = I.random_state(spec, 2602)
        model = P.Model.from_spec(spec, device=dev.index)
        t = lambda a: torch.tensor(a.reshape(-1), device=dev)
        out[name] = {"stages": S, "instances": spec.count,
                     "rows": dt_sweep(model, t(q0), t(qd0), dts, S, steps=2, tol=args.tol,
                                      max_iter=args.max_iter_uneven)}
    return out


def measure_scaling(P, args, dev):
    """Scaling study: serial hinge-rod chains of N links, batch 256, dt = 0.1,
    four stages; L-BFGS (m = 8) and Newton on the same inputs, at most
    args.max_iter_scaling iterations per step (the study compares the cost
    per iteration). Each (N, solver) runs args.scaling_steps steps forward
    in one launch, fewer when a one-step probe says they would take more
    than args.scaling_budget seconds (the row says how many), and a forward
    + adjoint pass (end-state loss) over the first min(steps, 8) steps (fewer
    when their forward alone would exceed half of args.scaling_adjoint_budget)."""
    import numpy as np
    import torch
    from paper_1709_04145_b300 import inputs as I
    from paper_1709_04145_b300.autograd import rollout_differentiable
    rows = []
    warm = False  # the first forward + adjoint in a process also loads kernels: one untimed call
    for N in args.scaling_links:
        w = I.scaling_chains(N, n_steps=args.scaling_steps)
        spec = w["spec"]
        S, dt, m = w["stages"], w["dt"], w["history"]
        batch = P.Batch([P.Model.from_spec(spec, device=dev.index)], max_stages=S, max_history=m,
                        newton=True)
        qp, qc = _state_tensors(P, [(w["q0"], w["qd0"])], S, dt, dev)
        x0 = torch.tensor(w["q0"].reshape(-1), device=dev)
        v0 = torch.tensor(w["qd0"].reshape(-1), device=dev)
        for name, sv in (("lbfgs", P.LBFGS), ("newton", P.NEWTON)):
            run = lambda T_: P.rollout(batch, qp, qc, None, T_, dt, S, sv, m, w["tol"],
                                       args.max_iter_scaling, want_traj=False)
            ms1, _ = _timed(lambda: run(1))
            T = int(max(1, min(args.scaling_steps, args.scaling_budget * 1e3 // max(ms1, 1e-3))))
            ms, out = _timed(lambda: run(T))
            # the adjoint pass over up to 8 steps, fewer where their forward
            # alone would take more than half the row's budget
            Ta = max(1, min(T, 8, int(0.5 * args.scaling_adjoint_budget * 1e3 // max(ms1, 1e-3))))
            tau = torch.zeros((Ta, batch.D), dtype=torch.float64, device=dev)

            def fwd_adj():
                xg = x0.clone().requires_grad_()
                vg = v0.clone().requires_grad_()
                tg = tau.clone().requires_grad_()
                qe, _, _ = rollout_differentiable(batch, xg, vg, tg, dt, S, solver=sv, history=m,
                                                  tol=w["tol"], max_iter=args.max_iter_scaling,
                                                  checkpoint_every=8, on_unsolved="keep")
                (qe ** 2).sum().backward()
                return tg.grad
            if not warm:
                fwd_adj()
                warm = True
            ms_fa, _ = _timed(fwd_adj)
            its = float(out["iters"].float().mean().item() / T)
            rows.append({"links": N, "solver": name, "instances": spec.count, "timesteps": T,
                         "fwd_ms": ms, "fwd_ms_per_step": ms / T,
                         "fwd_ms_per_iteration": ms / max(its * T, 1e-9),
                         "fwd_link_steps_per_s": spec.count * N * T / (ms / 1e3),
                         "fwd_adjoint_steps": Ta, "fwd_adjoint_ms": ms_fa,
                         "iters_per_step": its, "step_outcomes": step_outcomes(out)})
        del batch
        torch.cuda.empty_cache()
    return {"rows": rows, "dt": 0.1, "stages": 4, "max_iter_per_step": args.max_iter_scaling,
            "steps_requested": args.scaling_steps, "budget_s_per_row": args.scaling_budget,
            "adjoint_budget_s_per_row": args.scaling_adjoint_budget}


def measure_damped_system(P, args, dev, peak_tflops):
    """The LM iteration's damped system alone (pbad_damped_gram_solve: Gram
    matrix, Cholesky, solves; one CTA per instance) at the scaling study's
    largest Newton size: 256 instances, S n = 4 x args.damped_links, random
    J = N(0, 1) + 3 I, lambda = 1e-3. Algorithmic flops per instance: the
    lower triangle of J^T J, n^2 (n + 1) / 2 FMAs; the Cholesky, n^3 / 3
    flops; the two solves, 2 n^2."""
    import torch
    n, count = 4 * args.damped_links, 256
    gen = torch.Generator(device=dev).manual_seed(11)
    J = torch.randn((count, n, n), dtype=torch.float64, device=dev, generator=gen)
    J += 3.0 * torch.eye(n, dtype=torch.float64, device=dev)
    g = torch.randn((count, n), dtype=torch.float64, device=dev, generator=gen)
    P.damped_gram_solve(J, g, 1e-3)
    ms = min(_timed(lambda: P.damped_gram_solve(J, g, 1e-3))[0] for _ in range(2))
    _, _, _, st = P.damped_gram_solve(J, g, 1e-3)
    flops = count * (n * n * (n + 1) + n ** 3 / 3 + 2 * n * n)
    tf = flops / (ms / 1e3) / 1e12
    res = {"instances": count, "n": n, "ms": ms, "flops": flops, "achieved_tflops": tf,
           "frac_of_fp64_peak": tf / peak_tflops, "factored_fraction": float((st == 0).float().mean()),
           "note": "one CTA (128 threads) per instance; 256 CTAs on 148 SMs at 2 CTAs/SM"}
    del J, g
    torch.cuda.empty_cache()
    return res


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1709_04145_b300 as P

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    w = workload(args, rank)
    spec = w["spec"]
    S, dt, m = w["stages"], w["dt"], w["history"]
    nodes, _ = P.colloc(S)
    q_prev0_h = (w["q0"] + nodes[0] * dt * w["qd0"]).reshape(-1)
    q_cur0_h = w["q0"].reshape(-1)
    model = P.Model.from_spec(spec, device=local)
    batch = P.Batch([model], max_stages=S, max_history=m)
    if args.threads == 0:
        mapping, tuned, trials = autotune(P, batch, args, w)
    else:
        mapping, tuned, trials = args.mapping, args.threads, []
    batch.set_threads(tuned)
    batch.set_mapping(mapping)
    q_prev0 = torch.tensor(q_prev0_h, device=dev)
    q_cur0 = torch.tensor(q_cur0_h, device=dev)
    T = w["n_steps"]
    out = dict(q_prev=torch.empty(batch.D, dtype=torch.float64, device=dev),
               q_cur=torch.empty(batch.D, dtype=torch.float64, device=dev),
               status=torch.empty(batch.n_instances, dtype=torch.int32, device=dev),
               iters=torch.empty(batch.n_instances, dtype=torch.int32, device=dev),
               evals=torch.empty(batch.n_instances, dtype=torch.int32, device=dev),
               grads=torch.empty(batch.n_instances, dtype=torch.int32, device=dev),
               step_status=torch.empty((w["n_steps"], batch.n_instances), dtype=torch.int32,
                                       device=dev),
               step_rnorm=torch.empty((w["n_steps"], batch.n_instances), dtype=torch.float64,
                                      device=dev),
               traj_prev=None, traj_cur=None)

    def launch():
        P.rollout(batch, q_prev0, q_cur0, None, T, dt, S, P.LBFGS, m, w["tol"], w["max_iter"],
                  out=out)

    # one rollout = one persistent kernel, captured in a CUDA graph
    launch()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            launch()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2

    for _ in range(args.warmup):
        g.replay()
    torch.cuda.synchronize()
    peak_gflops = P.fp64_peak(local)

    clocks = ClockSampler(local)
    if not args.no_clocks:
        clocks.start()
        time.sleep(0.5)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    cur = torch.cuda.current_stream()
    for k in range(args.steps):
        flush.fill_(float(k))  # L2 flush between timed steps (outside the events)
        ev[k][0].record(cur)
        g.replay()
        ev[k][1].record(cur)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms_steps = [a.elapsed_time(b) for a, b in ev]
    clk = clocks.stop() if not args.no_clocks else None
    ms = sum(ms_steps) / len(ms_steps)
    if world > 1:
        ms = max_over_ranks(ms, dist, dev)

    status = out["status"].cpu().numpy()
    iters = out["iters"].cpu().numpy()
    evals = out["evals"].cpu().numpy()
    grads = out["grads"].cpu().numpy()
    link_steps = spec.count * spec.n_links * T
    value = job_throughput(link_steps, world, ms)

    # roofline of the rollout kernel (the only kernel of the timed region)
    flops = rollout_flops(spec, S, m, evals, grads, iters)
    achieved = flops / (ms / 1e3) / 1e12
    peak = peak_gflops / 1e3

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        qp_h = torch.tensor(q_prev0_h).pin_memory()
        qc_h = torch.tensor(q_cur0_h).pin_memory()
        res_h = torch.empty(batch.D, dtype=torch.float64).pin_memory()
        st_h = torch.empty(batch.n_instances, dtype=torch.int32).pin_memory()
        qp_d = torch.empty_like(q_prev0)
        qc_d = torch.empty_like(q_cur0)
        out2 = dict(out)
        torch.cuda.synchronize()
        t_e2e = []
        e2e_steps = max(1, min(args.steps, args.e2e_steps))
        for k in range(e2e_steps):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(cur)
            qp_d.copy_(qp_h, non_blocking=True)
            qc_d.copy_(qc_h, non_blocking=True)
            P.rollout(batch, qp_d, qc_d, None, T, dt, S, P.LBFGS, m, w["tol"], w["max_iter"],
                      out=out2)
            res_h.copy_(out2["q_cur"], non_blocking=True)
            st_h.copy_(out2["status"], non_blocking=True)
            e1.record(cur)
            torch.cuda.synchronize()
            t_e2e.append(e0.elapsed_time(e1))
        ms_e = sum(t_e2e) / len(t_e2e)
        if world > 1:
            ms_e = max_over_ranks(ms_e, dist, dev)
        e2e = {"value": job_throughput(link_steps, world, ms_e), "unit": UNIT,
               "h2d_bytes_per_step": 2 * batch.D * 8,
               "d2h_bytes_per_step": batch.D * 8 + batch.n_instances * 4,
               "ms_per_step": ms_e, "steps": e2e_steps}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded generators; no dataset)",
        "config": {"workload": f"batched ball-joint capsule chains: {spec.count} x {spec.n_links} "
                               f"links, dt={dt}, {S} stages, L-BFGS m={m}, {T} steps per rollout, "
                               "one persistent launch in a CUDA graph",
                   "instances_per_gpu": spec.count, "links": spec.n_links, "timesteps": T,
                   "stages": S, "solver": "lbfgs", "history": m, "tol": w["tol"],
                   "max_iter_per_step": w["max_iter"], "parallelism": f"instances sharded, {world} GPU",
                   "threads_per_block": tuned,
                   "mapping": "link (one lane per stage and link)" if mapping == P.MAP_LINK
                              else "stage (one lane per stage)",
                   "autotune_ms_2_steps": {f"{'link' if t.mapping else 'stage'}/{t.threads}":
                                           (t.ms if np.isfinite(t.ms) else None) for t in trials},
                   "capsule_radius_m": float(spec.radius[0, 0]),
                   "l2": "flushed between timed steps (512 MB write outside the events)"},
        "solver_stats": {"converged_fraction": float((status == 0).mean()),
                         "worst_status_counts": {P.STATUS[k]: int((status == k).sum())
                                                 for k in range(6)},
                         "step_outcomes": step_outcomes(out),
                         "solved_link_steps_per_s": value * step_outcomes(out)["solved_fraction"],
                         "floor_note": "STALLED = line search failed at |r| <= 1e3 x the binary64 "
                                       "rounding floor of r (solved to rounding)",
                         "iters_per_step": float(iters.mean() / T),
                         "evals_per_step": float(evals.mean() / T),
                         "gradient_evals_per_step": float(grads.mean() / T)},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "traffic": rollout_traffic(mapping, S, spec.n_links, float(evals.sum())),
                     "traffic_unit": "bytes per launch (DRAM read + write per instance-evaluation "
                                     "from an ncu capture of this kernel build, times the "
                                     "launch's evaluations; null without a capture of this build)",
                     "peak_source": "measured FP64 FMA probe (pbad_fp64_peak) on this GPU",
                     "flops_per_launch": flops},
        "gpu_launches": args.steps,
        "e2e": e2e,
        "clocks": clk,
    }
    if rank == 0 and args.plain_instances > 0:
        plain = measure_plain(P, w, args, dev)
        line["plain"] = plain
        line["batched_vs_plain"] = value / world / plain["value"]
    if rank == 0 and args.pendulum:
        line["plain_pendulum"] = measure_pendulum(P, args, dev)
    if rank == 0 and args.companion_steps > 0:
        line["companions"] = measure_companions(P, args, dev)
    if rank == 0 and args.throughput_instances > 0:
        tp = measure_throughput_point(P, args, dev, tuned, mapping)
        tp["frac_of_fp64_peak"] = tp["achieved_tflops"] / peak
        line["throughput_point"] = tp
    if rank == 0 and args.adjoint_steps > 0:
        line["fwd_adjoint"] = measure_adjoint(P, args, dev)
    if rank == 0 and args.uneven_steps > 0:
        line["uneven_batch"] = measure_uneven(P, args, dev)
    if rank == 0 and args.scaling_steps > 0:
        line["scaling_study"] = measure_scaling(P, args, dev)
    if rank == 0 and args.damped_links > 0:
        line["damped_system"] = measure_damped_system(P, args, dev, peak)
    if rank == 0 and args.drag_steps > 0:
        line["drag"] = measure_drag(P, args, dev)
    if rank == 0 and args.f32_steps > 0:
        line["mixed_precision"] = measure_mixed_precision(P, args, dev)
        line["mixed_precision"]["double_float_residual"] = measure_df64(P, args, dev)
    if rank == 0 and args.dt_sweep:
        line["dt_sweep"] = measure_dt_sweep(P, args, dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, sample = cpu_oracle_rate(w, n_inst=min(os.cpu_count() or 1, 16), n_steps=0,
                                              budget_s=args.cpu_sample_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": sample}
        # the same oracle on one core (one process, one instance)
        rate1, _, sample1 = cpu_oracle_rate(w, n_inst=1, n_steps=0,
                                            budget_s=args.cpu_sample_seconds / 3)
        line["cpu_baseline"]["single_core"] = {"value": rate1, "unit": UNIT, "sample": sample1}
        # the fair CPU baseline: the same L-BFGS with O(N) evaluations
        # (Algorithm DERIV for the residuals, its tangent for the gradient)
        cnt = {}
        rate_f, cores_f, sample_f = cpu_oracle_rate(w, n_inst=min(os.cpu_count() or 1, 16),
                                                    n_steps=0, budget_s=args.cpu_sample_seconds,
                                                    fast=True, counts=cnt)
        line["cpu_baseline"]["o_n_evaluation"] = {"value": rate_f, "unit": UNIT, "cores": cores_f,
                                                  "kind": "oracle L-BFGS, O(N) evaluation",
                                                  "sample": sample_f}
        # the oracle's iteration and evaluation counts beside the GPU's on the
        # same instances (the GPU's over all T steps of the timed rollout)
        ni, ns = cnt["n_inst"], cnt["n_steps"]
        line["cpu_baseline"]["o_n_evaluation"]["counts_side_by_side"] = {
            "instances": ni, "oracle_steps": ns, "gpu_steps": T,
            "oracle_iters_per_step": sum(cnt["iters"]) / (ni * ns),
            "gpu_iters_per_step": float(iters[:ni].mean() / T),
            "oracle_evals_per_step": sum(cnt["evals"]) / (ni * ns),
            "gpu_evals_per_step": float(evals[:ni].mean() / T)}
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_reference(args):
    """The CPU oracle as it stands, on the host cores, same workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workload(args)
    spec = w["spec"]
    n_inst = min(os.cpu_count() or 1, 16)
    for _ in range(args.warmup):
        cpu_oracle_rate(w, n_inst=min(2, n_inst), n_steps=1, budget_s=1)
    rates = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r, cores, sample = cpu_oracle_rate(w, n_inst=n_inst, n_steps=0,
                                           budget_s=args.cpu_sample_seconds)
        rates.append(r)
    wall = time.perf_counter() - t0
    value = statistics.median(rates)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded generators; no dataset)", "impl": "reference",
            "config": {"workload": f"batched ball-joint capsule chains: {spec.count} x {spec.n_links} "
                                   f"links, dt={w['dt']}, {w['stages']} stages, L-BFGS "
                                   f"m={w['history']}, {w['n_steps']} steps per rollout",
                       "max_iter_per_step": w["max_iter"], "tol": w["tol"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
