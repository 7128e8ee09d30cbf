"""Solver choice per bucket, time-step sweeps and mapping autotuners.

The paper compares L-BFGS and LM (Newton) per time step and finds the
better one depends on the step size and the body (Section 6.1, Fig.
OPTProf). `choose_solvers` makes that choice for each bucket of a batch
from a short probe: it runs the bucket alone with each solver over the
first steps of its own inputs and keeps the solver with the smaller device
time per converged instance-step. `dt_sweep` reports, for a range of step
sizes, what each solver achieves on a model. The mapping autotuners time
the instance-to-lane mappings and block sizes (`autotune_mapping`), the
mapping of each bucket inside one launch (`autotune_bucket_mapping`) and
which Newton buckets run a CTA per instance (`autotune_newton_cta`). All
of them only time launches of the library; their decision rules (`pick`,
`pick_mapping`, `pick_threads`, `choose_bucket_mappings`,
`newton_cta_candidates`) are plain host logic with CPU tests.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import LBFGS, NEWTON, Batch, colloc, rollout


@dataclass
class ProbeResult:
    """Outcome of one solver on one bucket: device milliseconds of the probe
    launch, converged instance-steps and all instance-steps."""
    solver: int
    ms: float
    converged: int
    total: int
    iters_per_step: float = 0.0
    extra: dict = field(default_factory=dict)

    @property
    def ms_per_converged(self) -> float:
        return self.ms / self.converged if self.converged > 0 else float("inf")


def pick(results) -> int:
    """The solver with the smallest time per converged instance-step; if no
    solver converges anything, the one with the most converged steps, then
    the fastest. Ties go to L-BFGS (no dense storage)."""
    results = list(results)
    if not results:
        raise ValueError("no probe results")
    if any(r.converged > 0 for r in results):
        return min(results, key=lambda r: (r.ms_per_converged, r.solver)).solver
    return min(results, key=lambda r: (-r.converged, r.ms, r.solver)).solver


def _timed(fn):
    import torch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    out = fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), out


def probe(model, q_prev, q_cur, tau_seq, n_steps: int, dt: float, stages: int, solver: int,
          history: int = 8, tol: float = 1e-8, max_iter: int = 100, threads: int = 32) -> ProbeResult:
    """Runs one bucket alone for n_steps with one solver (after a one-step
    warm-up launch) and counts its converged instance-steps. q_prev/q_cur:
    DOF-packed device tensors of this bucket; tau_seq: (n_steps * D) device
    tensor or None."""
    batch = Batch([model], max_stages=stages, max_history=history, newton=(solver == NEWTON))
    batch.set_threads(threads)
    tau1 = None if tau_seq is None else tau_seq[:batch.D].contiguous()
    rollout(batch, q_prev, q_cur, tau1, 1, dt, stages, solver, history, tol, max_iter,
            want_traj=False)
    converged = 0
    qp, qc = q_prev, q_cur
    ms = 0.0
    iters = 0.0
    for t in range(n_steps):
        tau_t = None if tau_seq is None else tau_seq[t * batch.D:(t + 1) * batch.D].contiguous()
        dms, out = _timed(lambda: rollout(batch, qp, qc, tau_t, 1, dt, stages, solver, history,
                                          tol, max_iter, want_traj=False))
        ms += dms
        converged += int((out["status"] == 0).sum().item())
        iters += float(out["iters"].float().mean().item())
        qp, qc = out["q_prev"], out["q_cur"]
    return ProbeResult(solver, ms, converged, model.count * n_steps, iters / n_steps)


def choose_solvers(batch: Batch, q_prev, q_cur, tau_seq, dt: float, stages: int,
                   probe_steps: int = 2, history: int = 8, tol: float = 1e-8,
                   max_iter: dict | None = None, threads: int = 32):
    """One solver per model of `batch` (LBFGS or NEWTON), chosen from probes
    over the first `probe_steps` steps of each bucket's own inputs.
    tau_seq: (n >= probe_steps steps, D) DOF-packed device tensor or None.
    Returns (solvers, {model index: [ProbeResult, ...]})."""
    max_iter = max_iter or {LBFGS: 100, NEWTON: 100}
    solvers, report = [], {}
    for k, m in enumerate(batch.models):
        a, b = int(batch.dof_off[k]), int(batch.dof_off[k + 1])
        tau_k = None
        if tau_seq is not None:
            tau_k = tau_seq[:probe_steps, a:b].contiguous().reshape(-1)
        res = [probe(m, q_prev[a:b].contiguous(), q_cur[a:b].contiguous(), tau_k, probe_steps, dt,
                     stages, sv, history, tol, max_iter[sv], threads)
               for sv in (LBFGS, NEWTON)]
        solvers.append(pick(res))
        report[k] = res
    return solvers, report


def dt_sweep(model, q0, qd0, dts, stages: int, steps: int = 2, history: int = 8, tol: float = 1e-8,
             max_iter: int = 100, threads: int = 32):
    """For each step size: converged fraction, iterations per step and device
    ms per step of each solver over `steps` steps from (q0, qd0) (device
    tensors, DOF-packed), zero torques. Returns a list of dicts."""
    rows = []
    nodes, _ = colloc(stages)
    for dt in dts:
        q_prev = (q0 + float(nodes[0]) * dt * qd0).contiguous()
        row = {"dt": float(dt)}
        for name, sv in (("lbfgs", LBFGS), ("newton", NEWTON)):
            r = probe(model, q_prev, q0, None, steps, dt, stages, sv, history, tol, max_iter,
                      threads)
            row[name] = {"converged_fraction": r.converged / r.total,
                         "iters_per_step": r.iters_per_step, "ms_per_step": r.ms / steps}
        rows.append(row)
    return rows


__all__ = ["ProbeResult", "pick", "probe", "choose_solvers", "dt_sweep"]


# ---------------------------------------------------------------- mapping
@dataclass
class MappingTrial:
    """Device milliseconds of one probe launch under an instance-to-lane
    mapping and a block size (ms = inf: the mapping does not serve it)."""
    mapping: int
    threads: int
    ms: float


def pick_mapping(trials):
    """(mapping, threads) of the fastest trial; ties go to the stage mapping
    (every topology and solver) and then to fewer threads per block."""
    trials = [t for t in trials if np.isfinite(t.ms)]
    if not trials:
        raise ValueError("no mapping served the probe")
    best = min(trials, key=lambda t: (t.ms, t.mapping, t.threads))
    return best.mapping, best.threads


def pick_threads(times, rel_tol: float = 0.01) -> int:
    """Block size from {threads: ms} of a short probe: the smallest block
    within rel_tol of the fastest. A short probe cannot see the tail of a
    long rollout, where a block holds its SM slot until its slowest warp
    is done, so near-ties go to the smaller block."""
    finite = {t: ms for t, ms in times.items() if np.isfinite(ms)}
    if not finite:
        raise ValueError("no block size served the probe")
    best = min(finite.values())
    return min(t for t, ms in finite.items() if ms <= best * (1.0 + rel_tol))


def autotune_mapping(batch: Batch, probe_fn, mappings=(0, 1), threads=(32, 64, 128), repeats=1):
    """Times probe_fn() (a short rollout of the workload on `batch`) under
    every mapping and block size, after one untimed call of each, and leaves
    the batch at the fastest. Returns (mapping, threads, trials)."""
    from ._native import PBADError
    trials = []
    for mp in mappings:
        batch.set_mapping(mp)
        for th in threads:
            batch.set_threads(th)
            try:
                probe_fn()
            except PBADError:
                trials.append(MappingTrial(mp, th, float("inf")))
                continue
            ms = min(_timed(probe_fn)[0] for _ in range(repeats))
            trials.append(MappingTrial(mp, th, ms))
    mp, th = pick_mapping(trials)
    batch.set_mapping(mp)
    batch.set_threads(th)
    return mp, th, trials


def choose_bucket_mappings(n_buckets: int, time_fn, stage: int = 0, link: int = 1):
    """Greedy per-bucket mapping choice (host logic): starting from every
    bucket stage-mapped, bucket k = 0, 1, ... is switched to the link mapping
    and kept there if time_fn(mappings) (milliseconds, inf where the launch
    is refused) falls. Returns (mappings, trials), trials[k] = (ms before,
    ms with bucket k link-mapped)."""
    chosen = [stage] * n_buckets
    best = time_fn(chosen)
    trials = []
    for k in range(n_buckets):
        cand = list(chosen)
        cand[k] = link
        ms = time_fn(cand)
        trials.append((best, ms))
        if ms < best:
            chosen, best = cand, ms
    return chosen, trials


def autotune_bucket_mapping(batch: Batch, probe_fn, repeats=1):
    """Chooses the mapping bucket by bucket inside one launch by
    choose_bucket_mappings, timing probe_fn() (a short rollout on `batch`)
    after one untimed call per candidate; buckets the link mapping cannot
    take (not a chain, more than 32 stage-links, Newton) are refused by the
    library and stay stage-mapped. Leaves the batch at the choice; returns
    (mappings, trials)."""
    from . import MAP_LINK, MAP_STAGE
    from ._native import PBADError

    def time_fn(mappings):
        batch.set_bucket_mapping(mappings)
        try:
            probe_fn()
        except PBADError:
            return float("inf")
        return min(_timed(probe_fn)[0] for _ in range(repeats))

    chosen, trials = choose_bucket_mappings(len(batch.models), time_fn, MAP_STAGE, MAP_LINK)
    batch.set_bucket_mapping(chosen)
    return chosen, trials


def newton_cta_candidates(sizes):
    """Thresholds of the Newton CTA mode worth timing for buckets of the
    given S n (host logic): 4097 (every bucket one warp per instance) and
    each distinct size up to 4096, which puts the buckets at least that
    large in CTA mode."""
    return [4097] + sorted({int(s) for s in sizes if 1 <= int(s) <= 4096}, reverse=True)


def autotune_newton_cta(batch: Batch, probe_fn, stages: int, repeats=1):
    """Times probe_fn() (a short Newton rollout on `batch`) at each threshold
    of newton_cta_candidates over the batch's buckets (S n at `stages`),
    after one untimed call each, and leaves the batch at the fastest.
    Returns (threshold, {threshold: ms})."""
    sizes = [stages * m.n_dof for m in batch.models]
    trials = {}
    for t in newton_cta_candidates(sizes):
        batch.set_newton_cta_min(t)
        probe_fn()
        trials[t] = min(_timed(probe_fn)[0] for _ in range(repeats))
    best = min(trials, key=trials.get)
    batch.set_newton_cta_min(best)
    return best, trials
