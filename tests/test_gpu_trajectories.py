"""Trajectory parity on the workloads the benchmark times, at their full
batch sizes and in their launch configurations: sampled instances' whole
trajectories, per-step statuses and exit |r| against the CPU oracle.

Comparison rule, step by step for each sampled instance:
  - the step's status equals the oracle's;
  - a converged step (|r| < tol on both sides): every coordinate agrees to
    |dq| <= 1e-6 max(1, |q|) (per element: relative 1e-6 with an absolute
    floor of 1e-6 rad). Both sides stop at |r| < tol = 1e-8 and the smallest
    singular value of these step Jacobians is ~0.7 or more, so each step's
    solution is fixed to ~1.4e-8; the observed growth over 20 steps is below
    4e-8;
  - the first step that ends unsolved must end with the same status, and
    the comparison of that instance stops there: the iterates of an
    unsolved step are not fixed by the step equations and decorrelate from
    the oracle's at the rounding level. Its exit |r| must agree within a
    factor of 2 where the step ended in a failed line search or damping
    loop (LS_FAIL, STALLED: the point where descent stopped); at the
    iteration cap (MAX_ITER) it depends on the path the iterates took (a
    25-link chain ended at 3.5e-5 on the GPU and 4.2e-3 in the oracle after
    100 LM iterations) and is not compared;
  - two exceptions are counted instead of failed, and each test bounds how
    many sampled instances may end so: a step that converges on one side on
    its last allowed iteration and ends MAX_ITER on the other (the outcome
    at the iteration cap turns on the rounding of the last iterate), and an
    unsolved step that ends MAX_ITER on one side and in a failed damping
    loop (LS_FAIL or STALLED) on the other (both unsolved: which stopping
    rule fires first depends on the path the decorrelated iterates take).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1709_04145_b300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-8


def _compare(name, b, st, rn, traj, ref, tol=TOL, cap=None):
    """Applies the rule above to one instance; returns the number of steps
    compared as converged (cap: list that collects the instances that ended
    at the iteration cap on one side only)."""
    conv = 0
    for k in range(len(st)):
        pair = {int(st[k]), int(ref["step_status"][k])}
        if st[k] != ref["step_status"][k] and (pair == {0, 1} or pair in ({1, 2}, {1, 5})):
            assert cap is not None, (name, b, k, st[k], ref["step_status"][k])
            cap.append((name, b, k))
            break
        assert st[k] == ref["step_status"][k], (name, b, k, st[k], ref["step_status"][k])
        if st[k] == 0:
            q = ref["traj_cur"][k]
            err = np.abs(traj[k] - q)
            assert np.all(err <= 1e-6 * np.maximum(1.0, np.abs(q))), (name, b, k, err.max())
            assert rn[k] < tol and ref["step_rnorm"][k] < tol
            conv += 1
        else:
            if st[k] != 1:
                assert 0.5 <= rn[k] / ref["step_rnorm"][k] <= 2.0, (name, b, k, rn[k],
                                                                   ref["step_rnorm"][k])
            break
    return conv


def _run(P, specs_states, S, dt, T, solvers, max_iter, taus=None, mapping=None):
    import torch
    dev = torch.device("cuda:0")
    batch = P.Batch([P.Model.from_spec(s) for s, _ in specs_states], max_stages=S, max_history=8,
                    newton=True)
    if mapping is not None:
        batch.set_mapping(mapping)
    nodes, _ = O.colloc(S)
    qc = np.concatenate([q0.reshape(-1) for _, (q0, _) in specs_states])
    qp = np.concatenate([(q0 + nodes[0] * dt * qd0).reshape(-1) for _, (q0, qd0) in specs_states])
    tau = None
    if taus is not None:
        tau = torch.tensor(np.concatenate([t.reshape(T, -1) for t in taus], axis=1).reshape(-1),
                           device=dev)
    out = P.rollout(batch, torch.tensor(qp, device=dev), torch.tensor(qc, device=dev), tau, T, dt,
                    S, solvers, 8, TOL, max_iter)
    res = {k: out[k].cpu().numpy() for k in ("traj_cur", "step_status", "step_rnorm")}
    return batch, res


def _check_bucket(batch, res, k, spec, state, tau, S, dt, T, solver, max_iter, sample, cap=None):
    q0, qd0 = state
    nodes, _ = O.colloc(S)
    n = spec.n_dof
    i0, d0 = int(batch.inst_off[k]), int(batch.dof_off[k])
    conv = 0
    for b in sample:
        om = O.OracleModel.from_spec(spec, int(b))
        qp = q0[b] + nodes[0] * dt * qd0[b]
        tq = tau[:, b] if tau is not None else np.zeros((T, n))
        ref = om.rollout(S, dt, qp, q0[b], tq, solver, 8, TOL, max_iter)
        traj = res["traj_cur"][:, d0 + b * n:d0 + (b + 1) * n]
        conv += _compare(spec.name, b, res["step_status"][:, i0 + b], res["step_rnorm"][:, i0 + b],
                         traj, ref, cap=cap)
    return conv


def test_ball_chains_newton_20_steps():
    """The batched workload (4096 ten-link ball chains, three stages, dt
    0.033) solved by Newton, 20 steps, twelve sampled instances."""
    import paper_1709_04145_b300 as P
    w = I.ball_chains(count=4096, n_links=10, n_steps=20)
    spec = w["spec"]
    batch, res = _run(P, [(spec, (w["q0"], w["qd0"]))], 3, w["dt"], 20, P.NEWTON, 100)
    sample = np.linspace(0, spec.count - 1, 12).astype(int)
    cap = []
    conv = _check_bucket(batch, res, 0, spec, (w["q0"], w["qd0"]), None, 3, w["dt"], 20, "lm",
                         100, sample, cap)
    # ~3% of steps end unsolved and each instance is compared up to its
    # first one: about half the sampled instance-steps are compared converged
    assert conv >= 12 * 20 * 0.4, conv
    assert len(cap) <= 1, cap


def test_uneven_batch_chosen_solvers_4_steps():
    """The uneven batch in one launch with the solver choice's solvers
    (Newton for the 1024 humanoids and the 2048 five-link chains, L-BFGS
    for the 1024 fifty-link chains), torques, dt 0.05, two stages, 4
    steps: sampled humanoids and five-link chains whole, the fifty-link
    chains' first step."""
    import paper_1709_04145_b300 as P
    u = I.uneven_batch(n_steps=4)
    specs, states, taus = u["specs"], u["states"], u["taus"]
    batch, res = _run(P, list(zip(specs, states)), 2, u["dt"], 4, [P.NEWTON, P.LBFGS, P.NEWTON],
                      100, taus=taus)
    cap = []
    conv = _check_bucket(batch, res, 0, specs[0], states[0], taus[0], 2, u["dt"], 4, "lm", 100,
                         np.linspace(0, specs[0].count - 1, 10).astype(int), cap)
    conv += _check_bucket(batch, res, 2, specs[2], states[2], taus[2], 2, u["dt"], 4, "lm", 100,
                          np.linspace(0, specs[2].count - 1, 10).astype(int), cap)
    assert conv >= 40, conv
    assert len(cap) <= 2, cap
    # the fifty-link chains (L-BFGS): the first step's status and exit |r|
    spec, (q0, qd0), tau = specs[1], states[1], taus[1]
    nodes, _ = O.colloc(2)
    i0 = int(batch.inst_off[1])
    for b in (0, 511, 1023):
        om = O.OracleModel.from_spec(spec, b)
        ref = om.rollout(2, u["dt"], q0[b] + nodes[0] * u["dt"] * qd0[b], q0[b], tau[:1, b], "lbfgs",
                         8, TOL, 100)
        assert res["step_status"][0, i0 + b] == ref["step_status"][0], b


def test_scaling_chains_newton_25_links():
    """Scaling study's 25-link hinge chains (256 instances, four stages, dt
    0.1), Newton, 5 steps, sampled instances up to their first unsolved
    step."""
    import paper_1709_04145_b300 as P
    ws = I.scaling_chains(25, n_steps=5)
    spec = ws["spec"]
    batch, res = _run(P, [(spec, (ws["q0"], ws["qd0"]))], 4, ws["dt"], 5, P.NEWTON, 100)
    cap = []
    _check_bucket(batch, res, 0, spec, (ws["q0"], ws["qd0"]), None, 4, ws["dt"], 5, "lm", 100,
                  [0, 11, 22, 100, 150, 200, 255], cap)
    assert len(cap) <= 2, cap


def test_ball_chains_lbfgs_link_parallel_first_steps():
    """The benchmark's own configuration (4096 ten-link ball chains, L-BFGS
    m = 8, 50 iterations, link-parallel mapping): no step converges on either
    side; the first step ends with the oracle's status, at an |r| of the
    same size (the iterates of 50 L-BFGS iterations at condition ~1e8
    differ beyond the rounding level, so no closer agreement is defined)."""
    import paper_1709_04145_b300 as P
    w = I.ball_chains(count=4096, n_links=10, n_steps=2)
    spec = w["spec"]
    batch, res = _run(P, [(spec, (w["q0"], w["qd0"]))], 3, w["dt"], 2, P.LBFGS, 50,
                      mapping=P.MAP_LINK)
    nodes, _ = O.colloc(3)
    for b in (0, 1365, 2730, 4095):
        om = O.OracleModel.from_spec(spec, b)
        ref = om.rollout(3, w["dt"], w["q0"][b] + nodes[0] * w["dt"] * w["qd0"][b], w["q0"][b],
                         np.zeros((1, spec.n_dof)), "lbfgs", 8, TOL, 50)
        assert res["step_status"][0, b] == ref["step_status"][0], b
        assert 0.25 <= res["step_rnorm"][0, b] / ref["step_rnorm"][0] <= 4.0, b
