"""Edge cases of the CUDA path through the C ABI: the sizes and arguments the
library rejects before any launch, the largest stage count, the smallest
body (one link, one instance), and the rest state whose step equations hold
at the initial guess (Section 4: with no force and no motion, the objective's
minimiser is the state itself)."""
import dataclasses

import numpy as np
import pytest

import parity_bounds as PB
from oracle import oracle as O
from paper_1709_04145_b300 import inputs as I

pytestmark = pytest.mark.gpu


def _dev():
    import torch
    return torch.device("cuda:0")


def _t(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64).reshape(-1), device=_dev())


def test_rejects_empty_and_out_of_range_arguments():
    import paper_1709_04145_b300 as P
    from paper_1709_04145_b300.models import mass_moments, rest_transforms
    spec = I.rod_chain(2, 3, name="rod3")
    # a model without instances
    with pytest.raises(P.PBADError, match="ARG"):
        P.Model(spec.parent, spec.jtype, spec.axis, mass_moments(spec)[:0],
                rest_transforms(spec)[:0], spec.gravity)
    batch = P.Batch([P.Model.from_spec(spec)], max_stages=2, max_history=4)
    q = _t(np.zeros(batch.D))
    qs = _t(np.zeros(2 * batch.D))
    bad_eval = [dict(stages=0), dict(stages=3), dict(dt=0.0), dict(dt=float("nan")),
                dict(dt=-0.01)]
    for kw in bad_eval:
        a = dict(dt=0.01, stages=1)
        a.update(kw)
        with pytest.raises(P.PBADError, match="ARG"):
            P.eval_objective_grad(batch, qs, q, q, None, a["dt"], a["stages"])
    bad_roll = [dict(n_steps=0), dict(n_steps=-1), dict(history=5), dict(history=-1),
                dict(tol=-1.0), dict(max_iter=-1), dict(stages=0), dict(stages=3),
                dict(solver=P.NEWTON)]  # Newton needs a batch made with newton=True
    for kw in bad_roll:
        a = dict(n_steps=2, dt=0.01, stages=1, solver=P.LBFGS, history=4, tol=1e-9, max_iter=10)
        a.update(kw)
        with pytest.raises(P.PBADError, match="ARG"):
            P.rollout(batch, q, q, None, a["n_steps"], a["dt"], a["stages"], a["solver"],
                      a["history"], a["tol"], a["max_iter"], want_traj=False,
                      want_step_log=False)


def test_eval_at_the_largest_stage_count_matches_oracle():
    """Five stages (the largest the library builds): E, r and the gradient
    per element, under both instance-to-lane mappings (5 x 4 = 20 lanes per
    ball chain in the link mapping) and on trees (stage mapping)."""
    import paper_1709_04145_b300 as P
    S, dt = 5, 0.02
    chains = [I.rod_chain(3, 3, name="rod3"), I.ball_chain(5, 4, seed=51, radius=0.12)]
    tree = I.humanoid(2, seed=52)
    rng = np.random.default_rng(53)

    def case(spec):
        B, n = spec.count, spec.n_dof
        q_cur = rng.uniform(-0.6, 0.6, size=(B, n))
        q_prev = q_cur + rng.normal(0, 0.02, size=(B, n))
        tau = rng.normal(0, 0.3, size=(B, n))
        qs = q_cur[:, None, :] + rng.normal(0, 0.03, size=(B, S, n))
        return q_prev, q_cur, tau, qs

    for specs, mappings in ((chains, (P.MAP_STAGE, P.MAP_LINK)), ([tree], (P.MAP_STAGE,))):
        batch = P.Batch([P.Model.from_spec(s) for s in specs], max_stages=S, max_history=8)
        cases = [case(s) for s in specs]
        cat = lambda j: _t(np.concatenate([c[j].reshape(-1) for c in cases]))
        for mapping in mappings:
            batch.set_mapping(mapping)
            E, g, r = P.eval_objective_grad(batch, cat(3), cat(0), cat(1), cat(2), dt, S)
            E = E.cpu().numpy()
            grads = batch.unpack(g.cpu().numpy(), S)
            resids = batch.unpack(r.cpu().numpy(), S)
            for k, spec in enumerate(specs):
                qp, qc, ta, qs = cases[k]
                for b in range(spec.count):
                    om = O.OracleModel.from_spec(spec, b)
                    Eo, ro, go, rb, gb = PB.oracle_eval_bounds(om, S, dt, qs[b], qp[b], qc[b], ta[b])
                    assert abs(E[batch.inst_off[k] + b] - Eo) <= PB.REL_EVAL * max(abs(Eo), 1.0)
                    assert PB.ratio(resids[k][b], ro, rb) <= 1.0, (mapping, spec.name, b)
                    assert PB.ratio(grads[k][b], go, gb) <= 1.0, (mapping, spec.name, b)


@pytest.mark.parametrize("S", [1, 2])
def test_one_link_one_instance_rollout_matches_oracle(S):
    """The smallest body: one rod on a hinge, one instance, 30 L-BFGS steps
    under both mappings, every step's status and the trajectory."""
    import paper_1709_04145_b300 as P
    spec = I.rod_chain(1, 1, name="rod1")
    dt, n_steps, tol = 0.01, 30, 1e-9
    q0 = np.array([0.7])
    qd0 = np.array([-0.4])
    nodes, _ = O.colloc(S)
    qp0 = q0 + nodes[0] * dt * qd0
    om = O.OracleModel.from_spec(spec, 0)
    ref = om.rollout(S, dt, qp0, q0, np.zeros((n_steps, 1)), "lbfgs", 8, tol, 1000)
    assert ref["status"] == 0
    batch = P.Batch([P.Model.from_spec(spec)], max_stages=S, max_history=8)
    for mapping in (P.MAP_STAGE, P.MAP_LINK):
        batch.set_mapping(mapping)
        out = P.rollout(batch, _t(qp0), _t(q0), None, n_steps, dt, S, P.LBFGS, 8, tol, 1000)
        assert np.array_equal(out["step_status"].cpu().numpy().reshape(-1), ref["step_status"])
        traj = out["traj_cur"].cpu().numpy().reshape(n_steps, 1)
        assert np.max(np.abs(traj - ref["traj_cur"])) <= 1e-7, mapping


@pytest.mark.parametrize("S", [1, 2, 3])
def test_rest_state_stays_bitwise_unchanged(S):
    """No gravity, no torque, q_prev = q_cur: the step equations hold at the
    initial guess (every stage at q_cur), so every step ends CONVERGED
    without an iteration and the state is bitwise unchanged over 50 steps,
    for both solvers and both mappings. The tolerance is twice the rounding
    floor of r, the most the residual of an exact root can show in binary64.
    The same holds hanging straight down under gravity (q = 0)."""
    import paper_1709_04145_b300 as P
    dt, n_steps = 0.05, 50
    spec = I.ball_chain(5, 4, seed=9, radius=0.1)
    flat = dataclasses.replace(spec, gravity=np.zeros(3))
    q = np.random.default_rng(7).uniform(-0.5, 0.5, (spec.count, spec.n_dof))
    for body, q0 in ((flat, q), (spec, np.zeros_like(q))):
        tol = 2.0 * max(O.OracleModel.from_spec(body, b).floor(S, dt) for b in range(body.count))
        batch = P.Batch([P.Model.from_spec(body)], max_stages=S, max_history=8, newton=True)
        for solver in (P.LBFGS, P.NEWTON):
            for mapping in ((P.MAP_STAGE, P.MAP_LINK) if solver == P.LBFGS else (P.MAP_STAGE,)):
                batch.set_mapping(mapping)
                out = P.rollout(batch, _t(q0), _t(q0), None, n_steps, dt, S, solver, 8, tol, 100)
                st = out["step_status"].cpu().numpy()
                assert np.all(st == 0), (solver, mapping, st)
                assert np.all(out["iters"].cpu().numpy() == 0), (solver, mapping)
                traj = out["traj_cur"].cpu().numpy().reshape(n_steps, -1)
                assert np.array_equal(traj, np.broadcast_to(q0.reshape(-1), traj.shape))
