"""Per-step outcomes of the CUDA rollouts against the oracle: each step's
status and the |r|_2 it ended at (pbad_rollout's step logs), and the
STALLED status (a line search / LM damping that cannot lower E at |r| below
1e3 times the binary64 rounding floor)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1709_04145_b300 import inputs as I

pytestmark = pytest.mark.gpu


def _t(a, dev):
    import torch
    return torch.tensor(np.ascontiguousarray(a).reshape(-1), device=dev)


def test_pendulum_step_log_matches_oracle():
    import torch

    import paper_1709_04145_b300 as P
    dev = torch.device("cuda:0")
    w = I.pendulum3()
    spec = w["spec"]
    T = 40
    batch = P.Batch([P.Model.from_spec(spec)], max_stages=1, max_history=w["history"])
    q0 = w["q0"]
    out = P.rollout(batch, _t(q0, dev), _t(q0, dev), None, T, w["dt"], 1, P.LBFGS,
                    w["history"], w["tol"], 2000)
    st = out["step_status"].cpu().numpy()[:, 0]
    rn = out["step_rnorm"].cpu().numpy()[:, 0]
    om = O.OracleModel.from_spec(spec, 0)
    ref = om.rollout(1, w["dt"], q0[0], q0[0], np.zeros((T, 3)), "lbfgs", w["history"],
                     w["tol"], 2000)
    assert np.array_equal(st, ref["step_status"])
    assert np.all(rn[st == 0] < w["tol"]) and np.all(ref["step_rnorm"][st == 0] < w["tol"])
    assert int(out["status"][0]) == ref["status"]


@pytest.mark.parametrize("solver,S,dt", [("lm", 2, 0.05), ("lbfgs", 1, 0.01)])
def test_step_log_status_and_exit_residual_match_oracle(solver, S, dt):
    """Five-link hinge chains (LM with two stages at the uneven batch's dt
    0.05; L-BFGS with one stage at dt 0.01, where it converges): every
    step's status equals the oracle's while the trajectories agree, and so
    does the |r| it ended at (relative 1e-6 where the step did not converge;
    below tol where it did)."""
    import torch

    import paper_1709_04145_b300 as P
    dev = torch.device("cuda:0")
    T, tol = 6, 1e-8
    spec = I.rod_chain(40, 5, name="rods5")
    q0, qd0 = I.random_state(spec, 91)
    nodes, _ = O.colloc(S)
    qp = q0 + nodes[0] * dt * qd0
    sv, mi = (P.NEWTON, 100) if solver == "lm" else (P.LBFGS, 2000)
    batch = P.Batch([P.Model.from_spec(spec)], max_stages=S, max_history=8, newton=True)
    out = P.rollout(batch, _t(qp, dev), _t(q0, dev), None, T, dt, S, sv, 8, tol, mi)
    st = out["step_status"].cpu().numpy()
    rn = out["step_rnorm"].cpu().numpy()
    traj = out["traj_cur"].cpu().numpy().reshape(T, spec.count, spec.n_dof)
    compared = 0
    for b in range(0, spec.count, 5):
        om = O.OracleModel.from_spec(spec, b)
        ref = om.rollout(S, dt, qp[b], q0[b], np.zeros((T, spec.n_dof)), solver, 8, tol, mi)
        for k in range(T):
            # compare while the trajectories still agree (the iterates of an
            # unconverged step decorrelate at the rounding level)
            if np.max(np.abs(traj[k, b] - ref["traj_cur"][k])) > 1e-6:
                break
            assert st[k, b] == ref["step_status"][k], (b, k, st[k, b], ref["step_status"][k])
            if st[k, b] == 0:
                assert rn[k, b] < tol and ref["step_rnorm"][k] < tol
            else:
                assert abs(rn[k, b] - ref["step_rnorm"][k]) <= 1e-6 * ref["step_rnorm"][k]
            compared += 1
    assert compared >= 8 * T // 2


def test_unconverged_lbfgs_first_step_matches_oracle_status():
    """L-BFGS on the uneven batch's five-link chains (dt 0.05, two stages,
    torques) ends its steps at the 100-iteration cap on both sides: the first
    step's status agrees, and its exit |r| is of the same size (the iterates
    of 100 iterations on a Gauss-Newton matrix of condition ~1e10 differ
    beyond the rounding level, so no closer agreement is defined)."""
    import torch

    import paper_1709_04145_b300 as P
    dev = torch.device("cuda:0")
    u = I.uneven_batch(n_steps=1)
    spec, (q0, qd0), tau = u["specs"][2], u["states"][2], u["taus"][2]
    S, dt = u["stages"], u["dt"]
    nodes, _ = O.colloc(S)
    qp = q0 + nodes[0] * dt * qd0
    batch = P.Batch([P.Model.from_spec(spec)], max_stages=S, max_history=8)
    out = P.rollout(batch, _t(qp, dev), _t(q0, dev), _t(tau, dev), 1, dt, S, P.LBFGS, 8, u["tol"], 100)
    st = out["step_status"].cpu().numpy()[0]
    rn = out["step_rnorm"].cpu().numpy()[0]
    for b in range(0, spec.count, 128):
        om = O.OracleModel.from_spec(spec, b)
        ref = om.rollout(S, dt, qp[b], q0[b], tau[:, b], "lbfgs", 8, u["tol"], 100)
        assert st[b] == ref["step_status"][0], (b, st[b], ref["step_status"][0])
        if st[b] != 0:
            assert 0.25 <= rn[b] / ref["step_rnorm"][0] <= 4.0, (b, rn[b], ref["step_rnorm"][0])


def test_lm_at_zero_tolerance_ends_stalled_on_the_gpu():
    """With tol = 0 no step can converge; LM's damping loop then fails at
    the rounding floor and every step must end STALLED, at an |r| below
    1e3 times the oracle's floor."""
    import torch

    import paper_1709_04145_b300 as P
    dev = torch.device("cuda:0")
    S, dt, T = 2, 0.01, 4
    spec = I.rod_chain(33, 5, name="rods5")
    q0, qd0 = I.random_state(spec, 3)
    nodes, _ = O.colloc(S)
    qp = q0 + nodes[0] * dt * qd0
    batch = P.Batch([P.Model.from_spec(spec)], max_stages=S, max_history=8, newton=True)
    out = P.rollout(batch, _t(qp, dev), _t(q0, dev), None, T, dt, S, P.NEWTON, 8, 0.0, 100)
    st = out["step_status"].cpu().numpy()
    rn = out["step_rnorm"].cpu().numpy()
    assert np.all(st == 5), np.unique(st, return_counts=True)
    for b in range(spec.count):
        fl = O.OracleModel.from_spec(spec, b).floor(S, dt)
        assert np.all(rn[:, b] <= 1e3 * fl) and np.all(rn[:, b] > 0)
    assert np.all(out["status"].cpu().numpy() == 5)
