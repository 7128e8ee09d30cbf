"""Newton with one CTA per instance (buckets with S n >= 128 unknowns: the
instance's four warps split the Jacobian columns and form the Gram matrix
and the Cholesky factor together) against the CPU oracle's LM."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1709_04145_b300 import inputs as I

pytestmark = pytest.mark.gpu


def _t(a, dev):
    import torch
    return torch.tensor(np.ascontiguousarray(a).reshape(-1), device=dev)


def test_cta_newton_ball_chains_match_oracle():
    """22-link ball chains, three stages (S n = 198), dt 0.01, 3 steps,
    tol 1e-6: every step's status and the whole trajectory."""
    import torch

    import paper_1709_04145_b300 as P
    dev = torch.device("cuda:0")
    S, dt, T, tol = 3, 0.01, 3, 1e-6
    spec = I.ball_chain(6, 22, seed=3, radius=0.15)
    q0, qd0 = I.random_state(spec, 5, pose_scale=0.2, vel_sigma=0.2)
    nodes, _ = O.colloc(S)
    qp = q0 + nodes[0] * dt * qd0
    batch = P.Batch([P.Model.from_spec(spec)], max_stages=S, max_history=8, newton=True)
    out = P.rollout(batch, _t(qp, dev), _t(q0, dev), None, T, dt, S, P.NEWTON, 8, tol, 100)
    st = out["step_status"].cpu().numpy()
    traj = out["traj_cur"].cpu().numpy().reshape(T, spec.count, spec.n_dof)
    conv = 0
    for b in (0, 2, 5):
        om = O.OracleModel.from_spec(spec, b)
        ref = om.rollout(S, dt, qp[b], q0[b], np.zeros((T, spec.n_dof)), "lm", 8, tol, 100)
        assert np.array_equal(st[:, b], ref["step_status"]), (b, st[:, b], ref["step_status"])
        for k in range(T):
            if st[k, b] != 0:
                break
            err = np.abs(traj[k, b] - ref["traj_cur"][k])
            assert np.all(err <= 1e-6 * np.maximum(1.0, np.abs(ref["traj_cur"][k]))), (b, k, err.max())
            conv += 1
    assert conv >= 6


def test_cta_newton_scaling_chains_first_step():
    """The scaling study's 50-link hinge chains (four stages, S n = 200, dt
    0.1), 20-iteration cap: the first step's status (it ends at the cap on
    both sides; the |r| reached there depends on the iterates' path, see
    the trajectory tests' rule)."""
    import torch

    import paper_1709_04145_b300 as P
    dev = torch.device("cuda:0")
    ws = I.scaling_chains(50, n_steps=1)
    spec, S, dt = ws["spec"], ws["stages"], ws["dt"]
    nodes, _ = O.colloc(S)
    qp = ws["q0"] + nodes[0] * dt * ws["qd0"]
    batch = P.Batch([P.Model.from_spec(spec)], max_stages=S, max_history=8, newton=True)
    out = P.rollout(batch, _t(qp, dev), _t(ws["q0"], dev), None, 1, dt, S, P.NEWTON, 8, 1e-8, 20)
    st = out["step_status"].cpu().numpy()[0]
    rn = out["step_rnorm"].cpu().numpy()[0]
    for b in (0, 128, 255):
        om = O.OracleModel.from_spec(spec, b)
        ref = om.rollout(S, dt, qp[b], ws["q0"][b], np.zeros((1, spec.n_dof)), "lm", 8, 1e-8, 20)
        assert st[b] == ref["step_status"][0], (b, st[b], ref["step_status"][0])
        if st[b] not in (0, 1):
            assert 0.5 <= rn[b] / ref["step_rnorm"][0] <= 2.0, (b, rn[b], ref["step_rnorm"][0])
        assert rn[b] < out["step_rnorm"].new_tensor([1e30]).item()


def test_cta_newton_adjoint_after_rollout():
    """The adjoint (one warp per instance) of a step solved in CTA mode,
    against the oracle's dense adjoint."""
    import torch

    import paper_1709_04145_b300 as P
    dev = torch.device("cuda:0")
    S, dt = 3, 0.01
    spec = I.ball_chain(4, 22, seed=3, radius=0.15)
    q0, qd0 = I.random_state(spec, 7, pose_scale=0.2, vel_sigma=0.2)
    nodes, _ = O.colloc(S)
    qp = q0 + nodes[0] * dt * qd0
    batch = P.Batch([P.Model.from_spec(spec)], max_stages=S, max_history=8, newton=True)
    out = P.step(batch, _t(qp, dev), _t(q0, dev), None, dt, S, P.NEWTON, 8, 1e-6, 100)
    st = out["status"].cpu().numpy()
    rng = np.random.default_rng(8)
    gbar = rng.normal(size=S * batch.D)
    gp, gc, gt, bst = P.step_backward(batch, _t(qp, dev), _t(q0, dev), None, out["q_stages"],
                                      _t(gbar, dev), dt, S)
    qs = out["q_stages"].cpu().numpy()
    n = spec.n_dof
    checked = 0
    for b in range(spec.count):
        if st[b] != 0:
            continue
        om = O.OracleModel.from_spec(spec, b)
        sl, ssl = slice(b * n, (b + 1) * n), slice(S * b * n, S * (b + 1) * n)
        rp, rc, rt = om.step_adjoint(S, dt, qp[b], q0[b], np.zeros(n), qs[ssl], gbar[ssl])
        for got, ref in ((gp, rp), (gc, rc), (gt, rt)):
            got = got.cpu().numpy()[sl]
            assert np.max(np.abs(got - ref)) <= 1e-6 * np.max(np.abs(ref)), b
        checked += 1
    assert checked >= 2


@pytest.mark.parametrize("S,N,dt", [(1, 200, 0.01), (4, 50, 0.1)])
def test_cta_newton_first_iterate_matches_oracle(S, N, dt):
    """One Newton iteration (Gram matrix, factorisation, solve, damping) on
    hinge chains in CTA mode - S n = 200, including the scaling study's
    200-link chains at one stage - from the same initial guess on both
    sides. The iterate agrees per element within the larger of 1e-6
    max(1, |q|) and the rounding bound of the damped system kappa eps |dx|,
    kappa the condition number of H + lambda_0 I at the initial guess (the
    four-stage 50-link Gram matrix J^T J is singular in binary64, so its
    damped condition number is ~1e12 / lambda_0 ~ 3e13 and the two sides'
    summation orders differ by up to ~1e-4 in its weak directions). The
    sharp check is the step's backward error: the GPU's step dx solves the
    oracle's damped system, |(H + lambda_0 I) dx + g| <= S n eps
    (|H + lambda_0 I| |dx| + |g|) in the max norm (a Cholesky solve's
    bound; a step taken at 10 lambda_0 misses it by 5x). The |r| of the
    iterate is not compared: its second-order part amplifies the weak
    directions (4.6e-4 relative measured)."""
    import torch

    import paper_1709_04145_b300 as P
    dev = torch.device("cuda:0")
    spec = I.rod_chain(4, N, name=f"rod{N}")
    q0, qd0 = I.random_state(spec, 5, pose_scale=0.2, vel_sigma=0.2)
    nodes, _ = O.colloc(S)
    qp = q0 + nodes[0] * dt * qd0
    batch = P.Batch([P.Model.from_spec(spec)], max_stages=S, max_history=8, newton=True)
    out = P.rollout(batch, _t(qp, dev), _t(q0, dev), None, 1, dt, S, P.NEWTON, 8, 1e-12, 1,
                    want_stages=True)
    traj = out["traj_cur"].cpu().numpy().reshape(spec.count, N)
    stages = out["stages_traj"].cpu().numpy()[0].reshape(spec.count, S * N)
    st = out["step_status"].cpu().numpy()[0]
    for b in (0, 3):
        om = O.OracleModel.from_spec(spec, b)
        ref = om.rollout(S, dt, qp[b], q0[b], np.zeros((1, N)), "lm", 8, 1e-12, 1)
        assert st[b] == ref["step_status"][0], (b, st[b], ref["step_status"][0])
        q = ref["traj_cur"][0]
        x0 = om.step(S, dt, qp[b], q0[b], np.zeros(N), "lm", 8, 1e-12, 0)[0]
        x1 = om.step(S, dt, qp[b], q0[b], np.zeros(N), "lm", 8, 1e-12, 1)[0]
        _, r, _, J = om.eval(S, dt, x0, qp[b], q0[b], np.zeros(N), want_jac=True)
        if S == 1:
            H, g = om.hmass(x0.reshape(-1)) / dt**2, r
        else:
            H, g = J.T @ J, J.T @ r
        A = H + 1e-12 * np.diag(H).max() * np.eye(len(H))
        kappa = np.linalg.cond(A)
        bound = kappa * np.finfo(float).eps * np.abs(x1 - x0).max()
        err = np.abs(traj[b] - q)
        assert np.all(err <= np.maximum(1e-6 * np.maximum(1.0, np.abs(q)), bound)), (b, err.max(),
                                                                                    bound)

        def backward_error(dx):
            res = A @ dx + g
            return np.abs(res).max() / (np.abs(A).sum(1).max() * np.abs(dx).max() + np.abs(g).max())
        be_bound = S * N * np.finfo(float).eps
        assert backward_error((x1 - x0).reshape(-1)) <= be_bound  # the oracle took the full step
        assert backward_error(stages[b] - x0.reshape(-1)) <= be_bound, b


def test_cta_threshold_moves_small_systems_to_cta_mode():
    """pbad_batch_set_newton_cta_min: ten-link ball chains at three stages
    (S n = 90, one warp per instance by default) in CTA mode after the
    threshold drops to 64 (the batch's workspace grows for it): the same
    statuses as one warp per instance and as the oracle, converged steps
    equal to the oracle's per element to 1e-6 max(1, |q|); raising the
    threshold to 4097 puts the batch back on one warp per instance, bit for
    bit."""
    import torch

    import paper_1709_04145_b300 as P
    dev = torch.device("cuda:0")
    S, dt, T, tol = 3, 0.02, 4, 1e-8
    spec = I.ball_chain(13, 10, seed=8, radius=0.15)
    q0, qd0 = I.random_state(spec, 9, pose_scale=0.3, vel_sigma=0.3)
    nodes, _ = O.colloc(S)
    qp = q0 + nodes[0] * dt * qd0
    batch = P.Batch([P.Model.from_spec(spec)], max_stages=S, max_history=8, newton=True)
    run = lambda: {k: v.cpu().numpy() for k, v in
                   P.rollout(batch, _t(qp, dev), _t(q0, dev), None, T, dt, S, P.NEWTON, 8, tol,
                             100).items() if hasattr(v, "cpu")}
    warp = run()
    batch.set_newton_cta_min(64)
    cta = run()
    batch.set_newton_cta_min(4097)
    warp2 = run()
    for key in ("traj_cur", "step_status", "iters"):
        assert np.array_equal(warp[key], warp2[key]), key
    n = spec.n_dof
    compared = 0
    for b in (0, 6, 12):
        om = O.OracleModel.from_spec(spec, b)
        ref = om.rollout(S, dt, qp[b], q0[b], np.zeros((T, n)), "lm", 8, tol, 100)
        for k in range(T):
            assert cta["step_status"][k, b] == ref["step_status"][k] == warp["step_status"][k, b]
            if ref["step_status"][k] != 0:
                break
            q = ref["traj_cur"][k]
            for res in (cta, warp):
                err = np.abs(res["traj_cur"][k, b * n:(b + 1) * n] - q)
                assert np.all(err <= 1e-6 * np.maximum(1.0, np.abs(q))), (b, k, err.max())
            compared += 1
    assert compared >= 6
    from paper_1709_04145_b300._native import PBADError
    with pytest.raises(PBADError):
        batch.set_newton_cta_min(0)
