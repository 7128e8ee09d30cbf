"""Drag potential (Section 6.2) on the CUDA path against the oracle: single
evaluations, rollouts with both solvers, the adjoint, and the batch-creation
rule for the one-stage drag storage."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1709_04145_b300 import inputs as I

pytestmark = pytest.mark.gpu

REL_EVAL = 1e-10
DRAG = 0.6


def _relerr(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def _specs():
    return [I.rod_chain(5, 3, name="rod3"), I.ball_chain(7, 4, seed=81, radius=0.1),
            I.humanoid(3, seed=82)]


@pytest.mark.parametrize("S", [1, 2, 3, 4])
def test_eval_with_drag_matches_oracle(S):
    import torch
    import paper_1709_04145_b300 as P
    dt = 0.02
    specs = _specs()
    batch = P.Batch([P.Model.from_spec(s, drag=DRAG) for s in specs], max_stages=5, max_history=8)
    rng = np.random.default_rng(83)
    cases = []
    for s in specs:
        B, n = s.count, s.n_dof
        qc = rng.uniform(-0.6, 0.6, (B, n))
        cases.append((qc + rng.normal(0, 0.02, (B, n)), qc, rng.normal(0, 0.3, (B, n)),
                      qc[:, None, :] + rng.normal(0, 0.03, (B, S, n))))
    dev = torch.device("cuda:0")
    cat = lambda j: torch.tensor(np.concatenate([c[j].reshape(-1) for c in cases]), device=dev)
    E, grad, resid = P.eval_objective_grad(batch, cat(3), cat(0), cat(1), cat(2), dt, S)
    torch.cuda.synchronize()
    E = E.cpu().numpy()
    grads = batch.unpack(grad.cpu().numpy(), S)
    resids = batch.unpack(resid.cpu().numpy(), S)
    for k, spec in enumerate(specs):
        qp, qc, ta, qs = cases[k]
        for b in range(spec.count):
            om = O.OracleModel.from_spec(spec, b, drag=DRAG)
            Eo, ro, go, _ = om.eval(S, dt, qs[b], qp[b], qc[b], ta[b], True)
            assert abs(E[batch.inst_off[k] + b] - Eo) <= REL_EVAL * max(abs(Eo), 1.0), (spec.name, b)
            assert _relerr(resids[k][b].reshape(-1), ro) < REL_EVAL, (spec.name, b)
            assert _relerr(grads[k][b].reshape(-1), go) < REL_EVAL, (spec.name, b)


@pytest.mark.parametrize("S,solver", [(1, "lbfgs"), (2, "lm"), (3, "lm")])
def test_rollout_with_drag_matches_oracle(S, solver):
    import torch
    import paper_1709_04145_b300 as P
    specs = [I.rod_chain(3, 4, name="rod4"), I.ball_chain(2, 3, seed=84, radius=0.2)]
    sv = P.LBFGS if solver == "lbfgs" else P.NEWTON
    batch = P.Batch([P.Model.from_spec(s, drag=DRAG) for s in specs], max_stages=3, max_history=8,
                    newton=True)
    dt, n_steps, tol = 0.01, 6, 1e-9
    nodes, _ = O.colloc(S)
    states = [I.random_state(s, 85 + k, pose_scale=0.4, vel_sigma=0.3) for k, s in enumerate(specs)]
    taus = [I.torques(s, n_steps, 87 + k, sigma=0.1) for k, s in enumerate(specs)]
    qps = [q0 + nodes[0] * dt * qd0 for q0, qd0 in states]
    dev = torch.device("cuda:0")
    qc = torch.tensor(np.concatenate([q0.reshape(-1) for q0, _ in states]), device=dev)
    qp = torch.tensor(np.concatenate([x.reshape(-1) for x in qps]), device=dev)
    tau = torch.tensor(np.concatenate([t.reshape(n_steps, -1) for t in taus], axis=1).reshape(-1),
                       device=dev)
    out = P.rollout(batch, qp, qc, tau, n_steps, dt, S, sv, 8, tol, 2000 if sv == P.LBFGS else 100)
    traj = out["traj_cur"].cpu().numpy()
    st = out["status"].cpu().numpy()
    n_conv = 0
    for k, spec in enumerate(specs):
        for b in range(spec.count):
            om = O.OracleModel.from_spec(spec, b, drag=DRAG)
            ref = om.rollout(S, dt, qps[k][b], states[k][0][b], taus[k][:, b, :], solver, 8, tol,
                             2000 if sv == P.LBFGS else 100)
            a = batch.dof_off[k] + b * spec.n_dof
            assert ref["status"] == st[batch.inst_off[k] + b], (spec.name, b)
            if ref["status"] == 0:
                n_conv += 1
                assert np.max(np.abs(traj[:, a:a + spec.n_dof] - ref["traj_cur"])) <= 1e-7, (spec.name, b)
    assert n_conv >= 4


def test_step_backward_with_drag_matches_oracle():
    import torch
    import paper_1709_04145_b300 as P
    S, dt = 2, 0.02
    specs = [I.rod_chain(3, 4, name="rod4"), I.humanoid(2, seed=88)]
    batch = P.Batch([P.Model.from_spec(s, drag=DRAG) for s in specs], max_stages=S, max_history=8,
                    newton=True)
    nodes, _ = O.colloc(S)
    states = [I.random_state(s, 89 + k, pose_scale=0.4, vel_sigma=0.3) for k, s in enumerate(specs)]
    q0 = np.concatenate([st[0].reshape(-1) for st in states])
    qd0 = np.concatenate([st[1].reshape(-1) for st in states])
    qp = q0 + nodes[0] * dt * qd0
    rng = np.random.default_rng(90)
    tau = rng.normal(0, 0.1, batch.D)
    dev = torch.device("cuda:0")
    t = lambda a: torch.tensor(a, device=dev)
    out = P.step(batch, t(qp), t(q0), t(tau), dt, S, P.NEWTON, 8, 1e-10, 100)
    assert (out["status"] == 0).all()
    gbar = rng.normal(size=S * batch.D)
    gp, gc, gt, st = P.step_backward(batch, t(qp), t(q0), t(tau), out["q_stages"], t(gbar), dt, S)
    torch.cuda.synchronize()
    assert (st == 0).all()
    qs_h = out["q_stages"].cpu().numpy()
    gp, gc, gt = gp.cpu().numpy(), gc.cpu().numpy(), gt.cpu().numpy()
    for k, spec in enumerate(specs):
        for b in range(spec.count):
            om = O.OracleModel.from_spec(spec, b, drag=DRAG)
            a = batch.dof_off[k] + b * spec.n_dof
            sl, ssl = slice(a, a + spec.n_dof), slice(S * a, S * (a + spec.n_dof))
            rp, rc, rt = om.step_adjoint(S, dt, qp[sl], q0[sl], tau[sl], qs_h[ssl], gbar[ssl])
            assert _relerr(gp[sl], rp) < 1e-7, (spec.name, b)
            assert _relerr(gc[sl], rc) < 1e-7, (spec.name, b)
            assert _relerr(gt[sl], rt) < 1e-7, (spec.name, b)


def test_drag_set_after_batch_creation():
    """A one-stage call needs the drag storage reserved at batch creation;
    stage counts >= 2 do not."""
    import torch
    import paper_1709_04145_b300 as P
    from paper_1709_04145_b300._native import lib
    spec = I.rod_chain(2, 3)
    model = P.Model.from_spec(spec)
    batch = P.Batch([model], max_stages=2, max_history=4)
    assert lib().pbad_model_set_drag(model._h, DRAG) == 0
    assert lib().pbad_model_set_drag(model._h, -1.0) != 0
    dev = torch.device("cuda:0")
    q = torch.zeros(batch.D, dtype=torch.float64, device=dev)
    with pytest.raises(P.PBADError):
        P.eval_objective_grad(batch, q, q, q, None, 0.02, 1)
    E, _, _ = P.eval_objective_grad(batch, torch.zeros(2 * batch.D, dtype=torch.float64, device=dev),
                                    q, q, None, 0.02, 2)
    assert torch.isfinite(E).all()
