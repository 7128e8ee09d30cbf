"""Translation joints and the free 6-DOF root on the CUDA path against the
oracle: evaluations, rollouts with both solvers, the step adjoint, and body
point Jacobians."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1709_04145_b300 import inputs as I

pytestmark = pytest.mark.gpu

REL_EVAL = 1e-10


def _relerr(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("S", [1, 2, 3])
@pytest.mark.parametrize("drag", [0.0, 0.4])
def test_eval_free_root_matches_oracle(S, drag):
    import torch
    import paper_1709_04145_b300 as P
    dt = 0.03
    specs = [I.free_chain(9, 4), I.free_chain(5, 2)]
    batch = P.Batch([P.Model.from_spec(s, drag=drag) for s in specs], max_stages=3, max_history=8)
    rng = np.random.default_rng(91)
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
            om = O.OracleModel.from_spec(spec, b, drag=drag)
            Eo, ro, go, _ = om.eval(S, dt, qs[b], qp[b], qc[b], ta[b], True)
            assert abs(E[batch.inst_off[k] + b] - Eo) <= REL_EVAL * max(abs(Eo), 1.0), (spec.name, b)
            assert _relerr(resids[k][b].reshape(-1), ro) < REL_EVAL, (spec.name, b)
            assert _relerr(grads[k][b].reshape(-1), go) < REL_EVAL, (spec.name, b)


@pytest.mark.parametrize("S,solver", [(1, "lbfgs"), (1, "lm"), (2, "lm")])
def test_free_root_rollout_matches_oracle(S, solver):
    import torch
    import paper_1709_04145_b300 as P
    w = I.swimmers_free(count=6, n_steps=8)
    spec, dt = w["spec"], w["dt"]
    sv = P.LBFGS if solver == "lbfgs" else P.NEWTON
    batch = P.Batch([P.Model.from_spec(spec, drag=w["drag"])], max_stages=S, max_history=8,
                    newton=True)
    nodes, _ = O.colloc(S)
    qp = w["q0"] + nodes[0] * dt * w["qd0"]
    dev = torch.device("cuda:0")
    t = lambda a: torch.tensor(np.ascontiguousarray(a).reshape(-1), device=dev)
    tol, mi = (1e-10, 500) if sv == P.LBFGS else (1e-10, 100)
    out = P.rollout(batch, t(qp), t(w["q0"]), None, 8, dt, S, sv, 8, tol, mi)
    traj = out["traj_cur"].cpu().numpy()
    st = out["status"].cpu().numpy()
    n = spec.n_dof
    for b in range(spec.count):
        om = O.OracleModel.from_spec(spec, b, drag=w["drag"])
        ref = om.rollout(S, dt, qp[b], w["q0"][b], np.zeros((8, n)), solver, 8, tol, mi)
        assert ref["status"] == st[b] == 0, (b, ref["status"], st[b])
        assert np.max(np.abs(traj[:, b * n:(b + 1) * n] - ref["traj_cur"])) <= 1e-7, b


def test_free_root_step_backward_matches_oracle():
    import torch
    import paper_1709_04145_b300 as P
    S, dt = 2, 0.02
    spec = I.free_chain(4, 3)
    batch = P.Batch([P.Model.from_spec(spec, drag=0.3)], max_stages=S, max_history=8, newton=True)
    nodes, _ = O.colloc(S)
    q0, qd0 = I.random_state(spec, 92, pose_scale=0.4, vel_sigma=0.3)
    qp = q0 + nodes[0] * dt * qd0
    rng = np.random.default_rng(93)
    tau = rng.normal(0, 0.1, batch.D)
    dev = torch.device("cuda:0")
    t = lambda a: torch.tensor(np.ascontiguousarray(a).reshape(-1), device=dev)
    out = P.step(batch, t(qp), t(q0), t(tau), dt, S, P.NEWTON, 8, 1e-10, 100)
    assert (out["status"] == 0).all()
    gbar = rng.normal(size=S * batch.D)
    gp, gc, gt, st = P.step_backward(batch, t(qp), t(q0), t(tau), out["q_stages"], t(gbar), dt, S)
    torch.cuda.synchronize()
    assert (st == 0).all()
    qs_h = out["q_stages"].cpu().numpy()
    gp, gc, gt = gp.cpu().numpy(), gc.cpu().numpy(), gt.cpu().numpy()
    n = spec.n_dof
    qp_f, q0_f = qp.reshape(-1), q0.reshape(-1)
    for b in range(spec.count):
        om = O.OracleModel.from_spec(spec, b, drag=0.3)
        sl, ssl = slice(b * n, (b + 1) * n), slice(S * b * n, S * (b + 1) * n)
        rp, rc, rt = om.step_adjoint(S, dt, qp_f[sl], q0_f[sl], tau[sl], qs_h[ssl], gbar[ssl])
        assert _relerr(gp[sl], rp) < 1e-7, b
        assert _relerr(gc[sl], rc) < 1e-7, b
        assert _relerr(gt[sl], rt) < 1e-7, b


def test_free_root_point_jacobian():
    import torch
    import paper_1709_04145_b300 as P
    from paper_1709_04145_b300.autograd import link_points
    spec = I.free_chain(3, 3)
    batch = P.Batch([P.Model.from_spec(spec)], max_stages=1, max_history=0)
    rng = np.random.default_rng(94)
    q = rng.uniform(-0.5, 0.5, (3, spec.n_dof))
    pl = rng.normal(0, 0.3, (3, 3))
    dev = torch.device("cuda:0")
    link = 3
    pos, jac = link_points(batch, torch.tensor(q.reshape(-1), device=dev), [link],
                           torch.tensor(pl, device=dev))
    pos, jac = pos.cpu().numpy(), jac.cpu().numpy().reshape(3, 3, spec.n_dof)
    for b in range(3):
        om = O.OracleModel.from_spec(spec, b)
        ref = om.fk(q[b])[link] @ np.append(pl[b], 1.0)
        assert np.max(np.abs(pos[b] - ref[:3])) < 1e-12
        h = 1e-6
        Jfd = np.stack([(om.fk(q[b] + h * e)[link] @ np.append(pl[b], 1.0) -
                         om.fk(q[b] - h * e)[link] @ np.append(pl[b], 1.0))[:3] / (2 * h)
                        for e in np.eye(spec.n_dof)], axis=1)
        assert np.max(np.abs(jac[b] - Jfd)) < 1e-7
