"""Penalty contact of Eq. FRI on the CUDA path against the oracle (one
stage): evaluations with points in the ground, rollouts of a free chain
falling onto the ground with both solvers, the step adjoint, and the
refusal for two or more stages."""
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


def _contact(spec, d1=200.0, d2=30.0):
    links = [l for l in range(spec.n_links) if spec.length[0, l] > 0]
    pts = [[0.0, 0.0, 0.0] for _ in links] + [[0.0, 0.0, -spec.length[0, l]] for l in links]
    return dict(link=links + links, point=pts, z0=0.0, d1=d1, d2=d2)


def test_eval_with_contact_matches_oracle():
    import torch
    import paper_1709_04145_b300 as P
    spec = I.free_chain(24, 3)
    contact = _contact(spec)
    batch = P.Batch([P.Model.from_spec(spec, drag=0.2, contact=contact)], max_stages=2,
                    max_history=8)
    rng = np.random.default_rng(101)
    B, n = spec.count, spec.n_dof
    qc = np.concatenate([rng.uniform(-0.3, 0.3, (B, 2)), rng.uniform(0.1, 0.6, (B, 1)),
                         rng.uniform(-0.6, 0.6, (B, n - 3))], axis=1)
    qp = qc + rng.normal(0, 0.01, (B, n))
    qs = qc + rng.normal(0, 0.02, (B, n))
    qs[:, 2] -= 0.2  # drive tips below the ground
    tau = rng.normal(0, 0.2, (B, n))
    dev = torch.device("cuda:0")
    t = lambda a: torch.tensor(a.reshape(-1), device=dev)
    E, grad, resid = P.eval_objective_grad(batch, t(qs), t(qp), t(qc), t(tau), 0.02, 1)
    E, grad = E.cpu().numpy(), grad.cpu().numpy().reshape(B, n)
    active = 0
    for b in range(B):
        om = O.OracleModel.from_spec(spec, b, drag=0.2, contact=contact)
        Eo, ro, go, _ = om.eval(1, 0.02, qs[b], qp[b], qc[b], tau[b], True)
        Eo0 = O.OracleModel.from_spec(spec, b, drag=0.2).eval(1, 0.02, qs[b], qp[b], qc[b], tau[b], False)[0]
        active += Eo != Eo0
        assert abs(E[b] - Eo) <= REL_EVAL * max(abs(Eo), 1.0), b
        assert _relerr(grad[b], go) < REL_EVAL, b
    assert active >= B // 2


@pytest.mark.parametrize("solver", ["lm", "lbfgs"])
def test_falling_chain_rollout_matches_oracle(solver):
    import torch
    import paper_1709_04145_b300 as P
    spec = I.free_chain(4, 3)
    contact = _contact(spec, d1=300.0, d2=20.0)
    sv = P.NEWTON if solver == "lm" else P.LBFGS
    batch = P.Batch([P.Model.from_spec(spec, drag=0.1, contact=contact)], max_stages=1,
                    max_history=8, newton=True)
    rng = np.random.default_rng(102)
    n = spec.n_dof
    q0 = np.concatenate([np.zeros((4, 2)), np.full((4, 1), 0.25), rng.uniform(-0.4, 0.4, (4, n - 3))], axis=1)
    dt, n_steps, tol = 0.01, 30, 1e-9
    mi = 100 if sv == P.NEWTON else 2000
    dev = torch.device("cuda:0")
    t = lambda a: torch.tensor(np.ascontiguousarray(a).reshape(-1), device=dev)
    out = P.rollout(batch, t(q0), t(q0), None, n_steps, dt, 1, sv, 8, tol, mi)
    traj = out["traj_cur"].cpu().numpy()
    st = out["status"].cpu().numpy()
    touched = 0
    for b in range(4):
        om = O.OracleModel.from_spec(spec, b, drag=0.1, contact=contact)
        ref = om.rollout(1, dt, q0[b], q0[b], np.zeros((n_steps, n)), solver, 8, tol, mi)
        assert ref["status"] == st[b] == 0, (b, ref["status"], st[b])
        assert np.max(np.abs(traj[:, b * n:(b + 1) * n] - ref["traj_cur"])) <= 1e-7, b
        z = [min((om.fk(q)[l] @ np.array([0, 0, -spec.length[0, l], 1.0]))[2] for l in range(1, spec.n_links))
             for q in ref["traj_cur"]]
        touched += min(z) < 0
    assert touched >= 2  # the chains reach the ground within the rollout


def test_contact_step_backward_matches_oracle():
    import torch
    import paper_1709_04145_b300 as P
    spec = I.free_chain(3, 2)
    contact = _contact(spec)
    batch = P.Batch([P.Model.from_spec(spec, contact=contact)], max_stages=1, max_history=8,
                    newton=True)
    rng = np.random.default_rng(103)
    n = spec.n_dof
    q0 = np.concatenate([np.zeros((3, 2)), np.full((3, 1), 0.1), rng.uniform(-0.5, 0.5, (3, n - 3))], axis=1)
    qp = q0 + rng.normal(0, 0.005, q0.shape)
    tau = rng.normal(0, 0.1, (3, n))
    dev = torch.device("cuda:0")
    t = lambda a: torch.tensor(np.ascontiguousarray(a).reshape(-1), device=dev)
    dt = 0.01
    # tolerance above the FP64 floor of r with the contact stiffness in it
    out = P.step(batch, t(qp), t(q0), t(tau), dt, 1, P.NEWTON, 8, 1e-9, 100)
    conv = out["status"].cpu().numpy() == 0
    assert conv.sum() >= 2
    gbar = rng.normal(size=batch.D)
    gp, gc, gt, st = P.step_backward(batch, t(qp), t(q0), t(tau), out["q_stages"], t(gbar), dt, 1)
    torch.cuda.synchronize()
    qs_h = out["q_stages"].cpu().numpy()
    gp, gc, gt = gp.cpu().numpy(), gc.cpu().numpy(), gt.cpu().numpy()
    for b in np.flatnonzero(conv):
        assert st[b] == 0
        om = O.OracleModel.from_spec(spec, b, contact=contact)
        sl = slice(b * n, (b + 1) * n)
        rp, rc, rt = om.step_adjoint(1, dt, qp[b], q0[b], tau[b], qs_h[sl], gbar[sl])
        assert _relerr(gp[sl], rp) < 1e-7, b
        assert _relerr(gc[sl], rc) < 1e-7, b
        assert _relerr(gt[sl], rt) < 1e-7, b


def test_contact_needs_one_stage():
    import torch
    import paper_1709_04145_b300 as P
    spec = I.free_chain(2, 2)
    batch = P.Batch([P.Model.from_spec(spec, contact=_contact(spec))], max_stages=2, max_history=4)
    q = torch.zeros(2 * batch.D, dtype=torch.float64, device="cuda:0")
    with pytest.raises(P.PBADError):
        P.eval_objective_grad(batch, q, q[:batch.D], q[:batch.D], None, 0.02, 2)


@pytest.mark.parametrize("solver", ["lbfgs", "lm"])
def test_spider_steps_match_oracle(solver):
    """Section 6.2's spider body (free root, four legs, six ground contact
    points): the first steps of both solvers against the oracle, step by
    step from the same states; the objective never rises within a step."""
    import torch
    import paper_1709_04145_b300 as P
    w = I.spiders(count=3, n_steps=4)
    spec, dt = w["spec"], w["dt"]
    sv = P.LBFGS if solver == "lbfgs" else P.NEWTON
    mi = 500 if sv == P.LBFGS else 100
    batch = P.Batch([P.Model.from_spec(spec, drag=w["drag"], contact=w["contact"])], max_stages=1,
                    max_history=8, newton=True)
    n = spec.n_dof
    dev = torch.device("cuda:0")
    t = lambda a: torch.tensor(np.ascontiguousarray(a).reshape(-1), device=dev)
    qc = w["q0"].copy()
    qp = w["q0"] - dt * w["qd0"]
    agree = 0
    for step in range(4):
        out = P.step(batch, t(qp), t(qc), None, dt, 1, sv, 8, w["tol"], mi)
        qs = out["q_stages"].cpu().numpy().reshape(spec.count, n)
        st = out["status"].cpu().numpy()
        E0, _, _ = P.eval_objective_grad(batch, t(2 * qc - qp), t(qp), t(qc), None, dt, 1)
        E1, _, _ = P.eval_objective_grad(batch, t(qs), t(qp), t(qc), None, dt, 1)
        assert (E1.cpu().numpy() <= E0.cpu().numpy() * (1 + 1e-9) + 1e-12).all()
        for b in range(spec.count):
            om = O.OracleModel.from_spec(spec, b, drag=w["drag"], contact=w["contact"])
            q_o, st_o, _, _ = om.step(1, dt, qp[b], qc[b], np.zeros(n), solver, 8, w["tol"], mi)
            if st_o == st[b] == 0:
                assert np.max(np.abs(q_o.reshape(-1) - qs[b])) <= 1e-7, (step, b)
                agree += 1
        # continue from the oracle's states so that every step starts equal
        nxt = np.stack([O.OracleModel.from_spec(spec, b, drag=w["drag"], contact=w["contact"])
                        .step(1, dt, qp[b], qc[b], np.zeros(n), solver, 8, w["tol"], mi)[0].reshape(-1)
                        for b in range(spec.count)])
        qp, qc = qc, nxt
    assert agree >= 3
