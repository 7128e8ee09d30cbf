"""Implicit-function adjoint of converged steps and differentiable rollouts
on the CUDA path, against the oracle's dense adjoint and finite differences."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1709_04145_b300 import inputs as I

pytestmark = pytest.mark.gpu


def _relerr(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("S", [1, 2, 3])
def test_step_backward_matches_oracle(S):
    import torch

    import paper_1709_04145_b300 as P
    dev = torch.device("cuda:0")
    specs = [I.rod_chain(3, 4, name="rod4"), I.ball_chain(3, 3, seed=41, radius=0.15),
             I.humanoid(2, seed=42)]
    batch = P.Batch([P.Model.from_spec(s) for s in specs], max_stages=3, max_history=8, newton=True)
    dt = 0.02
    nodes, _ = O.colloc(S)
    rng = np.random.default_rng(5)
    states = [I.random_state(s, 50 + k, pose_scale=0.4, vel_sigma=0.3) for k, s in enumerate(specs)]
    q0 = np.concatenate([st[0].reshape(-1) for st in states])
    qd0 = np.concatenate([st[1].reshape(-1) for st in states])
    qp = q0 + nodes[0] * dt * qd0
    tau = rng.normal(0, 0.1, batch.D)
    t = lambda a: torch.tensor(a, device=dev)
    # tolerance above the FP64 floor of r (~1e-10 for three stages at this dt)
    out = P.step(batch, t(qp), t(q0), t(tau), dt, S, P.NEWTON, 8, 1e-10 if S < 3 else 1e-9, 100)
    assert (out["status"] == 0).all()
    qs = out["q_stages"]
    gbar = rng.normal(size=S * batch.D)
    gp, gc, gt, st = P.step_backward(batch, t(qp), t(q0), t(tau), qs, t(gbar), dt, S)
    torch.cuda.synchronize()
    assert (st == 0).all()
    qs_h = qs.cpu().numpy()
    gp, gc, gt = gp.cpu().numpy(), gc.cpu().numpy(), gt.cpu().numpy()
    for k, spec in enumerate(specs):
        for b in range(spec.count):
            om = O.OracleModel.from_spec(spec, b)
            a = batch.dof_off[k] + b * spec.n_dof
            sl = slice(a, a + spec.n_dof)
            ssl = slice(S * a, S * (a + spec.n_dof))
            rp, rc, rt = om.step_adjoint(S, dt, qp[sl], q0[sl], tau[sl], qs_h[ssl], gbar[ssl])
            tol = 1e-7
            assert _relerr(gp[sl], rp) < tol, (spec.name, b, _relerr(gp[sl], rp))
            assert _relerr(gc[sl], rc) < tol, (spec.name, b)
            assert _relerr(gt[sl], rt) < tol, (spec.name, b)


def _ee_problem(count=2, n_steps=6):
    spec = I.humanoid(count, seed=61)
    q0, qd0 = I.random_state(spec, 62, pose_scale=0.3, vel_sigma=0.3)
    tau = I.torques(spec, n_steps, 63, sigma=0.1)
    # end effector: tip of limb 1's last link (link 4), target in a 1 m ball
    link = 4
    tip = np.zeros((count, 3))
    tip[:, 2] = -spec.length[:, link]
    return spec, q0, qd0, tau, link, tip


def test_rollout_gradient_matches_finite_differences():
    import torch

    import paper_1709_04145_b300 as P
    from paper_1709_04145_b300.autograd import points_differentiable, rollout_differentiable
    dev = torch.device("cuda:0")
    S, dt, n_steps = 2, 0.033, 6
    spec, q0, qd0, tau, link, tip = _ee_problem(2, n_steps)
    batch = P.Batch([P.Model.from_spec(spec)], max_stages=S, max_history=8, newton=True)
    target = torch.tensor(np.random.default_rng(64).normal(0, 0.3, (spec.count, 3)), device=dev)
    tip_t = torch.tensor(tip, device=dev)
    kw = dict(dt=dt, stages=S, solver=P.NEWTON, tol=1e-10, max_iter=100, checkpoint_every=4)

    def loss(q0_, qd0_, tau_):
        qc, qp, st = rollout_differentiable(batch, q0_, qd0_, tau_, **kw)
        assert (st == 0).all()
        p = points_differentiable(batch, qc, [link], tip_t)
        return ((p - target) ** 2).sum()

    x0 = torch.tensor(q0.reshape(-1), device=dev, requires_grad=True)
    v0 = torch.tensor(qd0.reshape(-1), device=dev, requires_grad=True)
    tt = torch.tensor(tau.reshape(n_steps, -1), device=dev, requires_grad=True)
    L = loss(x0, v0, tt)
    L.backward()
    h = 1e-5
    rng = np.random.default_rng(65)
    with torch.no_grad():
        for name, var, grad in (("q0", x0, x0.grad), ("qd0", v0, v0.grad), ("tau", tt, tt.grad)):
            flat = var.view(-1)
            for idx in rng.choice(flat.numel(), size=4, replace=False):
                old = flat[idx].item()
                flat[idx] = old + h
                Lp = loss(x0, v0, tt).item()
                flat[idx] = old - h
                Lm = loss(x0, v0, tt).item()
                flat[idx] = old
                fd = (Lp - Lm) / (2 * h)
                g = grad.view(-1)[idx].item()
                assert abs(g - fd) <= 1e-4 * max(1.0, abs(fd)), (name, idx, g, fd)


def test_rollout_gradient_matches_oracle_dense_adjoint():
    """Chains the oracle's dense per-step adjoint over the same trajectory."""
    import torch

    import paper_1709_04145_b300 as P
    from paper_1709_04145_b300.autograd import rollout_differentiable
    dev = torch.device("cuda:0")
    S, dt, n_steps = 2, 0.033, 5
    spec = I.ball_chain(2, 4, seed=71, radius=0.15)
    q0, qd0 = I.random_state(spec, 72, pose_scale=0.3, vel_sigma=0.3)
    tau = I.torques(spec, n_steps, 73, sigma=0.1)
    batch = P.Batch([P.Model.from_spec(spec)], max_stages=S, max_history=8, newton=True)
    w_c = np.random.default_rng(74).normal(size=batch.D)
    x0 = torch.tensor(q0.reshape(-1), device=dev, requires_grad=True)
    v0 = torch.tensor(qd0.reshape(-1), device=dev, requires_grad=True)
    tt = torch.tensor(tau.reshape(n_steps, -1), device=dev, requires_grad=True)
    qc, qp, st = rollout_differentiable(batch, x0, v0, tt, dt, S, P.NEWTON, tol=1e-10,
                                        max_iter=100, checkpoint_every=2)
    (qc * torch.tensor(w_c, device=dev)).sum().backward()
    nodes, _ = O.colloc(S)
    n = spec.n_dof
    for b in range(spec.count):
        om = O.OracleModel.from_spec(spec, b)
        sl = slice(b * n, (b + 1) * n)
        # forward with the oracle, keeping every step's state and stages
        qprev = q0[b] + nodes[0] * dt * qd0[b]
        qcur = q0[b].copy()
        hist = []
        for t in range(n_steps):
            qs, status, *_ = om.step(S, dt, qprev, qcur, tau[t, b], "lm", 8, 1e-10, 100)
            assert status == 0
            hist.append((qprev, qcur, qs))
            qprev, qcur = qs[S - 2], qs[S - 1]
        a_cur, a_prev = w_c[sl].copy(), np.zeros(n)
        g_tau = np.zeros((n_steps, n))
        for t in range(n_steps - 1, -1, -1):
            qpv, qcv, qs = hist[t]
            gbar = np.zeros((S, n))
            gbar[S - 1] += a_cur
            gbar[S - 2] += a_prev
            gp, gc, gt = om.step_adjoint(S, dt, qpv, qcv, tau[t, b], qs, gbar)
            a_prev, a_cur = gp, gc
            g_tau[t] = gt
        assert _relerr(x0.grad[sl].cpu().numpy(), a_prev + a_cur) < 1e-6
        assert _relerr(v0.grad[sl].cpu().numpy(), nodes[0] * dt * a_prev) < 1e-6
        assert _relerr(tt.grad[:, sl].cpu().numpy(), g_tau) < 1e-6


@pytest.mark.parametrize("S", [1, 2])
def test_step_backward_large_ball_rotations(S):
    """Newton step and its adjoint with ball joints turned 1-2.6 rad (the
    closed-form branch of the exponential map and of its derivatives in
    the Jacobian columns), against the oracle's dense adjoint."""
    import torch

    import paper_1709_04145_b300 as P
    dev = torch.device("cuda:0")
    spec = I.ball_chain(6, 3, seed=43, radius=0.15)
    batch = P.Batch([P.Model.from_spec(spec)], max_stages=S, max_history=8, newton=True)
    dt = 0.01
    nodes, _ = O.colloc(S)
    rng = np.random.default_rng(6)
    B, n = spec.count, spec.n_dof
    v = rng.normal(size=(B, n // 3, 3))
    v /= np.linalg.norm(v, axis=-1, keepdims=True)
    q0 = (v * rng.uniform(1.0, 2.6, size=(B, n // 3, 1))).reshape(B, n)
    qd0 = rng.normal(0, 0.3, size=(B, n))
    qp = q0 + nodes[0] * dt * qd0
    tau = rng.normal(0, 0.1, B * n)
    t = lambda a: torch.tensor(np.ascontiguousarray(a).reshape(-1), device=dev)
    out = P.step(batch, t(qp), t(q0), t(tau), dt, S, P.NEWTON, 8, 1e-9, 100)
    st = out["status"].cpu().numpy()
    assert (st == 0).sum() >= B - 1
    qs = out["q_stages"]
    gbar = rng.normal(size=S * batch.D)
    gp, gc, gt, bst = P.step_backward(batch, t(qp), t(q0), t(tau), qs, t(gbar), dt, S)
    torch.cuda.synchronize()
    qs_h = qs.cpu().numpy()
    gp, gc, gt, bst = gp.cpu().numpy(), gc.cpu().numpy(), gt.cpu().numpy(), bst.cpu().numpy()
    qp_f, q0_f = qp.reshape(-1), q0.reshape(-1)
    checked = 0
    for b in range(B):
        if st[b] != 0:
            continue
        assert bst[b] == 0
        om = O.OracleModel.from_spec(spec, b)
        sl, ssl = slice(b * n, (b + 1) * n), slice(S * b * n, S * (b + 1) * n)
        rp, rc, rt = om.step_adjoint(S, dt, qp_f[sl], q0_f[sl], tau[sl], qs_h[ssl], gbar[ssl])
        assert _relerr(gp[sl], rp) < 1e-7, b
        assert _relerr(gc[sl], rc) < 1e-7, b
        assert _relerr(gt[sl], rt) < 1e-7, b
        checked += 1
    assert checked >= B - 1


def test_unsolved_steps_flag_their_instances_gradients():
    """A step that ends unsolved (here MAX_ITER under a one-iteration cap)
    breaks the implicit-function theorem: its instance's gradients come back
    NaN (or zero), adjoint_status names the failure, and instances whose
    steps all converged keep the gradients they get without the flag."""
    import torch

    import paper_1709_04145_b300 as P
    from paper_1709_04145_b300.autograd import rollout_differentiable
    dev = torch.device("cuda:0")
    S, dt, n_steps = 2, 0.033, 4
    spec = I.ball_chain(6, 4, seed=81, radius=0.15)
    q0, qd0 = I.random_state(spec, 82, pose_scale=0.3, vel_sigma=0.3)
    tau = I.torques(spec, n_steps, 83, sigma=0.1)
    # instances 0-2 move fast (their steps need five LM iterations), 3-5
    # slowly (four): a four-iteration cap leaves only the first three unsolved
    qd0[:3] *= 8.0
    qd0[3:] *= 0.1
    tau[:, 3:] *= 0.1
    batch = P.Batch([P.Model.from_spec(spec)], max_stages=S, max_history=8, newton=True)
    n = spec.n_dof
    grads = {}
    for mode in ("keep", "nan", "zero"):
        x0 = torch.tensor(q0.reshape(-1), device=dev, requires_grad=True)
        v0 = torch.tensor(qd0.reshape(-1), device=dev, requires_grad=True)
        tt = torch.tensor(tau.reshape(n_steps, -1), device=dev, requires_grad=True)
        adj = torch.full((spec.count,), -1, dtype=torch.int32, device=dev)
        qc, qp, st = rollout_differentiable(batch, x0, v0, tt, dt, S, P.NEWTON, tol=1e-10,
                                            max_iter=4, checkpoint_every=2, on_unsolved=mode,
                                            adjoint_status=adj)
        qc.sum().backward()
        grads[mode] = (x0.grad.cpu().numpy(), v0.grad.cpu().numpy(), tt.grad.cpu().numpy(),
                       st.cpu().numpy(), adj.cpu().numpy())
    st, adj = grads["nan"][3], grads["nan"][4]
    unsolved = ~np.isin(st, [0, 5])
    assert unsolved.any() and not unsolved.all(), st
    assert np.array_equal(unsolved, ~np.isin(adj, [0, 5])), (st, adj)
    for b in range(spec.count):
        sl = slice(b * n, (b + 1) * n)
        gk, gn, gz = grads["keep"], grads["nan"], grads["zero"]
        for k in range(3):
            blk = (lambda a: a[sl]) if k < 2 else (lambda a: a[:, sl])
            if unsolved[b]:
                assert np.all(np.isnan(blk(gn[k]))), (b, k)
                assert np.all(blk(gz[k]) == 0.0), (b, k)
                assert np.all(np.isfinite(blk(gk[k]))), (b, k)
            else:
                assert np.array_equal(blk(gn[k]), blk(gk[k])), (b, k)
                assert np.array_equal(blk(gz[k]), blk(gk[k])), (b, k)


def test_kept_stages_give_the_recomputed_gradients_bitwise(monkeypatch):
    """keep_stages=True (the forward pass keeps every step's stages, the
    backward pass recomputes nothing) gives the same gradient bits and the
    same adjoint status as recomputing each checkpoint segment, whether the
    forward pass ran as one launch or as one launch per segment, with two
    fast-moving instances unsolved under an eight-iteration cap."""
    import torch

    import paper_1709_04145_b300 as P
    from paper_1709_04145_b300 import autograd as AG
    from paper_1709_04145_b300.autograd import rollout_differentiable
    dev = torch.device("cuda:0")
    S, dt, n_steps = 2, 0.033, 7
    spec = I.humanoid(6, seed=95)
    q0, qd0 = I.random_state(spec, 96, pose_scale=0.3, vel_sigma=0.3)
    qd0[:2] *= 6.0
    tau = I.torques(spec, n_steps, 97, sigma=0.1)
    batch = P.Batch([P.Model.from_spec(spec)], max_stages=S, max_history=8, newton=True)
    w = torch.tensor(np.random.default_rng(98).normal(size=batch.D), device=dev)
    res = {}
    for keep, one_launch_bytes in ((False, AG.ONE_LAUNCH_TRAJ_BYTES), (False, 0),
                                   (True, AG.ONE_LAUNCH_TRAJ_BYTES)):
        monkeypatch.setattr(AG, "ONE_LAUNCH_TRAJ_BYTES", one_launch_bytes)
        x0 = torch.tensor(q0.reshape(-1), device=dev, requires_grad=True)
        v0 = torch.tensor(qd0.reshape(-1), device=dev, requires_grad=True)
        tt = torch.tensor(tau.reshape(n_steps, -1), device=dev, requires_grad=True)
        adj = torch.full((spec.count,), -1, dtype=torch.int32, device=dev)
        qc, qp, st = rollout_differentiable(batch, x0, v0, tt, dt, S, P.NEWTON, tol=1e-10,
                                            max_iter=8, checkpoint_every=3, on_unsolved="keep",
                                            adjoint_status=adj, keep_stages=keep)
        ((qc * w).sum() + (qp * w).sum()).backward()
        res[(keep, one_launch_bytes)] = [a.cpu().numpy() for a in
                                         (x0.grad, v0.grad, tt.grad, st, adj, qc.detach())]
    runs = list(res.values())
    for other in runs[1:]:
        for a, b in zip(runs[0], other):
            assert np.array_equal(a, b, equal_nan=True)
    st = runs[0][3]
    assert (st == 0).any() and (st != 0).any(), st  # both kinds of instance


@pytest.mark.parametrize("S", [1, 2])
def test_segment_backward_equals_chained_step_backward(S):
    """pbad_rollout_backward over a segment (one launch) gives what chaining
    pbad_step_backward step by step from the host gives."""
    import torch

    import paper_1709_04145_b300 as P
    dev = torch.device("cuda:0")
    dt, T = 0.033, 5
    spec = I.humanoid(5, seed=91)
    q0, qd0 = I.random_state(spec, 92, pose_scale=0.3, vel_sigma=0.3)
    tau = I.torques(spec, T, 93, sigma=0.1).reshape(T, -1)
    batch = P.Batch([P.Model.from_spec(spec)], max_stages=S, max_history=8, newton=True)
    nodes, _ = O.colloc(S)
    t = lambda a: torch.tensor(np.ascontiguousarray(a).reshape(-1), device=dev)
    qp0, qc0, tt = t(q0 + nodes[0] * dt * qd0), t(q0), t(tau).view(T, -1)
    # (the comparison is of two orchestrations of the same per-step adjoint:
    # it holds whether or not the steps converged)
    out = P.rollout(batch, qp0, qc0, tt.reshape(-1), T, dt, S, P.NEWTON, 8, 1e-10, 100,
                    want_stages=True)
    rng = np.random.default_rng(94)
    a_prev, a_cur = t(rng.normal(size=batch.D)), t(rng.normal(size=batch.D))
    ap, ac, gt, st = P.rollout_backward(batch, qp0, qc0, tt.reshape(-1), out["stages_traj"], T, dt,
                                        S, a_prev, a_cur)
    assert (st.cpu().numpy() == 0).all()
    # the same chain from the host, one pbad_step_backward per step
    states, qp, qc = [], qp0, qc0
    for k in range(T):
        o = P.step(batch, qp, qc, tt[k].contiguous(), dt, S, P.NEWTON, 8, 1e-10, 100)
        states.append((qp, qc, o["q_stages"]))
        qp, qc = o["q_prev"], o["q_cur"]
    n = spec.n_dof
    bp, bc = a_prev.clone(), a_cur.clone()
    gts = [None] * T
    for k in range(T - 1, -1, -1):
        qpk, qck, qs = states[k]
        gbar = torch.zeros(S * batch.D, dtype=torch.float64, device=dev)
        gv = gbar.view(spec.count, S, n)
        gv[:, S - 1, :] += bc.view(spec.count, n)
        if S >= 2:
            gv[:, S - 2, :] += bp.view(spec.count, n)
        gp_, gc_, g_, _ = P.step_backward(batch, qpk, qck, tt[k].contiguous(), qs, gbar, dt, S)
        if S == 1:
            gc_ = gc_ + bp
        bp, bc = gp_, gc_
        gts[k] = g_
    def rel(x, y):
        x, y = x.cpu().numpy(), y.cpu().numpy()
        return np.max(np.abs(x - y)) / np.max(np.abs(y))
    assert rel(ap, bp) < 1e-12 and rel(ac, bc) < 1e-12
    assert rel(gt, torch.stack(gts)) < 1e-12
