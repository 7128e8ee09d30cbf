"""CUDA path vs the CPU oracle, element by element, through the C ABI."""
import numpy as np
import pytest

import parity_bounds as PB
from oracle import oracle as O
from paper_1709_04145_b300 import inputs as I

pytestmark = pytest.mark.gpu

# Relative tolerance of single objective/gradient evaluations (FP64 on both
# sides; the CUDA path contracts to FMA and sums in another order).
REL_EVAL = 1e-10


def _torch():
    import torch
    return torch


def _pbad():
    import paper_1709_04145_b300 as P
    return P


def _relerr(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def _specs():
    return [
        I.rod_chain(5, 3, name="rod3"),
        I.ball_chain(7, 4, seed=11, radius=0.1),
        I.humanoid(3, seed=12),
        I.rod_chain(33, 7, name="rod7"),  # ragged count: spans several warps
    ]


def _random_case(spec, S, seed, dt):
    rng = np.random.default_rng(seed)
    B, n = spec.count, spec.n_dof
    q_cur = rng.uniform(-0.6, 0.6, size=(B, n))
    q_prev = q_cur + rng.normal(0, 0.02, size=(B, n))
    tau = rng.normal(0, 0.3, size=(B, n))
    qs = q_cur[:, None, :] + rng.normal(0, 0.03, size=(B, S, n))
    return q_prev, q_cur, tau, qs


@pytest.mark.parametrize("S", [1, 2, 3, 4])
def test_eval_matches_oracle(S):
    torch = _torch()
    P = _pbad()
    dt = 0.02
    specs = _specs()
    models = [P.Model.from_spec(s) for s in specs]
    batch = P.Batch(models, max_stages=5, max_history=8)
    cases = [_random_case(s, S, 100 + k, dt) for k, s in enumerate(specs)]
    dev = torch.device("cuda:0")
    cat = lambda idx: torch.tensor(np.concatenate([c[idx].reshape(-1) for c in cases]), device=dev)
    q_prev, q_cur, tau, qs = cat(0), cat(1), cat(2), cat(3)
    E, grad, resid = P.eval_objective_grad(batch, qs, q_prev, q_cur, tau, dt, S)
    torch.cuda.synchronize()
    E = E.cpu().numpy()
    grads = batch.unpack(grad.cpu().numpy(), S)
    resids = batch.unpack(resid.cpu().numpy(), S)
    for k, spec in enumerate(specs):
        qp, qc, ta, q_s = cases[k]
        for b in range(spec.count):
            om = O.OracleModel.from_spec(spec, b)
            Eo, ro, go, rb, gb = PB.oracle_eval_bounds(om, S, dt, q_s[b], qp[b], qc[b], ta[b])
            Eg = E[batch.inst_off[k] + b]
            assert abs(Eg - Eo) <= REL_EVAL * max(abs(Eo), 1.0), (spec.name, b, Eg, Eo)
            assert _relerr(resids[k][b].reshape(-1), ro) < REL_EVAL, (spec.name, b)
            assert _relerr(grads[k][b].reshape(-1), go) < REL_EVAL, (spec.name, b)
            # per element: each component to 1e-10 of itself, with an absolute
            # floor from the binary64 rounding bound of r (the largest component
            # alone would let small ones pass loosely)
            assert PB.ratio(resids[k][b], ro, rb) <= 1.0, (spec.name, b)
            assert PB.ratio(grads[k][b], go, gb) <= 1.0, (spec.name, b)


def test_eval_without_tau_and_single_instance():
    torch = _torch()
    P = _pbad()
    spec = I.rod_chain(1, 1, name="rod1")
    batch = P.Batch([P.Model.from_spec(spec)], max_stages=2, max_history=0)
    dev = torch.device("cuda:0")
    q = torch.tensor([0.3], dtype=torch.float64, device=dev)
    qs = torch.tensor([0.31, 0.33], dtype=torch.float64, device=dev)
    E, grad, resid = P.eval_objective_grad(batch, qs, q - 0.01, q, None, 0.05, 2)
    om = O.OracleModel.from_spec(spec, 0)
    Eo, ro, go, _ = om.eval(2, 0.05, [0.31, 0.33], [0.29], [0.3], [0.0], True)
    assert abs(E.item() - Eo) <= REL_EVAL * abs(Eo)
    assert _relerr(grad.cpu().numpy(), go) < REL_EVAL
    assert _relerr(resid.cpu().numpy(), ro) < REL_EVAL


def test_pendulum_rollout_matches_oracle():
    """3-link planar rod pendulum, dt = 0.01, one stage, L-BFGS history 5,
    |grad| < 1e-10, 200 steps: max |dq| <= 1e-7 rad over the trajectory."""
    torch = _torch()
    P = _pbad()
    w = I.pendulum3()
    spec = w["spec"]
    batch = P.Batch([P.Model.from_spec(spec)], max_stages=1, max_history=5)
    dev = torch.device("cuda:0")
    q0 = torch.tensor(w["q0"].reshape(-1), device=dev)
    out = P.rollout(batch, q0, q0, None, w["n_steps"], w["dt"], 1, P.LBFGS, 5, w["tol"], 1000)
    torch.cuda.synchronize()
    om = O.OracleModel.from_spec(spec, 0)
    ref = om.rollout(1, w["dt"], w["q0"][0], w["q0"][0], np.zeros((w["n_steps"], 3)), "lbfgs", 5,
                     w["tol"], 1000)
    assert ref["status"] == 0
    assert int(out["status"][0]) == 0
    dq = np.max(np.abs(out["traj_cur"].cpu().numpy() - ref["traj_cur"]))
    assert dq <= 1e-7, dq


@pytest.mark.parametrize("S", [1, 2, 3])
def test_rollout_matches_oracle_chains(S):
    """Hinge and ball chains with torques, L-BFGS, several steps."""
    torch = _torch()
    P = _pbad()
    dt = 0.01
    n_steps = 6
    specs = [I.rod_chain(3, 4, name="rod4"), I.ball_chain(2, 3, seed=21, radius=0.2)]
    models = [P.Model.from_spec(s) for s in specs]
    batch = P.Batch(models, max_stages=3, max_history=8)
    states = [I.random_state(s, 30 + k, pose_scale=0.4, vel_sigma=0.3) for k, s in enumerate(specs)]
    taus = [I.torques(s, n_steps, 40 + k, sigma=0.1) for k, s in enumerate(specs)]
    nodes, _ = O.colloc(S)
    qps = [q0 + nodes[0] * dt * qd0 for q0, qd0 in states]
    dev = torch.device("cuda:0")
    q_cur = torch.tensor(np.concatenate([q0.reshape(-1) for q0, _ in states]), device=dev)
    q_prev = torch.tensor(np.concatenate([qp.reshape(-1) for qp in qps]), device=dev)
    tau = torch.tensor(np.concatenate([t.reshape(n_steps, -1) for t in taus], axis=1).reshape(-1),
                       device=dev)
    tol = 1e-9
    out = P.rollout(batch, q_prev, q_cur, tau, n_steps, dt, S, P.LBFGS, 8, tol, 2000)
    torch.cuda.synchronize()
    traj = out["traj_cur"].cpu().numpy()
    st = out["status"].cpu().numpy()
    for k, spec in enumerate(specs):
        for b in range(spec.count):
            om = O.OracleModel.from_spec(spec, b)
            ref = om.rollout(S, dt, qps[k][b], states[k][0][b], taus[k][:, b, :], "lbfgs", 8, tol, 2000)
            a = batch.dof_off[k] + b * spec.n_dof
            got = traj[:, a:a + spec.n_dof]
            assert ref["status"] == st[batch.inst_off[k] + b]
            if ref["status"] == 0:
                assert np.max(np.abs(got - ref["traj_cur"])) <= 1e-7, (spec.name, b)


def _rollout_case(specs, S, dt, n_steps, seed, pose=0.4, vel=0.3, sigma=0.1):
    states = [I.random_state(s, seed + k, pose_scale=pose, vel_sigma=vel) for k, s in enumerate(specs)]
    taus = [I.torques(s, n_steps, seed + 50 + k, sigma=sigma) for k, s in enumerate(specs)]
    nodes, _ = O.colloc(S)
    qps = [q0 + nodes[0] * dt * qd0 for q0, qd0 in states]
    return states, taus, qps


def _check_rollout(batch, specs, solvers, S, dt, n_steps, tol, max_iter, seed, dq_tol=1e-7, **kw):
    torch = _torch()
    P = _pbad()
    states, taus, qps = _rollout_case(specs, S, dt, n_steps, seed, **kw)
    dev = torch.device("cuda:0")
    q_cur = torch.tensor(np.concatenate([q0.reshape(-1) for q0, _ in states]), device=dev)
    q_prev = torch.tensor(np.concatenate([qp.reshape(-1) for qp in qps]), device=dev)
    tau = torch.tensor(np.concatenate([t.reshape(n_steps, -1) for t in taus], axis=1).reshape(-1),
                       device=dev)
    out = P.rollout(batch, q_prev, q_cur, tau, n_steps, dt, S, solvers, 8, tol, max_iter)
    torch.cuda.synchronize()
    traj = out["traj_cur"].cpu().numpy()
    st = out["status"].cpu().numpy()
    it = out["iters"].cpu().numpy()
    n_conv = 0
    for k, spec in enumerate(specs):
        name = "lbfgs" if solvers[k] == P.LBFGS else "lm"
        for b in range(spec.count):
            om = O.OracleModel.from_spec(spec, b)
            ref = om.rollout(S, dt, qps[k][b], states[k][0][b], taus[k][:, b, :], name, 8, tol,
                             max_iter)
            a = batch.dof_off[k] + b * spec.n_dof
            got = traj[:, a:a + spec.n_dof]
            assert ref["status"] == st[batch.inst_off[k] + b], (spec.name, b)
            if ref["status"] == 0:
                n_conv += 1
                assert np.max(np.abs(got - ref["traj_cur"])) <= dq_tol, (spec.name, b)
                if name == "lm":  # Newton: the same iterations, up to one per step at the tol
                    assert abs(ref["iters"] - it[batch.inst_off[k] + b]) <= n_steps, (spec.name, b)
    return n_conv


@pytest.mark.parametrize("S", [1, 2, 3])
def test_newton_rollout_matches_oracle(S):
    P = _pbad()
    specs = [I.rod_chain(3, 5, name="rod5"), I.ball_chain(4, 3, seed=23, radius=0.15),
             I.humanoid(2, seed=24)]
    batch = P.Batch([P.Model.from_spec(s) for s in specs], max_stages=3, max_history=8, newton=True)
    n_conv = _check_rollout(batch, specs, [P.NEWTON] * 3, S, 0.02, 5, 1e-9, 100, 300)
    assert n_conv >= 7


def test_uneven_batch_mixed_solvers_one_launch():
    """Trees on Newton, long and short hinge chains on L-BFGS, one launch."""
    P = _pbad()
    specs = [I.humanoid(3, seed=31), I.rod_chain(2, 12, name="rod12"), I.rod_chain(37, 3, name="rod3")]
    batch = P.Batch([P.Model.from_spec(s) for s in specs], max_stages=2, max_history=8, newton=True)
    n_conv = _check_rollout(batch, specs, [P.NEWTON, P.LBFGS, P.LBFGS], 2, 0.01, 4, 1e-9, 3000, 400,
                            sigma=0.1)
    assert n_conv >= 30


def test_newton_status_codes():
    """tol = 0 with one iteration forces MAX_ITER; NaN torques give NONFINITE."""
    torch = _torch()
    P = _pbad()
    spec = I.rod_chain(2, 3, name="rod3")
    batch = P.Batch([P.Model.from_spec(spec)], max_stages=2, max_history=8, newton=True)
    dev = torch.device("cuda:0")
    q = torch.tensor(np.tile([0.3, -0.2, 0.1], 2), device=dev)
    out = P.rollout(batch, q, q, None, 2, 0.02, 2, P.NEWTON, 8, 0.0, 1)
    assert out["status"].cpu().tolist() == [1, 1]
    tau = torch.full((2 * 6,), float("nan"), dtype=torch.float64, device=dev)
    out = P.rollout(batch, q, q, tau, 2, 0.02, 2, P.NEWTON, 8, 1e-9, 50)
    assert out["status"].cpu().tolist() == [4, 4]
    out = P.rollout(batch, q, q, tau, 2, 0.02, 2, P.LBFGS, 8, 1e-9, 50)
    assert out["status"].cpu().tolist() == [4, 4]


@pytest.mark.parametrize("S", [1, 2, 3])
def test_rollout_gradient_evaluation_counts(S):
    """L-BFGS forms dE/dq at a step's first point, at every accepted trial and
    where the approximate-Wolfe test reads it, and nowhere else: n_steps +
    iterations <= gradient evaluations <= evaluations. Newton forms Jr at a
    step's start and after every accepted iteration that does not end the
    step. (The parity tests above check that the trajectories are the ones
    the oracle's every-trial gradients give.)"""
    torch = _torch()
    P = _pbad()
    specs = [I.ball_chain(5, 4, seed=91, radius=0.15), I.rod_chain(6, 5, name="rod5")]
    batch = P.Batch([P.Model.from_spec(s) for s in specs], max_stages=3, max_history=8, newton=True)
    n_steps, dt = 4, 0.02
    states, taus, qps = _rollout_case(specs, S, dt, n_steps, 92)
    dev = torch.device("cuda:0")
    q_cur = torch.tensor(np.concatenate([q0.reshape(-1) for q0, _ in states]), device=dev)
    q_prev = torch.tensor(np.concatenate([qp.reshape(-1) for qp in qps]), device=dev)
    for sv in (P.LBFGS, P.NEWTON):
        out = P.rollout(batch, q_prev, q_cur, None, n_steps, dt, S, sv, 8, 1e-9, 60)
        ev = out["evals"].cpu().numpy()
        gr = out["grads"].cpu().numpy()
        it = out["iters"].cpu().numpy()
        assert (gr <= ev).all()
        if sv == P.LBFGS:
            assert (gr >= n_steps + it).all()
            if S >= 2:  # line searches that end in LS_FAIL reject on E alone
                assert gr.sum() < ev.sum()
        else:  # one build per step start and per accepted iteration, less the last
            assert (np.abs(gr - it) <= n_steps).all()


def _large_rotations(B, n, S, rng):
    """Ball-joint exp-map vectors with |theta| in [1, 2.6]: the closed-form
    branch of the exponential map's coefficients (|theta|^2 >= 1)."""
    def draw(shape):
        v = rng.normal(size=shape + (3,))
        v /= np.linalg.norm(v, axis=-1, keepdims=True)
        return (v * rng.uniform(1.0, 2.6, size=shape + (1,))).reshape(shape[:-1] + (n,))
    q_cur = draw((B, n // 3))
    q_prev = q_cur + rng.normal(0, 0.02, size=(B, n))
    qs = q_cur[:, None, :] + rng.normal(0, 0.03, size=(B, S, n))
    return q_prev, q_cur, qs


@pytest.mark.parametrize("S", [1, 2, 3])
def test_eval_large_ball_rotations(S):
    """E, r and dE/dq at rotations of 1-2.6 rad per ball joint (the series
    covers |theta| < 1 on the GPU), against the oracle's own exp map."""
    torch = _torch()
    P = _pbad()
    spec = I.ball_chain(9, 4, seed=13, radius=0.12)
    batch = P.Batch([P.Model.from_spec(spec)], max_stages=S, max_history=8)
    rng = np.random.default_rng(14)
    B, n, dt = spec.count, spec.n_dof, 0.02
    q_prev, q_cur, qs = _large_rotations(B, n, S, rng)
    tau = rng.normal(0, 0.3, size=(B, n))
    dev = torch.device("cuda:0")
    t = lambda a: torch.tensor(np.ascontiguousarray(a).reshape(-1), device=dev)
    E, grad, resid = P.eval_objective_grad(batch, t(qs), t(q_prev), t(q_cur), t(tau), dt, S)
    torch.cuda.synchronize()
    E, grad, resid = E.cpu().numpy(), grad.cpu().numpy(), resid.cpu().numpy()
    for b in range(B):
        om = O.OracleModel.from_spec(spec, b)
        Eo, ro, go, _ = om.eval(S, dt, qs[b].reshape(-1), q_prev[b], q_cur[b], tau[b], True)
        sl = slice(b * S * n, (b + 1) * S * n)
        assert abs(E[b] - Eo) <= REL_EVAL * max(abs(Eo), 1.0), b
        assert _relerr(resid[sl], ro) < REL_EVAL, b
        assert _relerr(grad[sl], go) < REL_EVAL, b


def _general_moments(count, N, rng):
    """Mass moments of a few point masses per link off the frame's z axis:
    full symmetric Sigma and an off-axis centroid (not axially symmetric)."""
    mm = np.zeros((count, N, 10))
    for b in range(count):
        for l in range(N):
            M = np.zeros((4, 4))
            for _ in range(4):
                p = np.append(rng.normal(0, 0.2, 3) + [0, 0, -0.4], 1.0)
                M += rng.uniform(0.1, 0.5) * np.outer(p, p)
            mm[b, l] = [M[0, 0], M[0, 1], M[0, 2], M[1, 1], M[1, 2], M[2, 2], M[0, 3], M[1, 3],
                        M[2, 3], M[3, 3]]
    return mm


@pytest.mark.parametrize("S", [1, 2, 3])
def test_eval_general_mass_moments(S):
    """Links that are not symmetric about their z axis take the general mass
    product; E, r and dE/dq against the oracle."""
    torch = _torch()
    P = _pbad()
    spec = I.ball_chain(7, 3, seed=15, radius=0.1)
    rng = np.random.default_rng(16)
    B, N, n, dt = spec.count, spec.n_links, spec.n_dof, 0.02
    mm = _general_moments(B, N, rng)
    rest = np.stack([O.rest_from_spec(spec, b) for b in range(B)])
    model = P.Model(spec.parent, spec.jtype, spec.axis, mm, rest, spec.gravity)
    batch = P.Batch([model], max_stages=S, max_history=8)
    q_prev, q_cur, tau, qs = _random_case(spec, S, 17, dt)
    dev = torch.device("cuda:0")
    t = lambda a: torch.tensor(np.ascontiguousarray(a).reshape(-1), device=dev)
    E, grad, resid = P.eval_objective_grad(batch, t(qs), t(q_prev), t(q_cur), t(tau), dt, S)
    torch.cuda.synchronize()
    E, grad, resid = E.cpu().numpy(), grad.cpu().numpy(), resid.cpu().numpy()
    for b in range(B):
        om = O.OracleModel(spec.parent, spec.jtype, spec.axis, mm[b], rest[b], spec.gravity)
        Eo, ro, go, _ = om.eval(S, dt, qs[b].reshape(-1), q_prev[b], q_cur[b], tau[b], True)
        sl = slice(b * S * n, (b + 1) * S * n)
        assert abs(E[b] - Eo) <= REL_EVAL * max(abs(Eo), 1.0), b
        assert _relerr(resid[sl], ro) < REL_EVAL, b
        assert _relerr(grad[sl], go) < REL_EVAL, b


@pytest.mark.parametrize("S", [1, 2, 3])
def test_eval_rotations_straddling_the_series_switch(S):
    """E, r and dE/dq (residual and tangent passes, both mappings) with every
    ball joint's |theta| within 1e-6 .. 1e-2 of 1 rad on either side: the
    kernels switch from the power series of the exponential map's
    coefficients to their closed forms at |theta|^2 = 1, and both branches
    must give the oracle's values (its own switch sits at |theta| = 0.5)."""
    torch = _torch()
    P = _pbad()
    spec = I.ball_chain(10, 4, seed=17, radius=0.12)
    batch = P.Batch([P.Model.from_spec(spec)], max_stages=S, max_history=8)
    rng = np.random.default_rng(18)
    B, n, dt = spec.count, spec.n_dof, 0.02

    def near_one(shape):
        v = rng.normal(size=shape + (3,))
        v /= np.linalg.norm(v, axis=-1, keepdims=True)
        mag = 1.0 + rng.choice([-1.0, 1.0], size=shape + (1,)) * 10.0 ** rng.uniform(-6, -2, size=shape + (1,))
        return (v * mag).reshape(shape[:-1] + (-1,))

    q_cur = near_one((B, n // 3))
    q_prev = near_one((B, n // 3))
    qs = near_one((B, S, n // 3))
    tau = rng.normal(0, 0.3, size=(B, n))
    dev = torch.device("cuda:0")
    t = lambda a: torch.tensor(np.ascontiguousarray(a).reshape(-1), device=dev)
    for mapping in (P.MAP_STAGE, P.MAP_LINK):
        batch.set_mapping(mapping)
        E, grad, resid = P.eval_objective_grad(batch, t(qs), t(q_prev), t(q_cur), t(tau), dt, S)
        E, grad, resid = E.cpu().numpy(), grad.cpu().numpy(), resid.cpu().numpy()
        for b in range(B):
            om = O.OracleModel.from_spec(spec, b)
            Eo, ro, go, _ = om.eval(S, dt, qs[b].reshape(-1), q_prev[b], q_cur[b], tau[b], True)
            sl = slice(b * S * n, (b + 1) * S * n)
            assert abs(E[b] - Eo) <= REL_EVAL * max(abs(Eo), 1.0), (mapping, b)
            assert _relerr(resid[sl], ro) < REL_EVAL, (mapping, b)
            assert _relerr(grad[sl], go) < REL_EVAL, (mapping, b)
