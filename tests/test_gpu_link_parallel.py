"""The link-parallel mapping (one lane per stage and link, PBAD_MAP_LINK)
against the CPU oracle, element by element through the C ABI: evaluations,
L-BFGS rollouts, the largest group (S N = 32 lanes), ragged instance counts,
several groups per warp, and the requests it does not serve."""
import numpy as np
import pytest

import parity_bounds as PB
from oracle import oracle as O
from paper_1709_04145_b300 import inputs as I

pytestmark = pytest.mark.gpu

REL_EVAL = 1e-10  # evaluation parity (FP64 both sides, sums in other orders)


def _relerr(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def _case(spec, S, seed):
    rng = np.random.default_rng(seed)
    B, n = spec.count, spec.n_dof
    q_cur = rng.uniform(-0.6, 0.6, size=(B, n))
    q_prev = q_cur + rng.normal(0, 0.02, size=(B, n))
    tau = rng.normal(0, 0.3, size=(B, n))
    qs = q_cur[:, None, :] + rng.normal(0, 0.03, size=(B, S, n))
    return q_prev, q_cur, tau, qs


def _eval_both(specs, S, dt, seed):
    import torch

    import paper_1709_04145_b300 as P
    dev = torch.device("cuda:0")
    batch = P.Batch([P.Model.from_spec(s) for s in specs], max_stages=5, max_history=8)
    cases = [_case(s, S, seed + k) for k, s in enumerate(specs)]
    cat = lambda idx: torch.tensor(np.concatenate([c[idx].reshape(-1) for c in cases]), device=dev)
    args = (cat(3), cat(0), cat(1), cat(2), dt, S)
    res = {}
    for mp in (P.MAP_STAGE, P.MAP_LINK):
        batch.set_mapping(mp)
        E, g, r = P.eval_objective_grad(batch, *args)
        res[mp] = (E.cpu().numpy(), batch.unpack(g.cpu().numpy(), S), batch.unpack(r.cpu().numpy(), S))
    return batch, cases, res


@pytest.mark.parametrize("S", [1, 2, 3, 4])
def test_link_parallel_eval_matches_oracle(S):
    import paper_1709_04145_b300 as P
    dt = 0.02
    specs = [I.rod_chain(5, 3, name="rod3"), I.ball_chain(7, 4, seed=11, radius=0.1),
             I.rod_chain(33, 7, name="rod7"),  # ragged count: several warps
             I.rod_chain(3, 1, name="rod1")]
    batch, cases, res = _eval_both(specs, S, dt, 100)
    E, grads, resids = res[P.MAP_LINK]
    Es, grads_s, _ = res[P.MAP_STAGE]
    for k, spec in enumerate(specs):
        qp, qc, ta, q_s = cases[k]
        for b in range(spec.count):
            om = O.OracleModel.from_spec(spec, b)
            Eo, ro, go, rb, gb = PB.oracle_eval_bounds(om, S, dt, q_s[b], qp[b], qc[b], ta[b])
            Eg = E[batch.inst_off[k] + b]
            assert abs(Eg - Eo) <= REL_EVAL * max(abs(Eo), 1.0), (spec.name, b, Eg, Eo)
            assert _relerr(resids[k][b].reshape(-1), ro) < REL_EVAL, (spec.name, b)
            assert _relerr(grads[k][b].reshape(-1), go) < REL_EVAL, (spec.name, b)
            # per element, with the floor from the rounding bound of r
            assert PB.ratio(resids[k][b], ro, rb) <= 1.0, (spec.name, b)
            assert PB.ratio(grads[k][b], go, gb) <= 1.0, (spec.name, b)
            # and the two mappings agree to rounding
            assert _relerr(grads[k][b], grads_s[k][b]) < REL_EVAL, (spec.name, b)


@pytest.mark.parametrize("S,N", [(4, 8), (3, 10), (2, 16), (1, 32)])
def test_link_parallel_eval_full_warp_groups(S, N):
    """Groups of exactly 30-32 lanes (one instance per warp), ball joints."""
    import paper_1709_04145_b300 as P
    dt = 0.033
    specs = [I.ball_chain(5, N, seed=40 + N, radius=0.15)]
    batch, cases, res = _eval_both(specs, S, dt, 200 + S)
    E, grads, resids = res[P.MAP_LINK]
    qp, qc, ta, q_s = cases[0]
    for b in range(specs[0].count):
        om = O.OracleModel.from_spec(specs[0], b)
        Eo, ro, go, rb, gb = PB.oracle_eval_bounds(om, S, dt, q_s[b], qp[b], qc[b], ta[b])
        assert abs(E[b] - Eo) <= REL_EVAL * max(abs(Eo), 1.0), (b, E[b], Eo)
        assert _relerr(resids[0][b].reshape(-1), ro) < REL_EVAL, b
        assert _relerr(grads[0][b].reshape(-1), go) < REL_EVAL, b
        assert PB.ratio(resids[0][b], ro, rb) <= 1.0, b
        assert PB.ratio(grads[0][b], go, gb) <= 1.0, b


def test_link_parallel_eval_free_root_chain():
    """Translation joint at the root (the free 6-DOF root), two stages."""
    import paper_1709_04145_b300 as P
    w = I.swimmers_free(count=9, n_steps=1)
    spec = w["spec"]
    assert spec.jtype[0] == I.TRANSLATION
    batch, cases, res = _eval_both([spec], 2, 0.05, 300)
    E, grads, resids = res[P.MAP_LINK]
    qp, qc, ta, q_s = cases[0]
    for b in range(spec.count):
        om = O.OracleModel.from_spec(spec, b)
        Eo, ro, go, _ = om.eval(2, 0.05, q_s[b], qp[b], qc[b], ta[b], True)
        assert abs(E[b] - Eo) <= REL_EVAL * max(abs(Eo), 1.0), b
        assert _relerr(grads[0][b].reshape(-1), go) < REL_EVAL, b


def test_link_parallel_pendulum_rollout_matches_oracle():
    """The plain-method pendulum (3 rods, dt = 0.01, one stage, L-BFGS m = 5,
    |r| < 1e-10, 200 steps): max |dq| <= 1e-7 rad, every step's status."""
    import torch

    import paper_1709_04145_b300 as P
    w = I.pendulum3()
    spec = w["spec"]
    batch = P.Batch([P.Model.from_spec(spec)], max_stages=1, max_history=5)
    batch.set_mapping(P.MAP_LINK)
    dev = torch.device("cuda:0")
    q0 = torch.tensor(w["q0"].reshape(-1), device=dev)
    out = P.rollout(batch, q0, q0, None, w["n_steps"], w["dt"], 1, P.LBFGS, 5, w["tol"], 1000)
    om = O.OracleModel.from_spec(spec, 0)
    ref = om.rollout(1, w["dt"], w["q0"][0], w["q0"][0], np.zeros((w["n_steps"], 3)), "lbfgs", 5,
                     w["tol"], 1000)
    assert ref["status"] == 0 and int(out["status"][0]) == 0
    assert np.array_equal(out["step_status"].cpu().numpy()[:, 0], ref["step_status"])
    dq = np.max(np.abs(out["traj_cur"].cpu().numpy() - ref["traj_cur"]))
    assert dq <= 1e-7, dq


@pytest.mark.parametrize("S", [1, 2, 3])
def test_link_parallel_rollout_matches_oracle(S):
    """Hinge and ball chains with torques, L-BFGS, six steps; several
    instances per warp for the short chains."""
    import torch

    import paper_1709_04145_b300 as P
    dt, n_steps, tol = 0.01, 6, 1e-9
    specs = [I.rod_chain(7, 4, name="rod4"), I.ball_chain(3, 3, seed=21, radius=0.2)]
    batch = P.Batch([P.Model.from_spec(s) for s in specs], max_stages=3, max_history=8)
    batch.set_mapping(P.MAP_LINK)
    states = [I.random_state(s, 30 + k, pose_scale=0.4, vel_sigma=0.3) for k, s in enumerate(specs)]
    taus = [I.torques(s, n_steps, 40 + k, sigma=0.1) for k, s in enumerate(specs)]
    nodes, _ = O.colloc(S)
    qps = [q0 + nodes[0] * dt * qd0 for q0, qd0 in states]
    dev = torch.device("cuda:0")
    q_cur = torch.tensor(np.concatenate([q0.reshape(-1) for q0, _ in states]), device=dev)
    q_prev = torch.tensor(np.concatenate([qp.reshape(-1) for qp in qps]), device=dev)
    tau = torch.tensor(np.concatenate([t.reshape(n_steps, -1) for t in taus], axis=1).reshape(-1),
                       device=dev)
    out = P.rollout(batch, q_prev, q_cur, tau, n_steps, dt, S, P.LBFGS, 8, tol, 2000)
    traj = out["traj_cur"].cpu().numpy()
    st = out["status"].cpu().numpy()
    sst = out["step_status"].cpu().numpy()
    for k, spec in enumerate(specs):
        for b in range(spec.count):
            om = O.OracleModel.from_spec(spec, b)
            ref = om.rollout(S, dt, qps[k][b], states[k][0][b], taus[k][:, b, :], "lbfgs", 8, tol,
                             2000)
            g = int(batch.inst_off[k]) + b
            a = int(batch.dof_off[k]) + b * spec.n_dof
            # the worst status agrees; every step's status and the trajectory
            # where the oracle converged every step (the iterates of an
            # unconverged L-BFGS step decorrelate at the rounding level)
            assert ref["status"] == st[g], (spec.name, b)
            if ref["status"] == 0:
                assert np.array_equal(sst[:, g], ref["step_status"]), (spec.name, b)
                assert np.max(np.abs(traj[:, a:a + spec.n_dof] - ref["traj_cur"])) <= 1e-7, (spec.name, b)


def test_link_parallel_step_outputs_stages():
    """pbad_step through the link mapping returns the same stages as the
    stage mapping (to the solver tolerance), one stage, where L-BFGS
    converges."""
    import torch

    import paper_1709_04145_b300 as P
    S, dt = 1, 0.01
    spec = I.ball_chain(11, 5, seed=5, radius=0.2)
    q0, qd0 = I.random_state(spec, 6, pose_scale=0.3, vel_sigma=0.3)
    nodes, _ = O.colloc(S)
    dev = torch.device("cuda:0")
    qp = torch.tensor((q0 + nodes[0] * dt * qd0).reshape(-1), device=dev)
    qc = torch.tensor(q0.reshape(-1), device=dev)
    batch = P.Batch([P.Model.from_spec(spec)], max_stages=S, max_history=8)
    res = {}
    for mp in (P.MAP_STAGE, P.MAP_LINK):
        batch.set_mapping(mp)
        res[mp] = P.step(batch, qp, qc, None, dt, S, P.LBFGS, 8, 1e-9, 2000)
    sa = res[P.MAP_STAGE]["status"].cpu().numpy()
    sb = res[P.MAP_LINK]["status"].cpu().numpy()
    both = (sa == 0) & (sb == 0)
    assert both.sum() >= spec.count // 2, (sa, sb)
    n = spec.n_dof
    for key, w in (("q_stages", S * n), ("q_prev", n), ("q_cur", n)):
        a = res[P.MAP_STAGE][key].cpu().numpy().reshape(spec.count, w)[both]
        b = res[P.MAP_LINK][key].cpu().numpy().reshape(spec.count, w)[both]
        assert np.max(np.abs(a - b)) <= 1e-8, key


def test_link_parallel_rejects_what_it_does_not_serve():
    import torch

    import paper_1709_04145_b300 as P
    dev = torch.device("cuda:0")
    cases = [
        ([I.humanoid(2, seed=3)], 2, P.LBFGS),                 # a tree
        ([I.rod_chain(2, 17, name="rod17")], 2, P.LBFGS),      # 34 lanes per instance
        ([I.rod_chain(2, 4, name="rod4")], 2, P.NEWTON),       # Newton
        ([I.rod_chain(2, 4, name="rod4")], 2, P.LBFGS_F32),    # binary32 direction
    ]
    for specs, S, sv in cases:
        batch = P.Batch([P.Model.from_spec(s) for s in specs], max_stages=S, max_history=8,
                        newton=True)
        batch.set_mapping(P.MAP_LINK)
        q = torch.zeros(batch.D, dtype=torch.float64, device=dev)
        with pytest.raises(P.PBADError, match="UNSUPPORTED"):
            P.rollout(batch, q, q, None, 1, 0.01, S, sv, 8, 1e-8, 10)
    # one stage with drag is left to the stage mapping
    spec = I.rod_chain(2, 4, name="rod4")
    batch = P.Batch([P.Model.from_spec(spec, drag=0.3)], max_stages=1, max_history=8)
    batch.set_mapping(P.MAP_LINK)
    q = torch.zeros(batch.D, dtype=torch.float64, device=dev)
    with pytest.raises(P.PBADError, match="UNSUPPORTED"):
        P.eval_objective_grad(batch, q, q, q, None, 0.01, 1)
    with pytest.raises(P.PBADError, match="ARG"):
        batch.set_mapping(7)


def test_link_parallel_full_size_ball_chains():
    """The batched workload's 4096 ten-link ball chains (three stages, 30
    lanes per instance): evaluation parity on sampled instances, and two
    rollout steps whose per-step statuses and exit |r| follow the stage
    mapping's."""
    import torch

    import paper_1709_04145_b300 as P
    w = I.ball_chains(count=4096, n_links=10, n_steps=2)
    spec, S, dt = w["spec"], w["stages"], w["dt"]
    dev = torch.device("cuda:0")
    batch = P.Batch([P.Model.from_spec(spec)], max_stages=S, max_history=8)
    nodes, _ = O.colloc(S)
    qp_h = w["q0"] + nodes[0] * dt * w["qd0"]
    rng = np.random.default_rng(7)
    qs_h = w["q0"][:, None, :] + rng.normal(0, 0.02, (spec.count, S, spec.n_dof))
    t = lambda a: torch.tensor(np.ascontiguousarray(a).reshape(-1), device=dev)
    batch.set_mapping(P.MAP_LINK)
    E, g, r = P.eval_objective_grad(batch, t(qs_h), t(qp_h), t(w["q0"]), None, dt, S)
    E, g = E.cpu().numpy(), g.cpu().numpy().reshape(spec.count, S * spec.n_dof)
    for b in np.linspace(0, spec.count - 1, 12).astype(int):
        om = O.OracleModel.from_spec(spec, int(b))
        Eo, _, go, _, gb = PB.oracle_eval_bounds(om, S, dt, qs_h[b], qp_h[b], w["q0"][b],
                                                 np.zeros(spec.n_dof))
        assert abs(E[b] - Eo) <= REL_EVAL * abs(Eo), b
        assert _relerr(g[b], go) < REL_EVAL, b
        assert PB.ratio(g[b], go, gb) <= 1.0, b
    outs = {}
    for mp in (P.MAP_STAGE, P.MAP_LINK):
        batch.set_mapping(mp)
        outs[mp] = P.rollout(batch, t(qp_h), t(w["q0"]), None, 2, dt, S, P.LBFGS, 8, w["tol"], 3)
    sa = outs[P.MAP_STAGE]["step_status"].cpu().numpy()
    sb = outs[P.MAP_LINK]["step_status"].cpu().numpy()
    ra = outs[P.MAP_STAGE]["step_rnorm"].cpu().numpy()
    rb = outs[P.MAP_LINK]["step_rnorm"].cpu().numpy()
    # three-iteration steps: the same decisions on almost every instance,
    # and the same exit residual to a relative 1e-6 where they agree
    same = sa[0] == sb[0]
    assert same.mean() > 0.99, same.mean()
    close = np.abs(ra[0] - rb[0]) <= 1e-6 * np.abs(ra[0])
    assert close[same].mean() > 0.99
