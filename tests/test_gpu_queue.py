"""Instance queue of the L-BFGS rollouts (pbad_batch_set_queue): with the
launch capped at a few blocks, groups that finish an instance take the next
one from the bucket's counter. Every instance's results are bitwise the ones
of the launch without a queue (one group per instance from the start), and
instances handed out by the queue match the oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1709_04145_b300 import inputs as I

pytestmark = pytest.mark.gpu

KEYS = ("traj_prev", "traj_cur", "q_prev", "q_cur", "status", "iters", "evals", "grads")


def _inputs(specs, S, dt, n_steps, seed):
    import torch
    states = [I.random_state(s, seed + k, pose_scale=0.4, vel_sigma=0.3) for k, s in enumerate(specs)]
    taus = [I.torques(s, n_steps, seed + 50 + k, sigma=0.1) for k, s in enumerate(specs)]
    nodes, _ = O.colloc(S)
    qps = [q0 + nodes[0] * dt * qd0 for q0, qd0 in states]
    dev = torch.device("cuda:0")
    q_cur = torch.tensor(np.concatenate([q0.reshape(-1) for q0, _ in states]), device=dev)
    q_prev = torch.tensor(np.concatenate([qp.reshape(-1) for qp in qps]), device=dev)
    tau = torch.tensor(np.concatenate([t.reshape(n_steps, -1) for t in taus], axis=1).reshape(-1),
                       device=dev)
    return states, taus, qps, q_prev, q_cur, tau


def _run(P, batch, q_prev, q_cur, tau, n_steps, dt, S, solvers, max_blocks, max_iter):
    import torch
    batch.set_queue(max_blocks)
    out = P.rollout(batch, q_prev, q_cur, tau, n_steps, dt, S, solvers, 8, 1e-9, max_iter)
    torch.cuda.synchronize()
    return {k: out[k].cpu().numpy() for k in KEYS}


def _assert_same(a, b):
    for k in KEYS:
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("S", [1, 2, 3])
def test_queue_bitwise_equals_static_assignment(S):
    import paper_1709_04145_b300 as P
    specs = [I.rod_chain(300, 3, name="rod3"), I.ball_chain(150, 2, seed=71, radius=0.2)]
    batch = P.Batch([P.Model.from_spec(s) for s in specs], max_stages=3, max_history=8)
    n_steps, dt = 3, 0.02
    _, _, _, qp, qc, tau = _inputs(specs, S, dt, n_steps, 700)
    ref = _run(P, batch, qp, qc, tau, n_steps, dt, S, P.LBFGS, -1, 200)
    for cap in (2, 5):  # one and a few blocks per bucket
        got = _run(P, batch, qp, qc, tau, n_steps, dt, S, P.LBFGS, cap, 200)
        _assert_same(got, ref)


def test_queue_with_binary32_direction_buckets():
    """Two buckets on the binary32-direction L-BFGS share the capped blocks."""
    import paper_1709_04145_b300 as P
    specs = [I.rod_chain(90, 4, name="rod4"), I.ball_chain(70, 3, seed=73, radius=0.2)]
    batch = P.Batch([P.Model.from_spec(s) for s in specs], max_stages=2, max_history=8)
    n_steps, dt, S = 3, 0.02, 2
    _, _, _, qp, qc, tau = _inputs(specs, S, dt, n_steps, 710)
    ref = _run(P, batch, qp, qc, tau, n_steps, dt, S, P.LBFGS_F32, -1, 100)
    got = _run(P, batch, qp, qc, tau, n_steps, dt, S, P.LBFGS_F32, 2, 100)
    _assert_same(got, ref)


def test_queue_ignored_by_mixed_solver_launches():
    """A launch with Newton and L-BFGS buckets runs without the queue."""
    import paper_1709_04145_b300 as P
    specs = [I.humanoid(3, seed=72), I.rod_chain(90, 4, name="rod4")]
    batch = P.Batch([P.Model.from_spec(s) for s in specs], max_stages=2, max_history=8, newton=True)
    n_steps, dt, S = 2, 0.02, 2
    _, _, _, qp, qc, tau = _inputs(specs, S, dt, n_steps, 715)
    solvers = [P.NEWTON, P.LBFGS]
    ref = _run(P, batch, qp, qc, tau, n_steps, dt, S, solvers, -1, 100)
    got = _run(P, batch, qp, qc, tau, n_steps, dt, S, solvers, 1, 100)
    _assert_same(got, ref)


def test_queued_instances_match_oracle():
    """One block of 32 one-stage groups for 120 chains: instances 32..119 are
    all handed out by the queue."""
    import paper_1709_04145_b300 as P
    spec = I.rod_chain(120, 3, name="rod3")
    batch = P.Batch([P.Model.from_spec(spec)], max_stages=1, max_history=8)
    n_steps, dt, S = 4, 0.01, 1
    states, taus, qps, qp, qc, tau = _inputs([spec], S, dt, n_steps, 720)
    got = _run(P, batch, qp, qc, tau, n_steps, dt, S, P.LBFGS, 1, 2000)
    n = spec.n_dof
    for b in [0, 31, 32, 33, 64, 95, 118, 119]:
        om = O.OracleModel.from_spec(spec, b)
        ref = om.rollout(S, dt, qps[0][b], states[0][0][b], taus[0][:, b, :], "lbfgs", 8, 1e-9, 2000)
        assert ref["status"] == got["status"][b] == 0, b
        assert np.max(np.abs(got["traj_cur"][:, b * n:(b + 1) * n] - ref["traj_cur"])) <= 1e-7, b


def test_resident_queue_on_a_batch_above_residency():
    """65536 ten-link ball chains (the throughput workload), one step of 3
    iterations: the queue capped at the resident blocks (max_blocks = 0)
    gives the static assignment's results."""
    import torch
    import paper_1709_04145_b300 as P
    w = I.ball_chains(count=65536, n_steps=1)
    spec, S, dt, m = w["spec"], w["stages"], w["dt"], w["history"]
    nodes, _ = O.colloc(S)
    dev = torch.device("cuda:0")
    qc = torch.tensor(w["q0"].reshape(-1), device=dev)
    qp = torch.tensor((w["q0"] + nodes[0] * dt * w["qd0"]).reshape(-1), device=dev)
    batch = P.Batch([P.Model.from_spec(spec)], max_stages=S, max_history=m)
    outs = []
    for cap in (-1, 0):
        batch.set_queue(cap)
        o = P.rollout(batch, qp, qc, None, 1, dt, S, P.LBFGS, m, w["tol"], 3, want_traj=False)
        torch.cuda.synchronize()
        outs.append({k: o[k].cpu().numpy() for k in ("q_prev", "q_cur", "status", "iters", "evals",
                                                     "grads")})
    for k in outs[0]:
        assert np.array_equal(outs[0][k], outs[1][k]), k
