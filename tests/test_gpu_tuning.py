"""Per-bucket solver choice on the GPU: one solver per model, and the choice
follows the probes (on 5-link hinge chains at dt = 0.05 with two stages
L-BFGS converges nothing within its cap while Newton converges)."""
import numpy as np
import pytest

from paper_1709_04145_b300 import inputs as I

pytestmark = pytest.mark.gpu


def test_choose_solvers_per_bucket():
    import torch
    import paper_1709_04145_b300 as P
    from paper_1709_04145_b300.tuning import choose_solvers
    specs = [I.rod_chain(64, 5, name="rod5"), I.humanoid(32, seed=71)]
    S, dt = 2, 0.05
    nodes, _ = P.colloc(S)
    states = [I.random_state(s, 72 + k) for k, s in enumerate(specs)]
    dev = torch.device("cuda:0")
    qc = torch.tensor(np.concatenate([q0.reshape(-1) for q0, _ in states]), device=dev)
    qp = torch.tensor(np.concatenate([(q0 + nodes[0] * dt * qd0).reshape(-1) for q0, qd0 in states]),
                      device=dev)
    batch = P.Batch([P.Model.from_spec(s) for s in specs], max_stages=S, max_history=8, newton=True)
    solvers, report = choose_solvers(batch, qp, qc, None, dt, S, probe_steps=1, tol=1e-8,
                                     max_iter={P.LBFGS: 30, P.NEWTON: 30})
    assert len(solvers) == 2 and all(s in (P.LBFGS, P.NEWTON) for s in solvers)
    rod = {r.solver: r for r in report[0]}
    assert rod[P.LBFGS].converged < rod[P.NEWTON].converged
    assert solvers[0] == P.NEWTON
    # the chosen solvers run in one launch
    out = P.rollout(batch, qp, qc, None, 2, dt, S, solvers, 8, 1e-8, 30, want_traj=False)
    assert np.isin(out["status"].cpu().numpy(), [0, 1, 2, 3]).all()


def test_autotuners_leave_a_consistent_batch():
    """autotune_bucket_mapping and autotune_newton_cta time real launches and
    leave the batch at their choice: the link mapping only where the library
    accepts it (here the ten-link chains), a Newton threshold among the
    candidates, and a rollout at the chosen settings matches the settings'
    own rollout bit for bit."""
    import torch
    import paper_1709_04145_b300 as P
    from paper_1709_04145_b300.tuning import (autotune_bucket_mapping, autotune_newton_cta,
                                              newton_cta_candidates)
    specs = [I.ball_chain(96, 10, seed=81, radius=0.15), I.humanoid(16, seed=82)]
    S, dt = 3, 0.01
    nodes, _ = P.colloc(S)
    states = [I.random_state(s, 83 + k, pose_scale=0.2, vel_sigma=0.2) for k, s in enumerate(specs)]
    dev = torch.device("cuda:0")
    qc = torch.tensor(np.concatenate([q0.reshape(-1) for q0, _ in states]), device=dev)
    qp = torch.tensor(np.concatenate([(q0 + nodes[0] * dt * qd0).reshape(-1) for q0, qd0 in states]),
                      device=dev)
    batch = P.Batch([P.Model.from_spec(s) for s in specs], max_stages=S, max_history=8, newton=True)
    lb = lambda: P.rollout(batch, qp, qc, None, 1, dt, S, P.LBFGS, 8, 1e-8, 20, want_traj=False)
    chosen, trials = autotune_bucket_mapping(batch, lb)
    assert chosen[1] == P.MAP_STAGE and trials[1][1] == float("inf")  # a tree: refused
    assert np.isfinite(trials[0][1])  # the ten-link chains (S N = 30) were timed link-mapped
    a = lb()["q_cur"].cpu().numpy()
    b = lb()["q_cur"].cpu().numpy()
    assert np.array_equal(a, b)
    batch.set_bucket_mapping(None)
    nw = lambda: P.rollout(batch, qp, qc, None, 1, dt, S, P.NEWTON, 8, 1e-8, 20, want_traj=False)
    t, times = autotune_newton_cta(batch, nw, S)
    assert t in newton_cta_candidates([S * m.n_dof for m in batch.models]) and t in times
    assert all(np.isfinite(v) for v in times.values())
    out = nw()
    assert np.isin(out["status"].cpu().numpy(), [0, 1, 2, 3, 5]).all()  # nothing non-finite
