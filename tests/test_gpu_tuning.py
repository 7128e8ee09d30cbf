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
