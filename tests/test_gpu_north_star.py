"""Long-trajectory parity: 200 steps solved to the same tolerance on both
sides end within max |dq| <= 1e-7 rad of the oracle's trajectory, beyond the
three-rod pendulum - five-link hinge chains solved by Newton at two and
three stages and by L-BFGS at one stage (under both lane mappings), with
ragged instance counts. Every step must end solved on both sides
(CONVERGED, or STALLED at the binary64 rounding floor of r: which of the
two a step at the floor reports turns on rounding, so only solved-ness is
compared step by step)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1709_04145_b300 import inputs as I

pytestmark = pytest.mark.gpu

T, DT = 200, 0.01
SOLVED = (0, 5)


def _run(spec, q0, qd0, S, solver_name, tol, max_iter, mapping=None):
    import torch

    import paper_1709_04145_b300 as P
    dev = torch.device("cuda:0")
    solver = {"lm": P.NEWTON, "lbfgs": P.LBFGS}[solver_name]
    batch = P.Batch([P.Model.from_spec(spec)], max_stages=S, max_history=8,
                    newton=solver == P.NEWTON)
    if mapping is not None:
        batch.set_mapping(mapping)
    nodes, _ = O.colloc(S)
    qp = torch.tensor((q0 + nodes[0] * DT * qd0).reshape(-1), device=dev)
    qc = torch.tensor(q0.reshape(-1), device=dev)
    out = P.rollout(batch, qp, qc, None, T, DT, S, solver, 8, tol, max_iter)
    return out["traj_cur"].cpu().numpy(), out["step_status"].cpu().numpy()


def _check(spec, q0, qd0, S, solver_name, tol, max_iter, traj, st, sample):
    n = spec.n_dof
    nodes, _ = O.colloc(S)
    worst = 0.0
    for b in sample:
        om = O.OracleModel.from_spec(spec, b)
        ref = om.rollout(S, DT, q0[b] + nodes[0] * DT * qd0[b], q0[b], np.zeros((T, n)), solver_name,
                         8, tol, max_iter)
        assert np.isin(ref["step_status"], SOLVED).all(), (b, "oracle")
        assert np.isin(st[:, b], SOLVED).all(), (b, "gpu")
        dq = np.max(np.abs(traj[:, b * n:(b + 1) * n] - ref["traj_cur"]))
        assert dq <= 1e-7, (b, dq)
        worst = max(worst, dq)
    return worst


@pytest.mark.parametrize("S,tol", [(2, 1e-10), (3, 1e-9)])
def test_newton_200_steps_hinge_chains(S, tol):
    spec = I.rod_chain(37, 5, name="rod5")  # ragged: 37 instances, one warp each
    q0, qd0 = I.random_state(spec, 77, pose_scale=0.5, vel_sigma=0.5)
    traj, st = _run(spec, q0, qd0, S, "lm", tol, 100)
    _check(spec, q0, qd0, S, "lm", tol, 100, traj, st, (0, 1, 2, 3, 18, 36))


@pytest.mark.parametrize("mapping", ["stage", "link"])
def test_lbfgs_200_steps_one_stage_hinge_chains(mapping):
    import paper_1709_04145_b300 as P
    spec = I.rod_chain(45, 5, name="rod5")  # ragged over 32-lane groups and warps
    q0, qd0 = I.random_state(spec, 77, pose_scale=0.5, vel_sigma=0.5)
    mp = P.MAP_STAGE if mapping == "stage" else P.MAP_LINK
    traj, st = _run(spec, q0, qd0, 1, "lbfgs", 1e-10, 1000, mapping=mp)
    _check(spec, q0, qd0, 1, "lbfgs", 1e-10, 1000, traj, st, (0, 1, 2, 3, 31, 44))
