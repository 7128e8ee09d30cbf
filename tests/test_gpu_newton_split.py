"""The one-warp Newton (LM) rollout with its trial-point residual passes
spread over the warp's replicas (pbad_batch_set_newton_split, the default)
gives bit for bit the results of every replica evaluating the whole pass:
trajectories, stages, per-step statuses and exit |r|, iteration and
evaluation counts. Trees (depth-first numbered humanoids), chains, two to
four stages (16, 10 and 8 replicas, with surplus lanes at three stages),
more links than replicas, and steps whose damping loop rejects trials."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1709_04145_b300 import inputs as I

pytestmark = pytest.mark.gpu


def _run(batch, specs, S, dt, n_steps, max_iter, split, seed):
    import torch

    import paper_1709_04145_b300 as P
    dev = torch.device("cuda:0")
    nodes, _ = O.colloc(S)
    states = [I.random_state(s, seed + k, pose_scale=0.4, vel_sigma=1.5) for k, s in enumerate(specs)]
    taus = [I.torques(s, n_steps, seed + 50 + k, sigma=0.2) for k, s in enumerate(specs)]
    q_cur = torch.tensor(np.concatenate([q0.reshape(-1) for q0, _ in states]), device=dev)
    q_prev = torch.tensor(np.concatenate([(q0 + nodes[0] * dt * qd0).reshape(-1)
                                          for q0, qd0 in states]), device=dev)
    tau = torch.tensor(np.concatenate([t.reshape(n_steps, -1) for t in taus], axis=1).reshape(-1),
                       device=dev)
    batch.set_newton_split(split)
    out = P.rollout(batch, q_prev, q_cur, tau, n_steps, dt, S, P.NEWTON, 8, 1e-10, max_iter,
                    want_stages=True)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items() if v is not None}


@pytest.mark.parametrize("S,specs,dt,n_steps,max_iter", [
    (2, lambda: [I.humanoid(40, seed=201), I.rod_chain(9, 5, name="rod5")], 0.033, 6, 30),
    (3, lambda: [I.ball_chain(23, 10, seed=202, radius=0.15)], 0.033, 4, 25),
    (4, lambda: [I.rod_chain(7, 25, name="rod25"), I.humanoid(5, seed=203)], 0.02, 3, 12),
])
def test_split_trial_passes_give_the_same_bits(S, specs, dt, n_steps, max_iter):
    import paper_1709_04145_b300 as P
    specs = specs()
    batch = P.Batch([P.Model.from_spec(s) for s in specs], max_stages=S, max_history=8,
                    newton=True)
    batch.set_newton_cta_min(4097)  # one warp per instance: the mode the split serves
    full = _run(batch, specs, S, dt, n_steps, max_iter, False, 210 + S)
    split = _run(batch, specs, S, dt, n_steps, max_iter, True, 210 + S)
    for key in ("traj_prev", "traj_cur", "stages_traj", "q_prev", "q_cur", "status", "iters",
                "evals", "grads", "step_status", "step_rnorm"):
        assert np.array_equal(full[key], split[key], equal_nan=True), key
    # the damping loop did reject trials (more evaluations than accepted
    # iterations plus one per step), so trial passes were exercised
    assert (full["evals"] > full["iters"] + n_steps).any()


def test_split_setting_rejects_bad_values():
    import paper_1709_04145_b300 as P
    from paper_1709_04145_b300._native import lib
    batch = P.Batch([P.Model.from_spec(I.rod_chain(2, 3, name="rod3"))], max_stages=2,
                    max_history=4, newton=True)
    assert lib().pbad_batch_set_newton_split(batch._h, 2) == -1
    assert lib().pbad_batch_set_newton_split(None, 1) == -1
