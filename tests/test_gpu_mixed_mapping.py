"""Per-bucket mappings in one launch (pbad_batch_set_bucket_mapping): a
batch whose link-mapped L-BFGS chains share the launch with stage-mapped
L-BFGS buckets, a Newton tree and CTA-mode Newton chains. Every bucket must
give bit for bit what it gives in a launch of its own mapping (each block
runs the same device function on the same inputs), and the link-mapped
bucket must match the oracle step by step."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1709_04145_b300 import inputs as I

pytestmark = pytest.mark.gpu

S, DT, TOL, M, MAX_ITER = 1, 0.01, 1e-8, 8, 1000  # one stage: L-BFGS solves Eq. EQ


def _specs():
    return [I.ball_chain(37, 5, seed=21, radius=0.2),  # link-mapped: S N = 5 lanes, 6 per warp
            I.rod_chain(45, 7, name="rod7"),  # stage-mapped L-BFGS
            I.humanoid(9, seed=22),  # Newton, stage mapping
            I.rod_chain(3, 130, name="rod130")]  # Newton, S n = 130: CTA per instance


def _states(specs):
    out = []
    for k, s in enumerate(specs):
        q0, qd0 = I.random_state(s, 300 + k, pose_scale=0.3, vel_sigma=0.3)
        out.append((q0, qd0))
    return out


def _roll(P, specs, states, solvers, mappings, T=6):
    import torch
    dev = torch.device("cuda:0")
    batch = P.Batch([P.Model.from_spec(s) for s in specs], max_stages=S, max_history=M, newton=True)
    if mappings is not None:
        batch.set_bucket_mapping(mappings)
    nodes, _ = O.colloc(S)
    qc = np.concatenate([q0.reshape(-1) for q0, _ in states])
    qp = np.concatenate([(q0 + nodes[0] * DT * qd0).reshape(-1) for q0, qd0 in states])
    out = P.rollout(batch, torch.tensor(qp, device=dev), torch.tensor(qc, device=dev), None, T, DT,
                    S, solvers, M, TOL, MAX_ITER)
    return batch, {k: v.cpu().numpy() for k, v in out.items() if hasattr(v, "cpu")}


def _bucket(batch, res, k, key):
    if key in ("traj_cur", "traj_prev", "q_cur", "q_prev"):
        a, b = int(batch.dof_off[k]), int(batch.dof_off[k + 1])
    else:
        a, b = int(batch.inst_off[k]), int(batch.inst_off[k + 1])
    return res[key][..., a:b]


def test_mixed_launch_equals_single_mapping_launches():
    import paper_1709_04145_b300 as P
    specs = _specs()
    states = _states(specs)
    solvers = [P.LBFGS, P.LBFGS, P.NEWTON, P.NEWTON]
    batch, mixed = _roll(P, specs, states, solvers, [P.MAP_LINK, P.MAP_STAGE, P.MAP_STAGE, P.MAP_STAGE])
    keys = ("traj_cur", "step_status", "step_rnorm", "status", "iters", "evals")
    for k, spec in enumerate(specs):
        mp = P.MAP_LINK if k == 0 else P.MAP_STAGE
        b1, alone = _roll(P, [spec], [states[k]], [solvers[k]], [mp])
        for key in keys:
            got = _bucket(batch, mixed, k, key)
            ref = _bucket(b1, alone, 0, key)
            assert np.array_equal(got, ref, equal_nan=True), (spec.name, key)


def test_mixed_launch_link_bucket_matches_oracle():
    """The link-mapped bucket of the mixed launch against the oracle: equal
    per-step statuses; converged steps agree per element to 1e-6 max(1, |q|)
    (both sides stop at |r| < 1e-8 on well-conditioned one-step systems)."""
    import paper_1709_04145_b300 as P
    specs = _specs()
    states = _states(specs)
    T = 6
    batch, res = _roll(P, specs, states, [P.LBFGS, P.LBFGS, P.NEWTON, P.NEWTON],
                       [P.MAP_LINK, -1, -1, -1], T)
    spec, (q0, qd0) = specs[0], states[0]
    nodes, _ = O.colloc(S)
    n = spec.n_dof
    traj = _bucket(batch, res, 0, "traj_cur")
    st = _bucket(batch, res, 0, "step_status")
    compared = 0
    for b in (0, 1, 17, 36):
        om = O.OracleModel.from_spec(spec, b)
        ref = om.rollout(S, DT, q0[b] + nodes[0] * DT * qd0[b], q0[b], np.zeros((T, n)), "lbfgs", M,
                         TOL, MAX_ITER)
        for t in range(T):
            assert st[t, b] == ref["step_status"][t], (b, t)
            if st[t, b] != 0:
                break
            q = ref["traj_cur"][t]
            err = np.abs(traj[t, b * n:(b + 1) * n] - q)
            assert np.all(err <= 1e-6 * np.maximum(1.0, np.abs(q))), (b, t, err.max())
            compared += 1
    assert compared >= 12


def test_bucket_mapping_refusals_and_clear():
    """A link mapping on a bucket it cannot serve is refused (a tree, a
    Newton bucket); -1 and clearing fall back to the batch's mapping."""
    import paper_1709_04145_b300 as P
    from paper_1709_04145_b300._native import PBADError
    specs = _specs()
    states = _states(specs)
    solvers = [P.LBFGS, P.LBFGS, P.NEWTON, P.NEWTON]
    for bad in ([P.MAP_STAGE, P.MAP_STAGE, P.MAP_LINK, P.MAP_STAGE],   # humanoid: a tree
                [P.MAP_STAGE, P.MAP_STAGE, P.MAP_STAGE, P.MAP_LINK]):  # Newton, N > 32
        with pytest.raises(PBADError):
            _roll(P, specs, states, solvers, bad, T=1)
    b_stage, r_stage = _roll(P, specs, states, solvers, None, T=2)
    b_clear, r_clear = _roll(P, specs, states, solvers, [-1, -1, -1, -1], T=2)
    assert np.array_equal(r_stage["traj_cur"], r_clear["traj_cur"])
    with pytest.raises(PBADError):
        b_clear.set_bucket_mapping([7, 0, 0, 0])
    b_clear.set_bucket_mapping(None)
