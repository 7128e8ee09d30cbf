"""The double-float residual pass (PBAD_PRECISION_DF64, link mapping)
against the binary64 oracle: at random points its E, r and gradient agree
to the evaluation tolerance; at a solved step its residual error stays
within 2^6 times the binary64 rounding floor (48 significant bits against
53), while the binary64 pass stays within twice the floor."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1709_04145_b300 import inputs as I

pytestmark = pytest.mark.gpu


def _t(a, dev):
    import torch
    return torch.tensor(np.ascontiguousarray(a).reshape(-1), device=dev)


def _relerr(a, b):
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("S", [1, 3])
def test_df64_eval_random_points(S):
    import torch

    import paper_1709_04145_b300 as P
    dev = torch.device("cuda:0")
    spec = I.ball_chain(9, 10 if S == 3 else 8, seed=31, radius=0.15)
    rng = np.random.default_rng(32)
    B, n = spec.count, spec.n_dof
    qc = rng.uniform(-0.6, 0.6, (B, n))
    qp = qc + rng.normal(0, 0.02, (B, n))
    qs = qc[:, None, :] + rng.normal(0, 0.03, (B, S, n))
    tau = rng.normal(0, 0.3, (B, n))
    batch = P.Batch([P.Model.from_spec(spec)], max_stages=S, max_history=8)
    batch.set_mapping(P.MAP_LINK)
    batch.set_precision(P.PRECISION_DF64)
    E, g, r = P.eval_objective_grad(batch, _t(qs, dev), _t(qp, dev), _t(qc, dev), _t(tau, dev), 0.033, S)
    E, g, r = E.cpu().numpy(), g.cpu().numpy().reshape(B, -1), r.cpu().numpy().reshape(B, -1)
    for b in range(B):
        om = O.OracleModel.from_spec(spec, b)
        Eo, ro, go, _ = om.eval(S, 0.033, qs[b], qp[b], qc[b], tau[b], True)
        assert abs(E[b] - Eo) <= 1e-10 * abs(Eo), b
        assert _relerr(r[b], ro) <= 1e-10, b
        assert _relerr(g[b], go) <= 1e-10, b


def test_df64_residual_error_at_a_solved_step():
    import torch

    import paper_1709_04145_b300 as P
    dev = torch.device("cuda:0")
    w = I.ball_chains(count=64, n_links=10, n_steps=1)
    spec, S, dt = w["spec"], w["stages"], w["dt"]
    nodes, _ = O.colloc(S)
    qp = w["q0"] + nodes[0] * dt * w["qd0"]
    batch = P.Batch([P.Model.from_spec(spec)], max_stages=S, max_history=8, newton=True)
    out = P.step(batch, _t(qp, dev), _t(w["q0"], dev), None, dt, S, P.NEWTON, 8, 1e-8, 100)
    st = out["status"].cpu().numpy()
    qs = out["q_stages"]
    res = {}
    for prec in (P.PRECISION_F64, P.PRECISION_DF64):
        batch.set_mapping(P.MAP_LINK)
        batch.set_precision(prec)
        _, _, r = P.eval_objective_grad(batch, qs, _t(qp, dev), _t(w["q0"], dev), None, dt, S)
        res[prec] = r.cpu().numpy().reshape(spec.count, -1)
    qs_h = qs.cpu().numpy().reshape(spec.count, S, spec.n_dof)
    checked = 0
    for b in range(spec.count):
        if st[b] != 0:
            continue
        om = O.OracleModel.from_spec(spec, b)
        _, ro, _, _ = om.eval(S, dt, qs_h[b], qp[b], w["q0"][b], np.zeros(spec.n_dof), False)
        fl = om.floor(S, dt)
        assert np.linalg.norm(res[P.PRECISION_F64][b] - ro) <= 2 * fl, b
        assert np.linalg.norm(res[P.PRECISION_DF64][b] - ro) <= 64 * fl, b
        checked += 1
    assert checked >= spec.count * 0.9


def test_df64_needs_the_link_mapping():
    import torch

    import paper_1709_04145_b300 as P
    spec = I.rod_chain(2, 3, name="rod3")
    batch = P.Batch([P.Model.from_spec(spec)], max_stages=2, max_history=8)
    batch.set_precision(P.PRECISION_DF64)
    q = torch.zeros(batch.D, dtype=torch.float64, device="cuda:0")
    with pytest.raises(P.PBADError, match="UNSUPPORTED"):
        P.eval_objective_grad(batch, torch.zeros(2 * batch.D, dtype=torch.float64, device="cuda:0"),
                              q, q, None, 0.01, 2)
    with pytest.raises(P.PBADError, match="ARG"):
        batch.set_precision(5)
