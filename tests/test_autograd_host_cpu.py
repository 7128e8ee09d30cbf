"""Host logic of the differentiable rollout (checkpoints, segment
recomputation, kept stages, the adjoint's segment order) on the CPU, with
the two launches replaced by a linear two-stage step whose adjoint is
written out here: every forward form (one launch, one launch per segment,
stages kept) gives the gradients of the unrolled map, and the backward
pass hands each segment launch the stages of exactly that segment."""
import numpy as np
import pytest
import torch

from paper_1709_04145_b300 import autograd as AG

# one step (two stages): s0 = a c + b p + tau, s1 = c2 c + d p + e tau;
# the state moves to (q_prev, q_cur) = (s0, s1)
CA, CB, CC, CD, CE = 0.9, -0.3, 1.1, 0.2, 0.5


def _step(p, c, t):
    return CA * c + CB * p + t, CC * c + CD * p + CE * t


class _Batch:
    def __init__(self, D):
        self.D = D
        self.n_instances = D


def _fake_rollout(calls):
    def rollout(batch, q_prev, q_cur, tau_seq, n_steps, dt, S, solver, history, tol, max_iter,
                want_traj=True, want_step_log=True, want_stages=False, out=None, stream=None):
        calls.append(("fwd", n_steps))
        tau = tau_seq.reshape(n_steps, -1)
        p, c = q_prev.clone(), q_cur.clone()
        tp, tc, st = [], [], []
        for k in range(n_steps):
            s0, s1 = _step(p, c, tau[k])
            st.append(torch.stack([s0, s1], dim=1).reshape(-1))  # [instance][stage]
            p, c = s0, s1
            tp.append(p)
            tc.append(c)
        res = dict(q_prev=p, q_cur=c, status=torch.zeros(batch.n_instances, dtype=torch.int32))
        if want_traj:
            res["traj_prev"], res["traj_cur"] = torch.stack(tp), torch.stack(tc)
        if want_stages:
            res["stages_traj"] = torch.stack(st)
        return res
    return rollout


def _fake_backward(calls):
    def rollout_backward(batch, q_prev0, q_cur0, tau_seq, stages_traj, n_steps, dt, S, a_prev,
                         a_cur, stream=None):
        calls.append(("bwd", n_steps))
        tau = tau_seq.reshape(n_steps, -1)
        # the stages handed over must be this segment's, from its start state
        p, c = q_prev0, q_cur0
        for k in range(n_steps):
            s0, s1 = _step(p, c, tau[k])
            assert torch.equal(stages_traj[k], torch.stack([s0, s1], dim=1).reshape(-1)), k
            p, c = s0, s1
        g_tau = torch.zeros_like(tau)
        ap, ac = a_prev.clone(), a_cur.clone()
        for k in range(n_steps - 1, -1, -1):
            g_tau[k] = ap + CE * ac
            ap, ac = CB * ap + CD * ac, CA * ap + CC * ac
        return ap, ac, g_tau, torch.zeros(batch.n_instances, dtype=torch.int32)
    return rollout_backward


def _unrolled_gradients(q0, qd0, tau, node_prev, dt, w_c, w_p):
    """d/d(q0, qd0, tau) of w_c . q_cur + w_p . q_prev after all steps, by
    finite-dimensional linearity: each input's unit vector pushed through."""
    def run(q0_, qd0_, tau_):
        p, c = q0_ + node_prev * dt * qd0_, q0_.copy()
        for k in range(tau_.shape[0]):
            p, c = CA * c + CB * p + tau_[k], CC * c + CD * p + CE * tau_[k]
        return float(w_c @ c + w_p @ p)
    base = run(q0, qd0, tau)
    gq = np.array([run(q0 + e, qd0, tau) - base for e in np.eye(q0.size)])
    gv = np.array([run(q0, qd0 + e, tau) - base for e in np.eye(q0.size)])
    gt = np.zeros_like(tau)
    for k in range(tau.shape[0]):
        for i in range(tau.shape[1]):
            t2 = tau.copy()
            t2[k, i] += 1.0
            gt[k, i] = run(q0, qd0, t2) - base
    return gq, gv, gt


@pytest.mark.parametrize("n_steps,k", [(7, 3), (8, 4), (5, 8), (1, 1)])
def test_every_forward_form_gives_the_unrolled_gradients(monkeypatch, n_steps, k):
    D, dt = 4, 0.05
    rng = np.random.default_rng(10 + n_steps)
    q0, qd0 = rng.normal(size=D), rng.normal(size=D)
    tau = rng.normal(size=(n_steps, D))
    w_c, w_p = rng.normal(size=D), rng.normal(size=D)
    node_prev = float(AG.colloc(2)[0][0])
    ref = _unrolled_gradients(q0, qd0, tau, node_prev, dt, w_c, w_p)
    results = {}
    for form, keep, one_launch in (("one launch", False, 1 << 30), ("per segment", False, 0),
                                   ("kept stages", True, 1 << 30)):
        calls = []
        monkeypatch.setattr(AG, "rollout", _fake_rollout(calls))
        monkeypatch.setattr(AG, "rollout_backward", _fake_backward(calls))
        monkeypatch.setattr(AG, "ONE_LAUNCH_TRAJ_BYTES", one_launch)
        x0 = torch.tensor(q0, requires_grad=True)
        v0 = torch.tensor(qd0, requires_grad=True)
        tt = torch.tensor(tau, requires_grad=True)
        qc, qp, st = AG.rollout_differentiable(_Batch(D), x0, v0, tt, dt, 2, checkpoint_every=k,
                                               on_unsolved="keep", keep_stages=keep)
        ((qc * torch.tensor(w_c)).sum() + (qp * torch.tensor(w_p)).sum()).backward()
        got = (x0.grad.numpy(), v0.grad.numpy(), tt.grad.numpy())
        for g, r in zip(got, ref):
            assert np.allclose(g, r, rtol=1e-12, atol=1e-12), form
        n_seg = -(-n_steps // k)
        fwd = [c for c in calls if c[0] == "fwd"]
        bwd = [c for c in calls if c[0] == "bwd"]
        # forward launches: one, or one per segment; recomputes: one per segment
        n_fwd = (1 if one_launch or keep else n_seg) + (0 if keep else n_seg)
        assert len(fwd) == n_fwd, (form, calls)
        # the backward walks the segments last to first
        assert [c[1] for c in bwd] == [min(k, n_steps - s) for s in
                                       range((n_seg - 1) * k, -1, -k)], (form, calls)
        results[form] = got
    for g1, g2 in zip(results["one launch"], results["per segment"]):
        assert np.array_equal(g1, g2)
