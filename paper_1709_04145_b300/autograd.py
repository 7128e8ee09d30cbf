"""Differentiable rollouts: a torch.autograd.Function over the CUDA rollout
whose backward pass applies the implicit-function-theorem adjoint of every
converged step (pbad_step_backward), recomputing the steps of each segment
from states checkpointed every ``checkpoint_every`` steps.

State convention: a rollout starts from (q0, qd0); the node before t_0 is
q_prev0 = q0 + node_prev * dt * qd0 (node_prev < 0 in units of dt), and each
step maps (q_prev, q_cur) to (stage S-1, stage S) (for one stage: (q_cur,
stage 1)). All tensors are DOF-packed float64 CUDA tensors of the batch.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import Batch, LBFGS, NEWTON, colloc, rollout, step, step_backward
from ._native import check, lib


def _scatter_stage(batch: Batch, S: int, stage: int, vec: torch.Tensor, out: torch.Tensor):
    """out (stage-packed) [:, stage, :] += vec (DOF-packed), model by model."""
    for k, m in enumerate(batch.models):
        a, b = int(batch.dof_off[k]), int(batch.dof_off[k + 1])
        blk = out[S * a:S * b].view(m.count, S, m.n_dof)
        blk[:, stage, :] += vec[a:b].view(m.count, m.n_dof)


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q0, qd0, tau_seq, batch, cfg):
        S, dt, n_steps, k = cfg["stages"], cfg["dt"], cfg["n_steps"], cfg["checkpoint_every"]
        nodes, _ = colloc(S)
        q_prev = (q0 + nodes[0] * dt * qd0).contiguous()
        q_cur = q0.contiguous()
        ckpts = []
        status = torch.zeros(batch.n_instances, dtype=torch.int32, device=q0.device)
        for s0 in range(0, n_steps, k):
            s1 = min(s0 + k, n_steps)
            ckpts.append((s0, s1, q_prev.clone(), q_cur.clone()))
            out = rollout(batch, q_prev, q_cur, tau_seq[s0:s1].contiguous(), s1 - s0, dt, S,
                          cfg["solver"], cfg["history"], cfg["tol"], cfg["max_iter"],
                          want_traj=False)
            status = torch.maximum(status, out["status"])
            q_prev, q_cur = out["q_prev"], out["q_cur"]
        ctx.batch, ctx.cfg, ctx.ckpts = batch, cfg, ckpts
        ctx.save_for_backward(tau_seq)
        ctx.node_prev = float(nodes[0])
        ctx.mark_non_differentiable(status)
        return q_cur, q_prev, status

    @staticmethod
    def backward(ctx, g_cur, g_prev, _g_status):
        (tau_seq,) = ctx.saved_tensors
        batch, cfg = ctx.batch, ctx.cfg
        S, dt = cfg["stages"], cfg["dt"]
        dev = tau_seq.device
        a_cur = g_cur.clone() if g_cur is not None else torch.zeros(batch.D, dtype=torch.float64, device=dev)
        a_prev = g_prev.clone() if g_prev is not None else torch.zeros_like(a_cur)
        g_tau = torch.zeros_like(tau_seq)
        for s0, s1, qp0, qc0 in reversed(ctx.ckpts):
            # recompute the segment step by step, keeping every step's stages
            states = []
            qp, qc = qp0, qc0
            for t in range(s0, s1):
                out = step(batch, qp, qc, tau_seq[t].contiguous(), dt, S, cfg["solver"],
                           cfg["history"], cfg["tol"], cfg["max_iter"])
                states.append((qp, qc, out["q_stages"]))
                qp, qc = out["q_prev"], out["q_cur"]
            for t in range(s1 - 1, s0 - 1, -1):
                qp, qc, qs = states[t - s0]
                gbar = torch.zeros(S * batch.D, dtype=torch.float64, device=dev)
                _scatter_stage(batch, S, S - 1, a_cur, gbar)
                if S >= 2:
                    _scatter_stage(batch, S, S - 2, a_prev, gbar)
                gp, gc, gt, st = step_backward(batch, qp, qc, tau_seq[t].contiguous(), qs, gbar, dt, S)
                if S == 1:  # q_prev' = q_cur passes through
                    gc = gc + a_prev
                a_prev, a_cur = gp, gc
                g_tau[t] = gt
        g_q0 = a_prev + a_cur
        g_qd0 = ctx.node_prev * dt * a_prev
        return g_q0, g_qd0, g_tau, None, None


def rollout_differentiable(batch: Batch, q0, qd0, tau_seq, dt: float, stages: int,
                           solver=NEWTON, history: int = 8, tol: float = 1e-10,
                           max_iter: int = 100, checkpoint_every: int = 8):
    """Differentiable rollout of tau_seq.shape[0] steps from (q0, qd0).
    Returns (q_cur, q_prev, status) after the last step; q_cur and q_prev
    carry gradients to q0, qd0 and tau_seq."""
    cfg = dict(stages=stages, dt=dt, n_steps=int(tau_seq.shape[0]), solver=solver,
               history=history, tol=tol, max_iter=max_iter, checkpoint_every=checkpoint_every)
    return _Rollout.apply(q0, qd0, tau_seq, batch, cfg)


def link_points(batch: Batch, q, link, point_local, want_jac: bool = True, stream=None):
    """World positions (instances, 3) of one body point per instance and the
    Jacobians (3*D, per model [count][3][n]) from the CUDA kernel."""
    pos = torch.empty((batch.n_instances, 3), dtype=torch.float64, device=q.device)
    jac = torch.empty(3 * batch.D, dtype=torch.float64, device=q.device) if want_jac else None
    links = np.ascontiguousarray(link, dtype=np.int32).reshape(len(batch.models))
    s = torch.cuda.current_stream() if stream is None else stream
    check(lib().pbad_link_points(batch._h, C.c_void_p(q.data_ptr()),
                                 links.ctypes.data_as(C.POINTER(C.c_int32)),
                                 C.c_void_p(point_local.data_ptr()), C.c_void_p(pos.data_ptr()),
                                 C.c_void_p(jac.data_ptr()) if jac is not None else None,
                                 C.c_void_p(s.cuda_stream)), "pbad_link_points")
    return pos, jac


class _Points(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q, batch, link, point_local):
        pos, jac = link_points(batch, q.contiguous(), link, point_local)
        ctx.batch = batch
        ctx.save_for_backward(jac)
        return pos

    @staticmethod
    def backward(ctx, g_pos):
        (jac,) = ctx.saved_tensors
        batch = ctx.batch
        g_q = torch.empty(batch.D, dtype=torch.float64, device=g_pos.device)
        for k, m in enumerate(batch.models):
            a, b = int(batch.dof_off[k]), int(batch.dof_off[k + 1])
            i0, i1 = int(batch.inst_off[k]), int(batch.inst_off[k + 1])
            J = jac[3 * a:3 * b].view(m.count, 3, m.n_dof)
            g_q[a:b] = torch.einsum("bi,bin->bn", g_pos[i0:i1], J).reshape(-1)
        return g_q, None, None, None


def points_differentiable(batch: Batch, q, link, point_local):
    """Differentiable world positions (instances, 3) of one point per
    instance (e.g. an end effector)."""
    return _Points.apply(q, batch, link, point_local)
