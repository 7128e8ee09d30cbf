"""Differentiable rollouts: a torch.autograd.Function over the CUDA rollout
whose backward pass applies the implicit-function-theorem adjoint of every
converged step. The forward pass is one persistent launch over all steps
(one per segment when the whole trajectory would exceed
ONE_LAUNCH_TRAJ_BYTES); states are checkpointed every ``checkpoint_every``
steps, and going back over each segment takes two launches: a rollout that recomputes
the segment's steps and keeps their stages, and pbad_rollout_backward,
which walks them in reverse. With ``keep_stages=True`` the forward pass
keeps every step's stages instead (S n doubles per instance-step: 36 MB for
1024 twenty-link trees over 64 two-stage steps), and the backward pass runs
only the pbad_rollout_backward launches; the gradients are bitwise those of
the recomputing form, which re-runs the same launches on the same inputs.

The adjoint of a step is the implicit-function theorem at its root, r = 0,
so it holds only for steps solved to the tolerance (CONVERGED) or to the
binary64 floor of r (STALLED). An instance with any other step (MAX_ITER,
LS_FAIL, CHOL_FAIL, NONFINITE), or whose adjoint system is singular, gets
NaN gradients by default (``on_unsolved="nan"``; ``"zero"`` masks them,
``"keep"`` applies the adjoint anyway), and ``adjoint_status`` reports it.

State convention: a rollout starts from (q0, qd0); the node before t_0 is
q_prev0 = q0 + node_prev * dt * qd0 (node_prev < 0 in units of dt), and each
step maps (q_prev, q_cur) to (stage S-1, stage S) (for one stage: (q_cur,
stage 1)). All tensors are DOF-packed float64 CUDA tensors of the batch.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import Batch, LBFGS, NEWTON, colloc, rollout, rollout_backward
from ._native import check, lib

CONVERGED, STALLED = 0, 5
# the forward pass runs in one launch when its whole trajectory (q_prev and
# q_cur of every step) fits in this many bytes, else one launch per segment
ONE_LAUNCH_TRAJ_BYTES = 1 << 30
_RANK = torch.tensor([0, 2, 3, 4, 5, 1], dtype=torch.int32)  # severity of status 0..5


def worse_status(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """Element-wise worst of two status tensors in the order CONVERGED <
    STALLED < MAX_ITER < LS_FAIL < CHOL_FAIL < NONFINITE."""
    rank = _RANK.to(a.device)
    return torch.where(rank[b.long()] > rank[a.long()], b, a)


def _dof_instance(batch: Batch, dev) -> torch.Tensor:
    """Instance index of every DOF of the batch's DOF-packed arrays."""
    idx = [np.repeat(np.arange(int(batch.inst_off[k]), int(batch.inst_off[k + 1])), m.n_dof)
           for k, m in enumerate(batch.models)]
    return torch.tensor(np.concatenate(idx), dtype=torch.long, device=dev)


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q0, qd0, tau_seq, batch, cfg):
        S, dt, n_steps, k = cfg["stages"], cfg["dt"], cfg["n_steps"], cfg["checkpoint_every"]
        nodes, _ = colloc(S)
        q_prev = (q0 + nodes[0] * dt * qd0).contiguous()
        q_cur = q0.contiguous()
        ckpts = []
        kept = []  # per segment (stages_traj, status) when keep_stages
        traj_bytes = 2 * n_steps * batch.D * 8
        if cfg["keep_stages"] or traj_bytes <= ONE_LAUNCH_TRAJ_BYTES:
            # every step in one persistent launch (each instance's warp carries
            # its state from step to step exactly as separate launches would,
            # so the backward pass's segment recomputes end bitwise at the
            # checkpoints); the checkpoints are the trajectory's rows at the
            # segment starts
            out = rollout(batch, q_prev, q_cur, tau_seq.contiguous(), n_steps, dt, S,
                          cfg["solver"], cfg["history"], cfg["tol"], cfg["max_iter"],
                          want_traj=True, want_step_log=False, want_stages=cfg["keep_stages"])
            status = out["status"]
            for s0 in range(0, n_steps, k):
                s1 = min(s0 + k, n_steps)
                if s0 > 0:
                    q_prev, q_cur = out["traj_prev"][s0 - 1], out["traj_cur"][s0 - 1]
                ckpts.append((s0, s1, q_prev.clone(), q_cur.clone()))
                if cfg["keep_stages"]:
                    # (the worst status over all steps: the adjoint status is
                    # the worst over the segments either way)
                    kept.append((out["stages_traj"][s0:s1], status))
            q_prev, q_cur = out["q_prev"], out["q_cur"]  # the end state
            del out
        else:
            # a trajectory too large to hold: one launch per segment, keeping
            # only the checkpoints
            status = torch.zeros(batch.n_instances, dtype=torch.int32, device=q0.device)
            for s0 in range(0, n_steps, k):
                s1 = min(s0 + k, n_steps)
                ckpts.append((s0, s1, q_prev.clone(), q_cur.clone()))
                out = rollout(batch, q_prev, q_cur, tau_seq[s0:s1].contiguous(), s1 - s0, dt, S,
                              cfg["solver"], cfg["history"], cfg["tol"], cfg["max_iter"],
                              want_traj=False, want_step_log=False)
                status = worse_status(status, out["status"])
                q_prev, q_cur = out["q_prev"], out["q_cur"]
        ckpts.append((n_steps, n_steps, q_prev.clone(), q_cur.clone()))
        ctx.batch, ctx.cfg, ctx.ckpts, ctx.kept = batch, cfg, ckpts, kept
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
        # worst over the steps of (the step's own status, the adjoint's status)
        adj = torch.zeros(batch.n_instances, dtype=torch.int32, device=dev)
        segs = ctx.ckpts
        for si in range(len(segs) - 2, -1, -1):
            s0, s1, qp0, qc0 = segs[si]
            tau_seg = tau_seq[s0:s1].contiguous()
            if ctx.kept:
                stages_traj, seg_status = ctx.kept[si]
            else:
                # recompute the segment in one launch, keeping every step's stages
                out = rollout(batch, qp0, qc0, tau_seg, s1 - s0, dt, S, cfg["solver"],
                              cfg["history"], cfg["tol"], cfg["max_iter"], want_traj=False,
                              want_step_log=False, want_stages=True)
                # the same launch on the same inputs: the recomputed segment must
                # end bitwise where the forward pass's did
                ep, ec = segs[si + 1][2], segs[si + 1][3]
                if not (torch.equal(out["q_prev"], ep) and torch.equal(out["q_cur"], ec)):
                    raise RuntimeError("rollout recompute diverged from the forward pass "
                                       f"(steps {s0}..{s1 - 1})")
                stages_traj, seg_status = out["stages_traj"], out["status"]
            adj = worse_status(adj, seg_status)
            # the adjoint of the segment's steps, in reverse, in one launch
            a_prev, a_cur, g_seg, st = rollout_backward(batch, qp0, qc0, tau_seg, stages_traj,
                                                        s1 - s0, dt, S, a_prev.contiguous(),
                                                        a_cur.contiguous())
            adj = worse_status(adj, st)
            g_tau[s0:s1] = g_seg
        g_q0 = a_prev + a_cur
        g_qd0 = ctx.node_prev * dt * a_prev
        if cfg["adjoint_status"] is not None:
            cfg["adjoint_status"].copy_(adj)
        mode = cfg["on_unsolved"]
        if mode != "keep":
            bad_inst = (adj != CONVERGED) & (adj != STALLED)
            if bool(bad_inst.any()):
                bad = bad_inst[_dof_instance(batch, dev)]
                fill = float("nan") if mode == "nan" else 0.0
                g_q0 = g_q0.masked_fill(bad, fill)
                g_qd0 = g_qd0.masked_fill(bad, fill)
                g_tau = g_tau.masked_fill(bad[None, :].expand_as(g_tau), fill)
        return g_q0, g_qd0, g_tau, None, None


def rollout_differentiable(batch: Batch, q0, qd0, tau_seq, dt: float, stages: int,
                           solver=NEWTON, history: int = 8, tol: float = 1e-10,
                           max_iter: int = 100, checkpoint_every: int = 8,
                           on_unsolved: str = "nan", adjoint_status=None,
                           keep_stages: bool = False):
    """Differentiable rollout of tau_seq.shape[0] steps from (q0, qd0).
    Returns (q_cur, q_prev, status) after the last step (status: the worst
    step status per instance); q_cur and q_prev carry gradients to q0, qd0
    and tau_seq. The implicit-function adjoint is valid at steps that ended
    CONVERGED or STALLED; the gradients of an instance with any other step,
    or with a singular adjoint system, are set to NaN (on_unsolved="nan"),
    to zero ("zero"), or left as computed ("keep"). adjoint_status, an int32
    CUDA tensor (instances,), receives in the backward pass the worst over
    the steps of each recomputed step's status and its adjoint's status.
    keep_stages=True keeps every step's stages from the forward pass (S n
    doubles per instance-step) so that the backward pass recomputes nothing;
    the gradients are the same bits."""
    if on_unsolved not in ("nan", "zero", "keep"):
        raise ValueError("on_unsolved must be 'nan', 'zero' or 'keep'")
    cfg = dict(stages=stages, dt=dt, n_steps=int(tau_seq.shape[0]), solver=solver,
               history=history, tol=tol, max_iter=max_iter, checkpoint_every=checkpoint_every,
               on_unsolved=on_unsolved, adjoint_status=adjoint_status,
               keep_stages=bool(keep_stages))
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
