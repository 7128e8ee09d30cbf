"""B300-native position-based articulated dynamics (Pan & Manocha, arXiv
1709.04145): Python front end of the CUDA library ``libpbad.so``.

Every step of the hot path runs in the library's kernels; this module only
marshals arguments (PyTorch tensors for device memory and streams). Importing
the package does not load the library; the first call does, and fails loudly
if it has not been built.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import inputs
from ._native import PBADError, check, lib

__all__ = ["Model", "Batch", "colloc", "eval_objective_grad", "step", "rollout", "fp64_peak",
           "step_backward", "rollout_backward", "PBADError", "LBFGS", "NEWTON", "LBFGS_F32", "MAP_STAGE", "MAP_LINK",
           "STATUS", "inputs"]

LBFGS = 0
NEWTON = 1
# L-BFGS with the two-loop recursion in binary32 (line search and every
# evaluation binary64): the mixed-precision option
LBFGS_F32 = 2
# instance-to-lane mappings (pbad_batch_set_mapping)
MAP_STAGE = 0
MAP_LINK = 1
# arithmetic of the evaluation's residual pass (pbad_batch_set_precision)
PRECISION_F64 = 0
PRECISION_DF64 = 1
STATUS = {0: "CONVERGED", 1: "MAX_ITER", 2: "LS_FAIL", 3: "CHOL_FAIL", 4: "NONFINITE",
          5: "STALLED"}


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _tptr(t):
    """Device pointer of a CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("arrays must be contiguous CUDA tensors")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def colloc(stages: int):
    """(nodes (S+2,), W (S, S+2)) from the library's own table."""
    nodes = np.zeros(stages + 2)
    W = np.zeros((stages, stages + 2))
    check(lib().pbad_colloc(stages, _dptr(nodes), _dptr(W)), "pbad_colloc")
    return nodes, W


def fp64_peak(device: int = 0) -> float:
    """Measured FP64 FMA throughput of the device, GFLOP/s."""
    out = C.c_double(0)
    check(lib().pbad_fp64_peak(device, C.byref(out)), "pbad_fp64_peak")
    return out.value


def fp64_mma_peak(device: int = 0) -> float:
    """Measured FP64 tensor-core (mma.sync m8n8k4) throughput, GFLOP/s."""
    out = C.c_double(0)
    check(lib().pbad_fp64_mma_peak(device, C.byref(out)), "pbad_fp64_mma_peak")
    return out.value


def damped_gram_solve(J, g, lam: float, stream=None):
    """The LM iteration's damped system for a batch of square Jacobians
    (pbad_damped_gram_solve): J (count, n, n) with J[b, c] column c of J_b,
    g (count, n). Returns (H, L, dl, status): H = J^T J, L the Cholesky
    factor of H + lam I stored column-major (L[b, c, r] = L_b[r][c], r >= c),
    dl = -(H + lam I)^-1 g, status 0 or CHOL_FAIL per instance."""
    import torch
    count, n = int(J.shape[0]), int(J.shape[1])
    if tuple(J.shape) != (count, n, n) or tuple(g.shape) != (count, n):
        raise ValueError("J must be (count, n, n) and g (count, n)")
    H = torch.empty_like(J)
    L = torch.zeros_like(J)
    dl = torch.empty_like(g)
    st = torch.empty(count, dtype=torch.int32, device=J.device)
    check(lib().pbad_damped_gram_solve(count, n, _tptr(J), _tptr(g), float(lam), _tptr(H), _tptr(L),
                                        _tptr(dl), _tptr(st), _stream(stream)),
          "pbad_damped_gram_solve")
    return H, L, dl, st


class Model:
    """One topology with ``count`` instances (pbad_model)."""

    def __init__(self, parent, jtype, axis, mass_moment, rest, gravity, device: int = 0,
                 drag: float = 0.0, contact: dict | None = None):
        parent = np.ascontiguousarray(parent, dtype=np.int32)
        jtype = np.ascontiguousarray(jtype, dtype=np.int32)
        axis = np.ascontiguousarray(axis, dtype=np.float64).reshape(-1, 3)
        N = parent.shape[0]
        mass_moment = np.ascontiguousarray(mass_moment, dtype=np.float64).reshape(-1, N, 10)
        rest = np.ascontiguousarray(rest, dtype=np.float64).reshape(-1, N, 12)
        gravity = np.ascontiguousarray(gravity, dtype=np.float64).reshape(3)
        count = mass_moment.shape[0]
        if rest.shape[0] != count:
            raise ValueError("mass_moment and rest disagree on the instance count")
        h = C.c_void_p()
        check(lib().pbad_model_create(N, _iptr(parent), _iptr(jtype), _dptr(axis), count,
                                      _dptr(mass_moment), _dptr(rest), _dptr(gravity), device,
                                      C.byref(h)), "pbad_model_create")
        self._h = h
        self.n_links = N
        self.count = count
        self.device = device
        nl, nd, cnt = C.c_int32(), C.c_int32(), C.c_int64()
        check(lib().pbad_model_info(h, C.byref(nl), C.byref(nd), C.byref(cnt)), "pbad_model_info")
        self.n_dof = nd.value
        self.drag = float(drag)
        if self.drag != 0.0:
            check(lib().pbad_model_set_drag(h, self.drag), "pbad_model_set_drag")
        self.contact = None
        if contact is not None:
            self.set_contact(**contact)

    def set_contact(self, link, point, z0: float = 0.0, d1: float = 0.0, d2: float = 0.0):
        """Penalty contact of Eq. FRI against the ground z < z0 at body points
        point[k] (link frame) of link[k] (one stage only; set before creating
        batches)."""
        lk = np.ascontiguousarray(np.asarray(link).reshape(-1), dtype=np.int32)
        pt = np.ascontiguousarray(np.asarray(point, dtype=np.float64).reshape(-1, 3))
        check(lib().pbad_model_set_contact(self._h, int(lk.shape[0]), _iptr(lk), _dptr(pt),
                                           float(z0), float(d1), float(d2)),
              "pbad_model_set_contact")
        self.contact = dict(link=lk, point=pt, z0=z0, d1=d1, d2=d2)

    @classmethod
    def from_spec(cls, spec: "inputs.BodySpec", device: int = 0, drag: float = 0.0,
                  contact: dict | None = None) -> "Model":
        """drag: coefficient c of the drag potential (Section 6.2), per unit
        mass; contact: keyword arguments of set_contact (Eq. FRI)."""
        from .models import mass_moments, rest_transforms
        return cls(spec.parent, spec.jtype, spec.axis, mass_moments(spec), rest_transforms(spec),
                   spec.gravity, device, drag, contact)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().pbad_model_destroy(h)
            self._h = None


class Batch:
    """An ordered list of models with solver workspace (pbad_batch).

    DOF-packed tensors have length D (models concatenated, each [count][n]);
    use ``pack``/``unpack`` to convert from/to per-model (count, n) arrays.
    """

    def __init__(self, models, max_stages: int = 5, max_history: int = 16, newton: bool = False):
        self.models = list(models)
        arr = (C.c_void_p * len(self.models))(*[m._h for m in self.models])
        h = C.c_void_p()
        check(lib().pbad_batch_create(len(self.models), arr, max_stages, max_history,
                                      1 if newton else 0, C.byref(h)), "pbad_batch_create")
        self._h = h
        self.max_stages = max_stages
        self.max_history = max_history
        ni, nd, wb = C.c_int64(), C.c_int64(), C.c_int64()
        check(lib().pbad_batch_info(h, C.byref(ni), C.byref(nd), C.byref(wb)), "pbad_batch_info")
        self.n_instances = ni.value
        self.D = nd.value
        self.workspace_bytes = wb.value
        self.device = self.models[0].device
        self.dof_off = np.cumsum([0] + [m.count * m.n_dof for m in self.models])
        self.inst_off = np.cumsum([0] + [m.count for m in self.models])

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().pbad_batch_destroy(h)
            self._h = None

    def set_threads(self, threads: int):
        """Threads per block of the solver kernels (32, 64, 96, 128)."""
        check(lib().pbad_batch_set_threads(self._h, int(threads)), "pbad_batch_set_threads")
        self.threads = int(threads)

    def set_mapping(self, mapping: int):
        """Instance-to-lane mapping of the evaluation and L-BFGS kernels:
        MAP_STAGE (one lane per stage, the default) or MAP_LINK (one lane
        per stage and link; serial chains with stages * links <= 32)."""
        check(lib().pbad_batch_set_mapping(self._h, int(mapping)), "pbad_batch_set_mapping")
        self.mapping = int(mapping)

    def set_bucket_mapping(self, mappings):
        """Per-bucket mapping of steps and rollouts (MAP_STAGE, MAP_LINK or -1
        for the batch's); None clears it. Buckets of different mappings still
        share one persistent launch."""
        if mappings is None:
            check(lib().pbad_batch_set_bucket_mapping(self._h, None), "pbad_batch_set_bucket_mapping")
            self.bucket_mapping = None
            return
        arr = np.ascontiguousarray(mappings, dtype=np.int32).reshape(len(self.models))
        check(lib().pbad_batch_set_bucket_mapping(self._h, _iptr(arr)), "pbad_batch_set_bucket_mapping")
        self.bucket_mapping = [int(x) for x in arr]

    def set_newton_cta_min(self, min_sn: int):
        """Newton buckets with stages x DOFs >= min_sn run one CTA of four
        warps per instance (default 128; 4097: never)."""
        check(lib().pbad_batch_set_newton_cta_min(self._h, int(min_sn)),
              "pbad_batch_set_newton_cta_min")

    def set_newton_split(self, on: bool):
        """One-warp Newton buckets with two or more stages: spread the
        residual pass at each trial point of the damping loop over the
        warp's replicas (True, the default) or have every replica evaluate
        it (False). Both give the same bits."""
        check(lib().pbad_batch_set_newton_split(self._h, 1 if on else 0),
              "pbad_batch_set_newton_split")

    def set_precision(self, precision: int):
        """Arithmetic of eval_objective_grad's residual pass: PRECISION_F64
        (default) or PRECISION_DF64 (double-float after the joint rotations;
        needs MAP_LINK). Rollouts always evaluate in binary64."""
        check(lib().pbad_batch_set_precision(self._h, int(precision)), "pbad_batch_set_precision")

    def set_queue(self, max_blocks: int):
        """Instance queue of the L-BFGS rollouts: at most max_blocks blocks,
        groups take the next instance when done (0 = the GPU's resident
        blocks; < 0 = off, the default)."""
        check(lib().pbad_batch_set_queue(self._h, int(max_blocks)), "pbad_batch_set_queue")

    def pack(self, per_model, stages: int = 0):
        """Concatenates per-model arrays (count, n) (or (count, S, n)) into one
        flat array (numpy or torch, whatever was given)."""
        flats = [a.reshape(-1) for a in per_model]
        if hasattr(flats[0], "detach"):
            import torch
            return torch.cat(flats).contiguous()
        return np.concatenate(flats)

    def unpack(self, flat, stages: int = 0):
        """Splits a DOF- or stage-packed flat array into per-model views."""
        out = []
        mult = max(stages, 1)
        for k, m in enumerate(self.models):
            a, b = self.dof_off[k] * mult, self.dof_off[k + 1] * mult
            shape = (m.count, stages, m.n_dof) if stages else (m.count, m.n_dof)
            out.append(flat[a:b].reshape(shape))
        return out


def _solvers(batch: Batch, solvers):
    if solvers is None:
        return None
    if isinstance(solvers, int):
        solvers = [solvers] * len(batch.models)
    arr = np.ascontiguousarray(solvers, dtype=np.int32)
    if arr.shape[0] != len(batch.models):
        raise ValueError("one solver per model")
    return arr


def eval_objective_grad(batch: Batch, q_star, q_prev, q_cur, tau, dt: float, stages: int,
                        want_resid: bool = True, stream=None):
    """Objective E (per instance), dE/dq_* (stage-packed) and the stage
    residuals r (stage-packed) at the given stage configurations."""
    import torch
    dev = q_star.device
    E = torch.empty(batch.n_instances, dtype=torch.float64, device=dev)
    grad = torch.empty(stages * batch.D, dtype=torch.float64, device=dev)
    resid = torch.empty_like(grad) if want_resid else None
    check(lib().pbad_eval_objective_grad(batch._h, _tptr(q_star), _tptr(q_prev), _tptr(q_cur),
                                         _tptr(tau), float(dt), int(stages), _tptr(E),
                                         _tptr(grad), _tptr(resid), _stream(stream)),
          "pbad_eval_objective_grad")
    return E, grad, resid


def step(batch: Batch, q_prev, q_cur, tau, dt: float, stages: int, solver=LBFGS,
         history: int = 8, tol: float = 1e-10, max_iter: int = 1000, stream=None):
    """One time step. Returns dict(q_prev, q_cur, q_stages, status, iters)."""
    import torch
    dev = q_prev.device
    qp = torch.empty(batch.D, dtype=torch.float64, device=dev)
    qc = torch.empty_like(qp)
    qs = torch.empty(stages * batch.D, dtype=torch.float64, device=dev)
    st = torch.empty(batch.n_instances, dtype=torch.int32, device=dev)
    it = torch.empty_like(st)
    sv = _solvers(batch, solver)
    check(lib().pbad_step(batch._h, _tptr(q_prev), _tptr(q_cur), _tptr(tau), float(dt),
                          int(stages), _iptr(sv) if sv is not None else None, int(history),
                          float(tol), int(max_iter), _tptr(qp), _tptr(qc), _tptr(qs), _tptr(st),
                          _tptr(it), _stream(stream)), "pbad_step")
    return dict(q_prev=qp, q_cur=qc, q_stages=qs, status=st, iters=it)


def rollout(batch: Batch, q_prev0, q_cur0, tau_seq, n_steps: int, dt: float, stages: int,
            solver=LBFGS, history: int = 8, tol: float = 1e-10, max_iter: int = 1000,
            want_traj: bool = True, want_step_log: bool = True, want_stages: bool = False,
            out=None, stream=None):
    """n_steps steps in one persistent launch. tau_seq: (n_steps*D) or None.
    Returns dict(traj_prev, traj_cur (n_steps, D) or None, q_prev, q_cur,
    status (worst over the steps), iters, evals, grads, step_status, step_rnorm
    ((n_steps, instances): each step's status and the |r|_2 it ended at, or
    None)). ``out`` may supply preallocated output tensors (same keys) so that
    the call allocates nothing (e.g. inside a CUDA graph)."""
    import torch
    dev = q_cur0.device
    if out is None:
        out = dict(q_prev=torch.empty(batch.D, dtype=torch.float64, device=dev),
                   q_cur=torch.empty(batch.D, dtype=torch.float64, device=dev),
                   status=torch.empty(batch.n_instances, dtype=torch.int32, device=dev),
                   iters=torch.empty(batch.n_instances, dtype=torch.int32, device=dev),
                   evals=torch.empty(batch.n_instances, dtype=torch.int32, device=dev),
                   grads=torch.empty(batch.n_instances, dtype=torch.int32, device=dev),
                   traj_prev=None, traj_cur=None)
        if want_traj:
            out["traj_prev"] = torch.empty((n_steps, batch.D), dtype=torch.float64, device=dev)
            out["traj_cur"] = torch.empty((n_steps, batch.D), dtype=torch.float64, device=dev)
        if want_stages:
            out["stages_traj"] = torch.empty((n_steps, stages * batch.D), dtype=torch.float64,
                                             device=dev)
        if want_step_log:
            out["step_status"] = torch.empty((n_steps, batch.n_instances), dtype=torch.int32,
                                             device=dev)
            out["step_rnorm"] = torch.empty((n_steps, batch.n_instances), dtype=torch.float64,
                                            device=dev)
    sv = _solvers(batch, solver)
    check(lib().pbad_rollout(batch._h, _tptr(q_prev0), _tptr(q_cur0), _tptr(tau_seq),
                             int(n_steps), float(dt), int(stages),
                             _iptr(sv) if sv is not None else None, int(history), float(tol),
                             int(max_iter), _tptr(out.get("traj_prev")),
                             _tptr(out.get("traj_cur")), _tptr(out["q_prev"]),
                             _tptr(out["q_cur"]), _tptr(out["status"]), _tptr(out["iters"]),
                             _tptr(out.get("evals")), _tptr(out.get("grads")),
                             _tptr(out.get("step_status")), _tptr(out.get("step_rnorm")),
                             _tptr(out.get("stages_traj")), _stream(stream)), "pbad_rollout")
    return out


def rollout_backward(batch: Batch, q_prev0, q_cur0, tau_seq, stages_traj, n_steps: int, dt: float,
                     stages: int, a_prev, a_cur, stream=None):
    """Implicit-function adjoint of n_steps consecutive steps in one launch
    (reverse order): returns (a_prev0, a_cur0, g_tau (n_steps, D), status)
    for the loss gradients a_prev, a_cur of the state after the last step;
    stages_traj (n_steps, S*D) as a rollout with want_stages writes it."""
    import torch
    dev = q_cur0.device
    ap = torch.empty(batch.D, dtype=torch.float64, device=dev)
    ac = torch.empty_like(ap)
    gt = torch.empty((n_steps, batch.D), dtype=torch.float64, device=dev)
    st = torch.empty(batch.n_instances, dtype=torch.int32, device=dev)
    check(lib().pbad_rollout_backward(batch._h, _tptr(q_prev0), _tptr(q_cur0), _tptr(tau_seq),
                                      _tptr(stages_traj), int(n_steps), float(dt), int(stages),
                                      _tptr(a_prev), _tptr(a_cur), _tptr(ap), _tptr(ac), _tptr(gt),
                                      _tptr(st), _stream(stream)), "pbad_rollout_backward")
    return ap, ac, gt, st


def step_backward(batch: Batch, q_prev, q_cur, tau, q_star, g_bar, dt: float, stages: int,
                  stream=None):
    """Implicit-function adjoint of one converged step: returns (gq_prev,
    gq_cur, gtau, status) for g_bar = dL/dq_* (stage-packed)."""
    import torch
    dev = q_star.device
    gp = torch.empty(batch.D, dtype=torch.float64, device=dev)
    gc = torch.empty_like(gp)
    gt = torch.empty_like(gp)
    st = torch.empty(batch.n_instances, dtype=torch.int32, device=dev)
    check(lib().pbad_step_backward(batch._h, _tptr(q_prev), _tptr(q_cur), _tptr(tau),
                                   _tptr(q_star), _tptr(g_bar), float(dt), int(stages), _tptr(gp),
                                   _tptr(gc), _tptr(gt), _tptr(st), _stream(stream)),
          "pbad_step_backward")
    return gp, gc, gt, st
