"""ctypes front end of the CPU oracle (``pbad_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers. The product path never imports this
module, and this module never imports the product package.

Builds ``libpbad_oracle.so`` with gcc on first use if it is missing.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pbad_oracle.c")
_LIB = os.path.join(_HERE, "libpbad_oracle.so")

HINGE, BALL, TRANSLATION = 0, 1, 2
# solver names of step/rollout: L-BFGS, Levenberg-Marquardt, and L-BFGS whose
# two-loop recursion runs in binary32 (line search and evaluations binary64)
SOLVERS = {"lbfgs": 0, "lm": 1, "lbfgs32": 2}
STATUS = {0: "CONVERGED", 1: "MAX_ITER", 2: "LS_FAIL", 3: "CHOL_FAIL", 4: "NONFINITE",
          5: "STALLED"}


def build(force: bool = False) -> str:
    """Compiles the oracle (plain C99, FP64, no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-D_DEFAULT_SOURCE",
                               "-ffp-contract=off", "-fPIC", "-shared", "-o",
                               _LIB, _SRC, "-lm"])
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        vp = C.c_void_p
        L.om_model_new.restype = vp
        L.om_model_new.argtypes = [C.c_int, ip, ip, dp, dp, dp, dp]
        L.om_model_free.argtypes = [vp]
        L.om_n_dof.restype = C.c_int
        L.om_n_dof.argtypes = [vp]
        L.om_fk.argtypes = [vp, dp, dp]
        L.om_link_dT.argtypes = [vp, dp, C.c_int, dp]
        L.om_link_ddT.argtypes = [vp, dp, C.c_int, C.c_int, C.c_int, dp]
        L.om_joint_rot.argtypes = [C.c_int, dp, dp, dp]
        L.om_joint_drot.argtypes = [C.c_int, dp, dp, C.c_int, dp]
        L.om_joint_ddrot.argtypes = [C.c_int, dp, dp, C.c_int, C.c_int, dp]
        L.om_legendre_roots.restype = C.c_int
        L.om_legendre_roots.argtypes = [C.c_int, dp]
        L.om_colloc.restype = C.c_int
        L.om_colloc.argtypes = [C.c_int, dp, dp]
        L.om_colloc_vel.argtypes = [C.c_int, dp]
        L.om_model_set_drag.argtypes = [vp, C.c_double]
        L.om_model_set_contact.argtypes = [vp, C.c_int, ip, dp, C.c_double, C.c_double,
                                           C.c_double]
        L.om_mass_moment_rod.argtypes = [C.c_double, C.c_double, dp]
        L.om_mass_moment_capsule.argtypes = [C.c_double, C.c_double, C.c_double, dp]
        L.om_hmass.argtypes = [vp, dp, dp]
        L.om_eval.restype = C.c_double
        L.om_eval.argtypes = [vp, C.c_int, C.c_double, dp, dp, dp, dp, dp, dp, dp]
        L.om_resid_known_jac.argtypes = [vp, C.c_int, C.c_double, dp, dp, dp, dp, dp]
        L.om_step.restype = C.c_int
        L.om_step.argtypes = [vp, C.c_int, C.c_double, dp, dp, dp, C.c_int, C.c_int,
                              C.c_double, C.c_int, C.c_int, dp, ip, ip, dp]
        L.om_rollout.restype = C.c_int
        L.om_rollout.argtypes = [vp, C.c_int, C.c_double, dp, dp, dp, C.c_int, C.c_int,
                                 C.c_int, C.c_double, C.c_int, C.c_int, dp, dp, dp, dp, ip, ip,
                                 ip, dp]
        L.om_eval_fast.restype = C.c_double
        L.om_eval_fast.argtypes = [vp, C.c_int, C.c_double, dp, dp, dp, dp, dp, dp]
        L.om_model_set_fast.argtypes = [vp, C.c_int]
        L.om_floor.restype = C.c_double
        L.om_floor.argtypes = [vp, C.c_int, C.c_double]
        L.om_status_worse.restype = C.c_int
        L.om_status_worse.argtypes = [C.c_int, C.c_int]
        L.om_step_adjoint.restype = C.c_int
        L.om_step_adjoint.argtypes = [vp, C.c_int, C.c_double, dp, dp, dp, dp, dp, dp, dp, dp]
        L.om_rnea.restype = C.c_int
        L.om_rnea.argtypes = [vp, dp, dp, dp, dp]
        L.om_rk4.restype = C.c_int
        L.om_rk4.argtypes = [vp, dp, dp, dp, C.c_double, C.c_int]
        L.om_deriv.argtypes = [vp, dp, dp, dp]
        L.om_lbfgs_direction.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, dp, dp, dp,
                                         C.c_double, dp, dp, C.c_int, dp]
        L.om_precond_apply.argtypes = [vp, C.c_int, C.c_double, dp, dp, dp]
        L.om_contact_gn.argtypes = [vp, C.c_double, dp, dp, dp]
        _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(C.POINTER(C.c_int))


def _null():
    return C.POINTER(C.c_double)()


# --------------------------------------------------------------------------
# stand-alone functions
# --------------------------------------------------------------------------

def legendre_roots(n: int) -> np.ndarray:
    x = np.zeros(max(n, 1))
    _, xp = _d(x)
    lib().om_legendre_roots(n, xp)
    return x[:n].copy() if n else np.zeros(0)


def colloc(S: int):
    """(nodes (S+2,), W (S, S+2)) in units of dt and 1/dt^2."""
    nodes = np.zeros(S + 2)
    W = np.zeros((S, S + 2))
    rc = lib().om_colloc(S, nodes.ctypes.data_as(C.POINTER(C.c_double)),
                         W.ctypes.data_as(C.POINTER(C.c_double)))
    if rc != 0:
        raise ValueError("unsupported stage count")
    return nodes, W


def colloc_vel(S: int) -> np.ndarray:
    """First-derivative weights V (S, S+2) in units of 1/dt: the stage-node
    velocities of the collocation polynomial (S >= 2) or the backward
    difference [0, -1, 1] of the drag potential (S = 1)."""
    V = np.zeros((S, S + 2))
    if lib().om_colloc_vel(S, V.ctypes.data_as(C.POINTER(C.c_double))) != 0:
        raise ValueError("unsupported stage count")
    return V


def mass_moment_rod(m: float, L: float) -> np.ndarray:
    out = np.zeros(10)
    lib().om_mass_moment_rod(m, L, out.ctypes.data_as(C.POINTER(C.c_double)))
    return out


def mass_moment_capsule(m: float, L: float, r: float) -> np.ndarray:
    out = np.zeros(10)
    lib().om_mass_moment_capsule(m, L, r, out.ctypes.data_as(C.POINTER(C.c_double)))
    return out


def joint_rot(jtype: int, axis, q, k: int | None = None, m: int | None = None):
    """R, dR/dq_k or d2R/dq_k dq_m of one joint (3x3)."""
    axis, ap = _d(np.asarray(axis, dtype=np.float64).reshape(3))
    q, qp = _d(np.atleast_1d(np.asarray(q, dtype=np.float64)))
    out = np.zeros(9)
    op = out.ctypes.data_as(C.POINTER(C.c_double))
    if k is None:
        lib().om_joint_rot(jtype, ap, qp, op)
    elif m is None:
        lib().om_joint_drot(jtype, ap, qp, k, op)
    else:
        lib().om_joint_ddrot(jtype, ap, qp, k, m, op)
    return out.reshape(3, 3)


# --------------------------------------------------------------------------
# models
# --------------------------------------------------------------------------

def mass_moments_from_spec(spec, b: int) -> np.ndarray:
    N = spec.n_links
    mm = np.zeros((N, 10))
    for l in range(N):
        if spec.shape[l] == 0:
            mm[l] = mass_moment_rod(spec.mass[b, l], spec.length[b, l])
        else:
            mm[l] = mass_moment_capsule(spec.mass[b, l], spec.length[b, l], spec.radius[b, l])
    return mm


def rest_from_spec(spec, b: int) -> np.ndarray:
    N = spec.n_links
    rest = np.zeros((N, 3, 4))
    rest[:, :, :3] = spec.rest_rot
    rest[:, :, 3] = spec.attach[b]
    return rest.reshape(N, 12)


class OracleModel:
    """One articulated body (one instance) in the oracle."""

    def __init__(self, parent, jtype, axis, mm, rest, gravity, drag: float = 0.0,
                 contact=None):
        self.parent, pp = _i(parent)
        self.jtype, jp = _i(jtype)
        self.axis, ap = _d(np.asarray(axis).reshape(-1, 3))
        self.mm, mp = _d(np.asarray(mm).reshape(-1, 10))
        self.rest, rp = _d(np.asarray(rest).reshape(-1, 12))
        self.gravity, gp = _d(gravity)
        self.n_links = int(self.parent.shape[0])
        h = lib().om_model_new(self.n_links, pp, jp, ap, mp, rp, gp)
        if not h:
            raise ValueError("malformed model")
        self._h = C.c_void_p(h)
        self.n_dof = lib().om_n_dof(self._h)
        self.drag = float(drag)
        lib().om_model_set_drag(self._h, self.drag)
        if contact is not None:
            self.set_contact(**contact)

    def set_contact(self, link, point, z0=0.0, d1=0.0, d2=0.0):
        """Eq. FRI penalty contact against the ground z < z0 at body points
        point[k] (link frame) of link[k]; one stage only."""
        lk, lp = _i(np.asarray(link).reshape(-1))
        pt, pp = _d(np.asarray(point, dtype=np.float64).reshape(-1, 3))
        if lib().om_model_set_contact(self._h, int(lk.shape[0]), lp, pp, float(z0), float(d1),
                                      float(d2)) != 0:
            raise ValueError("contact link out of range")
        self._contact = (lk, pt)

    @classmethod
    def from_spec(cls, spec, b: int = 0, drag: float = 0.0, contact=None):
        return cls(spec.parent, spec.jtype, spec.axis, mass_moments_from_spec(spec, b),
                   rest_from_spec(spec, b), spec.gravity, drag, contact)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.om_model_free(h)
            self._h = None

    def fk(self, q):
        q, qp = _d(q)
        T = np.zeros((self.n_links, 4, 4))
        lib().om_fk(self._h, qp, T.ctypes.data_as(C.POINTER(C.c_double)))
        return T

    def link_dT(self, q, l: int):
        q, qp = _d(q)
        out = np.zeros((self.n_dof, 4, 4))
        lib().om_link_dT(self._h, qp, l, out.ctypes.data_as(C.POINTER(C.c_double)))
        return out

    def deriv(self, q, G):
        """Algorithm DERIV (O(N)): d/dq of sum_l <G_l, T_l(q)> for fixed 3x4
        seeds G (N, 3, 4). Returns (n,)."""
        q, qp = _d(q)
        G, gp = _d(np.asarray(G, dtype=np.float64).reshape(-1, 12))
        r = np.zeros(self.n_dof)
        lib().om_deriv(self._h, qp, gp, r.ctypes.data_as(C.POINTER(C.c_double)))
        return r

    def link_ddT(self, q, l: int, d: int, e: int):
        q, qp = _d(q)
        out = np.zeros((4, 4))
        lib().om_link_ddT(self._h, qp, l, d, e, out.ctypes.data_as(C.POINTER(C.c_double)))
        return out

    def hmass(self, q):
        q, qp = _d(q)
        H = np.zeros((self.n_dof, self.n_dof))
        lib().om_hmass(self._h, qp, H.ctypes.data_as(C.POINTER(C.c_double)))
        return H

    def eval(self, S: int, dt: float, qs, q_prev, q_cur, tau, want_grad=True, want_jac=False):
        """Returns (E, r, grad, Jr); grad / Jr are None unless requested."""
        n = self.n_dof
        qs, qsp = _d(np.asarray(qs).reshape(S * n))
        q_prev, pp = _d(q_prev)
        q_cur, cp = _d(q_cur)
        tau, tp = _d(tau)
        r = np.zeros(S * n)
        g = np.zeros(S * n) if want_grad else None
        J = np.zeros((S * n, S * n)) if want_jac else None
        E = lib().om_eval(self._h, S, dt, qsp, pp, cp, tp,
                          r.ctypes.data_as(C.POINTER(C.c_double)),
                          g.ctypes.data_as(C.POINTER(C.c_double)) if g is not None else _null(),
                          J.ctypes.data_as(C.POINTER(C.c_double)) if J is not None else _null())
        return E, r, g, J

    def eval_fast(self, S: int, dt: float, qs, q_prev, q_cur, tau):
        """(E, r, grad) by the O(N) evaluation (Algorithm DERIV and its
        tangent) that the CPU baseline times; no contact points."""
        n = self.n_dof
        qs, qsp = _d(np.asarray(qs).reshape(S * n))
        q_prev, pp = _d(q_prev)
        q_cur, cp = _d(q_cur)
        tau, tp = _d(tau)
        r = np.zeros(S * n)
        g = np.zeros(S * n)
        E = lib().om_eval_fast(self._h, S, dt, qsp, pp, cp, tp,
                               r.ctypes.data_as(C.POINTER(C.c_double)),
                               g.ctypes.data_as(C.POINTER(C.c_double)))
        return E, r, g

    def set_fast(self, fast: bool):
        """Makes step/rollout's L-BFGS evaluate in O(N) (om_eval_fast)."""
        lib().om_model_set_fast(self._h, int(bool(fast)))

    def resid_known_jac(self, S: int, dt: float, qs, q_prev, q_cur):
        n = self.n_dof
        qs, qsp = _d(np.asarray(qs).reshape(S * n))
        q_prev, pp = _d(q_prev)
        q_cur, cp = _d(q_cur)
        Jp = np.zeros((S * n, n))
        Jc = np.zeros((S * n, n))
        lib().om_resid_known_jac(self._h, S, dt, qsp, pp, cp,
                                 Jp.ctypes.data_as(C.POINTER(C.c_double)),
                                 Jc.ctypes.data_as(C.POINTER(C.c_double)))
        return Jp, Jc

    def step(self, S, dt, q_prev, q_cur, tau, solver="lbfgs", history=8, tol=1e-10,
             max_iter=None, precond=True):
        n = self.n_dof
        sv = SOLVERS[solver]
        if max_iter is None:
            max_iter = 100 if sv == 1 else 1000
        q_prev, pp = _d(q_prev)
        q_cur, cp = _d(q_cur)
        tau, tp = _d(tau)
        qs = np.zeros(S * n)
        it = C.c_int(0)
        ev = C.c_int(0)
        rn = C.c_double(0)
        st = lib().om_step(self._h, S, dt, pp, cp, tp, sv, history, tol, max_iter,
                           int(precond), qs.ctypes.data_as(C.POINTER(C.c_double)),
                           C.byref(it), C.byref(ev), C.byref(rn))
        self.last_rnorm = rn.value
        return qs.reshape(S, n), st, it.value, ev.value

    def precond_apply(self, S: int, dt: float, q_cur, v):
        """P v with the L-BFGS preconditioner built at q_cur (v: S n)."""
        n = self.n_dof
        q_cur, cp = _d(q_cur)
        v, vp_ = _d(np.asarray(v).reshape(S * n))
        out = np.zeros(S * n)
        lib().om_precond_apply(self._h, S, dt, cp, vp_, out.ctypes.data_as(C.POINTER(C.c_double)))
        return out

    def contact_gn(self, dt: float, q, q_cur):
        """The contact term (n x n) of the one-stage Gauss-Newton matrix at q."""
        n = self.n_dof
        q, qp_ = _d(q)
        q_cur, cp = _d(q_cur)
        H = np.zeros((n, n))
        lib().om_contact_gn(self._h, dt, qp_, cp, H.ctypes.data_as(C.POINTER(C.c_double)))
        return H

    def floor(self, S: int, dt: float) -> float:
        """Rounding floor of |r|_2 for one step (see om_floor); a step whose
        line search cannot lower E at |r| <= 1e3 floor ends STALLED."""
        return lib().om_floor(self._h, S, dt)

    def rollout(self, S, dt, q_prev0, q_cur0, tau_seq, solver="lbfgs", history=8,
                tol=1e-10, max_iter=None, precond=True):
        """Returns dict(traj_prev, traj_cur (n_steps, n), q_prev, q_cur, status
        (worst over the steps), iters, evals, step_status (n_steps,), step_rnorm
        (n_steps,): each step's status and exit |r|_2)."""
        n = self.n_dof
        sv = SOLVERS[solver]
        if max_iter is None:
            max_iter = 100 if sv == 1 else 1000
        tau_seq, tsp = _d(np.asarray(tau_seq).reshape(-1, n))
        n_steps = tau_seq.shape[0]
        q_prev0, pp = _d(q_prev0)
        q_cur0, cp = _d(q_cur0)
        tp_ = np.zeros((n_steps, n))
        tc_ = np.zeros((n_steps, n))
        qpo = np.zeros(n)
        qco = np.zeros(n)
        it = C.c_int(0)
        ev = C.c_int(0)
        sst = np.zeros(n_steps, dtype=np.int32)
        srn = np.zeros(n_steps)
        fp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
        st = lib().om_rollout(self._h, S, dt, pp, cp, tsp, n_steps, sv, history, tol,
                              max_iter, int(precond), fp(tp_), fp(tc_), fp(qpo), fp(qco),
                              C.byref(it), C.byref(ev),
                              sst.ctypes.data_as(C.POINTER(C.c_int)), fp(srn))
        return dict(traj_prev=tp_, traj_cur=tc_, q_prev=qpo, q_cur=qco, status=st,
                    iters=it.value, evals=ev.value, step_status=sst, step_rnorm=srn)

    def step_adjoint(self, S, dt, q_prev, q_cur, tau, qs, gbar):
        n = self.n_dof
        q_prev, pp = _d(q_prev)
        q_cur, cp = _d(q_cur)
        tau, tp = _d(tau)
        qs, qsp = _d(np.asarray(qs).reshape(S * n))
        gbar, gp = _d(np.asarray(gbar).reshape(S * n))
        gqp = np.zeros(n)
        gqc = np.zeros(n)
        gt = np.zeros(n)
        fp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
        rc = lib().om_step_adjoint(self._h, S, dt, pp, cp, tp, qsp, gp, fp(gqp), fp(gqc), fp(gt))
        if rc != 0:
            raise RuntimeError("singular residual Jacobian")
        return gqp, gqc, gt

    def rnea(self, q, qd, qdd):
        q, qp = _d(q)
        qd, vp = _d(qd)
        qdd, ap = _d(qdd)
        tau = np.zeros(self.n_dof)
        rc = lib().om_rnea(self._h, qp, vp, ap, tau.ctypes.data_as(C.POINTER(C.c_double)))
        if rc != 0:
            raise ValueError("RNEA supports hinge joints only")
        return tau

    def rk4(self, q, qd, tau, h: float, n_steps: int):
        q = np.array(q, dtype=np.float64)
        qd = np.array(qd, dtype=np.float64)
        tau, tp = _d(tau)
        rc = lib().om_rk4(self._h, q.ctypes.data_as(C.POINTER(C.c_double)),
                          qd.ctypes.data_as(C.POINTER(C.c_double)), tp, h, n_steps)
        if rc != 0:
            raise RuntimeError("RK4 failed")
        return q, qd


def lbfgs_direction(sh, yh, rho, gamma, P, g, head: int, nh: int, f32: bool = False):
    """The two-loop recursion of the oracle's L-BFGS (binary64, or the
    binary32 variant) on explicit data: ring sh, yh (m, n) with the newest
    pair at head-1, rho (m,), H0 = gamma P with P dense (n, n). Returns d."""
    sh, sp = _d(sh)
    yh, yp = _d(yh)
    rho, rp = _d(rho)
    P, pp = _d(P)
    g, gp = _d(g)
    m, n = sh.shape
    d = np.zeros(n)
    lib().om_lbfgs_direction(n, nh, m, head, sp, yp, rp, gamma, pp, gp, int(f32),
                             d.ctypes.data_as(C.POINTER(C.c_double)))
    return d


def initial_prev(q0, qd0, S: int, dt: float):
    """q at the node k-1+alpha_{S-1} from q0 and an initial velocity:
    q_prev = q0 + node_prev * dt * qd0 (node_prev < 0)."""
    nodes, _ = colloc(S)
    return q0 + nodes[0] * dt * qd0
