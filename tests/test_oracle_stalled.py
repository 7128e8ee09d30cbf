"""Pins of the oracle's rounding floor of |r| and of the STALLED status.

The floor (om_floor) claims to bound the binary64 rounding error of the step
residual: checked here against the same residual evaluated with 40 decimal
digits (mpmath), written from its definitions - S = 1: the gradient of the
energy of Eq. EQ; S = 2: Eq. HOC, the gradient at each stage of the
transform-weighted inertial and gravity terms with the collocation
accelerations held fixed - by numerical differentiation in high precision.
The STALLED status (a failed line search / LM damping at |r| <= 1e3 floor)
is checked on cases that end at the floor (LM at tol = 0) and on the
severity order of the worst-over-steps status.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1709_04145_b300 import inputs as I

mpmath = pytest.importorskip("mpmath")
mp = mpmath.mp


def _mp_fk(spec, b, q):
    """World 4x4 transforms of every link at q (mpmath), from the spec's
    parent array, joint types, hinge axes and rest transforms."""
    N = spec.n_links
    T = []
    d = 0
    for l in range(N):
        X = mp.matrix(4, 4)
        for r in range(3):
            for c in range(3):
                X[r, c] = mp.mpf(float(spec.rest_rot[l, r, c]))
            X[r, 3] = mp.mpf(float(spec.attach[b, l, r]))
        X[3, 3] = 1
        assert spec.jtype[l] == I.HINGE
        u = [mp.mpf(float(x)) for x in spec.axis[l]]
        th = q[d]
        d += 1
        K = mp.matrix([[0, -u[2], u[1]], [u[2], 0, -u[0]], [-u[1], u[0], 0]])
        R = mp.eye(3) + mp.sin(th) * K + (1 - mp.cos(th)) * (K * K)
        J = mp.eye(4)
        for r in range(3):
            for c in range(3):
                J[r, c] = R[r, c]
        Tl = X * J
        p = spec.parent[l]
        T.append(T[p] * Tl if p >= 0 else Tl)
    return T


def _mp_M(spec, b, l):
    """int rho [p;1][p;1]^T dp of a uniform thin rod from the joint to
    (0, 0, -L): the second moment of a uniform segment."""
    assert spec.shape[l] == I.ROD
    m, L = mp.mpf(float(spec.mass[b, l])), mp.mpf(float(spec.length[b, l]))
    M = mp.matrix(4, 4)
    M[2, 2] = m * L * L / 3
    M[2, 3] = M[3, 2] = -m * L / 2
    M[3, 3] = m
    return M


def _tr_ABt(A, B):
    return mp.fsum(A[r, c] * B[r, c] for r in range(3) for c in range(4))


def _mp_residual(spec, b, S, dt, qs, qp, qc):
    """Stage residuals at 40 digits: S = 1 the gradient of Eq. EQ; S >= 2
    Eq. HOC with the collocation weights of the oracle's table."""
    mp.dps = 40
    n = spec.n_dof
    g = [mp.mpf(float(x)) for x in spec.gravity]
    nodes, W = O.colloc(S)
    W = [[mp.mpf(float(x)) / (mp.mpf(dt) ** 2) for x in row] for row in W]
    Ms = [_mp_M(spec, b, l) for l in range(spec.n_links)]
    qn = [[mp.mpf(float(x)) for x in v] for v in (qp, qc)] + \
         [[mp.mpf(float(x)) for x in qs[i]] for i in range(S)]
    Tn = [_mp_fk(spec, b, v) for v in qn]

    def grav(T, l):
        M = Ms[l]
        return mp.fsum(g[r] * mp.fsum(T[r, c] * M[c, 3] for c in range(4)) for r in range(3))

    r = []
    for i in range(S):
        A = []
        for l in range(spec.n_links):
            Al = mp.matrix(4, 4)
            for j in range(S + 2):
                Al += W[i][j] * Tn[j][l]
            A.append(Al)

        def phi(*x, i=i, A=A):
            T = _mp_fk(spec, b, list(x))
            if S == 1:
                # Eq. EQ: tr(D M D^T)/(2 dt^2) - g.T[mc; m], D = T - 2 T_k + T_{k-1}
                e = 0
                for l in range(spec.n_links):
                    D = (T[l] - 2 * Tn[1][l] + Tn[0][l]) * (1 / mp.mpf(dt))
                    e += _tr_ABt(D * Ms[l], D) / 2 - grav(T[l], l)
                return e
            # Eq. HOC at stage i: d/dx of sum_l T_l(x) : (A_il M_l) - g.T_l(x)[mc; m]
            return mp.fsum(_tr_ABt(T[l], A[l] * Ms[l]) - grav(T[l], l)
                           for l in range(spec.n_links))

        x0 = qn[2 + i]
        for d in range(n):
            e = [0] * n
            e[d] = 1
            r.append(mp.diff(phi, x0, tuple(e)))
    return np.array([float(v) for v in r])


@pytest.mark.parametrize("S,dt", [(1, 0.01), (2, 0.02)])
def test_floor_bounds_the_binary64_rounding_of_the_residual(S, dt):
    spec = I.rod_chain(2, 3, name="rods3")
    rng = np.random.default_rng(11 + S)
    for b in range(2):
        om = O.OracleModel.from_spec(spec, b)
        qc = rng.uniform(-0.7, 0.7, spec.n_dof)
        qp = qc + rng.normal(0, 0.02, spec.n_dof)
        qs = qc[None, :] + rng.normal(0, 0.03, (S, spec.n_dof))
        _, r64, _, _ = om.eval(S, dt, qs, qp, qc, np.zeros(spec.n_dof))
        r_exact = _mp_residual(spec, b, S, dt, qs, qp, qc)
        # the high-precision residual is the one the oracle computes ...
        assert np.max(np.abs(r64 - r_exact)) <= 1e-9 * np.max(np.abs(r_exact))
        # ... and its binary64 rounding error lies below the floor
        err = np.linalg.norm(r64 - r_exact)
        fl = om.floor(S, dt)
        assert err <= fl, (err, fl)
        assert fl < 1e-6 * np.linalg.norm(r_exact)


def test_status_severity_order():
    L = O.lib()
    order = [0, 5, 1, 2, 3, 4]  # CONVERGED < STALLED < MAX_ITER < LS_FAIL < CHOL_FAIL < NONFINITE
    for a_i, a in enumerate(order):
        for b_i, b in enumerate(order):
            assert L.om_status_worse(a, b) == order[max(a_i, b_i)]


def test_lm_at_zero_tolerance_ends_stalled_at_the_floor():
    spec = I.rod_chain(2, 5, name="rods5")
    q0, qd0 = I.random_state(spec, 3)
    nodes, _ = O.colloc(2)
    for b in range(2):
        om = O.OracleModel.from_spec(spec, b)
        qp = q0[b] + nodes[0] * 0.01 * qd0[b]
        res = om.rollout(2, 0.01, qp, q0[b], np.zeros((6, spec.n_dof)), "lm", 8, 0.0, 100)
        fl = om.floor(2, 0.01)
        st, rn = res["step_status"], res["step_rnorm"]
        # no step can meet tol = 0: each ends when the damping can no longer
        # lower E, which happens at the floor
        assert np.all(st == 5), st
        assert np.all(rn <= 1e3 * fl) and np.all(rn > 0)
        assert res["status"] == 5


def test_step_log_matches_single_steps():
    """Per-step status and exit |r| of a rollout equal those of the same
    steps taken one at a time."""
    w = I.pendulum3()
    spec = w["spec"]
    om = O.OracleModel.from_spec(spec, 0)
    q0 = w["q0"][0]
    res = om.rollout(1, w["dt"], q0, q0, np.zeros((5, 3)), "lbfgs", 5, 1e-10, 1000)
    qp, qc = q0.copy(), q0.copy()
    for k in range(5):
        qs, st, _, _ = om.step(1, w["dt"], qp, qc, np.zeros(3), "lbfgs", 5, 1e-10, 1000)
        assert st == res["step_status"][k]
        assert om.last_rnorm == res["step_rnorm"][k]
        assert (st != 0) or om.last_rnorm < 1e-10
        qp, qc = qc, qs[0]
    assert np.array_equal(qc, res["q_cur"])
