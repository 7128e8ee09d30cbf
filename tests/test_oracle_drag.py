"""Pins of the oracle's drag potential (Section 6.2, Q_drag; Appendix A):
velocity weights exact on polynomials, the integral against quadrature over
rod points, derivatives against central differences, the per-step velocity
decay of one stage, and dissipation."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1709_04145_b300 import inputs as I


def relerr(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def fd(f, x, h=1e-6):
    x = np.asarray(x, float)
    cols = []
    for k in range(x.size):
        e = np.zeros_like(x)
        e[k] = h
        cols.append((np.asarray(f(x + e)) - np.asarray(f(x - e))) / (2 * h))
    return np.stack(cols, axis=-1)


@pytest.mark.parametrize("S", [2, 3, 4])
def test_velocity_weights_differentiate_polynomials(S):
    nodes, _ = O.colloc(S)
    V = O.colloc_vel(S)
    for k in range(S + 2):  # exact for degree <= K = S + 1
        got = V @ nodes ** k
        want = k * nodes[2:] ** (k - 1) if k > 0 else np.zeros(S)
        assert np.max(np.abs(got - want)) < 1e-10, (S, k)


def test_velocity_weights_one_stage_is_backward_difference():
    assert np.array_equal(O.colloc_vel(1), np.array([[0.0, -1.0, 1.0]]))


def test_drag_integral_equals_rod_quadrature():
    """E(c) - E(0) for one stage = c/dt^2 int rho |P(q) - P(q_k)|^2 along the
    rods (2-point Gauss-Legendre is exact for the quadratic integrand)."""
    spec = I.rod_chain(1, 4)
    rng = np.random.default_rng(21)
    qc = rng.uniform(-1, 1, 4)
    qp = qc + rng.normal(0, 0.05, 4)
    q = qc + rng.normal(0, 0.05, 4)
    dt, c = 0.03, 0.8
    om0 = O.OracleModel.from_spec(spec, 0)
    om1 = O.OracleModel.from_spec(spec, 0, drag=c)
    dE = om1.eval(1, dt, q, qp, qc, np.zeros(4), False)[0] - om0.eval(1, dt, q, qp, qc, np.zeros(4), False)[0]
    x, w = np.polynomial.legendre.leggauss(2)
    T1, T0 = om0.fk(q), om0.fk(qc)
    ref = 0.0
    for l in range(4):
        L, m = spec.length[0, l], spec.mass[0, l]
        for xi, wi in zip(x, w):
            p = np.array([0, 0, -(xi + 1) * L / 2, 1.0])
            d = (T1[l] - T0[l]) @ p
            ref += wi * m / 2 * (d[:3] @ d[:3])
    ref *= c / dt ** 2
    assert abs(dE - ref) < 1e-10 * max(abs(ref), 1.0)


def test_zero_drag_is_bitwise_unchanged():
    spec = I.ball_chain(1, 3, seed=22, radius=0.1)
    n = spec.n_dof
    rng = np.random.default_rng(23)
    qc = rng.uniform(-0.5, 0.5, n); qp = qc + rng.normal(0, 0.02, n)
    for S in (1, 2, 3):
        qs = (qc + rng.normal(0, 0.02, (S, n))).reshape(-1)
        a = O.OracleModel.from_spec(spec, 0).eval(S, 0.03, qs, qp, qc, np.zeros(n), True)
        b = O.OracleModel.from_spec(spec, 0, drag=0.0).eval(S, 0.03, qs, qp, qc, np.zeros(n), True)
        assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


@pytest.mark.parametrize("S", [1, 2, 3])
@pytest.mark.parametrize("which", ["rod", "ball"])
def test_drag_derivatives_fd(S, which):
    spec = {"rod": I.rod_chain(1, 4), "ball": I.ball_chain(1, 3, seed=24, radius=0.1)}[which]
    om = O.OracleModel.from_spec(spec, 0, drag=0.7)
    n = om.n_dof
    rng = np.random.default_rng(25)
    qc = rng.uniform(-0.5, 0.5, n); qp = qc + rng.normal(0, 0.02, n)
    tau = rng.normal(0, 0.2, n)
    qs = (qc + rng.normal(0, 0.02, (S, n))).reshape(-1)
    dt = 0.033
    E, r, g, J = om.eval(S, dt, qs, qp, qc, tau, True, True)
    assert relerr(g, fd(lambda x: om.eval(S, dt, x, qp, qc, tau, False)[0], qs)) < 1e-6
    assert relerr(J, fd(lambda x: om.eval(S, dt, x, qp, qc, tau, False)[1], qs)) < 1e-6
    Jp, Jc = om.resid_known_jac(S, dt, qs, qp, qc)
    assert relerr(Jp, fd(lambda x: om.eval(S, dt, qs, x, qc, tau, False)[1], qp)) < 1e-6
    assert relerr(Jc, fd(lambda x: om.eval(S, dt, qs, qp, x, tau, False)[1], qc)) < 1e-6


def test_drag_decay_per_step_one_stage():
    """One stage, no gravity: the drag force -2 c rho v / dt makes a body's
    velocity decay by 1/(1 + 2c) per step (rho (v' - v)/dt + 2 c rho v'/dt = 0).
    A rod spinning slowly about a fixed hinge is that body up to the chord
    error of the rotation per step (~(omega dt)^2)."""
    c = 0.35
    mm = O.mass_moment_rod(1.0, 1.0)
    rest = np.array([1.0, 0, 0, 0, 0, 1.0, 0, 0, 0, 0, 1.0, 0])
    om = O.OracleModel([-1], [0], [[0.0, 1.0, 0.0]], mm, rest, np.zeros(3), drag=c)
    dt, omega0, n_steps = 1e-3, 0.1, 12
    q0 = np.zeros(1)
    out = om.rollout(1, dt, q0 - dt * omega0, q0, np.zeros((n_steps, 1)), "lm", 8, 1e-13, 100)
    assert out["status"] == 0
    th = np.concatenate([[q0[0] - dt * omega0, q0[0]], out["traj_cur"][:, 0]])
    dth = np.diff(th)
    ratios = dth[1:] / dth[:-1]
    assert np.max(np.abs(ratios - 1.0 / (1.0 + 2.0 * c))) < 1e-7, ratios


def test_drag_dissipates():
    """Kinetic energy of a swinging chain after the same steps is lower with
    drag (two stages)."""
    spec = I.rod_chain(1, 3)
    nodes, _ = O.colloc(2)
    q0 = np.array([0.5, -0.3, 0.2])
    dt, n_steps = 0.01, 80
    kin = []
    for c in (0.0, 2.0):
        om = O.OracleModel.from_spec(spec, 0, drag=c)
        out = om.rollout(2, dt, q0, q0, np.zeros((n_steps, 3)), "lm", 8, 1e-9, 100)
        assert out["status"] == 0
        v = (out["traj_cur"][-1] - out["traj_prev"][-1]) / ((0.0 - nodes[0]) * dt)
        kin.append(0.5 * v @ om.hmass(out["traj_cur"][-1]) @ v)
    assert kin[1] < 0.5 * kin[0], kin
