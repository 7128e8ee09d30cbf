"""Pins of the oracle's translation joint and the free 6-DOF root built from
it (translation + ball at one origin; Section 6.2's swimmer body):
derivatives against central differences, an exact free-fall parabola, and
exact conservation of linear momentum without external forces."""
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


def test_translation_joint_moves_the_frame():
    spec = I.free_chain(1, 2)
    om = O.OracleModel.from_spec(spec, 0)
    q = np.array([0.3, -0.2, 0.5, 0, 0, 0, 0])
    T = om.fk(q)
    assert np.allclose(T[0][:3, 3], q[:3]) and np.allclose(T[0][:3, :3], np.eye(3))
    assert np.allclose(T[1][:3, 3], q[:3])                          # ball at the same origin
    assert np.allclose(T[2][:3, 3], q[:3] + np.array([0, 0, -1.0]))  # tip of the first rod


@pytest.mark.parametrize("S", [1, 2, 3])
def test_free_root_derivatives_fd(S):
    spec = I.free_chain(1, 3)
    om = O.OracleModel.from_spec(spec, 0, drag=0.3)
    n = om.n_dof
    rng = np.random.default_rng(31)
    qc = rng.uniform(-0.5, 0.5, n); qp = qc + rng.normal(0, 0.02, n)
    tau = rng.normal(0, 0.2, n)
    qs = (qc + rng.normal(0, 0.02, (S, n))).reshape(-1)
    dt = 0.03
    E, r, g, J = om.eval(S, dt, qs, qp, qc, tau, True, True)
    assert relerr(g, fd(lambda x: om.eval(S, dt, x, qp, qc, tau, False)[0], qs)) < 1e-6
    assert relerr(J, fd(lambda x: om.eval(S, dt, x, qp, qc, tau, False)[1], qs)) < 1e-6
    Jp, Jc = om.resid_known_jac(S, dt, qs, qp, qc)
    assert relerr(Jp, fd(lambda x: om.eval(S, dt, qs, x, qc, tau, False)[1], qp)) < 1e-6
    assert relerr(Jc, fd(lambda x: om.eval(S, dt, qs, qp, x, tau, False)[1], qc)) < 1e-6


@pytest.mark.parametrize("S", [1, 2, 3])
def test_free_fall_parabola(S):
    """A rod on a free root released without spin falls along the exact
    parabola x(t) = x0 + v0 t + g t^2 / 2: the collocation polynomial of
    degree S + 1 >= 2 reproduces a quadratic exactly."""
    spec = I.free_chain(1, 1)
    om = O.OracleModel.from_spec(spec, 0)
    nodes, _ = O.colloc(S)
    dt, n_steps = 0.05, 20
    v0 = np.array([0.4, -0.1, 2.0])
    q0 = np.zeros(6)
    qd0 = np.concatenate([v0, np.zeros(3)])
    # tolerance above the FP64 floor of r for S >= 2 (weights ~ 1/dt^2 x positions)
    out = om.rollout(S, dt, q0 + nodes[0] * dt * qd0, q0, np.zeros((n_steps, 6)), "lm", 8,
                     1e-12 if S == 1 else 1e-9, 100)
    assert out["status"] == 0
    t = dt * np.arange(1, n_steps + 1)
    # the quadratic through the two known nodes: x(t_p) = v0 t_p at t_p = nodes[0] dt
    v = v0 - 0.5 * spec.gravity * nodes[0] * dt
    ref = v[None, :] * t[:, None] + 0.5 * spec.gravity[None, :] * t[:, None] ** 2
    assert np.max(np.abs(out["traj_cur"][:, :3] - ref)) < 1e-9
    assert np.max(np.abs(out["traj_cur"][:, 3:])) < 1e-10  # no spin appears


def _com(om, spec, q):
    T = om.fk(q)
    mm = O.mass_moments_from_spec(spec, 0)
    mc = np.zeros(3)
    m = 0.0
    for l in range(spec.n_links):
        mc += T[l][:3, :3] @ mm[l, 6:9] + mm[l, 9] * T[l][:3, 3]
        m += mm[l, 9]
    return mc / m


@pytest.mark.parametrize("S", [1, 2])
def test_free_chain_conserves_linear_momentum(S):
    """No gravity, no drag, no torques: the translation coordinates'
    residual is the total mass times the collocated second difference of the
    centre of mass, so the centre of mass moves on a straight line at
    constant speed over the node sequence."""
    spec = I.free_chain(1, 4)
    spec.gravity = np.zeros(3)
    om = O.OracleModel.from_spec(spec, 0)
    rng = np.random.default_rng(32)
    n = om.n_dof
    q0 = np.concatenate([np.zeros(3), rng.uniform(-0.5, 0.5, n - 3)])
    qd0 = rng.normal(0, 1.0, n)
    nodes, _ = O.colloc(S)
    dt, n_steps = 0.02, 25
    out = om.rollout(S, dt, q0 + nodes[0] * dt * qd0, q0, np.zeros((n_steps, n)), "lm", 8,
                     1e-11 if S == 1 else 1e-9, 100)
    assert out["status"] == 0
    c = np.array([_com(om, spec, q) for q in out["traj_cur"]])
    v = np.diff(c, axis=0) / dt
    assert np.max(np.abs(v - v[0])) < 1e-7 * max(1.0, np.abs(v[0]).max())
