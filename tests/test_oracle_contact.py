"""Pins of the oracle's penalty contact (Eq. FRI, Section 6.2): the energy
against a direct sum over the contact points, derivatives against central
differences with points in contact, and the static penetration of a body
resting on the ground."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1709_04145_b300 import inputs as I


def relerr(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def fd(f, x, h=1e-7):
    x = np.asarray(x, float)
    cols = []
    for k in range(x.size):
        e = np.zeros_like(x)
        e[k] = h
        cols.append((np.asarray(f(x + e)) - np.asarray(f(x - e))) / (2 * h))
    return np.stack(cols, axis=-1)


def _tips(spec):
    """One contact point at the tip of every body link."""
    links = [l for l in range(spec.n_links) if spec.length[0, l] > 0]
    pts = [[0.0, 0.0, -spec.length[0, l]] for l in links]
    return links, pts


def _case(seed=41):
    spec = I.free_chain(1, 3)
    links, pts = _tips(spec)
    contact = dict(link=links, point=pts, z0=0.0, d1=200.0, d2=30.0)
    rng = np.random.default_rng(seed)
    n = spec.n_dof
    qc = np.concatenate([[0.1, -0.2, 0.35], rng.uniform(-0.4, 0.4, n - 3)])
    qp = qc + rng.normal(0, 0.01, n)
    q = qc + rng.normal(0, 0.01, n)
    q[2] = 0.2  # root low enough that some tips are below z = 0
    return spec, contact, q, qc, qp


def test_contact_energy_is_the_point_sum():
    spec, contact, q, qc, qp = _case()
    dt = 0.02
    om0 = O.OracleModel.from_spec(spec, 0)
    om1 = O.OracleModel.from_spec(spec, 0, contact=contact)
    n = spec.n_dof
    dE = om1.eval(1, dt, q, qp, qc, np.zeros(n), False)[0] - om0.eval(1, dt, q, qp, qc, np.zeros(n), False)[0]
    T1, T0 = om0.fk(q), om0.fk(qc)
    ref, active = 0.0, 0
    for l, p in zip(contact["link"], contact["point"]):
        P = (T1[l] @ np.append(p, 1.0))[:3]
        Pk = (T0[l] @ np.append(p, 1.0))[:3]
        d = max(0.0, contact["z0"] - P[2])
        vt = (P[:2] - Pk[:2]) / dt
        ref += contact["d1"] * d * d + contact["d2"] * d * d * (vt @ vt)
        active += d > 0
    assert active >= 1
    assert abs(dE - ref) < 1e-11 * max(abs(ref), 1.0)


def test_contact_derivatives_fd():
    spec, contact, q, qc, qp = _case()
    om = O.OracleModel.from_spec(spec, 0, contact=contact)
    n = spec.n_dof
    tau = np.random.default_rng(42).normal(0, 0.1, n)
    dt = 0.02
    E, r, g, J = om.eval(1, dt, q, qp, qc, tau, True, True)
    assert relerr(g, fd(lambda x: om.eval(1, dt, x, qp, qc, tau, False)[0], q)) < 1e-6
    assert relerr(J, fd(lambda x: om.eval(1, dt, x, qp, qc, tau, False)[1], q)) < 1e-6
    Jp, Jc = om.resid_known_jac(1, dt, q, qp, qc)
    assert relerr(Jp, fd(lambda x: om.eval(1, dt, q, x, qc, tau, False)[1], qp)) < 1e-6
    assert relerr(Jc, fd(lambda x: om.eval(1, dt, q, qp, x, tau, False)[1], qc)) < 1e-6


def test_resting_penetration_balances_weight():
    """A rod on a free root lying flat with both ends on the ground comes to
    rest (with drag to take out the bounce) where the two penalty forces
    2 D1 d carry its weight: d = m g / (4 D1) at each end."""
    spec = I.free_chain(1, 1)
    L, m, D1 = 1.0, 1.0, 500.0
    contact = dict(link=[1, 1], point=[[0, 0, 0.0], [0, 0, -L]], z0=0.0, d1=D1, d2=5.0)
    om = O.OracleModel.from_spec(spec, 0, drag=0.2, contact=contact)
    # lying along x: rotate the rod (local -z) by +pi/2 about y
    q0 = np.array([0.0, 0.0, 0.005, 0.0, np.pi / 2, 0.0])
    dt, n_steps = 0.01, 300
    out = om.rollout(1, dt, q0, q0, np.zeros((n_steps, 6)), "lm", 8, 1e-9, 100)
    assert out["status"] == 0
    T = om.fk(out["traj_cur"][-1])
    ends = [(T[1] @ np.array([0, 0, z, 1.0]))[2] for z in (0.0, -L)]
    want = -m * 9.81 / (4 * D1)
    assert max(abs(e - want) for e in ends) < 2e-3 * abs(want), (ends, want)
