"""Pins of the two oracle routines that shape the iteration path: the L-BFGS
preconditioner (the initial inverse Hessian of the two-loop recursion) and
the contact term of the one-stage Gauss-Newton matrix (Eq. FRI's penalty).

- Preconditioner, one stage: for one rod on a hinge, P = dt^2 / (m L^2 / 3),
  the textbook moment of inertia of a rod about its end (times the 1e-8
  regularisation of the joint block); for one capsule on a ball joint at
  theta = 0, P^-1 dt^2 is its inertia tensor about the joint, tr(Sigma) I -
  Sigma from the (separately pinned) second moment.
- Preconditioner, several stages: for one rod on a hinge without gravity, at
  a state where every node coincides, the stage residuals are linear in the
  stage angles to first order with Jacobian Jr = What (x) B, so P must invert
  the Gauss-Newton matrix 2 Jr^T Jr of Eq. EQHOC, with Jr the oracle's dense
  Jacobian (pinned by finite differences).
- Contact term: for a body on a free root with its contact point at the
  ball joint's origin, the point is the translation coordinates themselves,
  so the Gauss-Newton term is the exact Hessian of the penalty energy: the
  finite-difference Hessian of E in the translation block minus the kinetic
  part m / dt^2 I (gravity is linear there).
"""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_1709_04145_b300 import inputs as I

REG = 1e-8  # the joint blocks' regularisation (a fraction of their mean diagonal)


@pytest.mark.parametrize("q", [0.0, 0.4, -1.1])
def test_one_stage_preconditioner_is_the_rod_inertia(q):
    dt, m, L = 0.02, 0.7, 1.3
    om = O.OracleModel.from_spec(I.rod_chain(1, 1, length=L, mass=m, name="rod1"), 0)
    Pv = om.precond_apply(1, dt, [q], [1.0])
    exact = dt * dt / (m * L * L / 3.0 * (1.0 + REG))
    assert abs(Pv[0] / exact - 1.0) < 1e-14


def test_one_stage_preconditioner_of_a_ball_joint_is_the_inertia_tensor():
    dt = 0.02
    spec = I.ball_chain(1, 1, seed=3, radius=0.1)
    om = O.OracleModel.from_spec(spec, 0)
    mm = O.mass_moments_from_spec(spec, 0)[0]
    Sig = np.array([[mm[0], mm[1], mm[2]], [mm[1], mm[3], mm[4]], [mm[2], mm[4], mm[5]]])
    Ij = np.trace(Sig) * np.eye(3) - Sig
    B = Ij + REG * np.trace(Ij) / 3.0 * np.eye(3)
    P = np.stack([om.precond_apply(1, dt, np.zeros(3), e) for e in np.eye(3)], axis=1)
    assert np.max(np.abs(P @ B / dt ** 2 - np.eye(3))) < 1e-13


@pytest.mark.parametrize("S", [2, 3, 4])
def test_several_stage_preconditioner_inverts_the_gauss_newton_matrix(S):
    dt = 0.02
    spec = I.rod_chain(1, 1, length=1.3, mass=0.7, name="rod1")
    om = O.OracleModel.from_spec(dataclasses.replace(spec, gravity=np.zeros(3)), 0)
    q = np.array([0.3])
    _, r, _, J = om.eval(S, dt, np.tile(q, (S, 1)), q, q, np.zeros(1), True, True)
    assert np.max(np.abs(r)) < 1e-9  # every node at q: the residuals vanish
    H = 2.0 * J.T @ J
    P = np.stack([om.precond_apply(S, dt, q, e) for e in np.eye(S)], axis=1)
    # exact but for the regularisation, which enters squared (B^2); with B
    # instead of B^2 in the joint block the product would be B I (B = 0.39)
    assert np.max(np.abs(P @ H - np.eye(S))) < 3.0 * REG


def test_contact_gauss_newton_term_is_the_penalty_hessian():
    dt = 0.02
    spec = I.free_chain(1, 1)
    om = O.OracleModel.from_spec(spec, 0)
    om.set_contact([1], [[0.0, 0.0, 0.0]], z0=0.0, d1=2000.0, d2=100.0)
    n = om.n_dof
    rng = np.random.default_rng(4)
    q_cur = np.zeros(n)
    q_cur[2] = -0.01  # in the ground
    q_cur[3:] = rng.uniform(-0.3, 0.3, 3)
    q_prev = q_cur.copy()
    q_prev[0] -= 0.003
    q = q_cur.copy()
    q[0] += 0.004
    q[1] -= 0.002
    q[2] = -0.015  # deeper, and sliding: normal and tangential terms
    Hc = om.contact_gn(dt, q, q_cur)
    h = 1e-6
    Hfd = np.zeros((3, 3))
    for a in range(3):
        qp, qm = q.copy(), q.copy()
        qp[a] += h
        qm[a] -= h
        gp = om.eval(1, dt, qp, q_prev, q_cur, np.zeros(n))[2]
        gm = om.eval(1, dt, qm, q_prev, q_cur, np.zeros(n))[2]
        Hfd[:, a] = (gp[:3] - gm[:3]) / (2.0 * h)
    m = O.mass_moments_from_spec(spec, 0)[1][9]
    Hpen = Hfd - m / dt ** 2 * np.eye(3)
    assert np.max(np.abs(Hc[:3, :3] - Hpen)) <= 1e-6 * np.max(np.abs(Hpen))
    assert abs(Hc[2, 2]) > 1000.0 and abs(Hc[0, 2]) > 1.0  # both terms are active
    # the rotation coordinates do not move the point
    assert np.max(np.abs(Hc[3:, :])) == 0.0 and np.max(np.abs(Hc[:, 3:])) == 0.0
    # out of the ground the term vanishes
    q_up = q.copy()
    q_up[2] = 0.2
    assert np.max(np.abs(om.contact_gn(dt, q_up, q_cur))) == 0.0
