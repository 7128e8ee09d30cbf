"""Pins of the oracle's L-BFGS search direction, binary64 and the
mixed-precision variant (binary32 two-loop recursion, binary64 line search
and evaluations):

- the two-loop recursion equals -H g with H the textbook BFGS inverse update
  (Nocedal & Wright, Eq. 6.17) applied to H0 = gamma P over the stored pairs,
  oldest first, built as a dense matrix;
- the secant equation H y = s holds for the newest pair;
- the binary32 variant stays within binary32 rounding of both, and differs
  from the binary64 result (it really rounds);
- a time step solved with the binary32 direction reaches the same solution as
  Levenberg-Marquardt (the fixed point is set by the step equations, not by
  the solver's path).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1709_04145_b300 import inputs as I


def relerr(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def _problem(n, m, seed, f32=False):
    """Pairs y = A s of an SPD A (every s^T y > 0), an SPD P, a gradient."""
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(n, n))
    A = A @ A.T + n * np.eye(n)
    sh = rng.normal(size=(m, n))
    yh = sh @ A.T
    if f32:  # the binary32 variant stores the pairs rounded
        sh = sh.astype(np.float32).astype(np.float64)
        yh = yh.astype(np.float32).astype(np.float64)
    rho = 1.0 / np.einsum("ij,ij->i", sh, yh)
    Q = rng.normal(size=(n, n))
    P = Q @ Q.T / n + np.eye(n)
    g = rng.normal(size=n)
    return sh, yh, rho, P, g


def _dense_h(sh, yh, rho, gamma, P, head, nh):
    """H after the BFGS inverse updates of the nh newest pairs, oldest first."""
    m, n = sh.shape
    H = gamma * P
    for c in range(nh - 1, -1, -1):
        j = (head - 1 - c) % m
        V = np.eye(n) - rho[j] * np.outer(yh[j], sh[j])
        H = V.T @ H @ V + rho[j] * np.outer(sh[j], sh[j])
    return H


@pytest.mark.parametrize("n,m,head,nh", [(12, 5, 2, 5), (30, 8, 0, 8), (9, 8, 6, 3), (7, 4, 1, 0)])
def test_two_loop_equals_dense_bfgs(n, m, head, nh):
    sh, yh, rho, P, g = _problem(n, m, 100 + n + head)
    gamma = 0.37
    d = O.lbfgs_direction(sh, yh, rho, gamma, P, g, head, nh)
    H = _dense_h(sh, yh, rho, gamma, P, head, nh)
    assert relerr(d, -H @ g) < 1e-12


@pytest.mark.parametrize("n,m,head,nh", [(12, 5, 2, 5), (30, 8, 0, 8), (9, 8, 6, 3), (7, 4, 1, 0)])
def test_two_loop_f32_within_rounding(n, m, head, nh):
    sh, yh, rho, P, g = _problem(n, m, 200 + n + head, f32=True)
    gamma = 0.37
    d32 = O.lbfgs_direction(sh, yh, rho, gamma, P, g, head, nh, f32=True)
    d64 = O.lbfgs_direction(sh, yh, rho, gamma, P, g, head, nh)
    H = _dense_h(sh, yh, rho, gamma, P, head, nh)
    # binary32 unit roundoff 6e-8 times the recursion's length and the
    # conditioning of these pairs (cond(A) ~ 10)
    assert relerr(d32, -H @ g) < 2e-5
    assert relerr(d32, d64) < 2e-5
    assert relerr(d32, d64) > 1e-10  # not silently binary64
    # every component is a binary32 number widened
    assert np.array_equal(d32.astype(np.float32).astype(np.float64), d32)


@pytest.mark.parametrize("f32", [False, True])
def test_secant_equation_newest_pair(f32):
    """H y_newest = s_newest for any H0: with g = y_newest, d = -s_newest."""
    n, m, head, nh = 15, 6, 4, 6
    sh, yh, rho, P, _ = _problem(n, m, 300, f32=f32)
    j = (head - 1) % m
    d = O.lbfgs_direction(sh, yh, rho, 2.5, P, yh[j], head, nh, f32=f32)
    assert relerr(d, -sh[j]) < (2e-5 if f32 else 1e-12)


@pytest.mark.parametrize("dt", [0.01, 0.033])
@pytest.mark.parametrize("spec", ["rod", "ball", "humanoid"])
def test_f32_direction_step_reaches_lm_solution(spec, dt):
    """One stage (Eq. EQ), where L-BFGS converges: the binary32 direction
    reaches Levenberg-Marquardt's solution."""
    s = {"rod": I.rod_chain(1, 4), "ball": I.ball_chain(1, 4, seed=31, radius=0.2),
         "humanoid": I.humanoid(1, seed=33)}[spec]
    om = O.OracleModel.from_spec(s, 0)
    n = om.n_dof
    rng = np.random.default_rng(32)
    qc = rng.uniform(-0.4, 0.4, n)
    qp = qc + rng.normal(0, 0.01, n)
    tau = rng.normal(0, 0.1, n)
    tol = 1e-9
    q_lm, st_lm, _, _ = om.step(1, dt, qp, qc, tau, "lm", 8, tol, 100)
    q32, st32, it32, _ = om.step(1, dt, qp, qc, tau, "lbfgs32", 8, tol, 2000)
    q64, st64, it64, _ = om.step(1, dt, qp, qc, tau, "lbfgs", 8, tol, 2000)
    assert st_lm == 0 and st32 == 0 and st64 == 0
    assert np.max(np.abs(q32 - q_lm)) < 1e-9
    # the rounded direction costs few extra iterations on these problems
    assert it32 <= 1.25 * it64 + 5, (it32, it64)


def test_f32_direction_rollout_matches_lbfgs():
    """20 steps of a swinging rod chain (one stage): binary32 and binary64
    directions give the same trajectory to the solver tolerance."""
    spec = I.rod_chain(1, 3)
    om = O.OracleModel.from_spec(spec, 0)
    q0 = np.array([0.6, -0.2, 0.3])
    dt, n_steps = 0.01, 20
    a = om.rollout(1, dt, q0, q0, np.zeros((n_steps, 3)), "lbfgs", 8, 1e-10, 2000)
    b = om.rollout(1, dt, q0, q0, np.zeros((n_steps, 3)), "lbfgs32", 8, 1e-10, 2000)
    assert a["status"] == 0 and b["status"] == 0
    assert np.max(np.abs(a["traj_cur"] - b["traj_cur"])) < 1e-9
