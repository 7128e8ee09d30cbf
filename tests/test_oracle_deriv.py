"""Pin of the oracle's O(N) Algorithm DERIV path (tree form, Section 5)
against the brute-force derivative along root-to-link paths, an independent
O(N^2) computation: sum_l <G_l, dT_l/dq> for random seeds G, on chains of
hinges and balls, a humanoid tree and a free root (translation + ball), and
the stage residual of Eq. HOC recovered from its own seeds."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1709_04145_b300 import inputs as I


def relerr(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def _brute(om, q, G):
    r = np.zeros(om.n_dof)
    for l in range(om.n_links):
        dT = om.link_dT(q, l)  # (n, 4, 4)
        r += np.einsum("dij,ij->d", dT[:, :3, :], G[l])
    return r


@pytest.mark.parametrize("which", ["rod", "ball", "humanoid", "free"])
def test_deriv_equals_path_derivative(which):
    spec = {"rod": I.rod_chain(1, 7), "ball": I.ball_chain(1, 6, seed=41, radius=0.1),
            "humanoid": I.humanoid(1, seed=42), "free": I.free_chain(1, 4)}[which]
    om = O.OracleModel.from_spec(spec, 0)
    rng = np.random.default_rng(43)
    for _ in range(3):
        q = rng.uniform(-0.7, 0.7, om.n_dof)
        G = rng.normal(size=(om.n_links, 3, 4))
        assert relerr(om.deriv(q, G), _brute(om, q, G)) < 1e-12


def test_deriv_is_linear_in_the_seeds_and_zero_for_zero_seeds():
    om = O.OracleModel.from_spec(I.humanoid(1, seed=44), 0)
    rng = np.random.default_rng(45)
    q = rng.uniform(-0.5, 0.5, om.n_dof)
    G1, G2 = rng.normal(size=(2, om.n_links, 3, 4))
    assert np.array_equal(om.deriv(q, np.zeros_like(G1)), np.zeros(om.n_dof))
    r = om.deriv(q, 2.0 * G1 - 3.0 * G2)
    assert relerr(r, 2.0 * om.deriv(q, G1) - 3.0 * om.deriv(q, G2)) < 1e-12


@pytest.mark.parametrize("S", [2, 3])
def test_deriv_reproduces_stage_residual(S):
    """r_i of Eq. HOC is DERIV at q_i with the seeds (sum_j W_ij T_l(q_j)) M_l
    - g [m c; m]^T, minus tau (no drag or contact)."""
    spec = I.ball_chain(1, 4, seed=46, radius=0.15)
    om = O.OracleModel.from_spec(spec, 0)
    n = om.n_dof
    rng = np.random.default_rng(47)
    dt = 0.02
    qc = rng.uniform(-0.4, 0.4, n)
    qp = qc + rng.normal(0, 0.02, n)
    qs = qc[None, :] + rng.normal(0, 0.02, (S, n))
    tau = rng.normal(0, 0.1, n)
    _, r, _, _ = om.eval(S, dt, qs.reshape(-1), qp, qc, tau, False)
    nodes, W = O.colloc(S)
    Ts = [om.fk(x) for x in [qp, qc] + list(qs)]          # nodes: prev, cur, stages
    mm = O.mass_moments_from_spec(spec, 0)                  # (N, 10)
    g = np.array(spec.gravity, dtype=float) if hasattr(spec, "gravity") else np.array([0, 0, -9.81])
    for i in range(S):
        G = np.zeros((om.n_links, 3, 4))
        for l in range(om.n_links):
            s = mm[l]
            M = np.array([[s[0], s[1], s[2], s[6]], [s[1], s[3], s[4], s[7]],
                          [s[2], s[4], s[5], s[8]], [s[6], s[7], s[8], s[9]]])
            A = sum(W[i, j] / dt ** 2 * Ts[j][l][:3, :] for j in range(S + 2))
            G[l] = A @ M - np.outer(g, s[6:10])
        ri = om.deriv(qs[i], G) - tau
        assert relerr(ri, r[i * n:(i + 1) * n]) < 1e-10, i


@pytest.mark.parametrize("S", [1, 2, 3, 4])
def test_o_n_evaluation_equals_brute_force(S):
    """The O(N) evaluation the CPU baseline times (Algorithm DERIV for the
    stage residuals and its tangent for the Eq. EQHOC gradient) gives the
    brute-force evaluation's E, r and dE/dq on chains, a tree and a free
    root, with drag."""
    rng = np.random.default_rng(40 + S)
    specs = [I.rod_chain(2, 5, name="rod5"), I.ball_chain(2, 6, seed=3, radius=0.15),
             I.humanoid(2, seed=4), I.free_chain(2, 4, name="free4")]
    for spec in specs:
        for drag in (0.0, 0.4):
            om = O.OracleModel.from_spec(spec, 1, drag=drag)
            n = spec.n_dof
            qc = rng.uniform(-0.6, 0.6, n)
            qp = qc + rng.normal(0, 0.02, n)
            qs = qc[None] + rng.normal(0, 0.03, (S, n))
            tau = rng.normal(0, 0.3, n)
            E, r, g, _ = om.eval(S, 0.033, qs, qp, qc, tau, True)
            Ef, rf, gf = om.eval_fast(S, 0.033, qs, qp, qc, tau)
            assert abs(E - Ef) <= 1e-12 * abs(E), (spec.name, drag)
            assert np.max(np.abs(r - rf)) <= 1e-12 * np.max(np.abs(r)), (spec.name, drag)
            assert np.max(np.abs(g - gf)) <= 1e-12 * np.max(np.abs(g)), (spec.name, drag)


def test_o_n_lbfgs_rollout_follows_brute_force():
    """The oracle's L-BFGS with the O(N) evaluation takes the same steps as
    with the brute-force one (the evaluations agree to rounding)."""
    w = I.pendulum3()
    spec = w["spec"]
    om = O.OracleModel.from_spec(spec, 0)
    q0 = w["q0"][0]
    ref = om.rollout(1, w["dt"], q0, q0, np.zeros((30, 3)), "lbfgs", 5, w["tol"], 1000)
    om.set_fast(True)
    fast = om.rollout(1, w["dt"], q0, q0, np.zeros((30, 3)), "lbfgs", 5, w["tol"], 1000)
    assert ref["status"] == fast["status"] == 0
    assert np.max(np.abs(ref["traj_cur"] - fast["traj_cur"])) <= 1e-9
