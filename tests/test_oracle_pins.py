"""Pins of the CPU oracle against facts that do not come from the oracle:
quadrature of the body integrals, closed forms, finite differences, a
Newton-Euler reference, invariants and the paper's qualitative claims."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1709_04145_b300 import inputs as I

G = 9.81


def fd(f, x, h=1e-6):
    x = np.asarray(x, dtype=np.float64)
    cols = []
    for k in range(x.size):
        xp = x.copy(); xp.flat[k] += h
        xm = x.copy(); xm.flat[k] -= h
        cols.append((np.asarray(f(xp)) - np.asarray(f(xm))) / (2 * h))
    return np.stack(cols, axis=-1)


def relerr(a, b):
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300)


# ---------------------------------------------------------------- mass moments
def _moment_from_points(pts, wts):
    """int [p;1][p;1]^T dm by quadrature, in the 10-entry layout."""
    P = np.concatenate([pts, np.ones((pts.shape[0], 1))], axis=1)
    M = (P * wts[:, None]).T @ P
    return np.array([M[0, 0], M[0, 1], M[0, 2], M[1, 1], M[1, 2], M[2, 2], M[0, 3], M[1, 3],
                     M[2, 3], M[3, 3]])


def test_rod_moment_equals_gauss_legendre():
    # Eq. ATOM's integral along a uniform rod: 2-point Gauss-Legendre is exact
    # for the quadratic integrand.
    m, L = 1.7, 1.3
    x, w = np.polynomial.legendre.leggauss(2)
    z = -(x + 1) * L / 2
    pts = np.stack([0 * z, 0 * z, z], axis=1)
    ref = _moment_from_points(pts, w * m / 2)
    assert relerr(O.mass_moment_rod(m, L), ref) < 1e-14


def _capsule_quadrature(m, L, r, nq=12):
    """Tensor Gauss-Legendre quadrature over the cylinder and both
    hemispheres in cylindrical/spherical coordinates (exact for the
    polynomial integrands)."""
    x, w = np.polynomial.legendre.leggauss(nq)
    u = (x + 1) / 2
    wu = w / 2
    # azimuth: the uniform rule is exact for the trigonometric polynomials here
    uph = np.arange(nq) / nq
    wph = np.full(nq, 1.0 / nq)
    pts, wts = [], []
    # cylinder: rho in [0, r], phi in [0, 2pi], z in [-L, 0]
    for i in range(nq):
        for j in range(nq):
            for k in range(nq):
                rho, ph, z = r * u[i], 2 * np.pi * uph[j], -L * u[k]
                pts.append([rho * np.cos(ph), rho * np.sin(ph), z])
                wts.append(wu[i] * wph[j] * wu[k] * r * 2 * np.pi * L * rho)
    # hemispheres: s in [0, r], polar angle th in [0, pi/2] from the cap axis
    for zc, sgn in [(0.0, 1.0), (-L, -1.0)]:
        for i in range(nq):
            for j in range(nq):
                for k in range(nq):
                    s, th, ph = r * u[i], np.pi / 2 * u[j], 2 * np.pi * uph[k]
                    pts.append([s * np.sin(th) * np.cos(ph), s * np.sin(th) * np.sin(ph),
                                zc + sgn * s * np.cos(th)])
                    wts.append(wu[i] * wu[j] * wph[k] * r * np.pi / 2 * 2 * np.pi * s * s * np.sin(th))
    pts, wts = np.array(pts), np.array(wts)
    vol = np.pi * r * r * L + 4.0 / 3.0 * np.pi * r ** 3
    return _moment_from_points(pts, wts * m / vol)


@pytest.mark.parametrize("m,L,r", [(1.0, 1.0, 0.05), (0.7, 0.5, 0.3), (2.0, 1.5, 0.15)])
def test_capsule_moment_equals_quadrature(m, L, r):
    assert relerr(O.mass_moment_capsule(m, L, r), _capsule_quadrature(m, L, r)) < 1e-9


def test_capsule_thin_limit_is_rod():
    assert relerr(O.mass_moment_capsule(1.3, 0.9, 1e-7), O.mass_moment_rod(1.3, 0.9)) < 1e-6


def test_product_mass_moments_agree_with_oracle():
    from paper_1709_04145_b300 import models as M
    spec = I.humanoid(4, seed=3)
    got = M.mass_moments(spec)
    for b in range(4):
        assert relerr(got[b], O.mass_moments_from_spec(spec, b)) < 1e-13


# --------------------------------------------------------------- collocation
def test_legendre_roots_closed_forms():
    assert np.allclose(O.legendre_roots(1), [0.0], atol=1e-16)
    assert np.allclose(O.legendre_roots(2), [-1 / np.sqrt(3), 1 / np.sqrt(3)], atol=1e-15)
    assert np.allclose(O.legendre_roots(3), [-np.sqrt(0.6), 0, np.sqrt(0.6)], atol=1e-15)
    for n in range(1, 7):
        assert np.allclose(O.legendre_roots(n), np.polynomial.legendre.leggauss(n)[0], atol=1e-14)


@pytest.mark.parametrize("S", [1, 2, 3, 4, 5])
def test_colloc_weights_differentiate_polynomials(S):
    nodes, W = O.colloc(S)
    K = S + 1
    for p in range(K + 1):
        vals = nodes ** p
        exact = p * (p - 1) * nodes[2:] ** max(p - 2, 0) if p >= 2 else np.zeros(S)
        assert np.allclose(W @ vals, exact, atol=1e-10 * max(1, np.abs(W).max()))
    assert np.allclose(W.sum(axis=1), 0, atol=1e-11)
    assert nodes[-1] == 1.0 and nodes[1] == 0.0
    if S >= 2:
        assert np.isclose(nodes[0], nodes[-2] - 1.0)


def test_colloc_tables_printed_values():
    nodes, W = O.colloc(1)
    assert np.allclose(W, [[1, -2, 1]])
    nodes, W = O.colloc(2)
    assert np.allclose(nodes, [-0.5, 0, 0.5, 1])
    assert np.allclose(W, [[0, 4, -8, 4], [-4, 16, -20, 8]])


# ------------------------------------------------------ joint rotations / FK
@pytest.mark.parametrize("theta", [[0.3, -0.2, 0.1], [1e-3, 2e-3, -1e-3], [0.0, 0.0, 0.0],
                                   [0.4, 0.2, 0.1], [1.2, -0.7, 2.0]])
def test_expmap_derivatives(theta):
    theta = np.array(theta, dtype=np.float64)
    R = O.joint_rot(1, [0, 0, 1], theta)
    assert np.allclose(R @ R.T, np.eye(3), atol=1e-14)
    # exp of a skew matrix by scipy as an independent reference
    from scipy.linalg import expm
    K = np.array([[0, -theta[2], theta[1]], [theta[2], 0, -theta[0]], [-theta[1], theta[0], 0]])
    assert np.allclose(R, expm(K), atol=1e-14)
    for k in range(3):
        dR = O.joint_rot(1, [0, 0, 1], theta, k)
        num = fd(lambda t: O.joint_rot(1, [0, 0, 1], t).reshape(-1), theta)[:, k].reshape(3, 3)
        assert np.max(np.abs(dR - num)) < 1e-8
        for m in range(3):
            ddR = O.joint_rot(1, [0, 0, 1], theta, k, m)
            num2 = fd(lambda t: O.joint_rot(1, [0, 0, 1], t, k).reshape(-1), theta)[:, m].reshape(3, 3)
            assert np.max(np.abs(ddR - num2)) < 1e-7


def test_fk_derivatives_fd():
    spec = I.humanoid(1, seed=7)
    om = O.OracleModel.from_spec(spec, 0)
    q = np.random.default_rng(0).uniform(-0.5, 0.5, om.n_dof)
    for l in [0, 4, 12, 19]:
        dT = om.link_dT(q, l)
        num = fd(lambda x: om.fk(x)[l].reshape(-1), q)
        assert np.max(np.abs(dT.reshape(om.n_dof, 16).T - num)) < 1e-8
        for d, e in [(0, 1), (2, 5), (4, 4), (30, 31)]:
            dd = om.link_ddT(q, l, d, e)
            num2 = fd(lambda x: om.link_dT(x, l)[d].reshape(-1), q)[:, e]
            assert np.max(np.abs(dd.reshape(-1) - num2)) < 1e-7


# ----------------------------------------------------- objective and gradients
def _rod_quadrature_energy(om, spec, q, qc, qp, dt, nq=3):
    """Eq. EQ by quadrature along the rods: rho/(2dt^2)|P - 2P_k + P_k-1|^2 and
    -rho g.P at Gauss-Legendre points of every rod."""
    x, w = np.polynomial.legendre.leggauss(nq)
    T1, T0, Tm = om.fk(q), om.fk(qc), om.fk(qp)
    E = 0.0
    for l in range(spec.n_links):
        L, m = spec.length[0, l], spec.mass[0, l]
        for xi, wi in zip(x, w):
            p = np.array([0, 0, -(xi + 1) * L / 2, 1.0])
            dm = wi * m / 2
            D = (T1[l] - 2 * T0[l] + Tm[l]) @ p
            E += dm * (D[:3] @ D[:3]) / (2 * dt * dt)
            E -= dm * (spec.gravity @ (T1[l] @ p)[:3])
    return E


def test_energy_equals_body_quadrature():
    spec = I.rod_chain(1, 4)
    om = O.OracleModel.from_spec(spec, 0)
    rng = np.random.default_rng(1)
    qc = rng.uniform(-1, 1, 4)
    qp = qc + rng.normal(0, 0.05, 4)
    q = qc + rng.normal(0, 0.05, 4)
    E, *_ = om.eval(1, 0.03, q, qp, qc, np.zeros(4), False)
    assert abs(E - _rod_quadrature_energy(om, spec, q, qc, qp, 0.03)) < 1e-12 * max(1, abs(E))


def test_appendix_a_expansion():
    # Appendix A: the kinetic part of Eq. EQ equals rho/(2dt^2)(I(1,1) - 4I(1,k)
    # + 2I(1,k-1)) + const, with I(a,b) = [T_a^T T_b] : M; the constant is the
    # q-independent 4I(k,k) + I(k-1,k-1) - 4I(k-1,k).
    spec = I.ball_chain(1, 3, seed=4)
    om = O.OracleModel.from_spec(spec, 0)
    mm = O.mass_moments_from_spec(spec, 0)
    rng = np.random.default_rng(2)
    n = om.n_dof
    qc = rng.uniform(-0.5, 0.5, n); qp = qc + rng.normal(0, 0.05, n); q = qc + rng.normal(0, 0.05, n)
    dt = 0.05
    Ek = om.eval(1, dt, q, qp, qc, np.zeros(n), False)[0]
    # remove gravity with a zero-gravity model
    om0 = O.OracleModel(spec.parent, spec.jtype, spec.axis, mm, O.rest_from_spec(spec, 0), np.zeros(3))
    Ek = om0.eval(1, dt, q, qp, qc, np.zeros(n), False)[0]
    T1, T0, Tm = om.fk(q), om.fk(qc), om.fk(qp)

    def Iab(Ta, Tb):
        s = 0.0
        for l in range(spec.n_links):
            v = mm[l]
            M = np.array([[v[0], v[1], v[2], v[6]], [v[1], v[3], v[4], v[7]],
                          [v[2], v[4], v[5], v[8]], [v[6], v[7], v[8], v[9]]])
            A = Ta[l].copy(); A[3] = 0
            Bm = Tb[l].copy(); Bm[3] = 0
            s += np.sum((A.T @ Bm) * M)
        return s
    full = (Iab(T1, T1) + 4 * Iab(T0, T0) + Iab(Tm, Tm) - 4 * Iab(T1, T0) - 4 * Iab(Tm, T0)
            + 2 * Iab(T1, Tm)) / (2 * dt * dt)
    assert abs(Ek - full) < 1e-9 * max(1, abs(full))


@pytest.mark.parametrize("S", [1, 2, 3])
@pytest.mark.parametrize("which", ["rod", "ball", "tree"])
def test_gradient_and_jacobian_fd(S, which):
    spec = {"rod": I.rod_chain(1, 4), "ball": I.ball_chain(1, 3, seed=5, radius=0.1),
            "tree": I.humanoid(1, seed=6)}[which]
    om = O.OracleModel.from_spec(spec, 0)
    n = om.n_dof
    rng = np.random.default_rng(3)
    qc = rng.uniform(-0.5, 0.5, n); qp = qc + rng.normal(0, 0.02, n)
    tau = rng.normal(0, 0.2, n)
    qs = (qc + rng.normal(0, 0.02, (S, n))).reshape(-1)
    dt = 0.033
    E, r, g, J = om.eval(S, dt, qs, qp, qc, tau, True, True)
    gfd = fd(lambda x: om.eval(S, dt, x, qp, qc, tau, False)[0], qs)
    Jfd = fd(lambda x: om.eval(S, dt, x, qp, qc, tau, False)[1], qs)
    assert relerr(g, gfd) < 1e-6
    assert relerr(J, Jfd) < 1e-6
    if S == 1:
        assert relerr(r, g) < 1e-15  # the residual of Eq. PBAD is dE/dq of Eq. EQ
        assert np.allclose(J, J.T, rtol=0, atol=1e-8 * np.abs(J).max())
    Jp, Jc = om.resid_known_jac(S, dt, qs, qp, qc)
    assert relerr(Jp, fd(lambda x: om.eval(S, dt, qs, x, qc, tau, False)[1], qp)) < 1e-6
    assert relerr(Jc, fd(lambda x: om.eval(S, dt, qs, qp, x, tau, False)[1], qc)) < 1e-6


def test_residual_is_pbad_equation_by_quadrature():
    # Eq. PBAD: int dP/dq^T [rho (P - 2P_k + P_k-1)/dt^2 - f] dp with dP/dq
    # from finite differences of point positions (quadrature along rods)
    spec = I.rod_chain(1, 3)
    om = O.OracleModel.from_spec(spec, 0)
    rng = np.random.default_rng(4)
    qc = rng.uniform(-1, 1, 3); qp = qc + rng.normal(0, 0.05, 3); q = qc + rng.normal(0, 0.05, 3)
    dt = 0.02
    x, w = np.polynomial.legendre.leggauss(3)
    res = np.zeros(3)
    T0, Tm = om.fk(qc), om.fk(qp)
    for l in range(3):
        for xi, wi in zip(x, w):
            p = np.array([0, 0, -(xi + 1) * 0.5, 1.0])
            dm = wi / 2
            pos = lambda qq: (om.fk(qq)[l] @ p)[:3]
            J = fd(pos, q)
            acc = (pos(q) - 2 * (T0[l] @ p)[:3] + (Tm[l] @ p)[:3]) / dt ** 2
            res += dm * J.T @ (acc - spec.gravity)
    r = om.eval(1, dt, q, qp, qc, np.zeros(3), False)[1]
    assert relerr(r, res) < 1e-7


def test_mass_matrix_equals_rnea_crba():
    spec = I.rod_chain(1, 5)
    om = O.OracleModel.from_spec(spec, 0)
    q = np.random.default_rng(5).uniform(-1, 1, 5)
    H = om.hmass(q)
    om0 = O.OracleModel(spec.parent, spec.jtype, spec.axis, O.mass_moments_from_spec(spec, 0),
                        O.rest_from_spec(spec, 0), np.zeros(3))
    Mcol = np.stack([om0.rnea(q, np.zeros(5), e) for e in np.eye(5)], axis=1)
    assert relerr(H, Mcol) < 1e-12


def test_rnea_gravity_is_potential_gradient():
    spec = I.rod_chain(1, 4)
    om = O.OracleModel.from_spec(spec, 0)
    q = np.random.default_rng(6).uniform(-1, 1, 4)
    tau_g = om.rnea(q, np.zeros(4), np.zeros(4))  # = dV/dq

    def V(qq):
        T = om.fk(qq)
        return -sum(spec.mass[0, l] * spec.gravity @ (T[l] @ np.array([0, 0, -0.5, 1]))[:3]
                    for l in range(4))
    assert relerr(tau_g, fd(V, q)) < 1e-8


# ----------------------------------------------------------------- dynamics
def test_single_pendulum_small_angle_period():
    # uniform rod about one end: T = 2 pi sqrt(2 L / (3 g)) = 1.637947 s
    spec = I.rod_chain(1, 1)
    om = O.OracleModel.from_spec(spec, 0)
    dt = 1e-3
    n = 2600
    q0 = np.array([1e-3])
    res = om.rollout(1, dt, q0, q0, np.zeros((n, 1)), "lbfgs", 5, 1e-12)
    x = np.concatenate([[1e-3], res["traj_cur"][:, 0]])
    t = np.arange(n + 1) * dt
    idx = np.where(np.sign(x[:-1]) != np.sign(x[1:]))[0]
    zc = t[idx] - x[idx] * dt / (x[idx + 1] - x[idx])
    period = 2 * (zc[1] - zc[0])
    exact = 2 * np.pi * np.sqrt(2 * 1.0 / (3 * G))
    assert abs(exact - 1.637947) < 1e-6
    assert abs(period - exact) / exact < 1e-3


@pytest.mark.parametrize("S", [1, 2, 3])
def test_rest_invariance(S):
    spec = I.ball_chain(1, 4, seed=9, radius=0.1)
    mm = O.mass_moments_from_spec(spec, 0)
    om0 = O.OracleModel(spec.parent, spec.jtype, spec.axis, mm, O.rest_from_spec(spec, 0), np.zeros(3))
    q = np.random.default_rng(7).uniform(-0.5, 0.5, om0.n_dof)
    res = om0.rollout(S, 0.05, q, q, np.zeros((20, om0.n_dof)), "lbfgs", 8, 1e-10)
    assert res["status"] == 0 and np.array_equal(res["traj_cur"][-1], q)
    om = O.OracleModel.from_spec(spec, 0)  # hanging straight down under gravity
    z = np.zeros(om.n_dof)
    res = om.rollout(S, 0.05, z, z, np.zeros((20, om.n_dof)), "lbfgs", 8, 1e-10)
    assert np.array_equal(res["traj_cur"][-1], z)


@pytest.mark.parametrize("N,S", [(5, 1), (3, 2), (2, 3)])
def test_lbfgs_and_lm_agree(N, S):
    spec = I.rod_chain(1, N)
    om = O.OracleModel.from_spec(spec, 0)
    rng = np.random.default_rng(8)
    qc = rng.uniform(-0.8, 0.8, N); qp = qc - 0.01 * rng.normal(size=N)
    a, sa, *_ = om.step(S, 0.02, qp, qc, np.zeros(N), "lbfgs", 8, 1e-10, 5000)
    b, sb, *_ = om.step(S, 0.02, qp, qc, np.zeros(N), "lm", 8, 1e-10)
    assert sa == 0 and sb == 0
    assert np.max(np.abs(a - b)) < 1e-9


def _order(S):
    spec = I.rod_chain(1, 2)
    om = O.OracleModel.from_spec(spec, 0)
    q0 = np.array([0.6, -0.4])
    t_end = 0.4
    qref, _ = om.rk4(q0, np.zeros(2), np.zeros(2), 1e-4, int(round(t_end / 1e-4)))
    errs = []
    dts = [0.02, 0.01, 0.005]
    for dt in dts:
        nodes, _ = O.colloc(S)
        # start from rest: q_prev at node k-1+alpha from the RK4 solution
        qp = q0 if S == 1 else om.rk4(q0, np.zeros(2), np.zeros(2), 1e-5,
                                      int(round(-nodes[0] * dt / 1e-5)))[0]
        steps = int(round(t_end / dt))
        res = om.rollout(S, dt, qp, q0, np.zeros((steps, 2)), "lm", 8, 1e-11)
        errs.append(np.max(np.abs(res["q_cur"] - qref)))
    return np.polyfit(np.log(dts), np.log(errs), 1)[0]


def test_convergence_order_vs_newton_euler_rk4():
    # Section 6.1: a K-th order position-based collocation behaves like RK of
    # order K-1; K = 2 (one stage) is first order.
    assert 0.8 < _order(1) < 1.4
    assert _order(2) > 1.6


def test_second_order_dissipates_more_than_third():
    # Fig. SWING: K = 2 loses energy quickly, K = 3 preserves it much better.
    spec = I.rod_chain(1, 3)
    om = O.OracleModel.from_spec(spec, 0)
    q0 = np.array([1.2, 0.0, 0.0])
    dt, n = 0.01, 150

    def energy(qp, qc, h):
        qm = 0.5 * (qp + qc)
        v = (qc - qp) / h
        T = om.fk(qm)
        V = -sum(spec.gravity @ (T[l] @ np.array([0, 0, -0.5, 1]))[:3] for l in range(3))
        return 0.5 * v @ om.hmass(qm) @ v + V

    E0 = energy(q0, q0, 1.0)
    out = {}
    for S in [1, 2]:
        nodes, _ = O.colloc(S)
        res = om.rollout(S, dt, q0, q0, np.zeros((n, 3)), "lm", 8, 1e-10)
        h = -nodes[0] * dt
        out[S] = abs(energy(res["traj_prev"][-1], res["traj_cur"][-1], h) - E0)
    assert out[2] < 0.5 * out[1]


# ------------------------------------------------------------------- adjoint
def test_step_adjoint_matches_finite_differences():
    spec = I.rod_chain(1, 3)
    om = O.OracleModel.from_spec(spec, 0)
    rng = np.random.default_rng(9)
    S, dt = 2, 0.02
    qc = rng.uniform(-0.5, 0.5, 3); qp = qc - 0.01 * rng.normal(size=3)
    tau = rng.normal(0, 0.1, 3)
    gbar = rng.normal(size=(S * 3))

    def L(qp_, qc_, tau_):
        qs, st, *_ = om.step(S, dt, qp_, qc_, tau_, "lm", 8, 1e-13)
        return gbar @ qs.reshape(-1)
    qs, *_ = om.step(S, dt, qp, qc, tau, "lm", 8, 1e-13)
    gp, gc, gt = om.step_adjoint(S, dt, qp, qc, tau, qs, gbar)
    h = 1e-6
    assert relerr(gp, fd(lambda x: L(x, qc, tau), qp, h)) < 1e-5
    assert relerr(gc, fd(lambda x: L(qp, x, tau), qc, h)) < 1e-5
    assert relerr(gt, fd(lambda x: L(qp, qc, x), tau, h)) < 1e-5


@pytest.mark.parametrize("k", [None, 0, 2])
def test_expmap_continuous_across_series_switch(k):
    """The oracle's exponential map switches from its power series to closed
    forms at |theta| = 0.5: R, dR and d2R just below and just above agree to
    rounding (a dropped or wrong low-order series term would show as a jump)."""
    u = np.array([0.6, -0.48, 0.64])  # unit direction
    lo, hi = 0.5 * (1 - 1e-14) * u, 0.5 * (1 + 1e-14) * u
    assert np.linalg.norm(lo) < 0.5 <= np.linalg.norm(hi)
    args = () if k is None else (k,)
    a, b = O.joint_rot(1, [0, 0, 1], lo, *args), O.joint_rot(1, [0, 0, 1], hi, *args)
    assert np.max(np.abs(a - b)) < 1e-13
    if k is not None:
        a2 = O.joint_rot(1, [0, 0, 1], lo, k, 1)
        b2 = O.joint_rot(1, [0, 0, 1], hi, k, 1)
        assert np.max(np.abs(a2 - b2)) < 1e-12
