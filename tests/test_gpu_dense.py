"""pbad_damped_gram_solve (the LM iteration's damped system, Section 5)
against its plain definition: H = J^T J, the Cholesky factor of
H + lambda I and dl = -(H + lambda I)^-1 g, computed here with numpy in
binary64. Sizes span one tile, several 64 x 64 tiles and ragged edges."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

EPS = np.finfo(float).eps


def _case(count, n, seed, lam):
    import torch
    import paper_1709_04145_b300 as P
    rng = np.random.default_rng(seed)
    J = rng.normal(size=(count, n, n)) + 3.0 * np.eye(n)  # J[b, c] = column c of J_b
    g = rng.normal(size=(count, n))
    dev = torch.device("cuda:0")
    H, L, dl, st = P.damped_gram_solve(torch.tensor(J, device=dev), torch.tensor(g, device=dev), lam)
    torch.cuda.synchronize()
    return J, g, H.cpu().numpy(), L.cpu().numpy(), dl.cpu().numpy(), st.cpu().numpy()


@pytest.mark.parametrize("n", [1, 37, 64, 150, 300])
def test_damped_gram_solve_matches_definition(n):
    lam = 1e-3
    J, g, H, L, dl, st = _case(3, n, 40 + n, lam)
    assert np.all(st == 0)
    for b in range(J.shape[0]):
        Jm = J[b].T  # rows: residual components
        Href = Jm.T @ Jm
        # forward error bound of a length-n dot product: n eps sum |a_k b_k|
        bound = 2 * n * EPS * (np.abs(Jm).T @ np.abs(Jm))
        assert np.all(np.abs(H[b] - Href) <= bound), b
        A = Href + lam * np.eye(n)
        Lref = np.linalg.cholesky(A)
        Lg = np.tril(L[b].T)  # stored column-major: L[b, c, r] = L[r][c]
        kappa = np.linalg.cond(A)
        assert np.max(np.abs(Lg - Lref)) <= 10 * n * EPS * np.sqrt(kappa) * np.max(np.abs(Lref)), b
        ref = np.linalg.solve(A, -g[b])
        assert np.max(np.abs(dl[b] - ref)) <= 10 * n * EPS * kappa * np.max(np.abs(ref)), b


def test_damped_gram_solve_reports_indefinite_systems():
    """lambda below minus the largest eigenvalue of J^T J: the first pivot is
    negative, the instance ends CHOL_FAIL; the others still solve."""
    import torch
    import paper_1709_04145_b300 as P
    rng = np.random.default_rng(7)
    n = 70
    J = 0.1 * rng.normal(size=(2, n, n)) + 3.0 * np.eye(n)  # instance 0: eig(J^T J) > 1
    J[1] *= 1e-3  # instance 1: J^T J tiny, so H - 1 I is negative definite
    g = rng.normal(size=(2, n))
    dev = torch.device("cuda:0")
    lam = -1.0
    H, L, dl, st = P.damped_gram_solve(torch.tensor(J, device=dev), torch.tensor(g, device=dev), lam)
    st = st.cpu().numpy()
    assert P.STATUS[int(st[1])] == "CHOL_FAIL"
    Jm = J[0].T
    A = Jm.T @ Jm + lam * np.eye(n)
    assert np.linalg.eigvalsh(A).min() > 0
    assert st[0] == 0
    ref = np.linalg.solve(A, -g[0])
    kappa = np.linalg.cond(A)
    got = dl.cpu().numpy()[0]
    assert np.max(np.abs(got - ref)) <= 10 * n * EPS * kappa * np.max(np.abs(ref))


def test_damped_gram_solve_arguments():
    import torch
    import paper_1709_04145_b300 as P
    from paper_1709_04145_b300._native import PBADError
    dev = torch.device("cuda:0")
    J = torch.zeros((0, 5, 5), dtype=torch.float64, device=dev)
    g = torch.zeros((0, 5), dtype=torch.float64, device=dev)
    _, _, _, st = P.damped_gram_solve(J, g, 1.0)  # count 0: nothing launched
    assert st.numel() == 0
    J = torch.eye(3, dtype=torch.float64, device=dev)[None]
    g = torch.ones((1, 3), dtype=torch.float64, device=dev)
    with pytest.raises(PBADError):
        P.damped_gram_solve(J, g, float("nan"))
    H, L, dl, st = P.damped_gram_solve(J, g, 1.0)  # (I + I) dl = -1
    assert st.item() == 0
    assert np.allclose(dl.cpu().numpy(), -0.5, rtol=0, atol=1e-15)
