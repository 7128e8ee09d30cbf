"""Per-element bounds for comparing one evaluation of the CUDA path with the
oracle's (Eq. EQ for one stage, Eq. EQHOC for several).

A check normalised by the largest component lets a small component carry an
error as large as 1e-10 of the largest one. These bounds hold each component
to 1e-10 of itself, plus an absolute floor derived from the binary64
rounding of the quantity:

- stage residual r_k: REL |r_k| + 2 floor, where floor is the oracle's
  bound on the rounding error of r (om_floor: eps times the magnitudes of
  the terms that cancel in Eq. HOC), once per side;
- gradient for one stage: the gradient is r itself (Eq. PBAD), same bound;
- gradient for several stages, 2 Jr^T r: component i moves by at most
  2 sum_k |Jr_ki| |dr_k| when every r_k moves by dr_k, so its floor is
  4 floor sum_k |Jr_ki| (both sides' r within floor), with Jr the oracle's
  dense residual Jacobian at the same point.
"""
import numpy as np

REL_EVAL = 1e-10


def oracle_eval_bounds(om, S, dt, qs, q_prev, q_cur, tau):
    """The oracle's (E, r, grad) at one point with the per-element bounds of
    r and of the gradient."""
    Eo, ro, go, J = om.eval(S, dt, np.asarray(qs).reshape(-1), q_prev, q_cur, tau, True, S > 1)
    fl = om.floor(S, dt)
    r_bound = REL_EVAL * np.abs(ro) + 2.0 * fl
    if S == 1:
        g_bound = REL_EVAL * np.abs(go) + 2.0 * fl
    else:
        g_bound = REL_EVAL * np.abs(go) + 4.0 * fl * np.abs(J).sum(axis=0)
    return Eo, ro, go, r_bound, g_bound


def ratio(got, ref, bound):
    """Largest |got - ref| / bound over the components (<= 1 passes)."""
    got = np.asarray(got, dtype=np.float64).reshape(-1)
    return float(np.max(np.abs(got - ref) / bound))


def eval_elementwise_errors(om, S, dt, qs, q_prev, q_cur, tau, resid, grad):
    """Largest ratios of the residual's and the gradient's component errors
    to their bounds; resid / grad are the (S n) vectors of one instance."""
    _, ro, go, rb, gb = oracle_eval_bounds(om, S, dt, qs, q_prev, q_cur, tau)
    return ratio(resid, ro, rb), ratio(grad, go, gb)
