"""The per-element evaluation bounds the GPU parity tests use: they accept
the oracle's own two evaluations of one point (the O(N^2) path products and
the O(N) Algorithm DERIV path sum in different orders), and they reject an
error in the smallest component that a check normalised by the largest
component would pass."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1709_04145_b300 import inputs as I
from parity_bounds import REL_EVAL, eval_elementwise_errors


def _point(spec, S, rng):
    n = spec.n_dof
    q_cur = rng.uniform(-0.6, 0.6, n)
    q_prev = q_cur + rng.normal(0, 0.02, n)
    tau = rng.normal(0, 0.3, n)
    qs = q_cur[None, :] + rng.normal(0, 0.03, (S, n))
    return qs, q_prev, q_cur, tau


@pytest.mark.parametrize("S", [1, 2, 3])
def test_bounds_accept_the_two_oracle_paths_and_reject_a_small_component_error(S):
    dt = 0.02
    rng = np.random.default_rng(500 + S)
    for spec in (I.rod_chain(2, 3, name="rod3"), I.ball_chain(2, 4, seed=11, radius=0.1),
                 I.humanoid(2, seed=12)):
        for b in range(spec.count):
            om = O.OracleModel.from_spec(spec, b)
            qs, q_prev, q_cur, tau = _point(spec, S, rng)
            _, rf, gf = om.eval_fast(S, dt, qs, q_prev, q_cur, tau)
            er, eg = eval_elementwise_errors(om, S, dt, qs, q_prev, q_cur, tau, rf, gf)
            assert er <= 1e-2 and eg <= 1e-2, (spec.name, b, er, eg)
            # half the old max-normalised tolerance, put on the smallest component
            i = int(np.argmin(np.abs(gf)))
            g_bad = gf.copy()
            g_bad[i] += 0.5 * REL_EVAL * np.max(np.abs(gf))
            j = int(np.argmin(np.abs(rf)))
            r_bad = rf.copy()
            r_bad[j] += 0.5 * REL_EVAL * np.max(np.abs(rf))
            er, eg = eval_elementwise_errors(om, S, dt, qs, q_prev, q_cur, tau, r_bad, g_bad)
            assert er > 1.0 and eg > 1.0, (spec.name, b, er, eg)
