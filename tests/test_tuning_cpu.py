"""Host logic of the per-bucket solver choice (no GPU)."""
import math

from paper_1709_04145_b300.tuning import ProbeResult, pick

LBFGS, NEWTON = 0, 1


def test_pick_prefers_less_time_per_converged_step():
    a = ProbeResult(LBFGS, ms=100.0, converged=10, total=20)   # 10 ms per converged step
    b = ProbeResult(NEWTON, ms=60.0, converged=20, total=20)   # 3 ms per converged step
    assert pick([a, b]) == NEWTON
    a = ProbeResult(LBFGS, ms=10.0, converged=20, total=20)
    assert pick([a, b]) == LBFGS


def test_pick_when_nothing_converges():
    a = ProbeResult(LBFGS, ms=10.0, converged=0, total=20)
    b = ProbeResult(NEWTON, ms=50.0, converged=0, total=20)
    assert math.isinf(a.ms_per_converged)
    assert pick([a, b]) == LBFGS  # fastest
    c = ProbeResult(NEWTON, ms=50.0, converged=1, total=20)
    assert pick([a, c]) == NEWTON  # any convergence beats none


def test_pick_ties_go_to_lbfgs():
    a = ProbeResult(LBFGS, ms=20.0, converged=10, total=10)
    b = ProbeResult(NEWTON, ms=20.0, converged=10, total=10)
    assert pick([b, a]) == LBFGS
