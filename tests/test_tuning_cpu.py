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


def test_worse_status_order():
    import torch

    from paper_1709_04145_b300.autograd import worse_status
    order = [0, 5, 1, 2, 3, 4]
    a = torch.tensor([x for x in order for _ in order], dtype=torch.int32)
    b = torch.tensor([y for _ in order for y in order], dtype=torch.int32)
    got = worse_status(a, b).tolist()
    want = [order[max(i, j)] for i in range(6) for j in range(6)]
    assert got == want


def test_pick_mapping_fastest_then_stage_then_fewer_threads():
    from paper_1709_04145_b300.tuning import MappingTrial, pick_mapping
    inf = float("inf")
    t = [MappingTrial(0, 32, 10.0), MappingTrial(1, 32, 6.0), MappingTrial(1, 64, 6.0),
         MappingTrial(0, 64, 9.0), MappingTrial(1, 128, inf)]
    assert pick_mapping(t) == (1, 32)
    t = [MappingTrial(1, 32, 5.0), MappingTrial(0, 64, 5.0)]
    assert pick_mapping(t) == (0, 64)
    t = [MappingTrial(1, 32, inf), MappingTrial(0, 128, 7.0)]
    assert pick_mapping(t) == (0, 128)
    import pytest
    with pytest.raises(ValueError):
        pick_mapping([MappingTrial(1, 32, inf)])


def test_choose_bucket_mappings_greedy():
    """Each bucket is switched to the link mapping only where the launch gets
    faster; refused candidates (inf) stay stage-mapped."""
    from paper_1709_04145_b300.tuning import choose_bucket_mappings
    inf = float("inf")
    # bucket 0 refused, bucket 1 helps, bucket 2 hurts once 1 is link-mapped
    table = {(0, 0, 0): 10.0, (1, 0, 0): inf, (0, 1, 0): 7.0, (0, 1, 1): 8.0}
    calls = []

    def time_fn(m):
        calls.append(tuple(m))
        return table[tuple(m)]

    chosen, trials = choose_bucket_mappings(3, time_fn)
    assert chosen == [0, 1, 0]
    assert trials == [(10.0, inf), (10.0, 7.0), (7.0, 8.0)]
    assert calls == [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 1, 1)]
    chosen, _ = choose_bucket_mappings(2, lambda m: 5.0)
    assert chosen == [0, 0]  # ties keep the stage mapping


def test_newton_cta_candidates():
    from paper_1709_04145_b300.tuning import newton_cta_candidates
    assert newton_cta_candidates([68, 90, 68]) == [4097, 90, 68]
    assert newton_cta_candidates([5000, 800]) == [4097, 800]  # above 4096: never CTA
    assert newton_cta_candidates([]) == [4097]


def test_pick_threads_prefers_small_blocks_on_near_ties():
    from paper_1709_04145_b300.tuning import pick_threads
    assert pick_threads({32: 391.0, 64: 391.7, 128: 388.4}) == 32  # within 1%
    assert pick_threads({32: 400.0, 64: 391.7, 128: 380.0}) == 128
    assert pick_threads({32: float("inf"), 64: 10.0, 128: 10.05}) == 64
