"""Host logic of the benchmark's reporting, on the CPU: the per-step outcome
record, the status names against the library's codes, and the algorithmic
flop count that the roofline divides by the kernel time."""
import numpy as np
import torch

import bench
import paper_1709_04145_b300 as P
from paper_1709_04145_b300 import inputs as I


def test_status_names_follow_the_library_codes():
    assert tuple(P.STATUS[k] for k in range(len(bench.STATUS_NAMES))) == bench.STATUS_NAMES


def test_step_outcomes_of_a_synthetic_log():
    # 3 steps x 4 instances: statuses and exit |r| chosen by hand
    st = torch.tensor([[0, 5, 1, 2], [0, 0, 4, 2], [5, 0, 1, 3]], dtype=torch.int32)
    rn = torch.tensor([[1e-9, 2e-9, 5.0, 7.0], [3e-9, 1e-9, float("nan"), 8.0],
                       [4e-9, 2e-9, 6.0, float("inf")]], dtype=torch.float64)
    rec = bench.step_outcomes({"step_status": st, "step_rnorm": rn})
    assert rec["instance_steps"] == 12
    assert rec["fractions"] == {"CONVERGED": 4 / 12, "MAX_ITER": 2 / 12, "LS_FAIL": 2 / 12,
                                "CHOL_FAIL": 1 / 12, "NONFINITE": 1 / 12, "STALLED": 2 / 12}
    assert rec["solved_fraction"] == 6 / 12
    finite = np.array([1e-9, 2e-9, 5.0, 7.0, 3e-9, 1e-9, 8.0, 4e-9, 2e-9, 6.0])
    assert rec["exit_rnorm_median"] == float(np.median(finite))
    assert rec["exit_rnorm_max"] == 8.0 and rec["exit_rnorm_nonfinite"] == 2
    # one bucket's slice of the instances
    rec1 = bench.step_outcomes({"step_status": st, "step_rnorm": rn}, slice(0, 2))
    assert rec1["instance_steps"] == 6 and rec1["solved_fraction"] == 1.0


def test_rollout_flops_are_linear_in_the_counters():
    spec = I.ball_chain(2, 10, seed=1)
    S, m = 3, 8
    one = lambda a: np.array([a, 0])
    # one residual pass of a ten-link ball chain at three stages: 3 x 10 x (540 + 24 x 3)
    assert bench.rollout_flops(spec, S, m, one(1), one(0), one(0)) == 3 * 10 * (540 + 72)
    # one tangent pass: 3 x 10 x (680 + 72); one L-BFGS iteration: S n (8 m + 26 + 2 S)
    assert bench.rollout_flops(spec, S, m, one(0), one(1), one(0)) == 3 * 10 * (680 + 72)
    assert bench.rollout_flops(spec, S, m, one(0), one(0), one(1)) == S * 30 * (8 * m + 26 + 2 * S)
    ev, gr, it = np.array([137, 140]), np.array([17, 18]), np.array([15, 16])
    total = bench.rollout_flops(spec, S, m, ev, gr, it)
    parts = sum(bench.rollout_flops(spec, S, m, ev * (k == 0), gr * (k == 1), it * (k == 2))
                for k in range(3))
    assert total == parts
    # one stage: the gradient is the residual (no tangent pass), the energy terms are added
    hinge = I.rod_chain(1, 4, name="rod4")
    assert bench.rollout_flops(hinge, 1, 5, np.array([1]), np.array([1]), np.array([0])) == \
        4 * (347 + 24 + 54)
