"""The evaluation entry point whose scratch is a fixed device array of the
library (for callers that cannot allocate device memory when they evaluate)
must give the results of the batch entry point. Collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

from paper_1709_04145_b300 import inputs as I

pytestmark = pytest.mark.gpu

REL_EVAL = 1e-10  # the tolerance of the evaluation parity tests


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _case(spec, S, seed, dev):
    import torch
    rng = np.random.default_rng(seed)
    B, n = spec.count, spec.n_dof
    q_cur = rng.uniform(-0.6, 0.6, size=(B, n))
    q_prev = q_cur + rng.normal(0, 0.02, size=(B, n))
    tau = rng.normal(0, 0.3, size=(B, n))
    qs = q_cur[:, None, :] + rng.normal(0, 0.03, size=(B, S, n))
    t = lambda a: torch.tensor(np.ascontiguousarray(a).reshape(-1), device=dev)
    return t(q_prev), t(q_cur), t(tau), t(qs)


@pytest.mark.parametrize("S", [1, 3])
def test_static_scratch_matches_batch_entry_point(S):
    import torch

    import paper_1709_04145_b300 as P
    from paper_1709_04145_b300._native import lib
    dev = torch.device("cuda:0")
    spec = I.ball_chain(45, 4, seed=5, radius=0.1)
    model = P.Model.from_spec(spec)
    batch = P.Batch([model], max_stages=S, max_history=0)
    L = lib()
    for call in range(2):  # two calls in a row: the shared scratch keeps stale contents
        q_prev, q_cur, tau, qs = _case(spec, S, 70 + call, dev)
        E_ref, g_ref, r_ref = P.eval_objective_grad(batch, qs, q_prev, q_cur, tau, 0.02, S)
        E = torch.empty(spec.count, dtype=torch.float64, device=dev)
        g = torch.empty(S * batch.D, dtype=torch.float64, device=dev)
        r = torch.empty_like(g)
        stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info(dev)[0]
        rc = L.pbad_eval_objective_grad_static(model._h, _ptr(qs), _ptr(q_prev), _ptr(q_cur),
                                               _ptr(tau), 0.02, S, _ptr(E), _ptr(g), _ptr(r),
                                               stream)
        assert rc == 0, L.pbad_last_error()
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info(dev)[0]
        if call == 1:
            # the first call in a process may load the library's device code
            # (which brings the static array); a later call allocates nothing
            assert free_after == free_before, (free_before, free_after)
        for got, ref in ((E, E_ref), (g, g_ref), (r, r_ref)):
            got, ref = got.cpu().numpy(), ref.cpu().numpy()
            assert np.max(np.abs(got - ref)) <= REL_EVAL * np.max(np.abs(ref))


def test_static_scratch_rejects_oversized_problem():
    import torch

    import paper_1709_04145_b300 as P
    from paper_1709_04145_b300._native import lib
    dev = torch.device("cuda:0")
    spec = I.ball_chain(20000, 10, seed=6, radius=0.1)
    model = P.Model.from_spec(spec)
    n = spec.count * spec.n_dof
    x = torch.zeros(3 * n, dtype=torch.float64, device=dev)
    E = torch.empty(spec.count, dtype=torch.float64, device=dev)
    L = lib()
    rc = L.pbad_eval_objective_grad_static(model._h, _ptr(x), _ptr(x), _ptr(x), None, 0.02, 3,
                                           _ptr(E), _ptr(x), None, None)
    assert rc == -1
    msg = L.pbad_last_error().decode()
    assert "scratch" in msg and "bytes" in msg
