"""Failure paths on the GPU, without faulting, trapping or hanging it.

- divergence (relative residual above 1e10, Sec. 5) and the iteration limit are
  reported as status codes with the history so far, like the oracle;
- a bounded device-side wait that can never be satisfied (a row of the
  triangular factor that waits for itself: a flag nothing sets) expires after
  about a second, the call returns PMG_ERR_TIMEOUT, and the CUDA context stays
  usable for the next solve.
"""
import time

import numpy as np
import pytest

from paper_1901_01685_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def pmg():
    from paper_1901_01685_gb300 import pmg as P
    P.lib()
    return P


def test_divergence_is_reported_like_the_oracle(torch_mod, pmg, oracle_mod):
    torch = torch_mod
    # dropping every off-diagonal ILUT entry leaves a diagonal smoother: the cycle diverges
    S = pmg.Solver(0, 3, 4, drop_tol=1e30)
    O = oracle_mod.Hierarchy(0, 3, 4, tau=1e30)
    f = O.rhs()
    u0 = inputs.initial_guess(O.N[0], 1)
    u, it, hist, st = S.solve(torch.as_tensor(f, device="cuda"), torch.as_tensor(u0, device="cuda"),
                              max_iter=100, allow=(pmg.PMG_ERR_DIVERGED,))
    _, ho, ito, sto = O.solve(f, u0, 1e-8, 100)
    assert st == pmg.PMG_ERR_DIVERGED and sto == "diverged"
    assert abs(it - ito) <= 1 and hist[-1] > 1e10
    m = min(it, ito)
    assert np.all(np.abs(hist[:m] - ho[:m]) <= 1e-10 * np.maximum(1.0, ho[:m]))


def test_iteration_limit_is_reported(torch_mod, pmg, oracle_mod):
    torch = torch_mod
    S = pmg.Solver(0, 3, 5)
    O = oracle_mod.Hierarchy(0, 3, 5)
    f = O.rhs()
    u0 = inputs.initial_guess(O.N[0], 1)
    u, it, hist, st = S.solve(torch.as_tensor(f, device="cuda"), torch.as_tensor(u0, device="cuda"),
                              rel_tol=1e-30, max_iter=1, allow=(pmg.PMG_ERR_MAXITER,))
    _, ho, _, _ = O.solve(f, u0, 1e-30, 1)
    assert st == pmg.PMG_ERR_MAXITER and it == 1
    assert abs(hist[0] - ho[0]) <= 1e-12


def test_expired_wait_returns_timeout_and_context_survives(torch_mod, pmg, oracle_mod):
    torch = torch_mod
    n = 4
    # row 2 lists itself as a dependency: its ready flag is never set by anyone
    rp = torch.tensor([0, 0, 1, 3, 4], dtype=torch.int32, device="cuda")
    ci = torch.tensor([0, 0, 2, 2], dtype=torch.int32, device="cuda")
    v = torch.tensor([0.5, 0.25, 0.125, 0.5], dtype=torch.float64, device="cuda")
    b = torch.ones(n, dtype=torch.float64, device="cuda")
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    t0 = time.time()
    with pytest.raises(pmg.PmgError) as e:
        pmg.pmg_lsolve_noalloc(n, rp, ci, v, b, y)
    assert e.value.status == pmg.PMG_ERR_TIMEOUT
    assert time.time() - t0 < 30
    # the context is still usable: a regular solve right after matches the oracle
    S = pmg.Solver(1, 2, 4)
    O = oracle_mod.Hierarchy(1, 2, 4)
    f = O.rhs()
    u0 = inputs.initial_guess(O.N[0], 2)
    u, it, hist, st = S.solve(torch.as_tensor(f, device="cuda"), torch.as_tensor(u0, device="cuda"))
    uo, ho, ito, _ = O.solve(f, u0)
    assert st == 0 and abs(it - ito) <= 1
    assert np.linalg.norm(u.cpu().numpy() - uo) <= 1e-10 * np.linalg.norm(uo)
