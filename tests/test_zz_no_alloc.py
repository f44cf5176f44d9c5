"""The allocation-free forward solve, pmg_lsolve_noalloc.

It serves callers that cannot allocate device memory (fixed memory pools,
plug-ins whose host owns every allocation, loops that must not allocate once
running): its scratch lives in a fixed array inside the library.  This file is
collected last so that a run stopping at the first failure has already run
every other test; it passes alone in a fresh process and after the others.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_noalloc_lsolve_matches_workspace_path(torch_mod):
    """Two calls in a row through the C-ABI, each compared with the library's
    workspace-based forward solve (PMG_OP_LSOLVE) and with scipy's triangular
    solve on the CPU oracle's own ILUT factor L (unit diagonal)."""
    torch = torch_mod
    import scipy.sparse
    import scipy.sparse.linalg
    from oracle import oracle as O
    from paper_1901_01685_gb300 import pmg
    S = pmg.Solver(pmg.PMG_QUARTER_ANNULUS, 3, 6)
    n, _, rp, ci, v = pmg.pmg_export_csr(S.h, 1, 0)
    Lo = O.Hierarchy(O.ANNULUS, 3, 6).csr("L", 0)
    Lu = scipy.sparse.csr_matrix((Lo.v, Lo.ci, Lo.rp), shape=(n, n)) + scipy.sparse.identity(n, format="csr")
    rp_d = torch.as_tensor(rp, device="cuda")
    ci_d = torch.as_tensor(ci, device="cuda")
    v_d = torch.as_tensor(v, device="cuda")
    rng = np.random.default_rng(21)
    for call in range(2):  # two calls in a row: the shared scratch must not leak state
        bh = rng.standard_normal(n)
        b = torch.as_tensor(bh, device="cuda")
        y_ref = torch.empty(n, dtype=torch.float64, device="cuda")
        S.apply(pmg.PMG_OP_LSOLVE, 0, None, b, y_ref)
        y = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        pmg.pmg_lsolve_noalloc(n, rp_d, ci_d, v_d, b, y)
        torch.cuda.synchronize()
        err = (y - y_ref).abs().max().item() / max(y_ref.abs().max().item(), 1e-300)
        assert err <= TOL, (call, err)
        y_cpu = scipy.sparse.linalg.spsolve_triangular(Lu, bh, lower=True)
        err_o = np.abs(y.cpu().numpy() - y_cpu).max() / np.abs(y_cpu).max()
        assert err_o <= TOL, (call, err_o)


def test_noalloc_rejects_sizes_above_its_limit(torch_mod):
    torch = torch_mod
    from paper_1901_01685_gb300 import pmg
    d = torch.zeros(4, dtype=torch.int32, device="cuda")
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(pmg.PmgError) as e:
        pmg.pmg_lsolve_noalloc((1 << 20) + 1, d, d, x, x, x)
    assert e.value.status == pmg.PMG_ERR_ARG
    assert "limit" in str(e.value)
