"""GPU parity: every hot-path step and whole solves through the C-ABI against
the FP64 CPU oracle on the same seeded inputs.

Tolerances (FP64 on both sides, different summation orders):
  single steps:            relative max-norm error <= 1e-12
  relative residual history: |difference| <= 1e-12 per V-cycle
  iteration count:          equal within 1
  final solution:           ||u_gpu - u_oracle|| / ||u_oracle|| <= 1e-10
"""
import numpy as np
import pytest

from paper_1901_01685_gb300 import inputs

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-12
HIST_TOL = 1e-12
U_TOL = 1e-10


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


_cache = {}


def _pair(pmg, oracle_mod, dom, p, k, proj=0, ex=0):
    key = (dom, p, k, proj, ex)
    if key not in _cache:
        S = pmg.Solver(dom, p, k, projection=proj, exact=ex)
        O = oracle_mod.Hierarchy(dom, p, k, projection=proj, exact=ex)
        _cache[key] = (S, O)
    return _cache[key]


def _dev(torch, a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


SMALL = [(0, 3, 5, 0, 0), (0, 3, 5, 1, 0), (1, 2, 5, 0, 0), (2, 2, 3, 0, 0), (0, 4, 6, 0, 1), (2, 3, 4, 1, 0),
         (3, 3, 5, 0, 0)]


@pytest.mark.parametrize("case", SMALL)
def test_steps_match_oracle(torch_mod, pmg, oracle_mod, case):
    torch = torch_mod
    S, O = _pair(pmg, oracle_mod, *case)
    rng = np.random.default_rng(11)
    for l in range(O.nlev):
        n, nc = O.N[l], O.coarse_N(l)
        x, b = rng.standard_normal(n), rng.standard_normal(n)
        y = torch.empty(n, dtype=torch.float64, device="cuda")
        S.apply(pmg.PMG_OP_RESIDUAL, l, _dev(torch, x), _dev(torch, b), y)
        assert _rel(y.cpu().numpy(), O.residual(l, b, x)) <= STEP_TOL
        S.apply(pmg.PMG_OP_SMOOTH, l, _dev(torch, x), _dev(torch, b), y)
        assert _rel(y.cpu().numpy(), O.smooth(l, b, x)) <= STEP_TOL
        yc = torch.empty(nc, dtype=torch.float64, device="cuda")
        S.apply(pmg.PMG_OP_RESTRICT, l, _dev(torch, x), None, yc)
        assert _rel(yc.cpu().numpy(), O.restrict(l, x)) <= STEP_TOL
        ec = rng.standard_normal(nc)
        S.apply(pmg.PMG_OP_PROLONG_ADD, l, _dev(torch, ec), _dev(torch, b), y)
        assert _rel(y.cpu().numpy(), O.prolong_add(l, ec, b)) <= STEP_TOL
        S.apply(pmg.PMG_OP_VCYCLE, l, _dev(torch, x), _dev(torch, b), y)
        assert _rel(y.cpu().numpy(), O.vcycle(l, b, x)) <= STEP_TOL


@pytest.mark.parametrize("case", SMALL)
def test_triangular_solves_match_oracle_factors(torch_mod, pmg, oracle_mod, case):
    import scipy.sparse
    import scipy.sparse.linalg
    torch = torch_mod
    S, O = _pair(pmg, oracle_mod, *case)
    rng = np.random.default_rng(12)
    for l in range(O.nlev):
        n = O.N[l]
        b = rng.standard_normal(n)
        Lc, Uc = O.csr("L", l), O.csr("U", l)
        L = scipy.sparse.csr_matrix((Lc.v, Lc.ci, Lc.rp), shape=Lc.shape) + scipy.sparse.identity(n, format="csr")
        U = scipy.sparse.csr_matrix((Uc.v, Uc.ci, Uc.rp), shape=Uc.shape)
        y = torch.empty(n, dtype=torch.float64, device="cuda")
        S.apply(pmg.PMG_OP_LSOLVE, l, None, _dev(torch, b), y)
        ref = scipy.sparse.linalg.spsolve_triangular(L, b, lower=True, unit_diagonal=True)
        assert _rel(y.cpu().numpy(), ref) <= STEP_TOL
        S.apply(pmg.PMG_OP_USOLVE, l, None, _dev(torch, b), y)
        ref = scipy.sparse.linalg.spsolve_triangular(U, b, lower=False)
        assert _rel(y.cpu().numpy(), ref) <= 1e-11


@pytest.mark.parametrize("case", SMALL)
def test_p1_steps_match_oracle(torch_mod, pmg, oracle_mod, case):
    torch = torch_mod
    S, O = _pair(pmg, oracle_mod, *case)
    rng = np.random.default_rng(13)
    for j in range(O.nh):
        n = O.NH[j]
        x, b = rng.standard_normal(n), rng.standard_normal(n)
        y = torch.empty(n, dtype=torch.float64, device="cuda")
        S.apply(pmg.PMG_OP_GS_FWD, j, _dev(torch, x), _dev(torch, b), y)
        assert _rel(y.cpu().numpy(), O.gs(j, b, x)) <= STEP_TOL
        S.apply(pmg.PMG_OP_GS_BWD, j, _dev(torch, x), _dev(torch, b), y)
        assert _rel(y.cpu().numpy(), O.gs(j, b, x, backward=True)) <= STEP_TOL
        S.apply(pmg.PMG_OP_HMG_VCYCLE, j, _dev(torch, x), _dev(torch, b), y)
        assert _rel(y.cpu().numpy(), O.hmg_vcycle(j, b, x)) <= STEP_TOL
    b = rng.standard_normal(O.NH[0])
    y = torch.empty(O.NH[0], dtype=torch.float64, device="cuda")
    S.apply(pmg.PMG_OP_COARSE_SOLVE, 0, None, _dev(torch, b), y)
    assert _rel(y.cpu().numpy(), O.coarse_solve(b)) <= STEP_TOL


def _check_solve(torch, S, O, seed=1):
    f = O.rhs()
    u0 = inputs.initial_guess(O.N[0], seed)
    u, it, hist, st = S.solve(_dev(torch, f), _dev(torch, u0))
    uo, histo, ito, sto = O.solve(f, u0)
    assert st == 0 and sto == "ok"
    assert abs(it - ito) <= 1, (it, ito)
    m = min(it, ito)
    assert np.abs(hist[:m] - histo[:m]).max() <= HIST_TOL, (hist, histo)
    un = u.cpu().numpy()
    assert np.linalg.norm(un - uo) <= U_TOL * np.linalg.norm(uo)
    return it, hist


@pytest.mark.parametrize("case", SMALL)
def test_solve_matches_oracle(torch_mod, pmg, oracle_mod, case):
    S, O = _pair(pmg, oracle_mod, *case)
    _check_solve(torch_mod, S, O)


@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_solve_full_size_annulus(torch_mod, pmg, oracle_mod, p):
    """Quarter annulus at h = 2^-8, p = 2..5 (~66k unknowns): the benchmark size."""
    S = pmg.Solver(0, p, 8)
    O = oracle_mod.Hierarchy(0, p, 8)
    it, hist = _check_solve(torch_mod, S, O)
    assert hist[-1] < 1e-8


def test_solve_host_buffers_match_device_path(torch_mod, pmg, oracle_mod):
    torch = torch_mod
    S, O = _pair(pmg, oracle_mod, 0, 3, 5, 0, 0)
    f = O.rhs()
    u0 = inputs.initial_guess(O.N[0], 3)
    u_dev, it, hist, _ = S.solve(_dev(torch, f), _dev(torch, u0))
    u_host = np.zeros(O.N[0])
    it2, hist2, _ = pmg.pmg_solve_host(S.h, S.ws, f, u0, 1e-8, 100, u_host)
    assert it == it2 and np.array_equal(hist, hist2)
    assert np.array_equal(u_host, u_dev.cpu().numpy())


def test_zero_residual_returns_immediately(torch_mod, pmg, oracle_mod):
    torch = torch_mod
    S, O = _pair(pmg, oracle_mod, 0, 3, 5, 0, 0)
    z = torch.zeros(O.N[0], dtype=torch.float64, device="cuda")
    u, it, hist, st = S.solve(z, z.clone())
    assert st == 0 and it == 0 and torch.count_nonzero(u).item() == 0


def test_exact_solution_is_fixed_point(torch_mod, pmg, oracle_mod):
    import scipy.sparse
    import scipy.sparse.linalg
    torch = torch_mod
    S, O = _pair(pmg, oracle_mod, 0, 3, 5, 0, 0)
    A = O.csr("A", 0)
    f = O.rhs()
    us = scipy.sparse.linalg.spsolve(scipy.sparse.csr_matrix((A.v, A.ci, A.rp), shape=A.shape).tocsc(), f)
    y = torch.empty(O.N[0], dtype=torch.float64, device="cuda")
    S.apply(pmg.PMG_OP_VCYCLE, 0, _dev(torch, us), _dev(torch, f), y)
    assert np.linalg.norm(y.cpu().numpy() - us) <= 1e-11 * np.linalg.norm(us)


def test_repeated_solves_are_deterministic(torch_mod, pmg, oracle_mod):
    torch = torch_mod
    S, O = _pair(pmg, oracle_mod, 1, 2, 5, 0, 0)
    f = _dev(torch, O.rhs())
    u0 = _dev(torch, inputs.initial_guess(O.N[0], 5))
    a, ita, ha, _ = S.solve(f, u0)
    b, itb, hb, _ = S.solve(f, u0)
    assert ita == itb and np.array_equal(ha, hb) and torch.equal(a, b)


def _check_bicgstab(torch, S, O, seed=1):
    f = O.rhs()
    u0 = inputs.initial_guess(O.N[0], seed)
    u, it, hist, st = S.solve_bicgstab(_dev(torch, f), _dev(torch, u0))
    uo, ho, ito, sto = O.bicgstab(f, u0)
    assert st == 0 and sto == "ok"
    assert abs(it - ito) <= 1, (it, ito)
    m = min(it, ito)
    assert np.abs(hist[:m] - ho[:m]).max() <= HIST_TOL, (hist, ho)
    if it == ito:
        assert np.linalg.norm(u.cpu().numpy() - uo) <= U_TOL * np.linalg.norm(uo)
    return it, hist


@pytest.mark.parametrize("case", SMALL)
def test_bicgstab_matches_oracle(torch_mod, pmg, oracle_mod, case):
    """BiCGSTAB preconditioned by the V-cycle (Sec. 5, Table 5) against the oracle's."""
    S, O = _pair(pmg, oracle_mod, *case)
    _check_bicgstab(torch_mod, S, O)


def test_bicgstab_full_size_annulus(torch_mod, pmg, oracle_mod):
    S = pmg.Solver(0, 3, 8)
    O = oracle_mod.Hierarchy(0, 3, 8)
    it, hist = _check_bicgstab(torch_mod, S, O)
    assert hist[-1] < 1e-8 and it <= 3


def test_steps_match_oracle_at_benchmark_size(torch_mod, pmg, oracle_mod):
    """Single steps at the benchmark size (quarter annulus, h = 2^-8, p = 3),
    where the kernels differ from the small cases: the clustered triangular
    solves on 257-row lines, the wide SpMV, and the wavefront Gauss-Seidel
    sweeps on the 255 x 255 P1 level (eight warps, every hand-off between
    them).  Each step within the per-step tolerance of the oracle's."""
    torch = torch_mod
    S = pmg.Solver(0, 3, 8)
    O = oracle_mod.Hierarchy(0, 3, 8)
    rng = np.random.default_rng(17)
    n = O.N[0]
    x, b = rng.standard_normal(n), rng.standard_normal(n)
    y = torch.empty(n, dtype=torch.float64, device="cuda")
    S.apply(pmg.PMG_OP_RESIDUAL, 0, _dev(torch, x), _dev(torch, b), y)
    assert _rel(y.cpu().numpy(), O.residual(0, b, x)) <= STEP_TOL
    S.apply(pmg.PMG_OP_SMOOTH, 0, _dev(torch, x), _dev(torch, b), y)
    assert _rel(y.cpu().numpy(), O.smooth(0, b, x)) <= STEP_TOL
    for j in range(2):
        nh = O.NH[j]
        xh, bh = rng.standard_normal(nh), rng.standard_normal(nh)
        yh = torch.empty(nh, dtype=torch.float64, device="cuda")
        S.apply(pmg.PMG_OP_GS_FWD, j, _dev(torch, xh), _dev(torch, bh), yh)
        assert _rel(yh.cpu().numpy(), O.gs(j, bh, xh)) <= STEP_TOL
        S.apply(pmg.PMG_OP_GS_BWD, j, _dev(torch, xh), _dev(torch, bh), yh)
        assert _rel(yh.cpu().numpy(), O.gs(j, bh, xh, backward=True)) <= STEP_TOL
