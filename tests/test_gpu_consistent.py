"""GPU parity of the consistent-mass transfers (Sec. 3 with the consistent
mass matrices of App. B in place of the lumped ones): the restriction,
prolongation and V-cycle steps and whole solves through the C-ABI against the
FP64 oracle set up with consistent=True.  The library inverts each level's
interior mass matrix by banded line solves along each grid direction (its
Kronecker structure); the oracle factors the assembled matrix as a whole, so
the two share no arithmetic beyond the quadrature rule.

Tolerances: those of test_gpu_parity (steps 1e-12 relative max norm,
residual histories 1e-12 per cycle, iterations within 1, solutions 1e-10),
widened where a mass solve enters to 8 eps kappa(M), the forward-error bound
of a backward-stable solve with the mass matrix M it inverts (kappa grows
with the degree: ~1e2 at q = 2, ~2e6 at q = 7 in 2D; two factorisations of M
in different orders differ by up to that much).  kappa is computed from the
oracle's assembled mass at h = 2^-4 (2^-3 for the cube), where it has
already levelled off in h.
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
        S = pmg.Solver(dom, p, k, projection=proj, exact=ex, transfer_mass=pmg.PMG_MASS_CONSISTENT)
        O = oracle_mod.Hierarchy(dom, p, k, projection=proj, exact=ex, consistent=True)
        _cache[key] = (S, O)
    return _cache[key]


def _dev(torch, a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


# annulus (weighted first direction), square, cube (three directions), the
# highest degree (half bandwidth 8), a ragged line length (k = 4, p = 7: 19
# interior functions a line, not a multiple of the 8-entry load batch)
CASES = [(0, 3, 5, 0, 0), (1, 2, 5, 0, 0), (2, 2, 3, 0, 0), (2, 3, 4, 1, 0), (0, 8, 4, 0, 0), (1, 7, 4, 0, 0),
         (0, 4, 6, 0, 1), (3, 3, 5, 0, 0)]


_kappa = {}


def _cond(oracle_mod, dom, q):
    """kappa_2 of the interior mass matrix of degree q (see the module docstring)."""
    key = (dom, q)
    if key not in _kappa:
        _kappa[key] = float(np.linalg.cond(_interior_mass(oracle_mod, dom, 3 if dom == 2 else 4, q)))
    return _kappa[key]


def _tol(base, kappa):
    return max(base, 8 * np.finfo(float).eps * kappa)


@pytest.mark.parametrize("case", CASES)
def test_transfer_steps_match_oracle(torch_mod, pmg, oracle_mod, case):
    torch = torch_mod
    S, O = _pair(pmg, oracle_mod, *case)
    dom, p = case[0], case[1]
    rng = np.random.default_rng(21)
    for l in range(O.nlev):
        n, nc = O.N[l], O.coarse_N(l)
        k_fine, k_coarse = _cond(oracle_mod, dom, p - l), _cond(oracle_mod, dom, p - l - 1)
        k_below = max(_cond(oracle_mod, dom, q) for q in range(1, p - l + 1))
        x, b = rng.standard_normal(n), rng.standard_normal(n)
        yc = torch.empty(nc, dtype=torch.float64, device="cuda")
        S.apply(pmg.PMG_OP_RESTRICT, l, _dev(torch, x), None, yc)
        assert _rel(yc.cpu().numpy(), O.restrict(l, x)) <= _tol(STEP_TOL, k_coarse)
        ec = rng.standard_normal(nc)
        y = torch.empty(n, dtype=torch.float64, device="cuda")
        S.apply(pmg.PMG_OP_PROLONG_ADD, l, _dev(torch, ec), _dev(torch, b), y)
        assert _rel(y.cpu().numpy(), O.prolong_add(l, ec, b)) <= _tol(STEP_TOL, k_fine)
        # in place: u += I e_c
        u = _dev(torch, b)
        S.apply(pmg.PMG_OP_PROLONG_ADD, l, _dev(torch, ec), u, u)
        assert _rel(u.cpu().numpy(), O.prolong_add(l, ec, b)) <= _tol(STEP_TOL, k_fine)
        S.apply(pmg.PMG_OP_VCYCLE, l, _dev(torch, x), _dev(torch, b), y)
        assert _rel(y.cpu().numpy(), O.vcycle(l, b, x)) <= _tol(STEP_TOL, k_below)


@pytest.mark.parametrize("case", CASES)
def test_solve_matches_oracle(torch_mod, pmg, oracle_mod, case):
    torch = torch_mod
    S, O = _pair(pmg, oracle_mod, *case)
    kappa = max(_cond(oracle_mod, case[0], q) for q in range(1, case[1] + 1))
    f = O.rhs()
    u0 = inputs.initial_guess(O.N[0], 3)
    u, it, hist, st = S.solve(_dev(torch, f), _dev(torch, u0))
    uo, histo, ito, sto = O.solve(f, u0)
    assert st == 0 and sto == "ok"
    assert abs(it - ito) <= 1, (it, ito)
    m = min(it, ito)
    assert np.abs(hist[:m] - histo[:m]).max() <= _tol(HIST_TOL, kappa), (hist, histo)
    assert np.linalg.norm(u.cpu().numpy() - uo) <= _tol(U_TOL, kappa) * np.linalg.norm(uo)


def _interior_mass(oracle_mod, dom, k, q):
    """Interior consistent mass matrix of degree q, dense, assembled by the oracle."""
    M = oracle_mod.full_matrix(dom, k, q, q, "mass")
    nr = len(M.rp) - 1
    D = np.zeros((nr, nr))
    for i in range(nr):
        D[i, M.ci[M.rp[i]:M.rp[i + 1]]] = M.v[M.rp[i]:M.rp[i + 1]]
    n, d = (1 << k) + q, 3 if dom == 2 else 2
    inner = np.arange(n ** d).reshape((n,) * d)[(slice(1, n - 1),) * d].ravel()
    return D[np.ix_(inner, inner)]


@pytest.mark.parametrize("dom,p,k", [(0, 3, 5), (2, 3, 3)])
def test_transfers_are_mass_adjoint(torch_mod, pmg, oracle_mod, dom, p, k):
    """With consistent masses I = M_q^{-1} P and R = M_c^{-1} P^T satisfy
    (I e_c)^T M_q v = (R v)^T M_c e_c for every e_c, v: the identity fails for
    the lumped masses and needs nothing from the oracle's factorisation, only
    its assembled mass matrices."""
    torch = torch_mod
    S = pmg.Solver(dom, p, k, transfer_mass=pmg.PMG_MASS_CONSISTENT)
    rng = np.random.default_rng(22)
    nlev = p - 1
    for l in range(nlev):
        q, qc = p - l, p - l - 1
        Mq, Mc = _interior_mass(oracle_mod, dom, k, q), _interior_mass(oracle_mod, dom, k, qc)
        n, nc = Mq.shape[0], Mc.shape[0]
        ec, v = rng.standard_normal(nc), rng.standard_normal(n)
        Ie = torch.zeros(n, dtype=torch.float64, device="cuda")
        S.apply(pmg.PMG_OP_PROLONG_ADD, l, _dev(torch, ec), Ie, Ie)
        Rv = torch.empty(nc, dtype=torch.float64, device="cuda")
        S.apply(pmg.PMG_OP_RESTRICT, l, _dev(torch, v), None, Rv)
        lhs = float(Ie.cpu().numpy() @ (Mq @ v))
        rhs = float(Rv.cpu().numpy() @ (Mc @ ec))
        scale = np.linalg.norm(Mq @ v) * np.linalg.norm(Ie.cpu().numpy()) + np.linalg.norm(Mc @ ec) * np.linalg.norm(Rv.cpu().numpy())
        kappa = max(_cond(oracle_mod, dom, q), _cond(oracle_mod, dom, qc))
        assert abs(lhs - rhs) <= _tol(1e-12, kappa) * scale, (l, lhs, rhs)


def test_batched_workspace_is_refused(torch_mod, pmg):
    S = pmg.Solver(0, 3, 5, transfer_mass=pmg.PMG_MASS_CONSISTENT, upload=False)
    S.max_rhs = 4
    with pytest.raises(pmg.PmgError) as e:
        S.upload()
    assert e.value.status == pmg.PMG_ERR_ARG
