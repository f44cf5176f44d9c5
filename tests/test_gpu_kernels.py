"""Every kernel variant of the triangular solves and Gauss-Seidel sweeps, pinned
with pmg_set_kernels, and the autotuner's choice: whole solves through the
C-ABI against the FP64 oracle with the single-solve tolerances (the variants
differ only in the order of floating-point summation):
  relative residual history: |difference| <= 1e-12 per V-cycle
  iteration count:          equal within 1
  final solution:           ||u_gpu - u_oracle|| / ||u_oracle|| <= 1e-10
"""
import numpy as np
import pytest

from paper_1901_01685_gb300 import inputs

pytestmark = pytest.mark.gpu

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


def _pair(pmg, oracle_mod, dom, p, k):
    key = (dom, p, k)
    if key not in _cache:
        _cache[key] = (pmg.Solver(dom, p, k, max_rhs=8), oracle_mod.Hierarchy(dom, p, k))
    return _cache[key]


def _dev(torch, a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _check_single(torch, S, O, seed=1):
    f = O.rhs()
    u0 = inputs.initial_guess(O.N[0], seed)
    u, it, hist, st = S.solve(_dev(torch, f), _dev(torch, u0))
    uo, ho, ito, sto = O.solve(f, u0)
    assert st == 0 and sto == "ok" and abs(it - ito) <= 1
    m = min(it, ito)
    assert np.abs(hist[:m] - ho[:m]).max() <= HIST_TOL
    assert np.linalg.norm(u.cpu().numpy() - uo) <= U_TOL * np.linalg.norm(uo)


def _check_batched(torch, pmg, S, O, nrhs=3):
    F = inputs.batched_rhs(O.rhs(), nrhs, seed=5)
    U0 = np.stack([inputs.initial_guess(O.N[0], 300 + r) for r in range(nrhs)])
    U, it, hist, st = S.solve_batched(_dev(torch, F), _dev(torch, U0), precision=pmg.PMG_PREC_FP64)
    assert st == 0
    Un = U.cpu().numpy()
    for r in range(nrhs):
        uo, ho, ito, sto = O.solve(F[r], U0[r])
        assert abs(it[r] - ito) <= 1
        m = min(it[r], ito)
        assert np.abs(hist[:m, r] - ho[:m]).max() <= HIST_TOL
        assert np.linalg.norm(Un[r] - uo) <= U_TOL * np.linalg.norm(uo)
    Um, itm, hm, stm = S.solve_batched(_dev(torch, F), _dev(torch, U0), precision=pmg.PMG_PREC_MIXED)
    assert stm == 0 and all(hm[itm[r] - 1, r] < 1e-8 for r in range(nrhs))


CASES = [(0, 3, 5), (1, 2, 5), (2, 2, 3)]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("single,sweep,cfg", [(0, 0, 0), (1, 1, 0), (0, 1, 0), (1, 0, 0),
                                              (3, 3, 0), (3, 3, 1), (3, 3, 2), (3, 3, 3), (3, 3, 4), (3, 3, 5),
                                              (3, 3, 6), (3, 3, 7), (3, 1, 2), (3, 2, 6)])
def test_single_vector_variants_match_oracle(torch_mod, pmg, oracle_mod, case, single, sweep, cfg):
    S, O = _pair(pmg, oracle_mod, *case)
    S.set_kernels(single=single, sweep_single=sweep, chain_cfg=cfg)
    _check_single(torch_mod, S, O)


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("batched,sweep", [(1, 1), (2, 2), (1, 2), (2, 1)])
def test_batched_variants_match_oracle(torch_mod, pmg, oracle_mod, case, batched, sweep):
    S, O = _pair(pmg, oracle_mod, *case)
    S.set_kernels(batched=batched, sweep_batched=sweep)
    _check_batched(torch_mod, pmg, S, O)


@pytest.mark.parametrize("case", CASES)
def test_autotuned_kernels_match_oracle(torch_mod, pmg, oracle_mod, case):
    S, O = _pair(pmg, oracle_mod, *case)
    kp, kh = S.autotune()
    assert len(kp) == O.nlev and len(kh) == O.nh
    assert all(v in ("windowed", "ring", "cluster") for d in kp for k, v in d.items() if k.startswith("single"))
    assert all(v in ("ring", "lines") for d in kp for k, v in d.items() if k.startswith("batched"))
    _check_single(torch_mod, S, O)
    _check_batched(torch_mod, pmg, S, O)


def test_set_kernels_rejects_invalid_variants(torch_mod, pmg, oracle_mod):
    S, O = _pair(pmg, oracle_mod, 1, 2, 5)
    before = S.info["kernels_p"]
    for tp, th in (([2 | (1 << 4) | (1 << 6) | (1 << 8) | (1 << 10)] * O.nlev, [0] * O.nh),  # single-vector variant 2
                   ([0] * O.nlev, [0] * O.nh)):           # batched variant 0 (single-vector kernel)
        with pytest.raises(pmg.PmgError) as e:
            pmg.pmg_set_kernels(S.h, tp, th)
        assert e.value.status == pmg.PMG_ERR_ARG
    assert pmg.pmg_info(S.h).as_dict()["kernels_p"] == before
