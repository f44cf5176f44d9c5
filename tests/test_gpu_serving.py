"""Continuous batching on the GPU: the slot calls of the C-ABI and the serving
loop.  A right-hand side that joins a running batch, or is served among other
requests of several problem keys, gives bit-for-bit the result of solving it
alone with pmg_solve_batched (every slot is one lane of fixed arithmetic)."""
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


def _dev(torch, a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _alone(torch, pmg, S, f, u0, prec):
    U, it, hist, st = S.solve_batched(_dev(torch, f[None]), _dev(torch, u0[None]), precision=prec)
    return U[0].cpu().numpy(), int(it[0])


@pytest.mark.parametrize("prec", [0, 1])
def test_slots_join_a_running_batch_and_match_alone(torch_mod, pmg, prec):
    torch = torch_mod
    S = pmg.Solver(0, 3, 6, max_rhs=8)
    f = S.rhs()
    F = inputs.batched_rhs(f, 5, seed=31)
    U0 = np.stack([inputs.initial_guess(S.N, 400 + r) for r in range(5)])
    h, ws = S.h, S.ws
    pmg.pmg_slots_load(h, ws, 0, _dev(torch, F[:3]), _dev(torch, U0[:3]))      # request A: slots 0..2
    cycles = 0
    pmg.pmg_slots_cycle(h, ws, prec)
    rel, state, iters = pmg.pmg_slots_wait(h, ws, 8)
    cycles += 1
    assert list(state[:3]) == [1, 1, 1] and list(iters[:3]) == [1, 1, 1]
    pmg.pmg_slots_load(h, ws, 5, _dev(torch, F[3:]), _dev(torch, U0[3:]))      # request B joins: slots 5..6
    while True:
        pmg.pmg_slots_cycle(h, ws, prec)
        rel, state, iters = pmg.pmg_slots_wait(h, ws, 8)
        cycles += 1
        if all(state[k] == 2 for k in (0, 1, 2, 5, 6)):
            break
        assert cycles < 50
    assert state[3] == 0 and state[4] == 0 and state[7] == 0
    got = {}
    for slot in (0, 1, 2, 5, 6):
        U = torch.empty((1, S.N), dtype=torch.float64, device="cuda")
        pmg.pmg_slots_read(h, ws, slot, U)
        got[slot] = U[0].cpu().numpy()
    pmg.pmg_slots_release(h, ws, 0, 8)
    assert pmg.pmg_slots_wait(h, ws, 8)[1].tolist() == [0] * 8
    for slot, r in ((0, 0), (1, 1), (2, 2), (5, 3), (6, 4)):
        ua, ita = _alone(torch, pmg, S, F[r], U0[r], prec)      # reuses the workspace: after the reads
        assert iters[slot] == ita and rel[slot] < 1e-8
        assert np.array_equal(got[slot], ua)


def test_slot_calls_check_their_arguments(torch_mod, pmg):
    torch = torch_mod
    S = pmg.Solver(1, 2, 5, max_rhs=4)
    F = _dev(torch, np.ones((2, S.N)))
    pmg.pmg_slots_load(S.h, S.ws, 0, F, F)
    with pytest.raises(pmg.PmgError) as e:                 # slot 1 is active
        pmg.pmg_slots_load(S.h, S.ws, 1, F, F)
    assert e.value.status == pmg.PMG_ERR_BUSY
    with pytest.raises(pmg.PmgError) as e:                 # past the last slot
        pmg.pmg_slots_load(S.h, S.ws, 3, F, F)
    assert e.value.status == pmg.PMG_ERR_ARG
    pmg.pmg_slots_cycle(S.h, S.ws, 0)
    with pytest.raises(pmg.PmgError) as e:                 # the cycle was not waited for
        pmg.pmg_slots_cycle(S.h, S.ws, 0)
    assert e.value.status == pmg.PMG_ERR_BUSY
    assert pmg.pmg_slots_wait(S.h, S.ws, 4) is not None
    S1 = pmg.Solver(1, 2, 5, max_rhs=1)                    # no slots in a one-right-hand-side workspace
    with pytest.raises(pmg.PmgError) as e:
        pmg.pmg_slots_cycle(S1.h, S1.ws, 0)
    assert e.value.status == pmg.PMG_ERR_ARG


@pytest.mark.parametrize("prec", [0, 1])
def test_served_mix_matches_each_request_alone(torch_mod, pmg, prec):
    """A Poisson stream over four keys (2D and 3D, several degrees) through the
    serving loop; every request's result equals its solve alone, bit for bit."""
    torch = torch_mod
    from paper_1901_01685_gb300 import serve
    keys = [(0, 2, 5), (0, 3, 5), (1, 2, 6), (2, 2, 3)]
    be = serve.GpuBackend(autotune=False)
    srv = serve.Server(be, slots=16, precision=prec)
    srv.prewarm(keys)
    rhs = {k: (srv.keys[k].handle["S"].rhs(), srv.keys[k].handle["S"].N) for k in keys}
    reqs = serve.request_mix(keys, 24, lambda k: rhs[k], seed=5, max_rhs=6)
    stats = serve.run_stream(srv, reqs, serve.poisson_arrivals(24, rate=400.0, seed=9))
    assert stats["completed"] == 24 and stats["p99_ms"] >= stats["p50_ms"] > 0
    alone = {k: pmg.Solver(*k, max_rhs=8) for k in keys}
    for r in reqs:
        assert r.status == "done" and r.relres.max() < 1e-8
        S = alone[r.key]
        U, it, hist, st = S.solve_batched(_dev(torch, r.F), _dev(torch, r.U0), precision=prec)
        assert np.array_equal(it, r.iters)
        assert np.array_equal(U.cpu().numpy(), r.U)
    srv.close()
