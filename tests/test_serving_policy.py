"""Scheduling policy of the serving loop (paper_1901_01685_gb300.serve) on the
CPU, with a simulated backend: every request completes with its own result,
requests join a running batch between cycles (continuous batching), keys are
admitted by device memory with least-recently-used eviction of idle keys, and
requests that can never fit are refused."""
import numpy as np
import pytest

from paper_1901_01685_gb300 import serve


class FakeBackend:
    """Slots converge after the number of cycles written in F[r, 0]; the
    'solution' is 2 F.  Memory per key comes from a table."""

    def __init__(self, sizes, budget):
        self.sizes = sizes
        self.budget = budget
        self.created, self.freed, self.loads = [], [], []

    def memory_budget(self):
        return self.budget

    def bytes_needed(self, key, slots):
        return self.sizes[key]

    def create(self, key, slots):
        self.created.append(key)
        return {"key": key, "state": np.zeros(slots, np.int32), "iters": np.zeros(slots, np.int32),
                "need": np.zeros(slots, np.int32), "F": [None] * slots, "U": [None] * slots, "res": None}

    def free(self, h):
        assert not (h["state"] == serve.ACTIVE).any(), "evicted a key with active slots"
        self.freed.append(h["key"])

    def load(self, h, s0, F, U0):
        self.loads.append((h["key"], s0, F.shape[0]))
        for r in range(F.shape[0]):
            s = s0 + r
            assert h["state"][s] != serve.ACTIVE
            h["state"][s], h["iters"][s], h["need"][s] = serve.ACTIVE, 0, int(F[r, 0])
            h["F"][s], h["U"][s] = F[r], U0[r].copy()

    def cycle(self, h, precision, tol):
        assert h["res"] is None, "cycle issued before the previous one was waited for"
        act = h["state"] == serve.ACTIVE
        h["iters"][act] += 1
        for s in np.nonzero(act)[0]:
            if h["iters"][s] >= h["need"][s]:
                h["state"][s] = serve.CONVERGED
                h["U"][s] = 2 * h["F"][s]
        h["res"] = (np.zeros(len(h["state"])), h["state"].copy(), h["iters"].copy())

    def poll(self, h, blocking=False):
        res, h["res"] = h["res"], None
        return res

    def read(self, h, s0, n):
        return np.stack([h["U"][s] for s in range(s0, s0 + n)])

    def release(self, h, s0, n):
        h["state"][s0:s0 + n] = serve.FREE


def _req(rid, key, nrhs, need, N=4):
    F = np.full((nrhs, N), float(need))
    F[:, 1:] = rid + np.arange(nrhs)[:, None]
    return serve.Request(rid=rid, key=key, F=F, U0=np.zeros((nrhs, N)))


def _run(server, now0=0.0, limit=10000):
    done, now = [], now0
    while server.pending_work():
        now += 1.0
        done += server.step(now)
        limit -= 1
        assert limit > 0, "server did not drain"
    return done, now


def test_every_request_completes_with_its_own_result():
    be = FakeBackend({(0, 2, 5): 10, (1, 3, 5): 10, (2, 2, 3): 10}, budget=100)
    srv = serve.Server(be, slots=8, precision=1)
    keys = list(be.sizes)
    reqs = [_req(i, keys[i % 3], 1 + i % 4, 2 + (i * 7) % 5) for i in range(30)]
    for r in reqs:
        srv.submit(r, now=0.0)
    done, _ = _run(srv)
    assert sorted(r.rid for r in done) == list(range(30))
    for r in reqs:
        assert r.status == "done"
        assert np.array_equal(r.U, 2 * r.F)
        assert np.array_equal(r.iters, np.full(r.nrhs, int(r.F[0, 0])))


def test_request_joins_a_running_batch_between_cycles():
    be = FakeBackend({(0, 2, 5): 10}, budget=100)
    srv = serve.Server(be, slots=8)
    a = srv.submit(_req(0, (0, 2, 5), 2, need=6), now=0.0)
    srv.step(1.0)                                   # loads A, first cycle
    srv.step(2.0)                                   # A: cycle 2
    b = srv.submit(_req(1, (0, 2, 5), 1, need=2), now=2.5)
    t = 3.0
    while b.status != "done":
        srv.step(t)
        t += 1.0
    assert a.status == "running"                    # B finished while A was still iterating
    assert b.t_done - b.t_admitted == 2.0           # exactly its own two cycles
    _run(srv, t)
    assert a.status == "done" and a.iters.tolist() == [6, 6]


def test_keys_are_admitted_by_memory_with_lru_eviction_of_idle_keys():
    k1, k2, k3 = (0, 2, 5), (0, 3, 5), (1, 2, 5)
    be = FakeBackend({k1: 40, k2: 40, k3: 40}, budget=90)
    srv = serve.Server(be, slots=4)
    srv.submit(_req(0, k1, 1, 2), now=0.0)
    srv.submit(_req(1, k2, 1, 2), now=0.0)
    _run(srv)
    assert set(srv.keys) == {k1, k2} and srv.used == 80
    srv.keys[k1].last_used = 10.0                   # k2 is the least recently used
    srv.submit(_req(2, k3, 1, 2), now=20.0)
    _run(srv, 20.0)
    assert be.freed == [k2] and set(srv.keys) == {k1, k3} and srv.evictions == 1


def test_busy_keys_are_not_evicted():
    k1, k2 = (0, 2, 5), (0, 3, 5)
    be = FakeBackend({k1: 60, k2: 60}, budget=100)
    srv = serve.Server(be, slots=4)
    a = srv.submit(_req(0, k1, 1, 5), now=0.0)
    srv.step(1.0)
    b = srv.submit(_req(1, k2, 1, 1), now=1.5)
    srv.step(2.0)
    assert k2 not in srv.keys and b.status == "queued"      # waits: k1 is busy
    _run(srv, 2.0)
    assert a.status == "done" and b.status == "done" and be.freed == [k1]


def test_requests_that_cannot_fit_are_refused():
    be = FakeBackend({(0, 2, 5): 10, (2, 5, 5): 1000}, budget=100)
    srv = serve.Server(be, slots=4)
    big = srv.submit(_req(0, (0, 2, 5), 5, 1), now=0.0)     # more right-hand sides than slots
    huge = srv.submit(_req(1, (2, 5, 5), 1, 1), now=0.0)    # hierarchy larger than the budget
    ok = srv.submit(_req(2, (0, 2, 5), 4, 1), now=0.0)
    _run(srv)
    assert big.status == "rejected" and huge.status == "rejected" and ok.status == "done"


def test_slots_are_contiguous_and_reused():
    be = FakeBackend({(0, 2, 5): 10}, budget=100)
    srv = serve.Server(be, slots=6)
    for i, (n, need) in enumerate([(2, 3), (3, 1), (1, 2), (3, 2)]):
        srv.submit(_req(i, (0, 2, 5), n, need), now=0.0)
    _run(srv)
    for key, s0, n in be.loads:
        assert 0 <= s0 and s0 + n <= 6
    assert [l[1:] for l in be.loads[:3]] == [(0, 2), (2, 3), (5, 1)]
    assert be.loads[3][1:] == (2, 3)                # the request of 3 reuses the freed run


def test_poisson_arrivals_are_seeded_and_have_the_requested_rate():
    a = serve.poisson_arrivals(4000, rate=50.0, seed=3)
    b = serve.poisson_arrivals(4000, rate=50.0, seed=3)
    assert np.array_equal(a, b) and np.all(np.diff(a) > 0)
    mean_gap = a[-1] / len(a)
    assert abs(mean_gap - 1 / 50.0) < 4 * (1 / 50.0) / np.sqrt(len(a))   # 4 standard errors of the mean


def test_router_keeps_keys_on_one_server_and_balances_new_keys():
    """Several GPUs: each key lives on one server (no request of a key runs
    elsewhere); new keys go to the least-loaded server; every result is right."""
    keys = [(0, 2, 5), (0, 3, 5), (1, 2, 5), (1, 3, 5), (2, 2, 3)]
    backends = [FakeBackend({k: 10 for k in keys}, budget=100) for _ in range(2)]
    router = serve.Router([serve.Server(b, slots=8) for b in backends])
    reqs = [_req(i, keys[i % len(keys)], 1 + i % 3, 2 + i % 4) for i in range(25)]
    for r in reqs:
        router.submit(r, now=0.0)
    now = 0.0
    while router.pending_work():
        now += 1.0
        router.step(now)
    assert all(r.status == "done" and np.array_equal(r.U, 2 * r.F) for r in reqs)
    served = [{l[0] for l in b.loads} for b in backends]
    assert served[0].isdisjoint(served[1]) and served[0] | served[1] == set(keys)
    assert all(served), "both servers took keys"
    assert router.cycles > 0
