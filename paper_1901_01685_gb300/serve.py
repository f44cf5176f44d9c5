"""Serving loop: continuous batching of p-multigrid solves (the paper has no
counterpart; it measures single solves, Sec. 5 and App. C).

Requests (a problem key (domain, p, log2 1/h), 1..S right-hand sides with
initial guesses) arrive over time.  The server keeps one hierarchy per key
resident on the device with a workspace of S right-hand-side slots and its
own CUDA stream.  Between V-cycles of a key it retires the slots that
converged (or diverged), hands their requests back, and loads waiting requests
of that key into free slots, so requests join and leave a running batch
(continuous batching, `pmg_slots_*` in the C-ABI).  Keys run on separate
streams, so their cycles overlap on the device.  Hierarchies are admitted by
device memory: a new key is set up only if its arena and workspace fit in the
budget, after evicting idle keys least recently used first.  A slot's result
does not depend on the other slots or on when it was loaded (per-lane
arithmetic), so every result equals the same request solved alone.

The scheduling policy is plain Python over a backend interface; `GpuBackend`
drives the CUDA library, and the tests also drive the policy with a simulated
backend on the CPU.
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Dict, List, Optional, Tuple

import numpy as np

from . import inputs

Key = Tuple[int, int, int]          # (domain, p, log2 1/h)

FREE, ACTIVE, CONVERGED, DIVERGED = 0, 1, 2, 3


@dataclasses.dataclass
class Request:
    rid: int
    key: Key
    F: np.ndarray                   # (nrhs, N) right-hand sides
    U0: np.ndarray                  # (nrhs, N) initial guesses
    t_arrival: float = 0.0
    t_admitted: Optional[float] = None
    t_done: Optional[float] = None
    U: Optional[np.ndarray] = None
    iters: Optional[np.ndarray] = None
    relres: Optional[np.ndarray] = None
    status: str = "queued"          # queued | running | done | diverged | rejected

    @property
    def nrhs(self) -> int:
        return int(self.F.shape[0])

    @property
    def latency(self) -> Optional[float]:
        return None if self.t_done is None else self.t_done - self.t_arrival


class _KeyState:
    def __init__(self, key: Key, handle, nbytes: int, slots: int):
        self.key = key
        self.handle = handle
        self.nbytes = nbytes
        self.slot_req: List[Optional[int]] = [None] * slots     # request id per slot
        self.pending = False                                    # a cycle is in flight
        self.last_used = 0.0

    def busy(self) -> bool:
        return self.pending or any(r is not None for r in self.slot_req)

    def free_run(self, n: int) -> Optional[int]:
        """First slot of a run of n free slots, or None."""
        run = 0
        for i, r in enumerate(self.slot_req):
            run = run + 1 if r is None else 0
            if run == n:
                return i - n + 1
        return None


class Server:
    """Continuous-batching server over a backend (see GpuBackend for the interface)."""

    def __init__(self, backend, slots: int = 64, hbm_budget: Optional[int] = None, precision: int = 1,
                 rel_tol: float = 1e-8, max_cycles: int = 100):
        self.backend = backend
        self.slots = slots
        self.budget = hbm_budget if hbm_budget is not None else backend.memory_budget()
        self.precision = precision
        self.rel_tol = rel_tol
        self.max_cycles = max_cycles
        self.keys: Dict[Key, _KeyState] = {}
        self.queue: Dict[Key, collections.deque] = collections.defaultdict(collections.deque)
        self.requests: Dict[int, Request] = {}
        self.used = 0
        self.evictions = 0
        self.cycles = 0

    # --------------------------------------------------------------- intake
    def submit(self, req: Request, now: Optional[float] = None) -> Request:
        req.t_arrival = time.perf_counter() if now is None else now
        self.requests[req.rid] = req
        if req.nrhs < 1 or req.nrhs > self.slots:
            req.status = "rejected"
            req.t_done = req.t_arrival
            return req
        self.queue[req.key].append(req)
        return req

    def pending_work(self) -> bool:
        return any(self.queue.values()) or any(k.busy() for k in self.keys.values())

    # ------------------------------------------------------------ residency
    def _admit_key(self, key: Key) -> Optional[_KeyState]:
        ks = self.keys.get(key)
        if ks is not None:
            return ks
        need = self.backend.bytes_needed(key, self.slots)
        if need > self.budget:
            return None
        # evict idle keys (no slots in use, nothing queued), least recently used first
        if self.used + need > self.budget:
            idle = sorted((k for k in self.keys.values() if not k.busy() and not self.queue[k.key]),
                          key=lambda k: k.last_used)
            for victim in idle:
                if self.used + need <= self.budget:
                    break
                self.backend.free(victim.handle)
                self.used -= victim.nbytes
                del self.keys[victim.key]
                self.evictions += 1
        if self.used + need > self.budget:
            return None
        handle = self.backend.create(key, self.slots)
        ks = _KeyState(key, handle, need, self.slots)
        self.keys[key] = ks
        self.used += need
        return ks

    # ------------------------------------------------------------ scheduling
    def _retire(self, ks: _KeyState, state, iters, relres, now: float) -> List[Request]:
        done: List[Request] = []
        by_req: Dict[int, List[int]] = collections.defaultdict(list)
        for s, rid in enumerate(ks.slot_req):
            if rid is not None:
                by_req[rid].append(s)
        for rid, sl in by_req.items():
            req = self.requests[rid]
            st = [int(state[s]) for s in sl]
            over = [int(iters[s]) >= self.max_cycles for s in sl]
            if all(x in (CONVERGED, DIVERGED) or o for x, o in zip(st, over)):
                s0, n = sl[0], len(sl)
                req.U = self.backend.read(ks.handle, s0, n)
                req.iters = np.array([int(iters[s]) for s in sl])
                req.relres = np.array([float(relres[s]) for s in sl])
                self.backend.release(ks.handle, s0, n)
                for s in sl:
                    ks.slot_req[s] = None
                req.status = "diverged" if DIVERGED in st else ("done" if all(x == CONVERGED for x in st)
                                                                 else "maxiter")
                req.t_done = now
                done.append(req)
        return done

    def _fill(self, ks: _KeyState, now: float) -> None:
        q = self.queue[ks.key]
        while q:
            req = q[0]
            s0 = ks.free_run(req.nrhs)
            if s0 is None:
                break
            q.popleft()
            self.backend.load(ks.handle, s0, req.F, req.U0)
            for s in range(s0, s0 + req.nrhs):
                ks.slot_req[s] = req.rid
            req.status = "running"
            req.t_admitted = now

    def step(self, now: Optional[float] = None) -> List[Request]:
        """One non-blocking scheduling pass; returns the requests completed in it."""
        now = time.perf_counter() if now is None else now
        done: List[Request] = []
        # keys with waiting requests become resident if memory allows; a key
        # that cannot fit even in an empty device is refused
        for key, q in self.queue.items():
            if q and key not in self.keys and self._admit_key(key) is None and \
                    self.backend.bytes_needed(key, self.slots) > self.budget:
                while q:
                    req = q.popleft()
                    req.status = "rejected"
                    req.t_done = now
                    done.append(req)
        for ks in list(self.keys.values()):
            if ks.pending:
                res = self.backend.poll(ks.handle, blocking=False)
                if res is None:
                    continue
                ks.pending = False
                relres, state, iters = res
                done += self._retire(ks, state, iters, relres, now)
            self._fill(ks, now)
            if any(r is not None for r in ks.slot_req):
                self.backend.cycle(ks.handle, self.precision, self.rel_tol)
                ks.pending = True
                ks.last_used = now
                self.cycles += 1
        return done

    def prewarm(self, keys: List[Key], threads: int = 4) -> None:
        """Sets up the hierarchies of `keys` on the host in parallel (the setup
        is native code and releases the interpreter), then makes them resident
        as far as the memory budget allows."""
        import concurrent.futures
        prep = getattr(self.backend, "prepare", None)
        if prep is not None:
            with concurrent.futures.ThreadPoolExecutor(threads) as ex:
                list(ex.map(prep, keys))
        for key in keys:
            self._admit_key(key)

    def drain(self, idle_sleep: float = 2e-4) -> List[Request]:
        done: List[Request] = []
        while self.pending_work():
            got = self.step()
            done += got
            if not got:
                time.sleep(idle_sleep)
        return done

    def close(self):
        for ks in self.keys.values():
            self.backend.free(ks.handle)
        self.keys.clear()
        self.used = 0


class Router:
    """Requests over several servers, one per GPU (the solves are independent:
    no collective, host-side routing only).  A key stays on the server that
    took it first, where its hierarchy is resident; a new key goes to the
    server with the fewest right-hand sides outstanding.  Same interface as
    Server (submit, step, pending_work, drain, close)."""

    def __init__(self, servers: List[Server]):
        assert servers, "a router needs at least one server"
        self.servers = servers
        self.home: Dict[Key, int] = {}

    def _load(self, i: int) -> int:
        srv = self.servers[i]
        queued = sum(r.nrhs for q in srv.queue.values() for r in q)
        running = sum(1 for ks in srv.keys.values() for rid in ks.slot_req if rid is not None)
        return queued + running

    def submit(self, req: Request, now: Optional[float] = None) -> Request:
        if req.key not in self.home:
            self.home[req.key] = min(range(len(self.servers)), key=self._load)
        return self.servers[self.home[req.key]].submit(req, now)

    def pending_work(self) -> bool:
        return any(s.pending_work() for s in self.servers)

    def step(self, now: Optional[float] = None) -> List[Request]:
        done: List[Request] = []
        for srv in self.servers:
            done += srv.step(now)
        return done

    @property
    def cycles(self) -> int:
        return sum(s.cycles for s in self.servers)

    @property
    def evictions(self) -> int:
        return sum(s.evictions for s in self.servers)

    def drain(self, idle_sleep: float = 2e-4) -> List[Request]:
        done: List[Request] = []
        while self.pending_work():
            got = self.step()
            done += got
            if not got:
                time.sleep(idle_sleep)
        return done

    def close(self):
        for srv in self.servers:
            srv.close()


def run_stream(server: Server, requests: List[Request], arrivals: np.ndarray, idle_sleep: float = 1e-4) -> dict:
    """Feeds `requests` at the given arrival offsets (seconds from start) and
    serves until all are done.  Returns latency percentiles and throughput."""
    order = np.argsort(arrivals, kind="stable")
    t0 = time.perf_counter()
    nxt = 0
    done: List[Request] = []
    while nxt < len(order) or server.pending_work():
        now = time.perf_counter()
        while nxt < len(order) and arrivals[order[nxt]] <= now - t0:
            r = requests[order[nxt]]
            server.submit(r, now=t0 + float(arrivals[order[nxt]]))
            nxt += 1
        got = server.step(now)
        done += got
        if not got:
            time.sleep(idle_sleep)
    t_end = time.perf_counter()
    served = [r for r in requests if r.latency is not None and r.status != "rejected"]
    lat = np.array([r.latency for r in served])
    # queueing: arrival to the request's load into slots; service: load to result
    queue = np.array([r.t_admitted - r.t_arrival for r in served if r.t_admitted is not None])
    service = np.array([r.t_done - r.t_admitted for r in served if r.t_admitted is not None])
    solves = sum(r.nrhs for r in requests if r.status in ("done", "maxiter", "diverged"))

    def pct(a, q):
        return 1e3 * float(np.percentile(a, q)) if a.size else None

    return {"requests": len(requests), "completed": sum(r.status == "done" for r in requests),
            "rejected": sum(r.status == "rejected" for r in requests),
            "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99),
            "mean_ms": 1e3 * float(lat.mean()) if lat.size else None,
            "queue_p50_ms": pct(queue, 50), "queue_p99_ms": pct(queue, 99),
            "service_p50_ms": pct(service, 50), "service_p99_ms": pct(service, 99),
            "makespan_s": t_end - t0, "solves": solves, "solves_per_s": solves / (t_end - t0),
            "cycles": server.cycles, "evictions": server.evictions}


def poisson_arrivals(n: int, rate: float, seed: int = 7) -> np.ndarray:
    """Arrival offsets (s) of a Poisson process with the given rate (seeded)."""
    u = np.maximum(inputs.uniform01(seed, n), 1e-300)
    return np.cumsum(-np.log(u) / rate)


def request_mix(keys: List[Key], n: int, rhs_of_key, seed: int = 11, max_rhs: int = 16) -> List[Request]:
    """n requests, keys uniform over `keys`, 1..max_rhs right-hand sides each.
    rhs_of_key(key) gives (f, N) for the key's load vector."""
    u = inputs.uniform01(seed, 2 * n)
    out = []
    for i in range(n):
        key = keys[min(int(u[2 * i] * len(keys)), len(keys) - 1)]
        nr = 1 + min(int(u[2 * i + 1] * max_rhs), max_rhs - 1)
        f, N = rhs_of_key(key)
        F = inputs.batched_rhs(f, nr, seed=1000 + 7 * i)
        U0 = np.stack([inputs.initial_guess(N, 50000 + 31 * i + r) for r in range(nr)])
        out.append(Request(rid=i, key=key, F=F, U0=U0))
    return out


class GpuBackend:
    """The CUDA library behind the server: one Solver (hierarchy + arena +
    S-slot workspace) and one stream per resident key."""

    def __init__(self, device: str = "cuda", autotune: bool = True, budget_fraction: float = 0.8):
        import torch
        from . import pmg
        self.torch, self.pmg = torch, pmg
        self.device = device
        self.autotune = autotune
        self.budget_fraction = budget_fraction
        self._hier = {}             # key -> host hierarchy handle kept for size queries

    def memory_budget(self) -> int:
        free, _total = self.torch.cuda.mem_get_info()
        return int(free * self.budget_fraction)

    def bytes_needed(self, key: Key, slots: int) -> int:
        pmg = self.pmg
        self.prepare(key)
        h = self._hier[key]
        return int(pmg.pmg_info(h).device_bytes + pmg.pmg_workspace_bytes(h, slots))

    def prepare(self, key: Key):
        """Host setup of a key's hierarchy (assembly, ILUT, transfers); thread-safe."""
        if key not in self._hier:
            self._hier[key] = self.pmg.pmg_setup(*key)

    def create(self, key: Key, slots: int):
        torch, pmg = self.torch, self.pmg
        self.prepare(key)
        S = pmg.Solver(*key, device=self.device, upload=False, max_rhs=slots, handle=self._hier.pop(key))
        S.upload(self.device)
        if self.autotune:
            S.autotune()
        stream = torch.cuda.Stream(device=self.device)
        return {"S": S, "stream": stream, "slots": slots}

    def free(self, handle):
        handle["stream"].synchronize()
        S = handle["S"]
        S.__del__()
        S.ws = None
        S.h = None

    def load(self, handle, slot0: int, F: np.ndarray, U0: np.ndarray):
        torch, pmg = self.torch, self.pmg
        s = handle["stream"]
        with torch.cuda.stream(s):
            Fd = torch.as_tensor(np.ascontiguousarray(F), device=self.device)
            Ud = torch.as_tensor(np.ascontiguousarray(U0), device=self.device)
            pmg.pmg_slots_load(handle["S"].h, handle["S"].ws, slot0, Fd, Ud, stream=s)
            handle.setdefault("keep", []).append((Fd, Ud))     # alive until the copies ran

    def cycle(self, handle, precision: int, rel_tol: float):
        self.pmg.pmg_slots_cycle(handle["S"].h, handle["S"].ws, precision, rel_tol, stream=handle["stream"])

    def poll(self, handle, blocking: bool = False):
        res = self.pmg.pmg_slots_wait(handle["S"].h, handle["S"].ws, handle["slots"], blocking=blocking)
        if res is not None:
            handle["keep"] = []
        return res

    def read(self, handle, slot0: int, n: int) -> np.ndarray:
        torch, pmg = self.torch, self.pmg
        s = handle["stream"]
        S = handle["S"]
        with torch.cuda.stream(s):
            U = torch.empty((n, S.N), dtype=torch.float64, device=self.device)
            pmg.pmg_slots_read(S.h, S.ws, slot0, U, stream=s)
            out = U.cpu()                      # waits for the copy on this stream
        return out.numpy()

    def release(self, handle, slot0: int, n: int):
        self.pmg.pmg_slots_release(handle["S"].h, handle["S"].ws, slot0, n, stream=handle["stream"])
