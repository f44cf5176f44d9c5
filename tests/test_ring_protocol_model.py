"""Executable model of the ring kernel's hand-over protocol (k_lpc in
csrc/kernels_batched.cuh), explored under random interleavings on the CPU.

Per line: producer warps fill a ring of S hand-over slots (row ix -> slot
ix mod S); each slot carries one value per lane (s_i for that lane's
right-hand side) plus a row of coefficients written one per lane and read in
full by every chain lane.  A pending value means "slot empty".  The chain
lanes take the rows in order, read the row's coefficients, then release
their own lane's slot.  Lanes run independently (independent thread
scheduling): the model schedules every lane of every warp as its own thread.

The properties checked are the ones the kernel relies on:
  1. with a producer count dividing S and the producer warp converging
     (__syncwarp) before overwriting the coefficients and before publishing,
     every chain lane reads exactly the coefficients of the row it processes,
     and the protocol never deadlocks;
  2. without the convergence, some interleaving makes a chain lane read the
     coefficients of another row (the race the kernel fixed);
  3. with a producer count that does not divide S, some interleaving fills a
     slot with a later row before the earlier one was taken.
"""
import random

import pytest

PENDING = None


class Model:
    def __init__(self, lanes, slots, producers, rows, converge, seed):
        self.L, self.S, self.P, self.rows = lanes, slots, producers, rows
        self.converge = converge
        self.rng = random.Random(seed)
        self.sb = [[PENDING] * lanes for _ in range(slots)]     # s values (row index as payload)
        self.cb = [[-1] * lanes for _ in range(slots)]          # coefficients (row index as payload)
        self.errors = []
        # producer lane state: (next row, phase)
        self.prod = {(p, l): [p, "wait_free"] for p in range(producers) for l in range(lanes)}
        self.chain = {l: [0, "wait_filled"] for l in range(lanes)}
        self.barrier = {p: [set(), 0] for p in range(producers)}   # arrived lanes, generation

    def step_producer(self, p, l):
        st = self.prod[(p, l)]
        ix, phase = st[0], st[1]
        if ix >= self.rows:
            return False
        k = ix % self.S
        if phase == "wait_free":
            if self.sb[k][l] is not PENDING:
                return False
            st[1] = "sync1" if self.converge else "write_cb"
            return True
        if phase in ("sync1", "sync2"):
            arrived, gen = self.barrier[p]
            if len(st) < 3:
                st.append(gen)
            if st[2] != gen:              # the barrier completed since this lane arrived
                st.pop()
                st[1] = "write_cb" if phase == "sync1" else "publish"
                return True
            arrived.add(l)
            if len(arrived) == self.L:
                self.barrier[p] = [set(), gen + 1]
            return False
        if phase == "write_cb":
            self.cb[k][l] = ix
            st[1] = "sync2" if self.converge else "publish"
            return True
        if phase == "publish":
            if self.sb[k][l] is not PENDING:
                self.errors.append(("overwrite", ix, l))
            self.sb[k][l] = ix
            st[0], st[1] = ix + self.P, "wait_free"
            return True
        raise AssertionError(phase)

    def step_chain(self, l):
        st = self.chain[l]
        ix = st[0]
        if ix >= self.rows:
            return False
        k = ix % self.S
        if self.sb[k][l] is PENDING:
            return False
        if self.sb[k][l] != ix:
            self.errors.append(("wrong s", ix, l, self.sb[k][l]))
        if any(c != ix for c in self.cb[k]):
            self.errors.append(("stale coefficients", ix, l, list(self.cb[k])))
        self.sb[k][l] = PENDING                   # release after the pushes consumed the coefficients
        st[0] = ix + 1
        return True

    def run(self):
        actors = [("p", p, l) for p in range(self.P) for l in range(self.L)] + [("c", l) for l in range(self.L)]
        idle = 0
        while True:
            done = all(v[0] >= self.rows for v in self.chain.values())
            if done:
                return True
            a = self.rng.choice(actors)
            moved = self.step_producer(a[1], a[2]) if a[0] == "p" else self.step_chain(a[1])
            idle = 0 if moved else idle + 1
            if idle > 50 * len(actors):
                # nobody can move: check it is a real deadlock, not an unlucky draw
                if not any((self.step_producer(a[1], a[2]) if a[0] == "p" else self.step_chain(a[1]))
                           for a in actors):
                    return False
                idle = 0


@pytest.mark.parametrize("producers", [1, 2, 4, 8])
def test_protocol_is_correct_and_deadlock_free(producers):
    for seed in range(60):
        m = Model(lanes=4, slots=8, producers=producers, rows=40, converge=True, seed=seed)
        assert m.run(), f"deadlock (P={producers}, seed={seed})"
        assert not m.errors, m.errors[:3]


def test_without_warp_convergence_a_chain_lane_reads_another_rows_coefficients():
    hits = 0
    for seed in range(200):
        m = Model(lanes=4, slots=8, producers=4, rows=40, converge=False, seed=seed)
        m.run()
        hits += any(e[0] == "stale coefficients" for e in m.errors)
    assert hits > 0


def test_a_producer_count_not_dividing_the_slots_breaks_slot_ownership():
    hits = 0
    for seed in range(200):
        m = Model(lanes=2, slots=8, producers=3, rows=40, converge=True, seed=seed)
        finished = m.run()
        hits += (not finished) or any(e[0] in ("wrong s", "overwrite") for e in m.errors)
    assert hits > 0
