"""Executable model of the hand-over between consecutive lines of one cluster
in the clustered triangular solve (k_lp4 with several lines a cluster, in
csrc/kernels.cuh), explored under random interleavings on the CPU.

A cluster takes a group of consecutive lines at a time.  The chain of line k
pushes each finished value of its line into a buffer in the shared memory of
line k+1's producer CTA; that producer polls the buffer for the entries its
rows need (not necessarily all of them), then moves on to the next group:
it resets a receiving buffer to "pending" and meets the other CTAs at one
cluster barrier per group.  The chain of line k may still be storing the last
values of its line when line k+1's producer, done early, resets a buffer for
the next group.

The kernel alternates between two buffers by group parity.  The model checks:
  1. with two buffers, every value a producer reads belongs to its own group
     (no stale value from an earlier group) and nothing deadlocks;
  2. with one buffer, some interleaving lets a late store of the previous
     group land after the reset, so that the producer reads a stale value
     (the race the second buffer removes).
"""
import random

import pytest

PENDING = None


def run(nx, groups, buffers, seed):
    rnd = random.Random(seed)
    buf = [[PENDING] * nx for _ in range(buffers)]
    arrived = {}                                   # barrier of group g: set of parties arrived
    # entries line k+1's rows need from line k in each group: a prefix-heavy random subset
    needs = [sorted(rnd.sample(range(nx), rnd.randint(1, nx))) for _ in range(groups)]
    errors = []

    def barrier(g, who):
        arrived.setdefault(g, set()).add(who)
        while len(arrived[g]) < 2:
            yield

    def chain():
        for g in range(groups):
            yield from barrier(g, "chain")
            b = buf[g % buffers]
            for ix in range(nx):
                b[ix] = (g, ix)                        # one store a step
                yield

    def producer():
        for g in range(groups):
            b = buf[g % buffers]
            for ix in range(nx):                       # reset before the group's barrier
                b[ix] = PENDING
            yield
            yield from barrier(g, "producer")
            for ix in needs[g]:
                while b[ix] is PENDING:
                    yield
                if b[ix] != (g, ix):
                    errors.append((g, ix, b[ix]))
                yield

    threads = [chain(), producer()]
    live = list(threads)
    steps = 0
    while live:
        t = rnd.choice(live)
        try:
            next(t)
        except StopIteration:
            live.remove(t)
        steps += 1
        if steps > 200000:
            raise AssertionError("no progress (deadlock)")
    return errors


@pytest.mark.parametrize("seed", range(200))
def test_two_buffers_never_read_a_stale_value(seed):
    assert run(nx=6, groups=6, buffers=2, seed=seed) == []


def test_one_buffer_reads_a_stale_value_in_some_interleaving():
    stale = sum(1 for seed in range(400) if run(nx=6, groups=6, buffers=1, seed=seed))
    assert stale > 0
