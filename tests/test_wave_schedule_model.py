"""Executable model of the wavefront Gauss-Seidel sweep's schedule (k_gs_wave
in csrc/kernels.cuh), run on the CPU against the sequential sweep.

The sweep's lower solve on an m x m grid (9-point stencil, lexicographic
order, first index fastest) is x(l, c) = t - c_SW x(l-1, c-1) - c_S x(l-1, c)
- c_SE x(l-1, c+1) - c_W x(l, c-1).  The kernel gives grid line l = 32 w + k
to lane k of warp w; at step s lane k computes column s - 2k.  Lane k - 1's
output of the previous step is the line below at column c + 1 (one shuffle);
lane 0 of warp w > 0 reads warp w - 1's lane 31 from a boundary buffer, and
starts with that line's column 0 in its history.  The products with the two
older values of the line below (SW, S) of the next point are formed during the
current step.  Inactive steps (columns outside the line) produce zeros that
must not disturb active lanes.

The model follows the kernel step by step, lane by lane, warp after warp (the
boundary buffer holds the finished lower line), and checks:
  1. the result equals the sequential sweep to rounding, for sizes with one
     or several warps and ragged last warps;
  2. dropping the column-0 preload of lane 0 (the fault the benchmark-size
     parity test once caught) gives a wrong result whenever there are two or
     more warps, so the check has teeth.
"""
import numpy as np
import pytest


def sequential(m, t, C):
    x = np.zeros((m, m))
    for l in range(m):
        for c in range(m):
            i = l * m + c

            def X(ll, cc):
                return x[ll, cc] if 0 <= ll < m and 0 <= cc < m else 0.0
            x[l, c] = (t[i] - C[i, 0] * X(l - 1, c - 1) - C[i, 1] * X(l - 1, c)
                       - C[i, 2] * X(l - 1, c + 1) - C[i, 3] * X(l, c - 1))
    return x.ravel()


def wavefront(m, t, C, preload=True):
    nw = (m + 31) // 32
    x = np.full(m * m, np.nan)
    incoming = None                      # boundary line of the previous warp
    for w in range(nw):
        steps = m + 62

        def data(k, s):
            l, c = 32 * w + k, s - 2 * k
            if l < m and 0 <= c < m:
                i = l * m + c
                return t[i], C[i]
            return 0.0, np.zeros(4)

        bm1, bm2, xl, got = np.zeros(32), np.zeros(32), np.zeros(32), np.zeros(32)
        if w > 0 and preload:
            bm1[0] = incoming[0]
        part = np.array([data(k, 0)[0] - data(k, 0)[1][0] * bm2[k] - data(k, 0)[1][1] * bm1[k] for k in range(32)])
        outgoing = np.zeros(m) if w + 1 < nw else None
        for s in range(steps):
            out, newpart, bs_all = np.zeros(32), np.zeros(32), np.zeros(32)
            for k in range(32):
                l, c = 32 * w + k, s - 2 * k
                bs = 0.0 if k == 0 else got[k]
                if k == 0 and w > 0 and s + 1 < m:
                    bs = incoming[s + 1]
                _, cq = data(k, s)
                tn, cn = data(k, s + 1)
                o1 = part[k] - cq[3] * xl[k]
                pn1 = tn - cn[0] * bm1[k]
                o = o1 - cq[2] * bs
                newpart[k] = pn1 - cn[1] * bs
                active = l < m and 0 <= c < m
                o = o if active else 0.0
                out[k], bs_all[k] = o, bs
                if active:
                    x[l * m + c] = o
                    if k == 31 and outgoing is not None:
                        outgoing[c] = o
            got = np.concatenate([[out[0]], out[:-1]])      # shuffle up by one lane
            xl, bm2, bm1, part = out.copy(), bm1.copy(), bs_all.copy(), newpart
        incoming = outgoing
    return x


@pytest.mark.parametrize("m", [2, 3, 17, 31, 32, 33, 64, 70])
def test_wavefront_schedule_equals_sequential_sweep(m):
    rng = np.random.default_rng(m)
    t = rng.standard_normal(m * m)
    C = 0.3 * rng.standard_normal((m * m, 4))
    ref = sequential(m, t, C)
    got = wavefront(m, t, C)
    assert not np.isnan(got).any()
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("m", [33, 64])
def test_missing_boundary_preload_is_detected(m):
    rng = np.random.default_rng(7)
    t = rng.standard_normal(m * m)
    C = 0.3 * rng.standard_normal((m * m, 4))
    ref = sequential(m, t, C)
    bad = wavefront(m, t, C, preload=False)
    assert np.abs(bad - ref).max() > 1e-6 * np.abs(ref).max()
