"""Python access to the plain FP64 CPU oracle (pmg_oracle.c).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use this
module.  The library in ``paper_1901_01685_gb300`` never imports it, and this
module never imports the library.

The C source follows the paper (arXiv 1901.01685) step by step; see the header
of ``pmg_oracle.c`` for the readings of passages the paper leaves open.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pmg_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")

ANNULUS, SQUARE, CUBE, CDR_SQUARE = 0, 1, 2, 3
U_SINPROD, U_PAPER_B1 = 0, 1
INDIRECT, DIRECT = 0, 1
STATUS = {0: "ok", 1: "arg", 2: "oom", 3: "zero_pivot", 4: "diverged", 5: "maxiter"}

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (single thread, -O2, no FP contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        L.or_bspline.restype = C.c_double
        L.or_bspline.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_int]
        L.or_gauss.argtypes = [C.c_int, dp, dp]
        L.or_u_exact.restype = C.c_double
        L.or_u_exact.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double]
        L.or_f_source.restype = C.c_double
        L.or_f_source.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double]
        L.or_setup.restype = C.c_void_p
        L.or_setup.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int,
                               C.c_int, C.c_int, C.c_int, C.c_int, ip]
        L.or_free.argtypes = [C.c_void_p]
        for name in ("or_nlev", "or_nh"):
            getattr(L, name).argtypes = [C.c_void_p]
        for name in ("or_level_N", "or_level_q", "or_hlevel_N"):
            getattr(L, name).argtypes = [C.c_void_p, C.c_int]
        L.or_get_csr.argtypes = [C.c_void_p, C.c_int, C.c_int, ip, ip, ip, ip, ip, dp]
        L.or_get_ml.argtypes = [C.c_void_p, C.c_int, dp]
        L.or_get_rhs.argtypes = [C.c_void_p, dp]
        L.or_residual.argtypes = [C.c_void_p, C.c_int, dp, dp, dp]
        L.or_smooth.argtypes = [C.c_void_p, C.c_int, dp, dp]
        L.or_restrict.argtypes = [C.c_void_p, C.c_int, dp, dp]
        L.or_prolong_add.argtypes = [C.c_void_p, C.c_int, dp, dp]
        L.or_coarse_solve.argtypes = [C.c_void_p, dp, dp]
        L.or_hmg_vcycle.argtypes = [C.c_void_p, C.c_int, dp, dp]
        L.or_gs.argtypes = [C.c_void_p, C.c_int, C.c_int, dp, dp]
        L.or_vcycle.argtypes = [C.c_void_p, C.c_int, dp, dp]
        L.or_solve.argtypes = [C.c_void_p, dp, dp, C.c_double, C.c_int, dp, dp, ip]
        L.or_l2_error.restype = C.c_double
        L.or_l2_error.argtypes = [C.c_void_p, dp]
        L.or_ilut.argtypes = [C.c_int, ip, ip, dp, C.c_double, C.c_double, ip, ip,
                              ip, ip, dp, ip, ip, dp, C.c_int]
        L.or_ilut_budget.argtypes = [C.c_longlong, C.c_int, C.c_double]
        L.or_use_consistent.argtypes = [C.c_void_p]
        L.or_full_matrix.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, ip, ip, ip, ip, ip, dp]
        L.or_full_load.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, dp]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_int))


class CSR:
    """Minimal CSR triple with a dense view for small checks."""

    def __init__(self, nr, nc, rp, ci, v):
        self.shape = (nr, nc)
        self.rp, self.ci, self.v = rp, ci, v

    @property
    def nnz(self):
        return int(self.rp[-1])

    def dense(self) -> np.ndarray:
        a = np.zeros(self.shape)
        for i in range(self.shape[0]):
            s, e = self.rp[i], self.rp[i + 1]
            a[i, self.ci[s:e]] += self.v[s:e]
        return a

    def matvec(self, x: np.ndarray) -> np.ndarray:
        rows = np.repeat(np.arange(self.shape[0]), np.diff(self.rp))
        y = np.zeros(self.shape[0])
        np.add.at(y, rows, self.v * x[self.ci])
        return y


def bspline(p: int, ne: int, i: int, x: float, deriv: int = 0) -> float:
    return lib().or_bspline(p, ne, i, x, deriv)


def gauss(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().or_gauss(n, _dp(x), _dp(w))
    return x, w


def u_exact(dom, ex, x, y, z=0.0):
    return lib().or_u_exact(dom, ex, x, y, z)


def f_source(dom, ex, x, y, z=0.0):
    return lib().or_f_source(dom, ex, x, y, z)


def ilut_budget(nnz: int, n: int, m: float) -> int:
    return lib().or_ilut_budget(nnz, n, m)


def ilut(a: CSR, tau: float, fill: float):
    """ILUT of a caller matrix; returns (L strict lower, U upper with diagonal)."""
    n = a.shape[0]
    rp = np.ascontiguousarray(a.rp, dtype=np.int32)
    ci = np.ascontiguousarray(a.ci, dtype=np.int32)
    v = np.ascontiguousarray(a.v, dtype=np.float64)
    cap = n * n + 1
    lrp = np.zeros(n + 1, np.int32); urp = np.zeros(n + 1, np.int32)
    lci = np.zeros(cap, np.int32); uci = np.zeros(cap, np.int32)
    lv = np.zeros(cap); uv = np.zeros(cap)
    nl = C.c_int(); nu = C.c_int()
    st = lib().or_ilut(n, _ip(rp), _ip(ci), _dp(v), tau, fill, C.byref(nl), C.byref(nu),
                       _ip(lrp), _ip(lci), _dp(lv), _ip(urp), _ip(uci), _dp(uv), cap)
    if st:
        raise RuntimeError(f"or_ilut failed: {STATUS.get(st, st)}")
    return (CSR(n, n, lrp, lci[:nl.value].copy(), lv[:nl.value].copy()),
            CSR(n, n, urp, uci[:nu.value].copy(), uv[:nu.value].copy()))


def full_matrix(dom: int, k: int, q: int, r: int, kind: str) -> CSR:
    """Full-space (no boundary elimination) stiffness ('stiff') or mass ('mass') matrix,
    test degree q, trial degree r, h = 2^-k."""
    kk = {"stiff": 0, "mass": 1}[kind]
    nr, nc, nnz = C.c_int(), C.c_int(), C.c_int()
    L = lib()
    st = L.or_full_matrix(dom, k, q, r, kk, C.byref(nr), C.byref(nc), C.byref(nnz), None, None, None)
    if st:
        raise RuntimeError(STATUS.get(st, st))
    rp = np.zeros(nr.value + 1, np.int32); ci = np.zeros(nnz.value, np.int32); v = np.zeros(nnz.value)
    st = L.or_full_matrix(dom, k, q, r, kk, C.byref(nr), C.byref(nc), C.byref(nnz), _ip(rp), _ip(ci), _dp(v))
    if st:
        raise RuntimeError(STATUS.get(st, st))
    return CSR(nr.value, nc.value, rp, ci, v)


def full_load(dom: int, ex: int, k: int, q: int) -> np.ndarray:
    d = 3 if dom == CUBE else 2
    n = (1 << k) + q
    out = np.zeros(n ** d)
    st = lib().or_full_load(dom, ex, k, q, _dp(out))
    if st:
        raise RuntimeError(STATUS.get(st, st))
    return out


class Hierarchy:
    """Oracle p-multigrid hierarchy: operators, ILUT factors, transfers and the
    p = 1 h-multigrid levels for one (domain, p, h) problem."""

    def __init__(self, domain: int, p: int, k: int, tau: float = 1e-12, fill: float = 1.0,
                 projection: int = INDIRECT, exact: int = U_SINPROD, nu1: int = 1, nu2: int = 1,
                 coarse_cycles: int = 2, consistent: bool = False):
        st = C.c_int()
        self._L = lib()
        self._h = self._L.or_setup(domain, p, k, tau, fill, projection, exact, nu1, nu2,
                                   coarse_cycles, C.byref(st))
        if not self._h:
            raise RuntimeError(f"or_setup failed: {STATUS.get(st.value, st.value)}")
        # transfers with the consistent mass matrices instead of the lumped ones (App. B)
        if consistent:
            cst = self._L.or_use_consistent(self._h)
            if cst:
                raise RuntimeError(f"or_use_consistent failed: {STATUS.get(cst, cst)}")
        self.domain, self.p, self.k, self.projection = domain, p, k, projection
        self.nlev = self._L.or_nlev(self._h)
        self.nh = self._L.or_nh(self._h)
        self.N = [self._L.or_level_N(self._h, l) for l in range(self.nlev)]
        self.q = [self._L.or_level_q(self._h, l) for l in range(self.nlev)]
        self.NH = [self._L.or_hlevel_N(self._h, j) for j in range(self.nh)]

    def __del__(self):
        if getattr(self, "_h", None):
            self._L.or_free(self._h)
            self._h = None

    # ---- exported data ----
    def csr(self, which: str, level: int) -> CSR:
        w = {"A": 0, "L": 1, "U": 2, "P": 3, "Pt": 4, "A1": 5, "Pc": 6, "Rc": 7}[which]
        nr, nc, nnz = C.c_int(), C.c_int(), C.c_int()
        st = self._L.or_get_csr(self._h, w, level, C.byref(nr), C.byref(nc), C.byref(nnz), None, None, None)
        if st:
            raise RuntimeError(f"no matrix {which} at level {level}")
        rp = np.zeros(nr.value + 1, np.int32); ci = np.zeros(nnz.value, np.int32); v = np.zeros(nnz.value)
        self._L.or_get_csr(self._h, w, level, C.byref(nr), C.byref(nc), C.byref(nnz), _ip(rp), _ip(ci), _dp(v))
        return CSR(nr.value, nc.value, rp, ci, v)

    def lumped_mass(self, level: int) -> np.ndarray:
        n = self.N[level] if level < self.nlev else self.NH[0]
        out = np.zeros(n)
        if self._L.or_get_ml(self._h, level, _dp(out)):
            raise RuntimeError("bad level")
        return out

    def rhs(self) -> np.ndarray:
        f = np.zeros(self.N[0])
        self._L.or_get_rhs(self._h, _dp(f))
        return f

    def coarse_N(self, level: int) -> int:
        return self.N[level + 1] if level + 1 < self.nlev else self.NH[0]

    # ---- hot-path steps ----
    def residual(self, level, f, u):
        r = np.zeros(self.N[level])
        self._L.or_residual(self._h, level, _dp(np.ascontiguousarray(f)), _dp(np.ascontiguousarray(u)), _dp(r))
        return r

    def smooth(self, level, f, u):
        u = np.array(u, dtype=np.float64, copy=True)
        self._L.or_smooth(self._h, level, _dp(np.ascontiguousarray(f)), _dp(u))
        return u

    def restrict(self, level, r):
        rc = np.zeros(self.coarse_N(level))
        self._L.or_restrict(self._h, level, _dp(np.ascontiguousarray(r)), _dp(rc))
        return rc

    def prolong_add(self, level, ec, u):
        u = np.array(u, dtype=np.float64, copy=True)
        self._L.or_prolong_add(self._h, level, _dp(np.ascontiguousarray(ec)), _dp(u))
        return u

    def coarse_solve(self, r1):
        e1 = np.zeros(self.NH[0])
        self._L.or_coarse_solve(self._h, _dp(np.ascontiguousarray(r1)), _dp(e1))
        return e1

    def hmg_vcycle(self, j, b, x):
        x = np.array(x, dtype=np.float64, copy=True)
        self._L.or_hmg_vcycle(self._h, j, _dp(np.ascontiguousarray(b)), _dp(x))
        return x

    def gs(self, j, b, x, backward=False):
        x = np.array(x, dtype=np.float64, copy=True)
        self._L.or_gs(self._h, j, int(backward), _dp(np.ascontiguousarray(b)), _dp(x))
        return x

    def vcycle(self, level, f, u):
        u = np.array(u, dtype=np.float64, copy=True)
        self._L.or_vcycle(self._h, level, _dp(np.ascontiguousarray(f)), _dp(u))
        return u

    def solve(self, f, u0, tol=1e-8, maxit=100):
        u = np.zeros(self.N[0])
        hist = np.zeros(maxit)
        it = C.c_int()
        st = self._L.or_solve(self._h, _dp(np.ascontiguousarray(f)), _dp(np.ascontiguousarray(u0)),
                              tol, maxit, _dp(u), _dp(hist), C.byref(it))
        return u, hist[: it.value].copy(), it.value, STATUS.get(st, st)

    def bicgstab(self, f, u0, tol=1e-8, maxit=100, precond=None):
        """BiCGSTAB (van der Vorst, SIAM J. Sci. Stat. Comput. 13, 1992) with
        right preconditioning by one p-multigrid V-cycle with zero initial guess
        per application (Sec. 5, "p-Multigrid as a preconditioner"; two
        applications per iteration).  Stops when the recursively updated
        residual satisfies ||r|| / ||r0|| < tol, tested after the half step (s)
        and after the full step; an exit at the half step counts the iteration
        in progress.  `precond(v)` replaces the V-cycle when given.
        Returns (u, history of relative residuals per iteration, iterations,
        status)."""
        A = self.csr("A", 0)
        M = precond if precond is not None else (lambda v: self.vcycle(0, v, np.zeros_like(v)))
        x = np.array(u0, dtype=np.float64, copy=True)
        r = np.asarray(f, dtype=np.float64) - A.matvec(x)
        r0n = np.linalg.norm(r)
        if r0n == 0.0:
            return x, np.zeros(0), 0, "ok"
        rhat = r.copy()
        p = np.zeros_like(r)
        v = np.zeros_like(r)
        rho_prev = alpha = omega = 1.0
        hist = []
        for it in range(1, maxit + 1):
            rho = float(rhat @ r)
            if rho == 0.0:
                return x, np.array(hist), it - 1, "breakdown"
            if it == 1:
                p = r.copy()
            else:
                beta = (rho / rho_prev) * (alpha / omega)
                p = r + beta * (p - omega * v)
            phat = M(p)
            v = A.matvec(phat)
            alpha = rho / float(rhat @ v)
            s = r - alpha * v
            if np.linalg.norm(s) / r0n < tol:
                x = x + alpha * phat
                hist.append(np.linalg.norm(s) / r0n)
                return x, np.array(hist), it, "ok"
            shat = M(s)
            t = A.matvec(shat)
            omega = float(t @ s) / float(t @ t)
            x = x + alpha * phat + omega * shat
            r = s - omega * t
            rel = np.linalg.norm(r) / r0n
            hist.append(rel)
            if rel < tol:
                return x, np.array(hist), it, "ok"
            if not rel <= 1e10:
                return x, np.array(hist), it, "diverged"
            rho_prev = rho
        return x, np.array(hist), maxit, "maxiter"

    def l2_error(self, u) -> float:
        return self._L.or_l2_error(self._h, _dp(np.ascontiguousarray(u, dtype=np.float64)))
