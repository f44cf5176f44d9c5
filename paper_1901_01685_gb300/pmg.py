"""Thin ctypes binding of the C-ABI in include/pmg.h.

Functions carry the C names and only marshal arguments: torch tensors become
device pointers, the current torch CUDA stream becomes the cudaStream_t, and
torch provides the device memory for the hierarchy arena and the workspaces.
Every step of the solve runs in the CUDA kernels of libpmg.so; there is no
CPU fallback, and importing this module fails loudly if the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_LIB_PATH = _build.LIB

PMG_OK, PMG_ERR_ARG, PMG_ERR_OOM, PMG_ERR_ZERO_PIVOT, PMG_ERR_DIVERGED, PMG_ERR_MAXITER, \
    PMG_ERR_TIMEOUT, PMG_ERR_CUDA, PMG_ERR_BUSY, PMG_ERR_STATE = range(10)
STATUS_NAMES = {0: "ok", 1: "arg", 2: "oom", 3: "zero_pivot", 4: "diverged", 5: "maxiter",
                6: "timeout", 7: "cuda", 8: "busy", 9: "state"}
PMG_QUARTER_ANNULUS, PMG_UNIT_SQUARE, PMG_UNIT_CUBE, PMG_CDR_SQUARE = 0, 1, 2, 3
PMG_U_SINPROD, PMG_U_PAPER_B1 = 0, 1
PMG_PROJ_INDIRECT, PMG_PROJ_DIRECT = 0, 1
PMG_MASS_LUMPED, PMG_MASS_CONSISTENT = 0, 1   # transfer mass matrix (Sec. 3, App. B)
(PMG_OP_RESIDUAL, PMG_OP_SMOOTH, PMG_OP_LSOLVE, PMG_OP_USOLVE, PMG_OP_RESTRICT, PMG_OP_PROLONG_ADD,
 PMG_OP_COARSE_SOLVE, PMG_OP_VCYCLE, PMG_OP_GS_FWD, PMG_OP_GS_BWD, PMG_OP_HMG_VCYCLE) = range(11)
PMG_MAX_LEVELS = 16
PMG_PREC_FP64, PMG_PREC_MIXED, PMG_PREC_MIXED_FP16, PMG_PREC_MIXED_BF16 = 0, 1, 2, 3

# every symbol include/pmg.h declares
EXPORTS = ("pmg_default_options", "pmg_setup", "pmg_info", "pmg_upload", "pmg_rhs", "pmg_workspace_bytes",
           "pmg_workspace_create", "pmg_solve", "pmg_solve_host", "pmg_solve_bicgstab", "pmg_solve_batched", "pmg_slots_load", "pmg_slots_cycle",
           "pmg_slots_wait", "pmg_slots_read", "pmg_slots_release", "pmg_autotune", "pmg_set_kernels", "pmg_apply",
           "pmg_export_csr",
           "pmg_export_lumped", "pmg_l2_error", "pmg_ws_profile", "pmg_ws_stats", "pmg_lsolve_noalloc",
           "pmg_ws_destroy", "pmg_destroy", "pmg_last_error")
PMG_NKERN = 8
KERNEL_CLASSES = ("residual", "transfer", "lsolve", "usolve", "gauss_seidel", "p1", "coarse", "norm")


class pmg_options(C.Structure):
    _fields_ = [("drop_tol", C.c_double), ("fill_factor", C.c_double), ("nu_pre", C.c_int),
                ("nu_post", C.c_int), ("projection", C.c_int), ("coarse_cycles", C.c_int),
                ("exact", C.c_int), ("transfer_mass", C.c_int)]


_L16 = C.c_int * PMG_MAX_LEVELS
_LL16 = C.c_longlong * PMG_MAX_LEVELS


class pmg_info_t(C.Structure):
    _fields_ = [("dim", C.c_int), ("p", C.c_int), ("log2_inv_h", C.c_int), ("nlevels", C.c_int),
                ("degree", _L16), ("n", _L16), ("nnz_A", _LL16), ("nnz_L", _LL16), ("nnz_U", _LL16),
                ("nnz_P", _LL16), ("depth_L", _L16), ("depth_U", _L16), ("nhlevels", C.c_int),
                ("n_h", _L16), ("nnz_h", _LL16), ("depth_gs", _L16), ("device_bytes", C.c_size_t),
                ("setup_ms_assembly", C.c_double), ("setup_ms_ilut", C.c_double),
                ("setup_ms_transfer", C.c_double), ("setup_ms_hmg", C.c_double),
                ("cycle_bytes", C.c_double), ("cycle_flops", C.c_double), ("tune_p", _L16), ("tune_h", _L16)]

    def as_dict(self) -> dict:
        nl, nh = self.nlevels, self.nhlevels
        d = {k: getattr(self, k) for k in ("dim", "p", "log2_inv_h", "nlevels", "nhlevels", "device_bytes",
                                          "setup_ms_assembly", "setup_ms_ilut", "setup_ms_transfer",
                                          "setup_ms_hmg", "cycle_bytes", "cycle_flops")}
        for k in ("degree", "n", "nnz_A", "nnz_L", "nnz_U", "nnz_P", "depth_L", "depth_U"):
            d[k] = list(getattr(self, k))[:nl]
        for k in ("n_h", "nnz_h", "depth_gs"):
            d[k] = list(getattr(self, k))[:nh]
        names = ("windowed", "ring", "lines", "cluster")
        d["kernels_p"] = [{f: names[(v >> (2 * b)) & 3] for b, f in enumerate(
            ("single_L", "single_U", "batched64_L", "batched64_U", "batched32_L", "batched32_U"))}
            for v in list(self.tune_p)[:nl]]
        for v, k in zip(list(self.tune_p)[:nl], d["kernels_p"]):
            k["chain_cfg_L"], k["chain_cfg_U"] = (v >> 12) & 7, (v >> 15) & 7
        sweep = ("windowed", "ring", "wavefront", "cluster")
        d["kernels_h"] = [{f: (sweep if b < 2 else names)[(v >> (2 * b)) & 3] for b, f in enumerate(
            ("single_fwd", "single_bwd", "batched_fwd", "batched_bwd"))} for v in list(self.tune_h)[:nh]]
        for v, k in zip(list(self.tune_h)[:nh], d["kernels_h"]):
            k["chain_cfg_fwd"], k["chain_cfg_bwd"] = (v >> 8) & 7, (v >> 11) & 7
        return d


class pmg_stats_t(C.Structure):
    _fields_ = [("ms", C.c_double * PMG_NKERN), ("launches", C.c_longlong * PMG_NKERN),
                ("bytes", C.c_double * PMG_NKERN), ("total_launches", C.c_longlong),
                ("graph_launches", C.c_longlong)]

    def as_dict(self) -> dict:
        return {"total_launches": self.total_launches, "graph_launches": self.graph_launches,
                "per_class": {KERNEL_CLASSES[k]: {"ms": self.ms[k], "launches": self.launches[k],
                                                   "bytes": self.bytes[k]} for k in range(PMG_NKERN)}}


_lib = None


def lib():
    """Loads libpmg.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        if not _build.up_to_date():
            _build.build()
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"libpmg.so missing at {_LIB_PATH}: the CUDA path is required")
        L = C.CDLL(_LIB_PATH)
        vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
        L.pmg_default_options.argtypes = [C.POINTER(pmg_options)]
        L.pmg_setup.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(pmg_options), C.POINTER(vp)]
        L.pmg_info.argtypes = [vp, C.POINTER(pmg_info_t)]
        L.pmg_upload.argtypes = [vp, vp, C.c_size_t, vp]
        L.pmg_rhs.argtypes = [vp, dp]
        L.pmg_workspace_bytes.argtypes = [vp, C.c_int, C.POINTER(C.c_size_t)]
        L.pmg_workspace_create.argtypes = [vp, C.c_int, vp, C.c_size_t, vp, C.POINTER(vp)]
        L.pmg_solve.argtypes = [vp, vp, vp, vp, C.c_double, C.c_int, vp, ip, dp, C.c_int, vp]
        L.pmg_solve_bicgstab.argtypes = [vp, vp, vp, vp, C.c_double, C.c_int, vp, ip, dp, C.c_int, vp]
        L.pmg_solve_host.argtypes = [vp, vp, dp, dp, C.c_double, C.c_int, dp, ip, dp, C.c_int, vp]
        L.pmg_solve_batched.argtypes = [vp, vp, C.c_int, vp, vp, C.c_double, C.c_int, C.c_int, vp, ip, dp, vp]
        L.pmg_slots_load.argtypes = [vp, vp, C.c_int, C.c_int, vp, vp, vp]
        L.pmg_slots_cycle.argtypes = [vp, vp, C.c_int, C.c_double, vp]
        L.pmg_slots_wait.argtypes = [vp, vp, C.c_int, ip, dp, ip, ip]
        L.pmg_slots_read.argtypes = [vp, vp, C.c_int, C.c_int, vp, vp]
        L.pmg_slots_release.argtypes = [vp, vp, C.c_int, C.c_int, vp]
        L.pmg_autotune.argtypes = [vp, vp, vp]
        L.pmg_set_kernels.argtypes = [vp, ip, ip]
        L.pmg_apply.argtypes = [vp, vp, C.c_int, C.c_int, vp, vp, vp, vp]
        L.pmg_export_csr.argtypes = [vp, C.c_int, C.c_int, ip, ip, C.POINTER(C.c_longlong), ip, ip, dp]
        L.pmg_export_lumped.argtypes = [vp, C.c_int, dp]
        L.pmg_l2_error.argtypes = [vp, dp, dp]
        L.pmg_ws_profile.argtypes = [vp, C.c_int]
        L.pmg_ws_stats.argtypes = [vp, C.POINTER(pmg_stats_t), C.c_int]
        L.pmg_lsolve_noalloc.argtypes = [C.c_int, vp, vp, vp, vp, vp, vp]
        L.pmg_ws_destroy.argtypes = [vp]
        L.pmg_destroy.argtypes = [vp]
        L.pmg_last_error.restype = C.c_char_p
        for name in EXPORTS:
            if name != "pmg_last_error":
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


class PmgError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().pmg_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")


def _check(st: int, where: str, allow=()):
    if st != PMG_OK and st not in allow:
        raise PmgError(st, where)
    return st


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t) -> C.c_void_p:
    if t is None:
        return C.c_void_p(0)
    import torch
    assert isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()
    return C.c_void_p(t.data_ptr())


# ---------------------------------------------------------------------------
# C entry points, same names as the C-ABI
# ---------------------------------------------------------------------------
def pmg_default_options() -> pmg_options:
    o = pmg_options()
    _check(lib().pmg_default_options(C.byref(o)), "pmg_default_options")
    return o


def pmg_setup(domain: int, p: int, log2_inv_h: int, opt: pmg_options | None = None) -> C.c_void_p:
    h = C.c_void_p()
    _check(lib().pmg_setup(domain, p, log2_inv_h, C.byref(opt) if opt is not None else None, C.byref(h)),
           "pmg_setup")
    return h


def pmg_info(h) -> pmg_info_t:
    info = pmg_info_t()
    _check(lib().pmg_info(h, C.byref(info)), "pmg_info")
    return info


def pmg_upload(h, arena, stream=None):
    _check(lib().pmg_upload(h, _ptr(arena), arena.numel() * arena.element_size(), _stream(stream)), "pmg_upload")


def pmg_rhs(h, n: int) -> np.ndarray:
    f = np.zeros(n)
    _check(lib().pmg_rhs(h, _dp(f)), "pmg_rhs")
    return f


def pmg_workspace_bytes(h, max_rhs: int = 1) -> int:
    b = C.c_size_t()
    _check(lib().pmg_workspace_bytes(h, max_rhs, C.byref(b)), "pmg_workspace_bytes")
    return b.value


def pmg_workspace_create(h, max_rhs, mem, stream=None) -> C.c_void_p:
    ws = C.c_void_p()
    _check(lib().pmg_workspace_create(h, max_rhs, _ptr(mem), mem.numel() * mem.element_size(), _stream(stream),
                                      C.byref(ws)), "pmg_workspace_create")
    return ws


def pmg_solve(h, ws, f, u0, rel_tol, max_iter, u, hist_cap=256, stream=None, allow=()):
    iters = C.c_int()
    hist = np.zeros(hist_cap)
    st = lib().pmg_solve(h, ws, _ptr(f), _ptr(u0), rel_tol, max_iter, _ptr(u), C.byref(iters), _dp(hist),
                         hist_cap, _stream(stream))
    _check(st, "pmg_solve", allow)
    return iters.value, hist[: min(iters.value, hist_cap)].copy(), st


def pmg_solve_bicgstab(h, ws, f, u0, rel_tol, max_iter, u, hist_cap=256, stream=None, allow=()):
    iters = C.c_int()
    hist = np.zeros(hist_cap)
    st = lib().pmg_solve_bicgstab(h, ws, _ptr(f), _ptr(u0), rel_tol, max_iter, _ptr(u), C.byref(iters), _dp(hist),
                                  hist_cap, _stream(stream))
    _check(st, "pmg_solve_bicgstab", allow)
    return iters.value, hist[: min(iters.value, hist_cap)].copy(), st


def pmg_solve_host(h, ws, f: np.ndarray, u0: np.ndarray, rel_tol, max_iter, u: np.ndarray, hist_cap=256,
                   stream=None, allow=()):
    iters = C.c_int()
    hist = np.zeros(hist_cap)
    st = lib().pmg_solve_host(h, ws, _dp(f), _dp(u0), rel_tol, max_iter, _dp(u), C.byref(iters), _dp(hist),
                              hist_cap, _stream(stream))
    _check(st, "pmg_solve_host", allow)
    return iters.value, hist[: min(iters.value, hist_cap)].copy(), st


def pmg_solve_batched(h, ws, nrhs, F, U0, rel_tol, max_iter, precision, U, stream=None, allow=()):
    """F, U0, U: device tensors of nrhs x n doubles (right-hand side k in row k).
    Returns (iters per right-hand side, history [cycles x nrhs], status)."""
    iters = np.zeros(nrhs, np.int32)
    hist = np.zeros((max_iter, nrhs))
    st = lib().pmg_solve_batched(h, ws, nrhs, _ptr(F), _ptr(U0), rel_tol, max_iter, precision, _ptr(U),
                                 _ip(iters), _dp(hist), _stream(stream))
    _check(st, "pmg_solve_batched", allow)
    return iters, hist[: int(iters.max(initial=0))].copy(), st


PMG_SLOT_FREE, PMG_SLOT_ACTIVE, PMG_SLOT_CONVERGED, PMG_SLOT_DIVERGED = 0, 1, 2, 3


def pmg_slots_load(h, ws, slot0, F, U0, stream=None):
    """F, U0: device tensors (n, N) loaded into slots slot0 .. slot0+n-1."""
    _check(lib().pmg_slots_load(h, ws, slot0, F.shape[0], _ptr(F), _ptr(U0), _stream(stream)), "pmg_slots_load")


def pmg_slots_cycle(h, ws, precision, rel_tol=1e-8, stream=None):
    _check(lib().pmg_slots_cycle(h, ws, precision, rel_tol, _stream(stream)), "pmg_slots_cycle")


def pmg_slots_wait(h, ws, max_rhs, blocking=True):
    """Returns None while the last slot operation runs, else (relres, state, iters) per slot."""
    ready = C.c_int()
    rel = np.zeros(max_rhs)
    state = np.zeros(max_rhs, np.int32)
    iters = np.zeros(max_rhs, np.int32)
    _check(lib().pmg_slots_wait(h, ws, int(bool(blocking)), C.byref(ready), _dp(rel), _ip(state), _ip(iters)),
           "pmg_slots_wait")
    return (rel, state, iters) if ready.value else None


def pmg_slots_read(h, ws, slot0, U, stream=None):
    _check(lib().pmg_slots_read(h, ws, slot0, U.shape[0], _ptr(U), _stream(stream)), "pmg_slots_read")


def pmg_slots_release(h, ws, slot0, n, stream=None):
    _check(lib().pmg_slots_release(h, ws, slot0, n, _stream(stream)), "pmg_slots_release")


def pmg_autotune(h, ws, stream=None):
    _check(lib().pmg_autotune(h, ws, _stream(stream)), "pmg_autotune")


def pmg_set_kernels(h, tune_p, tune_h):
    tp = np.ascontiguousarray(tune_p, dtype=np.int32)
    th = np.ascontiguousarray(tune_h, dtype=np.int32)
    _check(lib().pmg_set_kernels(h, _ip(tp), _ip(th)), "pmg_set_kernels")


def pmg_apply(h, ws, op, level, x, b, y, stream=None):
    _check(lib().pmg_apply(h, ws, op, level, _ptr(x), _ptr(b), _ptr(y), _stream(stream)), "pmg_apply")


def pmg_export_csr(h, which: int, level: int):
    nr, nc, nnz = C.c_int(), C.c_int(), C.c_longlong()
    L = lib()
    _check(L.pmg_export_csr(h, which, level, C.byref(nr), C.byref(nc), C.byref(nnz), None, None, None),
           "pmg_export_csr")
    rp = np.zeros(nr.value + 1, np.int32)
    ci = np.zeros(nnz.value, np.int32)
    v = np.zeros(nnz.value)
    _check(L.pmg_export_csr(h, which, level, C.byref(nr), C.byref(nc), C.byref(nnz), _ip(rp), _ip(ci), _dp(v)),
           "pmg_export_csr")
    return nr.value, nc.value, rp, ci, v


def pmg_export_lumped(h, level: int, n: int) -> np.ndarray:
    out = np.zeros(n)
    _check(lib().pmg_export_lumped(h, level, _dp(out)), "pmg_export_lumped")
    return out


def pmg_l2_error(h, u: np.ndarray) -> float:
    e = C.c_double()
    _check(lib().pmg_l2_error(h, _dp(np.ascontiguousarray(u, dtype=np.float64)), C.byref(e)), "pmg_l2_error")
    return e.value


def pmg_ws_profile(ws, enable: bool):
    _check(lib().pmg_ws_profile(ws, int(bool(enable))), "pmg_ws_profile")


def pmg_ws_stats(ws, reset: bool = False) -> pmg_stats_t:
    st = pmg_stats_t()
    _check(lib().pmg_ws_stats(ws, C.byref(st), int(bool(reset))), "pmg_ws_stats")
    return st


def pmg_lsolve_noalloc(n: int, rp, ci, v, b, y, stream=None):
    """y = L^{-1} b with scratch in the library's fixed device array (no allocation)."""
    _check(lib().pmg_lsolve_noalloc(n, _ptr(rp), _ptr(ci), _ptr(v), _ptr(b), _ptr(y), _stream(stream)),
           "pmg_lsolve_noalloc")


def pmg_ws_destroy(ws):
    lib().pmg_ws_destroy(ws)


def pmg_destroy(h):
    lib().pmg_destroy(h)


def pmg_last_error() -> str:
    return lib().pmg_last_error().decode(errors="replace")


# ---------------------------------------------------------------------------
# Convenience owner: hierarchy + torch-allocated arena + one workspace
# ---------------------------------------------------------------------------
class Solver:
    """Owns a hierarchy, its device arena and one workspace (torch memory)."""

    def __init__(self, domain: int, p: int, log2_inv_h: int, projection: int = PMG_PROJ_INDIRECT,
                 exact: int = PMG_U_SINPROD, drop_tol: float = 1e-12, fill_factor: float = 1.0,
                 nu_pre: int = 1, nu_post: int = 1, coarse_cycles: int = 2, device: str = "cuda",
                 upload: bool = True, max_rhs: int = 1, handle=None, transfer_mass: int = 0):
        if handle is not None:
            self.h = handle            # adopt a hierarchy set up elsewhere (pmg_setup)
        else:
            opt = pmg_default_options()
            opt.projection, opt.exact, opt.drop_tol, opt.fill_factor = projection, exact, drop_tol, fill_factor
            opt.nu_pre, opt.nu_post, opt.coarse_cycles = nu_pre, nu_post, coarse_cycles
            opt.transfer_mass = transfer_mass
            self.h = pmg_setup(domain, p, log2_inv_h, opt)
        self.info = pmg_info(self.h).as_dict()
        self.N = self.info["n"][0]
        self.arena = self.mem = self.ws = None
        self.max_rhs = max_rhs
        if upload:
            self.upload(device)

    def upload(self, device="cuda"):
        import torch
        nbytes = max(self.info["device_bytes"], 256)
        self.arena = torch.empty((nbytes + 255) // 256 * 32, dtype=torch.float64, device=device)
        pmg_upload(self.h, self.arena)
        wb = pmg_workspace_bytes(self.h, self.max_rhs)
        self.mem = torch.empty((wb + 255) // 256 * 32, dtype=torch.float64, device=device)
        self.ws = pmg_workspace_create(self.h, self.max_rhs, self.mem)

    def rhs(self) -> np.ndarray:
        return pmg_rhs(self.h, self.N)

    def solve(self, f, u0, rel_tol=1e-8, max_iter=100, u=None, allow=()):
        import torch
        if u is None:
            u = torch.empty_like(u0)
        it, hist, st = pmg_solve(self.h, self.ws, f, u0, rel_tol, max_iter, u, allow=allow)
        return u, it, hist, st

    def solve_bicgstab(self, f, u0, rel_tol=1e-8, max_iter=100, u=None, allow=()):
        """BiCGSTAB preconditioned by one V-cycle per application (Sec. 5, Table 5)."""
        import torch
        if u is None:
            u = torch.empty_like(u0)
        it, hist, st = pmg_solve_bicgstab(self.h, self.ws, f, u0, rel_tol, max_iter, u, allow=allow)
        return u, it, hist, st

    def autotune(self):
        """Times the kernel variants of every solve on this device and keeps the fastest."""
        pmg_autotune(self.h, self.ws)
        self.info = pmg_info(self.h).as_dict()
        return self.info["kernels_p"], self.info["kernels_h"]

    def set_kernels(self, single=1, batched=1, sweep_single=1, sweep_batched=1, chain_cfg=7):
        """One variant for every level: single-vector solves 0 (windowed), 1
        (ring) or 3 (chain and producers on clusters of two CTAs per line, chain
        configuration chain_cfg 0..7); single-vector sweeps also 2 (wavefront,
        2D levels); batched solves 1 (ring) or 2 (lines per CTA)."""
        tp = (single | (single << 2) | (batched << 4) | (batched << 6) | (batched << 8) | (batched << 10) |
              (chain_cfg << 12) | (chain_cfg << 15))
        th = (sweep_single | (sweep_single << 2) | (sweep_batched << 4) | (sweep_batched << 6) |
              (chain_cfg << 8) | (chain_cfg << 11))
        pmg_set_kernels(self.h, [tp] * self.info["nlevels"], [th] * self.info["nhlevels"])
        self.info = pmg_info(self.h).as_dict()

    def solve_batched(self, F, U0, rel_tol=1e-8, max_iter=100, precision=PMG_PREC_FP64, U=None, allow=()):
        """F, U0: (nrhs, n) float64 device tensors.  Returns (U, iters, hist, status)."""
        import torch
        if U is None:
            U = torch.empty_like(U0)
        it, hist, st = pmg_solve_batched(self.h, self.ws, F.shape[0], F, U0, rel_tol, max_iter, precision, U,
                                         allow=allow)
        return U, it, hist, st

    def apply(self, op, level, x, b, y):
        pmg_apply(self.h, self.ws, op, level, x, b, y)
        return y

    def __del__(self):
        try:
            if self.ws is not None:
                pmg_ws_destroy(self.ws)
            if getattr(self, "h", None):
                pmg_destroy(self.h)
        except Exception:
            pass
