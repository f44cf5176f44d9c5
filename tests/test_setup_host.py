"""Host logic of the library (no GPU work): the C-ABI library loads and exports
every declared symbol, and its host-side setup (assembly, ILUT, transfers, P1
levels, load vector) agrees with the independent oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pmg():
    from paper_1901_01685_gb300 import pmg as P
    P.lib()
    return P


def test_library_exports_every_declared_symbol(pmg):
    header = open(os.path.join(ROOT, "include", "pmg.h")).read()
    declared = set(re.findall(r"^\s*(?:pmg_status|const char\*)\s+(pmg_\w+)\s*\(", header, re.M))
    assert declared, "no declarations found"
    lib = ctypes.CDLL(pmg._LIB_PATH)
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert declared == set(pmg.EXPORTS)


def test_default_options_match_paper(pmg):
    o = pmg.pmg_default_options()
    assert o.drop_tol == 1e-12 and o.fill_factor == 1.0          # Sec. 3 "Smoother"
    assert o.nu_pre == 1 and o.nu_post == 1                      # Sec. 5
    assert o.coarse_cycles == 2                                   # Sec. 3
    assert o.transfer_mass == pmg.PMG_MASS_LUMPED                 # Sec. 3: lumped mass in the transfers


def test_setup_rejects_unknown_transfer_mass(pmg):
    o = pmg.pmg_default_options()
    o.transfer_mass = 2
    with pytest.raises(pmg.PmgError) as e:
        pmg.pmg_setup(0, 3, 5, o)
    assert e.value.status == pmg.PMG_ERR_ARG


@pytest.mark.parametrize("bad", [(0, 1, 5), (0, 9, 5), (0, 3, 2), (2, 2, 7), (5, 3, 5)])
def test_setup_rejects_bad_arguments(pmg, bad):
    with pytest.raises(pmg.PmgError) as e:
        pmg.pmg_setup(*bad)
    assert e.value.status == pmg.PMG_ERR_ARG


def _same_csr(lib_csr, ocsr, tol):
    nr, nc, rp, ci, v = lib_csr
    assert (nr, nc) == ocsr.shape
    assert np.array_equal(rp, ocsr.rp) and np.array_equal(ci, ocsr.ci), "sparsity pattern differs"
    scale = max(np.abs(ocsr.v).max(), 1e-300)
    assert np.abs(v - ocsr.v).max() <= tol * scale


CASES = [
    (0, 3, 5, 0, 0),   # quarter annulus, h = 2^-5, p = 3, indirect (the small configuration)
    (0, 3, 5, 1, 0),   # direct projection
    (1, 2, 5, 0, 0),   # unit square
    (2, 2, 3, 0, 0),   # unit cube
    (0, 4, 6, 0, 1),   # annulus, paper's benchmark-1 solution
    (3, 3, 5, 0, 0),   # benchmark 2: convection-diffusion-reaction, unit square
    (3, 2, 4, 1, 0),
]


@pytest.mark.parametrize("dom,p,k,proj,ex", CASES)
def test_setup_matches_oracle(pmg, oracle_mod, dom, p, k, proj, ex):
    opt = pmg.pmg_default_options()
    opt.projection, opt.exact = proj, ex
    h = pmg.pmg_setup(dom, p, k, opt)
    try:
        oh = oracle_mod.Hierarchy(dom, p, k, projection=proj, exact=ex)
        info = pmg.pmg_info(h).as_dict()
        assert info["nlevels"] == oh.nlev and info["n"] == oh.N and info["nhlevels"] == oh.nh
        for l in range(oh.nlev):
            _same_csr(pmg.pmg_export_csr(h, 0, l), oh.csr("A", l), 1e-13)
            _same_csr(pmg.pmg_export_csr(h, 1, l), oh.csr("L", l), 1e-12)
            _same_csr(pmg.pmg_export_csr(h, 2, l), oh.csr("U", l), 1e-12)
            _same_csr(pmg.pmg_export_csr(h, 3, l), oh.csr("P", l), 1e-13)
            ml = pmg.pmg_export_lumped(h, l, oh.N[l])
            assert np.abs(ml - oh.lumped_mass(l)).max() <= 1e-13 * ml.max()
        ml1 = pmg.pmg_export_lumped(h, oh.nlev, oh.NH[0])
        assert np.abs(ml1 - oh.lumped_mass(oh.nlev)).max() <= 1e-13 * ml1.max()
        for j in range(oh.nh):
            _same_csr(pmg.pmg_export_csr(h, 4, j), oh.csr("A1", j), 1e-13)
        f = pmg.pmg_rhs(h, oh.N[0])
        fo = oh.rhs()
        assert np.abs(f - fo).max() <= 1e-13 * np.abs(fo).max()
        # solve depths are reported and bounded by the number of rows
        assert all(0 < d <= n for d, n in zip(info["depth_L"], info["n"]))
    finally:
        pmg.pmg_destroy(h)


def test_l2_error_matches_oracle(pmg, oracle_mod):
    h = pmg.pmg_setup(0, 3, 4)
    try:
        oh = oracle_mod.Hierarchy(0, 3, 4)
        u = np.random.default_rng(0).standard_normal(oh.N[0]) * 1e-3
        assert abs(pmg.pmg_l2_error(h, u) - oh.l2_error(u)) <= 1e-12 * oh.l2_error(u)
    finally:
        pmg.pmg_destroy(h)


def test_calls_reject_null_and_out_of_order_arguments(pmg):
    import ctypes as C
    L = pmg.lib()
    h = pmg.pmg_setup(0, 2, 3)
    try:
        # solve without a workspace / before upload
        st = L.pmg_solve(h, None, None, None, 1e-8, 10, None, None, None, 0, None)
        assert st == pmg.PMG_ERR_ARG
        # upload into a buffer that is too small is refused before any device work
        st = L.pmg_upload(h, C.c_void_p(256), 16, None)
        assert st == pmg.PMG_ERR_ARG
        # misaligned arena
        info = pmg.pmg_info(h)
        st = L.pmg_upload(h, C.c_void_p(257), info.device_bytes, None)
        assert st == pmg.PMG_ERR_ARG
        st = L.pmg_workspace_create(h, 0, None, 0, None, None)
        assert st == pmg.PMG_ERR_ARG
        assert pmg.pmg_last_error() != ""
    finally:
        pmg.pmg_destroy(h)


def test_kernel_choice_words_decode(pmg):
    """pmg_info_t.tune_p / tune_h: 2-bit variant fields, then 3-bit chain
    configurations (bits 12-14 / 15-17 of tune_p, 8-10 / 11-13 of tune_h).
    Defaults after setup: clustered single-vector solves with four lines a
    cluster (configuration 7), wavefront single-vector sweeps, ring kernels
    for the batched forms."""
    S = pmg.Solver(0, 3, 5, upload=False)
    for k in S.info["kernels_p"]:
        assert (k["single_L"], k["single_U"]) == ("cluster", "cluster")
        assert (k["chain_cfg_L"], k["chain_cfg_U"]) == (7, 7)
        assert k["batched64_L"] == k["batched32_U"] == "ring"
    for k in S.info["kernels_h"]:
        assert (k["single_fwd"], k["single_bwd"]) == ("wavefront", "wavefront")
        assert (k["chain_cfg_fwd"], k["chain_cfg_bwd"]) == (7, 7)
    info = pmg.pmg_info_t()
    info.nlevels, info.nhlevels = 1, 1
    info.tune_p[0] = 3 | (1 << 2) | (1 << 4) | (2 << 6) | (1 << 8) | (2 << 10) | (5 << 12) | (6 << 15)
    info.tune_h[0] = 2 | (3 << 2) | (1 << 4) | (2 << 6) | (4 << 8) | (3 << 11)
    d = info.as_dict()
    kp, kh = d["kernels_p"][0], d["kernels_h"][0]
    assert (kp["single_L"], kp["single_U"], kp["batched64_L"], kp["batched64_U"]) == ("cluster", "ring", "ring", "lines")
    assert (kp["batched32_L"], kp["batched32_U"], kp["chain_cfg_L"], kp["chain_cfg_U"]) == ("ring", "lines", 5, 6)
    assert (kh["single_fwd"], kh["single_bwd"], kh["batched_fwd"], kh["batched_bwd"]) == ("wavefront", "cluster", "ring", "lines")
    assert (kh["chain_cfg_fwd"], kh["chain_cfg_bwd"]) == (4, 3)
