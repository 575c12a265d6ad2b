"""The C ABI library loads without a GPU, exports every symbol include/lrtddft.h declares,
validates arguments on the host, and its host-side geometry (bases, G-sets, K) agrees with
the oracle's independent construction."""
import ctypes as C
import math
import os
import re

import numpy as np
import pytest

from oracle import crystal, response, xc
from paper_2510_01875_gb300 import binding, build
from paper_2510_01875_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "lrtddft.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lrtddft_\w+)\s*\(", txt)))


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 19
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(binding.SIGNATURES)


def test_status_strings(lib):
    for s in range(8):
        assert lib.lrtddft_status_string(s)
    assert lib.lrtddft_status_string(99) == b"unknown status"


def _host_ctx(wl):
    lib = binding.load()
    cell = binding.lrt_cell()
    cell.lattice[:] = list(np.asarray(wl.lattice).reshape(-1))
    pos = np.ascontiguousarray(wl.positions)
    cell.natoms = wl.natoms
    cell.positions = pos.ctypes.data_as(C.POINTER(C.c_double))
    cell.Z, cell.r_c, cell.ecut = wl.Z, wl.r_c, wl.ecut
    cell.potential = binding.POT[wl.potential]
    cell.basis = binding.BASIS[wl.basis]
    km = binding.lrt_kmesh()
    km.n[:] = list(wl.kmesh)
    km.scheme = binding.KSCHEME[wl.kscheme]
    kern = binding.lrt_kernel(binding.KERNEL[wl.kernel], *wl.fxc_params)
    opt = binding.lrt_options(0, 0, 1)   # LRT_FLAG_HOST_ONLY
    q = np.ascontiguousarray(wl.q)
    nG = np.ascontiguousarray(wl.nG, dtype=np.int32)
    om = np.ascontiguousarray(wl.omega)
    h = C.c_void_p()
    st = lib.lrtddft_create(C.byref(cell), C.byref(km), wl.nbands, wl.T, None, wl.nq,
                            q.ctypes.data_as(C.POINTER(C.c_double)),
                            nG.ctypes.data_as(C.POINTER(C.c_int)), wl.nw,
                            om.ctypes.data_as(C.POINTER(C.c_double)), wl.eta, C.byref(kern),
                            C.byref(opt), C.byref(h))
    return st, h


def _create_status(wl):
    st, h = _host_ctx(wl)
    if st == 0:
        binding.load().lrtddft_destroy(h)
    return st


def test_argument_validation(lib):
    wl = W.tiny()
    assert _create_status(wl) == 0
    bad = [wl.replace(T=0.0), wl.replace(eta=-1.0), wl.replace(nbands=0),
           wl.replace(omega=wl.omega[::-1].copy()), wl.replace(nbands=10000),
           wl.replace(kmesh=(0, 2, 2)), wl.replace(q=np.array([[np.nan, 0, 0], [0.1, 0, 0]])),
           wl.replace(nG=np.array([0, 5])),
           # q equal to a reciprocal-lattice vector
           wl.replace(q=np.stack([crystal.reciprocal(wl.lattice)[0], wl.q[1]]))]
    for b in bad:
        assert _create_status(b) == binding.LRT_EINVAL


def test_host_only_context_refuses_compute(lib):
    st, h = _host_ctx(W.tiny())
    assert st == 0
    assert lib.lrtddft_chi0_assemble(h, 0, 1, None) == binding.LRT_ESTATE
    assert lib.lrtddft_dyson_solve(h, 0, 1, None) == binding.LRT_ESTATE
    S = np.zeros(100)
    assert lib.lrtddft_dsf(h, S.ctypes.data_as(C.POINTER(C.c_double))) == binding.LRT_ESTATE
    lib.lrtddft_destroy(h)


def test_params_and_adjoint_validation(lib):
    st, h = _host_ctx(W.tiny(kernel="fxc_model"))
    assert st == 0
    D = C.POINTER(C.c_double)
    k = binding.lrt_kernel(2, 1.0, 0.1, 0.05)
    for T, eta in ((0.0, 0.01), (-1.0, 0.01), (0.1, 0.0), (float("nan"), 0.01), (0.1, float("inf"))):
        assert lib.lrtddft_set_params(h, T, eta, C.byref(k)) == binding.LRT_EINVAL
    assert lib.lrtddft_set_params(h, 0.1, 0.01, C.byref(binding.lrt_kernel(7, 0, 0, 0))) == binding.LRT_EINVAL
    assert lib.lrtddft_set_params(h, 0.1, 0.01, C.byref(binding.lrt_kernel(2, float("nan"), 0, 0))) \
        == binding.LRT_EINVAL
    assert lib.lrtddft_set_params(h, 0.1, 0.01, None) == binding.LRT_EINVAL
    # valid parameters on a context without a GPU: refused by state, not by the arguments
    assert lib.lrtddft_set_params(h, 0.1, 0.01, C.byref(k)) == binding.LRT_ESTATE
    tau = np.linspace(0.0, 1.0, 4)
    g = np.zeros(5)
    gF = np.zeros((2, 4))
    assert lib.lrtddft_itcf_vjp(h, 4, tau.ctypes.data_as(D), None, g.ctypes.data_as(D)) == binding.LRT_EINVAL
    big = np.array([0.0, 1e9])
    assert lib.lrtddft_itcf_vjp(h, 2, big.ctypes.data_as(D), gF.ctypes.data_as(D),
                                g.ctypes.data_as(D)) == binding.LRT_EINVAL
    assert lib.lrtddft_jacobian(h, 0, None, None, None) == binding.LRT_EINVAL
    assert lib.lrtddft_dsf_vjp(h, gF.ctypes.data_as(D), g.ctypes.data_as(D)) == binding.LRT_ESTATE
    lib.lrtddft_destroy(h)


@pytest.mark.parametrize("wl", [W.tiny(), W.tiny(kscheme="commensurate", nq=1), W.al1_fcc_k8_b24(),
                                W.tiny(basis="fixed", seed=3), W.tiny(kernel="fxc_model", seed=4)])
def test_host_geometry_matches_oracle(lib, wl):
    if wl.kscheme == "commensurate" and wl.name.startswith("tiny"):
        wl = wl.replace(q=np.array([0.5 * crystal.reciprocal(wl.lattice)[1]]))
    st, h = _host_ctx(wl)
    assert st == 0
    sz = (C.c_int64 * 8)()
    lib.lrtddft_query(h, sz)
    nk, npw = sz[2], sz[5]
    for iq in range(wl.nq):
        nG = int(wl.nG[iq])
        m = np.zeros((nG, 3), dtype=np.int32)
        K = np.zeros(nG)
        assert lib.lrtddft_get_gset(h, iq, m.ctypes.data_as(C.POINTER(C.c_int32)),
                                    K.ctypes.data_as(C.POINTER(C.c_double))) == 0
        gs = crystal.response_gset(wl.lattice, wl.q[iq], nG)
        assert np.array_equal(m, gs)
        assert np.allclose(K, response.kernel_diag(wl, wl.q[iq], gs), rtol=1e-13, atol=0)
        mil = np.zeros((2, nk, npw, 3), dtype=np.int32)
        npk = np.zeros((2, nk), dtype=np.int32)
        assert lib.lrtddft_get_basis(h, iq, mil.ctypes.data_as(C.POINTER(C.c_int32)),
                                     npk.ctypes.data_as(C.POINTER(C.c_int32))) == 0
        kp, kqp = crystal.pair_meshes(wl.lattice, wl.kmesh, wl.q[iq], wl.kscheme)
        for s, pts in enumerate((kp, kqp)):
            for ik in range(0, nk, max(1, nk // 7)):
                ref = response.basis_for(wl, pts[ik])
                assert npk[s, ik] == len(ref)
                got = mil[s, ik, :npk[s, ik]]
                assert np.array_equal(got, ref)
                assert np.all(mil[s, ik, npk[s, ik]:] == np.iinfo(np.int32).min)
    lib.lrtddft_destroy(h)


def test_tuning_flags_and_hooks_on_host(lib):
    st, h = _host_ctx(W.tiny())
    assert st == 0
    # LRT_TUNE_AUTO | SINGLE_Q | PAIR_SIMT | FINE_ACCUM | HALF_TILES | ZERO_SIMT are the known flags
    for flags in (0, 1, 2, 4, 7, 8, 15, 16, 31, 32, 63):
        assert lib.lrtddft_set_tuning(h, flags, -1, 0) == 0, flags
    for flags in (64, 128, -1):
        assert lib.lrtddft_set_tuning(h, flags, -1, 0) == binding.LRT_EINVAL, flags
    for v, u in ((2, 0), (-2, 0), (0, 100), (0, -64)):
        assert lib.lrtddft_set_tuning(h, 0, v, u) == binding.LRT_EINVAL, (v, u)
    assert lib.lrtddft_set_tuning(h, 0, 1, 128) == 0
    v, u = C.c_int(), C.c_int()
    assert lib.lrtddft_get_tuning(h, C.byref(v), C.byref(u)) == 0
    assert (v.value, u.value) == (-1, 0)   # no tensor-core launch has run
    r = C.c_int(-1)
    assert lib.lrtddft_get_tile_rows(h, C.byref(r)) == 0 and r.value == 0
    # the spectral chi0 engine: bin width >= 0, order 1 or 3
    for hh, order in ((-1.0, 3), (0.01, 2), (float("inf"), 3)):
        assert lib.lrtddft_set_spectral(h, hh, order) == binding.LRT_EINVAL, (hh, order)
    assert lib.lrtddft_set_spectral(h, 0.01, 3) == 0
    assert lib.lrtddft_set_spectral(h, 0.0, 0) == 0
    x0, nb = C.c_double(-1.0), C.c_longlong(-1)
    assert lib.lrtddft_get_spectral_grid(h, 0, C.byref(x0), C.byref(nb)) == 0
    assert (x0.value, nb.value) == (0.0, 0)
    assert lib.lrtddft_get_spectral_grid(h, 9, C.byref(x0), C.byref(nb)) == binding.LRT_EINVAL
    out = np.zeros(16)
    D = C.POINTER(C.c_double)
    assert lib.lrtddft_get_pair_densities(h, 0, out.ctypes.data_as(D)) == binding.LRT_ESTATE
    assert lib.lrtddft_get_pair_densities(h, 5, out.ctypes.data_as(D)) == binding.LRT_EINVAL
    assert lib.lrtddft_get_pair_densities(h, 0, None) == binding.LRT_EINVAL
    lib.lrtddft_destroy(h)
