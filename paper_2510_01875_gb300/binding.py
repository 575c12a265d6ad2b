"""Python binding of liblrtddft (C ABI in include/lrtddft.h): argument marshalling only.

Every step of the response path runs in the CUDA library; this module converts a
`workloads.Workload` into the C structs, allocates numpy output buffers and checks status
codes.  `load()` raises if the library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from .workloads import Workload

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblrtddft.so")

LRT_OK, LRT_EINVAL, LRT_ENOMEM, LRT_ECUDA, LRT_ESINGULAR, LRT_ETIMEOUT, LRT_ESTATE, LRT_EUNSUPPORTED = range(8)
POT = {"empty_core": 0, "zero": 1}
BASIS = {"sphere": 0, "fixed": 1}
KSCHEME = {"commensurate": 0, "tr_symmetric": 1}
KERNEL = {"rpa": 0, "rpa_alda": 1, "fxc_model": 2}
PREC = {"fp64": 0, "fp16x3": 1, "bf16x3": 2}
ITCF = {"fold": 0, "direct": 1}


class LrtError(RuntimeError):
    def __init__(self, fn, status, detail):
        super().__init__(f"{fn}: {status} ({detail})")
        self.status = status


class lrt_cell(C.Structure):
    _fields_ = [("lattice", C.c_double * 9), ("natoms", C.c_int), ("positions", C.POINTER(C.c_double)),
                ("Z", C.c_double), ("r_c", C.c_double), ("ecut", C.c_double), ("potential", C.c_int),
                ("basis", C.c_int)]


class lrt_kmesh(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("scheme", C.c_int)]


class lrt_kernel(C.Structure):
    _fields_ = [("kind", C.c_int), ("A", C.c_double), ("B", C.c_double), ("C", C.c_double)]


class lrt_options(C.Structure):
    _fields_ = [("precision", C.c_int), ("device", C.c_int), ("flags", C.c_int)]


class lrt_atten_params(C.Structure):
    _fields_ = [("d_min", C.c_int), ("d_max", C.c_int), ("w_min", C.c_double), ("w_max", C.c_double),
                ("n_w", C.c_int), ("lambda_f", C.c_double), ("lambda_c", C.c_double),
                ("n_targets", C.c_int), ("feat_lo", C.c_double), ("feat_hi", C.c_double),
                ("low_exclude", C.c_double), ("accept_mean", C.c_double), ("accept_rms", C.c_double),
                ("average", C.c_int), ("ntau", C.c_int), ("retain_floor", C.c_double)]


MAXDEG = 8


class lrt_atten_report(C.Structure):
    _fields_ = [("n_accepted", C.c_int), ("targets", C.c_int * 4), ("degree", C.c_int * MAXDEG),
                ("window", C.c_int * MAXDEG), ("score", C.c_double * MAXDEG),
                ("mean_ratio", C.c_double * MAXDEG), ("rms_ratio", C.c_double * MAXDEG),
                ("accepted", C.c_int * MAXDEG)]


# name -> (restype, argtypes); every symbol include/lrtddft.h declares
_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
SIGNATURES = {
    "lrtddft_create": (C.c_int, [C.POINTER(lrt_cell), C.POINTER(lrt_kmesh), C.c_int, C.c_double, _D, C.c_int,
                                 _D, C.POINTER(C.c_int), C.c_int, _D, C.c_double, C.POINTER(lrt_kernel),
                                 C.POINTER(lrt_options), C.POINTER(_P)]),
    "lrtddft_destroy": (C.c_int, [_P]),
    "lrtddft_status_string": (C.c_char_p, [C.c_int]),
    "lrtddft_last_error": (C.c_char_p, []),
    "lrtddft_query": (C.c_int, [_P, C.POINTER(C.c_int64)]),
    "lrtddft_chi0_assemble": (C.c_int, [_P, C.c_int, C.c_int, _P]),
    "lrtddft_dyson_solve": (C.c_int, [_P, C.c_int, C.c_int, _P]),
    "lrtddft_dsf": (C.c_int, [_P, _D]),
    "lrtddft_dsf_device": (C.c_int, [_P, _P, _P]),
    "lrtddft_itcf_laplace": (C.c_int, [_P, C.c_int, _D, C.c_int, _D, _D]),
    "lrtddft_itcf_laplace_device": (C.c_int, [_P, C.c_int, _P, C.c_int, _P, _P, _P]),
    "lrtddft_set_params": (C.c_int, [_P, C.c_double, C.c_double, C.POINTER(lrt_kernel)]),
    "lrtddft_set_tuning": (C.c_int, [_P, C.c_int, C.c_int, C.c_int]),
    "lrtddft_get_tuning": (C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "lrtddft_get_tile_rows": (C.c_int, [_P, C.POINTER(C.c_int)]),
    "lrtddft_set_spectral": (C.c_int, [_P, C.c_double, C.c_int]),
    "lrtddft_get_spectral_grid": (C.c_int, [_P, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
    "lrtddft_graph_capture": (C.c_int, [_P, C.c_int, _P, C.c_int, _P, _P, _P]),
    "lrtddft_graph_launch": (C.c_int, [_P, _P]),
    "lrtddft_jacobian": (C.c_int, [_P, C.c_int, _D, _D, _D]),
    "lrtddft_itcf_vjp": (C.c_int, [_P, C.c_int, _D, _D, _D]),
    "lrtddft_dsf_vjp": (C.c_int, [_P, _D, _D]),
    "lrtddft_attenuate": (C.c_int, [_P, C.POINTER(lrt_atten_params), _D, C.POINTER(lrt_atten_report)]),
    "lrtddft_attenuate_noalloc": (C.c_int, [_P, C.POINTER(lrt_atten_params), _D,
                                            C.POINTER(lrt_atten_report)]),
    "lrtddft_profile": (C.c_int, [_P, C.c_int]),
    "lrtddft_profile_read": (C.c_int, [_P, _D]),
    "lrtddft_set_orbitals": (C.c_int, [_P, C.c_int, _D, _D, _D]),
    "lrtddft_set_orbitals_async": (C.c_int, [_P, C.c_int, _D, _D, _D]),
    "lrtddft_get_orbitals": (C.c_int, [_P, C.c_int, _D]),
    "lrtddft_get_basis": (C.c_int, [_P, C.c_int, _I32, _I32]),
    "lrtddft_get_ground_state": (C.c_int, [_P, C.c_int, _D, _D, _D, _D]),
    "lrtddft_get_gset": (C.c_int, [_P, C.c_int, _I32, _D]),
    "lrtddft_get_chi0": (C.c_int, [_P, C.c_int, _D]),
    "lrtddft_get_pair_densities": (C.c_int, [_P, C.c_int, _D]),
    "lrtddft_get_chi_col0": (C.c_int, [_P, C.c_int, _D]),
    "lrtddft_get_frequencies": (C.c_int, [_P, _D, C.POINTER(C.c_int)]),
    "lrtddft_set_eta_list": (C.c_int, [_P, C.c_int, _D]),
    "lrtddft_get_eta_list": (C.c_int, [_P, C.POINTER(C.c_int), _D]),
    "lrtddft_eta_scan": (C.c_int, [_P, C.c_int, _D, C.c_double, _D, _D, C.POINTER(C.c_int)]),
    "lrtddft_dielectric": (C.c_int, [_P, _D, _D]),
    "lrtddft_measure_fp64": (C.c_int, [C.c_int, _D]),
    "lrtddft_row_plan": (C.c_int, [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int), _I32]),
    "lrtddft_kubo_greenwood": (C.c_int, [_P, C.c_int, _D, C.c_int, _D, C.c_double, _D, _D, _D, _D,
                                         C.POINTER(C.c_int)]),
    "lrtddft_kubo_greenwood_attenuate": (C.c_int, [_P, C.POINTER(lrt_atten_params), _D,
                                                   C.POINTER(lrt_atten_report), _D]),
}

_lib = None


def load():
    """Load liblrtddft.so; raises when it is missing (build it with __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: the CUDA library must be built first")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _check(fn: str, st: int):
    if st != LRT_OK:
        lib = load()
        raise LrtError(fn, lib.lrtddft_status_string(st).decode(), lib.lrtddft_last_error().decode())


def measure_fp64(device: int = 0) -> float:
    """Measured FP64 FMA rate of the device's CUDA cores, TFLOP/s."""
    lib = load()
    v = C.c_double()
    _check("lrtddft_measure_fp64", lib.lrtddft_measure_fp64(device, C.byref(v)))
    return v.value


def row_plan(nG: int):
    """Row plan of the split contraction for nG G vectors (host only):
    (super-tiles, list sub-blocks, most G blocks per super-tile, row pair of (G, G') [nG, nG])."""
    lib = load()
    n_st, n_list, mb = C.c_int(), C.c_int(), C.c_int()
    rp = np.zeros((nG, nG), dtype=np.int32)
    _check("lrtddft_row_plan", lib.lrtddft_row_plan(nG, C.byref(n_st), C.byref(n_list), C.byref(mb),
                                                    rp.ctypes.data_as(_I32)))
    return n_st.value, n_list.value, mb.value, rp


def atten_params(**kw) -> lrt_atten_params:
    """An lrt_atten_params with library defaults for every field not given."""
    p = lrt_atten_params()
    for f, _ in lrt_atten_params._fields_:
        setattr(p, f, 0)
    p.average = 1
    for k, v in kw.items():
        setattr(p, k, v)
    return p


class Context:
    """One lrt_ctx built from a Workload."""

    def __init__(self, wl: Workload, precision: str = "fp64", device: int = 0,
                 occupations: Optional[np.ndarray] = None):
        lib = load()
        self.wl = wl
        cell = lrt_cell()
        cell.lattice[:] = [float(x) for x in np.asarray(wl.lattice).reshape(-1)]
        self._pos = np.ascontiguousarray(wl.positions, dtype=np.float64)
        cell.natoms = wl.natoms
        cell.positions = _dp(self._pos)
        cell.Z, cell.r_c, cell.ecut = wl.Z, wl.r_c, wl.ecut
        cell.potential = POT[wl.potential]
        cell.basis = BASIS[wl.basis]
        km = lrt_kmesh()
        km.n[:] = list(wl.kmesh)
        km.scheme = KSCHEME[wl.kscheme]
        kern = lrt_kernel(KERNEL[wl.kernel], *[float(x) for x in wl.fxc_params])
        opt = lrt_options(PREC[precision], device, 0)
        q = np.ascontiguousarray(wl.q, dtype=np.float64)
        nG = np.ascontiguousarray(wl.nG, dtype=np.int32)
        om = np.ascontiguousarray(wl.omega, dtype=np.float64)
        occ = None if occupations is None else np.ascontiguousarray(occupations, dtype=np.float64)
        h = _P()
        st = lib.lrtddft_create(C.byref(cell), C.byref(km), wl.nbands, wl.T,
                                None if occ is None else _dp(occ), wl.nq, _dp(q),
                                nG.ctypes.data_as(C.POINTER(C.c_int)), wl.nw, _dp(om), wl.eta,
                                C.byref(kern), C.byref(opt), C.byref(h))
        _check("lrtddft_create", st)
        self.h = h
        sz = (C.c_int64 * 8)()
        _check("lrtddft_query", lib.lrtddft_query(h, sz))
        self.nq, self.nw, self.nk, self.nb, self.nGmax, self.npw, self.nwi, _ = list(sz)
        self.neta = 1
        self.lib = lib

    def _rows(self, *rest):
        """Shape of a per-(q, eta) output: (nq, *rest) for one eta, (nq, neta, *rest) for a list."""
        return (self.nq,) + rest if self.neta == 1 else (self.nq, self.neta) + rest

    def close(self):
        if getattr(self, "h", None):
            self.lib.lrtddft_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- response steps ---
    def chi0_assemble(self, q0=0, q1=None, stream: int = 0):
        _check("lrtddft_chi0_assemble", self.lib.lrtddft_chi0_assemble(
            self.h, q0, self.nq if q1 is None else q1, _P(stream)))

    def dyson_solve(self, q0=0, q1=None, stream: int = 0):
        _check("lrtddft_dyson_solve", self.lib.lrtddft_dyson_solve(
            self.h, q0, self.nq if q1 is None else q1, _P(stream)))

    def dsf(self) -> np.ndarray:
        S = np.zeros(self._rows(self.nw))
        _check("lrtddft_dsf", self.lib.lrtddft_dsf(self.h, _dp(S)))
        return S

    def dsf_device(self, S_ptr: int, stream: int = 0):
        _check("lrtddft_dsf_device", self.lib.lrtddft_dsf_device(self.h, _P(S_ptr), _P(stream)))

    def itcf(self, tau, mode: str = "fold"):
        tau = np.ascontiguousarray(tau, dtype=np.float64)
        F = np.zeros(self._rows(len(tau)))
        m = np.zeros(self._rows(5))
        _check("lrtddft_itcf_laplace", self.lib.lrtddft_itcf_laplace(
            self.h, len(tau), _dp(tau), ITCF[mode], _dp(F), _dp(m)))
        return F, m

    def itcf_device(self, ntau: int, tau_ptr: int, F_ptr: int, metrics_ptr: int, mode="fold", stream: int = 0):
        _check("lrtddft_itcf_laplace_device", self.lib.lrtddft_itcf_laplace_device(
            self.h, ntau, _P(tau_ptr), ITCF[mode], _P(F_ptr), _P(metrics_ptr), _P(stream)))

    def set_tuning(self, auto: bool = False, single_q: bool = False, variant: int = -1, unit_stages: int = 0,
                   pair_simt: bool = False, fine_accum: bool = False, half_tiles: bool = False,
                   zero_simt: bool = False):
        """lrtddft_set_tuning: auto times the contraction's row-unit shapes, variants and unit
        sizes on the first launch of each shape; single_q launches the contraction once per q;
        pair_simt computes the split path's pair densities on the FP32 SIMT kernel instead of
        the tensor cores; fine_accum halves the FP32 accumulation period (32 stages);
        half_tiles makes every row unit 256 rows; zero_simt computes the w = 0 column on the
        CUDA cores instead of the tensor cores; variant (-1, 0, 1) and unit_stages (0 or a
        multiple of 64) force a choice."""
        flags = ((1 if auto else 0) | (2 if single_q else 0) | (4 if pair_simt else 0)
                 | (8 if fine_accum else 0) | (16 if half_tiles else 0) | (32 if zero_simt else 0))
        _check("lrtddft_set_tuning", self.lib.lrtddft_set_tuning(self.h, flags, variant, unit_stages))

    def get_tuning(self):
        v, u = C.c_int(), C.c_int()
        _check("lrtddft_get_tuning", self.lib.lrtddft_get_tuning(self.h, C.byref(v), C.byref(u)))
        return v.value, u.value

    def set_spectral(self, h: float, order: int = 3):
        """lrtddft_set_spectral: chi0 through a spectral function on a grid of spacing h (Ha)
        with Lagrange interpolation of the given order (1 or 3); h = 0 restores the direct sum."""
        _check("lrtddft_set_spectral", self.lib.lrtddft_set_spectral(self.h, float(h), int(order)))

    def get_spectral_grid(self, iq: int):
        x0, nb = C.c_double(), C.c_longlong()
        _check("lrtddft_get_spectral_grid", self.lib.lrtddft_get_spectral_grid(
            self.h, iq, C.byref(x0), C.byref(nb)))
        return x0.value, nb.value

    def get_tile_rows(self) -> int:
        r = C.c_int()
        _check("lrtddft_get_tile_rows", self.lib.lrtddft_get_tile_rows(self.h, C.byref(r)))
        return r.value

    def graph_capture(self, ntau: int, tau_ptr: int, S_ptr: int, F_ptr: int, metrics_ptr: int, mode="fold"):
        _check("lrtddft_graph_capture", self.lib.lrtddft_graph_capture(
            self.h, ntau, _P(tau_ptr), ITCF[mode], _P(S_ptr), _P(F_ptr), _P(metrics_ptr)))

    def graph_launch(self, stream: int = 0):
        _check("lrtddft_graph_launch", self.lib.lrtddft_graph_launch(self.h, _P(stream)))

    def set_params(self, T: float, eta: float, kernel: Optional[str] = None, fxc_params=None):
        """New T, eta (Ha) and kernel without new eigensolves; chi0 and chi must be recomputed."""
        kern = lrt_kernel(KERNEL[kernel or self.wl.kernel],
                          *[float(x) for x in (fxc_params if fxc_params is not None else self.wl.fxc_params)])
        _check("lrtddft_set_params", self.lib.lrtddft_set_params(self.h, float(T), float(eta), C.byref(kern)))
        self.neta = 1
        self.wl = self.wl.replace(T=float(T), eta=float(eta), kernel=kernel or self.wl.kernel,
                                  fxc_params=tuple(float(x) for x in (fxc_params if fxc_params is not None
                                                                      else self.wl.fxc_params)))

    def jacobian(self, tau=None):
        """(dS [nq][nw][5], dF [nq][ntau][5] or None) with respect to (T, eta, A, B, C)."""
        dS = np.zeros((self.nq, self.nw, 5))
        if tau is None:
            _check("lrtddft_jacobian", self.lib.lrtddft_jacobian(self.h, 0, None, _dp(dS), None))
            return dS, None
        tau = np.ascontiguousarray(tau, dtype=np.float64)
        dF = np.zeros((self.nq, len(tau), 5))
        _check("lrtddft_jacobian", self.lib.lrtddft_jacobian(self.h, len(tau), _dp(tau), _dp(dS), _dp(dF)))
        return dS, dF

    def itcf_vjp(self, tau, dL_dF):
        tau = np.ascontiguousarray(tau, dtype=np.float64)
        g = np.ascontiguousarray(dL_dF, dtype=np.float64).reshape(self.nq, len(tau))
        out = np.zeros(5)
        _check("lrtddft_itcf_vjp", self.lib.lrtddft_itcf_vjp(self.h, len(tau), _dp(tau), _dp(g), _dp(out)))
        return out

    def dsf_vjp(self, dL_dS):
        g = np.ascontiguousarray(dL_dS, dtype=np.float64).reshape(self.nq, self.nw)
        out = np.zeros(5)
        _check("lrtddft_dsf_vjp", self.lib.lrtddft_dsf_vjp(self.h, _dp(g), _dp(out)))
        return out

    def attenuate(self, params: Optional[lrt_atten_params] = None):
        p = params if params is not None else atten_params()
        Sp = np.zeros(self._rows(self.nw))
        rep = (lrt_atten_report * (self.nq * self.neta))()
        _check("lrtddft_attenuate", self.lib.lrtddft_attenuate(self.h, C.byref(p), _dp(Sp), rep))
        return Sp, [report_dict(r) for r in rep]

    def attenuate_noalloc(self, params: Optional[lrt_atten_params] = None):
        """lrtddft_attenuate without device allocation (fixed 16 MiB workspace in the library;
        calls must not overlap on the GPU)."""
        p = params if params is not None else atten_params()
        Sp = np.zeros(self._rows(self.nw))
        rep = (lrt_atten_report * (self.nq * self.neta))()
        _check("lrtddft_attenuate_noalloc",
               self.lib.lrtddft_attenuate_noalloc(self.h, C.byref(p), _dp(Sp), rep))
        return Sp, [report_dict(r) for r in rep]

    # --- the eta-convergence test (Sec. 2) ---
    def set_eta_list(self, etas):
        """Broadenings (Ha, strictly increasing) computed together by later assemblies; outputs
        then carry an eta axis after q."""
        e = np.ascontiguousarray(etas, dtype=np.float64)
        _check("lrtddft_set_eta_list", self.lib.lrtddft_set_eta_list(self.h, len(e), _dp(e)))
        self.neta = len(e)

    def get_eta_list(self) -> np.ndarray:
        n = C.c_int()
        _check("lrtddft_get_eta_list", self.lib.lrtddft_get_eta_list(self.h, C.byref(n), None))
        e = np.zeros(n.value)
        _check("lrtddft_get_eta_list", self.lib.lrtddft_get_eta_list(self.h, C.byref(n), _dp(e)))
        return e

    def eta_scan(self, tau, tol: float):
        """(F [nq][neta][ntau], metrics [nq][neta][5], reference eta index [nq])."""
        tau = np.ascontiguousarray(tau, dtype=np.float64)
        F = np.zeros((self.nq, self.neta, len(tau)))
        m = np.zeros((self.nq, self.neta, 5))
        ref = np.zeros(self.nq, dtype=np.int32)
        _check("lrtddft_eta_scan", self.lib.lrtddft_eta_scan(
            self.h, len(tau), _dp(tau), float(tol), _dp(F), _dp(m), ref.ctypes.data_as(C.POINTER(C.c_int))))
        return F, m, ref

    # --- dielectric properties (Sec. 3, Eqs. 10-11) ---
    def dielectric(self, S) -> dict:
        """chi, 1/eps, eps and sigma at the w >= 0 samples from S (rows as dsf returns them)."""
        S = np.ascontiguousarray(S, dtype=np.float64)
        npos = int(np.sum(np.asarray(self.wl.omega) >= 0.0))
        out = np.zeros(self._rows(npos, 8))
        _check("lrtddft_dielectric", self.lib.lrtddft_dielectric(self.h, _dp(S), _dp(out)))
        z = lambda k: out[..., k] + 1j * out[..., k + 1]
        return {"w": np.asarray(self.wl.omega)[np.asarray(self.wl.omega) >= 0.0], "chi": z(0),
                "eps_inv": z(2), "eps": z(4), "sigma": z(6)}

    # --- Kubo-Greenwood route (App. A.3) ---
    def kubo_greenwood(self, etas, tau, tol: float) -> dict:
        e = np.ascontiguousarray(etas, dtype=np.float64)
        tau = np.ascontiguousarray(tau, dtype=np.float64)
        ne = len(e)
        sigma = np.zeros((ne, self.nw), dtype=np.complex128)
        S = np.zeros((ne, self.nw))
        F = np.zeros((ne, len(tau)))
        m = np.zeros((ne, 5))
        ref = C.c_int()
        _check("lrtddft_kubo_greenwood", self.lib.lrtddft_kubo_greenwood(
            self.h, ne, _dp(e), len(tau), _dp(tau), float(tol), sigma.ctypes.data_as(_D), _dp(S), _dp(F),
            _dp(m), C.byref(ref)))
        return {"sigma": sigma, "S": S, "F": F, "metrics": m, "eta_ref": ref.value}

    def kubo_greenwood_attenuate(self, params: Optional[lrt_atten_params] = None):
        p = params if params is not None else atten_params()
        Sp = np.zeros(self.nw)
        rep = lrt_atten_report()
        npos = int(np.sum(np.asarray(self.wl.omega) >= 0.0))
        out = np.zeros((npos, 8))
        _check("lrtddft_kubo_greenwood_attenuate", self.lib.lrtddft_kubo_greenwood_attenuate(
            self.h, C.byref(p), _dp(Sp), C.byref(rep), _dp(out)))
        z = lambda k: out[:, k] + 1j * out[:, k + 1]
        return Sp, report_dict(rep), {"chi_star": z(0), "eps_inv": z(2), "eps": z(4), "sigma": z(6)}

    # --- instrumentation ---
    def profile(self, enable: bool = True):
        _check("lrtddft_profile", self.lib.lrtddft_profile(self.h, 1 if enable else 0))

    def profile_read(self) -> dict:
        out = np.zeros(8)
        _check("lrtddft_profile_read", self.lib.lrtddft_profile_read(self.h, _dp(out)))
        return {"launches": int(out[0]), "chi0_launches": int(out[1]), "chi0_ms": float(out[2]),
                "rho_launches": int(out[3]), "rho_ms": float(out[4]), "chi0_cmac": float(out[5])}

    # --- hooks ---
    def set_orbitals(self, iq: int, eps: np.ndarray, coeff: np.ndarray, occ: Optional[np.ndarray] = None):
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        cf = np.ascontiguousarray(coeff, dtype=np.complex128)
        oc = None if occ is None else np.ascontiguousarray(occ, dtype=np.float64)
        _check("lrtddft_set_orbitals", self.lib.lrtddft_set_orbitals(
            self.h, iq, _dp(eps), cf.ctypes.data_as(_D), None if oc is None else _dp(oc)))

    def set_orbitals_async(self, iq: int, eps: np.ndarray, coeff: np.ndarray,
                           occ: Optional[np.ndarray] = None):
        """Pipelined set_orbitals: coeff (ideally page-locked, e.g. a pinned torch tensor's
        numpy view) is copied while earlier work runs and must stay unchanged until the next
        chi0_assemble of iq has been followed by a call that returns results."""
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        if coeff.dtype != np.complex128 or not coeff.flags.c_contiguous:
            raise ValueError("coeff must be a C-contiguous complex128 array (it is read after the call)")
        oc = None if occ is None else np.ascontiguousarray(occ, dtype=np.float64)
        _check("lrtddft_set_orbitals_async", self.lib.lrtddft_set_orbitals_async(
            self.h, iq, _dp(eps), coeff.ctypes.data_as(_D), None if oc is None else _dp(oc)))

    def get_orbitals(self, iq: int, out: Optional[np.ndarray] = None) -> np.ndarray:
        if out is None:
            out = np.zeros((2, self.nk, self.nb, self.npw), dtype=np.complex128)
        _check("lrtddft_get_orbitals", self.lib.lrtddft_get_orbitals(self.h, iq, out.ctypes.data_as(_D)))
        return out

    def get_basis(self, iq: int):
        m = np.zeros((2, self.nk, self.npw, 3), dtype=np.int32)
        n = np.zeros((2, self.nk), dtype=np.int32)
        _check("lrtddft_get_basis", self.lib.lrtddft_get_basis(
            self.h, iq, m.ctypes.data_as(_I32), n.ctypes.data_as(_I32)))
        return m, n

    def get_ground_state(self, iq: int):
        e = np.zeros((2, self.nk, self.nb))
        f = np.zeros((2, self.nk, self.nb))
        w = np.zeros((2, self.nk, self.nb))
        mu = C.c_double()
        _check("lrtddft_get_ground_state", self.lib.lrtddft_get_ground_state(
            self.h, iq, _dp(e), _dp(f), _dp(w), C.byref(mu)))
        return e, f, mu.value, w

    def get_gset(self, iq: int):
        nG = int(self.wl.nG[iq])
        m = np.zeros((nG, 3), dtype=np.int32)
        K = np.zeros(nG)
        _check("lrtddft_get_gset", self.lib.lrtddft_get_gset(self.h, iq, m.ctypes.data_as(_I32), _dp(K)))
        return m, K

    def get_chi0(self, iq: int) -> np.ndarray:
        nG = int(self.wl.nG[iq])
        out = np.zeros((self.neta * self.nwi, nG, nG), dtype=np.complex128)
        _check("lrtddft_get_chi0", self.lib.lrtddft_get_chi0(self.h, iq, out.ctypes.data_as(_D)))
        return out if self.neta == 1 else out.reshape(self.neta, self.nwi, nG, nG)

    def get_pair_densities(self, iq: int) -> np.ndarray:
        """rho[p][G] of q index iq from the context's pair-density kernel (test hook)."""
        nG = int(self.wl.nG[iq])
        out = np.zeros((self.nk * self.nb * self.nb, nG), dtype=np.complex128)
        _check("lrtddft_get_pair_densities",
               self.lib.lrtddft_get_pair_densities(self.h, iq, out.ctypes.data_as(_D)))
        return out

    def get_chi_col0(self, iq: int) -> np.ndarray:
        nG = int(self.wl.nG[iq])
        out = np.zeros((self.neta * self.nwi, nG), dtype=np.complex128)
        _check("lrtddft_get_chi_col0", self.lib.lrtddft_get_chi_col0(self.h, iq, out.ctypes.data_as(_D)))
        return out if self.neta == 1 else out.reshape(self.neta, self.nwi, nG)

    def get_frequencies(self):
        f = np.zeros(self.nwi)
        h = C.c_int()
        _check("lrtddft_get_frequencies", self.lib.lrtddft_get_frequencies(self.h, _dp(f), C.byref(h)))
        return f, h.value


def report_dict(r: lrt_atten_report) -> dict:
    degs = []
    for i in range(MAXDEG):
        if r.degree[i] < 0:
            continue
        degs.append({"d": r.degree[i], "m": r.window[i], "score": r.score[i],
                     "mean_ratio": r.mean_ratio[i], "rms_ratio": r.rms_ratio[i],
                     "accepted": bool(r.accepted[i])})
    return {"n_accepted": r.n_accepted, "targets": [t for t in r.targets if t >= 0], "degrees": degs}
