"""GPU: response G-sets beyond the shared-memory Dyson solver (N_G > 118), where each Dyson
matrix (and its transpose in the adjoint) lives in a per-block slice of a global workspace.
Through the C ABI, against the FP64 oracle:

 - FP64 path with ragged N_G = 130 and 200 in one context: chi0, chi_00, S to 1e-10 of the
   per-q max norm, F and the metrics to 1e-10 relative;
 - FP16x3 path on the same workload at the split-precision bounds (chi0 3e-5 of the max norm,
   F 1e-5 pointwise);
 - FP64 adjoint at N_G = 130 (f_xc model kernel) against the oracle's analytic tangents, 1e-8
   of each parameter's max |dF|.
"""
import numpy as np
import pytest

from oracle import adjoint, pipeline, response
from paper_2510_01875_gb300 import binding, build
from paper_2510_01875_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return binding.load()


def large():
    wl = W.tiny(seed=51, nq=2, nw=24, kmesh=(2, 2, 2), nbands=8)
    return wl.replace(nG=np.array([130, 200]))


def run(wl, prec):
    c = binding.Context(wl, prec)
    c.chi0_assemble()
    c.dyson_solve()
    tau = response.tau_grid(wl.T, wl.ntau)
    F, m = c.itcf(tau)
    out = {"S": c.dsf(), "F": F, "metrics": m, "chi0": [c.get_chi0(i) for i in range(wl.nq)],
           "chi": [c.get_chi_col0(i) for i in range(wl.nq)]}
    c.close()
    return out


def rel_max(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.fixture(scope="module")
def oracle_runs():
    wl = large()
    return wl, [pipeline.run_q(wl, iq, keep_chi0=True) for iq in range(wl.nq)]


def test_fp64_large_ng_against_oracle(oracle_runs):
    wl, ref = oracle_runs
    g = run(wl, "fp64")
    for iq in range(wl.nq):
        r = ref[iq]
        assert g["chi0"][iq].shape[1] == wl.nG[iq]
        assert rel_max(g["chi0"][iq], r["chi0"]) < TOL, iq
        assert rel_max(g["chi"][iq][:, 0], r["chi00"]) < TOL, iq
        assert rel_max(g["S"][iq], r["S"]) < TOL, iq
        assert np.abs(g["F"][iq] / r["F"] - 1).max() < TOL, iq
        assert np.abs(g["metrics"][iq] / r["metrics"] - 1).max() < TOL, iq


def test_split_large_ng_against_oracle(oracle_runs):
    wl, ref = oracle_runs
    g = run(wl, "fp16x3")
    for iq in range(wl.nq):
        r = ref[iq]
        assert rel_max(g["chi0"][iq], r["chi0"]) < 3e-5, iq
        assert np.abs(g["F"][iq] / r["F"] - 1).max() < 1e-5, iq


def test_fp64_adjoint_large_ng_against_oracle_tangents():
    wl = W.tiny(seed=52, nq=1, nw=20, kmesh=(2, 2, 2), nbands=8, kernel="fxc_model", nG=130)
    tau = response.tau_grid(wl.T, 8)
    c = binding.Context(wl, "fp64")
    c.chi0_assemble()
    c.dyson_solve()
    dS, dF = c.jacobian(tau)
    c.close()
    t = adjoint.tangents_q(wl, 0, tau)
    for j in range(5):
        ref = t["dF"][:, j]
        scale = np.abs(ref).max()
        if scale == 0.0:
            assert np.all(dF[0, :, j] == 0.0), j
            continue
        assert np.abs(dF[0, :, j] - ref).max() / scale < 1e-8, j
