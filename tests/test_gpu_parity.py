"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, element by element,
on seeded workloads that span several tiles with ragged tails.

Tolerances (FP64 path): chi0 and S to 1e-10 of their per-q max norm, F and the metrics to
1e-10 relative (F > 0).  Only gauge-invariant outputs are compared (chi0, chi, S, F)."""
import math

import numpy as np
import pytest

from oracle import crystal, pipeline, response
from paper_2510_01875_gb300 import binding, build
from paper_2510_01875_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return binding.load()


def gpu_run(wl, precision="fp64"):
    ctx = binding.Context(wl, precision)
    ctx.chi0_assemble()
    ctx.dyson_solve()
    S = ctx.dsf()
    tau = response.tau_grid(wl.T, wl.ntau)
    F, m = ctx.itcf(tau)
    chi0 = [ctx.get_chi0(iq) for iq in range(wl.nq)]
    chi = [ctx.get_chi_col0(iq) for iq in range(wl.nq)]
    freqs, hcol = ctx.get_frequencies()
    gs = [ctx.get_ground_state(iq) for iq in range(wl.nq)]
    ctx.close()
    return {"S": S, "F": F, "metrics": m, "chi0": chi0, "chi": chi, "freqs": freqs, "hcol": hcol,
            "gs": gs}


def rel_max(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def compare(wl, g, tol=TOL, chi0_tol=None):
    chi0_tol = tol if chi0_tol is None else chi0_tol
    for iq in range(wl.nq):
        r = pipeline.run_q(wl, iq, keep_chi0=True)
        assert np.allclose(g["freqs"], r["freqs"], rtol=0, atol=0)
        assert g["hcol"] == r["hcol"]
        eps, _, mu, wgt = g["gs"][iq]
        ref_gs = response.ground_state(wl, iq)
        nb = wl.nbands
        assert np.abs(eps[0][:, :nb] - ref_gs["eps_k"][:, :nb]).max() < 1e-10
        assert np.abs(eps[1][:, :nb] - ref_gs["eps_kq"][:, :nb]).max() < 1e-10
        # band weights (split multiplets at the band cut) agree
        nbr = ref_gs["nb"]
        assert np.array_equal(wgt[0][:, :nbr], ref_gs["w_k"]) and not wgt[0][:, nbr:].any()
        assert np.array_equal(wgt[1][:, :nbr], ref_gs["w_kq"]) and not wgt[1][:, nbr:].any()
        if not math.isnan(r["mu"]):
            assert abs(mu - r["mu"]) < 1e-10
        assert rel_max(g["chi0"][iq], r["chi0"]) < chi0_tol, "chi0"
        assert rel_max(g["chi"][iq][:, 0], r["chi00"]) < tol, "chi_00"
        assert rel_max(g["S"][iq], r["S"]) < tol, "S"
        assert np.abs(g["F"][iq] / r["F"] - 1).max() < tol, "F"
        assert np.abs(g["metrics"][iq] / r["metrics"] - 1).max() < tol, "metrics"


CASES = {
    # two displaced atoms in a cubic cell, time-reversal-symmetric mesh, 2 q
    "tiny_tr": W.tiny(),
    # fixed basis, static f_xc model kernel
    "tiny_fixed_fxc": W.tiny(seed=3, basis="fixed", kernel="fxc_model", nG=11, nbands=9),
    # zero potential, RPA
    "tiny_free_rpa": W.tiny(seed=5, potential="zero", kernel="rpa", natoms_displaced=False,
                            nbands=10, ecut=2.5),
    # ragged tiles: 70 bands (two 64-band tiles), 19 G (three 8-G blocks), 45 frequencies
    "ragged": W.tiny(seed=9, nq=1, nbands=70, ecut=5.0, nG=19, nw=45, kmesh=(2, 1, 2)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp64_parity_small(name):
    wl = CASES[name]
    compare(wl, gpu_run(wl))


def test_fp64_parity_commensurate():
    wl = W.tiny(seed=11, kscheme="commensurate", nq=1, natoms_displaced=False, kmesh=(4, 4, 4),
                ecut=2.5, nbands=12)
    wl = wl.replace(q=np.array([0.25 * crystal.reciprocal(wl.lattice)[1] + 0.25 * crystal.reciprocal(wl.lattice)[2]]))
    compare(wl, gpu_run(wl))


def test_fp64_parity_al1_fcc_k8():
    """The fcc Al, 8^3 mesh, 24 bands, 15 G, 256 frequencies workload, in full."""
    wl = W.al1_fcc_k8_b24()
    compare(wl, gpu_run(wl))


def test_detailed_balance_on_gpu():
    wl = W.tiny(seed=13, nq=1, nw=41, wmin_ev=-40.0, wmax_ev=40.0)
    g = gpu_run(wl)
    S = g["S"][0]
    beta = 1.0 / wl.T
    for j in range(wl.nw // 2 + 1, wl.nw):
        jm = wl.nw - 1 - j
        assert abs(S[jm] - math.exp(-beta * wl.omega[j]) * S[j]) < 1e-10 * np.abs(S).max()


def test_itcf_direct_mode_and_symmetry():
    wl = W.tiny(seed=13, nq=1, nw=41, wmin_ev=-40.0, wmax_ev=40.0)
    ctx = binding.Context(wl)
    ctx.chi0_assemble()
    ctx.dyson_solve()
    S = ctx.dsf()
    beta = 1.0 / wl.T
    tau = np.linspace(0.0, beta, 33)
    Ff, _ = ctx.itcf(tau, "fold")
    Fd, _ = ctx.itcf(tau, "direct")
    ctx.close()
    assert np.abs(Ff[0] - Ff[0][::-1]).max() < 1e-13 * Ff.max()
    ref = response.itcf_direct(wl.omega, S[0], tau)
    assert np.abs(Fd[0] / ref - 1).max() < 1e-12


def test_call_order_errors():
    wl = W.tiny(nq=1)
    ctx = binding.Context(wl)
    with pytest.raises(binding.LrtError) as e:
        ctx.dyson_solve()
    assert e.value.status == "calls out of order"
    with pytest.raises(binding.LrtError):
        ctx.dsf()
    with pytest.raises(binding.LrtError):
        ctx.chi0_assemble(0, 5)
    ctx.close()
