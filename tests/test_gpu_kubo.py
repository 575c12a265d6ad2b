"""GPU: the Kubo-Greenwood route of the eta-convergence test (App. A.3) through the C ABI
against the oracle (FP64): sigma_KG, S*_KG and F*_KG per eta and the Sec. 2 metrics to 1e-10,
the reference-eta index against the oracle's rule on the same metrics, and the attenuated S*_KG
with the filtered chi*, eps and sigma (Kramers-Kronig, Eqs. 10-11)."""
import numpy as np
import pytest

from oracle import attenuation, etascan, kubo, response
from paper_2510_01875_gb300 import binding, build
from paper_2510_01875_gb300 import workloads as W

pytestmark = pytest.mark.gpu

WL = W.tiny(nq=1, kmesh=(3, 3, 3), nbands=10, nw=81, wmin_ev=-20.0, wmax_ev=60.0)
ETAS = [W.ev(x) for x in (0.2, 0.35, 0.5, 0.8)]


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return binding.load()


def test_kubo_greenwood_scan_and_filter():
    tau = response.tau_grid(WL.T, WL.ntau)
    tol = 2e-2
    ctx = binding.Context(WL, "fp64")
    r = ctx.kubo_greenwood(ETAS, tau, tol)
    ref_scan = kubo.kg_scan(WL, ETAS, tau)
    for j, o in enumerate(ref_scan):
        assert np.abs(r["sigma"][j] - o["sigma"]).max() <= 1e-10 * np.abs(o["sigma"]).max(), j
        assert np.abs(r["S"][j] - o["S"]).max() <= 1e-10 * np.abs(o["S"]).max(), j
        assert np.abs(r["F"][j] / o["F"] - 1).max() <= 1e-10, j
        assert np.abs(r["metrics"][j] / o["metrics"] - 1).max() <= 1e-10, j
    assert r["eta_ref"] == etascan.reference_eta(r["metrics"], tol)
    Sp, rep, der = ctx.kubo_greenwood_attenuate()
    ctx.close()
    o = ref_scan[r["eta_ref"]]
    Sp_o, rep_o, w, chi, eps, sigma = kubo.kg_filtered(WL, o["S"], o["S0"], attenuation.AttenParams())
    assert rep["n_accepted"] == rep_o["n_accepted"]
    assert np.abs(Sp - Sp_o).max() <= 1e-9 * np.abs(Sp_o).max()
    for key, ref in (("chi_star", chi), ("eps", eps), ("sigma", sigma)):
        assert np.abs(der[key] - ref).max() <= 1e-9 * np.abs(ref).max(), key
