"""Pins of the oracle's Kubo-Greenwood route (App. A.3): the optical-limit L(w) against this
oracle's own Adler-Wiser chi0 at small q (an independent route: pair densities by G-space
correlation at finite q), the w -> 0 limit of S*_KG, and the relations of Eqs. 10-11."""
import math

import numpy as np

from oracle import crystal, kubo, response
from paper_2510_01875_gb300 import workloads as W

BASE = W.tiny(nq=1, kmesh=(2, 2, 2), nbands=8, nG=3, nw=11, wmin_ev=2.0, wmax_ev=40.0)


def _aw_interband_over_q2(qm):
    """(1/3) sum over q along x, y, z of chi0_00(q, w)/q^2 with the intraband pairs (n = n')
    removed: the trace/3 of the interband optical limit as |q| -> 0."""
    freqs = np.asarray(BASE.omega)
    out = []
    for a in range(3):
        q = np.zeros(3)
        q[a] = qm
        wl = BASE.replace(q=q[None])
        gs = response.ground_state(wl, 0)
        rho = response.pair_densities(wl, gs, crystal.response_gset(wl.lattice, q, 1)).reshape(-1, 1)
        d, df = response.pair_weights(gs)
        inter = 1.0 - np.eye(gs["nb"])[None].repeat(wl.nk, axis=0)
        out.append(response.chi0(rho, d, df * inter.reshape(-1), freqs, wl.eta, wl.nk,
                                 crystal.volume(wl.lattice))[:, 0, 0] / qm ** 2)
    return np.mean(out, axis=0)


def _kg_L(qm):
    wl = BASE.replace(q=np.array([[qm, 0.0, 0.0]]))
    d, g = kubo.kg_pairs(wl, response.ground_state(wl, 0))
    return kubo.kg_L(d, g, np.asarray(BASE.omega), wl.eta)


def test_kg_is_the_optical_limit_of_adler_wiser():
    errs = []
    for qm in (2e-4, 1e-4):
        L = _kg_L(qm)
        errs.append(np.abs(_aw_interband_over_q2(qm) - L).max() / np.abs(L).max())
    assert errs[0] / errs[1] > 3.5          # the difference is O(q^2)
    assert errs[1] < 2e-4


def test_kg_s_zero_is_the_limit_of_s():
    wl = W.tiny(nq=1, kmesh=(2, 2, 2), nbands=8, nw=31, wmin_ev=-20.0, wmax_ev=40.0)
    gs = response.ground_state(wl, 0)
    _, _, S0 = kubo.kg_spectra(wl, gs, wl.eta)
    d, g = kubo.kg_pairs(wl, gs)
    h = 1e-4
    L = kubo.kg_L(d, g, np.array([h, 2 * h]), wl.eta)
    im = (1.0 / (1.0 - 4 * math.pi * L) - 1.0).imag
    n = response.density(wl)
    ref = -(wl.T / (math.pi * n)) * (4 * im[0] / h - im[1] / (2 * h)) / 3
    assert abs(S0 - ref) < 2e-8 * abs(ref)
    assert S0 > 0


def test_kg_relations_of_eqs_10_11():
    wl = W.tiny(nq=1, kmesh=(2, 2, 2), nbands=8, nw=31, wmin_ev=1.0, wmax_ev=40.0)
    gs = response.ground_state(wl, 0)
    sigma, S, _ = kubo.kg_spectra(wl, gs, wl.eta)
    d, g = kubo.kg_pairs(wl, gs)
    L = kubo.kg_L(d, g, np.asarray(wl.omega), wl.eta)
    w = np.asarray(wl.omega)
    eps = 1 + 4j * math.pi * sigma / w                     # Eq. 11
    np.testing.assert_allclose(eps, 1 - 4 * math.pi * L, rtol=1e-13)
    chi_star = 1 / eps - 1                                 # Eq. 10 with v chi = chi*
    n = response.density(wl)
    np.testing.assert_allclose(S, -chi_star.imag / (math.pi * n * (-np.expm1(-w / wl.T))), rtol=1e-13)
    assert np.all(S > 0)
