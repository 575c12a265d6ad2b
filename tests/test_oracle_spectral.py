"""Pins of the oracle's spectral-function chi0 (oracle/spectral.py) against mathematics that does
not go through its own formulas:
 - Lagrange weights of order m reproduce every polynomial of degree <= m exactly (and not
   degree m + 1);
 - with every pole on a grid node the spectral chi0 equals the direct Adler-Wiser sum;
 - on a real cell the error against the direct sum falls as h^(m+1).
"""
import numpy as np
import pytest

from oracle import crystal, response, spectral
from paper_2510_01875_gb300 import workloads as W


@pytest.mark.parametrize("order", [1, 3])
def test_weights_reproduce_polynomials(order):
    rng = np.random.default_rng(5)
    x = rng.uniform(-3.0, 4.0, 200)
    h = 0.37
    x0, nb = spectral.grid(x, h)
    j0, Wt = spectral.lagrange_weights(x, x0, h, order)
    assert j0.min() >= 0 and (j0 + order).max() <= nb - 1
    nodes = x0 + h * (j0[:, None] + np.arange(order + 1)[None, :])
    for k in range(order + 1):
        assert np.abs((Wt * nodes ** k).sum(axis=1) - x ** k).max() <= 1e-12 * (1 + np.abs(x) ** k).max()
    miss = np.abs((Wt * nodes ** (order + 1)).sum(axis=1) - x ** (order + 1)).max()
    assert miss > 1e-6


def _cell():
    wl = W.tiny(seed=61, nq=1, nw=30, kmesh=(2, 2, 2), nbands=8, nG=7)
    gset = crystal.response_gset(wl.lattice, wl.q[0], int(wl.nG[0]))
    gs = response.ground_state(wl, 0)
    rho = response.pair_densities(wl, gs, gset).reshape(-1, len(gset))
    delta, df = response.pair_weights(gs)
    freqs, _ = response.internal_frequencies(wl.omega)
    return wl, rho, delta, df, freqs, crystal.volume(wl.lattice)


@pytest.mark.parametrize("order", [1, 3])
def test_poles_on_nodes_equal_direct_sum(order):
    wl, rho, delta, df, freqs, om = _cell()
    h = 0.01
    delta = -h * np.round(-delta / h)   # move every pole onto a node of the grid
    ref = response.chi0(rho, delta, df, freqs, wl.eta, wl.nk, om)
    got, _, _ = spectral.chi0_spectral(rho, delta, df, freqs, wl.eta, wl.nk, om, h, order)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("order", [1, 3])
def test_error_falls_as_h_to_the_order_plus_one(order):
    wl, rho, delta, df, freqs, om = _cell()
    ref = response.chi0(rho, delta, df, freqs, wl.eta, wl.nk, om)
    errs = []
    hs = [wl.eta / 8, wl.eta / 16, wl.eta / 32]
    for h in hs:
        got, _, _ = spectral.chi0_spectral(rho, delta, df, freqs, wl.eta, wl.nk, om, h, order)
        errs.append(np.abs(got - ref).max() / np.abs(ref).max())
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(r - (order + 1)) < 0.35 for r in rates), (errs, rates)
    # and the bound (h/eta)^(m+1) holds with a modest constant
    assert errs[-1] <= 2.0 * (hs[-1] / wl.eta) ** (order + 1)
