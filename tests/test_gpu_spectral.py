"""GPU: chi0 through a spectral function (lrtddft_set_spectral) against the oracle's spectral
form (oracle/spectral.py, pinned to the direct sum) and against the direct engine.

 - FP64 context: the grid (x_0, n_b) equals the oracle's; chi0 at every internal frequency
   within 1e-10 of the oracle's spectral chi0 (orders 1 and 3), and S(q, w) (with its exact
   w -> 0 limit) within 1e-10 of the oracle's S built from that chi0;
 - an eta list: every eta's chi0 from the one spectral function, against the oracle per eta;
 - split context: FP32 pair sums with compensated accumulation, within 1e-5 of the oracle,
   also at N_G = 200 (a smaller staged chunk);
 - against the direct engine at h = eta/16, order 3: within the interpolation bound;
 - the adjoint and graph capture are refused, and bad arguments are rejected.
"""
import numpy as np
import pytest

from oracle import crystal, response, spectral
from paper_2510_01875_gb300 import binding, build
from paper_2510_01875_gb300 import workloads as W

pytestmark = pytest.mark.gpu

WL = W.tiny(seed=71, nq=2, nw=50, kmesh=(3, 3, 3), nbands=10, nG=9)


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return binding.load()


def _oracle_parts(wl, iq):
    gset = crystal.response_gset(wl.lattice, wl.q[iq], int(wl.nG[iq]))
    gs = response.ground_state(wl, iq)
    rho = response.pair_densities(wl, gs, gset).reshape(-1, len(gset))
    delta, df = response.pair_weights(gs)
    freqs, hcol = response.internal_frequencies(wl.omega)
    return gset, rho, delta, df, freqs, hcol, crystal.volume(wl.lattice)


def _ctx(wl, prec, h, order):
    c = binding.Context(wl, prec)
    c.set_spectral(h, order)
    c.chi0_assemble()
    c.dyson_solve()
    return c


@pytest.mark.parametrize("order", [1, 3])
def test_fp64_spectral_against_oracle(order):
    wl = WL
    h = wl.eta / 8
    c = _ctx(wl, "fp64", h, order)
    S = c.dsf()
    n = response.density(wl)
    for iq in range(wl.nq):
        gset, rho, delta, df, freqs, hcol, om = _oracle_parts(wl, iq)
        ref, x0, nb = spectral.chi0_spectral(rho, delta, df, freqs, wl.eta, wl.nk, om, h, order)
        gx0, gnb = c.get_spectral_grid(iq)
        assert gnb == nb and abs(gx0 - x0) <= 1e-12 * max(1.0, abs(x0))
        got = c.get_chi0(iq)
        assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()
        # S from that chi0, with the exact w -> 0 limit (its eta derivative is the pair sum's)
        K = response.kernel_diag(wl, wl.q[iq], gset)
        chiG0 = response.dyson_column0(ref, K)
        deta = response.chi0_eta_derivative(rho, delta, df, 0.0, wl.eta, wl.nk, om)
        S0 = response.s_zero(response.chi00_derivative(ref[hcol], deta, K), wl.T, n)
        S_ref = response.dsf(chiG0[:, 0], wl.omega, S0, wl.T, n)
        assert np.abs(S[iq] - S_ref).max() <= 1e-10 * np.abs(S_ref).max()
    c.close()


def test_eta_list_from_one_spectral_function():
    wl = WL.replace(q=WL.q[:1], nG=WL.nG[:1])
    etas = np.array([0.5, 1.0, 2.0]) * wl.eta
    h = wl.eta / 8
    c = binding.Context(wl, "fp64")
    c.set_spectral(h, 3)
    c.set_eta_list(etas)
    c.chi0_assemble()
    got = c.get_chi0(0)   # [eta][w][G][G']
    _, rho, delta, df, freqs, _, om = _oracle_parts(wl, 0)
    for j, eta in enumerate(etas):
        ref, _, _ = spectral.chi0_spectral(rho, delta, df, freqs, eta, wl.nk, om, h, 3)
        assert np.abs(got[j] - ref).max() <= 1e-10 * np.abs(ref).max(), j
    c.close()


@pytest.mark.parametrize("prec", ["fp16x3", "bf16x3"])
def test_split_spectral_against_oracle(prec):
    wl = WL
    h = wl.eta / 8
    c = _ctx(wl, prec, h, 3)
    for iq in range(wl.nq):
        _, rho, delta, df, freqs, _, om = _oracle_parts(wl, iq)
        ref, _, _ = spectral.chi0_spectral(rho, delta, df, freqs, wl.eta, wl.nk, om, h, 3)
        got = c.get_chi0(iq)
        assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max(), iq
    c.close()


def test_split_spectral_large_g_set():
    """N_G = 200: the moments kernel stages 16 sorted pairs per chunk instead of 32 (two chunks
    of 200 pair densities next to the FP32 bin totals fill the shared memory)."""
    wl = W.tiny(seed=73, nq=1, nw=24, kmesh=(2, 2, 2), nbands=8, nG=200)
    h = wl.eta / 8
    c = _ctx(wl, "fp16x3", h, 3)
    _, rho, delta, df, freqs, _, om = _oracle_parts(wl, 0)
    ref, _, _ = spectral.chi0_spectral(rho, delta, df, freqs, wl.eta, wl.nk, om, h, 3)
    got = c.get_chi0(0)
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()
    c.close()


def test_spectral_against_direct_engine():
    wl = WL
    direct = binding.Context(wl, "fp64")
    direct.chi0_assemble()
    c = _ctx(wl, "fp64", wl.eta / 16, 3)
    for iq in range(wl.nq):
        a, b = c.get_chi0(iq), direct.get_chi0(iq)
        # order-3 interpolation of 1/(w - x + i eta) at h = eta/16: about (1/16)^4 relative
        assert np.abs(a - b).max() <= 2.0 * (1.0 / 16) ** 4 * np.abs(b).max(), iq
    c.close()
    direct.close()


def test_refusals_and_arguments():
    wl = W.tiny(seed=72, nq=1, nw=20)
    c = binding.Context(wl, "fp64")
    for h, order in ((-1.0, 3), (0.01, 2), (float("nan"), 3)):
        with pytest.raises(binding.LrtError):
            c.set_spectral(h, order)
    c.set_spectral(wl.eta / 4, 1)
    c.chi0_assemble()
    c.dyson_solve()
    with pytest.raises(binding.LrtError):
        c.jacobian(response.tau_grid(wl.T, 4))
    c.set_spectral(0.0)   # back to the direct engine: the adjoint runs
    c.chi0_assemble()
    c.dyson_solve()
    c.jacobian(response.tau_grid(wl.T, 4))
    c.close()
