"""Pins of the oracle's analytic tangents of F(q, tau) (oracle/adjoint.py).

The tangents are propagated by hand through occupations, weights, chi0, Dyson, S and the
Laplace fold; they are checked here against central differences of the oracle's plain
forward path (a separate computation), at fixed absolute tau.
"""
import numpy as np
import pytest

from oracle import adjoint, response
from paper_2510_01875_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _shift(wl, j, h):
    if j == 0:
        return wl.replace(T=wl.T + h)
    if j == 1:
        return wl.replace(eta=wl.eta + h)
    p = list(wl.fxc_params)
    p[j - 2] += h
    return wl.replace(fxc_params=tuple(p))


def _fd(wl, iq, tau, j, h):
    fp = adjoint.itcf_at(_shift(wl, j, h), iq, tau)
    fm = adjoint.itcf_at(_shift(wl, j, -h), iq, tau)
    return (fp - fm) / (2.0 * h)


@pytest.mark.parametrize("kscheme", ["tr_symmetric", "commensurate"])
def test_tangents_match_central_differences(kscheme):
    wl = W.tiny(seed=11, nq=1, kernel="fxc_model", kscheme=kscheme, nw=48, T_ev=4.0, eta_ev=0.6)
    tau = response.tau_grid(wl.T, 16)
    t = adjoint.tangents_q(wl, 0, tau)
    # the plain forward path and the tangent code agree on F itself
    np.testing.assert_allclose(t["F"], adjoint.itcf_at(wl, 0, tau), rtol=1e-12)
    steps = [1e-4 * wl.T, 1e-4 * wl.eta, 1e-4, 1e-4, 1e-4]
    for j, h in enumerate(steps):
        fd = _fd(wl, 0, tau, j, h)
        scale = max(np.abs(fd).max(), 1e-300)
        err = np.abs(t["dF"][:, j] - fd).max() / scale
        assert err < 2e-6, (j, err)


def test_tangents_with_omega_zero_on_grid():
    # omega = 0 on the grid: S(0) comes from the h-limit form, which depends on T directly
    wl = W.tiny(seed=12, nq=1, kernel="fxc_model", nw=41, wmin_ev=-20.0, wmax_ev=20.0)
    assert np.any(wl.omega == 0.0)
    tau = response.tau_grid(wl.T, 9)
    t = adjoint.tangents_q(wl, 0, tau)
    for j, h in ((0, 1e-4 * wl.T), (1, 1e-4 * wl.eta), (3, 1e-4)):
        fd = _fd(wl, 0, tau, j, h)
        assert np.abs(t["dF"][:, j] - fd).max() / np.abs(fd).max() < 2e-6


@pytest.mark.parametrize("kernel", ["rpa", "rpa_alda"])
def test_kernel_parameters_do_not_enter_rpa_and_alda(kernel):
    wl = W.tiny(seed=13, nq=1, kernel=kernel, nw=24)
    t = adjoint.tangents_q(wl, 0, response.tau_grid(wl.T, 5))
    assert np.all(t["dF"][:, 2:] == 0.0)
    assert np.abs(t["dF"][:, :2]).max() > 0.0


def test_vjp_is_the_contracted_tangent():
    wl = W.tiny(seed=14, nq=2, kernel="fxc_model", nw=24)
    tau = response.tau_grid(wl.T, 6)
    g = np.random.default_rng(0).standard_normal((2, 6))
    full = sum(g[i] @ adjoint.tangents_q(wl, i, tau)["dF"] for i in range(2))
    np.testing.assert_allclose(adjoint.vjp(wl, tau, g), full, rtol=1e-13)
