"""Pins of the oracle's dielectric post-processing (Sec. 3 closing relations, Eqs. 10-11):
the Kramers-Kronig transform on a damped oscillator, whose real and imaginary parts are known
in closed form, and the identities between chi, 1/eps, eps and sigma."""
import math

import numpy as np

from oracle import dielectric as D


def _oscillator(w, A=-1.0, w0=1.0, g=0.3):
    """chi(w) = A / (w0^2 - w^2 - i g w): causal (poles in the lower half plane), Im chi odd."""
    return A / (w0 * w0 - w * w - 1j * g * w)


def test_kramers_kronig_reproduces_a_damped_oscillator():
    errs = []
    for h in (0.04, 0.02, 0.01):
        w = np.arange(0.0, 40.0 + 0.5 * h, h)
        chi = _oscillator(w)
        re = D.kramers_kronig(w, chi.imag)
        inner = w < 10.0   # away from the truncation at 40
        errs.append(np.abs(re[inner] - chi.real[inner]).max() / np.abs(chi.real).max())
    # at least second order in h (the error falls 40x from h = 0.04 to 0.02) down to the floor
    # set by the truncation of the integral at w = 40 (5e-7 here)
    assert errs[0] / errs[1] > 4.0
    assert errs[2] < 1e-6 and errs[1] < 1e-6


def test_kramers_kronig_at_zero_is_the_static_integral():
    """At w = 0 the formula is the regular integral (2/pi) int Im chi(w')/w' dw' = chi(0)."""
    h = 0.005
    w = np.arange(0.0, 60.0 + 0.5 * h, h)
    chi = _oscillator(w)
    re = D.kramers_kronig(w, chi.imag)
    assert abs(re[0] - chi[0].real) < 1e-4 * abs(chi[0].real)


def test_dielectric_identities():
    w = np.linspace(0.0, 3.0, 31)
    chi = _oscillator(w)
    q = 0.7
    eps_inv, eps, sigma = D.dielectric(chi, q, w)
    np.testing.assert_allclose(eps_inv, 1 + 4 * math.pi / q ** 2 * chi, rtol=1e-15)
    np.testing.assert_allclose(eps * eps_inv, np.ones_like(eps), rtol=1e-14)
    # eps = 1 + (4 pi i/w) sigma (Eq. 11)
    np.testing.assert_allclose(1 + 4j * math.pi / w[1:] * sigma[1:], eps[1:], rtol=1e-13)


def test_im_chi_inverts_the_fluctuation_dissipation_relation():
    T, n = 0.3, 0.027
    w = np.linspace(0.0, 2.0, 21)[1:]
    im = -np.abs(np.sin(w))
    S = -im / (math.pi * n * (-np.expm1(-w / T)))
    np.testing.assert_allclose(D.im_chi_from_dsf(S, w, T, n), im, rtol=1e-14)
