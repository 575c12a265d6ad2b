"""Oracle: dielectric properties from a (filtered) dynamic structure factor.

Test infrastructure only (see oracle/__init__.py).

Sec. 3 (after the workflow figure) and App. A.2 (Eqs. 10 and 11): once S_p(q,w) is known, the
fluctuation-dissipation theorem (Eq. 8) gives Im chi, the Kramers-Kronig relation gives Re chi,
and the dielectric function and the conductivity follow:
  Im chi(q,w) = -pi n (1 - e^{-beta w}) S(q,w)                     (Eq. 8 solved for Im chi)
  Re chi(q,w) = (2/pi) P int_0^inf w' Im chi(q,w') / (w'^2 - w^2) dw'   (Kramers-Kronig for a
                response whose imaginary part is odd in w)
  1/eps(q,w)  = 1 + (4 pi/q^2) chi(q,w)                            (Eq. 10)
  sigma(q,w)  = (i w/(4 pi)) (1 - eps(q,w))                        (Eq. 11 solved for sigma)

Discretisation of the principal value (a reading; the paper gives none): Maclaurin's formula
(Ohta and Ishida, Appl. Spectrosc. 42, 952 (1988)) on the uniformly spaced samples
w_j >= 0 of the grid, spacing h:
  Re chi(w_i) = (2/pi) 2h sum_{j: i - j odd} w_j Im chi(w_j) / (w_j^2 - w_i^2),
which skips the singular node and is second order in h; the part of the integral below the
first sample and above the last one is not included (truncation).  At w = 0 the sum is the
regular integral (2/pi) int Im chi(w')/w' dw'.

Pinned by (tests/test_oracle_dielectric.py): a damped oscillator chi = A/(w0^2 - w^2 - i g w),
whose real part the transform of its imaginary part must reproduce to the truncation and
O(h^2) discretisation errors (the error falls 4x per halving of h), and the identities of
Eqs. 10-11 on it.
"""
from __future__ import annotations

import math

import numpy as np


def positive_samples(omega):
    """Indices of the w >= 0 samples (uniformly spaced) and their spacing."""
    w = np.asarray(omega)
    sel = np.where(w >= 0.0)[0]
    if len(sel) < 3:
        raise ValueError("at least 3 samples with w >= 0 are needed")
    h = w[sel[1]] - w[sel[0]]
    if np.abs(np.diff(w[sel]) - h).max() > 1e-9 * h:
        raise ValueError("the w >= 0 samples must be uniformly spaced")
    return sel, h


def im_chi_from_dsf(S, omega, T, n):
    """Im chi = -pi n (1 - e^{-w/T}) S (Eq. 8)."""
    w = np.asarray(omega)
    return -math.pi * n * (-np.expm1(-w / T)) * np.asarray(S)


def kramers_kronig(w, imchi):
    """Re chi at the uniform samples w (>= 0) from Im chi there, by Maclaurin's formula."""
    w = np.asarray(w, dtype=np.float64)
    imchi = np.asarray(imchi, dtype=np.float64)
    N = len(w)
    h = w[1] - w[0]
    idx = np.arange(N)
    out = np.zeros(N)
    for i in range(N):
        j = idx[(idx - i) % 2 == 1]          # the nodes of the other parity
        out[i] = (2.0 / math.pi) * 2.0 * h * np.sum(w[j] * imchi[j] / (w[j] ** 2 - w[i] ** 2))
    return out


def dielectric(chi, q, w, v=None):
    """(1/eps, eps, sigma) from chi at |q| and the frequencies w (Eqs. 10 and 11); v overrides
    the Coulomb factor 4 pi/q^2 (v = 1 for a response already scaled by it)."""
    chi = np.asarray(chi, dtype=np.complex128)
    vq = (4.0 * math.pi / (q * q)) if v is None else v
    eps_inv = 1.0 + vq * chi
    eps = 1.0 / eps_inv
    sigma = 1j * np.asarray(w) / (4.0 * math.pi) * (1.0 - eps)
    return eps_inv, eps, sigma


def from_dsf(S, omega, T, n, q, v=None):
    """For one q: (w, chi, 1/eps, eps, sigma) on the w >= 0 samples of the caller's grid."""
    sel, _ = positive_samples(omega)
    w = np.asarray(omega)[sel]
    im = im_chi_from_dsf(np.asarray(S)[sel], w, T, n)
    chi = kramers_kronig(w, im) + 1j * im
    eps_inv, eps, sigma = dielectric(chi, q, w, v)
    return w, chi, eps_inv, eps, sigma
