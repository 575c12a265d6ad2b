"""Oracle: the Adler-Wiser chi0 through a spectral function on a grid of transition energies and
a transform of it to the frequency grid (an engine variant that the paper does not use: it
removes the number of frequencies from the cost of the pair sum).

Test infrastructure only (see oracle/__init__.py).

With x_p = -Delta_p = eps_n'k+q - eps_nk, the direct sum (response.chi0)
    chi0_GG'(w) = pref sum_p P_p(G,G') df_p / (w - x_p + i eta),   P_p = rho_p(G) rho_p*(G'),
is replaced by
    A_b(G,G')   = sum_p P_p(G,G') df_p L_b(x_p)                    (the spectral function)
    chi0_GG'(w) = pref sum_b A_b(G,G') / (w - x_b + i eta)         (its transform)
on the uniform grid x_b = x_0 + b h, where L_b(x) are the Lagrange interpolation weights of
order m on the m + 1 grid nodes around x: m = 1, the two nodes x_j <= x < x_{j+1}; m = 3, the
four nodes x_{j-1} .. x_{j+2}.  For each pair this replaces 1/(w - x_p + i eta) by its order-m
interpolant in x_p, so the relative error of chi0 is O((h/eta)^(m+1)).
Grid (a reading; any grid covering the poles would do): over the pairs with df_p != 0,
x_0 = h (floor(min x_p / h) - 1) and n_b = floor((max x_p - x_0)/h) + 3, so every node used
lies on the grid.  pref = 2/(N_k Omega), as in response.chi0.

Pinned by tests/test_oracle_spectral.py: the weights reproduce polynomials of degree <= m
exactly (sum_b L_b(x) x_b^k = x^k); poles placed on grid nodes give the direct sum to rounding;
the error against the direct sum falls as h^(m+1) on a random cell.
"""
from __future__ import annotations

import math

import numpy as np


def grid(x: np.ndarray, h: float):
    """(x_0, n_b) of the bin grid covering the poles x (see the module docstring)."""
    if len(x) == 0:
        return 0.0, 0
    x0 = h * (math.floor(float(np.min(x)) / h) - 1.0)
    nb = int(math.floor((float(np.max(x)) - x0) / h)) + 3
    return x0, nb


def lagrange_weights(x: np.ndarray, x0: float, h: float, order: int):
    """(first node index j0 [len(x)], weights W [len(x), order + 1]) of each x on the grid."""
    t = (np.asarray(x, dtype=np.float64) - x0) / h
    j = np.floor(t)
    f = t - j
    j = j.astype(np.int64)
    if order == 1:
        return j, np.stack([1.0 - f, f], axis=1)
    if order == 3:
        # nodes at offsets -1, 0, 1, 2 from j; f in [0, 1)
        W = np.stack([-f * (f - 1.0) * (f - 2.0) / 6.0,
                      (f + 1.0) * (f - 1.0) * (f - 2.0) / 2.0,
                      -(f + 1.0) * f * (f - 2.0) / 2.0,
                      (f + 1.0) * f * (f - 1.0) / 6.0], axis=1)
        return j - 1, W
    raise ValueError("order must be 1 or 3")


def spectral_function(rho_flat, delta, df, h: float, order: int):
    """A [n_b][G][G'] and the grid (x_0, n_b): A_b = sum_p rho_p rho_p^H df_p L_b(x_p) over the
    pairs with df_p != 0."""
    keep = df != 0.0
    x = -np.asarray(delta)[keep]
    w = np.asarray(df)[keep]
    r = rho_flat[keep]
    x0, nb = grid(x, h)
    nG = rho_flat.shape[1]
    A = np.zeros((nb, nG, nG), dtype=np.complex128)
    if nb == 0:
        return A, x0, nb
    j0, W = lagrange_weights(x, x0, h, order)
    for c in range(order + 1):
        b = j0 + c
        coef = w * W[:, c]
        for bb in np.unique(b):
            sel = b == bb
            rs = r[sel]
            A[bb] += (rs * coef[sel][:, None]).T @ rs.conj()
    return A, x0, nb


def chi0_from_spectral(A, x0: float, h: float, freqs, eta: float, nk: int, omega_cell: float):
    """chi0[w, G, G'] = pref sum_b A_b(G,G') / (w - x_b + i eta)."""
    nb = A.shape[0]
    xb = x0 + h * np.arange(nb)
    kern = 1.0 / (np.asarray(freqs)[:, None] - xb[None, :] + 1j * eta)
    pref = 2.0 / (nk * omega_cell)
    return pref * np.einsum("wb,bgh->wgh", kern, A)


def chi0_spectral(rho_flat, delta, df, freqs, eta, nk, omega_cell, h: float, order: int = 3):
    """The spectral-function chi0 on the internal frequencies: (chi0, x_0, n_b)."""
    A, x0, nb = spectral_function(rho_flat, delta, df, h, order)
    return chi0_from_spectral(A, x0, h, freqs, eta, nk, omega_cell), x0, nb
