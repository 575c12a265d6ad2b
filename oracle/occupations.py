"""Oracle: Fermi-Dirac occupations and the chemical potential.

Test infrastructure only (see oracle/__init__.py).

f(eps) = 1 / (1 + exp((eps - mu)/T)), spin-unpolarised (factor 2 outside).
mu solves (2/N_k) sum_{k,n} f(eps_nk) = N_e, found by plain bisection.

Pinned by: electron-count neutrality to 1e-13 and, at zero potential on a dense mesh,
agreement with the free-gas Fermi-Dirac integral (tests/test_oracle_basics.py).
"""
from __future__ import annotations

import numpy as np
from scipy.special import expit


def fermi(eps, mu: float, T: float):
    return expit(-(np.asarray(eps) - mu) / T)


def electron_count(eps, mu: float, T: float, nk: int, weights=None) -> float:
    f = fermi(eps, mu, T)
    if weights is not None:
        f = f * weights
    return 2.0 * float(np.sum(f)) / nk


def chemical_potential(eps, T: float, nelec: float, nk: int, weights=None) -> float:
    """Bisection for mu with 200 halvings of [min(eps) - 60 T, max(eps) + 60 T]; `weights`
    (band weights of a split degenerate multiplet, else 1) multiply each state's count."""
    eps = np.asarray(eps)
    cap = eps.size if weights is None else float(np.sum(weights))
    if 2.0 * cap / nk < nelec:
        raise ValueError("not enough bands to hold the electrons")
    lo = float(eps.min()) - 60.0 * T
    hi = float(eps.max()) + 60.0 * T
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if electron_count(eps, mid, T, nk, weights) < nelec:
            lo = mid
        else:
            hi = mid
        if hi - lo <= 0.0:
            break
    return 0.5 * (lo + hi)
