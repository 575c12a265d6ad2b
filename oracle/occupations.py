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


def electron_count(eps, mu: float, T: float, nk: int) -> float:
    return 2.0 * float(np.sum(fermi(eps, mu, T))) / nk


def chemical_potential(eps, T: float, nelec: float, nk: int) -> float:
    """Bisection for mu with 200 halvings of [min(eps) - 60 T, max(eps) + 60 T]."""
    eps = np.asarray(eps)
    if 2.0 * eps.size / nk < nelec:
        raise ValueError("not enough bands to hold the electrons")
    lo = float(eps.min()) - 60.0 * T
    hi = float(eps.max()) + 60.0 * T
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if electron_count(eps, mid, T, nk) < nelec:
            lo = mid
        else:
            hi = mid
        if hi - lo <= 0.0:
            break
    return 0.5 * (lo + hi)
