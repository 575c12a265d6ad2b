"""Oracle: the eta-convergence test and the attenuation started from the Kubo-Greenwood
conductivity (App. A.3).

Test infrastructure only (see oracle/__init__.py).

The optical limit q -> 0 of the interband Adler-Wiser response, on the k mesh of q index 0 of
the workload (readings: the paper starts from sigma_KG of an external code; here it is built
from the same orbitals as the rest of the path, trace/3 of the conductivity tensor):
  p_nn'(k) = <nk| -i grad |n'k> = sum_G c*_nk(G) (k + G) c_n'k(G)          momentum matrix
  L(w)     = lim chi0_inter(q, w)/q^2
           = (2/(N_k Omega)) sum_{k, n, n'} df_nn' (|p_nn'|^2/3) / Delta^2 / (w + Delta + i eta),
             Delta = eps_nk - eps_n'k, df_nn' = w_nk w_n'k (f_nk - f_n'k) (band weights as in the
             Adler-Wiser sum); pairs with Delta = 0 have df = 0 and are left out
  sigma_KG(w) = i w L(w)                  (continuity: sigma = i w chi/q^2, so that Eq. 11's
                                           eps = 1 + 4 pi i sigma/w is 1 - (4 pi/q^2) chi0)
  eps_KG(w)   = 1 + 4 pi i sigma_KG(w)/w = 1 - 4 pi L(w)
  chi*_KG(w)  = v(q) chi_KG(q, w) = 1/eps_KG(w) - 1          (Eqs. 10 and 12, v(q) = 4 pi/q^2)
  S*_KG(w)    = -Im chi*_KG(w) / (pi n (1 - e^{-w/T}))        (Eq. 13, hbar = 1, with the pi of
                                                               the library's reading)
  S*_KG(0)    = (T/(pi n)) Re d(1/eps_KG)/d eta at w = 0 = (T/(pi n)) Re[4 pi L_eta(0)/eps_KG(0)^2],
                L_eta = dL/d eta (L depends on w + i eta only, as in the S(q,0) limit)
  F*_KG       = the detailed-balance fold of Eq. 1 over S*_KG (Eq. 14, F* = v(q) F_KG)
After the reference eta is found (etascan.reference_eta), S*_KG at that eta is attenuated
(attenuation.attenuate) and the filtered chi*, eps and sigma follow from it (dielectric.py with
v = 1, since chi* already carries v(q)).

Pinned by (tests/test_oracle_kubo.py): L(w) against the Adler-Wiser chi0 of this oracle at small
q (interband pairs, averaged over three orthogonal q directions), which it approaches as q^2;
S*_KG(0) against the w -> 0 limit of S*_KG(w) (Richardson); and the algebra of
Eqs. 10-11 between sigma, eps and chi*.
"""
from __future__ import annotations

import math

import numpy as np

from . import attenuation, crystal, dielectric, response


def momentum_matrices(lattice, k, basis, C) -> np.ndarray:
    """p[a][n, n'] = sum_G conj(C[G, n]) (k + G)_a C[G, n'] for a = x, y, z."""
    kg = k[None, :] + basis @ crystal.reciprocal(lattice)
    return np.array([C.conj().T @ (kg[:, a][:, None] * C) for a in range(3)])


def kg_pairs(wl, gs):
    """(Delta_p, g_p) over the pairs (k, n, n') with Delta != 0: g_p = pref df |p|^2 / (3 Delta^2)."""
    pref = 2.0 / (wl.nk * crystal.volume(wl.lattice))
    deltas, gs_ = [], []
    for ik in range(wl.nk):
        P = momentum_matrices(wl.lattice, gs["k"][ik], gs["basis_k"][ik], gs["C_k"][ik])
        p2 = np.sum(np.abs(P) ** 2, axis=0)
        e, f, w = gs["eps_k"][ik], gs["f_k"][ik], gs["w_k"][ik]
        d = e[:, None] - e[None, :]
        df = (f[:, None] - f[None, :]) * w[:, None] * w[None, :]
        m = d != 0.0
        deltas.append(d[m])
        gs_.append(pref * df[m] * p2[m] / (3.0 * d[m] ** 2))
    return np.concatenate(deltas), np.concatenate(gs_)


def kg_L(delta, g, freqs, eta) -> np.ndarray:
    """L(w) = sum_p g_p / (w + Delta_p + i eta)."""
    return np.array([np.sum(g / (w + delta + 1j * eta)) for w in freqs])


def kg_spectra(wl, gs, eta):
    """For one eta on the workload's grid: sigma_KG(w) (sigma(0) = 0), S*_KG(w), and S*_KG(0)."""
    delta, g = kg_pairs(wl, gs)
    omega = np.asarray(wl.omega)
    L = kg_L(delta, g, omega, eta)
    n = response.density(wl)
    T = wl.T
    sigma = 1j * omega * L
    chi_star = 1.0 / (1.0 - 4.0 * math.pi * L) - 1.0
    L0 = np.sum(g / (delta + 1j * eta))
    L0_eta = np.sum(g * (-1j) / (delta + 1j * eta) ** 2)
    eps0 = 1.0 - 4.0 * math.pi * L0
    S0 = T * (4.0 * math.pi * L0_eta / eps0 ** 2).real / (math.pi * n)
    S = np.zeros(len(omega))
    for j, w in enumerate(omega):
        S[j] = S0 if w == 0.0 else -chi_star[j].imag / (math.pi * n * (-math.expm1(-w / T)))
    return sigma, S, S0


def kg_scan(wl, etas, tau):
    """Per eta: sigma [nw], S* [nw], F* [ntau], metrics [5] (F of Eq. 1 and the Sec. 2 metrics)."""
    gs = response.ground_state(wl, 0)
    n = response.density(wl)
    out = []
    for eta in etas:
        sigma, S, S0 = kg_spectra(wl, gs, eta)
        wp, Sp = response.positive_branch(S, wl.omega, S0)
        out.append({"sigma": sigma, "S": S, "S0": S0,
                    "F": response.itcf_fold(wp, Sp, tau, wl.T),
                    "metrics": response.itcf_metrics(wp, Sp, wl.T, n)})
    return out


def kg_filtered(wl, S, S0, params: attenuation.AttenParams):
    """Attenuated S*_KG and the filtered chi*, eps and sigma at the w >= 0 samples."""
    Sp, rep = attenuation.attenuate(wl.omega, S, S0, wl.T, wl.ntau, params)
    w, chi, eps_inv, eps, sigma = dielectric.from_dsf(Sp, wl.omega, wl.T, response.density(wl),
                                                      q=None, v=1.0)
    return Sp, rep, w, chi, eps, sigma
