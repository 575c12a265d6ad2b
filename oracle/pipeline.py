"""Oracle: the whole response path for one workload, q by q.

Test infrastructure only (see oracle/__init__.py).

Order of steps (the paper's workflow, Sec. 3 workflow figure, with the response engine
ahead of it): ground state -> pair densities -> chi0 -> Dyson -> S (Eq. 8) -> F (Eq. 1),
F-tilde (Eq. 2) and metrics -> attenuation (Sec. 3).
"""
from __future__ import annotations

import numpy as np

from . import crystal, response


def run_q(wl, iq: int, keep_chi0: bool = False, freqs_subset=None) -> dict:
    """Everything for q index iq.  freqs_subset (indices into the internal frequency list)
    restricts chi0 and Dyson to a slice of frequencies (for timing samples)."""
    q = wl.q[iq]
    gset = crystal.response_gset(wl.lattice, q, int(wl.nG[iq]))
    gs = response.ground_state(wl, iq)
    rho = response.pair_densities(wl, gs, gset)              # [k, n, n', G]
    rho_flat = rho.reshape(-1, len(gset))
    delta, df = response.pair_weights(gs)
    freqs, hcol = response.internal_frequencies(wl.omega)
    if freqs_subset is not None:
        freqs = freqs[freqs_subset]
    om = crystal.volume(wl.lattice)
    chi0 = response.chi0(rho_flat, delta, df, freqs, wl.eta, wl.nk, om)
    K = response.kernel_diag(wl, q, gset)
    chiG0 = response.dyson_column0(chi0, K)
    out = {"gset": gset, "mu": gs["mu"], "K": K, "chi00": chiG0[:, 0], "freqs": freqs,
           "hcol": hcol, "delta": delta, "df": df}
    if keep_chi0:
        out["chi0"] = chi0
    if freqs_subset is not None:
        return out
    n = response.density(wl)
    deta = response.chi0_eta_derivative(rho_flat, delta, df, 0.0, wl.eta, wl.nk, om)
    S0 = response.s_zero(response.chi00_derivative(chi0[hcol], deta, K), wl.T, n)
    S = response.dsf(chiG0[:, 0], wl.omega, S0, wl.T, n)
    wp, Sp = response.positive_branch(S, wl.omega, S0)
    tau = response.tau_grid(wl.T, wl.ntau)
    out.update({"S": S, "S0": S0, "wp": wp, "Sp": Sp, "tau": tau,
                "dchi00_deta0": response.chi00_derivative(chi0[hcol], deta, K),
                "F": response.itcf_fold(wp, Sp, tau, wl.T),
                "metrics": response.itcf_metrics(wp, Sp, wl.T, n)})
    return out


def run(wl, keep_chi0: bool = False) -> list:
    return [run_q(wl, iq, keep_chi0) for iq in range(wl.nq)]
