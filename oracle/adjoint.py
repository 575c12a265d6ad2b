"""Oracle: analytic forward-mode tangents of F(q, tau) and S(q, w) with respect to
theta = (T, eta, A, B, C).

Test infrastructure only (see oracle/__init__.py).  The GPU path differentiates in reverse
mode (vector-Jacobian product); this module propagates the five tangents forward through
every step, in the order of the forward path, so the two share nothing but the definitions:

  occupations  f = 1/(1 + e^{(eps - mu)/T});  df/dT = f(1 - f) [(eps - mu)/T^2 + mu'/T],
               mu' = dmu/dT from d/dT (2/N_k) sum w f = 0 (k mesh of the q, band weights w);
  weights      w_p(w) = df_p/(w + Delta_p + i eta):  dw_p/dT = (d df_p/dT)/(w + Delta_p + i eta),
               dw_p/deta = -i df_p/(w + Delta_p + i eta)^2;
  chi0         the Adler-Wiser sum of each weight tangent;
  kernel       K_GG = 4 pi/|q+G|^2 + A f_ALDA (1 + B |q+G|^2) e^{-C |q+G|^2} for the f_xc
               model (tangents of A, B, C; zero for RPA and RPA+ALDA); f_ALDA is the zero-
               temperature value at the mean density, so K does not depend on T;
  Dyson        M = 1 - chi0 K, chi_{:,0} = M^{-1} chi0_{:,0}:
               d chi_{:,0} = M^{-1} [d chi0 (K chi_{:,0} + e_0) + chi0 dK chi_{:,0}];
  S (Eq. 8)    S = -Im chi_00/(pi n (1 - e^{-w/T})); at w = 0 the limit
               S(0) = (T/(pi n)) Re s, s = d chi_00/d eta = [M^{-1} E v]_0, E = d chi0/d eta,
               v = K chi_{:,0} + e_0, whose tangents are second derivatives:
               d(M^{-1} E v) = M^{-1} [dE v + E dv - dM M^{-1} E v],  dM = -(d chi0 K + chi0 dK),
               dE/dT = sum_p rho rho* (-i d df_p/dT)/(w + Delta_p + i eta)^2,
               dE/deta = sum_p rho rho* (-2 df_p)/(w + Delta_p + i eta)^3;
  F (Eq. 1)    the detailed-balance fold; tau is held fixed (absolute), so T also enters
               through e^{-(1/T - tau) w}.
"""
from __future__ import annotations

import math

import numpy as np

from . import crystal, response, xc

NTHETA = 5   # T, eta, A, B, C


def _mu_tangent(gs, T: float) -> float:
    """dmu/dT at fixed orbitals: the electron count over the k mesh stays N_e."""
    f = gs["f_k"]
    w = gs["w_k"]
    g = w * f * (1.0 - f)
    den = float(np.sum(g))
    if den == 0.0:
        return 0.0
    return -float(np.sum(g * (gs["eps_k"] - gs["mu"]))) / (T * den)


def occupation_tangents(gs, T: float, fixed: bool):
    """(df_k/dT, df_kq/dT); zero when the occupations are supplied by the caller."""
    if fixed:
        return np.zeros_like(gs["f_k"]), np.zeros_like(gs["f_kq"])
    mup = _mu_tangent(gs, T)
    out = []
    for tag in ("k", "kq"):
        f = gs["f_" + tag]
        e = gs["eps_" + tag]
        out.append(f * (1.0 - f) * ((e - gs["mu"]) / (T * T) + mup / T))
    return out[0], out[1]


def kernel_tangents(wl, q, gset) -> np.ndarray:
    """dK_GG/d(A, B, C) as [3][N_G]."""
    out = np.zeros((3, len(gset)))
    if wl.kernel != "fxc_model":
        return out
    A, Bp, C = wl.fxc_params
    Bm = crystal.reciprocal(wl.lattice)
    qg = q[None, :] + gset @ Bm
    qg2 = np.einsum("ij,ij->i", qg, qg)
    fa = xc.fxc_alda(response.density(wl))
    e = np.exp(-C * qg2)
    out[0] = fa * (1.0 + Bp * qg2) * e
    out[1] = A * fa * qg2 * e
    out[2] = -A * fa * (1.0 + Bp * qg2) * qg2 * e
    return out


def tangents_q(wl, iq: int, tau) -> dict:
    """F and S of q index iq at the absolute imaginary times tau, and their tangents
    dF[ntau][5], dS[nw][5] (order T, eta, A, B, C)."""
    q = wl.q[iq]
    T = wl.T
    beta = 1.0 / T
    tau = np.asarray(tau, dtype=np.float64)
    gset = crystal.response_gset(wl.lattice, q, int(wl.nG[iq]))
    gs = response.ground_state(wl, iq)
    rho = response.pair_densities(wl, gs, gset).reshape(-1, len(gset))
    delta, df = response.pair_weights(gs)
    dfk, dfkq = occupation_tangents(gs, T, wl.occupations is not None)
    ddf = (dfk[:, :, None] - dfkq[:, None, :]) * gs["w_k"][:, :, None] * gs["w_kq"][:, None, :]
    ddf = ddf.reshape(-1)
    freqs, hcol = response.internal_frequencies(wl.omega)
    om = crystal.volume(wl.lattice)
    pref = 2.0 / (wl.nk * om)
    nG = len(gset)
    K = response.kernel_diag(wl, q, gset)
    dK = kernel_tangents(wl, q, gset)
    n = response.density(wl)

    chi00 = np.zeros(len(freqs), dtype=np.complex128)
    dchi00 = np.zeros((len(freqs), NTHETA), dtype=np.complex128)
    e0 = np.zeros(nG, dtype=np.complex128)
    e0[0] = 1.0
    s0 = 0.0
    ds0 = np.zeros(NTHETA, dtype=np.complex128)
    for iw, w in enumerate(freqs):
        den = w + delta + 1j * wl.eta
        wt = df / den
        c0 = pref * ((rho * wt[:, None]).T @ rho.conj())
        dc_T = pref * ((rho * (ddf / den)[:, None]).T @ rho.conj())
        dc_eta = pref * ((rho * (-1j * df / den ** 2)[:, None]).T @ rho.conj())
        M = np.eye(nG) - c0 * K[None, :]
        x = response.solve_gauss(M[None], c0[None, :, 0].copy())[0]
        chi00[iw] = x[0]
        v = K * x + e0
        rhs = np.stack([dc_T @ v, dc_eta @ v] + [c0 @ (dK[j] * x) for j in range(3)])
        dx = response.solve_gauss(np.repeat(M[None], NTHETA, axis=0), rhs)
        dchi00[iw] = dx[:, 0]
        if iw == hcol:
            # s = d chi_00/d eta at w = 0 and its tangents (second derivatives of chi_00)
            y = response.solve_gauss(M[None], (dc_eta @ v)[None])[0]
            s0 = y[0]
            dE = [pref * ((rho * (-1j * ddf / den ** 2)[:, None]).T @ rho.conj()),
                  pref * ((rho * (-2.0 * df / den ** 3)[:, None]).T @ rho.conj())]
            dc = [dc_T, dc_eta]
            r = []
            for j in range(NTHETA):
                dKj = dK[j - 2] if j >= 2 else np.zeros(nG)
                dcj = dc[j] if j < 2 else np.zeros_like(c0)
                dv = dKj * x + K * dx[j]
                dM = -(dcj * K[None, :] + c0 * dKj[None, :])
                t = dc_eta @ dv - dM @ y
                if j < 2:
                    t = t + dE[j] @ v
                r.append(t)
            ds0 = response.solve_gauss(np.repeat(M[None], NTHETA, axis=0), np.stack(r))[:, 0]

    # S on the caller's grid and its tangents (Eq. 8)
    nw = len(wl.omega)
    S = np.zeros(nw)
    dS = np.zeros((nw, NTHETA))
    for j, w in enumerate(wl.omega):
        if w == 0.0:
            S[j], dS[j] = _s0_and_tangent(s0, ds0, T, n)
            continue
        g = 1.0 / (-math.expm1(-beta * w))
        S[j] = -chi00[j].imag * g / (math.pi * n)
        dS[j] = -dchi00[j].imag * g / (math.pi * n)
        dg = math.exp(-beta * w) * w / (T * T) * g * g
        dS[j, 0] += -chi00[j].imag * dg / (math.pi * n)
    S0, dS0 = _s0_and_tangent(s0, ds0, T, n)

    # F (Eq. 1, detailed-balance fold) at fixed absolute tau
    wp, Sp = response.positive_branch(S, wl.omega, S0)
    w_arr = np.asarray(wl.omega)
    pos = w_arr >= 0.0
    dSp = dS[pos]
    if len(wp) != int(np.sum(pos)):
        dSp = np.concatenate([dS0[None, :], dSp])
    wtr = response.trapezoid_weights(wp)
    e1 = np.exp(-np.outer(tau, wp))
    e2 = np.exp(-np.outer(beta - tau, wp))
    F = (e1 + e2) @ (wtr * Sp)
    dF = (e1 + e2) @ (wtr[:, None] * dSp)
    dF[:, 0] += (e2 * wp[None, :] / (T * T)) @ (wtr * Sp)
    return {"F": F, "dF": dF, "S": S, "dS": dS, "chi00": chi00, "dchi00": dchi00,
            "freqs": freqs, "hcol": hcol}


def _s0_and_tangent(s, ds, T, n):
    """S(0) = (T/(pi n)) Re s, s = d chi_00/d eta at w = 0, and its tangents."""
    S0 = T * s.real / (math.pi * n)
    dS0 = np.array(T * ds.real / (math.pi * n), dtype=np.float64)
    dS0[0] += s.real / (math.pi * n)
    return S0, dS0


def itcf_at(wl, iq: int, tau) -> np.ndarray:
    """F(q, tau) of the plain forward path at absolute tau (for central differences)."""
    r = response
    q = wl.q[iq]
    gset = crystal.response_gset(wl.lattice, q, int(wl.nG[iq]))
    gs = r.ground_state(wl, iq)
    rho = r.pair_densities(wl, gs, gset).reshape(-1, len(gset))
    delta, df = r.pair_weights(gs)
    freqs, hcol = r.internal_frequencies(wl.omega)
    c0 = r.chi0(rho, delta, df, freqs, wl.eta, wl.nk, crystal.volume(wl.lattice))
    K = r.kernel_diag(wl, q, gset)
    chi00 = r.dyson_column0(c0, K)[:, 0]
    n = r.density(wl)
    om = crystal.volume(wl.lattice)
    deta = r.chi0_eta_derivative(rho, delta, df, 0.0, wl.eta, wl.nk, om)
    S0 = r.s_zero(r.chi00_derivative(c0[hcol], deta, K), wl.T, n)
    S = r.dsf(chi00, wl.omega, S0, wl.T, n)
    wp, Sp = r.positive_branch(S, wl.omega, S0)
    return r.itcf_fold(wp, Sp, tau, wl.T)


def vjp(wl, tau, dL_dF) -> np.ndarray:
    """sum_{q, tau} dL/dF(q, tau) dF(q, tau)/dtheta for all q (reverse product of the
    forward tangents)."""
    g = np.zeros(NTHETA)
    for iq in range(wl.nq):
        t = tangents_q(wl, iq, tau)
        g += np.asarray(dL_dF[iq]) @ t["dF"]
    return g
