"""Oracle: pair densities, Adler-Wiser chi0, Dyson, S(q,w) and F(q,tau).

Test infrastructure only (see oracle/__init__.py).

Definitions (Hartree atomic units, spin factor 2, Omega = cell volume, N_k = k points):
  pair p = (k, n, n'),  Delta_p = eps_nk - eps_n'k+q,  df_p = f_nk - f_n'k+q
  rho_p(G) = <nk| e^{-i(q+G).r} |n'k+q> = sum_G1 c*_nk(G1) c_n'k+q(G1+G)      (direct
             G-space correlation; no FFT)
  w_p(w)   = df_p / (w + Delta_p + i eta)
  chi0_GG'(q,w) = (2/(N_k Omega)) sum_p rho_p(G) rho_p*(G') w_p(w)            (Adler-Wiser)
  K_GG = 4 pi/|q+G|^2 + f_xc                                                    (diagonal)
  chi = (1 - chi0 K)^{-1} chi0; only chi_{G,0} is solved for.
  S(q,w) = -Im chi_00(q,w) / (pi n (1 - e^{-beta w}))          fluctuation-dissipation, Eq. 8
           (hbar = 1; the 1/pi makes int w S dw = q^2/2, the f-sum rule)
  S(q,0) = lim_{w->0} of Eq. 8 = -(T/(pi n)) d Im chi_00/dw at w = 0 (Im chi_00(0) = 0 on the
           time-reversal-symmetric pair meshes).  chi0 depends on w and eta only through
           w + i eta and K on neither, so chi_00 is a function of w + i eta and
           d chi_00/dw = -i d chi_00/d eta:  S(q,0) = (T/(pi n)) Re d chi_00/d eta (w = 0), with
           d chi_00/d eta from the Dyson chain rule d x = M^{-1} (d chi0/d eta)(K x + e_0),
           d chi0/d eta = (2/(N_k Omega)) sum_p rho_p(G) rho_p*(G') (-i df_p)/(w + Delta_p + i eta)^2
  F(q,tau) = int dw S(q,w) e^{-tau w}                        two-sided Laplace transform, Eq. 1
           = int_0^wmax S(w) [e^{-tau w} + e^{-(beta-tau) w}] dw   using detailed balance
             S(-w) = e^{-beta w} S(w) (FOLD mode, trapezoid over the w >= 0 samples)
  F-tilde(tau) = F(tau) - F(0)                                                    Eq. 2
  metrics: F(beta/2), int_0^beta F dtau, F-tilde(beta/2), int_0^beta F-tilde dtau and the static
  response chi(q) = -n int_0^beta F dtau (Sec. 2).  The tau integral is done exactly per w:
  int_0^beta [e^{-tau w} + e^{-(beta-tau) w}] dtau = 2 (1 - e^{-beta w}) / w.

Pinned by (tests/test_oracle_response.py): the discrete and continuum Lindhard functions at
zero potential, S(q,0) against the analytic w-derivative of the discrete Lindhard sum and
against the limit of S(q,w) (Richardson extrapolation in w), the exact discrete f-sum rule, detailed balance to rounding on time-reversal
symmetric meshes, the analytic Laplace transform of a model spectrum, the scalar and K = 0
limits of Dyson, the Dyson residual, pair-density orthonormality and completeness, and a
brute-force chi0 built by real-space FFT products on a tiny cell.
"""
from __future__ import annotations

import math

import numpy as np

from . import crystal, occupations, xc

DEGEN_TOL = 1e-6  # Ha; eigenvalues this close to the last kept band form one multiplet
EXTRA_BANDS = 8   # eigenpairs computed beyond nbands to see a multiplet split by the cut


def _lookup(basis: np.ndarray):
    lo = basis.min(axis=0)
    shape = basis.max(axis=0) - lo + 1
    lut = -np.ones(tuple(shape), dtype=np.int64)
    idx = basis - lo
    lut[idx[:, 0], idx[:, 1], idx[:, 2]] = np.arange(len(basis))
    return lo, shape, lut


def pair_density(Ck, basis_k, Ckq, basis_kq, gset) -> np.ndarray:
    """rho[n, n', iG] = sum_G1 conj(Ck[G1, n]) Ckq[G1+G, n'] over G1 with G1+G in basis_kq."""
    lo, shape, lut = _lookup(basis_kq)
    nb = Ck.shape[1]
    rho = np.zeros((nb, Ckq.shape[1], len(gset)), dtype=np.complex128)
    for ig, G in enumerate(gset):
        t = basis_k + G[None, :] - lo[None, :]
        ok = np.all((t >= 0) & (t < shape[None, :]), axis=1)
        j = -np.ones(len(basis_k), dtype=np.int64)
        j[ok] = lut[t[ok, 0], t[ok, 1], t[ok, 2]]
        v = j >= 0
        rho[:, :, ig] = Ck[v].conj().T @ Ckq[j[v]]
    return rho


def basis_for(wl, k):
    if wl.basis == "fixed":
        return crystal.sphere_basis(wl.lattice, np.zeros(3), wl.ecut)
    return crystal.sphere_basis(wl.lattice, k, wl.ecut)


def density(wl) -> float:
    return wl.Z * wl.natoms / crystal.volume(wl.lattice)


def band_weights(e, nbands: int) -> np.ndarray:
    """Weights of the computed bands e (ascending): 1 for the lowest nbands, 0 above, except
    that a degenerate multiplet (|e_n - e_{nbands-1}| <= DEGEN_TOL) split by the cut keeps
    its share j/m on each of its m members (j of them below the cut).  The projector onto
    "the lowest nbands states" is then gauge-invariant, which it is not when the cut runs
    through a multiplet (e.g. at high-symmetry k of a Gamma-centred mesh)."""
    e = np.asarray(e)
    w = np.zeros(len(e))
    w[:nbands] = 1.0
    mem = np.where(np.abs(e - e[nbands - 1]) <= DEGEN_TOL)[0]
    j, m = int(np.sum(mem < nbands)), len(mem)
    if m > j:
        if mem.max() >= len(e) - 1:
            raise ValueError("degenerate multiplet at the band cut extends past the computed bands")
        w[mem] = j / m
    return w


def ground_state(wl, iq: int):
    """Eigenpairs on the k and k+q meshes of q index iq, band weights, occupations and mu.
    Arrays carry nb >= nbands bands: nbands plus any members of a multiplet split by the cut."""
    q = wl.q[iq]
    kpts, kqpts = crystal.pair_meshes(wl.lattice, wl.kmesh, q, wl.kscheme)
    out = {"k": kpts, "kq": kqpts, "eps_k": [], "eps_kq": [], "C_k": [], "C_kq": [],
           "basis_k": [], "basis_kq": [], "w_k": [], "w_kq": []}
    for tag, pts in (("k", kpts), ("kq", kqpts)):
        for kv in pts:
            b = basis_for(wl, kv)
            nfull = min(len(b), wl.nbands + EXTRA_BANDS)
            e, C = crystal.eigenstates(wl.lattice, wl.positions, wl.Z, wl.r_c, kv, b, nfull,
                                       wl.potential)
            out["eps_" + tag].append(e)
            out["C_" + tag].append(C)
            out["basis_" + tag].append(b)
            if wl.occupations is not None:
                w = np.zeros(nfull)
                w[:wl.nbands] = 1.0
            else:
                w = band_weights(e, wl.nbands)
            out["w_" + tag].append(w)
    nb = max(int(np.max(np.nonzero(w)[0])) + 1 for w in out["w_k"] + out["w_kq"])
    for tag in ("k", "kq"):
        out["eps_" + tag] = np.array([e[:nb] for e in out["eps_" + tag]])
        out["C_" + tag] = [C[:, :nb] for C in out["C_" + tag]]
        out["w_" + tag] = np.array([w[:nb] for w in out["w_" + tag]])
    out["nb"] = nb
    nelec = wl.Z * wl.natoms
    if wl.occupations is not None:
        out["mu"] = float("nan")
        out["f_k"] = np.zeros((wl.nk, nb))
        out["f_kq"] = np.zeros((wl.nk, nb))
        out["f_k"][:, :wl.nbands] = np.asarray(wl.occupations[iq][0])
        out["f_kq"][:, :wl.nbands] = np.asarray(wl.occupations[iq][1])
    else:
        mu = occupations.chemical_potential(out["eps_k"], wl.T, nelec, wl.nk, out["w_k"])
        out["mu"] = mu
        out["f_k"] = occupations.fermi(out["eps_k"], mu, wl.T)
        out["f_kq"] = occupations.fermi(out["eps_kq"], mu, wl.T)
    return out


def pair_densities(wl, gs, gset) -> np.ndarray:
    """rho[k, n, n', G] for all k of the mesh."""
    return np.array([pair_density(gs["C_k"][i], gs["basis_k"][i], gs["C_kq"][i], gs["basis_kq"][i], gset)
                     for i in range(wl.nk)])


def pair_weights(gs):
    """Delta_p and df_p = w_nk w_n'k+q (f_nk - f_n'k+q) flattened in (k, n, n') order (the band
    weights w are 1 except on a multiplet split by the band cut)."""
    d = gs["eps_k"][:, :, None] - gs["eps_kq"][:, None, :]
    df = gs["f_k"][:, :, None] - gs["f_kq"][:, None, :]
    df = df * gs["w_k"][:, :, None] * gs["w_kq"][:, None, :]
    return d.reshape(-1), df.reshape(-1)


def internal_frequencies(omega: np.ndarray):
    """The frequencies chi is evaluated at: the grid, plus w = 0 appended when 0 is not on it
    (S(q,0) is needed by the Laplace transform of Eq. 1).  Returns (freqs, index of w = 0)."""
    w = np.array(omega, dtype=np.float64)
    zero = np.where(w == 0.0)[0]
    if len(zero):
        return w, int(zero[0])
    return np.concatenate([w, [0.0]]), len(w)


def chi0(rho_flat, delta, df, freqs, eta, nk, omega_cell) -> np.ndarray:
    """chi0[w, G, G'] = (2/(N_k Omega)) sum_p rho_p(G) rho_p*(G') df_p/(w + Delta_p + i eta)."""
    out = np.zeros((len(freqs), rho_flat.shape[1], rho_flat.shape[1]), dtype=np.complex128)
    pref = 2.0 / (nk * omega_cell)
    for iw, w in enumerate(freqs):
        wt = df / (w + delta + 1j * eta)
        out[iw] = pref * ((rho_flat * wt[:, None]).T @ rho_flat.conj())
    return out


def chi0_eta_derivative(rho_flat, delta, df, w, eta, nk, omega_cell) -> np.ndarray:
    """d chi0[G, G']/d eta at frequency w:
    (2/(N_k Omega)) sum_p rho_p(G) rho_p*(G') (-i df_p) / (w + Delta_p + i eta)^2."""
    pref = 2.0 / (nk * omega_cell)
    wt = -1j * df / (w + delta + 1j * eta) ** 2
    return pref * ((rho_flat * wt[:, None]).T @ rho_flat.conj())


def chi00_derivative(chi0w: np.ndarray, dchi0w: np.ndarray, K: np.ndarray) -> complex:
    """d chi_00 at one frequency for a change d chi0 at fixed K (Dyson chain rule):
    M = 1 - chi0 K, x = M^{-1} chi0_{:,0}, d x = M^{-1} d chi0 (K x + e_0); returns d x_0."""
    N = len(K)
    M = np.eye(N) - chi0w * K[None, :]
    x = solve_gauss(M[None], chi0w[None, :, 0].copy())[0]
    v = K * x
    v[0] += 1.0
    return complex(solve_gauss(M[None], (dchi0w @ v)[None])[0][0])


def kernel_diag(wl, q, gset) -> np.ndarray:
    """K_GG = 4 pi/|q+G|^2 + f_xc for the workload's kernel choice."""
    B = crystal.reciprocal(wl.lattice)
    qg = q[None, :] + gset @ B
    qg2 = np.einsum("ij,ij->i", qg, qg)
    K = 4.0 * math.pi / qg2
    n = density(wl)
    if wl.kernel == "rpa":
        return K
    if wl.kernel == "rpa_alda":
        return K + xc.fxc_alda(n)
    if wl.kernel == "fxc_model":
        A, Bp, C = wl.fxc_params
        return K + np.array([xc.fxc_model(math.sqrt(v), n, A, Bp, C) for v in qg2])
    raise ValueError(wl.kernel)


def solve_gauss(M: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Gaussian elimination with partial pivoting, vectorised over the leading batch axis.
    M[batch, N, N], b[batch, N] -> x with M x = b."""
    A = M.copy()
    x = b.copy()
    nb, N, _ = A.shape
    rows = np.arange(nb)
    for c in range(N):
        piv = c + np.argmax(np.abs(A[:, c:, c]), axis=1)
        if np.any(np.abs(A[rows, piv, c]) == 0.0):
            raise np.linalg.LinAlgError("singular Dyson matrix")
        tmp = A[rows, c, :].copy()
        A[rows, c, :] = A[rows, piv, :]
        A[rows, piv, :] = tmp
        tb = x[rows, c].copy()
        x[rows, c] = x[rows, piv]
        x[rows, piv] = tb
        for r in range(c + 1, N):
            fac = A[:, r, c] / A[:, c, c]
            A[:, r, c:] -= fac[:, None] * A[:, c, c:]
            x[:, r] -= fac * x[:, c]
    for c in range(N - 1, -1, -1):
        x[:, c] = (x[:, c] - np.einsum("bj,bj->b", A[:, c, c + 1:], x[:, c + 1:])) / A[:, c, c]
    return x


def dyson_column0(chi0w: np.ndarray, K: np.ndarray) -> np.ndarray:
    """chi_{G,0} from (1 - chi0 K) chi_{:,0} = chi0_{:,0}; returns [w, G]."""
    N = chi0w.shape[1]
    M = np.eye(N)[None, :, :] - chi0w * K[None, None, :]
    return solve_gauss(M, chi0w[:, :, 0].copy())


def dsf(chi00_int: np.ndarray, omega: np.ndarray, S0: float, T: float, n: float) -> np.ndarray:
    """S on the caller's grid from chi_00 at the internal frequencies (Eq. 8); S0 at w = 0."""
    beta = 1.0 / T
    S = np.zeros(len(omega))
    for j, w in enumerate(omega):
        if w == 0.0:
            S[j] = S0
        else:
            S[j] = -chi00_int[j].imag / (math.pi * n * (-math.expm1(-beta * w)))
    return S


def s_zero(dchi00_deta0: complex, T: float, n: float) -> float:
    """S(q,0) = (T/(pi n)) Re d chi_00/d eta at w = 0 (the w -> 0 limit of Eq. 8)."""
    return T * dchi00_deta0.real / (math.pi * n)


def positive_branch(S, omega, S0):
    """(w_j, S_j) over w >= 0 in ascending order, with w = 0 included (value S0 if the grid
    lacks it)."""
    w = np.asarray(omega)
    pos = w >= 0.0
    wp, Sp = w[pos], np.asarray(S)[pos]
    if len(wp) == 0 or wp[0] != 0.0:
        wp = np.concatenate([[0.0], wp])
        Sp = np.concatenate([[S0], Sp])
    return wp, Sp


def trapezoid_weights(x: np.ndarray) -> np.ndarray:
    w = np.zeros(len(x))
    if len(x) < 2:
        return w
    dx = np.diff(x)
    w[:-1] += 0.5 * dx
    w[1:] += 0.5 * dx
    return w


def itcf_fold(wp, Sp, tau, T) -> np.ndarray:
    """F(tau) = sum_j wt_j S_j [e^{-tau w_j} + e^{-(beta - tau) w_j}] (Eq. 1 + detailed balance)."""
    beta = 1.0 / T
    wt = trapezoid_weights(wp)
    tau = np.asarray(tau)
    ker = np.exp(-np.outer(tau, wp)) + np.exp(-np.outer(beta - tau, wp))
    return ker @ (wt * Sp)


def itcf_direct(omega, S, tau) -> np.ndarray:
    """F(tau) = trapezoid over the full grid of S(w) e^{-tau w} (Eq. 1, no folding)."""
    wt = trapezoid_weights(np.asarray(omega))
    return np.exp(-np.outer(np.asarray(tau), omega)) @ (wt * S)


def itcf_metrics(wp, Sp, T, n) -> np.ndarray:
    """[F(beta/2), int_0^beta F, Ftilde(beta/2), int_0^beta Ftilde, -n int_0^beta F]."""
    beta = 1.0 / T
    wt = trapezoid_weights(wp)
    Fhalf = float(itcf_fold(wp, Sp, [0.5 * beta], T)[0])
    F0 = float(itcf_fold(wp, Sp, [0.0], T)[0])
    tint = np.where(wp > 0.0, -2.0 * np.expm1(-beta * np.where(wp > 0, wp, 1.0)) / np.where(wp > 0, wp, 1.0),
                    2.0 * beta)
    Fint = float(np.sum(wt * Sp * tint))
    return np.array([Fhalf, Fint, Fhalf - F0, Fint - beta * F0, -n * Fint])


def tau_grid(T: float, ntau: int) -> np.ndarray:
    return np.linspace(0.0, 0.5 / T, ntau)
