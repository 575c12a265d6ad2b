"""Oracle: constraints-based attenuation of narrow-band fluctuations (Sec. 3).

Test infrastructure only (see oracle/__init__.py).

S_TDDFT = S_p + S_n and F_TDDFT = F_p + F_n (Sec. 3, Eqs. 3-4).  The steps, in the
paper's order:
 1. target frequencies: the power spectrum of dS/dw over a featureless range; the
    n_targets strongest local maxima (Sec. 3, the PSD figure), ignoring the lowest
    5 % of Fourier frequencies;
 2. a Savitzky-Golay filter (local least-squares polynomial of degree d over a window of
    m = 2 round(w / (2 dw)) + 1 samples, Savitzky & Golay 1964); at the edges the
    polynomial of the first / last full window is evaluated at the edge points;
 3. grid search over (d, w) scored by AICc = N ln(RSS/N) + 2k + 2k(k+1)/(N-k-1),
    k = trace of the smoother matrix, plus lambda_f * ln(max(R_f, r0) / r0) with R_f = (power
    of the filtered dS/dw kept in +-2 bins around the targets) / (the raw power there) and
    r0 = 1e-4, plus lambda_c * (sum of squared second differences of the filtered S / the
    same for the raw S); lambda_f = lambda_c = N unless given (the paper states neither
    the weights nor the form; the logarithm puts the frequency penalty on the scale of the
    N ln(RSS/N) term, so it can outweigh the fit gain of keeping a narrow band); the optimal window is chosen per degree; near ties (1e-9
    relative) go to the fewest sign changes of the filtered dS/dw (the minimal stationary
    point condition), then to the smaller window;
 4. constraints in imaginary time: F_n = Laplace transform of S - S_p (Eq. 5) with
    mean  Fbar_n = (1/beta) int_0^beta F_n dtau and RMS
    sigma_n = [(1/beta) int_0^beta (F_n - Fbar_n)^2 dtau]^{1/2} (Eq. 7 read with beta as
    the interval and the 1/beta inside the root); accepted if |Fbar_n| / F(beta/2) and
    sigma_n / F(beta/2) are below the thresholds (defaults 0.4 % and 0.0042 %, Sec. 3);
 5. S_p = mean over the accepted degrees of their filtered spectra (Sec. 4.1); if none
    passes, S_p = S and the report says so.

The filter acts on the uniformly spaced samples with w >= 0 of the caller's grid.

Pinned by (tests/test_oracle_attenuation.py): the SG filter (polynomial exactness, the
classic 5-point table, the hat diagonal of the edge rows against the explicit projection
V (V^T V)^{-1} V^T), the Hann periodogram against its closed form as a sum of geometric
series, the target bins of planted cosines (with the low-frequency exclusion), and AICc,
the trace of the smoother and the curvature ratio on a hand-worked 10-sample example.
The weights and the form of the score are readings (the paper states neither); given
those readings every ingredient of the selection is pinned.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import response


@dataclasses.dataclass
class AttenParams:
    d_min: int = 1
    d_max: int = 4
    w_min: float = 0.0          # window grid, Ha (0 -> 4 dw)
    w_max: float = 0.0          # (0 -> a quarter of the filtered range)
    n_w: int = 24
    lambda_f: float = -1.0      # < 0 -> N
    lambda_c: float = -1.0      # < 0 -> N
    n_targets: int = 2
    feat_lo: float = -1.0       # featureless range, Ha (< 0 -> central 90 % of the samples)
    feat_hi: float = -1.0
    low_exclude: float = 0.05
    accept_mean: float = 4e-3
    accept_rms: float = 4.2e-5
    average: bool = True
    retain_floor: float = 1e-4  # r0 of the frequency penalty


def window_points(w: float, dw: float) -> int:
    return 2 * int(math.floor(w / (2.0 * dw) + 0.5)) + 1


def sg_filter(y: np.ndarray, d: int, m: int):
    """Savitzky-Golay smoothing by a least-squares fit per window (QR of the window's
    Vandermonde matrix).  Returns (filtered y, diagonal of the smoother matrix)."""
    N = len(y)
    h = m // 2
    t = np.arange(-h, h + 1) / h
    V = np.vander(t, d + 1, increasing=True)
    Q, R = np.linalg.qr(V)
    out = np.empty(N)
    hat = np.empty(N)
    # interior windows: fit y[j-h .. j+h], evaluate at the centre (offset 0)
    for j in range(h, N - h):
        c = np.linalg.solve(R, Q.T @ y[j - h:j + h + 1])
        out[j] = c[0]
        hat[j] = float(Q[h] @ Q[h])
    # edges: the polynomial of the first / last full window at the edge points
    c0 = np.linalg.solve(R, Q.T @ y[:m])
    c1 = np.linalg.solve(R, Q.T @ y[N - m:])
    for j in range(h):
        out[j] = np.polyval(c0[::-1], t[j])
        hat[j] = float(Q[j] @ Q[j])
        jj = N - h + j
        out[jj] = np.polyval(c1[::-1], t[h + 1 + j])
        hat[jj] = float(Q[h + 1 + j] @ Q[h + 1 + j])
    return out, hat


def derivative(y: np.ndarray, dw: float, i0: int, i1: int) -> np.ndarray:
    """Central differences (y[j+1] - y[j-1]) / (2 dw) for j = i0..i1."""
    j = np.arange(i0, i1 + 1)
    return (y[j + 1] - y[j - 1]) / (2.0 * dw)


def periodogram(D: np.ndarray) -> np.ndarray:
    """|sum_j hann_j (D_j - mean D) e^{-2 pi i j k / L}|^2 for k = 0..L//2."""
    L = len(D)
    j = np.arange(L)
    hann = 0.5 - 0.5 * np.cos(2.0 * math.pi * j / (L - 1))
    x = hann * (D - D.mean())
    k = np.arange(L // 2 + 1)
    E = np.exp(-2j * math.pi * np.outer(k, j) / L)
    return np.abs(E @ x) ** 2


def targets(P: np.ndarray, n_targets: int, low_exclude: float):
    K = len(P) - 1
    kmin = max(1, int(math.ceil(low_exclude * K)))
    peaks = [k for k in range(kmin + 1, K) if P[k] > P[k - 1] and P[k] >= P[k + 1]]
    peaks.sort(key=lambda k: (-P[k], k))
    return sorted(peaks[:n_targets])


def target_bins(tg, K):
    bins = set()
    for k in tg:
        for b in range(k - 2, k + 3):
            if 0 <= b <= K:
                bins.add(b)
    return sorted(bins)


def aicc(rss: float, N: int, k: float) -> float:
    """Corrected Akaike criterion of a linear smoother: N ln(RSS/N) + 2k + 2k(k+1)/(N-k-1),
    k = trace of the smoother matrix (its effective number of parameters)."""
    return N * math.log(max(rss, 1e-300) / N) + 2.0 * k + 2.0 * k * (k + 1.0) / (N - k - 1.0)


def retention(P_raw: np.ndarray, P_filt: np.ndarray, bins) -> float:
    """R_f: power of the filtered dS/dw kept in the target bins / the raw power there."""
    raw = float(np.sum(P_raw[bins])) if len(bins) else 0.0
    return float(np.sum(P_filt[bins])) / raw if raw > 0 else 0.0


def curvature_ratio(yf: np.ndarray, y: np.ndarray) -> float:
    """sum of squared second differences of the filtered spectrum / the same of the raw one."""
    raw = float(np.sum(np.diff(y, 2) ** 2))
    return float(np.sum(np.diff(yf, 2) ** 2)) / raw if raw > 0 else 0.0


def sign_changes(D: np.ndarray) -> int:
    s = np.sign(D)
    s = s[s != 0]
    return int(np.sum(s[1:] != s[:-1]))


def laplace_fold(wp, Sp, tau, T):
    return response.itcf_fold(wp, Sp, tau, T)


def attenuate(omega, S, S0, T, ntau, p: AttenParams):
    """One q.  omega / S: the caller's grid and DSF; S0: S at w = 0 (used when 0 is not on
    the grid).  Returns (S_p on the caller's grid, report dict)."""
    omega = np.asarray(omega)
    S = np.asarray(S)
    sel = np.where(omega >= 0.0)[0]
    y = S[sel]
    N = len(y)
    dw = omega[sel[1]] - omega[sel[0]]
    # featureless range for the spectrum of dS/dw
    if p.feat_lo < 0.0 or p.feat_hi < 0.0:
        i0 = max(1, int(math.floor(0.05 * (N - 1))))
        i1 = min(N - 2, int(math.ceil(0.95 * (N - 1))))
    else:
        i0 = max(1, int(np.searchsorted(omega[sel], p.feat_lo)))
        i1 = min(N - 2, int(np.searchsorted(omega[sel], p.feat_hi, side="right")) - 1)
    D = derivative(y, dw, i0, i1)
    P = periodogram(D)
    K = len(P) - 1
    tg = targets(P, p.n_targets, p.low_exclude)
    bins = target_bins(tg, K)
    lf = N if p.lambda_f < 0 else p.lambda_f
    lc = N if p.lambda_c < 0 else p.lambda_c
    w_lo = p.w_min if p.w_min > 0 else 4.0 * dw
    w_hi = p.w_max if p.w_max > 0 else 0.25 * N * dw
    ms = sorted({window_points(w, dw) for w in np.linspace(w_lo, w_hi, p.n_w)})
    tau = response.tau_grid(T, ntau)
    beta = 1.0 / T
    wpos, Spos = response.positive_branch(S, omega, S0)
    off = len(wpos) - N                     # 1 when S0 was prepended
    Fref_half = float(laplace_fold(wpos, Spos, [0.5 * beta], T)[0])
    report = {"targets": tg, "degrees": []}
    accepted = []
    for d in range(p.d_min, p.d_max + 1):
        best = None
        for m in ms:
            if m < d + 2 or m > N:
                continue
            yf, hat = sg_filter(y, d, m)
            rss = float(np.sum((yf - y) ** 2))
            k = float(np.sum(hat))
            if N - k - 1.0 <= 0.0:
                continue
            Df = derivative(yf, dw, i0, i1)
            rf = retention(P, periodogram(Df), bins)
            fpen = math.log(max(rf, p.retain_floor) / p.retain_floor)
            score = aicc(rss, N, k) + lf * fpen + lc * curvature_ratio(yf, y)
            cand = (score, sign_changes(Df), m, yf)
            if best is None:
                best = cand
            else:
                tie = abs(score - best[0]) <= 1e-9 * abs(best[0])
                if (not tie and score < best[0]) or (tie and (cand[1], m) < (best[1], best[2])):
                    best = cand
        if best is None:
            continue
        score, _, m, yf = best
        Sn = np.zeros(len(wpos))
        Sn[off:] = y - yf
        Fn = laplace_fold(wpos, Sn, tau, T)
        wt = response.trapezoid_weights(tau)
        Fbar = float(np.sum(wt * Fn)) * 2.0 / beta
        sig = math.sqrt(max(float(np.sum(wt * (Fn - Fbar) ** 2)) * 2.0 / beta, 0.0))
        rm, rs = abs(Fbar) / Fref_half, sig / Fref_half
        ok = rm <= p.accept_mean and rs <= p.accept_rms
        report["degrees"].append({"d": d, "m": m, "score": score, "mean_ratio": rm,
                                  "rms_ratio": rs, "accepted": ok})
        if ok:
            accepted.append((score, d, yf))
    Sp = S.copy()
    if accepted:
        if p.average:
            Sp[sel] = np.mean([a[2] for a in accepted], axis=0)
        else:
            Sp[sel] = min(accepted, key=lambda a: (a[0], a[1]))[2]
    report["n_accepted"] = len(accepted)
    return Sp, report
