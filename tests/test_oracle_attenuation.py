"""Pins of the oracle's Savitzky-Golay / AICc / constraints filter (Sec. 3)."""
import math

import numpy as np

from conftest import golden
from oracle import attenuation as A
from oracle import response


def test_sg_classic_table():
    for row in golden("savitzky_golay_quadratic.txt"):
        m = int(row[0])
        w = np.array(row[1:1 + m]) / row[1 + m]
        N = 4 * m
        for d in (2, 3):
            imp = np.zeros(N)
            imp[N // 2] = 1.0
            out, hat = A.sg_filter(imp, d, m)
            # response to a unit impulse = the (symmetric) smoothing weights
            got = out[N // 2 - m // 2:N // 2 + m // 2 + 1]
            assert np.abs(got - w[::-1]).max() < 1e-14
            assert abs(hat[N // 2] - w[m // 2]) < 1e-14


def test_sg_reproduces_polynomials():
    rng = np.random.default_rng(1)
    x = np.linspace(-1.0, 2.0, 61)
    for d in (1, 2, 3, 4):
        c = rng.normal(size=d + 1)
        y = np.polyval(c, x)
        for m in (d + 3 if (d + 3) % 2 else d + 4, 11, 21):
            out, _ = A.sg_filter(y, d, m)
            assert np.abs(out - y).max() < 1e-11 * np.abs(y).max()


def test_window_points_rule():
    assert A.window_points(3.65, 0.1) == 37
    assert A.window_points(1.0, 0.25) == 5
    assert A.window_points(0.1, 0.25) == 1


def _ringing_spectrum(nu=3.1, amp=0.02, N=801):
    """A smooth plasmon-like S plus a narrow-band oscillation of period 1/nu (in Ha)."""
    w = np.linspace(0.0, 4.0, N)
    Sp = w * np.exp(-((w - 1.2) ** 2) / 0.3) + 0.05 * w * np.exp(-w)
    Sn = amp * np.sin(2 * math.pi * nu * w / 0.05 * 0.05 * 8) * np.exp(-w / 3) * (w > 0.2)
    return w, Sp, Sn


def test_attenuation_removes_narrow_band_ringing():
    w, Sp, Sn = _ringing_spectrum()
    S = Sp + Sn
    T = 0.5
    p = A.AttenParams(accept_mean=1.0, accept_rms=1.0)
    out, rep = A.attenuate(w, S, S[0], T, 64, p)
    assert rep["n_accepted"] >= 1
    # the target is the injected oscillation: frequency index ~ (cycles over the range)
    D = A.derivative(S, w[1] - w[0], 40, 760)
    P = A.periodogram(D)
    assert P[rep["targets"]].max() == P[int(np.argmax(P[5:])) + 5]
    # the narrow band is attenuated: <1 % of its derivative power survives, and the output is
    # closer to the smooth part than the input everywhere the ringing lives
    Dout = A.derivative(out, w[1] - w[0], 40, 760)
    Pout = A.periodogram(Dout)
    t = rep["targets"][0]
    assert Pout[t - 2:t + 3].sum() < 1e-2 * P[t - 2:t + 3].sum()
    assert np.abs(out - Sp).max() < 0.5 * np.abs(S - Sp).max()


def test_attenuation_constraints_report():
    w, Sp, Sn = _ringing_spectrum(amp=0.005)
    S = Sp + Sn
    T = 0.5
    out, rep = A.attenuate(w, S, S[0], T, 64, A.AttenParams())
    for d in rep["degrees"]:
        # recompute the constraint ratios from their definitions (Eqs. 5 and 7)
        yf, _ = A.sg_filter(S, d["d"], d["m"])
        tau = response.tau_grid(T, 64)
        Fn = response.itcf_fold(w, S - yf, tau, T)
        Fref = response.itcf_fold(w, S, [1 / (2 * T)], T)[0]
        beta = 1 / T
        Fbar = np.trapezoid(Fn, tau) * 2 / beta
        sig = math.sqrt(np.trapezoid((Fn - Fbar) ** 2, tau) * 2 / beta)
        assert abs(d["mean_ratio"] - abs(Fbar) / Fref) < 1e-12
        assert abs(d["rms_ratio"] - sig / Fref) < 1e-12
        assert d["accepted"] == (d["mean_ratio"] <= 4e-3 and d["rms_ratio"] <= 4.2e-5)


def _geometric(alpha, L):
    """sum_{j=0}^{L-1} e^{i alpha j} in closed form."""
    z = np.exp(1j * alpha)
    if abs(z - 1.0) < 1e-14:
        return complex(L)
    return (1.0 - z ** L) / (1.0 - z)


def test_periodogram_of_a_cosine_matches_its_closed_form():
    """Hann window h_j = 1/2 - 1/2 cos(2 pi j/(L-1)) times cos(2 pi k0 j/L): its DFT is a sum of
    six geometric series, so |X_k|^2 follows in closed form at every bin (a wrong window, a
    shifted bin index or a missing factor would not)."""
    for L, k0 in ((64, 9), (101, 17), (200, 41)):
        j = np.arange(L)
        D = np.cos(2 * math.pi * k0 * j / L)
        P = A.periodogram(D)
        b, g = 2 * math.pi / (L - 1), 2 * math.pi * k0 / L
        for k in range(L // 2 + 1):
            t = 2 * math.pi * k / L
            X = 0.25 * (_geometric(g - t, L) + _geometric(-g - t, L))
            X -= 0.125 * sum(_geometric(s1 * b + s2 * g - t, L) for s1 in (1, -1) for s2 in (1, -1))
            assert abs(P[k] - abs(X) ** 2) < 1e-9 * P.max(), (L, k0, k)
        # the peak sits at k0 and carries (L/4)^2 to the order of the window's 1/L asymmetry
        assert int(np.argmax(P)) == k0
        assert abs(P[k0] / (L / 4) ** 2 - 1) < 4.0 / L


def test_targets_are_the_planted_cosines_above_the_low_exclusion():
    L = 240
    j = np.arange(L)
    D = (3.0 * np.cos(2 * math.pi * 4 * j / L) + 1.0 * np.cos(2 * math.pi * 29 * j / L)
         + 0.6 * np.cos(2 * math.pi * 71 * j / L) + 0.2 * np.cos(2 * math.pi * 95 * j / L))
    P = A.periodogram(D)
    # bins below ceil(0.05 * 120) = 6 are ignored: the strongest cosine (bin 4) is not a target
    assert A.targets(P, 2, 0.05) == [29, 71]
    assert A.targets(P, 1, 0.05) == [29]
    assert A.targets(P, 3, 0.05) == [29, 71, 95]
    assert A.targets(P, 2, 0.0) == [4, 29]
    assert A.target_bins([29, 71], 120) == [27, 28, 29, 30, 31, 69, 70, 71, 72, 73]
    assert A.target_bins([1], 120) == [0, 1, 2, 3]


def test_retention_is_the_kept_power_ratio():
    rng = np.random.default_rng(3)
    D = rng.normal(size=90)
    P = A.periodogram(D)
    bins = A.target_bins(A.targets(P, 2, 0.05), len(P) - 1)
    assert abs(A.retention(P, A.periodogram(0.3 * D), bins) - 0.09) < 1e-14
    assert A.retention(P, A.periodogram(np.zeros(90)), bins) == 0.0


def test_hat_diagonal_equals_the_explicit_projection():
    """The smoother's diagonal: interior and edge rows are v_j^T (V^T V)^{-1} v_j of the
    window's Vandermonde matrix V (normal equations by an explicit inverse, not QR)."""
    N = 40
    for d, m in ((1, 3), (2, 7), (3, 9), (4, 15)):
        h = m // 2
        t = np.arange(-h, h + 1) / h
        V = np.vander(t, d + 1, increasing=True)
        Hm = V @ np.linalg.inv(V.T @ V) @ V.T
        _, hat = A.sg_filter(np.zeros(N), d, m)
        for jj in range(h):
            assert abs(hat[jj] - Hm[jj, jj]) < 1e-13
            assert abs(hat[N - h + jj] - Hm[h + 1 + jj, h + 1 + jj]) < 1e-13
        assert np.abs(hat[h:N - h] - Hm[h, h]).max() < 1e-13


def test_aicc_and_penalties_on_a_hand_worked_example():
    """y_j = j^2, j = 0..9, linear SG over 3 points.  Worked by hand: interior outputs are the
    3-point means j^2 + 2/3; the edge lines through (0, 1, 4) and (49, 64, 81) give -1/3 and
    242/3 at the ends.  Residuals 2/3 (8 interior points) and -1/3 (two edges): RSS = 34/9.
    Hat diagonal 1/3 inside and 5/6 at the edges (V^T V = diag(3, 2)): k = 13/3.  Second
    differences: 2 everywhere for y (sum of squares 32), 1, 2 x 6, 1 for the filtered y (26)."""
    y = np.arange(10.0) ** 2
    yf, hat = A.sg_filter(y, 1, 3)
    want = np.array([-1 / 3] + [j * j + 2 / 3 for j in range(1, 9)] + [242 / 3])
    assert np.abs(yf - want).max() < 1e-12
    assert abs(hat[0] - 5 / 6) < 1e-15 and abs(hat[9] - 5 / 6) < 1e-15
    assert np.abs(hat[1:9] - 1 / 3).max() < 1e-15
    rss = float(np.sum((yf - y) ** 2))
    k = float(np.sum(hat))
    assert abs(rss - 34 / 9) < 1e-12 and abs(k - 13 / 3) < 1e-14
    # N ln(RSS/N) + 2k + 2k(k+1)/(N-k-1) = 10 ln(17/45) + 26/3 + 208/21
    assert abs(A.aicc(rss, 10, k) - (10 * math.log(17 / 45) + 26 / 3 + 208 / 21)) < 1e-12
    assert abs(A.curvature_ratio(yf, y) - 13 / 16) < 1e-14


def test_reported_score_is_the_sum_of_its_parts():
    """A one-window, one-degree search: the reported score is AICc + lambda_f ln(max(R_f, r0)/r0)
    + lambda_c x curvature ratio, each part recomputed from its definition."""
    w, Sp, Sn = _ringing_spectrum(amp=0.01, N=401)
    S = Sp + Sn
    dw = w[1] - w[0]
    p = A.AttenParams(d_min=2, d_max=2, w_min=20 * dw, w_max=20 * dw, n_w=1, lambda_f=7.0,
                      lambda_c=3.0)
    _, rep = A.attenuate(w, S, S[0], 0.5, 64, p)
    d = rep["degrees"][0]
    assert d["d"] == 2 and d["m"] == 21
    N = len(w)
    yf, hat = A.sg_filter(S, 2, 21)
    i0, i1 = int(math.floor(0.05 * (N - 1))), int(math.ceil(0.95 * (N - 1)))
    P = A.periodogram(A.derivative(S, dw, i0, i1))
    bins = A.target_bins(A.targets(P, 2, 0.05), len(P) - 1)
    rf = A.retention(P, A.periodogram(A.derivative(yf, dw, i0, i1)), bins)
    want = (A.aicc(float(np.sum((yf - S) ** 2)), N, float(np.sum(hat)))
            + 7.0 * math.log(max(rf, 1e-4) / 1e-4) + 3.0 * A.curvature_ratio(yf, S))
    assert abs(d["score"] - want) < 1e-12 * abs(want)
