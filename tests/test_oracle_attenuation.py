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
