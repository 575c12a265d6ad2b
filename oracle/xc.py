"""Oracle: the static exchange-correlation kernel of the Dyson step.

Test infrastructure only (see oracle/__init__.py).

ALDA at the mean density n (zero temperature, spin-unpolarised):
f_xc = d^2 (n eps_xc(n)) / dn^2 with
  exchange (Slater):  n eps_x = -(3/4)(3/pi)^{1/3} n^{4/3}  ->  f_x = -pi / k_F^2,
  correlation (Perdew-Wang 1992, unpolarised parameters):
    eps_c(r_s) = -2A(1 + a1 r_s) ln(1 + 1/Q),
    Q = 2A(b1 r_s^{1/2} + b2 r_s + b3 r_s^{3/2} + b4 r_s^2),
  and with r_s = (3/(4 pi n))^{1/3}:  f_c = (r_s^2 eps_c'' - 2 r_s eps_c') / (9 n).
The paper's runs use an adiabatic GGA kernel (App. A.1); the kernel here is the
local-density one the response engine is specified with.

Static kernel model: f_xc(|q+G|) = A f_ALDA (1 + B |q+G|^2) exp(-C |q+G|^2).

Pinned by: f_x = -pi/k_F^2 against a finite-difference second derivative of n eps_x,
eps_c(r_s = 2) = -0.0448 Ha (PW92 table value), and complex-step derivatives of eps_c
(tests/test_oracle_basics.py).
"""
from __future__ import annotations

import math

PW92_A = 0.031091
PW92_ALPHA1 = 0.21370
PW92_BETA = (7.5957, 3.5876, 1.6382, 0.49294)


def rs_of_n(n: float) -> float:
    return (3.0 / (4.0 * math.pi * n)) ** (1.0 / 3.0)


def kf_of_n(n: float) -> float:
    return (3.0 * math.pi * math.pi * n) ** (1.0 / 3.0)


def eps_x(n):
    return -0.75 * (3.0 / math.pi) ** (1.0 / 3.0) * n ** (1.0 / 3.0)


def eps_c(rs):
    """PW92 correlation energy per electron; accepts complex rs (complex-step tests)."""
    A, a1 = PW92_A, PW92_ALPHA1
    b1, b2, b3, b4 = PW92_BETA
    Q = 2.0 * A * (b1 * rs ** 0.5 + b2 * rs + b3 * rs ** 1.5 + b4 * rs ** 2)
    import cmath
    log = cmath.log if isinstance(rs, complex) else math.log
    return -2.0 * A * (1.0 + a1 * rs) * log(1.0 + 1.0 / Q)


def eps_c_derivs(rs: float):
    """(eps_c, d eps_c/d rs, d^2 eps_c/d rs^2), analytic."""
    A, a1 = PW92_A, PW92_ALPHA1
    b1, b2, b3, b4 = PW92_BETA
    s = math.sqrt(rs)
    Q = 2.0 * A * (b1 * s + b2 * rs + b3 * rs * s + b4 * rs * rs)
    Q1 = 2.0 * A * (0.5 * b1 / s + b2 + 1.5 * b3 * s + 2.0 * b4 * rs)
    Q2 = 2.0 * A * (-0.25 * b1 / (rs * s) + 0.75 * b3 / s + 2.0 * b4)
    L = math.log(1.0 + 1.0 / Q)
    D = Q * Q + Q
    e = -2.0 * A * (1.0 + a1 * rs) * L
    e1 = -2.0 * A * a1 * L + 2.0 * A * (1.0 + a1 * rs) * Q1 / D
    e2 = (4.0 * A * a1 * Q1 / D
          + 2.0 * A * (1.0 + a1 * rs) * (Q2 / D - Q1 * Q1 * (2.0 * Q + 1.0) / (D * D)))
    return e, e1, e2


def fx_alda(n: float) -> float:
    kf = kf_of_n(n)
    return -math.pi / (kf * kf)


def fc_alda(n: float) -> float:
    rs = rs_of_n(n)
    _, e1, e2 = eps_c_derivs(rs)
    return (rs * rs * e2 - 2.0 * rs * e1) / (9.0 * n)


def fxc_alda(n: float) -> float:
    return fx_alda(n) + fc_alda(n)


def fxc_model(qg: float, n: float, A: float, B: float, C: float) -> float:
    return A * fxc_alda(n) * (1.0 + B * qg * qg) * math.exp(-C * qg * qg)
