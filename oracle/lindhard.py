"""Oracle pins: the free-electron-gas (Lindhard) response, independent of the eigensolver path.

Test infrastructure only (see oracle/__init__.py).

  discrete_lindhard: chi0_GG(q,w) at zero potential, summing directly over plane-wave states
      (2/(N_k Omega)) sum_{k,G1} [f(e_{k+G1}) - f(e_{k+q+G1+G})] / (w + e_{k+G1} - e_{k+q+G1+G} + i eta)
      with e_p = |p|^2/2 and G1 running over the plane waves among the lowest nbands at k
      whose partner k+q+G1+G is among the lowest nbands at k+q.
  discrete_lindhard_dw: its frequency derivative, the same sum of
      -[f(e_{k+G1}) - f(e_{k+q+G1+G})] / (w + e_{k+G1} - e_{k+q+G1+G} + i eta)^2.
  continuum_lindhard: the finite-temperature Lindhard function at z = w + i eta,
      chi0(q,z) = 1/(2 pi^2 q) int_0^inf dk k f(k^2/2) [ln(z - q^2/2 + kq) - ln(z - q^2/2 - kq)
                                                      - ln(z + q^2/2 + kq) + ln(z + q^2/2 - kq)]
      (principal logarithms; Im z > 0 keeps every argument off the branch cut).
  imag_lindhard_eta0: the eta -> 0 closed form of Im chi0,
      -(T/(2 pi q)) [ln(1 + e^{(mu-E1)/T}) - ln(1 + e^{(mu-E2)/T})], E_{1,2} = (w/q -+ q/2)^2 / 2.
  static_lindhard_t0: the T = 0 static limit -(k_F/pi^2)[1/2 + (1-x^2)/(4x) ln|(1+x)/(1-x)|],
      x = q/(2 k_F).
  free_gas_mu: mu of the ideal Fermi gas at density n and temperature T.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, optimize
from scipy.special import expit

from . import crystal


def free_gas_density(mu: float, T: float) -> float:
    """n = (1/pi^2) int_0^inf k^2 f(k^2/2) dk."""
    kmax = math.sqrt(2.0 * max(mu, 0.0) + 80.0 * T)
    pts = [math.sqrt(2.0 * mu)] if mu > 0 else None
    val, _ = integrate.quad(lambda k: k * k * expit(-(0.5 * k * k - mu) / T), 0.0, kmax,
                            epsabs=0.0, epsrel=1e-13, limit=400, points=pts)
    return val / math.pi ** 2


def free_gas_mu(n: float, T: float) -> float:
    kf = (3.0 * math.pi ** 2 * n) ** (1.0 / 3.0)
    ef = 0.5 * kf * kf
    return optimize.brentq(lambda m: free_gas_density(m, T) - n, ef - 50.0 * T - 10.0, ef + 5.0,
                           xtol=1e-15, rtol=1e-15, maxiter=400)


def continuum_lindhard(q: float, w: float, eta: float, mu: float, T: float) -> complex:
    z = complex(w, eta)
    hq = 0.5 * q * q

    def integrand(k, part):
        f = expit(-(0.5 * k * k - mu) / T)
        val = (np.log(z - hq + k * q) - np.log(z - hq - k * q)
               - np.log(z + hq + k * q) + np.log(z + hq - k * q))
        return k * f * (val.real if part == 0 else val.imag)

    kmax = math.sqrt(2.0 * max(mu, 0.0) + 80.0 * T)
    # the logarithms change branch where their real parts vanish; f steps near sqrt(2 mu)
    cand = [abs(w / q - 0.5 * q), abs(w / q + 0.5 * q)]
    if mu > 0:
        cand.append(math.sqrt(2.0 * mu))
    pts = sorted({x for x in cand if 0.0 < x < kmax})
    re, _ = integrate.quad(integrand, 0.0, kmax, args=(0,), epsabs=0.0, epsrel=1e-12, limit=2000,
                           points=pts or None)
    im, _ = integrate.quad(integrand, 0.0, kmax, args=(1,), epsabs=0.0, epsrel=1e-12, limit=2000,
                           points=pts or None)
    return complex(re, im) / (2.0 * math.pi ** 2 * q)


def imag_lindhard_eta0(q: float, w: float, mu: float, T: float) -> float:
    e1 = 0.5 * (w / q - 0.5 * q) ** 2
    e2 = 0.5 * (w / q + 0.5 * q) ** 2
    return -(T / (2.0 * math.pi * q)) * (np.logaddexp(0.0, (mu - e1) / T) - np.logaddexp(0.0, (mu - e2) / T))


def static_lindhard_t0(q: float, kf: float) -> float:
    x = q / (2.0 * kf)
    return -(kf / math.pi ** 2) * (0.5 + (1.0 - x * x) / (4.0 * x) * math.log(abs((1.0 + x) / (1.0 - x))))


def lowest_planewaves(lattice, k, ecut, nbands):
    """Miller indices and energies of the nbands lowest plane waves at k within the cutoff
    sphere; also the energy of the next one (to check that the cut does not split a shell)."""
    b = crystal.sphere_basis(lattice, k, ecut)
    B = crystal.reciprocal(lattice)
    kg = k[None, :] + b @ B
    e = 0.5 * np.einsum("ij,ij->i", kg, kg)
    order = np.argsort(e, kind="stable")
    nxt = e[order[nbands]] if len(order) > nbands else math.inf
    return b[order[:nbands]], e[order[:nbands]], nxt


def discrete_lindhard(lattice, kpts, kqpts, ecut, nbands, G, mu, T, freqs, eta, dw=False):
    """Zero-potential chi0_GG at the frequencies, by direct plane-wave enumeration (dw: its
    derivative with respect to w, term by term)."""
    om = crystal.volume(lattice)
    nk = len(kpts)
    out = np.zeros(len(freqs), dtype=np.complex128)
    for k, kq in zip(kpts, kqpts):
        m1, e1, _ = lowest_planewaves(lattice, k, ecut, nbands)
        m2, e2, _ = lowest_planewaves(lattice, kq, ecut, nbands)
        index2 = {tuple(x): i for i, x in enumerate(m2)}
        for a in range(len(m1)):
            j = index2.get(tuple(m1[a] + G))
            if j is None:
                continue
            f1 = expit(-(e1[a] - mu) / T)
            f2 = expit(-(e2[j] - mu) / T)
            den = freqs + e1[a] - e2[j] + 1j * eta
            out += -(f1 - f2) / den ** 2 if dw else (f1 - f2) / den
    return 2.0 * out / (nk * om)
