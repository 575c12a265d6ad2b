"""Seeded synthetic workloads: empty-core aluminium cells shaped like the
warm-dense-matter systems of Sec. 4 (Al, Sec. 4.2 and App. A.1).

This module is the only code shared by the CUDA path and the oracle.  It
builds inputs only: lattice vectors, seeded ion positions, q vectors, the
frequency grid and the run parameters.  It holds none of the response
method's arithmetic (no basis sets, no Hamiltonians, no occupations, no
response functions).

Units are Hartree atomic units throughout (energies in Ha, lengths in bohr,
wave vectors in 1/bohr).  Random numbers come from a SplitMix64 counter
generator (Steele, Lea and Flood, 2014) with Box-Muller normals, so the same
seed gives the same cell on every machine.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Tuple

import numpy as np

HA_EV = 27.211386245988          # 1 Ha in eV (CODATA 2018)
BOHR_ANG = 0.529177210903        # 1 bohr in Angstrom (CODATA 2018)
SEED_BASE = 2510018750           # workload seed = SEED_BASE + workload index

AL_A = 7.65                      # fcc Al lattice constant, bohr (4.05 A, App. A.1)
AL_Z = 3.0                       # valence charge of the empty-core ion
AL_RC = 1.12                     # Ashcroft empty-core radius, bohr


def ev(x):
    """Electron-volts to Hartree."""
    return x / HA_EV


def inv_ang(x):
    """1/Angstrom to 1/bohr."""
    return x * BOHR_ANG


class SplitMix64:
    """SplitMix64 counter generator; uniform doubles in [0,1) from the top
    53 bits; normals by the Box-Muller transform."""

    MASK = (1 << 64) - 1

    def __init__(self, seed: int):
        self.state = seed & self.MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & self.MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & self.MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & self.MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def normal(self) -> float:
        u1 = self.uniform()
        while u1 <= 0.0:
            u1 = self.uniform()
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


def fcc_primitive(a: float) -> np.ndarray:
    """Rows are the primitive vectors of the fcc lattice."""
    return 0.5 * a * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]])


FCC_BASIS_FRAC = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])


def supercell(lattice: np.ndarray, basis_cart: np.ndarray, n: Tuple[int, int, int]):
    """Repeat a cell n[0] x n[1] x n[2] times; returns (lattice, positions)."""
    pos = []
    for i in range(n[0]):
        for j in range(n[1]):
            for k in range(n[2]):
                shift = i * lattice[0] + j * lattice[1] + k * lattice[2]
                for b in basis_cart:
                    pos.append(b + shift)
    big = np.array([n[0] * lattice[0], n[1] * lattice[1], n[2] * lattice[2]])
    return big, np.array(pos)


def displace(positions: np.ndarray, sigma: float, rng: SplitMix64) -> np.ndarray:
    """i.i.d. Gaussian displacements N(0, sigma^2) per Cartesian component."""
    out = positions.copy()
    for a in range(out.shape[0]):
        for c in range(3):
            out[a, c] += sigma * rng.normal()
    return out


def detector_cone(nq: int, qmag: float, rel_spread: float, half_angle_deg: float,
                  rng: SplitMix64) -> np.ndarray:
    """q vectors in a cone about x: |q| uniform in qmag*(1 +- rel_spread),
    polar angle uniform in [0, half_angle], azimuth uniform in [0, 2 pi)."""
    out = np.zeros((nq, 3))
    for i in range(nq):
        m = qmag * (1.0 + rel_spread * (2.0 * rng.uniform() - 1.0))
        th = math.radians(half_angle_deg) * rng.uniform()
        ph = 2.0 * math.pi * rng.uniform()
        out[i] = m * np.array([math.cos(th), math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph)])
    return out


@dataclasses.dataclass
class Workload:
    """One response calculation: cell, k-mesh, bands, q list and grids."""
    name: str
    lattice: np.ndarray            # (3,3) rows = lattice vectors, bohr
    positions: np.ndarray          # (natoms,3) Cartesian, bohr
    Z: float                       # ionic valence
    r_c: float                     # empty-core radius, bohr
    potential: str                 # "empty_core" or "zero"
    ecut: float                    # plane-wave cutoff 1/2|k+G|^2 <= ecut, Ha
    kmesh: Tuple[int, int, int]
    kscheme: str                   # "commensurate" or "tr_symmetric"
    nbands: int
    T: float                       # electron temperature, Ha
    eta: float                     # Lorentzian broadening, Ha
    q: np.ndarray                  # (nq,3) Cartesian, 1/bohr
    nG: np.ndarray                 # (nq,) response G-vectors per q
    omega: np.ndarray              # (nw,) real frequencies, Ha
    kernel: str = "rpa_alda"       # "rpa", "rpa_alda" or "fxc_model"
    fxc_params: Tuple[float, float, float] = (1.0, 0.0, 0.0)   # A, B, C of the f_xc(q) model
    ntau: int = 64
    basis: str = "sphere"          # "sphere" (per k) or "fixed" (1/2|G|^2 <= ecut, shared)
    occupations: Optional[np.ndarray] = None   # optional override, not used by the standard set

    @property
    def nq(self) -> int:
        return self.q.shape[0]

    @property
    def nw(self) -> int:
        return self.omega.shape[0]

    @property
    def nk(self) -> int:
        return int(np.prod(self.kmesh))

    @property
    def natoms(self) -> int:
        return self.positions.shape[0]

    def replace(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


def al1_fcc_k8_b24(zero_potential: bool = False) -> Workload:
    """fcc Al primitive cell, 8^3 Gamma mesh, 24 bands, T = 1 eV, one q = (0.5,0,0) 2pi/a
    (commensurate: (0,1/4,1/4) in reduced coordinates), 15 G, 256 omega on [0,60] eV."""
    a = AL_A
    return Workload(
        name="al1_fcc_k8_b24_q1_g15_w256" + ("_v0" if zero_potential else ""),
        lattice=fcc_primitive(a), positions=np.zeros((1, 3)), Z=AL_Z, r_c=AL_RC,
        potential="zero" if zero_potential else "empty_core", ecut=8.0,
        kmesh=(8, 8, 8), kscheme="commensurate", nbands=24, T=ev(1.0), eta=ev(0.2),
        q=np.array([[0.5 * 2.0 * math.pi / a, 0.0, 0.0]]), nG=np.array([15]),
        omega=np.linspace(0.0, ev(60.0), 256), kernel="rpa_alda")


def al1_fcc_k12_b120() -> Workload:
    """Same Al cell at T = 10 eV: 12^3 mesh, 120 bands (16 Ha cutoff), 59 G, 1024 omega on
    [-40,120] eV, eta = 0.5 eV, 8 q with |q| in [0.5,2.5] 1/A along x."""
    a = AL_A
    qs = np.array([[inv_ang(x), 0.0, 0.0] for x in np.linspace(0.5, 2.5, 8)])
    return Workload(
        name="al1_fcc_k12_b120_q8_g59_w1024",
        lattice=fcc_primitive(a), positions=np.zeros((1, 3)), Z=AL_Z, r_c=AL_RC,
        potential="empty_core", ecut=16.0, kmesh=(12, 12, 12), kscheme="tr_symmetric",
        nbands=120, T=ev(10.0), eta=ev(0.5), q=qs, nG=np.full(8, 59),
        omega=np.linspace(ev(-40.0), ev(120.0), 1024), kernel="rpa_alda")


def al32_k4_b400() -> Workload:
    """32-atom fcc supercell (2x2x2 conventional) with sigma = 0.15 bohr displacements,
    T = 5 eV, 4^3 mesh, 400 bands, 24 detector-cone q (|q| = 1.5 1/A +- 5 %, 3 degrees),
    N_G per q seeded-uniform in [60,200], 2048 omega on [-50,150] eV, eta = 0.3 eV."""
    rng = SplitMix64(SEED_BASE + 2)
    a = AL_A
    lat, pos = supercell(a * np.eye(3), FCC_BASIS_FRAC * a, (2, 2, 2))
    pos = displace(pos, 0.15, rng)
    qs = detector_cone(24, inv_ang(1.5), 0.05, 3.0, rng)
    nG = np.array([60 + int(rng.uniform() * 141) for _ in range(24)])
    return Workload(
        name="al32_k4_b400_q24_g60-200_w2048", lattice=lat, positions=pos, Z=AL_Z, r_c=AL_RC,
        potential="empty_core", ecut=8.0, kmesh=(4, 4, 4), kscheme="tr_symmetric",
        nbands=400, T=ev(5.0), eta=ev(0.3), q=qs, nG=nG,
        omega=np.linspace(ev(-50.0), ev(150.0), 2048), kernel="rpa_alda")


def al4_cubic_k6_b200() -> Workload:
    """4-atom conventional cubic Al cell, T = 20 eV, 6^3 mesh, 200 bands, 89 G, 16 q with
    |q| in [0.5,3] 1/A along x, 2048 omega on [-100,300] eV, eta = 0.5 eV,
    static f_xc(q) = A f_ALDA (1 + B q^2) exp(-C q^2) with (A,B,C) = (1, 0.1, 0.05)."""
    a = AL_A
    qs = np.array([[inv_ang(x), 0.0, 0.0] for x in np.linspace(0.5, 3.0, 16)])
    return Workload(
        name="al4_cubic_k6_b200_q16_g89_w2048", lattice=a * np.eye(3),
        positions=FCC_BASIS_FRAC * a, Z=AL_Z, r_c=AL_RC, potential="empty_core", ecut=8.0,
        kmesh=(6, 6, 6), kscheme="tr_symmetric", nbands=200, T=ev(20.0), eta=ev(0.5), q=qs,
        nG=np.full(16, 89), omega=np.linspace(ev(-100.0), ev(300.0), 2048),
        kernel="fxc_model", fxc_params=(1.0, 0.1, 0.05))


def al64_k2_b1600() -> Workload:
    """64-atom 4x4x4 primitive fcc supercell, sigma = 0.25 bohr, T = 50 eV, 2^3 mesh,
    1600 bands, 300 G, 48 detector-cone q, 4096 omega on [-200,600] eV, eta = 0.5 eV."""
    rng = SplitMix64(SEED_BASE + 4)
    a = AL_A
    lat, pos = supercell(fcc_primitive(a), np.zeros((1, 3)), (4, 4, 4))
    pos = displace(pos, 0.25, rng)
    qs = detector_cone(48, inv_ang(1.5), 0.05, 3.0, rng)
    return Workload(
        name="al64_k2_b1600_q48_g300_w4096", lattice=lat, positions=pos, Z=AL_Z, r_c=AL_RC,
        potential="empty_core", ecut=8.0, kmesh=(2, 2, 2), kscheme="tr_symmetric",
        nbands=1600, T=ev(50.0), eta=ev(0.5), q=qs, nG=np.full(48, 300),
        omega=np.linspace(ev(-200.0), ev(600.0), 4096), kernel="rpa_alda")


ALL = (al1_fcc_k8_b24, al1_fcc_k12_b120, al32_k4_b400, al4_cubic_k6_b200, al64_k2_b1600)


def tiny(seed: int = 7, nq: int = 2, kscheme: str = "tr_symmetric", potential: str = "empty_core",
         kernel: str = "rpa_alda", nbands: int = 8, ecut: float = 2.0, kmesh=(2, 2, 2),
         nw: int = 40, nG: int = 7, basis: str = "sphere", T_ev: float = 5.0,
         eta_ev: float = 0.5, wmin_ev: float = -30.0, wmax_ev: float = 60.0,
         natoms_displaced: bool = True) -> Workload:
    """A small seeded cell for tests: the fcc primitive Al cell, optionally with a
    displaced second atom (a 2-atom simple-cubic-like basis), few bands and a coarse mesh."""
    rng = SplitMix64(SEED_BASE + 1000 + seed)
    a = AL_A
    lat = fcc_primitive(a)
    pos = np.zeros((1, 3))
    if natoms_displaced:
        lat = a * np.eye(3)
        pos = displace(np.array([[0.0, 0.0, 0.0], [0.5 * a, 0.5 * a, 0.0]]), 0.2, rng)
    qs = []
    for i in range(nq):
        m = inv_ang(0.6 + 0.5 * i)
        th = 0.3 * rng.uniform()
        ph = 2.0 * math.pi * rng.uniform()
        qs.append(m * np.array([math.cos(th), math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph)]))
    return Workload(
        name=f"tiny{seed}", lattice=lat, positions=pos, Z=AL_Z, r_c=AL_RC, potential=potential,
        ecut=ecut, kmesh=tuple(kmesh), kscheme=kscheme, nbands=nbands, T=ev(T_ev), eta=ev(eta_ev),
        q=np.array(qs), nG=np.full(nq, nG), omega=np.linspace(ev(wmin_ev), ev(wmax_ev), nw),
        kernel=kernel, fxc_params=(1.0, 0.1, 0.05), basis=basis)
