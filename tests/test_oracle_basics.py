"""Pins of the oracle's building blocks: generator, lattice, occupations, xc kernel."""
import math

import numpy as np
import pytest

from conftest import golden
from oracle import crystal, lindhard, occupations, xc
from paper_2510_01875_gb300 import workloads as W


def test_splitmix64_reference_outputs():
    r = W.SplitMix64(0)
    assert [r.next_u64() for _ in range(3)] == [row[0] for row in golden("splitmix64_seed0.txt")]


def test_workloads_shapes():
    small, full, adj = W.al1_fcc_k8_b24(), W.al1_fcc_k12_b120(), W.al4_cubic_k6_b200()
    assert (small.nq, small.nw, small.nk, small.nbands, int(small.nG[0])) == (1, 256, 512, 24, 15)
    assert (full.nq, full.nw, full.nk, full.nbands, int(full.nG[0])) == (8, 1024, 1728, 120, 59)
    assert (adj.nq, adj.nw, adj.nk, adj.natoms) == (16, 2048, 216, 4)
    batched = W.al32_k4_b400()
    assert batched.natoms == 32 and batched.nq == 24 and 60 <= batched.nG.min() and batched.nG.max() <= 200
    qm = np.linalg.norm(batched.q, axis=1)
    assert np.all(np.abs(qm / W.inv_ang(1.5) - 1.0) <= 0.05 + 1e-12)
    ang = np.degrees(np.arccos(batched.q[:, 0] / qm))
    assert ang.max() <= 3.0 + 1e-9
    # the same seed gives the same cell
    assert np.array_equal(W.al32_k4_b400().positions, batched.positions)


def test_reciprocal_lattice():
    for lat in (W.fcc_primitive(W.AL_A), W.AL_A * np.eye(3), W.al32_k4_b400().lattice):
        B = crystal.reciprocal(lat)
        assert np.allclose(lat @ B.T, 2 * math.pi * np.eye(3), atol=1e-12)


def test_fcc_shell_closures():
    """|G| shells of the fcc primitive cell (a bcc reciprocal lattice): 1, 9, 15, 27, 51, 59,
    65, 89; of the simple cubic cell: 1, 7, 19, 27, 33, 57, 81, 93."""
    for lat, want in ((W.fcc_primitive(W.AL_A), [1, 9, 15, 27, 51, 59, 65, 89]),
                      (W.AL_A * np.eye(3), [1, 7, 19, 27, 33, 57, 81, 93])):
        B = crystal.reciprocal(lat)
        m = crystal._miller_candidates(lat, np.zeros(3), 6.0)
        g2 = np.round(np.einsum("ij,ij->i", m @ B, m @ B) / (B[0] @ B[0]) * 12).astype(int)
        vals = np.unique(g2)[:8]
        assert [int((g2 <= v).sum()) for v in vals] == want


def test_response_gset_order_and_zero_first():
    lat = W.fcc_primitive(W.AL_A)
    q = W.al1_fcc_k8_b24().q[0]
    gs = crystal.response_gset(lat, q, 15)
    assert len(gs) == 15 and not gs[0].any()
    B = crystal.reciprocal(lat)
    d = np.linalg.norm(q[None] + gs @ B, axis=1)
    # the set is the 15 smallest |q+G| (checked against all lattice vectors nearby)
    m = crystal._miller_candidates(lat, q, 6.0)
    allq = np.sort(np.linalg.norm(q[None] + m @ B, axis=1))
    assert d.max() <= allq[14] + 1e-9
    assert np.all(np.diff(d[1:]) >= -1e-9)


def test_hamiltonian_hermitian_and_free_limit():
    wl = W.tiny()
    k = np.array([0.1, -0.05, 0.2])
    b = crystal.sphere_basis(wl.lattice, k, wl.ecut)
    H = crystal.hamiltonian(wl.lattice, wl.positions, wl.Z, wl.r_c, k, b)
    assert np.allclose(H, H.conj().T, atol=1e-14)
    e0, _ = crystal.eigenstates(wl.lattice, wl.positions, wl.Z, wl.r_c, k, b, 6, potential="zero")
    kg = k[None] + b @ crystal.reciprocal(wl.lattice)
    assert np.allclose(e0, np.sort(0.5 * np.einsum("ij,ij->i", kg, kg))[:6], atol=1e-13)
    # the potential averages to zero: trace(H) equals the kinetic trace
    assert abs(np.trace(H).real - 0.5 * np.einsum("ij,ij->", kg, kg)) < 1e-10


def test_empty_core_form_factor():
    """v(G) of one ion at the origin is real, -(4 pi Z/(Omega G^2)) cos(G r_c); zero at G = 0."""
    lat = W.fcc_primitive(W.AL_A)
    m = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 1]])
    V = crystal.vion(lat, np.zeros((1, 3)), 3.0, 1.12, m)
    G = np.linalg.norm(m @ crystal.reciprocal(lat), axis=1)
    om = crystal.volume(lat)
    assert V[0] == 0
    assert np.allclose(V[1:], -(4 * math.pi * 3.0 / (om * G[1:] ** 2)) * np.cos(G[1:] * 1.12), rtol=1e-14)


def test_neutrality():
    rng = np.random.default_rng(3)
    eps = np.sort(rng.normal(0.0, 0.3, size=(27, 12)), axis=1)
    for T in (0.01, 0.1, 1.0):
        mu = occupations.chemical_potential(eps, T, 9.0, 27)
        assert abs(occupations.electron_count(eps, mu, T, 27) - 9.0) < 1e-13 * 9.0


def test_mu_matches_free_gas():
    """At zero potential on a dense mesh the discrete mu approaches the ideal-gas value."""
    lat = W.fcc_primitive(W.AL_A)
    T = W.ev(5.0)
    n = 3.0 / crystal.volume(lat)
    errs = []
    for nm in (4, 8, 12):
        kp = crystal.kmesh(lat, (nm, nm, nm), np.zeros(3))
        eps = np.array([lindhard.lowest_planewaves(lat, k, 12.0, 40)[1] for k in kp])
        errs.append(abs(occupations.chemical_potential(eps, T, 3.0, len(kp)) - lindhard.free_gas_mu(n, T)))
    assert errs[2] < errs[0] and errs[2] < 2e-3


def test_fx_closed_form():
    n = 0.02682
    h = 1e-4 * n
    f = lambda x: x * xc.eps_x(x)
    fd = (f(n + h) - 2 * f(n) + f(n - h)) / (h * h)
    assert abs(xc.fx_alda(n) - fd) < 1e-6 * abs(fd)
    assert abs(xc.fx_alda(n) + math.pi / xc.kf_of_n(n) ** 2) < 1e-15


def test_pw92_table_value():
    rs, e, tol = golden("pw92_correlation.txt")[0]
    assert abs(xc.eps_c(rs) - e) < tol


def test_pw92_derivatives_complex_step():
    for rs in (1.0, 2.073, 3.5):
        h = 1e-20
        cs = xc.eps_c(complex(rs, h)).imag / h
        e, e1, e2 = xc.eps_c_derivs(rs)
        assert abs(e - xc.eps_c(rs)) < 1e-16
        assert abs(e1 - cs) < 1e-13 * abs(cs)
        d = 1e-5
        e2fd = (xc.eps_c_derivs(rs + d)[1] - xc.eps_c_derivs(rs - d)[1]) / (2 * d)
        assert abs(e2 - e2fd) < 1e-7 * abs(e2fd)


def test_fc_against_numerical_second_derivative():
    n = 0.02682
    f = lambda x: x * xc.eps_c(xc.rs_of_n(x))
    for h in (2e-3 * n,):
        fd = (f(n + h) - 2 * f(n) + f(n - h)) / (h * h)
        assert abs(xc.fc_alda(n) - fd) < 1e-5 * abs(fd)


def test_fxc_model_reduces_to_alda():
    n = 0.02682
    assert xc.fxc_model(1.3, n, 1.0, 0.0, 0.0) == xc.fxc_alda(n)
    assert abs(xc.fxc_model(0.0, n, 2.0, 0.1, 0.05) - 2 * xc.fxc_alda(n)) < 1e-15
