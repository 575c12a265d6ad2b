"""Pins of the oracle's response path against closed forms, sum rules, symmetries and an
independent brute-force construction."""
import math

import numpy as np
import pytest

from oracle import crystal, lindhard, occupations, pipeline, response
from paper_2510_01875_gb300 import workloads as W


def _free_tiny(nbands=None):
    """Zero-potential fcc cell on a time-reversal-symmetric 3^3 mesh; nbands chosen so that
    the band cut never splits a degenerate plane-wave shell."""
    wl = W.tiny(potential="zero", natoms_displaced=False, kmesh=(3, 3, 3), ecut=3.0, nq=1, nG=9,
                nw=25, T_ev=3.0)
    kp, kqp = crystal.pair_meshes(wl.lattice, wl.kmesh, wl.q[0], wl.kscheme)
    for nb in range(14, 5, -1):
        ok = True
        for k in list(kp) + list(kqp):
            _, e, nxt = lindhard.lowest_planewaves(wl.lattice, k, wl.ecut, nb)
            if nxt - e[-1] < 1e-6:
                ok = False
                break
        if ok:
            return wl.replace(nbands=nb)
    raise RuntimeError("no clean band cut")


def test_chi0_zero_potential_equals_discrete_lindhard():
    wl = _free_tiny()
    r = pipeline.run_q(wl, 0, keep_chi0=True)
    chi0 = r["chi0"]
    kp, kqp = crystal.pair_meshes(wl.lattice, wl.kmesh, wl.q[0], wl.kscheme)
    scale = np.abs(chi0).max()
    for ig, G in enumerate(r["gset"]):
        ref = lindhard.discrete_lindhard(wl.lattice, kp, kqp, wl.ecut, wl.nbands, G, r["mu"], wl.T,
                                         r["freqs"], wl.eta)
        assert np.abs(chi0[:, ig, ig] - ref).max() < 1e-12 * scale
    off = chi0.copy()
    for ig in range(len(r["gset"])):
        off[:, ig, ig] = 0
    assert np.abs(off).max() < 1e-12 * scale


def test_s_zero_at_zero_potential_is_the_lindhard_derivative():
    """At V = 0, chi0 is diagonal (the discrete Lindhard sum L_G), so chi_00 = L_0/(1 - L_0 K_0)
    and d chi_00/dw = L_0'/(1 - L_0 K_0)^2 with L_0' the term-by-term w-derivative of the
    plane-wave sum: S(q,0) = -(T/(pi n)) Im d chi_00/dw at w = 0 (the limit of Eq. 8)."""
    wl = _free_tiny()
    r = pipeline.run_q(wl, 0)
    kp, kqp = crystal.pair_meshes(wl.lattice, wl.kmesh, wl.q[0], wl.kscheme)
    z = np.zeros(3, dtype=int)
    L = lindhard.discrete_lindhard(wl.lattice, kp, kqp, wl.ecut, wl.nbands, z, r["mu"], wl.T,
                                   np.array([0.0]), wl.eta)[0]
    dL = lindhard.discrete_lindhard(wl.lattice, kp, kqp, wl.ecut, wl.nbands, z, r["mu"], wl.T,
                                    np.array([0.0]), wl.eta, dw=True)[0]
    K0 = r["K"][0]
    n = response.density(wl)
    ref = -(wl.T / (math.pi * n)) * (dL / (1.0 - L * K0) ** 2).imag
    assert abs(r["S0"] - ref) < 1e-12 * abs(ref)
    assert abs(r["chi00"][r["hcol"]].imag) < 1e-13 * abs(r["chi00"][r["hcol"]])


@pytest.mark.parametrize("wmin_ev", [-30.0, 0.0])
def test_s_zero_is_the_limit_of_s(wmin_ev):
    """S(q,0) against the w -> 0 limit of Eq. 8 taken numerically: Im chi_00 is odd in w, so
    Im chi_00(h)/h = a + b h^2 + ..., and the Richardson combination (4 g(h) - g(2h))/3 of
    g(h) = Im chi_00(h)/h leaves O((h/eta)^4) (4e-10 here at h = 1e-4 Ha; it falls 16x per halving
    of h down to the rounding floor near 5e-11).  Covers 0 on and off the caller's grid."""
    wl = _db_workload().replace(omega=np.linspace(W.ev(wmin_ev), W.ev(40.0), 33))
    r = pipeline.run_q(wl, 0)
    h = 1e-4
    probe = pipeline.run_q(wl.replace(omega=np.array([h, 2 * h])), 0)
    g1, g2 = probe["chi00"][0].imag / h, probe["chi00"][1].imag / (2 * h)
    n = response.density(wl)
    ref = -(wl.T / (math.pi * n)) * (4 * g1 - g2) / 3
    assert abs(r["S0"] - ref) < 2e-9 * abs(ref)
    assert r["S0"] > 0


def test_discrete_lindhard_converges_to_continuum():
    lat = W.fcc_primitive(W.AL_A)
    T, eta = W.ev(5.0), W.ev(0.5)
    n = 3.0 / crystal.volume(lat)
    mu = lindhard.free_gas_mu(n, T)
    q = np.array([W.inv_ang(0.9), 0.0, 0.0])
    freqs = np.array([W.ev(5.0), W.ev(15.0), W.ev(25.0)])
    ref = np.array([lindhard.continuum_lindhard(np.linalg.norm(q), w, eta, mu, T) for w in freqs])
    errs = []
    for nm in (4, 8, 14):
        kp, kqp = crystal.pair_meshes(lat, (nm, nm, nm), q, "tr_symmetric")
        d = lindhard.discrete_lindhard(lat, kp, kqp, 8.0, 24, np.zeros(3, dtype=int), mu, T, freqs, eta)
        errs.append(np.abs(d - ref).max() / np.abs(ref).max())
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.03


def test_continuum_lindhard_limits():
    n = 0.02682
    kf = (3 * math.pi ** 2 * n) ** (1 / 3)
    T = W.ev(2.0)
    mu = lindhard.free_gas_mu(n, T)
    q = 0.8
    for w in (0.2, 0.5, 0.9):
        c = lindhard.continuum_lindhard(q, w, 1e-6, mu, T)
        assert abs(c.imag - lindhard.imag_lindhard_eta0(q, w, mu, T)) < 1e-4 * abs(c.imag)
    T0 = 1e-5
    mu0 = lindhard.free_gas_mu(n, T0)
    for qq in (0.3, 1.0, 2.5):
        c = lindhard.continuum_lindhard(qq, 0.0, 1e-7, mu0, T0)
        assert abs(c.real - lindhard.static_lindhard_t0(qq, kf)) < 2e-4 * abs(c.real)


def test_exact_discrete_fsum():
    """Fixed plane-wave basis, all bands: the double-commutator (f-sum) identity per k,
    sum_{n,n'} |rho_nn'(0)|^2 (f_n - f_n')(eps_n' - eps_n)
        = (q^2/2)(sum_n f_nk + sum_n f_n,k+q) + q.(J_k - J_k+q),  J_k = sum_n f_nk <k+G>_nk,
    holds exactly (summed over the mesh and scaled by 2/(N_k Omega) the first term is n q^2,
    the second is the current term of a finite mesh)."""
    lat = W.fcc_primitive(W.AL_A)
    B = crystal.reciprocal(lat)
    q = 0.5 * B[0] + 0.13 * B[1]
    base = W.tiny(natoms_displaced=True, kmesh=(2, 2, 2), ecut=1.2, basis="fixed",
                  kscheme="tr_symmetric", nq=1, nG=3, T_ev=8.0)
    lat = base.lattice
    npw = len(crystal.sphere_basis(lat, np.zeros(3), base.ecut))
    wl = base.replace(q=q[None], nbands=npw)
    gs = response.ground_state(wl, 0)
    gset = crystal.response_gset(lat, q, 3)
    rho = response.pair_densities(wl, gs, gset)[:, :, :, 0]
    Bl = crystal.reciprocal(lat)
    lhs = rhs = 0.0
    for ik in range(wl.nk):
        d = gs["eps_k"][ik][:, None] - gs["eps_kq"][ik][None, :]
        df = gs["f_k"][ik][:, None] - gs["f_kq"][ik][None, :]
        lhs += np.sum(np.abs(rho[ik]) ** 2 * df * (-d))
        pk = (np.abs(gs["C_k"][ik]) ** 2).T @ (gs["k"][ik][None] + gs["basis_k"][ik] @ Bl)
        pkq = (np.abs(gs["C_kq"][ik]) ** 2).T @ (gs["kq"][ik][None] + gs["basis_kq"][ik] @ Bl)
        Jk = gs["f_k"][ik] @ pk
        Jkq = gs["f_kq"][ik] @ pkq
        rhs += 0.5 * (q @ q) * (gs["f_k"][ik].sum() + gs["f_kq"][ik].sum()) + q @ (Jk - Jkq)
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)


def _db_workload():
    return W.tiny(nq=1, nw=41, wmin_ev=-40.0, wmax_ev=40.0, kmesh=(2, 2, 2), ecut=2.0, nbands=10)


def test_detailed_balance_and_odd_imaginary_part():
    wl = _db_workload()
    r = pipeline.run_q(wl, 0)
    w, S = wl.omega, r["S"]
    beta = 1.0 / wl.T
    smax = np.abs(S).max()
    for j in range(len(w)):
        jm = len(w) - 1 - j
        if w[j] > 0:
            assert abs(S[jm] - math.exp(-beta * w[j]) * S[j]) < 1e-10 * smax
            assert abs(r["chi00"][jm].imag + r["chi00"][j].imag) < 1e-12 * np.abs(r["chi00"]).max()


def test_passivity():
    wl = _db_workload()
    r = pipeline.run_q(wl, 0, keep_chi0=True)
    pos = r["freqs"] > 0
    assert np.all(r["S"] >= -1e-14 * np.abs(r["S"]).max())
    diag = np.einsum("wgg->wg", r["chi0"])[pos]
    assert np.all(diag.imag <= 1e-15 * np.abs(diag).max())


def test_itcf_analytic_spectrum():
    """S(w) = a w e^{-w/s} for w > 0: F_fold(tau) = a[(1/s + tau)^-2 + (1/s + beta - tau)^-2]."""
    a, s, T = 0.7, 0.4, 0.2
    beta = 1 / T
    w = np.linspace(0.0, 30.0, 60001)
    S = a * w * np.exp(-w / s)
    tau = np.linspace(0, beta / 2, 9)
    F = response.itcf_fold(w, S, tau, T)
    ref = a * ((1 / s + tau) ** -2 + (1 / s + beta - tau) ** -2)
    assert np.abs(F / ref - 1).max() < 1e-6
    m = response.itcf_metrics(w, S, T, 1.0)
    assert abs(m[0] - a * 2 * (1 / s + beta / 2) ** -2) < 1e-6 * m[0]
    # int_0^beta F dtau analytically: 2 a [s - 1/(1/s + beta)]
    assert abs(m[1] - 2 * a * (s - 1 / (1 / s + beta))) < 1e-6 * m[1]
    assert abs(m[3] - (m[1] - beta * response.itcf_fold(w, S, [0.0], T)[0])) < 1e-12


def test_itcf_symmetry_and_direct_mode():
    wl = _db_workload()
    r = pipeline.run_q(wl, 0)
    beta = 1 / wl.T
    tau = np.linspace(0, beta, 127)
    Ff = response.itcf_fold(r["wp"], r["Sp"], tau, wl.T)
    assert np.abs(Ff - Ff[::-1]).max() < 1e-14 * Ff.max()
    Fd = response.itcf_direct(wl.omega, r["S"], tau)
    # direct mode on a symmetric grid: symmetric up to the e^{-beta W} truncation
    assert np.abs(Fd - Fd[::-1]).max() < 1e-3 * Fd.max()
    assert np.abs(Fd - Ff).max() < 1e-3 * Ff.max()


def test_static_response_kramers_kronig():
    """-n int_0^beta F dtau = (2/pi) int_0^inf Im chi(w)/w dw = Re chi_00(0 + i eta)."""
    wl = W.tiny(nq=1, nw=3001, wmin_ev=0.0, wmax_ev=600.0, kmesh=(2, 2, 2), ecut=2.0, nbands=12)
    r = pipeline.run_q(wl, 0)
    chi_static = r["metrics"][4]
    re0 = r["chi00"][r["hcol"]].real
    assert abs(chi_static - re0) < 2e-3 * abs(re0)


def test_dyson_limits_and_residual():
    rng = np.random.default_rng(5)
    c = rng.normal(size=(6, 1, 1)) + 1j * rng.normal(size=(6, 1, 1))
    K = np.array([0.7])
    x = response.dyson_column0(c, K)
    assert np.allclose(x[:, 0], c[:, 0, 0] / (1 - c[:, 0, 0] * K[0]), rtol=1e-14)
    N = 9
    c = (rng.normal(size=(4, N, N)) + 1j * rng.normal(size=(4, N, N))) * 0.3
    assert np.allclose(response.dyson_column0(c, np.zeros(N)), c[:, :, 0], rtol=0, atol=1e-15)
    K = rng.uniform(0.5, 3.0, size=N)
    x = response.dyson_column0(c, K)
    M = np.eye(N)[None] - c * K[None, None, :]
    res = np.einsum("bij,bj->bi", M, x) - c[:, :, 0]
    assert np.abs(res).max() < 1e-12 * np.abs(c).max()


def test_pair_density_orthonormality_and_completeness():
    wl = W.tiny(nq=1, kmesh=(2, 2, 2), ecut=2.0, nbands=6)
    k = np.array([0.05, 0.1, -0.07])
    b = crystal.sphere_basis(wl.lattice, k, wl.ecut)
    _, C = crystal.eigenstates(wl.lattice, wl.positions, wl.Z, wl.r_c, k, b, 6)
    rho = response.pair_density(C, b, C, b, np.zeros((1, 3), dtype=int))
    assert np.abs(rho[:, :, 0] - np.eye(6)).max() < 1e-13
    # fixed basis, all bands, any q: the overlap at G = 0 is unitary
    lat = wl.lattice
    bf = crystal.sphere_basis(lat, np.zeros(3), 1.5)
    q = np.array([0.21, -0.13, 0.08])
    H1 = crystal.hamiltonian(lat, wl.positions, wl.Z, wl.r_c, k, bf)
    H2 = crystal.hamiltonian(lat, wl.positions, wl.Z, wl.r_c, k + q, bf)
    C1 = np.linalg.eigh(H1)[1]
    C2 = np.linalg.eigh(H2)[1]
    rho = response.pair_density(C1, bf, C2, bf, np.zeros((1, 3), dtype=int))[:, :, 0]
    assert np.abs(np.sum(np.abs(rho) ** 2, axis=1) - 1).max() < 1e-13


def _rho_realspace(lat, k, bk, Ck, kq, bkq, Ckq, gset, nr):
    """rho via orbitals on an nr^3 real-space grid: (1/N_r) sum_r u*_nk(r) u_n'k+q(r) e^{-iG.r},
    with u(r) = sum_G c(G) e^{iG.r} built by inverse FFT."""
    def to_grid(basis, C):
        g = np.zeros((C.shape[1], nr, nr, nr), dtype=np.complex128)
        idx = np.mod(basis, nr)
        for n in range(C.shape[1]):
            g[n][idx[:, 0], idx[:, 1], idx[:, 2]] = C[:, n]
        return np.fft.ifftn(g, axes=(1, 2, 3)) * nr ** 3
    uk = to_grid(bk, Ck)
    ukq = to_grid(bkq, Ckq)
    out = np.zeros((Ck.shape[1], Ckq.shape[1], len(gset)), dtype=np.complex128)
    for n in range(Ck.shape[1]):
        prod = np.fft.fftn(uk[n].conj()[None] * ukq, axes=(1, 2, 3)) / nr ** 3
        gi = np.mod(gset, nr)
        out[n] = prod[:, gi[:, 0], gi[:, 1], gi[:, 2]]
    return out


def test_bruteforce_chi0_realspace_route():
    """chi0 from real-space pair densities and an explicit loop over (k, n, n', G, G', w)."""
    wl = W.tiny(nq=1, kmesh=(2, 2, 2), ecut=1.5, nbands=5, nG=5, nw=6)
    r = pipeline.run_q(wl, 0, keep_chi0=True)
    gs = response.ground_state(wl, 0)
    om = crystal.volume(wl.lattice)
    nr = 16
    ref = np.zeros_like(r["chi0"])
    for ik in range(wl.nk):
        rho = _rho_realspace(wl.lattice, gs["k"][ik], gs["basis_k"][ik], gs["C_k"][ik], gs["kq"][ik],
                             gs["basis_kq"][ik], gs["C_kq"][ik], r["gset"], nr)
        for n in range(gs["nb"]):
            for m in range(gs["nb"]):
                d = gs["eps_k"][ik, n] - gs["eps_kq"][ik, m]
                f = (gs["f_k"][ik, n] - gs["f_kq"][ik, m]) * gs["w_k"][ik, n] * gs["w_kq"][ik, m]
                for iw, w in enumerate(r["freqs"]):
                    wt = f / (w + d + 1j * wl.eta)
                    for a in range(len(r["gset"])):
                        for b in range(len(r["gset"])):
                            ref[iw, a, b] += rho[n, m, a] * np.conj(rho[n, m, b]) * wt
    ref *= 2.0 / (wl.nk * om)
    assert np.abs(r["chi0"] - ref).max() < 1e-13 * np.abs(ref).max()


def _split_multiplet_case():
    """fcc primitive cell on a Gamma-centred mesh with a band cut that splits a degenerate
    multiplet at some k points (high-symmetry points keep the Oh degeneracies)."""
    lat = W.fcc_primitive(W.AL_A)
    q = 0.5 * crystal.reciprocal(lat)[1]
    base = W.tiny(natoms_displaced=False, kscheme="commensurate", kmesh=(2, 2, 2), ecut=2.5, nq=1,
                  nG=5, nw=12, T_ev=4.0)
    for nb in range(6, 16):
        wl = base.replace(q=q[None], nbands=nb)
        gs = response.ground_state(wl, 0)
        if np.any((gs["w_k"] > 0) & (gs["w_k"] < 1)) or np.any((gs["w_kq"] > 0) & (gs["w_kq"] < 1)):
            return wl, gs
    raise RuntimeError("no split multiplet found")


def test_band_weights_make_chi0_gauge_invariant():
    """A random unitary rotation inside each multiplet split by the band cut leaves chi0
    unchanged with the band weights, and changes it without them."""
    wl, gs = _split_multiplet_case()
    gset = crystal.response_gset(wl.lattice, wl.q[0], int(wl.nG[0]))
    freqs, _ = response.internal_frequencies(wl.omega)
    om = crystal.volume(wl.lattice)

    def chi0_of(g):
        rho = response.pair_densities(wl, g, gset).reshape(-1, len(gset))
        d, df = response.pair_weights(g)
        return response.chi0(rho, d, df, freqs, wl.eta, wl.nk, om)

    ref = chi0_of(gs)
    rng = np.random.default_rng(0)
    rot = dict(gs)
    for tag in ("k", "kq"):
        Cs = []
        for i, C in enumerate(gs["C_" + tag]):
            w = gs["w_" + tag][i]
            mem = np.where((w > 0) & (w < 1))[0]
            C = C.copy()
            if len(mem):
                X = rng.normal(size=(len(mem), len(mem))) + 1j * rng.normal(size=(len(mem), len(mem)))
                U, _ = np.linalg.qr(X)
                C[:, mem] = C[:, mem] @ U
            Cs.append(C)
        rot["C_" + tag] = Cs
    assert np.abs(chi0_of(rot) - ref).max() < 1e-12 * np.abs(ref).max()
    # with a plain cut at nbands the same rotation is visible
    plain, plain_rot = dict(gs), dict(rot)
    for g in (plain, plain_rot):
        for tag in ("k", "kq"):
            w = np.zeros_like(gs["w_" + tag])
            w[:, :wl.nbands] = 1.0
            g["w_" + tag] = w
    assert np.abs(chi0_of(plain_rot) - chi0_of(plain)).max() > 1e-6 * np.abs(ref).max()
