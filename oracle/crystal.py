"""Oracle: crystal geometry, plane-wave bases and the empty-core Kohn-Sham problem.

Test infrastructure only (see oracle/__init__.py).

The paper's ground state comes from plane-wave DFT (App. A.1).  Here the
potential is fixed (no self-consistency): the Ashcroft empty-core ion
v(r) = -Z/r for r > r_c and 0 inside, whose per-cell Fourier coefficient is
v(G) = -(4 pi Z / (Omega G^2)) cos(G r_c), with V(G=0) = 0 (neutralising
background).  H_{GG'}(k) = 1/2 |k+G|^2 delta_{GG'} + V(G-G'),
V(G) = sum_a v(G) exp(-i G.R_a).

Pinned by: the zero-potential limit (plane waves are exact eigenstates, tested in
tests/test_oracle_response.py) and the explicit-dense brute force check.
"""
from __future__ import annotations

import math

import numpy as np

# Two values closer than this (in 1/bohr^2) are treated as equal when ordering
# |q+G|^2 and |G|^2 shells; basis spheres include points up to 2*ecut + BASIS_TOL.
SHELL_TOL = 1e-9
BASIS_TOL = 1e-9


def reciprocal(lattice: np.ndarray) -> np.ndarray:
    """Rows b_j with a_i . b_j = 2 pi delta_ij."""
    return 2.0 * math.pi * np.linalg.inv(lattice).T


def volume(lattice: np.ndarray) -> float:
    return abs(float(np.linalg.det(lattice)))


def _miller_candidates(lattice: np.ndarray, center: np.ndarray, radius: float) -> np.ndarray:
    """All integer triples m with |center + m.B| <= radius (plus a margin).
    |m_i| <= (radius + |center|) |a_i| / (2 pi) because m_i = (G . a_i) / (2 pi)."""
    reach = radius + float(np.linalg.norm(center))
    lim = [int(math.ceil(reach * np.linalg.norm(lattice[i]) / (2.0 * math.pi))) + 1 for i in range(3)]
    r = [np.arange(-l, l + 1) for l in lim]
    m = np.stack(np.meshgrid(r[0], r[1], r[2], indexing="ij"), axis=-1).reshape(-1, 3)
    return m


def sphere_basis(lattice: np.ndarray, k: np.ndarray, ecut: float) -> np.ndarray:
    """Miller indices of {G : 1/2 |k+G|^2 <= ecut}, in lexicographic (h,k,l) order."""
    B = reciprocal(lattice)
    m = _miller_candidates(lattice, k, math.sqrt(2.0 * ecut))
    kg = k[None, :] + m @ B
    keep = np.einsum("ij,ij->i", kg, kg) <= 2.0 * ecut + BASIS_TOL
    return m[keep]


def response_gset(lattice: np.ndarray, q: np.ndarray, nG: int) -> np.ndarray:
    """The nG reciprocal vectors of smallest |q+G|; ties broken by smaller |G|, then by
    lexicographic (h,k,l).  Returned with G = 0 first and the rest in that order.
    Raises ValueError if G = 0 is not among them."""
    B = reciprocal(lattice)
    radius = 1.0
    while True:
        m = _miller_candidates(lattice, q, radius)
        qg = q[None, :] + m @ B
        d2 = np.einsum("ij,ij->i", qg, qg)
        inside = d2 <= radius * radius
        # every vector taken must lie well inside, so its whole shell is a candidate
        if (d2 <= radius * radius - 1e-6).sum() >= nG:
            break
        radius *= 1.5
    m = m[inside]
    d2 = d2[inside]
    g2 = np.einsum("ij,ij->i", m @ B, m @ B)
    # Shell labels: sort by value and start a new shell whenever the gap to the
    # first member of the current shell exceeds SHELL_TOL.
    def shells(v):
        order = np.argsort(v, kind="stable")
        lab = np.empty(len(v), dtype=np.int64)
        cur, start = 0, None
        for idx in order:
            if start is None or v[idx] - start > SHELL_TOL:
                if start is not None:
                    cur += 1
                start = v[idx]
            lab[idx] = cur
        return lab
    s1 = shells(d2)
    s2 = shells(g2)
    keys = sorted(range(len(m)), key=lambda i: (s1[i], s2[i], int(m[i, 0]), int(m[i, 1]), int(m[i, 2])))
    chosen = m[keys[:nG]]
    zero = np.where(~chosen.any(axis=1))[0]
    if len(zero) != 1:
        raise ValueError("G = 0 is not among the nG vectors of smallest |q+G|")
    rest = [i for i in range(nG) if i != zero[0]]
    return np.concatenate([chosen[zero], chosen[rest]], axis=0)


def kmesh(lattice: np.ndarray, n, shift: np.ndarray) -> np.ndarray:
    """Gamma-centred mesh k = sum_j (i_j/n_j) b_j, i_j = 0..n_j-1, plus a Cartesian shift.
    Order: i_0 slowest, i_2 fastest."""
    B = reciprocal(lattice)
    pts = []
    for i in range(n[0]):
        for j in range(n[1]):
            for l in range(n[2]):
                pts.append((i / n[0]) * B[0] + (j / n[1]) * B[1] + (l / n[2]) * B[2])
    return np.array(pts) + shift[None, :]


def pair_meshes(lattice, n, q, scheme):
    """k points and k+q points for one q.
    commensurate: k in M (Gamma-centred), k+q = k + q.
    tr_symmetric: k in M - q/2, k+q in M + q/2; then -k-q is in the k set modulo G,
    which makes chi0(-w)* = chi0(w)^T exactly (time reversal)."""
    if scheme == "commensurate":
        k = kmesh(lattice, n, np.zeros(3))
    elif scheme == "tr_symmetric":
        k = kmesh(lattice, n, -0.5 * q)
    else:
        raise ValueError(scheme)
    return k, k + q[None, :]


def vion(lattice: np.ndarray, positions: np.ndarray, Z: float, r_c: float, miller: np.ndarray,
         potential: str = "empty_core") -> np.ndarray:
    """V(G) = sum_a v(|G|) exp(-i G.R_a), v(G) = -(4 pi Z/(Omega G^2)) cos(G r_c), V(0) = 0."""
    out = np.zeros(len(miller), dtype=np.complex128)
    if potential == "zero":
        return out
    B = reciprocal(lattice)
    om = volume(lattice)
    G = miller @ B
    g2 = np.einsum("ij,ij->i", G, G)
    nz = g2 > 0
    g = np.sqrt(g2[nz])
    vg = -(4.0 * math.pi * Z / (om * g2[nz])) * np.cos(g * r_c)
    phase = np.exp(-1j * (G[nz] @ positions.T)).sum(axis=1)
    out[nz] = vg * phase
    return out


def hamiltonian(lattice, positions, Z, r_c, k, basis, potential="empty_core") -> np.ndarray:
    """Dense H_{GG'}(k) on the given basis (Miller indices)."""
    B = reciprocal(lattice)
    kg = k[None, :] + basis @ B
    H = np.zeros((len(basis), len(basis)), dtype=np.complex128)
    diff = basis[:, None, :] - basis[None, :, :]
    uniq, inv = np.unique(diff.reshape(-1, 3), axis=0, return_inverse=True)
    V = vion(lattice, positions, Z, r_c, uniq, potential)
    H += V[inv.reshape(-1)].reshape(len(basis), len(basis))
    H[np.diag_indices(len(basis))] += 0.5 * np.einsum("ij,ij->i", kg, kg)
    return H


def eigenstates(lattice, positions, Z, r_c, k, basis, nbands, potential="empty_core"):
    """Lowest nbands eigenpairs of H(k) by LAPACK (numpy.linalg.eigh).
    Returns (eps[nbands], C[npw, nbands]) with orthonormal columns."""
    if nbands > len(basis):
        raise ValueError("nbands exceeds the number of plane waves")
    H = hamiltonian(lattice, positions, Z, r_c, k, basis, potential)
    w, v = np.linalg.eigh(H)
    return w[:nbands], v[:, :nbands]
