"""GPU setup: the kept orbitals are eigenvectors of H(k) to FP64 accuracy.

The batched eigensolver's vectors carried residuals ||H v - eps v|| up to 1.6e-9 Ha on the
benchmark cell; the library refines them by one first-order step in the solver's eigenbasis
and a Lowdin re-orthonormalisation.  Checked here through the C ABI: the orbitals and
eigenvalues of every k point of both meshes against H(k) built independently by the oracle on
the library's own basis order, and their orthonormality."""
import numpy as np
import pytest

from oracle import crystal
from paper_2510_01875_gb300 import binding, build
from paper_2510_01875_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FULL = W.al1_fcc_k12_b120()
CASES = {
    "tiny": W.tiny(),
    "large_ng_cell": W.tiny(seed=51, nq=2, nw=24, kmesh=(2, 2, 2), nbands=8),
    # the benchmark cell: 120 bands of 331-334 plane waves, smallest and largest |q|
    "al1_16ha_b120": FULL.replace(kmesh=(2, 2, 2), q=FULL.q[[0, 7]], nG=FULL.nG[[0, 7]]),
}


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return binding.load()


@pytest.mark.parametrize("name", sorted(CASES))
def test_orbitals_are_eigenvectors(name):
    wl = CASES[name]
    ctx = binding.Context(wl, "fp64")
    worst_res, worst_orth = 0.0, 0.0
    for iq in range(wl.nq):
        coeff = ctx.get_orbitals(iq)
        miller, npw_k = ctx.get_basis(iq)
        eps, _, _, _ = ctx.get_ground_state(iq)
        meshes = crystal.pair_meshes(wl.lattice, wl.kmesh, wl.q[iq], wl.kscheme)
        for s in range(2):
            for ik, k in enumerate(meshes[s]):
                n = int(npw_k[s, ik])
                H = crystal.hamiltonian(wl.lattice, wl.positions, wl.Z, wl.r_c, k, miller[s, ik, :n],
                                        wl.potential)
                V = coeff[s, ik, :wl.nbands, :n].T          # [npw][nbands]
                R = H @ V - V * eps[s, ik, :wl.nbands][None, :]
                worst_res = max(worst_res, float(np.linalg.norm(R, axis=0).max()))
                worst_orth = max(worst_orth, float(np.abs(V.conj().T @ V - np.eye(wl.nbands)).max()))
                assert not coeff[s, ik, :, n:].any()       # padding rows stay zero
    ctx.close()
    assert worst_res <= 1e-12, worst_res
    assert worst_orth <= 1e-13, worst_orth
