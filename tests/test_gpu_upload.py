"""GPU: pipelined orbital uploads (lrtddft_set_orbitals_async) through the C ABI.

Two cells share lattice, k meshes, basis and q (the second atom displaced differently), so
the orbitals of one can be given to a context set up for the other:
 - after an asynchronous upload of cell B's orbitals (from page-locked memory), cell A's
   context assembles exactly what cell B's own context does;
 - until the next assembly, the results of the current orbitals stay valid (S and F of cell A
   are unchanged by a pending upload), and the upload then takes effect;
 - a later synchronous set_orbitals drops a pending upload.
"""
import numpy as np
import pytest

from oracle import response
from paper_2510_01875_gb300 import binding, build
from paper_2510_01875_gb300 import workloads as W

pytestmark = pytest.mark.gpu

WL_A = W.tiny(seed=51, nq=2, nw=48)
WL_B = WL_A.replace(positions=WL_A.positions + np.array([[0.0, 0.0, 0.0], [0.07, -0.05, 0.04]]),
                    name="tiny51b")
TAU = response.tau_grid(WL_A.T, 16)


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return binding.load()


def _forward(c):
    c.chi0_assemble()
    c.dyson_solve()
    return c.dsf(), c.itcf(TAU)[0]


def _pinned_orbitals(c):
    import torch
    out = []
    for iq in range(c.nq):
        e, f, _, _ = c.get_ground_state(iq)
        t = torch.empty((2, c.nk, c.nb, c.npw, 2), dtype=torch.float64).pin_memory()
        cf = t.numpy().view(np.complex128).reshape(2, c.nk, c.nb, c.npw)
        c.get_orbitals(iq, cf)
        out.append((e, cf, f, t))
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp16x3"])
def test_async_upload_equals_own_context(prec):
    a = binding.Context(WL_A, prec)
    b = binding.Context(WL_B, prec)
    assert (a.nk, a.nb, a.npw) == (b.nk, b.nb, b.npw)
    for iq in range(WL_A.nq):
        ma, na = a.get_basis(iq)
        mb, nb_ = b.get_basis(iq)
        assert np.array_equal(ma, mb) and np.array_equal(na, nb_)
    S_b, F_b = _forward(b)
    S_a, F_a = _forward(a)
    assert np.abs(S_a - S_b).max() > 1e-3 * np.abs(S_b).max()   # the cells differ
    orbs = _pinned_orbitals(b)
    for iq, (e, cf, f, _) in enumerate(orbs):
        a.set_orbitals_async(iq, e, cf, f)
    # pending uploads leave the current results in place
    S_keep = a.dsf()
    F_keep, _ = a.itcf(TAU)
    assert np.array_equal(S_keep, S_a) and np.array_equal(F_keep, F_a)
    S_new, F_new = _forward(a)
    assert np.abs(S_new - S_b).max() <= 1e-12 * np.abs(S_b).max()
    assert np.abs(F_new / F_b - 1).max() <= 1e-12
    # the adopted orbitals are the uploaded ones
    for iq, (e, cf, f, _) in enumerate(orbs):
        assert np.array_equal(a.get_orbitals(iq), cf)
        e2, f2, _, _ = a.get_ground_state(iq)
        assert np.array_equal(e2, e) and np.array_equal(f2, f)
    a.close()
    b.close()


def test_sync_set_drops_pending_upload():
    a = binding.Context(WL_A, "fp64")
    b = binding.Context(WL_B, "fp64")
    S_a, _ = _forward(a)
    own = [(a.get_ground_state(iq), a.get_orbitals(iq)) for iq in range(WL_A.nq)]
    orbs = _pinned_orbitals(b)
    for iq, (e, cf, f, _) in enumerate(orbs):
        a.set_orbitals_async(iq, e, cf, f)
    for iq, ((e, f, _, _), cf) in enumerate(own):
        a.set_orbitals(iq, e, cf, f)
    S_again, _ = _forward(a)
    assert np.abs(S_again - S_a).max() <= 1e-12 * np.abs(S_a).max()
    a.close()
    b.close()


def test_repeated_async_uploads_pipeline():
    """Three assemblies, each adopting the upload queued during the one before (A, B, A)."""
    a = binding.Context(WL_A, "fp16x3")
    b = binding.Context(WL_B, "fp16x3")
    S_b, _ = _forward(b)
    orbs_b = _pinned_orbitals(b)
    orbs_a = _pinned_orbitals(a)
    S_a, _ = _forward(a)
    results = []
    for orbs in (orbs_b, orbs_a, orbs_b):
        a.chi0_assemble()
        for iq, (e, cf, f, _) in enumerate(orbs):
            a.set_orbitals_async(iq, e, cf, f)   # for the next assembly, while this one runs
        a.dyson_solve()
        results.append(a.dsf())
    S_last, _ = _forward(a)
    # the first assembly ran on A's orbitals, the second on B's (uploaded during the first), ...
    for S, ref in zip(results + [S_last], (S_a, S_b, S_a, S_b)):
        assert np.abs(S - ref).max() <= 1e-12 * np.abs(ref).max()
    a.close()
    b.close()
