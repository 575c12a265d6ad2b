"""GPU: the split forms' w = 0 column (0 not on the caller's grid) against the FP64 oracle, on
the tensor cores (64 x 64 G tiles: one tile at N_G = 59, 2 x 2 at N_G = 89) and on the CUDA
cores (LRT_TUNE_ZERO_SIMT), for one eta and for an eta list (a launch per eta).

Bound: the split form's chi0 bound, 3e-5 (FP16x3) or 1e-4 (BF16x3) of the column's max norm.
"""
import numpy as np
import pytest

from oracle import pipeline
from paper_2510_01875_gb300 import binding, build
from paper_2510_01875_gb300 import workloads as W

pytestmark = pytest.mark.gpu

BOUND = {"fp16x3": 3e-5, "bf16x3": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return binding.load()


def _zero_column(wl, prec, zero_simt, etas=None):
    c = binding.Context(wl, prec)
    c.set_tuning(zero_simt=zero_simt)
    if etas is not None:
        c.set_eta_list(etas)
    c.chi0_assemble()
    freqs, hcol = c.get_frequencies()
    assert hcol == len(freqs) - 1 and freqs[hcol] == 0.0   # 0 is appended after the grid
    chi0 = c.get_chi0(0)
    c.close()
    return chi0, hcol


@pytest.mark.parametrize("prec", ["fp16x3", "bf16x3"])
@pytest.mark.parametrize("nG", [59, 89])
def test_zero_column_against_oracle(nG, prec):
    wl = W.tiny(seed=81, nq=1, nw=24, nbands=10, nG=nG)
    ref = pipeline.run_q(wl, 0, keep_chi0=True)["chi0"]
    tc, hcol = _zero_column(wl, prec, False)
    simt, _ = _zero_column(wl, prec, True)
    r0 = ref[hcol]
    tol = BOUND[prec] * np.abs(r0).max()
    assert np.abs(tc[hcol] - r0).max() <= tol
    assert np.abs(simt[hcol] - r0).max() <= tol
    # the other frequencies do not depend on how the w = 0 column is computed
    assert np.array_equal(tc[:hcol], simt[:hcol])


def test_zero_column_eta_list():
    wl = W.tiny(seed=82, nq=1, nw=24, nbands=10, nG=21)
    etas = np.array([0.5, 1.0, 2.0]) * wl.eta
    got, hcol = _zero_column(wl, "fp16x3", False, etas)   # [eta][w][G][G']
    for j, eta in enumerate(etas):
        r0 = pipeline.run_q(wl.replace(eta=eta), 0, keep_chi0=True)["chi0"][hcol]
        assert np.abs(got[j][hcol] - r0).max() <= BOUND["fp16x3"] * np.abs(r0).max(), j
