"""The 4-atom adjoint workload's shape on a smaller k mesh: 4-atom conventional cubic Al cell,
200 bands, 89 response G-vectors, 2048 frequencies on [-100, 300] eV, T = 20 eV,
eta = 0.5 eV, static f_xc(q) model; 2^3 k points instead of 6^3.

 - FP64 chi0 and S against the oracle (largest |q|) on a 64-frequency subset of the grid: the
   oracle's per-frequency loop over 3.2 x 10^5 pairs takes tens of seconds per 64 frequencies;
 - the FP16x3 Jacobian dF(q, tau)/d(T, eta, A, B, C) (64 tau on [0, beta/2]; smallest and
   largest |q|) against the FP64 adjoint's, per parameter, to 1e-4 of its max norm (the FP64
   adjoint equals the oracle's tangents to 1e-8 and central differences to 1e-6 in
   tests/test_gpu_adjoint.py).
"""
import numpy as np
import pytest

from oracle import pipeline, response
from paper_2510_01875_gb300 import binding, build
from paper_2510_01875_gb300 import workloads as W

pytestmark = pytest.mark.gpu

WL = W.al4_cubic_k6_b200().replace(kmesh=(2, 2, 2))


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return binding.load()


def test_adjoint_shape_fp64_against_oracle():
    j0 = int(np.searchsorted(WL.omega, W.ev(10.0)))
    wl = WL.replace(q=WL.q[15:16], nG=WL.nG[15:16], omega=WL.omega[j0:j0 + 64])
    ctx = binding.Context(wl, "fp64")
    ctx.chi0_assemble()
    ctx.dyson_solve()
    S = ctx.dsf()[0]
    chi0 = ctx.get_chi0(0)
    ctx.close()
    r = pipeline.run_q(wl, 0, keep_chi0=True)
    assert np.abs(chi0 - r["chi0"]).max() <= 1e-10 * np.abs(r["chi0"]).max()
    assert np.abs(S - r["S"]).max() <= 1e-10 * np.abs(r["S"]).max()


def test_adjoint_shape_split_jacobian():
    wl = WL.replace(q=WL.q[[0, 15]], nG=WL.nG[[0, 15]])
    tau = response.tau_grid(wl.T, 64)
    J = {}
    for prec in ("fp64", "fp16x3"):
        ctx = binding.Context(wl, prec)
        ctx.chi0_assemble()
        ctx.dyson_solve()
        J[prec] = ctx.jacobian(tau)[1]
        ctx.close()
    for j in range(5):
        ref = J["fp64"][..., j]
        err = np.abs(J["fp16x3"][..., j] - ref).max() / np.abs(ref).max()
        assert err <= 1e-4, (j, err)
