"""GPU: dielectric properties from a DSF (Sec. 3, Eqs. 10-11) through the C ABI against the
oracle's transform of the same spectra: chi (Kramers-Kronig by Maclaurin's formula), 1/eps,
eps and sigma to 1e-12 of each quantity's max norm (FP64; only the summation order differs)."""
import numpy as np
import pytest

from oracle import dielectric as D
from oracle import response
from paper_2510_01875_gb300 import binding, build
from paper_2510_01875_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return binding.load()


@pytest.mark.parametrize("wmin_ev", [0.0, -25.0])
def test_dielectric_against_oracle(wmin_ev):
    wl = W.tiny(nq=2, nw=81, wmin_ev=wmin_ev, wmax_ev=80.0)
    ctx = binding.Context(wl, "fp64")
    ctx.chi0_assemble()
    ctx.dyson_solve()
    S = ctx.dsf()
    Sp, _ = ctx.attenuate()
    for spec in (S, Sp):
        got = ctx.dielectric(spec)
        for iq in range(wl.nq):
            w, chi, ei, e, sg = D.from_dsf(spec[iq], wl.omega, wl.T, response.density(wl),
                                           float(np.linalg.norm(wl.q[iq])))
            assert np.array_equal(got["w"], w)
            for key, ref in (("chi", chi), ("eps_inv", ei), ("eps", e), ("sigma", sg)):
                assert np.abs(got[key][iq] - ref).max() <= 1e-12 * np.abs(ref).max(), (key, iq)
    ctx.close()
