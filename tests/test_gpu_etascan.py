"""GPU: the eta-convergence test (Sec. 2).  An eta list computes chi0 for every broadening in
one assembly (the tensor-core contraction takes the (eta, w) pairs as columns of one launch);
Dyson, S, F and the metrics then come per (q, eta).  Through the C ABI, against the FP64
oracle run once per eta: FP64 to 1e-10 (chi0 and S of the per-(q, eta) max norm, F and the
metrics relative), FP16x3 at the split bounds (F 1e-5 pointwise, S 1e-4 at its peaks, chi0
3e-5).  The reference-eta index is an integer decided from the metrics: it is checked against
the oracle's rule applied to the same metrics the GPU computed, and those metrics against the
oracle's."""
import numpy as np
import pytest

from oracle import etascan, pipeline, response
from paper_2510_01875_gb300 import binding, build
from paper_2510_01875_gb300 import workloads as W

pytestmark = pytest.mark.gpu

WL = W.tiny(nq=2, nw=41, wmin_ev=-20.0, wmax_ev=60.0)
ETAS = [W.ev(x) for x in (0.2, 0.35, 0.5, 0.8)]


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return binding.load()


@pytest.fixture(scope="module")
def oracle_runs():
    return {(j, iq): pipeline.run_q(WL.replace(eta=e), iq, keep_chi0=True)
            for j, e in enumerate(ETAS) for iq in range(WL.nq)}


def _gpu(prec):
    ctx = binding.Context(WL, prec)
    ctx.set_eta_list(ETAS)
    assert np.array_equal(ctx.get_eta_list(), np.array(ETAS))
    ctx.chi0_assemble()
    ctx.dyson_solve()
    S = ctx.dsf()
    F, m = ctx.itcf(response.tau_grid(WL.T, WL.ntau))
    chi0 = [ctx.get_chi0(iq) for iq in range(WL.nq)]
    return ctx, S, F, m, chi0


def _peaks(S):
    return [j for j in range(1, len(S) - 1) if S[j] > S[j - 1] and S[j] >= S[j + 1] and S[j] > 0.1 * S.max()]


def test_eta_list_fp64_against_oracle(oracle_runs):
    ctx, S, F, m, chi0 = _gpu("fp64")
    ctx.close()
    assert S.shape == (WL.nq, len(ETAS), WL.nw) and chi0[0].shape[0] == len(ETAS)
    for (j, iq), r in oracle_runs.items():
        c = chi0[iq][j]
        assert np.abs(c - r["chi0"]).max() <= 1e-10 * np.abs(r["chi0"]).max()
        assert np.abs(S[iq, j] - r["S"]).max() <= 1e-10 * np.abs(r["S"]).max()
        assert np.abs(F[iq, j] / r["F"] - 1).max() <= 1e-10
        assert np.abs(m[iq, j] / r["metrics"] - 1).max() <= 1e-10


def test_eta_list_split_against_oracle(oracle_runs):
    ctx, S, F, m, chi0 = _gpu("fp16x3")
    ctx.close()
    for (j, iq), r in oracle_runs.items():
        assert np.abs(chi0[iq][j] - r["chi0"]).max() <= 3e-5 * np.abs(r["chi0"]).max()
        assert np.abs(F[iq, j] / r["F"] - 1).max() <= 1e-5
        for p in _peaks(r["S"]):
            assert abs(S[iq, j, p] / r["S"][p] - 1) <= 1e-4


@pytest.mark.parametrize("prec", ["fp64", "fp16x3"])
def test_reference_eta(prec, oracle_runs):
    ctx, _, _, _, _ = _gpu(prec)
    tau = response.tau_grid(WL.T, WL.ntau)
    for tol in (1e-3, 2e-2, 1e-1):
        F, m, ref = ctx.eta_scan(tau, tol)
        for iq in range(WL.nq):
            assert ref[iq] == etascan.reference_eta(m[iq], tol)
    ctx.close()
    bound = 1e-10 if prec == "fp64" else 1e-5
    for (j, iq), r in oracle_runs.items():
        assert np.abs(m[iq, j] / r["metrics"] - 1).max() <= bound


def test_one_launch_equals_one_eta_at_a_time():
    """The columns of every eta in one contraction launch give the chi0 of separate contexts,
    one eta each (FP64: the same arithmetic, 1e-12; FP16x3: the power-of-two scale of the
    weights follows the smallest eta, so the 16-bit parts differ at the split's rounding)."""
    for prec, tol in (("fp64", 1e-12), ("fp16x3", 2e-5)):
        ctx, _, _, _, chi0 = _gpu(prec)
        ctx.close()
        for j, e in enumerate(ETAS):
            c1 = binding.Context(WL.replace(eta=e), prec)
            c1.chi0_assemble()
            for iq in range(WL.nq):
                one = c1.get_chi0(iq)
                assert np.abs(chi0[iq][j] - one).max() <= tol * np.abs(one).max(), (prec, j, iq)
            c1.close()


def test_adjoint_needs_one_eta_and_set_params_returns_to_one():
    ctx, _, _, _, _ = _gpu("fp64")
    with pytest.raises(binding.LrtError):
        ctx.jacobian(response.tau_grid(WL.T, 4))
    ctx.set_params(WL.T, ETAS[1])
    ctx.chi0_assemble()
    ctx.dyson_solve()
    S = ctx.dsf()
    ctx.close()
    r = pipeline.run_q(WL.replace(eta=ETAS[1]), 0)
    assert S.shape == (WL.nq, WL.nw)
    assert np.abs(S[0] - r["S"]).max() <= 1e-10 * np.abs(r["S"]).max()
