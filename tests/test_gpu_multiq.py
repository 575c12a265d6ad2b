"""GPU: many q of uneven size in one persistent tensor-core launch, its tuning choices, and
the captured CUDA graph of the forward path (through the C ABI).

 - q of different N_G (ragged) in one launch against the FP64 oracle at the split-precision
   bounds (chi0 3e-5 of the per-q max norm, F 1e-5 pointwise);
 - one launch for all q equals one launch per q to FP64 rounding (each unit computes the same
   FP32 partial sums; only the order of the FP64 reductions differs);
 - half row units (256 rows) equal the default 512-row units to FP64 rounding;
 - every (variant, unit size) and the autotuner agree with the defaults within 2e-6 on F and
   report the choice they made;
 - a graph replay reproduces the eager S and F and is refused after set_params.
"""
import numpy as np
import pytest

from oracle import pipeline, response
from paper_2510_01875_gb300 import binding, build
from paper_2510_01875_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return binding.load()


def ragged():
    wl = W.tiny(seed=31, nq=4, nw=45, kmesh=(3, 3, 3), nbands=10)
    return wl.replace(nG=np.array([7, 15, 9, 27]))


def run(wl, prec="fp16x3", **tune):
    c = binding.Context(wl, prec)
    if tune:
        c.set_tuning(**tune)
    c.chi0_assemble()
    c.dyson_solve()
    tau = response.tau_grid(wl.T, wl.ntau)
    F, _ = c.itcf(tau)
    out = {"S": c.dsf(), "F": F, "chi0": [c.get_chi0(i) for i in range(wl.nq)], "tuning": c.get_tuning(),
           "rows": c.get_tile_rows() if prec != "fp64" else None}
    c.close()
    return out


def test_ragged_q_in_one_launch_against_oracle():
    wl = ragged()
    g = run(wl)
    for iq in range(wl.nq):
        r = pipeline.run_q(wl, iq, keep_chi0=True)
        c0 = r["chi0"]
        assert np.abs(g["chi0"][iq] - c0).max() / np.abs(c0).max() < 3e-5, iq
        assert np.abs(g["F"][iq] / r["F"] - 1).max() < 1e-5, iq


def test_half_row_units_equal_full_units():
    """Every row unit a half (256 rows, one accumulator per CTA) against the default (512-row
    units; an odd last one is a half): each row accumulates the same FP32 partial sums in the
    same order, so only the order of the FP64 reductions differs."""
    wl = ragged()
    a = run(wl)
    b = run(wl, half_tiles=True)
    assert a["rows"] == 512 and b["rows"] == 256
    for iq in range(wl.nq):
        scale = np.abs(a["chi0"][iq]).max()
        assert np.abs(a["chi0"][iq] - b["chi0"][iq]).max() <= 1e-12 * scale
    np.testing.assert_allclose(a["F"], b["F"], rtol=1e-12)


def test_one_launch_equals_one_launch_per_q():
    wl = ragged()
    a = run(wl)
    b = run(wl, single_q=True)
    for iq in range(wl.nq):
        scale = np.abs(b["chi0"][iq]).max()
        assert np.abs(a["chi0"][iq] - b["chi0"][iq]).max() <= 1e-12 * scale
    np.testing.assert_allclose(a["F"], b["F"], rtol=1e-12)


@pytest.mark.parametrize("variant,unit_stages", [(0, 64), (1, 64), (1, 4096), (0, 128)])
def test_forced_choices_agree(variant, unit_stages):
    wl = W.tiny(seed=32, nq=2, nw=40, kmesh=(4, 4, 4), nbands=12, nG=15)
    ref = run(wl)
    g = run(wl, variant=variant, unit_stages=unit_stages)
    assert g["tuning"] == (variant, unit_stages)
    np.testing.assert_allclose(g["F"], ref["F"], rtol=2e-6)


def test_autotune_picks_a_candidate():
    wl = W.tiny(seed=33, nq=2, nw=40, kmesh=(4, 4, 4), nbands=12, nG=15)
    ref = run(wl)
    g = run(wl, auto=True)
    v, u = g["tuning"]
    assert v in (0, 1) and u in (1024, 4096, 16384) and g["rows"] in (256, 512)
    np.testing.assert_allclose(g["F"], ref["F"], rtol=2e-6)


def test_tuning_argument_checks():
    c = binding.Context(W.tiny(seed=34, nq=1), "fp16x3")
    for kw in (dict(variant=2), dict(variant=-2), dict(unit_stages=100), dict(unit_stages=-64)):
        with pytest.raises(binding.LrtError):
            c.set_tuning(**kw)
    c.close()


@pytest.mark.parametrize("prec", ["fp16x3", "fp64"])
def test_graph_replay_matches_eager(prec):
    torch = pytest.importorskip("torch")
    wl = ragged()
    tau = response.tau_grid(wl.T, wl.ntau)
    eager = run(wl, prec)
    c = binding.Context(wl, prec)
    dev = torch.device("cuda", 0)
    t = torch.tensor(tau, dtype=torch.float64, device=dev)
    S = torch.zeros((wl.nq, wl.nw), dtype=torch.float64, device=dev)
    F = torch.zeros((wl.nq, len(tau)), dtype=torch.float64, device=dev)
    M = torch.zeros((wl.nq, 5), dtype=torch.float64, device=dev)
    c.graph_capture(len(tau), t.data_ptr(), S.data_ptr(), F.data_ptr(), M.data_ptr())
    S.zero_()
    F.zero_()
    c.graph_launch()
    torch.cuda.synchronize()
    tol = 1e-12
    np.testing.assert_allclose(F.cpu().numpy(), eager["F"], rtol=tol)
    assert np.abs(S.cpu().numpy() - eager["S"]).max() <= tol * np.abs(eager["S"]).max()
    # results of the replay are visible to the ordinary calls
    assert np.abs(c.get_chi0(0) - eager["chi0"][0]).max() <= tol * np.abs(eager["chi0"][0]).max()
    c.set_params(wl.T, wl.eta)
    with pytest.raises(binding.LrtError):
        c.graph_launch()
    c.close()
