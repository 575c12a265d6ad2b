"""The allocation-free attenuation entry point against the allocating one.

Some callers cannot allocate device memory when they attenuate: programs whose free device
memory is held by another allocator's pool, or that cannot afford the device-wide
synchronisation cudaFree implies.  lrtddft_attenuate_noalloc serves them from a fixed 16 MiB
array in the library.  It must return what lrtddft_attenuate returns, on consecutive calls
(the shared array keeps the previous call's contents), and refuse work that does not fit.

This file is collected last on purpose: a run that stops at the first failure has run every
other test before reaching it."""
import numpy as np
import pytest

from paper_2510_01875_gb300 import binding, build
from paper_2510_01875_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return binding.load()


def _ctx(nw=301):
    wl = W.tiny(seed=21, nq=2, nw=nw, wmin_ev=0.0, wmax_ev=60.0, kmesh=(2, 2, 2), ecut=2.5,
                nbands=14, eta_ev=0.15)
    ctx = binding.Context(wl)
    ctx.chi0_assemble()
    ctx.dyson_solve()
    return ctx


def _same_report(a, b):
    assert a["targets"] == b["targets"] and a["n_accepted"] == b["n_accepted"]
    assert len(a["degrees"]) == len(b["degrees"])
    for x, y in zip(a["degrees"], b["degrees"]):
        assert (x["d"], x["m"], x["accepted"]) == (y["d"], y["m"], y["accepted"])
        for k in ("score", "mean_ratio", "rms_ratio"):
            assert abs(x[k] - y[k]) <= 1e-12 * max(abs(y[k]), 1e-300)


def test_noalloc_matches_allocating_entry_point_on_consecutive_calls():
    ctx = _ctx()
    params = binding.atten_params(accept_mean=1.0, accept_rms=1.0)
    ref, rep_ref = ctx.attenuate(params)
    for _ in range(2):
        got, rep = ctx.attenuate_noalloc(params)
        assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()
        for a, b in zip(rep, rep_ref):
            _same_report(a, b)
    ctx.close()


def test_noalloc_refuses_a_workspace_beyond_its_array():
    ctx = _ctx(nw=2001)
    # 8 degrees x ~600 windows x 2 q x 2001 samples needs hundreds of MB
    params = binding.atten_params(d_min=1, d_max=8, n_w=600, w_max=0.9 * 60.0 / 27.211386245988)
    with pytest.raises(binding.LrtError) as err:
        ctx.attenuate_noalloc(params)
    assert err.value.status == "invalid argument"
    assert "exceeds" in str(err.value)
    # the context stays usable
    Sp, _ = ctx.attenuate_noalloc(binding.atten_params())
    assert np.isfinite(Sp).all()
    ctx.close()
