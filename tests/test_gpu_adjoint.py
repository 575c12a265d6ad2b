"""GPU adjoint: derivatives of S(q, w) and F(q, tau) with respect to (T, eta, A, B, C)
through the C ABI (lrtddft_jacobian, lrtddft_itcf_vjp, lrtddft_dsf_vjp, lrtddft_set_params)
and the torch.autograd wrapper.

 - FP64 path against the oracle's analytic forward-mode tangents (oracle/adjoint.py):
   1e-8 of each parameter's max |dF| (the oracle tangents are pinned to central
   differences of the oracle's forward path in tests/test_oracle_adjoint.py);
 - split-precision paths (FP16x3 and BF16x3) against central differences of the FP64 forward
   (Richardson-extrapolated), within the 1e-4 gradient bound (three readings of it below);
 - FP64 path against the same central differences within 1e-6;
 - vector-Jacobian products equal the contracted Jacobians; set_params reproduces a
   freshly created context; the autograd wrapper returns the library's vjp.
"""
import numpy as np
import pytest

from oracle import adjoint, response
from paper_2510_01875_gb300 import binding, build
from paper_2510_01875_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return binding.load()


def _ctx(wl, prec="fp64"):
    c = binding.Context(wl, prec)
    c.chi0_assemble()
    c.dyson_solve()
    return c


CASES = {
    "tr_model": dict(seed=21, nq=2, kernel="fxc_model", nw=48, T_ev=4.0, eta_ev=0.6),
    "comm_model": dict(seed=22, nq=1, kernel="fxc_model", kscheme="commensurate", nw=40),
    "zero_on_grid": dict(seed=23, nq=1, kernel="fxc_model", nw=41, wmin_ev=-20.0, wmax_ev=20.0),
    "alda_ragged": dict(seed=24, nq=2, kernel="rpa_alda", nw=37, nG=9, nbands=11),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp64_jacobian_matches_oracle_tangents(name):
    wl = W.tiny(**CASES[name])
    tau = response.tau_grid(wl.T, 12)
    c = _ctx(wl)
    dS, dF = c.jacobian(tau)
    c.close()
    for iq in range(wl.nq):
        t = adjoint.tangents_q(wl, iq, tau)
        for j in range(5):
            ref = t["dF"][:, j]
            scale = np.abs(ref).max()
            if scale == 0.0:
                assert np.all(dF[iq, :, j] == 0.0), (name, iq, j)
                continue
            assert np.abs(dF[iq, :, j] - ref).max() / scale < 1e-8, (name, iq, j)
            refS = t["dS"][:, j]
            assert np.abs(dS[iq, :, j] - refS).max() / np.abs(refS).max() < 1e-8, (name, iq, j)


def _shifted(c, wl, j, h):
    p = [wl.T, wl.eta] + list(wl.fxc_params)
    p[j] += h
    c.set_params(p[0], p[1], fxc_params=p[2:])
    c.chi0_assemble()
    c.dyson_solve()


def _fd_fp64(wl, tau, gF, j, h):
    """Central difference of sum(gF * F) along parameter j on the FP64 GPU path, Richardson-
    extrapolated from steps h and 2h (truncation O(h^4))."""
    c = _ctx(wl, "fp64")
    d = []
    for step in (h, 2.0 * h):
        Fs = []
        for sgn in (1.0, -1.0):
            _shifted(c, wl, j, sgn * step)
            Fs.append(c.itcf(tau)[0])
        d.append(float(np.sum(gF * (Fs[0] - Fs[1]))) / (2.0 * step))
    c.close()
    return (4.0 * d[0] - d[1]) / 3.0


def _fd_fp64_jacobian(wl, tau, j, h):
    """dF(q, tau)/d theta_j [nq][ntau] by central differences of the FP64 GPU forward,
    Richardson-extrapolated from steps h and 2h (truncation O(h^4))."""
    c = _ctx(wl, "fp64")
    d = []
    for step in (h, 2.0 * h):
        Fs = []
        for sgn in (1.0, -1.0):
            _shifted(c, wl, j, sgn * step)
            Fs.append(c.itcf(tau)[0])
        d.append((Fs[0] - Fs[1]) / (2.0 * step))
    c.close()
    return (4.0 * d[0] - d[1]) / 3.0


@pytest.mark.parametrize("prec", ["fp16x3", "bf16x3"])
def test_split_gradient_against_fp64_central_differences(prec):
    """Gradients of F within 1e-4 of central differences of the FP64 forward (the split
    forward's own differences are no reference: its ~1e-6 rounding changes non-smoothly with
    the parameters).  Three readings of "gradient":
     - the Jacobian dF(q, tau)/d theta_j, per parameter, to 1e-4 of its max norm;
     - the gradient of sum_tau F (a cotangent of one sign), to 1e-4 relative;
     - a vector-Jacobian product with a random-sign cotangent g, to 1e-4 of the size of its
       terms, sum |g| |dF/d theta_j|: its value can cancel to any degree (here ~100x), which is
       a property of the cotangent, not of the adjoint."""
    wl = W.tiny(seed=25, nq=1, kernel="fxc_model", nw=64, T_ev=4.0, eta_ev=0.6, kmesh=(3, 3, 3),
                nbands=10, nG=9)
    tau = response.tau_grid(wl.T, 10)
    gF = np.random.default_rng(3).standard_normal((wl.nq, len(tau)))
    ones = np.ones((wl.nq, len(tau)))
    c = _ctx(wl, prec)
    _, J = c.jacobian(tau)
    g_rand = c.itcf_vjp(tau, gF)
    g_sum = c.itcf_vjp(tau, ones)
    c.close()
    for j, h in enumerate([1e-4 * wl.T, 1e-4 * wl.eta, 1e-4, 1e-4, 1e-4]):
        fd = _fd_fp64_jacobian(wl, tau, j, h)
        assert np.abs(J[:, :, j] - fd).max() <= 1e-4 * np.abs(fd).max(), (prec, j)
        assert abs(g_sum[j] - fd.sum()) <= 1e-4 * abs(fd.sum()), (prec, j, g_sum[j], fd.sum())
        assert abs(g_rand[j] - np.sum(gF * fd)) <= 1e-4 * np.sum(np.abs(gF * fd)), (prec, j)


def test_fp64_gradient_against_central_differences():
    wl = W.tiny(**CASES["tr_model"])
    tau = response.tau_grid(wl.T, 8)
    gF = np.random.default_rng(4).standard_normal((wl.nq, len(tau)))
    c = _ctx(wl, "fp64")
    grad = c.itcf_vjp(tau, gF)
    c.close()
    for j, h in enumerate([1e-4 * wl.T, 1e-4 * wl.eta, 1e-4, 1e-4, 1e-4]):
        fd = _fd_fp64(wl, tau, gF, j, h)
        assert abs(grad[j] - fd) <= 1e-6 * abs(fd), (j, grad[j], fd)


def test_vjps_are_contracted_jacobians():
    wl = W.tiny(**CASES["tr_model"])
    tau = response.tau_grid(wl.T, 7)
    c = _ctx(wl)
    dS, dF = c.jacobian(tau)
    rng = np.random.default_rng(5)
    gF = rng.standard_normal((wl.nq, len(tau)))
    gS = rng.standard_normal((wl.nq, wl.nw))
    np.testing.assert_allclose(c.itcf_vjp(tau, gF), np.einsum("qt,qtj->j", gF, dF), rtol=1e-12, atol=0)
    np.testing.assert_allclose(c.dsf_vjp(gS), np.einsum("qw,qwj->j", gS, dS), rtol=1e-12, atol=0)
    c.close()


def test_set_params_equals_fresh_context():
    wl = W.tiny(**CASES["tr_model"])
    wl2 = wl.replace(T=1.3 * wl.T, eta=0.8 * wl.eta, fxc_params=(0.7, 0.3, 0.02))
    tau = response.tau_grid(wl2.T, 9)
    a = _ctx(wl)
    a.set_params(wl2.T, wl2.eta, fxc_params=wl2.fxc_params)
    a.chi0_assemble()
    a.dyson_solve()
    Fa, _ = a.itcf(tau)
    Sa = a.dsf()
    b = _ctx(wl2)
    Fb, _ = b.itcf(tau)
    Sb = b.dsf()
    a.close()
    b.close()
    np.testing.assert_allclose(Fa, Fb, rtol=1e-12)
    assert np.abs(Sa - Sb).max() <= 1e-12 * np.abs(Sb).max()


def test_set_params_invalidates_results():
    wl = W.tiny(**CASES["tr_model"])
    c = _ctx(wl)
    c.set_params(wl.T, wl.eta)
    with pytest.raises(binding.LrtError):
        c.dsf()
    c.close()


def test_autograd_wrapper_returns_library_vjp():
    torch = pytest.importorskip("torch")
    from paper_2510_01875_gb300 import autograd as AG
    wl = W.tiny(**CASES["tr_model"])
    tau = response.tau_grid(wl.T, 6)
    c = binding.Context(wl, "fp64")
    theta = torch.tensor([wl.T, wl.eta, *wl.fxc_params], dtype=torch.float64, requires_grad=True)
    F = AG.itcf(theta, c, tau)
    wts = torch.linspace(0.5, 1.5, F.numel(), dtype=torch.float64).reshape(F.shape)
    (F * wts).sum().backward()
    ref = c.itcf_vjp(tau, wts.numpy())
    np.testing.assert_allclose(theta.grad.numpy(), ref, rtol=1e-12)
    # S wrapper, after another forward moved the context: backward restores its own state
    theta2 = torch.tensor([wl.T, wl.eta, *wl.fxc_params], dtype=torch.float64, requires_grad=True)
    S = AG.dsf(theta2, c)
    AG.itcf(theta.detach() * 1.01, c, tau)
    S.sum().backward()
    c.set_params(wl.T, wl.eta, fxc_params=wl.fxc_params)
    c.chi0_assemble()
    c.dyson_solve()
    np.testing.assert_allclose(theta2.grad.numpy(), c.dsf_vjp(np.ones((wl.nq, wl.nw))), rtol=1e-12)
    c.close()
