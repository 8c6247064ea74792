"""GPU adjoint sweep (C ABI and torch.autograd.Function) against the oracle.

The oracle's gradients are autograd of its FP64 map, themselves pinned to
central differences in the CPU suite; here the GPU reverse sweep is compared
with them on the same seeded inputs, and with central differences of the
oracle at a larger size.  Bars: FP64 plans 1e-7 relative; FP32 plans 1e-3
relative (to the largest component for the map gradient).
"""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


def _grad_case(n=16, nz=12, tgrid=(5, 6, 7), p1=400.0, precision="f64"):
    w = W.depleted_absorbing(n=n, nz=nz, tgrid=tgrid, xi=2.0, p1=p1)
    return w.with_(t_off=0.3, ddk_dT=-60.0, dn_dT=3e-4, precision=precision)


def _oracle_grads(w):
    from oracle import ssfm
    dT = torch.tensor(w.dT, dtype=torch.float64, requires_grad=True)
    w0 = torch.tensor(w.w0, dtype=torch.float64, requires_grad=True)
    zf = torch.tensor(w.z_focus, dtype=torch.float64, requires_grad=True)
    to = torch.tensor(w.t_off, dtype=torch.float64, requires_grad=True)
    eta = ssfm.run(w, w0=w0, z_focus=zf, t_off=to, dT=dT)[2]
    g = torch.autograd.grad(eta, (w0, zf, to, dT))
    return float(eta.detach()), [float(x) for x in g[:3]], g[3].numpy()


def _gpu_grads(w):
    import paper_2410_04994_gb300 as pkg
    from paper_2410_04994_gb300.autograd import efficiency
    plan = pkg.Plan(w, adjoint=True)
    dT = torch.tensor(w.dT, dtype=torch.float64, device="cuda", requires_grad=True)
    w0 = torch.tensor(w.w0, dtype=torch.float64, requires_grad=True)
    zf = torch.tensor(w.z_focus, dtype=torch.float64, requires_grad=True)
    to = torch.tensor(w.t_off, dtype=torch.float64, requires_grad=True)
    eta = efficiency(plan, w0, zf, to, dT)
    eta.backward()
    return float(eta.detach()), [float(w0.grad), float(zf.grad), float(to.grad)], dT.grad.cpu().numpy()


def _check(w, tol):
    eta_o, g_o, gT_o = _oracle_grads(w)
    eta_g, g_g, gT_g = _gpu_grads(w)
    assert abs(eta_g / eta_o - 1) < max(tol, 1e-4)
    for a, b in zip(g_g, g_o):
        assert abs(a - b) <= tol * abs(b) + 1e-12, (g_g, g_o)
    scale = np.abs(gT_o).max()
    assert np.abs(gT_g - gT_o).max() <= tol * scale, np.abs(gT_g - gT_o).max() / scale
    # the oven offset enters as a uniform dT (trilinear weights sum to one)
    assert abs(g_g[2] - gT_g.sum()) <= 10 * tol * np.abs(gT_g).sum()
    return g_g, gT_g


def test_adjoint_fp64_matches_oracle_autograd():
    _check(_grad_case(precision="f64"), 1e-7)


def test_adjoint_fp32_matches_oracle_autograd():
    _check(_grad_case(n=32, nz=40, tgrid=(8, 8, 16), precision="f32"), 1e-3)


def test_adjoint_undepleted_fp64():
    _check(_grad_case(precision="f64").with_(undepleted=True), 1e-7)


def test_adjoint_single_step_fp64():
    # one z-step over the whole crystal: keep Gamma h and psi h small
    _check(_grad_case(nz=1, p1=10.0, precision="f64").with_(dn_dT=1e-6, ddk_dT=-0.6), 1e-7)


def test_adjoint_fp32_vs_oracle_central_differences():
    """64 x 64, nz = 200, absorbing losses: the FP32 reverse sweep against
    central differences (h = 1e-4 relative) of the FP64 oracle."""
    from oracle import ssfm
    w = W.adjoint_case(n=64, nz=200, tgrid=(16, 16, 32))
    w = w.with_(t_off=0.2, ddk_dT=-30.0, dn_dT=1e-4)
    eta_g, g_g, gT_g = _gpu_grads(w)
    dT0 = torch.tensor(w.dT, dtype=torch.float64)

    def eta(**kw):
        return float(ssfm.run(w, **kw)[2])

    def fd(fun, x, h):
        return (fun(x + h) - fun(x - h)) / (2 * h)

    ref = [fd(lambda v: eta(w0=v), w.w0, 1e-4 * w.w0),
           fd(lambda v: eta(z_focus=v), w.z_focus, 1e-4 * w.z_focus),
           fd(lambda v: eta(t_off=v), w.t_off, 1e-4)]
    for a, b in zip(g_g, ref):
        assert abs(a - b) <= 1e-3 * abs(b), (g_g, ref)
    rng = np.random.default_rng(11)
    d = torch.tensor(rng.normal(size=tuple(dT0.shape)))
    dirder = fd(lambda s: eta(dT=dT0 + s * d), 0.0, 1e-3)
    got = float((torch.tensor(gT_g, dtype=torch.float64) * d).sum())
    assert abs(got - dirder) <= 1e-3 * abs(dirder), (got, dirder)


@pytest.mark.slow
def test_adjoint_full_size_fp32_vs_fp64_and_invariant():
    """256 x 256, nz = 2000, 64 x 64 x 128 map with sqrt(nz) checkpointing.
    The FP32 and FP64 reverse sweeps agree to 1e-3, and dJ/dT_off equals the
    sum of the node gradients in both."""
    w = W.adjoint_case()
    eta32, g32, gT32 = _gpu_grads(w)
    eta64, g64, gT64 = _gpu_grads(w.with_(precision="f64"))
    assert abs(eta32 / eta64 - 1) < 1e-4
    l1 = np.abs(gT64).sum()  # scale of dT-driven sensitivities (per kelvin)
    assert abs(g32[0] - g64[0]) <= 1e-3 * abs(g64[0])
    assert abs(g32[1] - g64[1]) <= 1e-3 * abs(g64[1])
    assert abs(g32[2] - g64[2]) <= 1e-3 * max(abs(g64[2]), l1)
    assert np.abs(gT32 - gT64).max() <= 1e-3 * np.abs(gT64).max()
    for g, gT in ((g32, gT32), (g64, gT64)):
        assert abs(g[2] - gT.sum()) <= 1e-3 * np.abs(gT).sum()


def test_autograd_with_plain_number_inputs():
    """Only w0 requires a gradient; z_focus and T_off are plain numbers and dT
    a tensor without grad: the backward returns no gradient for them, and
    w0's gradient equals the one of the all-tensor call."""
    import paper_2410_04994_gb300 as pkg
    from paper_2410_04994_gb300.autograd import efficiency
    w = _grad_case(precision="f64")
    _, g_all, _ = _gpu_grads(w)
    plan = pkg.Plan(w, adjoint=True)
    w0 = torch.tensor(w.w0, dtype=torch.float64, requires_grad=True)
    eta = efficiency(plan, w0, w.z_focus, w.t_off, torch.tensor(w.dT, device="cuda"))
    eta.backward()
    assert abs(float(w0.grad) - g_all[0]) <= 1e-12 * abs(g_all[0])
