"""The seeded synthetic inputs: the workloads have the sizes and distributions
stated for them (grids, z-steps, powers, focusing, temperature maps), and the
same seed gives the same inputs."""
import math

import numpy as np
import pytest

import workloads as W


def test_sweep_of_384_instances_on_three_grids():
    s = W.sweep_instances(with_maps=False)
    assert len(s) == 384
    sizes = [w.nx for w in s]
    assert sizes == [64] * 128 + [128] * 192 + [256] * 64
    assert all(w.ny == w.nx and w.nz == 2000 for w in s)
    assert sum(w.nx * w.ny for w in s) == 7_864_320          # grid points per z-step
    assert sum(w.point_steps for w in s) == 15_728_640_000
    p1 = np.array([w.p1 for w in s])
    toff = np.array([w.t_off for w in s])
    assert p1.min() >= 5.0 and p1.max() <= 60.0 and p1.std() > 10.0
    assert toff.min() >= -1.0 and toff.max() <= 1.0 and toff.std() > 0.4
    # xi = 0.3 * 20^(i/(n-1)) within each group: log-spaced from 0.3 to 6
    start = 0
    for n, count in W.SWEEP_GROUPS:
        g = s[start:start + count]
        xi = np.array([w.L / (w.w0 ** 2 * W.k_pump()) for w in g])   # L / (2 z_R)
        assert abs(xi[0] - 0.3) < 1e-12 and abs(xi[-1] - 6.0) < 1e-12
        assert np.allclose(np.diff(np.log(xi)), math.log(20.0) / (count - 1), rtol=1e-12)
        start += count
    # square window of ten entrance radii, focus at the centre, absorbing crystal
    for w in s[::37]:
        assert w.lx == w.ly
        assert abs(w.lx / (10 * W.beam_radius(0.0, w.w0, w.z_focus)) - 1) < 1e-12
        assert w.z_focus == w.L / 2
        assert (w.alpha_f, w.alpha_sh, w.beta_sh) == (W.ALPHA_F, W.ALPHA_SH, W.BETA_SH)
        assert (w.ddk_dT, w.dn_dT) == (W.DDK_DT, W.DN_DT)


def test_seeds_fix_the_inputs():
    a = W.sweep_instances(groups=((64, 3), (128, 2)))
    b = W.sweep_instances(groups=((64, 3), (128, 2)))
    c = W.sweep_instances(groups=((64, 3), (128, 2)), seed=2)
    for x, y in zip(a, b):
        assert x.p1 == y.p1 and x.t_off == y.t_off
        assert np.array_equal(x.dT, y.dT)
    assert not np.array_equal(a[0].dT, c[0].dT)
    assert a[0].p1 != c[0].p1


def test_temperature_map_recipe():
    """2 K exp(-2 r^2 / w(z)^2) + N(0, 0.01 K) on a 64 x 64 x 128 node grid over
    the field window and the crystal length."""
    w = W.sweep_instances(groups=((64, 2),))[1]
    assert w.dT.shape == (128, 64, 64) and w.dT.dtype == np.float32
    tz, ty, tx = w.dT.shape
    X = -w.t_lx / 2 + np.arange(tx) * w.t_lx / (tx - 1)
    Y = -w.t_ly / 2 + np.arange(ty) * w.t_ly / (ty - 1)
    Z = np.arange(tz) * w.L / (tz - 1)
    wz = np.array([W.beam_radius(z, w.w0, w.z_focus) for z in Z])
    r2 = X[None, None, :] ** 2 + Y[None, :, None] ** 2
    noise = w.dT - 2.0 * np.exp(-2.0 * r2 / wz[:, None, None] ** 2)
    n = noise.size
    assert abs(noise.mean()) < 4 * 0.01 / math.sqrt(n)
    assert abs(noise.std() / 0.01 - 1) < 0.02
    assert abs(float(w.dT.max()) - 2.0) < 0.06          # the peak on the axis at the focus


@pytest.mark.parametrize("name,n,nz,p1", [("depleted", 128, 1000, 50.0),
                                          ("adjoint", 256, 2000, 30.0),
                                          ("thermal", 1024, 8000, 100.0),
                                          ("plain", 32, 100, 10.0)])
def test_single_instance_workloads(name, n, nz, p1):
    w = W.full_size(name) if name != "depleted" else W.depleted_absorbing()
    assert (w.nx, w.ny, w.nz, w.p1) == (n, n, nz, p1)
    if name == "thermal":
        assert (w.hx, w.hy, w.hz, w.n_outer) == (128, 128, 256, 6)
        assert (w.wx, w.wy) == (2e-3, 1e-3)
    if name == "plain":
        assert w.precision == "f64" and w.dT is None and w.alpha_f == 0.0
    if name in ("depleted", "adjoint"):
        assert w.dT.shape == (128, 64, 64)
