"""Pins of the CPML oracle (the paper's convolutional PML boundary).

* With no damping and no frequency shift the memory variables stay zero and
  the scheme is the main one without sponge: the main oracle's traces, to
  rounding (nearest-node and trilinear sources and receivers, with and
  without a free surface).
* The gradient is the transpose of the modelling map: dot-product identity
  for wavelet -> traces, and central finite differences of the misfit.
* It absorbs: on a small grid, the error against a grid so large that no
  reflection reaches the receivers in the window is far below that of the
  Cerjan sponge of the same thickness.
* The layer's coefficients mean what they are for: the damping profile gives
  the continuous layer the nominal normal-incidence reflection R, and the
  recursion's b and c are the step integrals of the kernel whose transform
  is 1/s - 1 (quadrature).  A wrong factor or log base in the profile, a
  sign of c, or b without the frequency shift fails one of them.
"""
import numpy as np
import pytest

from oracle import cpml
from paper_2502_12350_gb300 import synth


def _tiny(density, nt=40, seed=3):
    return synth.small_case(seed=seed, nx=10, ny=9, nz=8, border=5, nt=nt, density=density,
                            n_src=2, n_rec=4, fpeak=30.0)


def _offgrid(w, seed):
    rng = np.random.default_rng(seed)
    w.src_xyz = w.src_xyz + rng.uniform(0.1, 0.9, w.src_xyz.shape) * w.h
    w.rec_xyz = w.rec_xyz + rng.uniform(0.1, 0.9, w.rec_xyz.shape) * w.h
    hi = (np.array([w.nx, w.ny, w.nz]) - 1) * w.h - 1e-3
    w.src_xyz = np.minimum(w.src_xyz, hi)
    w.rec_xyz = np.minimum(w.rec_xyz, hi)
    return w


def _below_surface(w):
    """Sources and receivers at least one plane below the top model plane."""
    w.src_xyz = w.src_xyz.copy()
    w.rec_xyz = w.rec_xyz.copy()
    w.src_xyz[:, 2] = np.maximum(w.src_xyz[:, 2], 2 * w.h)
    w.rec_xyz[:, 2] = np.maximum(w.rec_xyz[:, 2], 1 * w.h)
    return w


@pytest.mark.parametrize("density,xi,fs", [(False, 0, 0), (True, 0, 0), (True, 1, 0), (True, 0, 1),
                                           (False, 1, 1)])
def test_no_damping_is_the_main_scheme(oracle, density, xi, fs):
    w = _tiny(density)
    if xi:
        w = _offgrid(w, 8)
    if fs:
        w = _below_surface(w)
    g = oracle.make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, w.nt, cerjan=0.0, xyz_interp=xi,
                         free_surface=fs)
    ref = oracle.model(g, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, rho=w.rho)
    got = cpml.model(oracle, g, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, f0=0.0,
                     rho=w.rho, R=1.0)
    assert np.abs(ref).max() > 0
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("density,xi,fs", [(False, 0, 0), (True, 0, 0), (True, 1, 0), (True, 0, 1)])
def test_dot_product(oracle, density, xi, fs):
    w = _tiny(density, seed=4)
    if xi:
        w = _offgrid(w, 9)
    if fs:
        w = _below_surface(w)
    g = oracle.make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, w.nt, xyz_interp=xi,
                         free_surface=fs)
    rng = np.random.default_rng(5)
    wav = rng.standard_normal(w.nt)
    r = rng.standard_normal((int(w.rec_offset[-1]), w.nt))
    Fw = cpml.model(oracle, g, w.vel, w.src_xyz, wav, w.rec_offset, w.rec_xyz, f0=30.0, rho=w.rho)
    _, _, FTr = cpml.gradient(oracle, g, w.vel, w.src_xyz, wav, w.rec_offset, w.rec_xyz, Fw - r,
                              f0=30.0, rho=w.rho, return_dwav=True)
    w2 = rng.standard_normal(w.nt)
    Fw2 = cpml.model(oracle, g, w.vel, w.src_xyz, w2, w.rec_offset, w.rec_xyz, f0=30.0, rho=w.rho)
    lhs, rhs = np.sum(Fw2 * r), np.sum(w2 * FTr)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs))


@pytest.mark.parametrize("fs", [0, 1])
def test_gradient_matches_finite_differences(oracle, fs):
    w = _tiny(True, seed=6)
    if fs:
        w = _below_surface(w)
    g = oracle.make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, w.nt, free_surface=fs)
    rng = np.random.default_rng(7)
    vel = w.vel.astype(np.float64)
    dobs = cpml.model(oracle, g, vel * (1 + 0.03 * rng.standard_normal(vel.shape)), w.src_xyz,
                      w.wavelet, w.rec_offset, w.rec_xyz, f0=30.0, rho=w.rho)
    _, grad = cpml.gradient(oracle, g, vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, dobs,
                            f0=30.0, rho=w.rho)
    dc = np.zeros_like(vel)
    dc[1:-1, 1:-1, 1:-1] = rng.standard_normal(tuple(s - 2 for s in vel.shape)) * 50.0

    def J(v):
        d = cpml.model(oracle, g, v, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, f0=30.0,
                       rho=w.rho)
        return 0.5 * np.sum((d - dobs) ** 2)

    pred = np.sum(grad * dc)
    eps = 1e-3
    fd = (J(vel + eps * dc) - J(vel - eps * dc)) / (2 * eps)
    assert abs(fd - pred) <= 1e-6 * abs(pred)


def test_absorbs_better_than_the_sponge(oracle):
    """Receivers 4 cells from the model edge, 10-cell boundaries; the
    reference grid is 40 cells wider on every side (no reflection from it
    reaches the receivers in the window)."""
    n, b, h, dt, nt, cv, f = 24, 10, 10.0, 1e-3, 150, 2000.0, 25.0
    wav = synth.ricker(nt, dt, f).astype(np.float64)
    c = n // 2
    src = np.array([[c * h, c * h, c * h]])
    rec = np.array([[(n - 5) * h, c * h, c * h], [c * h, c * h, 4 * h], [3 * h, 3 * h, c * h]])
    vel = np.full((n, n, n), cv)
    g = oracle.make_grid(n, n, n, b, h, dt, nt)
    sponge = oracle.model(g, vel, src, wav, [0, 3], rec)
    pml = cpml.model(oracle, g, vel, src, wav, [0, 3], rec, f0=f)
    big, pad = n + 80, 40
    gb = oracle.make_grid(big, big, big, b, h, dt, nt, cerjan=0.0)
    ref = oracle.model(gb, np.full((big, big, big), cv), src + pad * h, wav, [0, 3],
                       rec + pad * h)
    e_sponge = np.linalg.norm(sponge - ref) / np.linalg.norm(ref)
    e_pml = np.linalg.norm(pml - ref) / np.linalg.norm(ref)
    # measured: sponge 2.5e-3, CPML 2.8e-6 relative error
    assert e_pml < 0.01 * e_sponge, (e_pml, e_sponge)
    assert e_pml < 1e-4, e_pml


def test_absorbs_with_a_free_surface(oracle):
    """Free surface on top, CPML on the other five faces: against a grid 40
    cells wider in x, y and below (the surface kept at the top model plane)
    the CPML traces err far less than those of the sponge."""
    n, b, h, dt, nt, cv, f = 24, 10, 10.0, 1e-3, 150, 2000.0, 25.0
    wav = synth.ricker(nt, dt, f).astype(np.float64)
    c = n // 2
    src = np.array([[c * h, c * h, 6 * h]])
    rec = np.array([[(n - 5) * h, c * h, 3 * h], [c * h, c * h, (n - 5) * h], [3 * h, 3 * h, 8 * h]])
    vel = np.full((n, n, n), cv)
    g = oracle.make_grid(n, n, n, b, h, dt, nt, free_surface=1)
    sponge = oracle.model(g, vel, src, wav, [0, 3], rec)
    pml = cpml.model(oracle, g, vel, src, wav, [0, 3], rec, f0=f)
    pad = 40
    bx, bz = n + 2 * pad, n + pad
    gb = oracle.make_grid(bx, bx, bz, b, h, dt, nt, cerjan=0.0, free_surface=1)
    shift = np.array([pad * h, pad * h, 0.0])
    ref = oracle.model(gb, np.full((bz, bx, bx), cv), src + shift, wav, [0, 3], rec + shift)
    e_sponge = np.linalg.norm(sponge - ref) / np.linalg.norm(ref)
    e_pml = np.linalg.norm(pml - ref) / np.linalg.norm(ref)
    assert e_pml < 0.01 * e_sponge, (e_pml, e_sponge)
    assert e_pml < 1e-4, e_pml


def _d_alpha(b, c, dt):
    """Damping d and frequency shift alpha recovered from the recursion's
    coefficients b = exp(-(d + alpha) dt), c = d (b - 1) / (d + alpha)."""
    s = -np.log(b) / dt
    d = np.where(s > 0, c * s / np.where(s > 0, b - 1.0, 1.0), 0.0)
    return d, s - d


def test_layer_reaches_the_nominal_reflection():
    """The damping profile is built for a nominal normal-incidence reflection
    R of the continuous layer, exp(-(2 / vmax) * integral of d over the layer)
    = R.  Integrating the oracle's d (recovered from its b and c) over a
    finely sampled layer gives back R, for several R and velocities."""
    from scipy.integrate import simpson
    B, h, dt, f0 = 400, 10.0, 1e-4, 15.0
    N = 2 * B + 10
    for R, vmax in ((1e-3, 3000.0), (1e-2, 1800.0), (1e-5, 4500.0)):
        b, cc = cpml.profiles(N, B, h, dt, vmax, f0, R)
        d, _ = _d_alpha(b, cc, dt)
        prof = np.concatenate([[0.0], d[N - B:]])  # inner edge (distance 0) to the outer face
        x = np.arange(B + 1) * h
        refl = np.exp(-2.0 / vmax * simpson(prof, x=x))
        assert abs(np.log(refl) / np.log(R) - 1.0) < 1e-4, (R, vmax, refl)
        # both faces carry the same layer
        np.testing.assert_allclose(d[:B][::-1], d[N - B:], rtol=1e-12)


def test_recursion_is_the_convolution_with_the_layer_kernel():
    """In the layer the derivative is (1/s) d/dx with s = 1 + d / (alpha + i w),
    and 1/s - 1 = -d / (d + alpha + i w) is the transform of the kernel
    -d exp(-(d + alpha) t) for t > 0.  With the field held constant over each
    step, the memory variable is the sum over past steps m of the kernel's
    integral over [m dt, (m + 1) dt], which must equal c b^m."""
    from scipy.integrate import quad
    B, h, dt, vmax, f0, R = 10, 12.5, 1e-3, 3500.0, 12.0, 1e-3
    N = 3 * B
    b, cc = cpml.profiles(N, B, h, dt, vmax, f0, R)
    d, alpha = _d_alpha(b, cc, dt)
    for i in (N - B, N - B // 2, N - 1, 0, B // 2):
        di, ai = d[i], alpha[i]
        assert di > 0 and ai >= 0
        kern = lambda t: -di * np.exp(-(di + ai) * t)
        # the kernel's Fourier transform is 1/s - 1 at a few frequencies
        for w in (0.0, 2 * np.pi * 7.0, 2 * np.pi * 30.0):
            re = quad(lambda t: kern(t) * np.cos(w * t), 0, np.inf, limit=400)[0]
            im = quad(lambda t: -kern(t) * np.sin(w * t), 0, np.inf, limit=400)[0]
            inv_s = (ai + 1j * w) / (ai + 1j * w + di)  # 1 / (1 + d / (alpha + i w))
            assert abs((re + 1j * im) - (inv_s - 1.0)) <= 1e-7 * abs(inv_s - 1.0)
        for m in range(6):
            want = quad(kern, m * dt, (m + 1) * dt)[0]
            assert abs(cc[i] * b[i] ** m - want) <= 1e-10 * abs(want), (i, m)
