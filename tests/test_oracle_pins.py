"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: exact
rational algebra, polynomial exactness, the discrete dispersion relation,
the 3-D free-space Green's function, discrete energy conservation, the
von Neumann stability bound, the adjoint dot-product identity and finite
differences of the misfit.
"""
from fractions import Fraction

import numpy as np
import pytest

from paper_2502_12350_gb300 import synth


def _solve_rational(M, rhs):
    n = len(M)
    A = [row[:] + [r] for row, r in zip(M, rhs)]
    for c in range(n):
        p = next(r for r in range(c, n) if A[r][c] != 0)
        A[c], A[p] = A[p], A[c]
        for r in range(n):
            if r != c and A[r][c] != 0:
                f = A[r][c] / A[c][c]
                A[r] = [a - f * b for a, b in zip(A[r], A[c])]
    return [A[i][n] / A[i][i] for i in range(n)]


def test_fd_coefficients_solve_taylor_system(oracle):
    """Sec. 2.1 (eighth order in space, radius 4): the symmetric weights
    c_0..c_4 are the unique solution of sum_k c_|k| k^p = 2 delta_{p,2} for
    even p <= 8, solved here in exact rational arithmetic."""
    M = [[Fraction(1 if p == 0 else 0)] + [Fraction(2 * k**p) for k in range(1, 5)]
         for p in range(0, 9, 2)]
    M[0][0] = Fraction(1)
    rhs = [Fraction(2 if p == 2 else 0) for p in range(0, 9, 2)]
    c = _solve_rational(M, rhs)
    assert c == [Fraction(-205, 72), Fraction(8, 5), Fraction(-1, 5), Fraction(8, 315),
                 Fraction(-1, 560)]
    np.testing.assert_array_equal(oracle.fd_coeffs(), np.array([float(x) for x in c]))


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_laplacian_exact_on_polynomials(oracle, axis):
    """The stencil differentiates x^p exactly for p <= 9 (eighth order) and
    not for p = 10, away from the zero exterior.  Errors are measured on the
    rounding scale max|u|/h^2."""
    sp = (0.7, 0.9, 1.3)
    g = oracle.make_grid(6, 7, 8, 6, 1.0, 1e-3, 1, spacing=sp)
    Nz, Ny, Nx = oracle.padded_shape(g)
    n_ax = (Nx, Ny, Nz)[axis]
    h = sp[axis]
    x1 = (np.arange(n_ax) - (n_ax - 1) / 2) * h
    shape = [1, 1, 1]
    shape[2 - axis] = n_ax
    X = np.broadcast_to(x1.reshape(shape), (Nz, Ny, Nx))
    inner = (slice(4, -4),) * 3
    for p in range(0, 11):
        u = np.ascontiguousarray(X**p)
        exact = p * (p - 1) * X ** max(p - 2, 0) if p >= 2 else np.zeros_like(X)
        got = oracle.laplacian(g, u)[inner]
        err = np.abs(got - exact[inner]).max() / (np.abs(u).max() / h**2)
        if p <= 9:
            assert err < 1e-12, (p, err)
        else:
            assert err > 1e-8, (p, err)


def test_stability_bound_matches_von_neumann(oracle):
    """Leapfrog with the 3-D radius-4 stencil is stable iff
    (c dt/h)^2 * 3 * max_theta(-c0 - 2 sum c_j cos j theta) <= 4; the bound
    0.4529 is derived here from the symbol, and the oracle grows without
    bound just above it and stays bounded just below it (sponge off)."""
    c = oracle.fd_coeffs()
    theta = np.linspace(0, np.pi, 200001)
    sym = -(c[0] + 2 * sum(c[j] * np.cos(j * theta) for j in range(1, 5)))
    lam = 3 * sym.max()
    bound = 2 / np.sqrt(lam)
    assert abs(bound - 0.45286) < 1e-4
    n, h = 20, 10.0
    rng = np.random.default_rng(0)
    for courant, grows in ((0.97 * bound, False), (1.05 * bound, True)):
        dt = courant * h / 2000.0
        g = oracle.make_grid(n, n, n, 0, h, dt, 1, cerjan=0.0)
        vel = np.full((n, n, n), 2000.0)
        u0 = rng.standard_normal((n, n, n))
        up, uc = oracle.advance(g, vel, u0, u0, 300)
        ratio = np.abs(uc).max() / np.abs(u0).max()
        assert (ratio > 1e3) == grows, (courant, ratio)


def test_plane_wave_dispersion_relation(oracle):
    """A discrete plane wave cos(k.x - w n dt) with
    (2/dt)^2 sin^2(w dt/2) = c^2 sum_a (-c0 - 2 sum_j c_j cos(j k_a h))/h^2
    is advanced exactly by the scheme, away from the boundary."""
    c = oracle.fd_coeffs()
    n, h, cv, dt, steps = 56, 10.0, 2500.0, 1.5e-3, 5
    kvec = np.array([0.9, -0.6, 0.45]) * np.pi / (6 * h)
    s = sum(-c[0] - 2 * sum(c[j] * np.cos(j * ka * h) for j in range(1, 5)) for ka in kvec) / h**2
    w = 2 / dt * np.arcsin(np.sqrt(cv**2 * s) * dt / 2)
    g = oracle.make_grid(n, n, n, 0, h, dt, 1, cerjan=0.0)
    z, y, x = np.meshgrid(*(np.arange(n) * h,) * 3, indexing="ij")
    phase = kvec[0] * x + kvec[1] * y + kvec[2] * z
    u_m1, u_0 = np.cos(phase + w * dt), np.cos(phase)
    up, uc = oracle.advance(g, np.full((n, n, n), cv), u_m1, u_0, steps)
    exact = np.cos(phase - w * steps * dt)
    m = 4 * steps + 1
    inner = (slice(m, -m),) * 3
    assert np.abs(uc[inner] - exact[inner]).max() < 1e-10
    # and the continuous dispersion relation would not match: the test has teeth
    w_cont = cv * np.linalg.norm(kvec)
    assert abs(w_cont - w) * steps * dt > 1e-6


def test_greens_function_homogeneous(oracle):
    """Eq. 1 with S = f(t) delta(x - x_S): in a homogeneous medium the
    pressure is f(t - r/c) / (4 pi c^2 r) at every distance (the scalar 3-D
    wave equation has no near-field term).  Recorded sample d[n] is taken
    from u^{n+1}, so it is compared with f((n+1) dt - r/c).  An 8 Hz Ricker
    at c = 2000 m/s and h = 10 m has at least 10 points per wavelength up to
    2.5 times its peak frequency, where the eighth-order scheme's dispersion
    error is about 1e-3; the walls are far enough (no sponge) that no
    reflection reaches a receiver inside the compared window."""
    n, b, h, dt, nt, cv, f = 48, 28, 10.0, 1e-3, 360, 2000.0, 8.0
    g = oracle.make_grid(n, n, n, b, h, dt, nt, cerjan=0.0)
    vel = np.full((n, n, n), cv)
    c = n // 2
    src = np.array([[c * h, c * h, c * h]])
    offs = np.array([10, 13, 16])
    rec = np.array([[(c + o) * h, c * h, c * h] for o in offs] +
                   [[c * h, c * h, (c - 12) * h]])
    amp = 1e5
    w = synth.ricker(nt, dt, f, amp).astype(np.float64)
    seis = oracle.model(g, vel, src, w, [0, len(rec)], rec)
    r_all = list(offs * h) + [12 * h]
    t = (np.arange(nt) + 1) * dt
    for tr, r in zip(seis, r_all):
        # the nearest reflection (wall at c + b cells) arrives after the window
        assert (2 * (c + b) - r / h) * h / cv > r / cv + 2.2 / f
        tau = t - r / cv - 1.0 / f
        arg = (np.pi * f * tau) ** 2
        exact = amp * (1 - 2 * arg) * np.exp(-arg) / (4 * np.pi * cv**2 * r)
        win = t < (r / cv + 2.2 / f)
        rel = np.linalg.norm(tr[win] - exact[win]) / np.linalg.norm(exact[win])
        assert rel < 1.5e-3, (r, rel)


def test_uniform_density_equals_constant_density(oracle):
    """Eq. 1: with rho = rho0 everywhere the mass term vanishes, the source
    term is divided by sqrt(rho0) and the recorded pressure is sqrt(rho0) q,
    so the seismograms equal the constant-density ones for any rho0 != 1
    (a factor applied on one side only, or rho used for sqrt(rho) on one
    side, breaks this)."""
    w = _tiny(False, nt=50, seed=4)
    g = oracle.make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, w.nt)
    d0 = oracle.model(g, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz)
    for rho0 in (2300.0, 0.37):
        rho = np.full(w.vel.shape, rho0)
        d1 = oracle.model(g, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, rho=rho)
        assert np.linalg.norm(d1 - d0) <= 1e-12 * np.linalg.norm(d0), rho0


@pytest.mark.parametrize("density", [False, True])
def test_source_receiver_reciprocity(oracle, density):
    """Reciprocity of the variable-density acoustic equation
    p_tt = rho c^2 div(grad(p) / rho) + f delta(x - x_s), whose q = p/sqrt(rho)
    form is Eq. 1 (right): rho c^2 times its source term makes the operator
    symmetric, so the pressure recorded at B from a source at A, times
    rho(A) c(A)^2, equals the pressure recorded at A from a source at B, times
    rho(B) c(B)^2.  The discrete scheme keeps this exactly (without sponge):
    its step is similar to a symmetric one through diag(c dt), and the source
    and receiver scales are 1/sqrt(rho) and sqrt(rho).  Dropping both
    sqrt(rho) factors, or using rho for sqrt(rho) on both sides, breaks it."""
    w = synth.small_case(seed=21, nx=14, ny=13, nz=12, border=4, nt=70, density=True,
                         n_src=1, n_rec=1, fpeak=30.0)
    rng = np.random.default_rng(8)
    vel = w.vel.astype(np.float64) * rng.uniform(0.9, 1.1, w.vel.shape)
    rho = (synth.gardner_density(vel).astype(np.float64) * rng.uniform(0.6, 1.6, vel.shape)
           if density else None)
    g = oracle.make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, w.nt, cerjan=0.0)
    a, b = np.array([3, 4, 5]), np.array([10, 8, 7])  # (x, y, z) nodes
    if density:
        rho[a[2], a[1], a[0]] *= 1.8  # a clearly different density at the two ends
    xa, xb = (a * w.h)[None, :], (b * w.h)[None, :]
    d_ab = oracle.model(g, vel, xa, w.wavelet, [0, 1], xb, rho=rho)[0]
    d_ba = oracle.model(g, vel, xb, w.wavelet, [0, 1], xa, rho=rho)[0]
    za = lambda p: (p[2], p[1], p[0])
    ka = vel[za(a)] ** 2 * (1.0 if rho is None else rho[za(a)])
    kb = vel[za(b)] ** 2 * (1.0 if rho is None else rho[za(b)])
    assert np.abs(d_ab).max() > 0
    np.testing.assert_allclose(d_ab * ka, d_ba * kb, rtol=0, atol=1e-11 * np.abs(d_ab * ka).max())
    if density:  # the identity is not the constant-density one
        assert abs(ka / kb - (vel[za(a)] / vel[za(b)]) ** 2) > 0.05 * ka / kb


@pytest.mark.parametrize("density", [False, True])
def test_gn_jacobian_column_matches_finite_differences(oracle, density):
    """One column of the Jacobian behind the Gauss-Newton diagonal:
    d d_r[m] / d c(x) = 2 c dt^2 sum_n G_{r,x}[m - n] a^n(x), with a^n the
    source-side term from ``forward_terms`` and G the impulse response from
    ``cell_response``, against central differences of the modelled data with
    respect to the velocity at one interior cell (first nt samples)."""
    from oracle import gn
    w = synth.small_case(seed=31, nx=9, ny=8, nz=8, border=4, nt=45, density=density,
                         n_src=1, n_rec=3, fpeak=40.0)
    g = oracle.make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, w.nt)
    vel = w.vel.astype(np.float64)
    rho = None if w.rho is None else w.rho.astype(np.float64)
    cell = (4, 3, 5)  # (x, y, z), not on the outermost model layer
    zyx = (cell[2], cell[1], cell[0])
    a = gn.forward_terms(g, vel, rho, w.src_xyz, w.wavelet, 0)[:, zyx[0], zyx[1], zyx[2]]
    G = gn.cell_response(g, vel, rho, cell, w.rec_xyz)
    nt = w.nt
    col = np.zeros_like(G)
    for m in range(nt):
        col[:, m] = sum(G[:, m - n] * a[n] for n in range(m + 1))
    col *= 2.0 * vel[zyx] * w.dt**2
    eps = 1e-4 * vel[zyx]
    vp, vm = vel.copy(), vel.copy()
    vp[zyx] += eps
    vm[zyx] -= eps
    dp = oracle.model(g, vp, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, rho=rho)
    dm = oracle.model(g, vm, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, rho=rho)
    fd = (dp - dm) / (2 * eps)
    assert np.abs(col).max() > 0
    np.testing.assert_allclose(col, fd, rtol=0, atol=1e-6 * np.abs(fd).max())
    # The label at that cell is the sum of squares of the whole column (the
    # Born data over the full linear-convolution length 2 nt - 1, summed over
    # the receivers), which ties the oracle's chain-rule factor to the one the
    # finite differences just checked.
    full = np.zeros((G.shape[0], 2 * nt - 1))
    for n in range(nt):
        full[:, n:n + nt] += G * a[n]
    full *= 2.0 * vel[zyx] * w.dt**2
    H = gn.separable(g, vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, rho=rho)
    np.testing.assert_allclose(H[zyx], np.sum(full**2), rtol=1e-9)


@pytest.mark.parametrize("density", [False, True])
def test_energy_conserved_without_sponge(oracle, density):
    """With g == 1, Dirichlet walls and no source the discrete energy
    <A^-1 (u^{n+1}-u^n), u^{n+1}-u^n> - <u^{n+1}, (lap - m2) u^n> is
    constant (the scheme is symplectic because lap is symmetric)."""
    n, h, dt = 18, 10.0, 1e-3
    rng = np.random.default_rng(1)
    vel = rng.uniform(1800, 3000, (n, n, n))
    rho = synth.gardner_density(vel).astype(np.float64) * rng.uniform(0.9, 1.1, (n, n, n)) if density else None
    g = oracle.make_grid(n, n, n, 3, h, dt, 1, cerjan=0.0)
    A, m2, gg, _ = oracle.prepare(g, vel, rho)
    assert np.all(gg == 1.0)
    shp = A.shape
    u0 = rng.standard_normal(shp)
    u1 = u0 + 0.01 * rng.standard_normal(shp)
    energies = []
    up, uc = u0, u1
    for _ in range(6):
        up, uc = oracle.advance(g, vel, up, uc, 7, rho=rho)
        un, un1 = up, uc  # u^{n}, u^{n+1} after the call
        Lu = oracle.laplacian(g, un) - m2 * un
        d = un1 - un
        energies.append(np.sum(d * d / A) - np.sum(un1 * Lu))
    e = np.array(energies)
    assert np.abs(e - e[0]).max() / abs(e[0]) < 1e-11


def _tiny(density, nt=40, seed=3):
    return synth.small_case(seed=seed, nx=12, ny=11, nz=10, border=5, nt=nt, density=density,
                            n_src=2, n_rec=5, fpeak=30.0)


@pytest.mark.parametrize("density", [False, True])
def test_adjoint_dot_product(oracle, density):
    """<F w, r> = <w, F^T r> for the linear map wavelet -> seismograms, with
    F^T r taken from the multiplier recursion of the gradient (the residual
    is made equal to r by choosing d_obs = F w - r)."""
    w = _tiny(density)
    g = oracle.make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, w.nt)
    rng = np.random.default_rng(5)
    wav = rng.standard_normal(w.nt)
    r = rng.standard_normal((int(w.rec_offset[-1]), w.nt))
    Fw = oracle.model(g, w.vel, w.src_xyz, wav, w.rec_offset, w.rec_xyz, rho=w.rho)
    _, _, FTr = oracle.gradient(g, w.vel, w.src_xyz, wav, w.rec_offset, w.rec_xyz, Fw - r,
                                rho=w.rho, return_dwav=True)
    w2 = rng.standard_normal(w.nt)
    Fw2 = oracle.model(g, w.vel, w.src_xyz, w2, w.rec_offset, w.rec_xyz, rho=w.rho)
    lhs, rhs = np.sum(Fw2 * r), np.sum(w2 * FTr)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs))


@pytest.mark.parametrize("density", [False, True])
def test_gradient_matches_finite_differences(oracle, density):
    """Central differences of J = 1/2 |d(c) - d_obs|^2 along a perturbation
    that vanishes on the outermost model layer agree with <grad J, dc> with
    an error that falls as eps^2."""
    w = _tiny(density)
    g = oracle.make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, w.nt)
    rng = np.random.default_rng(7)
    vel = w.vel.astype(np.float64)
    dobs = oracle.model(g, vel * (1 + 0.03 * rng.standard_normal(vel.shape)), w.src_xyz,
                        w.wavelet, w.rec_offset, w.rec_xyz, rho=w.rho)
    J0, grad = oracle.gradient(g, vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, dobs,
                               rho=w.rho)
    dc = np.zeros_like(vel)
    dc[1:-1, 1:-1, 1:-1] = rng.standard_normal(tuple(s - 2 for s in vel.shape))
    dc *= 50.0

    def J(v):
        d = oracle.model(g, v, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, rho=w.rho)
        return 0.5 * np.sum((d - dobs) ** 2)

    pred = np.sum(grad * dc)
    errs = []
    for eps in (1e-1, 1e-2, 1e-3):
        fd = (J(vel + eps * dc) - J(vel - eps * dc)) / (2 * eps)
        errs.append(abs(fd - pred) / abs(pred))
    assert errs[-1] < 1e-6, errs
    assert errs[1] < errs[0] * 0.05, errs


def test_gradient_bitwise_invariant_to_snapshot_mode(oracle):
    """All stored states vs checkpoint-and-recompute at several intervals
    give bitwise identical misfit and gradient."""
    w = _tiny(True, nt=37)
    g = oracle.make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, w.nt)
    dobs = np.zeros((int(w.rec_offset[-1]), w.nt))
    ref = oracle.gradient(g, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, dobs, rho=w.rho)
    for every in (1, 5, 16, 36):
        got = oracle.gradient(g, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, dobs,
                              rho=w.rho, snap_every=every)
        assert got[0] == ref[0]
        np.testing.assert_array_equal(got[1], ref[1])


def test_misfit_is_half_sum_of_squares(oracle):
    w = _tiny(False, nt=20)
    g = oracle.make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, w.nt)
    d = oracle.model(g, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz)
    rng = np.random.default_rng(2)
    dobs = d + rng.standard_normal(d.shape)
    J, _, seis = oracle.gradient(g, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, dobs,
                                 return_seis=True)
    np.testing.assert_array_equal(seis, d)
    assert abs(J - 0.5 * np.sum((d - dobs) ** 2)) < 1e-12 * J


def test_sponge_profile_and_coefficients(oracle):
    """Cerjan damping: per-axis exp(-(alpha d)^2) for depth d into the
    sponge, product over axes; A = c^2 dt^2 with edge-replicated c; m2 = 0
    for constant density and for a constant-density model with rho given."""
    nx, ny, nz, b = 5, 6, 7, 4
    g = oracle.make_grid(nx, ny, nz, b, 10.0, 1e-3, 1, cerjan=0.05)
    rng = np.random.default_rng(0)
    vel = rng.uniform(1500, 3000, (nz, ny, nx))
    A, m2, gg, sr = oracle.prepare(g, vel, np.full((nz, ny, nx), 2000.0))
    prof = lambda N: np.array([np.exp(-(0.05 * (b - i if i < b else (i - (N - 1 - b) if i > N - 1 - b else 0))) ** 2)
                               for i in range(N)])
    expect = prof(nz + 2 * b)[:, None, None] * prof(ny + 2 * b)[None, :, None] * prof(nx + 2 * b)[None, None, :]
    np.testing.assert_allclose(gg, expect, rtol=1e-15)
    assert gg[b:-b, b:-b, b:-b].min() == 1.0
    cpad = np.pad(vel, b, mode="edge")
    np.testing.assert_allclose(A, cpad**2 * 1e-6, rtol=1e-15)
    assert np.abs(m2).max() < 1e-12
    np.testing.assert_allclose(sr, np.sqrt(2000.0), rtol=1e-15)


def test_density_mass_term_closed_form(oracle):
    """m2 = lap(sqrt rho)/sqrt rho: for sqrt(rho) = exp(a x) the continuous
    value is a^2; the eighth-order stencil reproduces it to O(h^8)."""
    n, b, h = 16, 4, 10.0
    g = oracle.make_grid(n, n, n, b, h, 1e-3, 1)
    a = 0.004
    x = np.arange(n) * h
    srho = np.exp(a * x)[None, None, :] * np.ones((n, n, 1))
    _, m2, _, _ = oracle.prepare(g, np.full((n, n, n), 2000.0), srho**2)
    inner = m2[b + 4:-b - 4, b + 4:-b - 4, b + 4:-b - 4]
    np.testing.assert_allclose(inner, a * a, rtol=1e-8)


def test_fp32_mode_close_to_fp64(oracle):
    w = _tiny(True, nt=60)
    g = oracle.make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, w.nt)
    d64 = oracle.model(g, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, rho=w.rho)
    d32 = oracle.model(g, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, rho=w.rho,
                       precision=32)
    rel = np.linalg.norm(d32 - d64) / np.linalg.norm(d64)
    assert 0 < rel < 1e-5


def test_pseudo_hessian_brute_force(oracle):
    """P(x) = sum_n (g (lap - m2) u^n)^2 equals the sum of squares of the
    source-side Jacobian factor formed from stored wavefields with the
    oracle's own Laplacian (brute force on a tiny grid)."""
    w = _tiny(True, nt=15)
    w.src_xyz = w.src_xyz[:1]
    w.rec_offset = w.rec_offset[:2]
    w.rec_xyz = w.rec_xyz[: w.rec_offset[1]]
    g = oracle.make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, w.nt)
    _, ph = oracle.model(g, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, rho=w.rho,
                         phess=True)
    A, m2, gg, sr = oracle.prepare(g, w.vel, w.rho)
    # replay the wavefield with advance() plus manual source injection
    shp = A.shape
    b = w.border
    si = (np.floor(w.src_xyz[0] / w.h + 0.5).astype(int) + b)
    P = np.zeros(shp)
    up, uc = np.zeros(shp), np.zeros(shp)
    for n in range(w.nt):
        a = gg * (oracle.laplacian(g, uc) - m2 * uc)
        P += a * a
        up, uc = oracle.advance(g, w.vel, up, uc, 1, rho=w.rho)
        uc[si[2], si[1], si[0]] += w.dt**2 * float(w.wavelet[n]) / (w.h**3 * sr[si[2], si[1], si[0]])
    np.testing.assert_allclose(ph, P[b:-b, b:-b, b:-b], rtol=1e-12, atol=1e-300)


def test_aperture_windows(oracle):
    """A shot confined to an aperture window: (a) an aperture spanning the
    whole model is the unwindowed problem, bitwise; (b) by the finite domain
    of dependence of the radius-4 stencil (4 cells per step), a receiver d
    cells inside the window sponge's inner edge sees exactly the full-model
    data for the first floor(d/4) - 1 steps, and different data later."""
    w = synth.small_case(seed=14, nx=40, ny=36, nz=14, border=4, nt=90, density=True, n_src=1,
                         n_rec=3, fpeak=40.0)
    g = oracle.make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, w.nt)
    w.src_xyz = np.array([[20 * w.h, 18 * w.h, 6 * w.h]], np.float32)
    w.rec_xyz = np.array([[20 * w.h, 18 * w.h, 3 * w.h], [22 * w.h, 18 * w.h, 6 * w.h],
                          [20 * w.h, 20 * w.h, 8 * w.h]], np.float32)
    full = oracle.model(g, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, rho=w.rho)
    whole = oracle.model(g, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, rho=w.rho,
                         aperture=[[0, w.nx, 0, w.ny]])
    np.testing.assert_array_equal(whole, full)
    ap = [[12, 28, 10, 26]]
    win = oracle.model(g, w.vel, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, rho=w.rho,
                       aperture=ap)
    # receivers are >= 6 cells inside the aperture (10 from the window's
    # Dirichlet wall): no difference can reach them in the first step, and
    # once the physical wave has reached the window sponge the data differ
    np.testing.assert_allclose(win[:, :2], full[:, :2], rtol=1e-12, atol=1e-30)
    assert np.abs(win - full).max() > 1e-6 * np.abs(full).max()
