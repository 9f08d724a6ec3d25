"""Convolutional PML (CPML) absorbing boundary (TEST INFRASTRUCTURE ONLY).

The paper's modelling offers two absorbing boundaries: damping (the Cerjan
sponge of the main oracle) and the convolutional perfectly matched layer
(Sec. 2, after Roden and Gedney).  This module restates the CPML scheme
plainly with sparse matrices, FP64; only tests and the CPU baseline use it.

Scheme (readings; the paper gives no formula).  In the layer every spatial
derivative d/dx_a becomes (1/s_a) d/dx_a with s_a = 1 + d_a / (alpha_a + i w),
and the second derivative (1/s_a) d/dx_a ((1/s_a) d/dx_a) is written with two
memory variables per axis, updated by recursive convolution:
    psi_a^n  = b_a psi_a^{n-1}  + c_a D1_a u^n
    zeta_a^n = b_a zeta_a^{n-1} + c_a (D2_a u^n + D1_a psi_a^n)
    x^n      = sum_a (D2_a u^n + D1_a psi_a^n + zeta_a^n)
    u^{n+1}  = (2 - A m2) u^n - u^{n-1} + A x^n  (+ source)
with b_a = exp(-(d_a + alpha_a) dt) and c_a = d_a (b_a - 1) / (d_a + alpha_a).
D2_a is the eighth-order second difference along axis a (the main scheme's
stencil, so x = lap u outside the layer), D1_a the eighth-order central first
difference (weights 4/5, -1/5, 4/105, -1/280), both with the field zero
outside the padded grid.  The layer is the `border` cells on each face;
at depth r = dist / border (dist = 1 .. border cells):
    d_a = d0 r^2,   d0 = -3 v_max ln(R) / (2 border h),   alpha_a = pi f0 (1 - r),
R = 1e-3 the nominal reflection coefficient and f0 the source's peak
frequency.  No sponge factor is applied (g = 1).  With a free surface
(g.free_surface) the top face has no layer, D2_z reads the negated mirror
planes above the surface (the main scheme's image method) and the field is
held at zero on and above it.  Density enters as in the
main scheme (A = c^2 dt^2, m2 = lap(sqrt rho) / sqrt rho, source / sqrt rho,
receivers sqrt rho u); sources and receivers are at their nearest nodes, or
(g.xyz_interp = 1) spread over the 8 nodes of their cell with trilinear
weights w_e, as in the main scheme: the source adds w_e dt^2 w[n] /
(h^3 sqrt rho_e) at node e and a receiver records sum_e w_e sqrt(rho_e) u_e.

The gradient is the exact transpose of this recursion (reverse mode, written
out step by step below), with dJ/dA = sum_n lam^{n+1} (x^n - m2 u^n) and
dJ/dc = 2 c dt^2 dJ/dA on the model interior.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

D1W = np.array([4.0 / 5.0, -1.0 / 5.0, 4.0 / 105.0, -1.0 / 280.0])


def _d2(n, h, c, zs=-1):
    """Second difference; with a free surface at zs a neighbour j <= zs reads
    the negated mirror plane 2 zs - j (the main scheme's image method)."""
    M = sp.lil_matrix((n, n))
    for i in range(n):
        M[i, i] += c[0]
        for m in range(1, 5):
            for j in (i - m, i + m):
                sign = 1.0
                if zs >= 0 and j <= zs:
                    j, sign = 2 * zs - j, -1.0
                if 0 <= j < n:
                    M[i, j] += sign * c[m]
    return (M / (h * h)).tocsr()


def _d1(n, h):
    M = sp.lil_matrix((n, n))
    for i in range(n):
        for m in range(1, 5):
            if i + m < n:
                M[i, i + m] = D1W[m - 1]
            if i - m >= 0:
                M[i, i - m] = -D1W[m - 1]
    return (M / h).tocsr()


def profiles(N, border, h, dt, vmax, f0, R=1e-3, low_face=True):
    """(b, c) of one padded axis of length N (low_face=False: no layer at the
    low end, the top face under a free surface)."""
    L = border * h
    d0 = -3.0 * vmax * np.log(R) / (2.0 * L) if border > 0 else 0.0
    dist = np.zeros(N)
    for i in range(N):
        if i < border:
            dist[i] = border - i if low_face else 0
        elif i > N - 1 - border:
            dist[i] = i - (N - 1 - border)
    r = dist / max(border, 1)
    d = np.where(dist > 0, d0 * r * r, 0.0)
    alpha = np.where(dist > 0, np.pi * f0 * (1.0 - r), 0.0)
    b = np.exp(-(d + alpha) * dt)
    c = np.where(d + alpha > 0, d * (b - 1.0) / np.where(d + alpha > 0, d + alpha, 1.0), 0.0)
    return b, c


class Operators:
    """Sparse operators and coefficients of the CPML scheme on a padded grid."""

    def __init__(self, oracle, g, vel, rho, f0, R=1e-3):
        A, m2, _, sr = oracle.prepare(g, vel, rho)
        self.shape = A.shape
        Nz, Ny, Nx = self.shape
        h, dt = g.dx, g.dt
        assert g.dx == g.dy == g.dz
        c = oracle.fd_coeffs()
        # free surface: the top model plane (padded plane zs = border)
        self.zs = g.border if getattr(g, "free_surface", 0) else -1
        I = [sp.identity(n, format="csr") for n in (Nz, Ny, Nx)]
        d2 = [_d2(Nz, h, c, self.zs), _d2(Ny, h, c), _d2(Nx, h, c)]
        d1 = [_d1(n, h) for n in (Nz, Ny, Nx)]
        # axis order a = 0: x, 1: y, 2: z (C order [z][y][x], x fastest)
        self.D2 = [sp.kron(sp.kron(I[0], I[1]), d2[2]).tocsr(),
                   sp.kron(sp.kron(I[0], d2[1]), I[2]).tocsr(),
                   sp.kron(sp.kron(d2[0], I[1]), I[2]).tocsr()]
        self.D1 = [sp.kron(sp.kron(I[0], I[1]), d1[2]).tocsr(),
                   sp.kron(sp.kron(I[0], d1[1]), I[2]).tocsr(),
                   sp.kron(sp.kron(d1[0], I[1]), I[2]).tocsr()]
        self.D2T = [D.T.tocsr() for D in self.D2]
        vmax = float(np.max(vel))
        bc = [profiles(Nx, g.border, h, dt, vmax, f0, R), profiles(Ny, g.border, h, dt, vmax, f0, R),
              profiles(Nz, g.border, h, dt, vmax, f0, R, low_face=self.zs < 0)]
        # the field is held at zero on and above a free surface
        live = np.ones(self.shape)
        if self.zs >= 0:
            live[: self.zs + 1] = 0.0
        self.live = live.ravel()
        ones = np.ones(self.shape)
        self.b = [(bc[0][0][None, None, :] * ones).ravel(),
                  (bc[1][0][None, :, None] * ones).ravel(),
                  (bc[2][0][:, None, None] * ones).ravel()]
        self.c = [(bc[0][1][None, None, :] * ones).ravel(),
                  (bc[1][1][None, :, None] * ones).ravel(),
                  (bc[2][1][:, None, None] * ones).ravel()]
        self.A = A.ravel()
        self.m2 = m2.ravel()
        self.Bc = 2.0 - self.A * self.m2
        self.sr = sr.ravel()
        self.g = g

    def _index(self, i, j, k):
        g = self.g
        if not (0 <= i < g.nx and 0 <= j < g.ny and 0 <= k < g.nz):
            raise ValueError("point outside the model")
        b = g.border
        Nz, Ny, Nx = self.shape
        return ((k + b) * Ny + (j + b)) * Nx + (i + b)

    def points(self, xyz):
        """[(padded node, weight)]: the nearest node, or the trilinear
        weights of the cell holding the point (zero weights dropped)."""
        g = self.g
        f = [(xyz[0] - g.ox) / g.dx, (xyz[1] - g.oy) / g.dy, (xyz[2] - g.oz) / g.dz]
        if not getattr(g, "xyz_interp", 0):
            return [(self._index(*[int(np.floor(v + 0.5)) for v in f]), 1.0)]
        base = [int(np.floor(v)) for v in f]
        t = [v - b for v, b in zip(f, base)]
        out = []
        for di in (0, 1):
            for dj in (0, 1):
                for dk in (0, 1):
                    w = ((t[0] if di else 1 - t[0]) * (t[1] if dj else 1 - t[1]) *
                         (t[2] if dk else 1 - t[2]))
                    if w != 0.0:
                        out.append((self._index(base[0] + di, base[1] + dj, base[2] + dk), w))
        return out


def _shot(op, src_xyz, s, rec_offset, rec_xyz):
    """Source nodes and scales; receiver sampling matrix S (d = S u)."""
    g = op.g
    src = op.points(src_xyz[s])
    sn = np.array([n for n, _ in src], dtype=np.int64)
    scale = np.array([w * g.dt * g.dt / (g.dx * g.dy * g.dz * op.sr[n]) for n, w in src])
    nr = rec_offset[s + 1] - rec_offset[s]
    S = sp.lil_matrix((nr, op.A.size))
    for q, r in enumerate(range(rec_offset[s], rec_offset[s + 1])):
        for n, w in op.points(rec_xyz[r]):
            S[q, n] += w * op.sr[n]
    return sn, scale, S.tocsr()


def forward(op, wavelet, sn, scale, recs, keep=False):
    """Traces [n_rec][nt] (recs: the sampling matrix); with keep=True also
    x^n - m2 u^n for every step."""
    n = op.A.size
    nt = op.g.nt
    u, v = np.zeros(n), np.zeros(n)
    psi = [np.zeros(n) for _ in range(3)]
    zeta = [np.zeros(n) for _ in range(3)]
    tr = np.zeros((recs.shape[0], nt))
    terms = []
    for it in range(nt):
        x = np.zeros(n)
        for a in range(3):
            psi[a] = op.b[a] * psi[a] + op.c[a] * (op.D1[a] @ u)
            d2u = op.D2[a] @ u
            d1p = op.D1[a] @ psi[a]
            zeta[a] = op.b[a] * zeta[a] + op.c[a] * (d2u + d1p)
            x += d2u + d1p + zeta[a]
        if keep:
            terms.append(x - op.m2 * u)
        un = op.live * (op.Bc * u - v + op.A * x)
        np.add.at(un, sn, scale * wavelet[it])
        v, u = u, un
        tr[:, it] = recs @ u
    return (tr, terms) if keep else tr


def model(oracle, g, vel, src_xyz, wavelet, rec_offset, rec_xyz, f0, rho=None, R=1e-3):
    """Seismograms [total_rec][nt] of every shot with the CPML boundary."""
    op = Operators(oracle, g, np.asarray(vel, np.float64), rho, f0, R)
    src_xyz = np.asarray(src_xyz, np.float64).reshape(-1, 3)
    rec_xyz = np.asarray(rec_xyz, np.float64).reshape(-1, 3)
    out = np.zeros((int(rec_offset[-1]), g.nt))
    for s in range(len(src_xyz)):
        sn, scale, recs = _shot(op, src_xyz, s, rec_offset, rec_xyz)
        out[rec_offset[s]:rec_offset[s + 1]] = forward(op, np.asarray(wavelet, np.float64), sn,
                                                       scale, recs)
    return out


def gradient(oracle, g, vel, src_xyz, wavelet, rec_offset, rec_xyz, dobs, f0, rho=None, R=1e-3,
             return_dwav=False):
    """(J, dJ/dc [nz][ny][nx]) and optionally dJ/dw, by the transposed recursion."""
    vel = np.asarray(vel, np.float64)
    op = Operators(oracle, g, vel, rho, f0, R)
    src_xyz = np.asarray(src_xyz, np.float64).reshape(-1, 3)
    rec_xyz = np.asarray(rec_xyz, np.float64).reshape(-1, 3)
    wavelet = np.asarray(wavelet, np.float64)
    n, nt = op.A.size, g.nt
    gA = np.zeros(n)
    dwav = np.zeros(nt)
    J = 0.0
    for s in range(len(src_xyz)):
        sn, scale, recs = _shot(op, src_xyz, s, rec_offset, rec_xyz)
        tr, terms = forward(op, wavelet, sn, scale, recs, keep=True)
        res = tr - np.asarray(dobs, np.float64)[rec_offset[s]:rec_offset[s + 1]]
        J += 0.5 * float(np.sum(res * res))
        lam, mu = np.zeros(n), np.zeros(n)  # adjoints of u^{n+1} (u slot) and u^n (v slot)
        psib = [np.zeros(n) for _ in range(3)]
        zetab = [np.zeros(n) for _ in range(3)]
        for it in range(nt - 1, -1, -1):
            lam += recs.T @ res[:, it]                       # d[n] = S u^{n+1}
            dwav[it] += np.sum(scale * lam[sn])
            lam = op.live * lam                              # through the surface mask
            gA += lam * terms[it]                           # u^{n+1} = ... + A (x - m2 u)
            xb = op.A * lam                                  # adjoint of x^n
            ub = op.Bc * lam + mu                            # adjoint of u^n (so far)
            ub += sum(op.D2T[a] @ xb for a in range(3))
            for a in range(3):
                zt = zetab[a] + xb                           # adjoint of zeta_a^n
                y = op.c[a] * zt
                zetab[a] = op.b[a] * zt                      # adjoint of zeta_a^{n-1}
                ub += op.D2T[a] @ y
                pt = psib[a] - op.D1[a] @ xb - op.D1[a] @ y  # adjoint of psi_a^n (D1^T = -D1)
                psib[a] = op.b[a] * pt                       # adjoint of psi_a^{n-1}
                ub -= op.D1[a] @ (op.c[a] * pt)
            mu = -lam                                        # adjoint of u^{n-1} via the v slot
            lam = ub
    b = g.border
    gA = gA.reshape(op.shape)[b:b + g.nz, b:b + g.ny, b:b + g.nx]
    grad = 2.0 * vel * g.dt * g.dt * gA
    return (J, grad, dwav) if return_dwav else (J, grad)
