// Oracle for the Mamute acoustic propagator, adjoint and imaging condition.
//
// TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, obviously correct CPU
// restatement of the method in the paper (Eq. 1, Algorithm 1 and Algorithm 3),
// written in FP64 (with an optional FP32 mode used only for tolerance
// studies).  Only the tests, the smoke check and the CPU-baseline leg of the
// benchmark may load it; the product library never links, loads or calls it,
// and it shares no source with the CUDA path.
//
// Conventions (each is a reading of the paper where it is silent or ambiguous):
//  * Eq. 1 (left): d2p/dt2 = c^2 lap p + S.  Eq. 1 (right): with density,
//    q = p / sqrt(rho), d2q/dt2 = c^2 (lap q - m2 q) + S / sqrt(rho),
//    m2 = lap(sqrt rho) / sqrt rho.
//  * Sec. 2.1: second order in time (leapfrog), eighth order in space
//    (radius-4 central stencil, the example config's "stencil = 4").
//  * Sec. 2.1 absorbing boundary by damping (Cerjan): sponge of `border` cells
//    padded outside the model on all six faces; per-axis profile
//    g(d) = exp(-(alpha d)^2), d = depth into the sponge (1..border); the 3-D
//    factor is the product of the three axis profiles.  Parity unpinned: the
//    value alpha = 0.015 (Cerjan's; the paper gives none) -- only alpha = 0
//    (no damping, energy conserved) is pinned.  The update is
//    u^{n+1} = g (B u^n - g u^{n-1} + A lap u^n) + source, A = c^2 dt^2,
//    B = 2 - A m2.
//  * The wavefield is zero outside the padded grid (Dirichlet).  c and rho are
//    edge-replicated into the sponge; sqrt(rho) is further edge-replicated
//    (index clamping) when m2 is formed, so m2 vanishes in the outer layers.
//  * Sec. 2.2.2 layouts: models are z x y x x (x fastest), coordinates are
//    (x, y, z) metres from (ox, oy, oz), traces are [n_rec][ns].
//  * Source term f(t) delta(x - x_S): the delta becomes 1/(dx dy dz) at the
//    nearest node; w[n] is injected into u^{n+1}; receivers record
//    p = sqrt(rho) q at the nearest node from u^{n+1}; u^0 = u^{-1} = 0.
//  * Misfit (Algorithm 3, SeismicData::Misfit): J = 1/2 sum (d - d_obs)^2.
//  * Gradient (Sec. 2.1, adjoint-state method; Algorithm 3 backward loop and
//    imaging by cross-correlation): the exact transpose of the discrete
//    recursion, written in terms of the Lagrange multiplier lambda^{n+1} of
//    the equation that produces u^{n+1}:
//        lambda^k = (B + lap A) g lambda^{k+1} - g^2 lambda^{k+2}
//                   + R^T r^{k-1},
//        dJ/dA(x) = sum_k lambda^k(x) g(x) ((lap - m2) u^{k-1})(x),
//    and "MultiplyAdjoint" (Algorithm 3) is the chain rule
//    dJ/dc = 2 c dt^2 dJ/dA on the model interior (the derivative through
//    the edge replication into the sponge is not taken).
//  * Forward-state storage for the backward loop (Sec. 2.1, three
//    wavefield-management modes): all states kept, or states checkpointed
//    every `snap_every` steps and recomputed; recomputation is the same
//    function on the same data, so every mode gives bitwise the same result.
//  * Pseudo-Hessian (optional output): P(x) = sum_shots sum_n
//    (g (lap - m2) u^n)(x)^2, the squared source-side factor of the Jacobian.
//  * Free surface (Sec. 2, modelling options; free_surface = 1): the top
//    model plane (padded plane z_s = border) is a pressure-release surface,
//    imposed by the image method: the field is odd about z_s, so values at
//    planes z_s - m are read as -u(z_s + m) and u(z_s) = 0 (g = 0 on z <= z_s,
//    which also keeps the planes above the surface at zero); the top face
//    has no sponge.  Sources and receivers on the surface plane are rejected.
//    The mirrored Laplacian is symmetric on the cells below the surface, so
//    the adjoint keeps the same form.
//  * Off-grid points (xyz_interp = 1): trilinear weights over the (up to)
//    8 nodes around a source or receiver; the source is spread with weights
//    w_e dt^2 / (dx dy dz sqrt(rho_e)) and a receiver samples
//    sum_e w_e sqrt(rho_e) u_e (nodes with zero weight, and nodes on a free
//    surface, are dropped).  xyz_interp = 0 is the nearest node.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

// Radius-4 central coefficients for the second derivative (eighth order),
// c_0 .. c_4 (Sec. 2.1: eighth order in space).
const double kC[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};

struct Grid {
  int nx, ny, nz, border;
  double dx, dy, dz, dt;
  int nt;
  double ox, oy, oz;
  double cerjan;  // sponge constant alpha; 0 disables damping (g == 1)
  int free_surface;  // 1: pressure-release surface at the top model plane
  int xyz_interp;    // 0: nearest node, 1: trilinear weights
};

struct Dims {
  long Nx, Ny, Nz;
  long zs = -1;  // padded plane of the free surface, -1 without one
  long n() const { return Nx * Ny * Nz; }
  long at(long i, long j, long k) const { return (k * Ny + j) * Nx + i; }
};

Dims padded(const Grid& g) {
  Dims d;
  d.Nx = g.nx + 2L * g.border;
  d.Ny = g.ny + 2L * g.border;
  d.Nz = g.nz + 2L * g.border;
  d.zs = g.free_surface ? g.border : -1;
  return d;
}

long clampl(long v, long lo, long hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Per-axis Cerjan profile on the padded axis of length N.  With a free
// surface at plane zs (z axis only) the low face has no sponge and the
// factor is 0 on and above the surface.
std::vector<double> sponge_profile(long N, int border, double alpha, long zs = -1) {
  std::vector<double> p(N, 1.0);
  for (long i = 0; i < N; ++i) {
    long d = 0;
    if (i < border && zs < 0) d = border - i;
    else if (i > N - 1 - border) d = i - (N - 1 - border);
    double a = alpha * (double)d;
    p[i] = (zs >= 0 && i <= zs) ? 0.0 : std::exp(-a * a);
  }
  return p;
}

// Padded coefficient arrays, always formed in FP64.
struct Medium {
  Dims d;
  std::vector<double> c;      // padded velocity
  std::vector<double> A;      // c^2 dt^2
  std::vector<double> m2;     // lap(sqrt rho)/sqrt rho  (0 without density)
  std::vector<double> g;      // gx*gy*gz
  std::vector<double> srho;   // sqrt(rho) padded (1 without density)
};

// lap v at (i,j,k) with the value function `val` deciding the exterior rule.
template <typename F>
double lap_at(const Dims& d, const Grid& gr, long i, long j, long k, F val) {
  double sx = kC[0] * val(i, j, k), sy = kC[0] * val(i, j, k), sz = kC[0] * val(i, j, k);
  for (int m = 1; m <= 4; ++m) {
    sx += kC[m] * (val(i - m, j, k) + val(i + m, j, k));
    sy += kC[m] * (val(i, j - m, k) + val(i, j + m, k));
    sz += kC[m] * (val(i, j, k - m) + val(i, j, k + m));
  }
  return sx / (gr.dx * gr.dx) + sy / (gr.dy * gr.dy) + sz / (gr.dz * gr.dz);
  (void)d;
}

Medium build_medium(const Grid& gr, const double* vel, const double* rho) {
  Medium M;
  M.d = padded(gr);
  const Dims& d = M.d;
  const long n = d.n();
  M.c.assign(n, 0.0);
  M.A.assign(n, 0.0);
  M.m2.assign(n, 0.0);
  M.g.assign(n, 1.0);
  M.srho.assign(n, 1.0);
  const int b = gr.border;
#pragma omp parallel for schedule(static)
  for (long k = 0; k < d.Nz; ++k)
    for (long j = 0; j < d.Ny; ++j)
      for (long i = 0; i < d.Nx; ++i) {
        long mi = clampl(i - b, 0, gr.nx - 1), mj = clampl(j - b, 0, gr.ny - 1),
             mk = clampl(k - b, 0, gr.nz - 1);
        long src = (mk * gr.ny + mj) * gr.nx + mi;
        double cv = vel[src];
        M.c[d.at(i, j, k)] = cv;
        M.A[d.at(i, j, k)] = cv * cv * gr.dt * gr.dt;
        if (rho) M.srho[d.at(i, j, k)] = std::sqrt(rho[src]);
      }
  if (rho) {
    // m2 = lap(sqrt rho) / sqrt rho with sqrt(rho) edge-replicated beyond
    // the padded grid (index clamping).
    const std::vector<double>& s = M.srho;
    auto val = [&](long i, long j, long k) {
      return s[d.at(clampl(i, 0, d.Nx - 1), clampl(j, 0, d.Ny - 1), clampl(k, 0, d.Nz - 1))];
    };
#pragma omp parallel for schedule(static)
    for (long k = 0; k < d.Nz; ++k)
      for (long j = 0; j < d.Ny; ++j)
        for (long i = 0; i < d.Nx; ++i)
          M.m2[d.at(i, j, k)] = lap_at(d, gr, i, j, k, val) / s[d.at(i, j, k)];
  }
  std::vector<double> gx = sponge_profile(d.Nx, b, gr.cerjan);
  std::vector<double> gy = sponge_profile(d.Ny, b, gr.cerjan);
  std::vector<double> gz = sponge_profile(d.Nz, b, gr.cerjan, d.zs);
#pragma omp parallel for schedule(static)
  for (long k = 0; k < d.Nz; ++k)
    for (long j = 0; j < d.Ny; ++j)
      for (long i = 0; i < d.Nx; ++i) M.g[d.at(i, j, k)] = gx[i] * gy[j] * gz[k];
  return M;
}

// Nearest padded node of a coordinate triple; -1 when outside the model.
long node_of(const Grid& gr, const Dims& d, const double* xyz) {
  long i = (long)std::floor((xyz[0] - gr.ox) / gr.dx + 0.5);
  long j = (long)std::floor((xyz[1] - gr.oy) / gr.dy + 0.5);
  long k = (long)std::floor((xyz[2] - gr.oz) / gr.dz + 0.5);
  if (i < 0 || i >= gr.nx || j < 0 || j >= gr.ny || k < 0 || k >= gr.nz) return -1;
  return d.at(i + gr.border, j + gr.border, k + gr.border);
}

// lap of a wavefield (zero outside the padded grid) at one node, in type T.
// With a free surface, planes at or above it are read through the odd image.
template <typename T>
T lap_field(const Dims& d, const T* u, long i, long j, long k, T ix2, T iy2, T iz2) {
  auto v = [&](long a, long b, long c) -> T {
    T sign = T(1);
    if (d.zs >= 0 && c <= d.zs) {
      c = 2 * d.zs - c;
      sign = T(-1);
    }
    if (a < 0 || a >= d.Nx || b < 0 || b >= d.Ny || c < 0 || c >= d.Nz) return T(0);
    return sign * u[d.at(a, b, c)];
  };
  T c0 = (T)kC[0];
  T sx = c0 * v(i, j, k), sy = c0 * v(i, j, k), sz = c0 * v(i, j, k);
  for (int m = 1; m <= 4; ++m) {
    T cm = (T)kC[m];
    sx += cm * (v(i - m, j, k) + v(i + m, j, k));
    sy += cm * (v(i, j - m, k) + v(i, j + m, k));
    sz += cm * (v(i, j, k - m) + v(i, j, k + m));
  }
  return sx * ix2 + sy * iy2 + sz * iz2;
}

// Coefficients converted to the working type.
template <typename T>
struct Coef {
  std::vector<T> A, B, m2, g;
  T ix2, iy2, iz2;
};

template <typename T>
Coef<T> coef_of(const Medium& M, const Grid& gr) {
  Coef<T> c;
  const long n = M.d.n();
  c.A.resize(n); c.B.resize(n); c.m2.resize(n); c.g.resize(n);
#pragma omp parallel for schedule(static)
  for (long p = 0; p < n; ++p) {
    c.A[p] = (T)M.A[p];
    c.m2[p] = (T)M.m2[p];
    c.B[p] = (T)(2.0 - M.A[p] * M.m2[p]);
    c.g[p] = (T)M.g[p];
  }
  c.ix2 = (T)(1.0 / (gr.dx * gr.dx));
  c.iy2 = (T)(1.0 / (gr.dy * gr.dy));
  c.iz2 = (T)(1.0 / (gr.dz * gr.dz));
  return c;
}

// One leapfrog step (Table 1, ModelingStep):
// unew = g (B ucur - g uprev + A lap ucur), written into uprev's storage.
template <typename T>
void step(const Dims& d, const Coef<T>& c, T* uprev, const T* ucur) {
  std::vector<T> out(d.n());
#pragma omp parallel for schedule(static)
  for (long k = 0; k < d.Nz; ++k)
    for (long j = 0; j < d.Ny; ++j)
      for (long i = 0; i < d.Nx; ++i) {
        long p = d.at(i, j, k);
        T l = lap_field<T>(d, ucur, i, j, k, c.ix2, c.iy2, c.iz2);
        out[p] = c.g[p] * (c.B[p] * ucur[p] - c.g[p] * uprev[p] + c.A[p] * l);
      }
  std::memcpy(uprev, out.data(), sizeof(T) * d.n());
}

// Transposed step for the multiplier: returns
// (B + lap A) (g lam1) - g^2 lam2, written into lam2's storage.
void adjoint_step(const Dims& d, const Coef<double>& c, double* lam2, const double* lam1) {
  const long n = d.n();
  std::vector<double> w(n), Aw(n), out(n);
  for (long p = 0; p < n; ++p) {
    w[p] = c.g[p] * lam1[p];
    Aw[p] = c.A[p] * w[p];
  }
#pragma omp parallel for schedule(static)
  for (long k = 0; k < d.Nz; ++k)
    for (long j = 0; j < d.Ny; ++j)
      for (long i = 0; i < d.Nx; ++i) {
        long p = d.at(i, j, k);
        double l = lap_field<double>(d, Aw.data(), i, j, k, c.ix2, c.iy2, c.iz2);
        out[p] = c.B[p] * w[p] + l - c.g[p] * c.g[p] * lam2[p];
      }
  std::memcpy(lam2, out.data(), sizeof(double) * n);
}

// Shot domain for an aperture [a0, a1) x [a2, a3) of model columns: the
// window [a0, a1 + 2 border) x [a2, a3 + 2 border) x [0, Nz) of the global
// padded grid, with its own sponge profiles at the window faces (the sponge
// of an interior aperture sees the true model around it).
Medium window(const Medium& G, const Grid& gr, int a0, int a1, int a2, int a3) {
  Medium W;
  const int b = gr.border;
  W.d.Nx = (a1 - a0) + 2L * b;
  W.d.Ny = (a3 - a2) + 2L * b;
  W.d.Nz = G.d.Nz;
  W.d.zs = G.d.zs;
  const long n = W.d.n();
  W.c.resize(n); W.A.resize(n); W.m2.resize(n); W.g.resize(n); W.srho.resize(n);
  std::vector<double> gx = sponge_profile(W.d.Nx, b, gr.cerjan);
  std::vector<double> gy = sponge_profile(W.d.Ny, b, gr.cerjan);
  std::vector<double> gz = sponge_profile(W.d.Nz, b, gr.cerjan, W.d.zs);
  for (long k = 0; k < W.d.Nz; ++k)
    for (long j = 0; j < W.d.Ny; ++j)
      for (long i = 0; i < W.d.Nx; ++i) {
        long p = W.d.at(i, j, k), q = G.d.at(i + a0, j + a2, k);
        W.c[p] = G.c[q];
        W.A[p] = G.A[q];
        W.m2[p] = G.m2[q];
        W.srho[p] = G.srho[q];
        W.g[p] = gx[i] * gy[j] * gz[k];
      }
  return W;
}

// A source or receiver: padded nodes and their weights (the source weights
// include dt^2 / (dx dy dz sqrt(rho)), the receiver weights sqrt(rho)).
struct Point {
  std::vector<long> node;
  std::vector<double> w;
};

struct Shot {
  Point src;
  std::vector<Point> rec;
};

// Node of a coordinate in a shot window (nearest node); -1 outside the model
// or aperture.
long node_in(const Grid& gr, const Dims& d, const double* xyz, const int* ap) {
  long i = (long)std::floor((xyz[0] - gr.ox) / gr.dx + 0.5);
  long j = (long)std::floor((xyz[1] - gr.oy) / gr.dy + 0.5);
  long k = (long)std::floor((xyz[2] - gr.oz) / gr.dz + 0.5);
  if (i < 0 || i >= gr.nx || j < 0 || j >= gr.ny || k < 0 || k >= gr.nz) return -1;
  long a0 = 0, a2 = 0;
  if (ap) {
    if (i < ap[0] || i >= ap[1] || j < ap[2] || j >= ap[3]) return -1;
    a0 = ap[0];
    a2 = ap[2];
  }
  return d.at(i + gr.border - a0, j + gr.border - a2, k + gr.border);
}

// Nodes and interpolation weights of a coordinate (before the density and
// source scales): the nearest node with weight 1, or the trilinear weights
// of the cell that holds the point.  Returns -1 if the point (or one of its
// nodes with non-zero weight) lies outside the model or aperture, or if all
// of its weight falls on a free surface.
int locate(const Grid& gr, const Dims& d, const double* xyz, const int* ap, Point& P) {
  P.node.clear();
  P.w.clear();
  const long a0 = ap ? ap[0] : 0, a2 = ap ? ap[2] : 0;
  const long lo[3] = {a0, a2, 0};
  const long hi[3] = {ap ? ap[1] : gr.nx, ap ? ap[3] : gr.ny, gr.nz};
  if (!gr.xyz_interp) {
    long p = node_in(gr, d, xyz, ap);
    if (p < 0) return -1;
    if (d.zs >= 0 && p / (d.Nx * d.Ny) <= d.zs) return -1;
    P.node.push_back(p);
    P.w.push_back(1.0);
    return 0;
  }
  const double o[3] = {gr.ox, gr.oy, gr.oz}, h[3] = {gr.dx, gr.dy, gr.dz};
  long base[3];
  double t[3];
  for (int a = 0; a < 3; ++a) {
    const double f = (xyz[a] - o[a]) / h[a];
    base[a] = (long)std::floor(f);
    t[a] = f - (double)base[a];
  }
  for (int c = 0; c < 8; ++c) {
    long idx[3];
    double w = 1.0;
    for (int a = 0; a < 3; ++a) {
      const int up = (c >> a) & 1;
      idx[a] = base[a] + up;
      w *= up ? t[a] : 1.0 - t[a];
    }
    if (w == 0.0) continue;
    for (int a = 0; a < 3; ++a)
      if (idx[a] < lo[a] || idx[a] >= hi[a]) return -1;
    const long k = idx[2] + gr.border;
    if (d.zs >= 0 && k <= d.zs) continue;  // the field is zero on the surface
    P.node.push_back(d.at(idx[0] + gr.border - a0, idx[1] + gr.border - a2, k));
    P.w.push_back(w);
  }
  return P.node.empty() ? -1 : 0;
}

// Shot s with its medium (the global one, or its aperture window).
struct ShotSetup {
  Medium local;   // used only with an aperture
  const Medium* M;
  Shot sh;
  int a0, a2;
};

int make_shot(const Grid& gr, const Medium& G, int s, const double* src_xyz, const int* rec_offset,
              const double* rec_xyz, const int* aperture, ShotSetup& S) {
  const int* ap = aperture ? aperture + 4 * s : nullptr;
  if (ap) {
    if (ap[0] < 0 || ap[1] > gr.nx || ap[0] >= ap[1] || ap[2] < 0 || ap[3] > gr.ny || ap[2] >= ap[3])
      return -1;
    S.local = window(G, gr, ap[0], ap[1], ap[2], ap[3]);
    S.M = &S.local;
    S.a0 = ap[0];
    S.a2 = ap[2];
  } else {
    S.M = &G;
    S.a0 = S.a2 = 0;
  }
  const Medium& M = *S.M;
  Shot& sh = S.sh;
  sh.rec.clear();
  if (locate(gr, M.d, src_xyz + 3 * s, ap, sh.src)) return -1;
  for (size_t e = 0; e < sh.src.node.size(); ++e)
    sh.src.w[e] *= gr.dt * gr.dt / (gr.dx * gr.dy * gr.dz * M.srho[sh.src.node[e]]);
  for (int r = rec_offset[s]; r < rec_offset[s + 1]; ++r) {
    Point P;
    if (locate(gr, M.d, rec_xyz + 3 * (long)r, ap, P)) return -1;
    for (size_t e = 0; e < P.node.size(); ++e) P.w[e] *= M.srho[P.node[e]];
    sh.rec.push_back(P);
  }
  return 0;
}

// Source injection and receiver sampling of one shot.
template <typename T>
void inject(std::vector<T>& u, const Point& P, double amount) {
  for (size_t e = 0; e < P.node.size(); ++e) u[P.node[e]] += (T)(P.w[e] * amount);
}

template <typename T>
double sample(const std::vector<T>& u, const Point& P) {
  double v = 0.0;
  for (size_t e = 0; e < P.node.size(); ++e) v += P.w[e] * (double)u[P.node[e]];
  return v;
}

// Forward modelling of one shot in type T (Algorithm 1, "Forward
// propagation"; Table 1 ModelingStep + ReadReceiver).  trace[r*nt + n].
// If `phess` is given, adds sum_n (g (lap - m2) u^n)^2 into it (padded).
template <typename T>
void forward_shot(const Grid& gr, const Dims& d, const Coef<T>& c, const Shot& sh,
                  const double* wavelet, double* trace, double* phess) {
  const long n = d.n();
  std::vector<T> u0(n, T(0)), u1(n, T(0));  // u0 = u^{n-1}, u1 = u^n
  const long nr = (long)sh.rec.size();
  for (int it = 0; it < gr.nt; ++it) {
    if (phess) {
#pragma omp parallel for schedule(static)
      for (long k = 0; k < d.Nz; ++k)
        for (long j = 0; j < d.Ny; ++j)
          for (long i = 0; i < d.Nx; ++i) {
            long p = d.at(i, j, k);
            double a = (double)c.g[p] *
                       ((double)lap_field<T>(d, u1.data(), i, j, k, c.ix2, c.iy2, c.iz2) -
                        (double)c.m2[p] * (double)u1[p]);
            phess[p] += a * a;
          }
    }
    step<T>(d, c, u0.data(), u1.data());  // u0 <- u^{n+1}
    inject(u0, sh.src, wavelet[it]);
    for (long r = 0; r < nr; ++r) trace[r * gr.nt + it] = sample(u0, sh.rec[r]);
    std::swap(u0, u1);
  }
}

}  // namespace

extern "C" {

// Oracle grid descriptor (ctypes mirror in oracle/oracle.py).
typedef Grid oracle_grid;

// The five stencil coefficients c_0..c_4 (Sec. 2.1, eighth order).
void oracle_fd_coeffs(double* out5) {
  for (int m = 0; m < 5; ++m) out5[m] = kC[m];
}

// Padded coefficient arrays (each [Nz][Ny][Nx]); any output may be null.
int oracle_prepare(const oracle_grid* gr, const double* vel, const double* rho, double* A,
                   double* m2, double* g, double* srho) {
  Medium M = build_medium(*gr, vel, rho);
  const long n = M.d.n();
  if (A) std::memcpy(A, M.A.data(), sizeof(double) * n);
  if (m2) std::memcpy(m2, M.m2.data(), sizeof(double) * n);
  if (g) std::memcpy(g, M.g.data(), sizeof(double) * n);
  if (srho) std::memcpy(srho, M.srho.data(), sizeof(double) * n);
  return 0;
}

// lap of a padded field (zero outside), FP64, for stencil tests.
void oracle_laplacian(const oracle_grid* gr, const double* u, double* out) {
  Dims d = padded(*gr);
  for (long k = 0; k < d.Nz; ++k)
    for (long j = 0; j < d.Ny; ++j)
      for (long i = 0; i < d.Nx; ++i)
        out[d.at(i, j, k)] = lap_field<double>(d, u, i, j, k, 1.0 / (gr->dx * gr->dx),
                                               1.0 / (gr->dy * gr->dy), 1.0 / (gr->dz * gr->dz));
}

// Advances an arbitrary initial state n_steps with no source, FP64, in place:
// on entry uprev = u^{-1}, ucur = u^0; on exit uprev = u^{n-1}, ucur = u^n.
int oracle_advance(const oracle_grid* gr, const double* vel, const double* rho, double* uprev,
                   double* ucur, int n_steps) {
  Medium M = build_medium(*gr, vel, rho);
  Coef<double> c = coef_of<double>(M, *gr);
  const long n = M.d.n();
  for (int it = 0; it < n_steps; ++it) {
    step<double>(M.d, c, uprev, ucur);
    std::vector<double> t(uprev, uprev + n);
    std::memcpy(uprev, ucur, sizeof(double) * n);
    std::memcpy(ucur, t.data(), sizeof(double) * n);
  }
  return 0;
}

// Adds a shot-window array into the global padded array.
void scatter_add(const Dims& G, const Dims& W, int a0, int a2, const std::vector<double>& loc,
                 std::vector<double>& glob) {
  for (long k = 0; k < W.Nz; ++k)
    for (long j = 0; j < W.Ny; ++j)
      for (long i = 0; i < W.Nx; ++i) glob[G.at(i + a0, j + a2, k)] += loc[W.at(i, j, k)];
}

// Seismic modelling (Algorithm 1): seis[total_rec][nt].  precision 64 or 32.
// phess (nullable): pseudo-Hessian summed over shots, [nz][ny][nx] interior.
// aperture (nullable): [n_src][4] model columns per shot (see window()).
int oracle_model(const oracle_grid* gr, const double* vel, const double* rho, int n_src,
                 const double* src_xyz, const double* wavelet, const int* rec_offset,
                 const double* rec_xyz, int precision, double* seis, double* phess,
                 const int* aperture) {
  Medium G = build_medium(*gr, vel, rho);
  std::vector<double> ph;
  if (phess) ph.assign(G.d.n(), 0.0);
  for (int s = 0; s < n_src; ++s) {
    ShotSetup S;
    if (make_shot(*gr, G, s, src_xyz, rec_offset, rec_xyz, aperture, S)) return -1;
    const Medium& M = *S.M;
    std::vector<double> phl;
    if (phess) phl.assign(M.d.n(), 0.0);
    double* out = seis + (long)rec_offset[s] * gr->nt;
    if (precision == 32) {
      Coef<float> c = coef_of<float>(M, *gr);
      forward_shot<float>(*gr, M.d, c, S.sh, wavelet, out, phess ? phl.data() : nullptr);
    } else {
      Coef<double> c = coef_of<double>(M, *gr);
      forward_shot<double>(*gr, M.d, c, S.sh, wavelet, out, phess ? phl.data() : nullptr);
    }
    if (phess) scatter_add(G.d, M.d, S.a0, S.a2, phl, ph);
  }
  if (phess) {
    const int b = gr->border;
    for (long k = 0; k < gr->nz; ++k)
      for (long j = 0; j < gr->ny; ++j)
        for (long i = 0; i < gr->nx; ++i)
          phess[(k * gr->ny + j) * gr->nx + i] = ph[G.d.at(i + b, j + b, k + b)];
  }
  return 0;
}

// Misfit and gradient (Algorithm 3), FP64.  grad[nz][ny][nx] = dJ/dc.
// snap_every = 0 keeps every forward state; > 0 checkpoints the state pair
// every snap_every steps and recomputes each segment in the backward loop.
// seis_out (nullable) receives the modelled data [total_rec][nt].
// dwav (nullable) receives dJ/dw[n] = sum_shots src_scale lambda^{n+1}(x_s),
// the transpose of the linear map wavelet -> seismogram applied to the residual.
int oracle_gradient(const oracle_grid* gr, const double* vel, const double* rho, int n_src,
                    const double* src_xyz, const double* wavelet, const int* rec_offset,
                    const double* rec_xyz, const double* dobs, int snap_every, double* misfit,
                    double* grad, double* seis_out, double* dwav, const int* aperture) {
  Medium G = build_medium(*gr, vel, rho);
  const int nt = gr->nt;
  std::vector<double> gA_global(G.d.n(), 0.0);
  if (dwav) std::memset(dwav, 0, sizeof(double) * nt);
  double J = 0.0;
  const int seg = snap_every > 0 ? snap_every : nt;
  for (int s = 0; s < n_src; ++s) {
    ShotSetup S;
    if (make_shot(*gr, G, s, src_xyz, rec_offset, rec_xyz, aperture, S)) return -1;
    const Medium& M = *S.M;
    const Dims& d = M.d;
    const long n = d.n();
    Coef<double> c = coef_of<double>(M, *gr);
    std::vector<double> gA(n, 0.0);
    const Shot& sh = S.sh;
    const long nr = (long)sh.rec.size();
    const long roff = rec_offset[s];
    // Forward propagation, with the state pair (u^{m-1}, u^m) saved at every
    // segment start m = 0, seg, 2 seg, ... (ManageWavefield::SaveWavefield).
    std::vector<std::vector<double>> ck_prev, ck_cur;
    std::vector<double> d_mod(nr * nt);
    {
      std::vector<double> u0(n, 0.0), u1(n, 0.0);
      for (int it = 0; it < nt; ++it) {
        if (it % seg == 0) { ck_prev.push_back(u0); ck_cur.push_back(u1); }
        step<double>(d, c, u0.data(), u1.data());
        inject(u0, sh.src, wavelet[it]);
        for (long r = 0; r < nr; ++r) d_mod[r * nt + it] = sample(u0, sh.rec[r]);
        std::swap(u0, u1);
      }
    }
    if (seis_out) std::memcpy(seis_out + roff * nt, d_mod.data(), sizeof(double) * nr * nt);
    // Residual and misfit (SeismicData::Misfit).
    std::vector<double> res(nr * nt);
    for (long r = 0; r < nr; ++r)
      for (int it = 0; it < nt; ++it) {
        double v = d_mod[r * nt + it] - dobs[(roff + r) * nt + it];
        res[r * nt + it] = v;
        J += 0.5 * v * v;
      }
    // Backward propagation: lambda^k for k = nt .. 1 with cross-correlation
    // imaging against u^{k-1} (ModelingStep, RetrieveWavefield, imaging).
    std::vector<double> lam1(n, 0.0), lam2(n, 0.0);  // lambda^{k+1}, lambda^{k+2}
    const int nseg = (nt + seg - 1) / seg;
    for (int sg = nseg - 1; sg >= 0; --sg) {
      const int m0 = sg * seg, m1 = std::min(nt, m0 + seg);
      // Recompute u^{m0} .. u^{m1-1} from the saved pair.
      std::vector<std::vector<double>> states;
      {
        std::vector<double> u0 = ck_prev[sg], u1 = ck_cur[sg];
        for (int it = m0; it < m1; ++it) {
          states.push_back(u1);  // u^{it}
          if (it + 1 < m1) {
            step<double>(d, c, u0.data(), u1.data());
            inject(u0, sh.src, wavelet[it]);
            std::swap(u0, u1);
          }
        }
      }
      for (int k = m1; k > m0; --k) {  // lambda^k pairs with u^{k-1}
        adjoint_step(d, c, lam2.data(), lam1.data());  // lam2 <- (B+lap A) g lam1 - g^2 lam2
        for (long r = 0; r < nr; ++r) inject(lam2, sh.rec[r], res[r * nt + (k - 1)]);
        std::swap(lam1, lam2);  // lam1 = lambda^k, lam2 = lambda^{k+1}
        if (dwav) dwav[k - 1] += sample(lam1, sh.src);
        const std::vector<double>& u = states[k - 1 - m0];
#pragma omp parallel for schedule(static)
        for (long kk = 0; kk < d.Nz; ++kk)
          for (long j = 0; j < d.Ny; ++j)
            for (long i = 0; i < d.Nx; ++i) {
              long p = d.at(i, j, kk);
              double lu = lap_field<double>(d, u.data(), i, j, kk, c.ix2, c.iy2, c.iz2);
              gA[p] += lam1[p] * c.g[p] * (lu - c.m2[p] * u[p]);
            }
      }
    }
    scatter_add(G.d, d, S.a0, S.a2, gA, gA_global);
  }
  if (misfit) *misfit = J;
  // MultiplyAdjoint: dJ/dc = 2 c dt^2 dJ/dA on the interior.
  const int b = gr->border;
  for (long k = 0; k < gr->nz; ++k)
    for (long j = 0; j < gr->ny; ++j)
      for (long i = 0; i < gr->nx; ++i) {
        long p = G.d.at(i + b, j + b, k + b);
        grad[(k * gr->ny + j) * gr->nx + i] = 2.0 * G.c[p] * gr->dt * gr->dt * gA_global[p];
      }
  return 0;
}

// ---------------------------------------------------------------------------
// Gauss-Newton diagonal building blocks (no aperture; one medium).
//
// Jacobian of the recorded data with respect to A(x): the Born source of
// step n at x is q[n] = a^n(x) dA(x), a^n = g (lap - m2) u^n, injected like
// the source into u^{n+1}; with G_{r,x}[k] the sample k recorded at r for a
// unit injection at x in step 0, dd_r[m]/dA(x) = sum_n G_{r,x}[m - n] a^n(x).

// a^n(x) of one shot for every step n < nt and interior cell: a[nt][nz][ny][nx].
int oracle_forward_terms(const oracle_grid* gr, const double* vel, const double* rho, int shot,
                         const double* src_xyz, const double* wavelet, double* a) {
  Medium M = build_medium(*gr, vel, rho);
  const Dims& d = M.d;
  const long n = d.n();
  Coef<double> c = coef_of<double>(M, *gr);
  Point src;
  if (locate(*gr, d, src_xyz + 3 * shot, nullptr, src)) return -1;
  for (size_t e = 0; e < src.node.size(); ++e)
    src.w[e] *= gr->dt * gr->dt / (gr->dx * gr->dy * gr->dz * M.srho[src.node[e]]);
  const int b = gr->border;
  const long ni = (long)gr->nx * gr->ny * gr->nz;
  std::vector<double> u0(n, 0.0), u1(n, 0.0);
  for (int it = 0; it < gr->nt; ++it) {
    for (long k = 0; k < gr->nz; ++k)
      for (long j = 0; j < gr->ny; ++j)
        for (long i = 0; i < gr->nx; ++i) {
          long p = d.at(i + b, j + b, k + b);
          double l = lap_field<double>(d, u1.data(), i + b, j + b, k + b, c.ix2, c.iy2, c.iz2);
          a[it * ni + (k * gr->ny + j) * gr->nx + i] = c.g[p] * (l - c.m2[p] * u1[p]);
        }
    step<double>(d, c, u0.data(), u1.data());
    inject(u0, src, wavelet[it]);
    std::swap(u0, u1);
  }
  return 0;
}

// Impulse response of a unit injection into u^1 at interior cell (ci, cj, ck),
// recorded at n_rec receivers for nt samples: G[n_rec][nt].
int oracle_cell_response(const oracle_grid* gr, const double* vel, const double* rho, int ci,
                         int cj, int ck, int n_rec, const double* rec_xyz, double* G) {
  Medium M = build_medium(*gr, vel, rho);
  Coef<double> c = coef_of<double>(M, *gr);
  Shot sh;
  sh.src.node.push_back(M.d.at(ci + gr->border, cj + gr->border, ck + gr->border));
  sh.src.w.push_back(1.0);
  for (int r = 0; r < n_rec; ++r) {
    Point P;
    if (locate(*gr, M.d, rec_xyz + 3 * r, nullptr, P)) return -1;
    for (size_t e = 0; e < P.node.size(); ++e) P.w[e] *= M.srho[P.node[e]];
    sh.rec.push_back(P);
  }
  std::vector<double> imp(gr->nt, 0.0);
  imp[0] = 1.0;
  forward_shot<double>(*gr, M.d, c, sh, imp.data(), G, nullptr);
  return 0;
}

// The same responses for one receiver and every interior cell at once, from
// the multiplier recursion driven by a unit data impulse at the last sample:
// lambda^{nt-j}(x) = G_{r,x}[j].  Output G[nt][nz][ny][nx].
int oracle_receiver_response(const oracle_grid* gr, const double* vel, const double* rho,
                             const double* rec_xyz1, double* G) {
  Medium M = build_medium(*gr, vel, rho);
  const Dims& d = M.d;
  const long n = d.n();
  Coef<double> c = coef_of<double>(M, *gr);
  Point rp;
  if (locate(*gr, d, rec_xyz1, nullptr, rp)) return -1;
  for (size_t e = 0; e < rp.node.size(); ++e) rp.w[e] *= M.srho[rp.node[e]];
  const int nt = gr->nt, b = gr->border;
  const long ni = (long)gr->nx * gr->ny * gr->nz;
  std::vector<double> lam1(n, 0.0), lam2(n, 0.0);
  for (int k = nt; k >= 1; --k) {
    adjoint_step(d, c, lam2.data(), lam1.data());
    if (k == nt) inject(lam2, rp, 1.0);
    std::swap(lam1, lam2);  // lam1 = lambda^k
    const int j = nt - k;
    for (long kk = 0; kk < gr->nz; ++kk)
      for (long jj = 0; jj < gr->ny; ++jj)
        for (long ii = 0; ii < gr->nx; ++ii)
          G[j * ni + (kk * gr->ny + jj) * gr->nx + ii] = lam1[d.at(ii + b, jj + b, kk + b)];
  }
  return 0;
}

}  // extern "C"
