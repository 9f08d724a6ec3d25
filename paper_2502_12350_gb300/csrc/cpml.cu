// Convolutional PML (Sec. 2: the second absorbing boundary, after Roden and
// Gedney) for modelling and for the gradient.
//
// In the layer each derivative d/dx_a is (1/s_a) d/dx_a, s_a = 1 + d_a /
// (alpha_a + i w), and the second derivative is carried by two memory
// variables per axis, updated by recursive convolution.  With the unscaled
// eighth-order stencils D2_a (weights c0..c4) and D1_a (4/5, -1/5, 4/105,
// -1/280) and the memory variables scaled by h and h^2 (so that the update
// uses A = c^2 dt^2 / h^2 like the damping kernels):
//   psi_a'  = b_a psi_a  + c_a D1_a u
//   zeta_a' = b_a zeta_a + c_a (D2_a u + D1_a psi_a')
//   x       = sum_a (D2_a u + D1_a psi_a' + zeta_a')
//   u'      = (2 - M) u - v + A x + source,        M = A m2 h^2
// with b_a = exp(-(d_a + alpha_a) dt), c_a = d_a (b_a - 1) / (d_a + alpha_a)
// (profiles built on the host).  No sponge factor applies.  The gradient is
// the exact transpose of this recursion in the Lagrange multiplier lam of
// u', run backwards over stored imaging terms t = x - (M / A) u:
//   acc += lam t;  xb = A lam
//   per axis: y_a = c_a (zetab_a + xb),  zetab_a <- b_a (zetab_a + xb)
//             p_a = psib_a - D1_a (xb + y_a), psib_a <- b_a p_a,  z_a = c_a p_a
//   lam_new = (2 - M) lam + mu + sum_a (D2_a (xb + y_a) - D1_a z_a),  mu_new = -lam
// (D2 is symmetric, D1 antisymmetric, the field is zero outside the padded
// grid).  Outside the layer along an axis the memory variables and their
// multipliers stay zero.
//
// These kernels read neighbours straight from global memory (one point per
// thread, L1/L2 serve the reuse); the memory-variable terms are evaluated
// only within 4 cells of the layer along their axis.
#include "cpml.h"

#include <algorithm>

namespace mamute {

namespace {

__constant__ float kC2[5] = {MAMUTE_C0, MAMUTE_C1, MAMUTE_C2, MAMUTE_C3, MAMUTE_C4};
__constant__ float kD1[4] = {4.0f / 5.0f, -1.0f / 5.0f, 4.0f / 105.0f, -1.0f / 280.0f};

struct Pt {
  int x, y, z;
};

__device__ __forceinline__ long long idx(const VolDesc& V, int x, int y, int z) {
  return V.off + ((long long)z * V.Ny + y) * V.pitch + x;
}

// f at p + m along axis a (zero outside the window).
__device__ __forceinline__ float nb(const float* f, const VolDesc& V, Pt p, int a, int m) {
  int x = p.x, y = p.y, z = p.z;
  if (a == 0) x += m;
  else if (a == 1) y += m;
  else z += m;
  if (x < 0 || x >= V.Nx || y < 0 || y >= V.Ny || z < 0 || z >= V.Nz) return 0.0f;
  return f[idx(V, x, y, z)];
}

__device__ __forceinline__ float d2(const float* f, const VolDesc& V, Pt p, int a) {
  float s = kC2[0] * f[idx(V, p.x, p.y, p.z)];
#pragma unroll
  for (int m = 1; m <= 4; ++m) s = fmaf(kC2[m], nb(f, V, p, a, m) + nb(f, V, p, a, -m), s);
  return s;
}

__device__ __forceinline__ float d1(const float* f, const VolDesc& V, Pt p, int a) {
  float s = 0.0f;
#pragma unroll
  for (int m = 1; m <= 4; ++m) s = fmaf(kD1[m - 1], nb(f, V, p, a, m) - nb(f, V, p, a, -m), s);
  return s;
}

__device__ __forceinline__ void prof(const CpmlProf& c, const VolDesc& V, Pt p, int a, float& b,
                                     float& cc) {
  if (a == 0) {
    b = c.bx[V.gx_off + p.x];
    cc = c.cx[V.gx_off + p.x];
  } else if (a == 1) {
    b = c.by[V.gy_off + p.y];
    cc = c.cy[V.gy_off + p.y];
  } else {
    b = c.bz[p.z];
    cc = c.cz[p.z];
  }
}

__device__ __forceinline__ bool in_layer(float b, float cc) { return cc != 0.0f || b != 1.0f; }

// Within 4 cells of the layer along axis a: elsewhere D1_a and D2_a of a
// field that is zero outside the layer vanish, and are skipped.
__device__ __forceinline__ bool near_layer(const VolDesc& V, Pt p, int a) {
  const int q = a == 0 ? p.x : (a == 1 ? p.y : p.z);
  const int N = a == 0 ? V.Nx : (a == 1 ? V.Ny : V.Nz);
  return q < V.border + 4 || q >= N - V.border - 4;
}

template <typename F>
__device__ __forceinline__ void for_points(const VolDesc& V, F f) {
  const long long n = (long long)V.Nx * V.Ny * V.Nz;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    Pt p;
    p.x = (int)(q % V.Nx);
    p.y = (int)((q / V.Nx) % V.Ny);
    p.z = (int)(q / ((long long)V.Nx * V.Ny));
    f(p);
  }
}

__global__ void psi_kernel(CpmlArgs c) {
  const VolDesc V = c.vols[blockIdx.y];
  for_points(V, [&](Pt p) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float b, cc;
      prof(c.pr, V, p, a, b, cc);
      if (!in_layer(b, cc)) continue;
      const long long i = idx(V, p.x, p.y, p.z);
      c.psi[a][i] = fmaf(b, c.psi[a][i], cc * d1(c.u, V, p, a));
    }
  });
}

__global__ void step_kernel_pml(CpmlArgs c) {
  const VolDesc V = c.vols[blockIdx.y];
  for_points(V, [&](Pt p) {
    const long long i = idx(V, p.x, p.y, p.z);
    float x = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float d2u = d2(c.u, V, p, a);
      const float d1p = near_layer(V, p, a) ? d1(c.psi[a], V, p, a) : 0.0f;
      float b, cc;
      prof(c.pr, V, p, a, b, cc);
      float zt = 0.0f;
      if (in_layer(b, cc)) {
        zt = fmaf(b, c.zeta[a][i], cc * (d2u + d1p));
        c.zeta[a][i] = zt;
      }
      x += d2u + d1p + zt;
    }
    const long long g = ((long long)p.z * c.NyG + (p.y + V.cy0)) * c.pitchG + (p.x + V.cx0);
    const float A = c.A[g];
    const float M = c.M ? c.M[g] : 0.0f;
    const float u = c.u[i];
    float out = fmaf(A, x, fmaf(2.0f, u, -c.v[i]) - M * u);
    // source: w_e dt^2 w[n] / (h^3 sqrt rho_e) at the corners of its cell
    const int dx = p.x - V.src_x, dy = p.y - V.src_y, dz = p.z - V.src_z;
    if ((unsigned)dx < 2u && (unsigned)dy < 2u && (unsigned)dz < 2u)
      out = fmaf(c.vols[blockIdx.y].src_sc[dx + 2 * dy + 4 * dz], c.wn, out);
    c.v[i] = out;
    if (c.tstore) {  // imaging term x - m2 u (in units of the scaled A) on the interior
      const int bb = V.border, zi = p.z - bb, yi = p.y - bb, xi = p.x - bb;
      if (xi >= 0 && xi < V.nxi && yi >= 0 && yi < V.nyi && zi >= 0 && zi < V.nzi)
        c.tstore[V.toff + ((long long)zi * V.nyi + yi) * V.tpitch + (p.x - V.txoff)] =
            x - (M / A) * u;
    }
  });
}

__global__ void record_kernel(const float* __restrict__ u, const long long* __restrict__ node,
                              const RecEntry* __restrict__ rec, int ncol, float* __restrict__ dout) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < ncol) dout[c] = rec[c].fscale * u[node[c]];
}

// lam[node] += sum over the node's receiver entries of fscale * res[rec][n].
__global__ void inject_kernel(float* __restrict__ lam, const long long* __restrict__ unode,
                              const int* __restrict__ uptr, const int* __restrict__ ucol,
                              const RecEntry* __restrict__ rec, const int* __restrict__ colmap,
                              const float* __restrict__ res, int nt, int n, int n_nodes) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_nodes) return;
  float s = 0.0f;
  for (int e = uptr[k]; e < uptr[k + 1]; ++e) {
    const int c = ucol[e];
    s = fmaf(rec[c].fscale, res[(long long)colmap[c] * nt + n], s);
  }
  lam[unode[k]] += s;
}

__global__ void adj1_kernel(CpmlAdjArgs c) {
  const VolDesc V = c.vols[blockIdx.y];
  for_points(V, [&](Pt p) {
    const long long i = idx(V, p.x, p.y, p.z);
    const float l = c.lam[i];
    const int bb = V.border, zi = p.z - bb, yi = p.y - bb, xi = p.x - bb;
    if (xi >= 0 && xi < V.nxi && yi >= 0 && yi < V.nyi && zi >= 0 && zi < V.nzi)
      c.acc[i] = fmaf(l, c.tstore[V.toff + ((long long)zi * V.nyi + yi) * V.tpitch + (p.x - V.txoff)],
                      c.acc[i]);
    const long long g = ((long long)p.z * c.NyG + (p.y + V.cy0)) * c.pitchG + (p.x + V.cx0);
    const float xb = c.A[g] * l;
    c.xb[i] = xb;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float b, cc;
      prof(c.pr, V, p, a, b, cc);
      if (in_layer(b, cc)) {
        const float zt = c.zetab[a][i] + xb;
        c.y[a][i] = cc * zt;
        c.zetab[a][i] = b * zt;
      } else {
        c.y[a][i] = 0.0f;
      }
    }
  });
}

__global__ void adj2_kernel(CpmlAdjArgs c) {
  const VolDesc V = c.vols[blockIdx.y];
  for_points(V, [&](Pt p) {
    const long long i = idx(V, p.x, p.y, p.z);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float b, cc;
      prof(c.pr, V, p, a, b, cc);
      if (in_layer(b, cc)) {
        const float pt = c.psib[a][i] - (d1(c.xb, V, p, a) + d1(c.y[a], V, p, a));
        c.psib[a][i] = b * pt;
        c.z[a][i] = cc * pt;
      } else {
        c.z[a][i] = 0.0f;
      }
    }
  });
}

__global__ void adj3_kernel(CpmlAdjArgs c) {
  const VolDesc V = c.vols[blockIdx.y];
  for_points(V, [&](Pt p) {
    const long long i = idx(V, p.x, p.y, p.z);
    const long long g = ((long long)p.z * c.NyG + (p.y + V.cy0)) * c.pitchG + (p.x + V.cx0);
    const float l = c.lam[i];
    const float M = c.M ? c.M[g] : 0.0f;
    float s = fmaf(2.0f, l, -M * l) + c.mu[i];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (near_layer(V, p, a))
        s += (d2(c.xb, V, p, a) + d2(c.y[a], V, p, a)) - d1(c.z[a], V, p, a);
      else
        s += d2(c.xb, V, p, a);
    }
    c.mu[i] = s;     // becomes lam of the previous step (the host swaps the roles)
    c.lam[i] = -l;   // becomes mu
  });
}

dim3 grid_for(int n_vol, long long max_pts) {
  long long b = (max_pts + 255) / 256;
  const long long cap = std::max(1LL, 152LL * 8 / n_vol);
  if (b > cap) b = cap;
  return dim3((unsigned)(b < 1 ? 1 : b), (unsigned)n_vol);
}

}  // namespace

cudaError_t launch_cpml_forward(const CpmlArgs& c, int n_vol, long long max_pts, cudaStream_t s) {
  const dim3 g = grid_for(n_vol, max_pts);
  psi_kernel<<<g, 256, 0, s>>>(c);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  step_kernel_pml<<<g, 256, 0, s>>>(c);
  return cudaGetLastError();
}

cudaError_t launch_cpml_record(const float* u, const long long* node, const RecEntry* rec, int ncol,
                               float* dout, cudaStream_t s) {
  if (ncol <= 0) return cudaSuccess;
  record_kernel<<<(ncol + 127) / 128, 128, 0, s>>>(u, node, rec, ncol, dout);
  return cudaGetLastError();
}

cudaError_t launch_cpml_inject(float* lam, const long long* unode, const int* uptr,
                               const int* ucol, const RecEntry* rec, const int* colmap,
                               const float* res, int nt, int n, int n_nodes, cudaStream_t s) {
  if (n_nodes <= 0) return cudaSuccess;
  inject_kernel<<<(n_nodes + 127) / 128, 128, 0, s>>>(lam, unode, uptr, ucol, rec, colmap, res, nt,
                                                      n, n_nodes);
  return cudaGetLastError();
}

cudaError_t launch_cpml_adjoint(const CpmlAdjArgs& c, int n_vol, long long max_pts, cudaStream_t s) {
  const dim3 g = grid_for(n_vol, max_pts);
  adj1_kernel<<<g, 256, 0, s>>>(c);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  adj2_kernel<<<g, 256, 0, s>>>(c);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  adj3_kernel<<<g, 256, 0, s>>>(c);
  return cudaGetLastError();
}

}  // namespace mamute
