// Convolutional PML (Sec. 2: the second absorbing boundary, after Roden and
// Gedney) for modelling and for the gradient.
//
// In the layer each derivative d/dx_a is (1/s_a) d/dx_a, s_a = 1 + d_a /
// (alpha_a + i w), and the second derivative is carried by two memory
// variables per axis, updated by recursive convolution.  With the unscaled
// eighth-order stencils D2_a (weights c0..c4) and D1_a (4/5, -1/5, 4/105,
// -1/280) and the memory variables scaled by h and h^2 (so that the update
// uses A = c^2 dt^2 / h^2 like the damping kernels):
//   Psi_a'  = b_a Psi_a  + c_a D1_a u
//   Zeta_a' = b_a Zeta_a + c_a (D2_a u + D1_a Psi_a')
//   u'      = (2 - M) u - v + A (lap u + sum_a (D1_a Psi_a' + Zeta_a')) + source
// with b_a = exp(-(d_a + alpha_a) dt), c_a = d_a (b_a - 1) / (d_a + alpha_a)
// (profiles built on the host; b = 1, c = 0 outside the layer).  The main
// step kernel forms (2 - M) u - v + A lap u + source everywhere (damping
// factor 1); the kernels here add the memory-variable part of each axis on
// that axis's layer slabs, where it is non-zero, and the same amount to the
// stored imaging term A lap u - M u.
//
// The gradient is the exact transpose of this recursion.  In the adjoint
// level psi (the multiplier of u scaled by A, which the main kernel
// propagates with the forward operator itself), one reverse step is
//   per axis, in the layer:  y_a = c_a (Zb_a + psi),  Zb_a <- b_a (Zb_a + psi)
//                            p_a = Pb_a - D1_a (psi + y_a),  Pb_a <- b_a p_a,  z_a = c_a p_a
//   main adjoint step:       psi' = (2 - M) psi - psi_prev + A lap psi + injection
//   correction (per axis):   psi' += A sum_a (D2_a y_a - D1_a z_a)
// (Zb, Pb the multipliers of Zeta and Psi; D2 is symmetric, D1 antisymmetric,
// the fields are zero outside the padded window), and the imaging
// accumulator takes the corrected psi' against the stored term.
#include "cpml.h"

#include <algorithm>

namespace mamute {

namespace {

__constant__ float kC2[5] = {MAMUTE_C0, MAMUTE_C1, MAMUTE_C2, MAMUTE_C3, MAMUTE_C4};
__constant__ float kD1[4] = {4.0f / 5.0f, -1.0f / 5.0f, 4.0f / 105.0f, -1.0f / 280.0f};

constexpr int kZG = 4;  // cells per load group of the marching kernels

struct Pt {
  int x, y, z;
};

__device__ __forceinline__ long long idx(const VolDesc& V, int x, int y, int z) {
  return V.off + ((long long)z * V.Ny + y) * V.pitch + x;
}

// Element stride of axis a in a window's arrays.
__device__ __forceinline__ long long axis_stride(const VolDesc& V, int a) {
  return a == 0 ? 1LL : (a == 1 ? (long long)V.pitch : (long long)V.Ny * V.pitch);
}

// Neighbours p - 4 .. p + 4 along axis a of the point at element i (zero
// outside the window; the bounds are tested only near the window's faces).
// No kernel writes an array that it reads this way, so the loads take the
// read-only path and may be issued ahead of the kernel's stores.
__device__ __forceinline__ void column(const float* f, const VolDesc& V, Pt p, int a, long long i,
                                       float (&v)[9]) {
  const int q = a == 0 ? p.x : (a == 1 ? p.y : p.z);
  const int N = a == 0 ? V.Nx : (a == 1 ? V.Ny : V.Nz);
  const long long st = axis_stride(V, a);
  if (q >= 4 && q + 4 < N) {
#pragma unroll
    for (int m = -4; m <= 4; ++m) v[m + 4] = __ldg(f + i + m * st);
  } else {
#pragma unroll
    for (int m = -4; m <= 4; ++m) v[m + 4] = (q + m >= 0 && q + m < N) ? __ldg(f + i + m * st) : 0.0f;
  }
}

__device__ __forceinline__ float d2(const float* f, const VolDesc& V, Pt p, int a, long long i) {
  float v[9];
  column(f, V, p, a, i, v);
  float s = kC2[0] * v[4];
#pragma unroll
  for (int m = 1; m <= 4; ++m) s = fmaf(kC2[m], v[4 + m] + v[4 - m], s);
  return s;
}

__device__ __forceinline__ float d1(const float* f, const VolDesc& V, Pt p, int a, long long i) {
  float v[9];
  column(f, V, p, a, i, v);
  float s = 0.0f;
#pragma unroll
  for (int m = 1; m <= 4; ++m) s = fmaf(kD1[m - 1], v[4 + m] - v[4 - m], s);
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

// Index of p in the imaging-region layout, or -1 outside the region.
__device__ __forceinline__ long long region_index(const VolDesc& V, Pt p) {
  const int zi = p.z - V.border, yi = p.y - V.iy0, xi = p.x - V.ix0;
  if (xi < 0 || xi >= V.nxi || yi < 0 || yi >= V.nyi || zi < 0 || zi >= V.nzi) return -1;
  return V.toff + ((long long)zi * V.nyi + yi) * V.tpitch + (p.x - V.txoff);
}

// The slab pair of width w across axis A (2: z, 1: y) of window V, marched
// along A: blockIdx.z = 0 takes [0, lo), 1 takes [hi, N) with lo = min(w, N),
// hi = max(N - w, lo); one thread per column across the other two axes (x
// fastest), at element i0 with the marched coordinate 0 and element stride st.
// With merge, slabs less than 8 cells apart are marched as one range [0, N)
// by the blockIdx.z = 0 threads (for kernels whose queues reach 4 cells past
// their range into values that the range's own march writes).
template <int A>
struct Slab {
  int s0, s1;
  unsigned ncol;
  long long st, stA;  // strides along A in the window and in the coefficient grid
  __device__ __forceinline__ bool init(const VolDesc& V, const CpmlArgs& c, int w,
                                       bool merge = false) {
    const int N = A == 2 ? V.Nz : V.Ny;
    const int lo = min(w, N), hi = max(N - w, lo);
    s0 = blockIdx.z == 0 ? 0 : hi;
    s1 = blockIdx.z == 0 ? lo : N;
    if (merge && hi - lo < 8) {
      s0 = 0;
      s1 = blockIdx.z == 0 ? N : 0;
    }
    ncol = (unsigned)V.Nx * (unsigned)(A == 2 ? V.Ny : V.Nz);
    st = A == 2 ? (long long)V.Ny * V.pitch : (long long)V.pitch;
    stA = A == 2 ? (long long)c.NyG * c.pitchG : (long long)c.pitchG;
    return s0 < s1;
  }
  __device__ __forceinline__ Pt column(const VolDesc& V, unsigned q) const {
    const unsigned o = q / (unsigned)V.Nx;
    Pt p;
    p.x = (int)(q - o * (unsigned)V.Nx);
    p.y = A == 2 ? (int)o : 0;
    p.z = A == 2 ? 0 : (int)o;
    return p;
  }
  __device__ __forceinline__ static void at(Pt& p, int s) {
    if (A == 2)
      p.z = s;
    else
      p.y = s;
  }
  __device__ __forceinline__ static void profile(const CpmlProf& pr, const VolDesc& V, int s, float& b,
                                                 float& cc) {
    b = A == 2 ? pr.bz[s] : pr.by[V.gy_off + s];
    cc = A == 2 ? pr.cz[s] : pr.cy[V.gy_off + s];
  }
};

// Calls f(p) for every point within w cells of an x face of window V, one
// point per thread of the blockIdx.x range (x fastest, then y, then z).
template <typename F>
__device__ __forceinline__ void for_xslab(const VolDesc& V, int w, F f) {
  const int lx = min(w, V.Nx), hx = max(V.Nx - w, lx);
  const unsigned nx3 = (unsigned)(lx + V.Nx - hx);
  // fewer than 2^32 points (windows are checked on the host): 32-bit indices
  const long long n = (long long)nx3 * V.Ny * V.Nz;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const unsigned q32 = (unsigned)q;
    const unsigned r = q32 / nx3, zz = r / (unsigned)V.Ny;
    const int xx = (int)(q32 - r * nx3);
    Pt p;
    p.x = xx < lx ? xx : hx + (xx - lx);
    p.y = (int)(r - zz * (unsigned)V.Ny);
    p.z = (int)zz;
    f(p);
  }
}

// f at coordinate s of the column starting at element i0 (zero outside
// [0, N)); f is not written by the kernel that reads it this way.
__device__ __forceinline__ float sval(const float* f, long long i0, long long st, int s, int N) {
  return (s >= 0 && s < N) ? __ldg(f + i0 + s * st) : 0.0f;
}

__device__ __forceinline__ float d1q(const float (&v)[9]) {
  float s = 0.0f;
#pragma unroll
  for (int m = 1; m <= 4; ++m) s = fmaf(kD1[m - 1], v[4 + m] - v[4 - m], s);
  return s;
}

__device__ __forceinline__ float d2q(const float (&v)[9]) {
  float s = kC2[0] * v[4];
#pragma unroll
  for (int m = 1; m <= 4; ++m) s = fmaf(kC2[m], v[4 + m] + v[4 - m], s);
  return s;
}

__device__ __forceinline__ void shift(float (&v)[9], float next) {
#pragma unroll
  for (int m = 0; m < 8; ++m) v[m] = v[m + 1];
  v[8] = next;
}

__device__ __forceinline__ float coefA(const CpmlArgs& c, const VolDesc& V, Pt p) {
  return c.A[((long long)p.z * c.NyG + (p.y + V.cy0)) * c.pitchG + (p.x + V.cx0)];
}

// ---------------------------------------------------------------- forward
//
// Each axis's terms live in its own pair of layer slabs, so each update
// runs as one launch per axis: for z and y a kernel that marches the slab
// along the axis with one thread per column (x fastest), the neighbours
// along the axis in register queues and the loads of kZG cells issued
// before their stores; for x one point per thread, the x neighbours coming
// from the same cache lines as the neighbouring threads' points.  The
// correction adds each axis's part to u^{n+1} (and to the stored term) in
// turn.

template <int A>
__global__ void __launch_bounds__(256, 4) psi_march_kernel(CpmlArgs c) {
  const VolDesc V = c.vols[blockIdx.y];
  Slab<A> S;
  if (!S.init(V, c, V.border)) return;
  const int N = A == 2 ? V.Nz : V.Ny;
  for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < S.ncol; q += gridDim.x * blockDim.x) {
    const Pt p = S.column(V, q);
    const long long i0 = idx(V, p.x, p.y, p.z);
    float v[9];  // u at s - 4 .. s + 4
#pragma unroll
    for (int m = 0; m < 9; ++m) v[m] = sval(c.u, i0, S.st, S.s0 - 4 + m, N);
    for (int sg = S.s0; sg < S.s1; sg += kZG) {
      float mv[kZG], un[kZG], b[kZG], cc[kZG];
#pragma unroll
      for (int k = 0; k < kZG; ++k) {
        const int s = sg + k;
        b[k] = 1.0f;
        cc[k] = 0.0f;
        if (s < S.s1) Slab<A>::profile(c.pr, V, s, b[k], cc[k]);
        mv[k] = in_layer(b[k], cc[k]) ? c.m1[A][i0 + s * S.st] : 0.0f;
        un[k] = sval(c.u, i0, S.st, s + 5, N);
      }
#pragma unroll
      for (int k = 0; k < kZG; ++k) {
        if (in_layer(b[k], cc[k])) c.m1[A][i0 + (sg + k) * S.st] = fmaf(b[k], mv[k], cc[k] * d1q(v));
        shift(v, un[k]);
      }
    }
  }
}

template <int A>
__global__ void __launch_bounds__(256, 3) fcorr_march_kernel(CpmlArgs c) {
  const VolDesc V = c.vols[blockIdx.y];
  Slab<A> S;
  if (!S.init(V, c, V.border + 4)) return;
  const int N = A == 2 ? V.Nz : V.Ny;
  for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < S.ncol; q += gridDim.x * blockDim.x) {
    Pt p = S.column(V, q);
    const long long i0 = idx(V, p.x, p.y, p.z);
    const float* Acol = c.A + ((long long)p.z * c.NyG + (p.y + V.cy0)) * c.pitchG + (p.x + V.cx0);
    float um[9], pm[9];  // u and Psi_A at s - 4 .. s + 4
#pragma unroll
    for (int m = 0; m < 9; ++m) {
      um[m] = sval(c.u, i0, S.st, S.s0 - 4 + m, N);
      pm[m] = sval(c.m1[A], i0, S.st, S.s0 - 4 + m, N);
    }
    for (int sg = S.s0; sg < S.s1; sg += kZG) {
      float zt[kZG], o[kZG], ag[kZG], un[kZG], pn[kZG], b[kZG], cc[kZG];
#pragma unroll
      for (int k = 0; k < kZG; ++k) {
        const int s = sg + k;
        const bool in = s < S.s1;
        b[k] = 1.0f;
        cc[k] = 0.0f;
        if (in) Slab<A>::profile(c.pr, V, s, b[k], cc[k]);
        zt[k] = in_layer(b[k], cc[k]) ? c.m2[A][i0 + s * S.st] : 0.0f;
        o[k] = in ? c.out[i0 + s * S.st] : 0.0f;
        ag[k] = in ? __ldg(Acol + s * S.stA) : 0.0f;
        un[k] = sval(c.u, i0, S.st, s + 5, N);
        pn[k] = sval(c.m1[A], i0, S.st, s + 5, N);
      }
#pragma unroll
      for (int k = 0; k < kZG; ++k) {
        const int s = sg + k;
        if (s < S.s1) {  // every slab point is within border + 4 cells of a face across A
          const long long i = i0 + s * S.st;
          const float d1p = d1q(pm);
          float zn = 0.0f;
          if (in_layer(b[k], cc[k])) {
            zn = fmaf(b[k], zt[k], cc[k] * (d2q(um) + d1p));
            c.m2[A][i] = zn;
          }
          const float d = ag[k] * (d1p + zn);
          c.out[i] = o[k] + d;
          if (c.tstore) {
            Slab<A>::at(p, s);
            const long long r = region_index(V, p);
            if (r >= 0) c.tstore[r] += d;
          }
        }
        shift(um, un[k]);
        shift(pm, pn[k]);
      }
    }
  }
}

__global__ void psi_x_kernel(CpmlArgs c) {
  const VolDesc V = c.vols[blockIdx.y];
  for_xslab(V, V.border, [&](Pt p) {
    const long long i = idx(V, p.x, p.y, p.z);
    float b, cc;
    prof(c.pr, V, p, 0, b, cc);
    if (in_layer(b, cc)) c.m1[0][i] = fmaf(b, c.m1[0][i], cc * d1(c.u, V, p, 0, i));
  });
}

__global__ void fcorr_x_kernel(CpmlArgs c) {
  const VolDesc V = c.vols[blockIdx.y];
  for_xslab(V, V.border + 4, [&](Pt p) {
    const long long i = idx(V, p.x, p.y, p.z);
    const float d1p = d1(c.m1[0], V, p, 0, i);
    float b, cc;
    prof(c.pr, V, p, 0, b, cc);
    float zt = 0.0f;
    if (in_layer(b, cc)) {
      zt = fmaf(b, c.m2[0][i], cc * (d2(c.u, V, p, 0, i) + d1p));
      c.m2[0][i] = zt;
    }
    const float d = coefA(c, V, p) * (d1p + zt);
    c.out[i] += d;
    if (c.tstore) {
      const long long r = region_index(V, p);
      if (r >= 0) c.tstore[r] += d;
    }
  });
}

__global__ void record_kernel(const float* __restrict__ u, const long long* __restrict__ node,
                              const RecEntry* __restrict__ rec, int ncol, float* __restrict__ dout) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < ncol) dout[c] = rec[c].fscale * u[node[c]];
}

// ---------------------------------------------------------------- reverse
//
// One launch per axis and update, as in the forward pass.  For z and y one
// marched kernel forms both multipliers: y_a is pointwise, so it is made as
// each cell enters the register queue (its Zeta multiplier updated in the
// same place), and p_a once the cell's neighbours along a are in the queue.
// Where the two layers along a are less than 8 cells apart, one thread
// marches the whole column, so that no queue reads a y_a another thread is
// making.  For x, y_x comes from a pointwise kernel and p_x from one point
// per thread.  The correction adds each axis's part to psi^k and to the
// imaging accumulator in turn.

// Profile of cell s along A (b = 1, c = 0 outside the window).
template <int A>
__device__ __forceinline__ void prof_at(const CpmlProf& pr, const VolDesc& V, int N, int s, float& b,
                                        float& cc) {
  b = 1.0f;
  cc = 0.0f;
  if (s >= 0 && s < N) Slab<A>::profile(pr, V, s, b, cc);
}

template <int A>
__global__ void __launch_bounds__(256, 2) pre_march_kernel(CpmlArgs c) {
  const VolDesc V = c.vols[blockIdx.y];
  Slab<A> S;
  if (!S.init(V, c, V.border, true)) return;
  const int N = A == 2 ? V.Nz : V.Ny;
  for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < S.ncol; q += gridDim.x * blockDim.x) {
    const Pt p = S.column(V, q);
    const long long i0 = idx(V, p.x, p.y, p.z);
    // y_A of a cell entering the queue, c (Zb + psi) with Zb <- b (Zb + psi)
    // in the layer, zero elsewhere (zb: the cell's Zeta multiplier)
    auto enter = [&](int s, float psi, float zb, float b, float cc) -> float {
      if (!in_layer(b, cc)) return 0.0f;
      const long long i = i0 + s * S.st;
      const float zt = zb + psi;
      const float y = cc * zt;
      c.y[A][i] = y;
      c.m2[A][i] = b * zt;
      return y;
    };
    float ps[9], yq[9];  // psi^{k+1} and y_A at s - 4 .. s + 4
#pragma unroll
    for (int m = 0; m < 9; ++m) {
      const int s = S.s0 - 4 + m;
      float b, cc;
      prof_at<A>(c.pr, V, N, s, b, cc);
      ps[m] = sval(c.u, i0, S.st, s, N);
      const float zb = in_layer(b, cc) ? c.m2[A][i0 + s * S.st] : 0.0f;
      yq[m] = enter(s, ps[m], zb, b, cc);
    }
    for (int sg = S.s0; sg < S.s1; sg += kZG) {
      // loads of the group: the cells entering (sg + 5 ..) and finishing (sg ..)
      float pn[kZG], zb[kZG], be[kZG], ce[kZG], mv[kZG], bf[kZG], cf[kZG];
#pragma unroll
      for (int k = 0; k < kZG; ++k) {
        const int e = sg + 5 + k, f = sg + k;
        prof_at<A>(c.pr, V, N, e, be[k], ce[k]);
        pn[k] = sval(c.u, i0, S.st, e, N);
        zb[k] = in_layer(be[k], ce[k]) ? c.m2[A][i0 + e * S.st] : 0.0f;
        prof_at<A>(c.pr, V, f < S.s1 ? N : 0, f, bf[k], cf[k]);
        mv[k] = in_layer(bf[k], cf[k]) ? c.m1[A][i0 + f * S.st] : 0.0f;
      }
#pragma unroll
      for (int k = 0; k < kZG; ++k) {
        if (in_layer(bf[k], cf[k])) {
          const long long i = i0 + (sg + k) * S.st;
          const float pt = mv[k] - (d1q(ps) + d1q(yq));
          c.m1[A][i] = bf[k] * pt;
          c.z[A][i] = cf[k] * pt;
        }
        const float ye = enter(sg + 5 + k, pn[k], zb[k], be[k], ce[k]);
        shift(ps, pn[k]);
        shift(yq, ye);
      }
    }
  }
}

template <int A>
__global__ void __launch_bounds__(256, 3) acorr_march_kernel(CpmlArgs c) {
  const VolDesc V = c.vols[blockIdx.y];
  Slab<A> S;
  if (!S.init(V, c, V.border + 4)) return;
  const int N = A == 2 ? V.Nz : V.Ny;
  for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < S.ncol; q += gridDim.x * blockDim.x) {
    Pt p = S.column(V, q);
    const long long i0 = idx(V, p.x, p.y, p.z);
    const float* Acol = c.A + ((long long)p.z * c.NyG + (p.y + V.cy0)) * c.pitchG + (p.x + V.cx0);
    float yq[9], zq[9];  // y_A and z_A at s - 4 .. s + 4
#pragma unroll
    for (int m = 0; m < 9; ++m) {
      yq[m] = sval(c.y[A], i0, S.st, S.s0 - 4 + m, N);
      zq[m] = sval(c.z[A], i0, S.st, S.s0 - 4 + m, N);
    }
    for (int sg = S.s0; sg < S.s1; sg += kZG) {
      float yn[kZG], zn[kZG], o[kZG], ac[kZG], ag[kZG], ts[kZG];
      long long r[kZG];
#pragma unroll
      for (int k = 0; k < kZG; ++k) {
        const int f = sg + k;
        const bool in = f < S.s1;
        const long long i = i0 + f * S.st;
        yn[k] = sval(c.y[A], i0, S.st, f + 5, N);
        zn[k] = sval(c.z[A], i0, S.st, f + 5, N);
        o[k] = in ? c.out[i] : 0.0f;
        ag[k] = in ? __ldg(Acol + f * S.stA) : 0.0f;
        Slab<A>::at(p, f);
        r[k] = in ? region_index(V, p) : -1;
        ts[k] = r[k] >= 0 ? __ldg(c.tstore + r[k]) : 0.0f;
        ac[k] = r[k] >= 0 ? c.acc[i] : 0.0f;
      }
#pragma unroll
      for (int k = 0; k < kZG; ++k) {
        if (sg + k < S.s1) {  // every slab point is within border + 4 cells of a face across A
          const long long i = i0 + (sg + k) * S.st;
          const float d = ag[k] * (d2q(yq) - d1q(zq));
          c.out[i] = o[k] + d;
          if (r[k] >= 0) c.acc[i] = fmaf(d, ts[k], ac[k]);
        }
        shift(yq, yn[k]);
        shift(zq, zn[k]);
      }
    }
  }
}

__global__ void y_x_kernel(CpmlArgs c) {
  const VolDesc V = c.vols[blockIdx.y];
  for_xslab(V, V.border, [&](Pt p) {
    const long long i = idx(V, p.x, p.y, p.z);
    float b, cc;
    prof(c.pr, V, p, 0, b, cc);
    if (in_layer(b, cc)) {
      const float zt = c.m2[0][i] + c.u[i];
      c.y[0][i] = cc * zt;
      c.m2[0][i] = b * zt;
    }
  });
}

__global__ void z_x_kernel(CpmlArgs c) {
  const VolDesc V = c.vols[blockIdx.y];
  for_xslab(V, V.border, [&](Pt p) {
    const long long i = idx(V, p.x, p.y, p.z);
    float b, cc;
    prof(c.pr, V, p, 0, b, cc);
    if (in_layer(b, cc)) {
      const float pt = c.m1[0][i] - (d1(c.u, V, p, 0, i) + d1(c.y[0], V, p, 0, i));
      c.m1[0][i] = b * pt;
      c.z[0][i] = cc * pt;
    }
  });
}

__global__ void acorr_x_kernel(CpmlArgs c) {
  const VolDesc V = c.vols[blockIdx.y];
  for_xslab(V, V.border + 4, [&](Pt p) {
    const long long i = idx(V, p.x, p.y, p.z);
    const float d = coefA(c, V, p) * (d2(c.y[0], V, p, 0, i) - d1(c.z[0], V, p, 0, i));
    c.out[i] += d;
    const long long r = region_index(V, p);
    if (r >= 0) c.acc[i] = fmaf(d, c.tstore[r], c.acc[i]);
  });
}

dim3 grid_for(int n_vol, long long max_pts) {
  long long b = (max_pts + 255) / 256;
  const long long cap = std::max(1LL, 152LL * 16 / n_vol);
  if (b > cap) b = cap;
  return dim3((unsigned)(b < 1 ? 1 : b), (unsigned)n_vol);
}

}  // namespace

// Both slabs of a marched axis (blockIdx.z), one thread per column.
dim3 march_grid(int n_vol, long long max_cols) {
  const long long b = std::min((max_cols + 255) / 256, 65535LL);
  return dim3((unsigned)std::max(1LL, b), (unsigned)n_vol, 2);
}

cudaError_t launch_cpml_psi(const CpmlArgs& c, int n_vol, const CpmlExtent& e, cudaStream_t s) {
  psi_march_kernel<2><<<march_grid(n_vol, e.xy), 256, 0, s>>>(c);
  psi_march_kernel<1><<<march_grid(n_vol, e.xz), 256, 0, s>>>(c);
  psi_x_kernel<<<grid_for(n_vol, 2LL * e.border * e.yz), 256, 0, s>>>(c);
  return cudaGetLastError();
}

cudaError_t launch_cpml_fcorr(const CpmlArgs& c, int n_vol, const CpmlExtent& e, cudaStream_t s) {
  fcorr_march_kernel<2><<<march_grid(n_vol, e.xy), 256, 0, s>>>(c);
  fcorr_march_kernel<1><<<march_grid(n_vol, e.xz), 256, 0, s>>>(c);
  fcorr_x_kernel<<<grid_for(n_vol, 2LL * (e.border + 4) * e.yz), 256, 0, s>>>(c);
  return cudaGetLastError();
}

cudaError_t launch_cpml_pre(const CpmlArgs& c, int n_vol, const CpmlExtent& e, cudaStream_t s) {
  pre_march_kernel<2><<<march_grid(n_vol, e.xy), 256, 0, s>>>(c);
  pre_march_kernel<1><<<march_grid(n_vol, e.xz), 256, 0, s>>>(c);
  const dim3 g = grid_for(n_vol, 2LL * e.border * e.yz);
  y_x_kernel<<<g, 256, 0, s>>>(c);
  z_x_kernel<<<g, 256, 0, s>>>(c);
  return cudaGetLastError();
}

cudaError_t launch_cpml_acorr(const CpmlArgs& c, int n_vol, const CpmlExtent& e, cudaStream_t s) {
  acorr_march_kernel<2><<<march_grid(n_vol, e.xy), 256, 0, s>>>(c);
  acorr_march_kernel<1><<<march_grid(n_vol, e.xz), 256, 0, s>>>(c);
  acorr_x_kernel<<<grid_for(n_vol, 2LL * (e.border + 4) * e.yz), 256, 0, s>>>(c);
  return cudaGetLastError();
}

cudaError_t launch_cpml_record(const float* u, const long long* node, const RecEntry* rec, int ncol,
                               float* dout, cudaStream_t s) {
  if (ncol <= 0) return cudaSuccess;
  record_kernel<<<(ncol + 127) / 128, 128, 0, s>>>(u, node, rec, ncol, dout);
  return cudaGetLastError();
}

}  // namespace mamute
