// Per-model and per-shot kernels around the time loop: coefficient
// preparation, geometry scales, data layout changes, misfit and the final
// gradient / pseudo-Hessian assembly.
#include "aux.h"

namespace mamute {

namespace {

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// sqrt(rho) of the edge-replicated padded model at any integer node, from
// the per-cell FP64 square roots.
__device__ __forceinline__ double srho_at(const double* srho, int nx, int ny, int nz, int b, int i,
                                          int j, int k) {
  const int mi = clampi(i - b, 0, nx - 1), mj = clampi(j - b, 0, ny - 1), mk = clampi(k - b, 0, nz - 1);
  return srho[((long long)mk * ny + mj) * nx + mi];
}

__global__ void sqrt_kernel(const float* __restrict__ rho, long long n, double* __restrict__ out) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x)
    out[p] = sqrt((double)rho[p]);
}

// A = c^2 dt^2 / h^2 and M = c^2 dt^2 m2, m2 = lap(sqrt rho) / sqrt rho
// (Eq. 1 right), on the global padded grid; formed in FP64, stored FP32.
__global__ void prep_coef_kernel(CoefPrepArgs a) {
  const long long n = (long long)a.Nz * a.Ny * a.pitch;
  const double c[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(p % a.pitch);
    const int j = (int)((p / a.pitch) % a.Ny);
    const int k = (int)(p / ((long long)a.pitch * a.Ny));
    if (i >= a.Nx) {
      a.A[p] = 0.0f;
      if (a.M) a.M[p] = 0.0f;
      continue;
    }
    const int b = a.border;
    const int mi = clampi(i - b, 0, a.nx - 1), mj = clampi(j - b, 0, a.ny - 1),
              mk = clampi(k - b, 0, a.nz - 1);
    const double cv = (double)a.vel[((long long)mk * a.ny + mj) * a.nx + mi];
    const double A2 = cv * cv * a.dt * a.dt;
    a.A[p] = (float)(A2 / (a.h * a.h));
    if (a.M) {
      const double* sr = a.srho;
      const double s0 = srho_at(sr, a.nx, a.ny, a.nz, b, i, j, k);
      double sx = c[0] * s0, sy = c[0] * s0, sz = c[0] * s0;
      for (int m = 1; m <= 4; ++m) {
        sx += c[m] * (srho_at(sr, a.nx, a.ny, a.nz, b, i - m, j, k) +
                      srho_at(sr, a.nx, a.ny, a.nz, b, i + m, j, k));
        sy += c[m] * (srho_at(sr, a.nx, a.ny, a.nz, b, i, j - m, k) +
                      srho_at(sr, a.nx, a.ny, a.nz, b, i, j + m, k));
        sz += c[m] * (srho_at(sr, a.nx, a.ny, a.nz, b, i, j, k - m) +
                      srho_at(sr, a.nx, a.ny, a.nz, b, i, j, k + m));
      }
      const double m2 = (sx + sy + sz) / (a.h * a.h) / s0;
      a.M[p] = (float)(A2 * m2);
    }
  }
}

__global__ void max_kernel(const float* v, long long n, unsigned int* out) {
  float m = 0.0f;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(v[p]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// Receiver-node and source-corner scales from the model at their nodes,
// times the interpolation weights.
__global__ void geometry_kernel(GeomArgs a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < a.n_rec) {
    const long long cell = a.rec_cell[t];
    const double sr = a.rho ? sqrt((double)a.rho[cell]) : 1.0;
    const double cv = a.vel[cell];
    RecEntry& e = a.rec[t];
    const double w = e.wgt;
    e.fscale = (float)(w * sr);
    e.ascale = (float)(w * cv * cv * a.dt * a.dt * (double)a.rec_g[t] * sr);
  }
  if (t < a.n_src) {
    for (int c = 0; c < 8; ++c) {
      const long long cell = a.src_cell[8 * t + c];
      float sc = 0.0f;
      if (cell >= 0) {
        const double sr = a.rho ? sqrt((double)a.rho[cell]) : 1.0;
        sc = (float)((double)a.src_w[8 * t + c] * a.dt * a.dt / (a.h * a.h * a.h * sr));
      }
      a.vols[t].src_sc[c] = sc;
    }
  }
}

__global__ void combine_kernel(const float* __restrict__ ecol, const int* __restrict__ ptr,
                               const int* __restrict__ cols, int n_rec, int n0, int n1, int nt,
                               float* __restrict__ seis) {
  const int r = blockIdx.x;  // receivers on x (more than 65535 of them)
  if (r >= n_rec) return;
  const int b = ptr[r], e = ptr[r + 1];
  for (int n = n0 + blockIdx.y * blockDim.x + threadIdx.x; n < n1; n += gridDim.y * blockDim.x) {
    float v = 0.0f;
    for (int k = b; k < e; ++k) v += ecol[(long long)cols[k] * nt + n];
    seis[(long long)r * nt + n] = v;
  }
}

// seis[colmap[c]][n] = d_int[n][c] (32x32 tiles through shared memory).
__global__ void data_out_kernel(const float* __restrict__ d_int, const int* __restrict__ colmap,
                                int nt, int ncol, long long pitch, float* __restrict__ seis) {
  __shared__ float tile[32][33];
  const int c0 = blockIdx.x * 32, n0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int n = n0 + r, c = c0 + threadIdx.x;
    tile[r][threadIdx.x] = (n < nt && c < ncol) ? d_int[(long long)n * ncol + c] : 0.0f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int c = c0 + r, n = n0 + threadIdx.x;
    if (c < ncol && n < nt) seis[(long long)colmap[c] * pitch + n] = tile[threadIdx.x][r];
  }
}

// r_int[n][c] = (d_int[n][c] if given) - sign * src[colmap[c]][n]; per-block
// partial sums of 1/2 r^2 in FP64 (reduced in a fixed order afterwards).
__global__ void data_in_kernel(const float* __restrict__ src, const int* __restrict__ colmap,
                               int nt, int ncol, const float* __restrict__ d_int, float sign,
                               float* __restrict__ r_int, double* __restrict__ partial) {
  __shared__ float tile[32][33];
  __shared__ double red[32 * 8];
  const int c0 = blockIdx.x * 32, n0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int c = c0 + r, n = n0 + threadIdx.x;
    tile[r][threadIdx.x] = (c < ncol && n < nt) ? src[(long long)colmap[c] * nt + n] : 0.0f;
  }
  __syncthreads();
  double acc = 0.0;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int n = n0 + r, c = c0 + threadIdx.x;
    if (n < nt && c < ncol) {
      const long long idx = (long long)n * ncol + c;
      const float v = (d_int ? d_int[idx] : 0.0f) - sign * tile[threadIdx.x][r];
      r_int[idx] = v;
      acc += 0.5 * (double)v * (double)v;
    }
  }
  const int t = threadIdx.y * 32 + threadIdx.x;
  red[t] = acc;
  __syncthreads();
  if (t == 0 && partial) {
    double s = 0.0;
    for (int k = 0; k < 32 * (int)blockDim.y; ++k) s += red[k];
    partial[blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
}

// Misfit over two arrays in the same layout (the user's [n_rec][nt]): block b
// reduces samples [b * kMisfitChunk, (b + 1) * kMisfitChunk) into partial[b];
// the total is then formed by one warp in a fixed order.  Neither depends on
// the work decomposition of the time-step kernels.
constexpr long long kMisfitChunk = 16384;

__global__ void misfit_partial_kernel(const float* __restrict__ d, const float* __restrict__ dobs,
                                      long long n, double* __restrict__ partial) {
  __shared__ double red[256];
  const long long b = (long long)blockIdx.x * kMisfitChunk;
  const long long e = b + kMisfitChunk < n ? b + kMisfitChunk : n;
  double acc = 0.0;
  for (long long i = b + threadIdx.x; i < e; i += 256) {
    const float r = d[i] - dobs[i];
    acc += 0.5 * (double)r * (double)r;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void warp_total_kernel(const double* __restrict__ partial, int n, double* out) {
  const int lane = threadIdx.x & 31;
  const int per = (n + 31) / 32;
  const int b = lane * per, e = b + per < n ? b + per : n;
  double s = 0.0;
  for (int k = b; k < e; ++k) s += partial[k];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) *out = s;
}

__global__ void sum_partials_kernel(const double* partial, int n, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += partial[k];
    *out = s;
  }
}

// grad[z][y][x] = 2 / (c^3 dt^2) sum_s G_s, or phess = sum_s P_s / (c dt)^4,
// summed over shots in ascending order (deterministic).
__global__ void finalize_kernel(FinalizeArgs a) {
  const long long n = (long long)a.nx * a.ny * a.nz;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(p % a.nx), y = (int)((p / a.nx) % a.ny), z = (int)(p / ((long long)a.nx * a.ny));
    const int X = x + a.border, Y = y + a.border, Z = z + a.border;
    float acc = 0.0f;
    for (int s = 0; s < a.n_vol; ++s) {
      const VolDesc& V = a.vols[s];
      // the window's imaging region (its cells inside the model)
      const int lx = X - V.cx0, ly = Y - V.cy0;
      if (lx < V.ix0 || ly < V.iy0 || lx >= V.ix0 + V.nxi || ly >= V.iy0 + V.nyi) continue;
      acc += a.acc[V.off + ((long long)Z * V.Ny + ly) * V.pitch + lx];
    }
    const double cv = a.vel[p];
    double out;
    if (a.kind == 0) {
      out = 2.0 * (double)acc / (cv * cv * cv * a.dt * a.dt);
      if (z < a.zero_top) out = 0.0;
    } else {
      const double A2 = cv * cv * a.dt * a.dt;
      out = (double)acc / (A2 * A2);
    }
    a.out[p] = (float)out;
  }
}

int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

cudaError_t launch_prep_coef(const CoefPrepArgs& a, cudaStream_t s) {
  if (a.M) {
    const long long nm = (long long)a.nx * a.ny * a.nz;
    sqrt_kernel<<<grid_for(nm, 256), 256, 0, s>>>(a.rho, nm, a.srho);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const long long n = (long long)a.Nz * a.Ny * a.pitch;
  prep_coef_kernel<<<grid_for(n, 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_max(const float* v, long long n, unsigned int* out, cudaStream_t s) {
  max_kernel<<<grid_for(n, 256), 256, 0, s>>>(v, n, out);
  return cudaGetLastError();
}

cudaError_t launch_geometry(const GeomArgs& a, cudaStream_t s) {
  const int n = a.n_rec > a.n_src ? a.n_rec : a.n_src;
  if (n == 0) return cudaSuccess;
  geometry_kernel<<<(n + 127) / 128, 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_data_out(const float* d_int, const int* colmap, int nt, int ncol, float* seis,
                            cudaStream_t s) {
  if (ncol == 0) return cudaSuccess;
  dim3 g((ncol + 31) / 32, (nt + 31) / 32), b(32, 8);
  data_out_kernel<<<g, b, 0, s>>>(d_int, colmap, nt, ncol, nt, seis);
  return cudaGetLastError();
}

cudaError_t launch_data_out_range(const float* d_int, const int* colmap, int n0, int n1, int nt,
                                  int ncol, float* seis, cudaStream_t s) {
  if (ncol == 0 || n1 <= n0) return cudaSuccess;
  dim3 g((ncol + 31) / 32, (n1 - n0 + 31) / 32), b(32, 8);
  data_out_kernel<<<g, b, 0, s>>>(d_int + (long long)n0 * ncol, colmap, n1 - n0, ncol, nt,
                                  seis + n0);
  return cudaGetLastError();
}

cudaError_t launch_combine(const float* ecol, const int* ptr, const int* cols, int n_rec, int n0,
                           int n1, int nt, float* seis, cudaStream_t s) {
  if (n_rec == 0 || n1 <= n0) return cudaSuccess;
  const int by = (n1 - n0 + 127) / 128;
  dim3 g(n_rec, by < 8 ? by : 8);
  combine_kernel<<<g, 128, 0, s>>>(ecol, ptr, cols, n_rec, n0, n1, nt, seis);
  return cudaGetLastError();
}

int data_in_blocks(int nt, int ncol) { return ((ncol + 31) / 32) * ((nt + 31) / 32); }

cudaError_t launch_data_in(const float* src, const int* colmap, int nt, int ncol,
                           const float* d_int, float sign, float* r_int, double* partial,
                           double* total, cudaStream_t s) {
  if (ncol == 0) return cudaSuccess;
  dim3 g((ncol + 31) / 32, (nt + 31) / 32), b(32, 8);
  data_in_kernel<<<g, b, 0, s>>>(src, colmap, nt, ncol, d_int, sign, r_int, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !total) return e;
  sum_partials_kernel<<<1, 32, 0, s>>>(partial, g.x * g.y, total);
  return cudaGetLastError();
}

int misfit_blocks(long long n) { return (int)((n + kMisfitChunk - 1) / kMisfitChunk); }

cudaError_t launch_misfit(const float* d, const float* dobs, long long n, double* partial,
                         double* total, cudaStream_t s) {
  if (n <= 0) return cudaMemsetAsync(total, 0, sizeof(double), s);
  misfit_partial_kernel<<<misfit_blocks(n), 256, 0, s>>>(d, dobs, n, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  warp_total_kernel<<<1, 32, 0, s>>>(partial, misfit_blocks(n), total);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const FinalizeArgs& a, cudaStream_t s) {
  const long long n = (long long)a.nx * a.ny * a.nz;
  finalize_kernel<<<grid_for(n, 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace mamute
