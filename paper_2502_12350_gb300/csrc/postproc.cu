// Gradient smoothing filters and seismic-data time resampling.
//
// Smoothing (Sec. 2, FWI gradient preconditioning: Bessel or Laplace filter
// with lengths lx, ly, lz; Algorithm 3: GradientPreconditioning).  Both
// filters are inverses of constant-coefficient operators built from the
// 3-point second difference with reflecting ends, which the orthonormal
// DCT-II diagonalises along each axis with eigenvalues
//   lambda_a(k) = 4 (l_a / h)^2 sin^2(pi k / (2 n_a)).
// The Bessel filter (I - sum_a l_a^2 D_aa)^-1 multiplies mode k by
// 1 / (1 + sum_a lambda_a), the Laplace filter prod_a (I - l_a^2 D_aa)^-1 by
// prod_a 1 / (1 + lambda_a).  The transform along an axis is a dense
// n x n contraction applied to every line of the volume (axis_kernel, a
// shared-memory tiled FP32 product); forward along x, y, z, the spectral
// scaling, and the transposed transforms along z, y, x give the exact solve.
//
// Resampling (Sec. 2: time interpolation by nearest neighbour or sinc;
// Table 1 Interpolate).  The resampling of every trace is the same sparse
// matrix, built on the host in FP64 (see api.cu); each of its rows covers a
// contiguous run of input samples, so it is stored as a band (first column,
// length, tap-major weights) and applied to every trace by band_rows_kernel
// (one thread per output sample and kBT traces, each weight loaded once for
// them); its transpose is another banded matrix.
#include "postproc.h"

namespace mamute {

namespace {

// Block tile: kTL lines x kTI outputs over chunks of kTK inputs; each of the
// 256 threads accumulates kRL lines x kRI outputs, reading them from shared
// memory as float4s (3 loads per 32 FMAs).
constexpr int kTL = 128, kTI = 64, kTK = 16, kRL = 8, kRI = 4;
constexpr int kAP = kTL + 4;  // A row pitch: float4-aligned, x-axis stores spread over banks

// out[L, i] = sum_j M[i][j] in[L, j] for the lines L of one axis:
// element (L, j) sits at (L / inner) * outer + (L % inner) + j * astride.
__global__ void __launch_bounds__(256) axis_kernel(const float* __restrict__ in,
                                                   float* __restrict__ out,
                                                   const float* __restrict__ M, int n,
                                                   long long lines, long long inner,
                                                   long long outer, long long astride) {
  __shared__ __align__(16) float As[kTK][kAP];
  __shared__ __align__(16) float Bs[kTK][kTI];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const long long L0 = (long long)blockIdx.x * kTL;
  const int i0 = blockIdx.y * kTI;
  // The kTL x kTK elements of a chunk are 8 per thread, at the same lines and
  // chunk columns in every chunk, so the line offsets are computed once.
  // Along x (astride 1) consecutive threads take consecutive j (the lines are
  // a row apart); along y and z consecutive lines (inner-contiguous).
  constexpr int kAQ = kTL * kTK / 256;
  const bool xaxis = astride == 1;
  long long abase[kAQ];
  int al[kAQ], ajj[kAQ];
#pragma unroll
  for (int q = 0; q < kAQ; ++q) {
    const int e = threadIdx.x + 256 * q;
    al[q] = xaxis ? e / kTK : e % kTL;
    ajj[q] = xaxis ? e % kTK : e / kTL;
    const long long L = L0 + al[q];
    abase[q] = L < lines ? (L / inner) * outer + (L % inner) : -1;
  }
  float acc[kRL][kRI] = {};
  for (int j0 = 0; j0 < n; j0 += kTK) {
#pragma unroll
    for (int q = 0; q < kAQ; ++q) {
      const int j = j0 + ajj[q];
      As[ajj[q]][al[q]] = (abase[q] >= 0 && j < n) ? in[abase[q] + (long long)j * astride] : 0.0f;
    }
#pragma unroll
    for (int q = 0; q < kTI * kTK / 256; ++q) {
      const int e = threadIdx.x + 256 * q;
      const int jj = e % kTK, ii = e / kTK;
      const int i = i0 + ii, j = j0 + jj;
      Bs[jj][ii] = (i < n && j < n) ? M[(long long)i * n + j] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kTK; ++k) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[k][ty * kRL]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[k][ty * kRL + 4]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[k][tx * kRI]);
      const float a[kRL] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bb[kRI] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int r = 0; r < kRL; ++r)
#pragma unroll
        for (int c = 0; c < kRI; ++c) acc[r][c] = fmaf(a[r], bb[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < kRL; ++r) {
    const long long L = L0 + ty * kRL + r;
    if (L >= lines) continue;
    const long long base = (L / inner) * outer + (L % inner);
#pragma unroll
    for (int c = 0; c < kRI; ++c) {
      const int i = i0 + tx * kRI + c;
      if (i < n) out[base + (long long)i * astride] = acc[r][c];
    }
  }
}

// Spectral multiplier of the filter on DCT coefficients [nz][ny][nx].
__global__ void scale_kernel(float* __restrict__ u, int nx, int ny, int nz,
                             const float* __restrict__ lam, int mode) {
  const long long n = (long long)nx * ny * nz;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(p % nx), y = (int)((p / nx) % ny), z = (int)(p / ((long long)nx * ny));
    const float lx = lam[x], ly = lam[nx + y], lz = lam[nx + ny + z];
    const float m = mode == 1 ? 1.0f / (1.0f + lx + ly + lz)
                              : 1.0f / ((1.0f + lx) * (1.0f + ly) * (1.0f + lz));
    u[p] *= m;
  }
}

constexpr int kBT = 8;  // traces per thread

__global__ void band_rows_kernel(const float* __restrict__ x, int n_in, const int* __restrict__ c0,
                                 const int* __restrict__ len, const float* __restrict__ w,
                                 int n_out, int n_traces, float* __restrict__ y) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n_out) return;
  const int c = c0[m], L = len[m];
  const int ngroup = (n_traces + kBT - 1) / kBT;
  for (int tg = blockIdx.y; tg < ngroup; tg += gridDim.y) {
    const int t0 = tg * kBT;
    const float* xr[kBT];
    float acc[kBT];
#pragma unroll
    for (int t = 0; t < kBT; ++t) {
      xr[t] = x + (long long)min(t0 + t, n_traces - 1) * n_in + c;
      acc[t] = 0.0f;
    }
    for (int j = 0; j < L; ++j) {
      const float wj = __ldg(w + (long long)j * n_out + m);
#pragma unroll
      for (int t = 0; t < kBT; ++t) acc[t] = fmaf(wj, __ldg(xr[t] + j), acc[t]);
    }
#pragma unroll
    for (int t = 0; t < kBT; ++t)
      if (t0 + t < n_traces) y[(long long)(t0 + t) * n_out + m] = acc[t];
  }
}

__global__ void sub_kernel(const float* __restrict__ a, const float* __restrict__ b, long long n,
                           float* __restrict__ out) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x)
    out[p] = a[p] - b[p];
}

}  // namespace

cudaError_t launch_sub(const float* a, const float* b, long long n, float* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  long long blk = (n + 255) / 256;
  if (blk > 152 * 16) blk = 152 * 16;
  sub_kernel<<<(unsigned)blk, 256, 0, s>>>(a, b, n, out);
  return cudaGetLastError();
}

cudaError_t launch_axis(const float* in, float* out, const float* M, int n, long long lines,
                        long long inner, long long outer, long long astride, cudaStream_t s) {
  if (lines <= 0 || n <= 0) return cudaSuccess;
  dim3 g((unsigned)((lines + kTL - 1) / kTL), (unsigned)((n + kTI - 1) / kTI));
  axis_kernel<<<g, 256, 0, s>>>(in, out, M, n, lines, inner, outer, astride);
  return cudaGetLastError();
}

cudaError_t launch_spectral_scale(float* u, int nx, int ny, int nz, const float* lam, int mode,
                                  cudaStream_t s) {
  const long long n = (long long)nx * ny * nz;
  long long b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  scale_kernel<<<(unsigned)b, 256, 0, s>>>(u, nx, ny, nz, lam, mode);
  return cudaGetLastError();
}

cudaError_t launch_band_rows(const float* x, int n_in, const int* c0, const int* len,
                             const float* w, int n_out, int n_traces, float* y, cudaStream_t s) {
  if (n_traces <= 0 || n_out <= 0) return cudaSuccess;
  const int groups = (n_traces + kBT - 1) / kBT;
  dim3 g((unsigned)((n_out + 127) / 128), (unsigned)(groups < 65535 ? groups : 65535));
  band_rows_kernel<<<g, 128, 0, s>>>(x, n_in, c0, len, w, n_out, n_traces, y);
  return cudaGetLastError();
}

}  // namespace mamute
