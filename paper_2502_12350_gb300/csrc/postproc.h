// Launch interface of the smoothing and resampling kernels (internal to libmamute).
#pragma once

#include <cuda_runtime.h>

namespace mamute {

// out[L, i] = sum_j M[i][j] in[L, j] over the lines L of one axis of a
// volume; element (L, j) is at (L / inner) * outer + (L % inner) + j * astride.
cudaError_t launch_axis(const float* in, float* out, const float* M, int n, long long lines,
                        long long inner, long long outer, long long astride, cudaStream_t s);
// u[z][y][x] *= filter multiplier from lam = [lambda_x(nx) | lambda_y(ny) | lambda_z(nz)]
// (mode 1: Bessel, 2: Laplace).
cudaError_t launch_spectral_scale(float* u, int nx, int ny, int nz, const float* lam, int mode,
                                  cudaStream_t s);
// y[r][m] = sum_{j < len[m]} w[j][m] x[r][c0[m] + j] for every trace r: a
// banded matrix whose row m covers the contiguous columns c0[m] ..
// c0[m] + len[m] - 1, weights stored tap-major (w[j][m] at j n_out + m).
cudaError_t launch_band_rows(const float* x, int n_in, const int* c0, const int* len,
                             const float* w, int n_out, int n_traces, float* y, cudaStream_t s);

// out = a - b elementwise.
cudaError_t launch_sub(const float* a, const float* b, long long n, float* out, cudaStream_t s);

}  // namespace mamute
