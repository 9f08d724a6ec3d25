// Launch interface of the auxiliary kernels (internal to libmamute).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace mamute {

struct CoefPrepArgs {
  const float* vel;   // model [nz][ny][nx]
  const float* rho;   // model density or null
  int nx, ny, nz, border;
  int Nx, Ny, Nz, pitch;  // global padded grid
  double h, dt;
  float* A;           // [Nz][Ny][pitch]
  float* M;           // [Nz][Ny][pitch] or null
  double* srho;       // scratch [nz][ny][nx] (density only)
};

struct GeomArgs {
  const float* vel;
  const float* rho;
  int n_rec, n_src;
  const long long* rec_cell;  // model cell index per receiver entry
  const float* rec_g;         // sponge factor at the entry's node
  RecEntry* rec;
  const long long* src_cell;  // model cell of each of the 8 source-cell corners per shot (-1: unused)
  const float* src_w;         // interpolation weight of each corner
  VolDesc* vols;
  double h, dt;
};

struct FinalizeArgs {
  const float* acc;   // accumulator pool (read on each window's imaging region)
  const VolDesc* vols;
  int n_vol;
  const float* vel;   // model [nz][ny][nx]
  int nx, ny, nz, border;
  double dt;
  int kind;           // 0: gradient dJ/dc, 1: pseudo-Hessian
  int zero_top;
  float* out;         // [nz][ny][nx]
};

cudaError_t launch_prep_coef(const CoefPrepArgs& a, cudaStream_t s);
cudaError_t launch_max(const float* v, long long n, unsigned int* out, cudaStream_t s);
cudaError_t launch_geometry(const GeomArgs& a, cudaStream_t s);
cudaError_t launch_data_out(const float* d_int, const int* colmap, int nt, int ncol, float* seis,
                            cudaStream_t s);
// Samples [n0, n1) of the same transpose into seis rows of length nt.
cudaError_t launch_data_out_range(const float* d_int, const int* colmap, int n0, int n1, int nt,
                                  int ncol, float* seis, cudaStream_t s);
// seis[r][n] = sum over k in [ptr[r], ptr[r+1]) of ecol[cols[k]][n] (in
// that order), samples [n0, n1): receivers spread over several nodes.
cudaError_t launch_combine(const float* ecol, const int* ptr, const int* cols, int n_rec, int n0,
                           int n1, int nt, float* seis, cudaStream_t s);
int data_in_blocks(int nt, int ncol);
cudaError_t launch_data_in(const float* src, const int* colmap, int nt, int ncol,
                           const float* d_int, float sign, float* r_int, double* partial,
                           double* total, cudaStream_t s);
// J = 1/2 sum (d - dobs)^2 over n samples of two arrays in the same layout,
// FP64 partial sums in fixed blocks and a fixed-order total.
int misfit_blocks(long long n);
cudaError_t launch_misfit(const float* d, const float* dobs, long long n, double* partial,
                         double* total, cudaStream_t s);
cudaError_t launch_finalize(const FinalizeArgs& a, cudaStream_t s);

}  // namespace mamute
