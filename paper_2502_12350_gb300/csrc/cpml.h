// Launch interface of the convolutional-PML kernels (internal to libmamute).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace mamute {

// Per-axis layer coefficients b = exp(-(d + alpha) dt), c = d (b - 1) / (d + alpha):
// x and y profiles of every shot window (at VolDesc gx_off / gy_off), z shared.
struct CpmlProf {
  const float* bx;
  const float* cx;
  const float* by;
  const float* cy;
  const float* bz;
  const float* cz;
};

// One forward step of one shot window (pools in the VolDesc layout).
struct CpmlArgs {
  const VolDesc* vols; // one shot window per blockIdx.y
  CpmlProf pr;
  const float* A;      // c^2 dt^2 / h^2 on the global padded grid
  const float* M;      // A m2 h^2 or null
  int pitchG, NyG;     // layout of A and M
  const float* u;      // u^n
  float* v;            // u^{n-1}, receives u^{n+1}
  float* psi[3];       // memory variables (scaled by h), per axis x, y, z
  float* zeta[3];      // (scaled by h^2)
  float wn;            // wavelet sample of the step
  float* tstore;       // imaging term x - m2 u of the step on the interior, or null
};

// One reverse step of one shot window.
struct CpmlAdjArgs {
  const VolDesc* vols; // one shot window per blockIdx.y
  CpmlProf pr;
  const float* A;
  const float* M;
  int pitchG, NyG;
  float* lam;          // multiplier of u^{n+1}; receives -lam (the next mu)
  float* mu;           // multiplier of u^n through the previous-level slot; receives the next lam
  float* xb;           // scratch: A lam
  float* y[3];         // scratch: c_a (zetab_a + xb)
  float* z[3];         // scratch: c_a p_a
  float* psib[3];      // multipliers of the memory variables
  float* zetab[3];
  float* acc;          // sum over steps of lam (x - m2 u), padded layout
  const float* tstore; // imaging term of the step
};

// psi update, then the step, of every window (max_pts: points of the largest).
cudaError_t launch_cpml_forward(const CpmlArgs& c, int n_vol, long long max_pts, cudaStream_t s);
// dout[c] = rec[c].fscale * u[node[c]] for the ncol internal data columns.
cudaError_t launch_cpml_record(const float* u, const long long* node, const RecEntry* rec, int ncol,
                               float* dout, cudaStream_t s);
// lam[unode[k]] += sum_{e in [uptr[k], uptr[k+1])} rec[c].fscale res[colmap[c]][n], c = ucol[e].
cudaError_t launch_cpml_inject(float* lam, const long long* unode, const int* uptr,
                               const int* ucol, const RecEntry* rec, const int* colmap,
                               const float* res, int nt, int n, int n_nodes, cudaStream_t s);
cudaError_t launch_cpml_adjoint(const CpmlAdjArgs& c, int n_vol, long long max_pts, cudaStream_t s);

}  // namespace mamute
