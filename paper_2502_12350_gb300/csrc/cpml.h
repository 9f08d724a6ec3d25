// Launch interface of the convolutional-PML kernels (internal to libmamute).
//
// The CPML scheme is run as the damping-free main step (the TMA stencil
// kernels with g = 1, which form the whole update away from the layer) plus
// these kernels, which touch only the layer slabs of each shot window where
// the memory variables live or are read: per axis the `border` layer cells
// of its two faces, and 4 more cells inward where the eighth-order
// derivatives of the memory variables reach.
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

// Fields of one CPML launch, all in the pool layout of the shot windows
// (blockIdx.y selects the window) except A (global padded grid) and the
// term store / accumulator (imaging-region layout).
struct CpmlArgs {
  const VolDesc* vols;
  CpmlProf pr;
  const float* A;      // c^2 dt^2 / h^2 on the global padded grid
  int pitchG, NyG;     // layout of A
  const float* u;      // forward: u^n; reverse: the adjoint level being propagated (psi^{k+1})
  float* out;          // the main kernel's new level, corrected in place
  float* m1[3];        // forward: Psi_a (first memory variable, scaled by h); reverse: its multiplier
  float* m2[3];        // forward: Zeta_a (scaled by h^2); reverse: its multiplier
  float* y[3];         // reverse scratch: c_a (multiplier of Zeta_a + psi)
  float* z[3];         // reverse scratch: c_a p_a
  float* tstore;       // imaging term of this step (corrected in place, forward) or read (reverse); may be null
  float* acc;          // reverse: imaging accumulator (pool layout, corrected in place)
};

// Largest extents over the shot windows, for the grids of the forward kernels.
struct CpmlExtent {
  long long xy, xz, yz;  // Nx Ny, Nx Nz and Ny Nz of a window
  int border;            // layer width in cells
};

// Forward, before the main step: Psi_a <- b_a Psi_a + c_a D1_a u^n in the layer
// (one launch per axis: kCpmlAxisLaunches).
cudaError_t launch_cpml_psi(const CpmlArgs& c, int n_vol, const CpmlExtent& e, cudaStream_t s);
// Forward, after the main step: Zeta_a <- b_a Zeta_a + c_a (D2_a u^n + D1_a Psi_a) in the layer,
// u^{n+1} += A sum_a (D1_a Psi_a + Zeta_a) and the stored term likewise (one launch per axis).
cudaError_t launch_cpml_fcorr(const CpmlArgs& c, int n_vol, const CpmlExtent& e, cudaStream_t s);
constexpr int kCpmlAxisLaunches = 3;
// Reverse, before the main adjoint step: y_a, the Zeta multipliers, then p_a,
// the Psi multipliers and z_a, from the level psi^{k+1} (kCpmlPreLaunches
// launches: the marched z and y kernels, then y_x and p_x).
cudaError_t launch_cpml_pre(const CpmlArgs& c, int n_vol, const CpmlExtent& e, cudaStream_t s);
constexpr int kCpmlPreLaunches = 4;
// Reverse, after the main adjoint step: psi^k += A sum_a (D2_a y_a - D1_a z_a)
// and the imaging accumulator likewise (one launch per axis).
cudaError_t launch_cpml_acorr(const CpmlArgs& c, int n_vol, const CpmlExtent& e, cudaStream_t s);
// dout[c] = rec[c].fscale * u[node[c]] for the ncol internal data columns.
cudaError_t launch_cpml_record(const float* u, const long long* node, const RecEntry* rec, int ncol,
                               float* dout, cudaStream_t s);

}  // namespace mamute
