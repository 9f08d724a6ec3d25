// Launch interface of the time-step kernels (internal to libmamute).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace mamute {

enum StepMode {
  MODE_FWD = 0,
  MODE_FWD_PH = 1,
  MODE_FWD_STORE = 2,
  MODE_ADJ = 3,
  MODE_ADJ_STORED = 4,
  MODE_ADJ_TERM = 5,
  MODE_FWD_STORE_PH = 6,
};

struct StepArgs {
  const WorkItem* items;
  const VolDesc* vols;
  const ShotMaps* maps;
  const CoefMaps* cmaps;
  const float* gx;        // x profiles of all shots
  const float* gy;        // y profiles of all shots
  const float* gz;        // z profile (shared)
  // Tensor maps of the buffers this step reads, for shot 0; shot v uses
  // base + v * stride.
  const CUtensorMap* mF;  // halo map of the current level of the propagated field
  const CUtensorMap* mP;  // centre map of the previous level
  const CUtensorMap* mU;  // halo map of u^{k-1} (adjoint imaging)
  int sF, sP, sU;
  float wn;               // wavelet sample of this step (forward)
  float* fout;            // pool receiving the new level (buffer fcur ^ 1)
  float* acc;             // accumulator pool (pseudo-Hessian or imaging)
  float* tstore;          // imaging-term store for this step (all-states mode)
  int tstep;              // step index of the term read by the all-states adjoint
  const int* rec_ptr;     // per-item per-plane receiver offsets
  const RecEntry* rec;    // receiver entries
  float* dout;            // forward: data row of this step (internal columns), may be null
  const float* rin;       // adjoint: residual row injected at this step
  int* status;            // error flags
  int zs;                 // padded plane of a free surface (odd image above it), -1 if none
};

bool tile_supported(int tx, int ty);
// Resident CTAs per SM of a step kernel configuration (0 if it cannot run).
int step_blocks_per_sm(int tx, int ty, bool dens, int mode, int max_planes);
// max_planes: the largest ze - zb of the launch's items (sizes the per-plane table).
cudaError_t launch_step(const StepArgs& a, int n_items, int max_planes, int tx, int ty, bool dens,
                        int mode, cudaStream_t s);

}  // namespace mamute
