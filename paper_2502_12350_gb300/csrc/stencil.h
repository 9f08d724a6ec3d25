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

// Tensor maps of one shot for the two-level kernel (boxes of its tile):
//   [0] pool 0 halo  [1] pool 1 halo  [2] pool 0 centre  [3] pool 1 centre
//   [4] A centre     [5] A m2 centre
struct PairMaps {
  CUtensorMap m[6];
};

// Arguments of one two-level launch (steps n and n + 1, n even: u^n in pool
// 0, u^{n-1} in pool 1).
struct PairArgs {
  const WorkItem* items;  // one per tile, all planes
  const int4* nbrs;       // items of the four xy neighbours of each tile (-1: none)
  const VolDesc* vols;
  const PairMaps* pmaps;
  const float* gx;
  const float* gy;
  const float* gz;
  float wn0, wn1;         // wavelet samples of the two steps
  float* fout1;           // pool 1: receives u^{n+1}
  float* fout2;           // pool 0: receives u^{n+2}
  const int* rec_ptr;     // per-item per-plane receiver offsets (pair tiling)
  const RecEntry* rec;
  float* dout0;           // data rows of the two steps (internal columns), may be null
  float* dout1;
  int* flags;             // per tile: planes of u^{n+1} stored, plus epoch
  int epoch;              // flag value before this launch
  int* status;
};

// Compiled tile shapes of the two-level kernel (TY even; 2 rows per thread).
#define MAMUTE_PAIR_TILES(X) X(72, 32) X(64, 32) X(32, 16)

bool pair_tile_supported(int tx, int ty);
// occ != null: writes the resident CTAs per SM instead of launching.
cudaError_t launch_pair(const PairArgs& a, int n_items, int nz, int tx, int ty, bool dens,
                        cudaStream_t s, int* occ);

bool tile_supported(int tx, int ty);
// Resident CTAs per SM of a step kernel configuration (0 if it cannot run).
int step_blocks_per_sm(int tx, int ty, bool dens, int mode, int max_planes);
// max_planes: the largest ze - zb of the launch's items (sizes the per-plane table).
cudaError_t launch_step(const StepArgs& a, int n_items, int max_planes, int tx, int ty, bool dens,
                        int mode, cudaStream_t s);

}  // namespace mamute
