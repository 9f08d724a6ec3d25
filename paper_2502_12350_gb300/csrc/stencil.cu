// Time-step kernel front end: supported tile shapes, occupancy and launch
// (the kernel itself is in stencil_impl.cuh, instantiated in stencil_fwd.cu
// and stencil_adj.cu).
#include "stencil_impl.cuh"

namespace mamute {

bool tile_supported(int tx, int ty) {
#define MAMUTE_T(TX, TY) if (tx == TX && ty == TY) return true;
  MAMUTE_TILES(MAMUTE_T)
#undef MAMUTE_T
  return false;
}

static cudaError_t dispatch(const StepArgs& a, int n_items, int max_planes, int tx, int ty,
                            bool dens, int mode, cudaStream_t s, int* occ) {
  if (mode == MODE_FWD || mode == MODE_FWD_PH || mode == MODE_FWD_STORE ||
      mode == MODE_FWD_STORE_PH)
    return dispatch_forward(a, n_items, max_planes, tx, ty, dens, mode, s, occ);
  return dispatch_adjoint(a, n_items, max_planes, tx, ty, dens, mode, s, occ);
}

int step_blocks_per_sm(int tx, int ty, bool dens, int mode, int max_planes) {
  int occ = 0;
  StepArgs a{};
  if (dispatch(a, 0, max_planes, tx, ty, dens, mode, nullptr, &occ) != cudaSuccess) return 0;
  return occ;
}

cudaError_t launch_step(const StepArgs& a, int n_items, int max_planes, int tx, int ty, bool dens,
                        int mode, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  return dispatch(a, n_items, max_planes, tx, ty, dens, mode, s, nullptr);
}

}  // namespace mamute
