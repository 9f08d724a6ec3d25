// Instantiations of the adjoint time-step kernel (modes ADJ, ADJ_STORED, ADJ_TERM).
#include "stencil_impl.cuh"

namespace mamute {

cudaError_t dispatch_adjoint(const StepArgs& a, int n_items, int max_planes, int tx, int ty, bool dens,
                   int mode, cudaStream_t s, int* occ) {
  switch (mode) {
    case MODE_ADJ:
#define MAMUTE_T(TX, TY) \
  if (tx == TX && ty == TY) return launch_mode<TX, TY, MODE_ADJ>(a, n_items, max_planes, dens, s, occ);
      MAMUTE_TILES(MAMUTE_T)
#undef MAMUTE_T
      return cudaErrorInvalidValue;
    case MODE_ADJ_STORED:
#define MAMUTE_T(TX, TY) \
  if (tx == TX && ty == TY) return launch_mode<TX, TY, MODE_ADJ_STORED>(a, n_items, max_planes, dens, s, occ);
      MAMUTE_TILES(MAMUTE_T)
#undef MAMUTE_T
      return cudaErrorInvalidValue;
    case MODE_ADJ_TERM:
#define MAMUTE_T(TX, TY) \
  if (tx == TX && ty == TY) return launch_mode<TX, TY, MODE_ADJ_TERM>(a, n_items, max_planes, dens, s, occ);
      MAMUTE_TILES(MAMUTE_T)
#undef MAMUTE_T
      return cudaErrorInvalidValue;
  }
  return cudaErrorInvalidValue;
}

}  // namespace mamute
