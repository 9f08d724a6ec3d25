// Instantiations of the forward time-step kernel (modes FWD, FWD_PH, FWD_STORE,
// FWD_STORE_PH).
#include "stencil_impl.cuh"

namespace mamute {

cudaError_t dispatch_forward(const StepArgs& a, int n_items, int max_planes, int tx, int ty, bool dens,
                   int mode, cudaStream_t s, int* occ) {
  switch (mode) {
    case MODE_FWD:
#define MAMUTE_T(TX, TY) \
  if (tx == TX && ty == TY) return launch_mode<TX, TY, MODE_FWD>(a, n_items, max_planes, dens, s, occ);
      MAMUTE_TILES(MAMUTE_T)
#undef MAMUTE_T
      return cudaErrorInvalidValue;
    case MODE_FWD_PH:
#define MAMUTE_T(TX, TY) \
  if (tx == TX && ty == TY) return launch_mode<TX, TY, MODE_FWD_PH>(a, n_items, max_planes, dens, s, occ);
      MAMUTE_TILES(MAMUTE_T)
#undef MAMUTE_T
      return cudaErrorInvalidValue;
    case MODE_FWD_STORE:
#define MAMUTE_T(TX, TY) \
  if (tx == TX && ty == TY) return launch_mode<TX, TY, MODE_FWD_STORE>(a, n_items, max_planes, dens, s, occ);
      MAMUTE_TILES(MAMUTE_T)
#undef MAMUTE_T
      return cudaErrorInvalidValue;
    case MODE_FWD_STORE_PH:
#define MAMUTE_T(TX, TY) \
  if (tx == TX && ty == TY) return launch_mode<TX, TY, MODE_FWD_STORE_PH>(a, n_items, max_planes, dens, s, occ);
      MAMUTE_TILES(MAMUTE_T)
#undef MAMUTE_T
      return cudaErrorInvalidValue;
  }
  return cudaErrorInvalidValue;
}

}  // namespace mamute
