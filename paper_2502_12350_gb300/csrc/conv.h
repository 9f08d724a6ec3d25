// Launch interface of the network kernels (internal).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mamute {

struct ConvArgs {
  const uint16_t* x;     // [D][H][W][16] BF16
  const uint16_t* w;     // [27][16 out][16 in] BF16
  const float* bias;     // [16] or null
  int relu;
  const uint16_t* mask;  // [D][H][W][16] BF16 or null: output zeroed where mask <= 0
  float* y32;            // [D][H][W][16] or null
  uint16_t* y16;         // [D][H][W][16] or null
  int D, H, W;
};

struct WgradArgs {
  const uint16_t* x;     // layer input [D][H][W][16]
  const uint16_t* gy;    // output gradient [D][H][W][16]
  float* partial;        // wgrad_partial_floats() scratch
  int D, H, W;
};

int wgrad_blocks();
size_t wgrad_partial_floats();
int mse_blocks();
// TMA box of the tensor-core convolution's input map for a D x H x W
// volume: one halo plane of a row block, the activation viewed as
// [D][H][W][16] BF16 (innermost first: 16 channels, x, y, z), 32-byte
// swizzle, zero fill outside.
// Box of the forward convolution's halo-plane loads over the activation
// viewed as [D][H][4 W] 8-byte elements (no swizzle): {4 P, rows, 1, -}.
void conv_halo_box(int D, int H, int W, unsigned (&box)[4]);
cudaError_t launch_conv(const ConvArgs& a, const CUtensorMap& xmap, int* status, cudaStream_t s);
// Boxes of the weight-gradient kernel's maps over x (halo) and gy (tile),
// [D][H][W][16] BF16, 32-byte swizzle.
void conv_wgrad_halo_box(unsigned (&box)[4]);
void conv_gy_box(unsigned (&box)[4]);
cudaError_t launch_wgrad(const WgradArgs& a, const CUtensorMap& xmap, const CUtensorMap& gmap,
                         int* status, float* gw, float* gb, cudaStream_t s);
cudaError_t launch_pack(const float* w, uint16_t* fwd, uint16_t* bwd, cudaStream_t s);
cudaError_t launch_mse(long long N, const float* out, const float* tgt, const float* mask,
                       double n_mask, uint16_t* gy, double* partial, double* loss, cudaStream_t s);
cudaError_t launch_features(long long N, const float* vel, const float* ph, const float* hd,
                            unsigned int* pmax_bits, float v_ref, float v_scale, float lclip,
                            uint16_t* x16, float* target, cudaStream_t s);
cudaError_t launch_adam(int n, float* p, float* m, float* v, const float* g, float lr, float b1,
                        float b2, float eps, int step, cudaStream_t s);

}  // namespace mamute
