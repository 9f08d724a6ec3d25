// 3x3x3 'same' convolutions of the preconditioner network, BF16 in, FP32
// accumulate, on the tensor cores (mma.sync m16n8k16), with the loss and
// optimizer kernels that train it.
//
// Activations are channels-last [D][H][W][16] BF16 (fewer channels are
// zero-padded to 16); weights are [27 taps][16 out][16 in] BF16 for the
// forward product, with a flipped, transposed copy for the input gradient.
// A CTA owns a 16 (x) x 8 (y) tile of one z plane; each warp one row of 16
// voxels.  Per tap the 16 voxels x 16 input channels A fragment and the
// 16 x 16 weight B fragments come from shared memory through ldmatrix.
#include "conv.h"

#include <algorithm>

#include "common.cuh"

namespace mamute {

namespace {

constexpr int kTX = 16, kTY = 8;                       // output tile
constexpr int kHX = kTX + 2, kHY = kTY + 2, kHZ = 3;   // input halo tile
constexpr int kC = 16;                                 // channels (padded)
constexpr int kTaps = 27;

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float bf2f(uint16_t v) { return __uint_as_float((uint32_t)v << 16); }

__device__ __forceinline__ uint16_t f2bf(float f) {  // round to nearest even
  uint32_t u = __float_as_uint(f);
  if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)((u >> 16) | ((u & 0xffff) ? 0x40 : 0));
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

// Loads the (3, kHY, kHX) x 16-channel halo tile around (z, y0 - 1, x0 - 1)
// (zero outside the volume) as 16-byte halves.
__device__ __forceinline__ void load_halo(uint4* halo, const uint16_t* __restrict__ x, int D, int H,
                                          int W, int z, int y0, int x0) {
  for (int i = threadIdx.x; i < kHZ * kHY * kHX * 2; i += blockDim.x) {
    const int half = i & 1, v = i >> 1;
    const int hx = v % kHX, hy = (v / kHX) % kHY, hz = v / (kHX * kHY);
    const int gx = x0 + hx - 1, gy = y0 + hy - 1, gz = z + hz - 1;
    uint4 val = make_uint4(0, 0, 0, 0);
    if (gx >= 0 && gx < W && gy >= 0 && gy < H && gz >= 0 && gz < D)
      val = reinterpret_cast<const uint4*>(x + (((long long)gz * H + gy) * W + gx) * kC)[half];
    halo[i] = val;
  }
}

__global__ void __launch_bounds__(256) conv_fwd_kernel(ConvArgs a) {
  __shared__ __align__(128) uint4 halo[kHZ * kHY * kHX * 2];
  __shared__ __align__(128) uint4 wsm[kTaps * kC * 2];
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY, z = blockIdx.z;
  load_halo(halo, a.x, a.D, a.H, a.W, z, y0, x0);
  for (int i = threadIdx.x; i < kTaps * kC * 2; i += blockDim.x)
    wsm[i] = reinterpret_cast<const uint4*>(a.w)[i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mat = lane >> 3, r = lane & 7;
  float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
  const char* hb = reinterpret_cast<const char*>(halo);
  const char* wb = reinterpret_cast<const char*>(wsm);
  // A rows: voxel r + 8 (mat & 1), channel half (mat >> 1).
  const int avox = r + 8 * (mat & 1), ahalf = mat >> 1;
  // B rows: out channel r + 8 (mat >> 1), input-channel half (mat & 1).
  const int bco = r + 8 * (mat >> 1), bhalf = mat & 1;
#pragma unroll 3
  for (int tap = 0; tap < kTaps; ++tap) {
    const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
    uint32_t af[4], bf[4];
    const int hv = (dz * kHY + warp + dy) * kHX + dx + avox;
    ldsm_x4(af, hb + hv * 32 + ahalf * 16);
    ldsm_x4(bf, wb + (tap * kC + bco) * 32 + bhalf * 16);
    mma16816(acc[0], af, bf[0], bf[1]);
    mma16816(acc[1], af, bf[2], bf[3]);
  }
  // Epilogue: thread holds voxels g, g + 8 and channels nt*8 + 2t, +1.
  const int g = lane >> 2, t = lane & 3;
  const int y = y0 + warp;
  if (y >= a.H) return;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int xx = x0 + g + 8 * h;
    if (xx >= a.W) continue;
    const long long vox = ((long long)z * a.H + y) * a.W + xx;
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      const int co = nt * 8 + 2 * t;
      float v0 = acc[nt][2 * h] + (a.bias ? a.bias[co] : 0.f);
      float v1 = acc[nt][2 * h + 1] + (a.bias ? a.bias[co + 1] : 0.f);
      if (a.relu) {
        v0 = fmaxf(v0, 0.f);
        v1 = fmaxf(v1, 0.f);
      }
      if (a.mask) {
        if (!(bf2f(a.mask[vox * kC + co]) > 0.f)) v0 = 0.f;
        if (!(bf2f(a.mask[vox * kC + co + 1]) > 0.f)) v1 = 0.f;
      }
      if (a.y32) *reinterpret_cast<float2*>(a.y32 + vox * kC + co) = make_float2(v0, v1);
      if (a.y16)
        *reinterpret_cast<uint32_t*>(a.y16 + vox * kC + co) =
            (uint32_t)f2bf(v0) | ((uint32_t)f2bf(v1) << 16);
    }
  }
}

// Weight gradient: per CTA partial sums over its tiles of
// gw[tap][o][i] = sum_p gy[p][o] x[p + tap - 1][i] and gb[o] = sum_p gy[p][o].
__global__ void __launch_bounds__(256) conv_wgrad_kernel(WgradArgs a) {
  __shared__ __align__(128) uint4 halo[kHZ * kHY * kHX * 2];
  __shared__ __align__(128) uint4 gys[kTY * kTX * 2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mat = lane >> 3, r = lane & 7;
  // Taps of this warp: warp, warp + 8, warp + 16, warp + 24 (< 27).
  float acc[4][2][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;
  float bacc = 0.f;
  const int tiles_x = (a.W + kTX - 1) / kTX, tiles_y = (a.H + kTY - 1) / kTY;
  const long long n_tiles = (long long)tiles_x * tiles_y * a.D;
  const char* hb = reinterpret_cast<const char*>(halo);
  const char* gb = reinterpret_cast<const char*>(gys);
  for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int tx = (int)(tile % tiles_x), ty = (int)((tile / tiles_x) % tiles_y);
    const int z = (int)(tile / ((long long)tiles_x * tiles_y));
    const int x0 = tx * kTX, y0 = ty * kTY;
    __syncthreads();
    load_halo(halo, a.x, a.D, a.H, a.W, z, y0, x0);
    for (int i = threadIdx.x; i < kTY * kTX * 2; i += blockDim.x) {
      const int half = i & 1, v = i >> 1, vx = v % kTX, vy = v / kTX;
      const int xx = x0 + vx, yy = y0 + vy;
      uint4 val = make_uint4(0, 0, 0, 0);
      if (xx < a.W && yy < a.H)
        val = reinterpret_cast<const uint4*>(a.gy + (((long long)z * a.H + yy) * a.W + xx) * kC)[half];
      gys[i] = val;
    }
    __syncthreads();
    if (threadIdx.x < kC) {
      const uint16_t* g16 = reinterpret_cast<const uint16_t*>(gys);
      for (int v = 0; v < kTY * kTX; ++v) bacc += bf2f(g16[v * kC + threadIdx.x]);
    }
    for (int row = 0; row < kTY; ++row) {  // k step: the 16 voxels of one row
      uint32_t af[4];
      // A = gy^T: rows voxel r + 8 (mat >> 1), channel half (mat & 1), transposed.
      ldsm_x4_t(af, gb + (row * kTX + r + 8 * (mat >> 1)) * 32 + (mat & 1) * 16);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int tap = warp + 8 * i;
        if (tap < kTaps) {
          const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
          uint32_t bf[4];
          // B = shifted x: rows voxel r + 8 (mat & 1), channel half (mat >> 1), transposed.
          const int hv = (dz * kHY + row + dy) * kHX + dx + r + 8 * (mat & 1);
          ldsm_x4_t(bf, hb + hv * 32 + (mat >> 1) * 16);
          mma16816(acc[i][0], af, bf[0], bf[1]);
          mma16816(acc[i][1], af, bf[2], bf[3]);
        }
      }
    }
  }
  // Partial sums: d0 = (o = g, i = nt*8 + 2t), d1 = (g, +1), d2/d3 rows g + 8.
  const int g = lane >> 2, t = lane & 3;
  float* part = a.partial + (long long)blockIdx.x * (kTaps * kC * kC + kC);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int tap = warp + 8 * i;
    if (tap >= kTaps) continue;
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      const int ci = nt * 8 + 2 * t;
      float* p = part + tap * kC * kC;
      p[g * kC + ci] = acc[i][nt][0];
      p[g * kC + ci + 1] = acc[i][nt][1];
      p[(g + 8) * kC + ci] = acc[i][nt][2];
      p[(g + 8) * kC + ci + 1] = acc[i][nt][3];
    }
  }
  if (threadIdx.x < kC) part[kTaps * kC * kC + threadIdx.x] = bacc;
}

// Fixed-order sum of the per-CTA partials: gw [27][16][16], gb [16].
__global__ void wgrad_reduce_kernel(const float* __restrict__ partial, int n_parts,
                                    float* __restrict__ gw, float* __restrict__ gb) {
  const int n = kTaps * kC * kC + kC;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int p = 0; p < n_parts; ++p) s += partial[(long long)p * n + i];
    if (i < kTaps * kC * kC) gw[i] = (float)s;
    else gb[i - kTaps * kC * kC] = (float)s;
  }
}

// Forward and input-gradient BF16 weights from FP32 masters [27][o][i]:
// fwd[tap][o][i] = w[tap][o][i]; bwd[26 - tap][i][o] = w[tap][o][i].
__global__ void pack_kernel(const float* __restrict__ w, uint16_t* __restrict__ fwd,
                            uint16_t* __restrict__ bwd) {
  const int n = kTaps * kC * kC;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int tap = e / (kC * kC), o = (e / kC) % kC, i = e % kC;
    const uint16_t v = f2bf(w[e]);
    fwd[e] = v;
    if (bwd) bwd[((kTaps - 1 - tap) * kC + i) * kC + o] = v;
  }
}

// Mean squared error of channel 0 against the target over the masked
// voxels, FP64 partials; gy channel 0 = 2 (out - t) m / n_mask (BF16), other
// channels 0.
__global__ void mse_kernel(long long N, const float* __restrict__ out, const float* __restrict__ tgt,
                           const float* __restrict__ mask, double inv_n, uint16_t* __restrict__ gy,
                           double* __restrict__ partial) {
  __shared__ double red[256];
  double acc = 0.0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
       p += (long long)gridDim.x * blockDim.x) {
    const float m = mask ? mask[p] : 1.0f;
    const double r = ((double)out[p * kC] - (double)tgt[p]) * (double)m;
    acc += r * r;
    uint4* gp = reinterpret_cast<uint4*>(gy + p * kC);
    gp[0] = make_uint4(f2bf((float)(2.0 * r * inv_n)), 0, 0, 0);
    gp[1] = make_uint4(0, 0, 0, 0);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0] * inv_n;
}

__global__ void sum_kernel(const double* partial, int n, double* out) {
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += partial[i];
    *out = s;
  }
}

// Adam (Kingma and Ba 2015) with bias correction, FP32 master weights.
__global__ void adam_kernel(int n, float* __restrict__ p, float* __restrict__ m,
                            float* __restrict__ v, const float* __restrict__ g, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// Network inputs: channel 0 = (c - v_ref) / v_scale, channel 1 =
// max(log(P / Pmax), -lclip) / lclip, other channels 0 (BF16); target =
// log(H / P) when H is given.
__global__ void features_kernel(long long N, const float* __restrict__ vel,
                                const float* __restrict__ ph, const float* __restrict__ hd,
                                const unsigned int* __restrict__ pmax_bits, float v_ref,
                                float v_scale, float lclip, uint16_t* __restrict__ x16,
                                float* __restrict__ target) {
  const float pmax = fmaxf(__uint_as_float(*pmax_bits), 1e-30f);
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
       p += (long long)gridDim.x * blockDim.x) {
    const float c = (vel[p] - v_ref) / v_scale;
    const float lp = fmaxf(logf(fmaxf(ph[p], 1e-30f) / pmax), -lclip) / lclip;
    uint4* xp = reinterpret_cast<uint4*>(x16 + p * kC);
    xp[0] = make_uint4((uint32_t)f2bf(c) | ((uint32_t)f2bf(lp) << 16), 0, 0, 0);
    xp[1] = make_uint4(0, 0, 0, 0);
    if (hd && target) target[p] = logf(fmaxf(hd[p], 1e-30f) / fmaxf(ph[p], 1e-30f));
  }
}

__global__ void absmax_kernel(const float* v, long long n, unsigned int* out) {
  float m = 0.0f;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(v[p]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

}  // namespace

cudaError_t launch_features(long long N, const float* vel, const float* ph, const float* hd,
                            unsigned int* pmax_bits, float v_ref, float v_scale, float lclip,
                            uint16_t* x16, float* target, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(pmax_bits, 0, 4, s);
  if (e != cudaSuccess) return e;
  const int blocks = (int)std::min<long long>((N + 255) / 256, 152 * 16);
  absmax_kernel<<<blocks, 256, 0, s>>>(ph, N, pmax_bits);
  features_kernel<<<blocks, 256, 0, s>>>(N, vel, ph, hd, pmax_bits, v_ref, v_scale, lclip, x16,
                                         target);
  return cudaGetLastError();
}

int wgrad_blocks() { return 152 * 4; }
size_t wgrad_partial_floats() { return (size_t)wgrad_blocks() * (kTaps * kC * kC + kC); }
int mse_blocks() { return 152 * 4; }

cudaError_t launch_conv(const ConvArgs& a, cudaStream_t s) {
  dim3 grid((a.W + kTX - 1) / kTX, (a.H + kTY - 1) / kTY, a.D);
  conv_fwd_kernel<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_wgrad(const WgradArgs& a, float* gw, float* gb, cudaStream_t s) {
  conv_wgrad_kernel<<<wgrad_blocks(), 256, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  wgrad_reduce_kernel<<<(kTaps * kC * kC + kC + 255) / 256, 256, 0, s>>>(a.partial, wgrad_blocks(),
                                                                         gw, gb);
  return cudaGetLastError();
}

cudaError_t launch_pack(const float* w, uint16_t* fwd, uint16_t* bwd, cudaStream_t s) {
  pack_kernel<<<(kTaps * kC * kC + 255) / 256, 256, 0, s>>>(w, fwd, bwd);
  return cudaGetLastError();
}

cudaError_t launch_mse(long long N, const float* out, const float* tgt, const float* mask,
                       double n_mask, uint16_t* gy, double* partial, double* loss,
                       cudaStream_t s) {
  mse_kernel<<<mse_blocks(), 256, 0, s>>>(N, out, tgt, mask, 1.0 / n_mask, gy, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  sum_kernel<<<1, 32, 0, s>>>(partial, mse_blocks(), loss);
  return cudaGetLastError();
}

cudaError_t launch_adam(int n, float* p, float* m, float* v, const float* g, float lr, float b1,
                        float b2, float eps, int step, cudaStream_t s) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  adam_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, p, m, v, g, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

}  // namespace mamute
