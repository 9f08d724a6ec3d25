// 3x3x3 'same' convolutions of the preconditioner network, BF16 in, FP32
// accumulate, with the loss and optimizer kernels that train it.  Forward
// and input-gradient convolutions run on tcgen05 (conv_tc.cuh); the weight
// gradient, a reduction over voxels, on mma.sync m16n8k16.
//
// Activations are channels-last [D][H][W][16] BF16 (fewer channels are
// zero-padded to 16); weights are [27 taps][16 out][16 in] BF16 for the
// forward product, with a flipped, transposed copy for the input gradient.
#include "conv.h"

#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "tcgen05.cuh"

namespace mamute {

namespace {

constexpr int kTX = 16, kTY = 8;                       // output tile
constexpr int kHX = kTX + 2, kHY = kTY + 2;           // input halo tile (3 planes)
constexpr int kC = 16;                                 // channels (padded)
constexpr int kTaps = 27;

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

// Tiles of the weight-gradient kernel: 16 (x) x 8 (y) x 4 (z) output
// voxels, the 18 x 10 x 6 input halo and the gy tile stored with the
// 32-byte TMA swizzle (the 16-byte channel halves of voxel v swap when bit 2
// of v is set, so ldmatrix rows of consecutive voxels hit distinct banks).
constexpr int kFZ = 4;                                  // output planes per tile
constexpr int kFHZ = kFZ + 2;                           // halo planes
constexpr int kFHalo = kFHZ * kHY * kHX * kC * 2;       // bytes per halo buffer
static_assert(kFHalo % 256 == 0, "halo buffers must stay 256-byte aligned");

__device__ __forceinline__ int swz(int v, int half) { return 2 * v + (half ^ ((v >> 2) & 1)); }

#include "conv_tc.cuh"

// Weight gradient: per CTA partial sums over its tiles of
// gw[tap][o][i] = sum_p gy[p][o] x[p + tap - 1][i] and gb[o] = sum_p gy[p][o].
// Persistent like the forward kernel: per 16 x 8 x 4 tile one TMA load
// brings the 18 x 10 x 6 halo of x and one the 16 x 8 x 4 tile of gy (both
// with the 32-byte swizzle) into a double buffer.  Warp w accumulates taps
// w, w + 8, w + 16, w + 24; per output row the A fragment is gy^T (16 out
// channels x 16 voxels) and the B fragment the shifted x row.  Warp 0 also
// sums gy for the bias from its A fragments.
constexpr int kGTile = kFZ * kTY * kTX * kC * 2;  // bytes of a gy tile
static_assert(kGTile % 256 == 0, "gy tiles must stay 256-byte aligned");
constexpr int kWStage = kFHalo + kGTile;

__device__ __forceinline__ float2 bf2x2(uint32_t v) {
  return make_float2(__uint_as_float(v << 16), __uint_as_float(v & 0xffff0000u));
}

__global__ void __launch_bounds__(256, 2)
    conv_wgrad_kernel(const __grid_constant__ CUtensorMap xmap,
                      const __grid_constant__ CUtensorMap gmap, WgradArgs a, int* status) {
  extern __shared__ unsigned char wsm_raw[];
  unsigned char* dsm = wsm_raw + ((256 - (smem_u32(wsm_raw) & 255)) & 255);
  __shared__ uint64_t bar[2];
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mat = lane >> 3, r = lane & 7;
  const int tiles_x = (a.W + kTX - 1) / kTX, tiles_y = (a.H + kTY - 1) / kTY;
  const int tiles_z = (a.D + kFZ - 1) / kFZ;
  const long long n_tiles = (long long)tiles_x * tiles_y * tiles_z;
  auto issue = [&](int b, long long t) {
    const int x0 = (int)(t % tiles_x) * kTX;
    const int y0 = (int)((t / tiles_x) % tiles_y) * kTY;
    const int z0 = (int)(t / ((long long)tiles_x * tiles_y)) * kFZ;
    unsigned char* st = dsm + b * kWStage;
    mbar_arrive_expect_tx(&bar[b], kWStage);
    tma_load_4d(st, &xmap, 0, x0 - 1, y0 - 1, z0 - 1, &bar[b]);
    tma_load_4d(st + kFHalo, &gmap, 0, x0, y0, z0, &bar[b]);
  };
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_barrier_init();
    abort_flag = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0 && (long long)blockIdx.x < n_tiles) issue(0, blockIdx.x);
  float acc[4][2][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;
  float bsum[2] = {0.f, 0.f};  // warp 0: out channels g and g + 8
  int it = 0;
  bool issued_next = false;
  for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++it) {
    const int b = it & 1;
    issued_next = threadIdx.x == 0 && tile + gridDim.x < n_tiles;
    if (issued_next) issue(b ^ 1, tile + gridDim.x);
    if (!mbar_wait(&bar[b], (uint32_t)((it >> 1) & 1), status)) abort_flag = 1;
    __syncthreads();
    if (abort_flag) {
      if (issued_next) mbar_wait(&bar[b ^ 1], (uint32_t)(((it + 1) >> 1) & 1), status);
      return;
    }
    const unsigned char* hb = dsm + b * kWStage;
    const unsigned char* gb = hb + kFHalo;
#pragma unroll 2
    for (int row = 0; row < kFZ * kTY; ++row) {  // k step: the 16 voxels of one output row
      const int oz = row / kTY, oy = row % kTY;
      uint32_t af[4];
      // A = gy^T: rows voxel r + 8 (mat >> 1), channel half (mat & 1), transposed.
      ldsm_x4_t(af, gb + swz(row * kTX + r + 8 * (mat >> 1), mat & 1) * 16);
      if (warp == 0) {
        const float2 p0 = bf2x2(af[0]), p1 = bf2x2(af[1]), p2 = bf2x2(af[2]), p3 = bf2x2(af[3]);
        bsum[0] += (p0.x + p0.y) + (p2.x + p2.y);
        bsum[1] += (p1.x + p1.y) + (p3.x + p3.y);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int tap = warp + 8 * i;
        if (tap < kTaps) {
          const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
          uint32_t bf[4];
          // B = shifted x: rows voxel r + 8 (mat & 1), channel half (mat >> 1), transposed.
          const int hv = ((oz + dz) * kHY + oy + dy) * kHX + dx + r + 8 * (mat & 1);
          ldsm_x4_t(bf, hb + swz(hv, mat >> 1) * 16);
          mma16816(acc[i][0], af, bf[0], bf[1]);
          mma16816(acc[i][1], af, bf[2], bf[3]);
        }
      }
    }
    __syncthreads();  // stage b is free for the load issued next iteration
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
  if (warp == 0) {
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
      bsum[0] += __shfl_xor_sync(0xffffffffu, bsum[0], o);
      bsum[1] += __shfl_xor_sync(0xffffffffu, bsum[1], o);
    }
    if (t == 0) {
      part[kTaps * kC * kC + g] = bsum[0];
      part[kTaps * kC * kC + g + 8] = bsum[1];
    }
  }
}

// Fixed-order sum of the per-CTA partials in two stages: groups of
// kRedGroup partials (in order, FP64) into stage[g][i], then the groups (in
// order) into gw [27][16][16] and gb [16].
constexpr int kRedGroup = 16;

__global__ void wgrad_reduce1_kernel(const float* __restrict__ partial, int n_parts,
                                     double* __restrict__ stage) {
  const int n = kTaps * kC * kC + kC;
  const int g = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int p0 = g * kRedGroup, p1 = min(n_parts, p0 + kRedGroup);
  float v[kRedGroup];
#pragma unroll
  for (int j = 0; j < kRedGroup; ++j)
    v[j] = p0 + j < p1 ? partial[(long long)(p0 + j) * n + i] : 0.0f;
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kRedGroup; ++j) s += v[j];
  stage[(long long)g * n + i] = s;
}

__global__ void wgrad_reduce2_kernel(const double* __restrict__ stage, int n_groups,
                                     float* __restrict__ gw, float* __restrict__ gb) {
  const int n = kTaps * kC * kC + kC;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int g = 0; g < n_groups; ++g) s += stage[(long long)g * n + i];
  if (i < kTaps * kC * kC) gw[i] = (float)s;
  else gb[i - kTaps * kC * kC] = (float)s;
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

// Fixed-order sum of n partials by one warp: lane l adds its contiguous
// chunk in order, then the lanes combine in a fixed butterfly.
__global__ void sum_kernel(const double* partial, int n, double* out) {
  const int l = threadIdx.x, chunk = (n + 31) / 32;
  double s = 0.0;
  for (int i = l * chunk; i < min(n, (l + 1) * chunk); ++i) s += partial[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (l == 0) *out = s;
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

int wgrad_blocks() { return 152 * 2; }
// per-CTA partials, then the FP64 group sums of the two-stage reduction
size_t wgrad_partial_floats() {
  const size_t n = kTaps * kC * kC + kC;
  return (size_t)wgrad_blocks() * n + 2 * (size_t)((wgrad_blocks() + kRedGroup - 1) / kRedGroup) * n;
}
int mse_blocks() { return 152 * 4; }

void conv_wgrad_halo_box(unsigned (&box)[4]) {
  box[0] = kC;
  box[1] = kHX;
  box[2] = kHY;
  box[3] = kFHZ;
}

void conv_gy_box(unsigned (&box)[4]) {
  box[0] = kC;
  box[1] = kTX;
  box[2] = kTY;
  box[3] = kFZ;
}

// Blocking of the tensor-core convolution for a D x H x W volume: the
// tallest row block (at most 8 chunks of 128 outputs) whose halo slots leave
// room for a ring of 4 (each halo plane is consumed by one step), else the
// tallest with 3.
constexpr int kTcSmemMax = 232448;                  // dynamic shared memory per CTA
constexpr int kTcSlotBudget = kTcSmemMax - kTcWBytes - 1024;

static TcPlan tc_plan(int D, int H, int W) {
  TcPlan p{};
  // x segments of at most kTcMaxP - 2 voxels, as even as possible: a halo
  // row of P voxels is one TMA box row of 4 P 8-byte elements (<= 256)
  p.nxs = (W + kTcMaxP - 3) / (kTcMaxP - 2);
  p.SW = (W + p.nxs - 1) / p.nxs;
  p.P = p.SW + 2;
  auto shape = [&](int ry) {
    p.RY = ry;
    p.NCH = (p.RY * p.P + 127) / 128;
    // the halo box must cover the last chunk's reach
    p.rows = (p.NCH * 128 + 2 * p.P + 2 + p.P - 1) / p.P;
    p.slot_bytes = ((p.rows * p.P * 32 + 1023) / 1024) * 1024;
    p.ring = std::min(kTcMaxRing, kTcSlotBudget / p.slot_bytes);
  };
  const int ry_max = std::max(1, std::min(H, (kTcMaxChunks * 128) / p.P));
  int pick = 0;
  for (int want = 4; want >= 3 && !pick; --want)
    for (int ry = ry_max; ry >= 1; --ry) {
      shape(ry);
      if (p.rows <= 256 && p.ring >= want) {
        pick = ry;
        break;
      }
    }
  shape(pick > 0 ? pick : 1);
  p.nyb = (H + p.RY - 1) / p.RY;
  // z chunk: fewest rounds of 152 persistent CTAs x planes per item; ties
  // go to longer chunks (fewer re-loaded halo planes).
  long long best = -1;
  for (int zc = 1; zc <= std::min(D, 32); ++zc) {
    const long long items = (long long)p.nxs * p.nyb * ((D + zc - 1) / zc);
    const long long cost = ((items + 151) / 152) * zc;
    if (best < 0 || cost <= best) {
      best = cost;
      p.ZC = zc;
    }
  }
  p.nzc = (D + p.ZC - 1) / p.ZC;
  p.items = (long long)p.nxs * p.nyb * p.nzc;
  return p;
}

static size_t tc_smem_bytes(const TcPlan& p) {
  return (size_t)p.ring * p.slot_bytes + (size_t)kTcWBytes + 1024;
}

void conv_halo_box(int D, int H, int W, unsigned (&box)[4]) {
  const TcPlan p = tc_plan(D, H, W);
  box[0] = 4u * (unsigned)p.P;  // one halo row: P voxels of 4 8-byte elements
  box[1] = (unsigned)p.rows;
  box[2] = 1;
  box[3] = 1;
}

cudaError_t launch_conv(const ConvArgs& a, const CUtensorMap& xmap, int* status, cudaStream_t s) {
  const TcPlan p = tc_plan(a.D, a.H, a.W);
  // At least 116 KB so that one CTA runs per SM and TMEM allocation never
  // waits for another CTA of this kernel.
  const size_t sm = std::max<size_t>(tc_smem_bytes(p), 116 * 1024);
  static size_t attr = 0;
  if (sm > attr) {
    cudaError_t e =
        cudaFuncSetAttribute(conv_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    attr = sm;
  }
  const int grid = (int)std::min<long long>(p.items, 152);
  conv_tc_kernel<<<grid, kTcThreads, sm, s>>>(xmap, a, p, status);
  return cudaGetLastError();
}

cudaError_t launch_wgrad(const WgradArgs& a, const CUtensorMap& xmap, const CUtensorMap& gmap,
                         int* status, float* gw, float* gb, cudaStream_t s) {
  const long long n_tiles = (long long)((a.W + kTX - 1) / kTX) * ((a.H + kTY - 1) / kTY) *
                            ((a.D + kFZ - 1) / kFZ);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(conv_wgrad_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         2 * kWStage + 256);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int grid = (int)std::min<long long>(n_tiles, wgrad_blocks());
  conv_wgrad_kernel<<<grid, 256, 2 * kWStage + 256, s>>>(xmap, gmap, a, status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int n = kTaps * kC * kC + kC, groups = (grid + kRedGroup - 1) / kRedGroup;
  double* stage = reinterpret_cast<double*>(a.partial + (size_t)wgrad_blocks() * n);
  wgrad_reduce1_kernel<<<dim3((n + 127) / 128, groups), 128, 0, s>>>(a.partial, grid, stage);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  wgrad_reduce2_kernel<<<(n + 127) / 128, 128, 0, s>>>(stage, groups, gw, gb);
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
