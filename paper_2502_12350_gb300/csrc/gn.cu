// Gauss-Newton diagonal labels: discrete Fourier accumulation of the
// source-side imaging term and of the receiver-side impulse responses, and
// the Parseval assembly
//   H(x) = (2 c dt^2)^2 / N_f sum_k w_k (sum_r |G^_r(x,k)|^2)(sum_s |a^_s(x,k)|^2)
// over the retained frequency bins k of an N_f = 2 nt zero-padded DFT.
#include "gn.h"

#include <algorithm>
#include <cstdint>

#include "common.cuh"

namespace mamute {

namespace {

constexpr int kPts = 128;     // points per block
constexpr int kPP = 4;        // consecutive points per thread
constexpr int kChunk = 8;     // frequency bins per warp
constexpr int kMaxWarps = 16;

// Twiddles exp(-2 pi i bins[k] (n0 + t) / nf) for one time block, laid out
// [group][t][k'] with k = group * nbh + k' (zeros beyond nb).
__global__ void twiddle_kernel(int T, int n0, int nf, const int* __restrict__ bins, int nb,
                               int groups, int nbh, float2* __restrict__ W) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= groups * T * nbh) return;
  const int grp = i / (T * nbh), t = (i / nbh) % T, k = grp * nbh + i % nbh;
  if (k >= nb) {
    W[i] = make_float2(0.0f, 0.0f);
    return;
  }
  const long long m = ((long long)bins[k] * (long long)(n0 + t)) % nf;
  float sn, cs;
  sincospif(2.0f * (float)m / (float)nf, &sn, &cs);
  W[i] = make_float2(cs, -sn);
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// acc[k][x] += sum_t V[t][x] W[t][k], persistent over blocks of kPts points;
// blockIdx.y selects a group of bins (the bins are split over 1 or 2 CTAs
// per block of points so that two CTAs fit on an SM and one computes while
// the other loads or stores its accumulators).
// The T x nbh twiddles of the group are loaded once per CTA; the T x kPts samples of the
// next block arrive by bulk copies (one per sample row) into the other half
// of a double buffer while this block is accumulated.  Warp c owns bins
// [c kChunk, (c+1) kChunk) and lane g points 4g..4g+3, so per sample a
// thread does 4 x 8 complex MACs from one 16-byte read of V and four
// broadcast 16-byte reads of W.  VEC (N a multiple of 4): bulk copies and
// 16-byte accumulator accesses; otherwise plain loads.
template <bool VEC>
__global__ void __launch_bounds__(kMaxWarps * 32, 1)
    dft_kernel(const float* __restrict__ V, long long N, int T, int nb,
               const float2* __restrict__ W, float* __restrict__ re, float* __restrict__ im,
               int* status) {
  extern __shared__ float4 sm4[];
  __shared__ uint64_t bar[3];  // [0] twiddles, [1 + b] samples of buffer b
  __shared__ int abort_flag;
  const int nbp = (blockDim.x / 32) * kChunk;     // bins of this CTA's group
  const int kbase = blockIdx.y * nbp;
  W += (size_t)blockIdx.y * T * nbp;
  float2* Ws = reinterpret_cast<float2*>(sm4);   // [T][nbp]
  float* Vs = reinterpret_cast<float*>(Ws + T * nbp);  // [2][T][kPts]
  const long long nblk = (N + kPts - 1) / kPts;
  auto issue = [&](int b, long long blk) {
    const long long x0 = blk * kPts;
    const uint32_t bytes = (uint32_t)(min((long long)kPts, N - x0) * 4);
    mbar_arrive_expect_tx(&bar[1 + b], (uint32_t)T * bytes);
    for (int t = 0; t < T; ++t)
      bulk_load(Vs + ((size_t)b * T + t) * kPts, V + (long long)t * N + x0, bytes, &bar[1 + b]);
  };
  if (threadIdx.x == 0) {
    for (int i = 0; i < 3; ++i) mbar_init(&bar[i], 1);
    fence_barrier_init();
    abort_flag = 0;
  }
  __syncthreads();
  bool issued_next = false;  // thread 0: a sample copy into the other buffer is in flight
  if (VEC) {
    if (threadIdx.x == 0) {
      mbar_arrive_expect_tx(&bar[0], (uint32_t)(T * nbp * 8));
      bulk_load(Ws, W, (uint32_t)(T * nbp * 8), &bar[0]);
      issue(0, blockIdx.x);
    }
    if (!mbar_wait(&bar[0], 0, status)) abort_flag = 1;
  } else {
    for (int i = threadIdx.x; i < T * nbp; i += blockDim.x) Ws[i] = W[i];
  }
  const int g = threadIdx.x & 31, c = threadIdx.x >> 5;
  int it = 0;
  for (long long blk = blockIdx.x; blk < nblk; blk += gridDim.x, ++it) {
    const int b = it & 1;
    float* Vb = Vs + (size_t)b * T * kPts;
    const long long x0 = blk * kPts;
    if (VEC) {
      issued_next = threadIdx.x == 0 && blk + gridDim.x < nblk;
      if (issued_next) issue(b ^ 1, blk + gridDim.x);
    } else {
      for (int i = threadIdx.x; i < T * kPts; i += blockDim.x) {
        const int t = i / kPts, p = i % kPts;
        Vb[i] = x0 + p < N ? V[(long long)t * N + x0 + p] : 0.0f;
      }
    }
    const long long xb = x0 + kPP * g;
    const bool live = xb < N;
    float ar[kPP][kChunk], ai[kPP][kChunk];
#pragma unroll
    for (int j = 0; j < kChunk; ++j) {
      const int k = kbase + c * kChunk + j;
      if (VEC) {
        float4 rv = make_float4(0.f, 0.f, 0.f, 0.f), mv = rv;
        if (live && k < nb) {  // xb + 3 < N as N is a multiple of 4
          rv = *reinterpret_cast<const float4*>(re + (long long)k * N + xb);
          mv = *reinterpret_cast<const float4*>(im + (long long)k * N + xb);
        }
        ar[0][j] = rv.x; ar[1][j] = rv.y; ar[2][j] = rv.z; ar[3][j] = rv.w;
        ai[0][j] = mv.x; ai[1][j] = mv.y; ai[2][j] = mv.z; ai[3][j] = mv.w;
      } else {
#pragma unroll
        for (int q = 0; q < kPP; ++q) {
          const bool ok = k < nb && xb + q < N;
          ar[q][j] = ok ? re[(long long)k * N + xb + q] : 0.0f;
          ai[q][j] = ok ? im[(long long)k * N + xb + q] : 0.0f;
        }
      }
    }
    if (VEC && !mbar_wait(&bar[1 + b], (uint32_t)((it >> 1) & 1), status)) abort_flag = 1;
    __syncthreads();
    if (abort_flag) {
      if (issued_next) mbar_wait(&bar[1 + (b ^ 1)], (uint32_t)(((it + 1) >> 1) & 1), status);
      return;
    }
#pragma unroll 2
    for (int t = 0; t < T; ++t) {
      const float4 v = *reinterpret_cast<const float4*>(Vb + t * kPts + kPP * g);
      const float vq[kPP] = {v.x, v.y, v.z, v.w};
      const float4* w4 = reinterpret_cast<const float4*>(Ws + t * nbp + c * kChunk);
#pragma unroll
      for (int jj = 0; jj < kChunk / 2; ++jj) {
        const float4 w = w4[jj];  // bins 2jj and 2jj + 1
#pragma unroll
        for (int q = 0; q < kPP; ++q) {
          ar[q][2 * jj] = fmaf(vq[q], w.x, ar[q][2 * jj]);
          ai[q][2 * jj] = fmaf(vq[q], w.y, ai[q][2 * jj]);
          ar[q][2 * jj + 1] = fmaf(vq[q], w.z, ar[q][2 * jj + 1]);
          ai[q][2 * jj + 1] = fmaf(vq[q], w.w, ai[q][2 * jj + 1]);
        }
      }
    }
    if (live) {
#pragma unroll
      for (int j = 0; j < kChunk; ++j) {
        const int k = kbase + c * kChunk + j;
        if (k >= nb) continue;
        if (VEC) {
          *reinterpret_cast<float4*>(re + (long long)k * N + xb) =
              make_float4(ar[0][j], ar[1][j], ar[2][j], ar[3][j]);
          *reinterpret_cast<float4*>(im + (long long)k * N + xb) =
              make_float4(ai[0][j], ai[1][j], ai[2][j], ai[3][j]);
        } else {
#pragma unroll
          for (int q = 0; q < kPP; ++q) {
            if (xb + q < N) {
              re[(long long)k * N + xb + q] = ar[q][j];
              im[(long long)k * N + xb + q] = ai[q][j];
            }
          }
        }
      }
    }
    __syncthreads();  // buffer b is free for the copy issued next iteration
  }
}

// pw[k][x] += sum_v re[k][v N + x]^2 + im[k][v N + x]^2 over the nv windows
// of a batch (accumulators laid out [k][nv N]); then re = im = 0.
__global__ void power_kernel(int nb, long long N, int nv, float* __restrict__ re,
                             float* __restrict__ im, float* __restrict__ pw) {
  const long long n = (long long)nb * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long k = i / N, x = i % N;
    float acc = pw[i];
    for (int v = 0; v < nv; ++v) {
      const long long j = k * nv * N + v * N + x;
      const float a = re[j], b = im[j];
      acc = fmaf(a, a, fmaf(b, b, acc));
      re[j] = 0.0f;
      im[j] = 0.0f;
    }
    pw[i] = acc;
  }
}

// H[x] = 4 / (c^6 dt^4 nf) sum_k w_k R[k][x] S[k][x]  (FP64 sum).  The
// stored source-side term is A (lap - m2) u and the stored receiver-side
// term psi = A g lambda, so |a^|^2 |G^|^2 = |S^|^2 |R^|^2 / A^4 with
// A = c^2 dt^2, and (2 c dt^2)^2 / A^4 = 4 / (c^6 dt^4).
__global__ void assemble_kernel(long long N, int nb, const float* __restrict__ w,
                                const float* __restrict__ R, const float* __restrict__ S,
                                const float* __restrict__ vel, double dt, int nf,
                                float* __restrict__ H) {
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < N;
       x += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int k = 0; k < nb; ++k)
      acc += (double)w[k] * (double)R[(long long)k * N + x] * (double)S[(long long)k * N + x];
    const double c = vel[x];
    const double c2 = c * c;
    H[x] = (float)(4.0 * acc / (c2 * c2 * c2 * dt * dt * dt * dt * (double)nf));
  }
}

int blocks_for(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b > 152 * 32 ? 152 * 32 : (b < 1 ? 1 : b));
}

}  // namespace

int dft_padded_bins(int nb) { return ((nb + kChunk - 1) / kChunk) * kChunk; }

// Bins split over groups of CTAs: 2 groups above 64 bins, so that a CTA
// needs at most 8 warps and two CTAs fit on an SM.
static void dft_groups(int nb, int& groups, int& nbh) {
  const int nbp = dft_padded_bins(nb);
  groups = nbp > 64 ? 2 : 1;
  nbh = dft_padded_bins((nbp + groups - 1) / groups);
}

size_t dft_smem_bytes(int T, int nb) {
  int groups, nbh;
  dft_groups(nb, groups, nbh);
  return sizeof(float2) * T * nbh + sizeof(float) * 2 * T * kPts;
}

int dft_max_bins() { return kMaxWarps * kChunk; }

cudaError_t launch_dft(const float* V, long long N, int T, int n0, int nf, const int* bins, int nb,
                       float2* W, float* re, float* im, int* status, cudaStream_t s) {
  if (T <= 0 || N <= 0) return cudaSuccess;
  if (nb < 1 || nb > dft_max_bins()) return cudaErrorInvalidValue;
  int groups, nbh;
  dft_groups(nb, groups, nbh);  // groups * nbh <= dft_max_bins()
  twiddle_kernel<<<(groups * T * nbh + 255) / 256, 256, 0, s>>>(T, n0, nf, bins, nb, groups, nbh,
                                                                W);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t sm = dft_smem_bytes(T, nb);
  const bool vec = (N % 4) == 0 && ((uintptr_t)V % 16) == 0 && ((uintptr_t)W % 16) == 0 &&
                   ((uintptr_t)re % 16) == 0 && ((uintptr_t)im % 16) == 0;
  static size_t attr[2] = {0, 0};
  if (sm > attr[vec]) {
    e = vec ? cudaFuncSetAttribute(dft_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)
            : cudaFuncSetAttribute(dft_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    attr[vec] = sm;
  }
  const int threads = 32 * (nbh / kChunk);
  int per_sm = 1;
  e = vec ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dft_kernel<true>, threads, sm)
          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dft_kernel<false>, threads, sm);
  if (e != cudaSuccess) return e;
  const long long nblk = (N + kPts - 1) / kPts;
  const dim3 grid(
      (unsigned)std::min<long long>(nblk, std::max(1LL, 152LL * std::max(per_sm, 1) / groups)),
      (unsigned)groups);
  if (vec)
    dft_kernel<true><<<grid, threads, sm, s>>>(V, N, T, nb, W, re, im, status);
  else
    dft_kernel<false><<<grid, threads, sm, s>>>(V, N, T, nb, W, re, im, status);
  return cudaGetLastError();
}

cudaError_t launch_power(int nb, long long N, int nv, float* re, float* im, float* pw,
                         cudaStream_t s) {
  power_kernel<<<blocks_for((long long)nb * N), 256, 0, s>>>(nb, N, nv, re, im, pw);
  return cudaGetLastError();
}

cudaError_t launch_assemble(long long N, int nb, const float* w, const float* R, const float* S,
                            const float* vel, double dt, int nf, float* H, cudaStream_t s) {
  assemble_kernel<<<blocks_for(N), 256, 0, s>>>(N, nb, w, R, S, vel, dt, nf, H);
  return cudaGetLastError();
}

}  // namespace mamute
