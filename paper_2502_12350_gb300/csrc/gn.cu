// Gauss-Newton diagonal labels: discrete Fourier accumulation of the
// source-side imaging term and of the receiver-side impulse responses, and
// the Parseval assembly
//   H(x) = (2 c dt^2)^2 / N_f sum_k w_k (sum_r |G^_r(x,k)|^2)(sum_s |a^_s(x,k)|^2)
// over the retained frequency bins k of an N_f = 2 nt zero-padded DFT.
#include "gn.h"

#include <cstdint>

namespace mamute {

namespace {

constexpr int kPts = 128;   // points per CTA
constexpr int kPP = 4;      // consecutive points per thread
constexpr int kChunk = 16;  // frequency bins per thread
constexpr int kGroups = kPts / kPP;  // point groups: one warp

// Twiddles W[t][k] = exp(-2 pi i bins[k] (n0 + t) / nf) for one time block.
__global__ void twiddle_kernel(int T, int n0, int nf, const int* __restrict__ bins, int nb,
                               float2* __restrict__ W) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= T * nb) return;
  const int t = i / nb, k = i % nb;
  const long long m = ((long long)bins[k] * (long long)(n0 + t)) % nf;
  float sn, cs;
  sincospif(2.0f * (float)m / (float)nf, &sn, &cs);
  W[i] = make_float2(cs, -sn);
}

// acc[k][x] += sum_t V[t][x] W[t][k] for kPts points per CTA.  Warp c owns
// bins [c kChunk, (c+1) kChunk); lane g owns points 4g..4g+3 of the CTA, so
// per time sample a thread does 4 x 16 complex MACs from one 16-byte read of
// V and eight broadcast 16-byte reads of W (FP32 FMA bound, not LSU bound).
// VEC: N is a multiple of 4, so the accumulator rows take 16-byte accesses.
template <bool VEC>
__global__ void __launch_bounds__(256, 1)
    dft_kernel(const float* __restrict__ V, long long N, int T, int nb,
               const float2* __restrict__ W, float* __restrict__ re, float* __restrict__ im) {
  extern __shared__ float4 sm4[];
  float* Vs = reinterpret_cast<float*>(sm4);                // [T][kPts]
  const int nbp = (blockDim.x / 32) * kChunk;             // bins padded to the warps
  float2* Ws = reinterpret_cast<float2*>(Vs + T * kPts);  // [T][nbp], zero beyond nb
  const long long x0 = (long long)blockIdx.x * kPts;
  for (int i = threadIdx.x; i < T * nbp; i += blockDim.x) {
    const int t = i / nbp, k = i % nbp;
    Ws[i] = k < nb ? W[t * nb + k] : make_float2(0.0f, 0.0f);
  }
  for (int i = threadIdx.x; i < T * kPts; i += blockDim.x) {
    const int t = i / kPts, p = i % kPts;
    const long long x = x0 + p;
    Vs[i] = x < N ? V[(long long)t * N + x] : 0.0f;
  }
  __syncthreads();
  const int g = threadIdx.x & 31, c = threadIdx.x >> 5;
  const long long xb = x0 + kPP * g;
  if (xb >= N) return;
  float ar[kPP][kChunk], ai[kPP][kChunk];
#pragma unroll
  for (int j = 0; j < kChunk; ++j) {
    const int k = c * kChunk + j;
    if (VEC && k < nb) {  // xb + 3 < N as N is a multiple of 4
      const float4 r = *reinterpret_cast<const float4*>(re + (long long)k * N + xb);
      const float4 m = *reinterpret_cast<const float4*>(im + (long long)k * N + xb);
      ar[0][j] = r.x; ar[1][j] = r.y; ar[2][j] = r.z; ar[3][j] = r.w;
      ai[0][j] = m.x; ai[1][j] = m.y; ai[2][j] = m.z; ai[3][j] = m.w;
    } else {
#pragma unroll
      for (int q = 0; q < kPP; ++q) {
        const bool ok = k < nb && xb + q < N;
        ar[q][j] = ok ? re[(long long)k * N + xb + q] : 0.0f;
        ai[q][j] = ok ? im[(long long)k * N + xb + q] : 0.0f;
      }
    }
  }
#pragma unroll 2
  for (int t = 0; t < T; ++t) {
    const float4 v = *reinterpret_cast<const float4*>(Vs + t * kPts + kPP * g);
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
#pragma unroll
  for (int j = 0; j < kChunk; ++j) {
    const int k = c * kChunk + j;
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

size_t dft_smem_bytes(int T, int nb) {
  const int nbp = ((nb + kChunk - 1) / kChunk) * kChunk;
  return sizeof(float) * T * kPts + sizeof(float2) * T * nbp;
}

int dft_max_bins() { return (256 / 32) * kChunk; }

cudaError_t launch_dft(const float* V, long long N, int T, int n0, int nf, const int* bins, int nb,
                       float2* W, float* re, float* im, cudaStream_t s) {
  if (T <= 0) return cudaSuccess;
  if (nb < 1 || nb > dft_max_bins()) return cudaErrorInvalidValue;
  twiddle_kernel<<<(T * nb + 255) / 256, 256, 0, s>>>(T, n0, nf, bins, nb, W);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t sm = dft_smem_bytes(T, nb);
  const bool vec = (N % 4) == 0 && ((uintptr_t)re % 16) == 0 && ((uintptr_t)im % 16) == 0;
  static size_t attr[2] = {0, 0};
  if (sm > attr[vec]) {
    e = vec ? cudaFuncSetAttribute(dft_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)
            : cudaFuncSetAttribute(dft_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    attr[vec] = sm;
  }
  const int warps = (nb + kChunk - 1) / kChunk;
  const unsigned grid = (unsigned)((N + kPts - 1) / kPts);
  if (vec)
    dft_kernel<true><<<grid, 32 * warps, sm, s>>>(V, N, T, nb, W, re, im);
  else
    dft_kernel<false><<<grid, 32 * warps, sm, s>>>(V, N, T, nb, W, re, im);
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
