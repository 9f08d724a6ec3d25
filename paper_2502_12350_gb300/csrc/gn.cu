// Gauss-Newton diagonal labels: discrete Fourier accumulation of the
// source-side imaging term and of the receiver-side impulse responses, and
// the Parseval assembly
//   H(x) = (2 c dt^2)^2 / N_f sum_k w_k (sum_r |G^_r(x,k)|^2)(sum_s |a^_s(x,k)|^2)
// over the retained frequency bins k of an N_f = 2 nt zero-padded DFT.
#include "gn.h"

namespace mamute {

namespace {

constexpr int kPts = 64;    // points per CTA
constexpr int kChunk = 16;  // frequency bins per thread

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

// acc[k][x] += sum_t V[t][x] W[t][k] for kPts points per CTA; thread
// (p, c) owns point p and bins [c kChunk, (c+1) kChunk).
__global__ void __launch_bounds__(512) dft_kernel(const float* __restrict__ V, long long N, int T, int nb,
                           const float2* __restrict__ W, float* __restrict__ re,
                           float* __restrict__ im) {
  extern __shared__ float sm[];
  float* Vs = sm;                                        // [T][kPts]
  float2* Ws = reinterpret_cast<float2*>(sm + T * kPts);  // [T][nb]
  const long long x0 = (long long)blockIdx.x * kPts;
  for (int i = threadIdx.x; i < T * nb; i += blockDim.x) Ws[i] = W[i];
  for (int i = threadIdx.x; i < T * kPts; i += blockDim.x) {
    const int t = i / kPts, p = i % kPts;
    const long long x = x0 + p;
    Vs[i] = x < N ? V[(long long)t * N + x] : 0.0f;
  }
  __syncthreads();
  const int p = threadIdx.x % kPts, c = threadIdx.x / kPts;
  const long long x = x0 + p;
  if (x >= N) return;
  float ar[kChunk], ai[kChunk];
#pragma unroll
  for (int j = 0; j < kChunk; ++j) {
    const int k = c * kChunk + j;
    ar[j] = k < nb ? re[(long long)k * N + x] : 0.0f;
    ai[j] = k < nb ? im[(long long)k * N + x] : 0.0f;
  }
  for (int t = 0; t < T; ++t) {
    const float v = Vs[t * kPts + p];
    const float2* wr = Ws + t * nb + c * kChunk;
#pragma unroll
    for (int j = 0; j < kChunk; ++j) {
      if (c * kChunk + j < nb) {
        const float2 w = wr[j];
        ar[j] = fmaf(v, w.x, ar[j]);
        ai[j] = fmaf(v, w.y, ai[j]);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < kChunk; ++j) {
    const int k = c * kChunk + j;
    if (k < nb) {
      re[(long long)k * N + x] = ar[j];
      im[(long long)k * N + x] = ai[j];
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

size_t dft_smem_bytes(int T, int nb) { return sizeof(float) * T * kPts + sizeof(float2) * T * nb; }

int dft_max_bins() { return (512 / kPts) * kChunk; }

cudaError_t launch_dft(const float* V, long long N, int T, int n0, int nf, const int* bins, int nb,
                       float2* W, float* re, float* im, cudaStream_t s) {
  if (T <= 0) return cudaSuccess;
  twiddle_kernel<<<(T * nb + 255) / 256, 256, 0, s>>>(T, n0, nf, bins, nb, W);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t sm = dft_smem_bytes(T, nb);
  static size_t attr = 0;
  if (sm > attr) {
    e = cudaFuncSetAttribute(dft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    attr = sm;
  }
  const int chunks = (nb + kChunk - 1) / kChunk;
  dft_kernel<<<(int)((N + kPts - 1) / kPts), kPts * chunks, sm, s>>>(V, N, T, nb, W, re, im);
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
