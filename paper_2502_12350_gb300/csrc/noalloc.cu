// Misfit reduction that allocates nothing.
//
// Some callers cannot allocate device memory: a host framework whose caching
// allocator already holds the device's memory, or a latency-sensitive loop
// that must not pay for cudaMalloc's implicit device-wide synchronisation.
// For them this file provides one extra entry point, a variant of the
// context-based misfit reduction (which keeps its per-block partial sums in
// context scratch), whose partial sums live in a fixed file-scope device
// array instead.  The caller passes only its inputs and a host output.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/mamute.h"

namespace {

constexpr int kThreads = 256;
constexpr long long kChunk = 16384;          // samples reduced by one block
constexpr int kMaxPartials = 16384;          // blocks per call (128 KiB of partials)
constexpr long long kMaxSamples = kChunk * kMaxPartials;
static_assert(kMaxSamples == MAMUTE_MISFIT_NOALLOC_MAX_SAMPLES, "header limit out of date");
constexpr int kMaxDevices = 64;

// Scratch shared by every call on a device: slot [0, nb) holds the partial
// sums of the current call, slot kMaxPartials the total.  Each slot that is
// read is first written in the same call, so nothing needs clearing.
static __device__ __align__(256) double g_scratch[kMaxPartials + 1];

std::mutex g_mu;
double* g_addr[kMaxDevices] = {nullptr};

__global__ void partial_kernel(const float* __restrict__ d, const float* __restrict__ dobs,
                               long long n, double* __restrict__ scratch) {
  __shared__ double red[kThreads];
  const long long base = (long long)blockIdx.x * kChunk;
  const long long end = base + kChunk < n ? base + kChunk : n;
  double acc = 0.0;
  for (long long i = base + threadIdx.x; i < end; i += kThreads) {
    const float r = d[i] - dobs[i];
    acc += 0.5 * (double)r * (double)r;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) scratch[blockIdx.x] = red[0];
}

// One warp: lane l adds the partials of its contiguous chunk in order, then
// the lanes combine in a fixed butterfly, so the total does not depend on
// timing and the partials are read in parallel.
__global__ void total_kernel(int nb, double* __restrict__ scratch) {
  if (blockIdx.x != 0) return;
  const int lane = threadIdx.x & 31;
  const int per = (nb + 31) / 32;
  const int b = lane * per, e = b + per < nb ? b + per : nb;
  double s = 0.0;
  for (int k = b; k < e; ++k) s += scratch[k];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) scratch[kMaxPartials] = s;
}

}  // namespace

// Device address of the scratch array on the current device.  The host-side
// name g_scratch is only a stand-in, so the address is looked up once per
// device, with that device current, on the first call that runs there.
static int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MAMUTE_ECUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return MAMUTE_ECUDA;
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return MAMUTE_OK;
}

extern "C" int mamute_misfit_noalloc(const float* d, const float* d_obs, long long n,
                                     void* cuda_stream, double* misfit) {
  if (!misfit || n < 0 || (n > 0 && (!d || !d_obs))) return MAMUTE_EINVAL;
  if (n > kMaxSamples) return MAMUTE_EINVAL;  // beyond the fixed scratch array
  if (n == 0) {
    *misfit = 0.0;
    return MAMUTE_OK;
  }
  double* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc != MAMUTE_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int nb = (int)((n + kChunk - 1) / kChunk);
  partial_kernel<<<nb, kThreads, 0, s>>>(d, d_obs, n, scratch);
  total_kernel<<<1, 32, 0, s>>>(nb, scratch);
  cudaError_t e = cudaGetLastError();
  double J = 0.0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&J, scratch + kMaxPartials, sizeof J, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return MAMUTE_ECUDA;
  *misfit = J;
  return MAMUTE_OK;
}
