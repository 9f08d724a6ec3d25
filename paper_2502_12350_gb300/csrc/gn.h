// Launch interface of the Gauss-Newton diagonal kernels (internal).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

namespace mamute {

size_t dft_smem_bytes(int T, int nb);
int dft_max_bins();
// acc (re, im)[nb][N] += sum_{t<T} V[t][N] exp(-2 pi i bins[k] (n0 + t) / nf); W is
// scratch for T * dft_max_bins() twiddles; status collects bounded-wait timeouts.
cudaError_t launch_dft(const float* V, long long N, int T, int n0, int nf, const int* bins, int nb,
                       float2* W, float* re, float* im, int* status, cudaStream_t s);
// The same accumulation on the tensor cores (kind::tf32, hi / lo split, one
// accumulator pass per call).  vmap: V viewed as 3-D {N, T, 1} FP32, box
// {128, dft_tc_chunk(), 1}, no swizzle; W: dft_tc_image_bytes(T, nb) bytes of scratch
// (16-byte aligned); needs dft_tc_supported(N, nb) (N a multiple of 4, at
// most 128 bins) and 16-byte aligned re / im.  overwrite: re / im hold zeros
// (the first block of a batch), so the sums are stored without reading them.
int dft_tc_chunk();
size_t dft_tc_image_bytes(int T, int nb);
bool dft_tc_supported(long long N, int nb);
cudaError_t launch_dft_tc(const CUtensorMap& vmap, long long N, int T, int n0, int nf,
                          const int* bins, int nb, float* W, float* re, float* im, bool overwrite,
                          int* status, cudaStream_t s);
// pw[k][x] += sum over the nv windows of |acc[k][v N + x]|^2, then acc = 0.
cudaError_t launch_power(int nb, long long N, int nv, float* re, float* im, float* pw,
                         cudaStream_t s);
// H[x] = 4 / (c^6 dt^4 nf) sum_k w[k] R[k][x] S[k][x].
cudaError_t launch_assemble(long long N, int nb, const float* w, const float* R, const float* S,
                            const float* vel, double dt, int nf, float* H, cudaStream_t s);

}  // namespace mamute
