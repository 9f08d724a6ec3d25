// Gauss-Newton diagonal labels: discrete Fourier accumulation of the
// source-side imaging term and of the receiver-side impulse responses, and
// the Parseval assembly
//   H(x) = (2 c dt^2)^2 / N_f sum_k w_k (sum_r |G^_r(x,k)|^2)(sum_s |a^_s(x,k)|^2)
// over the retained frequency bins k of an N_f = 2 nt zero-padded DFT.
#include "gn.h"

#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "tcgen05.cuh"

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

// ---- Tensor-core form of the same accumulation (kind::tf32, 3 products).
//
// The block sum acc[k][x] += sum_t V[t][x] W[t][k] is a product of a
// (2 nb) x T twiddle matrix (rows: cos of bins 64 j .. 64 j + 63, then -sin
// of the same bins, per M tile j) with the T x N sample matrix.  Each
// operand x is split into tf32 parts hi = rna(x), lo = rna(x - hi) and the
// product is taken as A_hi B_hi + A_hi B_lo + A_lo B_hi (the dropped term is
// below FP32 rounding), with FP32 accumulation in tensor memory over all T
// samples of the block: the accumulators are read and written once per
// block instead of once per 64 samples.
//
// Operands in shared memory use the K-major canonical layout without
// swizzle: core matrices of 8 rows x 16 bytes (4 tf32), the 4 K-cores of a
// 16-sample chunk 128 bytes apart (LBO), 8-row groups 512 bytes apart
// (SBO).  A CTA takes tiles of 128 points; per 16-sample chunk the producer
// brings the 16 x 128 samples by TMA and the chunk's twiddle images (built
// in that layout by dft_image_kernel) by one bulk copy into a 4-stage ring,
// four warps split the samples into hi / lo rows, and one thread issues
// mt x 2 x 3 products M=128 N=128 K=8 into a double-buffered accumulator;
// four epilogue warps add (or, for the first block of a batch, store) the
// tile's accumulators to acc.

constexpr int kTcNP = 128;                    // points per tile (MMA N)
constexpr int kTcKC = 16;                     // samples per chunk
constexpr int kTcStages = 4;                  // ring of sample / twiddle stages
constexpr int kTcGroup = (kTcKC / 4) * 128;   // bytes per 8-row group (SBO)
constexpr int kTcImg = 128 * kTcKC * 4;       // bytes of one 128-row chunk image
constexpr int kTcMaxMt = 2;                   // M tiles: up to 128 bins
constexpr int kTcVBytes = kTcKC * kTcNP * 4;  // samples of one chunk
constexpr int kTcABytes = kTcMaxMt * 2 * kTcImg;
constexpr int kTcSBytes = 2 * kTcImg;         // hi and lo sample rows
constexpr int kTcSmem = kTcStages * (kTcVBytes + kTcABytes) + 2 * kTcSBytes + 1024;
constexpr int kTcDftThreads = 320;

// D f32 (bits 4-5 = 1), A and B tf32 (bits 7-9, 10-12 = 2), both K-major,
// N = 128 (bits 17-22: N >> 3), M = 128 (bits 24-28: M >> 4).
constexpr uint32_t kDftIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((128u >> 3) << 17) |
                               ((128u >> 4) << 24);

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Byte offset of element (row, k) in a canonical K-major image of 8-row
// groups with kTcKC / 4 K-cores each.
__device__ __forceinline__ int img_off(int row, int k) {
  return (row >> 3) * kTcGroup + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4;
}

// Twiddle images: for chunk c, M tile j and part p (0 hi, 1 lo) a 128 x 32
// image at W + ((c * mt + j) * 2 + p) * kTcImg bytes.
__global__ void dft_image_kernel(int T, int n0, int nf, const int* __restrict__ bins, int nb,
                                 int mt, int nchunks, float* __restrict__ W) {
  const int n = nchunks * mt * 128 * kTcKC;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int k = e % kTcKC, row = (e / kTcKC) % 128, j = (e / (kTcKC * 128)) % mt;
    const int c = e / (kTcKC * 128 * mt);
    const int t = c * kTcKC + k, bin = 64 * j + (row & 63);
    float v = 0.0f;
    if (t < T && bin < nb) {
      const long long m = ((long long)bins[bin] * (long long)(n0 + t)) % nf;
      float sn, cs;
      sincospif(2.0f * (float)m / (float)nf, &sn, &cs);
      v = row < 64 ? cs : -sn;
    }
    const float hi = tf32_rna(v), lo = tf32_rna(v - hi);
    char* base = reinterpret_cast<char*>(W) + (size_t)((c * mt + j) * 2) * kTcImg;
    *reinterpret_cast<float*>(base + img_off(row, k)) = hi;
    *reinterpret_cast<float*>(base + kTcImg + img_off(row, k)) = lo;
  }
}

struct DftTcArgs {
  const float* W;   // twiddle images
  float* re;
  float* im;
  long long N;
  int nb, mt, nchunks;
  int overwrite;    // the accumulators are zero: store instead of add
  int* status;
};

__global__ void __launch_bounds__(kTcDftThreads, 1)
    dft_tc_kernel(const __grid_constant__ CUtensorMap vmap, DftTcArgs a) {
  extern __shared__ unsigned char dft_raw[];
  unsigned char* sm = dft_raw + ((1024 - (smem_u32(dft_raw) & 1023)) & 1023);
  unsigned char* vraw = sm;                                   // stages of samples
  unsigned char* aimg = sm + kTcStages * kTcVBytes;           // stages of twiddle images
  unsigned char* bspl = aimg + kTcStages * kTcABytes;         // 2 buffers of hi / lo rows
  __shared__ uint64_t full[kTcStages], empty[kTcStages], sready[2], sfree[2], tfull[2], tempty[2],
      done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  volatile int* ab = &abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long ntiles = (a.N + kTcNP - 1) / kTcNP;
  const int nch = a.nchunks, mt = a.mt;
  const uint32_t abytes = (uint32_t)(mt * 2 * kTcImg);
  if (threadIdx.x == 0) {
    for (int i = 0; i < kTcStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 5);   // 4 split warps + the MMA commit
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&sready[i], 4);
      mbar_init(&sfree[i], 1);
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 4);
    }
    mbar_init(&done_bar, 1);
    fence_barrier_init();
    abort_flag = 0;
  }
  if (warp == 1) {
    tc_alloc(&tmem_base, 512);
    tc_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    // ---- producer: per chunk, the samples (TMA) and the twiddle images
    if (lane == 0) {
      tmap_acquire(&vmap);
      uint32_t q = 0;
      for (long long tile = blockIdx.x; tile < ntiles && !*ab; tile += gridDim.x)
        for (int c = 0; c < nch; ++c, ++q) {
          const int s = (int)(q % kTcStages), r = (int)(q / kTcStages);
          if (r > 0 && !tc_wait(&empty[s], (r & 1) ^ 1, a.status, ab)) break;
          mbar_arrive_expect_tx(&full[s], (uint32_t)kTcVBytes + abytes);
          tma_load_3d(vraw + s * kTcVBytes, &vmap, (int)(tile * kTcNP), c * kTcKC, 0, &full[s]);
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
                  "r"(smem_u32(aimg + s * kTcABytes)),
              "l"(reinterpret_cast<const char*>(a.W) + (size_t)c * abytes), "r"(abytes),
              "r"(smem_u32(&full[s]))
              : "memory");
        }
      if (*ab)  // let issued loads land before the CTA exits
        for (uint32_t k = 0; k < (uint32_t)kTcStages && k < q; ++k) {
          const uint32_t qq = q - 1 - k;
          mbar_wait(&full[qq % kTcStages], (qq / kTcStages) & 1, a.status);
        }
    }
  } else if (warp == 1) {
    // ---- MMA issuer
    if (lane == 0) {
      const uint32_t abase = smem_u32(aimg), bbase = smem_u32(bspl);
      uint32_t q = 0, p = 0;
      bool ok = true;
      for (long long tile = blockIdx.x; tile < ntiles && ok && !*ab; tile += gridDim.x, ++p) {
        const uint32_t tb = p & 1;
        if (p >= 2 && !(ok = tc_wait(&tempty[tb], ((p >> 1) & 1) ^ 1, a.status, ab))) break;
        for (int c = 0; c < nch && ok; ++c, ++q) {
          const uint32_t s = q % kTcStages, b = q & 1;
          if (!(ok = tc_wait(&full[s], (q / kTcStages) & 1, a.status, ab))) break;
          if (!(ok = tc_wait(&sready[b], (q >> 1) & 1, a.status, ab))) break;
          tc_fence_after();
          const uint32_t bhi = bbase + b * kTcSBytes, blo = bhi + kTcImg;
          for (int j = 0; j < mt; ++j) {
            const uint32_t ahi = abase + s * kTcABytes + (uint32_t)(j * 2 * kTcImg);
            const uint32_t alo = ahi + kTcImg;
            const uint32_t d = tmem + tb * 256u + (uint32_t)(j * 128);
#pragma unroll
            for (int ks = 0; ks < kTcKC / 8; ++ks) {
              const uint32_t ko = (uint32_t)ks * 256u;  // two K-cores per product
              const uint32_t acc0 = (c > 0 || ks > 0) ? 1u : 0u;
              constexpr uint32_t G = kTcGroup;
              tc_mma_tf32(d, tc_sdesc(ahi + ko, 128u, G), tc_sdesc(bhi + ko, 128u, G), kDftIdesc, acc0);
              tc_mma_tf32(d, tc_sdesc(ahi + ko, 128u, G), tc_sdesc(blo + ko, 128u, G), kDftIdesc, 1u);
              tc_mma_tf32(d, tc_sdesc(alo + ko, 128u, G), tc_sdesc(bhi + ko, 128u, G), kDftIdesc, 1u);
            }
          }
          tc_commit(&empty[s]);
          tc_commit(&sfree[b]);
        }
        if (ok) tc_commit(&tfull[tb]);
      }
      tc_commit(&done_bar);
      mbar_wait(&done_bar, 0, a.status);
    }
  } else if (warp < 6) {
    // ---- split: samples of point n = 32 (warp - 2) + lane into hi / lo rows
    const int n = 32 * (warp - 2) + lane;
    uint32_t q = 0;
    bool ok = true;
    for (long long tile = blockIdx.x; tile < ntiles && ok && !*ab; tile += gridDim.x)
      for (int c = 0; c < nch; ++c, ++q) {
        const int s = (int)(q % kTcStages), b = (int)(q & 1), rb = (int)(q >> 1);
        int got = 1;
        if (lane == 0) {
          got = tc_wait(&full[s], (q / kTcStages) & 1, a.status, ab) ? 1 : 0;
          if (got && rb > 0) got = tc_wait(&sfree[b], (rb & 1) ^ 1, a.status, ab) ? 1 : 0;
        }
        if (!(ok = __shfl_sync(0xffffffffu, got, 0) != 0)) break;
        const float* vr = reinterpret_cast<const float*>(vraw + s * kTcVBytes);
        unsigned char* hi = bspl + b * kTcSBytes;
        unsigned char* lo = hi + kTcImg;
#pragma unroll
        for (int k4 = 0; k4 < kTcKC / 4; ++k4) {
          float4 h, l;
          float* hp = &h.x;
          float* lp = &l.x;
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float x = vr[(k4 * 4 + e) * kTcNP + n];
            hp[e] = tf32_rna(x);
            lp[e] = tf32_rna(x - hp[e]);
          }
          *reinterpret_cast<float4*>(hi + img_off(n, k4 * 4)) = h;
          *reinterpret_cast<float4*>(lo + img_off(n, k4 * 4)) = l;
        }
        fence_async_smem();  // visible to the tensor cores (async proxy)
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&sready[b]);
          mbar_arrive(&empty[s]);  // the samples of this stage are read
        }
      }
  } else {
    // ---- epilogue: TMEM lane quarter q = warp & 3 (warps 6..9 -> 2, 3, 0, 1)
    const int quarter = warp & 3, row = quarter * 32 + lane;
    uint32_t p = 0;
    bool ok = true;
    for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++p) {
      const uint32_t tb = p & 1;
      int got = 0;
      if (lane == 0) got = tc_wait(&tfull[tb], (p >> 1) & 1, a.status, ab) ? 1 : 0;
      if (!(ok = __shfl_sync(0xffffffffu, got, 0) != 0)) break;
      tc_fence_after();
      const long long x0 = tile * kTcNP;
      for (int j = 0; j < mt; ++j) {
        const int bin = 64 * j + (row & 63);
        float* dst = (row < 64 ? a.re : a.im) + (long long)bin * a.N;
#pragma unroll 1
        for (int cb = 0; cb < kTcNP / 32; ++cb) {
          uint32_t r[32];
          tc_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + tb * 256u + (uint32_t)(j * 128 + cb * 32),
                  r);
          tc_wait_ld();
          const long long xb = x0 + cb * 32;
          if (bin < a.nb) {
            if (xb + 32 <= a.N) {
              float4* dp = reinterpret_cast<float4*>(dst + xb);
              if (a.overwrite) {
#pragma unroll
                for (int k = 0; k < 8; ++k)
                  dp[k] = make_float4(__uint_as_float(r[4 * k]), __uint_as_float(r[4 * k + 1]),
                                      __uint_as_float(r[4 * k + 2]), __uint_as_float(r[4 * k + 3]));
              } else {
                float4 v[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) v[k] = dp[k];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                  v[k].x += __uint_as_float(r[4 * k]);
                  v[k].y += __uint_as_float(r[4 * k + 1]);
                  v[k].z += __uint_as_float(r[4 * k + 2]);
                  v[k].w += __uint_as_float(r[4 * k + 3]);
                  dp[k] = v[k];
                }
              }
            } else {
              for (int k = 0; k < 32 && xb + k < a.N; ++k)
                dst[xb + k] = (a.overwrite ? 0.0f : dst[xb + k]) + __uint_as_float(r[k]);
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[tb]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tc_dealloc(tmem, 512);
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

int dft_tc_chunk() { return kTcKC; }

size_t dft_tc_image_bytes(int T, int nb) {
  const int mt = (nb + 63) / 64, nch = (T + kTcKC - 1) / kTcKC;
  return (size_t)nch * mt * 2 * kTcImg;
}

bool dft_tc_supported(long long N, int nb) { return N % 4 == 0 && nb >= 1 && nb <= 64 * kTcMaxMt; }

cudaError_t launch_dft_tc(const CUtensorMap& vmap, long long N, int T, int n0, int nf,
                          const int* bins, int nb, float* W, float* re, float* im, bool overwrite,
                          int* status, cudaStream_t s) {
  if (T <= 0 || N <= 0) return cudaSuccess;
  if (!dft_tc_supported(N, nb)) return cudaErrorInvalidValue;
  const int mt = (nb + 63) / 64, nch = (T + kTcKC - 1) / kTcKC;
  const int n = nch * mt * 128 * kTcKC;
  dft_image_kernel<<<(n + 255) / 256, 256, 0, s>>>(T, n0, nf, bins, nb, mt, nch, W);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  static bool attr = false;
  if (!attr) {
    e = cudaFuncSetAttribute(dft_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  DftTcArgs a{W, re, im, N, nb, mt, nch, overwrite ? 1 : 0, status};
  const long long ntiles = (N + kTcNP - 1) / kTcNP;
  const int grid = (int)std::min<long long>(ntiles, 152);
  dft_tc_kernel<<<grid, kTcDftThreads, kTcSmem, s>>>(vmap, a);
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
