// Internal declarations shared by the CUDA translation units of libmamute.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mamute {

// Radius-4 central weights of the eighth-order second derivative
// (Sec. 2.1: eighth order in space).  kC0x3 is 3 c0 (the centre term of the
// three axes).
#define MAMUTE_C0 (-205.0f / 72.0f)
#define MAMUTE_C1 (8.0f / 5.0f)
#define MAMUTE_C2 (-1.0f / 5.0f)
#define MAMUTE_C3 (8.0f / 315.0f)
#define MAMUTE_C4 (-1.0f / 560.0f)

constexpr int kHalo = 4;             // stencil radius
constexpr long long kSpinLimit = 1LL << 24;  // bounded mbarrier waits

// Error flags written by kernels (bit mask in the context status word).
constexpr int kErrTimeout = 1;

// One shot's propagation domain (a window of the global padded grid).
struct VolDesc {
  int Nx, Ny, Nz;        // local padded dimensions
  int pitch;             // floats per row of the shot's wavefield arrays
  int cx0, cy0;          // origin of the window in the global padded grid
  int gx_off, gy_off;    // offsets of the shot's x / y sponge profiles
  int src_x, src_y, src_z;  // source cell corner (0,0,0), local padded coordinates
  // dt^2 w_e / (h^3 sqrt(rho_e)) for the corners e = dx + 2 dy + 4 dz of the
  // source cell (nearest node: corner 0 only; trilinear: the 8 weights w_e)
  float src_sc[8];
  int border;            // sponge cells on each face
  // Imaging region: the window's cells that lie in the model, local x in
  // [ix0, ix0 + nxi), y in [iy0, iy0 + nyi), z in [border, border + nzi).  The
  // stored imaging terms cover it (rows of tpitch floats from local x =
  // txoff), and the gradient / pseudo-Hessian take the accumulator (pool
  // layout) on it.
  int ix0, iy0;
  int nxi, nyi, nzi;
  int txoff, tpitch;     // term store rows: local x in [txoff, txoff + tpitch)
  long long off;         // element offset of the shot's arrays in each pool
  long long slab;        // elements per wavefield array (Nz * Ny * pitch, rounded)
  long long toff;        // offset of the shot's region in one step of the term store
};

// One CTA's work: the w x h tile at (x0, y0) of one shot's padded window
// (local coordinates; x0 a multiple of 4, w <= TX, h <= TY), planes [zb, ze).
struct WorkItem {
  int vol, x0, y0, zb, ze, w, h;
  int rec_tab;  // offset of this item's per-plane receiver table, -1 if none
};

// A receiver as seen by the tile that owns it.
struct RecEntry {
  int lxy;        // lx + TX * ly inside the tile
  int col;        // column in the internal [nt][n_col] data layout
  int group;      // number of entries sharing this node if first of its group, else 0
  float fscale;   // forward sampling scale w sqrt(rho) at the node
  float ascale;   // adjoint injection scale w c^2 dt^2 g sqrt(rho) at the node
  float wgt;      // interpolation weight w of the node (1 for the nearest node)
  int pad1, pad2;
};

// Tensor maps of one shot (array of these in device memory).  Halo boxes are
// (TX+8) x (TY+8) x 1, centre boxes TX x TY x 1, for the forward tile (F) or
// the adjoint tile (A):
//   [0] u0 halo F   [1] u0 centre F   [2] u1 halo F   [3] u1 centre F
//   [4] p0 halo A   [5] p0 centre A   [6] p1 halo A   [7] p1 centre A
//   [8] accumulator centre F (pseudo-Hessian)
//   [9] u0 halo A  [10] u1 halo A    (forward field read by the imaging)
//  [11] accumulator centre A (imaging)
//  [12] term store (x, y, z, step) centre A, 4-D (all-states adjoint)
struct ShotMaps {
  CUtensorMap m[13];
};

// Global coefficient maps: [0] A centre, [1] M = A m2 centre.
struct CoefMaps {
  CUtensorMap m[2];
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: returns false (and records a timeout) if the phase does not
// complete within kSpinLimit polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* status) {
  for (long long i = 0; i < kSpinLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  atomicOr(status, kErrTimeout);
  return false;
}

__device__ __forceinline__ void tmap_acquire(const CUtensorMap* m) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(m) : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* m, int x, int y, int z,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(m), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* m, int x, int y, int z,
                                            int w, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(m), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
      : "memory");
}

// Named barrier among the compute warps only (id 1).
__device__ __forceinline__ void compute_sync(int nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

}  // namespace mamute
