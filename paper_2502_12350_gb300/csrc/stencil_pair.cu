// Two time levels per pass over HBM (temporal blocking of the forward step).
//
// The scheme is the same as the one-step kernel's (Eq. 1; Sec. 2.1), point by
// point and bit by bit: u^{n+1} = g (2 u^n - M u^n - g u^{n-1} + A lap u^n),
// then u^{n+2} from u^{n+1} and u^n.  One launch advances two steps:
//
//   * Each CTA owns a TX x TY tile of the padded grid (all planes) and marches
//     in z.  At iteration j it computes u^{n+1} on plane j (step A) and, four
//     planes behind, u^{n+2} on plane j - 4 (step B).
//   * Step A reads u^n with its xy halo from a TMA ring (as the one-step
//     kernel), u^{n-1}, A, A m2 from a second ring, writes u^{n+1} over
//     u^{n-1} and keeps it in a register queue for step B's z stencil.
//   * Step B needs the xy halo of u^{n+1} on plane j - 4, which the
//     neighbouring tiles compute.  Every CTA publishes how many planes of
//     u^{n+1} it has stored (a release store after a barrier of its compute
//     warps); a producer lane waits until the four neighbours (and the tile
//     itself) have published plane j - 4, then loads the halo'd plane from
//     L2 by TMA.  Step B then writes u^{n+2} over u^n: every neighbour has
//     finished step A on that plane, so it no longer reads u^n there.
//   * All tiles must run at once (they wait on each other), so the launch is
//     cooperative and uses at most one CTA per SM; every wait is bounded.
//
// HBM traffic per point and pair of steps: u^n, u^{n-1}, A, A m2 read once,
// u^{n+1} and u^{n+2} written once (24 B with density, 20 without), against
// 40 / 32 B for two one-step launches; the second reads of A, A m2 and the
// u^{n+1} halo come from L2.
//
// Each compute thread owns 4 consecutive x points on 2 rows (8 points), so
// the y neighbours of both rows come from 12 shared-memory loads instead of
// 20.
#include "stencil_impl.cuh"

namespace mamute {

namespace {

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void fence_acq_rel_gpu() {
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Tensor memory (TMEM) holds step B's z column of u^{n+1}: 9 planes x 8
// points per thread, in the 32 lanes of the warp's subpartition.
__device__ __forceinline__ void tm_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tm_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tm_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tm_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tm_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// 8 consecutive columns of this thread's lane: the 8 points of one plane.
__device__ __forceinline__ void tm_st8(uint32_t taddr, const F4& r0, const F4& r1) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
      "f"(r0.v[0]), "f"(r0.v[1]), "f"(r0.v[2]), "f"(r0.v[3]), "f"(r1.v[0]), "f"(r1.v[1]),
      "f"(r1.v[2]), "f"(r1.v[3])
      : "memory");
}
__device__ __forceinline__ void tm_ld8(uint32_t taddr, F4& r0, F4& r1) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(r0.v[0]), "=f"(r0.v[1]), "=f"(r0.v[2]), "=f"(r0.v[3]), "=f"(r1.v[0]), "=f"(r1.v[1]),
        "=f"(r1.v[2]), "=f"(r1.v[3])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tm_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Step B's lap for the 8 points of a thread, with the z column streamed from
// TMEM one pair of planes (z - 1 - m, z + 1 + m) at a time; the operations
// and their order are lap25's, so the values are bitwise the one-step
// kernel's.  slot(p) is the TMEM column address of plane p; c0, c1 are the
// centre rows (plane z).
template <int TX, typename Slot>
__device__ __forceinline__ void lap8_tm(const float* st, int lx, int ly0, const F4& c0,
                                        const F4& c1, Slot slot, int z, float (&oa)[4],
                                        float (&ob)[4]) {
  constexpr int RP = TX + 2 * kHalo;
  const float cw[4] = {MAMUTE_C1, MAMUTE_C2, MAMUTE_C3, MAMUTE_C4};
  const float* r0 = st + (ly0 + kHalo) * RP + lx;
  const float* r1 = r0 + RP;
  const F4 L0 = ld4s(r0), R0 = ld4s(r0 + 8), L1 = ld4s(r1), R1 = ld4s(r1 + 8);
  float xa[12], xb[12];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    xa[k] = L0.v[k];
    xa[4 + k] = c0.v[k];
    xa[8 + k] = R0.v[k];
    xb[k] = L1.v[k];
    xb[4 + k] = c1.v[k];
    xb[8 + k] = R1.v[k];
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    oa[e] = __fmul_rn(3.0f * MAMUTE_C0, c0.v[e]);
    ob[e] = __fmul_rn(3.0f * MAMUTE_C0, c1.v[e]);
  }
  F4 upp = c0, dnp = c1;  // rows at distance m from the pair (m = 0: the pair itself)
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const F4 up = ld4s(r0 + kHalo - (m + 1) * RP);  // row ly0 - 1 - m
    const F4 dn = ld4s(r1 + kHalo + (m + 1) * RP);  // row ly0 + 2 + m
    F4 zm0, zm1, zp0, zp1;
    tm_ld8(slot(z - 1 - m), zm0, zm1);
    tm_ld8(slot(z + 1 + m), zp0, zp1);
    tm_wait_ld();
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      // row ly0: y- = row ly0 - 1 - m, y+ = row ly0 + 1 + m
      float sa = __fadd_rn(__fadd_rn(__fadd_rn(xa[4 + e - (m + 1)], xa[4 + e + (m + 1)]),
                                     __fadd_rn(up.v[e], m == 0 ? c1.v[e] : dnp.v[e])),
                           __fadd_rn(zm0.v[e], zp0.v[e]));
      oa[e] = __fmaf_rn(cw[m], sa, oa[e]);
      // row ly0 + 1: y- = row ly0 - m, y+ = row ly0 + 2 + m
      float sb = __fadd_rn(__fadd_rn(__fadd_rn(xb[4 + e - (m + 1)], xb[4 + e + (m + 1)]),
                                     __fadd_rn(m == 0 ? c0.v[e] : upp.v[e], dn.v[e])),
                           __fadd_rn(zm1.v[e], zp1.v[e]));
      ob[e] = __fmaf_rn(cw[m], sb, ob[e]);
    }
    upp = up;
    dnp = dn;
  }
}

// lap for the 8 points of a thread (rows ly0 and ly0 + 1, columns lx..lx+3):
// halo stage `st` with row pitch TX + 8; z columns from q0 / q1 (one queue
// per row).  Operands reach lap25 in the same order as in lap4, so each
// point's value is bitwise the one-step kernel's.
template <int TX>
__device__ __forceinline__ void lap8(const float* st, int lx, int ly0, const F4 (&qa)[9],
                                     const F4 (&qb)[9], float (&oa)[4], float (&ob)[4]) {
  constexpr int RP = TX + 2 * kHalo;
  const float* r0 = st + (ly0 + kHalo) * RP + lx;  // row ly0, x from lx - 4
  const float* r1 = r0 + RP;
  F4 L0 = ld4s(r0), R0 = ld4s(r0 + 8), L1 = ld4s(r1), R1 = ld4s(r1 + 8);
  F4 up[4], dn[4];  // rows ly0 - 1 - m and ly0 + 2 + m (centre columns)
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    up[m] = ld4s(r0 + kHalo - (m + 1) * RP);
    dn[m] = ld4s(r1 + kHalo + (m + 1) * RP);
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    float xa[12], xb[12];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      xa[k] = L0.v[k];
      xa[4 + k] = qa[4].v[k];
      xa[8 + k] = R0.v[k];
      xb[k] = L1.v[k];
      xb[4 + k] = qb[4].v[k];
      xb[8 + k] = R1.v[k];
    }
    float a[4], b[4], c[4], d[4], f[4], g[4];
    // row ly0
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      a[m] = xa[4 + e - (m + 1)];
      b[m] = xa[4 + e + (m + 1)];
      c[m] = up[m].v[e];
      d[m] = m == 0 ? qb[4].v[e] : dn[m - 1].v[e];
      f[m] = qa[3 - m].v[e];
      g[m] = qa[5 + m].v[e];
    }
    oa[e] = lap25(qa[4].v[e], a, b, c, d, f, g);
    // row ly0 + 1
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      a[m] = xb[4 + e - (m + 1)];
      b[m] = xb[4 + e + (m + 1)];
      c[m] = m == 0 ? qa[4].v[e] : up[m - 1].v[e];
      d[m] = dn[m].v[e];
      f[m] = qb[3 - m].v[e];
      g[m] = qb[5 + m].v[e];
    }
    ob[e] = lap25(qb[4].v[e], a, b, c, d, f, g);
  }
}

template <int TX, int TY, bool DENS>
struct PairLayout {
  static constexpr int NCT = (TX / 4) * (TY / 2);
  static constexpr int NW = NCT / 32;
  static constexpr int HS = (TX + 2 * kHalo) * (TY + 2 * kHalo);
  static constexpr int CS = TX * TY;
  static constexpr int NSU = 6;  // u^n halo ring: 5 planes in use, 1 ahead
  static constexpr int NSC = 2;  // u^{n-1}, A, A m2 of step A
  static constexpr int NSV = 2;  // u^{n+1} halo + A, A m2 of step B
  static constexpr int NCA = DENS ? 3 : 2;  // centre arrays of step A
  static constexpr int NCB = DENS ? 2 : 1;  // centre arrays of step B (A, A m2)
  static constexpr int VS = HS + NCB * CS;  // floats per step-B stage
  static constexpr int NST = 8;  // "plane stored" barriers between the warps and the publisher
  static constexpr size_t base_bytes =
      sizeof(float) * ((size_t)NSU * HS + (size_t)NSC * NCA * CS + (size_t)NSV * VS + CS) +
      sizeof(uint64_t) * (2 * NSU + 2 * NSC + 2 * NSV + NST);
};

}  // namespace

template <int TX, int TY, bool DENS>
__global__ void __launch_bounds__((TX / 4) * (TY / 2) + 32, 1) pair_kernel(const PairArgs a) {
  using LY = PairLayout<TX, TY, DENS>;
  constexpr int NCT = LY::NCT, NW = LY::NW, HS = LY::HS, CS = LY::CS;
  constexpr int NSU = LY::NSU, NSC = LY::NSC, NSV = LY::NSV, NCA = LY::NCA;
  constexpr int VS = LY::VS;
  static_assert(NCT % 32 == 0, "whole compute warps");

  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* ringU = reinterpret_cast<float*>(smem_raw);
  float* ringC = ringU + NSU * HS;
  float* ringV = ringC + NSC * NCA * CS;
  float* otile = ringV + NSV * VS;
  uint64_t* bars = reinterpret_cast<uint64_t*>(otile + CS);
  uint64_t* fullU = bars;
  uint64_t* emptyU = fullU + NSU;
  uint64_t* fullC = emptyU + NSU;
  uint64_t* emptyC = fullC + NSC;
  uint64_t* fullV = emptyC + NSC;
  uint64_t* emptyV = fullV + NSV;
  uint64_t* stored = emptyV + NSV;  // plane j of u^{n+1} stored by every compute warp
  constexpr int NST = LY::NST;

  const WorkItem it = a.items[blockIdx.x];
  const int4 nb = a.nbrs[blockIdx.x];
  const VolDesc V = a.vols[it.vol];
  const PairMaps* pm = a.pmaps + it.vol;
  const int x0 = it.x0, y0 = it.y0;
  const int Nz = V.Nz;
  const int tid = threadIdx.x;

  // Per-plane data (sponge factor, receiver-entry range) straight from
  // global memory: shared memory is taken up by the rings.
  auto plane_info = [&](int j) {
    PlaneInfo pi;
    pi.gz = a.gz[j];
    pi.rb = pi.re = 0;
    if (it.rec_tab >= 0) {
      pi.rb = a.rec_ptr[it.rec_tab + j];
      pi.re = a.rec_ptr[it.rec_tab + j + 1];
    }
    pi.pad = 0;
    return pi;
  };
  if (tid == 0) {
    for (int s = 0; s < NSU; ++s) {
      mbar_init(&fullU[s], 1);
      mbar_init(&emptyU[s], NW);
    }
    for (int s = 0; s < NSC; ++s) {
      mbar_init(&fullC[s], 1);
      mbar_init(&emptyC[s], NW);
    }
    for (int s = 0; s < NSV; ++s) {
      mbar_init(&fullV[s], 1);
      mbar_init(&emptyV[s], NW);
    }
    for (int s = 0; s < NST; ++s) mbar_init(&stored[s], NW);
    fence_barrier_init();
  }
  __shared__ uint32_t tmem_base;
  constexpr uint32_t kTmCols = 256;  // 9 planes x 8 points per warp, 3 warps per lane group
  static_assert(((NW + 3) / 4) * 72 <= (int)kTmCols, "TMEM columns");
  if (tid < 32) {
    tm_alloc(&tmem_base, kTmCols);
    tm_relinquish();
  }
  tm_fence_before();
  __syncthreads();
  tm_fence_after();

  const int cx = V.cx0 + x0, cy = V.cy0 + y0;
  if (tid >= NCT) {
    // ------------------------------------------------------------ producers
    const int lane = tid - NCT;
    if (lane == 0) {
      // u^n planes -4 .. Nz+3 (halo'd) and u^{n-1}, A, A m2 of planes 0 .. Nz-1
      tmap_acquire(&pm->m[0]);
      tmap_acquire(&pm->m[3]);
      tmap_acquire(&pm->m[4]);
      if (DENS) tmap_acquire(&pm->m[5]);
      int nU = 0, nC = 0;
      auto drain = [&]() {
        for (int s = 0; s < NSU && s < nU; ++s)
          mbar_wait(&fullU[s], (uint32_t)(((nU - 1 - s) / NSU) & 1), a.status);
        for (int c = 0; c < NSC && c < nC; ++c)
          mbar_wait(&fullC[c], (uint32_t)(((nC - 1 - c) / NSC) & 1), a.status);
      };
      for (int i = 0; i < Nz + 2 * kHalo; ++i) {
        const int s = i % NSU, r = i / NSU;
        if (r > 0 && !mbar_wait(&emptyU[s], (r & 1) ^ 1, a.status)) {
          drain();
          return;
        }
        mbar_arrive_expect_tx(&fullU[s], HS * 4);
        tma_load_3d(ringU + s * HS, &pm->m[0], x0 - kHalo, y0 - kHalo, i - kHalo, &fullU[s]);
        ++nU;
        if (i >= 2 * kHalo) {
          const int j = i - 2 * kHalo;
          const int c = j % NSC, rc = j / NSC;
          if (rc > 0 && !mbar_wait(&emptyC[c], (rc & 1) ^ 1, a.status)) {
            drain();
            return;
          }
          mbar_arrive_expect_tx(&fullC[c], NCA * CS * 4);
          float* cd = ringC + c * NCA * CS;
          tma_load_3d(cd, &pm->m[3], x0, y0, j, &fullC[c]);
          tma_load_3d(cd + CS, &pm->m[4], cx, cy, j, &fullC[c]);
          if (DENS) tma_load_3d(cd + 2 * CS, &pm->m[5], cx, cy, j, &fullC[c]);
          ++nC;
        }
      }
    } else if (lane == 1) {
      // u^{n+1} planes 0 .. Nz-1 (halo'd, once this tile and its neighbours
      // have stored them) with A, A m2 of the same plane, for step B
      tmap_acquire(&pm->m[1]);
      tmap_acquire(&pm->m[4]);
      if (DENS) tmap_acquire(&pm->m[5]);
      int nV = 0;
      auto drain = [&]() {
        for (int s = 0; s < NSV && s < nV; ++s)
          mbar_wait(&fullV[s], (uint32_t)(((nV - 1 - s) / NSV) & 1), a.status);
      };
      // Waits (bounded) until this tile and its neighbours have published
      // plane z: the five flags are polled together, then one acquire fence.
      auto published = [&](int target) {
        const int t[5] = {(int)blockIdx.x, nb.x, nb.y, nb.z, nb.w};
        for (long long spin = 0; spin < kSpinLimit; ++spin) {
          bool ok = true;
#pragma unroll
          for (int k = 0; k < 5; ++k)
            if (t[k] >= 0 && ld_relaxed(a.flags + t[k]) < target) ok = false;
          if (ok) {
            fence_acq_rel_gpu();
            return true;
          }
        }
        atomicOr(a.status, kErrTimeout);
        return false;
      };
      for (int z = 0; z < Nz; ++z) {
        const int s = z % NSV, r = z / NSV;
        if (r > 0 && !mbar_wait(&emptyV[s], (r & 1) ^ 1, a.status)) {
          drain();
          return;
        }
        if (!published(a.epoch + z + 1)) {
          drain();
          return;
        }
        fence_proxy_async_global();  // the TMA reads below see the stores they waited for
        mbar_arrive_expect_tx(&fullV[s], VS * 4);
        float* vd = ringV + s * VS;
        tma_load_3d(vd, &pm->m[1], x0 - kHalo, y0 - kHalo, z, &fullV[s]);
        tma_load_3d(vd + HS, &pm->m[4], cx, cy, z, &fullV[s]);
        if (DENS) tma_load_3d(vd + HS + CS, &pm->m[5], cx, cy, z, &fullV[s]);
        ++nV;
      }
    } else if (lane == 2) {
      // Publisher: once every compute warp has stored plane j of u^{n+1},
      // make the stores visible at GPU scope and advance this tile's flag
      // (off the compute warps' path).
      for (int j = 0; j < Nz; ++j) {
        if (!mbar_wait(&stored[j % NST], (uint32_t)((j / NST) & 1), a.status)) return;
        __threadfence();
        st_release(a.flags + blockIdx.x, a.epoch + j + 1);
      }
    }
    return;
  }

  // -------------------------------------------------------------- consumers
  constexpr int RP = TX + 2 * kHalo;
  const int lx = (tid % (TX / 4)) * 4, ly0 = (tid / (TX / 4)) * 2;
  const int gxl = x0 + lx;
  const int lane = tid & 31;
  const bool col_ok = lx < it.w && gxl < V.Nx;
  bool row_ok[2];
  float gyv[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int y = y0 + ly0 + r;
    row_ok[r] = ly0 + r < it.h && y < V.Ny;
    // Tile rows start on even rows, so both rows of a thread are in the tile
    // or both past it (then computed from halo data but neither stored nor
    // used); past the window the field is zero.
    gyv[r] = y < V.Ny ? a.gy[V.gy_off + y] : 0.0f;
  }
  float gxv[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) gxv[e] = (gxl + e < V.Nx) ? a.gx[V.gx_off + gxl + e] : 0.0f;
  const int off0 = (ly0 + kHalo) * RP + lx + kHalo;  // centre of row ly0 in a halo stage

  bool dead = false;
  auto wait = [&](uint64_t* bar, uint32_t parity) {
    if (!dead && !mbar_wait(bar, parity, a.status)) dead = true;
  };
  auto release = [&](uint64_t* bar) {
    __syncwarp();
    if (lane == 0) mbar_arrive(bar);
  };
  // Stores a level on plane z, records its receivers and injects the source.
  auto finish = [&](F4 (&out)[2], int z, float wn, float* dout, float* fout) {
    // source: w_e dt^2 w[n] / (h^3 sqrt rho_e) at the corners of its cell
    const int dz = z - V.src_z;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int dy = y0 + ly0 + r - V.src_y;
      if ((unsigned)dz < 2u && (unsigned)dy < 2u) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int dx = gxl + e - V.src_x;
          if ((unsigned)dx < 2u) {
            const float sc = a.vols[it.vol].src_sc[dx + 2 * dy + 4 * dz];  // global: dynamic index
            if (sc != 0.0f) out[r].v[e] = __fmaf_rn(sc, wn, out[r].v[e]);
          }
        }
      }
    }
    const PlaneInfo pi = plane_info(z);
    if (pi.rb < pi.re) {
#pragma unroll
      for (int r = 0; r < 2; ++r)
        *reinterpret_cast<float4*>(otile + (ly0 + r) * TX + lx) =
            make_float4(out[r].v[0], out[r].v[1], out[r].v[2], out[r].v[3]);
      compute_sync(NCT);
      if (dout)
        for (int e = pi.rb + tid; e < pi.re; e += NCT) {
          const RecEntry re = a.rec[e];
          dout[re.col] = re.fscale * otile[re.lxy];
        }
      compute_sync(NCT);
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      if (!(row_ok[r] && col_ok)) continue;
      F4 o = out[r];
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (gxl + e >= V.Nx) o.v[e] = 0.0f;
      st4g(fout + V.off + ((long long)z * V.Ny + y0 + ly0 + r) * V.pitch + gxl, o);
    }
  };

  F4 qa[9], qb[9];  // u^n z columns of rows ly0, ly0 + 1 (registers)
  // u^{n+1} z columns in TMEM: plane p at columns wcol + 8 (p mod 9)
  const int warp = tid >> 5;
  const uint32_t tm_lane = (uint32_t)((warp & 3) * 32) << 16;
  const uint32_t wcol = tmem_base + (uint32_t)((warp >> 2) * 72);
  auto slot = [&](int p) { return tm_lane | (wcol + (uint32_t)(8 * ((p + 18) % 9))); };
  const F4 zero4 = {{0.f, 0.f, 0.f, 0.f}};
  for (int k = 0; k < 9; ++k) tm_st8(tm_lane | (wcol + 8 * k), zero4, zero4);  // planes < 0
  tm_wait_st();
  // Priming: u^n planes -4 .. 3.
  for (int i = 0; i < 2 * kHalo; ++i) {
    const int s = i % NSU;
    wait(&fullU[s], (i / NSU) & 1);
    qa[i] = ld4s(ringU + s * HS + off0);
    qb[i] = ld4s(ringU + s * HS + off0 + RP);
    if (i < kHalo || i - kHalo >= Nz) release(&emptyU[s]);
  }

  for (int j = 0; j < Nz + kHalo; ++j) {
    if (j < Nz) {
      // ---------------------------------------------------- step A, plane j
      {
        const int i = j + 2 * kHalo, s = i % NSU;
        wait(&fullU[s], (i / NSU) & 1);
        qa[8] = ld4s(ringU + s * HS + off0);
        qb[8] = ld4s(ringU + s * HS + off0 + RP);
        if (j + kHalo >= Nz) release(&emptyU[s]);
      }
      const int c = j % NSC;
      wait(&fullC[c], (j / NSC) & 1);
      const int su = (j + kHalo) % NSU;
      float la[4], lb[4];
      lap8<TX>(ringU + su * HS, lx, ly0, qa, qb, la, lb);
      const float* cs = ringC + c * NCA * CS + ly0 * TX + lx;
      const float gz = a.gz[j];
      F4 out[2];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const F4 prev = ld4s(cs + r * TX);
        const F4 Av = ld4s(cs + CS + r * TX);
        F4 Mv = {{0.f, 0.f, 0.f, 0.f}};
        if (DENS) Mv = ld4s(cs + 2 * CS + r * TX);
        const float gyz = __fmul_rn(gyv[r], gz);
        const F4& u = r ? qb[4] : qa[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float g = __fmul_rn(gxv[e], gyz);
          out[r].v[e] = update(u.v[e], prev.v[e], Av.v[e], Mv.v[e], g, r ? lb[e] : la[e], DENS);
        }
      }
      release(&emptyU[su]);
      release(&emptyC[c]);
      finish(out, j, a.wn0, a.dout0, a.fout1);
      // Plane j of u^{n+1} is stored by this warp; the publisher lane waits
      // for all of them.
      release(&stored[j % NST]);
      tm_st8(slot(j), out[0], out[1]);  // after release()'s __syncwarp: warp-wide
    } else {
      __syncwarp();
      tm_st8(slot(j), zero4, zero4);  // u^{n+1} is zero past the last plane
      qa[8] = zero4;
      qb[8] = zero4;
    }
    tm_wait_st();
    if (j >= kHalo) {
      // ---------------------------------------------- step B, plane j - 4
      const int z = j - kHalo;
      const int s = z % NSV;
      wait(&fullV[s], (z / NSV) & 1);
      F4 c0, c1;  // u^{n+1} on plane z
      __syncwarp();
      tm_ld8(slot(z), c0, c1);
      tm_wait_ld();
      float la[4], lb[4];
      lap8_tm<TX>(ringV + s * VS, lx, ly0, c0, c1, slot, z, la, lb);
      const float* cs = ringV + s * VS + HS + ly0 * TX + lx;
      const float gz = a.gz[z];
      F4 out[2];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const F4 Av = ld4s(cs + r * TX);
        F4 Mv = {{0.f, 0.f, 0.f, 0.f}};
        if (DENS) Mv = ld4s(cs + CS + r * TX);
        const float gyz = __fmul_rn(gyv[r], gz);
        const F4& u = r ? c1 : c0;
        const F4& prev = r ? qb[0] : qa[0];  // u^n on plane j - 4
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float g = __fmul_rn(gxv[e], gyz);
          out[r].v[e] = update(u.v[e], prev.v[e], Av.v[e], Mv.v[e], g, r ? lb[e] : la[e], DENS);
        }
      }
      release(&emptyV[s]);
      finish(out, z, a.wn1, a.dout1, a.fout2);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      qa[k] = qa[k + 1];
      qb[k] = qb[k + 1];
    }
  }
  // Every compute warp is done with TMEM: warp 0 returns the columns.
  tm_fence_before();
  compute_sync(NCT);
  if (warp == 0) {
    tm_fence_after();
    tm_dealloc(tmem_base, kTmCols);
  }
}

template <int TX, int TY, bool DENS>
static size_t pair_smem(int) {
  return PairLayout<TX, TY, DENS>::base_bytes;
}

template <int TX, int TY, bool DENS>
static cudaError_t pair_one(const PairArgs& a, int n_items, int nz, cudaStream_t s, int* occ) {
  const size_t sm = pair_smem<TX, TY, DENS>(nz);
  static size_t attr = 0;
  if (sm > attr) {
    cudaError_t e = cudaFuncSetAttribute(pair_kernel<TX, TY, DENS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    attr = sm;
  }
  const int threads = (TX / 4) * (TY / 2) + 32;
  if (occ)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, pair_kernel<TX, TY, DENS>, threads,
                                                         sm);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)n_items);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = s;
  cudaLaunchAttribute attrs[1];
  attrs[0].id = cudaLaunchAttributeCooperative;  // the tiles wait on each other
  attrs[0].val.cooperative = 1;
  cfg.attrs = attrs;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, pair_kernel<TX, TY, DENS>, a);
}

bool pair_tile_supported(int tx, int ty) {
#define MAMUTE_P(TX, TY) if (tx == TX && ty == TY) return true;
  MAMUTE_PAIR_TILES(MAMUTE_P)
#undef MAMUTE_P
  return false;
}

cudaError_t launch_pair(const PairArgs& a, int n_items, int nz, int tx, int ty, bool dens,
                        cudaStream_t s, int* occ) {
  if (!occ && n_items <= 0) return cudaSuccess;
#define MAMUTE_P(TX, TY)                                                          \
  if (tx == TX && ty == TY)                                                       \
    return dens ? pair_one<TX, TY, true>(a, n_items, nz, s, occ)                  \
                : pair_one<TX, TY, false>(a, n_items, nz, s, occ);
  MAMUTE_PAIR_TILES(MAMUTE_P)
#undef MAMUTE_P
  return cudaErrorInvalidValue;
}

}  // namespace mamute
