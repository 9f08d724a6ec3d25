// Forward and adjoint time steps of the eighth-order acoustic scheme
// (Eq. 1; Sec. 2.1; Table 1 ModelingStep + ReadReceiver; Algorithm 3
// backward loop with the cross-correlation imaging condition).
//
// One CTA owns a TX x TY tile of one shot's padded grid and marches through
// its planes in z (2.5-D blocking).  A producer warp streams, with TMA,
//   * the propagated field plane by plane with its 4-cell xy halo into a ring
//     of shared-memory stages (zero fill outside the grid = the Dirichlet
//     exterior), and
//   * the centre tiles of the other per-point arrays (previous level, A,
//     A m2, accumulator) into a second ring,
// both guarded by mbarriers.  Each compute thread owns 4 consecutive x points
// of one row and keeps the 9-plane z column of its points in a register
// queue, so only the xy neighbours are read from shared memory.
//
// Update (forward and adjoint alike; the adjoint runs the same operator on
// psi = A g lambda, which makes it the exact transpose of the forward):
//   out = g (2 u - M u - g prev + A lap u),   M = A m2 (0 without density)
// with A = c^2 dt^2 / h^2 and lap the unscaled 25-point sum.
#pragma once

#include "common.cuh"
#include "stencil.h"

namespace mamute {

namespace {

struct F4 {
  float v[4];
};

__device__ __forceinline__ F4 ld4s(const float* p) {
  float4 t = *reinterpret_cast<const float4*>(p);
  return F4{{t.x, t.y, t.z, t.w}};
}

__device__ __forceinline__ void st4g(float* p, const F4& a) {
  *reinterpret_cast<float4*>(p) = make_float4(a.v[0], a.v[1], a.v[2], a.v[3]);
}

// The 25-point sum for one point, in a fixed order of IEEE operations (no
// contraction freedom), so that every kernel that forms it for the same
// field gets bitwise the same value.
__device__ __forceinline__ float lap25(float u, const float (&xm)[4], const float (&xp)[4],
                                       const float (&ym)[4], const float (&yp)[4],
                                       const float (&zm)[4], const float (&zp)[4]) {
  const float cw[4] = {MAMUTE_C1, MAMUTE_C2, MAMUTE_C3, MAMUTE_C4};
  float acc = __fmul_rn(3.0f * MAMUTE_C0, u);
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    float s = __fadd_rn(__fadd_rn(__fadd_rn(xm[m], xp[m]), __fadd_rn(ym[m], yp[m])),
                        __fadd_rn(zm[m], zp[m]));
    acc = __fmaf_rn(cw[m], s, acc);
  }
  return acc;
}

// lap for the 4 points of a thread: halo stage `st` (row pitch TX + 8), row
// ly, columns lx..lx+3; the z column comes from the register queue q.
template <int TX>
__device__ __forceinline__ void lap4(const float* st, int lx, int ly, const F4 (&q)[9],
                                     float (&out)[4]) {
  constexpr int RP = TX + 2 * kHalo;
  const float* row = st + (ly + kHalo) * RP + lx;
  F4 L = ld4s(row), R = ld4s(row + 8);
  float xs[12];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    xs[e] = L.v[e];
    xs[4 + e] = q[4].v[e];
    xs[8 + e] = R.v[e];
  }
  F4 ym[4], yp[4];
#pragma unroll
  for (int m = 1; m <= 4; ++m) {
    ym[m - 1] = ld4s(row + kHalo - m * RP);
    yp[m - 1] = ld4s(row + kHalo + m * RP);
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    float a[4], b[4], c[4], d[4], f[4], g[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      a[m] = xs[4 + e - (m + 1)];
      b[m] = xs[4 + e + (m + 1)];
      c[m] = ym[m].v[e];
      d[m] = yp[m].v[e];
      f[m] = q[3 - m].v[e];
      g[m] = q[5 + m].v[e];
    }
    out[e] = lap25(q[4].v[e], a, b, c, d, f, g);
  }
}

__device__ __forceinline__ float update(float u, float prev, float A, float M, float g,
                                        float lap, bool dens) {
  float s = __fmaf_rn(2.0f, u, -__fmul_rn(g, prev));
  if (dens) s = __fmaf_rn(-M, u, s);
  s = __fmaf_rn(A, lap, s);
  return __fmul_rn(g, s);
}

// Imaging term A (lap - m2) u in the scheme's units: A lap u - M u.
__device__ __forceinline__ float img_term(float u, float A, float M, float lap, bool dens) {
  float t = __fmul_rn(A, lap);
  if (dens) t = __fmaf_rn(-M, u, t);
  return t;
}

template <int TX, int TY, bool ADJ, bool RECOMP>
struct Layout {
  static constexpr int NCT = (TX / 4) * TY;  // compute threads
  static constexpr int HS = (TX + 2 * kHalo) * (TY + 2 * kHalo);  // halo stage floats
  static constexpr int CS = TX * TY;  // centre tile floats
  // Halo ring depth: 5 planes in use plus 3 ahead (2 ahead when two halo'd
  // fields share each stage, to keep two CTAs per SM).
  static constexpr int NSU = (ADJ && RECOMP) ? 7 : 8;
  static constexpr int NSC = ADJ ? 4 : 3;  // centre ring depth
  static constexpr int NHALO = (ADJ && RECOMP) ? 2 : 1;  // halo'd fields per stage
};

// Per-plane metadata staged in shared memory: sponge factor gz and the
// receiver-entry range of the plane.
struct PlaneInfo {
  float gz;
  int rb, re, pad;
};

}  // namespace

// Kernel modes.
//   MODE_FWD        forward step
//   MODE_FWD_PH     forward step + pseudo-Hessian accumulation (acc += (g t)^2)
//   MODE_FWD_STORE  forward step + store of the imaging term t on the interior
//   MODE_FWD_STORE_PH  both of the above (all-terms gradient with pseudo-Hessian)
//   MODE_ADJ        adjoint step + imaging against a recomputed forward field
//   MODE_ADJ_STORED adjoint step + imaging against the stored imaging term
// Resident CTAs per SM the register budget is sized for: the adjoint with a
// recomputed forward field on large tiles needs more than 200 KB of shared
// memory per pair, so it runs one CTA per SM with the full register file.
template <int TX, int TY, int MODE>
struct MinBlocks {
  static constexpr int value = (MODE == MODE_ADJ && TX * TY >= 1024) ? 1 : 2;
};

template <int TX, int TY, bool DENS, int MODE>
__global__ void __launch_bounds__((TX / 4) * TY + 32, (MinBlocks<TX, TY, MODE>::value))
    step_kernel(const StepArgs a) {
  constexpr bool ADJ = (MODE == MODE_ADJ || MODE == MODE_ADJ_STORED || MODE == MODE_ADJ_TERM);
  constexpr bool RECOMP = (MODE == MODE_ADJ);
  constexpr bool ACC = (MODE == MODE_FWD_PH || MODE == MODE_FWD_STORE_PH || MODE == MODE_ADJ ||
                       MODE == MODE_ADJ_STORED);
  constexpr bool TERM = (MODE == MODE_ADJ_STORED);  // stored imaging term as a centre array
  using LY = Layout<TX, TY, ADJ, RECOMP>;
  constexpr int NCT = LY::NCT, HS = LY::HS, CS = LY::CS, NSU = LY::NSU, NSC = LY::NSC;
  constexpr int NHALO = LY::NHALO;
  constexpr int NC = 2 + (DENS ? 1 : 0) + (ACC ? 1 : 0) + (TERM ? 1 : 0);  // centre arrays
  constexpr int CI_PREV = 0, CI_A = 1, CI_M = 2, CI_ACC = DENS ? 3 : 2, CI_T = CI_ACC + 1;

  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* ring = reinterpret_cast<float*>(smem_raw);           // NSU * NHALO * HS
  float* cring = ring + NSU * NHALO * HS;                       // NSC * NC * CS
  float* otile = cring + NSC * NC * CS;                         // CS
  uint64_t* bars = reinterpret_cast<uint64_t*>(otile + CS);     // 2*NSU + 2*NSC
  uint64_t* fullF = bars;
  uint64_t* emptyF = bars + NSU;
  uint64_t* fullC = bars + 2 * NSU;
  uint64_t* emptyC = bars + 2 * NSU + NSC;
  PlaneInfo* pinfo = reinterpret_cast<PlaneInfo*>(bars + 2 * NSU + 2 * NSC);  // npl entries

  const WorkItem it = a.items[blockIdx.x];
  const VolDesc V = a.vols[it.vol];
  const ShotMaps* sm = a.maps + it.vol;
  const int x0 = it.x0, y0 = it.y0, zb = it.zb, ze = it.ze;
  const int npl = ze - zb;
  const int tid = threadIdx.x;

  for (int j = tid; j < npl; j += blockDim.x) {
    PlaneInfo pi;
    pi.gz = a.gz[zb + j];
    pi.rb = pi.re = 0;
    if (it.rec_tab >= 0) {
      pi.rb = a.rec_ptr[it.rec_tab + j];
      pi.re = a.rec_ptr[it.rec_tab + j + 1];
    }
    pi.pad = 0;
    pinfo[j] = pi;
  }
  if (tid == 0) {
    for (int s = 0; s < NSU; ++s) {
      mbar_init(&fullF[s], 1);
      mbar_init(&emptyF[s], NCT / 32);
    }
    for (int s = 0; s < NSC; ++s) {
      mbar_init(&fullC[s], 1);
      mbar_init(&emptyC[s], NCT / 32);
    }
    fence_barrier_init();
  }
  __syncthreads();

  // Maps of the buffers this launch reads (chosen by the host per step).
  const CUtensorMap* mapF = a.mF + (long long)it.vol * a.sF;
  const CUtensorMap* mapP = a.mP + (long long)it.vol * a.sP;
  const CUtensorMap* mapU = a.mU + (long long)it.vol * a.sU;  // forward field for imaging
  const CUtensorMap* mapAcc = &sm->m[ADJ ? 11 : 8];
  const CUtensorMap* mapT = &sm->m[12];
  const CUtensorMap* mapA = &a.cmaps->m[0];
  const CUtensorMap* mapM = &a.cmaps->m[1];

  if (tid >= NCT) {
    // ------------------------------------------------------------ producer
    if (tid == NCT) {
      tmap_acquire(mapF);
      tmap_acquire(mapP);
      tmap_acquire(mapA);
      if (DENS) tmap_acquire(mapM);
      if (RECOMP) tmap_acquire(mapU);
      if (ACC) tmap_acquire(mapAcc);
      if (TERM) tmap_acquire(mapT);
      const int nu = npl + 2 * kHalo;
      const int cx = V.cx0 + x0, cy = V.cy0 + y0;
      int nF = 0, nC = 0;  // loads issued into the halo and centre rings
      // After a wait runs out: let every load already issued land before the
      // CTA exits (bulk copies must not target the shared memory of a CTA
      // that has finished).  Stage s of a ring holds loads s, s + depth, ...;
      // the last one issued into it completes phase (count - 1).
      auto drain = [&]() {
        for (int s = 0; s < NSU && s < nF; ++s)
          mbar_wait(&fullF[s], (uint32_t)(((nF - 1 - s) / NSU) & 1), a.status);
        for (int c = 0; c < NSC && c < nC; ++c)
          mbar_wait(&fullC[c], (uint32_t)(((nC - 1 - c) / NSC) & 1), a.status);
      };
      for (int i = 0; i < nu; ++i) {
        const int s = i % NSU, r = i / NSU;
        if (r > 0 && !mbar_wait(&emptyF[s], (r & 1) ^ 1, a.status)) {
          drain();
          return;
        }
        // Above a free surface at plane zs the plane is the image of plane
        // 2 zs - p (the consumers negate it).
        const int p0 = zb - kHalo + i;
        const int p = (a.zs >= 0 && p0 < a.zs) ? 2 * a.zs - p0 : p0;
        mbar_arrive_expect_tx(&fullF[s], NHALO * HS * 4);
        float* dst = ring + s * NHALO * HS;
        tma_load_3d(dst, mapF, x0 - kHalo, y0 - kHalo, p, &fullF[s]);
        if (RECOMP) tma_load_3d(dst + HS, mapU, x0 - kHalo, y0 - kHalo, p, &fullF[s]);
        ++nF;
        if (i >= 2 * kHalo) {
          const int j = i - 2 * kHalo, q = zb + j;
          const int c = j % NSC, rc = j / NSC;
          if (rc > 0 && !mbar_wait(&emptyC[c], (rc & 1) ^ 1, a.status)) {
            drain();
            return;
          }
          mbar_arrive_expect_tx(&fullC[c], NC * CS * 4);
          float* cd = cring + c * NC * CS;
          tma_load_3d(cd + CI_PREV * CS, mapP, x0, y0, q, &fullC[c]);
          tma_load_3d(cd + CI_A * CS, mapA, cx, cy, q, &fullC[c]);
          if (DENS) tma_load_3d(cd + CI_M * CS, mapM, cx, cy, q, &fullC[c]);
          if (ACC) tma_load_3d(cd + CI_ACC * CS, mapAcc, x0, y0, q, &fullC[c]);
          if (TERM)
            tma_load_4d(cd + CI_T * CS, mapT, x0 - V.txoff, y0 - V.iy0, q - V.border, a.tstep,
                        &fullC[c]);
          ++nC;
        }
      }
    }
    return;
  }

  // -------------------------------------------------------------- consumers
  constexpr int RP = TX + 2 * kHalo;
  const int lx = (tid % (TX / 4)) * 4, ly = tid / (TX / 4);
  const int gxl = x0 + lx, gyl = y0 + ly;  // local padded coordinates of point 0
  const int lane = tid & 31;
  const bool row_ok = ly < it.h && gyl < V.Ny;
  const bool col_ok = lx < it.w && gxl < V.Nx;  // tile widths are multiples of 4
  float gxv[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) gxv[e] = (gxl + e < V.Nx) ? a.gx[V.gx_off + gxl + e] : 0.0f;
  const float gyv = row_ok ? a.gy[V.gy_off + gyl] : 0.0f;
  const int my_off = (ly + kHalo) * RP + lx + kHalo;  // centre of my row in a halo stage

  // A wait that runs out marks the CTA dead: it records the timeout and then
  // runs to completion without waiting, so every named barrier is reached.
  bool dead = false;
  auto wait = [&](uint64_t* bar, uint32_t parity) {
    if (!dead && !mbar_wait(bar, parity, a.status)) dead = true;
  };
  F4 q[9], qu[9];
  // z column entry of plane p from its ring stage (negated above a free
  // surface, where the stage holds the image plane).
  auto zload = [&](const float* st, int p) {
    F4 v = ld4s(st);
    if (a.zs >= 0 && p < a.zs) {
#pragma unroll
      for (int e = 0; e < 4; ++e) v.v[e] = -v.v[e];
    }
    return v;
  };
  // Priming: planes zb-4 .. zb+3 fill queue slots 0..7.
  for (int i = 0; i < 2 * kHalo; ++i) {
    const int s = i % NSU;
    wait(&fullF[s], (i / NSU) & 1);
    q[i] = zload(ring + s * NHALO * HS + my_off, zb - kHalo + i);
    if (RECOMP) qu[i] = zload(ring + s * NHALO * HS + HS + my_off, zb - kHalo + i);
    if (i < kHalo || zb - kHalo + i >= ze) {
      __syncwarp();
      if (lane == 0) mbar_arrive(&emptyF[s]);
    }
  }

  for (int j = 0; j < npl; ++j) {
    const int z = zb + j;
    {  // queue slot 8 <- plane z + 4
      const int i = j + 2 * kHalo, s = i % NSU;
      wait(&fullF[s], (i / NSU) & 1);
      q[8] = zload(ring + s * NHALO * HS + my_off, z + kHalo);
      if (RECOMP) qu[8] = zload(ring + s * NHALO * HS + HS + my_off, z + kHalo);
      if (z + kHalo >= ze) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&emptyF[s]);
      }
    }
    const int c = j % NSC;
    wait(&fullC[c], (j / NSC) & 1);
    const int su = (j + kHalo) % NSU;
    const float* st = ring + su * NHALO * HS;
    const float* cs = cring + c * NC * CS + ly * TX + lx;

    float lap[4];
    lap4<TX>(st, lx, ly, q, lap);
    const F4 prev = ld4s(cs + CI_PREV * CS);
    const F4 Av = ld4s(cs + CI_A * CS);
    F4 Mv = {{0.f, 0.f, 0.f, 0.f}};
    if (DENS) Mv = ld4s(cs + CI_M * CS);
    const PlaneInfo pi = pinfo[j];
    const float gyz = __fmul_rn(gyv, pi.gz);
    F4 out;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float g = __fmul_rn(gxv[e], gyz);
      out.v[e] = update(q[4].v[e], prev.v[e], Av.v[e], Mv.v[e], g, lap[e], DENS);
    }
    // Source injection (forward only): u^{n+1} += w_e dt^2 w[n] / (h^3 sqrt rho_e)
    // at the corners e of the source cell (one corner for the nearest node).
    if (!ADJ) {
      const int dz = z - V.src_z, dy = gyl - V.src_y;
      if ((unsigned)dz < 2u && (unsigned)dy < 2u) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int dx = gxl + e - V.src_x;
          if ((unsigned)dx < 2u) {
            const float sc = a.vols[it.vol].src_sc[dx + 2 * dy + 4 * dz];  // global: dynamic index
            if (sc != 0.0f) out.v[e] = __fmaf_rn(sc, a.wn, out.v[e]);
          }
        }
      }
    }
    // Receivers of this tile on this plane.
    {
      const int rb = pi.rb, re = pi.re;
      if (rb < re) {
        *reinterpret_cast<float4*>(otile + ly * TX + lx) =
            make_float4(out.v[0], out.v[1], out.v[2], out.v[3]);
        compute_sync(NCT);
        if (!ADJ) {
          if (a.dout)
            for (int e = rb + tid; e < re; e += NCT) {
              const RecEntry r = a.rec[e];
              a.dout[r.col] = r.fscale * otile[r.lxy];
            }
        } else {
          for (int e = rb + tid; e < re; e += NCT) {
            const RecEntry r = a.rec[e];
            if (r.group > 0) {
              float add = 0.0f;
              for (int k = 0; k < r.group; ++k) {
                const RecEntry rk = a.rec[e + k];
                add = __fmaf_rn(rk.ascale, a.rin[rk.col], add);
              }
              otile[r.lxy] += add;
            }
          }
        }
        compute_sync(NCT);
        if (ADJ) out = ld4s(otile + ly * TX + lx);
      }
    }
    // Interior store of the new adjoint level.
    if (MODE == MODE_ADJ_TERM) {
      const int zi = z - V.border, yi = gyl - V.iy0;
      if (row_ok && col_ok && yi >= 0 && yi < V.nyi && zi >= 0 && zi < V.nzi) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int xi = gxl + e - V.ix0;
          if (xi >= 0 && xi < V.nxi)
            a.tstore[V.toff + ((long long)zi * V.nyi + yi) * V.tpitch + (gxl + e - V.txoff)] =
                out.v[e];
        }
      }
    }
    // Imaging / accumulation.
    if (MODE == MODE_FWD_PH || MODE == MODE_FWD_STORE || MODE == MODE_FWD_STORE_PH ||
        MODE == MODE_ADJ || MODE == MODE_ADJ_STORED) {
      F4 t;
      if (MODE == MODE_ADJ) {
        float lu[4];
        lap4<TX>(st + HS, lx, ly, qu, lu);
#pragma unroll
        for (int e = 0; e < 4; ++e) t.v[e] = img_term(qu[4].v[e], Av.v[e], Mv.v[e], lu[e], DENS);
      } else if (MODE == MODE_ADJ_STORED) {
        t = ld4s(cs + CI_T * CS);
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) t.v[e] = img_term(q[4].v[e], Av.v[e], Mv.v[e], lap[e], DENS);
      }
      if (MODE == MODE_FWD_STORE || MODE == MODE_FWD_STORE_PH) {
        const int zi = z - V.border, yi = gyl - V.iy0;
        if (row_ok && col_ok && yi >= 0 && yi < V.nyi && zi >= 0 && zi < V.nzi) {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int xi = gxl + e - V.ix0;
            if (xi >= 0 && xi < V.nxi)
              a.tstore[V.toff + ((long long)zi * V.nyi + yi) * V.tpitch + (gxl + e - V.txoff)] =
                  t.v[e];
          }
        }
      }
      if (ACC) {
        const F4 acc = ld4s(cs + CI_ACC * CS);
        F4 nacc;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          if (ADJ) {
            nacc.v[e] = __fmaf_rn(out.v[e], t.v[e], acc.v[e]);
          } else {
            const float g = __fmul_rn(gxv[e], gyz);
            const float gt = __fmul_rn(g, t.v[e]);
            nacc.v[e] = __fmaf_rn(gt, gt, acc.v[e]);
          }
        }
        // (whole window; the gradient and pseudo-Hessian read its imaging region)
        if (row_ok && col_ok) {
          float* ap = a.acc + V.off + ((long long)z * V.Ny + gyl) * V.pitch + gxl;
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (gxl + e >= V.Nx) nacc.v[e] = 0.0f;
          st4g(ap, nacc);
        }
      }
    }
    // Store the new level over the previous one.
    if (row_ok && col_ok) {
      float* op = a.fout + V.off + ((long long)z * V.Ny + gyl) * V.pitch + gxl;
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (gxl + e >= V.Nx) out.v[e] = 0.0f;
      st4g(op, out);
    }
    // Release this plane's stages.
    __syncwarp();
    if (lane == 0) {
      mbar_arrive(&emptyF[su]);
      mbar_arrive(&emptyC[c]);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      q[k] = q[k + 1];
      if (RECOMP) qu[k] = qu[k + 1];
    }
  }
}

template <int TX, int TY, bool DENS, int MODE>
static size_t smem_bytes_base() {
  constexpr bool ADJ = (MODE == MODE_ADJ || MODE == MODE_ADJ_STORED || MODE == MODE_ADJ_TERM);
  constexpr bool RECOMP = (MODE == MODE_ADJ);
  constexpr bool ACC = (MODE == MODE_FWD_PH || MODE == MODE_FWD_STORE_PH || MODE == MODE_ADJ ||
                       MODE == MODE_ADJ_STORED);
  using LY = Layout<TX, TY, ADJ, RECOMP>;
  constexpr int NC = 2 + (DENS ? 1 : 0) + (ACC ? 1 : 0) + (MODE == MODE_ADJ_STORED ? 1 : 0);
  return sizeof(float) * (size_t)(LY::NSU * LY::NHALO * LY::HS + LY::NSC * NC * LY::CS + LY::CS) +
         sizeof(uint64_t) * (2 * LY::NSU + 2 * LY::NSC);
}

// Dynamic shared memory of one launch: rings, output tile, barriers and the
// per-plane table for up to max_planes planes per item.
template <int TX, int TY, bool DENS, int MODE>
static size_t smem_bytes(int max_planes) {
  return smem_bytes_base<TX, TY, DENS, MODE>() + sizeof(PlaneInfo) * (size_t)max_planes;
}

template <int TX, int TY, bool DENS, int MODE>
static cudaError_t launch_one(const StepArgs& a, int n_items, int max_planes, cudaStream_t s,
                              int* occupancy) {
  const size_t sm = smem_bytes<TX, TY, DENS, MODE>(max_planes);
  static size_t attr_bytes = 0;
  if (sm > attr_bytes) {
    cudaError_t e = cudaFuncSetAttribute(step_kernel<TX, TY, DENS, MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    attr_bytes = sm;
  }
  if (occupancy) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occupancy, step_kernel<TX, TY, DENS, MODE>,
                                                         (TX / 4) * TY + 32, sm);
  }
  step_kernel<TX, TY, DENS, MODE><<<n_items, (TX / 4) * TY + 32, sm, s>>>(a);
  return cudaGetLastError();
}

template <int TX, int TY, int MODE>
static cudaError_t launch_mode(const StepArgs& a, int n_items, int max_planes, bool dens,
                               cudaStream_t s, int* occ) {
  return dens ? launch_one<TX, TY, true, MODE>(a, n_items, max_planes, s, occ)
              : launch_one<TX, TY, false, MODE>(a, n_items, max_planes, s, occ);
}

// Compiled tile shapes (TX, TY).
#define MAMUTE_TILES(X) X(64, 16) X(64, 8) X(32, 16) X(32, 8) X(128, 8) X(72, 16) X(96, 8) X(48, 16)

cudaError_t dispatch_forward(const StepArgs& a, int n_items, int max_planes, int tx, int ty,
                             bool dens, int mode, cudaStream_t s, int* occ);
cudaError_t dispatch_adjoint(const StepArgs& a, int n_items, int max_planes, int tx, int ty,
                             bool dens, int mode, cudaStream_t s, int* occ);

}  // namespace mamute
