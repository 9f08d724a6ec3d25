// 3x3x3 convolution (forward and input gradient) on the 5th-generation
// tensor cores: tcgen05.mma with the accumulators in tensor memory, operands
// staged in shared memory by TMA.  Included by conv.cu inside its anonymous
// namespace (shares bf2f / f2bf and the constants there).
//
// Formulation.  A CTA owns a block of RY output rows (y) of an x segment of
// SW voxels and marches over a chunk of z planes.  Each halo plane of the
// block (rows y0-1 .., x from xs-1, width P = SW + 2 <= 64) arrives by one
// TMA load of long rows (the activation viewed as 8-byte elements, one box
// row per halo row, no swizzle): 32 bytes (16 channels) per voxel.  Two
// warps then swap the two 16-byte channel halves of every voxel whose
// shared-memory address has bit 7 set, in place, which gives the K-major
// SWIZZLE_32B operand layout of tcgen05 (one 32-byte row per M row, 8-row
// groups 256 bytes apart, the swizzle taken on absolute shared-memory
// addresses).  (A TMA load with the 32-byte swizzle itself is limited to
// 32-byte box rows, which move a few bytes per clock per SM.)  Output voxels are numbered f = ry * P + xx over the
// block (xx in [0, P): the last two columns of every row are junk and never
// stored), so the A rows of tap (dz, dy, dx) for the 128 outputs
// f0 .. f0+127 are the 128 consecutive halo voxels starting at
// f0 + dy P + dx of halo plane z + dz: one descriptor per tap and chunk, no
// data movement.
//
// Plane stacking.  Halo plane h feeds output planes h + 1, h and h - 1
// through the kernel's dz = 0, 1, 2 taps with the same A operand, so each
// halo plane is consumed once: per chunk, 9 (dy, dx) products of
// tcgen05.mma.kind::f16 M=128 N=64 K=16 (bf16 in, f32 accumulate) whose 64
// columns are the chunk's 4 accumulator slots of 16 output channels.  Plane
// p lives in slot p mod 4; at step h the slots hold planes h + 1 (first
// contribution: zeroed just before by an N=16 product with a zero B), h,
// h - 1 (last contribution) and h - 2 (complete, read by the epilogue
// meanwhile: its B columns are zero, so the products rewrite its values
// unchanged).  The B operand is the window of 4 blocks at offset (1 - h)
// mod 4 of the block sequence [dz2, dz1, dz0, 0, dz2, dz1, dz0] of the
// (dy, dx) tap's weights.  The epilogue warps read one voxel's 16 output
// channels per thread with tcgen05.ld and store 32 (bf16) or 64 (f32)
// contiguous bytes.
//
// Warp roles (384 threads): warp 0 lane 0 issues the TMA loads of halo
// planes into a ring of slots; warp 1 allocates TMEM and lane 0 issues
// the MMAs; warps 2-9 run the epilogue, two per TMEM lane quarter (warp w
// reads lanes 32 (w mod 4) ..), each taking every other chunk; warps 10-11
// swizzle each loaded halo plane.  Every wait is bounded; a timeout sets
// the status flag and a CTA-wide abort flag that ends every role's loop.

constexpr int kTcMaxRing = 6;        // halo plane slots (at most)
constexpr int kTcCols = 512;         // TMEM columns: 8 chunks x 4 plane slots x 16
constexpr int kTcMaxChunks = 8;
constexpr int kTcMaxP = 64;          // halo row width (x segment + 2): one TMA box row
constexpr int kTcEpiWarps = 8;
constexpr int kTcSwzWarps = 2;
constexpr int kTcThreads = 32 * (2 + kTcEpiWarps + kTcSwzWarps);
// B operand: per (dy, dx) tap, 7 blocks x 16 output channels (N rows) x 16
// input channels (K), K-major core matrices: 8-row groups 128 bytes apart,
// the two 8-channel K halves kTcWHalf bytes apart.
constexpr int kTcWBlocks = 7;
constexpr int kTcWHalf = kTcWBlocks * 16 * 16;   // bytes
constexpr int kTcWTap = 2 * kTcWHalf;            // bytes per (dy, dx) tap
constexpr int kTcWBytes = 9 * kTcWTap;

struct TcPlan {
  int P, SW, RY, NCH, rows, ZC, ring;
  int nxs, nyb, nzc;
  long long items;
  int slot_bytes;  // shared memory of one halo plane (multiple of 1024)
};

// Instruction descriptor, kind::f16: D f32 (bits 4-5 = 1), A and B bf16
// (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at
// bits 24-28.
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) |
                              ((128u >> 4) << 24);
constexpr uint32_t kTcIdesc64 = (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) |
                                ((128u >> 4) << 24);

__global__ void __launch_bounds__(kTcThreads, 1)
    conv_tc_kernel(const __grid_constant__ CUtensorMap xmap, ConvArgs a, TcPlan pl, int* status) {
  extern __shared__ unsigned char tc_raw[];
  // the 32-byte swizzle acts on address bits 4 and 7: slots on 1024 bytes
  unsigned char* sm = tc_raw + ((1024 - (smem_u32(tc_raw) & 1023)) & 1023);
  unsigned char* slots = sm;                               // ring x slot_bytes
  unsigned char* wts = sm + pl.ring * pl.slot_bytes;       // kTcWBytes, see kTcWBlocks
  __shared__ uint64_t full[kTcMaxRing], ready[kTcMaxRing], empty[kTcMaxRing], tfull[4], tempty[4],
      done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  volatile int* ab = &abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // B blocks: block j of tap (dy, dx) holds w[dz][dy][dx][o][i] for the dz of
  // the sequence [2, 1, 0, -, 2, 1, 0] (block 3 zero).  Each 16-byte piece
  // (8 input channels of one output channel) goes to the two blocks of its
  // dz; the global loads are issued together before the stores.
  {
    constexpr int kPieces = kTaps * kC * 2;  // 864 pieces of 8 bf16
    constexpr int kPer = (kPieces + kTcThreads - 1) / kTcThreads;
    const uint4* wg = reinterpret_cast<const uint4*>(a.w);
    uint4 pc[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int e = threadIdx.x + k * kTcThreads;
      if (e < kPieces) pc[k] = wg[e];
    }
    uint4* ws = reinterpret_cast<uint4*>(wts);
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int e = threadIdx.x + k * kTcThreads;
      if (e >= kPieces) continue;
      const int tap = e / (kC * 2), o = (e / 2) % kC, ih = e % 2;
      const int dz = tap / 9, t9 = tap % 9;
      const int j0 = 2 - dz;  // blocks j0 and j0 + 4
#pragma unroll
      for (int r = 0; r < 2; ++r)
        ws[(t9 * kTcWTap + ih * kTcWHalf) / 16 + (j0 + 4 * r) * 16 + o] = pc[k];
    }
    for (int e = threadIdx.x; e < 9 * 2 * 16; e += kTcThreads) {  // block 3: zeros
      const int t9 = e / 32, ih = (e / 16) % 2, o = e % 16;
      ws[(t9 * kTcWTap + ih * kTcWHalf) / 16 + 3 * 16 + o] = make_uint4(0u, 0u, 0u, 0u);
    }
  }
  fence_async_smem();  // visible to the tensor cores (async proxy)
  if (threadIdx.x == 0) {
    for (int i = 0; i < kTcMaxRing; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&ready[i], kTcSwzWarps);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 4; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], kTcEpiWarps);
    }
    mbar_init(&done_bar, 1);
    fence_barrier_init();
    abort_flag = 0;
  }
  if (warp == 1) {
    tc_alloc(&tmem_base, kTcCols);
    tc_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  auto geom = [&](long long it, int& xs, int& y0, int& z0, int& nz) {
    xs = (int)(it % pl.nxs) * pl.SW;
    y0 = (int)((it / pl.nxs) % pl.nyb) * pl.RY;
    z0 = (int)(it / ((long long)pl.nxs * pl.nyb)) * pl.ZC;
    nz = min(pl.ZC, a.D - z0);
  };

  if (warp == 0) {
    // ---- producer: halo planes z0 - 1 .. z0 + nz of each item, in order
    if (lane == 0) {
      const uint32_t tx = 32u * (uint32_t)pl.P * (uint32_t)pl.rows;
      uint32_t q = 0;
      for (long long it = blockIdx.x; it < pl.items && !*ab; it += gridDim.x) {
        int xs, y0, z0, nz;
        geom(it, xs, y0, z0, nz);
        for (int h = 0; h < nz + 2; ++h, ++q) {
          const int s = (int)(q % pl.ring);
          if (!tc_wait(&empty[s], ((q / pl.ring) & 1) ^ 1, status, ab)) break;
          unsigned char* dst = slots + (size_t)s * pl.slot_bytes;
          mbar_arrive_expect_tx(&full[s], tx);
          tma_load_3d(dst, &xmap, 4 * (xs - 1), y0 - 1, z0 - 1 + h, &full[s]);
        }
      }
      if (*ab)  // let issued loads land before the CTA exits
        for (uint32_t k = 0; k < (uint32_t)pl.ring && k < q; ++k) {
          const uint32_t qq = q - 1 - k;
          mbar_wait(&full[qq % pl.ring], (qq / pl.ring) & 1, status);
        }
    }
  } else if (warp == 1) {
    // ---- MMA issuer: one step per halo plane (global step counter t)
    if (lane == 0) {
      const uint32_t wbase = smem_u32(wts), sbase = smem_u32(slots);
      const uint64_t bw = tc_sdesc(wbase, (uint32_t)kTcWHalf, 128u);
      const uint64_t bzero = bw + 3ull * 16u;  // block 3 (zeros), N = 16
      const uint64_t rowoff[3] = {0ull, 2ull * (uint64_t)pl.P, 4ull * (uint64_t)pl.P};
      uint32_t t = 0;
      bool ok = true;
      for (long long it = blockIdx.x; it < pl.items && ok && !*ab; it += gridDim.x) {
        int xs, y0, z0, nz;
        geom(it, xs, y0, z0, nz);
        for (int k = 0; k < nz + 2; ++k, ++t) {
          const uint32_t hs = t % (uint32_t)pl.ring;
          if (!(ok = tc_wait(&ready[hs], (t / pl.ring) & 1, status, ab))) break;
          const uint32_t sn = (t + 1) & 3;  // slot of plane h + 1
          if (t >= 2 && !(ok = tc_wait(&tempty[sn], ((t - 2) >> 2) & 1, status, ab))) break;
          tc_fence_after();
          // start-address field (address >> 4) advanced by chunk * 128 +
          // dy * P + dx voxels of 32 bytes (2 units each)
          const uint64_t a0 = tc_sdesc(sbase + hs * (uint32_t)pl.slot_bytes, 16u, 256u, 6u);
          const uint64_t bwin = bw + (uint64_t)(((1u - t) & 3u) * 16u);
          for (int c = 0; c < pl.NCH; ++c) {
            const uint32_t d = tmem + (uint32_t)(c * 64);
            const uint64_t ac = a0 + (uint64_t)c * 256u;
            tc_mma(d + sn * 16u, ac, bzero, kTcIdesc, 0u);
#pragma unroll
            for (int t9 = 0; t9 < 9; ++t9) {
              const int dy = t9 / 3, dx = t9 % 3;
              tc_mma(d, ac + rowoff[dy] + 2ull * (uint64_t)dx,
                     bwin + (uint64_t)t9 * (uint64_t)(kTcWTap >> 4), kTcIdesc64, 1u);
            }
          }
          tc_commit(&empty[hs]);
          tc_commit(&tfull[(t + 3) & 3]);  // plane h - 1 complete
        }
      }
      tc_commit(&done_bar);  // every MMA issued above has completed
      mbar_wait(&done_bar, 0, status);
    }
  } else if (warp >= 2 + kTcEpiWarps) {
    // ---- swizzle: swap the channel halves of the voxels at addresses with
    // bit 7 set (voxels 4..7 of every 8 from the 1024-byte-aligned slot)
    const int sid = threadIdx.x - 32 * (2 + kTcEpiWarps);
    const int nvox = pl.rows * pl.P;
    uint32_t q = 0;
    bool ok = true;
    for (long long it = blockIdx.x; it < pl.items && ok && !*ab; it += gridDim.x) {
      int xs, y0, z0, nz;
      geom(it, xs, y0, z0, nz);
      for (int h = 0; h < nz + 2; ++h, ++q) {
        const int s = (int)(q % pl.ring);
        int got = 0;
        if (lane == 0) got = tc_wait(&full[s], (q / pl.ring) & 1, status, ab) ? 1 : 0;
        if (!(ok = __shfl_sync(0xffffffffu, got, 0) != 0)) break;
        uint4* vox = reinterpret_cast<uint4*>(slots + (size_t)s * pl.slot_bytes);
        for (int j = sid; j < (nvox + 1) / 2; j += 32 * kTcSwzWarps) {
          const int v = (j >> 2) * 8 + 4 + (j & 3);
          if (v < nvox) {
            const uint4 lo = vox[2 * v], hi = vox[2 * v + 1];
            vox[2 * v] = hi;
            vox[2 * v + 1] = lo;
          }
        }
        fence_async_smem();  // visible to the tensor cores (async proxy)
        __syncwarp();
        if (lane == 0) mbar_arrive(&ready[s]);
      }
    }
  } else {
    // ---- epilogue: one output voxel (16 channels) per thread and chunk
    const int quarter = warp & 3, half = (warp - 2) >> 2;
    const int row = quarter * 32 + lane;
    // block row and column of this thread's voxel in each of its chunks
    int rdiv[4], rmod[4];
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const int f = (half + 2 * cc) * 128 + row;
      rdiv[cc] = f / pl.P;
      rmod[cc] = f % pl.P;
    }
    float bias[kC];
#pragma unroll
    for (int o = 0; o < kC; ++o) bias[o] = a.bias ? a.bias[o] : 0.f;
    // Lane 0 waits and reads the abort flag for the warp, so the break and
    // the tcgen05.ld that follows (a .sync.aligned warp instruction) are
    // taken by the whole warp together.
    auto warp_stop = [&]() { return __shfl_sync(0xffffffffu, lane == 0 ? (int)(*ab != 0) : 0, 0) != 0; };
    uint32_t t = 0;
    bool ok = true;
    for (long long it = blockIdx.x; it < pl.items && ok && !warp_stop(); it += gridDim.x) {
      int xs, y0, z0, nz;
      geom(it, xs, y0, z0, nz);
      for (int k = 0; k < nz + 2; ++k, ++t) {
        const uint32_t sd = (t + 3) & 3;  // slot of plane h - 1
        int got = 0;
        if (lane == 0) got = tc_wait(&tfull[sd], (t >> 2) & 1, status, ab) ? 1 : 0;
        if (!(ok = __shfl_sync(0xffffffffu, got, 0) != 0)) break;
        tc_fence_after();
        if (k >= 2) {
          const int z = z0 + k - 2;
          for (int c0 = half; c0 < pl.NCH; c0 += 8) {  // up to 4 chunks per TMEM wait
            uint32_t r[64];
#pragma unroll
            for (int cc = 0; cc < 4; ++cc)
              if (c0 + 2 * cc < pl.NCH)
                tc_ld16(tmem + ((uint32_t)(quarter * 32) << 16) +
                            (uint32_t)((c0 + 2 * cc) * 64) + sd * 16u,
                        r + 16 * cc);
            tc_wait_ld();
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
              const int ry = rdiv[cc], xx = rmod[cc];
              const int y = y0 + ry, x = xs + xx;
              if (c0 + 2 * cc >= pl.NCH || ry >= pl.RY || xx >= pl.SW || y >= a.H || x >= a.W)
                continue;
              const long long vox = ((long long)z * a.H + y) * a.W + x;
              float v[kC];
#pragma unroll
              for (int o = 0; o < kC; ++o) {
                v[o] = __uint_as_float(r[cc * 16 + o]) + bias[o];
                if (a.relu) v[o] = fmaxf(v[o], 0.f);
              }
              if (a.mask) {
                const uint4* mp = reinterpret_cast<const uint4*>(a.mask + vox * kC);
                const uint4 m0 = mp[0], m1 = mp[1];
                const uint32_t mw[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
                for (int o = 0; o < kC; ++o) {
                  const uint16_t mb = (uint16_t)(mw[o >> 1] >> (16 * (o & 1)));
                  if (!(bf2f(mb) > 0.f)) v[o] = 0.f;
                }
              }
              if (a.y32) {
                float4* yp = reinterpret_cast<float4*>(a.y32 + vox * kC);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                  yp[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
              }
              if (a.y16) {  // round to nearest even, two values per conversion
                uint32_t pk[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                  const __nv_bfloat162 b2 = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
                  pk[q] = *reinterpret_cast<const uint32_t*>(&b2);
                }
                uint4* yp = reinterpret_cast<uint4*>(a.y16 + vox * kC);
                yp[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                yp[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
              }
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[sd]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tc_dealloc(tmem, kTcCols);
  }
}
