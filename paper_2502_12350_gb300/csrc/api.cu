// C ABI of libmamute: context, validation, planning and the modelling /
// gradient drivers (Algorithm 1 and Algorithm 3 of the paper).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mamute.h"
#include "aux.h"
#include "conv.h"
#include "gn.h"
#include "common.cuh"
#include "cpml.h"
#include "postproc.h"
#include "revolve.h"
#include "stencil.h"

using namespace mamute;

namespace {

// Stability bound of the 3-D eighth-order leapfrog scheme:
// (c dt / h)^2 * 3 * max_theta(-c0 - 2 sum c_j cos j theta) <= 4.
double cfl_bound() {
  const double c[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};
  double mx = 0.0;
  for (int i = 0; i <= 100000; ++i) {
    const double th = M_PI * i / 100000.0;
    double s = -c[0];
    for (int j = 1; j <= 4; ++j) s -= 2.0 * c[j] * std::cos(j * th);
    mx = std::max(mx, s);
  }
  return 2.0 / std::sqrt(3.0 * mx);
}

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

// A receiver's node with non-zero weight (nearest node: one per receiver;
// trilinear: up to 8), in the shot window's local padded coordinates.
struct NodeEntry {
  int lx, ly, lz;
  long long cell;  // model cell of the node
  int r;           // receiver
  int shot;
  float w;         // interpolation weight
};

struct Plan {
  int nx, ny, nz, b, Nx, Ny, Nz, pitchG, nt;
  double h, dt;
  bool dens;
  int tx, ty;             // forward tile
  int atx, aty;           // adjoint tile
  std::vector<VolDesc> vols;
  std::vector<WorkItem> items, aitems;
  std::vector<int> rec_ptr, arec_ptr;
  std::vector<RecEntry> rec, arec;
  std::vector<long long> rec_cell, arec_cell;
  std::vector<float> rec_g, arec_g;
  std::vector<int> colmap, acolmap;
  // receiver -> its internal columns (forward tiling), ascending; identity
  // when every receiver is one node
  std::vector<int> rcol_ptr, rcols;
  bool one_node = true;
  std::vector<long long> src_cell;  // 8 per shot (-1: corner not used)
  std::vector<float> src_w;         // 8 per shot
  int zs = -1;                      // padded plane of the free surface
  std::vector<float> gx, gy, gz;
  long long pool_elems = 0, term_elems = 0;
  int ncol = 0;   // internal data columns (receiver nodes)
  int nrec = 0;   // receivers
  std::vector<NodeEntry> ent;      // receiver nodes (input of the receiver tables)
  std::vector<int> fwd_col_of_ent; // forward-table column of each receiver node
  // two-level (temporal blocking) forward launches
  bool pairs = false;
  int ptx = 0, pty = 0;
  std::vector<WorkItem> pitems;
  std::vector<int4> pnbr;
  std::vector<int> prec_ptr;
  std::vector<RecEntry> prec;
  std::vector<long long> prec_cell;
  std::vector<float> prec_g;
  // convolutional PML instead of the sponge
  bool pml = false;
  double pml_f0 = 0.0, pml_r = 1e-3;
  float vmax = 0.f;  // max(vel), set by check_cfl
};

}  // namespace

struct mamute_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  // scratch (grow-only)
  DevBuf coefA, coefM, srho, pool[2], psi[2], acc, slots, tstore, dint, rint, dtmp, partial, misfit;
  DevBuf ident, rcolptr, rcols, ecol, srcw;  // receiver-node combination (trilinear)
  DevBuf smA, smMat, smLam;                  // gradient smoothing scratch
  std::vector<double> smKey, rsKey;          // what smMat / smLam and rsPtr / rsCol / rsW hold
  DevBuf pitems, pnbr, precptr, prec, pcells, pgvals, pmaps, pflags;  // two-level launches
  bool pair_graph_failed = false;  // cooperative launches could not be captured
  DevBuf rsPtr, rsCol, rsW, dmod, ddat;      // time resampling: band matrix (c0, len, weights), model- and data-axis traces
  DevBuf cpml, cprof, cnode, crec, ccell, cgval;  // convolutional PML
  DevBuf items, vols, maps, cmaps, recptr, rec, colmap, gx, gy, gz, cells, gvals, srccell,
      aitems, arecptr, arec, acolmap, acells, agvals;
  DevBuf hvel, hrho, hseis, hobs, hgrad, hphess;  // staging for the *_host calls
  DevBuf gnV, gnRe, gnIm, gnS, gnR, gnW, gnBins, gnWts, gnRow;  // GN-diagonal scratch
  DevBuf nnPartial, nnLoss;  // network scratch
  DevBuf slotmaps;           // tensor maps of the checkpoint slots
  int* status = nullptr;
  unsigned int* maxbits = nullptr;
  // timing hook
  bool timing = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool ev0_set = false;
  double loop_ms = 0.0;
  long long step_launches = 0, launches = 0;
  // event pairs around the DFT launches of mamute_gn_diagonal
  std::vector<cudaEvent_t> dft_ev;
  int dft_n = 0;
  double dft_ms = 0.0, dft_macs = 0.0;
  int max_planes = 1;  // planes per work item of the current call
  // captured time loop of the last mamute_model call and its signature
  cudaGraphExec_t graph = nullptr;
  std::vector<unsigned long long> graph_key;
  cudaStream_t capture = nullptr;  // private stream the time loop is captured on
  cudaStream_t copy = nullptr;     // seismogram transposes and copies to the host
  std::vector<cudaEvent_t> seg_ev;  // ends of the time-loop segments
  std::vector<ShotMaps> hmaps;     // host copy of the uploaded shot maps
};

namespace {

int fail(mamute_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return code;
}

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? MAMUTE_ENOMEM : MAMUTE_ECUDA, \
                  "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

cudaError_t ensure(DevBuf& b, size_t bytes) {
  if (bytes <= b.bytes && b.p) return cudaSuccess;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  if (bytes == 0) bytes = 256;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e == cudaSuccess) b.bytes = bytes;
  return e;
}

void release(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

template <typename T>
cudaError_t upload(DevBuf& b, const std::vector<T>& v, cudaStream_t s) {
  cudaError_t e = ensure(b, sizeof(T) * std::max<size_t>(v.size(), 1));
  if (e != cudaSuccess || v.empty()) return e;
  e = cudaMemcpyAsync(b.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);  // host vectors are released after the call
}

// Cerjan profile of one padded axis; with a free surface at plane zs (z axis
// only) the low face is not damped and the factor is 0 on and above it.
std::vector<float> sponge(int N, int b, double alpha, int zs = -1) {
  std::vector<float> p(N);
  for (int i = 0; i < N; ++i) {
    int d = 0;
    if (i < b && zs < 0) d = b - i;
    else if (i > N - 1 - b) d = i - (N - 1 - b);
    const double a = alpha * d;
    p[i] = (zs >= 0 && i <= zs) ? 0.0f : (float)std::exp(-a * a);
  }
  return p;
}

int env_int(const char* name, int dflt) {
  const char* v = getenv(name);
  return v ? atoi(v) : dflt;
}

// Tiling of one shot window: column starts (multiples of 4) and row starts.
struct Tiling {
  std::vector<int> xs, ys;  // boundaries, size ncols+1 / nrows+1
};

// Splits n into k pieces, each a multiple of `q` except possibly the last,
// as equal as possible.
std::vector<int> split(int n, int k, int q) {
  std::vector<int> b(1, 0);
  for (int i = 1; i < k; ++i) {
    long long e = (long long)n * i / k;
    e = (e + q / 2) / q * q;
    if (e <= b.back()) e = b.back() + q;
    if (e >= n) break;
    b.push_back((int)e);
  }
  b.push_back(n);
  return b;
}

int max_piece(const std::vector<int>& b) {
  int m = 0;
  for (size_t i = 1; i < b.size(); ++i) m = std::max(m, b[i] - b[i - 1]);
  return m;
}



// Receiver tables for one tiling (items ordered z block, row, column).
void build_receivers(Plan& P, int TX, int zsplit, const std::vector<NodeEntry>& ent,
                     const std::vector<int>& item_base, const std::vector<Tiling>& tilings,
                     std::vector<WorkItem>& items, std::vector<int>& rec_ptr,
                     std::vector<RecEntry>& rec, std::vector<long long>& cells,
                     std::vector<float>& gvals, std::vector<int>& colmap,
                     std::vector<int>* ent_of_col = nullptr) {
  struct Tmp {
    int item, z, lxy, r;
  };
  std::vector<Tmp> t;
  t.reserve(ent.size());
  for (int r = 0; r < (int)ent.size(); ++r) {
    const int s = ent[r].shot;
    const int lx = ent[r].lx, ly = ent[r].ly, lz = ent[r].lz;
    const Tiling& T = tilings[s];
    const int ti = (int)(std::upper_bound(T.xs.begin(), T.xs.end(), lx) - T.xs.begin()) - 1;
    const int tj = (int)(std::upper_bound(T.ys.begin(), T.ys.end(), ly) - T.ys.begin()) - 1;
    const int ncols = (int)T.xs.size() - 1, nrows = (int)T.ys.size() - 1;
    const int Nz = P.vols[s].Nz;
    const int zlen = (Nz + zsplit - 1) / zsplit;
    const int zb = std::min(lz / zlen, zsplit - 1);
    const int item = item_base[s] + (zb * nrows + tj) * ncols + ti;
    t.push_back(Tmp{item, lz, (lx - T.xs[ti]) + TX * (ly - T.ys[tj]), r});
  }
  std::sort(t.begin(), t.end(), [](const Tmp& a, const Tmp& b) {
    if (a.item != b.item) return a.item < b.item;
    if (a.z != b.z) return a.z < b.z;
    if (a.lxy != b.lxy) return a.lxy < b.lxy;
    return a.r < b.r;
  });
  rec.assign(t.size(), RecEntry{});
  cells.assign(t.size(), 0);
  gvals.assign(t.size(), 0.f);
  colmap.assign(t.size(), 0);
  rec_ptr.clear();
  for (auto& it : items) it.rec_tab = -1;
  size_t e = 0;
  while (e < t.size()) {
    const int item = t[e].item;
    size_t f = e;
    while (f < t.size() && t[f].item == item) ++f;
    WorkItem& W = items[item];
    W.rec_tab = (int)rec_ptr.size();
    const int npl = W.ze - W.zb;
    size_t k = e;
    for (int j = 0; j <= npl; ++j) {
      while (k < f && t[k].z < W.zb + j) ++k;
      rec_ptr.push_back((int)k);
    }
    e = f;
  }
  for (size_t i = 0; i < t.size(); ++i) {
    const NodeEntry& E = ent[t[i].r];
    RecEntry& R = rec[i];
    R.lxy = t[i].lxy;
    R.col = (int)i;
    R.group = 0;
    R.wgt = E.w;
    colmap[i] = E.r;
    cells[i] = E.cell;
    const VolDesc& V = P.vols[E.shot];
    gvals[i] = P.gx[V.gx_off + E.lx] * P.gy[V.gy_off + E.ly] * P.gz[E.lz];
  }
  if (ent_of_col) {
    ent_of_col->assign(t.size(), 0);
    for (size_t i = 0; i < t.size(); ++i) (*ent_of_col)[i] = t[i].r;
  }
  for (size_t i = 0; i < t.size();) {
    size_t j = i;
    while (j < t.size() && t[j].item == t[i].item && t[j].z == t[i].z && t[j].lxy == t[i].lxy) ++j;
    rec[i].group = (int)(j - i);
    i = j;
  }
}

// Chooses, among the compiled tile shapes, the shape, a row refinement and a
// split of the planes into z blocks that minimise the work of the busiest
// SM: ceil(items / SMs) items of (box-bound points x planes), divided by a
// factor for the resident warps (per-SM bandwidth falls off below about
// 16 warps).  Items beyond the resident slots run in later waves, which the
// same count captures.  MAMUTE_TX / MAMUTE_TY force a shape.
struct TileChoice {
  int tx = 64, ty = 16, zsplit = 1;
  std::vector<Tiling> tilings;
};

TileChoice choose_tiles(const std::vector<VolDesc>& vols, bool dens, int mode, int n_sm,
                        int force_tx, int force_ty, int force_z) {
  static const int shapes[][2] = {{64, 16}, {72, 16}, {48, 16}, {96, 8}, {64, 8},
                                  {128, 8}, {32, 16}, {32, 8}};
  static const int zsplits[] = {1, 2, 3, 4, 6, 8, 12, 16};
  TileChoice best;
  double best_cost = -1.0;
  const int Nz = vols.empty() ? 1 : vols[0].Nz;
  for (const auto& sh : shapes) {
    const int TX = sh[0], TY = sh[1];
    if (force_tx > 0 && (TX != force_tx || TY != force_ty)) continue;
    if (!tile_supported(TX, TY)) continue;
    const int per_sm = step_blocks_per_sm(TX, TY, dens, mode, Nz);
    if (per_sm < 1) continue;
    const int warps_cta = (TX / 4) * TY / 32;
    for (int r = 1; r <= 2; ++r) {
      std::vector<Tiling> tl;
      long long tiles = 0;
      double maxpts = 0.0;
      bool ok = true;
      for (const VolDesc& V : vols) {
        Tiling T;
        const int ncols = (V.Nx + TX - 1) / TX;
        const int nrows = std::min(V.Ny, r * ((V.Ny + TY - 1) / TY));
        T.xs = split(V.Nx, ncols, 4);
        T.ys = split(V.Ny, nrows, 1);
        if (max_piece(T.xs) > TX || max_piece(T.ys) > TY) { ok = false; break; }
        // rows refined only while tiles stay at least half full
        if (r > 1 && 2 * (V.Ny / nrows) < TY) { ok = false; break; }
        tiles += (long long)(T.xs.size() - 1) * (T.ys.size() - 1);
        // a CTA computes its whole box even when the tile is smaller
        maxpts = std::max(maxpts, std::max((double)max_piece(T.xs) * max_piece(T.ys),
                                           0.6 * TX * TY));
        tl.push_back(std::move(T));
      }
      if (!ok || tiles <= 0) continue;
      for (int zs : zsplits) {
        if (force_z > 0 && zs != force_z) continue;
        if (force_z <= 0 && zs > 1 && Nz / zs < 8) break;
        const long long items = tiles * zs;
        const long long per = (items + n_sm - 1) / n_sm;  // items on the busiest SM
        const double warps = (double)std::min<long long>(per_sm, per) * warps_cta;
        const double occ = std::min(1.0, warps / 16.0);
        // z-block priming reads 8 extra halo planes of one of ~4 arrays
        const double planes = (double)((Nz + zs - 1) / zs) + (zs > 1 ? 2.0 : 0.0);
        const double cost = (double)per * maxpts * planes / occ;
        if (env_int("MAMUTE_VERBOSE", 0) >= 2)
          fprintf(stderr, "mamute tiles: mode %d %dx%d rows x%d z%d: %d per SM, cost %.0f\n", mode, TX,
                  TY, r, zs, per_sm, cost);
        if (best_cost < 0 || cost < best_cost * (1.0 - 1e-3)) {
          best_cost = cost;
          best.tx = TX;
          best.ty = TY;
          best.zsplit = zs;
          best.tilings = tl;
        }
      }
    }
  }
  return best;
}

// adj_mode: the adjoint kernel mode the tiles are chosen for (MODE_ADJ when
// the forward states are recomputed, MODE_ADJ_STORED when every imaging term
// is kept: their shared-memory footprints, hence occupancies, differ).
int build_plan(mamute_ctx* ctx, const mamute_grid* g, bool dens, int n_src, const float* src_xyz,
               const int* rec_offset, const float* rec_xyz, const int* aperture, Plan& P,
               const int* tiles = nullptr, int adj_mode = MODE_ADJ) {
  if (!g) return fail(ctx, MAMUTE_EINVAL, "grid is NULL");
  if (g->nx < 1 || g->ny < 1 || g->nz < 1 || g->border < 0 || g->nt < 1)
    return fail(ctx, MAMUTE_EINVAL, "bad grid dimensions");
  if (!(g->h > 0.f) || !(g->dt > 0.f)) return fail(ctx, MAMUTE_EINVAL, "h and dt must be > 0");
  if (g->free_surface != 0 && g->free_surface != 1)
    return fail(ctx, MAMUTE_EINVAL, "free_surface must be 0 or 1");
  if (g->free_surface && g->nz < 5)
    return fail(ctx, MAMUTE_EINVAL, "a free surface needs nz >= 5 (the image of the stencil)");
  if (g->xyz_interp != 0 && g->xyz_interp != 1)
    return fail(ctx, MAMUTE_EINVAL, "xyz_interp must be 0 or 1");
  if (!(g->cerjan >= 0.f)) return fail(ctx, MAMUTE_EINVAL, "cerjan must be >= 0");
  if (g->pml != 0 && g->pml != 1) return fail(ctx, MAMUTE_EINVAL, "pml must be 0 or 1");
  if (g->pml) {
    if (!(g->pml_f0 >= 0.f)) return fail(ctx, MAMUTE_EINVAL, "pml_f0 must be >= 0");
    if (!(g->pml_r >= 0.f && g->pml_r < 1.f)) return fail(ctx, MAMUTE_EINVAL, "pml_r must be in [0, 1)");
    P.pml = true;
    P.pml_f0 = g->pml_f0;
    P.pml_r = g->pml_r > 0.f ? g->pml_r : 1e-3;
  }
  if (n_src < 1 || !src_xyz || !rec_offset) return fail(ctx, MAMUTE_EINVAL, "no shots");
  if (rec_offset[0] != 0) return fail(ctx, MAMUTE_EINVAL, "rec_offset[0] must be 0");
  for (int s = 0; s < n_src; ++s)
    if (rec_offset[s + 1] < rec_offset[s]) return fail(ctx, MAMUTE_EINVAL, "rec_offset decreasing");
  const int n_rec = rec_offset[n_src];
  if (n_rec > 0 && !rec_xyz) return fail(ctx, MAMUTE_EINVAL, "rec_xyz is NULL");
  P.nx = g->nx; P.ny = g->ny; P.nz = g->nz; P.b = g->border; P.nt = g->nt;
  P.h = g->h; P.dt = g->dt; P.dens = dens;
  P.Nx = P.nx + 2 * P.b; P.Ny = P.ny + 2 * P.b; P.Nz = P.nz + 2 * P.b;
  P.pitchG = (int)round_up(P.Nx, 8);
  const long long nmax = 1LL << 31;
  if ((long long)P.Nz * P.Ny * P.pitchG >= nmax * 4)
    return fail(ctx, MAMUTE_EINVAL, "grid too large");
  P.zs = g->free_surface ? P.b : -1;
  // The CPML replaces the sponge: damping factor 1 in the main step.
  const double alpha = P.pml ? 0.0 : (double)g->cerjan;
  P.gz = sponge(P.Nz, P.b, alpha, P.zs);
  // Model cells and weights of a point: its nearest node, or the trilinear
  // weights of the cell that holds it (zero weights dropped).  Nodes on a
  // free surface are dropped too (the field is zero there); false if the
  // point or a node it needs lies outside [lo, hi) or no node is left.
  struct Corner {
    int i, j, k;
    double w;
  };
  auto locate = [&](const float* xyz, const int lo[2], const int hi[2], std::vector<Corner>& out) {
    out.clear();
    const double f[3] = {((double)xyz[0] - g->ox) / g->h, ((double)xyz[1] - g->oy) / g->h,
                         ((double)xyz[2] - g->oz) / g->h};
    const int lim_lo[3] = {lo[0], lo[1], 0}, lim_hi[3] = {hi[0], hi[1], P.nz};
    if (!g->xyz_interp) {
      int id[3];
      for (int a = 0; a < 3; ++a) {
        id[a] = (int)std::floor(f[a] + 0.5);
        if (id[a] < lim_lo[a] || id[a] >= lim_hi[a]) return false;
      }
      if (P.zs >= 0 && id[2] == 0) return false;
      out.push_back(Corner{id[0], id[1], id[2], 1.0});
      return true;
    }
    int base[3];
    double t[3];
    for (int a = 0; a < 3; ++a) {
      base[a] = (int)std::floor(f[a]);
      t[a] = f[a] - (double)base[a];
    }
    for (int c = 0; c < 8; ++c) {
      int id[3];
      double w = 1.0;
      for (int a = 0; a < 3; ++a) {
        const int up = (c >> a) & 1;
        id[a] = base[a] + up;
        w *= up ? t[a] : 1.0 - t[a];
      }
      if (w == 0.0) continue;
      for (int a = 0; a < 3; ++a)
        if (id[a] < lim_lo[a] || id[a] >= lim_hi[a]) return false;
      if (P.zs >= 0 && id[2] == 0) continue;
      out.push_back(Corner{id[0], id[1], id[2], w});
    }
    return !out.empty();
  };
  std::vector<NodeEntry> ent;
  std::vector<int> rcount(n_rec, 0);
  std::vector<Corner> cs;
  long long off = 0, toff = 0;
  for (int s = 0; s < n_src; ++s) {
    int a0 = 0, a1 = P.nx, a2 = 0, a3 = P.ny;
    if (aperture) {
      a0 = aperture[4 * s]; a1 = aperture[4 * s + 1]; a2 = aperture[4 * s + 2]; a3 = aperture[4 * s + 3];
      if (a0 < 0 || a1 > P.nx || a0 >= a1 || a2 < 0 || a3 > P.ny || a2 >= a3)
        return fail(ctx, MAMUTE_EINVAL, "aperture of shot %d outside the model", s);
      if (a0 % 4) return fail(ctx, MAMUTE_EINVAL, "aperture x start of shot %d not a multiple of 4", s);
    }
    VolDesc V{};
    V.cx0 = a0; V.cy0 = a2;
    V.Nx = (a1 - a0) + 2 * P.b; V.Ny = (a3 - a2) + 2 * P.b; V.Nz = P.Nz;
    V.pitch = (int)round_up(V.Nx, 8);
    V.border = P.b; V.nzi = P.nz;
    // imaging region: window cells inside the model (model x = a0 - b + local x)
    V.ix0 = std::max(0, P.b - a0);
    V.nxi = std::min(V.Nx, P.nx + P.b - a0) - V.ix0;
    V.iy0 = std::max(0, P.b - a2);
    V.nyi = std::min(V.Ny, P.ny + P.b - a2) - V.iy0;
    V.slab = round_up((long long)V.Nz * V.Ny * V.pitch, 64);
    V.off = off; off += V.slab;
    // Term-store rows start on a 16-byte boundary of the local x axis (TMA).
    V.txoff = V.ix0 & ~3;
    V.tpitch = (int)round_up(V.ix0 - V.txoff + V.nxi, 4);
    V.toff = toff; toff += (long long)V.tpitch * V.nyi * V.nzi;
    V.gx_off = (int)P.gx.size(); V.gy_off = (int)P.gy.size();
    std::vector<float> px = sponge(V.Nx, P.b, alpha), py = sponge(V.Ny, P.b, alpha);
    P.gx.insert(P.gx.end(), px.begin(), px.end());
    P.gy.insert(P.gy.end(), py.begin(), py.end());
    const int lo[2] = {a0, a2}, hi[2] = {a1, a3};
    if (!locate(src_xyz + 3 * s, lo, hi, cs))
      return fail(ctx, MAMUTE_EINVAL, "source %d outside the model, its aperture or on the free surface", s);
    // corner (0,0,0) of the source's cell; the 8 scales are set on the device
    int bi = cs[0].i, bj = cs[0].j, bk = cs[0].k;
    for (const Corner& c : cs) {
      bi = std::min(bi, c.i); bj = std::min(bj, c.j); bk = std::min(bk, c.k);
    }
    V.src_x = bi + P.b - a0; V.src_y = bj + P.b - a2; V.src_z = bk + P.b;
    for (int e = 0; e < 8; ++e) {
      P.src_cell.push_back(-1);
      P.src_w.push_back(0.f);
    }
    for (const Corner& c : cs) {
      const int e = (c.i - bi) + 2 * (c.j - bj) + 4 * (c.k - bk);
      P.src_cell[8 * s + e] = ((long long)c.k * P.ny + c.j) * P.nx + c.i;
      P.src_w[8 * s + e] = (float)c.w;
    }
    for (int r = rec_offset[s]; r < rec_offset[s + 1]; ++r) {
      if (!locate(rec_xyz + 3 * (long long)r, lo, hi, cs))
        return fail(ctx, MAMUTE_EINVAL,
                    "receiver %d outside the model, the aperture of its shot or on the free surface", r);
      for (const Corner& c : cs)
        ent.push_back(NodeEntry{c.i + P.b - a0, c.j + P.b - a2, c.k + P.b,
                                ((long long)c.k * P.ny + c.j) * P.nx + c.i, r, s, (float)c.w});
      rcount[r] = (int)cs.size();
    }
    P.vols.push_back(V);
  }
  P.pool_elems = off;
  P.term_elems = toff;
  P.ncol = (int)ent.size();
  P.nrec = n_rec;
  P.one_node = true;
  for (int r = 0; r < n_rec; ++r) P.one_node = P.one_node && rcount[r] == 1;
  // Work items: one per tile, all planes, for the forward and adjoint kernels.
  int n_sm = 0;
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, ctx->device);
  if (n_sm < 1) n_sm = 1;
  const int fmode = dens ? MODE_FWD : MODE_FWD;
  auto pick = [&](int i, const char* env) { return (tiles && tiles[i] > 0) ? tiles[i] : env_int(env, 0); };
  TileChoice fc = choose_tiles(P.vols, dens, fmode, n_sm, pick(0, "MAMUTE_TX"), pick(1, "MAMUTE_TY"),
                               pick(2, "MAMUTE_ZSPLIT"));
  TileChoice ac = choose_tiles(P.vols, dens, adj_mode, n_sm, pick(3, "MAMUTE_ADJ_TX"),
                               pick(4, "MAMUTE_ADJ_TY"), pick(5, "MAMUTE_ADJ_ZSPLIT"));
  if (fc.tilings.empty() || ac.tilings.empty())
    return fail(ctx, MAMUTE_EINVAL, "unsupported tile shape");
  P.tx = fc.tx; P.ty = fc.ty; P.atx = ac.tx; P.aty = ac.ty;
  auto make_items = [&](const TileChoice& C, std::vector<WorkItem>& items, std::vector<int>& base) {
    items.clear();
    base.clear();
    for (int s = 0; s < n_src; ++s) {
      const VolDesc& V = P.vols[s];
      const Tiling& T = C.tilings[s];
      base.push_back((int)items.size());
      const int zlen = (V.Nz + C.zsplit - 1) / C.zsplit;
      for (int zb = 0; zb < C.zsplit; ++zb)
        for (size_t tj = 0; tj + 1 < T.ys.size(); ++tj)
          for (size_t ti = 0; ti + 1 < T.xs.size(); ++ti)
            items.push_back(WorkItem{s, T.xs[ti], T.ys[tj], zb * zlen, std::min(V.Nz, (zb + 1) * zlen),
                                     T.xs[ti + 1] - T.xs[ti], T.ys[tj + 1] - T.ys[tj], -1});
    }
  };
  std::vector<int> base;
  make_items(fc, P.items, base);
  std::vector<int> ent_of_col;
  build_receivers(P, P.tx, fc.zsplit, ent, base, fc.tilings, P.items, P.rec_ptr, P.rec,
                  P.rec_cell, P.rec_g, P.colmap, &ent_of_col);
  P.fwd_col_of_ent.assign(ent.size(), 0);
  for (size_t c = 0; c < ent_of_col.size(); ++c) P.fwd_col_of_ent[ent_of_col[c]] = (int)c;
  P.ent = ent;
  // receiver -> internal columns of the forward tables, ascending
  P.rcol_ptr.assign(n_rec + 1, 0);
  for (int c = 0; c < P.ncol; ++c) ++P.rcol_ptr[P.colmap[c] + 1];
  for (int r = 0; r < n_rec; ++r) P.rcol_ptr[r + 1] += P.rcol_ptr[r];
  P.rcols.assign(P.ncol, 0);
  {
    std::vector<int> fill(P.rcol_ptr.begin(), P.rcol_ptr.end() - 1);
    for (int c = 0; c < P.ncol; ++c) P.rcols[fill[P.colmap[c]]++] = c;
  }
  make_items(ac, P.aitems, base);
  build_receivers(P, P.atx, ac.zsplit, ent, base, ac.tilings, P.aitems, P.arec_ptr, P.arec,
                  P.arec_cell, P.arec_g, P.acolmap);
  if (env_int("MAMUTE_VERBOSE", 0))
    fprintf(stderr, "mamute plan: %d shots, forward tile %dx%d/%dz (%zu CTAs), adjoint tile %dx%d/%dz (%zu CTAs)\n",
            n_src, P.tx, P.ty, fc.zsplit, P.items.size(), P.atx, P.aty, ac.zsplit, P.aitems.size());
  return MAMUTE_OK;
}

CUresult encode3d(mamute_ctx* ctx, CUtensorMap* m, const float* base, int Nx, int Ny, int Nz,
                  int pitch, int bx, int by) {
  cuuint64_t dims[3] = {(cuuint64_t)Nx, (cuuint64_t)Ny, (cuuint64_t)Nz};
  cuuint64_t strides[2] = {(cuuint64_t)pitch * 4, (cuuint64_t)pitch * Ny * 4};
  cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
  cuuint32_t es[3] = {1, 1, 1};
  return ctx->encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)base, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

// Device-resident problem: coefficients, tables and maps for one call.
struct Run {
  Plan P;
  bool adj_maps = false;
};

cudaError_t aux_count(mamute_ctx* ctx, cudaError_t e) {
  ++ctx->launches;
  return e;
}

int check_cfl(mamute_ctx* ctx, Plan& P, const float* vel) {
  CK(cudaMemsetAsync(ctx->maxbits, 0, sizeof(unsigned int), ctx->stream));
  CK(aux_count(ctx, launch_max(vel, (long long)P.nx * P.ny * P.nz, ctx->maxbits, ctx->stream)));
  unsigned int bits = 0;
  CK(cudaMemcpyAsync(&bits, ctx->maxbits, sizeof bits, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  float vmax;
  std::memcpy(&vmax, &bits, sizeof vmax);
  P.vmax = vmax;
  const double courant = (double)vmax * P.dt / P.h;
  if (!(courant <= cfl_bound()))
    return fail(ctx, MAMUTE_ECFL, "max(c) dt / h = %.5f exceeds the stability bound %.5f", courant,
                cfl_bound());
  return MAMUTE_OK;
}

// Coefficients, geometry tables, pools and maps.
int setup(mamute_ctx* ctx, Plan& P, const float* vel, const float* rho, bool need_psi,
          bool need_acc) {
  const size_t nG = (size_t)P.Nz * P.Ny * P.pitchG;
  CK(ensure(ctx->coefA, nG * 4));
  if (P.dens) CK(ensure(ctx->coefM, nG * 4));
  if (P.dens) CK(ensure(ctx->srho, (size_t)P.nx * P.ny * P.nz * 8));
  CoefPrepArgs ca{vel, rho, P.nx, P.ny, P.nz, P.b, P.Nx, P.Ny, P.Nz, P.pitchG, P.h, P.dt,
                  (float*)ctx->coefA.p, P.dens ? (float*)ctx->coefM.p : nullptr,
                  P.dens ? (double*)ctx->srho.p : nullptr};
  CK(aux_count(ctx, launch_prep_coef(ca, ctx->stream)));
  const size_t pool = (size_t)P.pool_elems * 4;
  for (int i = 0; i < 2; ++i) CK(ensure(ctx->pool[i], pool));
  if (need_psi)
    for (int i = 0; i < 2; ++i) CK(ensure(ctx->psi[i], pool));
  if (need_acc) CK(ensure(ctx->acc, pool));
  CK(upload(ctx->vols, P.vols, ctx->stream));
  CK(upload(ctx->items, P.items, ctx->stream));
  CK(upload(ctx->recptr, P.rec_ptr, ctx->stream));
  CK(upload(ctx->rec, P.rec, ctx->stream));
  CK(upload(ctx->colmap, P.colmap, ctx->stream));
  CK(upload(ctx->cells, P.rec_cell, ctx->stream));
  CK(upload(ctx->gvals, P.rec_g, ctx->stream));
  CK(upload(ctx->aitems, P.aitems, ctx->stream));
  CK(upload(ctx->arecptr, P.arec_ptr, ctx->stream));
  CK(upload(ctx->arec, P.arec, ctx->stream));
  CK(upload(ctx->acolmap, P.acolmap, ctx->stream));
  CK(upload(ctx->acells, P.arec_cell, ctx->stream));
  CK(upload(ctx->agvals, P.arec_g, ctx->stream));
  CK(upload(ctx->srccell, P.src_cell, ctx->stream));
  CK(upload(ctx->srcw, P.src_w, ctx->stream));
  if (!P.one_node) {
    std::vector<int> iota(P.ncol);
    for (int c = 0; c < P.ncol; ++c) iota[c] = c;
    CK(upload(ctx->ident, iota, ctx->stream));
    CK(upload(ctx->rcolptr, P.rcol_ptr, ctx->stream));
    CK(upload(ctx->rcols, P.rcols, ctx->stream));
    CK(ensure(ctx->ecol, (size_t)P.ncol * P.nt * 4));
  }
  CK(upload(ctx->gx, P.gx, ctx->stream));
  CK(upload(ctx->gy, P.gy, ctx->stream));
  CK(upload(ctx->gz, P.gz, ctx->stream));
  // Scales at receivers (both tables) and sources.
  GeomArgs ga{vel, rho, (int)P.rec.size(), (int)P.vols.size(), (const long long*)ctx->cells.p,
              (const float*)ctx->gvals.p, (RecEntry*)ctx->rec.p, (const long long*)ctx->srccell.p,
              (const float*)ctx->srcw.p, (VolDesc*)ctx->vols.p, P.h, P.dt};
  CK(aux_count(ctx, launch_geometry(ga, ctx->stream)));
  GeomArgs gb{vel, rho, (int)P.arec.size(), 0, (const long long*)ctx->acells.p,
              (const float*)ctx->agvals.p, (RecEntry*)ctx->arec.p, nullptr, nullptr, nullptr,
              P.h, P.dt};
  CK(aux_count(ctx, launch_geometry(gb, ctx->stream)));
  // Tensor maps (layout in ShotMaps).
  std::vector<ShotMaps> maps(P.vols.size());
  for (size_t s = 0; s < P.vols.size(); ++s) {
    const VolDesc& V = P.vols[s];
    auto enc = [&](int slot, const void* base, int bx, int by) {
      return encode3d(ctx, &maps[s].m[slot], (const float*)base + V.off, V.Nx, V.Ny, V.Nz, V.pitch,
                      bx, by) == CUDA_SUCCESS;
    };
    bool ok = true;
    for (int b = 0; b < 2; ++b) {
      ok = ok && enc(2 * b + 0, ctx->pool[b].p, P.tx + 8, P.ty + 8);
      ok = ok && enc(2 * b + 1, ctx->pool[b].p, P.tx, P.ty);
      if (need_psi) {
        ok = ok && enc(4 + 2 * b + 0, ctx->psi[b].p, P.atx + 8, P.aty + 8);
        ok = ok && enc(4 + 2 * b + 1, ctx->psi[b].p, P.atx, P.aty);
        ok = ok && enc(9 + b, ctx->pool[b].p, P.atx + 8, P.aty + 8);
      }
    }
    if (need_acc) {
      ok = ok && enc(8, ctx->acc.p, P.tx, P.ty);
      ok = ok && enc(11, ctx->acc.p, P.atx, P.aty);
    }
    if (!ok) return fail(ctx, MAMUTE_ECUDA, "cuTensorMapEncodeTiled failed (shot %d)", (int)s);
  }
  CK(upload(ctx->maps, maps, ctx->stream));
  ctx->hmaps = maps;
  std::vector<CoefMaps> cm(2);  // [0]: forward tile boxes, [1]: adjoint tile boxes
  for (int v = 0; v < 2; ++v) {
    const int bx = v ? P.atx : P.tx, by = v ? P.aty : P.ty;
    if (encode3d(ctx, &cm[v].m[0], (const float*)ctx->coefA.p, P.Nx, P.Ny, P.Nz, P.pitchG, bx, by))
      return fail(ctx, MAMUTE_ECUDA, "cuTensorMapEncodeTiled failed (A)");
    if (P.dens &&
        encode3d(ctx, &cm[v].m[1], (const float*)ctx->coefM.p, P.Nx, P.Ny, P.Nz, P.pitchG, bx, by))
      return fail(ctx, MAMUTE_ECUDA, "cuTensorMapEncodeTiled failed (M)");
  }
  CK(upload(ctx->cmaps, cm, ctx->stream));
  return MAMUTE_OK;
}

// Launch accounting and the timing events around the time loop.
cudaError_t step_launch(mamute_ctx* ctx, const StepArgs& a, int n_items, int tx, int ty, bool dens,
                        int mode) {
  if (ctx->timing && !ctx->ev0_set) {
    cudaError_t e = cudaEventRecord(ctx->ev0, ctx->stream);
    if (e != cudaSuccess) return e;
    ctx->ev0_set = true;
  }
  ++ctx->step_launches;
  ++ctx->launches;
  cudaError_t e = launch_step(a, n_items, ctx->max_planes, tx, ty, dens, mode, ctx->stream);
  if (e == cudaSuccess && ctx->timing) e = cudaEventRecord(ctx->ev1, ctx->stream);
  return e;
}

// One DFT accumulation (twiddles + dft_kernel), timed by an event pair
// when the timing hook is on.
cudaError_t dft_launch(mamute_ctx* ctx, const float* V, long long N, int T, int n0, int nf,
                       const int* bins, int nb, float2* W, float* re, float* im) {
  cudaError_t e = cudaSuccess;
  if (ctx->timing) {
    while (ctx->dft_ev.size() < (size_t)2 * ctx->dft_n + 2) {
      cudaEvent_t ev = nullptr;
      e = cudaEventCreate(&ev);
      if (e != cudaSuccess) return e;
      ctx->dft_ev.push_back(ev);
    }
    e = cudaEventRecord(ctx->dft_ev[2 * ctx->dft_n], ctx->stream);
    if (e != cudaSuccess) return e;
  }
  ctx->launches += 2;
  if (dft_tc_supported(N, nb) && (uintptr_t)V % 16 == 0 && (uintptr_t)re % 16 == 0 &&
      (uintptr_t)im % 16 == 0 && (uintptr_t)W % 16 == 0) {
    // tensor cores: samples by TMA (V as {N, T, 1} FP32, boxes of 128 points
    // x one chunk of samples)
    CUtensorMap vmap;
    cuuint64_t dims[3] = {(cuuint64_t)N, (cuuint64_t)std::max(T, 1), 1};
    cuuint64_t strides[2] = {(cuuint64_t)N * 4, (cuuint64_t)N * std::max(T, 1) * 4};
    cuuint32_t box[3] = {128, (cuuint32_t)dft_tc_chunk(), 1};
    cuuint32_t es[3] = {1, 1, 1};
    if (ctx->encode(&vmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(V), dims, strides,
                    box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE))
      return cudaErrorInvalidValue;
    // every batch starts from zeroed accumulators: its first block stores
    e = launch_dft_tc(vmap, N, T, n0, nf, bins, nb, reinterpret_cast<float*>(W), re, im, n0 == 0,
                      ctx->status, ctx->stream);
  } else {
    e = launch_dft(V, N, T, n0, nf, bins, nb, W, re, im, ctx->status, ctx->stream);
  }
  if (e == cudaSuccess && ctx->timing && T > 0) {
    e = cudaEventRecord(ctx->dft_ev[2 * ctx->dft_n + 1], ctx->stream);
    ++ctx->dft_n;
    ctx->dft_macs += (double)N * T * nb;
  }
  return e;
}

constexpr int kShotMapStride = (int)(sizeof(ShotMaps) / sizeof(CUtensorMap));

// Map m[idx] of shot 0 in the uploaded per-shot map array.
const CUtensorMap* shot_map(mamute_ctx* ctx, int idx) {
  return &((const ShotMaps*)ctx->maps.p)[0].m[idx];
}

StepArgs fwd_args(mamute_ctx* ctx, const Plan& P, int n, const float* wavelet, float* dout,
                  int mode) {
  StepArgs a{};
  a.items = (const WorkItem*)ctx->items.p;
  a.vols = (const VolDesc*)ctx->vols.p;
  a.maps = (const ShotMaps*)ctx->maps.p;
  a.cmaps = (const CoefMaps*)ctx->cmaps.p;
  a.gx = (const float*)ctx->gx.p;
  a.gy = (const float*)ctx->gy.p;
  a.gz = (const float*)ctx->gz.p;
  a.mF = shot_map(ctx, 2 * (n & 1));            // u^n, halo
  a.mP = shot_map(ctx, 2 * ((n + 1) & 1) + 1);  // u^{n-1}, centre
  a.mU = a.mF;
  a.sF = a.sP = a.sU = kShotMapStride;
  a.wn = wavelet[n];
  a.fout = (float*)ctx->pool[(n + 1) & 1].p;
  a.acc = (float*)ctx->acc.p;
  a.tstore = (mode == MODE_FWD_STORE || mode == MODE_FWD_STORE_PH)
                 ? (float*)ctx->tstore.p + (size_t)n * P.term_elems
                 : nullptr;
  a.rec_ptr = (const int*)ctx->recptr.p;
  a.rec = (const RecEntry*)ctx->rec.p;
  a.dout = dout;
  a.rin = nullptr;
  a.status = ctx->status;
  a.zs = P.zs;
  return a;
}

int finish(mamute_ctx* ctx) {
  int st = 0;
  CK(cudaMemcpyAsync(&st, ctx->status, sizeof st, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->timing && ctx->ev0_set) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
    ctx->loop_ms = ms;
  }
  if (st & kErrTimeout) return fail(ctx, MAMUTE_ETIMEOUT, "a device-side wait ran out");
  return MAMUTE_OK;
}

int check_common(mamute_ctx* ctx, const mamute_grid* g, const float* vel, const float* wavelet) {
  if (!ctx) return MAMUTE_EINVAL;
  ctx->err.clear();
  ctx->ev0_set = false;
  ctx->loop_ms = 0.0;
  ctx->step_launches = 0;
  ctx->launches = 0;
  if (!vel || !wavelet || !g) return fail(ctx, MAMUTE_EINVAL, "NULL vel, wavelet or grid");
  CK(cudaSetDevice(ctx->device));
  CK(cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream));
  return MAMUTE_OK;
}

#define TRY(x)               \
  do {                       \
    int rc_ = (x);           \
    if (rc_ != MAMUTE_OK) return rc_; \
  } while (0)

// Two-level forward launches (stencil_pair.cu), on request (time_blocking =
// 2, or MAMUTE_PAIRS=1): one shot, no free surface, every tile resident at
// once (one CTA per SM).  Columns of the x split are
// multiples of 4 and at most TX wide; the rows are split as finely as the
// SMs allow (at least 8 rows per tile), so that all SMs get a tile.
bool plan_pairs(mamute_ctx* ctx, Plan& P, const mamute_opts* opts) {
  const int want = env_int("MAMUTE_PAIRS", opts && opts->time_blocking == 2 ? 1 : 0);
  if (want == 0 || P.vols.size() != 1 || P.zs >= 0 || P.nt < 2) return false;
  int n_sm = 0;
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, ctx->device);
  const VolDesc& V = P.vols[0];
  static const int shapes[][2] = {{72, 32}, {64, 32}, {32, 16}};
  for (const auto& sh : shapes) {
    const int TX = sh[0], TY = sh[1];
    if (!pair_tile_supported(TX, TY)) continue;
    int occ = 0;
    PairArgs dummy{};
    const cudaError_t oe = launch_pair(dummy, 0, V.Nz, TX, TY, P.dens, nullptr, &occ);
    if (env_int("MAMUTE_VERBOSE", 0))
      fprintf(stderr, "mamute pairs: tile %dx%d: %s, %d CTA(s) per SM\n", TX, TY,
              cudaGetErrorString(oe), occ);
    if (oe != cudaSuccess || occ < 1) {
      cudaGetLastError();
      continue;
    }
    const int ncols = (V.Nx + TX - 1) / TX;
    const long long slots = (long long)occ * n_sm;
    const int need_rows = (V.Ny + TY - 1) / TY;
    if ((long long)ncols * need_rows > slots) continue;
    int nrows = (int)std::min<long long>(slots / ncols, (V.Ny + 7) / 8);
    nrows = std::max(nrows, need_rows);
    Tiling T;
    T.xs = split(V.Nx, ncols, 4);
    // Row boundaries are even: a thread's two rows then lie in the same tile,
    // so the rows it computes past its tile (from halo data that the next
    // tile may already have overwritten) are never used as neighbours.
    T.ys = split(V.Ny, nrows, 2);
    if (max_piece(T.xs) > TX || max_piece(T.ys) > TY) continue;
    // a tile's 4-row halo must stay within its neighbours
    bool thin = false;
    for (size_t k = 1; k + 1 < T.ys.size(); ++k) thin = thin || T.ys[k] - T.ys[k - 1] < kHalo;
    if (thin) continue;
    const int nc = (int)T.xs.size() - 1, nr = (int)T.ys.size() - 1;
    P.pitems.clear();
    P.pnbr.clear();
    for (int tj = 0; tj < nr; ++tj)
      for (int ti = 0; ti < nc; ++ti) {
        P.pitems.push_back(WorkItem{0, T.xs[ti], T.ys[tj], 0, V.Nz, T.xs[ti + 1] - T.xs[ti],
                                    T.ys[tj + 1] - T.ys[tj], -1});
        auto id = [&](int a, int b) { return (a < 0 || a >= nc || b < 0 || b >= nr) ? -1 : b * nc + a; };
        P.pnbr.push_back(make_int4(id(ti - 1, tj), id(ti + 1, tj), id(ti, tj - 1), id(ti, tj + 1)));
      }
    std::vector<int> base(1, 0);
    std::vector<Tiling> tl(1, T);
    std::vector<int> colmap, ent_of_col;
    build_receivers(P, TX, 1, P.ent, base, tl, P.pitems, P.prec_ptr, P.prec, P.prec_cell,
                    P.prec_g, colmap, &ent_of_col);
    // the same internal data columns as the one-step tables
    for (size_t c = 0; c < P.prec.size(); ++c) P.prec[c].col = P.fwd_col_of_ent[ent_of_col[c]];
    P.ptx = TX;
    P.pty = TY;
    P.pairs = true;
    if (env_int("MAMUTE_VERBOSE", 0))
      fprintf(stderr, "mamute pairs: tile %dx%d, %d x %d tiles\n", TX, TY, nc, nr);
    return true;
  }
  return false;
}

// Tables, tensor maps and progress flags of the two-level launches.
int setup_pairs(mamute_ctx* ctx, const Plan& P, const float* vel, const float* rho) {
  CK(upload(ctx->pitems, P.pitems, ctx->stream));
  CK(upload(ctx->pnbr, P.pnbr, ctx->stream));
  CK(upload(ctx->precptr, P.prec_ptr, ctx->stream));
  CK(upload(ctx->prec, P.prec, ctx->stream));
  CK(upload(ctx->pcells, P.prec_cell, ctx->stream));
  CK(upload(ctx->pgvals, P.prec_g, ctx->stream));
  GeomArgs ga{vel, rho, (int)P.prec.size(), 0, (const long long*)ctx->pcells.p,
              (const float*)ctx->pgvals.p, (RecEntry*)ctx->prec.p, nullptr, nullptr, nullptr,
              P.h, P.dt};
  CK(aux_count(ctx, launch_geometry(ga, ctx->stream)));
  const VolDesc& V = P.vols[0];
  std::vector<PairMaps> pm(1);
  bool ok = true;
  for (int b = 0; b < 2; ++b) {
    const float* base = (const float*)ctx->pool[b].p + V.off;
    ok = ok && encode3d(ctx, &pm[0].m[b], base, V.Nx, V.Ny, V.Nz, V.pitch, P.ptx + 8, P.pty + 8) ==
                   CUDA_SUCCESS;
    ok = ok && encode3d(ctx, &pm[0].m[2 + b], base, V.Nx, V.Ny, V.Nz, V.pitch, P.ptx, P.pty) ==
                   CUDA_SUCCESS;
  }
  ok = ok && encode3d(ctx, &pm[0].m[4], (const float*)ctx->coefA.p, P.Nx, P.Ny, P.Nz, P.pitchG,
                      P.ptx, P.pty) == CUDA_SUCCESS;
  if (P.dens)
    ok = ok && encode3d(ctx, &pm[0].m[5], (const float*)ctx->coefM.p, P.Nx, P.Ny, P.Nz, P.pitchG,
                        P.ptx, P.pty) == CUDA_SUCCESS;
  else
    pm[0].m[5] = pm[0].m[4];
  if (!ok) return fail(ctx, MAMUTE_ECUDA, "cuTensorMapEncodeTiled failed (two-level maps)");
  CK(upload(ctx->pmaps, pm, ctx->stream));
  CK(ensure(ctx->pflags, P.pitems.size() * 4));
  return MAMUTE_OK;
}

// Gradient smoothing by the DCT-II diagonalisation of the Bessel / Laplace
// operators (see postproc.cu): forward transforms along x, y, z, the
// spectral multiplier, transposed transforms along z, y, x.
int do_smooth(mamute_ctx* ctx, int nx, int ny, int nz, double h, int mode, const float* lengths,
              const float* in, float* out) {
  const long long n = (long long)nx * ny * nz;
  if (mode == 0) {
    if (in != out) CK(cudaMemcpyAsync(out, in, (size_t)n * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    return MAMUTE_OK;
  }
  const int dims[3] = {nx, ny, nz};
  double L[3];
  for (int a = 0; a < 3; ++a) {
    const double l = lengths ? (double)lengths[a] : 0.0;
    if (!(l >= 0.0)) return fail(ctx, MAMUTE_EINVAL, "smoothing length %d is negative", a);
    L[a] = l > 0.0 ? l : 2.0 * h;
  }
  // C_a (orthonormal DCT-II, rows = modes) and its transpose, per axis, and
  // the eigenvalues of -l_a^2 D_aa; built and uploaded only when the sizes,
  // the spacing or the lengths differ from the previous call's.
  size_t off[3][2];
  size_t o = 0;
  for (int a = 0; a < 3; ++a) {
    off[a][0] = o;
    off[a][1] = o + (size_t)dims[a] * dims[a];
    o += 2 * (size_t)dims[a] * dims[a];
  }
  const std::vector<double> key = {(double)nx, (double)ny, (double)nz, h, L[0], L[1], L[2]};
  if (key != ctx->smKey) {
    ctx->smKey.clear();
    std::vector<float> mats(o), lam;
    for (int a = 0; a < 3; ++a) {
      const int m = dims[a];
      for (int k = 0; k < m; ++k)
        for (int i = 0; i < m; ++i) {
          const double sc = k == 0 ? std::sqrt(1.0 / m) : std::sqrt(2.0 / m);
          const float c = (float)(sc * std::cos(M_PI * k * (i + 0.5) / m));
          mats[off[a][0] + (size_t)k * m + i] = c;
          mats[off[a][1] + (size_t)i * m + k] = c;
        }
      for (int k = 0; k < m; ++k) {
        const double sn = std::sin(M_PI * k / (2.0 * m));
        lam.push_back((float)(4.0 * (L[a] / h) * (L[a] / h) * sn * sn));
      }
    }
    CK(upload(ctx->smMat, mats, ctx->stream));
    CK(upload(ctx->smLam, lam, ctx->stream));
    ctx->smKey = key;
  }
  CK(ensure(ctx->smA, (size_t)n * 4));
  const float* M = (const float*)ctx->smMat.p;
  float* A = (float*)ctx->smA.p;
  // axis geometry: lines, inner, outer, stride
  const long long g[3][4] = {{(long long)ny * nz, 1, nx, 1},
                             {(long long)nz * nx, nx, (long long)nx * ny, nx},
                             {(long long)nx * ny, (long long)nx * ny, 0, (long long)nx * ny}};
  auto pass = [&](int a, int inv, const float* src, float* dst) -> cudaError_t {
    ++ctx->launches;
    return launch_axis(src, dst, M + off[a][inv], dims[a], g[a][0], g[a][1], g[a][2], g[a][3],
                       ctx->stream);
  };
  CK(pass(0, 0, in, A));
  CK(pass(1, 0, A, out));
  CK(pass(2, 0, out, A));
  ++ctx->launches;
  CK(launch_spectral_scale(A, nx, ny, nz, (const float*)ctx->smLam.p, mode, ctx->stream));
  CK(pass(2, 1, A, out));
  CK(pass(1, 1, out, A));
  CK(pass(0, 1, A, out));
  return MAMUTE_OK;
}

// Rows of the resampling matrix (or of its transpose) as CSR, weights in FP64
// (see mamute_resample in the header for the definitions); do_resample turns
// them into a band.
void resample_csr(int nt_in, double dt_in, int nt_out, double dt_out, int mode, bool transpose,
                  std::vector<int>& ptr, std::vector<int>& col, std::vector<float>& w) {
  std::vector<std::vector<std::pair<int, double>>> rows(nt_out);
  if (mode == MAMUTE_INTERP_NEAREST) {
    for (int m = 0; m < nt_out; ++m) {
      const long long nn = (long long)std::floor(m * dt_out / dt_in + 0.5);
      if (nn >= 0 && nn < nt_in) rows[m].push_back({(int)nn, 1.0});
    }
  } else {
    const int W = 8;
    const double D = std::max(dt_in, dt_out);
    for (int m = 0; m < nt_out; ++m) {
      const double c = m * dt_out / dt_in, half = W * D / dt_in;
      const long long lo = std::max(0LL, (long long)std::floor(c - half) - 1);
      const long long hi = std::min((long long)nt_in - 1, (long long)std::ceil(c + half) + 1);
      for (long long nn = lo; nn <= hi; ++nn) {
        const double u = (m * dt_out - nn * dt_in) / D;
        if (!(std::fabs(u) < W)) continue;
        const double sinc = u == 0.0 ? 1.0 : std::sin(M_PI * u) / (M_PI * u);
        const double hann = 0.5 * (1.0 + std::cos(M_PI * u / W));
        rows[m].push_back({(int)nn, dt_in / D * sinc * hann});
      }
    }
  }
  ptr.clear();
  col.clear();
  w.clear();
  if (!transpose) {
    ptr.push_back(0);
    for (int m = 0; m < nt_out; ++m) {
      for (auto& e : rows[m]) {
        col.push_back(e.first);
        w.push_back((float)e.second);
      }
      ptr.push_back((int)col.size());
    }
    return;
  }
  std::vector<std::vector<std::pair<int, double>>> cols(nt_in);
  for (int m = 0; m < nt_out; ++m)
    for (auto& e : rows[m]) cols[e.first].push_back({m, e.second});
  ptr.push_back(0);
  for (int nn = 0; nn < nt_in; ++nn) {
    for (auto& e : cols[nn]) {
      col.push_back(e.first);
      w.push_back((float)e.second);
    }
    ptr.push_back((int)col.size());
  }
}

int do_resample(mamute_ctx* ctx, int ntr, int nt_in, double dt_in, int nt_out, double dt_out,
                int mode, int adjoint, const float* x, float* y) {
  if (ntr < 0 || nt_in < 1 || nt_out < 1 || !(dt_in > 0.0) || !(dt_out > 0.0) ||
      (mode != MAMUTE_INTERP_NEAREST && mode != MAMUTE_INTERP_SINC))
    return fail(ctx, MAMUTE_EINVAL, "resample: bad sizes, steps or mode");
  if (ntr == 0) return MAMUTE_OK;
  if (!x || !y) return fail(ctx, MAMUTE_EINVAL, "resample: NULL trace array");
  // the matrix is built and uploaded only when it differs from the previous call's
  const std::vector<double> key = {(double)nt_in, dt_in, (double)nt_out, dt_out, (double)mode,
                                   (double)(adjoint != 0)};
  if (key != ctx->rsKey) {
    ctx->rsKey.clear();
    std::vector<int> ptr, col;
    std::vector<float> w;
    resample_csr(nt_in, dt_in, nt_out, dt_out, mode, adjoint != 0, ptr, col, w);
    // as a band: row m covers columns c0[m] .. c0[m] + len[m] - 1 (a gap, if
    // any, holds zero weights), weights tap-major
    const int rows = (int)ptr.size() - 1;
    std::vector<int> c0(rows, 0), len(rows, 0);
    int K = 0;
    for (int m = 0; m < rows; ++m)
      if (ptr[m + 1] > ptr[m]) {
        c0[m] = col[ptr[m]];
        len[m] = col[ptr[m + 1] - 1] - c0[m] + 1;
        K = std::max(K, len[m]);
      }
    std::vector<float> wb((size_t)K * rows, 0.0f);
    for (int m = 0; m < rows; ++m)
      for (int k = ptr[m]; k < ptr[m + 1]; ++k) wb[(size_t)(col[k] - c0[m]) * rows + m] = w[k];
    CK(upload(ctx->rsPtr, c0, ctx->stream));
    CK(upload(ctx->rsCol, len, ctx->stream));
    CK(upload(ctx->rsW, wb, ctx->stream));
    ctx->rsKey = key;
  }
  ++ctx->launches;
  const int n_src = adjoint ? nt_out : nt_in, n_dst = adjoint ? nt_in : nt_out;
  CK(launch_band_rows(x, n_src, (const int*)ctx->rsPtr.p, (const int*)ctx->rsCol.p,
                     (const float*)ctx->rsW.p, n_dst, ntr, y, ctx->stream));
  return MAMUTE_OK;
}

// Data time axis of a call: nt_data samples of dt_data (time_interp != 0),
// else the modelling axis.
int check_interp(mamute_ctx* ctx, const mamute_grid* g, const mamute_opts* opts, int* ti,
                 int* ntd) {
  *ti = opts ? opts->time_interp : 0;
  *ntd = g->nt;
  if (*ti == 0) return MAMUTE_OK;
  if (*ti != MAMUTE_INTERP_NEAREST && *ti != MAMUTE_INTERP_SINC)
    return fail(ctx, MAMUTE_EINVAL, "time_interp must be 0, 1 or 2");
  if (opts->nt_data < 1 || !(opts->dt_data > 0.f))
    return fail(ctx, MAMUTE_EINVAL, "time_interp needs nt_data >= 1 and dt_data > 0");
  *ntd = opts->nt_data;
  return MAMUTE_OK;
}

// Samples [n0, n1) of the recorded data (internal [nt][ncol] layout) into
// the user's seis[n_rec][nt]: a transpose when every receiver is one node,
// else a transpose to per-node rows followed by the fixed-order sum of each
// receiver's nodes.
int data_to_user(mamute_ctx* ctx, const Plan& P, int n0, int n1, float* seis, cudaStream_t s) {
  if (P.one_node) {
    CK(aux_count(ctx, launch_data_out_range((const float*)ctx->dint.p, (const int*)ctx->colmap.p,
                                            n0, n1, P.nt, P.ncol, seis, s)));
    return MAMUTE_OK;
  }
  CK(aux_count(ctx, launch_data_out_range((const float*)ctx->dint.p, (const int*)ctx->ident.p, n0,
                                          n1, P.nt, P.ncol, (float*)ctx->ecol.p, s)));
  CK(aux_count(ctx, launch_combine((const float*)ctx->ecol.p, (const int*)ctx->rcolptr.p,
                                   (const int*)ctx->rcols.p, P.nrec, n0, n1, P.nt, seis, s)));
  return MAMUTE_OK;
}

// ---- Convolutional PML (Sec. 2, the second absorbing boundary) ----

// Layer coefficients of one padded axis of N cells with `border` layer cells
// at each end, appended to bo / co: b = exp(-(d + alpha) dt) and
// c = d (b - 1) / (d + alpha) with, at depth r = dist / border,
// d = d0 r^2, d0 = -3 vmax ln(R) / (2 border h), alpha = pi f0 (1 - r);
// b = 1, c = 0 outside the layer.  low_face = false: no layer at the low
// end (the top face under a free surface, whose image planes the main step
// kernel forms).
void cpml_profile(int N, int border, double h, double dt, double vmax, double f0, double R,
                  std::vector<float>& bo, std::vector<float>& co, bool low_face = true) {
  const double d0 = border > 0 ? -3.0 * vmax * std::log(R) / (2.0 * border * h) : 0.0;
  for (int i = 0; i < N; ++i) {
    int dist = 0;
    if (i < border) dist = low_face ? border - i : 0;
    else if (i > N - 1 - border) dist = i - (N - 1 - border);
    double b = 1.0, c = 0.0;
    if (dist > 0) {
      const double r = (double)dist / border;
      const double d = d0 * r * r, al = M_PI * f0 * (1.0 - r);
      b = std::exp(-(d + al) * dt);
      if (d + al > 0.0) c = d * (b - 1.0) / (d + al);
    }
    bo.push_back((float)b);
    co.push_back((float)c);
  }
}

// Pools of the CPML memory variables, each P.pool_elems floats in ctx->cpml:
// 0..2 Psi_a, 3..5 Zeta_a (their multipliers in the reverse pass), 6..8 y_a,
// 9..11 z_a (reverse scratch).
constexpr int kPmlPoolsModel = 6, kPmlPoolsGradient = 12;

struct PmlTables {
  CpmlArgs base{};          // buffers and profiles; u, out, tstore, acc set per launch
  CpmlExtent ext{};         // extents of the kernels' grids
};

// Profiles, the data columns' nodes and scales, and the pools (after setup()).
int cpml_setup(mamute_ctx* ctx, const Plan& P, const float* vel, const float* rho, int n_pools,
               PmlTables& T) {
  std::vector<float> bx, cx, by, cy, bz, cz;
  for (const VolDesc& V : P.vols) {
    if ((long long)V.Nx * V.Ny * V.Nz >= (1LL << 32))  // 32-bit shell indexing
      return fail(ctx, MAMUTE_EINVAL, "pml: a shot window of 2^32 points or more");
    cpml_profile(V.Nx, P.b, P.h, P.dt, P.vmax, P.pml_f0, P.pml_r, bx, cx);
    cpml_profile(V.Ny, P.b, P.h, P.dt, P.vmax, P.pml_f0, P.pml_r, by, cy);
    T.ext.xy = std::max(T.ext.xy, (long long)V.Nx * V.Ny);
    T.ext.xz = std::max(T.ext.xz, (long long)V.Nx * V.Nz);
    T.ext.yz = std::max(T.ext.yz, (long long)V.Ny * V.Nz);
  }
  T.ext.border = P.b;
  cpml_profile(P.Nz, P.b, P.h, P.dt, P.vmax, P.pml_f0, P.pml_r, bz, cz, P.zs < 0);
  std::vector<float> all;
  size_t off[6];
  const std::vector<float>* parts[6] = {&bx, &cx, &by, &cy, &bz, &cz};
  for (int k = 0; k < 6; ++k) {
    off[k] = all.size();
    all.insert(all.end(), parts[k]->begin(), parts[k]->end());
  }
  CK(upload(ctx->cprof, all, ctx->stream));
  const float* base = (const float*)ctx->cprof.p;
  // Data columns in the forward tables' order (the layout data_to_user
  // reads), sampled after the memory-variable correction of each step.
  std::vector<int> ent_of_col(P.ncol, 0);
  for (size_t e = 0; e < P.ent.size(); ++e) ent_of_col[P.fwd_col_of_ent[e]] = (int)e;
  std::vector<long long> node(P.ncol), cell(P.ncol);
  std::vector<RecEntry> rec(P.ncol);
  std::vector<float> gval(P.ncol, 1.0f);
  for (int c = 0; c < P.ncol; ++c) {
    const NodeEntry& E = P.ent[ent_of_col[c]];
    const VolDesc& V = P.vols[E.shot];
    node[c] = V.off + ((long long)E.lz * V.Ny + E.ly) * V.pitch + E.lx;
    cell[c] = E.cell;
    rec[c] = RecEntry{};
    rec[c].col = c;
    rec[c].wgt = E.w;
  }
  CK(upload(ctx->cnode, node, ctx->stream));
  CK(upload(ctx->ccell, cell, ctx->stream));
  CK(upload(ctx->crec, rec, ctx->stream));
  CK(upload(ctx->cgval, gval, ctx->stream));
  if (P.ncol > 0) {  // fscale = w sqrt(rho) of the columns
    GeomArgs ga{vel, rho, P.ncol, 0, (const long long*)ctx->ccell.p, (const float*)ctx->cgval.p,
                (RecEntry*)ctx->crec.p, nullptr, nullptr, nullptr, P.h, P.dt};
    CK(aux_count(ctx, launch_geometry(ga, ctx->stream)));
  }
  const size_t pool = (size_t)P.pool_elems * 4;
  CK(ensure(ctx->cpml, (size_t)n_pools * pool));
  CK(cudaMemsetAsync(ctx->cpml.p, 0, (size_t)n_pools * pool, ctx->stream));
  CpmlArgs& c = T.base;
  c.vols = (const VolDesc*)ctx->vols.p;
  c.pr = CpmlProf{base + off[0], base + off[1], base + off[2], base + off[3], base + off[4],
                  base + off[5]};
  c.A = (const float*)ctx->coefA.p;
  c.pitchG = P.pitchG;
  c.NyG = P.Ny;
  for (int k = 0; k < 3; ++k) {
    c.m1[k] = (float*)ctx->cpml.p + (size_t)k * P.pool_elems;
    c.m2[k] = (float*)ctx->cpml.p + (size_t)(3 + k) * P.pool_elems;
    c.y[k] = n_pools > 6 ? (float*)ctx->cpml.p + (size_t)(6 + k) * P.pool_elems : nullptr;
    c.z[k] = n_pools > 6 ? (float*)ctx->cpml.p + (size_t)(9 + k) * P.pool_elems : nullptr;
  }
  return MAMUTE_OK;
}

// One forward CPML step around the main step launch `main` (u^n in u, the
// main kernel writes u^{n+1} to out): the Psi update before it, the Zeta
// update and the correction of u^{n+1} (and of the stored term) after it,
// then the data sample of the step into drow (may be null).
template <typename Main>
int cpml_fwd_step(mamute_ctx* ctx, const Plan& P, const PmlTables& T, const float* u, float* out,
                  float* tstore, float* drow, Main main) {
  CpmlArgs c = T.base;
  c.u = u;
  c.out = out;
  c.tstore = tstore;
  const int nvol = (int)P.vols.size();
  if (ctx->timing && !ctx->ev0_set) {
    CK(cudaEventRecord(ctx->ev0, ctx->stream));
    ctx->ev0_set = true;
  }
  CK(launch_cpml_psi(c, nvol, T.ext, ctx->stream));
  ctx->launches += kCpmlAxisLaunches;
  TRY(main());
  CK(launch_cpml_fcorr(c, nvol, T.ext, ctx->stream));
  ctx->launches += kCpmlAxisLaunches;
  if (drow)
    CK(aux_count(ctx, launch_cpml_record(out, (const long long*)ctx->cnode.p,
                                         (const RecEntry*)ctx->crec.p, P.ncol, drow, ctx->stream)));
  if (ctx->timing) CK(cudaEventRecord(ctx->ev1, ctx->stream));
  return MAMUTE_OK;
}

// host_seis (host, may be NULL): the seismograms also go to this host array,
// segment by segment while later segments of the time loop run.
int run_model(mamute_ctx* ctx, const mamute_grid* g, const float* vel, const float* rho,
              int n_src, const float* src_xyz, const float* wavelet, const int* rec_offset,
              const float* rec_xyz, const mamute_opts* opts, float* seis,
              float* host_seis = nullptr) {
  TRY(check_common(ctx, g, vel, wavelet));
  Plan P;
  TRY(build_plan(ctx, g, rho != nullptr, n_src, src_xyz, rec_offset, rec_xyz,
                 opts ? opts->aperture : nullptr, P, opts ? opts->tiles : nullptr));
  ctx->max_planes = P.Nz;
  if (P.ncol > 0 && !seis) return fail(ctx, MAMUTE_EINVAL, "seis is NULL");
  int ti = 0, ntd = P.nt;
  TRY(check_interp(ctx, g, opts, &ti, &ntd));
  TRY(check_cfl(ctx, P, vel));
  const bool ph = opts && opts->phess;
  if (P.pml && ph) return fail(ctx, MAMUTE_EINVAL, "phess is not available with pml");
  TRY(setup(ctx, P, vel, rho, false, ph));
  PmlTables T;
  if (P.pml) TRY(cpml_setup(ctx, P, vel, rho, kPmlPoolsModel, T));
  const size_t pool = (size_t)P.pool_elems * 4;
  CK(cudaMemsetAsync(ctx->pool[0].p, 0, pool, ctx->stream));
  CK(cudaMemsetAsync(ctx->pool[1].p, 0, pool, ctx->stream));
  if (ph) CK(cudaMemsetAsync(ctx->acc.p, 0, pool, ctx->stream));
  CK(ensure(ctx->dint, (size_t)P.nt * std::max(P.ncol, 1) * 4));
  const int mode = ph ? MODE_FWD_PH : MODE_FWD;
  // Two time levels per launch where the problem allows it.
  const bool pairs = !ph && !P.pml && plan_pairs(ctx, P, opts);
  if (pairs) {
    TRY(setup_pairs(ctx, P, vel, rho));
    CK(cudaMemsetAsync(ctx->pflags.p, 0, P.pitems.size() * 4, ctx->stream));
  }
  // The time loop is captured into a CUDA graph and replayed while the plan,
  // the buffers and the wavelet stay the same (MAMUTE_GRAPHS=0 disables).
  std::vector<unsigned long long> key;
  // Seismograms stream to the host during the loop unless they are resampled
  // to a data time axis first.
  const bool stream_out = host_seis != nullptr && P.ncol > 0 && ti == 0;
  const bool use_graph = env_int("MAMUTE_GRAPHS", 1) != 0 && P.nt >= 8 &&
                         !(pairs && ctx->pair_graph_failed);
  if (use_graph) {
    auto push = [&](const void* p) { key.push_back((unsigned long long)(uintptr_t)p); };
    key.push_back((unsigned long long)P.nt);
    key.push_back((unsigned long long)P.items.size());
    key.push_back(((unsigned long long)P.tx << 32) | (unsigned)P.ty);
    key.push_back((unsigned long long)mode * 2 + P.dens);
    key.push_back((unsigned long long)P.ncol);
    key.push_back((unsigned long long)ctx->max_planes);
    for (const DevBuf* b : {&ctx->items, &ctx->vols, &ctx->maps, &ctx->cmaps, &ctx->gx, &ctx->gy,
                            &ctx->gz, &ctx->recptr, &ctx->rec, &ctx->acc, &ctx->dint,
                            &ctx->pool[0], &ctx->pool[1]})
      push(b->p);
    for (int n = 0; n < P.nt; ++n) {
      unsigned int u;
      std::memcpy(&u, &wavelet[n], 4);
      key.push_back(u);
    }
    key.push_back(pairs ? (((unsigned long long)P.ptx << 32) | (unsigned)P.pty) : 0);
    for (const DevBuf* b : {&ctx->pitems, &ctx->pnbr, &ctx->precptr, &ctx->prec, &ctx->pmaps,
                            &ctx->pflags})
      push(pairs ? b->p : nullptr);
    key.push_back(P.pml ? 1 : 0);
    for (const DevBuf* b : {&ctx->cpml, &ctx->cprof, &ctx->cnode, &ctx->crec})
      push(P.pml ? b->p : nullptr);
    key.push_back(stream_out ? 1 : 0);
    if (stream_out) {
      push(seis);
      push(host_seis);
    }
  }
  // Steps [t0, t1): pairs of steps (n even) by the two-level kernel, the
  // rest one at a time.
  auto run_steps = [&](int t0, int t1) -> int {
    int n = t0;
    while (n < t1) {
      float* drow = (float*)ctx->dint.p + (size_t)n * P.ncol;
      if (pairs && n % 2 == 0 && n + 1 < t1) {
        PairArgs a{};
        a.items = (const WorkItem*)ctx->pitems.p;
        a.nbrs = (const int4*)ctx->pnbr.p;
        a.vols = (const VolDesc*)ctx->vols.p;
        a.pmaps = (const PairMaps*)ctx->pmaps.p;
        a.gx = (const float*)ctx->gx.p;
        a.gy = (const float*)ctx->gy.p;
        a.gz = (const float*)ctx->gz.p;
        a.wn0 = wavelet[n];
        a.wn1 = wavelet[n + 1];
        a.fout1 = (float*)ctx->pool[1].p;
        a.fout2 = (float*)ctx->pool[0].p;
        a.rec_ptr = (const int*)ctx->precptr.p;
        a.rec = (const RecEntry*)ctx->prec.p;
        a.dout0 = P.ncol > 0 ? drow : nullptr;
        a.dout1 = P.ncol > 0 ? drow + P.ncol : nullptr;
        a.flags = (int*)ctx->pflags.p;
        a.epoch = (n / 2) * P.Nz;
        a.status = ctx->status;
        if (ctx->timing && !ctx->ev0_set) {
          CK(cudaEventRecord(ctx->ev0, ctx->stream));
          ctx->ev0_set = true;
        }
        ++ctx->step_launches;
        ++ctx->launches;
        CK(launch_pair(a, (int)P.pitems.size(), P.Nz, P.ptx, P.pty, P.dens, ctx->stream, nullptr));
        if (ctx->timing) CK(cudaEventRecord(ctx->ev1, ctx->stream));
        n += 2;
      } else if (P.pml) {
        StepArgs a = fwd_args(ctx, P, n, wavelet, nullptr, mode);
        TRY(cpml_fwd_step(ctx, P, T, (const float*)ctx->pool[n & 1].p, a.fout, nullptr,
                          P.ncol > 0 ? drow : nullptr, [&]() -> int {
                            CK(step_launch(ctx, a, (int)P.items.size(), P.tx, P.ty, P.dens, mode));
                            return MAMUTE_OK;
                          }));
        n += 1;
      } else {
        StepArgs a = fwd_args(ctx, P, n, wavelet, drow, mode);
        CK(step_launch(ctx, a, (int)P.items.size(), P.tx, P.ty, P.dens, mode));
        n += 1;
      }
    }
    return MAMUTE_OK;
  };
  auto launch_all = [&]() -> int {
    if (!stream_out) return run_steps(0, P.nt);
    // In 8 segments (even boundaries, so pairs do not straddle them): after
    // each, the copy stream transposes that segment's samples and copies them
    // to the host while the next segment runs.
    const int nseg = std::min(P.nt, 8);
    int t0 = 0;
    for (int k = 0; k < nseg; ++k) {
      int t1 = (int)((long long)P.nt * (k + 1) / nseg);
      if (k + 1 < nseg) t1 -= t1 % 2;
      if (t1 <= t0) continue;
      TRY(run_steps(t0, t1));
      CK(cudaEventRecord(ctx->seg_ev[k], ctx->stream));
      CK(cudaStreamWaitEvent(ctx->copy, ctx->seg_ev[k], 0));
      TRY(data_to_user(ctx, P, t0, t1, seis, ctx->copy));
      CK(cudaMemcpy2DAsync(host_seis + t0, (size_t)P.nt * 4, seis + t0, (size_t)P.nt * 4,
                           (size_t)(t1 - t0) * 4, (size_t)P.nrec, cudaMemcpyDeviceToHost,
                           ctx->copy));
      t0 = t1;
    }
    CK(cudaEventRecord(ctx->seg_ev[nseg], ctx->copy));
    CK(cudaStreamWaitEvent(ctx->stream, ctx->seg_ev[nseg], 0));
    return MAMUTE_OK;
  };
  if (stream_out) {
    if (!ctx->copy) CK(cudaStreamCreateWithFlags(&ctx->copy, cudaStreamNonBlocking));
    while ((int)ctx->seg_ev.size() < 9) {
      cudaEvent_t ev = nullptr;
      CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      ctx->seg_ev.push_back(ev);
    }
  }
  if (!use_graph) {
    TRY(launch_all());
  } else {
    if (!ctx->graph || ctx->graph_key != key) {
      if (ctx->graph) {
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
      }
      // Captured on a private stream (the caller's may be the legacy default
      // stream, which cannot be captured); the graph runs on the caller's.
      if (!ctx->capture) CK(cudaStreamCreateWithFlags(&ctx->capture, cudaStreamNonBlocking));
      CK(cudaStreamSynchronize(ctx->stream));
      const bool timing = ctx->timing;
      const long long sl0 = ctx->step_launches, l0 = ctx->launches;
      cudaStream_t user = ctx->stream;
      ctx->timing = false;  // no event records inside the capture
      ctx->stream = ctx->capture;
      cudaGraph_t gr = nullptr;
      cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
      const int rc = e == cudaSuccess ? launch_all() : MAMUTE_OK;
      if (e == cudaSuccess) e = cudaStreamEndCapture(ctx->stream, &gr);
      ctx->stream = user;
      ctx->timing = timing;
      ctx->step_launches = sl0;
      ctx->launches = l0;
      if (e == cudaSuccess && rc == MAMUTE_OK) e = cudaGraphInstantiate(&ctx->graph, gr, 0);
      if (gr) cudaGraphDestroy(gr);
      if (pairs && (rc != MAMUTE_OK || e != cudaSuccess)) {
        // Cooperative launches that cannot be captured: run them directly
        // from now on.
        cudaGetLastError();
        if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
        ctx->graph_key.clear();
        ctx->pair_graph_failed = true;
        ctx->err.clear();
        CK(cudaStreamSynchronize(ctx->stream));
        TRY(launch_all());
        goto loop_done;
      }
      if (rc != MAMUTE_OK) return rc;
      CK(e);
      ctx->graph_key = key;
    }
    if (ctx->timing) CK(cudaEventRecord(ctx->ev0, ctx->stream));
    CK(cudaGraphLaunch(ctx->graph, ctx->stream));
    if (ctx->timing) {
      CK(cudaEventRecord(ctx->ev1, ctx->stream));
      ctx->ev0_set = true;
    }
    const int loop = pairs ? (P.nt / 2 + P.nt % 2) : P.nt;
    ctx->step_launches = loop;
    ctx->launches += loop * (P.pml ? 2 * kCpmlAxisLaunches + (P.ncol > 0 ? 2 : 1) : 1) +
                     (stream_out ? std::min(P.nt, 8) * (P.one_node ? 1 : 2) : 0);
  }
loop_done:
  if (!stream_out) {
    if (ti == 0) {
      TRY(data_to_user(ctx, P, 0, P.nt, seis, ctx->stream));
    } else if (P.ncol > 0) {
      CK(ensure(ctx->dmod, (size_t)P.nrec * P.nt * 4));
      TRY(data_to_user(ctx, P, 0, P.nt, (float*)ctx->dmod.p, ctx->stream));
      TRY(do_resample(ctx, P.nrec, P.nt, P.dt, ntd, opts->dt_data, ti, 0,
                      (const float*)ctx->dmod.p, seis));
    }
    if (host_seis && P.ncol > 0)
      CK(cudaMemcpyAsync(host_seis, seis, (size_t)P.nrec * ntd * 4, cudaMemcpyDeviceToHost,
                         ctx->stream));
  }
  if (ph) {
    FinalizeArgs fa{(const float*)ctx->acc.p, (const VolDesc*)ctx->vols.p, (int)P.vols.size(), vel,
                    P.nx, P.ny, P.nz, P.b, P.dt, 1, 0, opts->phess};
    CK(aux_count(ctx, launch_finalize(fa, ctx->stream)));
  }
  return finish(ctx);
}

// Gradient (residual mode, d_in = d_obs) or transposed Jacobian (d_in = d_res).
int run_gradient(mamute_ctx* ctx, const mamute_grid* g, const float* vel, const float* rho,
                 int n_src, const float* src_xyz, const float* wavelet, const int* rec_offset,
                 const float* rec_xyz, const float* d_in, bool residual_mode,
                 const mamute_opts* opts, double* misfit, float* grad) {
  TRY(check_common(ctx, g, vel, wavelet));
  if (!grad) return fail(ctx, MAMUTE_EINVAL, "grad is NULL");
  Plan P;
  TRY(build_plan(ctx, g, rho != nullptr, n_src, src_xyz, rec_offset, rec_xyz,
                 opts ? opts->aperture : nullptr, P, opts ? opts->tiles : nullptr));
  ctx->max_planes = P.Nz;
  if (P.ncol > 0 && !d_in) return fail(ctx, MAMUTE_EINVAL, "data is NULL");
  int ti = 0, ntd = P.nt;
  TRY(check_interp(ctx, g, opts, &ti, &ntd));
  const int smode = opts ? opts->smooth_mode : 0;
  if (smode < 0 || smode > 2) return fail(ctx, MAMUTE_EINVAL, "smooth_mode must be 0, 1 or 2");
  TRY(check_cfl(ctx, P, vel));
  {
    // When every step's imaging term will be kept (the storage decision
    // below, made here ahead of it on the same figures), choose the adjoint
    // tiles for the stored-term kernel.
    const int ns = opts ? opts->n_snapshots : 0;
    bool keep_all = ns < 0 || P.pml;
    if (ns == 0 && !keep_all) {
      size_t fr = 0, tot = 0;
      CK(cudaMemGetInfo(&fr, &tot));
      const double fr_ = (opts && opts->check_mem > 0.f) ? opts->check_mem : 0.8;
      const double need = (double)P.nt * P.term_elems * 4;
      keep_all = need <= fr_ * ((double)fr + (double)ctx->tstore.bytes + (double)ctx->slots.bytes);
    }
    if (keep_all) {
      Plan Q;
      TRY(build_plan(ctx, g, rho != nullptr, n_src, src_xyz, rec_offset, rec_xyz,
                     opts ? opts->aperture : nullptr, Q, opts ? opts->tiles : nullptr,
                     MODE_ADJ_STORED));
      Q.vmax = P.vmax;
      P = std::move(Q);
      ctx->max_planes = P.Nz;
    }
  }
  const bool ph = opts && opts->phess;
  if (P.pml && ph) return fail(ctx, MAMUTE_EINVAL, "phess is not available with pml");
  if (P.pml && opts && opts->n_snapshots > 0)
    return fail(ctx, MAMUTE_EINVAL,
                "a pml gradient keeps every step's imaging term: n_snapshots must be 0 or -1");
  TRY(setup(ctx, P, vel, rho, true, true));
  PmlTables T;
  if (P.pml) TRY(cpml_setup(ctx, P, vel, rho, kPmlPoolsGradient, T));
  const size_t pool = (size_t)P.pool_elems * 4;
  const size_t ncol = std::max(P.ncol, 1);
  CK(ensure(ctx->dint, (size_t)P.nt * ncol * 4));
  CK(ensure(ctx->rint, (size_t)P.nt * ncol * 4));
  CK(ensure(ctx->partial, (size_t)std::max(misfit_blocks((long long)ntd * P.nrec), 1) * 8));
  for (int i = 0; i < 2; ++i) {
    CK(cudaMemsetAsync(ctx->pool[i].p, 0, pool, ctx->stream));
    CK(cudaMemsetAsync(ctx->psi[i].p, 0, pool, ctx->stream));
  }
  CK(cudaMemsetAsync(ctx->acc.p, 0, pool, ctx->stream));
  CK(cudaMemsetAsync(ctx->misfit.p, 0, 8, ctx->stream));
  // Storage mode.
  const int nsnap = opts ? opts->n_snapshots : 0;
  const double frac = (opts && opts->check_mem > 0.f) ? opts->check_mem : 0.8;
  bool all_mode = nsnap < 0;
  if (nsnap == 0) {
    // Automatic: keep every step's imaging term (no recomputation) when the
    // store fits in check_mem of the free memory, else revolve.
    size_t fr = 0, tot = 0;
    CK(cudaMemGetInfo(&fr, &tot));
    const size_t need = (size_t)P.nt * P.term_elems * 4;
    const double avail = (double)fr + (double)ctx->tstore.bytes + (double)ctx->slots.bytes;
    if ((double)need <= frac * avail) {
      release(ctx->slots);
      if (ensure(ctx->tstore, need) == cudaSuccess)
        all_mode = true;
      else
        cudaGetLastError();
    }
  }
  if (P.pml && !all_mode)
    return fail(ctx, MAMUTE_ENOMEM, "the imaging terms of %d steps (%.2f GB) do not fit", P.nt,
                (double)P.nt * P.term_elems * 4e-9);
  if (!all_mode && ctx->tstore.p) release(ctx->tstore);  // room for the slots
  int slots = 0;
  if (all_mode) {
    CK(ensure(ctx->tstore, (size_t)P.nt * P.term_elems * 4));
    bool pads = false;
    for (const VolDesc& V : P.vols) pads = pads || V.txoff != V.ix0 || V.tpitch != V.nxi;
    if (pads) CK(cudaMemsetAsync(ctx->tstore.p, 0, (size_t)P.nt * P.term_elems * 4, ctx->stream));
    for (size_t s = 0; s < P.vols.size(); ++s) {
      const VolDesc& V = P.vols[s];
      cuuint64_t dims[4] = {(cuuint64_t)V.tpitch, (cuuint64_t)V.nyi, (cuuint64_t)V.nzi,
                            (cuuint64_t)P.nt};
      cuuint64_t strides[3] = {(cuuint64_t)V.tpitch * 4, (cuuint64_t)V.tpitch * V.nyi * 4,
                               (cuuint64_t)P.term_elems * 4};
      cuuint32_t box[4] = {(cuuint32_t)P.atx, (cuuint32_t)P.aty, 1, 1};
      cuuint32_t es[4] = {1, 1, 1, 1};
      if (ctx->encode(&ctx->hmaps[s].m[12], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                      (float*)ctx->tstore.p + V.toff, dims, strides, box, es,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE))
        return fail(ctx, MAMUTE_ECUDA, "cuTensorMapEncodeTiled failed (term store)");
    }
    CK(upload(ctx->maps, ctx->hmaps, ctx->stream));
  } else if (nsnap > 0) {
    slots = std::min(nsnap, P.nt);
  } else {
    size_t fr = 0, tot = 0;
    CK(cudaMemGetInfo(&fr, &tot));
    const double per = 2.0 * (double)pool;
    // Slots this context already holds count as available.
    const double avail = (double)fr + (double)ctx->slots.bytes;
    slots = (int)std::min<double>(std::floor(frac * avail / per), (double)P.nt);
    if (slots < 0) slots = 0;
  }
  // Fewer slots if the allocation fails (fragmentation or a shared device).
  while (!all_mode && slots > 0 && ensure(ctx->slots, (size_t)slots * 2 * pool) != cudaSuccess) {
    cudaGetLastError();
    slots = slots * 3 / 4;
  }
  const int fmode_first = all_mode ? (ph ? MODE_FWD_STORE_PH : MODE_FWD_STORE)
                                    : (ph ? MODE_FWD_PH : MODE_FWD);
  // Buffers of the forward state: the two working pools (slot -1) or the two
  // halves of a checkpoint slot.  A restore only switches the state to the
  // slot's halves; the next step reads them through the slot's own maps and
  // writes to a working pool.
  struct Buf {
    int slot, part;
    bool operator==(const Buf& o) const { return slot == o.slot && part == o.part; }
  };
  const int nvol = (int)P.vols.size();
  if (!all_mode && slots > 0) {
    std::vector<CUtensorMap> sm((size_t)slots * nvol * 6);
    for (int k = 0; k < slots; ++k)
      for (int v = 0; v < nvol; ++v)
        for (int q = 0; q < 2; ++q) {
          const VolDesc& V = P.vols[v];
          const float* base = (const float*)((const char*)ctx->slots.p + ((size_t)k * 2 + q) * pool) + V.off;
          CUtensorMap* m = &sm[((size_t)k * nvol + v) * 6 + q * 3];
          if (encode3d(ctx, m + 0, base, V.Nx, V.Ny, V.Nz, V.pitch, P.tx + 8, P.ty + 8) ||
              encode3d(ctx, m + 1, base, V.Nx, V.Ny, V.Nz, V.pitch, P.tx, P.ty) ||
              encode3d(ctx, m + 2, base, V.Nx, V.Ny, V.Nz, V.pitch, P.atx + 8, P.aty + 8))
            return fail(ctx, MAMUTE_ECUDA, "cuTensorMapEncodeTiled failed (checkpoint slot)");
        }
    CK(upload(ctx->slotmaps, sm, ctx->stream));
  }
  auto buf_ptr = [&](Buf b) -> char* {
    return b.slot < 0 ? (char*)ctx->pool[b.part].p
                      : (char*)ctx->slots.p + ((size_t)b.slot * 2 + b.part) * pool;
  };
  // role 0: forward halo, 1: forward centre, 2: adjoint-box halo
  auto buf_map = [&](Buf b, int role, const CUtensorMap** m, int* stride) {
    if (b.slot < 0) {
      static const int idx[3][2] = {{0, 2}, {1, 3}, {9, 10}};
      *m = shot_map(ctx, idx[role][b.part]);
      *stride = kShotMapStride;
    } else {
      *m = (const CUtensorMap*)ctx->slotmaps.p + ((size_t)b.slot * nvol) * 6 + b.part * 3 + role;
      *stride = 6;
    }
  };
  Buf cur{-1, 0}, prev{-1, 1};  // u^0 and u^{-1}
  int sn = 0;                   // time level held in cur
  int recorded = 0;             // steps whose data sample is recorded
  auto fwd_step = [&](int n, bool first_sweep) -> int {
    const bool rec = first_sweep && n >= recorded;
    const int mode = rec ? fmode_first : MODE_FWD;
    StepArgs a = fwd_args(ctx, P, n, wavelet,
                          (rec && residual_mode) ? (float*)ctx->dint.p + (size_t)n * P.ncol : nullptr,
                          mode);
    Buf out = prev.slot < 0 ? prev : Buf{-1, cur.slot < 0 ? 1 - cur.part : 0};
    buf_map(cur, 0, &a.mF, &a.sF);
    buf_map(prev, 1, &a.mP, &a.sP);
    a.mU = a.mF;
    a.sU = a.sF;
    a.fout = (float*)buf_ptr(out);
    if (P.pml) {
      // the data sample is taken after the memory-variable correction
      float* drow = a.dout;
      a.dout = nullptr;
      TRY(cpml_fwd_step(ctx, P, T, (const float*)buf_ptr(cur), a.fout, a.tstore, drow,
                        [&]() -> int {
                          CK(step_launch(ctx, a, (int)P.items.size(), P.tx, P.ty, P.dens, mode));
                          return MAMUTE_OK;
                        }));
    } else {
      CK(step_launch(ctx, a, (int)P.items.size(), P.tx, P.ty, P.dens, mode));
    }
    if (rec) recorded = n + 1;
    prev = cur;
    cur = out;
    sn = n + 1;
    return MAMUTE_OK;
  };
  // Residual in the adjoint tile's column order: r = d - d_obs (or r = d_res).
  // The forward data are recorded in the forward tile's column order, so they
  // go through the user layout: seis (scratch) = data_out(d_int), then
  // r_int = data_in(seis - d_obs) in the adjoint order.
  auto make_residual = [&]() -> int {
    CK(ensure(ctx->dtmp, (size_t)P.nt * ncol * 4));
    if (ti != 0) {
      // Data on their own time axis: d = K d_model, r = d - d_obs, and the
      // adjoint source on the modelling axis is K^T r.
      CK(ensure(ctx->ddat, (size_t)std::max(P.nrec, 1) * ntd * 4));
      float* dmodel = (float*)ctx->dtmp.p;
      float* ddata = (float*)ctx->ddat.p;
      if (residual_mode) {
        TRY(data_to_user(ctx, P, 0, P.nt, dmodel, ctx->stream));
        TRY(do_resample(ctx, P.nrec, P.nt, P.dt, ntd, opts->dt_data, ti, 0, dmodel, ddata));
        ctx->launches += 3;
        CK(launch_misfit(ddata, d_in, (long long)ntd * P.nrec, (double*)ctx->partial.p,
                         (double*)ctx->misfit.p, ctx->stream));
        CK(launch_sub(ddata, d_in, (long long)ntd * P.nrec, ddata, ctx->stream));
        TRY(do_resample(ctx, P.nrec, P.nt, P.dt, ntd, opts->dt_data, ti, 1, ddata, dmodel));
      } else {
        TRY(do_resample(ctx, P.nrec, P.nt, P.dt, ntd, opts->dt_data, ti, 1, d_in, dmodel));
      }
      CK(aux_count(ctx, launch_data_in(dmodel, (const int*)ctx->acolmap.p, P.nt, P.ncol, nullptr,
                                       -1.0f, (float*)ctx->rint.p, nullptr, nullptr, ctx->stream)));
      return MAMUTE_OK;
    }
    if (residual_mode) {
      TRY(data_to_user(ctx, P, 0, P.nt, (float*)ctx->dtmp.p, ctx->stream));
      // r = seis - d_obs: first r_int = -(-seis) then subtract d_obs.
      CK(aux_count(ctx, launch_data_in((const float*)ctx->dtmp.p, (const int*)ctx->acolmap.p, P.nt, P.ncol,
                        nullptr, -1.0f, (float*)ctx->dint.p, nullptr, nullptr, ctx->stream)));
      CK(aux_count(ctx, launch_data_in(d_in, (const int*)ctx->acolmap.p, P.nt, P.ncol, (const float*)ctx->dint.p,
                        1.0f, (float*)ctx->rint.p, nullptr, nullptr, ctx->stream)));
      // The misfit is summed over the user's [n_rec][nt] layout, so it does
      // not depend on the tile shapes of either propagation.
      ctx->launches += 2;
      CK(launch_misfit((const float*)ctx->dtmp.p, d_in, (long long)P.nt * P.nrec,
                       (double*)ctx->partial.p, (double*)ctx->misfit.p, ctx->stream));
    } else {
      CK(aux_count(ctx, launch_data_in(d_in, (const int*)ctx->acolmap.p, P.nt, P.ncol, nullptr, -1.0f,
                        (float*)ctx->rint.p, nullptr, nullptr, ctx->stream)));
    }
    return MAMUTE_OK;
  };
  auto adj_step = [&](int i) -> int {  // adjoint index k = i + 1, imaging against u^i
    const int k = i + 1;
    StepArgs a{};
    a.items = (const WorkItem*)ctx->aitems.p;
    a.vols = (const VolDesc*)ctx->vols.p;
    a.maps = (const ShotMaps*)ctx->maps.p;
    a.cmaps = (const CoefMaps*)ctx->cmaps.p + 1;
    a.gx = (const float*)ctx->gx.p;
    a.gy = (const float*)ctx->gy.p;
    a.gz = (const float*)ctx->gz.p;
    a.mF = shot_map(ctx, 4 + 2 * ((k + 1) & 1));  // psi^{k+1}, halo
    a.mP = shot_map(ctx, 5 + 2 * (k & 1));        // psi^{k+2}, centre
    a.sF = a.sP = kShotMapStride;
    // u^i: the current level, or the previous one after the final extra step
    const Buf u = (sn == i) ? cur : prev;
    buf_map(u, 2, &a.mU, &a.sU);
    a.wn = 0.f;
    a.fout = (float*)ctx->psi[k & 1].p;
    a.acc = (float*)ctx->acc.p;
    a.tstore = nullptr;
    a.tstep = i;  // the all-states adjoint reads the term of step i through its map
    a.rec_ptr = (const int*)ctx->arecptr.p;
    a.rec = (const RecEntry*)ctx->arec.p;
    a.dout = nullptr;
    a.rin = (const float*)ctx->rint.p + (size_t)i * P.ncol;
    a.status = ctx->status;
    a.zs = P.zs;
    if (P.pml) {  // memory-variable multipliers from psi^{k+1}
      CpmlArgs c = T.base;
      c.u = (const float*)ctx->psi[(k + 1) & 1].p;
      CK(launch_cpml_pre(c, nvol, T.ext, ctx->stream));
      ctx->launches += kCpmlPreLaunches;
    }
    CK(step_launch(ctx, a, (int)P.aitems.size(), P.atx, P.aty, P.dens,
                   all_mode ? MODE_ADJ_STORED : MODE_ADJ));
    if (P.pml) {  // psi^k and the accumulator += the memory-variable part
      CpmlArgs c = T.base;
      c.u = (const float*)ctx->psi[(k + 1) & 1].p;
      c.out = (float*)ctx->psi[k & 1].p;
      c.tstore = (float*)ctx->tstore.p + (size_t)i * P.term_elems;
      c.acc = (float*)ctx->acc.p;
      CK(launch_cpml_acorr(c, nvol, T.ext, ctx->stream));
      ctx->launches += kCpmlAxisLaunches;
      if (ctx->timing) CK(cudaEventRecord(ctx->ev1, ctx->stream));
    }
    return MAMUTE_OK;
  };
  auto begin_adjoint = [&]() -> int {
    TRY(make_residual());
    if (P.pml)  // the memory variables' multipliers start at zero
      CK(cudaMemsetAsync(ctx->cpml.p, 0, (size_t)kPmlPoolsGradient * pool, ctx->stream));
    if (ph) {
      FinalizeArgs fa{(const float*)ctx->acc.p, (const VolDesc*)ctx->vols.p, (int)P.vols.size(),
                      vel, P.nx, P.ny, P.nz, P.b, P.dt, 1, 0, opts->phess};
      CK(aux_count(ctx, launch_finalize(fa, ctx->stream)));
      CK(cudaMemsetAsync(ctx->acc.p, 0, pool, ctx->stream));
    }
    return MAMUTE_OK;
  };
  if (all_mode) {
    for (int n = 0; n < P.nt; ++n) TRY(fwd_step(n, true));
    TRY(begin_adjoint());
    for (int i = P.nt - 1; i >= 0; --i) TRY(adj_step(i));
  } else {
    std::vector<RevAction> acts;
    long long nf = 0;
    revolve_plan(P.nt, slots, acts, nf);
    bool first_reverse = true;
    for (const RevAction& A : acts) {
      switch (A.kind) {
        case REV_ADVANCE:
          for (int n = A.a; n < A.b; ++n) TRY(fwd_step(n, first_reverse));
          break;
        case REV_STORE: {  // slot half (m & 1) holds u^m
          const Buf dc{A.a, sn & 1}, dp{A.a, (sn + 1) & 1};
          if (!(dc == cur))
            CK(cudaMemcpyAsync(buf_ptr(dc), buf_ptr(cur), pool, cudaMemcpyDeviceToDevice, ctx->stream));
          if (!(dp == prev))
            CK(cudaMemcpyAsync(buf_ptr(dp), buf_ptr(prev), pool, cudaMemcpyDeviceToDevice, ctx->stream));
          break;
        }
        case REV_RESTORE:
          if (A.a < 0) {
            CK(cudaMemsetAsync(ctx->pool[0].p, 0, pool, ctx->stream));
            CK(cudaMemsetAsync(ctx->pool[1].p, 0, pool, ctx->stream));
            cur = Buf{-1, 0};
            prev = Buf{-1, 1};
          } else {
            cur = Buf{A.a, A.b & 1};
            prev = Buf{A.a, (A.b + 1) & 1};
          }
          sn = A.b;
          break;
        case REV_REVERSE:
          if (first_reverse) {
            // The last forward step yields the final data sample; u^{nt-1}
            // stays in the previous-level buffer.
            if (recorded < P.nt) TRY(fwd_step(P.nt - 1, true));
            TRY(begin_adjoint());
            first_reverse = false;
          }
          if (!(sn == A.a || sn == A.a + 1)) return fail(ctx, MAMUTE_ECUDA, "checkpoint plan out of step");
          TRY(adj_step(A.a));
          break;
      }
    }
  }
  // MultiplyAdjoint, GradientPreconditioning, ZeroesNearSurface (Algorithm 3).
  const int ztop = opts ? std::max(0, std::min(opts->zero_top_planes, P.nz)) : 0;
  FinalizeArgs fa{(const float*)ctx->acc.p, (const VolDesc*)ctx->vols.p, (int)P.vols.size(), vel,
                  P.nx, P.ny, P.nz, P.b, P.dt, 0, smode ? 0 : ztop, grad};
  CK(aux_count(ctx, launch_finalize(fa, ctx->stream)));
  if (smode) {
    TRY(do_smooth(ctx, P.nx, P.ny, P.nz, P.h, smode, opts->smooth_len, grad, grad));
    if (ztop > 0)
      CK(cudaMemsetAsync(grad, 0, (size_t)ztop * P.nx * P.ny * 4, ctx->stream));
  }
  if (misfit) {
    double J = 0.0;
    CK(cudaMemcpyAsync(&J, ctx->misfit.p, sizeof J, cudaMemcpyDeviceToHost, ctx->stream));
    TRY(finish(ctx));
    *misfit = J;
    return MAMUTE_OK;
  }
  return finish(ctx);
}

// Gauss-Newton diagonal (see gn.cu): forward propagation of each shot storing
// the imaging term, adjoint propagation of a unit data impulse at each
// receiver storing psi, DFT accumulation in blocks of kT steps, Parseval.
int run_gn(mamute_ctx* ctx, const mamute_grid* g, const float* vel, const float* rho, int n_src,
           const float* src_xyz, const float* wavelet, const int* rec_offset, const float* rec_xyz,
           float band_rel, float* hdiag) {
  TRY(check_common(ctx, g, vel, wavelet));
  if (!hdiag) return fail(ctx, MAMUTE_EINVAL, "hdiag is NULL");
  if (!rec_offset || n_src < 1) return fail(ctx, MAMUTE_EINVAL, "no shots");
  const int nr0 = rec_offset[1] - rec_offset[0];
  if (nr0 < 1) return fail(ctx, MAMUTE_EINVAL, "no receivers");
  for (int s = 1; s < n_src; ++s) {
    if (rec_offset[s + 1] - rec_offset[s] != nr0)
      return fail(ctx, MAMUTE_EINVAL, "every shot must record at the same receivers");
    for (int r = 0; r < nr0; ++r)
      for (int d = 0; d < 3; ++d)
        if (rec_xyz[3 * (long long)(rec_offset[s] + r) + d] != rec_xyz[3 * (long long)r + d])
          return fail(ctx, MAMUTE_EINVAL, "every shot must record at the same receivers");
  }
  Plan P;
  TRY(build_plan(ctx, g, rho != nullptr, n_src, src_xyz, rec_offset, rec_xyz, nullptr, P));
  if (P.pml) return fail(ctx, MAMUTE_EINVAL, "the GN diagonal uses the sponge boundary (pml = 0)");
  if (!P.one_node)
    return fail(ctx, MAMUTE_EINVAL, "the Gauss-Newton diagonal needs receivers on grid nodes");
  ctx->max_planes = P.Nz;
  TRY(check_cfl(ctx, P, vel));
  // Compact interior term layout: slot k of the ring is [nz][ny][nx].
  auto compact_terms = [](Plan& Q) {
    long long toff = 0;
    for (VolDesc& V : Q.vols) {
      V.txoff = V.border;
      V.tpitch = V.nxi;
      V.toff = toff;
      toff += (long long)V.nxi * V.nyi * V.nzi;
    }
    Q.term_elems = toff;
  };
  compact_terms(P);
  TRY(setup(ctx, P, vel, rho, true, false));
  // Retained bins of the N_f = 2 nt DFT: where the wavelet spectrum is at
  // least band_rel of its peak (all bins for band_rel <= 0).
  const int nt = P.nt, nf = 2 * nt;
  std::vector<double> mag(nt + 1);
  double mmax = 0.0;
  for (int k = 0; k <= nt; ++k) {
    double re = 0.0, im = 0.0;
    for (int n = 0; n < nt; ++n) {
      const double ph = -2.0 * M_PI * (double)(((long long)k * n) % nf) / nf;
      re += wavelet[n] * std::cos(ph);
      im += wavelet[n] * std::sin(ph);
    }
    mag[k] = std::sqrt(re * re + im * im);
    mmax = std::max(mmax, mag[k]);
  }
  std::vector<int> bins;
  std::vector<float> wts;
  for (int k = 0; k <= nt; ++k)
    if (band_rel <= 0.f || mag[k] >= band_rel * mmax) {
      bins.push_back(k);
      wts.push_back((k == 0 || k == nt) ? 1.0f : 2.0f);
    }
  const int nb = (int)bins.size();
  ctx->dft_n = 0;
  ctx->dft_ms = ctx->dft_macs = 0.0;
  if (nb > dft_max_bins())
    return fail(ctx, MAMUTE_EINVAL, "%d frequency bins exceed the limit %d (raise band_rel)", nb,
                dft_max_bins());
  // Shots are propagated together and receivers B at a time (one unit
  // impulse per shot window), so each batch is one launch per step; the DFT
  // accumulators hold every window of the batch.
  const long long N = (long long)P.nx * P.ny * P.nz;
  // Samples per DFT accumulation: up to 1024 on the tensor cores (the
  // accumulators are read and written once per block; the first block of a
  // batch only writes them), 64 on the FP32 path (its twiddles and samples
  // live in shared memory).  Batches of B windows share each launch.
  // The longest block that still lets a batch hold every shot (fewer, fuller
  // batches matter more for the propagations than block length does for the
  // accumulation).
  // Receivers are batched independently of the shots, as many windows per
  // launch as fit (larger launches propagate faster), in equal batches.
  int kT = 64, B = n_src, Br = nr0;
  {
    size_t fr = 0, tot = 0;
    CK(cudaMemGetInfo(&fr, &tot));
    // buffers this context already holds for the labels count as available
    const double avail = (double)fr + (double)ctx->gnV.bytes + (double)ctx->gnRe.bytes +
                         (double)ctx->gnIm.bytes;
    const double fixed = 2.0 * nb * (double)N * 4.0;  // S and R
    // windows whose samples and accumulators fit in 0.6 of the memory
    auto fit = [&](int t) {
      const double per_vol = ((double)2 * nb + t) * (double)N * 4.0;
      return (int)std::max(1.0, std::min(1e6, std::floor((0.6 * avail - fixed) / per_vol)));
    };
    if (dft_tc_supported(N, nb)) {
      const int want = std::min(n_src, 16);
      kT = 256;
      for (int t : {1024, 512, 256}) {
        const int tt = std::min(t, (nt + 31) / 32 * 32);
        if (fit(tt) >= want) {
          kT = tt;
          break;
        }
      }
    }
    int cap = fit(kT);
    const int env_cap = env_int("MAMUTE_GN_BATCH", 0);  // smaller batches (profiling)
    if (env_cap > 0) cap = std::min(cap, env_cap);
    B = std::min(n_src, cap);
    const int nbr = (nr0 + cap - 1) / cap;
    Br = (nr0 + nbr - 1) / nbr;
    if (env_int("MAMUTE_VERBOSE", 0))
      fprintf(stderr, "mamute gn: %d bins, blocks of %d samples, batches of %d shot and %d receiver "
              "windows (%.1f GB available)\n", nb, kT, B, Br, avail * 1e-9);
  }
  const int Bmax = std::max(B, Br);
  CK(ensure(ctx->gnV, (size_t)kT * Bmax * N * 4));
  CK(ensure(ctx->gnRe, (size_t)nb * Bmax * N * 4));
  CK(ensure(ctx->gnIm, (size_t)nb * Bmax * N * 4));
  CK(ensure(ctx->gnS, (size_t)nb * N * 4));
  CK(ensure(ctx->gnR, (size_t)nb * N * 4));
  CK(ensure(ctx->gnW, std::max((size_t)kT * dft_max_bins() * 8, dft_tc_image_bytes(kT, nb))));
  CK(upload(ctx->gnBins, bins, ctx->stream));
  CK(upload(ctx->gnWts, wts, ctx->stream));
  CK(ensure(ctx->gnRow, (size_t)2 * std::max(P.ncol, 1) * 4));
  CK(cudaMemsetAsync(ctx->gnRe.p, 0, (size_t)nb * Bmax * N * 4, ctx->stream));
  CK(cudaMemsetAsync(ctx->gnIm.p, 0, (size_t)nb * Bmax * N * 4, ctx->stream));
  CK(cudaMemsetAsync(ctx->gnS.p, 0, (size_t)nb * N * 4, ctx->stream));
  CK(cudaMemsetAsync(ctx->gnR.p, 0, (size_t)nb * N * 4, ctx->stream));
  float* V = (float*)ctx->gnV.p;
  float* re = (float*)ctx->gnRe.p;
  float* im = (float*)ctx->gnIm.p;
  const size_t pool = (size_t)P.pool_elems * 4;
  // Item ranges of the windows [v0, v1) (items are grouped by window).
  auto range = [](const std::vector<WorkItem>& items, int v0, int v1, int& b, int& e) {
    b = 0;
    while (b < (int)items.size() && items[b].vol < v0) ++b;
    e = b;
    while (e < (int)items.size() && items[e].vol < v1) ++e;
  };
  // Source side: shots [s0, s1) at once.
  for (int s0 = 0; s0 < n_src; s0 += B) {
    const int s1 = std::min(n_src, s0 + B), nv = s1 - s0;
    const long long Nb = (long long)nv * N;
    int ib, ie;
    range(P.items, s0, s1, ib, ie);
    CK(cudaMemsetAsync(ctx->pool[0].p, 0, pool, ctx->stream));
    CK(cudaMemsetAsync(ctx->pool[1].p, 0, pool, ctx->stream));
    int done = 0;
    auto flush = [&](int upto) -> int {  // DFT of samples [done, upto)
      if (upto > done) {
        CK(dft_launch(ctx, V, Nb, upto - done, done, nf, (const int*)ctx->gnBins.p, nb,
                      (float2*)ctx->gnW.p, re, im));
        done = upto;
      }
      return MAMUTE_OK;
    };
    for (int n = 0; n < nt; ++n) {
      StepArgs a = fwd_args(ctx, P, n, wavelet, nullptr, MODE_FWD_STORE);
      a.items = (const WorkItem*)ctx->items.p + ib;
      a.tstore = V + (size_t)(n % kT) * Nb - (size_t)s0 * N;
      CK(step_launch(ctx, a, ie - ib, P.tx, P.ty, P.dens, MODE_FWD_STORE));
      if ((n + 1) % kT == 0) TRY(flush(n + 1));
    }
    TRY(flush(nt));
    CK(aux_count(ctx, launch_power(nb, N, nv, re, im, (float*)ctx->gnS.p, ctx->stream)));
  }
  // Receiver side: receiver r0 + b of the common set in window b, a unit data
  // impulse at the last sample.  Batches of Br windows: when Br exceeds the
  // shot plan's windows, a plan of Br whole-grid windows that each record
  // the common receiver set (their sources are never fired).
  Plan Pr;
  const Plan* R = &P;
  std::vector<int> roff(rec_offset, rec_offset + n_src + 1);
  if (Br > n_src) {
    std::vector<float> sxyz(3 * (size_t)Br), rxyz(3 * (size_t)Br * nr0);
    roff.assign(Br + 1, 0);
    for (int b = 0; b < Br; ++b) {
      for (int d = 0; d < 3; ++d) sxyz[3 * (size_t)b + d] = src_xyz[d];
      std::copy(rec_xyz, rec_xyz + 3 * (size_t)nr0, rxyz.begin() + 3 * (size_t)b * nr0);
      roff[b + 1] = (b + 1) * nr0;
    }
    TRY(build_plan(ctx, g, rho != nullptr, Br, sxyz.data(), roff.data(), rxyz.data(), nullptr, Pr));
    if (!Pr.one_node || Pr.Nz != P.Nz)
      return fail(ctx, MAMUTE_ECUDA, "receiver plan differs from the shot plan");
    Pr.vmax = P.vmax;
    compact_terms(Pr);
    TRY(setup(ctx, Pr, vel, rho, true, false));
    R = &Pr;
  }
  const size_t rpool = (size_t)R->pool_elems * 4;
  CK(ensure(ctx->gnRow, (size_t)2 * std::max(R->ncol, 1) * 4));
  float* zero_row = (float*)ctx->gnRow.p;
  float* imp_row = zero_row + std::max(R->ncol, 1);
  CK(cudaMemsetAsync(ctx->gnRow.p, 0, (size_t)2 * std::max(R->ncol, 1) * 4, ctx->stream));
  std::vector<int> col_of(R->ncol > 0 ? R->ncol : 1, -1);  // global receiver -> adjoint column
  for (int c = 0; c < R->ncol; ++c) col_of[R->acolmap[c]] = c;
  std::vector<float> row(std::max(R->ncol, 1));
  for (int r0 = 0; r0 < nr0; r0 += Br) {
    const int nv = std::min(Br, nr0 - r0);
    const long long Nb = (long long)nv * N;
    std::fill(row.begin(), row.end(), 0.0f);
    for (int b = 0; b < nv; ++b) row[col_of[roff[b] + r0 + b]] = 1.0f;
    CK(cudaMemcpyAsync(imp_row, row.data(), row.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemsetAsync(ctx->psi[0].p, 0, rpool, ctx->stream));
    CK(cudaMemsetAsync(ctx->psi[1].p, 0, rpool, ctx->stream));
    int ib, ie;
    range(R->aitems, 0, nv, ib, ie);
    int done = 0;
    auto flush = [&](int upto) -> int {
      if (upto > done) {
        CK(dft_launch(ctx, V, Nb, upto - done, done, nf, (const int*)ctx->gnBins.p, nb,
                      (float2*)ctx->gnW.p, re, im));
        done = upto;
      }
      return MAMUTE_OK;
    };
    for (int j = 0; j < nt; ++j) {  // adjoint index k = nt - j holds G[j]
      const int k = nt - j;
      StepArgs a{};
      a.items = (const WorkItem*)ctx->aitems.p + ib;
      a.vols = (const VolDesc*)ctx->vols.p;
      a.maps = (const ShotMaps*)ctx->maps.p;
      a.cmaps = (const CoefMaps*)ctx->cmaps.p + 1;
      a.gx = (const float*)ctx->gx.p;
      a.gy = (const float*)ctx->gy.p;
      a.gz = (const float*)ctx->gz.p;
      a.mF = shot_map(ctx, 4 + 2 * ((k + 1) & 1));  // psi^{k+1}, halo
      a.mP = shot_map(ctx, 5 + 2 * (k & 1));        // psi^{k+2}, centre
      a.mU = a.mF;
      a.sF = a.sP = a.sU = kShotMapStride;
      a.fout = (float*)ctx->psi[k & 1].p;
      a.tstore = V + (size_t)(j % kT) * Nb;
      a.rec_ptr = (const int*)ctx->arecptr.p;
      a.rec = (const RecEntry*)ctx->arec.p;
      a.rin = (j == 0) ? imp_row : zero_row;
      a.status = ctx->status;
      a.zs = R->zs;
      CK(step_launch(ctx, a, ie - ib, R->atx, R->aty, R->dens, MODE_ADJ_TERM));
      if ((j + 1) % kT == 0) TRY(flush(j + 1));
    }
    TRY(flush(nt));
    CK(aux_count(ctx, launch_power(nb, N, nv, re, im, (float*)ctx->gnR.p, ctx->stream)));
    CK(cudaStreamSynchronize(ctx->stream));  // the host impulse row is reused
  }
  CK(aux_count(ctx, launch_assemble(N, nb, (const float*)ctx->gnWts.p, (const float*)ctx->gnR.p,
                                    (const float*)ctx->gnS.p, vel, P.dt, nf, hdiag, ctx->stream)));
  TRY(finish(ctx));
  for (int i = 0; i < ctx->dft_n; ++i) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ctx->dft_ev[2 * i], ctx->dft_ev[2 * i + 1]));
    ctx->dft_ms += ms;
  }
  return MAMUTE_OK;
}

}  // namespace

extern "C" {

const char* mamute_strerror(int code) {
  switch (code) {
    case MAMUTE_OK: return "ok";
    case MAMUTE_EINVAL: return "invalid argument";
    case MAMUTE_ECFL: return "CFL stability condition violated";
    case MAMUTE_ENOMEM: return "out of device memory";
    case MAMUTE_ECUDA: return "CUDA error";
    case MAMUTE_ETIMEOUT: return "device-side wait timed out";
    case MAMUTE_EARCH: return "device is not sm_103";
  }
  return "unknown error";
}

const char* mamute_last_error(const mamute_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

double mamute_cfl_limit(void) { return cfl_bound(); }

int mamute_ctx_set_timing(mamute_ctx* ctx, int enable) {
  if (!ctx) return MAMUTE_EINVAL;
  if (enable && !ctx->ev0) {
    cudaSetDevice(ctx->device);
    if (cudaEventCreate(&ctx->ev0) != cudaSuccess || cudaEventCreate(&ctx->ev1) != cudaSuccess)
      return fail(ctx, MAMUTE_ECUDA, "cudaEventCreate failed");
  }
  ctx->timing = enable != 0;
  return MAMUTE_OK;
}

int mamute_ctx_last_timing(const mamute_ctx* ctx, double* loop_ms, long long* step_launches,
                           long long* total_launches) {
  if (!ctx) return MAMUTE_EINVAL;
  if (loop_ms) *loop_ms = ctx->loop_ms;
  if (step_launches) *step_launches = ctx->step_launches;
  if (total_launches) *total_launches = ctx->launches;
  return MAMUTE_OK;
}

int mamute_ctx_dft_timing(const mamute_ctx* ctx, double* dft_ms, long long* dft_launches,
                          double* complex_macs) {
  if (!ctx) return MAMUTE_EINVAL;
  if (dft_ms) *dft_ms = ctx->dft_ms;
  if (dft_launches) *dft_launches = ctx->dft_n;
  if (complex_macs) *complex_macs = ctx->dft_macs;
  return MAMUTE_OK;
}

int mamute_ctx_create(mamute_ctx** out, int device, void* stream) {
  if (!out) return MAMUTE_EINVAL;
  *out = nullptr;
  int cc_major = 0, cc_minor = 0;
  if (cudaSetDevice(device) != cudaSuccess) return MAMUTE_ECUDA;
  if (cudaDeviceGetAttribute(&cc_major, cudaDevAttrComputeCapabilityMajor, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&cc_minor, cudaDevAttrComputeCapabilityMinor, device) != cudaSuccess)
    return MAMUTE_ECUDA;
  if (cc_major != 10 || cc_minor != 3) return MAMUTE_EARCH;
  mamute_ctx* ctx = new mamute_ctx();
  ctx->device = device;
  ctx->stream = (cudaStream_t)stream;
  cudaDriverEntryPointQueryResult q;
  void* fn = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
          cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    delete ctx;
    return MAMUTE_ECUDA;
  }
  ctx->encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  if (cudaMalloc(&ctx->status, 256) != cudaSuccess || cudaMalloc(&ctx->maxbits, 256) != cudaSuccess ||
      ensure(ctx->misfit, 256) != cudaSuccess) {
    mamute_ctx_destroy(ctx);
    return MAMUTE_ENOMEM;
  }
  *out = ctx;
  return MAMUTE_OK;
}

void mamute_ctx_destroy(mamute_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  DevBuf* all[] = {&ctx->coefA, &ctx->coefM, &ctx->srho, &ctx->pool[0], &ctx->pool[1], &ctx->psi[0],
                   &ctx->psi[1], &ctx->acc, &ctx->slots, &ctx->tstore, &ctx->dint, &ctx->rint, &ctx->dtmp,
                   &ctx->partial, &ctx->misfit, &ctx->items, &ctx->vols, &ctx->maps, &ctx->cmaps,
                   &ctx->recptr, &ctx->rec, &ctx->colmap, &ctx->gx, &ctx->gy, &ctx->gz,
                   &ctx->cells, &ctx->gvals, &ctx->srccell, &ctx->aitems, &ctx->arecptr,
                   &ctx->arec, &ctx->acolmap, &ctx->acells, &ctx->agvals, &ctx->hvel,
                   &ctx->hrho, &ctx->hseis, &ctx->hobs, &ctx->hgrad, &ctx->hphess,
                   &ctx->gnV, &ctx->gnRe, &ctx->gnIm, &ctx->gnS, &ctx->gnR, &ctx->gnW,
                   &ctx->gnBins, &ctx->gnWts, &ctx->gnRow, &ctx->nnPartial, &ctx->nnLoss,
                   &ctx->slotmaps, &ctx->ident, &ctx->rcolptr, &ctx->rcols, &ctx->ecol,
                   &ctx->srcw, &ctx->smA, &ctx->smMat, &ctx->smLam, &ctx->rsPtr, &ctx->rsCol,
                   &ctx->rsW, &ctx->dmod, &ctx->ddat, &ctx->pitems, &ctx->pnbr, &ctx->precptr,
                   &ctx->prec, &ctx->pcells, &ctx->pgvals, &ctx->pmaps, &ctx->pflags,
                   &ctx->cpml, &ctx->cprof, &ctx->cnode, &ctx->crec, &ctx->ccell, &ctx->cgval};
  for (DevBuf* b : all) release(*b);
  if (ctx->status) cudaFree(ctx->status);
  if (ctx->maxbits) cudaFree(ctx->maxbits);
  for (cudaEvent_t ev : ctx->dft_ev) cudaEventDestroy(ev);
  if (ctx->ev0) cudaEventDestroy(ctx->ev0);
  if (ctx->ev1) cudaEventDestroy(ctx->ev1);
  if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
  if (ctx->capture) cudaStreamDestroy(ctx->capture);
  if (ctx->copy) cudaStreamDestroy(ctx->copy);
  for (cudaEvent_t ev : ctx->seg_ev) cudaEventDestroy(ev);
  delete ctx;
}

int mamute_model(mamute_ctx* ctx, const mamute_grid* grid, const float* vel, const float* rho,
                 int n_src, const float* src_xyz, const float* wavelet, const int* rec_offset,
                 const float* rec_xyz, const mamute_opts* opts, float* seis) {
  return run_model(ctx, grid, vel, rho, n_src, src_xyz, wavelet, rec_offset, rec_xyz, opts, seis);
}

int mamute_gradient(mamute_ctx* ctx, const mamute_grid* grid, const float* vel, const float* rho,
                    int n_src, const float* src_xyz, const float* wavelet, const int* rec_offset,
                    const float* rec_xyz, const float* d_obs, const mamute_opts* opts,
                    double* misfit, float* grad) {
  return run_gradient(ctx, grid, vel, rho, n_src, src_xyz, wavelet, rec_offset, rec_xyz, d_obs,
                      true, opts, misfit, grad);
}

int mamute_adjoint(mamute_ctx* ctx, const mamute_grid* grid, const float* vel, const float* rho,
                   int n_src, const float* src_xyz, const float* wavelet, const int* rec_offset,
                   const float* rec_xyz, const float* d_res, const mamute_opts* opts, float* grad) {
  return run_gradient(ctx, grid, vel, rho, n_src, src_xyz, wavelet, rec_offset, rec_xyz, d_res,
                      false, opts, nullptr, grad);
}

int mamute_model_host(mamute_ctx* ctx, const mamute_grid* g, const float* vel, const float* rho,
                      int n_src, const float* src_xyz, const float* wavelet, const int* rec_offset,
                      const float* rec_xyz, const mamute_opts* opts, float* seis) {
  if (!ctx || !g || !vel || !rec_offset || n_src < 1) return MAMUTE_EINVAL;
  TRY(check_common(ctx, g, vel, wavelet));
  int ti = 0, ntd = g->nt;
  TRY(check_interp(ctx, g, opts, &ti, &ntd));
  const size_t nm = (size_t)g->nx * g->ny * g->nz * 4;
  const size_t ns = (size_t)rec_offset[n_src] * ntd * 4;
  CK(ensure(ctx->hvel, nm));
  CK(cudaMemcpyAsync(ctx->hvel.p, vel, nm, cudaMemcpyHostToDevice, ctx->stream));
  if (rho) {
    CK(ensure(ctx->hrho, nm));
    CK(cudaMemcpyAsync(ctx->hrho.p, rho, nm, cudaMemcpyHostToDevice, ctx->stream));
  }
  CK(ensure(ctx->hseis, ns));
  mamute_opts o{};
  if (opts) o = *opts;
  if (opts && opts->phess) {
    CK(ensure(ctx->hphess, nm));
    o.phess = (float*)ctx->hphess.p;
  }
  if (ns && !seis) return fail(ctx, MAMUTE_EINVAL, "seis is NULL");
  TRY(run_model(ctx, g, (const float*)ctx->hvel.p, rho ? (const float*)ctx->hrho.p : nullptr, n_src,
                src_xyz, wavelet, rec_offset, rec_xyz, opts ? &o : nullptr, (float*)ctx->hseis.p,
                seis));
  if (opts && opts->phess)
    CK(cudaMemcpyAsync(opts->phess, ctx->hphess.p, nm, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return MAMUTE_OK;
}

int mamute_gradient_host(mamute_ctx* ctx, const mamute_grid* g, const float* vel, const float* rho,
                         int n_src, const float* src_xyz, const float* wavelet,
                         const int* rec_offset, const float* rec_xyz, const float* d_obs,
                         const mamute_opts* opts, double* misfit, float* grad) {
  if (!ctx || !g || !vel || !rec_offset || n_src < 1 || !grad) return MAMUTE_EINVAL;
  TRY(check_common(ctx, g, vel, wavelet));
  int ti = 0, ntd = g->nt;
  TRY(check_interp(ctx, g, opts, &ti, &ntd));
  const size_t nm = (size_t)g->nx * g->ny * g->nz * 4;
  const size_t ns = (size_t)rec_offset[n_src] * ntd * 4;
  CK(ensure(ctx->hvel, nm));
  CK(cudaMemcpyAsync(ctx->hvel.p, vel, nm, cudaMemcpyHostToDevice, ctx->stream));
  if (rho) {
    CK(ensure(ctx->hrho, nm));
    CK(cudaMemcpyAsync(ctx->hrho.p, rho, nm, cudaMemcpyHostToDevice, ctx->stream));
  }
  CK(ensure(ctx->hobs, ns));
  if (ns) CK(cudaMemcpyAsync(ctx->hobs.p, d_obs, ns, cudaMemcpyHostToDevice, ctx->stream));
  CK(ensure(ctx->hgrad, nm));
  mamute_opts o{};
  if (opts) o = *opts;
  if (opts && opts->phess) {
    CK(ensure(ctx->hphess, nm));
    o.phess = (float*)ctx->hphess.p;
  }
  TRY(run_gradient(ctx, g, (const float*)ctx->hvel.p, rho ? (const float*)ctx->hrho.p : nullptr,
                   n_src, src_xyz, wavelet, rec_offset, rec_xyz, (const float*)ctx->hobs.p, true,
                   opts ? &o : nullptr, misfit, (float*)ctx->hgrad.p));
  CK(cudaMemcpyAsync(grad, ctx->hgrad.p, nm, cudaMemcpyDeviceToHost, ctx->stream));
  if (opts && opts->phess)
    CK(cudaMemcpyAsync(opts->phess, ctx->hphess.p, nm, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return MAMUTE_OK;
}

int mamute_gn_diagonal(mamute_ctx* ctx, const mamute_grid* grid, const float* vel,
                       const float* rho, int n_src, const float* src_xyz, const float* wavelet,
                       const int* rec_offset, const float* rec_xyz, float band_rel, float* hdiag) {
  return run_gn(ctx, grid, vel, rho, n_src, src_xyz, wavelet, rec_offset, rec_xyz, band_rel, hdiag);
}

// ------------------------------------------------------------ network kernels
static int nn_begin(mamute_ctx* ctx) {
  if (!ctx) return MAMUTE_EINVAL;
  ctx->err.clear();
  CK(cudaSetDevice(ctx->device));
  return MAMUTE_OK;
}

static int nn_end(mamute_ctx* ctx) {
  CK(cudaStreamSynchronize(ctx->stream));
  return MAMUTE_OK;
}

// TMA map over a [D][H][W][16] BF16 activation (innermost first: channels,
// x, y, z) with the 32-byte swizzle and zero fill outside.
static CUresult encode_act(mamute_ctx* ctx, CUtensorMap* m, const void* p, int D, int H, int W,
                           const unsigned (&box)[4]) {
  cuuint64_t dims[4] = {16, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D};
  cuuint64_t strides[3] = {32, (cuuint64_t)W * 32, (cuuint64_t)W * H * 32};
  cuuint32_t cbox[4] = {box[0], box[1], box[2], box[3]};
  cuuint32_t es[4] = {1, 1, 1, 1};
  return ctx->encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(p), dims, strides,
                     cbox, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

// As nn_end, for kernels with bounded device-side waits.
static int nn_end_status(mamute_ctx* ctx) {
  int st = 0;
  CK(cudaMemcpyAsync(&st, ctx->status, sizeof st, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (st & kErrTimeout) return fail(ctx, MAMUTE_ETIMEOUT, "a device-side wait ran out");
  return MAMUTE_OK;
}

int mamute_conv3d(mamute_ctx* ctx, int D, int H, int W, const unsigned short* x,
                  const unsigned short* w, const float* bias, int relu,
                  const unsigned short* mask, float* y32, unsigned short* y16) {
  TRY(nn_begin(ctx));
  if (D < 1 || H < 1 || W < 1 || !x || !w || (!y32 && !y16))
    return fail(ctx, MAMUTE_EINVAL, "conv3d: bad arguments");
  if ((uintptr_t)x % 16 || (uintptr_t)w % 16)
    return fail(ctx, MAMUTE_EINVAL, "conv3d: x and w must be 16-byte aligned");
  ConvArgs a{x, w, bias, relu, mask, y32, y16, D, H, W};
  if ((uintptr_t)mask % 16 || (uintptr_t)y32 % 16 || (uintptr_t)y16 % 16)
    return fail(ctx, MAMUTE_EINVAL, "conv3d: mask and outputs must be 16-byte aligned");
  // halo rows as long boxes of 8-byte elements, no swizzle (the kernel
  // applies the operand swizzle in shared memory)
  CUtensorMap xmap;
  unsigned box[4];
  conv_halo_box(D, H, W, box);
  {
    cuuint64_t dims[3] = {(cuuint64_t)W * 4, (cuuint64_t)H, (cuuint64_t)D};
    cuuint64_t strides[2] = {(cuuint64_t)W * 32, (cuuint64_t)W * H * 32};
    cuuint32_t cbox[3] = {box[0], box[1], box[2]};
    cuuint32_t es[3] = {1, 1, 1};
    if (ctx->encode(&xmap, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<unsigned short*>(x), dims,
                    strides, cbox, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE))
      return fail(ctx, MAMUTE_ECUDA, "conv3d: cuTensorMapEncodeTiled failed");
  }
  CK(cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream));
  CK(launch_conv(a, xmap, ctx->status, ctx->stream));
  return nn_end_status(ctx);
}

int mamute_conv3d_wgrad(mamute_ctx* ctx, int D, int H, int W, const unsigned short* x,
                        const unsigned short* gy, float* gw, float* gb) {
  TRY(nn_begin(ctx));
  if (D < 1 || H < 1 || W < 1 || !x || !gy || !gw || !gb)
    return fail(ctx, MAMUTE_EINVAL, "conv3d_wgrad: bad arguments");
  if ((uintptr_t)x % 16 || (uintptr_t)gy % 16)
    return fail(ctx, MAMUTE_EINVAL, "conv3d_wgrad: x and gy must be 16-byte aligned");
  CK(ensure(ctx->nnPartial, wgrad_partial_floats() * 4));
  WgradArgs a{x, gy, (float*)ctx->nnPartial.p, D, H, W};
  CUtensorMap xmap, gmap;
  unsigned hbox[4], gbox[4];
  conv_wgrad_halo_box(hbox);
  conv_gy_box(gbox);
  if (encode_act(ctx, &xmap, x, D, H, W, hbox) || encode_act(ctx, &gmap, gy, D, H, W, gbox))
    return fail(ctx, MAMUTE_ECUDA, "conv3d_wgrad: cuTensorMapEncodeTiled failed");
  CK(cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream));
  CK(launch_wgrad(a, xmap, gmap, ctx->status, gw, gb, ctx->stream));
  return nn_end_status(ctx);
}

int mamute_conv3d_pack(mamute_ctx* ctx, const float* w, unsigned short* fwd,
                       unsigned short* bwd) {
  TRY(nn_begin(ctx));
  if (!w || !fwd) return fail(ctx, MAMUTE_EINVAL, "conv3d_pack: bad arguments");
  CK(launch_pack(w, fwd, bwd, ctx->stream));
  return nn_end(ctx);
}

int mamute_mse_loss(mamute_ctx* ctx, long long n, const float* out, const float* target,
                    const float* mask, double n_mask, double* loss, unsigned short* gy) {
  TRY(nn_begin(ctx));
  if (n < 1 || !out || !target || !gy || !(n_mask > 0))
    return fail(ctx, MAMUTE_EINVAL, "mse_loss: bad arguments");
  CK(ensure(ctx->nnPartial, std::max<size_t>(wgrad_partial_floats() * 4, (size_t)mse_blocks() * 8)));
  CK(ensure(ctx->nnLoss, 256));
  CK(launch_mse(n, out, target, mask, n_mask, gy, (double*)ctx->nnPartial.p,
                (double*)ctx->nnLoss.p, ctx->stream));
  if (loss) {
    double L = 0.0;
    CK(cudaMemcpyAsync(&L, ctx->nnLoss.p, 8, cudaMemcpyDeviceToHost, ctx->stream));
    TRY(nn_end(ctx));
    *loss = L;
    return MAMUTE_OK;
  }
  return nn_end(ctx);
}

int mamute_adam(mamute_ctx* ctx, int n, float* p, float* m, float* v, const float* g, float lr,
                float beta1, float beta2, float eps, int step) {
  TRY(nn_begin(ctx));
  if (n < 1 || !p || !m || !v || !g || step < 1)
    return fail(ctx, MAMUTE_EINVAL, "adam: bad arguments");
  CK(launch_adam(n, p, m, v, g, lr, beta1, beta2, eps, step, ctx->stream));
  return nn_end(ctx);
}

int mamute_nn_features(mamute_ctx* ctx, long long n, const float* vel, const float* phess,
                       const float* hdiag, float v_ref, float v_scale, float log_clip,
                       unsigned short* x16, float* target, float* pmax) {
  TRY(nn_begin(ctx));
  if (n < 1 || !vel || !phess || !x16 || !(v_scale > 0.f) || !(log_clip > 0.f))
    return fail(ctx, MAMUTE_EINVAL, "nn_features: bad arguments");
  CK(launch_features(n, vel, phess, hdiag, ctx->maxbits, v_ref, v_scale, log_clip, x16, target,
                     ctx->stream));
  if (pmax) {
    unsigned int bits = 0;
    CK(cudaMemcpyAsync(&bits, ctx->maxbits, 4, cudaMemcpyDeviceToHost, ctx->stream));
    TRY(nn_end(ctx));
    std::memcpy(pmax, &bits, 4);
    return MAMUTE_OK;
  }
  return nn_end(ctx);
}

int mamute_smooth(mamute_ctx* ctx, int nx, int ny, int nz, float h, int mode,
                  const float* lengths, const float* in, float* out) {
  TRY(nn_begin(ctx));
  if (nx < 1 || ny < 1 || nz < 1 || !(h > 0.f) || mode < 0 || mode > 2 || !in || !out)
    return fail(ctx, MAMUTE_EINVAL, "smooth: bad arguments");
  TRY(do_smooth(ctx, nx, ny, nz, h, mode, lengths, in, out));
  return nn_end(ctx);
}

int mamute_resample(mamute_ctx* ctx, int n_traces, int nt_in, float dt_in, int nt_out,
                    float dt_out, int mode, int adjoint, const float* x, float* y) {
  TRY(nn_begin(ctx));
  TRY(do_resample(ctx, n_traces, nt_in, dt_in, nt_out, dt_out, mode, adjoint, x, y));
  return nn_end(ctx);
}

int mamute_revolve_plan(int nt, int n_slots, long long* n_forward, int* n_actions, int* actions) {
  if (nt < 1 || n_slots < 0 || !n_forward || !n_actions) return MAMUTE_EINVAL;
  std::vector<RevAction> acts;
  long long nf = 0;
  if (revolve_plan(nt, n_slots, acts, nf)) return MAMUTE_EINVAL;
  *n_forward = nf;
  if (actions) {
    const int cap = *n_actions;
    for (int i = 0; i < (int)acts.size() && i < cap; ++i) {
      actions[3 * i] = acts[i].kind;
      actions[3 * i + 1] = acts[i].a;
      actions[3 * i + 2] = acts[i].b;
    }
  }
  *n_actions = (int)acts.size();
  return MAMUTE_OK;
}

}  // extern "C"
