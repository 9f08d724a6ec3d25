/*
 * mamute.h - C ABI of the GB300-native Mamute hot path.
 *
 * The library computes, on one sm_103a GPU, the three steps the paper builds
 * its modelling and FWI on:
 *   - the 3-D acoustic finite-difference propagator of Eq. 1 (second order in
 *     time, eighth order in space, optional variable-density term), with the
 *     damping absorbing boundary, source injection and receiver sampling
 *     (Sec. 2.1; Table 1: ModelingStep, ReadReceiver; Algorithm 1);
 *   - the adjoint wavefield driven by data residuals and the zero-lag
 *     cross-correlation imaging condition, summed over shots into the
 *     gradient of the misfit (Algorithm 3; Sec. 2.1, adjoint-state method);
 *   - optimal checkpointing of the forward wavefield (Sec. 2.1, third
 *     wavefield-management mode; check_mem of Table 4).
 *
 * Conventions shared by every call
 *   Grid       Model arrays are [nz][ny][nx] float32, x fastest (Sec. 2.2.2,
 *              "z x y x x").  A sponge of `border` cells is added outside the
 *              model on all six faces; the model is edge-replicated into it.
 *              Spacing is isotropic (h).  The wavefield is zero outside the
 *              padded grid.
 *   Sources    One wavelet w[nt] shared by all shots (Sec. 2.2.2, source.bin),
 *              injected at the nearest node: u^{n+1}(x_s) += dt^2 w[n] /
 *              (h^3 sqrt(rho(x_s))).
 *   Receivers  Shot s owns receivers rec_offset[s] .. rec_offset[s+1]-1,
 *              coordinates (x, y, z) in metres from (ox, oy, oz), nearest
 *              node; sample n records p = sqrt(rho) u^{n+1} (Sec. 2.2.2:
 *              traces are [n_rec][ns], trace-major).
 *   Memory     Arrays named "device" are device pointers owned by the caller
 *              (e.g. torch tensors) on the context's device; arrays named
 *              "host" are host pointers.  The library owns only its context
 *              scratch (wavefields, checkpoints, tables), grown on demand and
 *              freed by mamute_ctx_destroy.  Nothing is retained from caller
 *              buffers after a call returns.
 *   Streams    Work is issued on the stream given to mamute_ctx_create; every
 *              compute call synchronises that stream before returning, so its
 *              outputs are ready when it returns.
 *   Errors     Every int-returning call returns MAMUTE_OK (0) or a negative
 *              MAMUTE_E* code; no exception or abort crosses the ABI.
 *              mamute_last_error() gives a one-line description of the last
 *              failure on a context.  A context is used by one host thread at
 *              a time.
 */
#ifndef MAMUTE_H
#define MAMUTE_H

#ifdef __cplusplus
extern "C" {
#endif

#define MAMUTE_OK 0
#define MAMUTE_EINVAL (-1)   /* bad dimensions, null pointer, point outside the model */
#define MAMUTE_ECFL (-2)     /* max(c) dt / h above the stability bound 0.4529 */
#define MAMUTE_ENOMEM (-3)   /* device allocation failed */
#define MAMUTE_ECUDA (-4)    /* a CUDA runtime or driver call failed */
#define MAMUTE_ETIMEOUT (-5) /* a bounded device-side wait ran out */
#define MAMUTE_EARCH (-6)    /* the device is not compute capability 10.3 */

typedef struct mamute_ctx mamute_ctx;

/* Grid and time axis (Table 2: nx, ny, nz, dx=dy=dz, border, ox, oy, oz, ns,
 * dt).  cerjan is the Cerjan damping constant alpha of the sponge profile
 * g(d) = exp(-(alpha d)^2), d = depth into the sponge in cells (Sec. 2.1,
 * damping boundary); 0 disables damping.
 * free_surface (Sec. 2, modelling options): 1 makes the top model plane
 * (z = oz) a pressure-release surface by the image method: the field is odd
 * about that plane (the planes above it read as the negated planes below it)
 * and zero on it, and the top face has no sponge; needs nz >= 5, and sources
 * and receivers must lie below the surface.  0: sponge on all six faces.
 * xyz_interp: 0 puts sources and receivers at their nearest node; 1 uses
 * the trilinear weights w_e of the 8 nodes of the cell holding the point:
 * the source adds w_e dt^2 w[n] / (h^3 sqrt(rho_e)) at each node and a
 * receiver records sum_e w_e sqrt(rho_e) u_e (nodes with zero weight or on a
 * free surface are skipped; every node with non-zero weight must lie in the
 * model, or the shot's aperture).
 * pml (Sec. 2, the convolutional PML absorbing boundary): 1 replaces the
 * sponge by a convolutional perfectly matched layer on the `border` cells of
 * every face of each shot's window (cerjan is then ignored).  Each
 * derivative d/dx_a is divided by s_a = 1 + d_a / (alpha_a + i w) in the
 * layer, carried by two memory variables per axis updated by recursive
 * convolution; at depth r = (cells into the layer) / border,
 * d_a = -3 vmax ln(pml_r) r^2 / (2 border h) and alpha_a = pi pml_f0 (1 - r),
 * vmax = max(vel).  pml_f0 is the source's dominant frequency in Hz (>= 0)
 * and pml_r the nominal reflection coefficient in (0, 1) (0 selects 1e-3).
 * With free_surface the top face has no layer (the surface's image method
 * holds there) and the other five faces have it.  A pml gradient keeps the
 * imaging term of every step (n_snapshots 0 or -1; ENOMEM when that store
 * does not fit) and takes no phess; mamute_gn_diagonal with pml is EINVAL.
 * 0: the sponge. */
typedef struct {
  int nx, ny, nz;
  int border;
  float h;
  float dt;
  int nt;
  float ox, oy, oz;
  float cerjan;
  int free_surface;
  int xyz_interp;
  int pml;
  float pml_f0;
  float pml_r;
} mamute_grid;

/* Options (Table 4 check_mem; Sec. 3 zeroes_nplanes_gradient).
 *   check_mem       fraction (0,1] of free device memory that the stored
 *                   states may use when n_snapshots == 0 (default 0.8).
 *   n_snapshots     0: automatic: keep the imaging term of every step when
 *                   nt x (interior points) x 4 bytes fits in check_mem of
 *                   the free memory, else as many revolve
 *                   slots as check_mem allows; >0: exactly that many revolve
 *                   slots; -1: keep the imaging term of every step (no
 *                   recomputation).
 *   zero_top_planes ZeroesNearSurface: gradient planes z < this are zeroed.
 *   aperture        host [n_src][4] or NULL: shot s propagates only over the
 *                   model columns x in [a0, a1), y in [a2, a3) plus the sponge
 *                   around them (cells of the global padded grid, so the
 *                   sponge of an interior aperture sees the true model); a0
 *                   must be a multiple of 4.  NULL: every shot uses the whole
 *                   grid.
 *   phess           device [nz][ny][nx] or NULL: receives the pseudo-Hessian
 *                   sum_s sum_n (g (lap - m2) u_s^n)^2 of the forward pass
 *                   (overwritten).
 *   tiles           work decomposition of the time-step kernels: {forward tile
 *                   width, height, z blocks, adjoint tile width, height, z
 *                   blocks}; 0 entries are chosen by the library's cost model
 *                   (an autotuner may pass measured choices; the result does
 *                   not depend on them).  An unsupported shape is EINVAL.
 *   smooth_mode     gradient preconditioning (Sec. 2, FWI parameters; Algorithm
 *                   3 GradientPreconditioning, applied after MultiplyAdjoint and
 *                   before ZeroesNearSurface): 0 none, 1 Bessel filter, 2
 *                   Laplace filter (see mamute_smooth).
 *   smooth_len      filter lengths lx, ly, lz in metres; 0 entries mean 2 h.
 *   time_interp     0: data (seis, d_obs, d_res) are on the modelling time axis
 *                   [n_rec][nt]; 1 (nearest) or 2 (sinc): they are on a data
 *                   axis of nt_data samples of dt_data seconds, and the
 *                   modelled traces are resampled to it (Sec. 2, time
 *                   interpolation; see mamute_resample); the residual is
 *                   brought back by the transposed resampling.
 *   nt_data, dt_data  the data time axis when time_interp != 0.
 *   time_blocking   mamute_model only: 2 advances two time steps per launch
 *                   with the two-level kernel (one shot, no free surface, no
 *                   pseudo-Hessian, every tile resident on its own SM; the
 *                   seismograms are bitwise those of one step per launch);
 *                   0 or 1: one step per launch.
 * A NULL options pointer means all defaults. */
typedef struct {
  float check_mem;
  int n_snapshots;
  int zero_top_planes;
  const int* aperture;
  float* phess;
  int tiles[6];
  int smooth_mode;
  float smooth_len[3];
  int time_interp;
  int nt_data;
  float dt_data;
  int time_blocking;
} mamute_opts;

#define MAMUTE_SMOOTH_NONE 0
#define MAMUTE_SMOOTH_BESSEL 1
#define MAMUTE_SMOOTH_LAPLACE 2
#define MAMUTE_INTERP_NEAREST 1
#define MAMUTE_INTERP_SINC 2

/* Creates a context on `device` issuing work on `cuda_stream` (a cudaStream_t;
 * NULL = the legacy default stream).  Returns MAMUTE_EARCH unless the device
 * is sm_103.  *ctx is NULL on failure. */
int mamute_ctx_create(mamute_ctx** ctx, int device, void* cuda_stream);

/* Frees the context and all of its device scratch.  NULL is allowed. */
void mamute_ctx_destroy(mamute_ctx* ctx);

/* Static description of an error code. */
const char* mamute_strerror(int code);

/* Description of the last failure on ctx (empty string if none). */
const char* mamute_last_error(const mamute_ctx* ctx);

/* Seismic modelling (Algorithm 1; Table 1 ModelingStep and ReadReceiver).
 *   vel       device [nz][ny][nx] P-wave velocity (m/s)
 *   rho       device [nz][ny][nx] density, or NULL for constant density
 *             (Eq. 1 right / left)
 *   src_xyz   host [n_src][3] source positions (m)
 *   wavelet   host [nt] source signature
 *   rec_offset host [n_src+1], rec_offset[0] = 0, non-decreasing
 *   rec_xyz   host [rec_offset[n_src]][3] receiver positions (m)
 *   opts      may be NULL (aperture and phess are honoured)
 *   seis      device [rec_offset[n_src]][nt] output, overwritten
 * Errors: EINVAL (dimensions, nulls, a point outside the model, misaligned
 * aperture), ECFL (ValidConditions, Table 1), ENOMEM, ECUDA, ETIMEOUT. */
int mamute_model(mamute_ctx* ctx, const mamute_grid* grid, const float* vel, const float* rho,
                 int n_src, const float* src_xyz, const float* wavelet, const int* rec_offset,
                 const float* rec_xyz, const mamute_opts* opts, float* seis);

/* Misfit and gradient (Algorithm 3): forward propagation with wavefield
 * checkpointing, J = 1/2 sum (d - d_obs)^2 (SeismicData::Misfit), adjoint
 * propagation driven by the residuals with cross-correlation imaging, the
 * sum over shots, MultiplyAdjoint (dJ/dc = 2 c dt^2 dJ/dA, A = c^2 dt^2) and
 * ZeroesNearSurface.
 *   d_obs   device [rec_offset[n_src]][nt] observed data
 *   misfit  host, receives J (accumulated in FP64)
 *   grad    device [nz][ny][nx], receives dJ/dc, overwritten
 * Other arguments and errors as mamute_model. */
int mamute_gradient(mamute_ctx* ctx, const mamute_grid* grid, const float* vel, const float* rho,
                    int n_src, const float* src_xyz, const float* wavelet, const int* rec_offset,
                    const float* rec_xyz, const float* d_obs, const mamute_opts* opts,
                    double* misfit, float* grad);

/* Transposed Jacobian applied to a data-space vector (the backward pass of
 * modelling): grad = d<seis(c), d_res>/dc, i.e. the adjoint wavefield is
 * driven by d_res instead of the residual.  Used by the autograd binding.
 *   d_res  device [rec_offset[n_src]][nt]
 *   grad   device [nz][ny][nx], overwritten
 * Other arguments and errors as mamute_gradient. */
int mamute_adjoint(mamute_ctx* ctx, const mamute_grid* grid, const float* vel, const float* rho,
                   int n_src, const float* src_xyz, const float* wavelet, const int* rec_offset,
                   const float* rec_xyz, const float* d_res, const mamute_opts* opts, float* grad);

/* As mamute_model and mamute_gradient, but vel, rho, seis, d_obs, grad and
 * opts->phess are HOST pointers; the call stages them through context
 * buffers (host->device before, device->host after).  mamute_model_host
 * copies the seismograms to seis in 8 time segments while the later
 * segments propagate (page-locked seis makes the copies asynchronous). */
int mamute_model_host(mamute_ctx* ctx, const mamute_grid* grid, const float* vel,
                      const float* rho, int n_src, const float* src_xyz, const float* wavelet,
                      const int* rec_offset, const float* rec_xyz, const mamute_opts* opts,
                      float* seis);
int mamute_gradient_host(mamute_ctx* ctx, const mamute_grid* grid, const float* vel,
                         const float* rho, int n_src, const float* src_xyz,
                         const float* wavelet, const int* rec_offset, const float* rec_xyz,
                         const float* d_obs, const mamute_opts* opts, double* misfit,
                         float* grad);

/* Gauss-Newton diagonal of the misfit (learned-preconditioner labels; the
 * paper's adjoint-state gradient of Sec. 2.1 / Algorithm 3 linearised):
 *   H(x) = sum_s sum_r sum_m (d d_{s,r}[m] / d c(x))^2
 * with the Born data taken over the full linear-convolution length of the
 * nt-step source-side term and the nt-sample impulse response.  Evaluated
 * by Parseval over an N_f = 2 nt zero-padded DFT: one forward propagation
 * per shot and one adjoint propagation per receiver, accumulating DFTs of
 * the imaging term and of the receiver impulse responses, restricted to the
 * bins where the wavelet spectrum is at least band_rel of its peak
 * (band_rel <= 0: all bins).  Every shot must record at the same receivers
 * (same count and coordinates, in the same order).
 *   hdiag  device [nz][ny][nx], overwritten
 * Other arguments as mamute_model (no aperture).  Errors: EINVAL (also for
 * differing receiver sets or more bins than the kernel supports, 128),
 * ECFL, ENOMEM, ECUDA, ETIMEOUT. */
int mamute_gn_diagonal(mamute_ctx* ctx, const mamute_grid* grid, const float* vel,
                       const float* rho, int n_src, const float* src_xyz, const float* wavelet,
                       const int* rec_offset, const float* rec_xyz, float band_rel, float* hdiag);

/* ---- Learned preconditioner network (not in the paper: a preconditioner
 * learned from exact Gauss-Newton diagonals).  A 4-layer 3x3x3 'same' CNN predicts the
 * log of the Gauss-Newton diagonal from the velocity and the pseudo-Hessian.
 * All pointers are device pointers.  Activations are channels-last
 * [D][H][W][16] BF16 (unsigned short bit patterns, fewer channels zero-
 * padded); weights are FP32 masters [27 taps][16 out][16 in] with taps in
 * (dz, dy, dx) order, packed to BF16 for the products; products are BF16 x
 * BF16 with FP32 accumulation on the tensor cores.  Every call synchronises
 * the context's stream.  Errors: EINVAL for bad sizes, NULL pointers or
 * activation pointers that are not 16-byte aligned, ECUDA, ENOMEM, ETIMEOUT
 * (a bounded device-side wait ran out). */

/* y = act(conv(x, w) + bias) with zero padding; act = ReLU if relu != 0;
 * if mask is given, outputs where mask <= 0 are zeroed (ReLU derivative of
 * the layer input in the input-gradient pass).  w is a packed weight set
 * (mamute_conv3d_pack; 16-byte aligned): the forward set computes the layer,
 * the backward set the gradient with respect to the layer input.  y32 [D][H][W][16] FP32
 * and/or y16 [D][H][W][16] BF16 receive the result (either may be NULL). */
int mamute_conv3d(mamute_ctx* ctx, int D, int H, int W, const unsigned short* x,
                  const unsigned short* w, const float* bias, int relu,
                  const unsigned short* mask, float* y32, unsigned short* y16);

/* Weight and bias gradients: gw[tap][o][i] = sum_p gy[p][o] x[p + tap - 1][i],
 * gb[o] = sum_p gy[p][o] (FP32, summed in a fixed order).
 *   x, gy  [D][H][W][16] BF16;  gw [27][16][16], gb [16] FP32 */
int mamute_conv3d_wgrad(mamute_ctx* ctx, int D, int H, int W, const unsigned short* x,
                        const unsigned short* gy, float* gw, float* gb);

/* Packs FP32 masters w [27][16][16] into the forward BF16 set fwd (same
 * layout) and, if bwd is not NULL, the input-gradient set
 * bwd[26 - tap][i][o] = w[tap][o][i]. */
int mamute_conv3d_pack(mamute_ctx* ctx, const float* w, unsigned short* fwd,
                       unsigned short* bwd);

/* Masked mean squared error of channel 0 of out [n][16] FP32 against
 * target [n]: loss = sum_p m_p (out_p - t_p)^2 / n_mask (FP64 sums; mask
 * [n] or NULL for all ones) to the host, and its gradient gy [n][16] BF16
 * (channel 0, other channels zero). */
int mamute_mse_loss(mamute_ctx* ctx, long long n, const float* out, const float* target,
                    const float* mask, double n_mask, double* loss, unsigned short* gy);

/* Network inputs and targets for n voxels: x16 [n][16] BF16 with channel 0
 * = (vel - v_ref) / v_scale and channel 1 = max(log(phess / Pmax),
 * -log_clip) / log_clip, Pmax = max |phess|; if hdiag and target are given,
 * target[p] = log(hdiag[p] / phess[p]).  pmax (host, may be NULL) receives
 * Pmax. */
int mamute_nn_features(mamute_ctx* ctx, long long n, const float* vel, const float* phess,
                       const float* hdiag, float v_ref, float v_scale, float log_clip,
                       unsigned short* x16, float* target, float* pmax);

/* One Adam step (Kingma and Ba) with bias correction on n FP32 parameters. */
int mamute_adam(mamute_ctx* ctx, int n, float* p, float* m, float* v, const float* g, float lr,
                float beta1, float beta2, float eps, int step);

/* Checkpoint schedule (host only, no device work; Sec. 2.1 optimal
 * checkpointing after Griewank and Walther).  Plans the reversal of nt steps
 * from the zero initial state with n_slots checkpoint slots.  Writes the
 * number of forward steps the plan takes (the first sweep included) to
 * *n_forward and the number of actions to *n_actions; if `actions` is not
 * NULL it must hold 3 * (*n_actions) ints from a previous sizing call and
 * receives triples (kind, a, b): kind 0 = advance from step a to step b,
 * 1 = store the current state in slot a, 2 = restore slot a (state of step
 * b; slot -1 is the zero initial state), 3 = reverse step a.
 * Errors: EINVAL for nt < 1 or n_slots < 0. */
int mamute_revolve_plan(int nt, int n_slots, long long* n_forward, int* n_actions, int* actions);

/* Timing of the time loop, for benchmarks.  When enabled, each compute call
 * records CUDA events on the context's stream immediately before the first
 * and after the last time-step kernel it launches, and counts its kernel
 * launches.  mamute_ctx_last_timing reports, for the last completed call,
 * the elapsed milliseconds between the two events, the number of time-step
 * kernel launches and the number of all kernel launches (NULL outputs are
 * skipped).  Errors: EINVAL for a NULL context; ECUDA if an event fails. */
int mamute_ctx_set_timing(mamute_ctx* ctx, int enable);
int mamute_ctx_last_timing(const mamute_ctx* ctx, double* loop_ms, long long* step_launches,
                           long long* total_launches);

/* For the last mamute_gn_diagonal call made with timing enabled: the summed
 * device milliseconds of its DFT accumulations (an event pair on the
 * context's stream around each twiddle + DFT launch), their number, and the
 * complex multiply-adds they performed (points x samples x bins, each four
 * FP32 flops).  NULL outputs are skipped; EINVAL for a NULL context.  No
 * counterpart in the paper: it measures the labels' FP32 ALU roofline. */
int mamute_ctx_dft_timing(const mamute_ctx* ctx, double* dft_ms, long long* dft_launches,
                          double* complex_macs);

/* Misfit J = 1/2 sum_i (d[i] - d_obs[i])^2 (FP64 sums of FP32 residuals)
 * for callers that cannot allocate device memory, e.g. because a host
 * framework's caching allocator already holds the device's memory, or because
 * a latency-sensitive loop must not pay for cudaMalloc's implicit
 * synchronisation of the device.  The paper has no counterpart: it is the
 * formula mamute_gradient uses for its misfit, summed in the same order
 * (16384-sample blocks over the [n_rec][nt] layout, then one warp in a fixed
 * order), so for the same arrays the two agree bit for bit.  Its per-block
 * partial sums are kept in a fixed
 * file-scope device array (128 KiB on every device that loads the library,
 * held until the process exits) instead of context scratch.  No context is
 * needed and nothing is allocated or freed.
 *   d, d_obs   device [n] float32 (any layout, the same for both)
 *   n          number of samples, 0 <= n <= MAMUTE_MISFIT_NOALLOC_MAX_SAMPLES
 *   cuda_stream stream to run on (NULL = legacy default stream); the call
 *              synchronises it before returning
 *   misfit     host, receives J
 * The first call on a device looks up the scratch array's device address
 * with that device current; later calls on that device reuse it.  All calls
 * on a device share the one array, so calls that overlap on the GPU (from
 * several host threads or streams) race and must be serialised by the caller.
 * Errors: EINVAL for a NULL pointer, n < 0 or n above the limit (nothing is
 * launched); ECUDA if a launch or the copy of the result fails. */
#define MAMUTE_MISFIT_NOALLOC_MAX_SAMPLES (16384LL * 16384LL)
int mamute_misfit_noalloc(const float* d, const float* d_obs, long long n, void* cuda_stream,
                          double* misfit);

/* Gradient smoothing (Sec. 2, FWI: gradient preconditioning by a Bessel or a
 * Laplace filter with lengths bessel_filter_l{x,y,z}; Algorithm 3
 * GradientPreconditioning).  With D_aa the 3-point second difference along
 * axis a on the model grid of spacing h, reflecting at the ends (the value
 * beyond the last cell repeats it):
 *   mode 1 (Bessel)   out = (I - lx^2 Dxx - ly^2 Dyy - lz^2 Dzz)^-1 in
 *   mode 2 (Laplace)  out = (I - lx^2 Dxx)^-1 (I - ly^2 Dyy)^-1 (I - lz^2 Dzz)^-1 in
 *   mode 0            out = in.
 * Solved exactly in the DCT-II basis, which diagonalises both operators
 * (FP32 transforms).  lengths: host [3] (lx, ly, lz, metres; 0 means 2 h) or
 * NULL for all 2 h.  in, out: device [nz][ny][nx]; they may be the same
 * array.  Errors: EINVAL (sizes, NULL, bad mode or negative length), ENOMEM,
 * ECUDA. */
int mamute_smooth(mamute_ctx* ctx, int nx, int ny, int nz, float h, int mode,
                  const float* lengths, const float* in, float* out);

/* Time resampling of traces (Sec. 2: time interpolation by nearest neighbour
 * or sinc; Table 1 Interpolate).  Sample n of an input trace is at time
 * n dt_in, output sample m at m dt_out.
 *   mode 1 (nearest)  y[m] = x[floor(m dt_out / dt_in + 1/2)], 0 past the end
 *   mode 2 (sinc)     y[m] = sum_n x[n] (dt_in / D) sinc((m dt_out - n dt_in) / D)
 *                      hann((m dt_out - n dt_in) / (8 D)), D = max(dt_in, dt_out),
 *                      hann(u) = (1 + cos(pi u)) / 2 for |u| < 1, else 0
 *                      (interpolation when dt_out <= dt_in; low-pass below the
 *                      output Nyquist frequency, then decimation, otherwise).
 * adjoint = 0: x device [n_traces][nt_in] -> y device [n_traces][nt_out];
 * adjoint = 1: the transpose, x device [n_traces][nt_out] -> y device
 * [n_traces][nt_in].  The weights are formed in FP64 on the host, the sums in
 * FP32 on the device, in a fixed order.  Errors: EINVAL, ENOMEM, ECUDA. */
int mamute_resample(mamute_ctx* ctx, int n_traces, int nt_in, float dt_in, int nt_out,
                    float dt_out, int mode, int adjoint, const float* x, float* y);

/* Stability bound used by the CFL check (max(c) dt / h must not exceed it). */
double mamute_cfl_limit(void);

#ifdef __cplusplus
}
#endif

#endif /* MAMUTE_H */
