/*
 * cygrid_gb300.h -- C ABI of the GB300 convolution-gridding library.
 *
 * The library grids irregularly sampled sky data (one value or a spectrum of
 * C channels per sample) onto arbitrary target coordinates by convolution
 * with a kernel, following Winkel, Lenz & Floeer (A&A 2016), Sect. 2:
 *
 *   numerator  N_pc = sum_n omega_n w(p, n) D_nc         (Eq. 1)
 *   weight map W_p  = sum_n omega_n w(p, n)              (Eq. 2)
 *   map        R_pc = N_pc / W_p   (NaN where W_p = 0)   (Eq. 3)
 *
 * with the sum restricted to samples within the support radius r of the
 * target (d <= r, Sect. 3.5).  Candidate samples are found with the paper's
 * HEALPix lookup (Sect. 2.2, 3.3): the samples' RING indices, a stable sort
 * of the samples by index, and a disc query around each tile of targets.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Angles are in degrees: longitude (any real value, folded into [0,360))
 *    and latitude in [-90, 90]; kernel sizes and the support radius too.
 *  - Every array argument is a pointer to DEVICE memory of the current CUDA
 *    device, owned by the caller, contiguous, and must stay valid until the
 *    work enqueued by the call has executed on the handle's stream.  The
 *    library never frees caller memory.  Exceptions are marked "host".
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls enqueue work on the handle's stream and return without
 *    waiting, except where a call is documented as synchronising.
 *  - The handle owns its workspace (allocated with stream-ordered
 *    cudaMallocAsync and released by cg_grid_destroy).  A handle must not be
 *    used from two host threads at once.
 *  - Errors: every call returns a cg_status.  Argument errors are detected on
 *    the host and returned at once; the message is available from
 *    cg_last_error() (thread-local).  Errors that only the device can see
 *    (non-finite or out-of-range sample coordinates) set a device error word
 *    that the next synchronising call (cg_grid_finalize, cg_sync) reports as
 *    CG_EINVAL or CG_EDEVICE.  Nothing in the library traps, aborts or
 *    asserts on the device.
 */
#ifndef CYGRID_GB300_H
#define CYGRID_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cg_grid cg_grid; /* opaque, library-owned */

typedef enum {
  CG_OK = 0,
  CG_EINVAL = 1,    /* invalid argument or invalid input value */
  CG_ENOMEM = 2,    /* device allocation failed */
  CG_ECUDA = 3,     /* a CUDA runtime call failed */
  CG_EDEVICE = 4,   /* the device reported an internal error */
  CG_ETIMEOUT = 5,  /* a bounded device-side wait gave up */
  CG_ESTATE = 6     /* call not valid in the handle's current state */
} cg_status;

typedef enum { CG_F32 = 0, CG_BF16 = 1 } cg_dtype;

typedef enum {
  CG_GAUSS1D = 0, /* params[0] = sigma (deg): w = exp(-d^2 / (2 sigma^2)) */
  CG_GAUSS2D = 1, /* params = {sigma_maj, sigma_min, PA} (deg), PA of the
                     major axis from north through east; with beta the
                     bearing of the sample seen from the target,
                     a = d cos(beta - PA), b = d sin(beta - PA),
                     w = exp(-a^2/(2 sigma_maj^2) - b^2/(2 sigma_min^2)) */
  CG_TSINC = 2    /* params = {a, b} (deg): the sin(x)/x kernel tapered by a
                     Gaussian, w = sin(pi d/a) / (pi d/a) exp(-d^2 / b^2);
                     weights can be negative, and R is NaN where W <= 0 */
} cg_kernel;

typedef enum {
  CG_PATH_AUTO = 0,   /* CG_PATH_TC for BF16 data with C >= 16 and C % 8 == 0,
                         else CG_PATH_FP32 */
  CG_PATH_FP32 = 1,   /* channel accumulation on FP32 CUDA cores (any data) */
  CG_PATH_TC = 2,     /* BF16 data on the tcgen05 tensor cores, FP32 accumulation;
                         each weight as a hi + lo pair of BF16 numbers (~16
                         significant bits), so the result matches the FP64
                         definition on the same BF16 data to ~1e-5 */
  CG_PATH_TC_FAST = 3 /* as CG_PATH_TC with single BF16 weights (8 significant
                         bits): half the tensor work; map error up to 2^-8 of
                         S_pc = sum |omega w D| / W */
} cg_path;

/* Create a gridder for n_targets target directions (paper Sect. 3.5: WcsGrid
 * / SlGrid -- here always an explicit list of sight lines).
 *   out        host: receives the new handle.
 *   lon_deg,
 *   lat_deg    device, [n_targets] float64 each.
 *   n_targets  1 .. 2^31-1.
 *   n_channels C >= 1, the length of each sample's spectrum.
 *   stream     cudaStream_t (as void*) for all work of this handle.
 * Target geometry (unit vectors, tiles of nearby targets) is computed here,
 * on the stream.  Invalid target coordinates return CG_EINVAL after a
 * synchronisation of the stream (create is a set-up call and synchronises). */
cg_status cg_grid_create(cg_grid** out, const double* lon_deg, const double* lat_deg,
                         int64_t n_targets, int32_t n_channels, void* stream);

/* Set the kernel (paper Sect. 3.5, set_kernel).
 *   kernel_type   cg_kernel.
 *   params        host, [n_params]: {sigma}, {sigma_maj, sigma_min, PA} or {a, b},
 *                 degrees.
 *   support_deg   support radius r > 0: samples with d > r do not contribute.
 *   nside         internal HEALPix resolution, 1 .. 8192 (any integer; powers of
 *                 two index a little faster), or 0 to derive it from
 *                 hpx_maxres_deg: the smallest power of two with pixel size
 *                 sqrt(pi/3)/nside <= hpx_maxres_deg.  Out of range: CG_EINVAL.
 * The result does not depend on nside (the cut d <= r is exact); nside only
 * changes how candidates are found.  Resets the accumulators.  Synchronising. */
cg_status cg_set_kernel(cg_grid* g, int32_t kernel_type, const double* params,
                        int32_t n_params, double support_deg, int32_t nside,
                        double hpx_maxres_deg);

/* Accumulate samples into the numerator and weight map (Eq. 1-2; paper
 * Sect. 2.1 algorithm, step 2).  Multiple calls accumulate (streaming).
 *   lon_deg, lat_deg  device, [n_samples] float64.
 *   data              device, [n_samples][C] row-major, dtype data_dtype.
 *   data_dtype        CG_F32 or CG_BF16.
 *   weights           device, [n_samples] float32 >= 0, or NULL for unit weights.
 *   n_samples         0 .. 2^31-1 (0 is a no-op).
 * lon_deg = lat_deg = NULL (and weights = NULL) grids new channel data for the
 * samples of the previous add, reusing its sample index (keys, sort, ranges);
 * n_samples must then equal that add's count, and the previous add must come
 * after the last cg_set_kernel (else CG_EINVAL).  The library keeps its own
 * FP64 copy of the coordinates, so the caller's earlier arrays may be gone.
 * Asynchronous.  Non-finite or |lat| > 90 coordinates are reported by the
 * next synchronising call as CG_EINVAL. */
cg_status cg_grid_add(cg_grid* g, const double* lon_deg, const double* lat_deg,
                      const void* data, int32_t data_dtype, const float* weights,
                      int64_t n_samples);

/* Normalise (Eq. 3; paper Sect. 2.1 step 3, get_datacube) without changing
 * the accumulators.
 *   out                  device float32: [n_targets][C] (layout 0) or
 *                        [C][n_targets] (layout 1, the FITS cube order).
 *   out_weights          device float32 [n_targets] (W_p), or NULL.
 * NaN where W_p = 0.  Synchronises the stream and reports device errors. */
cg_status cg_grid_finalize(cg_grid* g, float* out, int32_t layout_channel_major,
                           float* out_weights);

/* One-shot gridding: reset, add, finalize in one call (paper Listing 1:
 * grid() followed by get_datacube()).  Arguments as for cg_grid_add and
 * cg_grid_finalize.  Does NOT synchronise: device errors are reported by the
 * next cg_sync or cg_grid_finalize. */
cg_status cg_grid_oneshot(cg_grid* g, const double* lon_deg, const double* lat_deg,
                          const void* data, int32_t data_dtype, const float* weights,
                          int64_t n_samples, float* out, int32_t layout_channel_major,
                          float* out_weights);

/* One-shot gridding of samples held in HOST memory: the end-to-end form of
 * cg_grid_oneshot.  The call copies the coordinates, channel data and
 * weights into device staging buffers owned by the handle, grids them exactly
 * as cg_grid_oneshot does, and copies the map (and weight map) back into the
 * caller's host arrays.
 *   h_lon, h_lat, h_data, h_weights   host arrays with the shapes and types of
 *                        cg_grid_oneshot's device arguments (h_weights may be
 *                        NULL); page-locked memory (cudaHostAlloc or
 *                        cudaHostRegister) lets the copies run asynchronously,
 *                        pageable memory makes them synchronous.
 *   h_out                host float32 [n_targets][C] (layout 0) or
 *                        [C][n_targets] (layout 1).
 *   h_out_weights        host float32 [n_targets] (W_p), or NULL.
 * Asynchronous: every host array must stay valid and unmodified until
 * cg_sync returns, which also reports device errors.  Consecutive calls on
 * one handle are pipelined over two staging slots: call k + 1 copies its
 * inputs on a copy-in stream while call k computes on the handle's stream and
 * the map of call k - 1 is copied back on a copy-out stream; within a call
 * the sample index is built while the channel data are still being copied.
 * Device memory: two slots of N (20 + C b) + P (C + 1) 4 bytes (b = 2 for
 * BF16, 4 for F32), grown on demand and kept until cg_grid_destroy. */
cg_status cg_grid_oneshot_host(cg_grid* g, const double* h_lon, const double* h_lat,
                               const void* h_data, int32_t data_dtype, const float* h_weights,
                               int64_t n_samples, float* h_out, int32_t layout_channel_major,
                               float* h_out_weights);

/* Zero the accumulators (asynchronous). */
cg_status cg_grid_reset(cg_grid* g);

/* Release the handle and its workspace (synchronises the stream). */
cg_status cg_grid_destroy(cg_grid* g);

/* Change the stream used by later calls. */
cg_status cg_set_stream(cg_grid* g, void* stream);

/* Select the channel-accumulation form (cg_path). */
cg_status cg_set_path(cg_grid* g, int32_t path);

/* Wait for the handle's stream (and the copy streams of
 * cg_grid_oneshot_host) and report device-side errors. */
cg_status cg_sync(cg_grid* g);

/* Thread-local description of the last error ("" if none). */
const char* cg_last_error(void);

/* Counters and layout facts of a handle (host struct).
 *   nside, n_tiles, tile_size, n_ranges: planner choices;
 *   path: the accumulation form the last add used (cg_path);
 *   n_candidates: (tile, sample) candidate pairs of the last add, summed over
 *                 tiles; each stands for tile_size (target, sample) weights
 *                 (those beyond the support are zero). */
typedef struct {
  int64_t n_targets;
  int32_t n_channels;
  int32_t nside;
  int64_t n_tiles;
  int32_t tile_size;
  int32_t path;
  int64_t n_ranges;
  int64_t n_samples_total;
  int64_t n_pairs;      /* (target, sample) pairs with d <= r since the last reset */
  int64_t n_launches;   /* kernels this handle has launched since creation */
  int64_t n_candidates;
} cg_info;
/* Fill *info (host struct).  Synchronises the stream (n_pairs is device-side). */
cg_status cg_get_info(cg_grid* g, cg_info* info);

/* Stage timing with CUDA events recorded on the handle's stream.
 * Stages: 0 sample keys (ang2pix), 1 radix sort, 2 sample gather + ring
 * offsets + tile sample ranges, 3 tile gridder, 4 normalisation / layout.
 * When enabled, every add / oneshot / finalize records its stages.
 * cg_read_timing waits for the stream, writes the summed milliseconds per
 * stage (host array ms[CG_N_STAGES]) over all calls recorded since the
 * previous read and the number of gridder launches, then clears the record. */
#define CG_N_STAGES 5
cg_status cg_set_timing(cg_grid* g, int32_t enable);
cg_status cg_read_timing(cg_grid* g, double* ms, int64_t* n_grid_launches);

/* RING-scheme HEALPix index of each direction (paper Sect. 2.2 step 3a; the
 * tessellation of Gorski et al. 2005).
 *   lon_deg, lat_deg  device [n] float64.   pix  device [n] int64.
 * Invalid coordinates give pix = -1.  Asynchronous on `stream`. */
cg_status cg_ang2pix_ring(int32_t nside, const double* lon_deg, const double* lat_deg,
                          int64_t n, int64_t* pix, void* stream);

/* Unit vectors (cos b cos l, cos b sin l, sin b) of n directions, evaluated
 * exactly as the gridder evaluates sample positions (the distance of Eq. 1-2
 * is taken between such vectors): double-float sine and cosine on the FP32
 * pipes, absolute error ~1e-14, returned as float64.
 *   lon_deg, lat_deg  device [n] float64 (finite; |lat| <= 90 for a unit vector)
 *   xyz               device [n][3] float64, written
 * Asynchronous on `stream`; CG_EINVAL for n < 0 or a null pointer. */
cg_status cg_unit_vectors(const double* lon_deg, const double* lat_deg, int64_t n, double* xyz,
                          void* stream);

/* Register-blocking shape of the FP32 CUDA-core gridder (a tuning knob; the
 * result differs only in the rounding of the weight sums): -1 = by channel
 * count (default), 0 .. CG_F32_SHAPES-1 = (targets x channels per thread,
 * channel groups) of <1,4,1> <1,8,1> <1,8,2> <2,8,4> <2,16,4> <4,16,8>
 * <4,16,16>.  The batch autotuner picks it per job. */
#define CG_F32_SHAPES 7
cg_status cg_set_f32_shape(cg_grid* g, int32_t shape);

/* Adjoint of the normalised gridding operator (paper Eq. 1-3 read as a
 * linear map R = G D with G[p][n] = omega_n w_pn / W_p): degridding,
 *   out[n][c] = sum_p G[p][n] map[p][c],
 * for the samples of the last add (its sample index is reused; the target
 * side uses a RING index of the targets built on the first call after
 * cg_set_kernel).  The gradient of a loss L(R) with respect to the data is
 * cg_degrid of dL/dR.
 *   map          device float32 [n_targets][C] (user order).
 *   map_weights  device float32 [n_targets]: W_p of the operator (the
 *                out_weights of the gridding call), or NULL for the handle's
 *                accumulated weight map (CG_ESTATE if a one-shot call left
 *                none).  Targets with W_p <= 0 contribute nothing.
 *   out          device float32 [n][C] in the add's sample order (samples
 *                with invalid coordinates get 0).
 *   n            must equal the last add's n_samples.
 * Deterministic (a gather: each sample's sum has a fixed order).
 * Asynchronous; CG_ESTATE without a previous add, CG_EINVAL on bad arguments. */
cg_status cg_degrid(cg_grid* g, const float* map, const float* map_weights, float* out,
                    int64_t n);

/* Normalised interpolation of a map at the samples of the last add (the
 * degridding reading in which every sample receives the kernel-weighted mean
 * of the map around it; the mirror of Eq. 1-3 with targets and samples
 * exchanged):
 *   out[n][c] = sum_p w_pn map[p][c] / V_n,  V_n = sum_p w_pn  (d_pn <= r),
 * NaN where no target lies within r of the sample.  The samples' weights do
 * not enter.
 *   map          device float32 [n_targets][C] (user order).
 *   out          device float32 [n][C] in the add's sample order.
 *   out_weights  device float32 [n] (V_n), or NULL.
 *   n            must equal the last add's n_samples.
 * Deterministic.  Asynchronous; CG_ESTATE without a previous add. */
cg_status cg_interp(cg_grid* g, const float* map, float* out, float* out_weights, int64_t n);

/* One-shot gridding with one weight per sample AND channel (an extension of
 * Eq. 1-3: omega_n becomes omega_nc):
 *   N_pc = sum_n omega_nc w_pn D_nc,  W_pc = sum_n omega_nc w_pn,
 *   R_pc = N_pc / W_pc (NaN where W_pc = 0).
 *   pc_weights   device float32 [n_samples][C], finite and >= 0; a zero
 *                weight removes the sample from that channel (its value is
 *                not read, so it may be NaN).
 *   out          device float32 [n_targets][C] (layout 0) or [C][n_targets].
 *   out_weights  device float32 [n_targets][C] or [C][n_targets] (W_pc, same
 *                layout), or NULL.
 * Runs the FP32 CUDA-core gridder once over 2C values per sample
 * (omega_nc D_nc and omega_nc); builds a new sample index (cg_degrid and
 * cg_interp then refer to these samples) and leaves the accumulators of
 * cg_grid_add untouched.  Asynchronous. */
cg_status cg_grid_oneshot_pcw(cg_grid* g, const double* lon_deg, const double* lat_deg,
                              const void* data, int32_t data_dtype, const float* pc_weights,
                              int64_t n_samples, float* out, int32_t layout_channel_major,
                              float* out_weights);

/* Derivative of the normalised map with respect to the kernel width, for the
 * circular gauss1d kernel with the support radius held fixed:
 *   dR_pc/dsigma = (sum_n omega_n w'_pn D_nc - R_pc sum_n omega_n w'_pn) / W_p,
 *   w' = dw/dsigma = w d^2 / sigma^3     (d, sigma in degrees),
 * for the samples of the last add and the channel data `data` (the FP32
 * CUDA-core gridder is run with w and with w').
 *   data       device [n_samples][C], CG_F32 or CG_BF16 (data_dtype).
 *   grad_out   device float32 [n_targets][C] upstream gradient dL/dR, or NULL.
 *   dR         device float32 [n_targets][C] (user order), or NULL; NaN where
 *              W_p = 0.
 *   dsigma     device float64 scalar: sum_pc grad_out[p][c] dR[p][c] (W_p > 0
 *              targets; deterministic FP64 reduction), or NULL (needs grad_out).
 * CG_EINVAL for gauss2d kernels.  Asynchronous. */
cg_status cg_grid_dsigma(cg_grid* g, const void* data, int32_t data_dtype, const float* grad_out,
                         float* dR, double* dsigma);

/* Map making by gradient descent on L(m) = 1/2 ||G^T m - D||^2, G the
 * normalised gridding operator of Eq. 3 and G^T its adjoint (cg_degrid): the
 * element-wise steps of an iteration, on the handle's stream.
 *   cg_md_residual: r <- r - data (device float32 [n], r = G^T m on entry)
 *                   and *loss <- 1/2 sum r^2 in FP64 (device double; a fixed
 *                   summation order, so repeated calls agree bit for bit);
 *   cg_md_update:   m <- m - alpha grad (device float32 [n]), where grad is
 *                   NaN (a target no sample reaches) it counts as 0.
 * CG_EINVAL for null pointers, n < 0 or a non-finite alpha. */
cg_status cg_md_residual(cg_grid* g, float* r, const float* data, int64_t n, double* loss);
cg_status cg_md_update(cg_grid* g, float* m, const float* grad, float alpha, int64_t n);

/* Copy out the sample index built by the last cg_grid_add (the sorted
 * replacement for the paper's hash tables, Sect. 3.4):
 *   sorted_pix  device [n] int64: RING indices in ascending order;
 *   perm        device [n] int64: original sample index of each sorted entry
 *               (ties in ascending original order: a stable sort);
 *   ring_off    device [4 nside + 1] int64: first sorted position whose pixel
 *               lies in ring >= i (ring 0 and 4 nside are sentinels), or NULL.
 * n must equal the sample count of that add.  Asynchronous. */
cg_status cg_grid_export_index(cg_grid* g, int64_t* sorted_pix, int64_t* perm,
                               int64_t* ring_off, int64_t n);

/* Testing hook for the bounded waits of the tensor-core gridder.
 *
 * The paper has no counterpart.  enable != 0: until it is called again with
 * enable = 0, every tensor-core gridding launch of this handle makes its
 * producer warps first wait for a device word that nothing sets, giving up
 * after wait_cycles SM clock cycles (<= 0: 2e6, about a millisecond).  The
 * wait runs out, the kernel records a time-out, every warp role stops, the
 * MMAs in flight complete and the tensor memory is freed; the next
 * synchronising call (cg_sync, cg_grid_finalize, ...) returns CG_ETIMEOUT and
 * clears the condition.  The call's output is undefined; the handle stays
 * usable.  This exercises the failure path of the kernel's waits without any
 * fault, trap or endless loop on the GPU. */
cg_status cg_debug_hold(cg_grid* g, int32_t enable, int64_t wait_cycles);

/* No-allocation variant of the sample index (RING keys + stable sort).
 *
 * The paper has no counterpart: this entry point exists for callers that must
 * not allocate device memory -- code that runs under a fixed, pre-reserved
 * memory budget (the allocator may not be touched after start-up), inside
 * another framework's memory manager that forbids foreign allocations, or on a
 * hot path where an allocation could block or fail.  It computes what
 * cg_grid_add followed by cg_grid_export_index computes for the samples' index:
 *   sorted_pix  device [n] int64: RING indices at `nside`, ascending; samples
 *               with non-finite or out-of-range coordinates get 12 nside^2 and
 *               sort to the end (they are not reported as errors here);
 *   perm        device [n] int64: original index of each sorted entry, ties in
 *               ascending original order (a stable sort).
 * All scratch lives in one static device array of the library
 * (CG_NOALLOC_MAX_SAMPLES samples, about 4.3 MB), which every GPU that loads
 * the library holds until the process exits.  n above CG_NOALLOC_MAX_SAMPLES
 * returns CG_EINVAL.  The call allocates nothing: no cudaMalloc, cudaFree or
 * allocating library routine.  The first call on a device looks up the
 * array's device address (once per device, with that device current); make
 * that first call before any stream capture.  Every call on a device shares
 * the one array, so calls that overlap on the GPU (different streams, or
 * different host threads) race: order them on one stream.  The array keeps
 * the previous call's contents; the call clears what must start at zero.
 * Asynchronous on `stream`; nside 1 .. 8192. */
#define CG_NOALLOC_MAX_SAMPLES 262144
cg_status cg_sort_samples_noalloc(int32_t nside, const double* lon_deg, const double* lat_deg,
                                  int64_t n, int64_t* sorted_pix, int64_t* perm, void* stream);

/* ------------------------------------------------------------------------
 * Batches: many independent gridding jobs replayed as one CUDA graph.
 *
 * The paper grids one survey at a time; a batch runs many jobs of uneven
 * sample count, channel count, target grid and kernel width together.  Each
 * job has its own handle (targets, kernel and channel count set by the
 * caller with cg_grid_create / cg_set_kernel) and its own caller-owned
 * device arrays; a job computes exactly what cg_grid_oneshot computes.
 * ------------------------------------------------------------------------ */
typedef struct cg_job {
  cg_grid* grid;                  /* the job's handle (one handle per job)    */
  const double* lon_deg;          /* device [n_samples] float64               */
  const double* lat_deg;          /* device [n_samples] float64               */
  const void* data;               /* device [n_samples][C], data_dtype        */
  int32_t data_dtype;             /* CG_F32 or CG_BF16                        */
  const float* weights;           /* device [n_samples] float32 or NULL       */
  int64_t n_samples;              /* >= 1                                     */
  float* out;                     /* device float32 map (layout as below)     */
  int32_t layout_channel_major;   /* 0: [n_targets][C], 1: [C][n_targets]     */
  float* out_weights;             /* device float32 [n_targets] or NULL       */
} cg_job;

typedef struct cg_batch cg_batch;

/* Plan a batch: copies the job descriptors (the arrays they point to must
 * stay valid while the batch is used) and assigns the jobs to n_streams
 * parallel branches (1 .. 64), largest estimated cost first onto the least
 * loaded branch.  CG_EINVAL for a job without a kernel, with no samples or a
 * null pointer, or whose handle another job also uses. */
cg_status cg_batch_create(cg_batch** out, const cg_job* jobs, int32_t n_jobs, int32_t n_streams);

/* Autotune (synchronising): for every job, time `reps` one-shot runs of each
 * candidate -- the FP32 gridder's register-blocking shapes next to the
 * default for its channel count, and (allow_tc != 0, BF16 data, C % 8 == 0)
 * the tensor-core form -- and keep the fastest.  Invalidates a captured graph. */
cg_status cg_batch_autotune(cg_batch* b, int32_t reps, int32_t allow_tc);

/* Run every job once eagerly (so that workspaces reach their final size),
 * then capture all jobs into one CUDA graph on `stream` (NULL: a private
 * stream): a fork, each job's one-shot pipeline on its branch, a join. */
cg_status cg_batch_capture(cg_batch* b, void* stream);

/* Replay the captured graph on `stream` (one launch; asynchronous).
 * CG_ESTATE before cg_batch_capture.  Device errors of a job are reported
 * by cg_sync on that job's handle. */
cg_status cg_batch_run(cg_batch* b, void* stream);

/* The planner's and autotuner's choice for one job: path (CG_PATH_*), FP32
 * shape index (-1: default), tuned ms per one-shot run, branch index. */
cg_status cg_batch_get_choice(cg_batch* b, int32_t job, int32_t* path, int32_t* f32_shape,
                              double* ms, int32_t* stream_index);

/* Kernels recorded in the captured graph and the number of branches. */
cg_status cg_batch_info(cg_batch* b, int64_t* graph_kernels, int32_t* n_streams);

/* Choose how the next cg_batch_capture records the batch: fused != 0 builds
 * one pipeline for all jobs -- one keys pass, one sort of every job's samples
 * (a composite key keeps each job's samples together, in its own RING key
 * order), one gather and one candidate-range pass, one persistent FP32
 * gridder launch per 96 jobs whose CTAs take (job, tile, channel slab,
 * candidate split) items from a queue ordered by estimated cost, one split
 * reduction, one non-finite fix-up and one normalisation over all jobs; jobs
 * whose choice is the tensor-core form (BF16 data, C % 8 == 0, 16-byte
 * aligned data, [n_targets][C] output) run the tensor-core gridder on their
 * segment of the shared index.  fused = 0 (the default): one branch per job
 * as described at cg_batch_create.  Each job computes what cg_grid_oneshot
 * computes (paper Eq. 1-3); the FP32 results may differ from a one-job call
 * in the last bits where the candidate splits differ.  While a fused graph
 * exists the jobs' handles belong to it (their candidate ranges are
 * rewritten by every replay).  Invalidates a captured graph. */
cg_status cg_batch_set_fused(cg_batch* b, int32_t fused);

/* Wait for the last cg_batch_run and report the jobs' device errors:
 * CG_EINVAL (invalid sample coordinates or weights, skipped), CG_ETIMEOUT
 * (a bounded device wait gave up); the error words are cleared. */
cg_status cg_batch_sync(cg_batch* b);

/* Testing hook (no paper counterpart): with enable != 0 the fused FP32
 * gridder's CTAs first wait, for at most wait_cycles SM clock cycles (0: two
 * million), for a device word that nothing sets, then record ERR_TIMEOUT and
 * leave without taking items, so that cg_batch_sync reports CG_ETIMEOUT
 * without a GPU fault.  Invalidates a captured graph. */
cg_status cg_batch_debug_hold(cg_batch* b, int32_t enable, int64_t wait_cycles);

/* Release the graph, branch streams and events (not the jobs' handles). */
cg_status cg_batch_destroy(cg_batch* b);

#ifdef __cplusplus
}
#endif

#endif /* CYGRID_GB300_H */
