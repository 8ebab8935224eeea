/*
 * epic.h - C ABI of the GB300 EPIC/EPICal library.
 *
 * EPIC (E-field Parallel Imaging Correlator) direct imaging and the EPICal
 * feedback calibration of Beardsley et al., "An Efficient Feedback
 * Calibration Algorithm for Direct Imaging Radio Telescopes".  Per time
 * sample t and channel c (one "frame"):
 *   E'_a = E_a / g_a                       gain correction          (Eq. 8)
 *   E'_j = sum_a W_a(r_j - r_a) E'_a        gridding                 (Eq. 9)
 *   E'(s_k) = (1/Na) sum_j e^{+2 pi i ...} E'_j   2D FFT             (Eq. 10)
 *   I'(s_k) += |E'(s_k)|^2 / T             square and average (Sec. 2.1)
 *   K_a += E_a conj(E'(s0)), P_a += |E_a|^2  EPICal correlation (Eqs. 12, 15)
 * and per calibration interval the damped gain update (Eqs. 15-17).
 *
 * Conventions (all calls):
 *  - Every call returns an epic_status; on failure epic_last_error() gives a
 *    thread-local message.  No call aborts the process.
 *  - "device" pointers are CUDA global-memory pointers on the plan's device
 *    (e.g. torch tensor data_ptr()); "host" pointers are ordinary memory.
 *    The caller owns every buffer it passes; the plan owns its tables,
 *    gains and accumulators.  Host arrays given to create/configure are
 *    copied before the call returns.
 *  - Work is enqueued on the plan's stream and is asynchronous unless the
 *    description says "synchronous".  Device faults surface as
 *    EPIC_ERR_CUDA on a later call or on epic_plan_sync().
 *  - A plan is not thread-safe; use one plan per host thread and stream.
 *  - Complex numbers are interleaved (re, im) pairs.
 */
#ifndef EPIC_H
#define EPIC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct epic_plan_s* epic_plan_t;

typedef enum {
  EPIC_OK = 0,
  EPIC_ERR_INVALID_ARG = 1,    /* bad pointer, size, enum or gamma */
  EPIC_ERR_GRID_TOO_SMALL = 2, /* a gridding stencil falls outside [0, N) */
  EPIC_ERR_CUDA = 3,           /* a CUDA runtime call failed */
  EPIC_ERR_OOM = 4,            /* device or host allocation failed */
  EPIC_ERR_NUMERIC = 5,        /* EPICal held antennas (non-finite / tiny D) */
  EPIC_ERR_TIMEOUT = 6,        /* a bounded device wait gave up */
  EPIC_ERR_UNSUPPORTED = 7,    /* valid request this build cannot run */
  EPIC_ERR_STATE = 8           /* call out of order (e.g. update before image) */
} epic_status;

typedef enum { EPIC_KERNEL_GAUSSIAN = 0, EPIC_KERNEL_TOPHAT = 1 } epic_kernel_type;
typedef enum { EPIC_IN_CI4 = 0, EPIC_IN_COMPLEX64 = 1 } epic_input_format;
typedef enum { EPIC_PREC_FP32 = 0, EPIC_PREC_FP16 = 1, EPIC_PREC_BF16 = 2 } epic_precision;
/* Kernel structure of epic_image.  FUSED: one persistent launch keeps each
 * frame in one SM (N <= 128).  UNFUSED: the plain path, row spectra pass
 * through device memory in batches (N = 32..512).  CLUSTER:
 * one persistent launch in which a thread-block cluster (8 CTAs for N = 256,
 * 16 for N = 512) shares each frame through distributed shared memory.
 * PIPED: the fused path in warp-specialised form (N = 64 or 128, Na <= 512):
 * producer warps grid and row-transform frame t + 1 while consumer warps
 * column-transform frame t, handing frames over through two shared-memory
 * slots (FUSED keeps the form with two CTA barriers per step of two
 * frames, measured faster on this build).  AUTO picks FUSED for N <= 128, else UNFUSED
 * (measured faster than CLUSTER on this build). */
typedef enum {
  EPIC_PATH_AUTO = 0, EPIC_PATH_FUSED = 1, EPIC_PATH_UNFUSED = 2, EPIC_PATH_CLUSTER = 3,
  EPIC_PATH_PIPED = 4
} epic_path;

/* Plan description (Sec. 2.1: antenna positions, grid, kernel, channels). */
typedef struct {
  int n_ant;                   /* Na >= 1 */
  const double* ant_xy_m;      /* host [Na][2]: planar East, North positions, metres */
  int n_chan;                  /* C >= 1 */
  const double* freq_hz;       /* host [C]: channel centre frequencies */
  int grid_n;                  /* N: power of two, 16..128 (FUSED), 32..512 (UNFUSED) */
  double cell_wavelengths;     /* grid cell du in wavelengths (0.5 = full sky) */
  int kernel;                  /* epic_kernel_type: antenna illumination W_a */
  int kernel_support;          /* K: odd stencil side in cells, 1..7 */
  double kernel_param;         /* Gaussian sigma in cells / tophat side in metres */
  int input;                   /* epic_input_format of the voltages */
  const float* voltage_scale;  /* host [C] multiplier per channel, or NULL = 1 */
  const unsigned char* flags;  /* host [Na], 1 = antenna flagged, or NULL */
  int precision;               /* epic_precision of the FFT: FP32, or FP16 / BF16
                                  (column DFT on tensor cores, UNFUSED/AUTO path) */
  void* cuda_stream;           /* cudaStream_t for all work; NULL = default */
  int path;                    /* epic_path */
  size_t workspace_bytes;      /* UNFUSED batch scratch budget; 0 = 2 GiB */
  const double* kernel_param_ant;  /* host [Na]: kernel_param per antenna (heterogeneous
                                      illumination patterns), or NULL = kernel_param for all */
  int batch_persistent;        /* UNFUSED FP32, N = 256 or 512: 1 = every epic_image call is one
                                  persistent cooperative launch over all its batches (grid
                                  barriers between the row, column and correlation phases);
                                  0 = one launch per kernel and batch; epic_autotune may switch it */
} epic_plan_desc;

/* Read-only facts about a plan (epic_plan_get_info). */
typedef struct {
  int n_ant, n_chan, grid_n, kernel_support;
  int window_rows;             /* max over channels of occupied grid rows */
  int cal_kx, cal_ky;          /* calibrator pixel, -1 before epical_configure */
  int ctas;                    /* persistent CTAs used by epic_image */
  int units_per_chan;          /* time segments per channel per call */
  size_t smem_bytes;           /* dynamic shared memory of the image kernel */
  long long frames_pending;    /* frames correlated since the last update */
  long long iteration;         /* completed EPICal updates */
  int path;                    /* epic_path in use (never AUTO) */
  int batch_time;              /* UNFUSED: time samples per batch (0 before use) */
} epic_plan_info;

/* Result of epic_autotune. */
typedef struct {
  int path;                    /* epic_path that was tuned */
  int units_target;            /* FUSED: work units per CTA aimed for */
  int batch_time;              /* UNFUSED: time samples per batch (0 = scratch budget) */
  int cols_target;             /* UNFUSED: column-FFT units per SM aimed for */
  double ms_default, ms_best;  /* epic_image time before / after tuning */
  int candidates;              /* launch shapes timed */
  int row_table;               /* UNFUSED FP32 row kernel: gather table -1 auto, 0 L1, 1 shared memory */
  int row_frames;              /* UNFUSED FP32 row kernel: frames per step (1 or 2) */
  int batch_persistent;        /* UNFUSED FP32: one persistent launch per call (1) or batched (0) */
} epic_tune_result;

/* Build the gridding tables of Eq. 9 for every (channel, antenna): the
 * stencil centre is the nearest cell to u_a/du + N/2 (u_a = r_a f / c),
 * taps are normalised to sum 1 (W(0) = 1, Sec. 2.1).  The kernels grid by
 * gathering: the plan also lists, for every FFT lane, the taps that land on
 * its grid cells (at most 255 taps on one cell).  Uploads tables and sets
 * all gains to 1.  Synchronous.  *out receives the plan.
 * Errors: INVALID_ARG (sizes, enums, NULL arrays), GRID_TOO_SMALL,
 * UNSUPPORTED (N or Na outside the built kernels, or more than 255 taps on
 * one grid cell), CUDA, OOM. */
epic_status epic_plan_create(epic_plan_t* out, const epic_plan_desc* desc);

/* Free the plan and its device memory (waits for its stream). NULL is OK. */
epic_status epic_plan_destroy(epic_plan_t plan);

/* Use another stream for subsequent work. */
epic_status epic_plan_set_stream(epic_plan_t plan, void* cuda_stream);

/* Fill *info.  Host only. */
epic_status epic_plan_get_info(epic_plan_t plan, epic_plan_info* info);

/* Replace the current gains g_a (Eq. 8 divides by them).  gains: host
 * [C][Na] complex128.  Zero or non-finite gains give INVALID_ARG.
 * Synchronous upload. */
epic_status epic_set_gains(epic_plan_t plan, const double* gains);

/* Image one batch of frames (Eqs. 8-10 and the square-and-average step):
 * image[c][ky][kx] (+)= (1/n_time) sum_t |E'(s_k, t)|^2 for every channel.
 * d_volt: device [n_time][C][Na], one byte per sample (EPIC_IN_CI4) or
 * complex float32 (EPIC_IN_COMPLEX64).  d_image: device [C][N][N] float64,
 * pixel (N/2, N/2) is the phase centre, l = (kx - N/2)/(N du).
 * accumulate = 0 overwrites d_image, else adds.  If EPICal is configured
 * the same pass accumulates K_a and P_a of Eqs. 12 and 15 with the
 * uncalibrated E_a into the plan.  Asynchronous.
 * Errors: INVALID_ARG (NULL, n_time < 1), CUDA. */
epic_status epic_image(epic_plan_t plan, const void* d_volt, long long n_time,
                       double* d_image, int accumulate);

/* epic_image on host buffers: copies h_volt (layout as d_volt) to the
 * device, images it and copies the [C][N][N] float64 image back to
 * h_image.  Uses plan-owned device staging buffers (grown on demand).
 * Pinned host memory makes the copies faster.  Synchronous. */
epic_status epic_image_host(epic_plan_t plan, const void* h_volt, long long n_time,
                            double* h_image, int accumulate);

/* epic_image_host for callers that cannot allocate device memory (a
 * real-time loop that may not add a device-synchronising cudaMalloc between
 * intervals, a process held to a device-memory budget fixed at start-up, or
 * host code running where CUDA allocation calls are not allowed).  The paper
 * has no counterpart: this is a deployment variant of the same imaging
 * kernel.  It allocates nothing: voltages and the image are staged through
 * one 32 MiB file-scope device array that every GPU loading the library
 * holds until exit; T is processed in chunks that fit beside the image.
 * Arguments and result as epic_image_host.  The image [C][N][N] float64 plus
 * one time sample of voltages must fit in 32 MiB, else INVALID_ARG with a
 * message.  The call needs a plan on the fused FP32 path (EPIC_PATH_FUSED,
 * what AUTO picks for N <= 128 at FP32); every other path (UNFUSED, CLUSTER,
 * PIPED, FP16/BF16) needs plan scratch and gives UNSUPPORTED before the array
 * is touched.  The first call on a device looks up the array's device address
 * (make that first call before any stream capture); the address is kept for
 * the life of the device's context, so do not call this entry point on a
 * device after cudaDeviceReset.  All calls share the array: calls whose GPU
 * work overlaps (several host threads or plans on different streams) race
 * and must be serialised by the caller.  Synchronous. */
epic_status epic_image_host_static(epic_plan_t plan, const void* h_volt, long long n_time,
                                   double* h_image, int accumulate);

/* Batching form, autotuner: times candidate launch shapes of epic_image on
 * this batch (FUSED: work units per CTA, i.e. the time-segment length of a
 * persistent CTA's work unit; UNFUSED: time samples per batch and
 * column-FFT work units per SM, then for FP32 the row kernel's variant:
 * gather table in shared memory or read through L1, one or two frames per
 * step, and for N = 256 / 512 whether a call runs as one persistent
 * launch), keeps the fastest in the plan and reports it in *out (may be
 * NULL).  d_image is overwritten; EPICal sums are left
 * untouched.  Synchronous.  The paper has no counterpart (run-time tuning
 * of this implementation). */
epic_status epic_autotune(epic_plan_t plan, const void* d_volt, long long n_time, double* d_image,
                          epic_tune_result* out);

/* Batching form, CUDA graph: capture one calibration interval, epic_image
 * of d_volt (n_time samples, all channels) into d_image followed, when
 * EPICal is configured, by epical_update writing d_gains_out (may be NULL),
 * into a graph owned by the plan.  Buffers are bound at capture; the plan
 * stream must not be the legacy default stream.  Replace the graph by
 * capturing again.  Synchronous. */
epic_status epic_graph_capture(epic_plan_t plan, const void* d_volt, long long n_time, double* d_image,
                               double* d_gains_out);

/* Replay the captured interval on the plan stream (one interval: image and,
 * if configured, the gain update).  Asynchronous.  Errors: STATE if no
 * graph was captured. */
epic_status epic_graph_launch(epic_plan_t plan);

/* Arm EPICal (Sec. 2.2).  (cal_l, cal_m): calibrator direction; the pixel
 * used is the nearest pixel centre.  Model: n_src point sources, host
 * src_lmS [n_src][3] rows (l, m, S) with apparent fluxes S, used for every
 * channel; V^M_ab = sum_s S_s exp(-2 pi i (u_a - u_b) . s).  The plan
 * forms D_a = sum_{b != a} conj(A_{0,b}) V^M_ab once (Eq. 16 denominator
 * over Na), A_{0,a} being the exact response of the calibrator pixel to
 * antenna a.  gamma in [0, 1) is the damping of Eq. 17.  g0: host [C][Na]
 * complex128 initial gains or NULL = 1.  Resets the accumulators.
 * Synchronous.  Errors: INVALID_ARG (gamma, pixel outside the image,
 * n_src < 1), CUDA. */
epic_status epical_configure(epic_plan_t plan, double cal_l, double cal_m,
                             int n_src, const double* src_lmS, double gamma,
                             const double* g0);

/* EPICal update of Eqs. 15-17 from the frames imaged since the last update:
 * C_a = <K_a> - conj(A_{0,a}) <P_a> / conj(g_a),
 * g_a <- (1 - gamma) C_a / D_a + gamma g_a, then clears K, P.  Flagged
 * antennas, |D_a| below 1e-30 and non-finite results keep the old gain and
 * are counted (see epic_plan_sync).  d_gains_out: device [C][Na]
 * complex128 copy of the new gains, or NULL.  d_status: device [C][Na]
 * int32 (1 = held), or NULL.  Asynchronous.
 * Errors: STATE (not configured, or no frames since the last update). */
epic_status epical_update(epic_plan_t plan, double* d_gains_out, int* d_status);

/* Multiple-pixel and direction-dependent EPICal (Sec. 6, "Multiple pixel
 * correlations"): correlate every raw antenna signal with the E-field at
 * n_pix calibration pixels instead of the single calibrator pixel, to bring
 * more of the sky's power into the loop at O(Na n_pix) per sample.
 * pix_lm: host [n_pix][2] directions (l, m), each mapped to its nearest
 * pixel centre (two directions on one pixel give INVALID_ARG).  Uses the
 * model sources and gamma of the preceding epical_configure.  Per channel
 * and pixel p the plan forms A_{p,a} (exact response of pixel p to antenna
 * a) and D_{p,a} = sum_{b != a} conj(A_{p,b}) V^M_ab.  From then on
 * epic_image stores E'(s_p, t) of every frame and correlates,
 * K_{a,p} += E_a(t) conj(E'(s_p, t)) (Eq. 12 per pixel, a [Na x T] by
 * [T x n_pix] product per channel), and epical_update applies, with
 * C_{a,p} = <K_{a,p}> - conj(A_{p,a}) <P_a> / conj(g_a) (Eq. 15 per pixel):
 *   imaging gains   g_a <- (1 - gamma) sum_p conj(D_{p,a}) C_{a,p} /
 *                          sum_p |D_{p,a}|^2 + gamma g_a
 *                   (least squares over the pixels of the fixed point
 *                   C_{a,p} = g_a D_{p,a}; Eq. 16 when n_pix = 1),
 *   per direction   g_{a,p} <- (1 - gamma) C_{a,p} / D_{p,a} + gamma g_{a,p}
 *                   (each pixel solved independently, Eqs. 16-17),
 * holding flagged antennas, vanishing denominators and non-finite results
 * as epical_update does.  Per-direction solutions start from the current
 * gains.  Resets the accumulators.  epical_configure returns the plan to the
 * single-pixel form.  The multiple-pixel sums are not part of
 * epical_get_state.  Needs the fused FP32 path (N <= 128), else
 * UNSUPPORTED; epic_image_host_static refuses plans in this form (it needs
 * the tap buffer, plan scratch of T x C x n_pix complex64, grown by
 * epic_image on demand).  Synchronous.
 * Errors: STATE (EPICal not configured), INVALID_ARG, UNSUPPORTED, OOM, CUDA. */
epic_status epical_configure_pixels(epic_plan_t plan, int n_pix, const double* pix_lm);

/* Per-direction gain solutions of the multiple-pixel form to host
 * [C][Na][n_pix] complex128 (pixels in the order given to
 * epical_configure_pixels).  Synchronous.  Errors: STATE if the plan is not
 * in the multiple-pixel form. */
epic_status epical_get_direction_gains(epic_plan_t plan, double* h_gains);

/* Visibility-based comparison path (Sec. 4, noise trends; Sec. 5 checks the
 * LWA solutions the same way).  X-engine: every antenna pair's visibility
 * from the voltage stream EPICal uses,
 *   V[c][a][b] (+)= (1/n_time) sum_t E_a(t) conj(E_b(t)),
 * E_a = voltage_scale[c] x the raw sample (uncalibrated, flags ignored),
 * autocorrelations included.  d_volt: device [n_time][C][Na] as for
 * epic_image.  d_vis: device [C][Na][Na] complex128, caller-owned
 * (Hermitian: both triangles written); accumulate = 0 overwrites, else adds.
 * For 4-bit input the product runs on the tensor cores: the samples are
 * packed as FP16 integers into a plan-owned operand matrix (time segments
 * that keep it within 1 GiB, grown on demand) and multiplied by tcgen05 MMAs
 * with FP32 accumulation, every partial sum an integer below 2^24, so the
 * per-channel sums are exact.  Complex64 input runs on the CUDA cores in
 * FP32 (segments of 32768 samples added in FP64).
 * Asynchronous.  Errors: INVALID_ARG, OOM, CUDA, TIMEOUT (bounded waits of
 * the tensor-core kernel, through epic_plan_sync). */
epic_status epic_visibilities(epic_plan_t plan, const void* d_volt, long long n_time, double* d_vis,
                              int accumulate);

/* Visibility-based gain solve: minimise Eq. 21,
 *   chi^2 = sum_a sum_{b != a} |V_ab - g_a conj(g_b) V^M_ab|^2,
 * per channel by alternating least squares with every other iterate
 * averaged (StEFCal, Salvini & Wijnholds 2014; the paper names no solver):
 *   g_a <- sum_b V_ab g_b conj(V^M_ab) / sum_b |g_b V^M_ab|^2
 * over unflagged b != a with |u_a - u_b| >= min_baseline wavelengths (Sec. 5
 * leaves out baselines shorter than 10 wavelengths; 0 keeps all), until
 * max_a |g_new - g| <= tol max_a |g_new| or max_iter iterations.  V^M is
 * formed in FP64 from the point-source model of the last epical_configure
 * (V^M_ab = sum_s S_s e^{-2 pi i (u_a - u_b) . s}) on the first solve after
 * it.  The pair products run in FP32 (V and V^M rounded to FP32; the plan
 * holds 2 x C x Na x Na complex64 for them), the sums over antennas, the
 * update, the averaging and the stopping test in FP64, so the solution
 * agrees with an FP64 solve to about 1e-6; the stopping tolerance used is
 * max(tol, 1e-6).  d_vis: device [C][Na][Na]
 * complex128 (as from epic_visibilities).  d_gains: device [C][Na]
 * complex128, the start on input and the solution on output; flagged
 * antennas and antennas with no usable pair keep their start value.
 * h_iters: host [C] iterations used, or NULL (then the call is
 * asynchronous; else synchronous).
 * Errors: STATE (EPICal not configured), INVALID_ARG, UNSUPPORTED
 * (Na > 5120), OOM, CUDA. */
epic_status epic_visibility_solve(epic_plan_t plan, const double* d_vis, double* d_gains, int max_iter,
                                  double tol, double min_baseline, int* h_iters);

/* Gains taken as constant across a band of channels (Sec. 5: the LWA
 * demonstration averages the per-channel solutions across its central
 * channels to raise the signal to noise).  For every unflagged antenna the
 * gains of channels c_lo <= c < c_hi are replaced by their plain complex
 * mean (and 1/g with them); other channels and flagged antennas are left as
 * they are, and so is an antenna whose mean is zero or not finite.  Call
 * after epical_update; the next epic_image uses the averaged gains.
 * Asynchronous on the plan stream.
 * Errors: INVALID_ARG (NULL plan, unless 0 <= c_lo < c_hi <= C), CUDA. */
epic_status epical_average_channels(epic_plan_t plan, int c_lo, int c_hi);

/* Gain model across frequency (Sec. 6, "Fitting gain models": a low-order
 * polynomial in amplitude and in phase over a band of channels, a step
 * beyond the constant-across-band average of epical_average_channels).
 * For every unflagged antenna, the amplitudes |g| and the phases arg g of
 * channels c_lo <= c < c_hi (phases unwrapped along the band from c_lo, each
 * step taken within pi) are fitted by least squares with polynomials of
 * degrees deg_amp and deg_phase in x, the channel frequency mapped linearly
 * onto [-1, 1] over the band; the band's gains (and 1/g) are replaced by
 * A(x) e^{i Phi(x)}.  An antenna with a zero or non-finite gain in the band
 * is left as it is.  Call after epical_update.  FP64.  Synchronous.
 * Errors: INVALID_ARG (band, or degrees outside 0..7 or not below the
 * number of channels in the band), CUDA. */
epic_status epical_fit_bandpass(epic_plan_t plan, int c_lo, int c_hi, int deg_amp, int deg_phase);

/* Phase centre away from zenith (Sec. 2.1 footnote: a phase applied to the
 * electric fields as one phases visibilities).  Every voltage of antenna a
 * in channel c is multiplied by p_a = e^{+2 pi i u_a . s0}, s0 = (l0, m0),
 * u_a = r_a f_c / c, together with the gain correction (the stored
 * multiplier becomes p_a / g_a), so that the image is centred on s0:
 * pixel kx holds l = l0 + (kx - N/2)/(N du), and likewise for m.  EPICal
 * uses the phased responses (A_{0,a} p_a) and takes calibrator and
 * calibration-pixel directions relative to s0; the gains keep their Eq. 7
 * meaning and the gradient of epic_image_backward stays with respect to g.
 * (0, 0) returns to zenith.  EPICal must be configured again afterwards
 * (the call resets it).  Synchronous.
 * Errors: INVALID_ARG (l0^2 + m0^2 >= 1), OOM, CUDA. */
epic_status epic_set_phase_centre(epic_plan_t plan, double l0, double m0);

/* Failure detection (no counterpart in the paper): the warp-specialised
 * fused form (EPIC_PATH_PIPED) hands frames between its producer and
 * consumer warps through mbarriers, and the persistent unfused form
 * (batch_persistent) orders its phases with grid-wide barriers; every such
 * wait gives up after a bounded number of polls, the kernel then raises the
 * plan's error flag, stops waiting and runs to its end, and the next
 * epic_plan_sync returns EPIC_ERR_TIMEOUT (the image of that call is not
 * valid; the context stays usable).  This call sets that number of polls
 * for the plan's later launches of those forms (0 = the default: about
 * 10^6 for the mbarriers, 2^22 for the grid barrier); a small value makes
 * the waits run out, which is how the timeout path is tested.  Kernels that
 * have asynchronous copies in flight keep their own limits.  Host only.
 * Errors: INVALID_ARG (polls < 0). */
epic_status epic_plan_set_wait_limit(epic_plan_t plan, int polls);

/* Wait for the plan's stream.  *n_held (may be NULL) receives the number
 * of held (antenna, channel) gains since the previous sync; the call
 * returns EPIC_ERR_NUMERIC if it is non-zero.  Synchronous. */
epic_status epic_plan_sync(epic_plan_t plan, int* n_held);

/* Current gains to host [C][Na] complex128.  Synchronous. */
epic_status epical_get_gains(epic_plan_t plan, double* h_gains);

/* Checkpoint: EPICal state (gains, accumulators, counters) to host.  With
 * buf == NULL only *bytes is set.  Synchronous. */
epic_status epical_get_state(epic_plan_t plan, void* buf, size_t* bytes);

/* Resume from epical_get_state output of a plan with the same C and Na.
 * Errors: INVALID_ARG (size or header mismatch).  Synchronous. */
epic_status epical_set_state(epic_plan_t plan, const void* buf, size_t bytes);

/* Set the gains from device memory (d_gains: device [C][Na] complex128),
 * asynchronously on the plan stream; w = 1/g is formed on the device.  Zero
 * gains give non-finite multipliers (no check, no host round trip). */
epic_status epic_set_gains_device(epic_plan_t plan, const double* d_gains);

/* Differentiation form: gradient of a real loss L(I) of the dirty image
 * with respect to the complex gains.  Given d_dl_di = dL/dI (device
 * [C][N][N] float64, I as produced by epic_image on the same d_volt and the
 * plan's current gains), writes d_grad_g (device [C][Na] complex128) =
 * 2 dL/dconj(g), the convention of torch complex autograd, so that
 * dL = Re(conj(grad) dg).  Through w = 1/g (Eq. 8) and Eqs. 9-10:
 * dL/dconj(w_a) = (1/T) sum_t conj(E_a(t)) sum_k conj(A_{k,a}) R_k E'(s_k,t),
 * R = dL/dI, evaluated as inverse FFTs of R . E' followed by degridding;
 * every frame is recomputed, none is stored.  Flagged antennas get 0.
 * Fused path only (N <= 128), else UNSUPPORTED.  Asynchronous. */
epic_status epic_image_backward(epic_plan_t plan, const void* d_volt, long long n_time,
                                const double* d_dl_di, double* d_grad_g);

/* Arithmetic of the transforms in epic_image_backward: EPIC_PREC_FP32 (the
 * default) or EPIC_PREC_BF16, where two frames at a time go through the
 * four FFTs, the multiply by R and the shared-memory exchanges as BF16
 * pairs (gridding sums, degridding sums, the conj(E_a) products and the
 * accumulation stay FP32, the gradient sums FP64).  The BF16 gradient
 * carries the rounding of 8-bit significands through about 4 log2(N)
 * butterfly levels (a relative error of order 10^-2).  Host only; applies
 * to later calls.  Errors: INVALID_ARG (another precision). */
epic_status epic_plan_set_adjoint_precision(epic_plan_t plan, int precision);

/* Debug/test accessors (synchronous, host outputs). */
/* base_xy: host [C][Na][2] int32 stencil-centre cell (x, y); w: host
 * [C][Na][K][K] float64 normalised tap weights ([dy][dx]); either may be
 * NULL.  Flagged antennas have zero weights. */
epic_status epic_plan_get_grid_table(epic_plan_t plan, int* base_xy, double* w);

/* Unpack n 4-bit complex bytes (device d_in) to device float32 pairs
 * d_out [n][2] exactly (high nibble real, low nibble imaginary, two's
 * complement).  Asynchronous. */
epic_status epic_unpack_ci4(epic_plan_t plan, const unsigned char* d_in, float* d_out,
                            long long n);

/* Measurement aid (no counterpart in the paper): launch a grid of `blocks`
 * CTAs of 256 threads, each thread running 8 independent chains of
 * 16 * iters fused multiply-adds in FP32 (fp64 = 0) or FP64 (fp64 != 0), on
 * cuda_stream (cudaStream_t, NULL = default).  *flops receives the FLOP
 * count of the launch (2 per multiply-add), so that a caller timing the
 * launch with CUDA events obtains the device's FMA rate: the roofline
 * denominator of the FP32-arithmetic-bound imaging kernels.  d_sink: device
 * buffer of at least `blocks` floats (doubles for FP64), never written for
 * these arguments.  Asynchronous.  Errors: INVALID_ARG, CUDA. */
epic_status epic_measure_fma_peak(int fp64, int blocks, long long iters, void* d_sink,
                                  void* cuda_stream, double* flops);

/* Message of the last failed call on this thread ("" if none). */
const char* epic_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* EPIC_H */
