// Internal interface between the host plan (epic_plan.cpp) and the CUDA
// kernels (epic_kernels.cu).  Not part of the public C ABI.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>

namespace epic {

// Arguments of one fused imaging launch (gain correction, gridding, 2D FFT,
// square-accumulate and the EPICal correlation for every frame of a batch).
struct ImageArgs {
  const void* volt;        // device [T][C][Na] u8 (ci4) or float2
  int input_fmt;           // 0 = ci4, 1 = complex64
  long long n_time;        // T
  int n_chan, n_ant;       // C, Na
  int support;             // K
  const int* cell0;        // [C][Na] window cell of tap (0,0); -1 = flagged
  const float* wts;        // [C][Na][K*K] weights * (-1)^(jx+jy) / Na
  const float2* wgain;     // [C][Na] 1/g (gain correction multiplier)
  const float* vscale;     // [C] voltage scale, or nullptr
  const int2* win;         // [C] (first occupied grid row y0, occupied rows R)
  const int4* win4;        // [C] (y0, rows, x0, columns) of the occupied window
  const int* cellf;        // [C][Na] window cell (row * (N + N1) + col - x0); -1 = flagged
  const int* gofs;         // [C][rows_alloc][N1] first gather entry of each FFT lane,
                           // relative to the channel's first entry
  const uint4* gcnt;       // [C][rows_alloc][N1] entries of each column block j (byte j)
  const uint2* gent;       // gather entries (antenna, weight bits), lane by lane,
                           // grouped by column block j
  const int* gbase;        // [C + 1] first entry of each channel in gent
  int gsmem;               // 1: the channel's table is copied to shared memory per unit
  int piped;               // 1: warp-specialised form (epic_image_piped)
  int steps;               // fused form: frames per step (spectra slots), 1 or 2
  int* err;                // device flag: a bounded wait timed out (piped form)
  const float2* pixph;     // [C] (-1)^(k0x+k0y) e^{2 pi i (x0 k0x + y0 k0y)/N}
  const float2* twid;      // [N] e^{+2 pi i m / N}
  double* image;           // [C][N][N] accumulated with img_scale
  double img_scale;        // 1 / T_call
  int do_cal;              // accumulate K, P
  int k0x, k0y;            // calibrator pixel
  float pix_sign;          // (-1)^(k0x+k0y): centring factor of the image
  double2* kacc;           // [C][Na] sum_t E_a conj(P(t))
  double* pacc;            // [C][Na] sum_t |E_a|^2
  int segs;                // time segments per channel (units = C * segs)
  int rows_alloc;          // shared-memory grid rows (max R)
  int rs;                  // row stride of the transposed (swizzled) buffer
  int grid;                // CTAs launched
  size_t smem;             // dynamic shared memory bytes
  // multiple-pixel EPICal (0 pixels = off): the column-pass owner of each
  // calibration pixel stores E'(s_p, t) to ptap[t][C][npix] (tap order)
  int wait_limit;           // warp-specialised form: polls per bounded wait (0 = default)
  int npix;
  const uint2* ptab;       // [COLROUNDS][BT] (slot mask, first tap index) per thread
  const float2* pph;       // [C][npix] window-coordinate phase of each pixel
  float2* ptap;            // [T][C][npix] pixel taps of the call
};

// Shape facts of the fused image kernel for grid side n.
struct ImageKernelShape {
  int threads;             // CTA size
  int groups;              // 1-D FFTs in flight per CTA
  int max_ant;             // largest Na the kernel holds in registers
};

bool image_kernel_shape(int n, ImageKernelShape* out);
// Owner of image pixel (kx, ky) in the fused kernel's column pass: column
// round, thread index and register slot.
struct PixelOwner {
  int round, thread, slot;
};
bool image_pixel_owner(int n, int kx, int ky, PixelOwner* out);
int image_col_rounds(int n);

// Multiple-pixel EPICal (epic_multipix.cu).
struct MultiCorrArgs {
  const void* volt;        // device [T][C][Na] of the call
  int input_fmt;
  long long n_time;
  int n_chan, n_ant, npix;
  const float* vscale;     // [C] or nullptr
  const int* cell0;        // [C][Na]; < 0 = flagged (skipped)
  const float2* ptap;      // [T][C][npix] pixel taps
  double2* kmp;            // [C][Na][npix] sum_t E_a conj(tap_p)
  int segs;                // time segments per channel
};
cudaError_t launch_correlate_multi(const MultiCorrArgs& a, cudaStream_t s);
struct MultiUpdateArgs {
  int n_chan, n_ant, npix;
  double2* kmp;            // [C][Na][npix], cleared
  double2* kacc;           // [C][Na] single-pixel sums, cleared
  double* pacc;            // [C][Na], cleared
  double inv_frames;
  const double2* ap;       // [C][npix][Na] A_{p,a}
  const double2* dp;       // [C][npix][Na] D_{p,a}
  double2* gain;           // [C][Na] imaging gains (joint solution)
  float2* wgain;           // [C][Na] 1/g
  double2* gdir;           // [C][Na][npix] per-direction solutions
  const unsigned char* flags;
  double gamma, dmin;
  double2* gout;           // [C][Na] or nullptr
  int* status;             // [C][Na] or nullptr
  int* held_count;
  const double2* phase;    // [C][Na] phasing factors, or nullptr
};
cudaError_t launch_update_multi(const MultiUpdateArgs& a, cudaStream_t s);

// Visibility-based comparison path (epic_xengine.cu).
struct XengineArgs {
  const void* volt;        // device [T][C][Na]
  int input_fmt;
  long long n_time;
  int n_chan, n_ant;
  const float* vscale;     // [C] or nullptr
  double scale;            // 1 / T
  double2* vis;            // [C][Na][Na], accumulated (atomics)
};
cudaError_t launch_xengine(const XengineArgs& a, cudaStream_t s);
// Tensor-core X-engine for 4-bit input (epic_tc.cu): pack to FP16 Z
// [C][2 Na_p][Tp], then G = Z Z^T on tcgen05, upper-triangle tiles.
struct XeTcArgs {
  int n_chan, n_ant;
  int na_p;                // antennas padded to a multiple of 64
  int tp;                  // samples of this segment padded to a multiple of 64
  const float* vscale;     // [C] or nullptr
  double scale;            // 1 / T of the whole call
  double2* vis;            // [C][Na][Na]
  int accumulate;          // 1: add to vis, 0: overwrite
  int* err;                // bounded-wait timeout flag
};
cudaError_t xe_prepare();
bool xe_make_map(void* z, int n_chan, int na_p, int tp, void* tm);
cudaError_t launch_xengine_tc(const XeTcArgs& a, const void* volt, long long t0, int nt, void* z, const void* tm,
                              int sms, cudaStream_t s);
cudaError_t launch_model_vis(int n_chan, int n_ant, int n_src, const double2* ph, const double* flux,
                             float2* vm, cudaStream_t s);
struct StefcalArgs {
  int n_chan, n_ant;
  float2* vis32;           // [C][Na][Na] scratch: the visibilities rounded to FP32
  const float2* vm;        // [C][Na][Na] model visibilities (FP32)
  const double2* uv;       // [C][Na] antenna positions in wavelengths
  const unsigned char* flags;
  double min_baseline;     // wavelengths; shorter pairs are left out
  double tol;
  int max_iter;
  double2* gains;          // [C][Na] in: start, out: solution
  int* iters;              // [C] iterations used, or nullptr
};
// Rounds vis64 into a.vis32, then solves.
cudaError_t launch_stefcal(const StefcalArgs& a, const double2* vis64, cudaStream_t s);
int image_rs(int rows_alloc);
int image_rs_fused(int rows_alloc);

// Dynamic shared memory of the adjoint kernel (layout: window [rows][N],
// spectra [N][rs], FFT exchange, twiddles, E' [Na]).
// Dynamic shared memory of the adjoint kernel (bf16: the BF16 frame-pair form).
size_t adjoint_smem_bytes(int n, int rows_alloc, int rs, int n_ant, bool bf16);
// Row stride of the fused kernel's grid window, N + N1.
int image_window_stride(int n);
size_t image_smem_bytes(int n, int n_ant, int rs, int steps);
// Frames per step the fused kernel supports for grid side n (1 or 2).
int image_max_steps(int n);
// Shared memory of a channel's gather table (lane offsets + up to gmax entries).
size_t image_table_bytes(int rows_alloc, int n1, long long gmax);
// Lanes per 1-D FFT (N1) of the fused kernel: window column x is entry
// block j = x / N1 of lane x % N1.
int image_fft_lanes(int n);
// Opt in to the shared memory and report resident CTAs per SM.
cudaError_t image_kernel_prepare(int n, size_t smem, int n_ant, int steps, int* ctas_per_sm);
cudaError_t launch_image(int n, const ImageArgs& a, cudaStream_t s);

// Warp-specialised fused form (N = 64, 128): producer warps grid and row-FFT
// frame t + 1 while consumer warps column-FFT frame t (two spectra slots).
bool piped_supported(int n, int n_ant);
// Dynamic shared memory; gmax > 0 adds the gather table (gmax entries).
size_t piped_smem_bytes(int n, int n_ant, int rs, int rows_alloc, long long gmax);
cudaError_t piped_prepare(int n, size_t smem, bool table_in_smem, int* ctas_per_sm);
cudaError_t launch_piped(int n, const ImageArgs& a, cudaStream_t s);

struct UpdateArgs {
  int n_chan, n_ant;
  double2* kacc;           // [C][Na], cleared by the update
  double* pacc;            // [C][Na], cleared by the update
  double inv_frames;       // 1 / frames accumulated
  const double2* a0;       // [C][Na] A_{0,a}
  const double2* dden;     // [C][Na] D_a
  double2* gain;           // [C][Na] g (updated in place)
  float2* wgain;           // [C][Na] 1/g as float2 (updated)
  const unsigned char* flags;  // [Na]
  double gamma;
  double dmin;
  double2* gout;           // [C][Na] or nullptr
  int* status;             // [C][Na] or nullptr
  int* held_count;         // device counter
  const double2* phase;    // [C][Na] phasing to the phase centre (w = p / g), or nullptr
};
cudaError_t launch_update(const UpdateArgs& a, cudaStream_t s);

cudaError_t launch_unpack(const unsigned char* in, float2* out, long long n, cudaStream_t s);

// Adjoint (gain gradient) launch of the fused structure, N <= 128.
struct AdjointArgs {
  const void* volt;
  int input_fmt;
  long long n_time;
  int n_chan, n_ant, support;
  const int* cell0;
  const float* wts;
  const float2* wgain;
  const float* vscale;
  const int2* win;
  const float2* twid;
  const int* gofs;         // gridding gather (absolute columns): [C][rows_alloc][N1] lane offsets
  const uint4* gcnt;       // [C][rows_alloc][N1] entries per column group (bytes)
  const uint2* gent;       // entries (antenna, weight bits)
  const int* gbase;        // [C + 1] first entry of each channel
  const double* dldi;      // [C][N][N] dL/dI
  double2* dldw;           // [C][Na] accumulated dL/dconj(w), pre-zeroed
  double img_scale;        // 1 / T
  int segs, rows_alloc, rs, grid;
  size_t smem;
};
// bf16: spectra of two frames at a time as BF16 pairs (FP32 gridding,
// degridding and accumulation), else FP32 throughout.
cudaError_t launch_adjoint(int n, const AdjointArgs& a, bool bf16, cudaStream_t s);
// phase: [C][Na] phasing factors p (the multiplier is w = p / g), or nullptr.
cudaError_t launch_adjoint_finalize(int n_chan, int n_ant, const double2* dldw, const double2* gain,
                                    const double2* phase, const unsigned char* flags, double2* out,
                                    cudaStream_t s);
cudaError_t launch_set_gains(int n, const double2* g_in, double2* g, float2* w, const double2* phase,
                             cudaStream_t s);
// Complex mean of the gains of channels [c_lo, c_hi) per unflagged antenna.
cudaError_t launch_average_channels(int n_ant, int c_lo, int c_hi, const unsigned char* flags, double2* gain,
                                    float2* wgain, const double2* phase, cudaStream_t s);
// Polynomial gain model across channels [c_lo, c_hi); x: device [c_hi - c_lo] abscissa.
cudaError_t launch_fit_bandpass(int n_ant, int c_lo, int c_hi, int deg_amp, int deg_phase, const double* x,
                                const unsigned char* flags, double2* gain, float2* wgain, const double2* phase,
                                cudaStream_t s);

// Arguments of one batch of the plain unfused path (epic_unfused.cu).
struct UnfusedArgs {
  const void* volt;        // device [T][C][Na] (whole call; batches index into it)
  int input_fmt;
  int n_chan, n_ant, support, grid_n;
  const int* cell0;        // [C][Na] window cell of tap (0,0); -1 = flagged
  const float* wts;        // [C][Na][K*K] folded weights
  const float2* wgain;     // [C][Na] 1/g
  const float* vscale;     // [C] or nullptr
  const int2* win;         // [C] (y0, rows)
  const float2* twid;      // [N]
  float2* spec;            // scratch [nt*C][N][rs] transposed row spectra
  const int* gofs;         // [C][rows_alloc][N1] first gather entry of each row-FFT lane
  const uint4* gcnt;       // [C][rows_alloc][N1][ceil(N2/16)] entries per column group (bytes)
  const uint2* gent;       // gather entries (antenna, weight bits), lane by lane, by group
  const int* gbase;        // [C + 1] first entry of each channel
  float2* pix;             // scratch [nt*C] calibrator pixel per frame
  int rows_alloc, rs;
  double* image;           // [C][N][N]
  double img_scale;
  int do_cal, k0x, k0y;
  float pix_sign;
  double2* kacc;
  double* pacc;
  int cols_target;         // column-FFT work units per SM to aim for
  // plain FP32 path (window coordinates): the gather tables above hold
  // window columns; the calibrator pixel takes the window phase pixph
  const float2* pixph;     // [C] (-1)^(k0x+k0y) e^{2 pi i (x0 k0x + y0 k0y)/N}
  int max_cols;            // widest channel's occupied columns
  int gmax;                // most gather entries of one channel
  int* err;                // device flag: a bounded wait timed out
  int row_table;           // row kernel's gather table: -1 auto, 0 L1, 1 shared memory
  int row_frames;          // row kernel's frames per step, 1 or 2
  int sms;                 // SMs of the device (persistent form's work split)
  int wait_limit;          // persistent form: polls per grid-barrier wait (0 = default)
};
// One persistent cooperative launch for a whole call (N = 256, 512): rows,
// grid barrier, columns, grid barrier, correlation, per batch of nt_batch
// samples.  bar: device {count, generation, abort} (count reset here).
bool persistent_supported(int n);
cudaError_t launch_unfused_persistent(const UnfusedArgs& a, long long n_time, int nt_batch, unsigned* bar, int sms,
                                      cudaStream_t s);
bool unfused_supported(int n);
// Lanes per row FFT (N1) of the unfused kernels: absolute column x is gather
// group j = x / N1 of lane x % N1.
int unfused_fft_lanes(int n);
cudaError_t launch_correlate(const UnfusedArgs& a, long long t0, int nt, cudaStream_t s);

// Thread-block-cluster imaging for N = 256 / 512, epic_cluster.cu.
struct ClusterArgs {
  const void* volt;
  int input_fmt;
  long long n_time;
  int n_chan, n_ant, support;
  const int* rowcol;       // [C][Na] stencil top window row << 16 | first window column; -1 flagged
  const int* order;        // [C][Na] unflagged antennas sorted by stencil top row
  const int2* ranges;      // [C][CS] range of `order` whose stencils meet each CTA's rows
  const float* wts;        // [C][Na][K*K] folded weights
  const float2* wgain;     // [C][Na] 1/g
  const float* vscale;     // [C] or nullptr
  const int4* win4;        // [C] (y0, rows, x0, cols)
  const float2* twid;      // [N]
  const float2* pixph;     // [C] calibrator-pixel phase (window coordinates)
  double* image;
  double img_scale;
  int do_cal, k0x, k0y;
  double2* kacc;
  double* pacc;
  int segs, rpc_alloc, rs, grid;
  int frames_per_step;     // frames per pair of cluster barriers (spectra slots)
  size_t smem;
};
bool cluster_supported(int n);
int cluster_size(int n);
size_t cluster_smem_bytes(int n, int rpc_alloc, int rs, int frames_per_step);
cudaError_t cluster_prepare(int n, size_t smem, int* clusters);
cudaError_t launch_cluster(int n, const ClusterArgs& a, cudaStream_t s);

// Reduced-precision (tensor-core column DFT) batch, epic_tc.cu.
struct TcArgs {
  UnfusedArgs u;           // gridding inputs (window-column lists), image, pixel, EPICal sums
  void* hh;                // [C*N][tb_cap][kp] FP16/BF16 scaled row spectra
  float* fscale;           // [tb_cap*C] per-frame power-of-two scale s_f
  float* finv2;            // [tb_cap*C] 1 / s_f^2
  int tb_cap, kp, bf16;
  int* err;                // device flag: a bounded wait timed out
  void* gh;                // [tb_cap*C*r_alloc][kr] FP16/BF16 scaled window grid
  int kr;                  // K extent of the row DFT (2 x window columns, padded to 64)
  int r_alloc;             // grid rows per frame in gh (max occupied rows)
  const int4* win4;        // [C] (y0, rows, x0, cols)
  const void* tm_gh;       // host CUtensorMap over gh
  const void* tm_fr;       // host CUtensorMap over the row DFT matrix [2N][kr]
};
bool tc_make_row_maps(void* gh, void* dftr, long long rows_cap, int n, int kr, bool bf16, void* tm_gh,
                      void* tm_fr);
bool tc_supported(int n, int rows_alloc);
int tc_kp(int rows_alloc);
size_t tc_smem(int kp);
cudaError_t tc_prepare(bool bf16, size_t smem);
bool tc_make_maps(void* dft, void* hh, int n, int n_chan, int tb_cap, int kp, bool bf16, void* tm_dft,
                  void* tm_data);
cudaError_t launch_tc_batch(const TcArgs& a, const void* tm_dft, const void* tm_data, long long t0, int nt,
                            int sms, cudaStream_t s);
// Enqueue the four kernels of one batch of nt time samples starting at t0.
cudaError_t launch_unfused_batch(const UnfusedArgs& a, long long t0, int nt, int sms, cudaStream_t s);

}  // namespace epic

// ---- helpers for entry points outside epic_plan.cpp ----
struct epic_plan_s;
namespace epic {
// One fused imaging launch over a device batch: adds (img_scale * sum_t
// |E|^2) into d_image (no clearing) and, when EPICal is armed, counts the
// frames toward the next update.
int image_batch_scaled(epic_plan_s* p, const void* d_volt, long long n_time, double* d_image,
                       double img_scale);
size_t plan_frame_bytes(const epic_plan_s* p);   // voltages of one time sample, all channels
size_t plan_image_elems(const epic_plan_s* p);   // C * N * N
cudaStream_t plan_stream(const epic_plan_s* p);
int plan_device(const epic_plan_s* p);
int plan_path(const epic_plan_s* p);            // epic_path in use (never AUTO)
int set_error(int status, const char* msg);     // records epic_last_error(), returns status
}  // namespace epic
