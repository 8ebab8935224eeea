// Host side of the EPIC/EPICal C ABI: plan validation, FP64 table
// construction, device memory, launches.  See include/epic.h.
#include "../../include/epic.h"

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "epic_internal.h"

namespace {

// NVTX range over one entry point (named in timeline tools such as Nsight
// Systems; a no-op without an attached tool).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};


constexpr double kC = 299792458.0;  // speed of light, m/s
constexpr double kPi = 3.14159265358979323846;
constexpr double kDmin = 1e-30;     // |D_a| at or below this holds the gain

thread_local std::string g_last_error;

epic_status fail(epic_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

epic_status cuda_fail(cudaError_t e, const char* what) {
  return fail(EPIC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define EPIC_CUDA(call)                                          \
  do {                                                           \
    cudaError_t e_ = (call);                                     \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);          \
  } while (0)

template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaError_t alloc(size_t count) {
    release();
    if (count == 0) return cudaSuccess;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&p), count * sizeof(T));
    if (e == cudaSuccess) n = count;
    else p = nullptr;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
};

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

}  // namespace

namespace {
// Multiplier of Eq. 8 for entry i ([C][Na] order): w = p_i / g with the
// phasing factor p_i of the plan's phase centre (1 at zenith).
float2 gain_multiplier_host(const std::vector<double2>& phase, size_t i, double gr, double gi) {
  const double m2 = gr * gr + gi * gi;
  double wr = gr / m2, wi = -gi / m2;
  if (!phase.empty()) {
    const double2 q = phase[i];
    const double xr = wr * q.x - wi * q.y, xi = wr * q.y + wi * q.x;
    wr = xr;
    wi = xi;
  }
  return make_float2(static_cast<float>(wr), static_cast<float>(wi));
}
}  // namespace

struct epic_plan_s {
  // description
  int na = 0, nc = 0, n = 0, k = 0, input = 0, kernel = 0;
  double cell = 0.5, kparam = 0.5;
  std::vector<double> kparam_ant;   // per-antenna kernel parameter (empty: kparam for all)
  std::vector<double> ant;      // [Na][2]
  std::vector<double> freq;     // [C]
  std::vector<float> vscale;    // [C]
  std::vector<unsigned char> flags;  // [Na]
  cudaStream_t stream = nullptr;
  int device = 0;

  // host tables (FP64, as computed)
  std::vector<int> base;        // [C][Na][2]
  std::vector<double> w64;      // [C][Na][K*K]
  std::vector<int> y0, rows;    // [C]
  int rows_alloc = 0;

  // device tables
  DevBuf<int> d_cell0;          // [C][Na]
  DevBuf<float> d_wts;          // [C][Na][K*K] folded
  DevBuf<float2> d_wgain;       // [C][Na] 1/g
  DevBuf<double2> d_gain;       // [C][Na] g
  DevBuf<float> d_vscale;       // [C]
  DevBuf<int2> d_win;           // [C]
  DevBuf<int4> d_win4;          // [C] (y0, rows, x0, cols) for the fused kernel
  DevBuf<int> d_cellf;          // [C][Na] fused-kernel window cell of tap (0,0)
  DevBuf<int> d_gofs;           // [C][rows_alloc][N1] fused gather: first entry per FFT lane
  DevBuf<uint2> d_gent;         // fused gather entries (antenna << 5 | j, weight bits)
  DevBuf<int> d_gbase;          // [C + 1] first gather entry of each channel
  DevBuf<uint4> d_gcnt;         // [C][rows_alloc][N1] gather group lengths (bytes)
  DevBuf<int> d_ugofs;          // unfused gather: [C][rows_alloc][N1] lane offsets
  DevBuf<uint4> d_ugcnt;        // unfused gather: [C][rows_alloc][N1][ceil(N2/16)] group lengths
  DevBuf<uint2> d_ugent;        // unfused gather entries (antenna, weight bits)
  DevBuf<int> d_ugbase;         // [C + 1] first unfused gather entry of each channel
  int gsmem = 0;                // fused gather table held in shared memory
  bool piped = false;           // fused path in its warp-specialised form
  int steps = 1;                // fused form: frames per step
  DevBuf<float2> d_pixph;       // [C] calibrator-pixel phase in window coordinates
  std::vector<int> x0, cols;    // [C] first occupied column, occupied columns
  int rs_fused = 0;
  int gmax = 0;                 // most gather entries of one channel (window tables)
  DevBuf<float2> d_twid;        // [N]
  DevBuf<unsigned char> d_flags;  // [Na]

  // EPICal
  bool cal = false;
  int k0x = -1, k0y = -1;
  double gamma = 0.5;
  DevBuf<double2> d_a0, d_dden, d_kacc;
  DevBuf<double> d_pacc;
  DevBuf<int> d_held;
  long long frames = 0;
  long long iteration = 0;

  // launch shape
  epic::ImageKernelShape shape{};
  size_t smem = 0;
  int rs = 0;
  int ctas = 0;
  int sms = 0;

  // host-API staging
  DevBuf<unsigned char> d_stage_in;
  DevBuf<double> d_stage_img;

  // path and unfused scratch
  int path = EPIC_PATH_FUSED;
  size_t workspace_budget = static_cast<size_t>(2) << 30;
  DevBuf<float2> d_ws;          // unfused scratch: [nt*C] x (N*rs + 1)
  int ws_time = 0;              // time samples the scratch holds

  // differentiation form
  DevBuf<double2> d_dldw;       // [C][Na] dL/dconj(w) accumulator

  // launch-shape parameters (autotuner) and the captured interval graph
  int tune_units = 4;           // fused: work units per CTA to aim for
  int tune_nt = 0;              // unfused: time samples per batch (0 = budget)
  int tune_cols = 4;            // unfused: column units per SM to aim for
  int tune_row_table = -1;      // unfused row kernel: gather table -1 auto, 0 L1, 1 shared memory
  int tune_row_frames = 2;      // unfused row kernel: frames per step
  int wait_limit = 0;           // warp-specialised and persistent forms: polls per bounded wait (0 = default)
  int persistent = 0;           // unfused FP32, N = 256 / 512: one persistent launch per call
  int adjoint_precision = EPIC_PREC_FP32;   // arithmetic of the adjoint's transforms
  DevBuf<unsigned> d_gbar;      // grid barrier {count, generation, abort}
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;

  // reduced-precision form (tensor-core column DFT)
  int precision = EPIC_PREC_FP32;
  int kp = 0;                   // K extent of the DFT (2 x window rows, padded to 64)
  int tc_time = 0;              // time samples per batch
  DevBuf<uint16_t> d_tc_hh;     // [C*N][tc_time][kp]
  DevBuf<uint16_t> d_tc_dft;    // [2N][kp]
  DevBuf<float> d_tc_scale;     // [tc_time*C]
  DevBuf<float2> d_tc_pix;      // [tc_time*C]
  DevBuf<int> d_err;            // bounded-wait timeout flag
  alignas(64) unsigned char tm_dft[128];
  alignas(64) unsigned char tm_data[128];
  int kr = 0;                   // K extent of the row DFT (2 x window columns, padded to 64)
  DevBuf<uint16_t> d_tc_gh;     // [tc_time*C*rows_alloc][kr] scaled window grid
  DevBuf<uint16_t> d_tc_dftr;   // [2N][kr] row DFT over window columns
  alignas(64) unsigned char tm_gh[128];
  alignas(64) unsigned char tm_fr[128];

  // cluster path (N = 256 / 512)
  int cs = 0, rpc_alloc = 0, clusters = 0, cl_step = 1;
  DevBuf<int> d_rowcol, d_order;
  DevBuf<int2> d_ranges;

  // multiple-pixel / direction-dependent EPICal (Sec. 6); npix = 0: off
  std::vector<double> model;    // [n_src][3] (l, m, S) given to epical_configure
  int npix = 0;
  std::vector<int> pix_user;    // tap index -> caller's pixel index
  DevBuf<double2> d_ap, d_dp;   // [C][npix][Na] A_{p,a}, D_{p,a} (tap order)
  DevBuf<double2> d_kmp;        // [C][Na][npix] correlation sums
  DevBuf<double2> d_gdir;       // [C][Na][npix] per-direction solutions
  DevBuf<uint2> d_ptab;         // [COLROUNDS][BT] slot mask and first tap per thread
  DevBuf<float2> d_pph;         // [C][npix] window-coordinate pixel phases
  DevBuf<float2> d_ptap;        // [ptap_time][C][npix] pixel taps of a call
  long long ptap_time = 0;

  // visibility-based comparison (Sec. 4): model visibilities of the
  // configured model, formed on the first solve after epical_configure
  DevBuf<float2> d_vm;          // [C][Na][Na] (FP32)
  DevBuf<float2> d_vis32;       // [C][Na][Na] the solved visibilities in FP32
  DevBuf<double2> d_uv;         // [C][Na] positions in wavelengths
  DevBuf<int> d_iters;          // [C] solver iterations
  bool vm_stale = true;
  // tensor-core X-engine (4-bit input): FP16 operand scratch and its tensor map
  DevBuf<uint16_t> d_xe_z;      // [C][2 Na_p][xe_tp]
  int xe_tp = 0;                // samples per segment (multiple of 64); 0 = not set up
  alignas(64) unsigned char tm_xe[128];

  // phase centre (Sec. 2.1 footnote): E_a multiplied by p_a = e^{+2 pi i u_a . s0}
  double phase_l = 0.0, phase_m = 0.0;
  std::vector<double2> phase;   // [C][Na] host copy (empty: zenith, not phased)
  DevBuf<double2> d_phase;      // [C][Na] or null
  DevBuf<double> d_bx;          // [C] bandpass fit abscissa scratch
};

namespace {

epic_status check_plan(epic_plan_t p) {
  if (!p) return fail(EPIC_ERR_INVALID_ARG, "plan is NULL");
  return EPIC_OK;
}

// Segments per channel: enough work units to fill every CTA a few times,
// preferring a total that is a multiple of the CTA count.
int choose_segments(int n_chan, long long n_time, int ctas, int target = 4) {
  long long best = 1;
  const long long min_len = 16;
  for (long long s = 1; s <= 4096; ++s) {
    if (n_time / s < min_len && s > 1) break;
    best = s;
    const long long units = static_cast<long long>(n_chan) * s;
    if (units >= static_cast<long long>(target) * ctas && units % ctas == 0) return static_cast<int>(s);
    if (units >= 4LL * target * ctas) return static_cast<int>(s);
  }
  return static_cast<int>(best);
}

// A_{p,a} of channel c: exact response of image pixel (kx, ky) to antenna a
// through its stencil, (1/Na) sum_taps W_a(j) e^{+2 pi i (j - N/2).(k - N/2)/N},
// times the antenna's phasing factor when the plan has a phase centre.
void pixel_response(epic_plan_t p, int c, int kx, int ky, std::vector<std::complex<double>>& A) {
  const int Na = p->na, N = p->n, K = p->k, KK = K * K, h = (K - 1) / 2;
  A.assign(Na, 0.0);
  for (int a = 0; a < Na; ++a) {
    if (p->flags[a]) continue;
    const size_t ob = (static_cast<size_t>(c) * Na + a) * 2;
    const int bx = p->base[ob], by = p->base[ob + 1];
    const double* wa = &p->w64[(static_cast<size_t>(c) * Na + a) * KK];
    std::complex<double> s = 0.0;
    for (int dy = 0; dy < K; ++dy)
      for (int dx = 0; dx < K; ++dx) {
        const int jx = bx + dx - h, jy = by + dy - h;
        long long m = static_cast<long long>(jx - N / 2) * (kx - N / 2) +
                      static_cast<long long>(jy - N / 2) * (ky - N / 2);
        m %= N;
        if (m < 0) m += N;
        const double ph = 2.0 * kPi * static_cast<double>(m) / N;
        s += wa[dy * K + dx] * std::complex<double>(std::cos(ph), std::sin(ph));
      }
    A[a] = s / static_cast<double>(Na);
    if (!p->phase.empty()) {
      const double2 q = p->phase[static_cast<size_t>(c) * Na + a];
      A[a] *= std::complex<double>(q.x, q.y);
    }
  }
}

// D_a = sum_{b != a, unflagged} conj(A_b) V^M_ab for channel c with V^M
// from the point-source model: sum_s S_s e^{-2 pi i u_a.s} (B_s - conj(A_a)
// e^{+2 pi i u_a.s}), B_s = sum_b conj(A_b) e^{+2 pi i u_b.s}.
void model_denominator(epic_plan_t p, int c, const std::vector<std::complex<double>>& A,
                       std::vector<std::complex<double>>& D) {
  const int Na = p->na;
  const double f = p->freq[c];
  D.assign(Na, 0.0);
  const size_t n_src = p->model.size() / 3;
  std::vector<std::complex<double>> ph(Na);
  for (size_t si = 0; si < n_src; ++si) {
    const double l = p->model[3 * si], m = p->model[3 * si + 1], S = p->model[3 * si + 2];
    std::complex<double> B = 0.0;
    for (int b = 0; b < Na; ++b) {
      const double ux = (p->ant[2 * b] * f) / kC, uy = (p->ant[2 * b + 1] * f) / kC;
      const double arg = 2.0 * kPi * (ux * l + uy * m);
      ph[b] = std::complex<double>(std::cos(arg), std::sin(arg));  // e^{+2 pi i u_b.s}
      if (!p->flags[b]) B += std::conj(A[b]) * ph[b];
    }
    for (int a = 0; a < Na; ++a) D[a] += S * (std::conj(ph[a]) * B - std::conj(A[a]));
  }
}

// Nearest pixel centre of direction (l, m): l - l0 = (k - N/2) / (N du), with
// (l0, m0) the phase centre.
bool nearest_pixel(epic_plan_t p, double l, double m, int* kx, int* ky) {
  const int N = p->n;
  l -= p->phase_l;                         // image coordinates relative to the phase centre
  m -= p->phase_m;
  const double kxd = std::floor(l * N * p->cell + N / 2 + 0.5);
  const double kyd = std::floor(m * N * p->cell + N / 2 + 0.5);
  if (!(kxd >= 0 && kxd < N && kyd >= 0 && kyd < N)) return false;
  *kx = static_cast<int>(kxd);
  *ky = static_cast<int>(kyd);
  return true;
}

// Window-coordinate phase of pixel (kx, ky) in channel c:
// (-1)^(kx+ky) e^{2 pi i (x0 kx + y0 ky) / N}.
float2 window_phase(epic_plan_t p, int c, int kx, int ky) {
  const int N = p->n;
  const double sg = ((kx + ky) & 1) ? -1.0 : 1.0;
  long long m = static_cast<long long>(p->x0[c]) * kx + static_cast<long long>(p->y0[c]) * ky;
  m %= N;
  if (m < 0) m += N;
  const double th = 2.0 * kPi * static_cast<double>(m) / N;
  return make_float2(static_cast<float>(sg * std::cos(th)), static_cast<float>(sg * std::sin(th)));
}

// Tap buffer of the multiple-pixel form for calls of up to n_time samples
// (grown outside any stream capture: epic_graph_capture sizes it first).
epic_status ensure_ptap(epic_plan_t p, long long n_time) {
  if (p->npix < 1 || p->ptap_time >= n_time) return EPIC_OK;
  cudaError_t e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return cuda_fail(e, "stream sync before tap buffer growth");
  e = p->d_ptap.alloc(static_cast<size_t>(n_time) * p->nc * p->npix);
  if (e != cudaSuccess) {
    p->ptap_time = 0;
    return fail(EPIC_ERR_OOM, "pixel tap buffer allocation failed");
  }
  p->ptap_time = n_time;
  return EPIC_OK;
}

// Gridding of Eq. 9 inverted into per-lane gather lists.  The grid of
// channel c holds its occupied rows (window row r = y - y0[c]); an N-point
// row FFT runs on N1 lanes, lane n1 holding the columns x = n1 + N1 j.  For
// every lane (r, n1) the list holds the taps (antenna, folded weight) that
// land on its columns, grouped by j, with the group lengths as bytes
// (ceil(N2 / 16) 16-byte words per lane).  window: columns relative to the
// first occupied column x0[c] (a phase of every image pixel, removed where
// a pixel value is needed), else absolute.  ofs [C][rows_alloc][N1] is the
// lane's first entry relative to the channel's first (base [C + 1]).
epic_status build_gather(epic_plan_t p, const std::vector<float>& wts, int N1, bool window, std::vector<int>& ofs,
                         std::vector<uint4>& cnt, std::vector<uint2>& ent, std::vector<int>& base) {
  const int C = p->nc, Na = p->na, N = p->n, K = p->k, KK = K * K, h = (K - 1) / 2;
  const int N2 = N / N1, CW = (N2 + 15) / 16;
  const int RA = p->rows_alloc;
  ofs.assign(static_cast<size_t>(C) * RA * N1, 0);
  cnt.assign(static_cast<size_t>(C) * RA * N1 * CW, make_uint4(0, 0, 0, 0));
  base.assign(static_cast<size_t>(C) + 1, 0);
  ent.clear();
  std::vector<std::vector<std::pair<int, float>>> bucket(static_cast<size_t>(RA) * N1 * N2);
  for (int c = 0; c < C; ++c) {
    base[c] = static_cast<int>(ent.size());
    for (auto& l : bucket) l.clear();
    for (int a = 0; a < Na; ++a) {
      if (p->flags[a]) continue;
      const size_t ob = (static_cast<size_t>(c) * Na + a) * 2;
      const int r0 = p->base[ob + 1] - h - p->y0[c];
      const int xa = p->base[ob] - h - (window ? p->x0[c] : 0);
      const float* wf = &wts[(static_cast<size_t>(c) * Na + a) * KK];
      for (int dy = 0; dy < K; ++dy)
        for (int dx = 0; dx < K; ++dx) {
          const float w = wf[dy * K + dx];
          if (w == 0.0f) continue;
          const int x = xa + dx;
          bucket[(static_cast<size_t>(r0 + dy) * N1 + x % N1) * N2 + x / N1].emplace_back(a, w);
        }
    }
    for (int li = 0; li < RA * N1; ++li) {
      ofs[static_cast<size_t>(c) * RA * N1 + li] = static_cast<int>(ent.size()) - base[c];
      unsigned char cb[32] = {0};
      for (int j = 0; j < N2; ++j) {
        const auto& l = bucket[static_cast<size_t>(li) * N2 + j];
        if (l.size() > 255) return fail(EPIC_ERR_UNSUPPORTED, "more than 255 gridding taps on one grid cell");
        cb[j] = static_cast<unsigned char>(l.size());
        for (const auto& en : l) {
          uint2 q;
          q.x = static_cast<unsigned>(en.first);
          std::memcpy(&q.y, &en.second, sizeof(float));
          ent.push_back(q);
        }
      }
      std::memcpy(&cnt[(static_cast<size_t>(c) * RA * N1 + li) * CW], cb, sizeof(uint4) * CW);
    }
  }
  base[C] = static_cast<int>(ent.size());
  return EPIC_OK;
}

// Arguments of one fused launch over a device batch.// Arguments of one fused launch over a device batch.
epic::ImageArgs fused_args(epic_plan_t p, const void* d_volt, long long n_time, double* d_image,
                           double img_scale) {
  epic::ImageArgs a{};
  a.volt = d_volt;
  a.input_fmt = p->input;
  a.n_time = n_time;
  a.n_chan = p->nc;
  a.n_ant = p->na;
  a.support = p->k;
  a.cell0 = p->d_cell0.p;
  a.cellf = p->d_cellf.p;
  a.gofs = p->d_gofs.p;
  a.gent = p->d_gent.p;
  a.gbase = p->d_gbase.p;
  a.gcnt = p->d_gcnt.p;
  a.gsmem = p->gsmem;
  a.piped = p->piped ? 1 : 0;
  a.steps = p->steps;
  a.err = p->d_err.p;
  a.wts = p->d_wts.p;
  a.wgain = p->d_wgain.p;
  a.vscale = p->d_vscale.p;
  a.win = p->d_win.p;
  a.win4 = p->d_win4.p;
  a.pixph = p->d_pixph.p;
  a.twid = p->d_twid.p;
  a.image = d_image;
  a.img_scale = img_scale;
  a.do_cal = p->cal ? 1 : 0;
  a.k0x = p->cal ? p->k0x : 0;
  a.k0y = p->cal ? p->k0y : 0;
  a.pix_sign = ((a.k0x + a.k0y) & 1) ? -1.0f : 1.0f;
  a.kacc = p->d_kacc.p;
  a.pacc = p->d_pacc.p;
  a.segs = choose_segments(p->nc, n_time, p->ctas, p->tune_units);
  a.rows_alloc = p->rows_alloc;
  a.rs = p->rs_fused;
  const long long units = static_cast<long long>(p->nc) * a.segs;
  a.grid = static_cast<int>(std::min<long long>(units, p->ctas));
  a.smem = p->smem;
  a.npix = 0;                              // epic_image arms the pixel taps itself
  a.wait_limit = p->wait_limit;
  return a;
}

// Cluster path: one persistent launch of thread-block clusters.
epic_status image_cluster(epic_plan_t p, const void* d_volt, long long n_time, double* d_image) {
  epic::ClusterArgs a{};
  a.volt = d_volt;
  a.input_fmt = p->input;
  a.n_time = n_time;
  a.n_chan = p->nc;
  a.n_ant = p->na;
  a.support = p->k;
  a.rowcol = p->d_rowcol.p;
  a.order = p->d_order.p;
  a.ranges = p->d_ranges.p;
  a.wts = p->d_wts.p;
  a.wgain = p->d_wgain.p;
  a.vscale = p->d_vscale.p;
  a.win4 = p->d_win4.p;
  a.twid = p->d_twid.p;
  a.pixph = p->d_pixph.p;
  a.image = d_image;
  a.img_scale = 1.0 / static_cast<double>(n_time);
  a.do_cal = p->cal ? 1 : 0;
  a.k0x = p->cal ? p->k0x : 0;
  a.k0y = p->cal ? p->k0y : 0;
  a.kacc = p->d_kacc.p;
  a.pacc = p->d_pacc.p;
  a.segs = choose_segments(p->nc, n_time, p->clusters, p->tune_units);
  a.rpc_alloc = p->rpc_alloc;
  a.rs = p->rs_fused;
  a.frames_per_step = p->cl_step;
  const long long units = static_cast<long long>(p->nc) * a.segs;
  a.grid = static_cast<int>(std::min<long long>(units, p->clusters)) * p->cs;
  a.smem = p->smem;
  EPIC_CUDA(epic::launch_cluster(p->n, a, p->stream));
  if (p->cal) p->frames += n_time;
  return EPIC_OK;
}

// Plain unfused path: batches of time samples through the device scratch.
epic_status image_unfused(epic_plan_t p, const void* d_volt, long long n_time, double* d_image) {
  const int C = p->nc, N = p->n;
  // per time sample: row spectra [C][N][rs] and the calibrator pixel [C]
  const size_t per_t = static_cast<size_t>(C) * (static_cast<size_t>(N) * p->rs + 1);
  long long nt = static_cast<long long>(p->workspace_budget / (per_t * sizeof(float2)));
  if (p->tune_nt > 0 && p->tune_nt < nt) nt = p->tune_nt;
  if (nt < 1) nt = 1;
  if (nt > n_time) nt = n_time;
  if (nt > (1 << 20)) nt = 1 << 20;
  if (p->ws_time < nt) {
    cudaError_t e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream sync before scratch growth");
    e = p->d_ws.alloc(per_t * static_cast<size_t>(nt));
    if (e != cudaSuccess) {
      p->ws_time = 0;
      return fail(EPIC_ERR_OOM, "unfused scratch allocation failed");
    }
    p->ws_time = static_cast<int>(nt);
  }
  nt = std::min<long long>(nt, p->ws_time);
  epic::UnfusedArgs a{};
  a.volt = d_volt;
  a.input_fmt = p->input;
  a.n_chan = C;
  a.n_ant = p->na;
  a.support = p->k;
  a.grid_n = N;
  a.cell0 = p->d_cell0.p;
  a.wts = p->d_wts.p;
  a.wgain = p->d_wgain.p;
  a.vscale = p->d_vscale.p;
  a.win = p->d_win.p;
  a.twid = p->d_twid.p;
  const size_t cap = static_cast<size_t>(p->ws_time) * C;
  a.spec = p->d_ws.p;
  a.pix = a.spec + cap * N * p->rs;
  a.gofs = p->d_gofs.p;                    // window-column gather tables
  a.gcnt = p->d_gcnt.p;
  a.gent = p->d_gent.p;
  a.gbase = p->d_gbase.p;
  a.rows_alloc = p->rows_alloc;
  a.rs = p->rs;
  a.pixph = p->d_pixph.p;
  a.max_cols = *std::max_element(p->cols.begin(), p->cols.end());
  a.gmax = p->gmax;
  a.err = p->d_err.p;
  a.row_table = p->tune_row_table;
  a.row_frames = p->tune_row_frames;
  a.sms = p->sms;
  a.image = d_image;
  a.img_scale = 1.0 / static_cast<double>(n_time);
  a.do_cal = p->cal ? 1 : 0;
  a.k0x = p->cal ? p->k0x : 0;
  a.k0y = p->cal ? p->k0y : 0;
  a.pix_sign = ((a.k0x + a.k0y) & 1) ? -1.0f : 1.0f;
  a.kacc = p->d_kacc.p;
  a.pacc = p->d_pacc.p;
  a.cols_target = p->tune_cols;
  a.wait_limit = p->wait_limit;
  if (p->persistent && p->precision == EPIC_PREC_FP32 && epic::persistent_supported(N)) {
    a.row_frames = 1;
    EPIC_CUDA(epic::launch_unfused_persistent(a, n_time, static_cast<int>(nt), p->d_gbar.p, p->sms, p->stream));
    if (p->cal) p->frames += n_time;
    return EPIC_OK;
  }
  for (long long t0 = 0; t0 < n_time; t0 += nt) {
    const int n = static_cast<int>(std::min<long long>(nt, n_time - t0));
    EPIC_CUDA(epic::launch_unfused_batch(a, t0, n, p->sms, p->stream));
  }
  if (p->cal) p->frames += n_time;
  return EPIC_OK;
}

// float -> IEEE binary16 / bfloat16 bits, round to nearest even (host).
uint16_t to_half_bits(float f) {
  uint32_t x;
  std::memcpy(&x, &f, 4);
  const uint32_t sign = (x >> 16) & 0x8000u;
  const int e = static_cast<int>((x >> 23) & 0xff) - 127 + 15;
  uint32_t m = x & 0x7fffffu;
  if (e >= 31) return static_cast<uint16_t>(sign | 0x7c00u);
  if (e <= 0) {
    if (e < -10) return static_cast<uint16_t>(sign);
    m |= 0x800000u;
    const int sh = 14 - e;
    uint32_t v = m >> sh;
    const uint32_t rem = m & ((1u << sh) - 1), half = 1u << (sh - 1);
    if (rem > half || (rem == half && (v & 1))) ++v;
    return static_cast<uint16_t>(sign | v);
  }
  uint32_t v = (static_cast<uint32_t>(e) << 10) | (m >> 13);
  const uint32_t rem = m & 0x1fffu;
  if (rem > 0x1000u || (rem == 0x1000u && (v & 1))) ++v;
  return static_cast<uint16_t>(sign | v);
}

uint16_t to_bf16_bits(float f) {
  uint32_t x;
  std::memcpy(&x, &f, 4);
  const uint32_t lsb = (x >> 16) & 1u;
  x += 0x7fffu + lsb;
  return static_cast<uint16_t>(x >> 16);
}

// Reduced-precision form: FP32 gridding and row FFTs, FP16/BF16 tensor-core
// column DFT with per-frame power-of-two scaling, FP64 image accumulation.
epic_status image_tc(epic_plan_t p, const void* d_volt, long long n_time, double* d_image) {
  const int C = p->nc, N = p->n;
  if (p->tc_time == 0) {
    p->kr = ((2 * *std::max_element(p->cols.begin(), p->cols.end()) + 63) / 64) * 64;
    const size_t per_t = static_cast<size_t>(C) *
                         (static_cast<size_t>(N) * p->kp * 2 + static_cast<size_t>(p->rows_alloc) * p->kr * 2 +
                          2 * sizeof(float) + sizeof(float2));
    long long nt = static_cast<long long>(p->workspace_budget / per_t);
    nt = std::max<long long>(1, std::min<long long>(nt, 128));
    const size_t n_hh = static_cast<size_t>(C) * N * nt * p->kp;
    const size_t n_gh = static_cast<size_t>(nt) * C * p->rows_alloc * p->kr;
    cudaError_t es[] = {p->d_tc_hh.alloc(n_hh),
                        p->d_tc_dft.alloc(static_cast<size_t>(2) * N * p->kp),
                        p->d_tc_scale.alloc(static_cast<size_t>(2 * nt) * C),
                        p->d_tc_pix.alloc(static_cast<size_t>(nt) * C),
                        p->d_tc_gh.alloc(n_gh),
                        p->d_tc_dftr.alloc(static_cast<size_t>(2) * N * p->kr)};
    for (cudaError_t x : es)
      if (x != cudaSuccess) return fail(EPIC_ERR_OOM, "tensor-path scratch allocation failed");
    EPIC_CUDA(cudaMemset(p->d_tc_hh.p, 0, n_hh * 2));
    // real-expanded DFT over window rows: rows 2 ky + (re, im), columns 2 jw + (re, im)
    const bool bf = p->precision == EPIC_PREC_BF16;
    std::vector<uint16_t> dft(static_cast<size_t>(2) * N * p->kp);
    for (int ky = 0; ky < N; ++ky)
      for (int jw = 0; jw < p->kp / 2; ++jw) {
        const long long m = (static_cast<long long>(jw) * ky) % N;
        const double th = 2.0 * kPi * static_cast<double>(m) / N;
        const float cs = static_cast<float>(std::cos(th)), sn = static_cast<float>(std::sin(th));
        auto put = [&](int r, int k, float v) {
          dft[static_cast<size_t>(r) * p->kp + k] = bf ? to_bf16_bits(v) : to_half_bits(v);
        };
        put(2 * ky, 2 * jw, cs);
        put(2 * ky, 2 * jw + 1, -sn);
        put(2 * ky + 1, 2 * jw, sn);
        put(2 * ky + 1, 2 * jw + 1, cs);
      }
    EPIC_CUDA(cudaMemcpy(p->d_tc_dft.p, dft.data(), dft.size() * 2, cudaMemcpyHostToDevice));
    // row DFT over window columns x: rows 2 kx + (re, im), columns 2 x + (re, im)
    std::vector<uint16_t> dftr(static_cast<size_t>(2) * N * p->kr);
    for (int kx = 0; kx < N; ++kx)
      for (int x = 0; x < p->kr / 2; ++x) {
        const long long m = (static_cast<long long>(x) * kx) % N;
        const double th = 2.0 * kPi * static_cast<double>(m) / N;
        const float cs = static_cast<float>(std::cos(th)), sn = static_cast<float>(std::sin(th));
        auto put = [&](int r, int k, float v) {
          dftr[static_cast<size_t>(r) * p->kr + k] = bf ? to_bf16_bits(v) : to_half_bits(v);
        };
        put(2 * kx, 2 * x, cs);
        put(2 * kx, 2 * x + 1, -sn);
        put(2 * kx + 1, 2 * x, sn);
        put(2 * kx + 1, 2 * x + 1, cs);
      }
    EPIC_CUDA(cudaMemcpy(p->d_tc_dftr.p, dftr.data(), dftr.size() * 2, cudaMemcpyHostToDevice));
    if (!epic::tc_make_maps(p->d_tc_dft.p, p->d_tc_hh.p, N, C, static_cast<int>(nt), p->kp, bf, p->tm_dft,
                            p->tm_data) ||
        !epic::tc_make_row_maps(p->d_tc_gh.p, p->d_tc_dftr.p, static_cast<long long>(nt) * C * p->rows_alloc, N,
                                p->kr, bf, p->tm_gh, p->tm_fr))
      return fail(EPIC_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    p->tc_time = static_cast<int>(nt);
  }
  epic::TcArgs a{};
  epic::UnfusedArgs& u = a.u;
  u.volt = d_volt;
  u.input_fmt = p->input;
  u.n_chan = C;
  u.n_ant = p->na;
  u.support = p->k;
  u.grid_n = N;
  u.cell0 = p->d_cell0.p;
  u.wts = p->d_wts.p;
  u.wgain = p->d_wgain.p;
  u.vscale = p->d_vscale.p;
  u.win = p->d_win.p;
  u.twid = p->d_twid.p;
  u.spec = nullptr;
  u.gofs = p->d_gofs.p;                    // window-column gather tables
  u.gcnt = p->d_gcnt.p;
  u.gent = p->d_gent.p;
  u.gbase = p->d_gbase.p;
  u.pix = p->d_tc_pix.p;
  u.rows_alloc = p->rows_alloc;
  u.rs = p->rs;
  u.image = d_image;
  u.img_scale = 1.0 / static_cast<double>(n_time);
  u.do_cal = p->cal ? 1 : 0;
  u.k0x = p->cal ? p->k0x : 0;
  u.k0y = p->cal ? p->k0y : 0;
  u.pix_sign = ((u.k0x + u.k0y) & 1) ? -1.0f : 1.0f;
  u.kacc = p->d_kacc.p;
  u.pacc = p->d_pacc.p;
  u.cols_target = p->tune_cols;
  a.hh = p->d_tc_hh.p;
  a.fscale = p->d_tc_scale.p;
  a.finv2 = p->d_tc_scale.p + static_cast<size_t>(p->tc_time) * C;
  a.tb_cap = p->tc_time;
  a.kp = p->kp;
  a.bf16 = p->precision == EPIC_PREC_BF16 ? 1 : 0;
  a.err = p->d_err.p;
  a.gh = p->d_tc_gh.p;
  a.kr = p->kr;
  a.r_alloc = p->rows_alloc;
  a.win4 = p->d_win4.p;
  a.tm_gh = p->tm_gh;
  a.tm_fr = p->tm_fr;
  for (long long t0 = 0; t0 < n_time; t0 += p->tc_time) {
    const int n = static_cast<int>(std::min<long long>(p->tc_time, n_time - t0));
    EPIC_CUDA(epic::launch_tc_batch(a, p->tm_dft, p->tm_data, t0, n, p->sms, p->stream));
  }
  if (p->cal) p->frames += n_time;
  return EPIC_OK;
}

// Checks of the plan descriptor; the fused kernel's launch shape for it and
// which of the fused / unfused forms can take it.
epic_status validate_desc(const epic_plan_desc* d, epic::ImageKernelShape* shape, bool* fused_shape,
                          bool* unfused_ok) {
  if (d->n_ant < 1 || d->n_chan < 1) return fail(EPIC_ERR_INVALID_ARG, "n_ant and n_chan must be >= 1");
  if (!d->ant_xy_m || !d->freq_hz) return fail(EPIC_ERR_INVALID_ARG, "ant_xy_m and freq_hz are required");
  if (!is_pow2(d->grid_n) || d->grid_n < 16)
    return fail(EPIC_ERR_INVALID_ARG, "grid_n must be a power of two >= 16");
  if (!(d->cell_wavelengths > 0) || !std::isfinite(d->cell_wavelengths))
    return fail(EPIC_ERR_INVALID_ARG, "cell_wavelengths must be > 0");
  if (d->kernel_support < 1 || d->kernel_support > 7 || d->kernel_support % 2 == 0)
    return fail(EPIC_ERR_INVALID_ARG, "kernel_support must be odd, 1..7");
  if (d->kernel != EPIC_KERNEL_GAUSSIAN && d->kernel != EPIC_KERNEL_TOPHAT)
    return fail(EPIC_ERR_INVALID_ARG, "unknown kernel type");
  if (!(d->kernel_param > 0) || !std::isfinite(d->kernel_param))
    return fail(EPIC_ERR_INVALID_ARG, "kernel_param must be > 0");
  if (d->kernel_param_ant)
    for (int a = 0; a < d->n_ant; ++a)
      if (!(d->kernel_param_ant[a] > 0) || !std::isfinite(d->kernel_param_ant[a]))
        return fail(EPIC_ERR_INVALID_ARG, "kernel_param_ant must be > 0 for every antenna");
  if (d->input != EPIC_IN_CI4 && d->input != EPIC_IN_COMPLEX64)
    return fail(EPIC_ERR_INVALID_ARG, "unknown input format");
  if (d->precision != EPIC_PREC_FP32 && d->precision != EPIC_PREC_FP16 && d->precision != EPIC_PREC_BF16)
    return fail(EPIC_ERR_INVALID_ARG, "unknown precision");
  if (d->precision != EPIC_PREC_FP32 && (d->path == EPIC_PATH_FUSED || d->path == EPIC_PATH_PIPED))
    return fail(EPIC_ERR_UNSUPPORTED, "FP16/BF16 run on the tensor-core column DFT (not the fused path)");
  for (int c = 0; c < d->n_chan; ++c)
    if (!(d->freq_hz[c] > 0) || !std::isfinite(d->freq_hz[c]))
      return fail(EPIC_ERR_INVALID_ARG, "frequencies must be finite and > 0");
  for (int i = 0; i < 2 * d->n_ant; ++i)
    if (!std::isfinite(d->ant_xy_m[i])) return fail(EPIC_ERR_INVALID_ARG, "non-finite antenna position");

  if (d->path != EPIC_PATH_AUTO && d->path != EPIC_PATH_FUSED && d->path != EPIC_PATH_UNFUSED &&
      d->path != EPIC_PATH_CLUSTER && d->path != EPIC_PATH_PIPED)
    return fail(EPIC_ERR_INVALID_ARG, "unknown path");
  if (d->path == EPIC_PATH_CLUSTER &&
      (!epic::cluster_supported(d->grid_n) || d->n_ant > 256 * epic::cluster_size(d->grid_n) ||
       d->precision != EPIC_PREC_FP32))
    return fail(EPIC_ERR_UNSUPPORTED, "cluster path: FP32, grid_n 256 or 512, n_ant <= 256 x cluster size");
  *fused_shape = epic::image_kernel_shape(d->grid_n, shape) && d->n_ant <= shape->max_ant;
  *unfused_ok = epic::unfused_supported(d->grid_n);
  if (d->path == EPIC_PATH_PIPED && !epic::piped_supported(d->grid_n, d->n_ant))
    return fail(EPIC_ERR_UNSUPPORTED, "warp-specialised fused path: grid_n 64 or 128, n_ant <= 512");
  if ((d->path == EPIC_PATH_FUSED || d->path == EPIC_PATH_PIPED) && !*fused_shape)
    return fail(EPIC_ERR_UNSUPPORTED, "fused path: grid_n must be 16..128 and n_ant <= " +
                                          std::to_string(shape->max_ant > 0 ? shape->max_ant : 2048));
  if (d->path == EPIC_PATH_UNFUSED && !*unfused_ok)
    return fail(EPIC_ERR_UNSUPPORTED, "unfused path: grid_n must be 32..512");
  if (!*fused_shape && !*unfused_ok)
    return fail(EPIC_ERR_UNSUPPORTED, "grid_n must be 16..512 in this build");
  return EPIC_OK;
}

// Gridding tables of Eq. 9 in FP64 (stencil centres p->base, normalised
// taps p->w64), every channel's occupied window (y0, rows, x0, cols), and
// the device forms: cell0 [C][Na] = window row * N + absolute column of
// the first tap, wts [C][Na][K*K] = taps with the centring sign of Eq. 10
// and 1/Na folded in.
epic_status build_grid_tables(epic_plan_s* p, std::vector<int>& cell0, std::vector<float>& wts) {
  const int Na = p->na, C = p->nc, N = p->n, K = p->k, KK = K * K, h = (K - 1) / 2;
  p->base.assign(static_cast<size_t>(C) * Na * 2, 0);
  p->w64.assign(static_cast<size_t>(C) * Na * KK, 0.0);
  p->y0.assign(C, 0);
  p->rows.assign(C, 0);
  p->x0.assign(C, 0);
  p->cols.assign(C, 0);
  cell0.assign(static_cast<size_t>(C) * Na, -1);
  wts.assign(static_cast<size_t>(C) * Na * KK, 0.0f);
  int n_unflagged = 0;
  for (int a = 0; a < Na; ++a) n_unflagged += p->flags[a] ? 0 : 1;
  if (n_unflagged == 0) return fail(EPIC_ERR_INVALID_ARG, "every antenna is flagged");
  for (int c = 0; c < C; ++c) {
    const double f = p->freq[c];
    int ymin = N, ymax = -1;
    for (int a = 0; a < Na; ++a) {
      const double ux = (p->ant[2 * a] * f) / kC;
      const double uy = (p->ant[2 * a + 1] * f) / kC;
      const double px = ux / p->cell + N / 2;
      const double py = uy / p->cell + N / 2;
      const double bxd = std::floor(px + 0.5), byd = std::floor(py + 0.5);
      const size_t ob = (static_cast<size_t>(c) * Na + a) * 2;
      if (!(std::fabs(bxd) < 1e9 && std::fabs(byd) < 1e9)) {
        if (p->flags[a]) continue;
        return fail(EPIC_ERR_GRID_TOO_SMALL, "antenna far outside the grid");
      }
      const int bx = static_cast<int>(bxd), by = static_cast<int>(byd);
      p->base[ob] = bx;
      p->base[ob + 1] = by;
      if (p->flags[a]) continue;
      if (bx - h < 0 || bx + h >= N || by - h < 0 || by + h >= N) {
        char msg[160];
        std::snprintf(msg, sizeof msg, "antenna %d channel %d: stencil outside the %dx%d grid", a, c, N, N);
        return fail(EPIC_ERR_GRID_TOO_SMALL, msg);
      }
      double* w = &p->w64[(static_cast<size_t>(c) * Na + a) * KK];
      double sum = 0.0;
      const double kp = p->kparam_ant.empty() ? p->kparam : p->kparam_ant[a];
      const double half = (kp * f / kC) / p->cell / 2.0;
      for (int dy = 0; dy < K; ++dy)
        for (int dx = 0; dx < K; ++dx) {
          const int jx = bx + dx - h, jy = by + dy - h;
          double v;
          if (p->kernel == EPIC_KERNEL_GAUSSIAN) {
            const double ex = jx - px, ey = jy - py;
            const double d2 = ex * ex + ey * ey;
            v = std::exp(-d2 / (2.0 * kp * kp));
          } else {
            v = (std::fabs(jx - px) <= half && std::fabs(jy - py) <= half) ? 1.0 : 0.0;
          }
          w[dy * K + dx] = v;
          sum += v;
        }
      if (!(sum > 0))
        return fail(EPIC_ERR_INVALID_ARG, "gridding kernel has no support for antenna " + std::to_string(a));
      for (int i = 0; i < KK; ++i) w[i] /= sum;
      ymin = std::min(ymin, by - h);
      ymax = std::max(ymax, by + h);
    }
    p->y0[c] = ymin;
    p->rows[c] = ymax - ymin + 1;
    int xmin = N, xmax = -1;
    for (int a = 0; a < Na; ++a) {
      if (p->flags[a]) continue;
      const int bx = p->base[(static_cast<size_t>(c) * Na + a) * 2];
      xmin = std::min(xmin, bx - h);
      xmax = std::max(xmax, bx + h);
    }
    p->x0[c] = xmin;
    p->cols[c] = xmax - xmin + 1;
    p->rows_alloc = std::max(p->rows_alloc, p->rows[c]);
    for (int a = 0; a < Na; ++a) {
      if (p->flags[a]) continue;
      const size_t ob = (static_cast<size_t>(c) * Na + a) * 2;
      const int bx = p->base[ob], by = p->base[ob + 1];
      cell0[static_cast<size_t>(c) * Na + a] = (by - h - ymin) * N + (bx - h);
      const double* w = &p->w64[(static_cast<size_t>(c) * Na + a) * KK];
      float* wf = &wts[(static_cast<size_t>(c) * Na + a) * KK];
      for (int dy = 0; dy < K; ++dy)
        for (int dx = 0; dx < K; ++dx) {
          const int jx = bx + dx - h, jy = by + dy - h;
          const double sgn = ((jx + jy) & 1) ? -1.0 : 1.0;   // centring of Eq. 10
          wf[dy * K + dx] = static_cast<float>(w[dy * K + dx] * sgn / Na);
        }
    }
  }

  return EPIC_OK;
}

// Launch shape and path of the plan: the tensor-core form's K extent for
// FP16/BF16, else the fused kernel's frames per step and gather-table
// placement (or the warp-specialised form), the cluster form when asked
// for, else the plain unfused path; CTAs per launch.
epic_status choose_path(epic_plan_s* p, const epic_plan_desc* d, bool fused_shape, bool unfused_ok) {
  const int Na = p->na, N = p->n, KK = p->k * p->k;
  p->rs = epic::image_rs(p->rows_alloc);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  p->device = dev;
  int smem_optin = 0;
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, dev);
  bool fused = fused_shape && d->path != EPIC_PATH_UNFUSED && d->precision == EPIC_PREC_FP32;
  p->precision = d->precision;
  if (p->precision != EPIC_PREC_FP32) {
    if (!epic::tc_supported(N, p->rows_alloc))
      return fail(EPIC_ERR_UNSUPPORTED, "FP16/BF16 form: grid_n must be 128 or 256 and the array "
                                        "footprint at most 128 grid rows");
    p->kp = epic::tc_kp(p->rows_alloc);
    e = epic::tc_prepare(p->precision == EPIC_PREC_BF16, epic::tc_smem(p->kp));
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core kernel attributes");
  }
  p->rs_fused = epic::image_rs_fused(p->rows_alloc);
  if (fused && d->path == EPIC_PATH_PIPED && epic::piped_supported(N, Na)) {
    // warp-specialised form: two spectra slots; gather table in shared
    // memory when it fits (entries per channel <= Na K^2 + one per FFT lane)
    const long long gmax = static_cast<long long>(Na) * KK;   // entries per channel <= Na K^2
    const size_t s1 = epic::piped_smem_bytes(N, Na, p->rs_fused, p->rows_alloc, gmax);
    const size_t s0 = epic::piped_smem_bytes(N, Na, p->rs_fused, p->rows_alloc, 0);
    if (s1 <= static_cast<size_t>(smem_optin)) {
      p->piped = true;
      p->smem = s1;
      p->gsmem = 1;
    } else if (s0 <= static_cast<size_t>(smem_optin)) {
      p->piped = true;
      p->smem = s0;
      p->gsmem = 0;
    }
  }
  if (d->path == EPIC_PATH_PIPED && !p->piped)
    return fail(EPIC_ERR_UNSUPPORTED, "warp-specialised fused path: array footprint exceeds shared memory");
  if (fused && !p->piped) {
    // shape preference: two frames per step, then one; the gather table in
    // shared memory when it fits (entries per channel <= Na K^2 taps), else
    // read through L1
    const int n1 = epic::image_fft_lanes(N);
    const long long gmax = static_cast<long long>(Na) * KK;
    const size_t tab = epic::image_table_bytes(p->rows_alloc, n1, gmax);
    bool placed = false;
    for (int steps = epic::image_max_steps(N); steps >= 1 && !placed; --steps)
      for (int ts = 1; ts >= 0 && !placed; --ts) {
        const size_t need = epic::image_smem_bytes(N, Na, p->rs_fused, steps) + (ts ? tab : 0);
        if (need <= static_cast<size_t>(smem_optin)) {
          p->smem = need;
          p->gsmem = ts;
          p->steps = steps;
          placed = true;
        }
      }
    if (!placed) {
      const std::string msg = "array footprint needs " +
                              std::to_string(epic::image_smem_bytes(N, Na, p->rs_fused, 1)) +
                              " B of shared memory in the fused kernel (limit " +
                              std::to_string(smem_optin) + ")";
      if (d->path == EPIC_PATH_FUSED || !unfused_ok) return fail(EPIC_ERR_UNSUPPORTED, msg);
      fused = false;
    }
  }
  const bool want_cluster = !fused && p->precision == EPIC_PREC_FP32 && d->path == EPIC_PATH_CLUSTER &&
                            epic::cluster_supported(N) && Na <= 256 * epic::cluster_size(N);
  if (want_cluster) {
    p->cs = epic::cluster_size(N);
    p->rpc_alloc = (p->rows_alloc + p->cs - 1) / p->cs;
    // frames per pair of cluster barriers: as many spectra slots as fit, up to 4
    p->cl_step = 4;
    while (p->cl_step > 1 &&
           epic::cluster_smem_bytes(N, p->rpc_alloc, p->rs_fused, p->cl_step) > static_cast<size_t>(smem_optin))
      --p->cl_step;
    const size_t csm = epic::cluster_smem_bytes(N, p->rpc_alloc, p->rs_fused, p->cl_step);
    int ncl = 0;
    e = csm <= static_cast<size_t>(smem_optin) ? epic::cluster_prepare(N, csm, &ncl) : cudaErrorInvalidValue;
    if (e == cudaSuccess && ncl >= 1) {
      p->smem = csm;
      p->clusters = ncl;
      p->ctas = ncl * p->cs;
      p->path = EPIC_PATH_CLUSTER;
    } else if (d->path == EPIC_PATH_CLUSTER) {
      return e != cudaSuccess && e != cudaErrorInvalidValue ? cuda_fail(e, "cluster kernel attributes")
                                                            : fail(EPIC_ERR_UNSUPPORTED, "cluster kernel cannot be resident");
    } else {
      cudaGetLastError();
      p->cs = 0;
    }
  }
  if (p->path == EPIC_PATH_CLUSTER) {
    // tables built below with the device tables
  } else if (fused) {
    int per_sm = 0;
    e = p->piped ? epic::piped_prepare(N, p->smem, p->gsmem != 0, &per_sm)
                 : epic::image_kernel_prepare(N, p->smem, Na, p->steps, &per_sm);
    if (e != cudaSuccess || per_sm < 1)
      return e != cudaSuccess ? cuda_fail(e, "image kernel attributes")
                              : fail(EPIC_ERR_UNSUPPORTED, "image kernel cannot be resident");
    p->ctas = per_sm * p->sms;
    p->path = EPIC_PATH_FUSED;
  } else {
    p->smem = 0;
    p->ctas = p->sms;
    p->path = EPIC_PATH_UNFUSED;
  }

  return EPIC_OK;
}

// Cluster-path tables: each antenna's stencil (top row << 16 | first
// column) in window coordinates, the antennas of every channel sorted by
// top row, and per CTA of a cluster the sorted range whose stencil rows
// meet the CTA's row block (rows per CTA = ceil(rows / cluster size)).
void build_cluster_tables(const epic_plan_s* p, std::vector<int>& rowcol, std::vector<int>& order,
                          std::vector<int2>& ranges) {
  const int Na = p->na, C = p->nc, K = p->k, h = (K - 1) / 2;
  const int CS = p->cs;
  rowcol.assign(static_cast<size_t>(C) * Na, -1);
  order.assign(static_cast<size_t>(C) * Na, 0);
  ranges.assign(static_cast<size_t>(C) * CS, make_int2(0, 0));
  for (int c = 0; c < C; ++c) {
    std::vector<std::pair<int, int>> tops;
    for (int a = 0; a < Na; ++a) {
      if (p->flags[a]) continue;
      const size_t ob = (static_cast<size_t>(c) * Na + a) * 2;
      const int top = p->base[ob + 1] - h - p->y0[c];
      const int col = p->base[ob] - h - p->x0[c];
      rowcol[static_cast<size_t>(c) * Na + a] = (top << 16) | col;
      tops.emplace_back(top, a);
    }
    std::stable_sort(tops.begin(), tops.end());
    for (size_t i = 0; i < tops.size(); ++i) order[static_cast<size_t>(c) * Na + i] = tops[i].second;
    const int rpc = (p->rows[c] + CS - 1) / CS;
    for (int q = 0; q < CS; ++q) {
      const int lo_top = q * rpc - K + 1, hi_top = (q + 1) * rpc - 1;
      int lo = 0, hi = 0;
      while (lo < static_cast<int>(tops.size()) && tops[lo].first < lo_top) ++lo;
      hi = lo;
      while (hi < static_cast<int>(tops.size()) && tops[hi].first <= hi_top) ++hi;
      ranges[static_cast<size_t>(c) * CS + q] = make_int2(lo, hi);
    }
  }
}

}  // namespace

extern "C" {

const char* epic_last_error(void) { return g_last_error.c_str(); }

epic_status epic_plan_create(epic_plan_t* out, const epic_plan_desc* d) {
  const NvtxRange nvtx_range("epic_plan_create");
  if (!out || !d) return fail(EPIC_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  epic::ImageKernelShape shape{};
  bool fused_shape = false, unfused_ok = false;
  if (epic_status st = validate_desc(d, &shape, &fused_shape, &unfused_ok)) return st;

  epic_plan_s* p = new (std::nothrow) epic_plan_s();
  if (!p) return fail(EPIC_ERR_OOM, "host allocation failed");
  p->na = d->n_ant;
  p->nc = d->n_chan;
  p->n = d->grid_n;
  p->k = d->kernel_support;
  p->kernel = d->kernel;
  p->kparam = d->kernel_param;
  if (d->kernel_param_ant) p->kparam_ant.assign(d->kernel_param_ant, d->kernel_param_ant + d->n_ant);
  p->cell = d->cell_wavelengths;
  p->input = d->input;
  p->ant.assign(d->ant_xy_m, d->ant_xy_m + 2 * d->n_ant);
  p->freq.assign(d->freq_hz, d->freq_hz + d->n_chan);
  p->vscale.assign(d->n_chan, 1.0f);
  if (d->voltage_scale) p->vscale.assign(d->voltage_scale, d->voltage_scale + d->n_chan);
  p->flags.assign(d->n_ant, 0);
  if (d->flags)
    for (int a = 0; a < d->n_ant; ++a) p->flags[a] = d->flags[a] ? 1 : 0;
  p->stream = static_cast<cudaStream_t>(d->cuda_stream);
  p->shape = shape;
  if (d->workspace_bytes) p->workspace_budget = d->workspace_bytes;
  p->persistent = d->batch_persistent ? 1 : 0;

  // ---- gridding tables (Eq. 9), FP64 ----
  std::vector<int> cell0;
  std::vector<float> wts;
  if (epic_status st = build_grid_tables(p, cell0, wts)) {
    delete p;
    return st;
  }
  const int Na = p->na, C = p->nc, N = p->n, K = p->k, h = (K - 1) / 2;

  // ---- launch shape ----
  if (epic_status st = choose_path(p, d, fused_shape, unfused_ok)) {
    delete p;
    return st;
  }
  const bool fused = p->path == EPIC_PATH_FUSED;

  // ---- device tables ----
  std::vector<float2> twid(N);
  for (int m = 0; m < N; ++m)
    twid[m] = make_float2(static_cast<float>(std::cos(2.0 * kPi * m / N)),
                          static_cast<float>(std::sin(2.0 * kPi * m / N)));
  std::vector<int2> win(C);
  for (int c = 0; c < C; ++c) win[c] = make_int2(p->y0[c], p->rows[c]);
  std::vector<int4> win4(C);
  for (int c = 0; c < C; ++c) win4[c] = make_int4(p->y0[c], p->rows[c], p->x0[c], p->cols[c]);
  std::vector<int> cellf(static_cast<size_t>(C) * Na, -1);
  const int ws = fused ? epic::image_window_stride(N) : N;
  for (int c = 0; c < C; ++c)
    for (int a = 0; a < Na; ++a) {
      if (p->flags[a]) continue;
      const size_t ob = (static_cast<size_t>(c) * Na + a) * 2;
      const int bx = p->base[ob], by = p->base[ob + 1];
      cellf[static_cast<size_t>(c) * Na + a] = (by - h - p->y0[c]) * ws + (bx - h - p->x0[c]);
    }
  // gridding gather tables (see build_gather): the fused kernel, the plain
  // unfused path and the reduced-precision gridding use window columns, the
  // fused path's adjoint absolute columns
  std::vector<int> gofs, gbase, ugofs, ugbase;
  std::vector<uint4> gcnt, ugcnt;
  std::vector<uint2> gent, ugent;
  if (p->path == EPIC_PATH_FUSED || p->path == EPIC_PATH_UNFUSED) {
    const int n1 = p->path == EPIC_PATH_FUSED ? epic::image_fft_lanes(N) : epic::unfused_fft_lanes(N);
    if (epic_status st = build_gather(p, wts, n1, true, gofs, gcnt, gent, gbase)) {
      epic_plan_destroy(p);
      return st;
    }
    for (int c = 0; c < C; ++c) p->gmax = std::max(p->gmax, gbase[c + 1] - gbase[c]);
  }
  if (p->path == EPIC_PATH_FUSED) {
    const int n1 = epic::image_fft_lanes(N);
    if (epic_status st = build_gather(p, wts, n1, false, ugofs, ugcnt, ugent, ugbase)) {
      epic_plan_destroy(p);
      return st;
    }
  }
  std::vector<float2> pixph(C, make_float2(1.0f, 0.0f));
  std::vector<int> rowcol, order;
  std::vector<int2> ranges;
  if (p->path == EPIC_PATH_CLUSTER) build_cluster_tables(p, rowcol, order, ranges);
  std::vector<double2> gain(static_cast<size_t>(C) * Na, make_double2(1.0, 0.0));
  std::vector<float2> wgain(static_cast<size_t>(C) * Na, make_float2(1.0f, 0.0f));

  auto up = [&](auto& buf, const auto& host) -> cudaError_t {
    cudaError_t e2 = buf.alloc(host.size());
    if (e2 != cudaSuccess) return e2;
    return cudaMemcpy(buf.p, host.data(), host.size() * sizeof(host[0]), cudaMemcpyHostToDevice);
  };
  cudaError_t es[] = {up(p->d_cell0, cell0), up(p->d_wts, wts), up(p->d_wgain, wgain),
                      up(p->d_gain, gain), up(p->d_vscale, p->vscale), up(p->d_win, win),
                      up(p->d_twid, twid), up(p->d_flags, p->flags), up(p->d_win4, win4),
                      up(p->d_cellf, cellf), up(p->d_pixph, pixph), up(p->d_rowcol, rowcol),
                      up(p->d_order, order), up(p->d_ranges, ranges), up(p->d_gofs, gofs),
                      up(p->d_gent, gent), up(p->d_gbase, gbase), up(p->d_gcnt, gcnt),
                      up(p->d_ugofs, ugofs), up(p->d_ugcnt, ugcnt), up(p->d_ugent, ugent),
                      up(p->d_ugbase, ugbase)};
  for (cudaError_t x : es)
    if (x != cudaSuccess) {
      epic_plan_destroy(p);
      return x == cudaErrorMemoryAllocation ? fail(EPIC_ERR_OOM, "device allocation failed")
                                            : cuda_fail(x, "table upload");
    }
  cudaError_t e = p->d_held.alloc(1);
  if (e == cudaSuccess) e = cudaMemset(p->d_held.p, 0, sizeof(int));
  if (e == cudaSuccess) e = p->d_gbar.alloc(4);
  if (e == cudaSuccess) e = cudaMemset(p->d_gbar.p, 0, 4 * sizeof(unsigned));
  if (e == cudaSuccess) e = p->d_err.alloc(1);
  if (e == cudaSuccess) e = cudaMemset(p->d_err.p, 0, sizeof(int));
  if (e != cudaSuccess) {
    epic_plan_destroy(p);
    return cuda_fail(e, "counter");
  }
  *out = p;
  return EPIC_OK;
}

epic_status epic_plan_destroy(epic_plan_t p) {
  if (!p) return EPIC_OK;
  cudaStreamSynchronize(p->stream);
  p->d_cell0.release();
  p->d_wts.release();
  p->d_wgain.release();
  p->d_gain.release();
  p->d_vscale.release();
  p->d_win.release();
  p->d_win4.release();
  p->d_cellf.release();
  p->d_gofs.release();
  p->d_gent.release();
  p->d_gbase.release();
  p->d_gcnt.release();
  p->d_ugofs.release();
  p->d_ugcnt.release();
  p->d_ugent.release();
  p->d_ugbase.release();
  p->d_pixph.release();
  p->d_rowcol.release();
  p->d_order.release();
  p->d_ranges.release();
  p->d_twid.release();
  p->d_flags.release();
  p->d_a0.release();
  p->d_dden.release();
  p->d_kacc.release();
  p->d_pacc.release();
  p->d_held.release();
  p->d_stage_in.release();
  p->d_stage_img.release();
  p->d_ws.release();
  p->d_dldw.release();
  p->d_tc_hh.release();
  p->d_tc_dft.release();
  p->d_tc_scale.release();
  p->d_tc_pix.release();
  p->d_tc_gh.release();
  p->d_tc_dftr.release();
  p->d_gbar.release();
  p->d_err.release();
  p->d_ap.release();
  p->d_dp.release();
  p->d_kmp.release();
  p->d_gdir.release();
  p->d_ptab.release();
  p->d_pph.release();
  p->d_ptap.release();
  p->d_vm.release();
  p->d_vis32.release();
  p->d_xe_z.release();
  p->d_phase.release();
  p->d_bx.release();
  p->d_uv.release();
  p->d_iters.release();
  if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  delete p;
  return EPIC_OK;
}

epic_status epic_plan_set_stream(epic_plan_t p, void* stream) {
  if (epic_status s = check_plan(p)) return s;
  p->stream = static_cast<cudaStream_t>(stream);
  return EPIC_OK;
}

epic_status epic_plan_get_info(epic_plan_t p, epic_plan_info* info) {
  if (epic_status s = check_plan(p)) return s;
  if (!info) return fail(EPIC_ERR_INVALID_ARG, "info is NULL");
  info->n_ant = p->na;
  info->n_chan = p->nc;
  info->grid_n = p->n;
  info->kernel_support = p->k;
  info->window_rows = p->rows_alloc;
  info->cal_kx = p->cal ? p->k0x : -1;
  info->cal_ky = p->cal ? p->k0y : -1;
  info->ctas = p->ctas;
  info->units_per_chan = 0;
  info->smem_bytes = p->smem;
  info->frames_pending = p->frames;
  info->iteration = p->iteration;
  info->path = p->piped ? EPIC_PATH_PIPED : p->path;
  info->batch_time = p->ws_time;
  return EPIC_OK;
}

epic_status epic_set_gains(epic_plan_t p, const double* gains) {
  const NvtxRange nvtx_range("epic_set_gains");
  if (epic_status s = check_plan(p)) return s;
  if (!gains) return fail(EPIC_ERR_INVALID_ARG, "gains is NULL");
  const size_t n = static_cast<size_t>(p->nc) * p->na;
  std::vector<double2> g(n);
  std::vector<float2> w(n);
  for (size_t i = 0; i < n; ++i) {
    const double re = gains[2 * i], im = gains[2 * i + 1];
    const double m2 = re * re + im * im;
    if (!std::isfinite(re) || !std::isfinite(im) || !(m2 > 0))
      return fail(EPIC_ERR_INVALID_ARG, "gains must be finite and non-zero");
    g[i] = make_double2(re, im);
    w[i] = gain_multiplier_host(p->phase, i, re, im);
  }
  EPIC_CUDA(cudaMemcpyAsync(p->d_gain.p, g.data(), n * sizeof(double2), cudaMemcpyHostToDevice, p->stream));
  EPIC_CUDA(cudaMemcpyAsync(p->d_wgain.p, w.data(), n * sizeof(float2), cudaMemcpyHostToDevice, p->stream));
  EPIC_CUDA(cudaStreamSynchronize(p->stream));
  return EPIC_OK;
}

epic_status epic_image(epic_plan_t p, const void* d_volt, long long n_time, double* d_image,
                       int accumulate) {
  const NvtxRange nvtx_range("epic_image");
  if (epic_status s = check_plan(p)) return s;
  if (!d_volt || !d_image) return fail(EPIC_ERR_INVALID_ARG, "NULL device buffer");
  if (n_time < 1) return fail(EPIC_ERR_INVALID_ARG, "n_time must be >= 1");
  const size_t img_bytes = static_cast<size_t>(p->nc) * p->n * p->n * sizeof(double);
  if (!accumulate) EPIC_CUDA(cudaMemsetAsync(d_image, 0, img_bytes, p->stream));
  if (p->precision != EPIC_PREC_FP32) return image_tc(p, d_volt, n_time, d_image);
  if (p->path == EPIC_PATH_CLUSTER) return image_cluster(p, d_volt, n_time, d_image);
  if (p->path == EPIC_PATH_UNFUSED) return image_unfused(p, d_volt, n_time, d_image);
  epic::ImageArgs a = fused_args(p, d_volt, n_time, d_image, 1.0 / static_cast<double>(n_time));
  if (p->cal && p->npix > 0) {
    if (epic_status st = ensure_ptap(p, n_time)) return st;
    a.npix = p->npix;
    a.ptab = p->d_ptab.p;
    a.pph = p->d_pph.p;
    a.ptap = p->d_ptap.p;
  }
  EPIC_CUDA(epic::launch_image(p->n, a, p->stream));
  if (p->cal && p->npix > 0) {
    epic::MultiCorrArgs m{};
    m.volt = d_volt;
    m.input_fmt = p->input;
    m.n_time = n_time;
    m.n_chan = p->nc;
    m.n_ant = p->na;
    m.npix = p->npix;
    m.vscale = p->d_vscale.p;
    m.cell0 = p->d_cell0.p;
    m.ptap = p->d_ptap.p;
    m.kmp = p->d_kmp.p;
    // about two CTAs per SM, segments of at least 64 samples
    int segs = 1;
    while (static_cast<long long>(p->nc) * segs < 2LL * p->sms && n_time / (2 * segs) >= 64) segs *= 2;
    m.segs = segs;
    EPIC_CUDA(epic::launch_correlate_multi(m, p->stream));
  }
  if (p->cal) p->frames += n_time;
  return EPIC_OK;
}

epic_status epic_image_host(epic_plan_t p, const void* h_volt, long long n_time, double* h_image,
                            int accumulate) {
  const NvtxRange nvtx_range("epic_image_host");
  if (epic_status s = check_plan(p)) return s;
  if (!h_volt || !h_image) return fail(EPIC_ERR_INVALID_ARG, "NULL host buffer");
  if (n_time < 1) return fail(EPIC_ERR_INVALID_ARG, "n_time must be >= 1");
  const size_t elem = p->input == EPIC_IN_CI4 ? 1 : 8;
  const size_t in_bytes = static_cast<size_t>(n_time) * p->nc * p->na * elem;
  const size_t img_n = static_cast<size_t>(p->nc) * p->n * p->n;
  if (p->d_stage_in.n < in_bytes) {
    cudaError_t e = p->d_stage_in.alloc(in_bytes);
    if (e != cudaSuccess) return fail(EPIC_ERR_OOM, "staging allocation failed");
  }
  if (p->d_stage_img.n < img_n) {
    cudaError_t e = p->d_stage_img.alloc(img_n);
    if (e != cudaSuccess) return fail(EPIC_ERR_OOM, "staging allocation failed");
  }
  EPIC_CUDA(cudaMemcpyAsync(p->d_stage_in.p, h_volt, in_bytes, cudaMemcpyHostToDevice, p->stream));
  if (accumulate)
    EPIC_CUDA(cudaMemcpyAsync(p->d_stage_img.p, h_image, img_n * sizeof(double),
                              cudaMemcpyHostToDevice, p->stream));
  if (epic_status s = epic_image(p, p->d_stage_in.p, n_time, p->d_stage_img.p, accumulate)) return s;
  EPIC_CUDA(cudaMemcpyAsync(h_image, p->d_stage_img.p, img_n * sizeof(double), cudaMemcpyDeviceToHost,
                            p->stream));
  EPIC_CUDA(cudaStreamSynchronize(p->stream));
  return EPIC_OK;
}

epic_status epical_configure(epic_plan_t p, double cal_l, double cal_m, int n_src,
                             const double* src, double gamma, const double* g0) {
  const NvtxRange nvtx_range("epical_configure");
  if (epic_status s = check_plan(p)) return s;
  if (!(gamma >= 0.0 && gamma < 1.0)) return fail(EPIC_ERR_INVALID_ARG, "gamma must be in [0, 1)");
  if (n_src < 1 || !src) return fail(EPIC_ERR_INVALID_ARG, "at least one model source is required");
  const int Na = p->na, C = p->nc;
  int k0x = 0, k0y = 0;
  if (!nearest_pixel(p, cal_l, cal_m, &k0x, &k0y)) return fail(EPIC_ERR_INVALID_ARG, "calibrator outside the image");
  for (int si = 0; si < n_src; ++si)
    for (int j = 0; j < 3; ++j)
      if (!std::isfinite(src[3 * si + j])) return fail(EPIC_ERR_INVALID_ARG, "model sources must be finite");
  p->model.assign(src, src + 3 * static_cast<size_t>(n_src));
  const size_t n = static_cast<size_t>(C) * Na;
  std::vector<double2> a0(n), dd(n), g(n);
  std::vector<float2> w(n);
  std::vector<std::complex<double>> A, D;
  for (int c = 0; c < C; ++c) {
    pixel_response(p, c, k0x, k0y, A);
    model_denominator(p, c, A, D);
    for (int a = 0; a < Na; ++a) {
      const size_t i = static_cast<size_t>(c) * Na + a;
      a0[i] = make_double2(A[a].real(), A[a].imag());
      dd[i] = make_double2(D[a].real(), D[a].imag());
      double gr = 1.0, gi = 0.0;
      if (g0) {
        gr = g0[2 * i];
        gi = g0[2 * i + 1];
        if (!std::isfinite(gr) || !std::isfinite(gi) || !(gr * gr + gi * gi > 0))
          return fail(EPIC_ERR_INVALID_ARG, "initial gains must be finite and non-zero");
      }
      g[i] = make_double2(gr, gi);
      w[i] = gain_multiplier_host(p->phase, i, gr, gi);
    }
  }
  if (!p->d_a0.p) {
    cudaError_t es[] = {p->d_a0.alloc(n), p->d_dden.alloc(n), p->d_kacc.alloc(n), p->d_pacc.alloc(n)};
    for (cudaError_t x : es)
      if (x != cudaSuccess) return fail(EPIC_ERR_OOM, "EPICal allocation failed");
  }
  EPIC_CUDA(cudaMemcpyAsync(p->d_a0.p, a0.data(), n * sizeof(double2), cudaMemcpyHostToDevice, p->stream));
  EPIC_CUDA(cudaMemcpyAsync(p->d_dden.p, dd.data(), n * sizeof(double2), cudaMemcpyHostToDevice, p->stream));
  EPIC_CUDA(cudaMemcpyAsync(p->d_gain.p, g.data(), n * sizeof(double2), cudaMemcpyHostToDevice, p->stream));
  EPIC_CUDA(cudaMemcpyAsync(p->d_wgain.p, w.data(), n * sizeof(float2), cudaMemcpyHostToDevice, p->stream));
  {
    // pixel k0 of the window-coordinate transform
    std::vector<float2> ph(C);
    for (int c = 0; c < C; ++c) ph[c] = window_phase(p, c, k0x, k0y);
    EPIC_CUDA(cudaMemcpyAsync(p->d_pixph.p, ph.data(), C * sizeof(float2), cudaMemcpyHostToDevice,
                              p->stream));
  }
  EPIC_CUDA(cudaMemsetAsync(p->d_kacc.p, 0, n * sizeof(double2), p->stream));
  EPIC_CUDA(cudaMemsetAsync(p->d_pacc.p, 0, n * sizeof(double), p->stream));
  EPIC_CUDA(cudaStreamSynchronize(p->stream));
  p->k0x = k0x;
  p->k0y = k0y;
  p->gamma = gamma;
  p->cal = true;
  p->frames = 0;
  p->iteration = 0;
  p->npix = 0;                             // single-pixel form until epical_configure_pixels
  p->vm_stale = true;
  return EPIC_OK;
}

epic_status epic_visibilities(epic_plan_t p, const void* d_volt, long long n_time, double* d_vis,
                              int accumulate) {
  const NvtxRange nvtx_range("epic_visibilities");
  if (epic_status s = check_plan(p)) return s;
  if (!d_volt || !d_vis) return fail(EPIC_ERR_INVALID_ARG, "NULL device buffer");
  if (n_time < 1) return fail(EPIC_ERR_INVALID_ARG, "n_time must be >= 1");
  const size_t nv = static_cast<size_t>(p->nc) * p->na * p->na;
  if (p->input == EPIC_IN_CI4) {
    // tensor cores: FP16 integers, exact; time in segments that keep the
    // operand scratch within 1 GiB (and every FP32 sum below 2^24)
    const int na_p = (p->na + 63) / 64 * 64;
    const size_t row_bytes = static_cast<size_t>(p->nc) * 2 * na_p * sizeof(uint16_t);
    long long seg = static_cast<long long>((static_cast<size_t>(1) << 30) / row_bytes) / 64 * 64;
    seg = std::max<long long>(64, std::min<long long>(seg, 32768));
    seg = std::min<long long>(seg, (n_time + 63) / 64 * 64);
    if (p->xe_tp < seg) {
      EPIC_CUDA(cudaStreamSynchronize(p->stream));
      if (p->xe_tp == 0) EPIC_CUDA(epic::xe_prepare());
      if (p->d_xe_z.alloc(row_bytes / sizeof(uint16_t) * static_cast<size_t>(seg)) != cudaSuccess) {
        p->xe_tp = 0;
        return fail(EPIC_ERR_OOM, "X-engine operand scratch allocation failed");
      }
      if (!epic::xe_make_map(p->d_xe_z.p, p->nc, na_p, static_cast<int>(seg), p->tm_xe))
        return fail(EPIC_ERR_CUDA, "cuTensorMapEncodeTiled failed (X-engine)");
      p->xe_tp = static_cast<int>(seg);
    }
    epic::XeTcArgs x{};
    x.n_chan = p->nc;
    x.n_ant = p->na;
    x.na_p = na_p;
    x.tp = p->xe_tp;
    x.vscale = p->d_vscale.p;
    x.scale = 1.0 / static_cast<double>(n_time);
    x.vis = reinterpret_cast<double2*>(d_vis);
    x.err = p->d_err.p;
    for (long long t0 = 0; t0 < n_time; t0 += p->xe_tp) {
      const int nt = static_cast<int>(std::min<long long>(p->xe_tp, n_time - t0));
      x.accumulate = (t0 > 0 || accumulate) ? 1 : 0;
      EPIC_CUDA(epic::launch_xengine_tc(x, d_volt, t0, nt, p->d_xe_z.p, p->tm_xe, p->sms, p->stream));
    }
    return EPIC_OK;
  }
  if (!accumulate) EPIC_CUDA(cudaMemsetAsync(d_vis, 0, nv * sizeof(double2), p->stream));
  epic::XengineArgs a{};
  a.volt = d_volt;
  a.input_fmt = p->input;
  a.n_time = n_time;
  a.n_chan = p->nc;
  a.n_ant = p->na;
  a.vscale = p->d_vscale.p;
  a.scale = 1.0 / static_cast<double>(n_time);
  a.vis = reinterpret_cast<double2*>(d_vis);
  EPIC_CUDA(epic::launch_xengine(a, p->stream));
  return EPIC_OK;
}

epic_status epic_visibility_solve(epic_plan_t p, const double* d_vis, double* d_gains, int max_iter,
                                  double tol, double min_baseline, int* h_iters) {
  const NvtxRange nvtx_range("epic_visibility_solve");
  if (epic_status s = check_plan(p)) return s;
  if (!p->cal || p->model.empty()) return fail(EPIC_ERR_STATE, "configure EPICal (the model) first");
  if (!d_vis || !d_gains || max_iter < 1 || !(tol >= 0.0) || !(min_baseline >= 0.0))
    return fail(EPIC_ERR_INVALID_ARG, "bad solve arguments");
  const int C = p->nc, Na = p->na;
  const size_t nv = static_cast<size_t>(C) * Na * Na;
  if (static_cast<size_t>(Na) * (2 * sizeof(double2) + sizeof(float2)) > 200 * 1024)
    return fail(EPIC_ERR_UNSUPPORTED, "visibility solve holds the gains in shared memory (Na <= 5120)");
  if (p->vm_stale || !p->d_vm.p) {
    // phasors e_a(s) = e^{-2 pi i u_a . s} in FP64 on the host, V^M on the device
    const int ns = static_cast<int>(p->model.size() / 3);
    std::vector<double2> ph(static_cast<size_t>(C) * ns * Na);
    std::vector<double> flux(ns);
    std::vector<double2> uv(static_cast<size_t>(C) * Na);
    for (int si = 0; si < ns; ++si) flux[si] = p->model[3 * si + 2];
    for (int c = 0; c < C; ++c) {
      const double f = p->freq[c];
      for (int a = 0; a < Na; ++a)
        uv[static_cast<size_t>(c) * Na + a] = make_double2((p->ant[2 * a] * f) / kC, (p->ant[2 * a + 1] * f) / kC);
      for (int si = 0; si < ns; ++si)
        for (int a = 0; a < Na; ++a) {
          const double2 u = uv[static_cast<size_t>(c) * Na + a];
          const double arg = -2.0 * kPi * (u.x * p->model[3 * si] + u.y * p->model[3 * si + 1]);
          ph[(static_cast<size_t>(c) * ns + si) * Na + a] = make_double2(std::cos(arg), std::sin(arg));
        }
    }
    DevBuf<double2> d_ph;
    DevBuf<double> d_flux;
    cudaError_t es[] = {p->d_vm.alloc(nv), p->d_vis32.alloc(nv), p->d_uv.alloc(uv.size()), p->d_iters.alloc(C),
                        d_ph.alloc(ph.size()), d_flux.alloc(flux.size())};
    for (cudaError_t x : es)
      if (x != cudaSuccess) return fail(EPIC_ERR_OOM, "model visibility allocation failed");
    EPIC_CUDA(cudaMemcpyAsync(d_ph.p, ph.data(), ph.size() * sizeof(double2), cudaMemcpyHostToDevice, p->stream));
    EPIC_CUDA(cudaMemcpyAsync(d_flux.p, flux.data(), flux.size() * sizeof(double), cudaMemcpyHostToDevice,
                              p->stream));
    EPIC_CUDA(cudaMemcpyAsync(p->d_uv.p, uv.data(), uv.size() * sizeof(double2), cudaMemcpyHostToDevice,
                              p->stream));
    EPIC_CUDA(epic::launch_model_vis(C, Na, ns, d_ph.p, d_flux.p, p->d_vm.p, p->stream));
    EPIC_CUDA(cudaStreamSynchronize(p->stream));   // d_ph, d_flux are freed on return
    p->vm_stale = false;
  }
  epic::StefcalArgs a{};
  a.n_chan = C;
  a.n_ant = Na;
  a.vis32 = p->d_vis32.p;
  a.vm = p->d_vm.p;
  a.uv = p->d_uv.p;
  a.flags = p->d_flags.p;
  a.min_baseline = min_baseline;
  a.tol = tol;
  a.max_iter = max_iter;
  a.gains = reinterpret_cast<double2*>(d_gains);
  a.iters = p->d_iters.p;
  EPIC_CUDA(epic::launch_stefcal(a, reinterpret_cast<const double2*>(d_vis), p->stream));
  if (h_iters) {
    EPIC_CUDA(cudaMemcpyAsync(h_iters, p->d_iters.p, C * sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    EPIC_CUDA(cudaStreamSynchronize(p->stream));
  }
  return EPIC_OK;
}

epic_status epical_configure_pixels(epic_plan_t p, int n_pix, const double* pix_lm) {
  const NvtxRange nvtx_range("epical_configure_pixels");
  if (epic_status s = check_plan(p)) return s;
  if (!p->cal) return fail(EPIC_ERR_STATE, "configure EPICal (model, gamma) before its pixels");
  if (n_pix < 1 || !pix_lm) return fail(EPIC_ERR_INVALID_ARG, "need n_pix >= 1 and pix_lm");
  if (p->path != EPIC_PATH_FUSED || p->piped || p->precision != EPIC_PREC_FP32)
    return fail(EPIC_ERR_UNSUPPORTED, "multiple-pixel EPICal needs the fused FP32 path (N <= 128)");
  const int Na = p->na, C = p->nc, N = p->n;
  const int rounds = epic::image_col_rounds(N);
  epic::ImageKernelShape sh{};
  epic::image_kernel_shape(N, &sh);
  // owner of every pixel; taps ordered by (round, thread, slot) so that a
  // thread's taps of one round are consecutive
  struct Tap { int round, thread, slot, user, kx, ky; };
  std::vector<Tap> taps(n_pix);
  for (int i = 0; i < n_pix; ++i) {
    int kx = 0, ky = 0;
    if (!nearest_pixel(p, pix_lm[2 * i], pix_lm[2 * i + 1], &kx, &ky))
      return fail(EPIC_ERR_INVALID_ARG, "calibration pixel outside the image");
    epic::PixelOwner o{};
    if (!epic::image_pixel_owner(N, kx, ky, &o)) return fail(EPIC_ERR_UNSUPPORTED, "grid size");
    taps[i] = {o.round, o.thread, o.slot, i, kx, ky};
  }
  std::sort(taps.begin(), taps.end(), [](const Tap& x, const Tap& y) {
    return x.round != y.round ? x.round < y.round : x.thread != y.thread ? x.thread < y.thread : x.slot < y.slot;
  });
  for (int i = 1; i < n_pix; ++i)
    if (taps[i].kx == taps[i - 1].kx && taps[i].ky == taps[i - 1].ky)
      return fail(EPIC_ERR_INVALID_ARG, "two directions map to the same pixel");
  std::vector<uint2> tab(static_cast<size_t>(rounds) * sh.threads, make_uint2(0u, 0u));
  for (int i = n_pix - 1; i >= 0; --i) {
    uint2& e = tab[static_cast<size_t>(taps[i].round) * sh.threads + taps[i].thread];
    e.x |= 1u << taps[i].slot;
    e.y = static_cast<unsigned>(i);        // first (lowest) tap index of this thread and round
  }
  const size_t nap = static_cast<size_t>(C) * n_pix * Na;
  std::vector<double2> ap(nap), dp(nap);
  std::vector<float2> pph(static_cast<size_t>(C) * n_pix);
  std::vector<std::complex<double>> A, D;
  for (int c = 0; c < C; ++c)
    for (int i = 0; i < n_pix; ++i) {
      pixel_response(p, c, taps[i].kx, taps[i].ky, A);
      model_denominator(p, c, A, D);
      for (int a = 0; a < Na; ++a) {
        const size_t o = (static_cast<size_t>(c) * n_pix + i) * Na + a;
        ap[o] = make_double2(A[a].real(), A[a].imag());
        dp[o] = make_double2(D[a].real(), D[a].imag());
      }
      pph[static_cast<size_t>(c) * n_pix + i] = window_phase(p, c, taps[i].kx, taps[i].ky);
    }
  // per-direction solutions start from the current imaging gains
  const size_t n = static_cast<size_t>(C) * Na;
  std::vector<double2> g(n), gd(n * n_pix);
  EPIC_CUDA(cudaMemcpyAsync(g.data(), p->d_gain.p, n * sizeof(double2), cudaMemcpyDeviceToHost, p->stream));
  EPIC_CUDA(cudaStreamSynchronize(p->stream));
  for (size_t i = 0; i < n; ++i)
    for (int q = 0; q < n_pix; ++q) gd[i * n_pix + q] = g[i];
  cudaError_t es[] = {p->d_ap.alloc(nap), p->d_dp.alloc(nap), p->d_kmp.alloc(n * n_pix),
                      p->d_gdir.alloc(n * n_pix), p->d_ptab.alloc(tab.size()), p->d_pph.alloc(pph.size())};
  for (cudaError_t x : es)
    if (x != cudaSuccess) return fail(EPIC_ERR_OOM, "multiple-pixel EPICal allocation failed");
  p->d_ptap.release();
  p->ptap_time = 0;
  EPIC_CUDA(cudaMemcpyAsync(p->d_ap.p, ap.data(), nap * sizeof(double2), cudaMemcpyHostToDevice, p->stream));
  EPIC_CUDA(cudaMemcpyAsync(p->d_dp.p, dp.data(), nap * sizeof(double2), cudaMemcpyHostToDevice, p->stream));
  EPIC_CUDA(cudaMemcpyAsync(p->d_gdir.p, gd.data(), gd.size() * sizeof(double2), cudaMemcpyHostToDevice,
                            p->stream));
  EPIC_CUDA(cudaMemcpyAsync(p->d_ptab.p, tab.data(), tab.size() * sizeof(uint2), cudaMemcpyHostToDevice,
                            p->stream));
  EPIC_CUDA(cudaMemcpyAsync(p->d_pph.p, pph.data(), pph.size() * sizeof(float2), cudaMemcpyHostToDevice,
                            p->stream));
  EPIC_CUDA(cudaMemsetAsync(p->d_kmp.p, 0, n * n_pix * sizeof(double2), p->stream));
  EPIC_CUDA(cudaMemsetAsync(p->d_kacc.p, 0, n * sizeof(double2), p->stream));
  EPIC_CUDA(cudaMemsetAsync(p->d_pacc.p, 0, n * sizeof(double), p->stream));
  EPIC_CUDA(cudaStreamSynchronize(p->stream));
  p->pix_user.resize(n_pix);
  for (int i = 0; i < n_pix; ++i) p->pix_user[i] = taps[i].user;
  p->npix = n_pix;
  p->frames = 0;
  return EPIC_OK;
}

epic_status epical_get_direction_gains(epic_plan_t p, double* h_gains) {
  if (epic_status s = check_plan(p)) return s;
  if (!h_gains) return fail(EPIC_ERR_INVALID_ARG, "NULL output");
  if (p->npix < 1) return fail(EPIC_ERR_STATE, "multiple-pixel EPICal is not configured");
  const size_t n = static_cast<size_t>(p->nc) * p->na, P = p->npix;
  std::vector<double2> gd(n * P);
  EPIC_CUDA(cudaMemcpyAsync(gd.data(), p->d_gdir.p, gd.size() * sizeof(double2), cudaMemcpyDeviceToHost,
                            p->stream));
  EPIC_CUDA(cudaStreamSynchronize(p->stream));
  for (size_t i = 0; i < n; ++i)
    for (size_t q = 0; q < P; ++q) {
      const size_t o = (i * P + static_cast<size_t>(p->pix_user[q])) * 2;
      h_gains[o] = gd[i * P + q].x;
      h_gains[o + 1] = gd[i * P + q].y;
    }
  return EPIC_OK;
}

epic_status epical_average_channels(epic_plan_t p, int c_lo, int c_hi) {
  const NvtxRange nvtx_range("epical_average_channels");
  if (epic_status s = check_plan(p)) return s;
  if (!(0 <= c_lo && c_lo < c_hi && c_hi <= p->nc))
    return fail(EPIC_ERR_INVALID_ARG, "channel band must satisfy 0 <= c_lo < c_hi <= C");
  EPIC_CUDA(epic::launch_average_channels(p->na, c_lo, c_hi, p->d_flags.p, p->d_gain.p, p->d_wgain.p,
                                          p->d_phase.p, p->stream));
  return EPIC_OK;
}

epic_status epic_set_phase_centre(epic_plan_t p, double l0, double m0) {
  if (epic_status s = check_plan(p)) return s;
  if (!std::isfinite(l0) || !std::isfinite(m0) || !(l0 * l0 + m0 * m0 < 1.0))
    return fail(EPIC_ERR_INVALID_ARG, "phase centre must satisfy l0^2 + m0^2 < 1");
  const int C = p->nc, Na = p->na;
  const size_t n = static_cast<size_t>(C) * Na;
  if (l0 == 0.0 && m0 == 0.0) {
    p->phase.clear();
    p->d_phase.release();
  } else {
    p->phase.resize(n);
    for (int c = 0; c < C; ++c)
      for (int a = 0; a < Na; ++a) {
        const double f = p->freq[c];
        const double u = (p->ant[2 * a] * f) / kC, v = (p->ant[2 * a + 1] * f) / kC;
        const double arg = 2.0 * kPi * (u * l0 + v * m0);
        p->phase[static_cast<size_t>(c) * Na + a] = make_double2(std::cos(arg), std::sin(arg));
      }
    if (!p->d_phase.p && p->d_phase.alloc(n) != cudaSuccess)
      return fail(EPIC_ERR_OOM, "phase table allocation failed");
    EPIC_CUDA(cudaMemcpyAsync(p->d_phase.p, p->phase.data(), n * sizeof(double2), cudaMemcpyHostToDevice,
                              p->stream));
  }
  p->phase_l = l0;
  p->phase_m = m0;
  // multipliers of the current gains with the new phasing (in place)
  EPIC_CUDA(epic::launch_set_gains(static_cast<int>(n), p->d_gain.p, p->d_gain.p, p->d_wgain.p, p->d_phase.p,
                                   p->stream));
  EPIC_CUDA(cudaStreamSynchronize(p->stream));
  // calibrator pixel and responses depend on the phase centre
  p->cal = false;
  p->npix = 0;
  p->frames = 0;
  return EPIC_OK;
}

epic_status epical_fit_bandpass(epic_plan_t p, int c_lo, int c_hi, int deg_amp, int deg_phase) {
  const NvtxRange nvtx_range("epical_fit_bandpass");
  if (epic_status s = check_plan(p)) return s;
  if (!(0 <= c_lo && c_lo < c_hi && c_hi <= p->nc))
    return fail(EPIC_ERR_INVALID_ARG, "channel band must satisfy 0 <= c_lo < c_hi <= C");
  if (deg_amp < 0 || deg_phase < 0 || deg_amp > 7 || deg_phase > 7 || std::max(deg_amp, deg_phase) >= c_hi - c_lo)
    return fail(EPIC_ERR_INVALID_ARG, "degrees must be 0..7 and below the number of channels in the band");
  // abscissa: the band's frequencies mapped linearly onto [-1, 1]
  const int nb = c_hi - c_lo;
  double lo = p->freq[c_lo], hi = p->freq[c_lo];
  for (int c = c_lo; c < c_hi; ++c) {
    lo = std::min(lo, p->freq[c]);
    hi = std::max(hi, p->freq[c]);
  }
  std::vector<double> x(nb, 0.0);
  if (hi > lo)
    for (int k = 0; k < nb; ++k) x[k] = (p->freq[c_lo + k] - 0.5 * (lo + hi)) / (0.5 * (hi - lo));
  if (!p->d_bx.p && p->d_bx.alloc(p->nc) != cudaSuccess)
    return fail(EPIC_ERR_OOM, "bandpass scratch allocation failed");
  EPIC_CUDA(cudaMemcpyAsync(p->d_bx.p, x.data(), nb * sizeof(double), cudaMemcpyHostToDevice, p->stream));
  EPIC_CUDA(epic::launch_fit_bandpass(p->na, c_lo, c_hi, deg_amp, deg_phase, p->d_bx.p, p->d_flags.p, p->d_gain.p,
                                      p->d_wgain.p, p->d_phase.p, p->stream));
  EPIC_CUDA(cudaStreamSynchronize(p->stream));     // x is host memory of this call
  return EPIC_OK;
}

epic_status epical_update(epic_plan_t p, double* d_gains_out, int* d_status) {
  const NvtxRange nvtx_range("epical_update");
  if (epic_status s = check_plan(p)) return s;
  if (!p->cal) return fail(EPIC_ERR_STATE, "EPICal is not configured");
  if (p->frames < 1) return fail(EPIC_ERR_STATE, "no frames imaged since the last update");
  if (p->npix > 0) {
    epic::MultiUpdateArgs m{};
    m.n_chan = p->nc;
    m.n_ant = p->na;
    m.npix = p->npix;
    m.kmp = p->d_kmp.p;
    m.kacc = p->d_kacc.p;
    m.pacc = p->d_pacc.p;
    m.inv_frames = 1.0 / static_cast<double>(p->frames);
    m.ap = p->d_ap.p;
    m.dp = p->d_dp.p;
    m.gain = p->d_gain.p;
    m.wgain = p->d_wgain.p;
    m.gdir = p->d_gdir.p;
    m.flags = p->d_flags.p;
    m.gamma = p->gamma;
    m.dmin = kDmin;
    m.gout = reinterpret_cast<double2*>(d_gains_out);
    m.status = d_status;
    m.held_count = p->d_held.p;
    m.phase = p->d_phase.p;
    EPIC_CUDA(epic::launch_update_multi(m, p->stream));
    p->frames = 0;
    p->iteration += 1;
    return EPIC_OK;
  }
  epic::UpdateArgs u{};
  u.n_chan = p->nc;
  u.n_ant = p->na;
  u.kacc = p->d_kacc.p;
  u.pacc = p->d_pacc.p;
  u.inv_frames = 1.0 / static_cast<double>(p->frames);
  u.a0 = p->d_a0.p;
  u.dden = p->d_dden.p;
  u.gain = p->d_gain.p;
  u.wgain = p->d_wgain.p;
  u.flags = p->d_flags.p;
  u.gamma = p->gamma;
  u.dmin = kDmin;
  u.gout = reinterpret_cast<double2*>(d_gains_out);
  u.status = d_status;
  u.held_count = p->d_held.p;
  u.phase = p->d_phase.p;
  EPIC_CUDA(epic::launch_update(u, p->stream));
  p->frames = 0;
  p->iteration += 1;
  return EPIC_OK;
}

epic_status epic_plan_set_wait_limit(epic_plan_t p, int polls) {
  if (epic_status s = check_plan(p)) return s;
  if (polls < 0) return fail(EPIC_ERR_INVALID_ARG, "polls must be >= 0");
  p->wait_limit = polls;
  return EPIC_OK;
}

epic_status epic_plan_set_adjoint_precision(epic_plan_t p, int precision) {
  if (epic_status s = check_plan(p)) return s;
  if (precision != EPIC_PREC_FP32 && precision != EPIC_PREC_BF16)
    return fail(EPIC_ERR_INVALID_ARG, "adjoint precision must be EPIC_PREC_FP32 or EPIC_PREC_BF16");
  p->adjoint_precision = precision;
  return EPIC_OK;
}

epic_status epic_plan_sync(epic_plan_t p, int* n_held) {
  if (epic_status s = check_plan(p)) return s;
  EPIC_CUDA(cudaStreamSynchronize(p->stream));
  int held = 0, err = 0;
  EPIC_CUDA(cudaMemcpy(&held, p->d_held.p, sizeof(int), cudaMemcpyDeviceToHost));
  EPIC_CUDA(cudaMemset(p->d_held.p, 0, sizeof(int)));
  EPIC_CUDA(cudaMemcpy(&err, p->d_err.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (n_held) *n_held = held;
  if (err) {
    EPIC_CUDA(cudaMemset(p->d_err.p, 0, sizeof(int)));
    return fail(EPIC_ERR_TIMEOUT, "a bounded device wait timed out (a TMA-fed kernel gave up)");
  }
  if (held > 0) return fail(EPIC_ERR_NUMERIC, std::to_string(held) + " gains held by the EPICal update");
  return EPIC_OK;
}

epic_status epical_get_gains(epic_plan_t p, double* h_gains) {
  if (epic_status s = check_plan(p)) return s;
  if (!h_gains) return fail(EPIC_ERR_INVALID_ARG, "NULL output");
  const size_t n = static_cast<size_t>(p->nc) * p->na;
  EPIC_CUDA(cudaMemcpyAsync(h_gains, p->d_gain.p, n * sizeof(double2), cudaMemcpyDeviceToHost, p->stream));
  EPIC_CUDA(cudaStreamSynchronize(p->stream));
  return EPIC_OK;
}

namespace {
struct StateHeader {
  char magic[8];
  int n_chan, n_ant, cal, k0x, k0y, pad;
  double gamma;
  long long frames, iteration;
};
}  // namespace

epic_status epical_get_state(epic_plan_t p, void* buf, size_t* bytes) {
  if (epic_status s = check_plan(p)) return s;
  if (!bytes) return fail(EPIC_ERR_INVALID_ARG, "bytes is NULL");
  const size_t n = static_cast<size_t>(p->nc) * p->na;
  const size_t need = sizeof(StateHeader) + n * (sizeof(double2) * 2 + sizeof(double));
  if (!buf) {
    *bytes = need;
    return EPIC_OK;
  }
  if (*bytes < need) return fail(EPIC_ERR_INVALID_ARG, "state buffer too small");
  if (!p->cal) return fail(EPIC_ERR_STATE, "EPICal is not configured");
  StateHeader hd{};
  std::memcpy(hd.magic, "EPICST1", 8);
  hd.n_chan = p->nc;
  hd.n_ant = p->na;
  hd.cal = 1;
  hd.k0x = p->k0x;
  hd.k0y = p->k0y;
  hd.gamma = p->gamma;
  hd.frames = p->frames;
  hd.iteration = p->iteration;
  unsigned char* o = static_cast<unsigned char*>(buf);
  std::memcpy(o, &hd, sizeof hd);
  o += sizeof hd;
  EPIC_CUDA(cudaMemcpyAsync(o, p->d_gain.p, n * sizeof(double2), cudaMemcpyDeviceToHost, p->stream));
  EPIC_CUDA(cudaMemcpyAsync(o + n * sizeof(double2), p->d_kacc.p, n * sizeof(double2),
                            cudaMemcpyDeviceToHost, p->stream));
  EPIC_CUDA(cudaMemcpyAsync(o + 2 * n * sizeof(double2), p->d_pacc.p, n * sizeof(double),
                            cudaMemcpyDeviceToHost, p->stream));
  EPIC_CUDA(cudaStreamSynchronize(p->stream));
  *bytes = need;
  return EPIC_OK;
}

epic_status epical_set_state(epic_plan_t p, const void* buf, size_t bytes) {
  if (epic_status s = check_plan(p)) return s;
  if (!buf) return fail(EPIC_ERR_INVALID_ARG, "NULL state");
  if (!p->cal) return fail(EPIC_ERR_STATE, "configure EPICal before restoring its state");
  const size_t n = static_cast<size_t>(p->nc) * p->na;
  const size_t need = sizeof(StateHeader) + n * (sizeof(double2) * 2 + sizeof(double));
  if (bytes != need) return fail(EPIC_ERR_INVALID_ARG, "state size mismatch");
  StateHeader hd{};
  std::memcpy(&hd, buf, sizeof hd);
  if (std::memcmp(hd.magic, "EPICST1", 8) != 0 || hd.n_chan != p->nc || hd.n_ant != p->na)
    return fail(EPIC_ERR_INVALID_ARG, "state header does not match this plan");
  const unsigned char* i = static_cast<const unsigned char*>(buf) + sizeof hd;
  std::vector<double2> g(n);
  std::memcpy(g.data(), i, n * sizeof(double2));
  std::vector<float2> w(n);
  for (size_t k = 0; k < n; ++k) w[k] = gain_multiplier_host(p->phase, k, g[k].x, g[k].y);
  EPIC_CUDA(cudaMemcpyAsync(p->d_gain.p, g.data(), n * sizeof(double2), cudaMemcpyHostToDevice, p->stream));
  EPIC_CUDA(cudaMemcpyAsync(p->d_wgain.p, w.data(), n * sizeof(float2), cudaMemcpyHostToDevice, p->stream));
  EPIC_CUDA(cudaMemcpyAsync(p->d_kacc.p, i + n * sizeof(double2), n * sizeof(double2),
                            cudaMemcpyHostToDevice, p->stream));
  EPIC_CUDA(cudaMemcpyAsync(p->d_pacc.p, i + 2 * n * sizeof(double2), n * sizeof(double),
                            cudaMemcpyHostToDevice, p->stream));
  EPIC_CUDA(cudaStreamSynchronize(p->stream));
  p->k0x = hd.k0x;
  p->k0y = hd.k0y;
  p->gamma = hd.gamma;
  p->frames = hd.frames;
  p->iteration = hd.iteration;
  return EPIC_OK;
}

namespace {

// Median device time of `reps` epic_image calls on the plan stream.
epic_status time_image(epic_plan_t p, const void* d_volt, long long n_time, double* d_image, int reps,
                       double* ms_out) {
  cudaEvent_t e0, e1;
  EPIC_CUDA(cudaEventCreate(&e0));
  EPIC_CUDA(cudaEventCreate(&e1));
  std::vector<float> ms;
  epic_status st = epic_image(p, d_volt, n_time, d_image, 0);   // warm-up (and scratch growth)
  for (int r = 0; r < reps && st == EPIC_OK; ++r) {
    cudaEventRecord(e0, p->stream);
    st = epic_image(p, d_volt, n_time, d_image, 0);
    cudaEventRecord(e1, p->stream);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      st = cuda_fail(e, "autotune timing");
      break;
    }
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    ms.push_back(t);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != EPIC_OK) return st;
  std::sort(ms.begin(), ms.end());
  *ms_out = ms[ms.size() / 2];
  return EPIC_OK;
}

}  // namespace

epic_status epic_autotune(epic_plan_t p, const void* d_volt, long long n_time, double* d_image,
                          epic_tune_result* out) {
  const NvtxRange nvtx_range("epic_autotune");
  if (epic_status s = check_plan(p)) return s;
  if (!d_volt || !d_image || n_time < 1) return fail(EPIC_ERR_INVALID_ARG, "bad autotune arguments");
  const bool cal = p->cal;
  const long long frames = p->frames;
  p->cal = false;                         // tuning runs must not touch the EPICal sums
  epic_tune_result r{};
  r.path = p->path;
  double best = 0.0;
  epic_status st = EPIC_OK;
  const int reps = 3;
  if (p->path == EPIC_PATH_FUSED) {
    const int def = p->tune_units;
    st = time_image(p, d_volt, n_time, d_image, reps, &r.ms_default);
    best = r.ms_default;
    r.units_target = def;
    const int cand[] = {1, 2, 4, 8, 16, 32};
    for (int k : cand) {
      if (st != EPIC_OK) break;
      p->tune_units = k;
      double ms = 0;
      st = time_image(p, d_volt, n_time, d_image, reps, &ms);
      ++r.candidates;
      if (st == EPIC_OK && ms < best) {
        best = ms;
        r.units_target = k;
      }
    }
    p->tune_units = r.units_target;
  } else {
    const int def_nt = p->tune_nt, def_cols = p->tune_cols;
    st = time_image(p, d_volt, n_time, d_image, reps, &r.ms_default);
    best = r.ms_default;
    r.batch_time = p->ws_time;
    r.cols_target = def_cols;
    const int budget_nt = p->ws_time;     // largest batch the scratch budget allows
    for (int nt = 1; nt <= budget_nt && st == EPIC_OK; nt *= 2) {
      for (int ct : {2, 4, 8}) {
        p->tune_nt = nt;
        p->tune_cols = ct;
        double ms = 0;
        st = time_image(p, d_volt, n_time, d_image, reps, &ms);
        ++r.candidates;
        if (st != EPIC_OK) break;
        if (ms < best) {
          best = ms;
          r.batch_time = nt;
          r.cols_target = ct;
        }
      }
    }
    if (r.batch_time == budget_nt && def_nt == 0) r.batch_time = 0;
    p->tune_nt = r.batch_time;
    p->tune_cols = r.cols_target;
    // then the row kernel's variant: gather table in L1 or shared memory,
    // one or two frames per step
    r.row_table = p->tune_row_table;
    r.row_frames = p->tune_row_frames;
    if (p->precision == EPIC_PREC_FP32)
      for (int tb : {0, 1})
        for (int rf : {1, 2}) {
          if (st != EPIC_OK) break;
          p->tune_row_table = tb;
          p->tune_row_frames = rf;
          double ms = 0;
          st = time_image(p, d_volt, n_time, d_image, reps, &ms);
          ++r.candidates;
          if (st == EPIC_OK && ms < best) {
            best = ms;
            r.row_table = tb;
            r.row_frames = rf;
          }
        }
    p->tune_row_table = r.row_table;
    p->tune_row_frames = r.row_frames;
    // then one persistent launch per call against the batched launches
    r.batch_persistent = p->persistent;
    if (p->precision == EPIC_PREC_FP32 && epic::persistent_supported(p->n) && st == EPIC_OK) {
      const int def_pers = p->persistent;
      p->persistent = 1 - def_pers;
      double ms = 0;
      st = time_image(p, d_volt, n_time, d_image, reps, &ms);
      ++r.candidates;
      if (st == EPIC_OK && ms < best) {
        best = ms;
        r.batch_persistent = p->persistent;
      }
      p->persistent = r.batch_persistent;
    }
  }
  p->cal = cal;
  p->frames = frames;
  r.ms_best = best;
  if (out) *out = r;
  return st;
}

epic_status epic_graph_capture(epic_plan_t p, const void* d_volt, long long n_time, double* d_image,
                               double* d_gains_out) {
  const NvtxRange nvtx_range("epic_graph_capture");
  if (epic_status s = check_plan(p)) return s;
  if (!d_volt || !d_image || n_time < 1) return fail(EPIC_ERR_INVALID_ARG, "bad capture arguments");
  if (!p->stream) return fail(EPIC_ERR_INVALID_ARG, "graph capture needs a non-default plan stream");
  if (p->cal && p->frames != 0)
    return fail(EPIC_ERR_STATE, "update EPICal before capturing (frames are pending)");
  if (epic_status st = ensure_ptap(p, n_time)) return st;    // multiple-pixel taps
  if (p->path == EPIC_PATH_UNFUSED) {
    // allocate the batch scratch outside the capture
    const bool cal = p->cal;
    const long long frames = p->frames;
    p->cal = false;
    epic_status st = epic_image(p, d_volt, n_time, d_image, 0);
    p->cal = cal;
    p->frames = frames;
    if (st) return st;
  }
  EPIC_CUDA(cudaStreamSynchronize(p->stream));
  if (p->graph_exec) {
    cudaGraphExecDestroy(p->graph_exec);
    p->graph_exec = nullptr;
  }
  if (p->graph) {
    cudaGraphDestroy(p->graph);
    p->graph = nullptr;
  }
  const long long frames_before = p->frames;
  EPIC_CUDA(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
  epic_status st = epic_image(p, d_volt, n_time, d_image, 0);
  if (st == EPIC_OK && p->cal) st = epical_update(p, d_gains_out, nullptr);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(p->stream, &g);
  p->frames = frames_before;               // replays account for their own frames
  if (p->cal && st == EPIC_OK) p->iteration -= 1;
  if (st != EPIC_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&p->graph_exec, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(e, "cudaGraphInstantiate");
  }
  p->graph = g;
  return EPIC_OK;
}

epic_status epic_graph_launch(epic_plan_t p) {
  const NvtxRange nvtx_range("epic_graph_launch");
  if (epic_status s = check_plan(p)) return s;
  if (!p->graph_exec) return fail(EPIC_ERR_STATE, "no captured graph");
  EPIC_CUDA(cudaGraphLaunch(p->graph_exec, p->stream));
  if (p->cal) p->iteration += 1;
  return EPIC_OK;
}

epic_status epic_set_gains_device(epic_plan_t p, const double* d_gains) {
  const NvtxRange nvtx_range("epic_set_gains_device");
  if (epic_status s = check_plan(p)) return s;
  if (!d_gains) return fail(EPIC_ERR_INVALID_ARG, "d_gains is NULL");
  EPIC_CUDA(epic::launch_set_gains(p->nc * p->na, reinterpret_cast<const double2*>(d_gains), p->d_gain.p,
                                   p->d_wgain.p, p->d_phase.p, p->stream));
  return EPIC_OK;
}

epic_status epic_image_backward(epic_plan_t p, const void* d_volt, long long n_time,
                                const double* d_dl_di, double* d_grad_g) {
  const NvtxRange nvtx_range("epic_image_backward");
  if (epic_status s = check_plan(p)) return s;
  if (!d_volt || !d_dl_di || !d_grad_g) return fail(EPIC_ERR_INVALID_ARG, "NULL device buffer");
  if (n_time < 1) return fail(EPIC_ERR_INVALID_ARG, "n_time must be >= 1");
  if (p->path != EPIC_PATH_FUSED)
    return fail(EPIC_ERR_UNSUPPORTED, "the adjoint is built for the fused path (N <= 128)");
  const size_t n = static_cast<size_t>(p->nc) * p->na;
  if (!p->d_dldw.p) {
    cudaError_t e = p->d_dldw.alloc(n);
    if (e != cudaSuccess) return fail(EPIC_ERR_OOM, "gradient scratch allocation failed");
  }
  EPIC_CUDA(cudaMemsetAsync(p->d_dldw.p, 0, n * sizeof(double2), p->stream));
  epic::AdjointArgs a{};
  a.volt = d_volt;
  a.input_fmt = p->input;
  a.n_time = n_time;
  a.n_chan = p->nc;
  a.n_ant = p->na;
  a.support = p->k;
  a.cell0 = p->d_cell0.p;
  a.wts = p->d_wts.p;
  a.wgain = p->d_wgain.p;
  a.vscale = p->d_vscale.p;
  a.win = p->d_win.p;
  a.twid = p->d_twid.p;
  a.dldi = d_dl_di;
  a.dldw = p->d_dldw.p;
  a.img_scale = 1.0 / static_cast<double>(n_time);
  a.segs = choose_segments(p->nc, n_time, p->ctas, p->tune_units);
  a.rows_alloc = p->rows_alloc;
  a.rs = p->rs;
  const long long units = static_cast<long long>(p->nc) * a.segs;
  a.grid = static_cast<int>(std::min<long long>(units, p->ctas));
  a.gofs = p->d_ugofs.p;
  a.gcnt = p->d_ugcnt.p;
  a.gent = p->d_ugent.p;
  a.gbase = p->d_ugbase.p;
  const bool bf16 = p->adjoint_precision == EPIC_PREC_BF16;
  a.smem = epic::adjoint_smem_bytes(p->n, p->rows_alloc, p->rs, p->na, bf16);
  EPIC_CUDA(epic::launch_adjoint(p->n, a, bf16, p->stream));
  EPIC_CUDA(epic::launch_adjoint_finalize(p->nc, p->na, p->d_dldw.p, p->d_gain.p, p->d_phase.p, p->d_flags.p,
                                          reinterpret_cast<double2*>(d_grad_g), p->stream));
  return EPIC_OK;
}

epic_status epic_plan_get_grid_table(epic_plan_t p, int* base_xy, double* w) {
  if (epic_status s = check_plan(p)) return s;
  if (base_xy) std::memcpy(base_xy, p->base.data(), p->base.size() * sizeof(int));
  if (w) std::memcpy(w, p->w64.data(), p->w64.size() * sizeof(double));
  return EPIC_OK;
}

epic_status epic_unpack_ci4(epic_plan_t p, const unsigned char* d_in, float* d_out, long long n) {
  if (epic_status s = check_plan(p)) return s;
  if (n < 0 || (n > 0 && (!d_in || !d_out))) return fail(EPIC_ERR_INVALID_ARG, "bad unpack arguments");
  EPIC_CUDA(epic::launch_unpack(d_in, reinterpret_cast<float2*>(d_out), n, p->stream));
  return EPIC_OK;
}

}  // extern "C"

// ---- helpers for entry points outside this file ----
namespace epic {

int image_batch_scaled(epic_plan_s* p, const void* d_volt, long long n_time, double* d_image,
                       double img_scale) {
  if (!p || !d_volt || !d_image || n_time < 1) return fail(EPIC_ERR_INVALID_ARG, "bad batch");
  if (p->path != EPIC_PATH_FUSED)
    return fail(EPIC_ERR_UNSUPPORTED, "this call needs a plan on the fused path");
  if (p->cal && p->npix > 0)
    return fail(EPIC_ERR_UNSUPPORTED, "multiple-pixel EPICal needs its tap buffer (plan scratch)");
  const ImageArgs a = fused_args(p, d_volt, n_time, d_image, img_scale);
  cudaError_t e = launch_image(p->n, a, p->stream);
  if (e != cudaSuccess) return cuda_fail(e, "image launch");
  if (p->cal) p->frames += n_time;
  return EPIC_OK;
}

size_t plan_frame_bytes(const epic_plan_s* p) {
  return static_cast<size_t>(p->nc) * p->na * (p->input == EPIC_IN_CI4 ? 1 : 8);
}

size_t plan_image_elems(const epic_plan_s* p) { return static_cast<size_t>(p->nc) * p->n * p->n; }

cudaStream_t plan_stream(const epic_plan_s* p) { return p->stream; }

int plan_device(const epic_plan_s* p) { return p->device; }

int plan_path(const epic_plan_s* p) { return p->path; }

int set_error(int status, const char* msg) { return fail(static_cast<epic_status>(status), msg); }

}  // namespace epic
