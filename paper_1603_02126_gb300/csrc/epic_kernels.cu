// CUDA kernels of the EPIC imaging chain and the EPICal update (sm_103a).
//
// epic_image_fused<N>: one persistent launch images every frame (t, c) of a
// batch.  A CTA owns one work unit (channel c, a contiguous time segment) at
// a time and keeps that unit's running |E(s_k)|^2 sums in registers, so the
// only HBM traffic per frame is the Na voltage bytes.  The unit advances F
// frames per step (F spectra slots in shared memory), two CTA barriers per
// step:
//   row pass     EPICal correlation of the previous step's frames (Eqs. 12,
//                15); for every (frame, occupied grid row) the FFT lanes
//                gather their gridding taps (Eq. 9) from E' = E / g (Eq. 8)
//                in shared memory, then the N-point row FFT, written
//                transposed into the frame's slot;
//   column pass  N-point column FFTs (Eq. 10), |E|^2 accumulated in
//                registers, the calibrator pixel stored for the correlation;
//                then the next step's E' (4-bit unpack, gain) into shared
//                memory.
// The centring factor (-1)^(jx+jy) and the 1/Na of Eq. 10 are folded into
// the gridding weights by the plan; (-1)^(kx+ky) only matters for the
// calibrator pixel and is applied there.
//
// Each 1-D FFT of length N = N1 * N2 runs on a group of N1 lanes of one warp
// holding N2 points each: an N2-point DFT in registers, a twiddle
// e^{+2 pi i n1 k2 / N}, one exchange through shared memory, and N2/N1
// N1-point DFTs (the four-step decomposition).  Twiddles come from an FP64
// host table rounded to float.
#include "epic_fft.cuh"
#include "epic_fused_geo.cuh"
#include "epic_internal.h"

#include <cstdint>

namespace epic {
namespace {

using fft::cadd;
using fft::cmul;
using fft::csub;
using fft::Dft;
using fft::kFull;

constexpr double kPiD = 3.14159265358979323846;

// Raw voltage of antenna a in frame t, fetched one frame ahead: the 4-bit
// byte (ci4) or the complex64 value, unpacked only when it is used.
struct RawVolt {
  unsigned b;
  float2 f;
};

__device__ __forceinline__ RawVolt fetch_volt(const ImageArgs& A, long long t, int c, int a) {
  const size_t idx = (static_cast<size_t>(t) * A.n_chan + c) * A.n_ant + a;
  RawVolt r;
  if (A.input_fmt == 0) {
    r.b = __ldg(static_cast<const unsigned char*>(A.volt) + idx);
    r.f = make_float2(0.f, 0.f);
  } else {
    r.b = 0;
    r.f = __ldg(static_cast<const float2*>(A.volt) + idx);
  }
  return r;
}

__device__ __forceinline__ float2 unpack_volt(const ImageArgs& A, const RawVolt& r, float vs) {
  if (A.input_fmt == 0) {
    const int re = static_cast<int>(r.b << 24) >> 28;
    const int im = static_cast<int>(r.b << 28) >> 28;
    return make_float2(static_cast<float>(re) * vs, static_cast<float>(im) * vs);
  }
  return make_float2(r.f.x * vs, r.f.y * vs);
}

// One work unit (channel c, frames [t0, t1)) of the fused kernel, for an
// occupied window of at most N1 * NZ rows and columns: the grid is kept in
// window coordinates (first occupied row and column at 0), which only
// changes the phase of each image pixel, so every 1-D FFT has at most NZ
// non-zero inputs per lane and uses the pruned first-stage DFT.
//
// Gridding (Eq. 9) is a gather: the array layout is fixed for the plan, so
// the host lists, for every FFT lane (window row, lane n1), the taps that
// land on the lane's columns n1 + N1 j as entries (antenna, weight), grouped
// by j, with the group lengths as bytes of one 16-byte word per lane (loop
// bounds that do not wait on the entry loads).  Each frame the lane sums
// w * E'_a over its list straight into its FFT inputs; E'_a = E_a / g_a
// (Eq. 8) sits in shared memory, computed once per antenna while the
// previous step's column FFTs run.  No atomics, and the sum order is fixed.
//
// The unit advances F frames per step (F spectra slots): one row pass for
// the rows of all F frames, a CTA barrier, one column pass over all F
// frames, a barrier.  More work between barriers keeps more warps busy.
template <int N, int MAXA, int NZ, bool TS, int F>
__device__ __forceinline__ void fused_unit(const ImageArgs& A, int c, long long t0, long long t1,
                                           float2* Tt, float2* zg, const float2* tw, float2* pixs,
                                           float2* Es, int* sgofs, uint4* sgcnt, uint2* sgent) {
  using G = Geo<N>;
  constexpr int BT = G::BT, N1 = G::N1, N2 = G::N2, GROUPS = G::GROUPS, H = G::H;
  const int tid = threadIdx.x;
  const int g = tid / N1;
  const int n1 = tid % N1;
  constexpr int kGroupsPerWarp = 32 / N1;
  const int Na = A.n_ant;
  const int rs = A.rs;
  const size_t tslot = static_cast<size_t>(N) * rs;   // one frame's spectra

  const int4 wn = __ldg(A.win4 + c);                   // (y0, rows, x0, cols)
  const int R = wn.y;
  const float vs = A.vscale ? __ldg(A.vscale + c) : 1.0f;
  const float2* wg = A.wgain + static_cast<size_t>(c) * Na;
  // gather table of the channel: copied to shared memory for the unit (TS),
  // else read through L1
  const int gb = __ldg(A.gbase + c);
  const int* gofs = A.gofs + static_cast<size_t>(c) * A.rows_alloc * N1;
  const uint4* gcnt = A.gcnt + static_cast<size_t>(c) * A.rows_alloc * N1;
  const uint2* gent = A.gent + gb;
  if constexpr (TS) {
    const int gn = __ldg(A.gbase + c + 1) - gb;
    for (int i = tid; i < gn; i += BT) sgent[i] = __ldg(gent + i);
    for (int i = tid; i < R * N1; i += BT) {
      sgofs[i] = __ldg(gofs + i);
      sgcnt[i] = __ldg(gcnt + i);
    }
  }

  // calibrator pixel: column round, group, lane and register slot, phase
  const int pr = A.k0x / GROUPS, pg = A.k0x % GROUPS;
  const int pn1 = A.k0y % N1;
  const int pq = A.k0y / N1;
  const int pslot = (pq % H) * N1 + pq / H;
  const bool pix_owner = A.do_cal && g == pg && n1 == pn1;
  const float2 pph = A.do_cal ? __ldg(A.pixph + c) : make_float2(1.f, 0.f);

  float acc[G::NACC];
#pragma unroll
  for (int i = 0; i < G::NACC; ++i) acc[i] = 0.f;
  // raw voltages (scaled) of the current and previous step, for Eqs. 12, 15
  float2 kac[MAXA], ecur[F][MAXA], eprev[F][MAXA];
  float pac[MAXA];
#pragma unroll
  for (int i = 0; i < MAXA; ++i) {
    kac[i] = make_float2(0.f, 0.f);
    pac[i] = 0.f;
  }
  // first step: raw voltages and E' = E / g
#pragma unroll
  for (int f = 0; f < F; ++f)
#pragma unroll
    for (int i = 0; i < MAXA; ++i) {
      const int a = tid + BT * i;
      eprev[f][i] = make_float2(0.f, 0.f);
      ecur[f][i] = make_float2(0.f, 0.f);
      if (a < Na && t0 + f < t1) {
        ecur[f][i] = unpack_volt(A, fetch_volt(A, t0 + f, c, a), vs);
        Es[f * Na + a] = cmul(ecur[f][i], __ldg(wg + a));
      }
    }
  __syncthreads();

  int nprev = 0;                                       // frames of the previous step
  for (long long t = t0; t < t1; t += F) {
    const int nf = static_cast<int>(t1 - t < F ? t1 - t : F);
    const long long tn = t + F;                        // next step's first frame
    const int nfn = static_cast<int>(t1 - tn <= 0 ? 0 : (t1 - tn < F ? t1 - tn : F));
    // next step's voltages: pulled into L1 now, loaded after the row pass
    {
      const size_t esz = A.input_fmt == 0 ? 1 : sizeof(float2);
      for (int f = 0; f < nfn; ++f) {
        const size_t off = (static_cast<size_t>(tn + f) * A.n_chan + c) * Na * esz;
        const uintptr_t lo = (reinterpret_cast<uintptr_t>(A.volt) + off) & ~static_cast<uintptr_t>(127);
        const uintptr_t hi = reinterpret_cast<uintptr_t>(A.volt) + off + Na * esz;
        for (uintptr_t q = lo + static_cast<uintptr_t>(tid) * 128; q < hi; q += BT * 128)
          asm volatile("prefetch.global.L1 [%0];" ::"l"(q));
      }
    }

    // ---- B: correlation of the previous step, then gather + row FFTs ----
    if (A.do_cal) {
#pragma unroll
      for (int f = 0; f < F; ++f) {
        if (f < nprev) {
          const float2 p = pixs[f];
#pragma unroll
          for (int i = 0; i < MAXA; ++i) {
            const float2 e = eprev[f][i];
            kac[i].x += e.x * p.x + e.y * p.y;
            kac[i].y += e.y * p.x - e.x * p.y;
            pac[i] += e.x * e.x + e.y * e.y;
          }
        }
      }
    }
    // row tasks (frame, row) of the step; whole warps step through them
    // together (full-warp syncs in the FFT exchange); lanes past the last
    // task transform zeros and store nothing
    const int ntask = nf * R;
    for (int rb = g - g % kGroupsPerWarp; rb < ntask; rb += GROUPS) {
      const int task = rb + g % kGroupsPerWarp;
      const bool live = task < ntask;
      const int f = (F > 1 && live) ? task / R : 0;
      const int row = live ? task - f * R : 0;
      const float2* Ef = Es + f * Na;
      float2 v[N2];
#pragma unroll
      for (int j = 0; j < N2; ++j) v[j] = make_float2(0.f, 0.f);
      if (live) {
        const int li = row * N1 + n1;
        int e = TS ? sgofs[li] : __ldg(gofs + li);
        const uint4 cw = TS ? sgcnt[li] : __ldg(gcnt + li);
        const unsigned cv[4] = {cw.x, cw.y, cw.z, cw.w};
        const uint2* ge = TS ? sgent : gent;
#pragma unroll
        for (int j = 0; j < NZ; ++j) {
          const int cj = static_cast<int>((cv[j >> 2] >> (8 * (j & 3))) & 255u);
          float2 sum = make_float2(0.f, 0.f);
          for (int k = 0; k < cj; ++k) {
            const uint2 en = TS ? ge[e + k] : __ldg(ge + e + k);
            const float2 x = Ef[en.x];
            const float w = __uint_as_float(en.y);
            sum.x = fmaf(w, x.x, sum.x);
            sum.y = fmaf(w, x.y, sum.y);
          }
          e += cj;
          v[j] = sum;
        }
      }
      fft::fft_lanes_p<N1, N2, NZ>(v, n1, zg, tw, kFull);
      if (live) {
        float2* Tf = Tt + f * tslot;
        if constexpr (N1 % 8 == 0) {
          // kx = n1 + N1 h + N2 k1 = n1 (mod 8): one swizzled row index per thread
          float2* tb = Tf + n1 * rs + (row ^ n1);
#pragma unroll
          for (int h = 0; h < H; ++h)
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) tb[(N1 * h + N2 * k1) * rs] = v[h * N1 + k1];
        } else {
#pragma unroll
          for (int h = 0; h < H; ++h)
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) {
              const int kx = n1 + N1 * h + N2 * k1;
              Tf[kx * rs + (row ^ (kx & 7))] = v[h * N1 + k1];
            }
        }
      }
    }
    __syncthreads();

    // next step's voltages and gains, used after the column pass
    RawVolt nxt[F][MAXA];
    float2 gnx[MAXA];
#pragma unroll
    for (int i = 0; i < MAXA; ++i) {
      const int a = tid + BT * i;
      gnx[i] = (nfn > 0 && a < Na) ? __ldg(wg + a) : make_float2(0.f, 0.f);
#pragma unroll
      for (int f = 0; f < F; ++f)
        nxt[f][i] = (f < nfn && a < Na) ? fetch_volt(A, tn + f, c, a) : RawVolt{0u, make_float2(0.f, 0.f)};
    }

    // ---- C: column FFTs, |E|^2 accumulation, calibrator pixel ----
    const int jmax = (R - n1 + N1 - 1) / N1;             // this lane's rows n1 + N1 j < R
#pragma unroll
    for (int f = 0; f < F; ++f) {
      if (f < nf) {
        const float2* Tf = Tt + f * tslot;
#pragma unroll
        for (int r = 0; r < G::COLROUNDS; ++r) {
          const int kx = g + GROUPS * r;
          float2 v[N2];
          if constexpr (N1 % 8 == 0) {
            // kx = g (mod 8) and (n1 + N1 j) ^ s = (n1 ^ s) + N1 j for s < 8
            const float2* cb = Tf + kx * rs + (n1 ^ (g & 7));
#pragma unroll
            for (int j = 0; j < N2; ++j) v[j] = (j < NZ && j < jmax) ? cb[N1 * j] : make_float2(0.f, 0.f);
          } else {
#pragma unroll
            for (int j = 0; j < N2; ++j) {
              const int jw = n1 + N1 * j;
              v[j] = (j < NZ && jw < R) ? Tf[kx * rs + (jw ^ (kx & 7))] : make_float2(0.f, 0.f);
            }
          }
          fft::fft_lanes_p<N1, N2, NZ>(v, n1, zg, tw, kFull);
#pragma unroll
          for (int q = 0; q < N2; ++q) acc[r * N2 + q] += v[q].x * v[q].x + v[q].y * v[q].y;
          if (pix_owner && r == pr) {
#pragma unroll
            for (int q = 0; q < N2; ++q)
              if (q == pslot) pixs[f] = cmul(v[q], pph);
          }
          if (A.npix) {
            // multiple-pixel EPICal: this thread's calibration pixels of
            // the round (slot mask, index of its first tap)
            const uint2 tb = __ldg(A.ptab + r * BT + tid);
            if (tb.x) {
              float2* dst = A.ptap + (static_cast<size_t>(t + f) * A.n_chan + c) * A.npix;
              const float2* ph = A.pph + static_cast<size_t>(c) * A.npix;
#pragma unroll
              for (int q = 0; q < N2; ++q)
                if ((tb.x >> q) & 1u) {
                  const int pi = static_cast<int>(tb.y) + __popc(tb.x & ((1u << q) - 1u));
                  dst[pi] = cmul(v[q], __ldg(ph + pi));
                }
            }
          }
        }
      }
    }
    // ---- next step's E' (the row pass has finished reading Es) ----
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
      for (int i = 0; i < MAXA; ++i) {
        const int a = tid + BT * i;
        eprev[f][i] = ecur[f][i];
        if (f < nfn && a < Na) {
          ecur[f][i] = unpack_volt(A, nxt[f][i], vs);
          Es[f * Na + a] = cmul(ecur[f][i], gnx[i]);
        }
      }
    nprev = nf;
    __syncthreads();
  }

  // correlation of the unit's last step
  if (A.do_cal) {
#pragma unroll
    for (int f = 0; f < F; ++f) {
      if (f < nprev) {
        const float2 p = pixs[f];
#pragma unroll
        for (int i = 0; i < MAXA; ++i) {
          const float2 e = eprev[f][i];
          kac[i].x += e.x * p.x + e.y * p.y;
          kac[i].y += e.y * p.x - e.x * p.y;
          pac[i] += e.x * e.x + e.y * e.y;
        }
      }
    }
  }

  // flush the unit's partial sums (FP32 over one segment, FP64 across)
  double* img = A.image + static_cast<size_t>(c) * N * N;
#pragma unroll
  for (int r = 0; r < G::COLROUNDS; ++r) {
    const int kx = g + GROUPS * r;
#pragma unroll
    for (int h = 0; h < H; ++h)
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) {
        const int ky = n1 + N1 * h + N2 * k1;
        atomicAdd(img + ky * N + kx, static_cast<double>(acc[r * N2 + h * N1 + k1]) * A.img_scale);
      }
  }
  if (A.do_cal) {
    const int* cellf = A.cellf + static_cast<size_t>(c) * Na;
#pragma unroll
    for (int i = 0; i < MAXA; ++i) {
      const int a = tid + BT * i;
      if (a < Na && __ldg(cellf + a) >= 0) {
        const size_t o = static_cast<size_t>(c) * Na + a;
        atomicAdd(&A.kacc[o].x, static_cast<double>(kac[i].x));
        atomicAdd(&A.kacc[o].y, static_cast<double>(kac[i].y));
        atomicAdd(A.pacc + o, static_cast<double>(pac[i]));
      }
    }
  }
  __syncthreads();                                     // Es and pixs are reused by the next unit
}

template <int N, int MAXA, bool TS, int F>
__global__ void __launch_bounds__(Cfg<N>::BT, 1) epic_image_fused(const ImageArgs A) {
  using G = Geo<N>;
  constexpr int BT = G::BT, N1 = G::N1, N2 = G::N2, GROUPS = G::GROUPS;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* Tt = reinterpret_cast<float2*>(smem_raw);   // [F][N][rs] row spectra, transposed, swizzled
  float2* Z = Tt + F * N * A.rs;                       // [GROUPS][ZG] FFT exchange
  float2* tw = Z + GROUPS * G::ZG;                     // [N2][N1] twiddles
  float2* pixs = tw + N;                               // [4] calibrator pixels of the step
  float2* Es = pixs + 4;                               // [F][Na] gain-corrected voltages
  // gather table (TS): lane group lengths [rows_alloc * N1] (16-byte
  // aligned), lane offsets [rows_alloc * N1], entries [gmax]
  uint4* sgcnt = reinterpret_cast<uint4*>((reinterpret_cast<uintptr_t>(Es + F * A.n_ant) + 15) &
                                          ~static_cast<uintptr_t>(15));
  int* sgofs = reinterpret_cast<int*>(sgcnt + A.rows_alloc * N1);
  uint2* sgent = reinterpret_cast<uint2*>(sgofs + ((A.rows_alloc * N1 + 1) & ~1));

  const int tid = threadIdx.x;
  float2* zg = Z + (tid / N1) * G::ZG;
  // twiddles ordered [k2][n1]: e^{+2 pi i n1 k2 / N}
  for (int i = tid; i < N; i += BT) tw[i] = A.twid[(i % N1) * (i / N1)];
  __syncthreads();

  const long long T = A.n_time;
  const int units = A.n_chan * A.segs;
  for (int u = blockIdx.x; u < units; u += gridDim.x) {
    const int c = u / A.segs;
    const int s = u - c * A.segs;
    const long long t0 = T * s / A.segs;
    const long long t1 = T * (s + 1) / A.segs;
    if (t0 >= t1) continue;
    const int4 wn = __ldg(A.win4 + c);
    const int span = wn.y > wn.w ? wn.y : wn.w;          // occupied rows / columns
    if (span <= N1 * (N2 / 4))
      fused_unit<N, MAXA, N2 / 4, TS, F>(A, c, t0, t1, Tt, zg, tw, pixs, Es, sgofs, sgcnt, sgent);
    else if (span <= N1 * (N2 / 2))
      fused_unit<N, MAXA, N2 / 2, TS, F>(A, c, t0, t1, Tt, zg, tw, pixs, Es, sgofs, sgcnt, sgent);
    else
      fused_unit<N, MAXA, N2, TS, F>(A, c, t0, t1, Tt, zg, tw, pixs, Es, sgofs, sgcnt, sgent);
  }
}

// Multiplier of Eq. 8 with the phasing of the plan's phase centre:
// w = p / g (p = 1 when the plan is not phased).
__device__ __forceinline__ float2 gain_multiplier(double gr, double gi, const double2* phase, size_t i) {
  const double m2 = gr * gr + gi * gi;
  double wr = gr / m2, wi = -gi / m2;
  if (phase) {
    const double2 q = phase[i];
    const double xr = wr * q.x - wi * q.y, xi = wr * q.y + wi * q.x;
    wr = xr;
    wi = xi;
  }
  return make_float2(static_cast<float>(wr), static_cast<float>(wi));
}


// g and w = 1/g from device gains (no host round trip).
__global__ void set_gains_kernel(int n, const double2* __restrict__ g_in, double2* __restrict__ g,
                                 float2* __restrict__ w, const double2* __restrict__ phase) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double2 v = g_in[i];
  g[i] = v;
  w[i] = gain_multiplier(v.x, v.y, phase, i);
}

// Gains constant across channels c_lo .. c_hi - 1 (Sec. 5): per unflagged
// antenna, the complex mean of those channels' gains replaces each of them
// (FP64; a zero or non-finite mean leaves the antenna unchanged).
__global__ void average_channels_kernel(int n_ant, int c_lo, int c_hi, const unsigned char* __restrict__ flags,
                                        double2* __restrict__ gain, float2* __restrict__ wgain,
                                        const double2* __restrict__ phase) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n_ant || flags[a]) return;
  double sr = 0.0, si = 0.0;
  for (int c = c_lo; c < c_hi; ++c) {
    const double2 g = gain[static_cast<size_t>(c) * n_ant + a];
    sr += g.x;
    si += g.y;
  }
  const double inv = 1.0 / static_cast<double>(c_hi - c_lo);
  sr *= inv;
  si *= inv;
  const double m2 = sr * sr + si * si;
  if (!(m2 > 0.0) || !isfinite(m2)) return;
  for (int c = c_lo; c < c_hi; ++c) {
    const size_t i = static_cast<size_t>(c) * n_ant + a;
    gain[i] = make_double2(sr, si);
    wgain[i] = gain_multiplier(sr, si, phase, i);
  }
}

// Gain model across channels c_lo .. c_hi - 1 (Sec. 6, "Fitting gain
// models"), one thread per unflagged antenna, FP64: amplitudes and phases
// (unwrapped along the band, each step taken within pi) fitted by least
// squares with polynomials of degrees da and dp in the band abscissa x[]
// (normal equations, Gaussian elimination with partial pivoting); the
// band's gains become A(x) e^{i Phi(x)}.  An antenna with a zero or
// non-finite gain in the band is left as it is.
__global__ void fit_bandpass_kernel(int n_ant, int c_lo, int c_hi, int da, int dp, const double* __restrict__ x,
                                    const unsigned char* __restrict__ flags, double2* __restrict__ gain,
                                    float2* __restrict__ wgain, const double2* __restrict__ phase) {
  constexpr int kMaxDeg = 7;
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n_ant || flags[a]) return;
  const int nb = c_hi - c_lo;
  for (int c = c_lo; c < c_hi; ++c) {
    const double2 g = gain[static_cast<size_t>(c) * n_ant + a];
    if (!isfinite(g.x) || !isfinite(g.y) || (g.x == 0.0 && g.y == 0.0)) return;
  }
  double coef[2][kMaxDeg + 1];
  for (int which = 0; which < 2; ++which) {
    const int d = which == 0 ? da : dp;
    const int m = d + 1;
    double M[kMaxDeg + 1][kMaxDeg + 2];
    for (int i = 0; i < m; ++i)
      for (int j = 0; j <= m; ++j) M[i][j] = 0.0;
    double prev_raw = 0.0, prev = 0.0;
    for (int k = 0; k < nb; ++k) {
      const double2 g = gain[static_cast<size_t>(c_lo + k) * n_ant + a];
      double y;
      if (which == 0) {
        y = hypot(g.x, g.y);
      } else {
        const double raw = atan2(g.y, g.x);
        if (k == 0) {
          y = raw;
        } else {
          const double dd = raw - prev_raw;
          double dm = fmod(dd + kPiD, 2.0 * kPiD);
          if (dm < 0.0) dm += 2.0 * kPiD;
          dm -= kPiD;
          if (dm == -kPiD && dd > 0.0) dm = kPiD;
          y = prev + dm;
        }
        prev_raw = raw;
        prev = y;
      }
      double xp[2 * kMaxDeg + 1];
      xp[0] = 1.0;
      for (int i = 1; i <= 2 * d; ++i) xp[i] = xp[i - 1] * x[k];
      for (int i = 0; i < m; ++i) {
        for (int j = 0; j < m; ++j) M[i][j] += xp[i + j];
        M[i][m] += y * xp[i];
      }
    }
    for (int col = 0; col < m; ++col) {            // elimination with partial pivoting
      int piv = col;
      for (int r = col + 1; r < m; ++r)
        if (fabs(M[r][col]) > fabs(M[piv][col])) piv = r;
      if (piv != col)
        for (int j = 0; j <= m; ++j) {
          const double t = M[col][j];
          M[col][j] = M[piv][j];
          M[piv][j] = t;
        }
      for (int r = col + 1; r < m; ++r) {
        const double f = M[r][col] / M[col][col];
        for (int j = col; j <= m; ++j) M[r][j] -= f * M[col][j];
      }
    }
    for (int i = m - 1; i >= 0; --i) {
      double v = M[i][m];
      for (int j = i + 1; j < m; ++j) v -= M[i][j] * coef[which][j];
      coef[which][i] = v / M[i][i];
    }
  }
  for (int k = 0; k < nb; ++k) {
    double amp = 0.0, ph = 0.0;
    for (int i = da; i >= 0; --i) amp = amp * x[k] + coef[0][i];
    for (int i = dp; i >= 0; --i) ph = ph * x[k] + coef[1][i];
    double sn, cs;
    sincos(ph, &sn, &cs);
    const double gr = amp * cs, gi = amp * sn;
    if (!isfinite(gr) || !isfinite(gi) || (gr == 0.0 && gi == 0.0)) continue;
    const size_t i = static_cast<size_t>(c_lo + k) * n_ant + a;
    gain[i] = make_double2(gr, gi);
    wgain[i] = gain_multiplier(gr, gi, phase, i);
  }
}

// EPICal update (Eqs. 15-17) in FP64, one thread per (channel, antenna).
__global__ void epical_update_kernel(const UpdateArgs A) {
  const int n = A.n_chan * A.n_ant;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int a = i % A.n_ant;
  const double2 k = A.kacc[i];
  const double kx = k.x * A.inv_frames, ky = k.y * A.inv_frames;
  const double pb = A.pacc[i] * A.inv_frames;
  const double2 g = A.gain[i];
  const double2 a0 = A.a0[i];
  const double2 d = A.dden[i];
  // q = conj(A0) * P / conj(g)
  const double nr = a0.x * pb, ni = -a0.y * pb;   // conj(A0) * P
  const double gr = g.x, gi = -g.y;               // conj(g)
  const double gg = gr * gr + gi * gi;
  const double qr = (nr * gr + ni * gi) / gg;
  const double qi = (ni * gr - nr * gi) / gg;
  const double cr = kx - qr, ci = ky - qi;        // C_a (Eq. 15)
  const double dd = d.x * d.x + d.y * d.y;
  const double sr = (cr * d.x + ci * d.y) / dd;   // C / D (Eq. 16)
  const double si = (ci * d.x - cr * d.y) / dd;
  const double one_m = 1.0 - A.gamma;
  const double nxr = one_m * sr + A.gamma * g.x;  // Eq. 17
  const double nxi = one_m * si + A.gamma * g.y;
  const bool held = A.flags[a] != 0 || !(dd > A.dmin * A.dmin) || !isfinite(nxr) ||
                    !isfinite(nxi) || (nxr == 0.0 && nxi == 0.0);
  double2 out = g;
  if (!held) {
    out = make_double2(nxr, nxi);
    A.gain[i] = out;
    A.wgain[i] = gain_multiplier(nxr, nxi, A.phase, i);
  }
  if (A.status) A.status[i] = held ? 1 : 0;
  if (held && !A.flags[a]) atomicAdd(A.held_count, 1);
  if (A.gout) A.gout[i] = out;
  A.kacc[i] = make_double2(0.0, 0.0);
  A.pacc[i] = 0.0;
}

__global__ void unpack_ci4_kernel(const unsigned char* __restrict__ in, float2* __restrict__ out,
                                  long long n) {
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += stride) {
    const unsigned b = in[i];
    const int re = static_cast<int>(b << 24) >> 28;
    const int im = static_cast<int>(b << 28) >> 28;
    out[i] = make_float2(static_cast<float>(re), static_cast<float>(im));
  }
}

template <int N, int MAXA, int F>
cudaError_t prepare_nmf(size_t smem, int* ctas) {
  cudaError_t e = cudaFuncSetAttribute(epic_image_fused<N, MAXA, true, F>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(epic_image_fused<N, MAXA, false, F>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, epic_image_fused<N, MAXA, true, F>,
                                                       Cfg<N>::BT, smem);
}

// Frames per step: 2 for the 512-thread shapes (N = 64, 128), else 1.
template <int N>
constexpr int kMaxSteps = Cfg<N>::BT >= 512 ? 2 : 1;

// One antenna per thread when Na <= CTA size, else up to kMaxAntPerThread.
template <int N>
cudaError_t prepare_n(size_t smem, int n_ant, int steps, int* ctas) {
  if (steps == 2 && kMaxSteps<N> == 2) {
    if (n_ant <= Cfg<N>::BT) return prepare_nmf<N, 1, kMaxSteps<N>>(smem, ctas);
    return prepare_nmf<N, kMaxAntPerThread, kMaxSteps<N>>(smem, ctas);
  }
  if (n_ant <= Cfg<N>::BT) return prepare_nmf<N, 1, 1>(smem, ctas);
  return prepare_nmf<N, kMaxAntPerThread, 1>(smem, ctas);
}

template <int N, int MAXA, int F>
void launch_nmf(const ImageArgs& a, cudaStream_t s) {
  if (a.gsmem)
    epic_image_fused<N, MAXA, true, F><<<a.grid, Cfg<N>::BT, a.smem, s>>>(a);
  else
    epic_image_fused<N, MAXA, false, F><<<a.grid, Cfg<N>::BT, a.smem, s>>>(a);
}

template <int N>
cudaError_t launch_n(const ImageArgs& a, cudaStream_t s) {
  const bool two = a.steps == 2 && kMaxSteps<N> == 2;
  if (a.n_ant <= Cfg<N>::BT) {
    if (two) launch_nmf<N, 1, kMaxSteps<N>>(a, s);
    else launch_nmf<N, 1, 1>(a, s);
  } else {
    if (two) launch_nmf<N, kMaxAntPerThread, kMaxSteps<N>>(a, s);
    else launch_nmf<N, kMaxAntPerThread, 1>(a, s);
  }
  return cudaGetLastError();
}

template <int N>
void shape_n(ImageKernelShape* o) {
  o->threads = Cfg<N>::BT;
  o->groups = Geo<N>::GROUPS;
  o->max_ant = Cfg<N>::BT * kMaxAntPerThread;
}

}  // namespace

cudaError_t launch_average_channels(int n_ant, int c_lo, int c_hi, const unsigned char* flags, double2* gain,
                                    float2* wgain, const double2* phase, cudaStream_t s) {
  average_channels_kernel<<<(n_ant + 255) / 256, 256, 0, s>>>(n_ant, c_lo, c_hi, flags, gain, wgain, phase);
  return cudaGetLastError();
}

cudaError_t launch_fit_bandpass(int n_ant, int c_lo, int c_hi, int deg_amp, int deg_phase, const double* x,
                                const unsigned char* flags, double2* gain, float2* wgain, const double2* phase,
                                cudaStream_t s) {
  fit_bandpass_kernel<<<(n_ant + 127) / 128, 128, 0, s>>>(n_ant, c_lo, c_hi, deg_amp, deg_phase, x, flags, gain,
                                                           wgain, phase);
  return cudaGetLastError();
}

cudaError_t launch_set_gains(int n, const double2* g_in, double2* g, float2* w, const double2* phase,
                             cudaStream_t s) {
  set_gains_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, g_in, g, w, phase);
  return cudaGetLastError();
}

template <int N>
void owner_n(int kx, int ky, PixelOwner* o) {
  using G = Geo<N>;
  const int m = ky / G::N1;
  o->round = kx / G::GROUPS;
  o->thread = (kx % G::GROUPS) * G::N1 + ky % G::N1;
  o->slot = (m % G::H) * G::N1 + m / G::H;
}

bool image_pixel_owner(int n, int kx, int ky, PixelOwner* out) {
  if (kx < 0 || ky < 0 || kx >= n || ky >= n) return false;
  switch (n) {
    case 16: owner_n<16>(kx, ky, out); return true;
    case 32: owner_n<32>(kx, ky, out); return true;
    case 64: owner_n<64>(kx, ky, out); return true;
    case 128: owner_n<128>(kx, ky, out); return true;
    default: return false;
  }
}

int image_col_rounds(int n) {
  switch (n) {
    case 16: return Geo<16>::COLROUNDS;
    case 32: return Geo<32>::COLROUNDS;
    case 64: return Geo<64>::COLROUNDS;
    case 128: return Geo<128>::COLROUNDS;
    default: return 0;
  }
}

int image_window_stride(int n) {
  switch (n) {
    case 16: return 16 + Geo<16>::N1;
    case 32: return 32 + Geo<32>::N1;
    case 64: return 64 + Geo<64>::N1;
    case 128: return 128 + Geo<128>::N1;
    default: return 0;
  }
}

bool image_kernel_shape(int n, ImageKernelShape* out) {
  switch (n) {
    case 16: shape_n<16>(out); return true;
    case 32: shape_n<32>(out); return true;
    case 64: shape_n<64>(out); return true;
    case 128: shape_n<128>(out); return true;
    default: return false;
  }
}

int image_rs(int rows_alloc) {
  int rs = rows_alloc;
  while (rs % 16 != 4) ++rs;
  return rs;
}


int image_rs_fused(int rows_alloc) {
  int rs = ((rows_alloc + 7) / 8) * 8;     // room for the (row ^ (kx & 7)) swizzle
  while (rs % 16 != 8) rs += 8;
  return rs;
}

size_t image_smem_bytes(int n, int n_ant, int rs, int steps) {
  int groups = 0, zg = 0;
  switch (n) {
    case 16: groups = Geo<16>::GROUPS; zg = Geo<16>::ZG; break;
    case 32: groups = Geo<32>::GROUPS; zg = Geo<32>::ZG; break;
    case 64: groups = Geo<64>::GROUPS; zg = Geo<64>::ZG; break;
    case 128: groups = Geo<128>::GROUPS; zg = Geo<128>::ZG; break;
    default: return 0;
  }
  // spectra [F][N][rs], exchange, twiddles, calibrator pixels, E' [F][Na]
  const size_t elems = static_cast<size_t>(steps) * n * rs + static_cast<size_t>(groups) * zg + n + 4 +
                       static_cast<size_t>(steps) * n_ant;
  return elems * sizeof(float2);
}

size_t image_table_bytes(int rows_alloc, int n1, long long gmax) {
  return 16 + static_cast<size_t>(rows_alloc) * n1 * sizeof(uint4) +
         static_cast<size_t>((rows_alloc * n1 + 1) & ~1) * sizeof(int) + static_cast<size_t>(gmax) * sizeof(uint2);
}

int image_fft_lanes(int n) {
  switch (n) {
    case 16: return Geo<16>::N1;
    case 32: return Geo<32>::N1;
    case 64: return Geo<64>::N1;
    case 128: return Geo<128>::N1;
    default: return 0;
  }
}

int image_max_steps(int n) {
  switch (n) {
    case 16: return kMaxSteps<16>;
    case 32: return kMaxSteps<32>;
    case 64: return kMaxSteps<64>;
    case 128: return kMaxSteps<128>;
    default: return 1;
  }
}

cudaError_t image_kernel_prepare(int n, size_t smem, int n_ant, int steps, int* ctas) {
  switch (n) {
    case 16: return prepare_n<16>(smem, n_ant, steps, ctas);
    case 32: return prepare_n<32>(smem, n_ant, steps, ctas);
    case 64: return prepare_n<64>(smem, n_ant, steps, ctas);
    case 128: return prepare_n<128>(smem, n_ant, steps, ctas);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_image(int n, const ImageArgs& a, cudaStream_t s) {
  if (a.piped) return launch_piped(n, a, s);
  switch (n) {
    case 16: return launch_n<16>(a, s);
    case 32: return launch_n<32>(a, s);
    case 64: return launch_n<64>(a, s);
    case 128: return launch_n<128>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_update(const UpdateArgs& a, cudaStream_t s) {
  const int n = a.n_chan * a.n_ant;
  const int bt = 256;
  epical_update_kernel<<<(n + bt - 1) / bt, bt, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const unsigned char* in, float2* out, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int bt = 256;
  long long blocks = (n + bt - 1) / bt;
  if (blocks > 152 * 32) blocks = 152 * 32;
  unpack_ci4_kernel<<<static_cast<unsigned>(blocks), bt, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

}  // namespace epic
