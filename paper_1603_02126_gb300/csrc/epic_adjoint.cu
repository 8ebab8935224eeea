// Adjoint of the imaging chain (differentiation form), FP32 and BF16.
//
// For the loss L of the time-averaged image I, the gradient with respect to
// the conjugate gain multipliers w_a is accumulated per (channel, time
// segment) unit by recomputing every frame: gridding gather, row FFTs,
// column FFTs, multiply by R = dL/dI, inverse column FFTs into the grid
// window, inverse row FFTs, degridding of the K x K taps of every antenna
// and the product with conj(E_a(t)).  adjoint_finalize turns dL/dconj(w)
// into the gradient with respect to the gains (w = p / g).
#include "epic_fft.cuh"
#include "epic_fused_geo.cuh"
#include "epic_internal.h"

#include <cstdint>

namespace epic {
namespace {

using fft::cmul;

__device__ __forceinline__ float2 load_volt(const void* volt, int fmt, int n_chan, int n_ant,
                                           long long t, int c, int a) {
  const size_t idx = (static_cast<size_t>(t) * n_chan + c) * n_ant + a;
  if (fmt == 0) {
    const unsigned b = __ldg(static_cast<const unsigned char*>(volt) + idx);
    const int re = static_cast<int>(b << 24) >> 28;
    const int im = static_cast<int>(b << 28) >> 28;
    return make_float2(static_cast<float>(re), static_cast<float>(im));
  }
  return __ldg(static_cast<const float2*>(volt) + idx);
}

// Adjoint of the imaging chain (differentiation form).  With R = dL/dI for
// the dirty image I, X(t) the raw FFT of the folded grid of frame t, and
// W'_a the folded stencil weights, the gradient of L with respect to the
// conjugate gain multipliers is
//   dL/dconj(w_a) = (1/T) sum_t conj(E_a(t)) sum_j W'_a(j) [F^- (R . X(t))]_j
// (F^- = the conjugate transform).  Every frame is recomputed (nothing is
// stored): gridding as a per-lane gather from E' in shared memory (the plan's
// absolute-column tap lists) straight into the row FFTs, column FFTs,
// multiply by R, inverse column FFTs into the grid window, inverse row FFTs,
// degridding gather of the K x K taps per antenna.  E' of the next frame is
// formed during the degridding.  R for the unit's channel stays in registers.
template <int N, int MAXA>
__global__ void __launch_bounds__(Cfg<N>::BT, 1) epic_image_adjoint(const AdjointArgs A) {
  using G = Geo<N>;
  constexpr int BT = G::BT, N1 = G::N1, N2 = G::N2, GROUPS = G::GROUPS, H = G::H;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* Wg = reinterpret_cast<float2*>(smem_raw);   // [rows_alloc][N]
  float2* Tt = Wg + A.rows_alloc * N;                  // [N][rs] or [rows][N]
  float2* Z = Tt + N * A.rs;
  float2* tw = Z + GROUPS * G::ZG;
  float2* Es = tw + N;                                 // [Na] E / g of the current frame

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int g = tid / N1;
  const int n1 = tid % N1;
  const unsigned gmask = fft::group_mask<N1>(lane);
  float2* zg = Z + g * G::ZG;

  for (int i = tid; i < N; i += BT) tw[i] = A.twid[i];
  __syncthreads();

  const int Na = A.n_ant;
  const int K = A.support;
  const int KK = K * K;
  const long long T = A.n_time;
  const int units = A.n_chan * A.segs;

  for (int u = blockIdx.x; u < units; u += gridDim.x) {
    const int c = u / A.segs;
    const int s = u - c * A.segs;
    const long long t0 = T * s / A.segs;
    const long long t1 = T * (s + 1) / A.segs;
    if (t0 >= t1) continue;
    const int2 wn = __ldg(A.win + c);
    const int y0 = wn.x, R = wn.y;
    const float vs = A.vscale ? __ldg(A.vscale + c) : 1.0f;
    const int* cell0 = A.cell0 + static_cast<size_t>(c) * Na;
    const float* wts = A.wts + static_cast<size_t>(c) * Na * KK;
    const float2* wg = A.wgain + static_cast<size_t>(c) * Na;
    const double* rimg = A.dldi + static_cast<size_t>(c) * N * N;
    const int* gofs = A.gofs + static_cast<size_t>(c) * A.rows_alloc * N1;
    const uint4* gcnt = A.gcnt + static_cast<size_t>(c) * A.rows_alloc * N1;
    const uint2* gent = A.gent + __ldg(A.gbase + c);

    // R_k for this thread's pixels, in the column-FFT output order
    float rk[G::NACC];
#pragma unroll
    for (int r = 0; r < G::COLROUNDS; ++r) {
      const int kx = g + GROUPS * r;
#pragma unroll
      for (int h = 0; h < H; ++h)
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) {
          const int ky = n1 + N1 * h + N2 * k1;
          rk[r * N2 + h * N1 + k1] = static_cast<float>(__ldg(rimg + ky * N + kx));
        }
    }
    // raw voltages (scaled) of the unit's first frame and its E' = E / g
    float2 gac[MAXA], ecur[MAXA];
#pragma unroll
    for (int i = 0; i < MAXA; ++i) {
      const int a = tid + BT * i;
      gac[i] = make_float2(0.f, 0.f);
      ecur[i] = make_float2(0.f, 0.f);
      if (a < Na) {
        const float2 e = load_volt(A.volt, A.input_fmt, A.n_chan, Na, t0, c, a);
        ecur[i] = make_float2(e.x * vs, e.y * vs);
        Es[a] = cmul(ecur[i], __ldg(wg + a));
      }
    }
    __syncthreads();

    for (long long t = t0; t < t1; ++t) {
      // ---- B: gridding gather (Eq. 9, absolute columns n1 + N1 j) + row FFTs ----
      for (int row = g; row < R; row += GROUPS) {
        float2 v[N2];
        {
          const int li = row * N1 + n1;
          int e = __ldg(gofs + li);
          const uint4 cw = __ldg(gcnt + li);
          const unsigned cv[4] = {cw.x, cw.y, cw.z, cw.w};
#pragma unroll
          for (int j = 0; j < N2; ++j) {
            const int cj = static_cast<int>((cv[j >> 2] >> (8 * (j & 3))) & 255u);
            float2 sum = make_float2(0.f, 0.f);
            for (int k = 0; k < cj; ++k) {
              const uint2 en = __ldg(gent + e + k);
              const float2 x = Es[en.x];
              const float w = __uint_as_float(en.y);
              sum.x = fmaf(w, x.x, sum.x);
              sum.y = fmaf(w, x.y, sum.y);
            }
            e += cj;
            v[j] = sum;
          }
        }
        fft_group<N>(v, n1, zg, tw, gmask);
#pragma unroll
        for (int h = 0; h < H; ++h)
#pragma unroll
          for (int k1 = 0; k1 < N1; ++k1) Tt[(n1 + N1 * h + N2 * k1) * A.rs + row] = v[h * N1 + k1];
      }
      __syncthreads();

      // ---- C: column FFTs, multiply by R, inverse column FFTs into the window ----
#pragma unroll
      for (int r = 0; r < G::COLROUNDS; ++r) {
        const int kx = g + GROUPS * r;
        float2 v[N2];
#pragma unroll
        for (int j = 0; j < N2; ++j) {
          const int jw = n1 + N1 * j - y0;
          v[j] = (jw >= 0 && jw < R) ? Tt[kx * A.rs + jw] : make_float2(0.f, 0.f);
        }
        fft_group<N>(v, n1, zg, tw, gmask);
        // output slot h*N1 + k1 holds ky = n1 + N1*(h + H*k1): the inverse
        // transform's input slot j = h + H*k1; conjugate for F^-
        float2 u[N2];
#pragma unroll
        for (int h = 0; h < H; ++h)
#pragma unroll
          for (int k1 = 0; k1 < N1; ++k1) {
            const float rv = rk[r * N2 + h * N1 + k1];
            const float2 x = v[h * N1 + k1];
            u[h + H * k1] = make_float2(x.x * rv, -x.y * rv);
          }
        fft_group<N>(u, n1, zg, tw, gmask);
#pragma unroll
        for (int h = 0; h < H; ++h)
#pragma unroll
          for (int k1 = 0; k1 < N1; ++k1) {
            const int jw = n1 + N1 * h + N2 * k1 - y0;
            if (jw >= 0 && jw < R) {
              const float2 x = u[h * N1 + k1];
              Wg[jw * N + kx] = make_float2(x.x, -x.y);
            }
          }
      }
      __syncthreads();

      // ---- D: inverse row FFTs of the window rows, row-major into Tt ----
      for (int row = g; row < R; row += GROUPS) {
        float2 v[N2];
        float2* wr = Wg + row * N;
#pragma unroll
        for (int j = 0; j < N2; ++j) {
          const float2 x = wr[n1 + N1 * j];
          v[j] = make_float2(x.x, -x.y);
        }
        fft_group<N>(v, n1, zg, tw, gmask);
#pragma unroll
        for (int h = 0; h < H; ++h)
#pragma unroll
          for (int k1 = 0; k1 < N1; ++k1) {
            const float2 x = v[h * N1 + k1];
            Tt[row * N + n1 + N1 * h + N2 * k1] = make_float2(x.x, -x.y);
          }
      }
      __syncthreads();

      // ---- E: degrid and accumulate conj(E_a) Y_a ----
#pragma unroll
      for (int i = 0; i < MAXA; ++i) {
        const int a = tid + BT * i;
        if (a < Na) {
          const int c0 = __ldg(cell0 + a);
          if (c0 >= 0) {
            const float* wa = wts + static_cast<size_t>(a) * KK;
            float yr = 0.f, yi = 0.f;
            for (int dy = 0; dy < K; ++dy)
              for (int dx = 0; dx < K; ++dx) {
                const float w = __ldg(wa + dy * K + dx);
                const float2 b = Tt[c0 + dy * N + dx];
                yr += w * b.x;
                yi += w * b.y;
              }
            const float2 e = ecur[i];
            gac[i].x += e.x * yr + e.y * yi;     // conj(e) * y
            gac[i].y += e.x * yi - e.y * yr;
          }
          // next frame's raw voltages and E' (the row pass reads Es after the barrier)
          if (t + 1 < t1) {
            const float2 e = load_volt(A.volt, A.input_fmt, A.n_chan, Na, t + 1, c, a);
            ecur[i] = make_float2(e.x * vs, e.y * vs);
            Es[a] = cmul(ecur[i], __ldg(wg + a));
          }
        }
      }
      __syncthreads();                                 // Tt and Es are rewritten next frame
    }
#pragma unroll
    for (int i = 0; i < MAXA; ++i) {
      const int a = tid + BT * i;
      if (a < Na && cell0[a] >= 0) {
        const size_t o = static_cast<size_t>(c) * Na + a;
        atomicAdd(&A.dldw[o].x, static_cast<double>(gac[i].x) * A.img_scale);
        atomicAdd(&A.dldw[o].y, static_cast<double>(gac[i].y) * A.img_scale);
      }
    }
  }
}

// The BF16 form of the adjoint: the same four transforms per frame, with
// two frames (t, t + 1) carried together through every FFT, multiply and
// shared-memory exchange as fft::Cb2 values (BF16 pairs, one packed
// instruction per operation for both frames).  Gridding sums, the degridding
// sums and the conj(E_a) product stay FP32; the spectra are rounded to BF16
// once per butterfly.  A unit with an odd number of frames pairs its last
// frame with a zero frame.
template <int N, int MAXA>
__global__ void __launch_bounds__(Cfg<N>::BT, 1) epic_image_adjoint_b2(const AdjointArgs A) {
  using G = Geo<N>;
  using fft::Cb2;
  constexpr int BT = G::BT, N1 = G::N1, N2 = G::N2, GROUPS = G::GROUPS, H = G::H;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cb2* Wg = reinterpret_cast<Cb2*>(smem_raw);         // [rows_alloc][N]
  Cb2* Tt = Wg + A.rows_alloc * N;                     // [N][rs] or [rows][N]
  Cb2* Z = Tt + N * A.rs;
  Cb2* tw = Z + GROUPS * G::ZG;                        // [N] twiddles as splat pairs
  float2* Es = reinterpret_cast<float2*>(tw + N);      // [2][Na] E / g of the frame pair

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int g = tid / N1;
  const int n1 = tid % N1;
  const unsigned gmask = fft::group_mask<N1>(lane);
  Cb2* zg = Z + g * G::ZG;

  for (int i = tid; i < N; i += BT) {
    const float2 w = A.twid[i];
    tw[i] = Cb2{__float2bfloat162_rn(w.x), __float2bfloat162_rn(w.y)};
  }
  __syncthreads();

  const int Na = A.n_ant;
  const int K = A.support;
  const int KK = K * K;
  const long long T = A.n_time;
  const int units = A.n_chan * A.segs;
  float2* Es0 = Es;
  float2* Es1 = Es + Na;

  for (int u = blockIdx.x; u < units; u += gridDim.x) {
    const int c = u / A.segs;
    const int s = u - c * A.segs;
    const long long t0 = T * s / A.segs;
    const long long t1 = T * (s + 1) / A.segs;
    if (t0 >= t1) continue;
    const int2 wn = __ldg(A.win + c);
    const int y0 = wn.x, R = wn.y;
    const float vs = A.vscale ? __ldg(A.vscale + c) : 1.0f;
    const int* cell0 = A.cell0 + static_cast<size_t>(c) * Na;
    const float* wts = A.wts + static_cast<size_t>(c) * Na * KK;
    const float2* wg = A.wgain + static_cast<size_t>(c) * Na;
    const double* rimg = A.dldi + static_cast<size_t>(c) * N * N;
    const int* gofs = A.gofs + static_cast<size_t>(c) * A.rows_alloc * N1;
    const uint4* gcnt = A.gcnt + static_cast<size_t>(c) * A.rows_alloc * N1;
    const uint2* gent = A.gent + __ldg(A.gbase + c);

    // R_k for this thread's pixels (column-FFT output order), two pixels
    // per register as BF16 (splat when used)
    __nv_bfloat162 rk[G::NACC / 2];
#pragma unroll
    for (int r = 0; r < G::COLROUNDS; ++r) {
      const int kx = g + GROUPS * r;
#pragma unroll
      for (int h = 0; h < H; ++h)
#pragma unroll
        for (int k1 = 0; k1 < N1; k1 += 2) {
          const int ky = n1 + N1 * h + N2 * k1;
          rk[(r * N2 + h * N1 + k1) / 2] = __floats2bfloat162_rn(static_cast<float>(__ldg(rimg + ky * N + kx)),
                                                                 static_cast<float>(__ldg(rimg + (ky + N2) * N + kx)));
        }
    }
    // raw voltages (scaled) of the unit's first two frames and their E' = E / g
    float2 gac[MAXA], e0[MAXA], e1[MAXA];
#pragma unroll
    for (int i = 0; i < MAXA; ++i) {
      const int a = tid + BT * i;
      gac[i] = make_float2(0.f, 0.f);
      e0[i] = make_float2(0.f, 0.f);
      e1[i] = make_float2(0.f, 0.f);
      if (a < Na) {
        const float2 w = __ldg(wg + a);
        const float2 x0 = load_volt(A.volt, A.input_fmt, A.n_chan, Na, t0, c, a);
        e0[i] = make_float2(x0.x * vs, x0.y * vs);
        Es0[a] = cmul(e0[i], w);
        if (t0 + 1 < t1) {
          const float2 x1 = load_volt(A.volt, A.input_fmt, A.n_chan, Na, t0 + 1, c, a);
          e1[i] = make_float2(x1.x * vs, x1.y * vs);
        }
        Es1[a] = cmul(e1[i], w);
      }
    }
    __syncthreads();

    for (long long t = t0; t < t1; t += 2) {
      // ---- B: gridding gather of both frames (FP32 sums) + row FFTs ----
      for (int row = g; row < R; row += GROUPS) {
        Cb2 v[N2];
        {
          const int li = row * N1 + n1;
          int e = __ldg(gofs + li);
          const uint4 cw = __ldg(gcnt + li);
          const unsigned cv[4] = {cw.x, cw.y, cw.z, cw.w};
#pragma unroll
          for (int j = 0; j < N2; ++j) {
            const int cj = static_cast<int>((cv[j >> 2] >> (8 * (j & 3))) & 255u);
            float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f);
            for (int k = 0; k < cj; ++k) {
              const uint2 en = __ldg(gent + e + k);
              const float w = __uint_as_float(en.y);
              const float2 x0 = Es0[en.x], x1 = Es1[en.x];
              s0.x = fmaf(w, x0.x, s0.x);
              s0.y = fmaf(w, x0.y, s0.y);
              s1.x = fmaf(w, x1.x, s1.x);
              s1.y = fmaf(w, x1.y, s1.y);
            }
            e += cj;
            v[j] = fft::cb2_pack(s0, s1);
          }
        }
        fft_group<N>(v, n1, zg, tw, gmask);
#pragma unroll
        for (int h = 0; h < H; ++h)
#pragma unroll
          for (int k1 = 0; k1 < N1; ++k1) Tt[(n1 + N1 * h + N2 * k1) * A.rs + row] = v[h * N1 + k1];
      }
      __syncthreads();

      // ---- C: column FFTs, multiply by R, inverse column FFTs into the window ----
#pragma unroll
      for (int r = 0; r < G::COLROUNDS; ++r) {
        const int kx = g + GROUPS * r;
        Cb2 v[N2];
#pragma unroll
        for (int j = 0; j < N2; ++j) {
          const int jw = n1 + N1 * j - y0;
          v[j] = (jw >= 0 && jw < R) ? Tt[kx * A.rs + jw] : Cb2{__float2bfloat162_rn(0.f), __float2bfloat162_rn(0.f)};
        }
        fft_group<N>(v, n1, zg, tw, gmask);
        // output slot h*N1 + k1 holds ky = n1 + N1*(h + H*k1): the inverse
        // transform's input slot j = h + H*k1; conjugate for F^-
        Cb2 w[N2];
#pragma unroll
        for (int h = 0; h < H; ++h)
#pragma unroll
          for (int k1 = 0; k1 < N1; ++k1) {
            const int ri = r * N2 + h * N1 + k1;
            const __nv_bfloat162 rv = (ri & 1) ? __high2bfloat162(rk[ri >> 1]) : __low2bfloat162(rk[ri >> 1]);
            const Cb2 x = v[h * N1 + k1];
            w[h + H * k1] = Cb2{__hmul2(x.re, rv), __hneg2(__hmul2(x.im, rv))};
          }
        fft_group<N>(w, n1, zg, tw, gmask);
#pragma unroll
        for (int h = 0; h < H; ++h)
#pragma unroll
          for (int k1 = 0; k1 < N1; ++k1) {
            const int jw = n1 + N1 * h + N2 * k1 - y0;
            if (jw >= 0 && jw < R) {
              const Cb2 x = w[h * N1 + k1];
              Wg[jw * N + kx] = Cb2{x.re, __hneg2(x.im)};
            }
          }
      }
      __syncthreads();

      // ---- D: inverse row FFTs of the window rows, row-major into Tt ----
      for (int row = g; row < R; row += GROUPS) {
        Cb2 v[N2];
        const Cb2* wr = Wg + row * N;
#pragma unroll
        for (int j = 0; j < N2; ++j) {
          const Cb2 x = wr[n1 + N1 * j];
          v[j] = Cb2{x.re, __hneg2(x.im)};
        }
        fft_group<N>(v, n1, zg, tw, gmask);
#pragma unroll
        for (int h = 0; h < H; ++h)
#pragma unroll
          for (int k1 = 0; k1 < N1; ++k1) {
            const Cb2 x = v[h * N1 + k1];
            Tt[row * N + n1 + N1 * h + N2 * k1] = Cb2{x.re, __hneg2(x.im)};
          }
      }
      __syncthreads();

      // ---- E: degrid both frames (FP32 sums) and accumulate conj(E_a) Y_a ----
#pragma unroll
      for (int i = 0; i < MAXA; ++i) {
        const int a = tid + BT * i;
        if (a < Na) {
          const int c0 = __ldg(cell0 + a);
          if (c0 >= 0) {
            const float* wa = wts + static_cast<size_t>(a) * KK;
            float2 y0s = make_float2(0.f, 0.f), y1s = make_float2(0.f, 0.f);
            for (int dy = 0; dy < K; ++dy)
              for (int dx = 0; dx < K; ++dx) {
                const float w = __ldg(wa + dy * K + dx);
                const Cb2 b = Tt[c0 + dy * N + dx];
                y0s.x = fmaf(w, __low2float(b.re), y0s.x);
                y0s.y = fmaf(w, __low2float(b.im), y0s.y);
                y1s.x = fmaf(w, __high2float(b.re), y1s.x);
                y1s.y = fmaf(w, __high2float(b.im), y1s.y);
              }
            gac[i].x += e0[i].x * y0s.x + e0[i].y * y0s.y + e1[i].x * y1s.x + e1[i].y * y1s.y;
            gac[i].y += e0[i].x * y0s.y - e0[i].y * y0s.x + e1[i].x * y1s.y - e1[i].y * y1s.x;
          }
          // the next pair's raw voltages and E' (the row pass reads Es after the barrier)
          if (t + 2 < t1) {
            const float2 w = __ldg(wg + a);
            const float2 x0 = load_volt(A.volt, A.input_fmt, A.n_chan, Na, t + 2, c, a);
            e0[i] = make_float2(x0.x * vs, x0.y * vs);
            Es0[a] = cmul(e0[i], w);
            e1[i] = make_float2(0.f, 0.f);
            if (t + 3 < t1) {
              const float2 x1 = load_volt(A.volt, A.input_fmt, A.n_chan, Na, t + 3, c, a);
              e1[i] = make_float2(x1.x * vs, x1.y * vs);
            }
            Es1[a] = cmul(e1[i], w);
          }
        }
      }
      __syncthreads();                                 // Tt and Es are rewritten next pair
    }
#pragma unroll
    for (int i = 0; i < MAXA; ++i) {
      const int a = tid + BT * i;
      if (a < Na && cell0[a] >= 0) {
        const size_t o = static_cast<size_t>(c) * Na + a;
        atomicAdd(&A.dldw[o].x, static_cast<double>(gac[i].x) * A.img_scale);
        atomicAdd(&A.dldw[o].y, static_cast<double>(gac[i].y) * A.img_scale);
      }
    }
  }
}

// grad = 2 dL/dconj(g) = 2 dL/dconj(w) * (-1 / conj(g)^2); flagged -> 0.
__global__ void adjoint_finalize_kernel(int n, int n_ant, const double2* __restrict__ dldw,
                                        const double2* __restrict__ gain, const double2* __restrict__ phase,
                                        const unsigned char* __restrict__ flags,
                                        double2* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (flags[i % n_ant]) {
    out[i] = make_double2(0.0, 0.0);
    return;
  }
  const double2 g = gain[i];
  // w = p / g: dw/dg = -p / g^2, so 2 dL/dconj(g) = 2 dL/dconj(w) (-conj(p) / conj(g)^2)
  const double ar = g.x * g.x - g.y * g.y, ai = -2.0 * g.x * g.y;   // conj(g)^2
  const double den = ar * ar + ai * ai;
  double qr = -ar / den, qi = ai / den;                             // -1 / conj(g)^2
  if (phase) {
    const double2 q = phase[i];                                     // times conj(p)
    const double xr = qr * q.x + qi * q.y, xi = qi * q.x - qr * q.y;
    qr = xr;
    qi = xi;
  }
  const double2 d = dldw[i];
  out[i] = make_double2(2.0 * (d.x * qr - d.y * qi), 2.0 * (d.x * qi + d.y * qr));
}

template <int N>
cudaError_t adjoint_n(const AdjointArgs& a, bool bf16, cudaStream_t s) {
  void (*k)(AdjointArgs);
  if (a.n_ant <= Cfg<N>::BT) k = bf16 ? epic_image_adjoint_b2<N, 1> : epic_image_adjoint<N, 1>;
  else k = bf16 ? epic_image_adjoint_b2<N, kMaxAntPerThread> : epic_image_adjoint<N, kMaxAntPerThread>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(a.smem));
  if (e != cudaSuccess) return e;
  k<<<a.grid, Cfg<N>::BT, a.smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_adjoint(int n, const AdjointArgs& a, bool bf16, cudaStream_t s) {
  switch (n) {
    case 16: return adjoint_n<16>(a, bf16, s);
    case 32: return adjoint_n<32>(a, bf16, s);
    case 64: return adjoint_n<64>(a, bf16, s);
    case 128: return adjoint_n<128>(a, bf16, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_adjoint_finalize(int n_chan, int n_ant, const double2* dldw, const double2* gain,
                                    const double2* phase, const unsigned char* flags, double2* out,
                                    cudaStream_t s) {
  const int n = n_chan * n_ant;
  adjoint_finalize_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, n_ant, dldw, gain, phase, flags, out);
  return cudaGetLastError();
}

size_t adjoint_smem_bytes(int n, int rows_alloc, int rs, int n_ant, bool bf16) {
  int groups = 0, zg = 0;
  switch (n) {
    case 16: groups = Geo<16>::GROUPS; zg = Geo<16>::ZG; break;
    case 32: groups = Geo<32>::GROUPS; zg = Geo<32>::ZG; break;
    case 64: groups = Geo<64>::GROUPS; zg = Geo<64>::ZG; break;
    case 128: groups = Geo<128>::GROUPS; zg = Geo<128>::ZG; break;
    default: return 0;
  }
  // grid window [rows][N], transposed / row-major spectra [N][rs], exchange,
  // twiddles (8-byte elements: float2, or a BF16 pair of complex values),
  // then E' [Na] (two frames' worth in the BF16 form)
  static_assert(sizeof(fft::Cb2) == sizeof(float2), "Cb2 is an 8-byte element");
  const size_t elems = static_cast<size_t>(rows_alloc) * n + static_cast<size_t>(n) * rs +
                       static_cast<size_t>(groups) * zg + n + static_cast<size_t>(n_ant) * (bf16 ? 2 : 1);
  return elems * sizeof(float2);
}

}  // namespace epic
