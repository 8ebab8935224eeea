// Plain (unfused) FP32 EPIC imaging path for any grid side N = 32..512.
//
// Each step is its own kernel and hands its result to the next through HBM,
// one batch of frames at a time (frame f = t_local * C + c):
//   rows_gather    per frame: gain correction (Eq. 8) of every antenna into
//                  shared memory, then gridding (Eq. 9) as a gather straight
//                  into the FFT lanes of every occupied grid row (host-planned
//                  tap lists, no grid in device memory, no atomics) and the
//                  N-point row FFT, written transposed into Hs[f][kx][row];
//   cols_fft       N-point FFT of every column (Eq. 10), |E|^2 summed over
//                  the batch's frames in registers and added to the image;
//                  the owner of the calibrator pixel stores it per frame;
//   correlate      EPICal K_a += E_a conj(P), P_a += |E_a|^2 (Eqs. 12, 15).
// The grid window holds the occupied rows of each channel (as in the fused
// kernel); the centring signs and 1/Na are folded into the weights.
#include "epic_fft.cuh"
#include "epic_internal.h"

namespace epic {
namespace {

using fft::cmul;
using fft::kFull;

template <int N> struct UCfg;
template <> struct UCfg<32>  { static constexpr int N1 = 4,  N2 = 8; };
template <> struct UCfg<64>  { static constexpr int N1 = 8,  N2 = 8; };
template <> struct UCfg<128> { static constexpr int N1 = 8,  N2 = 16; };
template <> struct UCfg<256> { static constexpr int N1 = 16, N2 = 16; };
template <> struct UCfg<512> { static constexpr int N1 = 16, N2 = 32; };

constexpr int kUBT = 256;   // threads per CTA of the FFT kernels

__device__ __forceinline__ float2 load_volt_u(const void* volt, int fmt, size_t idx) {
  if (fmt == 0) {
    const unsigned b = __ldg(static_cast<const unsigned char*>(volt) + idx);
    const int re = static_cast<int>(b << 24) >> 28;
    const int im = static_cast<int>(b << 28) >> 28;
    return make_float2(static_cast<float>(re), static_cast<float>(im));
  }
  return __ldg(static_cast<const float2*>(volt) + idx);
}

// ---- gridding + row FFTs: one CTA per frame at a time ----
// Lane (window row, n1) of a row FFT sums w * E'_a over its tap list for
// each column group j (absolute column n1 + N1 j); lists and group lengths
// (one byte per j) come from the plan.  Whole warps step through the rows
// together; rows past the window transform zeros and store nothing.
template <int N>
__global__ void __launch_bounds__(kUBT, (N <= 128 ? 4 : 2)) rows_gather_kernel(const UnfusedArgs A, long long t0, int nt) {
  constexpr int N1 = UCfg<N>::N1, N2 = UCfg<N>::N2, H = N2 / N1;
  constexpr int GROUPS = kUBT / N1, GPW = 32 / N1;
  constexpr int CW = (N2 + 15) / 16;               // uint4 words of group lengths per lane
  using X = fft::Xchg<N1, N2>;
  __shared__ float2 tw[N];
  __shared__ float2 zbuf[GROUPS * X::ZG];
  extern __shared__ float2 Es[];                   // [Na] E / g of the current frame
  for (int i = threadIdx.x; i < N; i += kUBT) tw[i] = A.twid[i];
  const int g = threadIdx.x / N1, n1 = threadIdx.x % N1;
  float2* z = zbuf + g * X::ZG;
  const int C = A.n_chan, Na = A.n_ant;
  const long long frames = static_cast<long long>(nt) * C;
  // item = c * nt + tl: a CTA's consecutive items stay in one channel (its
  // tap lists stay in L1)
  for (long long it = blockIdx.x; it < frames; it += gridDim.x) {
    const int c = static_cast<int>(it / nt);
    const int tl = static_cast<int>(it - static_cast<long long>(c) * nt);
    const size_t f = static_cast<size_t>(tl) * C + c;
    const float vs = A.vscale ? __ldg(A.vscale + c) : 1.0f;
    __syncthreads();                               // previous frame's gathers are done
    for (int a = threadIdx.x; a < Na; a += kUBT) {
      const size_t vidx = (static_cast<size_t>(t0 + tl) * C + c) * Na + a;
      const float2 e = load_volt_u(A.volt, A.input_fmt, vidx);
      Es[a] = cmul(make_float2(e.x * vs, e.y * vs), __ldg(A.wgain + static_cast<size_t>(c) * Na + a));
    }
    __syncthreads();
    const int R = __ldg(A.win + c).y;
    const int* gofs = A.gofs + static_cast<size_t>(c) * A.rows_alloc * N1;
    const uint4* gcnt = A.gcnt + static_cast<size_t>(c) * A.rows_alloc * N1 * CW;
    const uint2* gent = A.gent + __ldg(A.gbase + c);
    for (int rb = g - g % GPW; rb < R; rb += GROUPS) {
      const int row = rb + g % GPW;
      const bool live = row < R;
      float2 v[N2];
#pragma unroll
      for (int j = 0; j < N2; ++j) v[j] = make_float2(0.f, 0.f);
      if (live) {
        const int li = row * N1 + n1;
        int e = __ldg(gofs + li);
        unsigned cv[4 * CW];
#pragma unroll
        for (int w = 0; w < CW; ++w) {
          const uint4 q = __ldg(gcnt + static_cast<size_t>(li) * CW + w);
          cv[4 * w] = q.x;
          cv[4 * w + 1] = q.y;
          cv[4 * w + 2] = q.z;
          cv[4 * w + 3] = q.w;
        }
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
      fft::fft_lanes<N1, N2>(v, n1, z, tw, kFull);
      if (live) {
        float2* dst = A.spec + f * N * A.rs + row;
#pragma unroll
        for (int h = 0; h < H; ++h)
#pragma unroll
          for (int k1 = 0; k1 < N1; ++k1) dst[static_cast<size_t>(n1 + N1 * h + N2 * k1) * A.rs] = v[h * N1 + k1];
      }
    }
  }
}

// ---- column FFTs + |E|^2: unit = (channel, block of GROUPS columns, time segment) ----
template <int N>
__global__ void __launch_bounds__(kUBT, (N <= 128 ? 3 : 2)) cols_fft_kernel(const UnfusedArgs A, int nt, int segs) {
  constexpr int N1 = UCfg<N>::N1, N2 = UCfg<N>::N2, H = N2 / N1;
  constexpr int GROUPS = kUBT / N1;
  constexpr int CBLK = (N + GROUPS - 1) / GROUPS;   // column blocks per channel
  using X = fft::Xchg<N1, N2>;
  __shared__ float2 tw[N];
  __shared__ float2 zbuf[GROUPS * X::ZG];
  for (int i = threadIdx.x; i < N; i += kUBT) tw[i] = A.twid[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int g = threadIdx.x / N1, n1 = threadIdx.x % N1;
  const unsigned gmask = fft::group_mask<N1>(lane);
  float2* z = zbuf + g * X::ZG;
  const int C = A.n_chan;
  const int units = C * CBLK * segs;
  for (int u = blockIdx.x; u < units; u += gridDim.x) {
    const int s = u % segs;
    const int cb = (u / segs) % CBLK;
    const int c = u / (segs * CBLK);
    const int kx = cb * GROUPS + g;
    const int tb = nt * s / segs, te = nt * (s + 1) / segs;
    const int2 wn = __ldg(A.win + c);
    const int y0 = wn.x, R = wn.y;
    const bool col_ok = kx < N;
    float acc[N2];
#pragma unroll
    for (int q = 0; q < N2; ++q) acc[q] = 0.f;
    const bool pix_group = A.do_cal && kx == A.k0x;
    const int pq = A.k0y / N1;
    const int pslot = (pq % H) * N1 + pq / H;
    for (int tl = tb; tl < te; ++tl) {
      if (!col_ok) continue;
      const size_t f = static_cast<size_t>(tl) * C + c;
      const float2* src = A.spec + (f * N + kx) * A.rs;
      float2 v[N2];
#pragma unroll
      for (int j = 0; j < N2; ++j) {
        const int jw = n1 + N1 * j - y0;
        v[j] = (jw >= 0 && jw < R) ? src[jw] : make_float2(0.f, 0.f);
      }
      fft::fft_lanes<N1, N2>(v, n1, z, tw, gmask);
#pragma unroll
      for (int q = 0; q < N2; ++q) acc[q] += v[q].x * v[q].x + v[q].y * v[q].y;
      if (pix_group && n1 == A.k0y % N1) {
#pragma unroll
        for (int q = 0; q < N2; ++q)
          if (q == pslot) A.pix[f] = make_float2(v[q].x * A.pix_sign, v[q].y * A.pix_sign);
      }
    }
    if (!col_ok) continue;
    double* img = A.image + static_cast<size_t>(c) * N * N;
#pragma unroll
    for (int h = 0; h < H; ++h)
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) {
        const int ky = n1 + N1 * h + N2 * k1;
        const double v = static_cast<double>(acc[h * N1 + k1]) * A.img_scale;
        if (segs == 1) img[ky * N + kx] += v;
        else atomicAdd(img + ky * N + kx, v);
      }
  }
}

// ---- EPICal correlation: one thread per (channel, antenna, time segment) ----
__global__ void correlate_kernel(const UnfusedArgs A, long long t0, int nt) {
  const int Na = A.n_ant, C = A.n_chan;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C * Na) return;
  const int c = i / Na, a = i % Na;
  if (__ldg(A.cell0 + i) < 0) return;
  const float vs = A.vscale ? __ldg(A.vscale + c) : 1.0f;
  const int tb = nt * blockIdx.y / gridDim.y, te = nt * (blockIdx.y + 1) / gridDim.y;
  float kr = 0.f, ki = 0.f, pp = 0.f;
  for (int tl = tb; tl < te; ++tl) {
    const size_t f = static_cast<size_t>(tl) * C + c;
    const float2 p = A.pix[f];
    const float2 e0 = load_volt_u(A.volt, A.input_fmt, (static_cast<size_t>(t0 + tl) * C + c) * Na + a);
    const float2 e = make_float2(e0.x * vs, e0.y * vs);
    kr += e.x * p.x + e.y * p.y;
    ki += e.y * p.x - e.x * p.y;
    pp += e.x * e.x + e.y * e.y;
  }
  if (gridDim.y == 1) {
    A.kacc[i].x += kr;
    A.kacc[i].y += ki;
    A.pacc[i] += pp;
  } else {
    atomicAdd(&A.kacc[i].x, static_cast<double>(kr));
    atomicAdd(&A.kacc[i].y, static_cast<double>(ki));
    atomicAdd(A.pacc + i, static_cast<double>(pp));
  }
}

// Time segments for the correlation: enough blocks to fill the GPU, at
// least 16 time samples each.
dim3 correlate_grid(int n_chan, int n_ant, int nt, int sms) {
  const int bx = (n_chan * n_ant + 255) / 256;
  int sy = 1;
  while (bx * sy < 4 * sms && nt / (2 * sy) >= 16) sy *= 2;
  return dim3(static_cast<unsigned>(bx), static_cast<unsigned>(sy));
}

template <int N>
cudaError_t launch_unfused_n(const UnfusedArgs& a, long long t0, int nt, int sms, cudaStream_t s) {
  constexpr int GROUPS = kUBT / UCfg<N>::N1;
  const size_t es_bytes = static_cast<size_t>(a.n_ant) * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(rows_gather_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(es_bytes));
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rows_gather_kernel<N>, kUBT, es_bytes);
  if (e != cudaSuccess) return e;
  const long long frames = static_cast<long long>(nt) * a.n_chan;
  long long rb = static_cast<long long>(per_sm > 0 ? per_sm : 1) * sms;
  if (rb > frames) rb = frames;
  rows_gather_kernel<N><<<static_cast<unsigned>(rb), kUBT, es_bytes, s>>>(a, t0, nt);
  constexpr int CBLK = (N + GROUPS - 1) / GROUPS;
  const int base_units = a.n_chan * CBLK;
  int segs = 1;
  while (base_units * segs < a.cols_target * sms && segs * 8 <= nt) segs *= 2;
  const int units = base_units * segs;
  const int cb = units < sms * 4 ? units : sms * 4;
  cols_fft_kernel<N><<<cb, kUBT, 0, s>>>(a, nt, segs);
  if (a.do_cal) correlate_kernel<<<correlate_grid(a.n_chan, a.n_ant, nt, sms), 256, 0, s>>>(a, t0, nt);
  return cudaGetLastError();
}

}  // namespace

bool unfused_supported(int n) { return n == 32 || n == 64 || n == 128 || n == 256 || n == 512; }

int unfused_fft_lanes(int n) {
  switch (n) {
    case 32: return UCfg<32>::N1;
    case 64: return UCfg<64>::N1;
    case 128: return UCfg<128>::N1;
    case 256: return UCfg<256>::N1;
    case 512: return UCfg<512>::N1;
    default: return 0;
  }
}

cudaError_t launch_correlate(const UnfusedArgs& a, long long t0, int nt, cudaStream_t s) {
  correlate_kernel<<<correlate_grid(a.n_chan, a.n_ant, nt, 152), 256, 0, s>>>(a, t0, nt);
  return cudaGetLastError();
}

cudaError_t launch_unfused_batch(const UnfusedArgs& a, long long t0, int nt, int sms, cudaStream_t s) {
  switch (a.grid_n) {
    case 32: return launch_unfused_n<32>(a, t0, nt, sms, s);
    case 64: return launch_unfused_n<64>(a, t0, nt, sms, s);
    case 128: return launch_unfused_n<128>(a, t0, nt, sms, s);
    case 256: return launch_unfused_n<256>(a, t0, nt, sms, s);
    case 512: return launch_unfused_n<512>(a, t0, nt, sms, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace epic
