// Visibility-based comparison path of the noise-trend study (Sec. 4): an
// X-engine forming every antenna pair's visibility from the same voltage
// stream EPICal uses, and the Eq. 21 gain solve on those visibilities.
//
//   xengine      V[c][a][b] += (s_c^2 / T) sum_t E_a(t) conj(E_b(t)) per channel, a
//                [Na x T] by [T x Na] complex product, tiled 64 x 64 per CTA
//                (4 x 4 outputs per thread, FP32 in registers, upper-triangle
//                tiles only, the lower triangle written as the conjugate).
//                For 4-bit input every product and partial sum is an integer
//                below 2^24, so the FP32 sums are exact.
//   model_vis    V^M[c][a][b] = sum_s S_s e_a(s) conj(e_b(s)), e_a(s) =
//                e^{-2 pi i u_a . s}, FP64 from host phasors, kept in FP32.
//   stefcal      Eq. 21 by alternating least squares with every other iterate
//                averaged (StEFCal): one CTA per channel, one warp per antenna
//                row at a time, FP32 products with FP64 reductions and
//                update, iterated in the kernel until
//                max_a |g_new - g| <= tol max_a |g_new| or max_iter.
#include <cuda_runtime.h>

#include <algorithm>

#include "epic_internal.h"

namespace epic {
namespace {

constexpr int kXT = 64;          // antennas per tile side
constexpr int kXK = 32;          // time samples per staged chunk
constexpr int kXThreads = 256;   // 16 x 16 threads, 4 x 4 outputs each
constexpr int kXSeg = 32768;     // samples per FP32 segment (exact for 4-bit input)

__device__ __forceinline__ float2 xload(const void* volt, int fmt, size_t idx) {
  if (fmt == 0) {
    const unsigned b = __ldg(static_cast<const unsigned char*>(volt) + idx);
    const int re = static_cast<int>(b << 24) >> 28;
    const int im = static_cast<int>(b << 28) >> 28;
    return make_float2(static_cast<float>(re), static_cast<float>(im));
  }
  return __ldg(static_cast<const float2*>(volt) + idx);
}

// blockIdx.x: channel * tile pairs + pair (upper triangle, row-major);
// blockIdx.y: time segment.
__global__ void __launch_bounds__(kXThreads) xengine_kernel(const XengineArgs A) {
  __shared__ __align__(16) float2 ea[kXK][kXT];
  __shared__ __align__(16) float2 eb[kXK][kXT];
  const int nb = (A.n_ant + kXT - 1) / kXT;
  const int pairs = nb * (nb + 1) / 2;
  const int c = blockIdx.x / pairs;
  int pr = blockIdx.x - c * pairs;
  int bi = 0;
  while (pr >= nb - bi) {                // (bi, bj) with bi <= bj
    pr -= nb - bi;
    ++bi;
  }
  const int bj = bi + pr;
  const int C = A.n_chan, Na = A.n_ant;
  const long long tb = static_cast<long long>(blockIdx.y) * kXSeg;
  const long long te = tb + kXSeg < A.n_time ? tb + kXSeg : A.n_time;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  for (long long t0 = tb; t0 < te; t0 += kXK) {
    __syncthreads();
    for (int i = threadIdx.x; i < kXK * kXT; i += kXThreads) {
      const int tt = i / kXT, k = i % kXT;
      const long long t = t0 + tt;
      const int a = bi * kXT + k, b = bj * kXT + k;
      const size_t row = (static_cast<size_t>(t) * C + c) * Na;
      ea[tt][k] = (t < te && a < Na) ? xload(A.volt, A.input_fmt, row + a) : make_float2(0.f, 0.f);
      eb[tt][k] = (t < te && b < Na) ? xload(A.volt, A.input_fmt, row + b) : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll 4
    for (int tt = 0; tt < kXK; ++tt) {
      float2 x[4], y[4];
      const float4 x01 = *reinterpret_cast<const float4*>(&ea[tt][ty * 4]);
      const float4 x23 = *reinterpret_cast<const float4*>(&ea[tt][ty * 4 + 2]);
      const float4 y01 = *reinterpret_cast<const float4*>(&eb[tt][tx * 4]);
      const float4 y23 = *reinterpret_cast<const float4*>(&eb[tt][tx * 4 + 2]);
      x[0] = make_float2(x01.x, x01.y); x[1] = make_float2(x01.z, x01.w);
      x[2] = make_float2(x23.x, x23.y); x[3] = make_float2(x23.z, x23.w);
      y[0] = make_float2(y01.x, y01.y); y[1] = make_float2(y01.z, y01.w);
      y[2] = make_float2(y23.x, y23.y); y[3] = make_float2(y23.z, y23.w);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          // E_a conj(E_b)
          acc[i][j].x = fmaf(x[i].x, y[j].x, fmaf(x[i].y, y[j].y, acc[i][j].x));
          acc[i][j].y = fmaf(x[i].y, y[j].x, fmaf(-x[i].x, y[j].y, acc[i][j].y));
        }
    }
  }
  const float vs = A.vscale ? __ldg(A.vscale + c) : 1.0f;
  const double scale = static_cast<double>(vs) * static_cast<double>(vs) * A.scale;
  double2* V = A.vis + static_cast<size_t>(c) * Na * Na;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int a = bi * kXT + ty * 4 + i, b = bj * kXT + tx * 4 + j;
      if (a >= Na || b >= Na) continue;
      if (bi == bj && b < a) continue;             // diagonal tile: upper half and the diagonal
      const double re = static_cast<double>(acc[i][j].x) * scale;
      const double im = static_cast<double>(acc[i][j].y) * scale;
      atomicAdd(&V[static_cast<size_t>(a) * Na + b].x, re);
      atomicAdd(&V[static_cast<size_t>(a) * Na + b].y, im);
      if (a != b) {
        atomicAdd(&V[static_cast<size_t>(b) * Na + a].x, re);
        atomicAdd(&V[static_cast<size_t>(b) * Na + a].y, -im);
      }
    }
}

// V^M[c][a][b] = sum_s S_s ph[c][s][a] conj(ph[c][s][b]) in FP64, stored
// rounded to FP32 for the solver; one thread per pair.
__global__ void model_vis_kernel(int n_chan, int n_ant, int n_src, const double2* __restrict__ ph,
                                 const double* __restrict__ flux, float2* __restrict__ vm) {
  const long long n = static_cast<long long>(n_chan) * n_ant * n_ant;
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const int b = static_cast<int>(i % n_ant);
  const int a = static_cast<int>((i / n_ant) % n_ant);
  const int c = static_cast<int>(i / (static_cast<long long>(n_ant) * n_ant));
  double re = 0.0, im = 0.0;
  for (int s = 0; s < n_src; ++s) {
    const double2 pa = ph[(static_cast<size_t>(c) * n_src + s) * n_ant + a];
    const double2 pb = ph[(static_cast<size_t>(c) * n_src + s) * n_ant + b];
    const double S = flux[s];
    re += S * (pa.x * pb.x + pa.y * pb.y);
    im += S * (pa.y * pb.x - pa.x * pb.y);
  }
  vm[i] = make_float2(static_cast<float>(re), static_cast<float>(im));
}

__global__ void to_f32_kernel(long long n, const double2* __restrict__ in, float2* __restrict__ out) {
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n; i += stride) {
    const double2 v = in[i];
    out[i] = make_float2(static_cast<float>(v.x), static_cast<float>(v.y));
  }
}

constexpr int kSThreads = 1024;
constexpr double kStefcalMinTol = 1e-6;   // smallest stopping tolerance with FP32 pair products

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One CTA per channel.  The per-pair products run in FP32 (V and V^M
// rounded to FP32, this GPU's FP64 rate being a small fraction of its FP32
// rate); each lane's partial sums go to FP64 for the warp reduction, the
// division, the averaging and the convergence test.  Shared memory: g (FP64)
// and gn [Na], g as FP32 [Na].
__global__ void __launch_bounds__(kSThreads) stefcal_kernel(const StefcalArgs A) {
  extern __shared__ __align__(16) double2 sg[];
  double2* g = sg;
  double2* gn = sg + A.n_ant;
  float2* gf = reinterpret_cast<float2*>(sg + 2 * A.n_ant);
  __shared__ double red_d[kSThreads / 32], red_m[kSThreads / 32];
  __shared__ int done;
  const int c = blockIdx.x, Na = A.n_ant;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = kSThreads / 32;
  const float2* V = A.vis32 + static_cast<size_t>(c) * Na * Na;
  const float2* VM = A.vm + static_cast<size_t>(c) * Na * Na;
  const double2* uv = A.uv + static_cast<size_t>(c) * Na;
  const double mb2 = A.min_baseline * A.min_baseline;
  double2* gio = A.gains + static_cast<size_t>(c) * Na;
  for (int a = threadIdx.x; a < Na; a += kSThreads) {
    g[a] = gio[a];
    gf[a] = make_float2(static_cast<float>(g[a].x), static_cast<float>(g[a].y));
  }
  if (threadIdx.x == 0) done = 0;
  __syncthreads();
  int it = 0;
  for (; it < A.max_iter; ++it) {
    for (int a = warp; a < Na; a += nw) {
      float nr = 0.f, ni = 0.f, den = 0.f;
      if (!A.flags[a]) {
        const double2 ua = uv[a];
        for (int b = lane; b < Na; b += 32) {
          if (b == a || A.flags[b]) continue;
          if (mb2 > 0.0) {
            const double2 ub = uv[b];
            const double dx = ua.x - ub.x, dy = ua.y - ub.y;
            if (dx * dx + dy * dy < mb2) continue;
          }
          const float2 gb = gf[b];
          const float2 m = VM[static_cast<size_t>(a) * Na + b];
          const float2 v = V[static_cast<size_t>(a) * Na + b];
          // z = g_b conj(VM_ab)
          const float zr = fmaf(gb.x, m.x, gb.y * m.y), zi = fmaf(gb.y, m.x, -gb.x * m.y);
          nr = fmaf(v.x, zr, fmaf(-v.y, zi, nr));
          ni = fmaf(v.x, zi, fmaf(v.y, zr, ni));
          den = fmaf(zr, zr, fmaf(zi, zi, den));
        }
      }
      const double snr = warp_sum(static_cast<double>(nr));
      const double sni = warp_sum(static_cast<double>(ni));
      const double sden = warp_sum(static_cast<double>(den));
      if (lane == 0) gn[a] = sden > 0.0 ? make_double2(snr / sden, sni / sden) : g[a];
    }
    __syncthreads();
    double dmax = 0.0, gmax = 0.0;
    for (int a = threadIdx.x; a < Na; a += kSThreads) {
      double2 x = gn[a];
      const double2 o = g[a];
      if (it & 1) x = make_double2(0.5 * (x.x + o.x), 0.5 * (x.y + o.y));
      gn[a] = x;
      dmax = fmax(dmax, hypot(x.x - o.x, x.y - o.y));
      gmax = fmax(gmax, hypot(x.x, x.y));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
      gmax = fmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
    }
    if (lane == 0) {
      red_d[warp] = dmax;
      red_m[warp] = gmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double d = 0.0, m = 0.0;
      for (int w = 0; w < nw; ++w) {
        d = fmax(d, red_d[w]);
        m = fmax(m, red_m[w]);
      }
      // FP32 pair products: changes below ~1e-6 are rounding, not progress
      done = (d <= fmax(A.tol, kStefcalMinTol) * m) ? 1 : 0;
    }
    for (int a = threadIdx.x; a < Na; a += kSThreads) {
      g[a] = gn[a];
      gf[a] = make_float2(static_cast<float>(gn[a].x), static_cast<float>(gn[a].y));
    }
    __syncthreads();
    if (done) {
      ++it;
      break;
    }
  }
  for (int a = threadIdx.x; a < Na; a += kSThreads) gio[a] = g[a];
  if (threadIdx.x == 0 && A.iters) A.iters[c] = it;
}

}  // namespace

cudaError_t launch_xengine(const XengineArgs& a, cudaStream_t s) {
  const int nb = (a.n_ant + kXT - 1) / kXT;
  const int pairs = nb * (nb + 1) / 2;
  const long long segs = (a.n_time + kXSeg - 1) / kXSeg;
  dim3 grid(static_cast<unsigned>(a.n_chan * pairs), static_cast<unsigned>(segs));
  xengine_kernel<<<grid, kXThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_model_vis(int n_chan, int n_ant, int n_src, const double2* ph, const double* flux,
                             float2* vm, cudaStream_t s) {
  const long long n = static_cast<long long>(n_chan) * n_ant * n_ant;
  model_vis_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(n_chan, n_ant, n_src, ph, flux, vm);
  return cudaGetLastError();
}

cudaError_t launch_stefcal(const StefcalArgs& a, const double2* vis64, cudaStream_t s) {
  const long long nv = static_cast<long long>(a.n_chan) * a.n_ant * a.n_ant;
  to_f32_kernel<<<static_cast<unsigned>(std::min<long long>((nv + 255) / 256, 152 * 16)), 256, 0, s>>>(
      nv, vis64, a.vis32);
  const size_t smem = static_cast<size_t>(a.n_ant) * (2 * sizeof(double2) + sizeof(float2));
  cudaError_t e = cudaFuncSetAttribute(stefcal_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  stefcal_kernel<<<a.n_chan, kSThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace epic
