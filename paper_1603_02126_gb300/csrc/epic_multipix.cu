// Multiple-pixel and direction-dependent EPICal (Sec. 6, "Multiple pixel
// correlations"): every raw antenna signal is correlated with the E-field at
// P calibration pixels instead of one, O(Na P) per sample.
//
// The fused imaging kernel stores the P pixel values of every frame
// (E'(s_p, t), formed with the current gains) to a tap buffer; the
// correlation here is then, per channel, the product of the [Na x T] voltage
// block with the conjugate [T x P] tap block,
//   K_{a,p} += sum_t E_a(t) conj(E'(s_p, t))      (Eq. 12 for every pixel),
// with the uncalibrated 4-bit or complex64 voltages.  The update combines
// the pixels per antenna (Eq. 15 per pixel, C_{a,p} = g_a D_{p,a} at the
// noise-free fixed point, least squares over p, Eq. 17 damping) and also
// advances one independent solution per direction (Eqs. 16-17 per pixel).
#include <cuda_runtime.h>

#include "epic_internal.h"

namespace epic {
namespace {

constexpr int kCorrThreads = 256;
constexpr int kPixBlock = 16;    // pixels held in registers per pass
constexpr int kTimeTile = 32;    // time samples of taps staged per barrier pair

__device__ __forceinline__ float2 load_raw(const void* volt, int fmt, size_t idx) {
  if (fmt == 0) {
    const unsigned b = __ldg(static_cast<const unsigned char*>(volt) + idx);
    const int re = static_cast<int>(b << 24) >> 28;
    const int im = static_cast<int>(b << 28) >> 28;
    return make_float2(static_cast<float>(re), static_cast<float>(im));
  }
  return __ldg(static_cast<const float2*>(volt) + idx);
}

// One CTA per (channel, time segment); threads own antennas, registers hold
// kPixBlock complex sums per antenna; taps of kTimeTile samples are staged
// in shared memory and read as broadcasts.  FP32 over the segment, FP64
// atomics across segments.
__global__ void __launch_bounds__(kCorrThreads) correlate_multi_kernel(const MultiCorrArgs A) {
  __shared__ float2 tap[kTimeTile][kPixBlock];
  const int c = blockIdx.x / A.segs;
  const int s = blockIdx.x - c * A.segs;
  const long long tb = A.n_time * s / A.segs, te = A.n_time * (s + 1) / A.segs;
  const int C = A.n_chan, Na = A.n_ant, P = A.npix;
  const float vs = A.vscale ? __ldg(A.vscale + c) : 1.0f;
  for (int ab = 0; ab < Na; ab += kCorrThreads) {
    const int a = ab + threadIdx.x;
    const bool live = a < Na && __ldg(A.cell0 + static_cast<size_t>(c) * Na + a) >= 0;
    for (int pb = 0; pb < P; pb += kPixBlock) {
      const int np = P - pb < kPixBlock ? P - pb : kPixBlock;
      float2 acc[kPixBlock];
#pragma unroll
      for (int j = 0; j < kPixBlock; ++j) acc[j] = make_float2(0.f, 0.f);
      for (long long t0 = tb; t0 < te; t0 += kTimeTile) {
        const int nt = static_cast<int>(te - t0 < kTimeTile ? te - t0 : kTimeTile);
        __syncthreads();
        for (int i = threadIdx.x; i < kTimeTile * kPixBlock; i += kCorrThreads) {
          const int tt = i / kPixBlock, j = i % kPixBlock;
          tap[tt][j] = (tt < nt && j < np)
                           ? __ldg(A.ptap + (static_cast<size_t>(t0 + tt) * C + c) * P + pb + j)
                           : make_float2(0.f, 0.f);
        }
        __syncthreads();
        if (live) {
#pragma unroll 4
          for (int tt = 0; tt < nt; ++tt) {
            const float2 e0 = load_raw(A.volt, A.input_fmt, (static_cast<size_t>(t0 + tt) * C + c) * Na + a);
            const float2 e = make_float2(e0.x * vs, e0.y * vs);
#pragma unroll
            for (int j = 0; j < kPixBlock; ++j) {
              const float2 q = tap[tt][j];
              acc[j].x = fmaf(e.x, q.x, fmaf(e.y, q.y, acc[j].x));   // Re(e conj(q))
              acc[j].y = fmaf(e.y, q.x, fmaf(-e.x, q.y, acc[j].y));  // Im(e conj(q))
            }
          }
        }
      }
      if (live) {
        double2* k = A.kmp + (static_cast<size_t>(c) * Na + a) * P + pb;
#pragma unroll
        for (int j = 0; j < kPixBlock; ++j)
          if (j < np) {
            atomicAdd(&k[j].x, static_cast<double>(acc[j].x));
            atomicAdd(&k[j].y, static_cast<double>(acc[j].y));
          }
      }
    }
  }
}

// FP64, one thread per (channel, antenna): Eq. 15 per pixel, the joint
// least-squares solution for the imaging gains and the per-direction
// solutions, then clears the accumulators.
__global__ void update_multi_kernel(const MultiUpdateArgs A) {
  const int n = A.n_chan * A.n_ant;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = i / A.n_ant, a = i - c * A.n_ant;
  const int P = A.npix;
  const bool flagged = A.flags[a] != 0;
  const double pb = A.pacc[i] * A.inv_frames;
  const double2 g = A.gain[i];
  const double gg = g.x * g.x + g.y * g.y;
  // conj(A) P / conj(g) = conj(A) P g / |g|^2
  const double one_m = 1.0 - A.gamma;
  double nr = 0.0, ni = 0.0, den = 0.0;
  for (int p = 0; p < P; ++p) {
    const size_t kp = static_cast<size_t>(i) * P + p;
    const size_t ap = (static_cast<size_t>(c) * P + p) * A.n_ant + a;
    const double2 k = A.kmp[kp];
    const double2 av = A.ap[ap];
    const double2 d = A.dp[ap];
    const double ar = av.x * pb, ai = -av.y * pb;            // conj(A) P
    const double qr = (ar * g.x - ai * g.y) / gg;            // (conj(A) P) g / |g|^2
    const double qi = (ar * g.y + ai * g.x) / gg;
    const double cr = k.x * A.inv_frames - qr, ci = k.y * A.inv_frames - qi;   // C_{a,p}
    nr += d.x * cr + d.y * ci;                               // conj(D) C
    ni += d.x * ci - d.y * cr;
    const double dd = d.x * d.x + d.y * d.y;
    den += dd;
    // per-direction solution (Eqs. 16-17 for this pixel)
    const double2 gd = A.gdir[kp];
    const double sr = (cr * d.x + ci * d.y) / dd, si = (ci * d.x - cr * d.y) / dd;
    const double xr = one_m * sr + A.gamma * gd.x, xi = one_m * si + A.gamma * gd.y;
    const bool hd = flagged || !(dd > A.dmin * A.dmin) || !isfinite(xr) || !isfinite(xi) ||
                    (xr == 0.0 && xi == 0.0);
    if (!hd) A.gdir[kp] = make_double2(xr, xi);
    A.kmp[kp] = make_double2(0.0, 0.0);
  }
  const double nxr = one_m * nr / den + A.gamma * g.x;
  const double nxi = one_m * ni / den + A.gamma * g.y;
  const bool held = flagged || !(den > A.dmin * A.dmin) || !isfinite(nxr) || !isfinite(nxi) ||
                    (nxr == 0.0 && nxi == 0.0);
  double2 out = g;
  if (!held) {
    out = make_double2(nxr, nxi);
    A.gain[i] = out;
    // w = p / g (p: phasing of the plan's phase centre, 1 if none)
    const double m2 = nxr * nxr + nxi * nxi;
    double wr = nxr / m2, wi = -nxi / m2;
    if (A.phase) {
      const double2 q = A.phase[i];
      const double xr = wr * q.x - wi * q.y, xi = wr * q.y + wi * q.x;
      wr = xr;
      wi = xi;
    }
    A.wgain[i] = make_float2(static_cast<float>(wr), static_cast<float>(wi));
  }
  if (A.status) A.status[i] = held ? 1 : 0;
  if (held && !flagged) atomicAdd(A.held_count, 1);
  if (A.gout) A.gout[i] = out;
  A.kacc[i] = make_double2(0.0, 0.0);
  A.pacc[i] = 0.0;
}

}  // namespace

cudaError_t launch_correlate_multi(const MultiCorrArgs& a, cudaStream_t s) {
  if (a.npix < 1 || a.n_time < 1) return cudaSuccess;
  correlate_multi_kernel<<<a.n_chan * a.segs, kCorrThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_update_multi(const MultiUpdateArgs& a, cudaStream_t s) {
  const int n = a.n_chan * a.n_ant;
  update_multi_kernel<<<(n + 255) / 256, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace epic
