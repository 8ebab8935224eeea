// Device FFT primitives shared by the imaging kernels (sm_103a).
//
// Dft<R>: in-register R-point DFT with the '+' sign of Eq. 10 (radix-2
// decimation in time, fully unrolled; twiddles are exact constants).
// fft_lanes<N1, N2>: one 1-D FFT of length N = N1 * N2 on N1 lanes of a warp,
// N2 points per lane: in-register N2-point DFT, twiddle e^{+2 pi i n1 k2 / N}
// from a float table, one exchange through shared memory, N2/N1 N1-point
// DFTs (four-step decomposition).
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace epic {
namespace fft {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// cos(2 pi m / 32) for m in [0, 8]: exact mathematical constants.
__host__ __device__ constexpr float cos32_q(int m) {
  return m == 0 ? 1.0f
       : m == 1 ? 0.98078528040323044913f
       : m == 2 ? 0.92387953251128675613f
       : m == 3 ? 0.83146961230254523708f
       : m == 4 ? 0.70710678118654752440f
       : m == 5 ? 0.55557023301960222474f
       : m == 6 ? 0.38268343236508977173f
       : m == 7 ? 0.19509032201612826785f
       : 0.0f;
}
// cos(2 pi m / 32) for any integer m, by symmetry.
__host__ __device__ constexpr float cos32(int m) {
  return ((m % 32) + 32) % 32 > 16 ? cos32(32 - (((m % 32) + 32) % 32))
       : ((m % 32) + 32) % 32 > 8 ? -cos32_q(16 - (((m % 32) + 32) % 32))
       : cos32_q(((m % 32) + 32) % 32);
}

// v * e^{+2 pi i K / R}, K a template argument: the quarter turns are
// swaps and sign flips, any other angle one complex multiply by exact
// constants.  (With k a run-time argument the compiler kept the case split
// as branches, even inside fully unrolled loops.)
template <int R, int K>
__device__ __forceinline__ float2 twiddle(float2 v) {
  constexpr int m = ((K * (32 / R)) % 32 + 32) % 32;
  if constexpr (m == 0) {
    return v;
  } else if constexpr (m == 8) {
    return make_float2(-v.y, v.x);
  } else if constexpr (m == 16) {
    return make_float2(-v.x, -v.y);
  } else if constexpr (m == 24) {
    return make_float2(v.y, -v.x);
  } else {
    constexpr float c = cos32(m), s = cos32(8 - m);
    return cmul(v, make_float2(c, s));
  }
}

// Radix-2 combination x[k] = e[k] + w^k o[k], x[k + R/2] = e[k] - w^k o[k]
// for k = 0 .. R/2 - 1, expanded at compile time.
template <int R, int K>
__device__ __forceinline__ void butterfly(float2 (&x)[R], const float2 (&e)[R / 2], const float2 (&o)[R / 2]) {
  const float2 t = twiddle<R, K>(o[K]);
  x[K] = cadd(e[K], t);
  x[K + R / 2] = csub(e[K], t);
}

template <int R, int... K>
__device__ __forceinline__ void combine(float2 (&x)[R], const float2 (&e)[R / 2], const float2 (&o)[R / 2],
                                        std::integer_sequence<int, K...>) {
  (butterfly<R, K>(x, e, o), ...);
}

// In-register DFT with the '+' sign of Eq. 10, natural order in and out
// (radix-2 decimation in time, fully unrolled).
template <int R>
struct Dft {
  static __device__ __forceinline__ void run(float2 (&x)[R]) {
    float2 e[R / 2], o[R / 2];
#pragma unroll
    for (int i = 0; i < R / 2; ++i) {
      e[i] = x[2 * i];
      o[i] = x[2 * i + 1];
    }
    Dft<R / 2>::run(e);
    Dft<R / 2>::run(o);
    combine<R>(x, e, o, std::make_integer_sequence<int, R / 2>{});
  }
};
template <>
struct Dft<1> {
  static __device__ __forceinline__ void run(float2 (&)[1]) {}
};


// R-point DFT of an input whose entries x[j], j >= NZ, are zero: the
// butterflies and copies that would only involve those zeros are skipped
// (compile-time pruning of the decimation-in-time recursion).
template <int R, int NZ>
struct DftP {
  static __device__ __forceinline__ void run(float2 (&x)[R]) {
    if constexpr (NZ >= R) {
      Dft<R>::run(x);
    } else if constexpr (NZ <= 1) {
#pragma unroll
      for (int k = 1; k < R; ++k) x[k] = x[0];
    } else {
      float2 e[R / 2], o[R / 2];
#pragma unroll
      for (int i = 0; i < R / 2; ++i) {
        e[i] = x[2 * i];
        o[i] = x[2 * i + 1];
      }
      DftP<R / 2, (NZ + 1) / 2>::run(e);
      DftP<R / 2, NZ / 2>::run(o);
      combine<R>(x, e, o, std::make_integer_sequence<int, R / 2>{});
    }
  }
};

// Padded exchange geometry of fft_lanes<N1, N2>.
template <int N1, int N2>
struct Xchg {
  static constexpr int ZS = N1 + 1;                              // padded row
  static constexpr int ZG0 = N2 * ZS;
  static constexpr int ZG = ZG0 + ((8 - ZG0 % 16) + 16) % 16;    // group stride
  static constexpr int H = N2 / N1;
  static_assert(N2 % N1 == 0, "N2 must be a multiple of N1");
  static_assert(32 % N1 == 0, "FFT groups must tile a warp");
};

// 1-D FFT of length N = N1 * N2 on a group of N1 lanes.
// In:  v[j] = x[n1 + N1 j], j < N2.
// Out: v[h N1 + k1] = X[n1 + N1 h + N2 k1], X[k] = sum_n x[n] e^{+2 pi i n k / N}.
// z: this group's exchange area (Xchg::ZG float2), tw: e^{+2 pi i m / N}.
template <int N1, int N2>
__device__ __forceinline__ void fft_lanes(float2 (&v)[N2], int n1, float2* z, const float2* tw,
                                          unsigned gmask) {
  constexpr int ZS = Xchg<N1, N2>::ZS, H = Xchg<N1, N2>::H;
  Dft<N2>::run(v);
#pragma unroll
  for (int k2 = 1; k2 < N2; ++k2) v[k2] = cmul(v[k2], tw[n1 * k2]);
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) z[k2 * ZS + n1] = v[k2];
  __syncwarp(gmask);
#pragma unroll
  for (int h = 0; h < H; ++h) {
    float2 u[N1];
#pragma unroll
    for (int m = 0; m < N1; ++m) u[m] = z[(n1 + N1 * h) * ZS + m];
    Dft<N1>::run(u);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) v[h * N1 + k1] = u[k1];
  }
  __syncwarp(gmask);
}

// fft_lanes for inputs that are zero beyond index N1 * NZ: v[j] for j >= NZ
// must be zero on entry (they are not read by the first-stage DFT).  tw2 is
// the twiddle table ordered [k2][n1] (tw2[k2 * N1 + n1] = e^{+2 pi i n1 k2 / N}),
// so that the lanes of a group read consecutive entries.
template <int N1, int N2, int NZ>
__device__ __forceinline__ void fft_lanes_p(float2 (&v)[N2], int n1, float2* z, const float2* tw2,
                                            unsigned gmask) {
  constexpr int ZS = Xchg<N1, N2>::ZS, H = Xchg<N1, N2>::H;
  DftP<N2, NZ>::run(v);
#pragma unroll
  for (int k2 = 1; k2 < N2; ++k2) v[k2] = cmul(v[k2], tw2[k2 * N1 + n1]);
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) z[k2 * ZS + n1] = v[k2];
  __syncwarp(gmask);
#pragma unroll
  for (int h = 0; h < H; ++h) {
    float2 u[N1];
#pragma unroll
    for (int m = 0; m < N1; ++m) u[m] = z[(n1 + N1 * h) * ZS + m];
    Dft<N1>::run(u);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) v[h * N1 + k1] = u[k1];
  }
  __syncwarp(gmask);
}

// Lane mask of the N1-lane group that contains `lane`.
template <int N1>
__device__ __forceinline__ unsigned group_mask(int lane) {
  return (N1 == 32) ? kFull : (((1u << N1) - 1u) << (lane & ~(N1 - 1)));
}

}  // namespace fft
}  // namespace epic
