// Device FFT primitives shared by the imaging kernels (sm_103a).
//
// Dft<R>: in-register R-point DFT with the '+' sign of Eq. 10 (radix-2
// decimation in time, fully unrolled; twiddles are exact constants).
// fft_lanes<N1, N2>: one 1-D FFT of length N = N1 * N2 on N1 lanes of a warp,
// N2 points per lane: in-register N2-point DFT, twiddle e^{+2 pi i n1 k2 / N}
// from a table, one exchange through shared memory, N2/N1 N1-point DFTs
// (four-step decomposition).
// The element type is float2 (one FP32 complex value) or Cb2 (the same
// complex sample of two independent transforms, real parts and imaginary
// parts each packed as a BF16 pair, so that every add and multiply acts on
// both transforms in one instruction).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <utility>

namespace epic {
namespace fft {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Two complex values (of two transforms): re = (re_0, re_1), im = (im_0, im_1).
struct Cb2 {
  __nv_bfloat162 re, im;
};

__device__ __forceinline__ Cb2 cadd(Cb2 a, Cb2 b) { return Cb2{__hadd2(a.re, b.re), __hadd2(a.im, b.im)}; }
__device__ __forceinline__ Cb2 csub(Cb2 a, Cb2 b) { return Cb2{__hsub2(a.re, b.re), __hsub2(a.im, b.im)}; }
// Element-wise complex product of the two pairs.
__device__ __forceinline__ Cb2 cmul(Cb2 a, Cb2 b) {
  return Cb2{__hfma2(a.re, b.re, __hneg2(__hmul2(a.im, b.im))), __hfma2(a.re, b.im, __hmul2(a.im, b.re))};
}

// Bits of the bfloat16 nearest to x (ties to even), at compile time, for
// the finite x of magnitude in [2^-126, 2^127) used here (and 0).
__host__ __device__ constexpr uint16_t bf16_bits(float x) {
  if (x == 0.0f) return 0;
  const uint16_t sign = x < 0.0f ? 0x8000u : 0u;
  float a = x < 0.0f ? -x : x;
  int e = 0;
  while (a >= 2.0f) {
    a *= 0.5f;
    ++e;
  }
  while (a < 1.0f) {
    a *= 2.0f;
    --e;
  }
  const float q = a * 128.0f;                   // in [128, 256): 7 fraction bits kept
  int qi = static_cast<int>(q);
  const float fr = q - static_cast<float>(qi);
  if (fr > 0.5f || (fr == 0.5f && (qi & 1))) ++qi;
  if (qi == 256) {
    qi = 128;
    ++e;
  }
  return static_cast<uint16_t>(sign | ((e + 127) << 7) | (qi - 128));
}

// (b, b) as a bfloat16 pair from its bits.
__device__ __forceinline__ __nv_bfloat162 bf2_splat(uint16_t b) {
  __nv_bfloat162_raw r;
  r.x = b;
  r.y = b;
  return __nv_bfloat162(r);
}

// Pack the FP32 values of two transforms into one Cb2.
__device__ __forceinline__ Cb2 cb2_pack(float2 v0, float2 v1) {
  return Cb2{__floats2bfloat162_rn(v0.x, v1.x), __floats2bfloat162_rn(v0.y, v1.y)};
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

// The same for a Cb2: quarter turns move the halves and flip signs, other
// angles multiply by the BF16-rounded constants (both transforms at once).
template <int R, int K>
__device__ __forceinline__ Cb2 twiddle(Cb2 v) {
  constexpr int m = ((K * (32 / R)) % 32 + 32) % 32;
  if constexpr (m == 0) {
    return v;
  } else if constexpr (m == 8) {
    return Cb2{__hneg2(v.im), v.re};
  } else if constexpr (m == 16) {
    return Cb2{__hneg2(v.re), __hneg2(v.im)};
  } else if constexpr (m == 24) {
    return Cb2{v.im, __hneg2(v.re)};
  } else {
    constexpr uint16_t c = bf16_bits(cos32(m)), s = bf16_bits(cos32(8 - m));
    return cmul(v, Cb2{bf2_splat(c), bf2_splat(s)});
  }
}

// Radix-2 combination x[k] = e[k] + w^k o[k], x[k + R/2] = e[k] - w^k o[k]
// for k = 0 .. R/2 - 1, expanded at compile time.
template <int R, int K, typename T>
__device__ __forceinline__ void butterfly(T (&x)[R], const T (&e)[R / 2], const T (&o)[R / 2]) {
  const T t = twiddle<R, K>(o[K]);
  x[K] = cadd(e[K], t);
  x[K + R / 2] = csub(e[K], t);
}

template <int R, typename T, int... K>
__device__ __forceinline__ void combine(T (&x)[R], const T (&e)[R / 2], const T (&o)[R / 2],
                                        std::integer_sequence<int, K...>) {
  (butterfly<R, K>(x, e, o), ...);
}

// In-register DFT with the '+' sign of Eq. 10, natural order in and out
// (radix-2 decimation in time, fully unrolled).
template <int R>
struct Dft {
  template <typename T>
  static __device__ __forceinline__ void run(T (&x)[R]) {
    T e[R / 2], o[R / 2];
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
  template <typename T>
  static __device__ __forceinline__ void run(T (&)[1]) {}
};


// R-point DFT of an input whose entries x[j], j >= NZ, are zero: the
// butterflies and copies that would only involve those zeros are skipped
// (compile-time pruning of the decimation-in-time recursion).
template <int R, int NZ>
struct DftP {
  template <typename T>
  static __device__ __forceinline__ void run(T (&x)[R]) {
    if constexpr (NZ >= R) {
      Dft<R>::run(x);
    } else if constexpr (NZ <= 1) {
#pragma unroll
      for (int k = 1; k < R; ++k) x[k] = x[0];
    } else {
      T e[R / 2], o[R / 2];
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
// z: this group's exchange area (Xchg::ZG elements), tw: e^{+2 pi i m / N}
// (for Cb2 elements each twiddle is a Cb2 of splat pairs).
template <int N1, int N2, typename T>
__device__ __forceinline__ void fft_lanes(T (&v)[N2], int n1, T* z, const T* tw, unsigned gmask) {
  constexpr int ZS = Xchg<N1, N2>::ZS, H = Xchg<N1, N2>::H;
  Dft<N2>::run(v);
#pragma unroll
  for (int k2 = 1; k2 < N2; ++k2) v[k2] = cmul(v[k2], tw[n1 * k2]);
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) z[k2 * ZS + n1] = v[k2];
  __syncwarp(gmask);
#pragma unroll
  for (int h = 0; h < H; ++h) {
    T u[N1];
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
