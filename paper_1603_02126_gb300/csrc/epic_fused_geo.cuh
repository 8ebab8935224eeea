// Launch geometry of the single-pass (fused) imaging kernels and of their
// adjoint: per grid size N, the N1 lanes of one 1-D FFT, the N2 points each
// lane holds, the CTA size, and the derived group / column-round counts.
#pragma once

#include <cuda_runtime.h>

#include "epic_fft.cuh"

namespace epic {

template <int N> struct Cfg;
template <> struct Cfg<16>  { static constexpr int N1 = 4, N2 = 4,  BT = 64; };
template <> struct Cfg<32>  { static constexpr int N1 = 4, N2 = 8,  BT = 128; };
template <> struct Cfg<64>  { static constexpr int N1 = 8, N2 = 8,  BT = 512; };
template <> struct Cfg<128> { static constexpr int N1 = 8, N2 = 16, BT = 512; };

constexpr int kMaxAntPerThread = 4;

template <int N>
struct Geo {
  static constexpr int N1 = Cfg<N>::N1, N2 = Cfg<N>::N2, BT = Cfg<N>::BT;
  static constexpr int GROUPS = BT / N1;
  static constexpr int COLROUNDS = N / GROUPS;
  static constexpr int NACC = COLROUNDS * N2;
  static constexpr int H = N2 / N1;
  static constexpr int ZS = N1 + 1;                       // padded exchange row
  static constexpr int ZG0 = N2 * ZS;
  static constexpr int ZG = ZG0 + ((8 - ZG0 % 16) + 16) % 16;  // group stride
  static_assert(N1 * N2 == N, "N1*N2 must be N");
  static_assert(N2 % N1 == 0, "N2 must be a multiple of N1");
  static_assert(N % GROUPS == 0, "columns must split evenly over groups");
  static_assert(32 % N1 == 0, "FFT groups must tile a warp");
};

// 1-D FFT of length N on a group of N1 lanes (see fft::fft_lanes); T is
// float2 or fft::Cb2.
template <int N, typename T>
__device__ __forceinline__ void fft_group(T (&v)[Geo<N>::N2], int n1, T* z, const T* tw, unsigned gmask) {
  fft::fft_lanes<Geo<N>::N1, Geo<N>::N2>(v, n1, z, tw, gmask);
}

}  // namespace epic
