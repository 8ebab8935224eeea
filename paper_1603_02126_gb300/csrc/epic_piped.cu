// Warp-specialised form of the fused imaging kernel (N = 64 and 128).
//
// The two-barrier fused kernel spends much of each frame filling and
// draining its phases: every warp waits at a CTA barrier between the row
// pass and the column pass.  Here the CTA is split into two roles joined by
// a two-slot pipeline in shared memory:
//   producers (warps 0-3)  frame t: unpack the voltages, multiply by 1/g
//       (Eq. 8), gather the gridding taps of every occupied row (Eq. 9) and
//       run its row FFT into spectra slot t mod 2; then signal "full";
//   consumers (warps 4-15) frame t: wait "full", evaluate the calibrator
//       pixel straight from the row spectra (one column DFT output) and
//       correlate it with every antenna (Eqs. 12, 15), run the column FFTs
//       (Eq. 10) and accumulate |E|^2 in registers; then signal "empty".
// So the producers build frame t+1 while the consumers transform frame t.
// The hand-off uses mbarriers; every wait has an iteration limit, after which
// the kernel raises the plan's error flag and runs to the end without
// waiting (results are then discarded by the host).
#include "epic_fft.cuh"
#include "epic_internal.h"

#include <cstdint>

namespace epic {
namespace {

using fft::cmul;
using fft::kFull;

constexpr int kBT = 512;            // threads per CTA
constexpr int kN1 = 8;              // lanes per 1-D FFT
constexpr int kProdWarps = 4;
constexpr int kProdThreads = kProdWarps * 32;
constexpr int kConsThreads = kBT - kProdThreads;
constexpr int kProdGroups = kProdThreads / kN1;   // 16 row FFTs in flight
constexpr int kConsGroups = kConsThreads / kN1;   // 48 column FFTs in flight
constexpr int kGroupsPerWarp = 32 / kN1;
constexpr int kBarProd = 1;         // named barrier of the producer warps
constexpr int kBarCons = 2;         // named barrier of the consumer warps
constexpr int kWaitLimit = 1 << 20;

template <int N>
struct PGeo {
  static constexpr int N2 = N / kN1;
  static constexpr int H = N2 / kN1;
  static constexpr int ZG = fft::Xchg<kN1, N2>::ZG;
  static constexpr int CR = (N + kConsGroups - 1) / kConsGroups;   // column rounds
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void named_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

__device__ __forceinline__ void mb_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mb_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mb_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase of the given parity (at most `limit` polls);
// after a timeout (or once any thread has timed out) it returns at once.
__device__ __forceinline__ void mb_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                        int* err, int limit) {
  if (*abort_flag) return;
  for (int i = 0; i < limit; ++i) {
    if (mb_try(bar, parity)) return;
    if ((i & 255) == 255 && *abort_flag) return;
  }
  *abort_flag = 1;
  atomicExch(err, 1);
}

__device__ __forceinline__ unsigned load_raw_ci4(const ImageArgs& A, long long t, int c, int a) {
  return __ldg(static_cast<const unsigned char*>(A.volt) +
               (static_cast<size_t>(t) * A.n_chan + c) * A.n_ant + a);
}

__device__ __forceinline__ float2 load_raw_c64(const ImageArgs& A, long long t, int c, int a) {
  return __ldg(static_cast<const float2*>(A.volt) + (static_cast<size_t>(t) * A.n_chan + c) * A.n_ant + a);
}

struct PipeSmem {
  float2* Tt;      // [2][N][rs] row spectra, transposed and swizzled
  float2* Z;       // [64 groups][ZG] FFT exchange
  float2* tw;      // [N2][N1] twiddles e^{+2 pi i n1 k2 / N}
  float2* Es;      // [2][Na] E / g
  float2* Er;      // [2][Na] E (raw, scaled) for the correlation
  float2* prow;    // [rows_alloc] calibrator-pixel weight of each window row
  uint64_t* bars;  // full[2], empty[2]
  int* abort_flag;
  uint4* sgcnt;    // [rows_alloc * N1] gather group lengths (TS)
  int* sgofs;      // [rows_alloc * N1] gather offsets (TS)
  uint2* sgent;    // [gmax] gather entries (TS)
};

// Producer role for one work unit: frames [t0, t1) of channel c; f is the
// CTA's running frame count (pipeline slot f mod 2, use f / 2 of that slot).
template <int N, int NZ, int MAXP, bool TS>
__device__ __forceinline__ long long producer_unit(const ImageArgs& A, const PipeSmem& S, int c,
                                                   long long t0, long long t1, long long f) {
  constexpr int N2 = PGeo<N>::N2, H = PGeo<N>::H;
  const int tid = threadIdx.x;                    // 0 .. kProdThreads - 1
  const int g = tid / kN1, n1 = tid % kN1;
  const int Na = A.n_ant, rs = A.rs;
  float2* zg = S.Z + g * PGeo<N>::ZG;
  const int R = __ldg(A.win4 + c).y;
  const float vs = A.vscale ? __ldg(A.vscale + c) : 1.0f;
  const float2* wg = A.wgain + static_cast<size_t>(c) * Na;
  const int gb = __ldg(A.gbase + c);
  const int* gofs = A.gofs + static_cast<size_t>(c) * A.rows_alloc * kN1;
  const uint4* gcnt = A.gcnt + static_cast<size_t>(c) * A.rows_alloc * kN1;
  const uint2* gent = A.gent + gb;

  if constexpr (TS) {
    named_sync(kBarProd, kProdThreads);           // previous unit's gathers are done
    const int gn = __ldg(A.gbase + c + 1) - gb;
    for (int i = tid; i < gn; i += kProdThreads) S.sgent[i] = __ldg(gent + i);
    for (int i = tid; i < R * kN1; i += kProdThreads) {
      S.sgofs[i] = __ldg(gofs + i);
      S.sgcnt[i] = __ldg(gcnt + i);
    }
  }

  // raw voltages of the unit's first frame
  unsigned rb[MAXP];
  float2 rf[MAXP];
#pragma unroll
  for (int i = 0; i < MAXP; ++i) {
    const int a = tid + kProdThreads * i;
    rb[i] = 0u;
    rf[i] = make_float2(0.f, 0.f);
    if (a < Na) {
      if (A.input_fmt == 0) rb[i] = load_raw_ci4(A, t0, c, a);
      else rf[i] = load_raw_c64(A, t0, c, a);
    }
  }

  for (long long t = t0; t < t1; ++t, ++f) {
    const int b = static_cast<int>(f & 1);
    const uint32_t ph = static_cast<uint32_t>((f >> 1) & 1);
    // slot b is free once the consumers have finished frame f - 2
    if (f >= 2) mb_wait(smem_addr(S.bars + 2 + b), ph ^ 1u, S.abort_flag, A.err,
                        A.wait_limit > 0 ? A.wait_limit : kWaitLimit);

    float2* Es = S.Es + b * Na;
    float2* Er = S.Er + b * Na;
#pragma unroll
    for (int i = 0; i < MAXP; ++i) {
      const int a = tid + kProdThreads * i;
      if (a < Na) {
        float2 e;
        if (A.input_fmt == 0) {
          const int re = static_cast<int>(rb[i] << 24) >> 28;
          const int im = static_cast<int>(rb[i] << 28) >> 28;
          e = make_float2(static_cast<float>(re) * vs, static_cast<float>(im) * vs);
        } else {
          e = make_float2(rf[i].x * vs, rf[i].y * vs);
        }
        Er[a] = e;
        Es[a] = cmul(e, __ldg(wg + a));
        // next frame's voltages, consumed one frame from now
        if (t + 1 < t1) {
          if (A.input_fmt == 0) rb[i] = load_raw_ci4(A, t + 1, c, a);
          else rf[i] = load_raw_c64(A, t + 1, c, a);
        }
      }
    }
    named_sync(kBarProd, kProdThreads);           // Es of this frame complete

    float2* Tt = S.Tt + static_cast<size_t>(b) * N * rs;
    for (int rbase = g - g % kGroupsPerWarp; rbase < R; rbase += kProdGroups) {
      const int row = rbase + g % kGroupsPerWarp;
      const bool live = row < R;
      float2 v[N2];
#pragma unroll
      for (int j = 0; j < N2; ++j) v[j] = make_float2(0.f, 0.f);
      if (live) {
        const int li = row * kN1 + n1;
        int e = TS ? S.sgofs[li] : __ldg(gofs + li);
        const uint4 cw = TS ? S.sgcnt[li] : __ldg(gcnt + li);
        const unsigned cv[4] = {cw.x, cw.y, cw.z, cw.w};
        const uint2* ge = TS ? S.sgent : gent;
#pragma unroll
        for (int j = 0; j < NZ; ++j) {
          const int cj = static_cast<int>((cv[j >> 2] >> (8 * (j & 3))) & 255u);
          float2 sum = make_float2(0.f, 0.f);
          for (int k = 0; k < cj; ++k) {
            const uint2 en = TS ? ge[e + k] : __ldg(ge + e + k);
            const float2 x = Es[en.x];
            const float w = __uint_as_float(en.y);
            sum.x = fmaf(w, x.x, sum.x);
            sum.y = fmaf(w, x.y, sum.y);
          }
          e += cj;
          v[j] = sum;
        }
      }
      fft::fft_lanes_p<kN1, N2, NZ>(v, n1, zg, S.tw, kFull);
      if (live) {
        // kx = n1 + N1 h + N2 k1 = n1 (mod 8): one swizzled row index per thread
        float2* tb = Tt + n1 * rs + (row ^ n1);
#pragma unroll
        for (int h = 0; h < H; ++h)
#pragma unroll
          for (int k1 = 0; k1 < kN1; ++k1) tb[(kN1 * h + N2 * k1) * rs] = v[h * kN1 + k1];
      }
    }
    mb_arrive(smem_addr(S.bars + b));             // slot b holds frame f
  }
  return f;
}

// Consumer role for one work unit (same frame numbering as the producers).
template <int N, int NZ, int MAXQ>
__device__ __forceinline__ long long consumer_unit(const ImageArgs& A, const PipeSmem& S, int c,
                                                   long long t0, long long t1, long long f) {
  constexpr int N2 = PGeo<N>::N2, H = PGeo<N>::H, CR = PGeo<N>::CR;
  const int q = threadIdx.x - kProdThreads;       // 0 .. kConsThreads - 1
  const int lane = q & 31;
  const int g = q / kN1, n1 = q % kN1;
  const int Na = A.n_ant, rs = A.rs;
  float2* zg = S.Z + (kProdGroups + g) * PGeo<N>::ZG;
  const int R = __ldg(A.win4 + c).y;
  const int jmax = (R - n1 + kN1 - 1) / kN1;      // this lane's rows n1 + N1 j < R
  const int kx0 = A.k0x;
  const int sw0 = kx0 & 7;

  // calibrator-pixel weights of the window rows for this channel:
  // e^{+2 pi i row k0y / N} times the window/centring phase
  if (A.do_cal) {
    named_sync(kBarCons, kConsThreads);           // previous unit's readers are done
    const float2 pph = __ldg(A.pixph + c);
    for (int r = q; r < R; r += kConsThreads)
      S.prow[r] = cmul(__ldg(A.twid + (r * A.k0y) % N), pph);
    named_sync(kBarCons, kConsThreads);
  }

  float acc[CR * N2];
#pragma unroll
  for (int i = 0; i < CR * N2; ++i) acc[i] = 0.f;
  float2 kac[MAXQ];
  float pac[MAXQ];
#pragma unroll
  for (int i = 0; i < MAXQ; ++i) {
    kac[i] = make_float2(0.f, 0.f);
    pac[i] = 0.f;
  }

  for (long long t = t0; t < t1; ++t, ++f) {
    const int b = static_cast<int>(f & 1);
    const uint32_t ph = static_cast<uint32_t>((f >> 1) & 1);
    mb_wait(smem_addr(S.bars + b), ph, S.abort_flag, A.err, A.wait_limit > 0 ? A.wait_limit : kWaitLimit);
    const float2* Tt = S.Tt + static_cast<size_t>(b) * N * rs;

    if (A.do_cal) {
      // calibrator pixel: column k0x of the row spectra times the row weights
      float2 p = make_float2(0.f, 0.f);
      for (int r = lane; r < R; r += 32) {
        const float2 x = Tt[kx0 * rs + (r ^ sw0)];
        const float2 w = S.prow[r];
        p.x += x.x * w.x - x.y * w.y;
        p.y += x.x * w.y + x.y * w.x;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        p.x += __shfl_xor_sync(kFull, p.x, o);
        p.y += __shfl_xor_sync(kFull, p.y, o);
      }
      const float2* Er = S.Er + b * Na;
#pragma unroll
      for (int i = 0; i < MAXQ; ++i) {
        const int a = q + kConsThreads * i;
        if (a < Na) {
          const float2 e = Er[a];
          kac[i].x += e.x * p.x + e.y * p.y;
          kac[i].y += e.y * p.x - e.x * p.y;
          pac[i] += e.x * e.x + e.y * e.y;
        }
      }
    }

#pragma unroll
    for (int r = 0; r < CR; ++r) {
      const int kx = g + kConsGroups * r;
      if (kx < N) {                               // warp-uniform
        float2 v[N2];
        // kx = g (mod 8) and (n1 + N1 j) ^ s = (n1 ^ s) + N1 j for s < 8
        const float2* cb = Tt + kx * rs + (n1 ^ (kx & 7));
#pragma unroll
        for (int j = 0; j < N2; ++j) v[j] = (j < NZ && j < jmax) ? cb[kN1 * j] : make_float2(0.f, 0.f);
        fft::fft_lanes_p<kN1, N2, NZ>(v, n1, zg, S.tw, kFull);
#pragma unroll
        for (int s = 0; s < N2; ++s) acc[r * N2 + s] += v[s].x * v[s].x + v[s].y * v[s].y;
      }
    }
    mb_arrive(smem_addr(S.bars + 2 + b));         // slot b may be refilled
  }

  // flush the unit's partial sums (FP32 over one segment, FP64 across)
  double* img = A.image + static_cast<size_t>(c) * N * N;
#pragma unroll
  for (int r = 0; r < CR; ++r) {
    const int kx = g + kConsGroups * r;
    if (kx < N) {
#pragma unroll
      for (int h = 0; h < H; ++h)
#pragma unroll
        for (int k1 = 0; k1 < kN1; ++k1) {
          const int ky = n1 + kN1 * h + N2 * k1;
          atomicAdd(img + ky * N + kx, static_cast<double>(acc[r * N2 + h * kN1 + k1]) * A.img_scale);
        }
    }
  }
  if (A.do_cal) {
    const int* cellf = A.cellf + static_cast<size_t>(c) * Na;
#pragma unroll
    for (int i = 0; i < MAXQ; ++i) {
      const int a = q + kConsThreads * i;
      if (a < Na && __ldg(cellf + a) >= 0) {
        const size_t o = static_cast<size_t>(c) * Na + a;
        atomicAdd(&A.kacc[o].x, static_cast<double>(kac[i].x));
        atomicAdd(&A.kacc[o].y, static_cast<double>(kac[i].y));
        atomicAdd(A.pacc + o, static_cast<double>(pac[i]));
      }
    }
  }
  return f;
}

template <int N, bool TS, int MAXP, int MAXQ>
__global__ void __launch_bounds__(kBT, 1) epic_image_piped(const ImageArgs A) {
  constexpr int N2 = PGeo<N>::N2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PipeSmem S;
  const int Na = A.n_ant;
  S.Tt = reinterpret_cast<float2*>(smem_raw);
  S.Z = S.Tt + 2 * static_cast<size_t>(N) * A.rs;
  S.tw = S.Z + 64 * PGeo<N>::ZG;
  S.Es = S.tw + N;
  S.Er = S.Es + 2 * Na;
  S.prow = S.Er + 2 * Na;
  S.bars = reinterpret_cast<uint64_t*>(S.prow + A.rows_alloc);
  S.abort_flag = reinterpret_cast<int*>(S.bars + 4);
  S.sgcnt = reinterpret_cast<uint4*>((reinterpret_cast<uintptr_t>(S.abort_flag + 2) + 15) &
                                     ~static_cast<uintptr_t>(15));
  S.sgofs = reinterpret_cast<int*>(S.sgcnt + A.rows_alloc * kN1);
  S.sgent = reinterpret_cast<uint2*>(S.sgofs + ((A.rows_alloc * kN1 + 1) & ~1));

  const int tid = threadIdx.x;
  for (int i = tid; i < N; i += kBT) S.tw[i] = A.twid[(i % kN1) * (i / kN1)];
  if (tid == 0) {
    mb_init(smem_addr(S.bars + 0), kProdThreads);
    mb_init(smem_addr(S.bars + 1), kProdThreads);
    mb_init(smem_addr(S.bars + 2), kConsThreads);
    mb_init(smem_addr(S.bars + 3), kConsThreads);
    *S.abort_flag = 0;
  }
  __syncthreads();

  const bool producer = tid < kProdThreads;
  const long long T = A.n_time;
  const int units = A.n_chan * A.segs;
  long long f = 0;
  for (int u = blockIdx.x; u < units; u += gridDim.x) {
    const int c = u / A.segs;
    const int s = u - c * A.segs;
    const long long t0 = T * s / A.segs;
    const long long t1 = T * (s + 1) / A.segs;
    if (t0 >= t1) continue;
    const int4 wn = __ldg(A.win4 + c);
    const int span = wn.y > wn.w ? wn.y : wn.w;
    if (producer) {
      if (span <= kN1 * (N2 / 4)) f = producer_unit<N, N2 / 4, MAXP, TS>(A, S, c, t0, t1, f);
      else if (span <= kN1 * (N2 / 2)) f = producer_unit<N, N2 / 2, MAXP, TS>(A, S, c, t0, t1, f);
      else f = producer_unit<N, N2, MAXP, TS>(A, S, c, t0, t1, f);
    } else {
      if (span <= kN1 * (N2 / 4)) f = consumer_unit<N, N2 / 4, MAXQ>(A, S, c, t0, t1, f);
      else if (span <= kN1 * (N2 / 2)) f = consumer_unit<N, N2 / 2, MAXQ>(A, S, c, t0, t1, f);
      else f = consumer_unit<N, N2, MAXQ>(A, S, c, t0, t1, f);
    }
  }
}

template <int N, bool TS>
cudaError_t piped_launch_t(const ImageArgs& a, cudaStream_t s, bool prepare_only, size_t smem, int* ctas) {
  auto k = epic_image_piped<N, TS, 4, 2>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  if (prepare_only) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k, kBT, smem);
  k<<<a.grid, kBT, a.smem, s>>>(a);
  return cudaGetLastError();
}

template <int N>
cudaError_t piped_dispatch(const ImageArgs& a, cudaStream_t s, bool prepare_only, size_t smem, bool ts,
                           int* ctas) {
  return ts ? piped_launch_t<N, true>(a, s, prepare_only, smem, ctas)
            : piped_launch_t<N, false>(a, s, prepare_only, smem, ctas);
}

}  // namespace

bool piped_supported(int n, int n_ant) {
  return (n == 64 || n == 128) && n_ant <= kProdThreads * 4 && n_ant <= kConsThreads * 2;
}

size_t piped_smem_bytes(int n, int n_ant, int rs, int rows_alloc, long long gmax) {
  int zg = 0;
  if (n == 64) zg = PGeo<64>::ZG;
  else if (n == 128) zg = PGeo<128>::ZG;
  else return 0;
  size_t b = (2 * static_cast<size_t>(n) * rs + 64 * static_cast<size_t>(zg) + n + 4 * static_cast<size_t>(n_ant) +
              rows_alloc) * sizeof(float2);
  b = (b + 7) & ~static_cast<size_t>(7);
  b += 4 * sizeof(uint64_t) + 2 * sizeof(int);
  if (gmax > 0) b += image_table_bytes(rows_alloc, kN1, gmax);
  return b;
}

cudaError_t piped_prepare(int n, size_t smem, bool ts, int* ctas) {
  ImageArgs dummy{};
  if (n == 64) return piped_dispatch<64>(dummy, nullptr, true, smem, ts, ctas);
  if (n == 128) return piped_dispatch<128>(dummy, nullptr, true, smem, ts, ctas);
  return cudaErrorInvalidValue;
}

cudaError_t launch_piped(int n, const ImageArgs& a, cudaStream_t s) {
  if (n == 64) return piped_dispatch<64>(a, s, false, a.smem, a.gsmem != 0, nullptr);
  if (n == 128) return piped_dispatch<128>(a, s, false, a.smem, a.gsmem != 0, nullptr);
  return cudaErrorInvalidValue;
}

}  // namespace epic
