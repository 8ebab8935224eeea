// Reduced-precision EPIC imaging: both 1-D transforms of Eq. 10 as
// tensor-core GEMMs (tcgen05, FP16 or BF16 operands, FP32 accumulation).
//
// Per batch of frames (frame f = t_local * C + c):
//   grid_lp      per frame, E' = E / g (Eq. 8) into shared memory and
//                S_f = sum_a |E'_a| / Na, an upper bound of every grid cell
//                and row-spectrum value (s_f = largest power of two with
//                s_f S_f < 1); FP32
//                gridding (Eq. 9) as a gather into the window grid (the
//                plain path's window-column lists), scaled by s_f and stored
//                FP16/BF16 as Gh[f R + jw][2 x + (re, im)]; the calibrator
//                pixel is summed in FP32 from the same cells;
//   tc_rows      H = Gh F_r^T with the real-expanded DFT over window columns
//                (outputs 2 kx + (re, im)); the epilogue writes each row's
//                spectrum K-major as Hh[c][kx][t][2 jw + (re, im)];
//   tc_cols      D[r][t] = sum_k' F[r][k'] Hh[c][kx][t][k'] with the
//                real-expanded DFT matrix F (rows r = 2 ky + (re, im),
//                columns k' = 2 jw + (re, im)); TMEM lane r then sums
//                D[r][t]^2 / s_t^2 over the frames t of the tile, lanes 2ky and
//                2ky+1 are added and the result goes to image[c][ky][kx]
//                (FP64 atomics).  |E|^2 does not depend on where the window
//                starts, so both DFTs use window coordinates.
// tc_cols is a persistent, warp-specialised kernel: warp 0 issues TMA loads
// (128B-swizzled; the CTA's DFT tile is loaded once, the data tiles stream
// through a 4-stage ring of 64-element K chunks, the next tile is
// prefetched into L2), warp 1 owns the TMEM allocation and issues
// tcgen05.mma from one thread (M = 128 DFT rows, N = 256 = 128 frames of
// two columns kx, kx + 1, K = 16 per instruction), warps 2-9 drain the
// double-buffered TMEM accumulators (one warp per column and lane
// quarter).  tc_rows (N = 256 outputs per MMA) and the X-engine (N = 256
// columns per MMA) stream both operands through a 4-stage ring, with
// epilogue warps 2-9.
// Every mbarrier wait is bounded; on timeout the kernel records an error
// flag, waits (bounded) for its copies and MMAs in flight and winds down.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>
#include <type_traits>

#include "epic_fft.cuh"
#include "epic_internal.h"

namespace epic {
namespace {

template <int N> struct LCfg;
template <> struct LCfg<128> { static constexpr int N1 = 8,  N2 = 16; };
template <> struct LCfg<256> { static constexpr int N1 = 16, N2 = 16; };

constexpr int kLBT = 256;

// Exponent k of the largest power of two s = 2^k with s * S < 1 (S > 0),
// from the float's exponent field, clamped to [-60, 60] so that s and 1/s^2
// are normal floats.
__device__ __forceinline__ int pow2_exp_below_inverse(float S) {
  if (!(S > 0.f)) return 0;
  const int e = static_cast<int>((__float_as_uint(S) >> 23) & 0xff) - 127;
  int k = -(e + 1);
  return k < -60 ? -60 : (k > 60 ? 60 : k);
}
__device__ __forceinline__ float exp2i(int k) {   // 2^k for k in [-126, 127]
  return __uint_as_float(static_cast<unsigned>(k + 127) << 23);
}

__device__ __forceinline__ float2 load_volt_tc(const void* volt, int fmt, size_t idx) {
  if (fmt == 0) {
    const unsigned b = __ldg(static_cast<const unsigned char*>(volt) + idx);
    const int re = static_cast<int>(b << 24) >> 28;
    const int im = static_cast<int>(b << 28) >> 28;
    return make_float2(static_cast<float>(re), static_cast<float>(im));
  }
  return __ldg(static_cast<const float2*>(volt) + idx);
}

// (re, im) rounded to the storage type, as one 4-byte store.
__device__ __forceinline__ void store_lp(__half* dst, float re, float im) {
  *reinterpret_cast<__half2*>(dst) = __floats2half2_rn(re, im);
}
__device__ __forceinline__ void store_lp(__nv_bfloat16* dst, float re, float im) {
  *reinterpret_cast<__nv_bfloat162*>(dst) = __floats2bfloat162_rn(re, im);
}

// ---- gridding into the low-precision window grid, FP32 calibrator pixel ----
// One frame at a time per CTA: E' = E / g (Eq. 8) into shared memory, then
// every lane (window row jw, n1) gathers the taps of its window columns
// x = n1 + N1 j (Eq. 9, the plan's window-column lists), scales by s_f and
// stores the cell rounded to FP16/BF16 into Gh[f R_alloc + jw][2x + re/im]
// (columns without taps get zeros).  The calibrator pixel, the Eq. 10 sum
// at k0, is accumulated from the FP32 cells with their absolute phases.
template <int N, typename T>
__global__ void __launch_bounds__(kLBT) grid_lp_kernel(const TcArgs A, long long t0, int nt) {
  constexpr int N1 = LCfg<N>::N1, N2 = LCfg<N>::N2;
  constexpr int GROUPS = kLBT / N1;
  constexpr int CW = (N2 + 15) / 16;
  extern __shared__ float2 Es[];                   // [Na] E / g of the current frame
  __shared__ float red[kLBT / 32];
  const int g = threadIdx.x / N1, n1 = threadIdx.x % N1;
  const int lane = threadIdx.x & 31;
  const int C = A.u.n_chan, Na = A.u.n_ant;
  const int nj = A.kr / (2 * N1);                  // column blocks held in Gh
  T* gh = static_cast<T*>(A.gh);
  const long long frames = static_cast<long long>(nt) * C;
  for (long long it = blockIdx.x; it < frames; it += gridDim.x) {
    const int c = static_cast<int>(it / nt);
    const int tl = static_cast<int>(it - static_cast<long long>(c) * nt);
    const size_t f = static_cast<size_t>(tl) * C + c;
    const float vs = A.u.vscale ? __ldg(A.u.vscale + c) : 1.0f;
    __syncthreads();
    // E' and S_f = sum_a |E'_a| / Na over unflagged antennas: an upper bound
    // of every grid cell and row-spectrum value (normalised taps, 1/Na folded)
    float sa = 0.f;
    for (int a = threadIdx.x; a < Na; a += kLBT) {
      const float2 e = load_volt_tc(A.u.volt, A.u.input_fmt, (static_cast<size_t>(t0 + tl) * C + c) * Na + a);
      const float2 ec = fft::cmul(make_float2(e.x * vs, e.y * vs), __ldg(A.u.wgain + static_cast<size_t>(c) * Na + a));
      Es[a] = ec;
      if (__ldg(A.u.cell0 + static_cast<size_t>(c) * Na + a) >= 0) sa += sqrtf(ec.x * ec.x + ec.y * ec.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sa += __shfl_xor_sync(fft::kFull, sa, o);
    if (lane == 0) red[threadIdx.x >> 5] = sa;
    __syncthreads();
    float S = 0.f;
#pragma unroll
    for (int w = 0; w < kLBT / 32; ++w) S += red[w];
    const int ke = pow2_exp_below_inverse(S / static_cast<float>(Na));
    const float sf = exp2i(ke);                    // s_f multiplies the cells
    if (threadIdx.x == 0) {
      A.fscale[f] = sf;
      A.finv2[f] = exp2i(-2 * ke);                 // 1 / s_f^2 multiplies |D|^2
    }
    const int4 wn = __ldg(A.win4 + c);             // (y0, rows, x0, cols)
    const int R = wn.y;
    const int nl = A.u.rows_alloc * N1;
    const int* gofs = A.u.gofs + static_cast<size_t>(c) * nl;
    const uint4* gcnt = A.u.gcnt + static_cast<size_t>(c) * nl * CW;
    const uint2* gent = A.u.gent + __ldg(A.u.gbase + c);
    float2 pix = make_float2(0.f, 0.f);
    for (int row = g; row < R; row += GROUPS) {
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
      T* dst = gh + (f * A.r_alloc + row) * static_cast<size_t>(A.kr);
#pragma unroll
      for (int j = 0; j < N2; ++j) {
        if (j >= nj) break;
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
        const int x = n1 + N1 * j;
        store_lp(dst + 2 * x, sum.x * sf, sum.y * sf);
        if (A.u.do_cal && cj > 0) {
          const int m = ((wn.z + x) * A.u.k0x + (wn.x + row) * A.u.k0y) & (N - 1);
          const float2 t = __ldg(A.u.twid + m);
          pix.x += sum.x * t.x - sum.y * t.y;
          pix.y += sum.x * t.y + sum.y * t.x;
        }
      }
    }
    if (A.u.do_cal) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        pix.x += __shfl_xor_sync(fft::kFull, pix.x, o);
        pix.y += __shfl_xor_sync(fft::kFull, pix.y, o);
      }
      if (lane == 0 && (pix.x != 0.f || pix.y != 0.f)) {
        atomicAdd(&A.u.pix[f].x, pix.x * A.u.pix_sign);
        atomicAdd(&A.u.pix[f].y, pix.y * A.u.pix_sign);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// tcgen05 / TMA / mbarrier helpers (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false on timeout or when another role has aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          int* err) {
  for (int i = 0; i < (1 << 22); ++i) {
    if (mbar_try(bar, parity)) return true;
    if ((i & 255) == 255 && *abort_flag) return false;
  }
  *abort_flag = 1;
  atomicExch(err, 1);
  return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* tm, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Bring one 3-D box into L2 ahead of its load (no shared memory, no barrier).
__device__ __forceinline__ void tma_prefetch_3d(const CUtensorMap* tm, int x, int y, int z) {
  asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];"
               ::"l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z)
               : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* tm, int x, int y, int z,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO); the leading offset is unused in this layout.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFF) >> 4);
  d |= static_cast<uint64_t>(16 >> 4) << 16;
  d |= static_cast<uint64_t>(1024 >> 4) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  d |= static_cast<uint64_t>(2) << 61;
  return d;
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

constexpr int kTcThreads = 320;          // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue
constexpr int kEpiWarps = 8;             // one per (column half, TMEM lane quarter)
constexpr int kTile = 128;               // DFT rows, and frames per column half
constexpr int kChunkBytes = kTile * 128; // one 64-element K chunk of a 128-row tile
constexpr int kColN = 256;               // MMA N of tc_cols: 128 frames of kx, then of kx + 1
constexpr int kColChunkBytes = kColN * 128;
constexpr int kColStages = 4;            // K-chunk ring of the data operand
constexpr uint32_t kColTmemCols = 512;   // tc_cols, tc_rows, X-engine: two 256-column accumulators

// Dynamic shared memory of tc_cols_kernel for a K extent of kp elements:
// the CTA's resident DFT tile and the data ring.
size_t tc_smem_bytes(int kp) {
  const size_t tile = static_cast<size_t>(kp / 64) * kChunkBytes;
  return 1024 /*alignment slack*/ + tile + kColStages * kColChunkBytes + 256 /*barriers*/;
}

// Column DFT GEMM.  A CTA owns one 128-row DFT tile (rows 2 ky + re/im),
// resident in shared memory, and walks the data tiles (channel, column
// pair kx and kx + 1, 128 frames): each MMA is M = 128 DFT rows by N = 256
// (the 128 frames of kx, then those of kx + 1; one 3-D TMA box of two
// columns) by K = 16, the shape that keeps the tensor pipe busiest for one
// CTA.  Data chunks stream through a 4-stage ring of 64-element K chunks;
// two 256-column TMEM accumulators alternate between the MMA and the
// epilogue.
template <bool kBf16>
__global__ void __launch_bounds__(kTcThreads, 1)
    tc_cols_kernel(const __grid_constant__ CUtensorMap tm_dft, const __grid_constant__ CUtensorMap tm_data,
                   const TcArgs A, int nt) {
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int kc_n = A.kp / 64;
  const uint32_t tile_bytes = static_cast<uint32_t>(kc_n) * kChunkBytes;
  unsigned char* sA = base;                         // the DFT tile (resident)
  unsigned char* sD = base + tile_bytes;            // data ring, kColStages chunks
  uint64_t* bars = reinterpret_cast<uint64_t*>(sD + kColStages * kColChunkBytes);
  // bars: [0, S) full; [S, 2S) empty; 2S + {0,1} tmem_full; 2S + {2,3}
  // tmem_empty; 2S + 4 dft_full; 2S + 5 drain
  constexpr int S = kColStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 6);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 2 * S + 7);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int C = A.u.n_chan, N = A.u.grid_n;
  const int MB = 2 * N / kTile;                     // DFT tiles
  const int tbk = (nt + kTile - 1) / kTile;
  const long long dtiles = static_cast<long long>(C) * (N / 2) * tbk;
  const int G = gridDim.x / MB;                     // CTAs per DFT tile (grid is a multiple of MB)
  const int mb = blockIdx.x % MB;
  const long long u0 = blockIdx.x / MB;

  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(smem_u32(bars + i), 1);
      mbar_init(smem_u32(bars + S + i), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(bars + 2 * S + i), 1);
      mbar_init(smem_u32(bars + 2 * S + 2 + i), kEpiWarps);
    }
    mbar_init(smem_u32(bars + 2 * S + 4), 1);
    mbar_init(smem_u32(bars + 2 * S + 5), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kColTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tm_dft)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tm_data)) : "memory");
      const uint32_t bdft = smem_u32(bars + 2 * S + 4);
      mbar_expect_tx(bdft, tile_bytes);
      for (int kc = 0; kc < kc_n; ++kc)
        tma_load_2d(smem_u32(sA + kc * kChunkBytes), &tm_dft, kc * 64, mb * kTile, bdft);
      long long it = 0;
      bool ok = true;
      for (long long u = u0; ok && u < dtiles; u += G) {
        const int tb = static_cast<int>(u % tbk);
        const int ck = static_cast<int>(u / tbk) * 2;   // c * N + kx, kx even
        // the next data tile into L2 now (first DFT tile's CTA), so that its
        // chunk loads find it there rather than in DRAM
        if (mb == 0 && u + G < dtiles) {
          const long long un = u + G;
          for (int kc = 0; kc < kc_n; ++kc)
            tma_prefetch_3d(&tm_data, kc * 64, static_cast<int>(un % tbk) * kTile, static_cast<int>(un / tbk) * 2);
        }
        for (int kc = 0; kc < kc_n; ++kc, ++it) {
          const int s = static_cast<int>(it % S);
          const uint32_t ph = static_cast<uint32_t>((it / S) & 1);
          if (!mbar_wait(smem_u32(bars + S + s), ph ^ 1, abort_flag, A.err)) {
            ok = false;
            break;
          }
          const uint32_t bfull = smem_u32(bars + s);
          mbar_expect_tx(bfull, kColChunkBytes);
          tma_load_3d(smem_u32(sD + s * kColChunkBytes), &tm_data, kc * 64, tb * kTile, ck, bfull);
        }
      }
      if (*abort_flag) {
        // let the copies still in flight land before the CTA exits (bounded)
        for (int w = 0; w < (1 << 22) && !mbar_try(smem_u32(bars + 2 * S + 4), 0); ++w) {
        }
        for (long long j = it > S ? it - S : 0; j < it; ++j) {
          const uint32_t bar = smem_u32(bars + j % S), ph = static_cast<uint32_t>((j / S) & 1);
          for (int w = 0; w < (1 << 22) && !mbar_try(bar, ph); ++w) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | ((kBf16 ? 1u : 0u) << 7) | ((kBf16 ? 1u : 0u) << 10) |
                             (static_cast<uint32_t>(kColN >> 3) << 17) |
                             (static_cast<uint32_t>(kTile >> 4) << 24);
      bool ok = mbar_wait(smem_u32(bars + 2 * S + 4), 0, abort_flag, A.err);
      tc_fence_after();
      long long it = 0;
      int i = 0;
      for (long long u = u0; ok && u < dtiles; u += G, ++i) {
        const int acc = i & 1;
        const uint32_t aph = static_cast<uint32_t>((i >> 1) & 1);
        if (!mbar_wait(smem_u32(bars + 2 * S + 2 + acc), aph ^ 1, abort_flag, A.err)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(acc * kColN);
        for (int kc = 0; kc < kc_n; ++kc, ++it) {
          const int s = static_cast<int>(it % S);
          const uint32_t ph = static_cast<uint32_t>((it / S) & 1);
          if (!mbar_wait(smem_u32(bars + s), ph, abort_flag, A.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(sA + kc * kChunkBytes), b0 = smem_u32(sD + s * kColChunkBytes);
#pragma unroll
          for (int k = 0; k < 4; ++k)
            mma_f16(d_tmem, sdesc_sw128(a0 + k * 32), sdesc_sw128(b0 + k * 32), idesc, (kc | k) != 0);
          mma_commit(smem_u32(bars + S + s));   // data chunk free once these MMAs finish
        }
        if (ok) mma_commit(smem_u32(bars + 2 * S + acc));   // accumulator ready
      }
      if (*abort_flag) {
        // wait (bounded) for the MMAs already issued before TMEM is freed
        const uint32_t drain = smem_u32(bars + 2 * S + 5);
        mma_commit(drain);
        for (int w = 0; w < (1 << 22) && !mbar_try(drain, 0); ++w) {
        }
      }
    }
  } else {
    // ---------------- epilogue (warps 2-9) ----------------
    const int q = warp & 3;                        // TMEM lane quarter of this warp
    const int half = (warp - 2) >> 2;              // column kx (0) or kx + 1 (1)
    const int r = mb * kTile + q * 32 + lane;      // DFT row = 2 ky + (re, im)
    const int ky = r >> 1;
    int i = 0;
    for (long long u = u0; u < dtiles; u += G, ++i) {
      const int acc = i & 1;
      const uint32_t ph = static_cast<uint32_t>((i >> 1) & 1);
      if (!mbar_wait(smem_u32(bars + 2 * S + acc), ph, abort_flag, A.err)) break;
      tc_fence_after();
      const int tb = static_cast<int>(u % tbk);
      const int ck = static_cast<int>(u / tbk) * 2 + half;
      const int c = ck / N, kx = ck % N;
      float sum = 0.f;
#pragma unroll
      for (int ch = 0; ch < kTile / 32; ++ch) {
        const int col = ch * 32;
        const int t = tb * kTile + col + lane;
        const float my_w = (t < nt) ? __ldg(A.finv2 + static_cast<size_t>(t) * C + c) : 0.f;
        float v[32];
        tmem_ld32(tmem_base + (static_cast<uint32_t>(q * 32) << 16) +
                      static_cast<uint32_t>(acc * kColN + half * kTile + col),
                  v);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float w = __shfl_sync(fft::kFull, my_w, j);
          sum = fmaf(v[j] * v[j], w, sum);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(bars + 2 * S + 2 + acc));
      const float other = __shfl_xor_sync(fft::kFull, sum, 1);
      if ((lane & 1) == 0)
        atomicAdd(A.u.image + (static_cast<size_t>(c) * N + ky) * N + kx,
                  static_cast<double>(sum + other) * A.u.img_scale);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kColTmemCols)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// X-engine on the tensor cores (visibility comparison path, 4-bit input).
// Per channel the voltages become a real matrix Z [2 Na_p][Tp] of FP16
// integers (row 2a = Re E_a, row 2a + 1 = Im E_a, time contiguous, zero
// padded); G = Z Z^T by tcgen05.mma (M = N = 128, K = 16 per instruction,
// FP32 accumulation in TMEM), tiles of 128 rows by 256 columns (two column
// blocks, M = 128, N = 256 per MMA) on or above the diagonal; the block of
// a tile that falls below the diagonal is computed but not written.  The
// 4-bit values and every partial sum are integers below 2^24, so G is
// exact.  Epilogue: Re V_ab = G[2a][2b] + G[2a+1][2b+1],
// Im V_ab = G[2a+1][2b] - G[2a][2b+1] (rows 2a and 2a+1 are adjacent TMEM
// lanes, exchanged by one shuffle), times s_c^2 / T in FP64.
// ---------------------------------------------------------------------------
constexpr int kXeStages = 4;                 // K-chunk ring (A and B chunk per stage)
constexpr int kXeThreads = 320;              // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue
constexpr int kXeN = 256;                    // columns per tile: two 128-row blocks of Z
constexpr uint32_t kXeStageBytes = kChunkBytes + kXeN * 128;

size_t xe_smem_bytes() { return 1024 + kXeStages * kXeStageBytes + 256; }

// volt [T][C][Na] 4-bit -> Z [C][2 Na_p][Tp] FP16; block = (channel, 32
// antennas, 64 samples); thread = (row r of the 64, 16 samples).
__global__ void __launch_bounds__(256) xe_pack_kernel(const unsigned char* __restrict__ volt, long long t0,
                                                      int nt, int n_chan, int n_ant, int na_p, int tp,
                                                      __half* __restrict__ z) {
  __shared__ unsigned char tile[64][33];
  const int c = blockIdx.x, ab = blockIdx.y * 32, tb = blockIdx.z * 64;
  for (int i = threadIdx.x; i < 64 * 32; i += 256) {
    const int tt = i / 32, k = i % 32;
    const int t = tb + tt, a = ab + k;
    tile[tt][k] = (t < nt && a < n_ant)
                      ? __ldg(volt + (static_cast<size_t>(t0 + t) * n_chan + c) * n_ant + a)
                      : static_cast<unsigned char>(0);
  }
  __syncthreads();
  const int r = threadIdx.x / 4, q = threadIdx.x % 4;     // row 2k + s of the block, 16-sample quarter
  const int k = r >> 1, sgn = r & 1;
  __align__(16) __half v[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const unsigned b = tile[q * 16 + j][k];
    const int x = sgn ? static_cast<int>(b << 28) >> 28 : static_cast<int>(b << 24) >> 28;
    v[j] = __int2half_rn(x);
  }
  __half* dst = z + (static_cast<size_t>(c) * 2 * na_p + 2 * ab + r) * tp + tb + q * 16;
  reinterpret_cast<uint4*>(dst)[0] = reinterpret_cast<const uint4*>(v)[0];
  reinterpret_cast<uint4*>(dst)[1] = reinterpret_cast<const uint4*>(v)[1];
}

__global__ void __launch_bounds__(kXeThreads, 1)
    xengine_tc_kernel(const __grid_constant__ CUtensorMap tm_z, const XeTcArgs A) {
  extern __shared__ __align__(1024) unsigned char xe_smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(xe_smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + kXeStages * kXeStageBytes);
  // bars: [0, S) full, [S, 2S) empty, 2S + {0, 1} tmem_full, 2S + {2, 3}
  // tmem_empty, 2S + 4 drain (MMAs in flight after a timeout)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kXeStages + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 2 * kXeStages + 6);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nb = 2 * A.na_p / kTile;                        // row blocks per channel
  const int nbp = (nb + 1) / 2;                             // column block pairs
  int pairs = 0;                                            // tiles per channel
  for (int i = 0; i < nb; ++i) pairs += nbp - i / 2;
  const long long tiles = static_cast<long long>(A.n_chan) * pairs;
  const int kc_n = A.tp / 64;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kXeStages; ++i) {
      mbar_init(smem_u32(bars + i), 1);
      mbar_init(smem_u32(bars + kXeStages + i), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(bars + 2 * kXeStages + i), 1);
      mbar_init(smem_u32(bars + 2 * kXeStages + 2 + i), 8);
    }
    mbar_init(smem_u32(bars + 2 * kXeStages + 4), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kColTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  // tile u -> (channel, row block bi, column blocks 2 bjp and 2 bjp + 1),
  // bjp >= bi / 2 (the pair reaches the diagonal)
  auto tile_of = [&](long long u, int* c, int* bi, int* bjp) {
    *c = static_cast<int>(u / pairs);
    int pr = static_cast<int>(u - static_cast<long long>(*c) * pairs);
    int i = 0;
    while (pr >= nbp - i / 2) {
      pr -= nbp - i / 2;
      ++i;
    }
    *bi = i;
    *bjp = i / 2 + pr;
  };

  if (warp == 0) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tm_z)) : "memory");
      long long it = 0;                                       // K chunks issued so far
      for (long long u = blockIdx.x; u < tiles && !*abort_flag; u += gridDim.x) {
        int c, bi, bjp;
        tile_of(u, &c, &bi, &bjp);
        const int ya = c * 2 * A.na_p + bi * kTile, yb = c * 2 * A.na_p + 2 * bjp * kTile;
        for (int kc = 0; kc < kc_n; ++kc, ++it) {
          const int s = static_cast<int>(it % kXeStages);
          const uint32_t ph = static_cast<uint32_t>((it / kXeStages) & 1);
          if (!mbar_wait(smem_u32(bars + kXeStages + s), ph ^ 1, abort_flag, A.err)) break;
          const uint32_t bfull = smem_u32(bars + s);
          mbar_expect_tx(bfull, kXeStageBytes);
          unsigned char* st = base + s * kXeStageBytes;
          tma_load_2d(smem_u32(st), &tm_z, kc * 64, ya, bfull);
          tma_load_2d(smem_u32(st + kChunkBytes), &tm_z, kc * 64, yb, bfull);
          tma_load_2d(smem_u32(st + 2 * kChunkBytes), &tm_z, kc * 64, yb + kTile, bfull);
        }
      }
      if (*abort_flag) {
        // let the last loads land before the CTA's shared memory is released
        for (long long j = it > kXeStages ? it - kXeStages : 0; j < it; ++j) {
          const uint32_t bar = smem_u32(bars + j % kXeStages), ph = static_cast<uint32_t>((j / kXeStages) & 1);
          for (int w = 0; w < (1 << 22) && !mbar_try(bar, ph); ++w) {
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | (static_cast<uint32_t>(kXeN >> 3) << 17) |
                             (static_cast<uint32_t>(kTile >> 4) << 24);   // FP16 x FP16 -> FP32
      long long it = 0;
      int i = 0;
      bool ok = true;
      for (long long u = blockIdx.x; ok && u < tiles; u += gridDim.x, ++i) {
        const int acc = i & 1;
        const uint32_t aph = (i >> 1) & 1;
        if (!mbar_wait(smem_u32(bars + 2 * kXeStages + 2 + acc), aph ^ 1, abort_flag, A.err)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(acc * kXeN);
        for (int kc = 0; kc < kc_n; ++kc, ++it) {
          const int s = static_cast<int>(it % kXeStages);
          const uint32_t ph = static_cast<uint32_t>((it / kXeStages) & 1);
          if (!mbar_wait(smem_u32(bars + s), ph, abort_flag, A.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(base + s * kXeStageBytes), b0 = a0 + kChunkBytes;
#pragma unroll
          for (int k = 0; k < 4; ++k)
            mma_f16(d_tmem, sdesc_sw128(a0 + k * 32), sdesc_sw128(b0 + k * 32), idesc, (kc | k) != 0);
          mma_commit(smem_u32(bars + kXeStages + s));          // stage free once these MMAs finish
        }
        if (ok) mma_commit(smem_u32(bars + 2 * kXeStages + acc));   // accumulator ready
      }
      if (*abort_flag) {
        // MMAs still in flight must finish before TMEM is released
        const uint32_t drain = smem_u32(bars + 2 * kXeStages + 4);
        mma_commit(drain);
        for (int w = 0; w < (1 << 22) && !mbar_try(drain, 0); ++w) {
        }
      }
    }
  } else {
    // epilogue: warp (2..9) & 3 is the TMEM lane quarter it may read, and
    // (warp - 2) / 4 the column block of the pair it writes
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;
    const int r = q * 32 + lane;                             // tile row 2a' + s
    int i = 0;
    for (long long u = blockIdx.x; u < tiles; u += gridDim.x, ++i) {
      const int acc = i & 1;
      const uint32_t aph = (i >> 1) & 1;
      if (!mbar_wait(smem_u32(bars + 2 * kXeStages + acc), aph, abort_flag, A.err)) break;
      tc_fence_after();
      int c, bi, bjp;
      tile_of(u, &c, &bi, &bjp);
      const int bj = 2 * bjp + half;
      const bool upper = bj >= bi;                           // else the block lies below the diagonal
      const int a = (bi * kTile + r) >> 1;                   // antenna of this lane pair
      const bool even = (lane & 1) == 0;
      const float vs = A.vscale ? __ldg(A.vscale + c) : 1.0f;
      const double sc = static_cast<double>(vs) * static_cast<double>(vs) * A.scale;
      double2* V = A.vis + static_cast<size_t>(c) * A.n_ant * A.n_ant;
#pragma unroll
      for (int ch = 0; ch < kTile / 32; ++ch) {
        float v[32];
        tmem_ld32(tmem_base + (static_cast<uint32_t>(q * 32) << 16) +
                      static_cast<uint32_t>(acc * kXeN + half * kTile + ch * 32),
                  v);
        // v[2j + s'] = G[r][bj*128 + ch*32 + 2j + s']; partner lane holds row r ^ 1
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float p0 = __shfl_xor_sync(fft::kFull, v[2 * j], 1);
          const float p1 = __shfl_xor_sync(fft::kFull, v[2 * j + 1], 1);
          if (even && upper) {
            const int b = (bj * kTile + ch * 32 + 2 * j) >> 1;
            if (a < A.n_ant && b < A.n_ant) {
              // row 2a: v = G[2a][2b], G[2a][2b+1]; partner: G[2a+1][2b], G[2a+1][2b+1]
              const double re = (static_cast<double>(v[2 * j]) + static_cast<double>(p1)) * sc;
              const double im = (static_cast<double>(p0) - static_cast<double>(v[2 * j + 1])) * sc;
              double2* o = V + static_cast<size_t>(a) * A.n_ant + b;
              if (A.accumulate) *o = make_double2(o->x + re, o->y + im);
              else *o = make_double2(re, im);
              if (bi != bj) {
                double2* m = V + static_cast<size_t>(b) * A.n_ant + a;
                if (A.accumulate) *m = make_double2(m->x + re, m->y - im);
                else *m = make_double2(re, -im);
              }
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(bars + 2 * kXeStages + 2 + acc));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kColTmemCols)
                 : "memory");
  }
}

// Row DFT of the precision form on the tensor cores: H = Gh F_r^T, rows =
// (frame, window row), K = 2 x window columns (re/im interleaved), outputs
// (kx, re/im) with F_r the real-expanded DFT over window columns.  Tile =
// (128 rows, 256 outputs): each MMA is M = 128 by N = 256 by K = 16.  Warp 0
// streams 64-element K chunks of both operands through a 4-stage mbarrier
// ring, warp 1 issues the MMAs into two 256-column TMEM accumulators, warps
// 2-9 (one per output half and lane quarter) write each lane's (re, im)
// pairs of its frame and window row straight into the column GEMM's K-major
// operand Hh[c][kx][t][2 jw + re/im], skipping rows past the channel's
// occupied rows (they stay zero).
constexpr int kRowN = 256;                       // outputs per tile
constexpr int kRowStages = 4;
constexpr uint32_t kRowStageBytes = kChunkBytes + kRowN * 128;   // A chunk + B chunk
size_t tc_rows_smem_bytes() { return 1024 + kRowStages * kRowStageBytes + 256; }

template <bool kBf16>
__global__ void __launch_bounds__(kTcThreads, 1)
    tc_rows_kernel(const __grid_constant__ CUtensorMap tm_gh, const __grid_constant__ CUtensorMap tm_fr,
                   const TcArgs A, int nt) {
  using T = typename std::conditional<kBf16, __nv_bfloat16, __half>::type;
  extern __shared__ __align__(1024) unsigned char tr_smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(tr_smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  constexpr int S = kRowStages;
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + S * kRowStageBytes);
  // bars: [0, S) full; [S, 2S) empty; 2S + {0,1} tmem_full; 2S + {2,3}
  // tmem_empty; 2S + 4 drain
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 2 * S + 6);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int C = A.u.n_chan, N = A.u.grid_n;
  const long long rows = static_cast<long long>(nt) * C * A.r_alloc;
  const long long mt_n = (rows + kTile - 1) / kTile;
  const int nt2 = 2 * N / kRowN;
  const long long tiles = mt_n * nt2;
  const int kc_n = A.kr / 64;

  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(smem_u32(bars + i), 1);
      mbar_init(smem_u32(bars + S + i), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(bars + 2 * S + i), 1);
      mbar_init(smem_u32(bars + 2 * S + 2 + i), kEpiWarps);
    }
    mbar_init(smem_u32(bars + 2 * S + 4), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kColTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tm_gh)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tm_fr)) : "memory");
      long long it = 0;
      bool ok = true;
      for (long long u = blockIdx.x; ok && u < tiles; u += gridDim.x) {
        const int mt = static_cast<int>(u / nt2), ot = static_cast<int>(u % nt2);
        for (int kc = 0; kc < kc_n; ++kc, ++it) {
          const int s = static_cast<int>(it % S);
          const uint32_t ph = static_cast<uint32_t>((it / S) & 1);
          if (!mbar_wait(smem_u32(bars + S + s), ph ^ 1, abort_flag, A.err)) {
            ok = false;
            break;
          }
          const uint32_t bfull = smem_u32(bars + s);
          mbar_expect_tx(bfull, kRowStageBytes);
          unsigned char* st = base + s * kRowStageBytes;
          tma_load_2d(smem_u32(st), &tm_gh, kc * 64, mt * kTile, bfull);
          tma_load_2d(smem_u32(st + kChunkBytes), &tm_fr, kc * 64, ot * kRowN, bfull);
        }
      }
      if (*abort_flag) {
        // let the copies still in flight land before the CTA exits (bounded)
        for (long long j = it > S ? it - S : 0; j < it; ++j) {
          const uint32_t bar = smem_u32(bars + j % S), ph = static_cast<uint32_t>((j / S) & 1);
          for (int w = 0; w < (1 << 22) && !mbar_try(bar, ph); ++w) {
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | ((kBf16 ? 1u : 0u) << 7) | ((kBf16 ? 1u : 0u) << 10) |
                             (static_cast<uint32_t>(kRowN >> 3) << 17) | (static_cast<uint32_t>(kTile >> 4) << 24);
      long long it = 0;
      int i = 0;
      bool ok = true;
      for (long long u = blockIdx.x; ok && u < tiles; u += gridDim.x, ++i) {
        const int acc = i & 1;
        const uint32_t aph = (i >> 1) & 1;
        if (!mbar_wait(smem_u32(bars + 2 * S + 2 + acc), aph ^ 1, abort_flag, A.err)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(acc * kRowN);
        for (int kc = 0; kc < kc_n; ++kc, ++it) {
          const int s = static_cast<int>(it % S);
          const uint32_t ph = static_cast<uint32_t>((it / S) & 1);
          if (!mbar_wait(smem_u32(bars + s), ph, abort_flag, A.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(base + s * kRowStageBytes), b0 = a0 + kChunkBytes;
#pragma unroll
          for (int k = 0; k < 4; ++k)
            mma_f16(d_tmem, sdesc_sw128(a0 + k * 32), sdesc_sw128(b0 + k * 32), idesc, (kc | k) != 0);
          mma_commit(smem_u32(bars + S + s));
        }
        if (ok) mma_commit(smem_u32(bars + 2 * S + acc));
      }
      if (*abort_flag) {
        // wait (bounded) for the MMAs already issued before TMEM is freed
        const uint32_t drain = smem_u32(bars + 2 * S + 4);
        mma_commit(drain);
        for (int w = 0; w < (1 << 22) && !mbar_try(drain, 0); ++w) {
        }
      }
    }
  } else {
    const int q = warp & 3;                        // TMEM lane quarter
    const int half = (warp - 2) >> 2;              // which 128 outputs of the tile
    T* hh = static_cast<T*>(A.hh);
    int i = 0;
    for (long long u = blockIdx.x; u < tiles; u += gridDim.x, ++i) {
      const int acc = i & 1;
      const uint32_t aph = (i >> 1) & 1;
      if (!mbar_wait(smem_u32(bars + 2 * S + acc), aph, abort_flag, A.err)) break;
      tc_fence_after();
      const int mt = static_cast<int>(u / nt2), ot = static_cast<int>(u % nt2);
      const long long row = static_cast<long long>(mt) * kTile + q * 32 + lane;
      const long long f = row / A.r_alloc;                 // frame tl * C + c
      const int jw = static_cast<int>(row - f * A.r_alloc);
      const int c = static_cast<int>(f % C), tl = static_cast<int>(f / C);
      const bool live = row < rows && jw < __ldg(A.win4 + (row < rows ? c : 0)).y;
#pragma unroll
      for (int ch = 0; ch < kTile / 32; ++ch) {
        float v[32];
        tmem_ld32(tmem_base + (static_cast<uint32_t>(q * 32) << 16) +
                      static_cast<uint32_t>(acc * kRowN + half * kTile + ch * 32),
                  v);
        if (live) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int kx = (ot * kRowN + half * kTile + ch * 32) / 2 + j;
            store_lp(hh + ((static_cast<size_t>(c) * N + kx) * A.tb_cap + tl) * A.kp + 2 * jw, v[2 * j], v[2 * j + 1]);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(bars + 2 * S + 2 + acc));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kColTmemCols)
                 : "memory");
  }
}

template <int N, typename T>
cudaError_t grid_lp_n(const TcArgs& a, long long t0, int nt, int sms, cudaStream_t s) {
  const size_t es_bytes = static_cast<size_t>(a.u.n_ant) * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(grid_lp_kernel<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(es_bytes));
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, grid_lp_kernel<N, T>, kLBT, es_bytes);
  if (e != cudaSuccess) return e;
  const long long frames = static_cast<long long>(nt) * a.u.n_chan;
  long long rb = static_cast<long long>(per_sm > 0 ? per_sm : 1) * sms;
  if (rb > frames) rb = frames;
  grid_lp_kernel<N, T><<<static_cast<unsigned>(rb), kLBT, es_bytes, s>>>(a, t0, nt);
  return cudaGetLastError();
}

}  // namespace

bool tc_supported(int n, int rows_alloc) { return (n == 128 || n == 256) && 2 * rows_alloc <= 256; }

int tc_kp(int rows_alloc) { return ((2 * rows_alloc + 63) / 64) * 64; }

size_t tc_smem(int kp) { return tc_smem_bytes(kp); }

cudaError_t tc_prepare(bool bf16, size_t smem) {
  cudaError_t e = bf16 ? cudaFuncSetAttribute(tc_rows_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              static_cast<int>(tc_rows_smem_bytes()))
                       : cudaFuncSetAttribute(tc_rows_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              static_cast<int>(tc_rows_smem_bytes()));
  if (e != cudaSuccess) return e;
  if (bf16)
    return cudaFuncSetAttribute(tc_cols_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(smem));
  return cudaFuncSetAttribute(tc_cols_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(smem));
}

// Tensor maps over the window grid Gh [rows_cap][kr] and the row DFT [2N][kr].
bool tc_make_row_maps(void* gh, void* dftr, long long rows_cap, int n, int kr, bool bf16, void* tm_gh,
                      void* tm_fr) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return false;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const CUtensorMapDataType dt = bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(kr) * 2};
  cuuint32_t box[2] = {64, static_cast<cuuint32_t>(kTile)};
  cuuint32_t es[2] = {1, 1};
  cuuint64_t dg[2] = {static_cast<cuuint64_t>(kr), static_cast<cuuint64_t>(rows_cap)};
  if (encode(static_cast<CUtensorMap*>(tm_gh), dt, 2, gh, dg, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  cuuint64_t df[2] = {static_cast<cuuint64_t>(kr), static_cast<cuuint64_t>(2 * n)};
  cuuint32_t box_fr[2] = {64, static_cast<cuuint32_t>(kRowN)};   // 256 outputs per tile
  return encode(static_cast<CUtensorMap*>(tm_fr), dt, 2, dftr, df, strides, box_fr, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_tc_batch(const TcArgs& a, const void* tm_dft, const void* tm_data, long long t0, int nt,
                            int sms, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (a.u.do_cal) e = cudaMemsetAsync(a.u.pix, 0, static_cast<size_t>(nt) * a.u.n_chan * sizeof(float2), s);
  if (e != cudaSuccess) return e;
  if (a.bf16) e = (a.u.grid_n == 128) ? grid_lp_n<128, __nv_bfloat16>(a, t0, nt, sms, s)
                                      : grid_lp_n<256, __nv_bfloat16>(a, t0, nt, sms, s);
  else e = (a.u.grid_n == 128) ? grid_lp_n<128, __half>(a, t0, nt, sms, s)
                               : grid_lp_n<256, __half>(a, t0, nt, sms, s);
  if (e != cudaSuccess) return e;
  {
    const long long rows = static_cast<long long>(nt) * a.u.n_chan * a.r_alloc;
    const long long tiles = (rows + kTile - 1) / kTile * (2 * a.u.grid_n / kRowN);
    const int grid = static_cast<int>(tiles < sms ? tiles : sms);
    const CUtensorMap* tg = static_cast<const CUtensorMap*>(a.tm_gh);
    const CUtensorMap* tf = static_cast<const CUtensorMap*>(a.tm_fr);
    if (a.bf16) tc_rows_kernel<true><<<grid, kTcThreads, tc_rows_smem_bytes(), s>>>(*tg, *tf, a, nt);
    else tc_rows_kernel<false><<<grid, kTcThreads, tc_rows_smem_bytes(), s>>>(*tg, *tf, a, nt);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const int MB = 2 * a.u.grid_n / kTile;           // 128-row DFT tiles
  const int grid = (sms / MB) * MB;
  const size_t smem = tc_smem_bytes(a.kp);
  const CUtensorMap* td = static_cast<const CUtensorMap*>(tm_dft);
  const CUtensorMap* tt = static_cast<const CUtensorMap*>(tm_data);
  if (a.bf16) tc_cols_kernel<true><<<grid, kTcThreads, smem, s>>>(*td, *tt, a, nt);
  else tc_cols_kernel<false><<<grid, kTcThreads, smem, s>>>(*td, *tt, a, nt);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (a.u.do_cal) e = launch_correlate(a.u, t0, nt, s);
  return e;
}

cudaError_t xe_prepare() {
  return cudaFuncSetAttribute(xengine_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(xe_smem_bytes()));
}

bool xe_make_map(void* z, int n_chan, int na_p, int tp, void* tm) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return false;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(tp), static_cast<cuuint64_t>(n_chan) * 2 * na_p};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(tp) * 2};
  cuuint32_t box[2] = {64, static_cast<cuuint32_t>(kTile)};
  cuuint32_t es[2] = {1, 1};
  return encode(static_cast<CUtensorMap*>(tm), CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, z, dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_xengine_tc(const XeTcArgs& a, const void* volt, long long t0, int nt, void* z, const void* tm,
                              int sms, cudaStream_t s) {
  dim3 pg(static_cast<unsigned>(a.n_chan), static_cast<unsigned>(a.na_p / 32), static_cast<unsigned>(a.tp / 64));
  xe_pack_kernel<<<pg, 256, 0, s>>>(static_cast<const unsigned char*>(volt), t0, nt, a.n_chan, a.n_ant, a.na_p,
                                    a.tp, static_cast<__half*>(z));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nb = 2 * a.na_p / kTile, nbp = (nb + 1) / 2;
  long long pairs = 0;
  for (int i = 0; i < nb; ++i) pairs += nbp - i / 2;
  const long long tiles = static_cast<long long>(a.n_chan) * pairs;
  const int grid = static_cast<int>(tiles < sms ? tiles : sms);
  xengine_tc_kernel<<<grid, kXeThreads, xe_smem_bytes(), s>>>(*static_cast<const CUtensorMap*>(tm), a);
  return cudaGetLastError();
}

// Tensor maps over the DFT matrix [2N][kp] and the spectra [C*N][tb_cap][kp].
bool tc_make_maps(void* dft, void* hh, int n, int n_chan, int tb_cap, int kp, bool bf16, void* tm_dft,
                  void* tm_data) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return false;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const CUtensorMapDataType dt = bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  {
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(kp), static_cast<cuuint64_t>(2 * n)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(kp) * 2};
    cuuint32_t box[2] = {64, static_cast<cuuint32_t>(kTile)};
    cuuint32_t es[2] = {1, 1};
    if (encode(static_cast<CUtensorMap*>(tm_dft), dt, 2, dft, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  {
    cuuint64_t dims[3] = {static_cast<cuuint64_t>(kp), static_cast<cuuint64_t>(tb_cap),
                          static_cast<cuuint64_t>(n_chan) * n};
    cuuint64_t strides[2] = {static_cast<cuuint64_t>(kp) * 2, static_cast<cuuint64_t>(kp) * 2 * tb_cap};
    cuuint32_t box[3] = {64, static_cast<cuuint32_t>(kTile), 2};   // columns kx, kx + 1
    cuuint32_t es[3] = {1, 1, 1};
    if (encode(static_cast<CUtensorMap*>(tm_data), dt, 3, hh, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

}  // namespace epic
