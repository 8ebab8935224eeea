// Plain (unfused) FP32 EPIC imaging path for any grid side N = 32..512.
//
// Each step is its own kernel and hands its result to the next through HBM,
// one batch of frames at a time (frame f = t_local * C + c):
//   rows_window    per step of F frames of one channel: gain correction
//                  (Eq. 8) of every antenna into shared memory, then gridding
//                  (Eq. 9) as a gather straight into the FFT lanes of every
//                  occupied grid row (host-planned tap lists, copied to
//                  shared memory once per channel when they fit) and the
//                  N-point row FFT, written transposed into Hs[f][kx][row];
//   cols_window    N-point FFT of every column (Eq. 10), |E|^2 summed over
//                  the batch's frames in registers and added to the image;
//                  the owner of the calibrator pixel stores it per frame.
//                  Each CTA's block of columns of the next frame is staged
//                  into shared memory by one TMA bulk copy while the current
//                  frame is transformed;
//   correlate      EPICal K_a += E_a conj(P), P_a += |E_a|^2 (Eqs. 12, 15).
// The grid is held in window coordinates (first occupied row and column of
// the channel at 0): the shift multiplies every image pixel by a phase,
// which |E|^2 does not see and the calibrator pixel gets back (plan table
// pixph).  Every FFT therefore has at most NZ non-zero inputs per lane and
// uses the pruned first-stage DFT.  The centring signs and 1/Na are folded
// into the gridding weights.
#include "epic_fft.cuh"
#include "epic_internal.h"

#include <cstdint>

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

constexpr int kUBT = 256;          // threads per CTA of the FFT kernels
constexpr int kRowFrames = 2;      // frames per step of the row kernel

__device__ __forceinline__ float2 load_volt_u(const void* volt, int fmt, size_t idx) {
  if (fmt == 0) {
    const unsigned b = __ldg(static_cast<const unsigned char*>(volt) + idx);
    const int re = static_cast<int>(b << 24) >> 28;
    const int im = static_cast<int>(b << 28) >> 28;
    return make_float2(static_cast<float>(re), static_cast<float>(im));
  }
  return __ldg(static_cast<const float2*>(volt) + idx);
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Bytes of the row kernel's per-channel gather table in shared memory.
__host__ __device__ inline size_t row_table_bytes(int rows_alloc, int n1, int cw, int gmax) {
  return static_cast<size_t>(rows_alloc) * n1 * cw * 16 + static_cast<size_t>(rows_alloc) * n1 * 4 +
         static_cast<size_t>(gmax) * 8;
}

// ---- gridding + row FFTs: a CTA owns a contiguous range of (channel, time) items ----
// Lane (window row, n1) of a row FFT sums w * E'_a over its tap list for
// each column block j (window column n1 + N1 j).  Whole warps step through
// the (frame, row) tasks together; lanes past the last task transform zeros
// and store nothing.
// Raw sample of one antenna: the 4-bit byte or the complex64 value.
struct RawU {
  unsigned b;
  float2 f;
};

__device__ __forceinline__ RawU fetch_raw(const void* volt, int fmt, size_t idx) {
  RawU r;
  if (fmt == 0) {
    r.b = __ldg(static_cast<const unsigned char*>(volt) + idx);
    r.f = make_float2(0.f, 0.f);
  } else {
    r.b = 0;
    r.f = __ldg(static_cast<const float2*>(volt) + idx);
  }
  return r;
}

__device__ __forceinline__ float2 unpack_raw(const RawU& r, int fmt) {
  if (fmt == 0) {
    const int re = static_cast<int>(r.b << 24) >> 28;
    const int im = static_cast<int>(r.b << 28) >> 28;
    return make_float2(static_cast<float>(re), static_cast<float>(im));
  }
  return r.f;
}

// Row stride of channel c's transposed spectra: its occupied rows rounded up
// to even (16-byte rows for the bulk copies of the column kernel).
__device__ __forceinline__ int chan_rs(int R) { return (R + 1) & ~1; }

// ---- gridding + row FFTs: a CTA owns a contiguous range of (channel, time) items ----
// Lane (window row, n1) of a row FFT sums w * E'_a over its tap list for
// each column block j (window column n1 + N1 j).  Whole warps step through
// the (frame, row) tasks together; lanes past the last task transform zeros
// and store nothing.  A step holds A.row_frames (1 or 2) consecutive
// samples of one channel; for Na <= 512 the next step's raw voltages and
// gain multipliers are loaded into registers while this step's rows are
// transformed.
template <int N, int NZ, bool TS>
__device__ __forceinline__ void rows_body(const UnfusedArgs& A, long long t0, int nt, const float2* tw,
                                          float2* zbuf, unsigned char* rsm, int cta, int ncta) {
  constexpr int N1 = UCfg<N>::N1, N2 = UCfg<N>::N2, H = N2 / N1;
  constexpr int GROUPS = kUBT / N1, GPW = 32 / N1;
  constexpr int CW = (N2 + 15) / 16;               // uint4 words of group lengths per lane
  constexpr int PF = 2;                            // antennas per thread held for the next step
  using X = fft::Xchg<N1, N2>;
  const int C = A.n_chan, Na = A.n_ant;
  const int F = A.row_frames;
  float2* Es = reinterpret_cast<float2*>(rsm);      // [kRowFrames][Na] E / g of the step's frames
  uint4* scnt = reinterpret_cast<uint4*>(rsm + ((static_cast<size_t>(kRowFrames) * Na * 8 + 15) &
                                                ~static_cast<size_t>(15)));
  int* sofs = reinterpret_cast<int*>(scnt + static_cast<size_t>(A.rows_alloc) * N1 * CW);
  uint2* sent = reinterpret_cast<uint2*>(sofs + ((A.rows_alloc * N1 + 1) & ~1));
  const int g = threadIdx.x / N1, n1 = threadIdx.x % N1;
  float2* z = zbuf + g * X::ZG;
  const long long frames = static_cast<long long>(nt) * C;
  const long long per = (frames + ncta - 1) / ncta;
  const long long ib = static_cast<long long>(cta) * per;
  const long long ie = ib + per < frames ? ib + per : frames;
  const bool regpf = Na <= PF * kUBT;
  // the step starting at item `it`: channel, first sample, frames
  auto step_of = [&](long long it, int* c, int* tl) {
    *c = static_cast<int>(it / nt);
    *tl = static_cast<int>(it - static_cast<long long>(*c) * nt);
    int nf = F;
    if (nf > nt - *tl) nf = nt - *tl;
    if (nf > ie - it) nf = static_cast<int>(ie - it);
    return nf;
  };
  RawU nxt[kRowFrames][PF];
  float2 wn[PF];
  if (regpf && ib < ie) {
    int c, tl;
    const int nf = step_of(ib, &c, &tl);
#pragma unroll
    for (int i = 0; i < PF; ++i) {
      const int a = threadIdx.x + kUBT * i;
      wn[i] = a < Na ? __ldg(A.wgain + static_cast<size_t>(c) * Na + a) : make_float2(0.f, 0.f);
#pragma unroll
      for (int f = 0; f < kRowFrames; ++f)
        if (a < Na && f < nf)
          nxt[f][i] = fetch_raw(A.volt, A.input_fmt, (static_cast<size_t>(t0 + tl + f) * C + c) * Na + a);
    }
  }
  int cur_c = -1;
  for (long long it = ib; it < ie;) {
    int c, tl;
    const int nf = step_of(it, &c, &tl);
    const float vs = A.vscale ? __ldg(A.vscale + c) : 1.0f;
    __syncthreads();                                // previous step's gathers are done
    if (TS && c != cur_c) {
      const int gb = __ldg(A.gbase + c), gn = __ldg(A.gbase + c + 1) - gb;
      const int nl = A.rows_alloc * N1;
      for (int i = threadIdx.x; i < gn; i += kUBT) sent[i] = __ldg(A.gent + gb + i);
      for (int i = threadIdx.x; i < nl; i += kUBT) sofs[i] = __ldg(A.gofs + static_cast<size_t>(c) * nl + i);
      for (int i = threadIdx.x; i < nl * CW; i += kUBT)
        scnt[i] = __ldg(A.gcnt + static_cast<size_t>(c) * nl * CW + i);
    }
    cur_c = c;
    if (regpf) {
#pragma unroll
      for (int i = 0; i < PF; ++i) {
        const int a = threadIdx.x + kUBT * i;
#pragma unroll
        for (int f = 0; f < kRowFrames; ++f)
          if (a < Na && f < nf) {
            const float2 e = unpack_raw(nxt[f][i], A.input_fmt);
            Es[f * Na + a] = cmul(make_float2(e.x * vs, e.y * vs), wn[i]);
          }
      }
    } else {
      for (int f = 0; f < nf; ++f)
        for (int a = threadIdx.x; a < Na; a += kUBT) {
          const size_t vidx = (static_cast<size_t>(t0 + tl + f) * C + c) * Na + a;
          const float2 e = load_volt_u(A.volt, A.input_fmt, vidx);
          Es[f * Na + a] = cmul(make_float2(e.x * vs, e.y * vs), __ldg(A.wgain + static_cast<size_t>(c) * Na + a));
        }
    }
    __syncthreads();
    // the next step's voltages: into registers (Na <= 512) or L2, while
    // this step's rows are transformed
    if (it + nf < ie) {
      int c2, tl2;
      const int nf2 = step_of(it + nf, &c2, &tl2);
      if (regpf) {
#pragma unroll
        for (int i = 0; i < PF; ++i) {
          const int a = threadIdx.x + kUBT * i;
          if (a < Na) wn[i] = __ldg(A.wgain + static_cast<size_t>(c2) * Na + a);
#pragma unroll
          for (int f = 0; f < kRowFrames; ++f)
            if (a < Na && f < nf2)
              nxt[f][i] = fetch_raw(A.volt, A.input_fmt, (static_cast<size_t>(t0 + tl2 + f) * C + c2) * Na + a);
        }
      } else {
        const size_t esz = A.input_fmt == 0 ? 1 : sizeof(float2);
        for (int f = 0; f < nf2; ++f) {
          const uintptr_t lo = reinterpret_cast<uintptr_t>(A.volt) +
                               ((static_cast<size_t>(t0 + tl2 + f) * C + c2) * Na) * esz;
          for (uintptr_t q = (lo & ~static_cast<uintptr_t>(127)) + static_cast<uintptr_t>(threadIdx.x) * 128;
               q < lo + Na * esz; q += kUBT * 128)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(q));
        }
      }
    }
    const int R = __ldg(A.win + c).y;
    const int rsc = chan_rs(R);
    const int nl = A.rows_alloc * N1;
    const int* gofs = TS ? sofs : A.gofs + static_cast<size_t>(c) * nl;
    const uint4* gcnt = TS ? scnt : A.gcnt + static_cast<size_t>(c) * nl * CW;
    const uint2* gent = TS ? sent : A.gent + __ldg(A.gbase + c);
    const int ntask = nf * R;
    for (int rb = g - g % GPW; rb < ntask; rb += GROUPS) {
      const int task = rb + g % GPW;
      const bool live = task < ntask;
      const int f = live ? task / R : 0;
      const int row = live ? task - f * R : 0;
      const float2* Ef = Es + f * Na;
      float2 v[N2];
#pragma unroll
      for (int j = 0; j < N2; ++j) v[j] = make_float2(0.f, 0.f);
      if (live) {
        const int li = row * N1 + n1;
        int e = gofs[li];
        unsigned cv[4 * CW];
#pragma unroll
        for (int w = 0; w < CW; ++w) {
          const uint4 q = gcnt[static_cast<size_t>(li) * CW + w];
          cv[4 * w] = q.x;
          cv[4 * w + 1] = q.y;
          cv[4 * w + 2] = q.z;
          cv[4 * w + 3] = q.w;
        }
#pragma unroll
        for (int j = 0; j < NZ; ++j) {
          const int cj = static_cast<int>((cv[j >> 2] >> (8 * (j & 3))) & 255u);
          float2 sum = make_float2(0.f, 0.f);
          for (int k = 0; k < cj; ++k) {
            const uint2 en = TS ? gent[e + k] : __ldg(gent + e + k);
            const float2 x = Ef[en.x];
            const float w = __uint_as_float(en.y);
            sum.x = fmaf(w, x.x, sum.x);
            sum.y = fmaf(w, x.y, sum.y);
          }
          e += cj;
          v[j] = sum;
        }
      }
      fft::fft_lanes_p<N1, N2, NZ>(v, n1, z, tw, kFull);
      if (live) {
        const size_t fr = static_cast<size_t>(tl + f) * C + c;
        float2* dst = A.spec + fr * N * A.rs + row;
#pragma unroll
        for (int h = 0; h < H; ++h)
#pragma unroll
          for (int k1 = 0; k1 < N1; ++k1)        // streaming stores: keep L2 for the tap lists
            __stcs(dst + static_cast<size_t>(n1 + N1 * h + N2 * k1) * rsc, v[h * N1 + k1]);
      }
    }
    it += nf;
  }
}

template <int N, int NZ, bool TS>
__global__ void __launch_bounds__(kUBT, (N <= 128 ? 3 : 2))
    rows_window_kernel(const UnfusedArgs A, long long t0, int nt) {
  constexpr int N1 = UCfg<N>::N1, N2 = UCfg<N>::N2;
  __shared__ float2 tw[N];                          // [k2][n1]: e^{+2 pi i n1 k2 / N}
  __shared__ float2 zbuf[(kUBT / N1) * fft::Xchg<N1, N2>::ZG];
  extern __shared__ __align__(16) unsigned char rsm[];
  for (int i = threadIdx.x; i < N; i += kUBT) tw[i] = A.twid[(i % N1) * (i / N1)];
  rows_body<N, NZ, TS>(A, t0, nt, tw, zbuf, rsm, blockIdx.x, gridDim.x);   // its first step syncs
}

// Bounded wait of one thread on an mbarrier phase; false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  for (int i = 0; i < (1 << 22); ++i) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// ---- column FFTs + |E|^2: unit = (channel, block of GROUPS columns, time segment) ----
// STAGE (N <= 256): thread 0 stages the unit's column block of frame i + 1
// (GROUPS x rs contiguous float2 of Hs) by a TMA bulk copy into the other of
// two shared-memory slots while frame i is transformed; it alone waits on
// the slot's mbarrier (bounded), then a CTA barrier hands the slot to all
// warps.  N = 512 reads the columns from global memory (the two slots and
// the FFT exchange would not leave room for two CTAs per SM).
// COH (persistent form): the spectra were written by other SMs earlier in
// the same launch, so they are read around L1 (ld.global.cg), and image
// updates are atomics (the unit-to-CTA mapping may change between batches).
template <int N, int NZ, bool STAGE, bool COH = false>
__device__ __forceinline__ bool cols_body(const UnfusedArgs& A, int nt, int segs, const float2* tw, float2* zbuf,
                                          float2* slot, uint64_t* bars, volatile int* abort_flag,
                                          uint32_t (&uses)[2], int cta, int ncta) {
  constexpr int N1 = UCfg<N>::N1, N2 = UCfg<N>::N2, H = N2 / N1;
  constexpr int GROUPS = kUBT / N1;
  constexpr int CBLK = (N + GROUPS - 1) / GROUPS;   // column blocks per channel
  constexpr int NCOL = N < GROUPS ? N : GROUPS;     // columns per block
  using X = fft::Xchg<N1, N2>;
  const int g = threadIdx.x / N1, n1 = threadIdx.x % N1;
  const int lane = threadIdx.x & 31;
  const unsigned gmask = fft::group_mask<N1>(lane);
  float2* z = zbuf + g * X::ZG;
  const int C = A.n_chan, rs = A.rs;                // frame stride N * rs
  const int units = C * CBLK * segs;
  bool ok = true;
  for (int u = cta; u < units && ok; u += ncta) {
    const int s = u % segs;
    const int cb = (u / segs) % CBLK;
    const int c = u / (segs * CBLK);
    const int kx = cb * GROUPS + g;
    const int tb = nt * s / segs, te = nt * (s + 1) / segs;
    const int R = __ldg(A.win + c).y;
    const int rsc = chan_rs(R);                      // this channel's row stride in Hs
    const uint32_t block_bytes = static_cast<uint32_t>(NCOL) * rsc * sizeof(float2);
    const bool col_ok = kx < N;
    float acc[N2];
#pragma unroll
    for (int q = 0; q < N2; ++q) acc[q] = 0.f;
    const bool pix_group = A.do_cal && kx == A.k0x;
    const int pq = A.k0y / N1;
    const int pslot = (pq % H) * N1 + pq / H;
    const float2 pph = A.do_cal ? __ldg(A.pixph + c) : make_float2(1.f, 0.f);
    if (STAGE && threadIdx.x == 0 && tb < te) {
      const float2* src = A.spec + (static_cast<size_t>(tb) * C + c) * N * rs + static_cast<size_t>(cb) * GROUPS * rsc;
      bulk_load(smem_addr(slot), src, block_bytes, smem_addr(bars));
    }
    for (int tl = tb; tl < te; ++tl) {
      const int i = tl - tb;
      const int sl = i & 1;
      if (STAGE) {
        if (threadIdx.x == 0) {
          if (tl + 1 < te) {                          // the other slot was freed by the last barrier
            const float2* src = A.spec + (static_cast<size_t>(tl + 1) * C + c) * N * rs +
                                static_cast<size_t>(cb) * GROUPS * rsc;
            bulk_load(smem_addr(slot + static_cast<size_t>(sl ^ 1) * NCOL * rs), src, block_bytes,
                      smem_addr(bars + (sl ^ 1)));
          }
          if (!mbar_wait_bounded(smem_addr(bars + sl), uses[sl] & 1u)) {
            *abort_flag = 1;
            atomicExch(A.err, 1);
          }
          ++uses[sl];
        }
        __syncthreads();
        if (*abort_flag) {
          ok = false;
          break;
        }
      }
      if (col_ok) {
        const float2* col = STAGE ? slot + static_cast<size_t>(sl) * NCOL * rs + static_cast<size_t>(g) * rsc
                                  : A.spec + (static_cast<size_t>(tl) * C + c) * N * rs + static_cast<size_t>(kx) * rsc;
        float2 v[N2];
#pragma unroll
        for (int j = 0; j < N2; ++j) {
          const int jw = n1 + N1 * j;
          v[j] = (j < NZ && jw < R) ? (STAGE ? col[jw] : (COH ? __ldcg(col + jw) : __ldcs(col + jw)))
                                    : make_float2(0.f, 0.f);
        }
        fft::fft_lanes_p<N1, N2, NZ>(v, n1, z, tw, gmask);
#pragma unroll
        for (int q = 0; q < N2; ++q) acc[q] += v[q].x * v[q].x + v[q].y * v[q].y;
        if (pix_group && n1 == A.k0y % N1) {
#pragma unroll
          for (int q = 0; q < N2; ++q)
            if (q == pslot) A.pix[static_cast<size_t>(tl) * C + c] = cmul(v[q], pph);
        }
      }
      if (STAGE) __syncthreads();                    // slot sl free for frame tl + 2
    }
    if (!ok || !col_ok) continue;
    double* img = A.image + static_cast<size_t>(c) * N * N;
#pragma unroll
    for (int h = 0; h < H; ++h)
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) {
        const int ky = n1 + N1 * h + N2 * k1;
        const double v = static_cast<double>(acc[h * N1 + k1]) * A.img_scale;
        if (segs == 1 && !COH) img[ky * N + kx] += v;
        else atomicAdd(img + ky * N + kx, v);
      }
  }
  // after a timeout: let this thread's copies still in flight land (bounded)
  if (STAGE && !ok && threadIdx.x == 0)
    for (int sl = 0; sl < 2; ++sl) mbar_wait_bounded(smem_addr(bars + sl), uses[sl] & 1u);
  return ok;
}

template <int N, int NZ, bool STAGE>
__global__ void __launch_bounds__(kUBT, (N <= 128 ? 3 : 2)) cols_window_kernel(const UnfusedArgs A, int nt, int segs) {
  constexpr int N1 = UCfg<N>::N1, N2 = UCfg<N>::N2;
  __shared__ float2 tw[N];
  __shared__ float2 zbuf[(kUBT / N1) * fft::Xchg<N1, N2>::ZG];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ int abort_flag;
  extern __shared__ __align__(128) float2 slot[];   // [2][NCOL][rs]
  for (int i = threadIdx.x; i < N; i += kUBT) tw[i] = A.twid[(i % N1) * (i / N1)];
  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bars + s)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_flag = 0;
  }
  __syncthreads();
  uint32_t uses[2] = {0u, 0u};                     // completed phases per slot (thread 0)
  cols_body<N, NZ, STAGE>(A, nt, segs, tw, zbuf, slot, bars, &abort_flag, uses, blockIdx.x, gridDim.x);
}

// ---- EPICal correlation: one thread per (channel, antenna, time segment) ----
__device__ __forceinline__ void corr_item(const UnfusedArgs& A, long long t0, int nt, int i, int sy, int nsy) {
  const int Na = A.n_ant, C = A.n_chan;
  const int c = i / Na, a = i % Na;
  if (__ldg(A.cell0 + i) < 0) return;
  const float vs = A.vscale ? __ldg(A.vscale + c) : 1.0f;
  const int tb = nt * sy / nsy, te = nt * (sy + 1) / nsy;
  float kr = 0.f, ki = 0.f, pp = 0.f;
  for (int tl = tb; tl < te; ++tl) {
    const size_t f = static_cast<size_t>(tl) * C + c;
    const float2 p = __ldcg(A.pix + f);            // written by another SM (persistent form)
    const float2 e0 = load_volt_u(A.volt, A.input_fmt, (static_cast<size_t>(t0 + tl) * C + c) * Na + a);
    const float2 e = make_float2(e0.x * vs, e0.y * vs);
    kr += e.x * p.x + e.y * p.y;
    ki += e.y * p.x - e.x * p.y;
    pp += e.x * e.x + e.y * e.y;
  }
  if (nsy == 1) {
    A.kacc[i].x += kr;
    A.kacc[i].y += ki;
    A.pacc[i] += pp;
  } else {
    atomicAdd(&A.kacc[i].x, static_cast<double>(kr));
    atomicAdd(&A.kacc[i].y, static_cast<double>(ki));
    atomicAdd(A.pacc + i, static_cast<double>(pp));
  }
}

__global__ void correlate_kernel(const UnfusedArgs A, long long t0, int nt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n_chan * A.n_ant) return;
  corr_item(A, t0, nt, i, blockIdx.y, gridDim.y);
}

// Time segments for the correlation: enough blocks to fill the GPU, at
// least 16 time samples each.
dim3 correlate_grid(int n_chan, int n_ant, int nt, int sms) {
  const int bx = (n_chan * n_ant + 255) / 256;
  int sy = 1;
  while (bx * sy < 4 * sms && nt / (2 * sy) >= 16) sy *= 2;
  return dim3(static_cast<unsigned>(bx), static_cast<unsigned>(sy));
}

// Grid-wide barrier of the persistent form (all CTAs co-resident: a
// cooperative launch).  Thread 0 of every CTA reads the generation, arrives
// on the counter; the last arriver resets the counter and advances the
// generation, the others wait for it with a bounded number of polls, after
// which the kernel's abort flag and the plan's error flag are raised and
// every CTA stops.  bar = {count, generation, abort}; limit = polls per
// wait (0: 2^22).
__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* err, int limit) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    volatile unsigned* vabort = bar + 2;
    const unsigned g = *vgen;
    __threadfence();
    int ok = *vabort == 0u;
    if (ok) {
      if (atomicAdd(bar, 1u) == gridDim.x - 1) {
        atomicExch(bar, 0u);
        __threadfence();
        atomicAdd(bar + 1, 1u);
      } else {
        int i = 0;
        const int lim = limit > 0 ? limit : (1 << 22);
        for (; i < lim && *vgen == g && *vabort == 0u; ++i) __nanosleep(64);
        if (*vgen == g) {
          ok = 0;
          atomicExch(bar + 2, 1u);
          atomicExch(err, 1);
        }
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// One launch for a whole epic_image call on the plain path: for every batch
// of samples the row phase, a grid barrier, the column phase, a grid
// barrier, the correlation phase (its result is read by no one before the
// next batch's column phase, two barriers later).  Gather tables through L1,
// column loads from global memory: the row and column phases then need the
// same shared memory (twiddles, FFT exchange) and fit side by side.
template <int N, int NZR, int NZC>
__global__ void __launch_bounds__(kUBT, (N <= 128 ? 3 : 2))
    unfused_persistent_kernel(const UnfusedArgs A, long long n_time, int nt_batch, unsigned* bar) {
  constexpr int N1 = UCfg<N>::N1, N2 = UCfg<N>::N2;
  constexpr int GROUPS = kUBT / N1;
  constexpr int CBLK = (N + GROUPS - 1) / GROUPS;
  __shared__ float2 tw[N];
  __shared__ float2 zbuf[GROUPS * fft::Xchg<N1, N2>::ZG];
  extern __shared__ __align__(16) unsigned char rsm[];
  for (int i = threadIdx.x; i < N; i += kUBT) tw[i] = A.twid[(i % N1) * (i / N1)];
  __syncthreads();
  __shared__ int unused_abort;
  uint32_t uses[2] = {0u, 0u};
  const int C = A.n_chan, Na = A.n_ant;
  for (long long t0 = 0; t0 < n_time; t0 += nt_batch) {
    const int nt = static_cast<int>(n_time - t0 < nt_batch ? n_time - t0 : nt_batch);
    rows_body<N, NZR, false>(A, t0, nt, tw, zbuf, rsm, blockIdx.x, gridDim.x);
    if (!grid_barrier(bar, A.err, A.wait_limit)) return;
    int segs = 1;
    while (C * CBLK * segs < A.cols_target * A.sms && segs * 8 <= nt) segs *= 2;
    cols_body<N, NZC, false, true>(A, nt, segs, tw, zbuf, nullptr, nullptr, &unused_abort, uses, blockIdx.x,
                                   gridDim.x);
    if (!grid_barrier(bar, A.err, A.wait_limit)) return;
    if (A.do_cal) {
      const int bx = (C * Na + 255) / 256;
      int sy = 1;
      while (bx * sy < 4 * A.sms && nt / (2 * sy) >= 16) sy *= 2;
      const long long items = static_cast<long long>(C) * Na * sy;
      for (long long k = static_cast<long long>(blockIdx.x) * kUBT + threadIdx.x; k < items;
           k += static_cast<long long>(gridDim.x) * kUBT)
        corr_item(A, t0, nt, static_cast<int>(k % (C * Na)), static_cast<int>(k / (C * Na)), sy);
    }
  }
}

template <int N, int NZR, int NZC>
cudaError_t persistent_launch(const UnfusedArgs& a, long long n_time, int nt_batch, unsigned* bar, int sms,
                              cudaStream_t s) {
  const size_t es = static_cast<size_t>(kRowFrames) * a.n_ant * sizeof(float2);
  auto kern = unfused_persistent_kernel<N, NZR, NZC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(es));
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kUBT, es);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  e = cudaMemsetAsync(bar, 0, 3 * sizeof(unsigned), s);   // count, generation, abort
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(per_sm * sms));
  cfg.blockDim = dim3(kUBT);
  cfg.dynamicSmemBytes = es;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a, n_time, nt_batch, bar);
}

template <int N>
cudaError_t launch_persistent_n(const UnfusedArgs& a, long long n_time, int nt_batch, unsigned* bar, int sms,
                                cudaStream_t s) {
  constexpr int N1 = UCfg<N>::N1, N2 = UCfg<N>::N2;
  if (a.max_cols <= N1 * (N2 / 2)) {
    if (a.rows_alloc <= N1 * (N2 / 2)) return persistent_launch<N, N2 / 2, N2 / 2>(a, n_time, nt_batch, bar, sms, s);
    return persistent_launch<N, N2 / 2, N2>(a, n_time, nt_batch, bar, sms, s);
  }
  if (a.rows_alloc <= N1 * (N2 / 2)) return persistent_launch<N, N2, N2 / 2>(a, n_time, nt_batch, bar, sms, s);
  return persistent_launch<N, N2, N2>(a, n_time, nt_batch, bar, sms, s);
}

template <int N, int NZ, bool TS>
cudaError_t rows_launch(const UnfusedArgs& a, long long t0, int nt, int sms, size_t smem, int per_sm,
                        cudaStream_t s) {
  const long long frames = static_cast<long long>(nt) * a.n_chan;
  long long rb = static_cast<long long>(per_sm > 0 ? per_sm : 1) * sms;
  const long long steps = (frames + a.row_frames - 1) / a.row_frames;
  if (rb > steps) rb = steps;
  rows_window_kernel<N, NZ, TS><<<static_cast<unsigned>(rb), kUBT, smem, s>>>(a, t0, nt);
  return cudaGetLastError();
}

// Shared memory, resident CTAs per SM and launch of the row kernel.  The
// gather table goes to shared memory when row_table is 1, or when it is -1
// and that keeps at least 3 CTAs per SM (2 for N >= 256); 0 reads it
// through L1.
template <int N, int NZ>
cudaError_t rows_dispatch(const UnfusedArgs& a, long long t0, int nt, int sms, cudaStream_t s) {
  constexpr int N1 = UCfg<N>::N1, N2 = UCfg<N>::N2, CW = (N2 + 15) / 16;
  const size_t es = static_cast<size_t>(kRowFrames) * a.n_ant * sizeof(float2);
  const size_t smem_ts = ((es + 15) & ~static_cast<size_t>(15)) + row_table_bytes(a.rows_alloc, N1, CW, a.gmax);
  int per_sm = 0;
  cudaError_t e = cudaSuccess;
  if (a.row_table != 0) {                           // -1: shared memory if that keeps the occupancy, 1: always
    e = cudaFuncSetAttribute(rows_window_kernel<N, NZ, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem_ts));
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rows_window_kernel<N, NZ, true>, kUBT, smem_ts);
    if (e == cudaSuccess && per_sm >= 1 && (a.row_table == 1 || per_sm >= (N <= 128 ? 3 : 2)))
      return rows_launch<N, NZ, true>(a, t0, nt, sms, smem_ts, per_sm, s);
    cudaGetLastError();
  }
  e = cudaFuncSetAttribute(rows_window_kernel<N, NZ, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(es));
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rows_window_kernel<N, NZ, false>, kUBT, es);
  if (e != cudaSuccess) return e;
  return rows_launch<N, NZ, false>(a, t0, nt, sms, es, per_sm, s);
}

template <int N, int NZ>
cudaError_t cols_launch(const UnfusedArgs& a, int nt, int sms, cudaStream_t s) {
  constexpr int GROUPS = kUBT / UCfg<N>::N1;
  constexpr int CBLK = (N + GROUPS - 1) / GROUPS;
  constexpr int NCOL = N < GROUPS ? N : GROUPS;
  constexpr bool STAGE = N <= 256;
  const size_t smem = STAGE ? static_cast<size_t>(2) * NCOL * a.rs * sizeof(float2) : 0;
  cudaError_t e = cudaFuncSetAttribute(cols_window_kernel<N, NZ, STAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cols_window_kernel<N, NZ, STAGE>, kUBT, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const int base_units = a.n_chan * CBLK;
  int segs = 1;
  while (base_units * segs < a.cols_target * sms && segs * 8 <= nt) segs *= 2;
  const int units = base_units * segs;
  const int cb = units < sms * per_sm ? units : sms * per_sm;
  cols_window_kernel<N, NZ, STAGE><<<cb, kUBT, smem, s>>>(a, nt, segs);
  return cudaGetLastError();
}

template <int N>
cudaError_t launch_unfused_n(const UnfusedArgs& a, long long t0, int nt, int sms, cudaStream_t s) {
  constexpr int N1 = UCfg<N>::N1, N2 = UCfg<N>::N2;
  // row FFTs pruned by the widest channel's occupied columns, column FFTs by
  // its occupied rows
  cudaError_t e;
  if (a.max_cols <= N1 * (N2 / 4)) e = rows_dispatch<N, N2 / 4>(a, t0, nt, sms, s);
  else if (a.max_cols <= N1 * (N2 / 2)) e = rows_dispatch<N, N2 / 2>(a, t0, nt, sms, s);
  else e = rows_dispatch<N, N2>(a, t0, nt, sms, s);
  if (e != cudaSuccess) return e;
  if (a.rows_alloc <= N1 * (N2 / 4)) e = cols_launch<N, N2 / 4>(a, nt, sms, s);
  else if (a.rows_alloc <= N1 * (N2 / 2)) e = cols_launch<N, N2 / 2>(a, nt, sms, s);
  else e = cols_launch<N, N2>(a, nt, sms, s);
  if (e != cudaSuccess) return e;
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

bool persistent_supported(int n) { return n == 256 || n == 512; }

cudaError_t launch_unfused_persistent(const UnfusedArgs& a, long long n_time, int nt_batch, unsigned* bar, int sms,
                                      cudaStream_t s) {
  switch (a.grid_n) {
    case 256: return launch_persistent_n<256>(a, n_time, nt_batch, bar, sms, s);
    case 512: return launch_persistent_n<512>(a, n_time, nt_batch, bar, sms, s);
    default: return cudaErrorInvalidValue;
  }
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
