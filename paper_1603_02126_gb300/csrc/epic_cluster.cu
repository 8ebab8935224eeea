// Thread-block-cluster EPIC imaging for grids that do not fit one SM
// (N = 256 with 8 CTAs per cluster, N = 512 with 16).
//
// One persistent launch images every frame of a batch.  The CTAs of a
// cluster share each frame: CTA q owns a block of the occupied grid rows and
// 32 image columns.  Per frame:
//   A  each CTA scatters the gain-corrected taps (Eqs. 8, 9) that fall in its
//      rows into its shared-memory grid block (window coordinates; lanes of
//      a warp hitting the same cell are merged before the atomic add);
//   B  N-point FFTs of its rows; every spectrum value goes straight to the
//      shared memory of the CTA that owns its column (distributed shared
//      memory stores), transposed and XOR-swizzled;
//   -- cluster barrier --
//   C  N-point FFTs of its 32 columns (Eq. 10), |E|^2 summed in registers;
//      the owner of the calibrator pixel broadcasts it to every CTA;
//   -- cluster barrier --
//      EPICal correlation of this frame for the CTA's share of antennas.
// Work units (channel, time segment) are assigned per cluster, so every CTA
// of a cluster runs the same loops and reaches every cluster barrier.
#include <cooperative_groups.h>

#include "epic_fft.cuh"
#include "epic_internal.h"

namespace cg = cooperative_groups;

namespace epic {
namespace {

using fft::cmul;
using fft::kFull;

template <int N> struct KCfg;
template <> struct KCfg<256> { static constexpr int CS = 8,  N1 = 16, N2 = 16; };
template <> struct KCfg<512> { static constexpr int CS = 16, N1 = 16, N2 = 32; };

constexpr int kKBT = 256;        // threads per CTA
constexpr int kColsPerCta = 32;  // image columns owned by one CTA

template <int N>
struct KGeo {
  static constexpr int CS = KCfg<N>::CS, N1 = KCfg<N>::N1, N2 = KCfg<N>::N2;
  static constexpr int GROUPS = kKBT / N1;                 // 16 FFT groups
  static constexpr int COLROUNDS = kColsPerCta / GROUPS;   // 2
  static constexpr int NACC = COLROUNDS * N2;
  static constexpr int H = N2 / N1;
  static constexpr int WS = N + N1;                        // grid-block row stride
  using X = fft::Xchg<N1, N2>;
  static_assert(CS * kColsPerCta == N, "columns split evenly over the cluster");
};

__device__ __forceinline__ float2 load_volt_k(const ClusterArgs& A, long long t, int c, int a) {
  const size_t idx = (static_cast<size_t>(t) * A.n_chan + c) * A.n_ant + a;
  if (A.input_fmt == 0) {
    const unsigned b = __ldg(static_cast<const unsigned char*>(A.volt) + idx);
    const int re = static_cast<int>(b << 24) >> 28;
    const int im = static_cast<int>(b << 28) >> 28;
    return make_float2(static_cast<float>(re), static_cast<float>(im));
  }
  return __ldg(static_cast<const float2*>(A.volt) + idx);
}

template <int N, int NZ>
__device__ __forceinline__ void cluster_unit(const ClusterArgs& A, cg::cluster_group& cluster, int c,
                                             long long t0, long long t1, float2* Wb, float2* Tt, float2* zg,
                                             const float2* tw2, float2* pixs) {
  using G = KGeo<N>;
  constexpr int BT = kKBT, N1 = G::N1, N2 = G::N2, GROUPS = G::GROUPS, H = G::H, WS = G::WS;
  constexpr int CS = G::CS;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int g = tid / N1;
  const int n1 = tid % N1;
  const unsigned gmask = fft::group_mask<N1>(lane);
  const int q = static_cast<int>(cluster.block_rank());
  const int Na = A.n_ant;
  const int K = A.support;
  const int KK = K * K;
  const int rs = A.rs;

  const int4 wn = __ldg(A.win4 + c);                        // (y0, rows, x0, cols)
  const int R = wn.y;
  const int rpc = (R + CS - 1) / CS;                        // rows per CTA
  const int r_lo = q * rpc;
  const int r_n = max(0, min(rpc, R - r_lo));               // rows this CTA owns
  const float vs = A.vscale ? __ldg(A.vscale + c) : 1.0f;
  const int* rcs = A.rowcol + static_cast<size_t>(c) * Na;  // stencil top row << 16 | first column
  const int* ord = A.order + static_cast<size_t>(c) * Na;   // antennas sorted by stencil row
  const int2 range = __ldg(A.ranges + static_cast<size_t>(c) * CS + q);
  const float* wts = A.wts + static_cast<size_t>(c) * Na * KK;
  const float2* wg = A.wgain + static_cast<size_t>(c) * Na;
  const int items = (range.y - range.x) * K;
  const int items_pad = ((items + BT - 1) / BT) * BT;

  // calibrator pixel: owning CTA, column round, group, lane and slot
  const int pcta = A.k0x / kColsPerCta, pcol = A.k0x % kColsPerCta;
  const int pr = pcol / GROUPS, pg = pcol % GROUPS;
  const int pn1 = A.k0y % N1;
  const int pq = A.k0y / N1;
  const int pslot = (pq % H) * N1 + pq / H;
  const bool pix_owner = A.do_cal && q == pcta && g == pg && n1 == pn1;
  const float2 pph = A.do_cal ? __ldg(A.pixph + c) : make_float2(1.f, 0.f);

  // this CTA correlates antennas a = q + CS * tid
  const int my_ant = q + CS * tid;
  const bool corr = A.do_cal && my_ant < Na && __ldg(rcs + min(my_ant, Na - 1)) >= 0;

  float acc[G::NACC];
#pragma unroll
  for (int i = 0; i < G::NACC; ++i) acc[i] = 0.f;
  float2 kac = make_float2(0.f, 0.f);
  float pac = 0.f;

  const int P = A.frames_per_step;                          // spectra slots in shared memory
  for (long long tb = t0; tb < t1; tb += P) {
    const int nf = static_cast<int>(min(static_cast<long long>(P), t1 - tb));
    for (int f = 0; f < nf; ++f) {
      const long long t = tb + f;
      float2* Ts = Tt + static_cast<size_t>(f) * kColsPerCta * rs;
      // ---- A: scatter the taps that fall in this CTA's rows ----
      for (int it = tid; it < items_pad; it += BT) {
        const bool in = it < items;
        const int i = in ? range.x + it / K : 0;
        const int dy = in ? it % K : 0;
        const int a = in ? __ldg(ord + i) : 0;
        const int rc = in ? __ldg(rcs + a) : -1;
        const int row = (rc >> 16) + dy - r_lo;
        const bool valid = rc >= 0 && row >= 0 && row < r_n;
        float2 ec = make_float2(0.f, 0.f);
        if (valid) {
          const float2 e = load_volt_k(A, t, c, a);
          ec = cmul(make_float2(e.x * vs, e.y * vs), __ldg(wg + a));
        }
        const int rowcell = valid ? row * WS + (rc & 0xffff) : -1 - lane;
        const unsigned peers = __match_any_sync(kFull, rowcell);
        const bool dup = __popc(peers) > 1;
        const float* wrow = wts + static_cast<size_t>(a) * KK + dy * K;
        if (!__any_sync(kFull, dup)) {
          if (valid) {
            for (int dx = 0; dx < K; ++dx) {
              const float w = __ldg(wrow + dx);
              atomicAdd(&Wb[rowcell + dx].x, w * ec.x);
              atomicAdd(&Wb[rowcell + dx].y, w * ec.y);
            }
          }
        } else {
          const int leader = __ffs(peers) - 1;
          for (int dx = 0; dx < K; ++dx) {
            const float w = valid ? __ldg(wrow + dx) : 0.f;
            const float vx = w * ec.x, vy = w * ec.y;
            float sx = 0.f, sy = 0.f;
#pragma unroll 1
            for (int src = 0; src < 32; ++src) {        // rare path: kept rolled
              const float ox = __shfl_sync(kFull, vx, src);
              const float oy = __shfl_sync(kFull, vy, src);
              if ((peers >> src) & 1u) {
                sx += ox;
                sy += oy;
              }
            }
            if (valid && lane == leader) {
              atomicAdd(&Wb[rowcell + dx].x, sx);
              atomicAdd(&Wb[rowcell + dx].y, sy);
            }
          }
        }
      }
      __syncthreads();

      // ---- B: row FFTs; spectra to the column owners' shared memory ----
      for (int lr = g; lr < r_n; lr += GROUPS) {
        const int row = r_lo + lr;                          // window row
        float2 v[N2];
        float2* wr = Wb + lr * WS;
#pragma unroll
        for (int j = 0; j < N2; ++j) v[j] = (j < NZ) ? wr[n1 + N1 * j] : make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < NZ; ++j) wr[n1 + N1 * j] = make_float2(0.f, 0.f);
        fft::fft_lanes_p<N1, N2, NZ>(v, n1, zg, tw2, gmask);
        // kx = n1 + N1 h + N2 k1: owner CTA kx / 32, column kx % 32 (= n1 mod 8)
        const int srow = row ^ (n1 & 7);
#pragma unroll
        for (int h = 0; h < H; ++h)
#pragma unroll
          for (int k1 = 0; k1 < N1; ++k1) {
            const int kx = n1 + N1 * h + N2 * k1;
            float2* dst = cluster.map_shared_rank(Ts, kx / kColsPerCta);
            dst[(kx % kColsPerCta) * rs + srow] = v[h * N1 + k1];
          }
      }
      __syncthreads();                                      // grid block reused by the next frame
    }
    cluster.sync();

    // ---- C: column FFTs of this CTA's 32 columns, every frame of the step ----
    const int jmax = (R - n1 + N1 - 1) / N1;
    for (int f = 0; f < nf; ++f) {
      const float2* Ts = Tt + static_cast<size_t>(f) * kColsPerCta * rs;
#pragma unroll
      for (int r = 0; r < G::COLROUNDS; ++r) {
        const int col = g + GROUPS * r;
        float2 v[N2];
        const float2* cb = Ts + col * rs + (n1 ^ (col & 7));
#pragma unroll
        for (int j = 0; j < N2; ++j) v[j] = (j < NZ && j < jmax) ? cb[N1 * j] : make_float2(0.f, 0.f);
        fft::fft_lanes_p<N1, N2, NZ>(v, n1, zg, tw2, gmask);
#pragma unroll
        for (int s = 0; s < N2; ++s) acc[r * N2 + s] += v[s].x * v[s].x + v[s].y * v[s].y;
        if (pix_owner && r == pr) {
          float2 p = make_float2(0.f, 0.f);
#pragma unroll
          for (int s = 0; s < N2; ++s)
            if (s == pslot) p = cmul(v[s], pph);
          for (int d = 0; d < CS; ++d) cluster.map_shared_rank(pixs, d)[f] = p;
        }
      }
    }
    cluster.sync();

    // ---- correlation of the step's frames (raw voltages, Eqs. 12, 15) ----
    if (corr) {
      for (int f = 0; f < nf; ++f) {
        const float2 p = pixs[f];
        const float2 e0 = load_volt_k(A, tb + f, c, my_ant);
        const float2 e = make_float2(e0.x * vs, e0.y * vs);
        kac.x += e.x * p.x + e.y * p.y;
        kac.y += e.y * p.x - e.x * p.y;
        pac += e.x * e.x + e.y * e.y;
      }
    }
  }

  // flush this CTA's columns and antennas (FP32 over the unit, FP64 across)
  double* img = A.image + static_cast<size_t>(c) * N * N;
#pragma unroll
  for (int r = 0; r < G::COLROUNDS; ++r) {
    const int kx = q * kColsPerCta + g + GROUPS * r;
#pragma unroll
    for (int h = 0; h < H; ++h)
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) {
        const int ky = n1 + N1 * h + N2 * k1;
        atomicAdd(img + ky * N + kx, static_cast<double>(acc[r * N2 + h * N1 + k1]) * A.img_scale);
      }
  }
  if (corr) {
    const size_t o = static_cast<size_t>(c) * Na + my_ant;
    atomicAdd(&A.kacc[o].x, static_cast<double>(kac.x));
    atomicAdd(&A.kacc[o].y, static_cast<double>(kac.y));
    atomicAdd(A.pacc + o, static_cast<double>(pac));
  }
}

template <int N>
__global__ void __launch_bounds__(kKBT, 1) epic_image_cluster(const ClusterArgs A) {
  using G = KGeo<N>;
  constexpr int CS = G::CS, N1 = G::N1, N2 = G::N2, GROUPS = G::GROUPS, WS = G::WS;
  cg::cluster_group cluster = cg::this_cluster();

  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* Wb = reinterpret_cast<float2*>(smem_raw);         // [rpc_alloc][WS] grid block
  float2* Tt = Wb + A.rpc_alloc * WS;                       // [P][32][rs] spectra of my columns
  float2* Z = Tt + static_cast<size_t>(A.frames_per_step) * kColsPerCta * A.rs;  // exchange
  float2* tw2 = Z + GROUPS * G::X::ZG;                      // [N2][N1] twiddles
  float2* pixs = tw2 + N;                                   // [P] calibrator pixels

  const int tid = threadIdx.x;
  float2* zg = Z + (tid / N1) * G::X::ZG;
  for (int i = tid; i < N; i += kKBT) tw2[i] = A.twid[(i % N1) * (i / N1)];
  for (int i = tid; i < A.rpc_alloc * WS; i += kKBT) Wb[i] = make_float2(0.f, 0.f);
  cluster.sync();                                           // every CTA of the cluster is resident

  const int cid = blockIdx.x / CS, ncl = gridDim.x / CS;
  const long long T = A.n_time;
  const int units = A.n_chan * A.segs;
  for (int u = cid; u < units; u += ncl) {
    const int c = u / A.segs;
    const int s = u - c * A.segs;
    const long long t0 = T * s / A.segs;
    const long long t1 = T * (s + 1) / A.segs;
    if (t0 >= t1) continue;                                 // cluster-uniform
    const int4 wn = __ldg(A.win4 + c);
    const int span = wn.y > wn.w ? wn.y : wn.w;
    if (span <= N1 * (N2 / 4))
      cluster_unit<N, N2 / 4>(A, cluster, c, t0, t1, Wb, Tt, zg, tw2, pixs);
    else if (span <= N1 * (N2 / 2))
      cluster_unit<N, N2 / 2>(A, cluster, c, t0, t1, Wb, Tt, zg, tw2, pixs);
    else
      cluster_unit<N, N2>(A, cluster, c, t0, t1, Wb, Tt, zg, tw2, pixs);
  }
  cluster.sync();                                           // no CTA leaves while others write to it
}

template <int N>
cudaError_t cluster_launch_n(const ClusterArgs& a, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(a.grid));
  cfg.blockDim = dim3(kKBT);
  cfg.dynamicSmemBytes = a.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = KCfg<N>::CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, epic_image_cluster<N>, a);
}

template <int N>
cudaError_t cluster_prepare_n(size_t smem, int* clusters) {
  cudaError_t e = cudaFuncSetAttribute(epic_image_cluster<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  if (KCfg<N>::CS > 8) {
    e = cudaFuncSetAttribute(epic_image_cluster<N>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(KCfg<N>::CS * 64));
  cfg.blockDim = dim3(kKBT);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = KCfg<N>::CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaOccupancyMaxActiveClusters(clusters, epic_image_cluster<N>, &cfg);
}

}  // namespace

bool cluster_supported(int n) { return n == 256 || n == 512; }

int cluster_size(int n) { return n == 256 ? KCfg<256>::CS : (n == 512 ? KCfg<512>::CS : 0); }

size_t cluster_smem_bytes(int n, int rpc_alloc, int rs, int frames_per_step) {
  size_t ws = 0, zg = 0, groups = 0;
  if (n == 256) {
    ws = KGeo<256>::WS;
    zg = KGeo<256>::X::ZG;
    groups = KGeo<256>::GROUPS;
  } else if (n == 512) {
    ws = KGeo<512>::WS;
    zg = KGeo<512>::X::ZG;
    groups = KGeo<512>::GROUPS;
  } else {
    return 0;
  }
  const size_t elems = static_cast<size_t>(rpc_alloc) * ws +
                       static_cast<size_t>(frames_per_step) * kColsPerCta * rs + groups * zg + n +
                       2 * static_cast<size_t>(frames_per_step);
  return elems * sizeof(float2);
}

cudaError_t cluster_prepare(int n, size_t smem, int* clusters) {
  if (n == 256) return cluster_prepare_n<256>(smem, clusters);
  if (n == 512) return cluster_prepare_n<512>(smem, clusters);
  return cudaErrorInvalidValue;
}

cudaError_t launch_cluster(int n, const ClusterArgs& a, cudaStream_t s) {
  if (n == 256) return cluster_launch_n<256>(a, s);
  if (n == 512) return cluster_launch_n<512>(a, s);
  return cudaErrorInvalidValue;
}

}  // namespace epic
