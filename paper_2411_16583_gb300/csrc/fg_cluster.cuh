// Y-fwd, Z with the compatibility projection and Y-inv in one pass whose working set lives
// in the distributed shared memory of a 16-CTA thread-block cluster (FP32, ny = nz = N).
//
// The projection (Eqs. mapping G, mechanicalsolve) couples the three components of one row
// i of the tensor only: A'_ij = n_j (A_im n_m) / |n|^2.  So a cluster takes one kx plane of
// one row (three components, N x N complex numbers: 1.5 MB at N = 256) and keeps it on chip
// across the three transforms:
//
//   stage 0  CTA r loads its slab of S = N/16 z-rows (y contiguous) of the three components
//            from S1 and transforms them along y                             [own tile]
//   stage 1  CTA r gathers the ky range [r S, (r+1) S) of every z from all 16 CTAs' own
//            tiles (distributed shared memory), transforms along z, projects, transforms
//            back along z                                                   [recv tile]
//   stage 2  CTA r gathers its z slab back, every ky, from all 16 recv tiles  [own tile]
//   stage 3  inverse transform along y and store to S1 in place
//
// with a cluster barrier between stages (and the last gather ends with one, so that no
// CTA leaves while a peer still reads its tiles).  The intermediate spectrum of the Y and Z
// passes never reaches HBM: the pass reads and writes the nine-component spectrum once
// (72.6 B per voxel at N = 256) where the three passes read and wrote it three times.
// In the host emulation the stages of all 16 CTAs of a cluster run one stage at a time, so
// the cluster barriers hold there too.
#pragma once
#include <atomic>
#include <vector>
#include "fg_ops.cuh"

#ifndef FG_EMU
#include <cooperative_groups.h>
#endif

namespace fg {

std::atomic<long long>& launch_counter();

constexpr int YZY_CLUSTER = 16;

// the projection of one row i of the tensor (components 3 i + j), zero mode kept on the
// stress-controlled components of the mask in coef[1]; coef[0] = 1/V
template <typename R>
FG_DEV void project_row(const PassArgs<R>& a, int kx, int ky, int kz, int i, cplx<R>* v) {
  using C = cplx<R>;
  const R n0 = a.rs[0][kx] * a.rc[1][ky] * a.rc[2][kz];
  const R n1 = a.rs[1][ky] * a.rc[0][kx] * a.rc[2][kz];
  const R n2 = a.rs[2][kz] * a.rc[0][kx] * a.rc[1][ky];
  const R nn = n0 * n0 + n1 * n1 + n2 * n2;
  const R s = nn > (R)0 ? a.coef[0] / nn : (R)0;
  const int mask = (int)a.coef[1];
  if (mask != 0 && kx == 0 && ky == 0 && kz == 0) {
#pragma unroll
    for (int j = 0; j < 3; ++j)
      v[j] = ((mask >> (3 * i + j)) & 1) ? cscale(v[j], a.coef[0]) : cmk<C>((R)0, (R)0);
    return;
  }
  C t = cadd(cadd(cscale(v[0], n0), cscale(v[1], n1)), cscale(v[2], n2));
  t = cscale(t, s);
  v[0] = cscale(t, n0);
  v[1] = cscale(t, n1);
  v[2] = cscale(t, n2);
}

// Frequency-space operators of the clustered pass.  ZRows: the projection, one tensor row
// (three components) per cluster, GROUPS = 3 clusters per kx plane.  ZWhole<Op>: a Z-pass
// operator on all its components (the chemistry's 1 -> 3 gradient and 3 -> 1 divergence),
// one cluster per kx plane.
template <typename R>
struct ZRows {
  static constexpr int CIN = 3, COUT = 3, GROUPS = 3;
  FG_DEV static void apply(const PassArgs<R>& a, int kx, int ky, int kz, int g, cplx<R>* v) {
    project_row(a, kx, ky, kz, g, v);
  }
};
template <class Op>
struct ZWhole {
  static constexpr int CIN = Op::CIN, COUT = Op::COUT, GROUPS = 1;
  template <typename R>
  FG_DEV static void apply(const PassArgs<R>& a, int kx, int ky, int kz, int, cplx<R>* v) {
    const R zs = a.dscal ? (R)a.dscal[0] : (R)0;
    Op::apply(a, kx, ky, kz, v, zs);
  }
};

template <typename R, int N, class Z = ZRows<R>>
struct YZYCluster {
  using C = cplx<R>;
  static constexpr int CI = Z::CIN, CO = Z::COUT, G = Z::GROUPS;
  static constexpr int CM = CI > CO ? CI : CO;
  static constexpr int S = N / YZY_CLUSTER;   // z rows (stage 0) or ky rows (stage 1) per CTA
  static constexpr int ROWS = CM * S;         // rows of the largest component count
  static constexpr int NT = round32(ROWS * tpr(N));
  using TFf = TileFFT<R, N, CI * S, NT, false>;  // forward transforms: the CI input rows
  using TFi = TileFFT<R, N, CO * S, NT, true>;   // inverse transforms: the CO output rows
  static constexpr int PITCH = TFf::PITCH;
  static constexpr int VMAX = TFf::VMAX > TFi::VMAX ? TFf::VMAX : TFi::VMAX;
  struct Locals {
    C v[VMAX];
    Acc<R> acc;
  };
  static constexpr size_t TILE = (size_t)ROWS * PITCH * sizeof(C);
  static size_t smem_bytes() { return 2 * TILE + N * sizeof(C); }
  static int clusters(int hx) { return hx * G; }

  // shared memory of the cluster's CTA q: the distributed shared memory window of that CTA
  // (mapa) on the GPU; the emulation's buffer of that CTA on the host
  FG_DEV static char* peer(char* local, char* const* sm, int q) {
#ifdef FG_EMU
    (void)local;
    return sm[q];
#else
    (void)sm;
    return cooperative_groups::this_cluster().map_shared_rank(local, q);
#endif
  }

  // own tile, recv tile and twiddles of a CTA's shared memory
  FG_DEV static C* own(char* sm) { return (C*)sm; }
  FG_DEV static C* recv(char* sm) { return (C*)(sm + TILE); }
  FG_DEV static C* twid(char* sm) { return (C*)(sm + 2 * TILE); }

  // Stage s of the CTA of rank `rank` in cluster `cid` (kx = cid / G, group g = cid % G:
  // components g CI + cc in, g CO + cc out).  local is the CTA's own shared memory; sm[q]
  // that of the cluster's CTA q in the emulation (unused on the GPU, where peer() maps it).
  // Tile rows (cc, r) hold component cc at z (own tile) or ky (recv tile) of the slab.
  template <class Loc>
  FG_DEV static void stage(int s, const PassArgs<R>& a, int cid, int rank, char* local,
                           char* const* sm, Loc* Ls) {
    const int kx = cid / G, g = cid % G;
    C* mine = own(local);
    C* rv = recv(local);
    C* tw = twid(local);
    const int ny = a.ny, nz = a.nz;
    if (s == 0) {
      FG_PHASE(NT)
      for (int m = tid; m < N; m += NT) tw[m] = a.tw[m];
      // S consecutive z-rows of length ny per component: one contiguous block each
      for (int e = tid; e < CI * S * N; e += NT) {
        const int q = e / N, y = e - q * N;
        const int cc = q / S, zz = q - cc * S;
        const long long gi = (long long)(g * CI + cc) * a.VH +
                             ((long long)kx * nz + rank * S + zz) * ny + y;
        mine[q * PITCH + pad16(y)] = a.cin[gi];
      }
      FG_END_PHASE
      tile_fft<TFf, 0>(Ls, mine, tw, NT);
    } else if (s == 1) {
      FG_PHASE(NT)
      // recv row (cc, kyy) holds every z of ky = rank S + kyy: z slab q of it is CTA q's
      for (int e = tid; e < CI * S * N; e += NT) {
        const int qrow = e / N, z = e - qrow * N;
        const int cc = qrow / S, kyy = qrow - cc * S;
        const int src = z / S, zz = z - src * S;
        const C* pt = own(peer(local, sm, src));
        rv[qrow * PITCH + pad16(z)] = pt[(cc * S + zz) * PITCH + pad16(rank * S + kyy)];
      }
      FG_END_PHASE
      tile_fft<TFf, 0>(Ls, rv, tw, NT);
      FG_PHASE(NT)
      for (int e = tid; e < S * N; e += NT) {
        const int kyy = e / N, kz = e - kyy * N;
        C v[CM];
#pragma unroll
        for (int cc = 0; cc < CI; ++cc) v[cc] = rv[(cc * S + kyy) * PITCH + pad16(kz)];
        Z::apply(a, kx, rank * S + kyy, kz, g, v);
#pragma unroll
        for (int cc = 0; cc < CO; ++cc) rv[(cc * S + kyy) * PITCH + pad16(kz)] = v[cc];
      }
      FG_END_PHASE
      tile_fft<TFi, 0>(Ls, rv, tw, NT);
    } else if (s == 2) {
      FG_PHASE(NT)
      // own row (cc, zz) gets every ky of z = rank S + zz: ky slab q of it is CTA q's
      for (int e = tid; e < CO * S * N; e += NT) {
        const int q = e / N, ky = e - q * N;
        const int cc = q / S, zz = q - cc * S;
        const int src = ky / S, kyy = ky - src * S;
        const C* pt = recv(peer(local, sm, src));
        mine[q * PITCH + pad16(ky)] = pt[(cc * S + kyy) * PITCH + pad16(rank * S + zz)];
      }
      FG_END_PHASE
    } else {
      tile_fft<TFi, 0>(Ls, mine, tw, NT);
      FG_PHASE(NT)
      for (int e = tid; e < CO * S * N; e += NT) {
        const int q = e / N, y = e - q * N;
        const int cc = q / S, zz = q - cc * S;
        const long long gi = (long long)(g * CO + cc) * a.VH +
                             ((long long)kx * nz + rank * S + zz) * ny + y;
        a.cout[gi] = mine[q * PITCH + pad16(y)];
      }
      FG_END_PHASE
    }
  }
};

#ifndef FG_EMU
template <class K, class A>
__global__ void __launch_bounds__(K::NT, 1) cluster_kernel(A a) {
  namespace cgr = cooperative_groups;
  extern __shared__ __align__(16) char smem[];
  typename K::Locals L;
  if (a.done && *a.done) return;  // the same flag for every CTA of the cluster
  cgr::cluster_group cluster = cgr::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int cid = (int)(blockIdx.x / YZY_CLUSTER);
  K::stage(0, a, cid, rank, smem, nullptr, &L);
  cluster.sync();
  K::stage(1, a, cid, rank, smem, nullptr, &L);
  cluster.sync();
  K::stage(2, a, cid, rank, smem, nullptr, &L);
  cluster.sync();  // no CTA leaves while a peer reads its tiles
  K::stage(3, a, cid, rank, smem, nullptr, &L);
}
#endif

// 1 when the device can keep at least one cluster of YZY_CLUSTER CTAs of K resident
template <class K, class A>
bool cluster_pass_available() {
#ifdef FG_EMU
  return true;
#else
  static const bool ok = []() {
    const size_t sm = K::smem_bytes();
    if (cudaFuncSetAttribute(cluster_kernel<K, A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sm) != cudaSuccess ||
        cudaFuncSetAttribute(cluster_kernel<K, A>, cudaFuncAttributeNonPortableClusterSizeAllowed,
                             1) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(YZY_CLUSTER, 1, 1);
    cfg.blockDim = dim3(K::NT, 1, 1);
    cfg.dynamicSmemBytes = sm;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = YZY_CLUSTER;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, cluster_kernel<K, A>, &cfg) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return n > 0;
  }();
  return ok;
#endif
}

// launches the fused pass over every (kx, row) cluster; returns 0 (no partial sums)
template <class K, class A>
int launch_cluster(const A& a, int nclusters, cudaStream_t st) {
  ++launch_counter();
#ifdef FG_EMU
  (void)st;
  const size_t sm = K::smem_bytes();
  std::vector<std::vector<char>> mem(YZY_CLUSTER, std::vector<char>(sm, 0));
  std::vector<std::vector<typename K::Locals>> Ls(YZY_CLUSTER,
                                                  std::vector<typename K::Locals>(K::NT));
  char* ptr[YZY_CLUSTER];
  for (int q = 0; q < YZY_CLUSTER; ++q) ptr[q] = mem[q].data();
  if (a.done && *a.done) return 0;
  for (int cid = 0; cid < nclusters; ++cid)
    for (int s = 0; s < 4; ++s)
      for (int r = 0; r < YZY_CLUSTER; ++r) K::stage(s, a, cid, r, ptr[r], ptr, Ls[r].data());
#else
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nclusters * YZY_CLUSTER), 1, 1);
  cfg.blockDim = dim3(K::NT, 1, 1);
  cfg.dynamicSmemBytes = K::smem_bytes();
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = YZY_CLUSTER;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, cluster_kernel<K, A>, a);
#endif
  return 0;
}

template <typename R, int N, class Z = ZRows<R>>
int run_yzy_cluster(const PassArgs<R>& a, cudaStream_t st) {
  using K = YZYCluster<R, N, Z>;
  return launch_cluster<K>(a, K::clusters(a.hx), st);
}
template <typename R, int N, class Z = ZRows<R>>
bool yzy_cluster_ok() {
  return cluster_pass_available<YZYCluster<R, N, Z>, PassArgs<R>>();
}

}  // namespace fg
