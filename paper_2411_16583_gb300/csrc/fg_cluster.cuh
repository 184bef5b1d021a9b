// Y-fwd, Z with the compatibility projection and Y-inv in one pass whose working set lives
// in the distributed shared memory of a 16-CTA thread-block cluster (FP32, ny = nz = N,
// N = R0 R1 a two-stage plan).
//
// The projection (Eqs. mapping G, mechanicalsolve) couples the three components of one row
// i of the tensor only: A'_ij = n_j (A_im n_m) / |n|^2.  So a cluster takes one kx plane of
// one row (three components, N x N complex numbers: 1.5 MB at N = 256) and keeps it on chip
// across the three transforms.  CTA r of the cluster owns the z slab [r S, (r+1) S) in the
// y stages and the ky slab [r S, (r+1) S) in the z stage (S = N / 16):
//
//   stage 0  load the S z-rows of each input component from HBM straight into registers
//            (radix-R0 step), one transpose through the own tile, radix-R1 step; each
//            thread then stores its ky values into the recv tile of the CTA that owns them
//            (remote stores to distributed shared memory, 16 lanes writing one 128-byte run)
//   stage 1  two-stage z-transform of the recv tile, the frequency-space operator (read
//            across the component rows), two-stage inverse z-transform whose last step
//            stores its z values into the own tile of the CTA that owns them
//   stage 2  two-stage inverse y-transform of the own tile, stored to HBM from registers
//
// Cluster barriers: one arrive at the start, waited on before the first remote store (every
// CTA of the cluster has started), and one after each push.  A tile is written remotely
// only in the stage before the one that reads it, so the two pushes never overlap a read.
// The pass reads and writes the nine-component spectrum once (72.6 B per voxel at N = 256)
// where the three passes read and wrote it three times.  In the host emulation the stages
// of the 16 CTAs run one stage at a time, which is what the barriers guarantee on the GPU.
#pragma once
#include <atomic>
#include <vector>
#include "fg_ops.cuh"

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
  static constexpr Plan P = make_plan(N);
  static_assert(P.S == 2, "the clustered pass takes a two-stage plan");
  static constexpr int R0 = P.r[0], R1 = P.r[1];
  static constexpr int T0 = N / R0, T1 = N / R1;  // butterflies per row in stage 0 / 1
  static constexpr int CI = Z::CIN, CO = Z::COUT, G = Z::GROUPS;
  static constexpr int CM = CI > CO ? CI : CO;
  static constexpr int S = N / YZY_CLUSTER;  // z rows (y stages) or ky rows (z stage) per CTA
  static constexpr int ROWS = CM * S;
  static constexpr int TM = T0 > T1 ? T0 : T1;
  static constexpr int RM = R0 > R1 ? R0 : R1;
  static constexpr int NT = round32(ROWS * TM);
  static constexpr int NSTAGES = 3;
  static constexpr int PITCH = row_pitch(N);
  struct Locals {
    C v[RM];
    Acc<R> acc;
  };
  static constexpr size_t TILE = (size_t)ROWS * PITCH * sizeof(C);
  static size_t smem_bytes() { return 2 * TILE + N * sizeof(C); }
  static int clusters(int hx) { return hx * G; }
  // resident CTAs per SM the register budget is sized for
  static constexpr int MINB = 2 * TILE + N * sizeof(C) <= 110 * 1024 ? 2 : 1;

  FG_DEV static C* own(char* sm) { return (C*)sm; }
  FG_DEV static C* recv(char* sm) { return (C*)(sm + TILE); }
  FG_DEV static C* twid(char* sm) { return (C*)(sm + 2 * TILE); }

  // stores v at element `off` of the tile that starts `base` bytes into the shared memory of
  // the cluster's CTA q: a remote store to distributed shared memory on the GPU (mapa of the
  // same offset in the own window), the emulation's buffer of CTA q on the host
  FG_DEV static void put(char* local, char* const* sm, int q, size_t base, int off, C v) {
#ifdef FG_EMU
    (void)local;
    ((C*)(sm[q] + base))[off] = v;
#else
    (void)sm;
    const unsigned la = (unsigned)__cvta_generic_to_shared(local + base + (size_t)off * sizeof(C));
    unsigned ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(la), "r"(q));
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(ra), "f"(v.x), "f"(v.y)
                 : "memory");
#endif
  }

  // every CTA of the cluster has started: waits on the arrive made at the kernel's start
  FG_DEV static void wait_started() {
#ifndef FG_EMU
    asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
#endif
  }

  // stage 0 of the plan on registers v = x[b + r T0]: radix-R0 DFT, outputs at b R0 + r
  template <bool INV>
  FG_DEV static void step0_store(C* v, C* row, int b) {
    Dft<R0, INV, C>::run(v);
#pragma unroll
    for (int r = 0; r < R0; ++r) row[pad16(b * R0 + r)] = v[r];
  }
  // stage 1 (Ns = R0): loads positions b + r T1, twiddles by exp(-+2 pi i r b / N), radix-R1
  // DFT; v then holds the natural-order outputs b + r T1
  template <bool INV>
  FG_DEV static void step1_load(C* v, const C* row, const C* tw, int b) {
#pragma unroll
    for (int r = 0; r < R1; ++r) v[r] = row[pad16(b + r * T1)];
#pragma unroll
    for (int r = 1; r < R1; ++r) {
      const C w = tw[r * b];
      v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
    }
    Dft<R1, INV, C>::run(v);
  }

  // Stage s of the CTA of rank `rank` in cluster `cid` (kx = cid / G, group g = cid % G:
  // components g CI + cc in, g CO + cc out).  local is the CTA's own shared memory; sm[q]
  // that of the cluster's CTA q in the emulation (unused on the GPU).  Tile row cc S + j
  // holds component cc at z = rank S + j (own tile) or ky = rank S + j (recv tile).
  template <class Loc>
  FG_DEV static void stage(int s, const PassArgs<R>& a, int cid, int rank, char* local,
                           char* const* sm, Loc* Ls) {
    const int kx = cid / G, g = cid % G;
    C* mine = own(local);
    C* rv = recv(local);
    C* tw = twid(local);
    const int ny = a.ny, nz = a.nz;
    if (s == 0) {
      // radix-R0 step straight from HBM (lanes along y: coalesced)
      FG_PHASE(NT)
      for (int m = tid; m < N; m += NT) tw[m] = a.tw[m];
      if (tid < CI * S * T0) {
        const int b = tid % T0, rho = tid / T0;
        const int cc = rho / S, zz = rho - cc * S;
        const C* in = a.cin + (long long)(g * CI + cc) * a.VH +
                      ((long long)kx * nz + rank * S + zz) * ny;
#pragma unroll
        for (int r = 0; r < R0; ++r) L.v[r] = in[b + r * T0];
        step0_store<false>(L.v, mine + rho * PITCH, b);
      }
      FG_END_PHASE
      // radix-R1 step, then each ky value to the recv tile of the CTA owning that ky (lanes
      // along z: the 16 lanes of one row of the destination write one contiguous run)
      FG_PHASE(NT)
      const bool act = tid < CI * S * T1;
      const int rho = tid % (CI * S), b = tid / (CI * S);
      if (act) step1_load<false>(L.v, mine + rho * PITCH, tw, b);
      wait_started();
      if (act) {
        const int cc = rho / S, zz = rho - cc * S;
#pragma unroll
        for (int r = 0; r < R1; ++r) {
          const int ky = b + r * T1, q = ky / S, kyy = ky - q * S;
          put(local, sm, q, TILE, (cc * S + kyy) * PITCH + pad16(rank * S + zz), L.v[r]);
        }
      }
      FG_END_PHASE
    } else if (s == 1) {
      // forward z-transform of the recv tile, radix-R0 step
      FG_PHASE(NT)
      if (tid < CI * S * T0) {
        const int b = tid % T0, rho = tid / T0;
        const C* row = rv + rho * PITCH;
#pragma unroll
        for (int r = 0; r < R0; ++r) L.v[r] = row[pad16(b + r * T0)];
        Dft<R0, false, C>::run(L.v);
      }
      FG_END_PHASE
      FG_PHASE(NT)
      if (tid < CI * S * T0) {
        const int b = tid % T0, rho = tid / T0;
#pragma unroll
        for (int r = 0; r < R0; ++r) rv[rho * PITCH + pad16(b * R0 + r)] = L.v[r];
      }
      FG_END_PHASE
      // radix-R1 step; each thread writes back the positions it read (natural order)
      FG_PHASE(NT)
      if (tid < CI * S * T1) {
        const int b = tid % T1, rho = tid / T1;
        C* row = rv + rho * PITCH;
        step1_load<false>(L.v, row, tw, b);
#pragma unroll
        for (int r = 0; r < R1; ++r) row[pad16(b + r * T1)] = L.v[r];
      }
      FG_END_PHASE
      // the operator on the CI components of each frequency, kept for output component co,
      // and the radix-R0 step of the inverse z-transform
      FG_PHASE(NT)
      if (tid < CO * S * T0) {
        const int b = tid % T0, rho = tid / T0;
        const int co = rho / S, kyy = rho - co * S;
#pragma unroll
        for (int r = 0; r < R0; ++r) {
          const int kz = b + r * T0;
          C w[CM];
#pragma unroll
          for (int ci = 0; ci < CI; ++ci) w[ci] = rv[(ci * S + kyy) * PITCH + pad16(kz)];
          Z::apply(a, kx, rank * S + kyy, kz, g, w);
          L.v[r] = w[co];
        }
        Dft<R0, true, C>::run(L.v);
      }
      FG_END_PHASE
      FG_PHASE(NT)
      if (tid < CO * S * T0) {
        const int b = tid % T0, rho = tid / T0;
#pragma unroll
        for (int r = 0; r < R0; ++r) rv[rho * PITCH + pad16(b * R0 + r)] = L.v[r];
      }
      FG_END_PHASE
      // radix-R1 step, then each z value to the own tile of the CTA owning that z
      FG_PHASE(NT)
      if (tid < CO * S * T1) {
        const int rho = tid % (CO * S), b = tid / (CO * S);
        const int co = rho / S, kyy = rho - co * S;
        step1_load<true>(L.v, rv + rho * PITCH, tw, b);
#pragma unroll
        for (int r = 0; r < R1; ++r) {
          const int z = b + r * T1, q = z / S, zz = z - q * S;
          put(local, sm, q, 0, (co * S + zz) * PITCH + pad16(rank * S + kyy), L.v[r]);
        }
      }
      FG_END_PHASE
    } else {
      // inverse y-transform of the own tile, stored to HBM from registers
      FG_PHASE(NT)
      if (tid < CO * S * T0) {
        const int b = tid % T0, rho = tid / T0;
        const C* row = mine + rho * PITCH;
#pragma unroll
        for (int r = 0; r < R0; ++r) L.v[r] = row[pad16(b + r * T0)];
        Dft<R0, true, C>::run(L.v);
      }
      FG_END_PHASE
      FG_PHASE(NT)
      if (tid < CO * S * T0) {
        const int b = tid % T0, rho = tid / T0;
#pragma unroll
        for (int r = 0; r < R0; ++r) mine[rho * PITCH + pad16(b * R0 + r)] = L.v[r];
      }
      FG_END_PHASE
      FG_PHASE(NT)
      if (tid < CO * S * T1) {
        const int b = tid % T1, rho = tid / T1;
        const int co = rho / S, zz = rho - co * S;
        step1_load<true>(L.v, mine + rho * PITCH, tw, b);
        C* out = a.cout + (long long)(g * CO + co) * a.VH +
                 ((long long)kx * nz + rank * S + zz) * ny;
#pragma unroll
        for (int r = 0; r < R1; ++r) out[b + r * T1] = L.v[r];
      }
      FG_END_PHASE
    }
  }
};

#ifndef FG_EMU
template <class K, class A>
__global__ void __launch_bounds__(K::NT, K::MINB) cluster_kernel(A a) {
  extern __shared__ __align__(16) char smem[];
  typename K::Locals L;
  if (a.done && *a.done) return;  // the same flag for every CTA of the cluster
  unsigned rank;
  asm("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
  const int cid = (int)(blockIdx.x / YZY_CLUSTER);
  asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
  K::stage(0, a, cid, (int)rank, smem, nullptr, &L);  // waits on that arrive before pushing
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
  K::stage(1, a, cid, (int)rank, smem, nullptr, &L);
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
  K::stage(2, a, cid, (int)rank, smem, nullptr, &L);
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
    for (int s = 0; s < K::NSTAGES; ++s)
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
