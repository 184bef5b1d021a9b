// Launch of the FFT pass kernels, and the per-size table of launchers that the runtime
// dispatches through (one table per transform length N and precision).
#pragma once
#include <atomic>
#include <type_traits>
#include <vector>
#include <cstring>
#include "fg_ops.cuh"
#include "fg_cluster.cuh"

namespace fg {

// Resident blocks per SM a kernel asks the compiler to fit (K::MINB when present): it caps
// the registers per thread at 65536 / (MINB NT), so that occupancy is not limited by
// registers before shared memory.
template <class K, class = void>
struct MinBlocks {
  static constexpr int value = 1;
};
template <class K>
struct MinBlocks<K, std::void_t<decltype(K::MINB)>> {
  static constexpr int value = K::MINB;
};

#ifndef FG_EMU
// Kernels without K::MINB keep the plain bound on the block size: an explicit minimum of
// one block lets the compiler spend more registers and halved the residency of the
// forward and Y/Z passes.
template <class K, class A>
__global__ void __launch_bounds__(K::NT) pass_kernel(A a) {
  extern __shared__ __align__(16) char smem[];
  typename K::Locals L;
  K::body(a, Dim3{(int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z},
          Dim3{(int)gridDim.x, (int)gridDim.y, (int)gridDim.z}, smem, &L);
}
template <class K, class A>
__global__ void __launch_bounds__(K::NT, MinBlocks<K>::value) pass_kernel_mb(A a) {
  extern __shared__ __align__(16) char smem[];
  typename K::Locals L;
  K::body(a, Dim3{(int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z},
          Dim3{(int)gridDim.x, (int)gridDim.y, (int)gridDim.z}, smem, &L);
}
#endif

// number of kernel launches issued by the library (all kernels, all contexts)
std::atomic<long long>& launch_counter();

// ------------------------------------------------------------------ grouped launches
//
// A batch of RVEs with equal grids runs each pass of an operator application as one
// launch over all members: block m P + b of the grouped kernel runs block b of member m
// (P blocks per member), with member m's pass arguments read from a device table.  The
// runtime finds the launches of one member's application by recording them: while a
// recorder is set on the calling thread, launch_pass stores the launch (the grouped
// launcher of its kernel, its grid and a copy of its arguments) instead of launching.
struct RecordedLaunch {
  void (*grouped)(const void* args, int members, Dim3 grid, cudaStream_t st);
  size_t arg_bytes;
  Dim3 grid;
  std::vector<char> args;
};
inline std::vector<RecordedLaunch>*& launch_recorder() {
  static thread_local std::vector<RecordedLaunch>* r = nullptr;
  return r;
}

#ifndef FG_EMU
// The block's member arguments are copied into shared memory first: the pass bodies then
// read them from memory that no global store can alias, as they read kernel parameters.
template <class K, class A>
FG_DEV void grouped_body(const A* __restrict__ args, Dim3 grid) {
  extern __shared__ __align__(16) char smem[];
  __shared__ __align__(16) A sa;
  typename K::Locals L;
  const int per = grid.x * grid.y * grid.z;
  const int m = (int)blockIdx.x / per, b = (int)blockIdx.x - m * per;
  static_assert(sizeof(A) % sizeof(int) == 0, "argument block of whole words");
  for (int i = (int)threadIdx.x; i < (int)(sizeof(A) / sizeof(int)); i += (int)blockDim.x)
    ((int*)&sa)[i] = ((const int*)(args + m))[i];
  __syncthreads();
  const int bx = b % grid.x, t = b / grid.x;
  K::body(sa, Dim3{bx, t % grid.y, t / grid.y}, grid, smem, &L);
}
template <class K, class A>
__global__ void __launch_bounds__(K::NT) grouped_kernel(const A* __restrict__ args, Dim3 grid) {
  grouped_body<K, A>(args, grid);
}
template <class K, class A>
__global__ void __launch_bounds__(K::NT, MinBlocks<K>::value)
    grouped_kernel_mb(const A* __restrict__ args, Dim3 grid) {
  grouped_body<K, A>(args, grid);
}
#endif

// One launch of kernel K over `members` members (argument table `args`: device memory on
// the GPU, host memory in the emulation), `grid` blocks each.
template <class K, class A>
void launch_grouped(const void* args, int members, Dim3 grid, cudaStream_t st) {
  static_assert(K::NT <= 1024, "a block holds at most 1024 threads");
  const size_t sm = K::smem_bytes();
  ++launch_counter();
  const A* av = (const A*)args;
#ifdef FG_EMU
  (void)st;
  std::vector<char> smem(sm);
  std::vector<typename K::Locals> Ls(K::NT);
  for (int m = 0; m < members; ++m)
    for (int z = 0; z < grid.z; ++z)
      for (int y = 0; y < grid.y; ++y)
        for (int x = 0; x < grid.x; ++x) {
          std::memset(smem.data(), 0, sm);
          K::body(av[m], Dim3{x, y, z}, grid, smem.data(), Ls.data());
        }
#else
  constexpr bool MB = MinBlocks<K>::value > 1;
  static const bool configured = [sm]() {
    if constexpr (MB)
      cudaFuncSetAttribute(grouped_kernel_mb<K, A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sm);
    else
      cudaFuncSetAttribute(grouped_kernel<K, A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sm);
    return true;
  }();
  (void)configured;
  const unsigned nb = (unsigned)members * (unsigned)(grid.x * grid.y * grid.z);
  if constexpr (MB)
    grouped_kernel_mb<K, A><<<nb, K::NT, sm, st>>>(av, grid);
  else
    grouped_kernel<K, A><<<nb, K::NT, sm, st>>>(av, grid);
#endif
}

// Launches kernel K with arguments A on `grid` blocks of K::NT threads.  Returns the
// number of blocks launched (the number of partial sums a reducing kernel writes).
template <class K, class A>
int launch_pass(const A& a, Dim3 grid, cudaStream_t st) {
  static_assert(K::NT <= 1024, "a block holds at most 1024 threads");
  if (std::vector<RecordedLaunch>* rec = launch_recorder()) {
    RecordedLaunch r;
    r.grouped = &launch_grouped<K, A>;
    r.arg_bytes = sizeof(A);
    r.grid = grid;
    r.args.resize(sizeof(A));
    std::memcpy(r.args.data(), &a, sizeof(A));
    rec->push_back(std::move(r));
    return grid.x * grid.y * grid.z;
  }
  const size_t sm = K::smem_bytes();
  ++launch_counter();
#ifdef FG_EMU
  (void)st;
  std::vector<char> smem(sm);
  std::vector<typename K::Locals> Ls(K::NT);
  for (int z = 0; z < grid.z; ++z)
    for (int y = 0; y < grid.y; ++y)
      for (int x = 0; x < grid.x; ++x) {
        std::memset(smem.data(), 0, sm);
        K::body(a, Dim3{x, y, z}, grid, smem.data(), Ls.data());
      }
#else
  constexpr bool MB = MinBlocks<K>::value > 1;
  static const bool configured = [sm]() {  // once per kernel, thread-safe
    if constexpr (MB)
      cudaFuncSetAttribute(pass_kernel_mb<K, A>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    else
      cudaFuncSetAttribute(pass_kernel<K, A>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    return true;
  }();
  (void)configured;
  if constexpr (MB)
    pass_kernel_mb<K, A><<<dim3(grid.x, grid.y, grid.z), K::NT, sm, st>>>(a);
  else
    pass_kernel<K, A><<<dim3(grid.x, grid.y, grid.z), K::NT, sm, st>>>(a);
#endif
  return grid.x * grid.y * grid.z;
}

template <typename R>
using PassFn = int (*)(const PassArgs<R>&, cudaStream_t);

// Launchers of one transform length.  x* use N = nx, y* use N = ny, z* use N = nz.
template <typename R>
struct SizeOps {
  int N;
  PassFn<R> xf_tangent, xf_cgtangent, xf_tangent_svk, xf_cgtangent_svk, xf_copy1, xf_copy3,
      xf_copy9;
  PassFn<R> xi_store1, xi_store3, xi_storedot1, xi_storedot9, xi_norm9, xi_pff, xi_chemflux, xi_chemop,
      xi_chemrhs, xi_cgupdate, xi_cgupdate_pc;
  // the fused chemistry CG: forward X with p = r + beta p, flux round trip, X-inv update
  PassFn<R> xf_cgchem, xr_chemflux, xi_cgchem;
  PassFn<R> yf, yi;
  PassFn<R> z_proj, z_lap, z_prec, z_grad, z_div;
  // the projection pass with 1 and 4 rows per block (register-direct sizes; null
  // elsewhere): tile shapes the autotuner times against the default
  PassFn<R> z_proj_rows[2];
  // Y-fwd, projection and Y-inv in one clustered pass (FP32, ny = nz = N of 128 or 256;
  // null elsewhere) and whether the device can run its clusters
  PassFn<R> yzy_proj;
  bool (*yzy_proj_ok)();
  // the chemistry's gradient (1 -> 3) and divergence (3 -> 1) chains as clustered passes
  PassFn<R> yzy_grad, yzy_div;
  bool (*yzy_chem_ok)();
  // FP64 only (null in the FP32 table): displacement at the corners and its transpose
  PassFn<R> xi_store9, z_disp, z_dispT;
};

template <class K, typename R>
int run_x(const PassArgs<R>& a, cudaStream_t st) {
  return launch_pass<K>(a, Dim3{K::grid_x(a.ny, a.nz), 1, 1}, st);
}
// one block row per component (9 components)
template <class K, typename R>
int run_x9(const PassArgs<R>& a, cudaStream_t st) {
  return launch_pass<K>(a, Dim3{K::grid_x(a.ny, a.nz), 9, 1}, st);
}
// Y and Z passes cover rows [row_lo, row_hi) when row_hi > 0 (a range of kx planes)
template <class K, typename R>
int run_y(const PassArgs<R>& a, cudaStream_t st) {
  const int rows = a.row_hi > 0 ? a.row_hi - a.row_lo : a.hx * a.nz;
  return launch_pass<K>(a, Dim3{(rows + K::ROWS - 1) / K::ROWS, a.ncomp, 1}, st);
}
template <class K, typename R>
int run_z(const PassArgs<R>& a, cudaStream_t st) {
  const int rows = a.row_hi > 0 ? a.row_hi - a.row_lo : a.hx * a.ny;
  return launch_pass<K>(a, Dim3{(rows + K::ROWS - 1) / K::ROWS, 1, 1}, st);
}

template <typename R, int N>
SizeOps<R> make_size_ops() {
  SizeOps<R> s{};
  s.N = N;
  if constexpr (N % 2 == 0) {
    s.xf_tangent = run_x<XFwd<R, N, PTangentNH<R>>, R>;
    s.xf_cgtangent = run_x<XFwd<R, N, PCgTangentNH<R>>, R>;
    s.xf_tangent_svk = run_x<XFwd<R, N, PTangentSVK<R>>, R>;
    s.xf_cgtangent_svk = run_x<XFwd<R, N, PCgTangentSVK<R>>, R>;
    s.xi_cgupdate = run_x<XInv<R, N, ECgUpdate<R>>, R>;
    s.xi_cgupdate_pc = run_x9<XInv<R, N, ECgUpdate1<R>, true>, R>;
    s.xf_copy1 = run_x<XFwd<R, N, PCopy<R, 1>>, R>;
    s.xf_copy3 = run_x<XFwd<R, N, PCopy<R, 3>>, R>;
    s.xf_copy9 = run_x<XFwd<R, N, PCopy<R, 9>>, R>;
    s.xi_store1 = run_x<XInv<R, N, EStore<R, 1>>, R>;
    s.xi_store3 = run_x<XInv<R, N, EStore<R, 3>>, R>;
    s.xi_storedot1 = run_x<XInv<R, N, EStoreDot<R, 1>>, R>;
    s.xi_storedot9 = run_x<XInv<R, N, EStoreDot<R, 9>>, R>;
    s.xi_norm9 = run_x<XInv<R, N, ENorm<R, 9>>, R>;
    s.xi_pff = run_x<XInv<R, N, EPff<R>>, R>;
    s.xi_chemflux = run_x<XInv<R, N, EChemFlux<R>>, R>;
    s.xi_chemop = run_x<XInv<R, N, EChemOp<R>>, R>;
    s.xi_chemrhs = run_x<XInv<R, N, EChemRhs<R>>, R>;
    s.xf_cgchem = run_x<XFwd<R, N, PCgChem<R>>, R>;
    s.xr_chemflux = run_x<XRound<R, N, EChemFluxRound<R>>, R>;
    s.xi_cgchem = run_x<XInv<R, N, ECgChemUpdate<R>>, R>;
    if constexpr (std::is_same<R, double>::value) s.xi_store9 = run_x<XInv<R, N, EStore<R, 9>>, R>;
  }
  if constexpr (Square<N>::OK) {  // register-direct two-stage passes
    s.yf = run_y<YPassD<R, N, false>, R>;
    s.yi = run_y<YPassD<R, N, true>, R>;
    s.z_proj = run_z<ZPassD<R, N, ZProject<R>>, R>;
    if constexpr (std::is_same<R, float>::value && N >= 64) {
      s.z_proj_rows[0] = run_z<ZPassD<R, N, ZProject<R>, 1>, R>;
      s.z_proj_rows[1] = run_z<ZPassD<R, N, ZProject<R>, 4>, R>;
    }

    s.z_lap = run_z<ZPassD<R, N, ZLaplace<R>>, R>;
    s.z_prec = run_z<ZPassD<R, N, ZPrecond<R>>, R>;
    s.z_grad = run_z<ZPassD<R, N, ZGrad<R>>, R>;
    s.z_div = run_z<ZPassD<R, N, ZDiv<R>>, R>;
    if constexpr (std::is_same<R, double>::value) {
      s.z_disp = run_z<ZPassD<R, N, ZDisp<R>>, R>;
      s.z_dispT = run_z<ZPassD<R, N, ZDispT<R>>, R>;
    }
  } else {
    s.yf = run_y<YPass<R, N, false>, R>;
    s.yi = run_y<YPass<R, N, true>, R>;
    s.z_proj = run_z<ZPass<R, N, ZProject<R>>, R>;
    s.z_lap = run_z<ZPass<R, N, ZLaplace<R>>, R>;
    s.z_prec = run_z<ZPass<R, N, ZPrecond<R>>, R>;
    s.z_grad = run_z<ZPass<R, N, ZGrad<R>>, R>;
    s.z_div = run_z<ZPass<R, N, ZDiv<R>>, R>;
    if constexpr (std::is_same<R, double>::value) {
      s.z_disp = run_z<ZPass<R, N, ZDisp<R>>, R>;
      s.z_dispT = run_z<ZPass<R, N, ZDispT<R>>, R>;
    }
  }
  if constexpr (std::is_same<R, float>::value && (N == 128 || N == 256)) {
    s.yzy_proj = run_yzy_cluster<R, N>;
    s.yzy_proj_ok = yzy_cluster_ok<R, N>;
    s.yzy_grad = run_yzy_cluster<R, N, ZWhole<ZGrad<R>>>;
    s.yzy_div = run_yzy_cluster<R, N, ZWhole<ZDiv<R>>>;
    s.yzy_chem_ok = [] {
      return yzy_cluster_ok<R, N, ZWhole<ZGrad<R>>>() && yzy_cluster_ok<R, N, ZWhole<ZDiv<R>>>();
    };
  }
  return s;
}

// Float-float launchers: the passes of the FP64 residual transforms only (projection of a
// nine-component field, the chemistry gradient-flux-divergence chain), reading and writing
// FP64 real fields.
template <int N>
SizeOps<ff> make_size_ops_ff() {
  SizeOps<ff> s{};
  s.N = N;
  if constexpr (N % 2 == 0) {
    s.xf_copy1 = run_x<XFwd<ff, N, PCopy<ff, 1>>, ff>;
    s.xf_copy3 = run_x<XFwd<ff, N, PCopy<ff, 3>>, ff>;
    s.xf_copy9 = run_x<XFwd<ff, N, PCopy<ff, 9>>, ff>;
    s.xi_norm9 = run_x<XInv<ff, N, ENorm<ff, 9>>, ff>;
    s.xi_chemflux = run_x<XInv<ff, N, EChemFlux<ff>>, ff>;
    s.xi_chemrhs = run_x<XInv<ff, N, EChemRhs<ff>>, ff>;
  }
  if constexpr (Square<N>::OK) {
    s.yf = run_y<YPassD<ff, N, false>, ff>;
    s.yi = run_y<YPassD<ff, N, true>, ff>;
    s.z_proj = run_z<ZPassD<ff, N, ZProject<ff>>, ff>;
    s.z_grad = run_z<ZPassD<ff, N, ZGrad<ff>>, ff>;
    s.z_div = run_z<ZPassD<ff, N, ZDiv<ff>>, ff>;
  } else {
    s.yf = run_y<YPass<ff, N, false>, ff>;
    s.yi = run_y<YPass<ff, N, true>, ff>;
    s.z_proj = run_z<ZPass<ff, N, ZProject<ff>>, ff>;
    s.z_grad = run_z<ZPass<ff, N, ZGrad<ff>>, ff>;
    s.z_div = run_z<ZPass<ff, N, ZDiv<ff>>, ff>;
  }
  return s;
}

// Registry: each instantiation unit registers the sizes it compiles.
template <typename R>
const SizeOps<R>* size_ops(int N);
void register_size_ops_f(const SizeOps<float>& s);
void register_size_ops_d(const SizeOps<double>& s);
void register_size_ops_ff(const SizeOps<ff>& s);

}  // namespace fg
