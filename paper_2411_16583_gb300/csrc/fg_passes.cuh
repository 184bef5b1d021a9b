// The five passes of one operator application y = F^-1[ Op_k . F[ Op_x(x) ] ] on an
// Nx x Ny x Nz periodic grid (Sec. 3.2; Eqs. mechanicalsolve, PFFA, PFFprecond,
// ChemresidualFourier_A).
//
//   X-fwd  real rows along x  -> fused pointwise prologue, R2C along x    -> S1 [c][kx][z][y]
//   Y-fwd  S1 rows along y    -> complex FFT along y, transposed store    -> S2 [c][kx][ky][z]
//   Z      S2 rows along z    -> FFT z, frequency-space operator, IFFT z  -> S2 (in place)
//   Y-inv  S2 (transposed)    -> inverse FFT along y                      -> S1
//   X-inv  S1 (transposed)    -> C2R along x, fused pointwise epilogue    -> real fields
//
// Every pass reads one side as whole contiguous rows and the other as runs of consecutive
// rows, so each global access is a contiguous segment.  Two real rows are transformed as
// one complex row (a + i b) and separated with the Hermitian symmetry of real data.
// The forward transform is unnormalised; the 1/V of the inverse is applied in the Z pass.
#pragma once
#include <type_traits>
#include "fg_fft.cuh"

namespace fg {

template <typename R>
struct PassArgs {
  using C = cplx<R>;
  using IO = io_t<R>;   // storage type of the real-space fields (FP64 for float-float)
  int nx, ny, nz, hx;   // hx = nx/2 + 1
  long long V, VH;      // voxels, half-spectrum points per component
  const IO* rin;        // real input fields (X-fwd prologue)
  IO* rout;             // real output fields (X-inv epilogue)
  IO* rout2;            // second real output (fused Krylov updates)
  const C* cin;         // complex input
  C* cout;              // complex output
  const C* tw;          // exp(-2 pi i m / N), m < N, for this pass's axis
  // per-axis frequency tables (Z pass), index k in [0, n_j) ([0, hx) for x)
  const R* rs[3];       // rotated scheme: (2/h_j) sin(pi k / n_j)
  const R* rc[3];       // rotated scheme: cos(pi k / n_j), exactly 0 at Nyquist
  const C* xi[3];       // forward difference: (exp(2 pi i k / n_j) - 1) / h_j
  const R* lap[3];      // 4 sin^2(pi k / n_j) / h_j^2
  const IO* aux[4];     // operator inputs (state, p, H, ...)
  R coef[4];            // operator constants
  const double* dscal;  // device scalars read by operators
  double* partials;     // one partial sum per block (reducing epilogues)
  const int* done;      // early exit when *done != 0 (converged Krylov loop)
  int ncomp;            // components (Y passes)
  int row_lo, row_hi;   // Y and Z passes: rows [row_lo, row_hi) only (row_hi = 0: all)
  int l2pf;             // X passes: prefetch the block's real-space rows into L2 first
};

// ------------------------------------------------------------------ L2 bulk prefetch
// cp.async.bulk.prefetch.L2 hands a contiguous range to the bulk-copy (TMA) unit, which
// brings it into L2 while the block goes on: the X passes issue it at their start for the
// real-space rows their prologue or epilogue reads, so those loads hit L2 instead of
// waiting on DRAM.  A hint only (no completion to wait for); ranges must start and end on
// 16-byte boundaries, and misaligned ones are skipped.  In the host emulation the range's
// first and last bytes are read instead, so the bounds-checked buffers catch a range that
// leaves its buffer.
FG_DEV void l2_prefetch(const void* p, long long bytes) {
  if (!p || bytes < 16) return;
  const unsigned long long u = (unsigned long long)p;
  if (u & 15) return;
  bytes &= ~15LL;
#ifdef FG_EMU
  volatile const char* c = (const char*)p;
  (void)c[0];
  (void)c[bytes - 1];
#else
  for (long long o = 0; o < bytes; o += (1LL << 20)) {
    const unsigned n = (unsigned)(bytes - o < (1LL << 20) ? bytes - o : (1LL << 20));
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"((const char*)p + o), "r"(n)
                 : "memory");
  }
#endif
}

// Epilogues that can load an element's operands apart from its update (Op::Ops,
// Op::load_ops, Op::apply_ops): X-inv then loads the operands of a group of elements
// before it updates any of them, so each thread has several loads in flight.
template <class Op, class = void>
struct HasOps : std::false_type {};
template <class Op>
struct HasOps<Op, std::void_t<typename Op::Ops>> : std::true_type {};
constexpr int XINV_GROUP = 4;

// Components of each real-space field an X-pass functor reads (0: none); functors that
// declare none are not prefetched.
template <class Op, class = void>
struct PfCounts {
  static constexpr int rin = 0, rout = 0, rout2 = 0, aux0 = 0, aux1 = 0;
};
template <class Op>
struct PfCounts<Op, std::void_t<decltype(Op::PF_AUX0)>> {
  static constexpr int rin = Op::PF_RIN, rout = Op::PF_ROUT, rout2 = Op::PF_ROUT2,
                       aux0 = Op::PF_AUX0, aux1 = Op::PF_AUX1;
};

// rows [e0, e0 + ne) (element offsets within a component) of `comps` components V apart
template <typename T>
FG_DEV void prefetch_rows(const T* p, int comps, long long V, long long e0, long long ne) {
  for (int c = 0; c < comps; ++c) l2_prefetch(p + c * V + e0, ne * (long long)sizeof(T));
}

template <class Op, typename R>
FG_DEV void prefetch_op_rows(const PassArgs<R>& a, long long e0, long long ne, int percomp) {
  using P = PfCounts<Op>;
  const int k = percomp;
  prefetch_rows(a.rin, k ? (P::rin ? 1 : 0) : P::rin, a.V, e0, ne);
  prefetch_rows(a.rout, k ? (P::rout ? 1 : 0) : P::rout, a.V, e0, ne);
  prefetch_rows(a.rout2, k ? (P::rout2 ? 1 : 0) : P::rout2, a.V, e0, ne);
  prefetch_rows(a.aux[0], k ? (P::aux0 ? 1 : 0) : P::aux0, a.V, e0, ne);
  prefetch_rows(a.aux[1], k ? (P::aux1 ? 1 : 0) : P::aux1, a.V, e0, ne);
}

// ------------------------------------------------------------------ tile sizing

constexpr int tpr(int N) { return N / make_plan(N).rmax; }
constexpr int round32(int n) { return (n + 31) / 32 * 32; }

constexpr int rows_x(int N, int ncomp, int csize) {
  int rows = 64;
  while (rows > 2 && (ncomp * (rows / 2) * row_pitch(N) * csize > 80 * 1024 ||
                      ncomp * (rows / 2) * tpr(N) > 1024 || ncomp * (rows / 2) > 64))
    rows /= 2;
  return rows;
}
constexpr int rows_y(int N, int csize) {
  int rows = 64;
  while (rows > 1 && (rows * row_pitch(N) * csize > 40 * 1024 || rows * tpr(N) > 512)) rows /= 2;
  return rows;
}
constexpr int rows_z(int N, int ncomp, int csize) {
  int rows = 16;
  while (rows > 1 && (ncomp * rows * row_pitch(N) * csize > 48 * 1024 ||
                      ncomp * rows * tpr(N) > 1024))
    rows /= 2;
  return rows;
}

// ------------------------------------------------------------------ block reduction
// Sums L.acc over the block into a.partials[block]; uses the `red` scratch (NT doubles).

#ifdef FG_EMU
#define FG_BLOCK_REDUCE(NT_, red, out)                     \
  {                                                        \
    double s_ = 0.0;                                       \
    for (int t_ = 0; t_ < (NT_); ++t_) s_ += Ls[t_].acc.value(); \
    out = s_;                                              \
  }
#else
#define FG_BLOCK_REDUCE(NT_, red, out)                                      \
  {                                                                         \
    double v_ = Ls[0].acc.value();                                          \
    for (int o_ = 16; o_ > 0; o_ >>= 1) v_ += __shfl_down_sync(0xffffffffu, v_, o_); \
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v_;                \
    __syncthreads();                                                        \
    if (threadIdx.x == 0) {                                                 \
      double s_ = 0.0;                                                      \
      for (int w_ = 0; w_ < (NT_) / 32; ++w_) s_ += red[w_];                \
      out = s_;                                                             \
    }                                                                       \
  }
#endif

FG_DEV long long block_linear(Dim3 b, int gx, int gy) {
  return ((long long)b.z * gy + b.y) * gx + b.x;
}

// ------------------------------------------------------------------ X-fwd

template <typename R, int N, class Op>
struct XFwd {
  using C = cplx<R>;
  static constexpr int CO = Op::COUT;
  static constexpr int ROWS = rows_x(N, CO, sizeof(C));
  static constexpr int CR = ROWS / 2;
  static constexpr int NROWS = CO * CR;
  static constexpr int NT = round32(NROWS * tpr(N));
  using TF = TileFFT<R, N, NROWS, NT, false>;
  static constexpr int PITCH = TF::PITCH;
  struct Locals {
    C v[TF::VMAX];
    Acc<R> acc;
  };
  static size_t smem_bytes() { return (size_t)(NROWS * PITCH + N) * sizeof(C) + NT * sizeof(double); }
  static int grid_x(int ny, int nz) { return (ny * nz + ROWS - 1) / ROWS; }

  template <class Loc>
  FG_DEV static void body(const PassArgs<R>& a, Dim3 bid, Dim3 grid, char* smem, Loc* Ls) {
    if (a.done && *a.done) return;
    C* tile = (C*)smem;
    C* tw = tile + NROWS * PITCH;
    double* red = (double*)(tw + N);
    (void)red;
    const int nrows = a.ny * a.nz;
    const int row0 = bid.x * ROWS;
    const int nr = nrows - row0 < ROWS ? nrows - row0 : ROWS;
    FG_PHASE(NT)
    if (a.l2pf && tid == 0) prefetch_op_rows<Op>(a, (long long)row0 * N, (long long)nr * N, 0);
    L.acc.zero();
    // device scalars of the fused Krylov updates, converted once per thread
    const R sc[2] = {a.dscal ? (R)a.dscal[0] : (R)0, a.dscal ? (R)a.dscal[1] : (R)0};
    for (int m = tid; m < N; m += NT) tw[m] = a.tw[m];
    for (int e = tid; e < ROWS * N; e += NT) {
      const int r = e / N, x = e - r * N;
      R out[CO];
      if (r < nr) {
        Op::apply(a, (long long)(row0 + r) * N + x, out, L.acc, sc);
      } else {
#pragma unroll
        for (int c = 0; c < CO; ++c) out[c] = (R)0;
      }
#pragma unroll
      for (int c = 0; c < CO; ++c) {
        C& z = tile[(c * CR + (r >> 1)) * PITCH + pad16(x)];
        if (r & 1) z.y = out[c]; else z.x = out[c];
      }
    }
    FG_END_PHASE
    tile_fft<TF, 0>(Ls, tile, tw, NT);
    FG_PHASE(NT)
    constexpr int H = N / 2 + 1;
    for (int e = tid; e < CO * nr * H; e += NT) {
      const int r = e % nr, t = e / nr;
      const int kx = t % H, c = t / H;
      const C* row = tile + (c * CR + (r >> 1)) * PITCH;
      const C zk = row[pad16(kx)];
      const C zn = row[pad16((N - kx) % N)];
      C val;
      if (!(r & 1)) {
        val = cmk<C>((zk.x + zn.x) * (R)0.5, (zk.y - zn.y) * (R)0.5);
      } else {
        const R dx = zk.x - zn.x, dy = zk.y + zn.y;
        val = cmk<C>(dy * (R)0.5, -dx * (R)0.5);
      }
      a.cout[c * a.VH + (long long)kx * nrows + row0 + r] = val;
    }
    FG_END_PHASE
    if constexpr (Op::RED) {
      double s = 0.0;
      FG_BLOCK_REDUCE(NT, red, s)
#ifdef FG_EMU
      a.partials[block_linear(bid, grid.x, grid.y)] = s;
#else
      if (threadIdx.x == 0) a.partials[block_linear(bid, grid.x, grid.y)] = s;
#endif
    }
  }
};

// ------------------------------------------------------------------ X-inv

// PERCOMP: one component per block (component = blockIdx.y), for epilogues that act on
// each component separately; the 1-component tile is 8x taller, so the transposed reads
// of the spectrum are runs of 64 rows.
template <typename R, int N, class Op, bool PERCOMP = false>
struct XInv {
  using C = cplx<R>;
  static constexpr int CI = Op::CIN;
  static constexpr int ROWS = rows_x(N, CI, sizeof(C));
  static constexpr int CR = ROWS / 2;
  static constexpr int NROWS = CI * CR;
  static constexpr int NT = round32(NROWS * tpr(N));
  using TF = TileFFT<R, N, NROWS, NT, true>;
  static constexpr int PITCH = TF::PITCH;
  struct Locals {
    C v[TF::VMAX];
    Acc<R> acc;
  };
  static constexpr size_t SMEM = (size_t)(NROWS * PITCH + N) * sizeof(C) + NT * sizeof(double);
  static size_t smem_bytes() { return SMEM; }
  static int grid_x(int ny, int nz) { return (ny * nz + ROWS - 1) / ROWS; }
  // blocks per SM the shared memory (227 KB usable, 1 KB reserved per block) and the
  // threads (2048) allow, at most 4, declared to the compiler so that registers do not cap
  // residency below it: the inverse pass is latency-bound on its loads (long-scoreboard
  // stalls)
  static constexpr int MINB_SMEM = (int)((227 * 1024) / (SMEM + 1024));
  static constexpr int MINB_THR = 2048 / NT;
  static constexpr int MINB_RAW = MINB_SMEM < MINB_THR ? MINB_SMEM : MINB_THR;
  static constexpr int MINB = MINB_RAW < 1 ? 1 : (MINB_RAW > 4 ? 4 : MINB_RAW);

  template <class Loc>
  FG_DEV static void body(const PassArgs<R>& a0, Dim3 bid, Dim3 grid, char* smem, Loc* Ls) {
    if (a0.done && *a0.done) return;
    PassArgs<R> a = a0;
    if constexpr (PERCOMP) {  // component bid.y: shift every per-component pointer
      const int cc = bid.y;
      a.cin += cc * a.VH;
      a.rout += cc * a.V;
      if (a.rout2) a.rout2 += cc * a.V;
      if (a.aux[0]) a.aux[0] += cc * a.V;
    }
    C* tile = (C*)smem;
    C* tw = tile + NROWS * PITCH;
    double* red = (double*)(tw + N);
    (void)red;
    const int nrows = a.ny * a.nz;
    const int row0 = bid.x * ROWS;
    const int nr = nrows - row0 < ROWS ? nrows - row0 : ROWS;
    FG_PHASE(NT)
    if (a.l2pf && tid == 0)
      prefetch_op_rows<Op>(a, (long long)row0 * N, (long long)nr * N, PERCOMP ? 1 : 0);
    L.acc.zero();
    for (int m = tid; m < N; m += NT) tw[m] = a.tw[m];
    constexpr int H = N / 2 + 1;
    constexpr int G = XINV_GROUP;
    // spectrum pairs of G elements loaded before any is unpacked into the tile
    for (int e0 = tid; e0 < CI * CR * H; e0 += G * NT) {
      C A[G], B[G];
#pragma unroll
      for (int u = 0; u < G; ++u) {
        const int e = e0 + u * NT;
        const int q = e % CR, t = e / CR;
        const int kx = t % H, c = t / H;
        const int r0 = 2 * q;
        if (e < CI * CR * H && r0 < nr) {
          const long long base = c * a.VH + (long long)kx * nrows + row0 + r0;
          A[u] = a.cin[base];
          B[u] = (r0 + 1 < nr) ? a.cin[base + 1] : cmk<C>((R)0, (R)0);
        }
      }
#pragma unroll
      for (int u = 0; u < G; ++u) {
        const int e = e0 + u * NT;
        const int q = e % CR, t = e / CR;
        const int kx = t % H, c = t / H;
        const int r0 = 2 * q;
        if (e < CI * CR * H && r0 < nr) {
          C* row = tile + (c * CR + q) * PITCH;
          if (kx == 0 || 2 * kx == N) {
            row[pad16(kx)] = cmk<C>(A[u].x, B[u].x);
          } else {
            row[pad16(kx)] = cmk<C>(A[u].x - B[u].y, A[u].y + B[u].x);
            row[pad16(N - kx)] = cmk<C>(A[u].x + B[u].y, B[u].x - A[u].y);
          }
        }
      }
    }
    FG_END_PHASE
    tile_fft<TF, 0>(Ls, tile, tw, NT);
    FG_PHASE(NT)
    const R sc[2] = {a.dscal ? (R)a.dscal[0] : (R)0, a.dscal ? (R)a.dscal[1] : (R)0};
    if constexpr (HasOps<Op>::value) {
      // groups of XINV_GROUP elements: every operand load of the group is issued before
      // the first update (elements are distinct, so no update feeds a load of the group)
      for (int e0 = tid; e0 < nr * N; e0 += XINV_GROUP * NT) {
        typename Op::Ops o[XINV_GROUP];
#pragma unroll
        for (int u = 0; u < XINV_GROUP; ++u) {
          const int e = e0 + u * NT;
          if (e < nr * N) {
            const int r = e / N, x = e - r * N;
            o[u] = Op::load_ops(a, (long long)(row0 + r) * N + x);
          }
        }
#pragma unroll
        for (int u = 0; u < XINV_GROUP; ++u) {
          const int e = e0 + u * NT;
          if (e < nr * N) {
            const int r = e / N, x = e - r * N;
            R val[CI];
#pragma unroll
            for (int c = 0; c < CI; ++c) {
              const C z = tile[(c * CR + (r >> 1)) * PITCH + pad16(x)];
              val[c] = (r & 1) ? z.y : z.x;
            }
            Op::apply_ops(a, (long long)(row0 + r) * N + x, o[u], val, L.acc, sc);
          }
        }
      }
    } else {
      for (int e = tid; e < nr * N; e += NT) {
        const int r = e / N, x = e - r * N;
        R val[CI];
#pragma unroll
        for (int c = 0; c < CI; ++c) {
          const C z = tile[(c * CR + (r >> 1)) * PITCH + pad16(x)];
          val[c] = (r & 1) ? z.y : z.x;
        }
        Op::apply(a, (long long)(row0 + r) * N + x, val, L.acc, sc);
      }
    }
    FG_END_PHASE
    if constexpr (Op::RED) {
      double s = 0.0;
      FG_BLOCK_REDUCE(NT, red, s)
#ifdef FG_EMU
      a.partials[block_linear(bid, grid.x, grid.y)] = s;
#else
      if (threadIdx.x == 0) a.partials[block_linear(bid, grid.x, grid.y)] = s;
#endif
    }
  }
};

// ------------------------------------------------------------------ X round trip

// Inverse x-transform, a pointwise map and the forward x-transform in one pass: the
// spectrum rows (transposed layout, CI components) come in, are turned into real rows
// (C2R) in shared memory, Op maps the CI real values of each voxel to CO values in place,
// and the forward R2C of those rows goes back out transposed.  The real-space
// intermediate never reaches global memory.  Op::apply(a, v, val[CI], out[CO], acc, sc);
// reducing ops write one partial sum per block.
template <typename R, int N, class Op>
struct XRound {
  using C = cplx<R>;
  static constexpr int CI = Op::CIN, CO = Op::COUT;
  static_assert(CI == CO, "the tile holds the same components before and after");
  static constexpr int ROWS = rows_x(N, CI, sizeof(C));
  static constexpr int CR = ROWS / 2;
  static constexpr int NROWS = CI * CR;
  static constexpr int NT = round32(NROWS * tpr(N));
  using TFi = TileFFT<R, N, NROWS, NT, true>;
  using TFf = TileFFT<R, N, NROWS, NT, false>;
  static constexpr int PITCH = TFi::PITCH;
  static constexpr int VMAX = TFi::VMAX > TFf::VMAX ? TFi::VMAX : TFf::VMAX;
  struct Locals {
    C v[VMAX];
    Acc<R> acc;
  };
  static size_t smem_bytes() { return (size_t)(NROWS * PITCH + N) * sizeof(C) + NT * sizeof(double); }
  static int grid_x(int ny, int nz) { return (ny * nz + ROWS - 1) / ROWS; }

  template <class Loc>
  FG_DEV static void body(const PassArgs<R>& a, Dim3 bid, Dim3 grid, char* smem, Loc* Ls) {
    if (a.done && *a.done) return;
    C* tile = (C*)smem;
    C* tw = tile + NROWS * PITCH;
    double* red = (double*)(tw + N);
    (void)red;
    const int nrows = a.ny * a.nz;
    const int row0 = bid.x * ROWS;
    const int nr = nrows - row0 < ROWS ? nrows - row0 : ROWS;
    constexpr int H = N / 2 + 1;
    FG_PHASE(NT)
    if (a.l2pf && tid == 0) prefetch_op_rows<Op>(a, (long long)row0 * N, (long long)nr * N, 0);
    L.acc.zero();
    for (int m = tid; m < N; m += NT) tw[m] = a.tw[m];
    for (int e = tid; e < CI * CR * H; e += NT) {
      const int q = e % CR, t = e / CR;
      const int kx = t % H, c = t / H;
      const int r0 = 2 * q;
      C* row = tile + (c * CR + q) * PITCH;
      if (r0 < nr) {
        const long long base = c * a.VH + (long long)kx * nrows + row0 + r0;
        const C A = a.cin[base];
        const C B = (r0 + 1 < nr) ? a.cin[base + 1] : cmk<C>((R)0, (R)0);
        if (kx == 0 || 2 * kx == N) {
          row[pad16(kx)] = cmk<C>(A.x, B.x);
        } else {
          row[pad16(kx)] = cmk<C>(A.x - B.y, A.y + B.x);
          row[pad16(N - kx)] = cmk<C>(A.x + B.y, B.x - A.y);
        }
      } else {  // rows past the grid: zeros, so the forward transform sees zero rows
        row[pad16(kx)] = cmk<C>((R)0, (R)0);
        if (kx != 0 && 2 * kx != N) row[pad16(N - kx)] = cmk<C>((R)0, (R)0);
      }
    }
    FG_END_PHASE
    tile_fft<TFi, 0>(Ls, tile, tw, NT);
    FG_PHASE(NT)
    const R sc[2] = {a.dscal ? (R)a.dscal[0] : (R)0, a.dscal ? (R)a.dscal[1] : (R)0};
    for (int e = tid; e < nr * N; e += NT) {
      const int r = e / N, x = e - r * N;
      R val[CI], out[CO];
#pragma unroll
      for (int c = 0; c < CI; ++c) {
        const C z = tile[(c * CR + (r >> 1)) * PITCH + pad16(x)];
        val[c] = (r & 1) ? z.y : z.x;
      }
      Op::apply(a, (long long)(row0 + r) * N + x, val, out, L.acc, sc);
#pragma unroll
      for (int c = 0; c < CO; ++c) {
        C& z = tile[(c * CR + (r >> 1)) * PITCH + pad16(x)];
        if (r & 1) z.y = out[c]; else z.x = out[c];
      }
    }
    // an odd last row's partner (the imaginary half of its complex row) is zero
    if (nr & 1)
      for (int e = tid; e < CO * N; e += NT) {
        const int c = e / N, x = e - c * N;
        tile[(c * CR + (nr >> 1)) * PITCH + pad16(x)].y = (R)0;
      }
    FG_END_PHASE
    tile_fft<TFf, 0>(Ls, tile, tw, NT);
    FG_PHASE(NT)
    for (int e = tid; e < CO * nr * H; e += NT) {
      const int r = e % nr, t = e / nr;
      const int kx = t % H, c = t / H;
      const C* row = tile + (c * CR + (r >> 1)) * PITCH;
      const C zk = row[pad16(kx)];
      const C zn = row[pad16((N - kx) % N)];
      C val;
      if (!(r & 1)) {
        val = cmk<C>((zk.x + zn.x) * (R)0.5, (zk.y - zn.y) * (R)0.5);
      } else {
        const R dx = zk.x - zn.x, dy = zk.y + zn.y;
        val = cmk<C>(dy * (R)0.5, -dx * (R)0.5);
      }
      a.cout[c * a.VH + (long long)kx * nrows + row0 + r] = val;
    }
    FG_END_PHASE
    if constexpr (Op::RED) {
      double s = 0.0;
      FG_BLOCK_REDUCE(NT, red, s)
#ifdef FG_EMU
      a.partials[block_linear(bid, grid.x, grid.y)] = s;
#else
      if (threadIdx.x == 0) a.partials[block_linear(bid, grid.x, grid.y)] = s;
#endif
    }
  }
};

// ------------------------------------------------------------------ Y passes

template <typename R, int N, bool INV>
struct YPass {
  using C = cplx<R>;
  static constexpr int ROWS = rows_y(N, sizeof(C));
  static constexpr int NT = round32(ROWS * tpr(N));
  using TF = TileFFT<R, N, ROWS, NT, INV>;
  static constexpr int PITCH = TF::PITCH;
  struct Locals {
    C v[TF::VMAX];
    Acc<R> acc;
  };
  static size_t smem_bytes() { return (size_t)(ROWS * PITCH + N) * sizeof(C); }
  static int grid_x(int hx, int nz) { return (hx * nz + ROWS - 1) / ROWS; }

  // element (row s of the (kx, z) rows, index n along y) in the [c][kx][ky][z] layout
  FG_DEV static long long tpos(int s, int n, int nz) {
    const int kx = s / nz, z = s - kx * nz;
    return ((long long)kx * N + n) * nz + z;
  }

  template <class Loc>
  FG_DEV static void body(const PassArgs<R>& a, Dim3 bid, Dim3 grid, char* smem, Loc* Ls) {
    if (a.done && *a.done) return;
    C* tile = (C*)smem;
    C* tw = tile + ROWS * PITCH;
    const int c = bid.y;
    const int nrows = a.row_hi > 0 ? a.row_hi : a.hx * a.nz;
    const int row0 = a.row_lo + bid.x * ROWS;
    const int nr = nrows - row0 < ROWS ? nrows - row0 : ROWS;
    const C* in = a.cin + c * a.VH;
    C* out = a.cout + c * a.VH;
    const bool rfast = a.nz >= 4;  // runs of consecutive rows are long enough to coalesce
    FG_PHASE(NT)
    for (int m = tid; m < N; m += NT) tw[m] = a.tw[m];
    for (int e = tid; e < nr * N; e += NT) {
      int r, n;
      if (!INV || !rfast) { r = e / N; n = e - r * N; }
      else { n = e / nr; r = e - n * nr; }
      const long long g = INV ? tpos(row0 + r, n, a.nz) : (long long)(row0 + r) * N + n;
      tile[r * PITCH + pad16(n)] = in[g];
    }
    FG_END_PHASE
    tile_fft<TF, 0>(Ls, tile, tw, NT);
    FG_PHASE(NT)
    for (int e = tid; e < nr * N; e += NT) {
      int r, n;
      if (INV || !rfast) { r = e / N; n = e - r * N; }
      else { n = e / nr; r = e - n * nr; }
      const long long g = INV ? (long long)(row0 + r) * N + n : tpos(row0 + r, n, a.nz);
      out[g] = tile[r * PITCH + pad16(n)];
    }
    FG_END_PHASE
  }
};

// ------------------------------------------------------------------ register-direct passes
// For a two-stage plan N = R0 R1 (64 = 8 x 8, 256 = 16 x 16, 128 = 16 x 8, 48 = 16 x 3,
// 80 = 16 x 5, ...) the first stage reads its butterfly inputs straight from global memory
// into registers (T0 = N / R0 butterflies per row) and the last
// stage writes its outputs straight to global memory: every element crosses shared
// memory once between the stages.  Thread-to-row maps are chosen per stage so that the
// global side of each stage is coalesced (row-fastest for transposed layouts).

template <int N>
struct Square {  // two-stage plans N = R0 R1: register-direct Y and Z passes
  static constexpr Plan P = make_plan(N);
  static constexpr bool OK = P.S == 2;
  static constexpr int R0 = P.r[0], R1 = P.r[1];
  static constexpr int T0 = N / R0, T1 = N / R1;  // butterflies per row in stage 0 and 1
  static constexpr int RM = R0 > R1 ? R0 : R1, TM = T0 > T1 ? T0 : T1;
};

// stage 0 (Ns = 1): v holds x[b + r T0], r < R0; outputs go to positions b R0 + r
// stage 1 (Ns = R0): v holds positions b + r T1, r < R1 (T1 = N / R1 = R0), twiddle
// exp(-+ 2 pi i r b / N); outputs land in natural order at b + r T1
template <typename C, int RAD, bool INV>
FG_DEV void square_stage1_twiddle(C* v, const C* tw, int b) {
#pragma unroll
  for (int r = 1; r < RAD; ++r) {
    const C w = tw[r * b];
    v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
  }
}

template <typename R, int N, bool INV>
struct YPassD {
  using C = cplx<R>;
  using SQ = Square<N>;
  static constexpr int R0 = SQ::R0, R1 = SQ::R1, T0 = SQ::T0, T1 = SQ::T1;
  // rows per block: the shared-memory budget of rows_y and at most YT threads: 512 for
  // equal radices (64 = 8 x 8, 256 = 16 x 16), 256 for unequal ones, whose stage with the
  // most butterflies sets the threads per row (at 128 = 16 x 8: 16 rows of 16 threads ran
  // the 128^3 operator application in 0.222 ms against 0.230 ms with 32 rows)
  static constexpr int ROWS_M = rows_y(N, sizeof(C));
  static constexpr int YT = SQ::R0 == SQ::R1 ? 512 : 256;
  static constexpr int ROWS = ROWS_M * SQ::TM <= YT ? ROWS_M : (YT / SQ::TM > 0 ? YT / SQ::TM : 1);
  static constexpr int NT = round32(ROWS * SQ::TM);
  static constexpr int PITCH = row_pitch(N);
  struct Locals {
    C v[SQ::RM];
    Acc<R> acc;
  };
  static size_t smem_bytes() { return (size_t)(ROWS * PITCH + N) * sizeof(C); }

  FG_DEV static long long tpos(int s, int n, int nz) {
    const int kx = s / nz, z = s - kx * nz;
    return ((long long)kx * N + n) * nz + z;
  }

  template <class Loc>
  FG_DEV static void body(const PassArgs<R>& a, Dim3 bid, Dim3 grid, char* smem, Loc* Ls) {
    if (a.done && *a.done) return;
    C* tile = (C*)smem;
    C* tw = tile + ROWS * PITCH;
    const int c = bid.y;
    const int nrows = a.row_hi > 0 ? a.row_hi : a.hx * a.nz;
    const int row0 = a.row_lo + bid.x * ROWS;
    const int nr = nrows - row0 < ROWS ? nrows - row0 : ROWS;
    const C* in = a.cin + c * a.VH;
    C* out = a.cout + c * a.VH;
    const bool rfast = a.nz >= 4;
    FG_PHASE(NT)
    for (int m = tid; m < N; m += NT) tw[m] = a.tw[m];
    if (tid < ROWS * T0) {
      int rho, b;  // inputs: transposed layout row-fastest, contiguous rows butterfly-fastest
      if (INV && rfast) { rho = tid % ROWS; b = tid / ROWS; }
      else { b = tid % T0; rho = tid / T0; }
      if (rho < nr) {
#pragma unroll
        for (int r = 0; r < R0; ++r) {
          const int n = b + r * T0;
          L.v[r] = in[INV ? tpos(row0 + rho, n, a.nz) : (long long)(row0 + rho) * N + n];
        }
      } else {
#pragma unroll
        for (int r = 0; r < R0; ++r) L.v[r] = cmk<C>((R)0, (R)0);
      }
      Dft<R0, INV, C>::run(L.v);
#pragma unroll
      for (int r = 0; r < R0; ++r) tile[rho * PITCH + pad16(b * R0 + r)] = L.v[r];
    }
    FG_END_PHASE
    FG_PHASE(NT)
    if (tid < ROWS * T1) {
      int rho, b;  // outputs: transposed layout row-fastest
      if (!INV && rfast) { rho = tid % ROWS; b = tid / ROWS; }
      else { b = tid % T1; rho = tid / T1; }
#pragma unroll
      for (int r = 0; r < R1; ++r) L.v[r] = tile[rho * PITCH + pad16(b + r * T1)];
      square_stage1_twiddle<C, R1, INV>(L.v, tw, b);
      Dft<R1, INV, C>::run(L.v);
      if (rho < nr) {
#pragma unroll
        for (int r = 0; r < R1; ++r) {
          const int n = b + r * T1;
          out[INV ? (long long)(row0 + rho) * N + n : tpos(row0 + rho, n, a.nz)] = L.v[r];
        }
      }
    }
    FG_END_PHASE
  }
};

// RZ > 0 overrides the rows per block (tile-shape variants the autotuner times)
template <typename R, int N, class Op, int RZ = 0>
struct ZPassD {
  using C = cplx<R>;
  using SQ = Square<N>;
  static constexpr int R0 = SQ::R0, R1 = SQ::R1, T0 = SQ::T0, T1 = SQ::T1;
  static constexpr int CI = Op::CIN;
  static constexpr int CO = Op::COUT;
  static constexpr int CM = CI > CO ? CI : CO;
  // rows per block: the shared-memory budget of rows_z, at most 1024 threads
  static constexpr int ROWS_M = rows_z(N, CM, sizeof(C));
  static constexpr int ROWS_T = 1024 / (CM * SQ::TM) > 0 ? 1024 / (CM * SQ::TM) : 1;
  static constexpr int ROWS = RZ > 0 ? RZ : (ROWS_M < ROWS_T ? ROWS_M : ROWS_T);
  static constexpr int NT = round32(CM * ROWS * SQ::TM);
  static constexpr int PITCH = row_pitch(N);
  struct Locals {
    C v[SQ::RM];
    Acc<R> acc;
  };
  static size_t smem_bytes() { return (size_t)(CM * ROWS * PITCH + N) * sizeof(C); }

  template <class Loc>
  FG_DEV static void body(const PassArgs<R>& a, Dim3 bid, Dim3 grid, char* smem, Loc* Ls) {
    if (a.done && *a.done) return;
    C* tile = (C*)smem;
    C* tw = tile + CM * ROWS * PITCH;
    const int nrows = a.row_hi > 0 ? a.row_hi : a.hx * a.ny;
    const int row0 = a.row_lo + bid.x * ROWS;
    const int nr = nrows - row0 < ROWS ? nrows - row0 : ROWS;
    // forward stage 0 from global
    FG_PHASE(NT)
    for (int m = tid; m < N; m += NT) tw[m] = a.tw[m];
    if (tid < CI * ROWS * T0) {
      const int b = tid % T0, q = tid / T0;  // q = c ROWS + rho
      const int rho = q % ROWS, c = q / ROWS;
      if (rho < nr) {
        const C* in = a.cin + c * a.VH + (long long)(row0 + rho) * N;
#pragma unroll
        for (int r = 0; r < R0; ++r) L.v[r] = in[b + r * T0];
      } else {
#pragma unroll
        for (int r = 0; r < R0; ++r) L.v[r] = cmk<C>((R)0, (R)0);
      }
      Dft<R0, false, C>::run(L.v);
      C* t = tile + q * PITCH;
#pragma unroll
      for (int r = 0; r < R0; ++r) t[pad16(b * R0 + r)] = L.v[r];
    }
    FG_END_PHASE
    // forward stage 1 in place (each thread reads and writes the same positions)
    FG_PHASE(NT)
    if (tid < CI * ROWS * T1) {
      const int b = tid % T1, q = tid / T1;
      C* t = tile + q * PITCH;
#pragma unroll
      for (int r = 0; r < R1; ++r) L.v[r] = t[pad16(b + r * T1)];
      square_stage1_twiddle<C, R1, false>(L.v, tw, b);
      Dft<R1, false, C>::run(L.v);
#pragma unroll
      for (int r = 0; r < R1; ++r) t[pad16(b + r * T1)] = L.v[r];
    }
    FG_END_PHASE
    // frequency-space operator on all components of each (row, kz)
    FG_PHASE(NT)
    const R zs = a.dscal ? (R)a.dscal[0] : (R)0;
    for (int e = tid; e < nr * N; e += NT) {
      const int r = e / N, n = e - r * N;
      const int s_ = row0 + r;
      const int kx = s_ / a.ny, ky = s_ - kx * a.ny;
      C v[CM];
#pragma unroll
      for (int c = 0; c < CI; ++c) v[c] = tile[(c * ROWS + r) * PITCH + pad16(n)];
      Op::apply(a, kx, ky, n, v, zs);
#pragma unroll
      for (int c = 0; c < CO; ++c) tile[(c * ROWS + r) * PITCH + pad16(n)] = v[c];
    }
    FG_END_PHASE
    // inverse stage 0: read, then write after the barrier
    FG_PHASE(NT)
    if (tid < CO * ROWS * T0) {
      const int b = tid % T0, q = tid / T0;
      const C* t = tile + q * PITCH;
#pragma unroll
      for (int r = 0; r < R0; ++r) L.v[r] = t[pad16(b + r * T0)];
      Dft<R0, true, C>::run(L.v);
    }
    FG_END_PHASE
    FG_PHASE(NT)
    if (tid < CO * ROWS * T0) {
      const int b = tid % T0, q = tid / T0;
      C* t = tile + q * PITCH;
#pragma unroll
      for (int r = 0; r < R0; ++r) t[pad16(b * R0 + r)] = L.v[r];
    }
    FG_END_PHASE
    // inverse stage 1 straight to global
    FG_PHASE(NT)
    if (tid < CO * ROWS * T1) {
      const int b = tid % T1, q = tid / T1;
      const int rho = q % ROWS, c = q / ROWS;
      const C* t = tile + q * PITCH;
#pragma unroll
      for (int r = 0; r < R1; ++r) L.v[r] = t[pad16(b + r * T1)];
      square_stage1_twiddle<C, R1, true>(L.v, tw, b);
      Dft<R1, true, C>::run(L.v);
      if (rho < nr) {
        C* o = a.cout + c * a.VH + (long long)(row0 + rho) * N;
#pragma unroll
        for (int r = 0; r < R1; ++r) o[b + r * T1] = L.v[r];
      }
    }
    FG_END_PHASE
  }
};

// ------------------------------------------------------------------ Z pass

template <typename R, int N, class Op>
struct ZPass {
  using C = cplx<R>;
  static constexpr int CI = Op::CIN;
  static constexpr int CO = Op::COUT;
  static constexpr int CM = CI > CO ? CI : CO;
  static constexpr int ROWS = rows_z(N, CM, sizeof(C));
  static constexpr int NT = round32(CM * ROWS * tpr(N));
  using TFf = TileFFT<R, N, CI * ROWS, NT, false>;
  using TFi = TileFFT<R, N, CO * ROWS, NT, true>;
  static constexpr int PITCH = TFf::PITCH;
  static constexpr int VMAX = TFf::VMAX > TFi::VMAX ? TFf::VMAX : TFi::VMAX;
  struct Locals {
    C v[VMAX];
    Acc<R> acc;
  };
  static size_t smem_bytes() { return (size_t)(CM * ROWS * PITCH + N) * sizeof(C); }
  static int grid_x(int hx, int ny) { return (hx * ny + ROWS - 1) / ROWS; }

  template <class Loc>
  FG_DEV static void body(const PassArgs<R>& a, Dim3 bid, Dim3 grid, char* smem, Loc* Ls) {
    if (a.done && *a.done) return;
    C* tile = (C*)smem;
    C* tw = tile + CM * ROWS * PITCH;
    const int nrows = a.row_hi > 0 ? a.row_hi : a.hx * a.ny;
    const int row0 = a.row_lo + bid.x * ROWS;
    const int nr = nrows - row0 < ROWS ? nrows - row0 : ROWS;
    FG_PHASE(NT)
    for (int m = tid; m < N; m += NT) tw[m] = a.tw[m];
    for (int e = tid; e < CI * nr * N; e += NT) {
      const int c = e / (nr * N), rem = e - c * (nr * N);
      const int r = rem / N, n = rem - r * N;
      tile[(c * ROWS + r) * PITCH + pad16(n)] = a.cin[c * a.VH + (long long)(row0 + r) * N + n];
    }
    FG_END_PHASE
    tile_fft<TFf, 0>(Ls, tile, tw, NT);
    FG_PHASE(NT)
    const R zs = a.dscal ? (R)a.dscal[0] : (R)0;
    for (int e = tid; e < nr * N; e += NT) {
      const int r = e / N, n = e - r * N;
      const int s = row0 + r;
      const int kx = s / a.ny, ky = s - kx * a.ny;
      C v[CM];
#pragma unroll
      for (int c = 0; c < CI; ++c) v[c] = tile[(c * ROWS + r) * PITCH + pad16(n)];
      Op::apply(a, kx, ky, n, v, zs);
#pragma unroll
      for (int c = 0; c < CO; ++c) tile[(c * ROWS + r) * PITCH + pad16(n)] = v[c];
    }
    FG_END_PHASE
    tile_fft<TFi, 0>(Ls, tile, tw, NT);
    FG_PHASE(NT)
    for (int e = tid; e < CO * nr * N; e += NT) {
      const int c = e / (nr * N), rem = e - c * (nr * N);
      const int r = rem / N, n = rem - r * N;
      a.cout[c * a.VH + (long long)(row0 + r) * N + n] = tile[(c * ROWS + r) * PITCH + pad16(n)];
    }
    FG_END_PHASE
  }
};

}  // namespace fg
