// Shared-memory tile FFT: several rows of length N transformed together by a block.
//
// Each stage is one radix-R step of the Stockham auto-sort formulation (Govindaraju et
// al., "High performance discrete Fourier transforms on graphics processors", SC 2008):
// butterfly b of a stage with Ns = product of the earlier radices reads elements
// b + r N/R, multiplies element r by exp(-+2 pi i r (b mod Ns) / (Ns R)), does an R-point
// DFT in registers and writes element r to (b / Ns) Ns R + (b mod Ns) + r Ns.  After the
// last stage the row is in natural order.  Stages run in place: a phase reads every
// butterfly's inputs into the thread's carried registers, the next phase writes them.
#pragma once
#include "fg_common.cuh"

namespace fg {

template <typename R, int N, int NROWS, int NT, bool INV>
struct TileFFT {
  using C = cplx<R>;
  static constexpr Plan P = make_plan(N);
  static constexpr int PITCH = row_pitch(N);

  template <int S>
  struct Stage {
    static constexpr int RAD = P.r[S];
    static constexpr int NS = plan_ns(N, S);
    static constexpr int NB = N / RAD;
    static constexpr int ITEMS = NROWS * NB;
    static constexpr int W = (ITEMS + NT - 1) / NT;
    static constexpr int TWS = N / (NS * RAD);

    FG_DEV static void load(int tid, C* v, const C* tile, const C* tw) {
#pragma unroll
      for (int w = 0; w < W; ++w) {
        const int item = tid + w * NT;
        if (W * NT == ITEMS || item < ITEMS) {
          const int row = item / NB, b = item - row * NB;
          const int k = b % NS;
          const C* t = tile + row * PITCH;
          C* x = v + w * RAD;
#pragma unroll
          for (int r = 0; r < RAD; ++r) x[r] = t[pad16(b + r * NB)];
          if (NS > 1) {
#pragma unroll
            for (int r = 1; r < RAD; ++r) {
              const C wt = tw[r * k * TWS];
              x[r] = INV ? cmulc(x[r], wt) : cmul(x[r], wt);
            }
          }
          Dft<RAD, INV, C>::run(x);
        }
      }
    }

    FG_DEV static void store(int tid, const C* v, C* tile) {
#pragma unroll
      for (int w = 0; w < W; ++w) {
        const int item = tid + w * NT;
        if (W * NT == ITEMS || item < ITEMS) {
          const int row = item / NB, b = item - row * NB;
          const int k = b % NS;
          const int j = (b / NS) * NS * RAD + k;
          C* t = tile + row * PITCH;
          const C* x = v + w * RAD;
#pragma unroll
          for (int r = 0; r < RAD; ++r) t[pad16(j + r * NS)] = x[r];
        }
      }
    }
  };

  template <int S>
  static constexpr int vneed() {
    if constexpr (S >= P.S) {
      return 1;
    } else {
      constexpr int here = Stage<S>::W * Stage<S>::RAD;
      constexpr int rest = vneed<S + 1>();
      return here > rest ? here : rest;
    }
  }
  static constexpr int VMAX = vneed<0>();
};

// Runs every stage of a TileFFT on `tile`; must be called from a kernel body that has
// the thread-locals array `Ls` in scope (see FG_PHASE).  Locals must hold `C v[VMAX]`.
template <class TF, int S, class Loc>
FG_DEV void tile_fft(Loc* Ls, typename TF::C* tile, const typename TF::C* tw, int nt) {
  if constexpr (S < TF::P.S) {
    FG_PHASE(nt)
    TF::template Stage<S>::load(tid, L.v, tile, tw);
    FG_END_PHASE
    FG_PHASE(nt)
    TF::template Stage<S>::store(tid, L.v, tile);
    FG_END_PHASE
    tile_fft<TF, S + 1>(Ls, tile, tw, nt);
  }
}

}  // namespace fg
