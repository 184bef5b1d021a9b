// Voxel-wise kernels: constitutive state and stress, damage driving force and history,
// chemistry coefficients, Krylov vector updates and the single-block finalisers that
// turn partial sums into the Krylov scalars.  All are grid-stride loops over voxels.
#pragma once
#include "fg_launch.cuh"

namespace fg {

constexpr int VEC_NT = 256;
constexpr int VEC_BLOCKS = 1216;  // 8 x 152 SMs

// Krylov scalars kept on the device (one block per solve).
struct KScal {
  double rz;     // <r, z> (z = r without preconditioner)
  double pq;     // <p, A p>
  double rr;     // <r, r>
  double bb;     // <b, b>
  double tol2;   // tol^2 <b, b>
  double alpha, beta;
  double aux;    // spare sum (mass, norms)
  double rr_best;  // smallest <r, r> at which the iterate was saved
  double pq0;      // <p, A p> of the first direction (p = b)
  int done, iters, maxit, status;
  int nosnap;      // 0 right after <r, r> fell to a quarter of rr_best (save the iterate)
  int snaps;       // iterates saved so far
  int indef;       // 1: continue through directions of negative curvature (Galerkin iterates)
  int negc;        // directions of negative curvature met
};

enum : int { ST_OK = 0, ST_INDEFINITE = 1, ST_DOMAIN = 2, ST_NUMERIC = 4 };

struct VArgs {
  long long n;          // elements processed
  long long V;          // voxels
  const void* in[16];   // inputs (meaning per kernel)
  void* out[6];         // outputs
  double s[10];         // scalars
  double* partials;     // per-block partial sums
  KScal* ks;            // Krylov scalars (may be null)
  const int* done;      // early exit
  int* flags;           // error flags (domain / numeric)
};

// Base of the element functors: AR is the type their per-thread sums accumulate in (the
// arithmetic type of the kernel), Pre the device scalars each thread reads once.
template <typename AR>
struct VecOp {
  using AccReal = AR;
  struct Pre {};
  FG_DEV static Pre pre(const VArgs&) { return Pre{}; }
};

// Generic grid-stride kernel: F::apply(a, i, acc, pre) for every element i.
template <class F>
struct VecKernel {
  static constexpr int NT = VEC_NT;
  using AR = typename F::AccReal;
  struct Locals {
    Acc<AR> acc;
  };
  static size_t smem_bytes() { return NT * sizeof(double); }
  template <class Loc>
  FG_DEV static void body(const VArgs& a, Dim3 bid, Dim3 grid, char* smem, Loc* Ls) {
    if (a.done && *a.done) return;
    double* red = (double*)smem;
    (void)red;
    FG_PHASE(NT)
    L.acc.zero();
    const typename F::Pre pre = F::pre(a);
    for (long long i = (long long)bid.x * NT + tid; i < a.n; i += (long long)grid.x * NT)
      F::apply(a, i, L.acc, pre);
    FG_END_PHASE
    if constexpr (F::RED) {
      double s = 0.0;
      FG_BLOCK_REDUCE(NT, red, s)
#ifdef FG_EMU
      a.partials[bid.x] = s;
#else
      if (threadIdx.x == 0) a.partials[bid.x] = s;
#endif
    }
  }
};

template <class F>
int launch_vec(const VArgs& a, cudaStream_t st) {
  long long nb = (a.n + VEC_NT - 1) / VEC_NT;
  int g = (int)(nb < VEC_BLOCKS ? (nb < 1 ? 1 : nb) : VEC_BLOCKS);
  if (F::RED) g = VEC_BLOCKS;  // fixed count of partial sums
  return launch_pass<VecKernel<F>>(a, Dim3{g, 1, 1}, st);
}

// Single-block finaliser: sums `npart` partials (in a fixed order) and calls F::fin.
template <class F>
struct FinKernel {
  static constexpr int NT = 256;
  struct Locals {
    Acc<double> acc;
  };
  static size_t smem_bytes() { return NT * sizeof(double); }
  template <class Loc>
  FG_DEV static void body(const VArgs& a, Dim3, Dim3, char* smem, Loc* Ls) {
    if (a.done && *a.done) return;
    double* red = (double*)smem;
    FG_PHASE(NT)
    double s = 0.0;
    for (long long i = tid; i < a.n; i += NT) s += a.partials[i];
    red[tid] = s;
    FG_END_PHASE
    FG_PHASE(NT)
    if (tid == 0) {
      double t = 0.0;
      for (int i = 0; i < NT; ++i) t += red[i];
      F::fin(a, t);
    }
    FG_END_PHASE
  }
};

template <class F>
void launch_fin(const VArgs& a, cudaStream_t st) {
  launch_pass<FinKernel<F>>(a, Dim3{1, 1, 1}, st);
}

// ================================================================== 3x3 helpers

FG_DEV double det3(const double* A) {
  return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
         A[2] * (A[3] * A[7] - A[4] * A[6]);
}
// cofactor matrix: cof(A) = det(A) A^-T
FG_DEV void cof3(const double* A, double* C) {
  C[0] = A[4] * A[8] - A[5] * A[7];
  C[1] = A[5] * A[6] - A[3] * A[8];
  C[2] = A[3] * A[7] - A[4] * A[6];
  C[3] = A[2] * A[7] - A[1] * A[8];
  C[4] = A[0] * A[8] - A[2] * A[6];
  C[5] = A[1] * A[6] - A[0] * A[7];
  C[6] = A[1] * A[5] - A[2] * A[4];
  C[7] = A[2] * A[3] - A[0] * A[5];
  C[8] = A[0] * A[4] - A[1] * A[3];
}

// Eigenvalues of a symmetric 3x3 matrix by the trigonometric closed form of
// O. K. Smith, "Eigenvalues of a symmetric 3x3 matrix", Comm. ACM 4 (1961) 168.
FG_DEV void sym_eig3(double a00, double a11, double a22, double a01, double a02, double a12,
                    double* e) {
  const double p1 = a01 * a01 + a02 * a02 + a12 * a12;
  const double q = (a00 + a11 + a22) / 3.0;
  const double b00 = a00 - q, b11 = a11 - q, b22 = a22 - q;
  const double p2 = b00 * b00 + b11 * b11 + b22 * b22 + 2.0 * p1;
  if (p2 <= 0.0) {
    e[0] = e[1] = e[2] = q;
    return;
  }
  const double p = sqrt(p2 / 6.0);
  const double ip = 1.0 / p;
  const double c00 = b00 * ip, c11 = b11 * ip, c22 = b22 * ip;
  const double c01 = a01 * ip, c02 = a02 * ip, c12 = a12 * ip;
  double r = 0.5 * (c00 * (c11 * c22 - c12 * c12) - c01 * (c01 * c22 - c12 * c02) +
                    c02 * (c01 * c12 - c11 * c02));
  r = r < -1.0 ? -1.0 : (r > 1.0 ? 1.0 : r);
  const double phi = acos(r) / 3.0;
  const double two_pi_3 = 2.0943951023931954923;
  e[0] = q + 2.0 * p * cos(phi);
  e[2] = q + 2.0 * p * cos(phi + two_pi_3);
  e[1] = 3.0 * q - e[0] - e[2];
}

// Per-voxel material (FP64 arrays, one per quantity).
struct MatPtrs {
  const double* lam;
  const double* mu;
  const double* Om;
  const double* c0;
};

// Elastic state of one voxel for either law: a = J_c^{-1/3}, F_e = a F, g = (1-d)^2,
// the pristine stress P0(F_e) and the power P0 : F_e (Eqs. Fc, Ee, psie0, pristine).
enum : int { LAW_SVK_ = 0, LAW_NH_ = 1 };

struct ElasticPoint {
  double a, g, Jc, lam, mu;
  double Fe[9], P0[9], P0Fe;
  double B[9], lnJe;  // Neo-Hookean: F^-T and ln J_e
  double S[6];        // Saint-Venant-Kirchhoff: S(E_e) as (xx, yy, zz, xy, xz, yz)
};

template <int LAW>
FG_DEV bool elastic_point(const double* F, double c, double d, double lam, double mu, double Om,
                          double c0, ElasticPoint& P) {
  P.Jc = 1.0 + Om * (c - c0);
  const double J = det3(F);
  if (!(P.Jc > 0.0) || !(J > 0.0)) return false;
  P.a = 1.0 / cbrt(P.Jc);
  P.g = (1.0 - d) * (1.0 - d);
  P.lam = lam;
  P.mu = mu;
#pragma unroll
  for (int k = 0; k < 9; ++k) P.Fe[k] = P.a * F[k];
  if constexpr (LAW == LAW_NH_) {
    // P0 = G (F_e - F_e^-T) + lam ln J_e F_e^-T, with F_e^-T = F^-T / a
    P.lnJe = log(P.a * P.a * P.a * J);
    double C[9];
    cof3(F, C);
    const double iJ = 1.0 / J, ia = 1.0 / P.a;
    double trCe = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      P.B[k] = C[k] * iJ;
      const double FeiT = P.B[k] * ia;
      P.P0[k] = mu * (P.Fe[k] - FeiT) + lam * P.lnJe * FeiT;
      trCe += P.Fe[k] * P.Fe[k];
    }
    P.P0Fe = mu * (trCe - 3.0) + 3.0 * lam * P.lnJe;
  } else {
    // E_e = (F_e^T F_e - I)/2, S = lam tr(E_e) I + 2 G E_e, P0 = F_e S
    double Ce[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        Ce[3 * i + j] = P.Fe[i] * P.Fe[j] + P.Fe[3 + i] * P.Fe[3 + j] + P.Fe[6 + i] * P.Fe[6 + j];
    const double trE = 0.5 * (Ce[0] + Ce[4] + Ce[8] - 3.0);
    const double Sxx = lam * trE + mu * (Ce[0] - 1.0), Syy = lam * trE + mu * (Ce[4] - 1.0);
    const double Szz = lam * trE + mu * (Ce[8] - 1.0);
    const double Sxy = mu * Ce[1], Sxz = mu * Ce[2], Syz = mu * Ce[5];
    P.S[0] = Sxx; P.S[1] = Syy; P.S[2] = Szz; P.S[3] = Sxy; P.S[4] = Sxz; P.S[5] = Syz;
    const double Sm[9] = {Sxx, Sxy, Sxz, Sxy, Syy, Syz, Sxz, Syz, Szz};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        P.P0[3 * i + j] = P.Fe[3 * i] * Sm[j] + P.Fe[3 * i + 1] * Sm[3 + j] + P.Fe[3 * i + 2] * Sm[6 + j];
    double sc = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) sc += Sm[k] * Ce[k];
    P.P0Fe = sc;
  }
  return true;
}

// reals per voxel of the packed tangent state
constexpr int state_size(int law) { return law == LAW_NH_ ? 12 : 18; }

// ---------------------------------------------------------------- mechanics state
// in: F (9 V) or uniform Fbar (s[0..8], when in[0] == null), c, d, material
// out0: P = (1-d)^2 a P0(a F) (9 V, FP64, may be null)
// out1: packed tangent state (precision R, may be null):
//   Neo-Hookean   B = F^-T (9), g a^2 G, g (G - lam ln J_e), g lam
//   St-V-Kirchhoff F (9), S (6), g a^2, g a^4 lam, g a^4 G

template <typename R, int LAW = LAW_NH_>
struct KMechState : VecOp<double> {
  static constexpr bool RED = false;
  FG_DEV static void apply(const VArgs& a, long long v, Acc<AccReal>&, const Pre&) {
    const long long V = a.V;
    const double* Fp = (const double*)a.in[0];
    double F[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) F[k] = Fp ? Fp[k * V + v] : a.s[k];
    const double c = ((const double*)a.in[1])[v];
    const double d = ((const double*)a.in[2])[v];
    const double lam = ((const double*)a.in[3])[v], mu = ((const double*)a.in[4])[v];
    const double Om = ((const double*)a.in[5])[v], c0 = ((const double*)a.in[6])[v];
    ElasticPoint P;
    if (!elastic_point<LAW>(F, c, d, lam, mu, Om, c0, P)) {
      atomicOr(a.flags, ST_DOMAIN);
      return;
    }
    if (a.out[0]) {
      double* Po = (double*)a.out[0];
      const double ga = P.g * P.a;
#pragma unroll
      for (int k = 0; k < 9; ++k) Po[k * V + v] = ga * P.P0[k];
    }
    if (a.out[1]) {
      R* st = (R*)a.out[1];
      if constexpr (LAW == LAW_NH_) {
#pragma unroll
        for (int k = 0; k < 9; ++k) st[k * V + v] = (R)P.B[k];
        st[9 * V + v] = (R)(P.g * P.a * P.a * P.mu);
        st[10 * V + v] = (R)(P.g * (P.mu - P.lam * P.lnJe));
        st[11 * V + v] = (R)(P.g * P.lam);
      } else {
        const double a2 = P.a * P.a;
#pragma unroll
        for (int k = 0; k < 9; ++k) st[k * V + v] = (R)F[k];
#pragma unroll
        for (int k = 0; k < 6; ++k) st[(9 + k) * V + v] = (R)P.S[k];
        st[15 * V + v] = (R)(P.g * a2);
        st[16 * V + v] = (R)(P.g * a2 * a2 * P.lam);
        st[17 * V + v] = (R)(P.g * a2 * a2 * P.mu);
      }
    }
  }
};

// ---------------------------------------------------------------- damage history
// H = max(H_t, g_c(x)/(2 l_c) D_f), D_f from the principal values of the undegraded
// Cauchy stress sigma = J^-1 a P0(a F) F^T (Eqs. Hist, SigDrivingForce).
// in: F, c, H_t, lam, mu, Om, c0, smax, gcr = g_c(x)/g_c (null: uniform) ; s0 = g_c/(2 l_c)
// out0: H ; out1 (when gcr): H_eff = H / gcr, the history the phase-field operator sees.
// Accumulates sum H_eff.
template <int LAW = LAW_NH_>
struct KHistory : VecOp<double> {
  static constexpr bool RED = true;
  FG_DEV static void apply(const VArgs& a, long long v, Acc<AccReal>& acc, const Pre&) {
    const long long V = a.V;
    const double* Fp = (const double*)a.in[0];
    double F[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) F[k] = Fp[k * V + v];
    const double c = ((const double*)a.in[1])[v];
    const double Ht = ((const double*)a.in[2])[v];
    ElasticPoint P;
    double Hn = Ht;
    if (elastic_point<LAW>(F, c, 0.0, ((const double*)a.in[3])[v], ((const double*)a.in[4])[v],
                           ((const double*)a.in[5])[v], ((const double*)a.in[6])[v], P)) {
      const double* P0 = P.P0;
      const double J = det3(F);
      const double s = P.a / J;
      double sg[9];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
          sg[3 * i + j] = s * (P0[3 * i] * F[3 * j] + P0[3 * i + 1] * F[3 * j + 1] +
                               P0[3 * i + 2] * F[3 * j + 2]);
      double e[3];
      sym_eig3(sg[0], sg[4], sg[8], 0.5 * (sg[1] + sg[3]), 0.5 * (sg[2] + sg[6]),
               0.5 * (sg[5] + sg[7]), e);
      const double smax = ((const double*)a.in[7])[v];
      double t = 0.0;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const double u = e[i] > 0.0 ? e[i] / smax : 0.0;
        t += u * u;
      }
      const double Df = t - 1.0 > 0.0 ? t - 1.0 : 0.0;
      const double* gcr = (const double*)a.in[8];
      const double Hc = a.s[0] * (gcr ? gcr[v] : 1.0) * Df;
      Hn = Hc > Ht ? Hc : Ht;
    } else {
      atomicOr(a.flags, ST_DOMAIN);
    }
    ((double*)a.out[0])[v] = Hn;
    if (a.out[1]) {
      const double He = Hn / ((const double*)a.in[8])[v];
      ((double*)a.out[1])[v] = He;
      acc.add(He);
    } else {
      acc.add(Hn);
    }
  }
};

// ---------------------------------------------------------------- chemistry
// K_c = D phi(d_t) c_t (1-c_t) C^-1, C = F^T F, stored (xx, yy, zz, xy, xz, yz) in R.
// in: F, c_t, d_t, D ; out0: K (6 V)
template <typename R>
struct KChemCond : VecOp<double> {
  static constexpr bool RED = false;
  FG_DEV static void apply(const VArgs& a, long long v, Acc<AccReal>&, const Pre&) {
    const long long V = a.V;
    const double* Fp = (const double*)a.in[0];
    double F[9], C[9], Ci[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) F[k] = Fp[k * V + v];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        C[3 * i + j] = F[i] * F[j] + F[3 + i] * F[3 + j] + F[6 + i] * F[6 + j];
    cof3(C, Ci);
    const double ct = ((const double*)a.in[1])[v];
    const double dt_ = ((const double*)a.in[2])[v];
    const double D = ((const double*)a.in[3])[v];
    const double phi = 0.9 * (1.0 - dt_) * (1.0 - dt_) + 0.1 * dt_ * dt_;
    const double s = D * phi * ct * (1.0 - ct) / det3(C);
    R* K = (R*)a.out[0];
    K[v] = (R)(s * Ci[0]);
    K[V + v] = (R)(s * Ci[4]);
    K[2 * V + v] = (R)(s * Ci[8]);
    K[3 * V + v] = (R)(s * Ci[1]);
    K[4 * V + v] = (R)(s * Ci[2]);
    K[5 * V + v] = (R)(s * Ci[5]);
  }
};

// Newton quantities at the iterate c (FP64):
//   out0 = mu~(c) = log(c/(1-c)) + mu_e / RT        (Eqs. muc, mue)
//   out1 = c - c_t - dt cdot_B                     (residual without the flux term)
//   out2 = c (1 - c) in precision R                (1/m of the Jacobian)
// mu_e = -(1-d)^2 Omega / (3 J_c) P0(F_e) : F_e / c_max  (d psi_e / dc at fixed F).
// in: c, c_t, cdot_B, F, d_t, lam, mu, Om, c0 ; s0 = dt, s1 = 1/RT, s2 = 1/c_max
template <typename R, int LAW = LAW_NH_>
struct KChemPrep : VecOp<double> {
  static constexpr bool RED = false;
  FG_DEV static void apply(const VArgs& a, long long v, Acc<AccReal>&, const Pre&) {
    const long long V = a.V;
    const double c = ((const double*)a.in[0])[v];
    const double ct = ((const double*)a.in[1])[v];
    const double cb = ((const double*)a.in[2])[v];
    if (!(c > 0.0 && c < 1.0)) {
      atomicOr(a.flags, ST_DOMAIN);
      return;
    }
    const double* Fp = (const double*)a.in[3];
    double F[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) F[k] = Fp[k * V + v];
    const double d = ((const double*)a.in[4])[v];
    const double lam = ((const double*)a.in[5])[v], mu = ((const double*)a.in[6])[v];
    const double Om = ((const double*)a.in[7])[v], c0 = ((const double*)a.in[8])[v];
    double mue = 0.0;
    if (Om != 0.0) {
      ElasticPoint P;
      if (elastic_point<LAW>(F, c, d, lam, mu, Om, c0, P)) {
        mue = -P.g * Om / (3.0 * P.Jc) * P.P0Fe * a.s[2];
      } else {
        atomicOr(a.flags, ST_DOMAIN);
      }
    }
    ((double*)a.out[0])[v] = log(c / (1.0 - c)) + mue * a.s[1];
    ((double*)a.out[1])[v] = c - ct - a.s[0] * cb;
    ((R*)a.out[2])[v] = (R)(c * (1.0 - c));
  }
};

// c = c_i + s0 dc with dc = y / m (y = m dc), 1/m = c_i (1 - c_i) or, with the full
// Jacobian, the stored in2 = 1/m (R); accumulates |s0 dc|^2.
// in0 = y (R), in1 = c_i, in2 = 1/m (R, may be null); out0 = c
template <typename R>
struct KChemUpdate : VecOp<double> {
  static constexpr bool RED = true;
  FG_DEV static void apply(const VArgs& a, long long v, Acc<AccReal>& acc, const Pre&) {
    const double ci = ((const double*)a.in[1])[v];
    const double im = a.in[2] ? (double)((const R*)a.in[2])[v] : ci * (1.0 - ci);
    const double dc = a.s[0] * (double)((const R*)a.in[0])[v] * im;
    const double cn = ci + dc;
    ((double*)a.out[0])[v] = cn;
    if (!(cn > 0.0 && cn < 1.0)) atomicOr(a.flags, ST_DOMAIN);
    acc.add(dc * dc);
  }
};

// ---------------------------------------------------------------- conversions / sums

// out0 (R) = s0 * in0 (FP64); accumulates |out|^2
template <typename R>
struct KScaleTo : VecOp<double> {
  static constexpr bool RED = true;
  FG_DEV static void apply(const VArgs& a, long long i, Acc<AccReal>& acc, const Pre&) {
    const R o = (R)(a.s[0] * ((const double*)a.in[0])[i]);
    ((R*)a.out[0])[i] = o;
    acc.add(o * o);
  }
};

// out0 (FP64) = in0 (R)
template <typename R>
struct KWiden : VecOp<double> {
  static constexpr bool RED = false;
  FG_DEV static void apply(const VArgs& a, long long i, Acc<AccReal>&, const Pre&) {
    ((double*)a.out[0])[i] = (double)((const R*)a.in[0])[i];
  }
};

// out0 (FP64) += in0 (R)
template <typename R>
struct KAddTo : VecOp<double> {
  static constexpr bool RED = false;
  FG_DEV static void apply(const VArgs& a, long long i, Acc<AccReal>&, const Pre&) {
    ((double*)a.out[0])[i] += (double)((const R*)a.in[0])[i];
  }
};

// out0 (FP64) = -sum_c in0[c] (R) * in1[c] (FP64), c < 9: minus the contraction of the
// adjoint field with the stress (the gradient of a loss with respect to log E)
template <typename R>
struct KAdjGradE : VecOp<double> {
  static constexpr bool RED = false;
  FG_DEV static void apply(const VArgs& a, long long v, Acc<AccReal>&, const Pre&) {
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 9; ++c)
      s += (double)((const R*)a.in[0])[c * a.V + v] * ((const double*)a.in[1])[c * a.V + v];
    ((double*)a.out[0])[v] = -s;
  }
};

// out0 = s0 in0 + s1 in1 + s2 in2 (FP64; in1, in2 may be null)
struct KLin3 : VecOp<double> {
  static constexpr bool RED = false;
  FG_DEV static void apply(const VArgs& a, long long i, Acc<AccReal>&, const Pre&) {
    double o = a.s[0] * ((const double*)a.in[0])[i];
    if (a.in[1]) o += a.s[1] * ((const double*)a.in[1])[i];
    if (a.in[2]) o += a.s[2] * ((const double*)a.in[2])[i];
    ((double*)a.out[0])[i] = o;
  }
};

// out0 = in0 / in1 (FP64)
struct KDivTo : VecOp<double> {
  static constexpr bool RED = false;
  FG_DEV static void apply(const VArgs& a, long long i, Acc<AccReal>&, const Pre&) {
    ((double*)a.out[0])[i] = ((const double*)a.in[0])[i] / ((const double*)a.in[1])[i];
  }
};

// out0 (FP64) = in0 + s0 * in1 (FP64)
struct KAxpyTo : VecOp<double> {
  static constexpr bool RED = false;
  FG_DEV static void apply(const VArgs& a, long long i, Acc<AccReal>&, const Pre&) {
    ((double*)a.out[0])[i] = ((const double*)a.in[0])[i] + a.s[0] * ((const double*)a.in[1])[i];
  }
};

// sum of in0 (FP64) and of in0^2 into (partials, partials + VEC_BLOCKS)
struct KSum : VecOp<double> {
  static constexpr bool RED = true;
  FG_DEV static void apply(const VArgs& a, long long i, Acc<AccReal>& acc, const Pre&) {
    acc.add(((const double*)a.in[0])[i]);
  }
};
struct KSumSq : VecOp<double> {
  static constexpr bool RED = true;
  FG_DEV static void apply(const VArgs& a, long long i, Acc<AccReal>& acc, const Pre&) {
    const double x = ((const double*)a.in[0])[i];
    acc.add(x * x);
  }
};
// out0 (FP64) = in0 (FP64) + s0..s8 pattern: F = F_t + dFbar (component = i / V)
struct KShiftF : VecOp<double> {
  static constexpr bool RED = false;
  FG_DEV static void apply(const VArgs& a, long long i, Acc<AccReal>&, const Pre&) {
    ((double*)a.out[0])[i] = ((const double*)a.in[0])[i] + a.s[i / a.V];
  }
};

// u += B_0 i_x + B_1 i_y + B_2 i_z at the corner of every voxel i (x fastest), the affine
// part (Fbar - I) x of one displacement component with B_j = (Fbar - I)_kj h_j.
// s[0..2] = B, s[3] = nx, s[4] = ny; out0 = u (V)
struct KAddAffine : VecOp<double> {
  static constexpr bool RED = false;
  FG_DEV static void apply(const VArgs& a, long long i, Acc<AccReal>&, const Pre&) {
    const long long nx = (long long)a.s[3], ny = (long long)a.s[4];
    const long long t = i / nx, ix = i - t * nx, iz = t / ny, iy = t - iz * ny;
    ((double*)a.out[0])[i] += a.s[0] * (double)ix + a.s[1] * (double)iy + a.s[2] * (double)iz;
  }
};

// ---------------------------------------------------------------- Krylov vectors

// CG start from x = 0: x = 0, r = b, p = b (in0 = b, out0 = x, out1 = r, out2 = p); sum b^2
template <typename R>
struct KCgInit : VecOp<R> {
  using AccReal = R;
  using Pre = typename VecOp<R>::Pre;
  static constexpr bool RED = true;
  FG_DEV static void apply(const VArgs& a, long long i, Acc<AccReal>& acc, const Pre&) {
    const R b = ((const R*)a.in[0])[i];
    ((R*)a.out[0])[i] = (R)0;
    ((R*)a.out[1])[i] = b;
    if (a.out[2]) ((R*)a.out[2])[i] = b;
    acc.add(b * b);
  }
};

// x += alpha p, r -= alpha q; sum r^2 (in0 = p, in1 = q, out0 = x, out1 = r)
template <typename R>
struct KCgXR : VecOp<R> {
  using AccReal = R;
  struct Pre {
    R al;
  };
  FG_DEV static Pre pre(const VArgs& a) { return Pre{(R)a.ks->alpha}; }
  static constexpr bool RED = true;
  FG_DEV static void apply(const VArgs& a, long long i, Acc<AccReal>& acc, const Pre& pr) {
    const R al = pr.al;
    R* x = (R*)a.out[0];
    R* r = (R*)a.out[1];
    x[i] += al * ((const R*)a.in[0])[i];
    const R rn = r[i] - al * ((const R*)a.in[1])[i];
    r[i] = rn;
    acc.add(rn * rn);
  }
};

// p = z + beta p (in0 = z, out0 = p)
template <typename R>
struct KCgP : VecOp<R> {
  using AccReal = R;
  struct Pre {
    R beta;
  };
  FG_DEV static Pre pre(const VArgs& a) { return Pre{(R)a.ks->beta}; }
  static constexpr bool RED = false;
  FG_DEV static void apply(const VArgs& a, long long i, Acc<AccReal>&, const Pre& pr) {
    R* p = (R*)a.out[0];
    p[i] = ((const R*)a.in[0])[i] + pr.beta * p[i];
  }
};

// r = b - q (in0 = b, in1 = q, out0 = r); sum r^2 and b^2 (two passes of partials)
template <typename R>
struct KResid : VecOp<R> {
  using AccReal = R;
  using Pre = typename VecOp<R>::Pre;
  static constexpr bool RED = true;
  FG_DEV static void apply(const VArgs& a, long long i, Acc<AccReal>& acc, const Pre&) {
    const R rv = ((const R*)a.in[0])[i] - ((const R*)a.in[1])[i];
    ((R*)a.out[0])[i] = rv;
    acc.add(rv * rv);
  }
};
template <typename R>
struct KSumSqR : VecOp<R> {
  using AccReal = R;
  using Pre = typename VecOp<R>::Pre;
  static constexpr bool RED = true;
  FG_DEV static void apply(const VArgs& a, long long i, Acc<AccReal>& acc, const Pre&) {
    const R x = ((const R*)a.in[0])[i];
    acc.add(x * x);
  }
};
template <typename R>
struct KCopy : VecOp<R> {
  using AccReal = R;
  using Pre = typename VecOp<R>::Pre;
  static constexpr bool RED = false;
  FG_DEV static void apply(const VArgs& a, long long i, Acc<AccReal>&, const Pre&) {
    ((R*)a.out[0])[i] = ((const R*)a.in[0])[i];
  }
};

// ---------------------------------------------------------------- finalisers

// CG start: bb = rr = rz = t; tol2 = s0^2 bb; maxit = s1; done when bb == 0
struct FCgStart {
  FG_DEV static void fin(const VArgs& a, double t) {
    KScal* k = a.ks;
    k->bb = t;
    k->rr = t;
    k->rz = t;
    k->tol2 = a.s[0] * a.s[0] * t;
    k->beta = 0.0;
    k->iters = 0;
    k->maxit = (int)a.s[1];
    k->status = 0;
    k->rr_best = t;
    k->nosnap = 1;
    k->snaps = 0;
    k->indef = (int)a.s[2];
    k->negc = 0;
    k->done = (t == 0.0 || t <= k->tol2) ? 1 : 0;
  }
};
// alpha = rz / <p, Ap>.  A direction of negative curvature either ends the solve
// (truncated CG) or, with indef set, is taken like any other: the Galerkin iterate exists
// whenever <p, Ap> != 0; only <p, Ap> = 0 or a non-finite value stops the solve.
struct FAlpha {
  FG_DEV static void fin(const VArgs& a, double t) {
    KScal* k = a.ks;
    k->pq = t;
    if (k->iters == 0) k->pq0 = t;
    if (k->indef && t < 0.0) {
      k->negc += 1;
      k->alpha = k->rz / t;
      return;
    }
    if (!(t > 0.0)) {
      k->status |= ST_INDEFINITE;
      k->done = 1;
      k->alpha = 0.0;
      return;
    }
    k->alpha = k->rz / t;
  }
};
// unpreconditioned CG: rr = t; beta = rr / rz; rz = rr; convergence
struct FBetaCg {
  FG_DEV static void fin(const VArgs& a, double t) {
    KScal* k = a.ks;
    k->iters += 1;
    k->rr = t;
    k->beta = t / k->rz;
    k->rz = t;
    if (t <= 0.25 * k->rr_best) {  // snapshot the iterate at every 4x drop of |r|^2
      k->rr_best = t;
      k->nosnap = 0;
      k->snaps += 1;
    } else {
      k->nosnap = 1;
    }
    if (!(t == t)) k->status |= ST_NUMERIC;
    if (t <= k->tol2 || k->iters >= k->maxit || !(t == t)) k->done = 1;
  }
};
// preconditioned CG, after the r update: rr = t; convergence
struct FResPcg {
  FG_DEV static void fin(const VArgs& a, double t) {
    KScal* k = a.ks;
    k->iters += 1;
    k->rr = t;
    if (!(t == t)) k->status |= ST_NUMERIC;
    if (t <= k->tol2 || k->iters >= k->maxit || !(t == t)) k->done = 1;
  }
};
// preconditioned CG, after z = P r: beta = <r,z>_new / <r,z>_old
struct FBetaPcg {
  FG_DEV static void fin(const VArgs& a, double t) {
    KScal* k = a.ks;
    k->beta = t / k->rz;
    k->rz = t;
  }
};
// PCG start: rr = t (s0 = tol, s1 = bb, s2 = maxit); done test
struct FPcgStart {
  FG_DEV static void fin(const VArgs& a, double t) {
    KScal* k = a.ks;
    k->rr = t;
    k->bb = a.s[1];
    k->tol2 = a.s[0] * a.s[0] * a.s[1];
    k->iters = 0;
    k->maxit = (int)a.s[2];
    k->status = 0;
    k->indef = 0;
    k->negc = 0;
    k->done = (a.s[1] == 0.0 || t <= k->tol2) ? 1 : 0;
  }
};
// PCG start, after z0 = P r0: rz = t
struct FPcgRz {
  FG_DEV static void fin(const VArgs& a, double t) { a.ks->rz = t; }
};
// after re-projecting the CG residual: rr = rz = |r|^2
struct FSetResidual {
  FG_DEV static void fin(const VArgs& a, double t) {
    a.ks->rr = t;
    a.ks->rz = t;
  }
};
// store a plain sum into ks->aux
struct FStore {
  FG_DEV static void fin(const VArgs& a, double t) { a.ks->aux = t; }
};

}  // namespace fg
