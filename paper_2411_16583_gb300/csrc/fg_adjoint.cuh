// Voxel-wise kernels of the discrete adjoint of one staggered step (Alg. 4), FP64.
//
// One converged step maps (c_t, F_t, d_t, H_t) to (c, F, d, H) through the chemistry
// residual f(c) = 0 (Eq. Chemresidualfc, with F~ = F_t + Fbar - Fbar_t frozen), the
// equilibrium G P(F, c, d) = 0 (Eq. mechanicalsolve), the history H = max(H_t, psi(F, c)),
// psi = g_c(x)/(2 l_c) D_f (Eqs. Hist, SigDrivingForce) and the phase field
// (g_c/l_c + 2 r H) d - g_c l_c lap d = 2 r H, r = g_c/g_c(x) (Eq. PFFA).  These kernels
// evaluate the pointwise pieces of its transpose; the solves run in the runtime.
#pragma once
#include "fg_pointwise.cuh"

namespace fg {

// K0(F_e)[X]: the pristine tangent dP0/dF_e applied to X, both laws (Eqs. psie0, pristine).
template <int LAW>
FG_DEV void k0_apply(const ElasticPoint& P, const double* X, double* out) {
  if constexpr (LAW == LAW_NH_) {
    // mu X + (mu - lam ln J_e) Bt X^T Bt + lam (Bt : X) Bt,  Bt = F_e^-T = F^-T / a
    double Bt[9], T[9];
    const double ia = 1.0 / P.a;
    double tr = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      Bt[k] = P.B[k] * ia;
      tr += Bt[k] * X[k];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int l = 0; l < 3; ++l)
        T[3 * i + l] = Bt[3 * i] * X[3 * l] + Bt[3 * i + 1] * X[3 * l + 1] + Bt[3 * i + 2] * X[3 * l + 2];
    const double m2 = P.mu - P.lam * P.lnJe;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const double M = T[3 * i] * Bt[j] + T[3 * i + 1] * Bt[3 + j] + T[3 * i + 2] * Bt[6 + j];
        out[3 * i + j] = P.mu * X[3 * i + j] + m2 * M + P.lam * tr * Bt[3 * i + j];
      }
  } else {
    // X S + F_e dS,  dS = lam tr(dE) I + 2 mu dE,  dE = sym(F_e^T X)
    double A[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        A[3 * i + j] = P.Fe[i] * X[j] + P.Fe[3 + i] * X[3 + j] + P.Fe[6 + i] * X[6 + j];
    double dS[9];
    const double trdE = A[0] + A[4] + A[8];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        dS[3 * i + j] = P.mu * (A[3 * i + j] + A[3 * j + i]) + (i == j ? P.lam * trdE : 0.0);
    const double S[9] = {P.S[0], P.S[3], P.S[4], P.S[3], P.S[1], P.S[5], P.S[4], P.S[5], P.S[2]};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        out[3 * i + j] = X[3 * i] * S[j] + X[3 * i + 1] * S[3 + j] + X[3 * i + 2] * S[6 + j] +
                         P.Fe[3 * i] * dS[j] + P.Fe[3 * i + 1] * dS[3 + j] + P.Fe[3 * i + 2] * dS[6 + j];
  }
}

FG_DEV void mat3_mul(const double* A, const double* B, double* C) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

// <s>_+ = sum_i max(e_i, 0) n_i n_i^T of a symmetric s (full 9 entries) with eigenvalues
// e[0] >= e[1] >= e[2], through the spectral projectors written as polynomials in s:
// with one positive eigenvalue e0 P0, P0 = (s - e1)(s - e2)/((e0 - e1)(e0 - e2)); with two,
// s - e2 P2, P2 = (s - e0)(s - e1)/((e2 - e0)(e2 - e1)).  In the first case both
// factors of the denominator are at least e0; in the second the factor e2 in front keeps
// the roundoff below eps |s|^2 / (e0 - e2).  The callers only come here with D_f > 0,
// where e0 >= sigma_max / sqrt(3).
FG_DEV void sym_pos_part(const double* s, const double* e, double* out) {
  if (e[2] >= 0.0) {
#pragma unroll
    for (int k = 0; k < 9; ++k) out[k] = s[k];
    return;
  }
  if (e[0] <= 0.0) {
#pragma unroll
    for (int k = 0; k < 9; ++k) out[k] = 0.0;
    return;
  }
  double A[9], B[9], M[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    A[k] = s[k];
    B[k] = s[k];
  }
  if (e[1] <= 0.0) {
    for (int i = 0; i < 3; ++i) {
      A[4 * i] -= e[1];
      B[4 * i] -= e[2];
    }
    mat3_mul(A, B, M);
    const double f = e[0] / ((e[0] - e[1]) * (e[0] - e[2]));
#pragma unroll
    for (int k = 0; k < 9; ++k) out[k] = f * M[k];
  } else {
    for (int i = 0; i < 3; ++i) {
      A[4 * i] -= e[0];
      B[4 * i] -= e[1];
    }
    mat3_mul(A, B, M);
    const double f = e[2] / ((e[2] - e[0]) * (e[2] - e[1]));
#pragma unroll
    for (int k = 0; k < 9; ++k) out[k] = s[k] - f * M[k];
  }
}

// psi = scale D_f(sigma) with scale = g_c(x)/(2 l_c), and (when D_f > 0) with
// S = dpsi/dsigma = scale (2 / sigma_max^2) <sigma>_+ and sigma = sym(P~ F^T)/J,
// P~ = a P0(a F):
//   Z = dpsi/dF = (a^2 K0[S F] + S P~)/J - (S : sigma) F^-T,
//   psi_c = (S F) : dP~/dc / J,  dP~/dc = -a Omega/(3 J_c) (P0 + K0[F_e]),
//   psi_E = dpsi/dlog E = S : sigma.
// Returns false outside the domain (det F <= 0 or J_c <= 0).
template <int LAW>
FG_DEV bool psi_terms(const double* F, double c, double lam, double mu, double Om, double c0,
                      double smax, double scale, double& psi, double* Z, double& psi_c,
                      double& psi_E) {
  ElasticPoint P;
  if (!elastic_point<LAW>(F, c, 0.0, lam, mu, Om, c0, P)) return false;
  const double J = det3(F);
  double Pt[9], sg[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) Pt[k] = P.a * P.P0[k];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      sg[3 * i + j] = (Pt[3 * i] * F[3 * j] + Pt[3 * i + 1] * F[3 * j + 1] + Pt[3 * i + 2] * F[3 * j + 2]) / J;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i + 1; j < 3; ++j) {
      const double m = 0.5 * (sg[3 * i + j] + sg[3 * j + i]);
      sg[3 * i + j] = m;
      sg[3 * j + i] = m;
    }
  double e[3];
  sym_eig3(sg[0], sg[4], sg[8], sg[1], sg[2], sg[5], e);
  double t = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double u = e[i] > 0.0 ? e[i] / smax : 0.0;
    t += u * u;
  }
  const double Df = t - 1.0 > 0.0 ? t - 1.0 : 0.0;
  psi = scale * Df;
  if (!(Df > 0.0)) {
#pragma unroll
    for (int k = 0; k < 9; ++k) Z[k] = 0.0;
    psi_c = 0.0;
    psi_E = 0.0;
    return true;
  }
  double S[9];
  sym_pos_part(sg, e, S);
  const double f = scale * 2.0 / (smax * smax);
  double SdS = 0.0;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    S[k] *= f;
    SdS += S[k] * sg[k];
  }
  double SF[9], KSF[9], SP[9];
  mat3_mul(S, F, SF);
  k0_apply<LAW>(P, SF, KSF);
  mat3_mul(S, Pt, SP);
  const double a2 = P.a * P.a;
  double FiT[9];  // F^-T (the Neo-Hookean ElasticPoint carries it)
  if constexpr (LAW == LAW_NH_) {
#pragma unroll
    for (int k = 0; k < 9; ++k) FiT[k] = P.B[k];
  } else {
    cof3(F, FiT);
#pragma unroll
    for (int k = 0; k < 9; ++k) FiT[k] /= J;
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) Z[k] = (a2 * KSF[k] + SP[k]) / J - SdS * FiT[k];
  double KFe[9];
  k0_apply<LAW>(P, P.Fe, KFe);
  const double da = -P.a * Om / (3.0 * P.Jc);
  double pc = 0.0;
#pragma unroll
  for (int k = 0; k < 9; ++k) pc += SF[k] * da * (P.P0[k] + KFe[k]);
  psi_c = pc / J;
  psi_E = SdS;
  return true;
}

// material pointers in consecutive VArgs inputs: lam, mu, Om, c0
FG_DEV void load_mat(const VArgs& a, int k, long long v, double& lam, double& mu, double& Om, double& c0) {
  lam = ((const double*)a.in[k])[v];
  mu = ((const double*)a.in[k + 1])[v];
  Om = ((const double*)a.in[k + 2])[v];
  c0 = ((const double*)a.in[k + 3])[v];
}

FG_DEV double opt_at(const void* p, long long v, double dflt) {
  return p ? ((const double*)p)[v] : dflt;
}

// rhs = sF + chi lamH Z (the mechanical adjoint right-hand side before G), chi = [psi > H_t]
// in: sF (9 V, may be null), lamH, F, c, H_t, lam, mu, Om, c0, smax, gcr (may be null)
// out0: rhs (9 V), out1: chi (V, may be null); s0 = g_c/(2 l_c)
template <int LAW>
struct KAdjRhsM : VecOp<double> {
  static constexpr bool RED = false;
  FG_DEV static void apply(const VArgs& a, long long v, Acc<AccReal>&, const Pre&) {
    const long long V = a.V;
    double F[9], Z[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) F[k] = ((const double*)a.in[2])[k * V + v];
    double lam, mu, Om, c0;
    load_mat(a, 5, v, lam, mu, Om, c0);
    const double scale = a.s[0] * opt_at(a.in[10], v, 1.0);
    double psi = 0.0, pc, pe;
    if (!psi_terms<LAW>(F, ((const double*)a.in[3])[v], lam, mu, Om, c0,
                        ((const double*)a.in[9])[v], scale, psi, Z, pc, pe)) {
      atomicOr(a.flags, ST_DOMAIN);
      return;
    }
    const double chi = psi > ((const double*)a.in[4])[v] ? 1.0 : 0.0;
    const double w = chi * ((const double*)a.in[1])[v];
    double* out = (double*)a.out[0];
#pragma unroll
    for (int k = 0; k < 9; ++k) out[k * V + v] = opt_at(a.in[0], k * V + v, 0.0) + w * Z[k];
    if (a.out[1]) ((double*)a.out[1])[v] = chi;
  }
};

// rhs_d = sd - dP/dd : lamM = sd + 2 (1 - d) a P0(a F) : lamM
// in: sd (may be null), lamM (9 V), F, c, d, lam, mu, Om, c0 ; out0: rhs_d
template <int LAW>
struct KAdjRhsD : VecOp<double> {
  static constexpr bool RED = false;
  FG_DEV static void apply(const VArgs& a, long long v, Acc<AccReal>&, const Pre&) {
    const long long V = a.V;
    double F[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) F[k] = ((const double*)a.in[2])[k * V + v];
    double lam, mu, Om, c0;
    load_mat(a, 5, v, lam, mu, Om, c0);
    const double d = ((const double*)a.in[4])[v];
    ElasticPoint P;
    if (!elastic_point<LAW>(F, ((const double*)a.in[3])[v], d, lam, mu, Om, c0, P)) {
      atomicOr(a.flags, ST_DOMAIN);
      return;
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) s += P.P0[k] * ((const double*)a.in[1])[k * V + v];
    ((double*)a.out[0])[v] = opt_at(a.in[0], v, 0.0) + 2.0 * (1.0 - d) * P.a * s;
  }
};

// lamH = sH + 2 r (1 - d) lamD, r = 1/gcr ; in: sH (may be null), lamD, d, gcr (may be null)
struct KAdjLamH : VecOp<double> {
  static constexpr bool RED = false;
  FG_DEV static void apply(const VArgs& a, long long v, Acc<AccReal>&, const Pre&) {
    const double d = ((const double*)a.in[2])[v];
    ((double*)a.out[0])[v] = opt_at(a.in[0], v, 0.0) +
                             2.0 * (1.0 - d) * ((const double*)a.in[1])[v] / opt_at(a.in[3], v, 1.0);
  }
};

// Outputs of the (F, H, d) block:
//   gE += -lamM : P + chi lamH psi_E,   gG += chi lamH psi - 2 r H (1 - d) lamD,
//   sH_t = (1 - chi) lamH,              gc_tot = sc - dP/dc : lamM + chi lamH psi_c
// in: lamM (9 V), lamD, lamH, sc (may be null), F, c, d, H, H_t, lam, mu, Om, c0, smax,
//     gcr (may be null) ; out0: gE, out1: gG, out2: sH_t, out3: gc_tot ; s0 = g_c/(2 l_c)
template <int LAW>
struct KAdjBlockOut : VecOp<double> {
  static constexpr bool RED = false;
  FG_DEV static void apply(const VArgs& a, long long v, Acc<AccReal>&, const Pre&) {
    const long long V = a.V;
    double F[9], Z[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) F[k] = ((const double*)a.in[4])[k * V + v];
    double lam, mu, Om, c0;
    load_mat(a, 9, v, lam, mu, Om, c0);
    const double c = ((const double*)a.in[5])[v];
    const double d = ((const double*)a.in[6])[v];
    const double gcr = opt_at(a.in[14], v, 1.0);
    ElasticPoint P;
    double psi = 0.0, psi_c = 0.0, psi_E = 0.0;
    if (!elastic_point<LAW>(F, c, d, lam, mu, Om, c0, P) ||
        !psi_terms<LAW>(F, c, lam, mu, Om, c0, ((const double*)a.in[13])[v], a.s[0] * gcr, psi, Z,
                        psi_c, psi_E)) {
      atomicOr(a.flags, ST_DOMAIN);
      return;
    }
    const double chi = psi > ((const double*)a.in[8])[v] ? 1.0 : 0.0;
    const double lD = ((const double*)a.in[1])[v];
    const double lH = ((const double*)a.in[2])[v];
    double KFe[9];
    k0_apply<LAW>(P, P.Fe, KFe);
    const double da = -P.a * Om / (3.0 * P.Jc);
    double lP = 0.0, lPc = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const double l = ((const double*)a.in[0])[k * V + v];
      lP += l * P.g * P.a * P.P0[k];
      lPc += l * P.g * da * (P.P0[k] + KFe[k]);
    }
    const double H = ((const double*)a.in[7])[v];
    ((double*)a.out[0])[v] += -lP + chi * lH * psi_E;
    ((double*)a.out[1])[v] += chi * lH * psi - 2.0 * H * (1.0 - d) * lD / gcr;
    ((double*)a.out[2])[v] = (1.0 - chi) * lH;
    ((double*)a.out[3])[v] = opt_at(a.in[3], v, 0.0) - lPc + chi * lH * psi_c;
  }
};

// Chemistry Jacobian M = dmu~/dc = 1/(c (1 - c)) + (dmu_e/dc)/RT at (c, F~, d_t);
// out0: w = 1/M, out1: b = g/M (the symmetric system (M^-1 + dt L) y = M^-1 g).
// in: c, g, F~, d_t, lam, mu, Om, c0 ; s0 = 1/RT, s1 = 1/c_max
template <int LAW>
struct KAdjChemM : VecOp<double> {
  static constexpr bool RED = false;
  FG_DEV static void apply(const VArgs& a, long long v, Acc<AccReal>&, const Pre&) {
    const long long V = a.V;
    const double c = ((const double*)a.in[0])[v];
    double m = 1.0 / (c * (1.0 - c));
    double lam, mu, Om, c0;
    load_mat(a, 4, v, lam, mu, Om, c0);
    if (Om != 0.0) {
      double F[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) F[k] = ((const double*)a.in[2])[k * V + v];
      ElasticPoint P;
      if (!elastic_point<LAW>(F, c, ((const double*)a.in[3])[v], lam, mu, Om, c0, P)) {
        atomicOr(a.flags, ST_DOMAIN);
        return;
      }
      double KFe[9];
      k0_apply<LAW>(P, P.Fe, KFe);
      double kf = 0.0;
#pragma unroll
      for (int k = 0; k < 9; ++k) kf += KFe[k] * P.Fe[k];
      const double q = P.P0Fe;
      m += P.g * Om * Om / (3.0 * P.Jc * P.Jc) * a.s[1] * (q + (kf + q) / 3.0) * a.s[0];
    }
    if (!(m > 0.0)) atomicOr(a.flags, ST_NUMERIC);
    const double w = 1.0 / m;
    ((double*)a.out[0])[v] = w;
    ((double*)a.out[1])[v] = w * ((const double*)a.in[1])[v];
  }
};

// Seeds of the step's inputs and parameter gradients from the chemistry multiplier lamC:
//   s = gl^T K gm, K = kappa C^-1, kappa = D phi(d_t) c_t (1 - c_t), C = F~^T F~,
//   gl = grad_f lamC, gm = grad_f mu~, Ll = L lamC ;
//   sc_t = lamC - dt (1 - 2 c_t)/(c_t (1 - c_t)) s
//   sd_t = -dt phi'/phi s + dt Ll 2 mu_e / ((1 - d_t) RT)
//   sF_t = dt kappa [(F w) u^T + (F u) w^T] - dt Ll dmu_e/dF / RT,  u = C^-1 gl, w = C^-1 gm
//   gD += -dt s,  gE += -dt Ll mu_e / RT
// in: lamC, gl (3 V), gm (3 V), Ll, c, c_t, d_t, F~, D, lam, mu, Om, c0
// out0: sc_t, out1: sd_t, out2: sF_t (9 V), out3: gD, out4: gE ; s0 = dt, s1 = 1/RT, s2 = 1/c_max
template <int LAW>
struct KAdjChemOut : VecOp<double> {
  static constexpr bool RED = false;
  FG_DEV static void apply(const VArgs& a, long long v, Acc<AccReal>&, const Pre&) {
    const long long V = a.V;
    const double dt = a.s[0], iRT = a.s[1];
    double F[9], Cm[9], Ci[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) F[k] = ((const double*)a.in[7])[k * V + v];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        Cm[3 * i + j] = F[i] * F[j] + F[3 + i] * F[3 + j] + F[6 + i] * F[6 + j];
    cof3(Cm, Ci);
    const double iC = 1.0 / det3(Cm);
    const double ct = ((const double*)a.in[5])[v];
    const double dtv = ((const double*)a.in[6])[v];
    const double phi = 0.9 * (1.0 - dtv) * (1.0 - dtv) + 0.1 * dtv * dtv;
    const double dphi = -1.8 * (1.0 - dtv) + 0.2 * dtv;
    const double kappa = ((const double*)a.in[8])[v] * phi * ct * (1.0 - ct);
    double gl[3], gm[3], u[3], w[3], Fu[3], Fw[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      gl[i] = ((const double*)a.in[1])[i * V + v];
      gm[i] = ((const double*)a.in[2])[i * V + v];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      u[i] = iC * (Ci[3 * i] * gl[0] + Ci[3 * i + 1] * gl[1] + Ci[3 * i + 2] * gl[2]);
      w[i] = iC * (Ci[3 * i] * gm[0] + Ci[3 * i + 1] * gm[1] + Ci[3 * i + 2] * gm[2]);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Fu[i] = F[3 * i] * u[0] + F[3 * i + 1] * u[1] + F[3 * i + 2] * u[2];
      Fw[i] = F[3 * i] * w[0] + F[3 * i + 1] * w[1] + F[3 * i + 2] * w[2];
    }
    const double s = kappa * (gl[0] * w[0] + gl[1] * w[1] + gl[2] * w[2]);
    const double Ll = ((const double*)a.in[3])[v];
    const double c = ((const double*)a.in[4])[v];
    double lam, mu, Om, c0;
    load_mat(a, 9, v, lam, mu, Om, c0);
    double mue = 0.0, mueF[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) mueF[k] = 0.0;
    if (Om != 0.0) {
      ElasticPoint P;
      if (!elastic_point<LAW>(F, c, dtv, lam, mu, Om, c0, P)) {
        atomicOr(a.flags, ST_DOMAIN);
        return;
      }
      double KFe[9];
      k0_apply<LAW>(P, P.Fe, KFe);
      const double pre = -P.g * Om / (3.0 * P.Jc) * a.s[2];
      mue = pre * P.P0Fe;
#pragma unroll
      for (int k = 0; k < 9; ++k) mueF[k] = pre * P.a * (KFe[k] + P.P0[k]);
    }
    ((double*)a.out[0])[v] = ((const double*)a.in[0])[v] - dt * (1.0 - 2.0 * ct) / (ct * (1.0 - ct)) * s;
    ((double*)a.out[1])[v] = -dt * dphi / phi * s + dt * Ll * 2.0 * mue * iRT / (1.0 - dtv);
    double* sF = (double*)a.out[2];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        sF[(3 * i + j) * V + v] = dt * kappa * (Fw[i] * u[j] + Fu[i] * w[j]) - dt * Ll * mueF[3 * i + j] * iRT;
    ((double*)a.out[3])[v] += -dt * s;
    ((double*)a.out[4])[v] += -dt * Ll * mue * iRT;
  }
};

// Fracture energy density g_c(x) (d^2/(2 l_c) + l_c/2 |grad_f d|^2) h^3 (Eq. crack):
// accumulated (the loss) and added to gG (its direct log g_c derivative); out1 = g_c(x) grad_f d.
// in: d, gd (3 V), gcr (may be null) ; out0: gG, out1: flux (3 V) ; s0 = g_c, s1 = l_c, s2 = h^3
struct KCrackLoss : VecOp<double> {
  static constexpr bool RED = true;
  FG_DEV static void apply(const VArgs& a, long long v, Acc<AccReal>& acc, const Pre&) {
    const long long V = a.V;
    const double gcx = a.s[0] * opt_at(a.in[2], v, 1.0);
    const double d = ((const double*)a.in[0])[v];
    double g2 = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const double g = ((const double*)a.in[1])[i * V + v];
      g2 += g * g;
      ((double*)a.out[1])[i * V + v] = gcx * g;
    }
    const double dens = gcx * (d * d / (2.0 * a.s[1]) + 0.5 * a.s[1] * g2) * a.s[2];
    if (a.out[0]) ((double*)a.out[0])[v] += dens;
    acc.add(dens);
  }
};

// dGamma/dd = h^3 (g_c(x) d / l_c + l_c grad_f^H (g_c(x) grad_f d)); in: d, div, gcr (may be
// null) ; out0: seed ; s0 = g_c, s1 = l_c, s2 = h^3
struct KCrackSeed : VecOp<double> {
  static constexpr bool RED = false;
  FG_DEV static void apply(const VArgs& a, long long v, Acc<AccReal>&, const Pre&) {
    const double gcx = a.s[0] * opt_at(a.in[2], v, 1.0);
    ((double*)a.out[0])[v] =
        a.s[2] * (gcx * ((const double*)a.in[0])[v] / a.s[1] + a.s[1] * ((const double*)a.in[1])[v]);
  }
};

// 1/m of the chemistry Newton with the full Jacobian m = 1/(c (1 - c)) + d(mu_e/RT)/dc,
// out0 (R), at (c, F~, d_t); in: c, F~, d_t, lam, mu, Om, c0 ; s0 = 1/RT, s1 = 1/c_max.
// Flags ST_NUMERIC where m <= 0.
template <typename R, int LAW>
struct KChemFullM : VecOp<double> {
  static constexpr bool RED = false;
  FG_DEV static void apply(const VArgs& a, long long v, Acc<AccReal>&, const Pre&) {
    const long long V = a.V;
    const double c = ((const double*)a.in[0])[v];
    double m = 1.0 / (c * (1.0 - c));
    double lam, mu, Om, c0;
    load_mat(a, 3, v, lam, mu, Om, c0);
    if (Om != 0.0) {
      double F[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) F[k] = ((const double*)a.in[1])[k * V + v];
      ElasticPoint P;
      if (!elastic_point<LAW>(F, c, ((const double*)a.in[2])[v], lam, mu, Om, c0, P)) {
        atomicOr(a.flags, ST_DOMAIN);
        return;
      }
      double KFe[9];
      k0_apply<LAW>(P, P.Fe, KFe);
      double kf = 0.0;
#pragma unroll
      for (int k = 0; k < 9; ++k) kf += KFe[k] * P.Fe[k];
      const double q = P.P0Fe;
      m += P.g * Om * Om / (3.0 * P.Jc * P.Jc) * a.s[1] * (q + (kf + q) / 3.0) * a.s[0];
    }
    if (!(m > 0.0)) atomicOr(a.flags, ST_NUMERIC);
    ((R*)a.out[0])[v] = (R)(1.0 / m);
  }
};

// <in0, in1> (FP64)
struct KDot : VecOp<double> {
  static constexpr bool RED = true;
  FG_DEV static void apply(const VArgs& a, long long i, Acc<AccReal>& acc, const Pre&) {
    acc.add(((const double*)a.in[0])[i] * ((const double*)a.in[1])[i]);
  }
};

}  // namespace fg
