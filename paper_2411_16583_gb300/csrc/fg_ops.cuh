// Pointwise parts fused into the FFT passes: the real-space prologues of X-fwd, the
// frequency-space operators of the Z pass and the real-space epilogues of X-inv.
#pragma once
#include "fg_passes.cuh"

namespace fg {

// ================================================================== Z-pass operators

// Compatibility projection (Eqs. mapping G, mechanicalsolve): A'_ij = n_j (A_im n_m)/|n|^2
// with the rotated-scheme vector n_j = (2/h_j) sin(q_j/2) prod_{m!=j} cos(q_m/2); zero
// where |n| = 0, except that under mixed macroscopic control the zero-frequency mode keeps
// the stress-controlled components (bit 3 i + j of the mask in coef[1]).
// coef[0] = 1/V (inverse DFT scaling).
template <typename R>
struct ZProject {
  using C = cplx<R>;
  static constexpr int CIN = 9, COUT = 9;
  FG_DEV static void apply(const PassArgs<R>& a, int kx, int ky, int kz, C* v, R zs) {
    const R n0 = a.rs[0][kx] * a.rc[1][ky] * a.rc[2][kz];
    const R n1 = a.rs[1][ky] * a.rc[0][kx] * a.rc[2][kz];
    const R n2 = a.rs[2][kz] * a.rc[0][kx] * a.rc[1][ky];
    const R nn = n0 * n0 + n1 * n1 + n2 * n2;
    const R s = nn > (R)0 ? a.coef[0] / nn : (R)0;
    const int mask = (int)a.coef[1];
    if (mask != 0 && kx == 0 && ky == 0 && kz == 0) {
#pragma unroll
      for (int k = 0; k < 9; ++k) v[k] = ((mask >> k) & 1) ? cscale(v[k], a.coef[0]) : cmk<C>((R)0, (R)0);
      return;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      C t = cadd(cadd(cscale(v[3 * i], n0), cscale(v[3 * i + 1], n1)), cscale(v[3 * i + 2], n2));
      t = cscale(t, s);
      v[3 * i] = cscale(t, n0);
      v[3 * i + 1] = cscale(t, n1);
      v[3 * i + 2] = cscale(t, n2);
    }
  }
};

// Phase-field spectral term (Eq. PFFA): g_c l_c |xi|^2 d^, coef[0] = g_c l_c / V.
template <typename R>
struct ZLaplace {
  using C = cplx<R>;
  static constexpr int CIN = 1, COUT = 1;
  FG_DEV static void apply(const PassArgs<R>& a, int kx, int ky, int kz, C* v, R zs) {
    const R l = a.lap[0][kx] + a.lap[1][ky] + a.lap[2][kz];
    v[0] = cscale(v[0], a.coef[0] * l);
  }
};

// Phase-field preconditioner (Eq. PFFprecond): r^ / (g_c/l_c + 2 Hbar + g_c l_c |xi|^2).
// coef[0] = 1/V, coef[1] = g_c/l_c, coef[2] = g_c l_c, dscal[0] = Hbar.
template <typename R>
struct ZPrecond {
  using C = cplx<R>;
  static constexpr int CIN = 1, COUT = 1;
  FG_DEV static void apply(const PassArgs<R>& a, int kx, int ky, int kz, C* v, R zs) {
    const R l = a.lap[0][kx] + a.lap[1][ky] + a.lap[2][kz];
    const R den = a.coef[1] + (R)2 * zs + a.coef[2] * l;
    v[0] = cscale(v[0], a.coef[0] / den);
  }
};

// Forward-difference gradient (chemistry, Eq. ChemresidualFourier_A): g_j^ = xi_j u^ / V.
template <typename R>
struct ZGrad {
  using C = cplx<R>;
  static constexpr int CIN = 1, COUT = 3;
  FG_DEV static void apply(const PassArgs<R>& a, int kx, int ky, int kz, C* v, R zs) {
    const C u = cscale(v[0], a.coef[0]);
    v[0] = cmul(a.xi[0][kx], u);
    v[1] = cmul(a.xi[1][ky], u);
    v[2] = cmul(a.xi[2][kz], u);
  }
};

// Adjoint of the forward difference: sum_j conj(xi_j) f_j^ / V (minus the divergence).
template <typename R>
struct ZDiv {
  using C = cplx<R>;
  static constexpr int CIN = 3, COUT = 1;
  FG_DEV static void apply(const PassArgs<R>& a, int kx, int ky, int kz, C* v, R zs) {
    C s = cadd(cadd(cmulc(v[0], a.xi[0][kx]), cmulc(v[1], a.xi[1][ky])), cmulc(v[2], a.xi[2][kz]));
    v[0] = cscale(s, a.coef[0]);
  }
};

// Displacement at the voxel corners from the split F = Fbar + grad u (Eq. Fsplit).  The
// rotated-scheme gradient of a corner field has the symbol i n_j e^{i sum_m q_m/2}, so the
// least-squares inverse multiplies F_ij^ by m_j = -i e^{-i sum q/2} n_j / |n|^2 (0 where
// |n| = 0).  disp_symbol returns n and w = -i e^{-i sum q/2} coef[0] / |n|^2; the half
// angle th_j = q_j/2 has cos th_j = rc_j and sin th_j = rs_j h_j / 2 = rs_j coef[1 + j].
template <typename R>
FG_DEV void disp_symbol(const PassArgs<R>& a, int kx, int ky, int kz, R* n, cplx<R>& w) {
  using C = cplx<R>;
  const R cx = a.rc[0][kx], cy = a.rc[1][ky], cz = a.rc[2][kz];
  const R sx = a.rs[0][kx], sy = a.rs[1][ky], sz = a.rs[2][kz];
  n[0] = sx * cy * cz;
  n[1] = sy * cx * cz;
  n[2] = sz * cx * cy;
  const R nn = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
  const R s = nn > (R)0 ? a.coef[0] / nn : (R)0;
  const C e = cmul(cmul(cmk<C>(cx, -sx * a.coef[1]), cmk<C>(cy, -sy * a.coef[2])),
                   cmk<C>(cz, -sz * a.coef[3]));
  w = cmk<C>(e.y * s, -e.x * s);  // -i e s
}

// u_i^ = sum_j m_j F_ij^ / V: nine components in, three out.
template <typename R>
struct ZDisp {
  using C = cplx<R>;
  static constexpr int CIN = 9, COUT = 3;
  FG_DEV static void apply(const PassArgs<R>& a, int kx, int ky, int kz, C* v, R zs) {
    R n[3];
    C w;
    disp_symbol(a, kx, ky, kz, n, w);
    C t[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
      t[i] = cmul(w, cadd(cadd(cscale(v[3 * i], n[0]), cscale(v[3 * i + 1], n[1])),
                          cscale(v[3 * i + 2], n[2])));
#pragma unroll
    for (int i = 0; i < 3; ++i) v[i] = t[i];
  }
};

// Transpose of ZDisp: G_ij^ = conj(m_j) r_i^ / V, three components in, nine out.
template <typename R>
struct ZDispT {
  using C = cplx<R>;
  static constexpr int CIN = 3, COUT = 9;
  FG_DEV static void apply(const PassArgs<R>& a, int kx, int ky, int kz, C* v, R zs) {
    R n[3];
    C w;
    disp_symbol(a, kx, ky, kz, n, w);
    const C wc = cmk<C>(w.x, -w.y);
    C r[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) r[i] = cmul(wc, v[i]);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) v[3 * i + j] = cscale(r[i], n[j]);
  }
};

// ================================================================== X-fwd prologues

template <typename R, int NC>
struct PCopy {
  static constexpr int COUT = NC;
  static constexpr bool RED = false;
  // components read per field (rin, rout, rout2, aux0, aux1), for the L2 prefetch
  static constexpr int PF_RIN = NC, PF_ROUT = 0, PF_ROUT2 = 0,
                       PF_AUX0 = 0, PF_AUX1 = 0;
  FG_DEV static void apply(const PassArgs<R>& a, long long v, R* out, Acc<R>&, const R*) {
#pragma unroll
    for (int c = 0; c < NC; ++c) out[c] = a.rin[c * a.V + v];
  }
};

// Neo-Hookean tangent K : dF from the packed per-voxel state
// (B = F^-T, s1 = g a^2 G, s2 = g (G - lam ln J_e), s3 = g lam; g = (1-d)^2):
//   K : dF = s1 dF + s2 B dF^T B + s3 (B : dF) B.
template <typename R>
FG_DEV void tangent_nh(const R* B, R s1, R s2, R s3, const R* p, R* t) {
  R m[9];  // M = B p^T : M_il = sum_k B_ik p_lk
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int l = 0; l < 3; ++l)
      m[3 * i + l] = B[3 * i] * p[3 * l] + B[3 * i + 1] * p[3 * l + 1] + B[3 * i + 2] * p[3 * l + 2];
  R bp = 0;
#pragma unroll
  for (int k = 0; k < 9; ++k) bp += B[k] * p[k];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const R mb = m[3 * i] * B[j] + m[3 * i + 1] * B[3 + j] + m[3 * i + 2] * B[6 + j];
      t[3 * i + j] = s1 * p[3 * i + j] + s2 * mb + s3 * bp * B[3 * i + j];
    }
}

// Saint-Venant-Kirchhoff tangent from the packed state (F, S, s1 = g a^2,
// s2 = g a^4 lam, s3 = g a^4 G): with M = F^T dF,
//   K : dF = s1 dF S + F (s2 tr(M) I + s3 (M + M^T)).
template <typename R>
FG_DEV void tangent_svk(const R* st, long long V, long long v, const R* p, R* t) {
  R F[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) F[k] = st[k * V + v];
  const R Sxx = st[9 * V + v], Syy = st[10 * V + v], Szz = st[11 * V + v];
  const R Sxy = st[12 * V + v], Sxz = st[13 * V + v], Syz = st[14 * V + v];
  const R s1 = st[15 * V + v], s2 = st[16 * V + v], s3 = st[17 * V + v];
  const R S[9] = {Sxx, Sxy, Sxz, Sxy, Syy, Syz, Sxz, Syz, Szz};
  R M[9];  // M_ij = sum_k F_ki p_kj
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) M[3 * i + j] = F[i] * p[j] + F[3 + i] * p[3 + j] + F[6 + i] * p[6 + j];
  const R tr = M[0] + M[4] + M[8];
  R W[9];  // s2 tr(M) I + s3 (M + M^T)
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) W[3 * i + j] = s3 * (M[3 * i + j] + M[3 * j + i]) + (i == j ? s2 * tr : (R)0);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const R pS = p[3 * i] * S[j] + p[3 * i + 1] * S[3 + j] + p[3 * i + 2] * S[6 + j];
      const R FW = F[3 * i] * W[j] + F[3 * i + 1] * W[3 + j] + F[3 * i + 2] * W[6 + j];
      t[3 * i + j] = s1 * pS + FW;
    }
}

template <typename R>
struct PTangentSVK {
  static constexpr int COUT = 9;
  static constexpr bool RED = false;
  // components read per field (rin, rout, rout2, aux0, aux1), for the L2 prefetch
  static constexpr int PF_RIN = 9, PF_ROUT = 0, PF_ROUT2 = 0,
                       PF_AUX0 = 18, PF_AUX1 = 0;
  FG_DEV static void apply(const PassArgs<R>& a, long long v, R* out, Acc<R>&, const R*) {
    R p[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) p[c] = a.rin[c * a.V + v];
    tangent_svk(a.aux[0], a.V, v, p, out);
  }
};

template <typename R>
struct PCgTangentSVK {
  static constexpr int COUT = 9;
  static constexpr bool RED = true;
  // components read per field (rin, rout, rout2, aux0, aux1), for the L2 prefetch
  static constexpr int PF_RIN = 9, PF_ROUT = 9, PF_ROUT2 = 0,
                       PF_AUX0 = 18, PF_AUX1 = 0;
  FG_DEV static void apply(const PassArgs<R>& a, long long v, R* out, Acc<R>& acc, const R* sc) {
    const R beta = sc[1];
    const R* __restrict__ r = a.rin;
    R* __restrict__ pp = a.rout;
    const long long V = a.V;
    R p[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) p[c] = r[c * V + v] + beta * pp[c * V + v];
    tangent_svk(a.aux[0], V, v, p, out);
#pragma unroll
    for (int c = 0; c < 9; ++c) pp[c * V + v] = p[c];
    const R sig = a.coef[1];
#pragma unroll
    for (int c = 0; c < 9; ++c) acc.add(p[c] * (out[c] + sig * p[c]));
  }
};

template <typename R>
struct PTangentNH {
  static constexpr int COUT = 9;
  static constexpr bool RED = false;
  // components read per field (rin, rout, rout2, aux0, aux1), for the L2 prefetch
  static constexpr int PF_RIN = 9, PF_ROUT = 0, PF_ROUT2 = 0,
                       PF_AUX0 = 12, PF_AUX1 = 0;
  FG_DEV static void apply(const PassArgs<R>& a, long long v, R* out, Acc<R>&, const R*) {
    R p[9], B[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) p[c] = a.rin[c * a.V + v];
    const R* st = a.aux[0];
#pragma unroll
    for (int c = 0; c < 9; ++c) B[c] = st[c * a.V + v];
    tangent_nh(B, st[9 * a.V + v], st[10 * a.V + v], st[11 * a.V + v], p, out);
  }
};

// Conjugate-gradient direction update fused with the tangent (mechanical CG):
//   p = r + beta p  (written back, in place),  tau = K : p,  accumulates <p, K p>.
// For a compatible p (every CG direction is a combination of projected fields)
// <p, K p> = <p, G K p>, so the step length is known before the inverse transform.
// A shifted system (G K G + sigma I) adds sigma |p|^2.
// rin = r, rout = p, aux0 = packed state, dscal[1] = beta, coef[1] = sigma.
template <typename R>
struct PCgTangentNH {
  static constexpr int COUT = 9;
  static constexpr bool RED = true;
  // components read per field (rin, rout, rout2, aux0, aux1), for the L2 prefetch
  static constexpr int PF_RIN = 9, PF_ROUT = 9, PF_ROUT2 = 0,
                       PF_AUX0 = 12, PF_AUX1 = 0;
  FG_DEV static void apply(const PassArgs<R>& a, long long v, R* out, Acc<R>& acc, const R* sc) {
    const R beta = sc[1];
    const R* __restrict__ r = a.rin;
    const R* __restrict__ st = a.aux[0];
    R* __restrict__ pp = a.rout;
    const long long V = a.V;
    // every load before the first store (r, p and the state never alias)
    R p[9], B[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) p[c] = r[c * V + v] + beta * pp[c * V + v];
#pragma unroll
    for (int c = 0; c < 9; ++c) B[c] = st[c * V + v];
    const R s1 = st[9 * V + v], s2 = st[10 * V + v], s3 = st[11 * V + v];
#pragma unroll
    for (int c = 0; c < 9; ++c) pp[c * V + v] = p[c];
    tangent_nh(B, s1, s2, s3, p, out);
    const R sig = a.coef[1];
#pragma unroll
    for (int c = 0; c < 9; ++c) acc.add(p[c] * (out[c] + sig * p[c]));
  }
};

// ================================================================== X-inv epilogues

// One component of the fused CG update (pointers already shifted to the component):
// r -= alpha (q + sigma p), x += alpha p; accumulates r^2.  rout = r, rout2 = x, aux0 = p,
// coef[1] = sigma (0 unless the system is shifted).
template <typename R>
struct ECgUpdate1 {
  static constexpr int CIN = 1;
  static constexpr bool RED = true;
  // components read per field (rin, rout, rout2, aux0, aux1), for the L2 prefetch
  static constexpr int PF_RIN = 0, PF_ROUT = 9, PF_ROUT2 = 9,
                       PF_AUX0 = 9, PF_AUX1 = 0;
  FG_DEV static void apply(const PassArgs<R>& a, long long v, const R* val, Acc<R>& acc, const R* sc) {
    apply_ops(a, v, load_ops(a, v), val, acc, sc);
  }
  // the operands of one element, loaded ahead of the update (grouped loads in X-inv)
  struct Ops {
    R r, x, p;
  };
  FG_DEV static Ops load_ops(const PassArgs<R>& a, long long v) {
    return Ops{a.rout[v], a.rout2[v], a.aux[0][v]};
  }
  FG_DEV static void apply_ops(const PassArgs<R>& a, long long v, const Ops& o, const R* val,
                               Acc<R>& acc, const R* sc) {
    const R al = sc[0];
    const R rn = o.r - al * (val[0] + a.coef[1] * o.p);
    a.rout[v] = rn;
    a.rout2[v] = o.x + al * o.p;
    acc.add(rn * rn);
  }
};

// Conjugate-gradient update fused with the inverse transform (mechanical CG): with
// q = G K p arriving as `val`, r -= alpha (q + sigma p) and x += alpha p; accumulates
// <r, r>.  rout = r, rout2 = x, aux0 = p, dscal[0] = alpha, coef[1] = sigma.
template <typename R>
struct ECgUpdate {
  static constexpr int CIN = 9;
  static constexpr bool RED = true;
  // components read per field (rin, rout, rout2, aux0, aux1), for the L2 prefetch
  static constexpr int PF_RIN = 0, PF_ROUT = 9, PF_ROUT2 = 9,
                       PF_AUX0 = 9, PF_AUX1 = 0;
  FG_DEV static void apply(const PassArgs<R>& a, long long v, const R* val, Acc<R>& acc, const R* sc) {
    const R al = sc[0];
    const R sig = a.coef[1];
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      const long long i = c * a.V + v;
      const R pc = a.aux[0][i];
      const R rn = a.rout[i] - al * (val[c] + sig * pc);
      a.rout[i] = rn;
      a.rout2[i] += al * pc;
      acc.add(rn * rn);
    }
  }
};

template <typename R, int NC>
struct EStore {
  static constexpr int CIN = NC;
  static constexpr bool RED = false;
  FG_DEV static void apply(const PassArgs<R>& a, long long v, const R* val, Acc<R>&, const R*) {
#pragma unroll
    for (int c = 0; c < NC; ++c) a.rout[c * a.V + v] = val[c];
  }
};

// store and accumulate <aux0, y>
template <typename R, int NC>
struct EStoreDot {
  static constexpr int CIN = NC;
  static constexpr bool RED = true;
  // components read per field (rin, rout, rout2, aux0, aux1), for the L2 prefetch
  static constexpr int PF_RIN = 0, PF_ROUT = 0, PF_ROUT2 = 0,
                       PF_AUX0 = NC, PF_AUX1 = 0;
  FG_DEV static void apply(const PassArgs<R>& a, long long v, const R* val, Acc<R>& acc, const R* sc) {
    apply_ops(a, v, load_ops(a, v), val, acc, sc);
  }
  struct Ops {
    R x[NC];
  };
  FG_DEV static Ops load_ops(const PassArgs<R>& a, long long v) {
    Ops o;
#pragma unroll
    for (int c = 0; c < NC; ++c) o.x[c] = a.aux[0][c * a.V + v];
    return o;
  }
  FG_DEV static void apply_ops(const PassArgs<R>& a, long long v, const Ops& o, const R* val,
                               Acc<R>& acc, const R*) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      a.rout[c * a.V + v] = val[c];
      acc.add(val[c] * o.x[c]);
    }
  }
};

// store and accumulate |y|^2
template <typename R, int NC>
struct ENorm {
  static constexpr int CIN = NC;
  static constexpr bool RED = true;
  FG_DEV static void apply(const PassArgs<R>& a, long long v, const R* val, Acc<R>& acc, const R* sc) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      a.rout[c * a.V + v] = val[c];
      acc.add(val[c] * val[c]);
    }
  }
};

// A(p) = [g_c/l_c + 2H] p + (spectral part); aux0 = p, aux1 = H, coef[0] = g_c/l_c.
template <typename R>
struct EPff {
  static constexpr int CIN = 1;
  static constexpr bool RED = true;
  // components read per field (rin, rout, rout2, aux0, aux1), for the L2 prefetch
  static constexpr int PF_RIN = 0, PF_ROUT = 0, PF_ROUT2 = 0,
                       PF_AUX0 = 1, PF_AUX1 = 1;
  FG_DEV static void apply(const PassArgs<R>& a, long long v, const R* val, Acc<R>& acc, const R* sc) {
    const R p = a.aux[0][v];
    const R y = (a.coef[0] + (R)2 * a.aux[1][v]) * p + val[0];
    a.rout[v] = y;
    acc.add(p * y);
  }
};

// chemistry flux K_c g, K_c symmetric stored as (xx, yy, zz, xy, xz, yz) in aux0
template <typename R>
struct EChemFlux {
  static constexpr int CIN = 3;
  static constexpr bool RED = false;
  // components read per field (rin, rout, rout2, aux0, aux1), for the L2 prefetch
  static constexpr int PF_RIN = 0, PF_ROUT = 0, PF_ROUT2 = 0,
                       PF_AUX0 = 6, PF_AUX1 = 0;
  FG_DEV static void apply(const PassArgs<R>& a, long long v, const R* g, Acc<R>&, const R*) {
    const R* K = a.aux[0];
    const long long V = a.V;
    const R kxx = K[v], kyy = K[V + v], kzz = K[2 * V + v];
    const R kxy = K[3 * V + v], kxz = K[4 * V + v], kyz = K[5 * V + v];
    a.rout[v] = kxx * g[0] + kxy * g[1] + kxz * g[2];
    a.rout[V + v] = kxy * g[0] + kyy * g[1] + kyz * g[2];
    a.rout[2 * V + v] = kxz * g[0] + kyz * g[1] + kzz * g[2];
  }
};

// chemistry Newton operator in y = m dc: y/m + dt L y; aux0 = y, aux1 = 1/m = c(1-c),
// coef[0] = dt; accumulates <y, A y>.
template <typename R>
struct EChemOp {
  static constexpr int CIN = 1;
  static constexpr bool RED = true;
  // components read per field (rin, rout, rout2, aux0, aux1), for the L2 prefetch
  static constexpr int PF_RIN = 0, PF_ROUT = 0, PF_ROUT2 = 0,
                       PF_AUX0 = 1, PF_AUX1 = 1;
  FG_DEV static void apply(const PassArgs<R>& a, long long v, const R* val, Acc<R>& acc, const R* sc) {
    const R y = a.aux[0][v];
    const R o = a.aux[1][v] * y + a.coef[0] * val[0];
    a.rout[v] = o;
    acc.add(y * o);
  }
};

// chemistry residual, stored negated as the Newton right-hand side:
// out = -(base + dt L mu~), base = c - c_t - dt cdot_B in aux0, coef[0] = dt;
// accumulates |out|^2.
template <typename R>
struct EChemRhs {
  static constexpr int CIN = 1;
  static constexpr bool RED = true;
  // components read per field (rin, rout, rout2, aux0, aux1), for the L2 prefetch
  static constexpr int PF_RIN = 0, PF_ROUT = 0, PF_ROUT2 = 0,
                       PF_AUX0 = 1, PF_AUX1 = 0;
  FG_DEV static void apply(const PassArgs<R>& a, long long v, const R* val, Acc<R>& acc, const R* sc) {
    const R o = -(a.aux[0][v] + a.coef[0] * val[0]);
    a.rout[v] = o;
    acc.add(o * o);
  }
};

// ================================================================== fused chemistry CG
// One iteration of the CG of the chemistry Newton system (y/m + dt L y, Eq. Chemderfc in
// y = m dc) with its vector updates folded into the operator passes, as in the mechanical
// CG: <p, A p> = <p, w p> + dt <grad_f p, K_c grad_f p> (w = 1/m) is summed in the forward
// X pass and in the flux round trip, so the step length is known before the inverse
// transform, whose epilogue forms q = w p + dt L p and applies the updates.

// p = r + beta p (in place), the transform input p, and the partial sums of w p^2.
// rin = r, rout = p, aux0 = w, dscal[1] = beta.
template <typename R>
struct PCgChem {
  static constexpr int COUT = 1;
  static constexpr bool RED = true;
  static constexpr int PF_RIN = 1, PF_ROUT = 1, PF_ROUT2 = 0, PF_AUX0 = 1, PF_AUX1 = 0;
  FG_DEV static void apply(const PassArgs<R>& a, long long v, R* out, Acc<R>& acc, const R* sc) {
    const R p = a.rin[v] + sc[1] * a.rout[v];
    a.rout[v] = p;
    out[0] = p;
    acc.add(a.aux[0][v] * p * p);
  }
};

// flux K_c g of the gradient g = grad_f p in the X round trip, and the partial sums of
// dt g . K_c g.  aux0 = K_c (6 components: xx, yy, zz, xy, xz, yz), coef[0] = dt.
template <typename R>
struct EChemFluxRound {
  static constexpr int CIN = 3, COUT = 3;
  static constexpr bool RED = true;
  static constexpr int PF_RIN = 0, PF_ROUT = 0, PF_ROUT2 = 0, PF_AUX0 = 6, PF_AUX1 = 0;
  FG_DEV static void apply(const PassArgs<R>& a, long long v, const R* g, R* out, Acc<R>& acc,
                           const R*) {
    const R* K = a.aux[0];
    const long long V = a.V;
    const R kxx = K[v], kyy = K[V + v], kzz = K[2 * V + v];
    const R kxy = K[3 * V + v], kxz = K[4 * V + v], kyz = K[5 * V + v];
    out[0] = kxx * g[0] + kxy * g[1] + kxz * g[2];
    out[1] = kxy * g[0] + kyy * g[1] + kyz * g[2];
    out[2] = kxz * g[0] + kyz * g[1] + kzz * g[2];
    acc.add(a.coef[0] * (g[0] * out[0] + g[1] * out[1] + g[2] * out[2]));
  }
};

// q = w p + dt L p from the divergence val, then r -= alpha q, x += alpha p and the partial
// sums of r^2.  rout = r, rout2 = x, aux0 = p, aux1 = w, coef[0] = dt, dscal[0] = alpha.
template <typename R>
struct ECgChemUpdate {
  static constexpr int CIN = 1;
  static constexpr bool RED = true;
  static constexpr int PF_RIN = 0, PF_ROUT = 1, PF_ROUT2 = 1, PF_AUX0 = 1, PF_AUX1 = 1;
  FG_DEV static void apply(const PassArgs<R>& a, long long v, const R* val, Acc<R>& acc, const R* sc) {
    apply_ops(a, v, load_ops(a, v), val, acc, sc);
  }
  struct Ops {
    R p, w, r, x;
  };
  FG_DEV static Ops load_ops(const PassArgs<R>& a, long long v) {
    return Ops{a.aux[0][v], a.aux[1][v], a.rout[v], a.rout2[v]};
  }
  FG_DEV static void apply_ops(const PassArgs<R>& a, long long v, const Ops& o, const R* val,
                               Acc<R>& acc, const R* sc) {
    const R al = sc[0];
    const R q = o.w * o.p + a.coef[0] * val[0];
    const R rn = o.r - al * q;
    a.rout[v] = rn;
    a.rout2[v] = o.x + al * o.p;
    acc.add(rn * rn);
  }
};

// ================================================================== float-float epilogues
// The float-float passes store their results as FP64 (the fields they serve are FP64)
// and accumulate norms in FP64.

template <int NC>
struct EStore<ff, NC> {
  static constexpr int CIN = NC;
  static constexpr bool RED = false;
  FG_DEV static void apply(const PassArgs<ff>& a, long long v, const ff* val, Acc<ff>&, const ff*) {
#pragma unroll
    for (int c = 0; c < NC; ++c) a.rout[c * a.V + v] = (double)val[c];
  }
};

template <int NC>
struct ENorm<ff, NC> {
  static constexpr int CIN = NC;
  static constexpr bool RED = true;
  FG_DEV static void apply(const PassArgs<ff>& a, long long v, const ff* val, Acc<ff>& acc, const ff*) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const double o = (double)val[c];
      a.rout[c * a.V + v] = o;
      acc.add(o * o);
    }
  }
};

// the flux K_c g in FP64 from the float-float gradient; aux0 = K_c (6 FP64 components)
template <>
struct EChemFlux<ff> {
  static constexpr int CIN = 3;
  static constexpr bool RED = false;
  static constexpr int PF_RIN = 0, PF_ROUT = 0, PF_ROUT2 = 0, PF_AUX0 = 6, PF_AUX1 = 0;
  FG_DEV static void apply(const PassArgs<ff>& a, long long v, const ff* gf, Acc<ff>&, const ff*) {
    const double* K = a.aux[0];
    const long long V = a.V;
    const double g[3] = {(double)gf[0], (double)gf[1], (double)gf[2]};
    const double kxx = K[v], kyy = K[V + v], kzz = K[2 * V + v];
    const double kxy = K[3 * V + v], kxz = K[4 * V + v], kyz = K[5 * V + v];
    a.rout[v] = kxx * g[0] + kxy * g[1] + kxz * g[2];
    a.rout[V + v] = kxy * g[0] + kyy * g[1] + kyz * g[2];
    a.rout[2 * V + v] = kxz * g[0] + kyz * g[1] + kzz * g[2];
  }
};

template <>
struct EChemRhs<ff> {
  static constexpr int CIN = 1;
  static constexpr bool RED = true;
  static constexpr int PF_RIN = 0, PF_ROUT = 0, PF_ROUT2 = 0, PF_AUX0 = 1, PF_AUX1 = 0;
  FG_DEV static void apply(const PassArgs<ff>& a, long long v, const ff* val, Acc<ff>& acc, const ff*) {
    const double o = -(a.aux[0][v] + (double)a.coef[0] * (double)val[0]);
    a.rout[v] = o;
    acc.add(o * o);
  }
};

}  // namespace fg
