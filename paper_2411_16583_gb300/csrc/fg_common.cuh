// Common device/host helpers of the GB300 FFT chemo-mechanical kernels.
//
// Kernels are written as a sequence of *phases* separated by block barriers.  A phase is
// straight-line per-thread code that reads and writes shared memory and the thread's own
// carried registers (`L`, a `Locals` struct).  Built for the GPU, a phase is the code of
// thread `threadIdx.x` followed by `__syncthreads()`.  Built with FG_EMU (the host
// emulation library used only by CPU tests), the same source runs every thread of a block
// in turn with its own `Locals`, which reproduces the barrier semantics exactly.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <cmath>

#define FG_HD __host__ __device__ __forceinline__
// code that runs inside kernels only (device-only in the GPU build)
#ifdef FG_EMU
#define FG_DEV inline
#else
#define FG_DEV __device__ __forceinline__
#endif

#ifdef FG_EMU
#define FG_PHASE(NT_)                       \
  for (int tid = 0; tid < (NT_); ++tid) {   \
    auto& L = Ls[tid];                      \
    (void)L;
#define FG_END_PHASE }
#else
#define FG_PHASE(NT_)                       \
  {                                         \
    const int tid = (int)threadIdx.x;       \
    auto& L = Ls[0];                        \
    (void)L;
#define FG_END_PHASE \
  }                  \
  __syncthreads();
#endif

#ifdef FG_EMU
// host stand-in of the device atomic used for error flags
inline int atomicOr(int* p, int v) {
  const int o = *p;
  *p = o | v;
  return o;
}
#endif

namespace fg {

struct Dim3 {
  int x, y, z;
};

// ------------------------------------------------------------------ per-thread sums
// FP64 kernels accumulate in FP64.  FP32 kernels accumulate a compensated pair of floats
// (Neumaier's summation): GB300 runs FP64 instructions at a small fraction of the FP32
// rate, and one FP64 operation per element throttled the FP32 passes.  The block
// reduction converts the pair to FP64.

template <typename R> struct Acc;
template <> struct Acc<double> {
  double s;
  FG_HD void zero() { s = 0.0; }
  FG_HD void add(double x) { s += x; }
  FG_HD double value() const { return s; }
};
template <> struct Acc<float> {
  float s, c;
  FG_HD void zero() { s = 0.f; c = 0.f; }
  FG_HD void add(float x) {
    const float t = s + x;
    c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
    s = t;
  }
  FG_HD double value() const { return (double)s + (double)c; }
};

// ------------------------------------------------------------------ float-float reals
// A real carried as the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2: about
// 48 significant bits from FP32 instructions alone (GB300 issues FP64 at a small fraction
// of its FP32 rate).  Sums use Knuth's error-free TwoSum and products the FMA form of
// Dekker's TwoProduct, renormalised as in the double-double algorithms of Dekker (1971)
// and Hida, Li and Bailey (2001); the quotient is one correction step of the float
// quotient.  The residual transforms of the mixed-precision mode run on it: stored in
// FP64, transformed in float-float.  FP32 addition and multiplication are IEEE in both
// builds; only explicit fmaf contracts.

struct ff {
  float hi, lo;
  FG_HD constexpr ff() : hi(0.f), lo(0.f) {}
  FG_HD constexpr ff(float h, float l) : hi(h), lo(l) {}
  // split of a double: hi its nearest float, lo the nearest float of the remainder
  FG_HD constexpr ff(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  FG_HD constexpr ff(int x) : hi((float)x), lo(0.f) {}
  FG_HD explicit operator double() const { return (double)hi + (double)lo; }
  FG_HD explicit operator int() const { return (int)hi; }
};

FG_HD ff ff_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return ff(s, (a - (s - bb)) + (b - bb));
}
FG_HD ff ff_quick_two_sum(float a, float b) {  // |a| >= |b| (or a = 0)
  const float s = a + b;
  return ff(s, b - (s - a));
}
// The sum of Dekker's add (the "sloppy" addition of the double-double literature): the low
// parts are added in one float operation, so the error is within a few units of 2^-48 of
// |a| + |b| (not of |a + b|): the norm-wise accuracy that transforms and projections need,
// at 11 float operations instead of 20.
FG_HD ff operator+(ff a, ff b) {
  const ff s = ff_two_sum(a.hi, b.hi);
  return ff_quick_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
FG_HD ff operator-(ff a) { return ff(-a.hi, -a.lo); }
FG_HD ff operator-(ff a, ff b) { return a + (-b); }
FG_HD ff operator*(ff a, ff b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return ff_quick_two_sum(p, e);
}
FG_HD ff operator/(ff a, ff b) {
  const float q1 = a.hi / b.hi;
  const ff r = a - ff(q1, 0.f) * b;
  const float q2 = r.hi / b.hi;
  return ff_quick_two_sum(q1, q2);
}
FG_HD ff& operator+=(ff& a, ff b) { return a = a + b; }
FG_HD ff& operator-=(ff& a, ff b) { return a = a - b; }
FG_HD ff& operator*=(ff& a, ff b) { return a = a * b; }
FG_HD bool operator>(ff a, ff b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
FG_HD bool operator<(ff a, ff b) { return b > a; }

struct ffc {  // complex float-float
  ff x, y;
};

// the type real-space fields of a precision are stored in: float-float transforms read
// and write FP64 fields
template <typename R> struct io_type { using type = R; };
template <> struct io_type<ff> { using type = double; };
template <typename R> using io_t = typename io_type<R>::type;

template <> struct Acc<ff> {  // float-float passes accumulate their FP64 outputs in FP64
  double s;
  FG_HD void zero() { s = 0.0; }
  FG_HD void add(double x) { s += x; }
  FG_HD double value() const { return s; }
};

// ------------------------------------------------------------------ complex arithmetic

template <typename R> struct ctype;
template <> struct ctype<float> { using type = float2; };
template <> struct ctype<double> { using type = double2; };
template <> struct ctype<ff> { using type = ffc; };
template <typename R> using cplx = typename ctype<R>::type;

template <typename C> FG_HD C cmk(decltype(C::x) a, decltype(C::x) b) {
  C c;
  c.x = a;
  c.y = b;
  return c;
}
template <typename C> FG_HD C cadd(C a, C b) { return cmk<C>(a.x + b.x, a.y + b.y); }
template <typename C> FG_HD C csub(C a, C b) { return cmk<C>(a.x - b.x, a.y - b.y); }
template <typename C> FG_HD C cmul(C a, C b) {
  return cmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename C> FG_HD C cmulc(C a, C b) {
  return cmk<C>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename C> FG_HD C cconj(C a) { return cmk<C>(a.x, -a.y); }
template <typename C> FG_HD C cscale(C a, decltype(C::x) s) { return cmk<C>(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename C> FG_HD C crot(C a) {
  return INV ? cmk<C>(-a.y, a.x) : cmk<C>(a.y, -a.x);
}

// ------------------------------------------------------------------ small DFT codelets
// y_k = sum_r v_r exp(-+ 2 pi i r k / R), in place, natural order in and out.

template <int R, bool INV, typename C> struct Dft;

template <bool INV, typename C> struct Dft<1, INV, C> {
  FG_HD static void run(C*) {}
};

template <bool INV, typename C> struct Dft<2, INV, C> {
  FG_HD static void run(C* v) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <bool INV, typename C> struct Dft<4, INV, C> {
  FG_HD static void run(C* v) {
    C s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    C s13 = cadd(v[1], v[3]), d13 = crot<INV>(csub(v[1], v[3]));
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    v[1] = cadd(d02, d13);
    v[3] = csub(d02, d13);
  }
};

template <bool INV, typename C> struct Dft<8, INV, C> {
  FG_HD static void run(C* v) {
    using R = decltype(C::x);
    const R h = (R)0.70710678118654752440;
    C e[4] = {v[0], v[2], v[4], v[6]};
    C o[4] = {v[1], v[3], v[5], v[7]};
    Dft<4, INV, C>::run(e);
    Dft<4, INV, C>::run(o);
    // o_k *= exp(-+ i pi k / 4)
    C o1 = INV ? cmk<C>(h * (o[1].x - o[1].y), h * (o[1].x + o[1].y))
               : cmk<C>(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));
    C o2 = crot<INV>(o[2]);
    C o3 = INV ? cmk<C>(-h * (o[3].x + o[3].y), h * (o[3].x - o[3].y))
               : cmk<C>(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);
    v[7] = csub(e[3], o3);
  }
};

// 16 = 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2.
template <bool INV, typename C> struct Dft<16, INV, C> {
  FG_HD static void run(C* v) {
    using R = decltype(C::x);
    // cos/sin of m pi / 8, m = 0..4
    const R c1 = (R)0.92387953251128675613, s1 = (R)0.38268343236508977173;
    const R h = (R)0.70710678118654752440;
    C a[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      C t[4] = {v[n2], v[4 + n2], v[8 + n2], v[12 + n2]};
      Dft<4, INV, C>::run(t);
#pragma unroll
      for (int k1 = 0; k1 < 4; ++k1) a[n2][k1] = t[k1];
    }
    // twiddle a[n2][k1] by W16^(n2 k1), W16 = exp(-+ 2 pi i / 16)
    const R ws = INV ? (R)1 : (R)-1;
    const R cw[10] = {(R)1, c1, h, s1, (R)0, -s1, -h, -c1, (R)-1, -c1};
    const R sw[10] = {(R)0, s1, h, c1, (R)1, c1, h, s1, (R)0, -s1};
#pragma unroll
    for (int n2 = 1; n2 < 4; ++n2)
#pragma unroll
      for (int k1 = 1; k1 < 4; ++k1) {
        const int m = n2 * k1;
        a[n2][k1] = cmul(a[n2][k1], cmk<C>(cw[m], ws * sw[m]));
      }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      C t[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
      Dft<4, INV, C>::run(t);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[k2];
    }
  }
};

template <bool INV, typename C> struct Dft<3, INV, C> {
  FG_HD static void run(C* v) {
    using R = decltype(C::x);
    const R s3 = (R)0.86602540378443864676;
    C t = cadd(v[1], v[2]);
    C d = csub(v[1], v[2]);
    C m = cmk<C>(v[0].x - (R)0.5 * t.x, v[0].y - (R)0.5 * t.y);
    C r = crot<INV>(cscale(d, s3));  // -+ i s3 (v1 - v2)
    v[0] = cadd(v[0], t);
    v[1] = cadd(m, r);
    v[2] = csub(m, r);
  }
};

template <bool INV, typename C> struct Dft<5, INV, C> {
  FG_HD static void run(C* v) {
    using R = decltype(C::x);
    const R c1 = (R)0.30901699437494742410, c2 = (R)-0.80901699437494742410;
    const R s1 = (R)0.95105651629515357212, s2 = (R)0.58778525229247312917;
    C t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    C d1 = csub(v[1], v[4]), d2 = csub(v[2], v[3]);
    C a1 = cmk<C>(v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y);
    C a2 = cmk<C>(v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y);
    C b1 = crot<INV>(cmk<C>(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y));
    C b2 = crot<INV>(cmk<C>(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y));
    v[0] = cadd(v[0], cadd(t1, t2));
    v[1] = cadd(a1, b1);
    v[4] = csub(a1, b1);
    v[2] = cadd(a2, b2);
    v[3] = csub(a2, b2);
  }
};

// ------------------------------------------------------------------ radix plans

struct Plan {
  int S;      // number of stages
  int r[6];   // radix of each stage
  int rmax;   // largest radix
};

constexpr Plan make_plan(int N) {
  Plan p{0, {1, 1, 1, 1, 1, 1}, 1};
  int n = N, p2 = 0, p3 = 0, p5 = 0;
  while (n % 2 == 0 && n > 1) { n /= 2; ++p2; }
  while (n % 3 == 0) { n /= 3; ++p3; }
  while (n % 5 == 0) { n /= 5; ++p5; }
  const int st2 = (p2 + 3) / 4;
  for (int s = 0; s < st2; ++s) {
    const int e = p2 / st2 + (s < p2 % st2 ? 1 : 0);
    p.r[p.S++] = 1 << e;
  }
  for (int s = 0; s < p3; ++s) p.r[p.S++] = 3;
  for (int s = 0; s < p5; ++s) p.r[p.S++] = 5;
  for (int s = 0; s < p.S; ++s) p.rmax = p.r[s] > p.rmax ? p.r[s] : p.rmax;
  return p;
}

constexpr bool plan_ok(int N) {
  int n = N;
  while (n % 2 == 0 && n > 1) n /= 2;
  while (n % 3 == 0) n /= 3;
  while (n % 5 == 0) n /= 5;
  return n == 1;
}

constexpr int plan_ns(int N, int s) {  // product of the radices before stage s
  Plan p = make_plan(N);
  int ns = 1;
  for (int i = 0; i < s; ++i) ns *= p.r[i];
  return ns;
}

// Padded shared-memory position of element i of a row: one spare slot per 16 elements
// so that the stride-R stores of a radix-R stage spread over the banks.
FG_HD constexpr int pad16(int i) { return i + (i >> 4); }
constexpr int row_pitch(int N) { return N + (N >> 4) + 1; }

}  // namespace fg
