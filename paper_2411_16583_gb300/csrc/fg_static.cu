// fg_mech_apply_noalloc: the FP32 mechanical operator application with every piece of
// scratch memory in one file-scope device array, for callers that cannot allocate GPU
// memory themselves (see include/fg.h).  Nothing here calls cudaMalloc or cudaFree.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "fg_pointwise.cuh"
#include "../../include/fg.h"

namespace fg {

constexpr int NA_MAX_EDGE = 64;
constexpr long long NA_MAX_V = (long long)NA_MAX_EDGE * NA_MAX_EDGE * NA_MAX_EDGE;
constexpr long long NA_MAX_VH = (long long)(NA_MAX_EDGE / 2 + 1) * NA_MAX_EDGE * NA_MAX_EDGE;
constexpr long long NA_MAX_PARTS = (long long)NA_MAX_EDGE * NA_MAX_EDGE + VEC_BLOCKS + 64;

constexpr long long na_align(long long b) { return (b + 255) / 256 * 256; }
// byte offsets of the pieces of the scratch array
constexpr long long NA_S1 = 0;
constexpr long long NA_S2 = NA_S1 + na_align(9 * NA_MAX_VH * (long long)sizeof(float2));
constexpr long long NA_STATE = NA_S2 + na_align(9 * NA_MAX_VH * (long long)sizeof(float2));
constexpr long long NA_TW = NA_STATE + na_align(12 * NA_MAX_V * (long long)sizeof(float));
constexpr long long NA_TAB = NA_TW + na_align(3 * NA_MAX_EDGE * (long long)sizeof(float2));
constexpr long long NA_XI = NA_TAB + na_align(9 * NA_MAX_EDGE * (long long)sizeof(float));
constexpr long long NA_PART = NA_XI + na_align(3 * NA_MAX_EDGE * (long long)sizeof(float2));
constexpr long long NA_KS = NA_PART + na_align(NA_MAX_PARTS * (long long)sizeof(double));
constexpr long long NA_BYTES = NA_KS + na_align((long long)sizeof(KScal));

}  // namespace fg

#ifndef FG_EMU
// Static scratch of fg_mech_apply_noalloc (about 32 MB), present on every device that
// loads the library.  Host code must not use its name as an address: the device address
// comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[fg::NA_BYTES];
#endif

namespace fg {

// message of fg_last_error (defined with the rest of the C ABI)
void set_last_error(const std::string& msg);

#ifndef FG_EMU
// device address of the scratch array on the current device, looked up once per device
static int noalloc_scratch(unsigned char** out) {
  static std::mutex m;
  static unsigned char* ptrs[256] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 256) {
    set_last_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return FG_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(m);
  if (!ptrs[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_last_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return FG_ERR_CUDA;
    }
    ptrs[dev] = (unsigned char*)p;
  }
  *out = ptrs[dev];
  return FG_OK;
}
#endif

}  // namespace fg

using namespace fg;

extern "C" int fg_mech_apply_noalloc(int nx, int ny, int nz, double hx, double hy, double hz,
                                     const double* F, const double* c, const double* d,
                                     const double* lam, const double* mu, const double* Omega,
                                     const double* c0, const float* x, float* y, double* dot,
                                     void* stream) {
  set_last_error("");
#ifdef FG_EMU
  (void)nx; (void)ny; (void)nz; (void)hx; (void)hy; (void)hz; (void)F; (void)c; (void)d;
  (void)lam; (void)mu; (void)Omega; (void)c0; (void)x; (void)y; (void)dot; (void)stream;
  set_last_error("fg_mech_apply_noalloc needs the GPU build");
  return FG_ERR_INVALID;
#else
  if (!F || !c || !d || !lam || !mu || !Omega || !c0 || !x || !y) {
    set_last_error("fg_mech_apply_noalloc: null pointer");
    return FG_ERR_INVALID;
  }
  if (nx < 2 || nx % 2 || ny < 1 || nz < 1 || nx > NA_MAX_EDGE || ny > NA_MAX_EDGE ||
      nz > NA_MAX_EDGE || !(hx > 0 && hy > 0 && hz > 0)) {
    set_last_error("fg_mech_apply_noalloc: grid must be even nx, every edge <= 64, h > 0");
    return FG_ERR_INVALID;
  }
  const SizeOps<float>* ox = size_ops<float>(nx);
  const SizeOps<float>* oy = size_ops<float>(ny);
  const SizeOps<float>* oz = size_ops<float>(nz);
  if (!ox || !oy || !oz || !ox->xf_tangent) {
    set_last_error("fg_mech_apply_noalloc: transform length not compiled in");
    return FG_ERR_INVALID;
  }
  unsigned char* base = nullptr;
  int rc = noalloc_scratch(&base);
  if (rc != FG_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const long long V = (long long)nx * ny * nz;
  const int hxn = nx / 2 + 1;
  const long long VH = (long long)hxn * ny * nz;
  float2* S1 = (float2*)(base + NA_S1);
  float2* S2 = (float2*)(base + NA_S2);
  float* state = (float*)(base + NA_STATE);
  float2* tw = (float2*)(base + NA_TW);
  float* tab = (float*)(base + NA_TAB);
  float2* xi = (float2*)(base + NA_XI);
  double* partials = (double*)(base + NA_PART);
  KScal* ks = (KScal*)(base + NA_KS);

  // frequency and twiddle tables of this grid (host FP64, rounded), copied in
  const int n[3] = {nx, ny, nz};
  const int len[3] = {hxn, ny, nz};
  const double h[3] = {hx, hy, hz};
  std::vector<float2> htw(3 * NA_MAX_EDGE), hxi(3 * NA_MAX_EDGE);
  std::vector<float> htab(9 * NA_MAX_EDGE, 0.f);
  for (int j = 0; j < 3; ++j) {
    for (int m = 0; m < n[j]; ++m) {
      const double a = 2.0 * M_PI * (double)m / (double)n[j];
      htw[j * NA_MAX_EDGE + m] = make_float2((float)cos(a), (float)(-sin(a)));
    }
    for (int k = 0; k < len[j]; ++k) {
      const int ks_ = (j > 0 && 2 * k > n[j]) ? k - n[j] : k;
      const double th = M_PI * (double)ks_ / (double)n[j];
      double co = cos(th);
      if (2 * std::abs(ks_) == n[j]) co = 0.0;
      htab[(0 * 3 + j) * NA_MAX_EDGE + k] = (float)(2.0 / h[j] * sin(th));
      htab[(1 * 3 + j) * NA_MAX_EDGE + k] = (float)co;
      htab[(2 * 3 + j) * NA_MAX_EDGE + k] = (float)(4.0 * sin(th) * sin(th) / (h[j] * h[j]));
      hxi[j * NA_MAX_EDGE + k] = make_float2((float)((cos(2 * th) - 1.0) / h[j]), (float)(sin(2 * th) / h[j]));
    }
  }
  cudaError_t e = cudaMemcpyAsync(tw, htw.data(), htw.size() * sizeof(float2), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(tab, htab.data(), htab.size() * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(xi, hxi.data(), hxi.size() * sizeof(float2), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    set_last_error(std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
    return FG_ERR_CUDA;
  }

  // the scalars (dot product, error flags) start at zero on every call
  e = cudaMemsetAsync(ks, 0, sizeof(KScal), st);
  if (e != cudaSuccess) {
    set_last_error(std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    return FG_ERR_CUDA;
  }
  // packed tangent state of (F, c, d) into the scratch
  VArgs v{};
  v.n = V;
  v.V = V;
  v.in[0] = F;
  v.in[1] = c;
  v.in[2] = d;
  v.in[3] = lam;
  v.in[4] = mu;
  v.in[5] = Omega;
  v.in[6] = c0;
  v.out[1] = state;
  v.partials = partials;
  v.flags = &ks->status;
  launch_vec<KMechState<float>>(v, st);

  auto pb = [&]() {
    PassArgs<float> a{};
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.hx = hxn;
    a.V = V;
    a.VH = VH;
    for (int j = 0; j < 3; ++j) {
      a.rs[j] = tab + (0 * 3 + j) * NA_MAX_EDGE;
      a.rc[j] = tab + (1 * 3 + j) * NA_MAX_EDGE;
      a.lap[j] = tab + (2 * 3 + j) * NA_MAX_EDGE;
      a.xi[j] = xi + j * NA_MAX_EDGE;
    }
    a.partials = partials;
    return a;
  };
  PassArgs<float> a = pb();
  a.tw = tw;
  a.rin = x;
  a.aux[0] = state;
  a.cout = S1;
  ox->xf_tangent(a, st);
  a = pb();
  a.tw = tw + NA_MAX_EDGE;
  a.cin = S1;
  a.cout = S2;
  a.ncomp = 9;
  oy->yf(a, st);
  a = pb();
  a.tw = tw + 2 * NA_MAX_EDGE;
  a.cin = S2;
  a.cout = S2;
  a.coef[0] = (float)(1.0 / (double)V);
  oz->z_proj(a, st);
  a = pb();
  a.tw = tw + NA_MAX_EDGE;
  a.cin = S2;
  a.cout = S1;
  a.ncomp = 9;
  oy->yi(a, st);
  a = pb();
  a.tw = tw;
  a.cin = S1;
  a.rout = y;
  a.aux[0] = x;
  const int nb = ox->xi_storedot9(a, st);
  VArgs f{};
  f.n = nb;
  f.partials = partials;
  f.ks = ks;
  launch_fin<FStore>(f, st);
  KScal hk;
  e = cudaMemcpyAsync(&hk, ks, sizeof(KScal), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(std::string("fg_mech_apply_noalloc: ") + cudaGetErrorString(e));
    return FG_ERR_CUDA;
  }
  if (hk.status & ST_DOMAIN) {
    set_last_error("fg_mech_apply_noalloc: det F <= 0 or J_c <= 0");
    return FG_ERR_DOMAIN;
  }
  if (dot) *dot = hk.aux;
  return FG_OK;
#endif
}

