// Host runtime of the solver: context and device memory, the operator pipelines, the
// Krylov / Newton / staggered drivers (Alg. 1-4) and the C ABI of include/fg.h.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <cmath>
#include <algorithm>
#include <array>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "fg_pointwise.cuh"
#include "fg_adjoint.cuh"
#include "../../include/fg.h"
#ifndef FG_EMU
#include <nvtx3/nvToolsExt.h>
#else
#include <sys/mman.h>
#include <unistd.h>
#endif

namespace fg {

// ------------------------------------------------------------------ size registry

template <typename R>
static std::map<int, SizeOps<R>>& registry() {
  static std::map<int, SizeOps<R>> m;
  return m;
}
std::atomic<long long>& launch_counter() {
  static std::atomic<long long> n{0};
  return n;
}

void register_size_ops_f(const SizeOps<float>& s) { registry<float>()[s.N] = s; }
void register_size_ops_d(const SizeOps<double>& s) { registry<double>()[s.N] = s; }
void register_size_ops_ff(const SizeOps<ff>& s) { registry<ff>()[s.N] = s; }
template <typename R>
const SizeOps<R>* size_ops(int N) {
  auto& m = registry<R>();
  auto it = m.find(N);
  return it == m.end() ? nullptr : &it->second;
}

// ------------------------------------------------------------------ errors

static thread_local std::string g_err;

// progress trace on stderr when the environment variable FG_VERBOSE is set
static bool verbose() {
  static const bool v = getenv("FG_VERBOSE") != nullptr;
  return v;
}
void set_last_error(const std::string& msg) { g_err = msg; }

// NVTX range over one solve phase (step, chemistry, mechanics, history, phase field,
// adjoint), for profilers that filter or group launches by range; without a tool attached
// the calls do nothing
struct Range {
#ifndef FG_EMU
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
#else
  explicit Range(const char*) {}
#endif
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

struct Fail {
  int code;
};

static void fail(int code, const std::string& msg) {
  g_err = msg;
  throw Fail{code};
}

// ------------------------------------------------------------------ device memory

#ifdef FG_EMU
// Emulated device memory is guarded: every buffer lies between two inaccessible pages and
// ends at the upper one (its start rounded down to 16 bytes), so a kernel that indexes
// past the end of a buffer, or far before its start, faults in the host tests instead of
// touching a neighbouring buffer.  FG_EMU_GUARD=start puts the start on the lower guard
// page instead, which catches any index below zero.
struct GuardedBlock {
  char* base;
  size_t len;
};
static std::mutex& guard_mutex() {
  static std::mutex m;
  return m;
}
static std::map<void*, GuardedBlock>& guard_blocks() {
  static std::map<void*, GuardedBlock> m;
  return m;
}
static void* dalloc(size_t n) {
  static const bool at_start = [] {
    const char* e = getenv("FG_EMU_GUARD");
    return e && strcmp(e, "start") == 0;
  }();
  const size_t pg = (size_t)sysconf(_SC_PAGESIZE);
  const size_t m = n ? n : 1;
  const size_t body = (m + pg - 1) / pg * pg;
  const size_t len = body + 2 * pg;
  void* b = mmap(nullptr, len, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
  if (b == MAP_FAILED) fail(FG_ERR_OOM, "host allocation failed");
  char* base = (char*)b;
  if (mprotect(base, pg, PROT_NONE) != 0 || mprotect(base + pg + body, pg, PROT_NONE) != 0) {
    munmap(b, len);
    fail(FG_ERR_OOM, "guard page setup failed");
  }
  char* p = at_start ? base + pg : base + pg + ((body - m) & ~(size_t)15);
  std::lock_guard<std::mutex> lk(guard_mutex());
  guard_blocks()[p] = GuardedBlock{base, len};
  return p;
}
static void dfree(void* p) {
  if (!p) return;
  GuardedBlock g{nullptr, 0};
  {
    std::lock_guard<std::mutex> lk(guard_mutex());
    auto it = guard_blocks().find(p);
    if (it == guard_blocks().end()) return;
    g = it->second;
    guard_blocks().erase(it);
  }
  munmap(g.base, g.len);
}
static void dcopy(void* d, const void* s, size_t n, cudaStream_t) { memcpy(d, s, n); }
static void dzero(void* d, size_t n, cudaStream_t) { memset(d, 0, n); }
static void dsync(cudaStream_t) {}
static void ccheck(const char*) {}
static void* hpinned(size_t n) { return dalloc(n); }
static void hfree(void* p) { dfree(p); }
#else
static void ccheck(const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) fail(FG_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
static void* dalloc(size_t n) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, n ? n : 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(FG_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  return p;
}
static void dfree(void* p) {
  if (p) cudaFree(p);
}
static void dcopy(void* d, const void* s, size_t n, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(d, s, n, cudaMemcpyDefault, st);
  if (e != cudaSuccess) fail(FG_ERR_CUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
}
static void dzero(void* d, size_t n, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(d, 0, n, st);
  if (e != cudaSuccess) fail(FG_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
}
static void dsync(cudaStream_t st) {
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) fail(FG_ERR_CUDA, std::string("cudaStreamSynchronize: ") + cudaGetErrorString(e));
  ccheck("kernel");
}
static void* hpinned(size_t n) {
  void* p = nullptr;
  if (cudaMallocHost(&p, n) != cudaSuccess) fail(FG_ERR_OOM, "cudaMallocHost failed");
  return p;
}
static void hfree(void* p) {
  if (p) cudaFreeHost(p);
}
#endif

// ------------------------------------------------------------------ context

enum { KS_MECH = 0, KS_PFF = 1, KS_CHEM = 2, KS_MISC = 3, KS_HBAR = 4, KS_N = 5 };

template <typename R>
struct Prec {
  using C = cplx<R>;
  using IO = io_t<R>;  // real-space fields (FP64 for the float-float set)
  bool on = false;
  C *S1 = nullptr, *S2 = nullptr;
  C *twx = nullptr, *twy = nullptr, *twz = nullptr;
  R *rs[3] = {}, *rc[3] = {}, *lap[3] = {};
  C* xi[3] = {};
  IO *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *b = nullptr, *z = nullptr;
  IO* xbest = nullptr;  // best-residual CG iterate
  IO *state = nullptr, *kc = nullptr, *w = nullptr, *Hr = nullptr, *tmp3 = nullptr;
  const SizeOps<R>*ox = nullptr, *oy = nullptr, *oz = nullptr;
};

// Recorded trajectory of fg_step calls for the adjoint: the step sizes and macroscopic
// deformation gradients, and checkpoints (c, F, d, H and Fbar, 12 V doubles) of the state
// before every `every`-th step.
struct Tape {
  int every = 1;
  std::vector<double> dts;
  std::vector<std::array<double, 9>> fbars;
  std::vector<double*> ckpt;
  std::vector<std::array<double, 9>> ckpt_fbar;
};

}  // namespace fg

struct fg_ctx {
  int device = 0;  // CUDA device the context lives on
  int nx = 0, ny = 0, nz = 0, hx = 0;
  int law = FG_NEOHOOKE;
  long long V = 0, VH = 0;
  double h[3] = {0, 0, 0};
  fg_opts o{};
  cudaStream_t st = nullptr;
  std::vector<void*> allocs;
  // FP64 fields
  double *F = nullptr, *Ft = nullptr, *c = nullptr, *ct = nullptr, *d = nullptr, *dt = nullptr;
  double *H = nullptr, *Ht = nullptr, *cdotB = nullptr, *P = nullptr, *GP = nullptr;
  double* gcr = nullptr;   // per-voxel g_c(x) / g_c, null for a uniform toughness
  double* Heff = nullptr;  // H g_c / g_c(x): the history of the phase-field operator (= H)
  double *Fbk = nullptr, *dF = nullptr;  // Newton line search: F before the update, dF
  double *mu = nullptr, *base = nullptr;
  double *lam = nullptr, *mu_ = nullptr, *Om = nullptr, *c0 = nullptr, *D = nullptr, *smax = nullptr;
  double* partials = nullptr;
  long long npartials = 0;
  fg::KScal* ks = nullptr;
  fg::KScal* ks_host = nullptr;
  int* flags = nullptr;
  int* flags_host = nullptr;
  fg::Prec<double> pd;
  fg::Prec<float> pf;
  fg::Prec<fg::ff> pe;  // float-float residual transforms (mixed mode, FP64 fields)
  bool ffres = false;   // the FP64 residual transforms run in float-float
  double Fbar[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  double Fbar_prev[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  double last_dt = 0.0;
  bool stepped = false;
  // launch-site profiling: event pairs around every launch of the enabled sites
  unsigned prof_mask = 0;
  std::vector<cudaEvent_t> prof_ev[8];
  std::vector<double> prof_frac[8];  // share of the full volume each recorded launch covers
  int prof_used[8] = {0};
  int kx_chunk[2] = {1, 1};          // kx planes per Y-Z-Y chunk (FP32, FP64)
  int xi_percomp = 1;                // fused CG update: one component per block
  int l2pf = 0;                      // X passes prefetch their real-space rows into L2
  int zrows = 0;                     // FP32 projection pass: 0 default tile, 1: 1 row, 2: 4 rows
  bool yzy_cluster = false;          // FP32 Y-Z-Y projection chain as one clustered pass
  bool yzy_cluster_chem = false;     // FP32 chemistry Y-Z-Y chains as clustered passes
  double tune_ms[4] = {0, 0, 0, 0};  // autotuner: X-inv update times [prefetch][per comp]
  int last_inner_refine = 0;
  bool strict = false;        // an iteration cap is an error in every mode (adjoint solves)
#ifndef FG_EMU
  // CUDA graphs of 16 fused mechanical CG iterations, [FP32, FP64][without, with the
  // re-projection at the end], and the kernels each holds
  cudaGraphExec_t cg_graph[2][2] = {};
  long long cg_graph_kernels[2][2] = {};
  bool graphs_off = false;
#endif
  int smask = 0;              // mixed control: stress-controlled components (bit 3 i + j)
  double Pbar[9] = {0};       // their prescribed mean first Piola stress
  double* mr[6] = {};         // MINRES work vectors (9 V doubles each), allocated on first use
  fg::Tape* tape = nullptr;   // recorded steps for fg_adjoint
};

namespace fg {

template <typename T>
static T* alloc_n(fg_ctx& c, long long n) {
  void* p = dalloc((size_t)n * sizeof(T));
  c.allocs.push_back(p);
  return (T*)p;
}

static void free_all(fg_ctx& c) {
  for (void* p : c.allocs) dfree(p);
  c.allocs.clear();
  hfree(c.ks_host);
  hfree(c.flags_host);
  c.ks_host = nullptr;
  c.flags_host = nullptr;
}

static bool is_mixed(const fg_ctx& c) { return c.o.precision == FG_MIXED; }

// per-axis frequency tables of one precision (host FP64, then rounded)
template <typename R>
static void build_tables(fg_ctx& c, Prec<R>& P) {
  using C = cplx<R>;
  const int n[3] = {c.nx, c.ny, c.nz};
  const int len[3] = {c.hx, c.ny, c.nz};
  for (int j = 0; j < 3; ++j) {
    std::vector<R> rs(len[j]), rc(len[j]), lap(len[j]);
    std::vector<C> xi(len[j]);
    for (int k = 0; k < len[j]; ++k) {
      const int ks = (j > 0 && 2 * k > n[j]) ? k - n[j] : k;  // signed index
      const double th = M_PI * (double)ks / (double)n[j];
      const double s = sin(th);
      double co = cos(th);
      if (2 * std::abs(ks) == n[j]) co = 0.0;
      rs[k] = (R)(2.0 / c.h[j] * s);
      rc[k] = (R)co;
      lap[k] = (R)(4.0 * s * s / (c.h[j] * c.h[j]));
      const double q = 2.0 * th;
      xi[k] = cmk<C>((R)((cos(q) - 1.0) / c.h[j]), (R)(sin(q) / c.h[j]));
    }
    P.rs[j] = alloc_n<R>(c, len[j]);
    P.rc[j] = alloc_n<R>(c, len[j]);
    P.lap[j] = alloc_n<R>(c, len[j]);
    P.xi[j] = alloc_n<C>(c, len[j]);
    dcopy(P.rs[j], rs.data(), len[j] * sizeof(R), c.st);
    dcopy(P.rc[j], rc.data(), len[j] * sizeof(R), c.st);
    dcopy(P.lap[j], lap.data(), len[j] * sizeof(R), c.st);
    dcopy(P.xi[j], xi.data(), len[j] * sizeof(C), c.st);
  }
  auto tw = [&](int N) {
    std::vector<C> t(N);
    for (int m = 0; m < N; ++m) {
      const double a = 2.0 * M_PI * (double)m / (double)N;
      t[m] = cmk<C>((R)cos(a), (R)(-sin(a)));
    }
    C* d = alloc_n<C>(c, N);
    dcopy(d, t.data(), N * sizeof(C), c.st);
    return d;
  };
  P.twx = tw(c.nx);
  P.twy = tw(c.ny);
  P.twz = tw(c.nz);
  dsync(c.st);
}

template <typename R>
static void setup_prec(fg_ctx& c, Prec<R>& P, int krylov_comps) {
  P.on = true;
  P.ox = size_ops<R>(c.nx);
  P.oy = size_ops<R>(c.ny);
  P.oz = size_ops<R>(c.nz);
  if (!P.ox || !P.oy || !P.oz || !P.ox->xf_tangent)
    fail(FG_ERR_INVALID, "grid size not compiled in (nx, ny, nz)");
  P.S1 = alloc_n<cplx<R>>(c, 9 * c.VH);
  P.S2 = alloc_n<cplx<R>>(c, 9 * c.VH);
  build_tables(c, P);
  const long long n = (long long)krylov_comps * c.V;
  P.x = alloc_n<R>(c, n);
  P.r = alloc_n<R>(c, n);
  P.p = alloc_n<R>(c, n);
  P.q = alloc_n<R>(c, n);
  P.b = alloc_n<R>(c, n);
  P.xbest = alloc_n<R>(c, n);
  P.z = alloc_n<R>(c, c.V);
  P.kc = alloc_n<R>(c, 6 * c.V);
  P.w = alloc_n<R>(c, c.V);
  P.Hr = alloc_n<R>(c, c.V);
  P.tmp3 = alloc_n<R>(c, 3 * c.V);
  if (krylov_comps == 9) P.state = alloc_n<R>(c, (long long)state_size(c.law) * c.V);
}

// The float-float set: its own tables and launchers; the spectra and the FP64 work
// fields it reads and writes are the FP64 set's (16-byte complex numbers in both).
static void setup_ff(fg_ctx& c) {
  Prec<ff>& P = c.pe;
  P.ox = size_ops<ff>(c.nx);
  P.oy = size_ops<ff>(c.ny);
  P.oz = size_ops<ff>(c.nz);
  if (!P.ox || !P.oy || !P.oz || !P.ox->xf_copy9)
    fail(FG_ERR_INVALID, "grid size not compiled in for the float-float residuals");
  static_assert(sizeof(ffc) == sizeof(double2), "float-float and FP64 spectra share buffers");
  P.S1 = (ffc*)c.pd.S1;
  P.S2 = (ffc*)c.pd.S2;
  build_tables(c, P);
  P.tmp3 = c.pd.tmp3;
  P.kc = c.pd.kc;
  P.on = true;
  c.ffres = true;
}

// ------------------------------------------------------------------ launch helpers

static VArgs vbase(fg_ctx& c, long long n) {
  VArgs v{};
  v.n = n;
  v.V = c.V;
  v.partials = c.partials;
  v.flags = c.flags;
  return v;
}

// ------------------------------------------------------------------ launch-site profiling

enum { SITE_XF = 0, SITE_YF = 1, SITE_Z = 2, SITE_YI = 3, SITE_XI = 4, SITE_CGXR = 5, SITE_N = 8 };
static constexpr int PROF_PAIRS = 32768;

struct ProfScope {
  fg_ctx& c;
  int site;
  bool on;
  ProfScope(fg_ctx& cc, int s, double frac = 1.0) : c(cc), site(s), on(false) {
#ifndef FG_EMU
    if ((c.prof_mask >> site) & 1u) {
      auto& v = c.prof_ev[site];
      const int k = c.prof_used[site];
      if (k < PROF_PAIRS) {
        if ((int)v.size() < 2 * (k + 1)) {
          cudaEvent_t a, b;
          cudaEventCreate(&a);
          cudaEventCreate(&b);
          v.push_back(a);
          v.push_back(b);
        }
        if ((int)c.prof_frac[site].size() < k + 1) c.prof_frac[site].push_back(0.0);
        c.prof_frac[site][k] = frac;
        cudaEventRecord(v[2 * k], c.st);
        on = true;
      }
    }
#else
    (void)frac;
#endif
  }
  ~ProfScope() {
#ifndef FG_EMU
    if (on) {
      cudaEventRecord(c.prof_ev[site][2 * c.prof_used[site] + 1], c.st);
      c.prof_used[site] += 1;
    }
#endif
  }
};

template <class F>
static void fin(fg_ctx& c, int slot, long long nparts, const int* done, double s0 = 0, double s1 = 0,
                double s2 = 0) {
  VArgs v = vbase(c, nparts);
  v.ks = c.ks + slot;
  v.done = done;
  v.s[0] = s0;
  v.s[1] = s1;
  v.s[2] = s2;
  launch_fin<F>(v, c.st);
}

static void read_ks(fg_ctx& c) {
  dcopy(c.ks_host, c.ks, KS_N * sizeof(KScal), c.st);
  dcopy(c.flags_host, c.flags, sizeof(int), c.st);
  dsync(c.st);
}

static double reduce_sum(fg_ctx& c, const double* x, long long n, bool sq) {
  VArgs v = vbase(c, n);
  v.in[0] = x;
  if (sq) launch_vec<KSumSq>(v, c.st);
  else launch_vec<KSum>(v, c.st);
  fin<FStore>(c, KS_MISC, VEC_BLOCKS, nullptr);
  read_ks(c);
  return c.ks_host[KS_MISC].aux;
}

// |x|^2 of a vector of precision R
template <typename R>
static double reduce_sum_r(fg_ctx& c, const R* x, long long n) {
  VArgs v = vbase(c, n);
  v.in[0] = x;
  launch_vec<KSumSqR<R>>(v, c.st);
  fin<FStore>(c, KS_MISC, VEC_BLOCKS, nullptr);
  read_ks(c);
  return c.ks_host[KS_MISC].aux;
}

template <typename R>
static PassArgs<R> pbase(fg_ctx& c, Prec<R>& P, const int* done) {
  PassArgs<R> a{};
  a.nx = c.nx;
  a.ny = c.ny;
  a.nz = c.nz;
  a.hx = c.hx;
  a.V = c.V;
  a.VH = c.VH;
  for (int j = 0; j < 3; ++j) {
    a.rs[j] = P.rs[j];
    a.rc[j] = P.rc[j];
    a.xi[j] = P.xi[j];
    a.lap[j] = P.lap[j];
  }
  a.partials = c.partials;
  a.done = done;
  a.l2pf = c.l2pf;
  return a;
}

// Y-fwd, Z op, Y-inv on the spectrum in S1 (ncomp_in comps) -> S1 (ncomp_out comps)
// Y-fwd, Z op, Y-inv on the spectrum in S1 (cin comps) -> S1 (cout comps).  The three
// passes run on chunks of consecutive kx planes sized to stay in L2 between them, so the
// intermediate spectrum S2 of a chunk is written and read back from L2 instead of HBM.
// `sites` (or null) names the profiling sites of the three passes.
template <typename R>
static void yzy(fg_ctx& c, Prec<R>& P, const int* done, int cin, PassFn<R> zop, int cout,
                const R* zcoef, const double* dscal, const int* sites = nullptr) {
  const int chunk = c.kx_chunk[sizeof(R) == 8 ? 1 : 0];
  for (int k0 = 0; k0 < c.hx; k0 += chunk) {
    const int k1 = k0 + chunk < c.hx ? k0 + chunk : c.hx;
    const double frac = (double)(k1 - k0) / (double)c.hx;
    PassArgs<R> a = pbase(c, P, done);
    a.tw = P.twy;
    a.cin = P.S1;
    a.cout = P.S2;
    a.ncomp = cin;
    a.row_lo = k0 * c.nz;
    a.row_hi = k1 * c.nz;
    {
      ProfScope ps(c, sites ? sites[0] : SITE_N - 1, frac);
      P.oy->yf(a, c.st);
    }
    a = pbase(c, P, done);
    a.tw = P.twz;
    a.cin = P.S2;
    a.cout = P.S2;
    for (int k = 0; k < 4; ++k) a.coef[k] = zcoef[k];
    a.dscal = dscal;
    a.row_lo = k0 * c.ny;
    a.row_hi = k1 * c.ny;
    {
      ProfScope ps(c, sites ? sites[1] : SITE_N - 1, frac);
      zop(a, c.st);
    }
    a = pbase(c, P, done);
    a.tw = P.twy;
    a.cin = P.S2;
    a.cout = P.S1;
    a.ncomp = cout;
    a.row_lo = k0 * c.nz;
    a.row_hi = k1 * c.nz;
    {
      ProfScope ps(c, sites ? sites[2] : SITE_N - 1, frac);
      P.oy->yi(a, c.st);
    }
  }
}

// Y-fwd, projection and Y-inv of a nine-component spectrum in S1: one clustered pass when
// the context uses it (FP32, ny = nz of 128 or 256), else the three passes
template <typename R>
static void yzy_proj(fg_ctx& c, Prec<R>& P, const int* done, const R* zc, const int* sites);
template <typename R>
static void yzy_chem(fg_ctx& c, Prec<R>& P, const int* done, bool grad, const R* zc);

// the projection pass of the context's tile shape (the autotuner's choice, FP32 only)
template <typename R>
static PassFn<R> zproj(const fg_ctx& c, const Prec<R>& P) {
  if (c.zrows > 0 && P.oz->z_proj_rows[c.zrows - 1]) return P.oz->z_proj_rows[c.zrows - 1];
  return P.oz->z_proj;
}

// the chemistry's Y-Z-Y chains (1 -> 3 gradient, 3 -> 1 divergence on S1): clustered
// passes when the context uses them, else the three passes
template <typename R>
static void yzy_chem(fg_ctx& c, Prec<R>& P, const int* done, bool grad, const R* zc) {
  if constexpr (std::is_same<R, float>::value) {
    if (c.yzy_cluster_chem) {
      PassArgs<R> a = pbase(c, P, done);
      a.tw = P.twz;
      a.cin = P.S1;
      a.cout = P.S1;
      for (int k = 0; k < 4; ++k) a.coef[k] = zc[k];
      (grad ? P.oz->yzy_grad : P.oz->yzy_div)(a, c.st);
      return;
    }
  }
  if (grad) yzy(c, P, done, 1, P.oz->z_grad, 3, zc, nullptr);
  else yzy(c, P, done, 3, P.oz->z_div, 1, zc, nullptr);
}

template <typename R>
static void yzy_proj(fg_ctx& c, Prec<R>& P, const int* done, const R* zc, const int* sites) {
  if constexpr (std::is_same<R, float>::value) {
    if (c.yzy_cluster && P.oz->yzy_proj) {
      PassArgs<R> a = pbase(c, P, done);
      a.tw = P.twz;
      a.cin = P.S1;
      a.cout = P.S1;
      for (int k = 0; k < 4; ++k) a.coef[k] = zc[k];
      ProfScope ps(c, sites ? sites[1] : SITE_N - 1, 1.0);
      P.oz->yzy_proj(a, c.st);
      return;
    }
  }
  yzy(c, P, done, 9, zproj(c, P), 9, zc, nullptr, sites);
}

// y = G : F^-1[ F[K : x] ] ; accumulates <x, y>; returns partial count
template <typename R>
static int op_mech(fg_ctx& c, Prec<R>& P, const R* x, R* y, const int* done) {
  PassArgs<R> a = pbase(c, P, done);
  a.tw = P.twx;
  a.rin = x;
  a.aux[0] = P.state;
  a.cout = P.S1;
  {
    ProfScope ps(c, SITE_XF);
    (c.law == FG_SVK ? P.ox->xf_tangent_svk : P.ox->xf_tangent)(a, c.st);
  }
  const R zc[4] = {(R)(1.0 / (double)c.V), (R)c.smask, 0, 0};
  static const int sites[3] = {SITE_YF, SITE_Z, SITE_YI};
  yzy_proj(c, P, done, zc, sites);
  a = pbase(c, P, done);
  a.tw = P.twx;
  a.cin = P.S1;
  a.rout = y;
  a.aux[0] = x;
  ProfScope ps(c, SITE_XI);
  return P.ox->xi_storedot9(a, c.st);
}

// y = G * x (projection of a tensor field), accumulates |y|^2
template <typename R>
static int op_gres(fg_ctx& c, Prec<R>& P, const io_t<R>* x, io_t<R>* y, const int* done) {
  PassArgs<R> a = pbase(c, P, done);
  a.tw = P.twx;
  a.rin = x;
  a.cout = P.S1;
  P.ox->xf_copy9(a, c.st);
  const R zc[4] = {(R)(1.0 / (double)c.V), (R)c.smask, 0, 0};
  yzy_proj(c, P, done, zc, (const int*)nullptr);
  a = pbase(c, P, done);
  a.tw = P.twx;
  a.cin = P.S1;
  a.rout = y;
  return P.ox->xi_norm9(a, c.st);
}

// y = [g_c/l_c + 2H] x + F^-1{ g_c l_c |xi|^2 x^ } ; accumulates <x, y>
template <typename R>
static int op_pff(fg_ctx& c, Prec<R>& P, const R* x, R* y, const R* H, const int* done) {
  PassArgs<R> a = pbase(c, P, done);
  a.tw = P.twx;
  a.rin = x;
  a.cout = P.S1;
  P.ox->xf_copy1(a, c.st);
  const R zc[4] = {(R)(c.o.gc * c.o.lc / (double)c.V), 0, 0, 0};
  yzy(c, P, done, 1, P.oz->z_lap, 1, zc, nullptr);
  a = pbase(c, P, done);
  a.tw = P.twx;
  a.cin = P.S1;
  a.rout = y;
  a.aux[0] = x;
  a.aux[1] = H;
  a.coef[0] = (R)(c.o.gc / c.o.lc);
  return P.ox->xi_pff(a, c.st);
}

// z = F^-1{ r^ / (g_c/l_c + 2 Hbar + g_c l_c |xi|^2) } ; accumulates <r, z>
template <typename R>
static int op_prec(fg_ctx& c, Prec<R>& P, const R* r, R* z, const int* done) {
  PassArgs<R> a = pbase(c, P, done);
  a.tw = P.twx;
  a.rin = r;
  a.cout = P.S1;
  P.ox->xf_copy1(a, c.st);
  const R zc[4] = {(R)(1.0 / (double)c.V), (R)(c.o.gc / c.o.lc), (R)(c.o.gc * c.o.lc), 0};
  yzy(c, P, done, 1, P.oz->z_prec, 1, zc, &c.ks[KS_HBAR].aux);
  a = pbase(c, P, done);
  a.tw = P.twx;
  a.cin = P.S1;
  a.rout = z;
  a.aux[0] = r;
  return P.ox->xi_storedot1(a, c.st);
}

// L u = grad_f^H (K_c grad_f u) into S1 (1 comp), K_c from P.kc
template <typename R>
static void op_chem_L(fg_ctx& c, Prec<R>& P, const io_t<R>* u, const int* done) {
  PassArgs<R> a = pbase(c, P, done);
  a.tw = P.twx;
  a.rin = u;
  a.cout = P.S1;
  P.ox->xf_copy1(a, c.st);
  const R zc[4] = {(R)(1.0 / (double)c.V), 0, 0, 0};
  yzy_chem(c, P, done, true, zc);
  a = pbase(c, P, done);
  a.tw = P.twx;
  a.cin = P.S1;
  a.rout = P.tmp3;
  a.aux[0] = P.kc;
  P.ox->xi_chemflux(a, c.st);
  a = pbase(c, P, done);
  a.tw = P.twx;
  a.rin = P.tmp3;
  a.cout = P.S1;
  P.ox->xf_copy3(a, c.st);
  yzy_chem(c, P, done, false, zc);
}

// y = x c(1-c) + dt L x ; accumulates <x, y>
template <typename R>
static int op_chem(fg_ctx& c, Prec<R>& P, const R* x, R* y, double dt, const int* done) {
  op_chem_L(c, P, x, done);
  PassArgs<R> a = pbase(c, P, done);
  a.tw = P.twx;
  a.cin = P.S1;
  a.rout = y;
  a.aux[0] = x;
  a.aux[1] = P.w;
  a.coef[0] = (R)dt;
  return P.ox->xi_chemop(a, c.st);
}

// b = -(base + dt L mu) into an FP64 field, transforms in FP64 or float-float ; returns
// |b|^2 partial count
template <typename R>
static int op_chem_rhs_p(fg_ctx& c, Prec<R>& P, double* b, double dt) {
  op_chem_L(c, P, c.mu, nullptr);
  PassArgs<R> a = pbase(c, P, nullptr);
  a.tw = P.twx;
  a.cin = P.S1;
  a.rout = b;
  a.aux[0] = c.base;
  a.coef[0] = (R)dt;
  return P.ox->xi_chemrhs(a, c.st);
}
static int op_chem_rhs(fg_ctx& c, double* b, double dt) {
  return c.ffres ? op_chem_rhs_p(c, c.pe, b, dt) : op_chem_rhs_p(c, c.pd, b, dt);
}

// y = G * x of FP64 fields with |y|^2 partial sums: the residual projection, in float-float
// transforms when the context runs them, else in FP64
static int gres64(fg_ctx& c, const double* x, double* y) {
  return c.ffres ? op_gres(c, c.pe, x, y, nullptr) : op_gres(c, c.pd, x, y, nullptr);
}

// ------------------------------------------------------------------ state kernels

template <typename R>
static void mech_state(fg_ctx& c, const double* F, const double* Fbar, double* Pout, R* state) {
  VArgs v = vbase(c, c.V);
  v.in[0] = F;
  if (!F)
    for (int k = 0; k < 9; ++k) v.s[k] = Fbar[k];
  v.in[1] = c.c;
  v.in[2] = c.d;
  v.in[3] = c.lam;
  v.in[4] = c.mu_;
  v.in[5] = c.Om;
  v.in[6] = c.c0;
  v.out[0] = Pout;
  v.out[1] = state;
  if (c.law == FG_SVK) launch_vec<KMechState<R, LAW_SVK_>>(v, c.st);
  else launch_vec<KMechState<R, LAW_NH_>>(v, c.st);
}

template <typename R>
static void to_prec(fg_ctx& c, const double* x, R* y, long long n, double s) {
  VArgs v = vbase(c, n);
  v.in[0] = x;
  v.out[0] = y;
  v.s[0] = s;
  launch_vec<KScaleTo<R>>(v, c.st);
}

static void check_flags(fg_ctx& c, const char* where) {
  if (*c.flags_host & ST_DOMAIN) {
    dzero(c.flags, sizeof(int), c.st);
    fail(FG_ERR_DOMAIN, std::string(where) + ": c left (0,1) or det F <= 0");
  }
  if (*c.flags_host & ST_NUMERIC) {
    dzero(c.flags, sizeof(int), c.st);
    fail(FG_ERR_NUMERIC, std::string(where) + ": non-finite value");
  }
}

// ------------------------------------------------------------------ Krylov drivers

// x_best = x when the last finaliser flagged a 4x drop of |r|^2 (kernel skipped otherwise)
template <typename R>
static void snap_iterate(fg_ctx& c, Prec<R>& P, long long n, KScal* ks) {
  VArgs v = vbase(c, n);
  v.done = &ks->nosnap;
  v.in[0] = P.x;
  v.out[0] = P.xbest;
  launch_vec<KCopy<R>>(v, c.st);
}

// a solve that stopped early (non-positive curvature or the iteration cap) returns the
// saved iterate when its own residual is larger: in an indefinite system CG residuals can
// grow long before a direction of negative curvature shows up
template <typename R>
static void keep_best(fg_ctx& c, Prec<R>& P, long long n, const KScal& k) {
  if (k.rr > k.rr_best) dcopy(P.x, P.xbest, n * sizeof(R), c.st);
}

// Conjugate gradients on P.b (n elements) from x = 0; result in P.x.  apply(p, q, done)
// computes q = A p and the partial sums of <p, q>, returning their count.
// Early stops and directions of negative curvature are counted into st (may be null).
template <typename R, class Apply>
static int cg_solve(fg_ctx& c, Prec<R>& P, long long n, int slot, double tol, int maxit, Apply apply,
                    fg_stats* st = nullptr) {
  int* truncated = st ? &st->cg_truncated : nullptr;
  KScal* ks = c.ks + slot;
  VArgs v = vbase(c, n);
  v.in[0] = P.b;
  v.out[0] = P.x;
  v.out[1] = P.r;
  v.out[2] = P.p;
  launch_vec<KCgInit<R>>(v, c.st);
  fin<FCgStart>(c, slot, VEC_BLOCKS, nullptr, tol, (double)maxit, (double)(c.o.cg_indefinite == 1));
  const int* done = &ks->done;
  int chunk = 4;
  while (true) {
    for (int j = 0; j < chunk; ++j) {
      const int nb = apply(P.p, P.q, done);
      fin<FAlpha>(c, slot, nb, done);
      VArgs u = vbase(c, n);
      u.ks = ks;
      u.done = done;
      u.in[0] = P.p;
      u.in[1] = P.q;
      u.out[0] = P.x;
      u.out[1] = P.r;
      {
        ProfScope ps(c, slot == KS_MECH ? SITE_CGXR : SITE_N - 1);
        launch_vec<KCgXR<R>>(u, c.st);
      }
      fin<FBetaCg>(c, slot, VEC_BLOCKS, done);
      snap_iterate(c, P, n, ks);
      VArgs w = vbase(c, n);
      w.ks = ks;
      w.done = done;
      w.in[0] = P.r;
      w.out[0] = P.p;
      launch_vec<KCgP<R>>(w, c.st);
    }
    read_ks(c);
    if (c.ks_host[slot].done) break;
    if (chunk < 16) chunk *= 2;
  }
  const KScal& k = c.ks_host[slot];
  if (st) st->cg_negcurv += k.negc;
  if (k.status & ST_NUMERIC) fail(FG_ERR_NUMERIC, "Krylov solve produced a non-finite value");
  if (k.status & ST_INDEFINITE) {
    // truncated CG: the iterate before the first direction of non-positive curvature, or
    // the saved best-residual iterate; with no iterate yet there is nothing to return
    if (k.iters == 0) fail(FG_ERR_NUMERIC, "Krylov operator not positive along the residual");
    keep_best(c, P, n, k);
    if (truncated) *truncated += 1;
    return k.iters;
  }
  if (k.rr > k.tol2 && k.iters >= maxit) {
    // an FP32 inner solve of the mixed mode is an inexact Newton step: its iterate is kept
    // and the FP64 outer residual decides; in FP64 mode the cap is an error
    if (!is_mixed(c) || c.strict) fail(FG_ERR_NOCONV, "Krylov solve hit max_cg");
    keep_best(c, P, n, k);
    if (truncated) *truncated += 1;
  }
  return k.iters;
}

// Chemistry CG (the linear solve of Alg. 3, operator y/m + dt L y) on P.b from x = 0 with
// the vector updates fused into the operator passes: the forward X pass forms
// p = r + beta p and <p, w p>, the flux round trip (inverse X, K_c g, forward X) adds
// dt <g, K_c g>, so alpha is known before the inverse transform, whose epilogue forms
// q = w p + dt L p and applies r -= alpha q, x += alpha p with the sums of r^2.  Per
// iteration: three X passes, two Y-Z-Y chains and two single-block finalisers; q and the
// real-space flux are never stored.
template <typename R>
static int cg_solve_chem(fg_ctx& c, Prec<R>& P, double dt, double tol, int maxit, fg_stats* st) {
  int* truncated = st ? &st->cg_truncated : nullptr;
  const long long n = c.V;
  const int slot = KS_CHEM;
  KScal* ks = c.ks + slot;
  VArgs v = vbase(c, n);
  v.in[0] = P.b;
  v.out[0] = P.x;
  v.out[1] = P.r;
  v.out[2] = P.p;
  launch_vec<KCgInit<R>>(v, c.st);
  fin<FCgStart>(c, slot, VEC_BLOCKS, nullptr, tol, (double)maxit, (double)(c.o.cg_indefinite == 1));
  const int* done = &ks->done;
  const double* sc = &ks->alpha;  // sc[0] = alpha, sc[1] = beta
  const R zc[4] = {(R)(1.0 / (double)c.V), 0, 0, 0};
  auto iteration = [&]() {
    PassArgs<R> a = pbase(c, P, done);
    a.tw = P.twx;
    a.rin = P.r;
    a.rout = P.p;
    a.aux[0] = P.w;
    a.dscal = sc;
    a.cout = P.S1;
    const int nb1 = P.ox->xf_cgchem(a, c.st);
    yzy_chem(c, P, done, true, zc);
    a = pbase(c, P, done);
    a.tw = P.twx;
    a.cin = P.S1;
    a.cout = P.S1;
    a.aux[0] = P.kc;
    a.coef[0] = (R)dt;
    a.partials = c.partials + nb1;  // after the forward pass's partial sums
    const int nb2 = P.ox->xr_chemflux(a, c.st);
    fin<FAlpha>(c, slot, nb1 + nb2, done);
    yzy_chem(c, P, done, false, zc);
    a = pbase(c, P, done);
    a.tw = P.twx;
    a.cin = P.S1;
    a.rout = P.r;
    a.rout2 = P.x;
    a.aux[0] = P.p;
    a.aux[1] = P.w;
    a.coef[0] = (R)dt;
    a.dscal = sc;
    const int nb = P.ox->xi_cgchem(a, c.st);
    fin<FBetaCg>(c, slot, nb, done);
    snap_iterate(c, P, n, ks);
  };
  int chunk = 4;
  while (true) {
    for (int j = 0; j < chunk; ++j) iteration();
    read_ks(c);
    if (c.ks_host[slot].done) break;
    if (chunk < 16) chunk *= 2;
  }
  const KScal& k = c.ks_host[slot];
  if (st) st->cg_negcurv += k.negc;
  if (k.status & ST_NUMERIC) fail(FG_ERR_NUMERIC, "Krylov solve produced a non-finite value");
  if (k.status & ST_INDEFINITE) {
    if (k.iters == 0) fail(FG_ERR_NUMERIC, "Krylov operator not positive along the residual");
    keep_best(c, P, n, k);
    if (truncated) *truncated += 1;
    return k.iters;
  }
  if (k.rr > k.tol2 && k.iters >= maxit) {
    if (!is_mixed(c) || c.strict) fail(FG_ERR_NOCONV, "Krylov solve hit max_cg");
    keep_best(c, P, n, k);
    if (truncated) *truncated += 1;
  }
  return k.iters;
}

// Mechanical CG (Alg. 1) on P.b from x = 0 with the vector updates fused into the
// operator passes: X-fwd forms p = r + beta p and <p, K p>, X-inv applies r -= alpha q,
// x += alpha p and sums |r|^2.  Per iteration: 5 passes + 2 single-block finalisers.
// sigma shifts the system to G K G + sigma I.  With negcurv != null a direction of negative
// curvature ends the solve without keeping an iterate: *negcurv is set and the caller
// re-solves (the shifted Newton of mech_newton); P.p then holds that direction.  indef
// overrides the option's treatment of negative curvature (1: take it, 0: stop; -1: option).
template <typename R>
static int cg_solve_mech(fg_ctx& c, Prec<R>& P, double tol, int maxit, fg_stats* st, double sigma = 0.0,
                         bool* negcurv = nullptr, int indef = -1) {
  int* truncated = st ? &st->cg_truncated : nullptr;
  const long long n = 9 * c.V;
  const int slot = KS_MECH;
  KScal* ks = c.ks + slot;
  VArgs v = vbase(c, n);
  v.in[0] = P.b;
  v.out[0] = P.x;
  v.out[1] = P.r;
  v.out[2] = P.p;
  launch_vec<KCgInit<R>>(v, c.st);
  fin<FCgStart>(c, slot, VEC_BLOCKS, nullptr, tol, (double)maxit,
                (double)(indef >= 0 ? indef : c.o.cg_indefinite == 1));
  const int* done = &ks->done;
  const double* sc = &ks->alpha;  // sc[0] = alpha, sc[1] = beta
  const R zc[4] = {(R)(1.0 / (double)c.V), (R)c.smask, 0, 0};
  long long launched = 0;
  // one fused iteration; the re-projection every 32 iterations
  auto iteration = [&]() {
    PassArgs<R> a = pbase(c, P, done);
    a.tw = P.twx;
    a.rin = P.r;
    a.rout = P.p;
    a.aux[0] = P.state;
    a.dscal = sc;
    a.coef[1] = (R)sigma;
    a.cout = P.S1;
    int nb;
    {
      ProfScope ps(c, SITE_XF);
      nb = (c.law == FG_SVK ? P.ox->xf_cgtangent_svk : P.ox->xf_cgtangent)(a, c.st);
    }
    fin<FAlpha>(c, slot, nb, done);
    {
      static const int sites[3] = {SITE_YF, SITE_Z, SITE_YI};
      yzy_proj(c, P, done, zc, sites);
    }
    a = pbase(c, P, done);
    a.tw = P.twx;
    a.cin = P.S1;
    a.rout = P.r;
    a.rout2 = P.x;
    a.aux[0] = P.p;
    a.dscal = sc;
    a.coef[1] = (R)sigma;
    {
      ProfScope ps(c, SITE_XI);
      nb = (c.xi_percomp ? P.ox->xi_cgupdate_pc : P.ox->xi_cgupdate)(a, c.st);
    }
    fin<FBetaCg>(c, slot, nb, done);
    snap_iterate(c, P, n, ks);
    if (++launched % 32 == 0) {
      // every CG vector is compatible in exact arithmetic; re-project r and p so that
      // roundoff in modes G does not see cannot build up and corrupt <p, K p>
      nb = op_gres(c, P, P.r, P.r, done);
      fin<FSetResidual>(c, slot, nb, done);
      op_gres(c, P, P.p, P.p, done);
    }
  };
  // chunks of 4, 12, then 16 iterations between host checks (iterations after convergence
  // exit at once on the device flag): from the third chunk on every chunk starts at a
  // multiple of 16 and either ends with the re-projection or has none, so it is replayed
  // from one of two CUDA graphs on streams that can be captured
  while (true) {
    const int cnt = launched == 0 ? 4 : (launched == 4 ? 12 : 16);
    bool ran = false;
#ifndef FG_EMU
    // graphs from iteration 32 on: every kernel of a chunk, the re-projection included, has
    // run once directly before it is captured
    if (cnt == 16 && launched >= 32 && sigma == 0.0 && !c.prof_mask && !c.graphs_off &&
        c.st != nullptr) {
      const int pi = sizeof(R) == 8 ? 1 : 0, var = (launched + 16) % 32 == 0 ? 1 : 0;
      cudaGraphExec_t& ex = c.cg_graph[pi][var];
      if (!ex) {  // capture once per context (the kernels read every scalar from the device)
        const long long k0 = launch_counter().load();
        const long long l0 = launched;
        cudaGraph_t g = nullptr;
        bool ok = cudaStreamBeginCapture(c.st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
          for (int j = 0; j < cnt; ++j) iteration();
          ok = cudaStreamEndCapture(c.st, &g) == cudaSuccess && g != nullptr;
        }
        launched = l0;                                   // captured, nothing ran
        const long long captured = launch_counter().load() - k0;
        launch_counter() -= captured;
        if (ok) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
        if (ok) {
          c.cg_graph_kernels[pi][var] = captured;
        } else {  // not capturable here: direct launches from now on
          ex = nullptr;
          c.graphs_off = true;
          cudaGetLastError();
        }
      }
      if (ex) {
        if (cudaGraphLaunch(ex, c.st) == cudaSuccess) {
          launch_counter() += c.cg_graph_kernels[pi][var];
          launched += cnt;
          ran = true;
          if (st) st->cg_graph_replays += 1;
        } else {
          c.graphs_off = true;
          cudaGetLastError();
        }
      }
    }
#endif
    if (!ran)
      for (int j = 0; j < cnt; ++j) iteration();
    read_ks(c);
    if (c.ks_host[slot].done) break;
  }
  const KScal& k = c.ks_host[slot];
  if (st) st->cg_negcurv += k.negc;
  if (k.status & ST_NUMERIC) fail(FG_ERR_NUMERIC, "Krylov solve produced a non-finite value");
  if (k.status & ST_INDEFINITE) {
    if (negcurv) {
      *negcurv = true;
      return k.iters;
    }
    if (k.iters == 0) fail(FG_ERR_NUMERIC, "Krylov operator not positive along the residual");
    keep_best(c, P, n, k);
    if (truncated) *truncated += 1;
    return k.iters;
  }
  if (k.rr > k.tol2 && k.iters >= maxit) {
    if (!is_mixed(c) || c.strict) fail(FG_ERR_NOCONV, "mechanical CG hit max_cg");
    keep_best(c, P, n, k);
    if (truncated) *truncated += 1;  // mixed mode: inexact Newton step, see cg_solve
  }
  return k.iters;
}

// Preconditioned CG for the phase field (Alg. 2) on P.b from x0 = P.x (V elements).
template <typename R>
static int pcg_pff(fg_ctx& c, Prec<R>& P, const R* H, double tol, int maxit) {
  const long long n = c.V;
  const int slot = KS_PFF;
  KScal* ks = c.ks + slot;
  // bb
  {
    VArgs v = vbase(c, n);
    v.in[0] = P.b;
    launch_vec<KSumSqR<R>>(v, c.st);
    fin<FStore>(c, slot, VEC_BLOCKS, nullptr);
  }
  read_ks(c);
  const double bb = c.ks_host[slot].aux;
  // r = b - A x0
  op_pff(c, P, P.x, P.q, H, nullptr);
  {
    VArgs v = vbase(c, n);
    v.in[0] = P.b;
    v.in[1] = P.q;
    v.out[0] = P.r;
    launch_vec<KResid<R>>(v, c.st);
    fin<FPcgStart>(c, slot, VEC_BLOCKS, nullptr, tol, bb, (double)maxit);
  }
  const int* done = &ks->done;
  {
    const int nb = op_prec(c, P, P.r, P.z, done);
    fin<FPcgRz>(c, slot, nb, done);
    VArgs v = vbase(c, n);
    v.done = done;
    v.in[0] = P.z;
    v.out[0] = P.p;
    launch_vec<KCopy<R>>(v, c.st);
  }
  int chunk = 4;
  while (true) {
    for (int j = 0; j < chunk; ++j) {
      int nb = op_pff(c, P, P.p, P.q, H, done);
      fin<FAlpha>(c, slot, nb, done);
      VArgs u = vbase(c, n);
      u.ks = ks;
      u.done = done;
      u.in[0] = P.p;
      u.in[1] = P.q;
      u.out[0] = P.x;
      u.out[1] = P.r;
      launch_vec<KCgXR<R>>(u, c.st);
      fin<FResPcg>(c, slot, VEC_BLOCKS, done);
      nb = op_prec(c, P, P.r, P.z, done);
      fin<FBetaPcg>(c, slot, nb, done);
      VArgs w = vbase(c, n);
      w.ks = ks;
      w.done = done;
      w.in[0] = P.z;
      w.out[0] = P.p;
      launch_vec<KCgP<R>>(w, c.st);
    }
    read_ks(c);
    if (c.ks_host[slot].done) break;
    if (chunk < 16) chunk *= 2;
  }
  const KScal& k = c.ks_host[slot];
  if (k.status & ST_NUMERIC) fail(FG_ERR_NUMERIC, "phase-field solve produced a non-finite value");
  if (k.status & ST_INDEFINITE) fail(FG_ERR_NUMERIC, "phase-field operator not positive definite");
  if (k.rr > k.tol2 && k.iters >= maxit && (!is_mixed(c) || c.strict))
    fail(FG_ERR_NOCONV, "phase-field PCG hit max_cg");
  return k.iters;
}

// ------------------------------------------------------------------ solves

static double mixed_tol(const fg_ctx& c, double tol) {
  return is_mixed(c) ? std::max(tol, c.o.cg_forcing) : tol;
}

// ||G*P(Fbar)|| with the fallbacks ||P(Fbar)||, then 1
// |G P - M P-bar*|^2 into c.GP from c.P: the equilibrium residual; under mixed control
// G keeps the mean of the stress-controlled components M and their prescribed mean
// stress P-bar* is subtracted
static double gres_residual(fg_ctx& c) {
  const int nb = gres64(c, c.P, c.GP);
  if (!c.smask) {
    fin<FStore>(c, KS_MISC, nb, nullptr);
    read_ks(c);
    return c.ks_host[KS_MISC].aux;
  }
  VArgs v = vbase(c, 9 * c.V);
  v.in[0] = c.GP;
  v.out[0] = c.GP;
  for (int k = 0; k < 9; ++k) v.s[k] = ((c.smask >> k) & 1) ? -c.Pbar[k] : 0.0;
  launch_vec<KShiftF>(v, c.st);
  return reduce_sum(c, c.GP, 9 * c.V, true);
}

static double residual_den(fg_ctx& c) {
  mech_state<double>(c, nullptr, c.Fbar, c.P, nullptr);
  const double g2 = gres_residual(c);
  check_flags(c, "residual");
  const double g = sqrt(g2);
  const double p = sqrt(reduce_sum(c, c.P, 9 * c.V, true));
  double den = g;
  if (den <= 1e-12 * p) den = p;
  if (den == 0.0) den = 1.0;
  return den;
}

// err_res of the current (F, c, d); leaves G*P in c.GP and the tangent state of
// precision R in P.state when state != null
template <typename R>
static double residual_mech(fg_ctx& c, double den, R* state) {
  mech_state<R>(c, c.F, nullptr, c.P, state);
  const double g2 = gres_residual(c);
  check_flags(c, "residual");
  return sqrt(g2) / den;
}

static double dotd(fg_ctx& c, const double* x, const double* y, long long n) {
  VArgs v = vbase(c, n);
  v.in[0] = x;
  v.in[1] = y;
  launch_vec<KDot>(v, c.st);
  fin<FStore>(c, KS_MISC, VEC_BLOCKS, nullptr);
  read_ks(c);
  return c.ks_host[KS_MISC].aux;
}

static void lin3(fg_ctx& c, double* out, long long n, double s0, const double* x0, double s1 = 0.0,
                 const double* x1 = nullptr, double s2 = 0.0, const double* x2 = nullptr) {
  VArgs v = vbase(c, n);
  v.in[0] = x0;
  v.in[1] = x1;
  v.in[2] = x2;
  v.out[0] = out;
  v.s[0] = s0;
  v.s[1] = s1;
  v.s[2] = s2;
  launch_vec<KLin3>(v, c.st);
}

// MINRES (Paige and Saunders, SIAM J. Numer. Anal. 12 (1975) 617) on the FP64 Newton
// system G K G dF = b, b = c.pd.b, from dF = 0 into c.pd.x.  Lanczos: A v_k = b_k v_{k-1} +
// a_k v_k + b_{k+1} v_{k+1} (b_1 = 0 in column 1); column k of the tridiagonal matrix is
// rotated by the Givens rotations G_{k-2}, G_{k-1} into (e_k, d_k, gbar_k), and G_k =
// (gbar_k, b_{k+1}) / gamma_k removes b_{k+1}; the rotated right-hand side gives
// phi_k = c phibar_{k-1}, phibar_k = -s phibar_{k-1}, |phibar_k| = |b - A x_k| (monotone),
// and x_k = x_{k-1} + phi_k w_k, w_k = (v_k - d_k w_{k-1} - e_k w_{k-2}) / gamma_k.  It is
// the fallback of the mechanical Newton where CG directions fail (a state whose tangent
// has negative eigenvalues).  Stops at |r| <= tol |b| or at maxit, where it keeps its
// iterate in both modes as the oracle's MINRES does (the Newton loop's own test on err_res
// then decides; an error only when strict).  Returns the iterations.
static int minres_mech(fg_ctx& c, double tol, int maxit) {
  Prec<double>& D = c.pd;
  const long long n = 9 * c.V;
  for (auto& p : c.mr)
    if (!p) p = alloc_n<double>(c, n);
  double *vp = c.mr[0], *v = c.mr[1], *u = c.mr[2], *w1 = c.mr[3], *w2 = c.mr[4], *w = c.mr[5];
  dzero(D.x, n * sizeof(double), c.st);
  dzero(vp, n * sizeof(double), c.st);
  dzero(w1, n * sizeof(double), c.st);
  dzero(w2, n * sizeof(double), c.st);
  const double beta1 = sqrt(dotd(c, D.b, D.b, n));
  if (beta1 == 0.0) return 0;
  lin3(c, v, n, 1.0 / beta1, D.b);
  double beta = 0.0, phibar = beta1, c1 = 1.0, s1 = 0.0, c2 = 1.0, s2 = 0.0;
  int it = 0;
  while (fabs(phibar) > tol * beta1) {
    if (it >= maxit) {
      if (c.strict) fail(FG_ERR_NOCONV, "mechanical MINRES hit max_cg");
      break;
    }
    ++it;
    op_mech(c, D, v, u, nullptr);  // u = A v_k
    const double alpha = dotd(c, v, u, n);
    lin3(c, u, n, 1.0, u, -alpha, v, -beta, vp);  // u = b_{k+1} v_{k+1}
    const double beta_next = sqrt(dotd(c, u, u, n));
    const double e = s2 * beta, t = c2 * beta;
    const double d = c1 * t + s1 * alpha;
    const double gbar = -s1 * t + c1 * alpha;
    const double gamma = hypot(gbar, beta_next);
    const double cr = gamma > 0.0 ? gbar / gamma : 1.0, sr = gamma > 0.0 ? beta_next / gamma : 0.0;
    const double phi = cr * phibar;
    phibar = -sr * phibar;
    if (!(gamma > 0.0) || !(phibar == phibar)) fail(FG_ERR_NUMERIC, "mechanical MINRES broke down");
    lin3(c, w, n, 1.0 / gamma, v, -d / gamma, w1, -e / gamma, w2);
    lin3(c, D.x, n, 1.0, D.x, phi, w);
    double* t3 = w2;  // w_{k-2} <- w_{k-1} <- w_k
    w2 = w1;
    w1 = w;
    w = t3;
    c2 = c1;
    s2 = s1;
    c1 = cr;
    s1 = sr;
    if (beta_next == 0.0) break;  // invariant subspace: x is exact
    double* t2 = vp;              // v_{k-1} <- v_k, v_{k+1} = u / b_{k+1}
    vp = v;
    v = t2;
    lin3(c, v, n, 1.0 / beta_next, u);
    beta = beta_next;
  }
  c.mr[0] = vp;
  c.mr[1] = v;
  c.mr[3] = w1;
  c.mr[4] = w2;
  c.mr[5] = w;
  return it;
}

// Newton correction of Alg. 1 in precision X: CG on (G K G + sigma I) dF = -G P from the
// tangent state in PX.state.  With cg_indefinite == 2 a solve that meets a direction p of
// negative curvature, Rayleigh quotient lam = <p, (A + sigma) p> / |p|^2 <= 0, sets
// sigma = 2 (sigma + |lam|), |lam| at least 1e-6 of the Rayleigh quotient of the
// right-hand side, and solves again from zero (a Rayleigh quotient only bounds the lowest
// eigenvalue from above: the geometric growth keeps the shifted system away from
// singular).  The correction is left in PX.x; returns the CG iterations.
template <typename X>
static int newton_solve(fg_ctx& c, Prec<X>& PX, double& sigma, fg_stats& s) {
  to_prec<X>(c, c.GP, PX.b, 9 * c.V, -1.0);
  int n = 0;
  for (int rs = 0;; ++rs) {
    bool neg = false;
    n += cg_solve_mech<X>(c, PX, mixed_tol(c, c.o.tol_cg), c.o.max_cg, &s, sigma,
                          c.o.cg_indefinite == 2 ? &neg : nullptr);
    if (!neg) return n;
    const KScal k = c.ks_host[KS_MECH];
    const double pp = reduce_sum_r<X>(c, PX.p, 9 * c.V);
    const double lam = pp > 0.0 ? k.pq / pp : 0.0;
    const double rho0 = k.bb > 0.0 ? fabs(k.pq0) / k.bb : 0.0;
    sigma = 2.0 * (sigma + std::max(fabs(lam), 1e-6 * rho0));
    s.newton_shifted += 1;
    if (verbose())
      fprintf(stderr, "[fg]   negative curvature at cg %d (lam %.3e): sigma %.3e\n", k.iters, lam, sigma);
    if (!(sigma == sigma) || sigma <= 0.0 || rs >= 12)
      fail(FG_ERR_NUMERIC, "mechanical Newton: shifted system still not positive");
  }
}

// Alg. 1 from the current F.  Each Newton correction is damped by halving (at most 10
// times) while F + lambda dF leaves the domain (det F <= 0 or J_c <= 0) or does not lower
// err_res; the residual of the accepted iterate is the next iteration's residual.  The
// shift sigma of newton_solve shrinks 4-fold per Newton iteration, so near a stable
// equilibrium the iteration is plain Newton.  Where the tangent has negative eigenvalues
// at the equilibrium itself, a shifted correction cannot lower the residual along them:
// when a CG correction (FP32 or FP64) fails the line search, the iteration is redone
// with FP64 MINRES on the unshifted system, and the rest of this solve uses it.
template <typename R>
static void mech_newton(fg_ctx& c, Prec<R>& P, double den, fg_stats& s, double err0 = -1.0) {
  Range range("mech_newton");
  bool hi = !is_mixed(c);  // Krylov in FP64
  bool mr = false;         // MINRES
  auto resid = [&]() {
    return hi ? residual_mech<double>(c, den, c.pd.state) : residual_mech<R>(c, den, P.state);
  };
  // err0 >= 0: the caller has just evaluated err_res at this F (c.P, c.GP current), so
  // only the tangent state is built, and nothing when F is converged already
  if (err0 >= 0.0 && err0 <= c.o.tol_newton) {
    s.err_mech = err0;
    return;
  }
  double err;
  if (err0 >= 0.0) {
    if (hi) mech_state<double>(c, c.F, nullptr, nullptr, c.pd.state);
    else mech_state<R>(c, c.F, nullptr, nullptr, P.state);
    check_flags(c, "tangent state");
    err = err0;
  } else {
    err = resid();
  }
  double sigma = 0.0;
  for (int it = 0;; ++it, sigma *= 0.25) {
    s.err_mech = err;
    if (!(err == err)) fail(FG_ERR_NUMERIC, "mechanical residual is not finite");
    if (err <= c.o.tol_newton) return;
    if (it >= c.o.max_newton) fail(FG_ERR_NOCONV, "mechanical Newton hit max_newton");
    int n;
    if (mr) {
      to_prec<double>(c, c.GP, c.pd.b, 9 * c.V, -1.0);
      n = minres_mech(c, mixed_tol(c, c.o.tol_cg), c.o.max_cg);
    } else {
      n = hi ? newton_solve<double>(c, c.pd, sigma, s) : newton_solve<R>(c, P, sigma, s);
    }
    s.cg_mech += n;
    s.newton_mech += 1;
    if (verbose())
      fprintf(stderr, "[fg] newton %d%s err %.3e cg %d rr/bb %.3e status %d snaps %d\n", it,
              mr ? " (minres)" : "", err, n,
              c.ks_host[KS_MECH].rr / (c.ks_host[KS_MECH].bb > 0 ? c.ks_host[KS_MECH].bb : 1.0),
              c.ks_host[KS_MECH].status, c.ks_host[KS_MECH].snaps);
    const double* dF;
    if (!hi) {
      // FP32 roundoff leaves traces of the correction in modes G never sees (the mean and
      // the null modes of the rotated scheme); project it in FP64 onto compatible
      // zero-mean fields before the update, as the exact correction is
      VArgs u = vbase(c, 9 * c.V);
      u.in[0] = P.x;
      u.out[0] = c.P;
      launch_vec<KWiden<R>>(u, c.st);
      gres64(c, c.P, c.dF);
      dF = c.dF;
    } else {
      dF = c.pd.x;
    }
    dcopy(c.Fbk, c.F, 9 * c.V * sizeof(double), c.st);
    double lam = 1.0;
    bool ok = false;
    for (int ls = 0; ls <= 10; ++ls, lam *= 0.5) {
      VArgs v = vbase(c, 9 * c.V);  // F = F_bk + lam dF
      v.in[0] = c.Fbk;
      v.in[1] = dF;
      v.out[0] = c.F;
      v.s[0] = lam;
      launch_vec<KAxpyTo>(v, c.st);
      double e = 0.0;
      try {
        e = resid();
      } catch (Fail& f) {
        if (f.code != FG_ERR_DOMAIN) throw;
        continue;
      }
      if (verbose()) fprintf(stderr, "[fg]   lambda %.4f err %.3e\n", lam, e);
      if (e < err) {
        err = e;
        ok = true;
        break;
      }
      s.newton_damped += 1;
    }
    if (!ok && !mr) {
      // the CG correction did not lower the FP64 residual: back to F_bk, FP64 MINRES from here
      dcopy(c.F, c.Fbk, 9 * c.V * sizeof(double), c.st);
      hi = true;
      mr = true;
      s.newton_minres += 1;
      err = resid();
      if (verbose()) fprintf(stderr, "[fg]   CG correction rejected: FP64 MINRES from here\n");
      continue;
    }
    if (!ok) fail(FG_ERR_NOCONV, "mechanical Newton: no decrease of err_res along the correction");
  }
}

struct FScaleAux {
  FG_DEV static void fin(const VArgs& a, double t) { a.ks->aux = t * a.s[0]; }
};

// H = max(H_t, g_c/(2 l_c) D_f(F, c)); Hbar = mean H to the device scalar
static void history(fg_ctx& c) {
  Range range("history");
  VArgs v = vbase(c, c.V);
  v.in[0] = c.F;
  v.in[1] = c.c;
  v.in[2] = c.Ht;
  v.in[3] = c.lam;
  v.in[4] = c.mu_;
  v.in[5] = c.Om;
  v.in[6] = c.c0;
  v.in[7] = c.smax;
  v.in[8] = c.gcr;
  v.out[0] = c.H;
  v.out[1] = c.gcr ? c.Heff : nullptr;
  v.s[0] = c.o.gc / (2.0 * c.o.lc);
  if (c.law == FG_SVK) launch_vec<KHistory<LAW_SVK_>>(v, c.st);
  else launch_vec<KHistory<LAW_NH_>>(v, c.st);
  fin<FScaleAux>(c, KS_HBAR, VEC_BLOCKS, nullptr, 1.0 / (double)c.V);
}

// H_eff = H / gcr after H was set or restored (nothing to do for a uniform toughness)
static void refresh_heff(fg_ctx& c) {
  if (!c.gcr) return;
  VArgs v = vbase(c, c.V);
  v.in[0] = c.H;
  v.in[1] = c.gcr;
  v.out[0] = c.Heff;
  launch_vec<KDivTo>(v, c.st);
}

// Hbar = mean H_eff of the stored history
static void hbar_from_sum(fg_ctx& c) {
  VArgs v = vbase(c, c.V);
  v.in[0] = c.Heff;
  launch_vec<KSum>(v, c.st);
  fin<FScaleAux>(c, KS_HBAR, VEC_BLOCKS, nullptr, 1.0 / (double)c.V);
}

template <typename R>
// Alg. 2 for d.  Returns whether d changed: with H = 0 the solution is d = 0 (the
// right-hand side 2H vanishes), which leaves an already zero d as it is.
static bool pff_solve(fg_ctx& c, Prec<R>& P, fg_stats& s) {
  Range range("pff_solve");
  const double hh = reduce_sum(c, c.Heff, c.V, true);
  if (hh == 0.0) {
    if (reduce_sum(c, c.d, c.V, true) == 0.0) return false;
    dzero(c.d, c.V * sizeof(double), c.st);
    return true;
  }
  if (!is_mixed(c)) {
    to_prec<double>(c, c.Heff, c.pd.b, c.V, 2.0);
    dcopy(c.pd.x, c.d, c.V * sizeof(double), c.st);
    s.cg_pff += pcg_pff<double>(c, c.pd, c.Heff, c.o.tol_pff_cg, c.o.max_cg);
    dcopy(c.d, c.pd.x, c.V * sizeof(double), c.st);
    return true;
  }
  // mixed: FP64 residual b - A d, FP32 PCG corrections
  to_prec<R>(c, c.Heff, P.Hr, c.V, 1.0);
  const double bb = 4.0 * hh;
  Prec<double>& D = c.pd;
  for (int it = 0;; ++it) {
    op_pff(c, D, c.d, D.q, c.Heff, nullptr);  // q = A d in FP64
    {
      VArgs t = vbase(c, c.V);  // b = 2H
      t.in[0] = c.Heff;
      t.out[0] = D.b;
      t.s[0] = 2.0;
      launch_vec<KScaleTo<double>>(t, c.st);
    }
    {
      VArgs v = vbase(c, c.V);  // r = b - A d
      v.in[0] = D.b;
      v.in[1] = D.q;
      v.out[0] = D.r;
      launch_vec<KResid<double>>(v, c.st);
      fin<FStore>(c, KS_MISC, VEC_BLOCKS, nullptr);
    }
    read_ks(c);
    const double rr = c.ks_host[KS_MISC].aux;
    if (rr <= c.o.tol_pff_cg * c.o.tol_pff_cg * bb) break;
    if (it >= 50) fail(FG_ERR_NOCONV, "phase-field refinement did not converge");
    to_prec<R>(c, D.r, P.b, c.V, 1.0);
    dzero(P.x, c.V * sizeof(R), c.st);
    s.cg_pff += pcg_pff<R>(c, P, P.Hr, std::max(c.o.tol_pff_cg, c.o.cg_forcing), c.o.max_cg);
    s.inner_refine += 1;
    VArgs u = vbase(c, c.V);
    u.in[0] = P.x;
    u.out[0] = c.d;
    launch_vec<KAddTo<R>>(u, c.st);
  }
  return true;
}

template <typename R>
static void chem_cond(fg_ctx& c, Prec<R>& P, const double* F, const double* ct, const double* dt) {
  VArgs v = vbase(c, c.V);
  v.in[0] = F;
  v.in[1] = ct;
  v.in[2] = dt;
  v.in[3] = c.D;
  v.out[0] = P.kc;
  launch_vec<KChemCond<R>>(v, c.st);
}

template <typename R>
static void chem_prep(fg_ctx& c, Prec<R>& P, double dt, const double* F) {
  VArgs v = vbase(c, c.V);
  v.in[0] = c.c;
  v.in[1] = c.ct;
  v.in[2] = c.cdotB;
  v.in[3] = F;
  v.in[4] = c.dt;
  v.in[5] = c.lam;
  v.in[6] = c.mu_;
  v.in[7] = c.Om;
  v.in[8] = c.c0;
  v.out[0] = c.mu;
  v.out[1] = c.base;
  v.out[2] = P.w;
  v.s[0] = dt;
  v.s[1] = 1.0 / c.o.RT;
  v.s[2] = 1.0 / c.o.cmax;
  if (c.law == FG_SVK) launch_vec<KChemPrep<R, LAW_SVK_>>(v, c.st);
  else launch_vec<KChemPrep<R, LAW_NH_>>(v, c.st);
  if (c.o.chem_full_jacobian) {  // 1/m with the elastic part of dmu~/dc as well
    VArgs u = vbase(c, c.V);
    u.in[0] = c.c;
    u.in[1] = F;
    u.in[2] = c.dt;
    u.in[3] = c.lam;
    u.in[4] = c.mu_;
    u.in[5] = c.Om;
    u.in[6] = c.c0;
    u.out[0] = P.w;
    u.s[0] = 1.0 / c.o.RT;
    u.s[1] = 1.0 / c.o.cmax;
    if (c.law == FG_SVK) launch_vec<KChemFullM<R, LAW_SVK_>>(u, c.st);
    else launch_vec<KChemFullM<R, LAW_NH_>>(u, c.st);
  }
}

template <typename R>
static void chem_solve(fg_ctx& c, Prec<R>& P, double dt, fg_stats& s) {
  Range range("chem_solve");
  chem_cond<R>(c, P, c.F, c.ct, c.dt);
  if (is_mixed(c)) chem_cond<double>(c, c.pd, c.F, c.ct, c.dt);
  dcopy(c.c, c.ct, c.V * sizeof(double), c.st);
  const double nct = sqrt(reduce_sum(c, c.ct, c.V, true));
  for (int it = 0;; ++it) {
    if (it >= c.o.max_chem_newton) fail(FG_ERR_NOCONV, "chemical Newton hit max_chem_newton");
    chem_prep<R>(c, P, dt, c.F);
    read_ks(c);
    check_flags(c, "chemistry");
    double* b64 = is_mixed(c) ? c.pd.b : (double*)P.b;
    op_chem_rhs(c, b64, dt);
    if (is_mixed(c)) to_prec<R>(c, b64, P.b, c.V, 1.0);
    const int n = cg_solve_chem<R>(c, P, dt, mixed_tol(c, c.o.tol_chem_cg), c.o.max_cg, &s);
    s.cg_chem += n;
    s.newton_chem += 1;
    // c = c_i + lambda y c_i (1 - c_i): halved (at most 10 times) while it leaves (0, 1)
    dcopy(c.base, c.c, c.V * sizeof(double), c.st);
    double lam = 1.0;
    for (int ls = 0;; ++ls, lam *= 0.5) {
      VArgs v = vbase(c, c.V);
      v.in[0] = P.x;
      v.in[1] = c.base;
      v.in[2] = c.o.chem_full_jacobian ? P.w : nullptr;
      v.out[0] = c.c;
      v.s[0] = lam;
      launch_vec<KChemUpdate<R>>(v, c.st);
      fin<FStore>(c, KS_MISC, VEC_BLOCKS, nullptr);
      read_ks(c);
      if (!(*c.flags_host & ST_DOMAIN)) break;
      dzero(c.flags, sizeof(int), c.st);
      if (ls >= 10) fail(FG_ERR_DOMAIN, "chemistry: c left (0,1) along the whole Newton correction");
      s.newton_damped += 1;
    }
    check_flags(c, "chemistry");
    const double rel = sqrt(c.ks_host[KS_MISC].aux) / nct;
    s.err_chem = rel;
    if (rel < c.o.tol_chem) return;
  }
}

template <typename R>
static void step_impl(fg_ctx& c, Prec<R>& P, double dt, const double* Fbar, fg_stats& s) {
  Range range("fg_step");
  const long long V = c.V;
  // t-state
  dcopy(c.Ft, c.F, 9 * V * sizeof(double), c.st);
  dcopy(c.ct, c.c, V * sizeof(double), c.st);
  dcopy(c.dt, c.d, V * sizeof(double), c.st);
  dcopy(c.Ht, c.H, V * sizeof(double), c.st);
  const double mass_t = reduce_sum(c, c.ct, V, false);
  const double src = reduce_sum(c, c.cdotB, V, false);
  // F = F_t + (Fbar_{t+dt} - Fbar_t)
  {
    VArgs v = vbase(c, 9 * V);
    v.in[0] = c.Ft;
    v.out[0] = c.F;
    for (int k = 0; k < 9; ++k) v.s[k] = Fbar[k] - c.Fbar[k];
    launch_vec<KShiftF>(v, c.st);
  }
  double Fbar_old[9];
  memcpy(Fbar_old, c.Fbar, sizeof(Fbar_old));
  memcpy(c.Fbar, Fbar, sizeof(c.Fbar));
  try {
    chem_solve<R>(c, P, dt, s);
    const double mass = reduce_sum(c, c.c, V, false);
    s.mass = mass;
    s.mass_err = (mass - (mass_t + dt * src)) / (mass != 0.0 ? mass : 1.0);
    // Alg. 4: the body (mechanics, history, phase field) runs at least once, also from a
    // state already in equilibrium, and the loop ends when the state it left is.  When the
    // phase-field solve leaves d as it was (no damage yet), F, c and d are the state of the
    // Newton's last err_res, with the same denominator: it is reused
    bool fresh = false;
    double den = 0.0, err = 0.0;
    for (int k = 0;; ++k) {
      if (!fresh) {
        den = residual_den(c);
        err = residual_mech<double>(c, den, nullptr);
      }
      s.err_mech = err;
      if (k > 0 && err <= c.o.tol_stag) break;
      if (k >= c.o.max_stag) fail(FG_ERR_NOCONV, "staggered scheme hit max_stag");
      mech_newton<R>(c, P, den, s, err);
      history(c);
      const bool dchanged = pff_solve<R>(c, P, s);
      s.stag += 1;
      fresh = !dchanged;
      if (fresh) err = s.err_mech;
    }
  } catch (Fail&) {
    // restore the t-state
    dcopy(c.F, c.Ft, 9 * V * sizeof(double), c.st);
    dcopy(c.c, c.ct, V * sizeof(double), c.st);
    dcopy(c.d, c.dt, V * sizeof(double), c.st);
    dcopy(c.H, c.Ht, V * sizeof(double), c.st);
    refresh_heff(c);
    memcpy(c.Fbar, Fbar_old, sizeof(c.Fbar));
    dsync(c.st);
    throw;
  }
  memcpy(c.Fbar_prev, Fbar_old, sizeof(Fbar_old));
  if (c.smask)  // the stress-controlled components of F-bar were unknowns: their mean
    for (int k = 0; k < 9; ++k)
      if ((c.smask >> k) & 1) c.Fbar[k] = reduce_sum(c, c.F + (long long)k * V, V, false) / (double)V;
  c.last_dt = dt;
  c.stepped = true;
  dsync(c.st);
}

// ------------------------------------------------------------------ adjoint

// state vector of the tape: c (V), F (9 V), d (V), H (V)
static void save_state(fg_ctx& c, double* buf) {
  const long long V = c.V;
  dcopy(buf, c.c, V * sizeof(double), c.st);
  dcopy(buf + V, c.F, 9 * V * sizeof(double), c.st);
  dcopy(buf + 10 * V, c.d, V * sizeof(double), c.st);
  dcopy(buf + 11 * V, c.H, V * sizeof(double), c.st);
}

static void load_state(fg_ctx& c, const double* buf, double* cc, double* F, double* d, double* H) {
  const long long V = c.V;
  dcopy(cc, buf, V * sizeof(double), c.st);
  dcopy(F, buf + V, 9 * V * sizeof(double), c.st);
  dcopy(d, buf + 10 * V, V * sizeof(double), c.st);
  dcopy(H, buf + 11 * V, V * sizeof(double), c.st);
}

// forgets the captured CG graphs (they bake in the stress mask and the kernel choices)
static void drop_graphs(fg_ctx& c) {
#ifndef FG_EMU
  for (auto& row : c.cg_graph)
    for (auto& ex : row)
      if (ex) {
        cudaGraphExecDestroy(ex);
        ex = nullptr;
      }
#else
  (void)c;
#endif
}

static void free_tape(fg_ctx& c) {
  if (!c.tape) return;
  for (double* p : c.tape->ckpt) dfree(p);
  delete c.tape;
  c.tape = nullptr;
}

// grad_f u (3 V) and grad_f^H f (V) of the chemistry operator, FP64
static void grad3(fg_ctx& c, const double* u, double* out) {
  Prec<double>& P = c.pd;
  PassArgs<double> a = pbase(c, P, nullptr);
  a.tw = P.twx;
  a.rin = u;
  a.cout = P.S1;
  P.ox->xf_copy1(a, c.st);
  const double zc[4] = {1.0 / (double)c.V, 0, 0, 0};
  yzy(c, P, nullptr, 1, P.oz->z_grad, 3, zc, nullptr);
  a = pbase(c, P, nullptr);
  a.tw = P.twx;
  a.cin = P.S1;
  a.rout = out;
  P.ox->xi_store3(a, c.st);
}

static void divadj(fg_ctx& c, const double* f, double* out) {
  Prec<double>& P = c.pd;
  PassArgs<double> a = pbase(c, P, nullptr);
  a.tw = P.twx;
  a.rin = f;
  a.cout = P.S1;
  P.ox->xf_copy3(a, c.st);
  const double zc[4] = {1.0 / (double)c.V, 0, 0, 0};
  yzy(c, P, nullptr, 3, P.oz->z_div, 1, zc, nullptr);
  a = pbase(c, P, nullptr);
  a.tw = P.twx;
  a.cin = P.S1;
  a.rout = out;
  P.ox->xi_store1(a, c.st);
}

// Displacement at the voxel corners (Eq. Fsplit), FP64: u~ (3 V) of F (9 V) by the
// least-squares inverse of the rotated gradient, and its transpose (9 V) of r (3 V).
static void disp_coef(const fg_ctx& c, double* zc) {
  zc[0] = 1.0 / (double)c.V;
  for (int j = 0; j < 3; ++j) zc[1 + j] = 0.5 * c.h[j];
}

static void disp_fluct(fg_ctx& c, const double* F, double* u) {
  Prec<double>& P = c.pd;
  PassArgs<double> a = pbase(c, P, nullptr);
  a.tw = P.twx;
  a.rin = F;
  a.cout = P.S1;
  P.ox->xf_copy9(a, c.st);
  double zc[4];
  disp_coef(c, zc);
  yzy(c, P, nullptr, 9, P.oz->z_disp, 3, zc, nullptr);
  a = pbase(c, P, nullptr);
  a.tw = P.twx;
  a.cin = P.S1;
  a.rout = u;
  P.ox->xi_store3(a, c.st);
}

static void disp_fluct_adj(fg_ctx& c, const double* r, double* g) {
  Prec<double>& P = c.pd;
  PassArgs<double> a = pbase(c, P, nullptr);
  a.tw = P.twx;
  a.rin = r;
  a.cout = P.S1;
  P.ox->xf_copy3(a, c.st);
  double zc[4];
  disp_coef(c, zc);
  yzy(c, P, nullptr, 3, P.oz->z_dispT, 9, zc, nullptr);
  a = pbase(c, P, nullptr);
  a.tw = P.twx;
  a.cin = P.S1;
  a.rout = g;
  P.ox->xi_store9(a, c.st);
}

// adds (Fbar - I) x at the corners to u (3 V)
static void disp_affine(fg_ctx& c, const double* Fbar, double* u) {
  for (int i = 0; i < 3; ++i) {
    VArgs v = vbase(c, c.V);
    v.out[0] = u + (long long)i * c.V;
    for (int j = 0; j < 3; ++j) v.s[j] = (Fbar[3 * i + j] - (i == j ? 1.0 : 0.0)) * c.h[j];
    v.s[3] = (double)c.nx;
    v.s[4] = (double)c.ny;
    launch_vec<KAddAffine>(v, c.st);
  }
}

// device buffers of one API call, freed on every exit path
struct Scratch {
  std::vector<void*> p;
  double* get(long long n) {
    p.push_back(nullptr);
    p.back() = dalloc((size_t)n * sizeof(double));
    return (double*)p.back();
  }
  ~Scratch() {
    for (void* q : p) dfree(q);
  }
};

static void axpy64(fg_ctx& c, double* out, const double* x, double s, const double* y, long long n) {
  VArgs v = vbase(c, n);  // out = x + s y
  v.in[0] = x;
  v.in[1] = y;
  v.out[0] = out;
  v.s[0] = s;
  launch_vec<KAxpyTo>(v, c.st);
}

// work space of the reverse pass (FP64)
struct AdjWork {
  double *lamM, *lamD, *lamH, *chi, *lamC, *gl, *gm, *Ll, *gctot, *tmpV, *sweepD;
  double* seeds[2];  // two seed sets (c V, F 9 V, d V, H V) = 12 V each
  double *gE, *gG, *gD;
  std::vector<double*> Q;  // GMRES basis
  std::vector<void*> mem;
  fg_ctx* c = nullptr;
  double* get(long long n) {
    double* p = (double*)dalloc((size_t)n * sizeof(double));
    mem.push_back(p);
    dzero(p, (size_t)n * sizeof(double), c->st);
    return p;
  }
  ~AdjWork() {
    for (void* p : mem) dfree(p);
  }
};

static const double* seed_c(const double* S, long long) { return S; }
static const double* seed_F(const double* S, long long V) { return S + V; }
static const double* seed_d(const double* S, long long V) { return S + 10 * V; }
static const double* seed_H(const double* S, long long V) { return S + 11 * V; }

// GKG lam = G rhs, lam in W.lamM (FP64 CG, negative curvature taken, caps are errors)
static int adj_solve_M(fg_ctx& c, const double* rhs, double* out) {
  Prec<double>& D = c.pd;
  op_gres(c, D, rhs, D.b, nullptr);
  const int n = cg_solve_mech<double>(c, D, c.o.tol_cg, c.o.max_cg, nullptr, 0.0, nullptr, 1);
  dcopy(out, D.x, 9 * c.V * sizeof(double), c.st);
  return n;
}

// A(H_eff) lam = rhs (phase-field PCG from zero)
static int adj_solve_D(fg_ctx& c, const double* rhs, double* out) {
  Prec<double>& D = c.pd;
  dcopy(D.b, rhs, c.V * sizeof(double), c.st);
  dzero(D.x, c.V * sizeof(double), c.st);
  const int n = pcg_pff<double>(c, D, c.Heff, c.o.tol_pff_cg, c.o.max_cg);
  dcopy(out, D.x, c.V * sizeof(double), c.st);
  return n;
}

template <int LAW>
static void adj_rhs_M(fg_ctx& c, const double* sF, const double* lamH, double* out, double* chi) {
  VArgs v = vbase(c, c.V);
  v.in[0] = sF;
  v.in[1] = lamH;
  v.in[2] = c.F;
  v.in[3] = c.c;
  v.in[4] = c.Ht;
  v.in[5] = c.lam;
  v.in[6] = c.mu_;
  v.in[7] = c.Om;
  v.in[8] = c.c0;
  v.in[9] = c.smax;
  v.in[10] = c.gcr;
  v.out[0] = out;
  v.out[1] = chi;
  v.s[0] = c.o.gc / (2.0 * c.o.lc);
  launch_vec<KAdjRhsM<LAW>>(v, c.st);
}

template <int LAW>
static void adj_rhs_D(fg_ctx& c, const double* sd, const double* lamM, double* out) {
  VArgs v = vbase(c, c.V);
  v.in[0] = sd;
  v.in[1] = lamM;
  v.in[2] = c.F;
  v.in[3] = c.c;
  v.in[4] = c.d;
  v.in[5] = c.lam;
  v.in[6] = c.mu_;
  v.in[7] = c.Om;
  v.in[8] = c.c0;
  v.out[0] = out;
  launch_vec<KAdjRhsD<LAW>>(v, c.st);
}

static void adj_lamH(fg_ctx& c, const double* sH, const double* lamD, double* out) {
  VArgs v = vbase(c, c.V);
  v.in[0] = sH;
  v.in[1] = lamD;
  v.in[2] = c.d;
  v.in[3] = c.gcr;
  v.out[0] = out;
  launch_vec<KAdjLamH>(v, c.st);
}

// one transposed Gauss-Seidel sweep: lamM = (GKG)^-1 G (sF + chi lamH Z),
// lamD = A^-1 (sd - dP/dd : lamM)
template <int LAW>
static void adj_sweep(fg_ctx& c, AdjWork& W, const double* sF, const double* sd, const double* lamH,
                      double* lamM, double* lamD, fg_adjoint_stats* as) {
  adj_rhs_M<LAW>(c, sF, lamH, c.dF, W.chi);
  const int nm = adj_solve_M(c, c.dF, lamM);
  adj_rhs_D<LAW>(c, sd, lamM, W.tmpV);
  const int nd = adj_solve_D(c, W.tmpV, lamD);
  if (as) {
    as->cg_mech += nm;
    as->cg_pff += nd;
    as->sweeps += 1;
  }
}

// Reverse of one converged step: the context holds the step's output state (c, F, d, H)
// and its t-state (c_t, F_t, d_t, H_t); S_out are the seeds of the outputs, S_in receives
// those of the inputs; gradients accumulate into W.gE, W.gG, W.gD.
template <int LAW>
static void adj_step(fg_ctx& c, AdjWork& W, const double* S_out, double* S_in, double dt,
                     const double* dFbar, fg_adjoint_stats* as) {
  const long long V = c.V;
  Prec<double>& D = c.pd;
  refresh_heff(c);
  hbar_from_sum(c);
  mech_state<double>(c, c.F, nullptr, nullptr, D.state);
  check_flags(c, "adjoint state");
  // (F, H, d) block
  adj_sweep<LAW>(c, W, seed_F(S_out, V), seed_d(S_out, V), seed_H(S_out, V), W.lamM, W.lamD, as);
  const double nchi = reduce_sum(c, W.chi, V, false);
  if (nchi > 0.0) {
    // GMRES on (I - T) lamD = lamD0, T x = sweep(0, 0, 2 r (1 - d) x).lamD
    const int m = std::max(1, std::min(c.o.max_stag, 60));
    while ((int)W.Q.size() < m + 1) W.Q.push_back(W.get(V));
    std::vector<double> Hm((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1, 0.0);
    const double beta = sqrt(dotd(c, W.lamD, W.lamD, V));
    int k = 0;
    bool conv = beta == 0.0;
    if (!conv) {
      VArgs v = vbase(c, V);
      v.in[0] = W.lamD;
      v.out[0] = W.Q[0];
      v.s[0] = 1.0 / beta;
      launch_vec<KScaleTo<double>>(v, c.st);
      g[0] = beta;
    }
    for (; !conv && k < m; ++k) {
      double* w = W.Q[k + 1];
      adj_lamH(c, nullptr, W.Q[k], W.tmpV);
      double* tM = c.Fbk;  // 9 V scratch
      adj_sweep<LAW>(c, W, nullptr, nullptr, W.tmpV, tM, W.sweepD, as);
      axpy64(c, w, W.Q[k], -1.0, W.sweepD, V);  // w = Q_k - T Q_k
      for (int j = 0; j <= k; ++j) {  // modified Gram-Schmidt
        const double h = dotd(c, W.Q[j], w, V);
        Hm[(size_t)j * m + k] = h;
        axpy64(c, w, w, -h, W.Q[j], V);
      }
      const double hn = sqrt(dotd(c, w, w, V));
      Hm[(size_t)(k + 1) * m + k] = hn;
      // Givens rotations of the Hessenberg column
      for (int j = 0; j < k; ++j) {
        const double a = Hm[(size_t)j * m + k], b = Hm[(size_t)(j + 1) * m + k];
        Hm[(size_t)j * m + k] = cs[j] * a + sn[j] * b;
        Hm[(size_t)(j + 1) * m + k] = -sn[j] * a + cs[j] * b;
      }
      const double a = Hm[(size_t)k * m + k], b = Hm[(size_t)(k + 1) * m + k];
      const double r = hypot(a, b);
      cs[k] = r > 0.0 ? a / r : 1.0;
      sn[k] = r > 0.0 ? b / r : 0.0;
      Hm[(size_t)k * m + k] = r;
      Hm[(size_t)(k + 1) * m + k] = 0.0;
      g[k + 1] = -sn[k] * g[k];
      g[k] = cs[k] * g[k];
      if (as) as->gmres += 1;
      if (fabs(g[k + 1]) <= c.o.tol_stag * beta || hn == 0.0) {
        conv = true;
        ++k;
        break;
      }
      VArgs v = vbase(c, V);
      v.in[0] = w;
      v.out[0] = w;
      v.s[0] = 1.0 / hn;
      launch_vec<KScaleTo<double>>(v, c.st);
    }
    if (!conv) fail(FG_ERR_NOCONV, "adjoint: GMRES on the phase-field multiplier hit max_stag");
    std::vector<double> y(k, 0.0);  // back substitution
    for (int i = k - 1; i >= 0; --i) {
      double t = g[i];
      for (int j = i + 1; j < k; ++j) t -= Hm[(size_t)i * m + j] * y[j];
      y[i] = t / Hm[(size_t)i * m + i];
    }
    dzero(W.lamD, V * sizeof(double), c.st);
    for (int j = 0; j < k; ++j) axpy64(c, W.lamD, W.lamD, y[j], W.Q[j], V);
    adj_lamH(c, seed_H(S_out, V), W.lamD, W.lamH);
    adj_rhs_M<LAW>(c, seed_F(S_out, V), W.lamH, c.dF, W.chi);
    const int nm = adj_solve_M(c, c.dF, W.lamM);
    if (as) as->cg_mech += nm;
  }
  adj_lamH(c, seed_H(S_out, V), W.lamD, W.lamH);
  {
    VArgs v = vbase(c, V);
    v.in[0] = W.lamM;
    v.in[1] = W.lamD;
    v.in[2] = W.lamH;
    v.in[3] = seed_c(S_out, V);
    v.in[4] = c.F;
    v.in[5] = c.c;
    v.in[6] = c.d;
    v.in[7] = c.H;
    v.in[8] = c.Ht;
    v.in[9] = c.lam;
    v.in[10] = c.mu_;
    v.in[11] = c.Om;
    v.in[12] = c.c0;
    v.in[13] = c.smax;
    v.in[14] = c.gcr;
    v.out[0] = W.gE;
    v.out[1] = W.gG;
    v.out[2] = (double*)seed_H(S_in, V);
    v.out[3] = W.gctot;
    v.s[0] = c.o.gc / (2.0 * c.o.lc);
    launch_vec<KAdjBlockOut<LAW>>(v, c.st);
  }
  // chemistry: F~ = F_t + (Fbar - Fbar_t)
  {
    VArgs v = vbase(c, 9 * V);
    v.in[0] = c.Ft;
    v.out[0] = c.Fbk;
    for (int k = 0; k < 9; ++k) v.s[k] = dFbar[k];
    launch_vec<KShiftF>(v, c.st);
  }
  chem_cond<double>(c, D, c.Fbk, c.ct, c.dt);
  chem_prep<double>(c, D, dt, c.Fbk);
  {
    VArgs v = vbase(c, V);
    v.in[0] = c.c;
    v.in[1] = W.gctot;
    v.in[2] = c.Fbk;
    v.in[3] = c.dt;
    v.in[4] = c.lam;
    v.in[5] = c.mu_;
    v.in[6] = c.Om;
    v.in[7] = c.c0;
    v.out[0] = D.w;
    v.out[1] = D.b;
    v.s[0] = 1.0 / c.o.RT;
    v.s[1] = 1.0 / c.o.cmax;
    launch_vec<KAdjChemM<LAW>>(v, c.st);
  }
  read_ks(c);
  if (*c.flags_host & ST_NUMERIC) {
    dzero(c.flags, sizeof(int), c.st);
    fail(FG_ERR_NUMERIC, "adjoint: chemistry Jacobian dmu/dc not positive");
  }
  check_flags(c, "adjoint chemistry");
  const int nc = cg_solve<double>(c, D, V, KS_CHEM, c.o.tol_chem_cg, c.o.max_cg,
                                  [&](const double* p, double* q, const int* done) {
                                    return op_chem(c, D, p, q, dt, done);
                                  });
  if (as) as->cg_chem += nc;
  dcopy(W.lamC, D.x, V * sizeof(double), c.st);
  grad3(c, W.lamC, W.gl);
  grad3(c, c.mu, W.gm);
  op_chem_L(c, D, W.lamC, nullptr);
  {
    PassArgs<double> a = pbase(c, D, nullptr);
    a.tw = D.twx;
    a.cin = D.S1;
    a.rout = W.Ll;
    D.ox->xi_store1(a, c.st);
  }
  {
    VArgs v = vbase(c, V);
    v.in[0] = W.lamC;
    v.in[1] = W.gl;
    v.in[2] = W.gm;
    v.in[3] = W.Ll;
    v.in[4] = c.c;
    v.in[5] = c.ct;
    v.in[6] = c.dt;
    v.in[7] = c.Fbk;
    v.in[8] = c.D;
    v.in[9] = c.lam;
    v.in[10] = c.mu_;
    v.in[11] = c.Om;
    v.in[12] = c.c0;
    v.out[0] = (double*)seed_c(S_in, V);
    v.out[1] = (double*)seed_d(S_in, V);
    v.out[2] = (double*)seed_F(S_in, V);
    v.out[3] = W.gD;
    v.out[4] = W.gE;
    v.s[0] = dt;
    v.s[1] = 1.0 / c.o.RT;
    v.s[2] = 1.0 / c.o.cmax;
    launch_vec<KAdjChemOut<LAW>>(v, c.st);
  }
  check_flags(c, "adjoint chemistry");
  if (as) as->steps += 1;
}

// Gamma_E of the stored phase field into the d seed of S; its direct log g_c gradient into gG
static double crack_loss(fg_ctx& c, AdjWork& W, double* S) {
  const long long V = c.V;
  grad3(c, c.d, W.gl);
  VArgs v = vbase(c, V);
  v.in[0] = c.d;
  v.in[1] = W.gl;
  v.in[2] = c.gcr;
  v.out[0] = W.gG;
  v.out[1] = W.gm;
  v.s[0] = c.o.gc;
  v.s[1] = c.o.lc;
  v.s[2] = c.h[0] * c.h[1] * c.h[2];
  launch_vec<KCrackLoss>(v, c.st);
  fin<FStore>(c, KS_MISC, VEC_BLOCKS, nullptr);
  read_ks(c);
  const double loss = c.ks_host[KS_MISC].aux;
  divadj(c, W.gm, W.tmpV);
  VArgs u = vbase(c, V);
  u.in[0] = c.d;
  u.in[1] = W.tmpV;
  u.in[2] = c.gcr;
  u.out[0] = (double*)seed_d(S, V);
  u.s[0] = c.o.gc;
  u.s[1] = c.o.lc;
  u.s[2] = c.h[0] * c.h[1] * c.h[2];
  launch_vec<KCrackSeed>(u, c.st);
  return loss;
}

template <typename R>
static double adjoint_impl(fg_ctx& c, Prec<R>& P, int loss, const double* sc, const double* sF,
                           const double* sd, double* gE, double* gG, double* gD, fg_adjoint_stats* as) {
  Range range("fg_adjoint");
  Tape& T = *c.tape;
  const long long V = c.V;
  const int nsteps = (int)T.dts.size();
  AdjWork W;
  W.c = &c;
  W.lamM = W.get(9 * V);
  W.lamD = W.get(V);
  W.lamH = W.get(V);
  W.chi = W.get(V);
  W.lamC = W.get(V);
  W.gl = W.get(3 * V);
  W.gm = W.get(3 * V);
  W.Ll = W.get(V);
  W.gctot = W.get(V);
  W.tmpV = W.get(V);
  W.sweepD = W.get(V);
  W.seeds[0] = W.get(12 * V);
  W.seeds[1] = W.get(12 * V);
  W.gE = W.get(V);
  W.gG = W.get(V);
  W.gD = W.get(V);
  // the state at the call (returned to afterwards): current and t-state
  double* fin_now = W.get(12 * V);
  double* fin_t = W.get(12 * V);
  save_state(c, fin_now);
  dcopy(fin_t, c.ct, V * sizeof(double), c.st);
  dcopy(fin_t + V, c.Ft, 9 * V * sizeof(double), c.st);
  dcopy(fin_t + 10 * V, c.dt, V * sizeof(double), c.st);
  dcopy(fin_t + 11 * V, c.Ht, V * sizeof(double), c.st);
  double fb_now[9], fb_prev[9];
  memcpy(fb_now, c.Fbar, sizeof(fb_now));
  memcpy(fb_prev, c.Fbar_prev, sizeof(fb_prev));
  const double last_dt = c.last_dt;
  const bool stepped = c.stepped;
  // loss seeds of the final state
  double* Sout = W.seeds[0];
  double* Sin = W.seeds[1];
  double value = 0.0;
  if (loss == FG_LOSS_CRACK_ENERGY) {
    value = crack_loss(c, W, Sout);
  } else {
    if (sc) dcopy(Sout, sc, V * sizeof(double), c.st);
    if (sF) dcopy(Sout + V, sF, 9 * V * sizeof(double), c.st);
    if (sd) dcopy(Sout + 10 * V, sd, V * sizeof(double), c.st);
  }
  const int every = T.every;
  std::vector<double*> snap(every + 1);
  for (auto& p : snap) p = W.get(12 * V);
  std::vector<std::array<double, 9>> snap_fb(every + 1);
  c.strict = true;
  try {
    for (int s = (int)T.ckpt.size() - 1; s >= 0; --s) {
      const int k0 = s * every, k1 = std::min(nsteps, k0 + every);
      // recompute the segment from its checkpoint
      load_state(c, T.ckpt[s], c.c, c.F, c.d, c.H);
      refresh_heff(c);
      memcpy(c.Fbar, T.ckpt_fbar[s].data(), sizeof(c.Fbar));
      dcopy(snap[0], T.ckpt[s], 12 * V * sizeof(double), c.st);
      snap_fb[0] = T.ckpt_fbar[s];
      for (int k = k0; k < k1; ++k) {
        fg_stats st{};
        step_impl<R>(c, P, T.dts[k], T.fbars[k].data(), st);
        if (as) as->recomputed += 1;
        save_state(c, snap[k - k0 + 1]);
        snap_fb[k - k0 + 1] = T.fbars[k];
      }
      // reverse through the segment
      for (int k = k1 - 1; k >= k0; --k) {
        const int j = k - k0;
        load_state(c, snap[j + 1], c.c, c.F, c.d, c.H);
        load_state(c, snap[j], c.ct, c.Ft, c.dt, c.Ht);
        // the chemistry of step k saw F~ = F_t + Fcmd_k - Fbar_t.  Under mixed control a
        // step stores Fbar_t = mean(F_t) on the stress-controlled components, which makes
        // F~ depend on that mean for every step after the first of the tape
        const bool mean_ctl = c.smask != 0 && k > 0;
        double dFb[9];
        for (int q = 0; q < 9; ++q) {
          double fbt = snap_fb[j][q];
          if (mean_ctl && ((c.smask >> q) & 1))
            fbt = reduce_sum(c, c.Ft + (long long)q * V, V, false) / (double)V;
          dFb[q] = snap_fb[j + 1][q] - fbt;
        }
        dzero(Sin, 12 * V * sizeof(double), c.st);
        if (c.law == FG_SVK) adj_step<LAW_SVK_>(c, W, Sout, Sin, T.dts[k], dFb, as);
        else adj_step<LAW_NH_>(c, W, Sout, Sin, T.dts[k], dFb, as);
        if (mean_ctl)  // dF~/dF_t = I - mean on the controlled components
          for (int q = 0; q < 9; ++q)
            if ((c.smask >> q) & 1) {
              double* sq = Sin + V + (long long)q * V;  // component q of the F seed
              VArgs v = vbase(c, V);
              v.in[0] = sq;
              v.out[0] = sq;
              v.s[0] = -reduce_sum(c, sq, V, false) / (double)V;
              launch_vec<KShiftF>(v, c.st);
            }
        std::swap(Sout, Sin);
      }
    }
  } catch (...) {
    c.strict = false;
    load_state(c, fin_now, c.c, c.F, c.d, c.H);
    load_state(c, fin_t, c.ct, c.Ft, c.dt, c.Ht);
    refresh_heff(c);
    memcpy(c.Fbar, fb_now, sizeof(fb_now));
    dsync(c.st);
    throw;
  }
  c.strict = false;
  load_state(c, fin_now, c.c, c.F, c.d, c.H);
  load_state(c, fin_t, c.ct, c.Ft, c.dt, c.Ht);
  refresh_heff(c);
  memcpy(c.Fbar, fb_now, sizeof(fb_now));
  memcpy(c.Fbar_prev, fb_prev, sizeof(fb_prev));
  c.last_dt = last_dt;
  c.stepped = stepped;
  if (gE) dcopy(gE, W.gE, V * sizeof(double), c.st);
  if (gG) dcopy(gG, W.gG, V * sizeof(double), c.st);
  if (gD) dcopy(gD, W.gD, V * sizeof(double), c.st);
  dsync(c.st);
  return value;
}

}  // namespace fg

using namespace fg;

template <typename R>
static double do_apply(fg_ctx& c, Prec<R>& P, int op, const R* x, R* y, double dt) {
  int nb = 0;
  switch (op) {
    case FG_OP_MECH:
      if (!P.state) fail(FG_ERR_INVALID, "fg_apply: no tangent state in this precision");
      mech_state<R>(c, c.F, nullptr, nullptr, P.state);
      nb = op_mech(c, P, x, y, nullptr);
      break;
    case FG_OP_GRES:
      nb = op_gres(c, P, x, y, nullptr);
      break;
    case FG_OP_PFF: {
      const R* H;
      if constexpr (sizeof(R) == 8) H = (const R*)c.Heff;
      else {
        to_prec<R>(c, c.Heff, P.Hr, c.V, 1.0);
        H = P.Hr;
      }
      nb = op_pff(c, P, x, y, H, nullptr);
      break;
    }
    case FG_OP_PFF_PREC:
      hbar_from_sum(c);
      nb = op_prec(c, P, x, y, nullptr);
      break;
    case FG_OP_CHEM:
      dcopy(c.ct, c.c, c.V * sizeof(double), c.st);
      dcopy(c.dt, c.d, c.V * sizeof(double), c.st);
      chem_cond<R>(c, P, c.F, c.c, c.d);
      chem_prep<R>(c, P, dt, c.F);
      nb = op_chem(c, P, x, y, dt, nullptr);
      break;
    default:
      fail(FG_ERR_INVALID, "fg_apply: unknown operator");
  }
  fin<FStore>(c, KS_MISC, nb, nullptr);
  read_ks(c);
  check_flags(c, "apply");
  return c.ks_host[KS_MISC].aux;
}

// ================================================================== C ABI

#define FG_API_BEGIN \
  g_err.clear();     \
  try {
#define FG_API_END                                     \
  }                                                    \
  catch (Fail & f) {                                   \
    return f.code;                                     \
  }                                                    \
  catch (std::exception & e) {                         \
    g_err = e.what();                                  \
    return FG_ERR_INVALID;                             \
  }                                                    \
  return FG_OK;

extern "C" {

void fg_default_opts(fg_opts* o) {
  memset(o, 0, sizeof(*o));
  o->precision = FG_FP64;
  o->gc = 1.0;
  o->lc = 2e-7;
  o->RT = 8.314462618 * 298.15;
  o->cmax = 3.0e4;
  o->tol_newton = 1e-9;
  o->tol_cg = 1e-10;
  o->tol_chem = 1e-9;
  o->tol_chem_cg = 1e-10;
  o->tol_pff_cg = 1e-10;
  o->tol_stag = 1e-9;
  o->cg_forcing = 1e-5;
  o->max_newton = 30;
  o->max_cg = 5000;
  o->max_chem_newton = 50;
  o->max_stag = 50;
  o->cuda_stream = nullptr;
  o->cg_indefinite = 2;
  o->l2_prefetch = 0;
  o->residual_ff = 1;
  o->cluster_pass = 1;
}

int fg_supported_size(int n) {
  const SizeOps<double>* s = size_ops<double>(n);
  return s != nullptr && size_ops<float>(n) != nullptr;
}

const char* fg_last_error(void) { return g_err.c_str(); }

long long fg_kernel_launches(void) { return launch_counter().load(); }

void fg_destroy(fg_ctx* ctx) {
  if (!ctx) return;
#ifndef FG_EMU
  cudaStreamSynchronize(ctx->st);
  for (auto& v : ctx->prof_ev)
    for (cudaEvent_t e : v) cudaEventDestroy(e);
#endif
  free_tape(*ctx);
#ifndef FG_EMU
  for (auto& row : ctx->cg_graph)
    for (auto& ex : row)
      if (ex) cudaGraphExecDestroy(ex);
#endif
  free_all(*ctx);
  delete ctx;
}

// file layout: magic "FGST", version 2, nx ny nz law smask (int32), Fbar[9], Fbar_prev[9],
// last_dt, stepped (as a double), Pbar[9], then c F d H and c_t F_t d_t H_t (24 V doubles).
// Version 1 files (no smask, no Pbar) still load and leave the stress control as it is.
static const char FG_MAGIC[4] = {'F', 'G', 'S', 'T'};

int fg_save(fg_ctx* c, const char* path) {
  FG_API_BEGIN
  if (!c || !path) fail(FG_ERR_INVALID, "fg_save: null argument");
  const long long V = c->V;
  std::vector<double> buf(24 * V);
  save_state(*c, buf.data());
  dcopy(buf.data() + 12 * V, c->ct, V * sizeof(double), c->st);
  dcopy(buf.data() + 13 * V, c->Ft, 9 * V * sizeof(double), c->st);
  dcopy(buf.data() + 22 * V, c->dt, V * sizeof(double), c->st);
  dcopy(buf.data() + 23 * V, c->Ht, V * sizeof(double), c->st);
  dsync(c->st);
  FILE* f = fopen(path, "wb");
  if (!f) fail(FG_ERR_INVALID, std::string("fg_save: cannot open ") + path);
  const int32_t hdr[6] = {2, c->nx, c->ny, c->nz, c->law, c->smask};
  double sc[29];
  memcpy(sc, c->Fbar, 9 * sizeof(double));
  memcpy(sc + 9, c->Fbar_prev, 9 * sizeof(double));
  sc[18] = c->last_dt;
  sc[19] = c->stepped ? 1.0 : 0.0;
  memcpy(sc + 20, c->Pbar, 9 * sizeof(double));
  bool ok = fwrite(FG_MAGIC, 1, 4, f) == 4 && fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
            fwrite(sc, sizeof(sc), 1, f) == 1 &&
            fwrite(buf.data(), sizeof(double), buf.size(), f) == buf.size();
  ok = (fclose(f) == 0) && ok;
  if (!ok) fail(FG_ERR_INVALID, std::string("fg_save: write failed: ") + path);
  FG_API_END
}

int fg_load(fg_ctx* c, const char* path) {
  FG_API_BEGIN
  if (!c || !path) fail(FG_ERR_INVALID, "fg_load: null argument");
  if (c->tape && !c->tape->dts.empty())  // the reverse pass recomputes the taped trajectory
    fail(FG_ERR_INVALID, "fg_load: steps are recorded on the tape");
  const long long V = c->V;
  FILE* f = fopen(path, "rb");
  if (!f) fail(FG_ERR_INVALID, std::string("fg_load: cannot open ") + path);
  char mg[4] = {};
  int32_t hdr[6] = {};
  double sc[29] = {};
  std::vector<double> buf(24 * V);
  bool ok = fread(mg, 1, 4, f) == 4 && fread(hdr, sizeof(int32_t), 5, f) == 5;
  const int version = ok ? hdr[0] : 0;
  if (ok && version == 2) ok = fread(hdr + 5, sizeof(int32_t), 1, f) == 1;
  if (ok) ok = fread(sc, sizeof(double), version == 2 ? 29 : 20, f) == (version == 2 ? 29u : 20u);
  if (!ok || memcmp(mg, FG_MAGIC, 4) != 0 || (version != 1 && version != 2) ||
      (version == 2 && (hdr[5] < 0 || hdr[5] > 511))) {
    fclose(f);
    fail(FG_ERR_INVALID, std::string("fg_load: not a state file of a known version: ") + path);
  }
  if (hdr[1] != c->nx || hdr[2] != c->ny || hdr[3] != c->nz || hdr[4] != c->law) {
    fclose(f);
    fail(FG_ERR_INVALID, "fg_load: the file's grid or law differs from the context's");
  }
  ok = fread(buf.data(), sizeof(double), buf.size(), f) == buf.size();
  fclose(f);
  if (!ok) fail(FG_ERR_INVALID, std::string("fg_load: truncated state file: ") + path);
  load_state(*c, buf.data(), c->c, c->F, c->d, c->H);
  dcopy(c->ct, buf.data() + 12 * V, V * sizeof(double), c->st);
  dcopy(c->Ft, buf.data() + 13 * V, 9 * V * sizeof(double), c->st);
  dcopy(c->dt, buf.data() + 22 * V, V * sizeof(double), c->st);
  dcopy(c->Ht, buf.data() + 23 * V, V * sizeof(double), c->st);
  refresh_heff(*c);
  memcpy(c->Fbar, sc, 9 * sizeof(double));
  memcpy(c->Fbar_prev, sc + 9, 9 * sizeof(double));
  c->last_dt = sc[18];
  c->stepped = sc[19] != 0.0;
  if (version == 2 && (hdr[5] != c->smask || memcmp(c->Pbar, sc + 20, 9 * sizeof(double)) != 0)) {
    c->smask = hdr[5];
    for (int k = 0; k < 9; ++k) c->Pbar[k] = c->smask ? sc[20 + k] : 0.0;
    drop_graphs(*c);
  }
  dsync(c->st);
  FG_API_END
}

int fg_set_stress_control(fg_ctx* c, int mask, const double Pbar[9]) {
  FG_API_BEGIN
  if (!c || mask < 0 || mask > 511 || (mask && !Pbar)) fail(FG_ERR_INVALID, "fg_set_stress_control: bad argument");
  if (c->tape && !c->tape->dts.empty())  // the reverse pass applies one mask to every step
    fail(FG_ERR_INVALID, "fg_set_stress_control: steps are recorded on the tape");
  c->smask = mask;
  for (int k = 0; k < 9; ++k) c->Pbar[k] = mask ? Pbar[k] : 0.0;
  drop_graphs(*c);
  FG_API_END
}

int fg_tape_begin(fg_ctx* c, int ckpt_every) {
  FG_API_BEGIN
  if (!c || ckpt_every < 1) fail(FG_ERR_INVALID, "fg_tape_begin: bad argument");
  free_tape(*c);
  c->tape = new Tape();
  c->tape->every = ckpt_every;
  FG_API_END
}

int fg_adjoint(fg_ctx* c, int loss, const double* seed_c, const double* seed_F, const double* seed_d,
               double* loss_value, double* grad_logE, double* grad_loggc, double* grad_logD,
               fg_adjoint_stats* st) {
  FG_API_BEGIN
  if (!c) fail(FG_ERR_INVALID, "fg_adjoint: null context");
  if (!c->tape || c->tape->dts.empty()) fail(FG_ERR_INVALID, "fg_adjoint: no recorded steps (fg_tape_begin, fg_step)");
  if (loss != FG_LOSS_CRACK_ENERGY && loss != FG_LOSS_SEEDS) fail(FG_ERR_INVALID, "fg_adjoint: loss");
  fg_adjoint_stats as;
  memset(&as, 0, sizeof(as));
  double v = is_mixed(*c)
                 ? adjoint_impl<float>(*c, c->pf, loss, seed_c, seed_F, seed_d, grad_logE, grad_loggc, grad_logD, &as)
                 : adjoint_impl<double>(*c, c->pd, loss, seed_c, seed_F, seed_d, grad_logE, grad_loggc, grad_logD, &as);
  if (loss_value) *loss_value = v;
  if (st) *st = as;
  FG_API_END
}

int fg_setup(fg_ctx** out, const fg_grid* g, const fg_phase* phases, int nphases,
             const uint8_t* phase_id, const double* cdot_B, const double* c_init,
             const double* log_E, const double* log_D, const double* log_gc,
             const double* log_smax, const fg_opts* opts) {
  FG_API_BEGIN
  if (!out || !g || !phases || nphases <= 0 || nphases > 255 || !phase_id || !cdot_B)
    fail(FG_ERR_INVALID, "fg_setup: null argument or bad phase count");
  *out = nullptr;
  if (g->nx < 2 || g->ny < 1 || g->nz < 1 || g->nx % 2)
    fail(FG_ERR_INVALID, "fg_setup: nx must be even and >= 2, ny, nz >= 1");
  if (!(g->hx > 0 && g->hy > 0 && g->hz > 0)) fail(FG_ERR_INVALID, "fg_setup: voxel size <= 0");
  if (!fg_supported_size(g->nx) || !fg_supported_size(g->ny) || !fg_supported_size(g->nz))
    fail(FG_ERR_INVALID, "fg_setup: transform length not compiled in");
  for (int k = 0; k < nphases; ++k) {
    if (phases[k].law != FG_NEOHOOKE && phases[k].law != FG_SVK)
      fail(FG_ERR_INVALID, "fg_setup: unknown constitutive law");
    if (phases[k].law != phases[0].law)
      fail(FG_ERR_INVALID, "fg_setup: every phase must use the same constitutive law");
    if (!(phases[k].E > 0) || !(phases[k].nu > -1 && phases[k].nu < 0.5) || !(phases[k].D >= 0) ||
        !(phases[k].sigma_max > 0))
      fail(FG_ERR_INVALID, "fg_setup: bad phase constants");
  }
  fg_opts o;
  if (opts) o = *opts;
  else fg_default_opts(&o);
  if (o.precision != FG_FP64 && o.precision != FG_MIXED) fail(FG_ERR_INVALID, "fg_setup: precision");
  if (!(o.gc > 0 && o.lc > 0 && o.RT > 0 && o.cmax > 0)) fail(FG_ERR_INVALID, "fg_setup: gc, lc, RT, cmax");
  if (o.cg_indefinite < 0 || o.cg_indefinite > 2) fail(FG_ERR_INVALID, "fg_setup: cg_indefinite");
  if (o.chem_full_jacobian != 0 && o.chem_full_jacobian != 1) fail(FG_ERR_INVALID, "fg_setup: chem_full_jacobian");
  if (o.l2_prefetch != 0 && o.l2_prefetch != 1) fail(FG_ERR_INVALID, "fg_setup: l2_prefetch");
  if (o.residual_ff != 0 && o.residual_ff != 1) fail(FG_ERR_INVALID, "fg_setup: residual_ff");
  if (o.z_columns != 0 && o.z_columns != 1 && o.z_columns != 4) fail(FG_ERR_INVALID, "fg_setup: z_columns");
  if (o.cluster_pass != 0 && o.cluster_pass != 1) fail(FG_ERR_INVALID, "fg_setup: cluster_pass");
  fg_ctx* c = new fg_ctx();
  try {
    c->law = phases[0].law;
#ifndef FG_EMU
    cudaGetDevice(&c->device);
#endif
    c->nx = g->nx;
    c->ny = g->ny;
    c->nz = g->nz;
    c->hx = g->nx / 2 + 1;
    c->V = (long long)g->nx * g->ny * g->nz;
    c->VH = (long long)c->hx * g->ny * g->nz;
    c->h[0] = g->hx;
    c->h[1] = g->hy;
    c->h[2] = g->hz;
    c->o = o;
    c->l2pf = o.l2_prefetch;
    c->zrows = o.z_columns == 1 ? 1 : (o.z_columns == 4 ? 2 : 0);
    c->st = (cudaStream_t)o.cuda_stream;
    const long long V = c->V;
    // per-voxel material on the host
    std::vector<double> lam(V), mu(V), Om(V), c0(V), D(V), sm(V), cin(V);
    for (long long v = 0; v < V; ++v) {
      const int id = phase_id[v];
      if (id >= nphases) fail(FG_ERR_INVALID, "fg_setup: phase id out of range");
      const fg_phase& p = phases[id];
      double E = p.E;
      if (log_E) E *= exp(log_E[v]);
      lam[v] = E * p.nu / ((1.0 + p.nu) * (1.0 - 2.0 * p.nu));
      mu[v] = E / (2.0 * (1.0 + p.nu));
      Om[v] = p.Omega;
      c0[v] = p.c0;
      D[v] = p.D * (log_D ? exp(log_D[v]) : 1.0);
      sm[v] = p.sigma_max * (log_smax ? exp(log_smax[v]) : 1.0);
      if (!(sm[v] > 0.0 && sm[v] < INFINITY)) fail(FG_ERR_INVALID, "fg_setup: sigma_max(x) not finite and > 0");
      cin[v] = c_init ? c_init[v] : p.c0;
      if (!(cin[v] > 0.0 && cin[v] < 1.0)) fail(FG_ERR_DOMAIN, "fg_setup: initial c outside (0,1)");
    }
    auto up = [&](const std::vector<double>& h) {
      double* d = alloc_n<double>(*c, V);
      dcopy(d, h.data(), V * sizeof(double), c->st);
      return d;
    };
    c->lam = up(lam);
    c->mu_ = up(mu);
    c->Om = up(Om);
    c->c0 = up(c0);
    c->D = up(D);
    c->smax = up(sm);
    c->c = up(cin);
    c->cdotB = alloc_n<double>(*c, V);
    dcopy(c->cdotB, cdot_B, V * sizeof(double), c->st);
    c->F = alloc_n<double>(*c, 9 * V);
    c->Ft = alloc_n<double>(*c, 9 * V);
    c->P = alloc_n<double>(*c, 9 * V);
    c->GP = alloc_n<double>(*c, 9 * V);
    c->Fbk = alloc_n<double>(*c, 9 * V);
    c->dF = alloc_n<double>(*c, 9 * V);
    c->ct = alloc_n<double>(*c, V);
    c->d = alloc_n<double>(*c, V);
    c->dt = alloc_n<double>(*c, V);
    c->H = alloc_n<double>(*c, V);
    c->Ht = alloc_n<double>(*c, V);
    if (log_gc) {
      std::vector<double> g(V);
      for (long long v = 0; v < V; ++v) g[v] = exp(log_gc[v]);
      c->gcr = up(g);
      c->Heff = alloc_n<double>(*c, V);
      dzero(c->Heff, V * sizeof(double), c->st);
    } else {
      c->Heff = c->H;
    }
    c->mu = alloc_n<double>(*c, V);
    c->base = alloc_n<double>(*c, V);
    {
      std::vector<double> F(9 * V, 0.0);
      for (int i = 0; i < 3; ++i)
        for (long long v = 0; v < V; ++v) F[(4 * i) * V + v] = 1.0;
      dcopy(c->F, F.data(), 9 * V * sizeof(double), c->st);
      dzero(c->d, V * sizeof(double), c->st);
      dzero(c->H, V * sizeof(double), c->st);
      dcopy(c->ct, c->c, V * sizeof(double), c->st);
      dzero(c->dt, V * sizeof(double), c->st);
      dzero(c->Ht, V * sizeof(double), c->st);
      dcopy(c->Ft, c->F, 9 * V * sizeof(double), c->st);
    }
    // one partial per block of the largest reducing launch (per-component X passes: 9
    // block rows of at least 2 rows each)
    c->npartials = 9LL * g->ny * g->nz + VEC_BLOCKS + 64;
    c->partials = alloc_n<double>(*c, c->npartials);
    c->ks = alloc_n<KScal>(*c, KS_N);
    dzero(c->ks, KS_N * sizeof(KScal), c->st);
    c->flags = alloc_n<int>(*c, 1);
    dzero(c->flags, sizeof(int), c->st);
    c->ks_host = (KScal*)hpinned(KS_N * sizeof(KScal));
    c->flags_host = (int*)hpinned(sizeof(int));
    {
      // kx planes per Y-Z-Y chunk: a chunk of the 9-component S2 spectrum should take
      // at most l2_fraction of the L2 cache
      double l2 = 64.0 * 1024.0;  // host emulation: a small cache so that tests cover chunking
#ifndef FG_EMU
      l2 = 0.0;
      int dev = 0, bytes = 0;
      cudaGetDevice(&dev);
      if (cudaDeviceGetAttribute(&bytes, cudaDevAttrL2CacheSize, dev) == cudaSuccess) l2 = bytes;
#endif
      const double frac = o.l2_fraction > 0.0 ? o.l2_fraction : 1.0;
      for (int k = 0; k < 2; ++k) {
        const double slab = 9.0 * g->ny * g->nz * (k ? 16.0 : 8.0);
        int ch = (l2 > 0.0 && frac < 1.0) ? (int)(frac * l2 / slab) : c->hx;
        c->kx_chunk[k] = ch < 1 ? 1 : (ch > c->hx ? c->hx : ch);
      }
    }
    // FP64 set with nine-component Krylov vectors in both modes: the mixed mode falls
    // back to it in the mechanical Newton
    setup_prec<double>(*c, c->pd, 9);
    if (o.precision == FG_MIXED) setup_prec<float>(*c, c->pf, 9);
    if (o.precision == FG_MIXED && o.residual_ff) setup_ff(*c);
    c->yzy_cluster = o.precision == FG_MIXED && o.cluster_pass && c->ny == c->nz &&
                     c->pf.oz->yzy_proj && c->pf.oz->yzy_proj_ok();
    c->yzy_cluster_chem = c->yzy_cluster && c->pf.oz->yzy_chem_ok();
    dsync(c->st);
  } catch (...) {
    fg_destroy(c);
    throw;
  }
  *out = c;
  FG_API_END
}

int fg_step(fg_ctx* c, double dt, const double Fbar[9], fg_stats* st) {
  fg_stats s;
  memset(&s, 0, sizeof(s));
  int rc = FG_OK;
  g_err.clear();
  try {
    if (!c || !Fbar || !(dt > 0)) fail(FG_ERR_INVALID, "fg_step: bad argument");
    Tape* T = c->tape;
    const bool ck = T && T->dts.size() % (size_t)T->every == 0;
    if (ck) {  // checkpoint of the state before this step
      double* buf = (double*)dalloc((size_t)12 * c->V * sizeof(double));
      T->ckpt.push_back(buf);
      std::array<double, 9> fb;
      memcpy(fb.data(), c->Fbar, sizeof(c->Fbar));
      T->ckpt_fbar.push_back(fb);
      save_state(*c, buf);
    }
    try {
      if (is_mixed(*c)) step_impl<float>(*c, c->pf, dt, Fbar, s);
      else step_impl<double>(*c, c->pd, dt, Fbar, s);
    } catch (Fail&) {
      if (ck) {
        dfree(T->ckpt.back());
        T->ckpt.pop_back();
        T->ckpt_fbar.pop_back();
      }
      throw;
    }
    if (T) {
      T->dts.push_back(dt);
      std::array<double, 9> fb;
      memcpy(fb.data(), Fbar, sizeof(fb));
      T->fbars.push_back(fb);
    }
  } catch (Fail& f) {
    rc = f.code;
  }
  s.status = rc;
  if (st) *st = s;
  return rc;
}

int fg_residual(fg_ctx* c, double* err_mech, double* err_chem, double* mass_sum) {
  FG_API_BEGIN
  if (!c) fail(FG_ERR_INVALID, "fg_residual: null context");
  if (err_mech) {
    const double den = residual_den(*c);
    *err_mech = residual_mech<double>(*c, den, nullptr);
  }
  if (err_chem) {
    *err_chem = 0.0;
    if (c->stepped) {
      // the last step's chemistry used F_t + (Fbar - Fbar_t), c_t and d_t
      VArgs v = vbase(*c, 9 * c->V);
      v.in[0] = c->Ft;
      v.out[0] = c->P;
      for (int k = 0; k < 9; ++k) v.s[k] = c->Fbar[k] - c->Fbar_prev[k];
      launch_vec<KShiftF>(v, c->st);
      chem_cond<double>(*c, c->pd, c->P, c->ct, c->dt);
      chem_prep<double>(*c, c->pd, c->last_dt, c->P);
      const int nb = op_chem_rhs(*c, c->pd.b, c->last_dt);
      fin<FStore>(*c, KS_MISC, nb, nullptr);
      read_ks(*c);
      const double nf = sqrt(c->ks_host[KS_MISC].aux);
      const double nct = sqrt(reduce_sum(*c, c->ct, c->V, true));
      *err_chem = nf / nct;
    }
  }
  if (mass_sum) *mass_sum = reduce_sum(*c, c->c, c->V, false);
  dsync(c->st);
  FG_API_END
}

int fg_apply(fg_ctx* c, int op, int prec, const void* x, void* y, double dt, double* dot) {
  FG_API_BEGIN
  if (!c || !x || !y) fail(FG_ERR_INVALID, "fg_apply: null argument");
  double d = 0.0;
  if (prec == 0) {
    if (!c->pd.state && (op == FG_OP_MECH)) fail(FG_ERR_INVALID, "fg_apply: FP64 tangent needs an FP64 context");
    if (c->pd.state == nullptr && op != FG_OP_GRES && !c->pd.on) fail(FG_ERR_INVALID, "fg_apply: FP64 operators unavailable");
    d = do_apply<double>(*c, c->pd, op, (const double*)x, (double*)y, dt);
  } else if (prec == 1) {
    if (!c->pf.on) fail(FG_ERR_INVALID, "fg_apply: FP32 operators need a mixed-precision context");
    if (op == FG_OP_GRES) fail(FG_ERR_INVALID, "fg_apply: residual projection is FP64 only");
    d = do_apply<float>(*c, c->pf, op, (const float*)x, (float*)y, dt);
  } else if (prec == 2) {
    if (!c->pe.on) fail(FG_ERR_INVALID, "fg_apply: float-float transforms need a mixed context with residual_ff");
    if (op != FG_OP_GRES) fail(FG_ERR_INVALID, "fg_apply: float-float transforms serve FG_OP_GRES only");
    const int nb = op_gres(*c, c->pe, (const double*)x, (double*)y, nullptr);
    fin<FStore>(*c, KS_MISC, nb, nullptr);
    read_ks(*c);
    d = c->ks_host[KS_MISC].aux;
  } else {
    fail(FG_ERR_INVALID, "fg_apply: prec must be 0, 1 or 2");
  }
  if (dot) *dot = d;
  FG_API_END
}

int fg_get_field(fg_ctx* c, int field, void* dst, int on_device) {
  FG_API_BEGIN
  if (!c || !dst) fail(FG_ERR_INVALID, "fg_get_field: null argument");
  const double* src = nullptr;
  long long n = c->V;
  switch (field) {
    case FG_FIELD_C: src = c->c; break;
    case FG_FIELD_F: src = c->F; n = 9 * c->V; break;
    case FG_FIELD_D: src = c->d; break;
    case FG_FIELD_H: src = c->H; break;
    case FG_FIELD_P:
      mech_state<double>(*c, c->F, nullptr, c->P, nullptr);
      src = c->P;
      n = 9 * c->V;
      break;
    default: fail(FG_ERR_INVALID, "fg_get_field: unknown field");
  }
  (void)on_device;
  dcopy(dst, src, n * sizeof(double), c->st);
  dsync(c->st);
  FG_API_END
}

int fg_displacement(fg_ctx* c, const double* F, const double* Fbar, double* u, int on_device) {
  FG_API_BEGIN
  if (!c || !u || (F == nullptr) != (Fbar == nullptr))
    fail(FG_ERR_INVALID, "fg_displacement: null argument (F and Fbar are given together)");
  (void)on_device;  // host and device pointers are both copied through device scratch
  const long long V = c->V;
  Scratch s;
  const double* Fd = c->F;
  if (F) {
    double* t = s.get(9 * V);
    dcopy(t, F, 9 * V * sizeof(double), c->st);
    Fd = t;
  }
  double* ud = s.get(3 * V);
  disp_fluct(*c, Fd, ud);
  disp_affine(*c, Fbar ? Fbar : c->Fbar, ud);
  dcopy(u, ud, 3 * V * sizeof(double), c->st);
  dsync(c->st);
  FG_API_END
}

int fg_displacement_adjoint(fg_ctx* c, const double* r, double* g, int on_device) {
  FG_API_BEGIN
  if (!c || !r || !g) fail(FG_ERR_INVALID, "fg_displacement_adjoint: null argument");
  (void)on_device;
  const long long V = c->V;
  Scratch s;
  double* rd = s.get(3 * V);
  double* gd = s.get(9 * V);
  dcopy(rd, r, 3 * V * sizeof(double), c->st);
  disp_fluct_adj(*c, rd, gd);
  dcopy(g, gd, 9 * V * sizeof(double), c->st);
  dsync(c->st);
  FG_API_END
}

int fg_set_field(fg_ctx* c, int field, const void* src, int on_device) {
  FG_API_BEGIN
  if (!c || !src) fail(FG_ERR_INVALID, "fg_set_field: null argument");
  if (c->tape && !c->tape->dts.empty())  // the reverse pass recomputes the taped trajectory
    fail(FG_ERR_INVALID, "fg_set_field: steps are recorded on the tape");
  double* dst = nullptr;
  double* dst_t = nullptr;
  long long n = c->V;
  switch (field) {
    case FG_FIELD_C: dst = c->c; dst_t = c->ct; break;
    case FG_FIELD_F: dst = c->F; dst_t = c->Ft; n = 9 * c->V; break;
    case FG_FIELD_D: dst = c->d; dst_t = c->dt; break;
    case FG_FIELD_H: dst = c->H; dst_t = c->Ht; break;
    default: fail(FG_ERR_INVALID, "fg_set_field: unknown or read-only field");
  }
  (void)on_device;
  dcopy(dst, src, n * sizeof(double), c->st);
  dcopy(dst_t, src, n * sizeof(double), c->st);
  if (field == FG_FIELD_H) refresh_heff(*c);
  dsync(c->st);
  FG_API_END
}

int fg_profile(fg_ctx* c, int site, int enable) {
  FG_API_BEGIN
  if (!c || site < 0 || site >= SITE_N - 1) fail(FG_ERR_INVALID, "fg_profile: bad site");
  if (enable) c->prof_mask |= 1u << site;
  else c->prof_mask &= ~(1u << site);
  c->prof_used[site] = 0;
  FG_API_END
}

int fg_profile_read(fg_ctx* c, int site, int* launches, double* total_ms, double* volumes) {
  FG_API_BEGIN
  if (!c || site < 0 || site >= SITE_N - 1 || !launches || !total_ms)
    fail(FG_ERR_INVALID, "fg_profile_read: bad argument");
  double t = 0.0, vol = 0.0;
  int n = 0;
#ifndef FG_EMU
  dsync(c->st);
  std::vector<float> ms(c->prof_used[site]);
  for (int k = 0; k < c->prof_used[site]; ++k)
    cudaEventElapsedTime(&ms[k], c->prof_ev[site][2 * k], c->prof_ev[site][2 * k + 1]);
  // launches that returned at once because their Krylov loop had converged (the tail of
  // the last batch of iterations) are not counted: below a fifth of the median
  std::vector<float> srt(ms);
  std::sort(srt.begin(), srt.end());
  const float med = srt.empty() ? 0.f : srt[srt.size() / 2];
  for (size_t k = 0; k < ms.size(); ++k)
    if (ms[k] >= 0.2f * med) {
      t += ms[k];
      vol += c->prof_frac[site][k];
      ++n;
    }
#endif
  *launches = n;
  *total_ms = t;
  if (volumes) *volumes = vol;
  FG_API_END
}

}  // extern "C"

struct fg_batch {
  std::vector<fg_ctx*> members;
  std::vector<cudaStream_t> own;    // streams created for the members
  std::vector<cudaStream_t> saved;  // the members' streams before the batch
  int threads = 1;
  cudaStream_t apply_st = nullptr;  // grouped operator applications
  std::vector<cudaStream_t> group_st;  // one stream per group, forked from apply_st
  std::vector<cudaEvent_t> group_ev;   // the forks' and joins' events
  void* dargs = nullptr;            // argument tables of the grouped launches (device)
  size_t dargs_bytes = 0;
};

// Grouped operator application over a batch.  Each member's application is recorded
// (launch_recorder: the pass launches it would issue, with their arguments); members whose
// sequences match (same kernels, same grids: equal grids and tuning) form a group, and each
// pass of a group runs as one launch over the group's members, their arguments in a device
// table laid out group by group and launch by launch.
struct GroupPlan {
  std::vector<std::vector<RecordedLaunch>> rec;  // per member
  std::vector<std::vector<int>> groups;          // member indices
  std::vector<char> table;                       // host copy of the argument tables
  std::vector<std::vector<size_t>> off;          // per group and launch: table offset
};

struct RecordScope {  // sets the calling thread's recorder for one scope
  explicit RecordScope(std::vector<RecordedLaunch>* r) { launch_recorder() = r; }
  ~RecordScope() { launch_recorder() = nullptr; }
};
struct FlagScope {  // clears a flag for one scope
  bool& f;
  bool old;
  explicit FlagScope(bool& f_) : f(f_), old(f_) { f = false; }
  ~FlagScope() { f = old; }
};

template <typename R>
static Prec<R>& prec_of(fg_ctx& c) {
  if constexpr (sizeof(R) == 4) return c.pf;
  else return c.pd;
}

// builds every member's tangent state of precision R from its F (as fg_apply does)
template <typename R>
static void batch_prepare(fg_batch& b) {
  for (fg_ctx* c : b.members) {
    Prec<R>& P = prec_of<R>(*c);
    if (!P.state) fail(FG_ERR_INVALID, "batch apply: a member has no tangent state in this precision");
    mech_state<R>(*c, c->F, nullptr, nullptr, P.state);
  }
  for (fg_ctx* c : b.members) dsync(c->st);
}

// The schedule knobs of the autotuner (kx planes per chunk, projection tile, X prefetch):
// they change the launches, not the values an application computes.
struct Knobs {
  int kx[2], zrows, l2pf;
  explicit Knobs(const fg_ctx& c) : kx{c.kx_chunk[0], c.kx_chunk[1]}, zrows(c.zrows), l2pf(c.l2pf) {}
  void put(fg_ctx& c) const {
    c.kx_chunk[0] = kx[0];
    c.kx_chunk[1] = kx[1];
    c.zrows = zrows;
    c.l2pf = l2pf;
  }
};

// records y_i = A_i x_i of every member (mechanical operator, precision R) and groups them;
// members of one grid are recorded with the knobs of the grid's first member, so that
// equal grids give equal launch sequences
template <typename R>
static void batch_plan(fg_batch& b, const void* const* x, void* const* y, GroupPlan& g) {
  const int n = (int)b.members.size();
  g.rec.assign(n, {});
  for (int i = 0; i < n; ++i) {
    fg_ctx& c = *b.members[i];
    int lead = i;
    for (int j = 0; j < i; ++j) {
      const fg_ctx& o = *b.members[j];
      if (o.nx == c.nx && o.ny == c.ny && o.nz == c.nz && o.law == c.law) {
        lead = j;
        break;
      }
    }
    const Knobs own(c);
    Knobs(*b.members[lead]).put(c);
    try {
      FlagScope fs(c.yzy_cluster);  // the clustered pass is not a recorded pass launch
      RecordScope rs(&g.rec[i]);
      op_mech(c, prec_of<R>(c), (const R*)x[i], (R*)y[i], nullptr);
    } catch (...) {
      own.put(c);
      throw;
    }
    own.put(c);
  }
  auto same = [&](int i, int j) {
    if (g.rec[i].size() != g.rec[j].size()) return false;
    for (size_t k = 0; k < g.rec[i].size(); ++k) {
      const RecordedLaunch &p = g.rec[i][k], &q = g.rec[j][k];
      if (p.grouped != q.grouped || p.grid.x != q.grid.x || p.grid.y != q.grid.y ||
          p.grid.z != q.grid.z)
        return false;
    }
    return true;
  };
  g.groups.clear();
  for (int i = 0; i < n; ++i) {
    bool put = false;
    for (auto& gr : g.groups)
      if (same(gr[0], i)) {
        gr.push_back(i);
        put = true;
        break;
      }
    if (!put) g.groups.push_back({i});
  }
  g.table.clear();
  g.off.assign(g.groups.size(), {});
  for (size_t q = 0; q < g.groups.size(); ++q) {
    const std::vector<int>& gr = g.groups[q];
    for (size_t k = 0; k < g.rec[gr[0]].size(); ++k) {
      const size_t at = (g.table.size() + 255) & ~(size_t)255;
      g.table.resize(at);
      g.off[q].push_back(at);
      for (int i : gr) {
        const std::vector<char>& a = g.rec[i][k].args;
        g.table.insert(g.table.end(), a.begin(), a.end());
      }
    }
  }
}

static void batch_stream(fg_batch& b) {
  for (const fg_ctx* c : b.members)
    if (c->device != b.members[0]->device)
      fail(FG_ERR_INVALID, "batch apply: the members live on different devices");
#ifndef FG_EMU
  cudaSetDevice(b.members[0]->device);
  if (!b.apply_st && cudaStreamCreateWithFlags(&b.apply_st, cudaStreamNonBlocking) != cudaSuccess)
    fail(FG_ERR_CUDA, "batch apply: cudaStreamCreate failed");
#endif
}

// copies the argument tables to the device (then waits: the host table is pageable)
static void batch_upload(fg_batch& b, const GroupPlan& g) {
  if (g.table.size() > b.dargs_bytes) {
    dfree(b.dargs);
    b.dargs = nullptr;
    b.dargs_bytes = 0;
    b.dargs = dalloc(g.table.size());
    b.dargs_bytes = g.table.size();
  }
  dcopy(b.dargs, g.table.data(), g.table.size(), b.apply_st);
  dsync(b.apply_st);
}

// one grouped launch per pass and group; the groups run concurrently on streams of their
// own, forked from and joined back into the batch's apply stream
static long long batch_launch(fg_batch& b, const GroupPlan& g) {
  const size_t G = g.groups.size();
#ifndef FG_EMU
  while (b.group_st.size() < G) {
    cudaStream_t s = nullptr;
    cudaEvent_t e = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
      fail(FG_ERR_CUDA, "batch apply: stream or event creation failed");
    b.group_st.push_back(s);
    b.group_ev.push_back(e);
  }
  if (b.group_ev.size() < G + 1) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
      fail(FG_ERR_CUDA, "batch apply: event creation failed");
    b.group_ev.push_back(e);
  }
  cudaEvent_t fork = b.group_ev[G];
  cudaEventRecord(fork, b.apply_st);
#endif
  long long nl = 0;
  for (size_t q = 0; q < G; ++q) {
    cudaStream_t st = b.apply_st;
#ifndef FG_EMU
    st = b.group_st[q];
    cudaStreamWaitEvent(st, fork, 0);
#endif
    const std::vector<RecordedLaunch>& seq = g.rec[g.groups[q][0]];
    for (size_t k = 0; k < seq.size(); ++k, ++nl)
      seq[k].grouped((const char*)b.dargs + g.off[q][k], (int)g.groups[q].size(), seq[k].grid, st);
#ifndef FG_EMU
    cudaEventRecord(b.group_ev[q], st);
    cudaStreamWaitEvent(b.apply_st, b.group_ev[q], 0);
#endif
  }
  return nl;
}

extern "C" {

int fg_batch_setup(fg_batch** out, int n, fg_ctx* const* members) {
  FG_API_BEGIN
  if (!out || n <= 0 || !members) fail(FG_ERR_INVALID, "fg_batch_setup: bad argument");
  for (int i = 0; i < n; ++i)
    if (!members[i]) fail(FG_ERR_INVALID, "fg_batch_setup: null member");
  fg_batch* b = new fg_batch();
  b->members.assign(members, members + n);
  for (int i = 0; i < n; ++i) {
    cudaStream_t s = nullptr;
#ifndef FG_EMU
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(members[i]->device);
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      cudaSetDevice(prev);
      for (size_t k = 0; k < b->own.size(); ++k) {
        b->members[k]->st = b->saved[k];
        cudaStreamDestroy(b->own[k]);
      }
      delete b;
      fail(FG_ERR_CUDA, "fg_batch_setup: cudaStreamCreate failed");
    }
    cudaSetDevice(prev);
#endif
    b->own.push_back(s);
    b->saved.push_back(members[i]->st);
    members[i]->st = s;
  }
  const unsigned hw = std::thread::hardware_concurrency();
  b->threads = (int)std::min<unsigned>(std::max(1u, hw ? hw : 1u), (unsigned)std::min(n, 32));
  *out = b;
  FG_API_END
}

int fg_batch_step(fg_batch* b, double dt, const double Fbar[9], fg_stats* st) {
  if (!b || !Fbar || !(dt > 0)) {
    g_err = "fg_batch_step: bad argument";
    return FG_ERR_INVALID;
  }
  const int n = (int)b->members.size();
  std::vector<int> rc(n, FG_OK);
  std::vector<fg_stats> ss(n);
  std::vector<std::string> msg(n);
  std::atomic<int> next{0};
  auto worker = [&]() {
    for (;;) {
      const int i = next.fetch_add(1);
      if (i >= n) return;
#ifndef FG_EMU
      cudaSetDevice(b->members[i]->device);
#endif
      rc[i] = fg_step(b->members[i], dt, Fbar, &ss[i]);
      msg[i] = g_err;
    }
  };
  std::vector<std::thread> pool;
  for (int t = 0; t < b->threads; ++t) pool.emplace_back(worker);
  for (auto& t : pool) t.join();
  int first = FG_OK;
  for (int i = 0; i < n; ++i) {
    if (st) st[i] = ss[i];
    if (rc[i] != FG_OK && first == FG_OK) {
      first = rc[i];
      g_err = "member " + std::to_string(i) + ": " + msg[i];
    }
  }
  return first;
}

int fg_batch_apply(fg_batch* b, int op, int prec, const void* const* x, void* const* y) {
  FG_API_BEGIN
  if (!b || !x || !y || op != FG_OP_MECH || (prec != 0 && prec != 1))
    fail(FG_ERR_INVALID, "fg_batch_apply: bad argument (FG_OP_MECH, precision 0 or 1)");
  const int n = (int)b->members.size();
  for (int i = 0; i < n; ++i)
    if (!x[i] || !y[i]) fail(FG_ERR_INVALID, "fg_batch_apply: null member vector");
  batch_stream(*b);
  GroupPlan g;
  if (prec == 1) {
    batch_prepare<float>(*b);
    batch_plan<float>(*b, x, y, g);
  } else {
    batch_prepare<double>(*b);
    batch_plan<double>(*b, x, y, g);
  }
  batch_upload(*b, g);
  batch_launch(*b, g);
  dsync(b->apply_st);
  FG_API_END
}

int fg_batch_time_apply(fg_batch* b, int prec, int napply, double ms[4], int info[3]) {
  FG_API_BEGIN
  if (!b || napply <= 0 || !ms || (prec != 0 && prec != 1))
    fail(FG_ERR_INVALID, "fg_batch_time_apply: bad argument");
#ifdef FG_EMU
  fail(FG_ERR_INVALID, "fg_batch_time_apply: needs the GPU build");
#else
  const int n = (int)b->members.size();
  const size_t es = prec == 1 ? sizeof(float) : sizeof(double);
  batch_stream(*b);
  std::vector<void*> xs(n, nullptr), ys(n, nullptr);
  std::vector<cudaEvent_t> ev(n, nullptr);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  auto cleanup = [&]() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (int i = 0; i < n; ++i) {
      if (ev[i]) cudaEventDestroy(ev[i]);
      dfree(xs[i]);
      dfree(ys[i]);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  try {
    for (int i = 0; i < n; ++i) {
      const size_t nb = (size_t)9 * b->members[i]->V * es;
      xs[i] = dalloc(nb);
      ys[i] = dalloc(nb);
      dzero(xs[i], nb, b->apply_st);
      cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    }
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    GroupPlan g;
    if (prec == 1) {
      batch_prepare<float>(*b);
      batch_plan<float>(*b, xs.data(), ys.data(), g);
    } else {
      batch_prepare<double>(*b);
      batch_plan<double>(*b, xs.data(), ys.data(), g);
    }
    batch_upload(*b, g);
    long long per_member = 0;
    for (const auto& r : g.rec) per_member += (long long)r.size();
    auto member_apply = [&](int i) {
      fg_ctx& c = *b->members[i];
      if (prec == 1) op_mech(c, c.pf, (const float*)xs[i], (float*)ys[i], nullptr);
      else op_mech(c, c.pd, (const double*)xs[i], (double*)ys[i], nullptr);
    };
    auto elapsed = [&]() {
      cudaEventRecord(e1, b->apply_st);
      dsync(b->apply_st);
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      return (double)t / napply;
    };
    // warm-up: one grouped application and one per member
    const long long nl = batch_launch(*b, g);
    for (int i = 0; i < n; ++i) member_apply(i);
    for (int i = 0; i < n; ++i) dsync(b->members[i]->st);
    dsync(b->apply_st);
    // (0) the grouped launches captured once as a CUDA graph and replayed
    if (cudaStreamBeginCapture(b->apply_st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      fail(FG_ERR_CUDA, "fg_batch_time_apply: stream capture failed");
    batch_launch(*b, g);
    if (cudaStreamEndCapture(b->apply_st, &graph) != cudaSuccess ||
        cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
      fail(FG_ERR_CUDA, "fg_batch_time_apply: graph capture failed");
    cudaEventRecord(e0, b->apply_st);
    for (int k = 0; k < napply; ++k) cudaGraphLaunch(exec, b->apply_st);
    ms[0] = elapsed();
    // (1) the grouped launches issued one by one
    cudaEventRecord(e0, b->apply_st);
    for (int k = 0; k < napply; ++k) batch_launch(*b, g);
    ms[1] = elapsed();
    // (2) each member's own launches, member after member on one stream
    {
      std::vector<cudaStream_t> keep(n);
      for (int i = 0; i < n; ++i) {
        keep[i] = b->members[i]->st;
        b->members[i]->st = b->apply_st;
      }
      try {
        cudaEventRecord(e0, b->apply_st);
        for (int k = 0; k < napply; ++k)
          for (int i = 0; i < n; ++i) member_apply(i);
        ms[2] = elapsed();
      } catch (...) {
        for (int i = 0; i < n; ++i) b->members[i]->st = keep[i];
        throw;
      }
      for (int i = 0; i < n; ++i) b->members[i]->st = keep[i];
    }
    // (3) each member's own launches on its own stream, all members at once
    cudaEventRecord(e0, b->apply_st);
    for (int i = 0; i < n; ++i) {
      cudaStreamWaitEvent(b->members[i]->st, e0, 0);
      for (int k = 0; k < napply; ++k) member_apply(i);
      cudaEventRecord(ev[i], b->members[i]->st);
      cudaStreamWaitEvent(b->apply_st, ev[i], 0);
    }
    ms[3] = elapsed();
    ccheck("fg_batch_time_apply");
    if (info) {
      info[0] = (int)g.groups.size();
      info[1] = (int)nl;
      info[2] = (int)per_member;
    }
  } catch (...) {
    cleanup();
    throw;
  }
  cleanup();
#endif
  FG_API_END
}

void fg_batch_destroy(fg_batch* b) {
  if (!b) return;
#ifndef FG_EMU
  if (b->apply_st) {
    cudaStreamSynchronize(b->apply_st);
    cudaStreamDestroy(b->apply_st);
  }
  for (cudaStream_t s : b->group_st) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->group_ev) cudaEventDestroy(e);
#endif
  if (b->dargs) dfree(b->dargs);
  for (size_t k = 0; k < b->members.size(); ++k) {
#ifndef FG_EMU
    cudaStreamSynchronize(b->own[k]);
    cudaStreamDestroy(b->own[k]);
#endif
    b->members[k]->st = b->saved[k];
  }
  delete b;
}

int fg_solve_mech(fg_ctx* c, const double Fbar[9], fg_stats* st) {
  fg_stats s;
  memset(&s, 0, sizeof(s));
  int rc = FG_OK;
  g_err.clear();
  try {
    if (!c || !Fbar) fail(FG_ERR_INVALID, "fg_solve_mech: bad argument");
    VArgs v = vbase(*c, 9 * c->V);  // F += Fbar - Fbar_old
    v.in[0] = c->F;
    v.out[0] = c->Fbk;
    for (int k = 0; k < 9; ++k) v.s[k] = Fbar[k] - c->Fbar[k];
    launch_vec<KShiftF>(v, c->st);
    dcopy(c->F, c->Fbk, 9 * c->V * sizeof(double), c->st);
    memcpy(c->Fbar, Fbar, sizeof(c->Fbar));
    const double den = residual_den(*c);
    if (is_mixed(*c)) mech_newton<float>(*c, c->pf, den, s);
    else mech_newton<double>(*c, c->pd, den, s);
    dsync(c->st);
  } catch (Fail& f) {
    rc = f.code;
  }
  s.status = rc;
  if (st) *st = s;
  return rc;
}

int fg_adjoint_mech(fg_ctx* c, const double* W, double* grad_logE, int* iters) {
  FG_API_BEGIN
  if (!c || !W || !grad_logE) fail(FG_ERR_INVALID, "fg_adjoint_mech: null argument");
  fg_stats s;
  memset(&s, 0, sizeof(s));
  const long long V = c->V;
  dcopy(c->P, W, 9 * V * sizeof(double), c->st);  // W -> device (P is scratch here)
  op_gres(*c, c->pd, c->P, c->GP, nullptr);        // G W
  int n = 0;
  auto run = [&](auto& P) {
    using R = typename std::remove_reference<decltype(*P.x)>::type;
    to_prec<R>(*c, c->GP, P.b, 9 * V, 1.0);
    mech_state<R>(*c, c->F, nullptr, c->P, P.state);  // tangent and stress at the solution
    n = cg_solve_mech<R>(*c, P, mixed_tol(*c, c->o.tol_cg), c->o.max_cg, nullptr);
    VArgs v = vbase(*c, V);
    v.in[0] = P.x;
    v.in[1] = c->P;
    v.out[0] = c->base;
    launch_vec<KAdjGradE<R>>(v, c->st);
  };
  if (is_mixed(*c)) run(c->pf);
  else run(c->pd);
  read_ks(*c);
  check_flags(*c, "adjoint");
  dcopy(grad_logE, c->base, V * sizeof(double), c->st);
  dsync(c->st);
  if (iters) *iters = n;
  FG_API_END
}

// Times the schedule choices of the mechanical CG that are selectable at run time and
// keeps the fastest: kx planes per Y-Z-Y chunk (whole volume, 40 % or 15 % of L2) and the
// per-component or 9-component X-inv update.
int fg_autotune(fg_ctx* c, double* ms_per_iteration) {
  FG_API_BEGIN
  if (!c) fail(FG_ERR_INVALID, "fg_autotune: null context");
  drop_graphs(*c);
#ifdef FG_EMU
  if (ms_per_iteration) *ms_per_iteration = 0.0;
#else
  const bool mixed = is_mixed(*c);
  const int k = mixed ? 0 : 1;
  const size_t es = mixed ? sizeof(float) : sizeof(double);
  int dev = 0, l2b = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&l2b, cudaDevAttrL2CacheSize, dev);
  const double slab = 9.0 * c->ny * c->nz * (mixed ? 8.0 : 16.0);
  std::vector<int> chunks = {c->hx};
  for (double f : {0.4, 0.15}) {
    int ch = (int)(f * l2b / slab);
    ch = ch < 1 ? 1 : (ch > c->hx ? c->hx : ch);
    if (std::find(chunks.begin(), chunks.end(), ch) == chunks.end()) chunks.push_back(ch);
  }
  void* x = dalloc(9 * c->V * es);
  void* y = dalloc(9 * c->V * es);
  dzero(x, 9 * c->V * es, c->st);
  if (mixed) mech_state<float>(*c, c->F, nullptr, nullptr, c->pf.state);
  else mech_state<double>(*c, c->F, nullptr, nullptr, c->pd.state);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto time_it = [&](auto&& f, int reps) {
    for (int i = 0; i < 2; ++i) f();
    cudaEventRecord(e0, c->st);
    for (int i = 0; i < reps; ++i) f();
    cudaEventRecord(e1, c->st);
    cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    return (double)t / reps;
  };
  double best = 1e300;
  int best_ch = c->kx_chunk[k];
  c->l2pf = 0;
  c->yzy_cluster = false;
  c->yzy_cluster_chem = false;
  for (int ch : chunks) {
    c->kx_chunk[k] = ch;
    const double t = mixed ? time_it([&] { op_mech(*c, c->pf, (const float*)x, (float*)y, nullptr); }, 5)
                           : time_it([&] { op_mech(*c, c->pd, (const double*)x, (double*)y, nullptr); }, 3);
    if (t < best) {
      best = t;
      best_ch = ch;
    }
  }
  c->kx_chunk[k] = best_ch;
  if (mixed) {  // tile shapes of the FP32 projection pass
    int best_z = 0;
    for (int zr = 1; zr <= 2; ++zr) {
      if (!c->pf.oz->z_proj_rows[zr - 1]) continue;
      c->zrows = zr;
      const double t = time_it([&] { op_mech(*c, c->pf, (const float*)x, (float*)y, nullptr); }, 5);
      if (t < best) {
        best = t;
        best_z = zr;
      }
    }
    c->zrows = best_z;
    const bool can_cluster = c->o.cluster_pass && c->ny == c->nz && c->pf.oz->yzy_proj &&
                             c->pf.oz->yzy_proj_ok();
    if (can_cluster) {  // the clustered Y-Z-Y pass against the best separate passes
      c->yzy_cluster = true;
      const double t = time_it([&] { op_mech(*c, c->pf, (const float*)x, (float*)y, nullptr); }, 5);
      c->yzy_cluster = t < best;
      if (t < best) best = t;
      // the chemistry chains, timed on the chemistry operator's transforms
      if (c->pf.oz->yzy_chem_ok()) {
        const float* xf = (const float*)x;
        double tc[2];
        for (int on = 0; on < 2; ++on) {
          c->yzy_cluster_chem = on != 0;
          tc[on] = time_it([&] { op_chem_L(*c, c->pf, xf, nullptr); }, 5);
        }
        c->yzy_cluster_chem = tc[1] < tc[0];
      }
    }
  }
  // X-inv update variants (alpha read from a zeroed scalar: x and r are unchanged)
  double* zero = (double*)dalloc(4 * sizeof(double));
  dzero(zero, 4 * sizeof(double), c->st);
  double tv[2][2];
  for (int pf = 0; pf < 2; ++pf)
  for (int pc = 0; pc < 2; ++pc) {
    auto run = [&]() {
      if (mixed) {
        PassArgs<float> a = pbase(*c, c->pf, nullptr);
        a.tw = c->pf.twx;
        a.cin = c->pf.S1;
        a.rout = (float*)y;
        a.rout2 = (float*)x;
        a.aux[0] = (const float*)x;
        a.dscal = zero;
        a.l2pf = pf;
        (pc ? c->pf.ox->xi_cgupdate_pc : c->pf.ox->xi_cgupdate)(a, c->st);
      } else {
        PassArgs<double> a = pbase(*c, c->pd, nullptr);
        a.tw = c->pd.twx;
        a.cin = c->pd.S1;
        a.rout = (double*)y;
        a.rout2 = (double*)x;
        a.aux[0] = (const double*)x;
        a.dscal = zero;
        a.l2pf = pf;
        (pc ? c->pd.ox->xi_cgupdate_pc : c->pd.ox->xi_cgupdate)(a, c->st);
      }
    };
    tv[pf][pc] = time_it(run, 5);
  }
  // the forward X pass of the CG with and without prefetch; the prefetch choice is made
  // on the pair of X passes of a CG iteration, which dominate the step
  double tf[2];
  for (int pf = 0; pf < 2; ++pf) {
    auto run = [&]() {
      if (mixed) {
        PassArgs<float> a = pbase(*c, c->pf, nullptr);
        a.tw = c->pf.twx;
        a.rin = (const float*)x;
        a.rout = (float*)y;
        a.aux[0] = c->pf.state;
        a.dscal = zero;
        a.cout = c->pf.S1;
        a.l2pf = pf;
        (c->law == FG_SVK ? c->pf.ox->xf_cgtangent_svk : c->pf.ox->xf_cgtangent)(a, c->st);
      } else {
        PassArgs<double> a = pbase(*c, c->pd, nullptr);
        a.tw = c->pd.twx;
        a.rin = (const double*)x;
        a.rout = (double*)y;
        a.aux[0] = c->pd.state;
        a.dscal = zero;
        a.cout = c->pd.S1;
        a.l2pf = pf;
        (c->law == FG_SVK ? c->pd.ox->xf_cgtangent_svk : c->pd.ox->xf_cgtangent)(a, c->st);
      }
    };
    tf[pf] = time_it(run, 5);
  }
  const double t0 = tf[0] + std::min(tv[0][0], tv[0][1]);
  const double t1 = tf[1] + std::min(tv[1][0], tv[1][1]);
  c->l2pf = t1 < t0 ? 1 : 0;
  c->xi_percomp = tv[c->l2pf][1] <= tv[c->l2pf][0] ? 1 : 0;
  c->tune_ms[0] = tv[0][0];
  c->tune_ms[1] = tv[0][1];
  c->tune_ms[2] = tv[1][0];
  c->tune_ms[3] = tv[1][1];
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  dsync(c->st);
  dfree(zero);
  dfree(x);
  dfree(y);
  ccheck("fg_autotune");
  if (ms_per_iteration) *ms_per_iteration = best;
#endif
  FG_API_END
}

int fg_autotune_report(fg_ctx* c, int choice[5], double xinv_ms[4]) {
  FG_API_BEGIN
  if (!c || !choice) fail(FG_ERR_INVALID, "fg_autotune_report: bad argument");
  choice[0] = c->kx_chunk[is_mixed(*c) ? 0 : 1];
  choice[1] = c->xi_percomp;
  choice[2] = c->l2pf;
  choice[3] = c->zrows == 1 ? 1 : (c->zrows == 2 ? 4 : 0);
  choice[4] = (c->yzy_cluster ? 1 : 0) + (c->yzy_cluster_chem ? 2 : 0);
  if (xinv_ms)
    for (int k = 0; k < 4; ++k) xinv_ms[k] = c->tune_ms[k];
  FG_API_END
}

int fg_time_apply(fg_ctx* c, int op, int prec, int n, double* ms) {
  FG_API_BEGIN
  if (!c || n <= 0 || !ms) fail(FG_ERR_INVALID, "fg_time_apply: bad argument");
#ifdef FG_EMU
  fail(FG_ERR_INVALID, "fg_time_apply: needs the GPU build");
#else
  const long long nel = (op == FG_OP_MECH || op == FG_OP_GRES) ? 9 * c->V : c->V;
  if (prec == 2 && (op != FG_OP_GRES || !c->pe.on))
    fail(FG_ERR_INVALID, "fg_time_apply: float-float transforms serve FG_OP_GRES of a mixed context");
  const size_t es = prec == 1 ? sizeof(float) : sizeof(double);
  void* x = dalloc(nel * es);
  void* y = dalloc(nel * es);
  dzero(x, nel * es, c->st);
  // prepare the operator state once with a first application
  double dummy = 0.0;
  if (prec == 0) dummy = do_apply<double>(*c, c->pd, op, (const double*)x, (double*)y, 1.0);
  else if (prec == 1) dummy = do_apply<float>(*c, c->pf, op, (const float*)x, (float*)y, 1.0);
  else op_gres(*c, c->pe, (const double*)x, (double*)y, nullptr);
  (void)dummy;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, c->st);
  for (int i = 0; i < n; ++i) {
    if (prec == 2) {
      op_gres(*c, c->pe, (const double*)x, (double*)y, nullptr);
    } else if (prec == 0) {
      Prec<double>& P = c->pd;
      switch (op) {
        case FG_OP_MECH: op_mech(*c, P, (const double*)x, (double*)y, nullptr); break;
        case FG_OP_GRES: op_gres(*c, P, (const double*)x, (double*)y, nullptr); break;
        case FG_OP_PFF: op_pff(*c, P, (const double*)x, (double*)y, (const double*)c->Heff, nullptr); break;
        case FG_OP_PFF_PREC: op_prec(*c, P, (const double*)x, (double*)y, nullptr); break;
        case FG_OP_CHEM: op_chem(*c, P, (const double*)x, (double*)y, 1.0, nullptr); break;
      }
    } else {
      Prec<float>& P = c->pf;
      switch (op) {
        case FG_OP_MECH: op_mech(*c, P, (const float*)x, (float*)y, nullptr); break;
        case FG_OP_PFF: op_pff(*c, P, (const float*)x, (float*)y, (const float*)P.Hr, nullptr); break;
        case FG_OP_PFF_PREC: op_prec(*c, P, (const float*)x, (float*)y, nullptr); break;
        case FG_OP_CHEM: op_chem(*c, P, (const float*)x, (float*)y, 1.0, nullptr); break;
      }
    }
  }
  cudaEventRecord(e1, c->st);
  cudaEventSynchronize(e1);
  float t = 0.f;
  cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  dfree(x);
  dfree(y);
  ccheck("fg_time_apply");
  *ms = (double)t / n;
#endif
  FG_API_END
}

#ifdef FG_EMU
// Test hook of the host emulation only (not part of the C ABI): writes one byte at
// `offset` from the start of a fresh guarded 64-byte buffer and frees it.  An offset
// outside [0, 64) must fault (past the end by default; below zero under
// FG_EMU_GUARD=start), which the tests observe in a child process.
int fg_emu_guard_probe(long long offset) {
  volatile char* p = (volatile char*)fg::dalloc(64);
  p[offset] = 1;
  fg::dfree((void*)p);
  return 0;
}
#endif

}  // extern "C"
