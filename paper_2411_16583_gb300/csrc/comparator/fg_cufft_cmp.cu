// Timed comparator of the fused mechanical operator: the same FP32 application
// y = F^-1[ G : F[ K(F, c, d) : x ] ] (Eq. mechanicalsolve) built the conventional way,
// from cuFFT's batched 3D real transforms (one plan over the nine components) and two
// separate element-wise kernels, the Neo-Hookean tangent in real space and the
// compatibility projection G in frequency space.  Each stage makes its own passes over
// HBM.  It is a benchmark baseline only (its own shared library, libfg_cufft.so, loaded by
// bench.py); the solver never calls it.
#include <cmath>
#include <string>
#include <vector>

#include <cufft.h>

#include "../fg_pointwise.cuh"

namespace fg {
// this library keeps its own launch counter, hidden from the solver library's
std::atomic<long long>& launch_counter() {
  static std::atomic<long long> n{0};
  return n;
}
}  // namespace fg

namespace {

using fg::VArgs;

std::string g_msg;

// tau = K : x per voxel from the packed Neo-Hookean state (B = F_e^-T, s1, s2, s3)
__global__ void k_tangent(const float* __restrict__ x, const float* __restrict__ st,
                          float* __restrict__ tau, long long V) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V;
       v += (long long)gridDim.x * blockDim.x) {
    float p[9], B[9], t[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) p[k] = x[k * V + v];
#pragma unroll
    for (int k = 0; k < 9; ++k) B[k] = st[k * V + v];
    fg::tangent_nh(B, st[9 * V + v], st[10 * V + v], st[11 * V + v], p, t);
#pragma unroll
    for (int k = 0; k < 9; ++k) tau[k * V + v] = t[k];
  }
}

// G on the half spectrum, layout [c][kz][ky][kx] (cuFFT's R2C output), with the rotated
// scheme n_j = rs_j(k_j) prod_{m != j} rc_m(k_m) and the 1/V of the inverse transform
__global__ void k_project(cufftComplex* __restrict__ A, const float* __restrict__ tab, int nx,
                          int ny, int nz, int tabn, float invV) {
  const int hx = nx / 2 + 1;
  const long long VH = (long long)hx * ny * nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < VH;
       i += (long long)gridDim.x * blockDim.x) {
    const int kx = (int)(i % hx);
    const int ky = (int)((i / hx) % ny);
    const int kz = (int)(i / ((long long)hx * ny));
    const float sx = tab[0 * tabn + kx], sy = tab[1 * tabn + ky], sz = tab[2 * tabn + kz];
    const float cx = tab[3 * tabn + kx], cy = tab[4 * tabn + ky], cz = tab[5 * tabn + kz];
    const float n0 = sx * cy * cz, n1 = sy * cx * cz, n2 = sz * cx * cy;
    const float nn = n0 * n0 + n1 * n1 + n2 * n2;
    const float s = nn > 0.f ? invV / nn : 0.f;
    cufftComplex v[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) v[k] = A[k * VH + i];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float tx = (v[3 * r].x * n0 + v[3 * r + 1].x * n1 + v[3 * r + 2].x * n2) * s;
      const float ty = (v[3 * r].y * n0 + v[3 * r + 1].y * n1 + v[3 * r + 2].y * n2) * s;
      A[(3 * r) * VH + i] = make_float2(tx * n0, ty * n0);
      A[(3 * r + 1) * VH + i] = make_float2(tx * n1, ty * n1);
      A[(3 * r + 2) * VH + i] = make_float2(tx * n2, ty * n2);
    }
  }
}

int fail(const std::string& m) {
  g_msg = m;
  return -1;
}

}  // namespace

#define FGC_API extern "C" __attribute__((visibility("default")))

FGC_API const char* fgc_last_error(void) { return g_msg.c_str(); }

// Builds the packed tangent state of (F, c, d) (device FP64 arrays, V or 9 V entries),
// applies the operator `reps` times to x (9 V floats) into y, and returns the mean time per
// application in *ms (CUDA events on `stream`).  Allocates and frees its own work space
// and cuFFT plans.  Returns 0, or -1 with a message in fgc_last_error().
FGC_API int fgc_mech_apply(int nx, int ny, int nz, double hx, double hy, double hz,
                           const double* F, const double* c, const double* d, const double* lam,
                           const double* mu, const double* Omega, const double* c0,
                           const float* x, float* y, int reps, float* ms, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const long long V = (long long)nx * ny * nz;
  const int hxn = nx / 2 + 1;
  const long long VH = (long long)hxn * ny * nz;
  const int tabn = std::max(nx, std::max(ny, nz));
  float* state = nullptr;
  float* tau = nullptr;
  cufftComplex* spec = nullptr;
  float* tab = nullptr;
  int* flags = nullptr;
  cufftHandle fwd = 0, inv = 0;
  bool have_fwd = false, have_inv = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = 0;
  auto ok = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && rc == 0) rc = fail(std::string(what) + ": " + cudaGetErrorString(e));
    return rc == 0;
  };
  if (reps < 1 || nx < 2 || nx % 2) return fail("fgc_mech_apply: bad argument");
  if (ok(cudaMalloc(&state, 12 * V * sizeof(float)), "cudaMalloc") &&
      ok(cudaMalloc(&tau, 9 * V * sizeof(float)), "cudaMalloc") &&
      ok(cudaMalloc(&spec, 9 * VH * sizeof(cufftComplex)), "cudaMalloc") &&
      ok(cudaMalloc(&tab, 6 * tabn * sizeof(float)), "cudaMalloc") &&
      ok(cudaMalloc(&flags, sizeof(int)), "cudaMalloc") &&
      ok(cudaMemsetAsync(flags, 0, sizeof(int), st), "cudaMemsetAsync")) {
    // per-axis tables of the rotated scheme, in FP64 on the host and rounded
    const int n[3] = {nx, ny, nz};
    const int len[3] = {hxn, ny, nz};
    const double h[3] = {hx, hy, hz};
    std::vector<float> ht(6 * tabn, 0.f);
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < len[j]; ++k) {
        const int ks = (j > 0 && 2 * k > n[j]) ? k - n[j] : k;
        const double th = M_PI * (double)ks / (double)n[j];
        ht[j * tabn + k] = (float)(2.0 / h[j] * std::sin(th));
        ht[(3 + j) * tabn + k] = (float)((2 * std::abs(ks) == n[j]) ? 0.0 : std::cos(th));
      }
    ok(cudaMemcpyAsync(tab, ht.data(), ht.size() * sizeof(float), cudaMemcpyHostToDevice, st),
       "cudaMemcpyAsync");
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
    v.flags = flags;
    if (rc == 0) fg::launch_vec<fg::KMechState<float>>(v, st);
    int dims[3] = {nz, ny, nx};
    if (rc == 0) {
      if (cufftPlanMany(&fwd, 3, dims, nullptr, 1, (int)V, nullptr, 1, (int)VH, CUFFT_R2C, 9) !=
          CUFFT_SUCCESS)
        rc = fail("cufftPlanMany (R2C) failed");
      else
        have_fwd = true;
    }
    if (rc == 0) {
      if (cufftPlanMany(&inv, 3, dims, nullptr, 1, (int)VH, nullptr, 1, (int)V, CUFFT_C2R, 9) !=
          CUFFT_SUCCESS)
        rc = fail("cufftPlanMany (C2R) failed");
      else
        have_inv = true;
    }
    if (rc == 0 && (cufftSetStream(fwd, st) != CUFFT_SUCCESS || cufftSetStream(inv, st) != CUFFT_SUCCESS))
      rc = fail("cufftSetStream failed");
    const int blocks = 4 * 152;
    auto apply = [&]() {
      k_tangent<<<blocks, 256, 0, st>>>(x, state, tau, V);
      if (cufftExecR2C(fwd, tau, spec) != CUFFT_SUCCESS) return false;
      k_project<<<blocks, 256, 0, st>>>(spec, tab, nx, ny, nz, tabn, (float)(1.0 / (double)V));
      return cufftExecC2R(inv, spec, y) == CUFFT_SUCCESS;
    };
    if (rc == 0 && !apply()) rc = fail("cuFFT execution failed");
    if (rc == 0 && ok(cudaEventCreate(&e0), "cudaEventCreate") &&
        ok(cudaEventCreate(&e1), "cudaEventCreate") &&
        ok(cudaEventRecord(e0, st), "cudaEventRecord")) {
      for (int r = 0; r < reps && rc == 0; ++r)
        if (!apply()) rc = fail("cuFFT execution failed");
      if (ok(cudaEventRecord(e1, st), "cudaEventRecord") &&
          ok(cudaEventSynchronize(e1), "cudaEventSynchronize")) {
        float t = 0.f;
        ok(cudaEventElapsedTime(&t, e0, e1), "cudaEventElapsedTime");
        if (ms) *ms = t / (float)reps;
      }
    }
    int hflags = 0;
    if (ok(cudaMemcpy(&hflags, flags, sizeof(int), cudaMemcpyDeviceToHost), "cudaMemcpy") && hflags)
      rc = fail("fgc_mech_apply: det F <= 0 or J_c <= 0");
    ok(cudaGetLastError(), "kernel launch");
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (have_fwd) cufftDestroy(fwd);
  if (have_inv) cufftDestroy(inv);
  cudaFree(state);
  cudaFree(tau);
  cudaFree(spec);
  cudaFree(tab);
  cudaFree(flags);
  return rc;
}
