// C-ABI plumbing: error reporting, default options and the batched operator apply.
#include <stdio.h>
#include <string.h>

#include <math.h>

#include <atomic>
#include <vector>
#include <string>

#include "kernels.cuh"

namespace cbs {

static thread_local std::string g_err;
static std::atomic<uint64_t> g_launches{0};
// launches counted by the calling thread: what a graph capture brackets, exact also while
// other threads (cbs_solve_cells) count their own
static thread_local uint64_t t_launches = 0;

void count_launches(uint64_t n) {
  g_launches.fetch_add(n, std::memory_order_relaxed);
  t_launches += n;
}
void uncount_launches(uint64_t n) {
  g_launches.fetch_sub(n, std::memory_order_relaxed);
  t_launches -= n;
}
uint64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }
uint64_t thread_launches() { return t_launches; }

void set_error(const std::string &msg) { g_err = msg; }

cbs_status cuda_fail(cudaError_t e, const char *what) {
  g_err = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return CBS_ECUDA;
}

}  // namespace cbs

using namespace cbs;

extern "C" const char *cbs_last_error(void) { return g_err.c_str(); }

extern "C" uint64_t cbs_kernel_launches(void) { return launches_so_far(); }

extern "C" cbs_status cbs_options_default(cbs_options *o) {
  if (!o) return CBS_EINVAL;
  memset(o, 0, sizeof(*o));
  o->tol = 1e-10;
  o->delta = 1e-10;
  o->rho_max = 1e-8;
  o->max_iter = 20000;
  o->precision = CBS_FP64;
  o->extraction = CBS_HANKEL;
  o->check_every = 8;
  o->inner_tol = 0.1;
  o->max_sweeps = 200;
  o->inner_max_iter = 1000;
  o->stall_sweeps = 12;
  o->energies_per_batch = 0;
  o->multi_shift = 0;
  o->stream = nullptr;
  o->family_tol = 0.0;
  o->stop_fraction = 1.0;
  o->points_per_wave = 0;
  o->conj_points = 1;
  return CBS_OK;
}

extern "C" cbs_status cbs_apply(const cbs_hamiltonian *h, int n_sys, const double *z, const double *E,
                                int L, const void *X, void *Y, int dtype, void *stream) {
  if (!h || !z || !E || !X || !Y || n_sys < 1 || L < 1 || L > 512) {
    set_error("cbs_apply: bad argument (need n_sys >= 1, 1 <= L <= 512, non-null pointers)");
    return CBS_EINVAL;
  }
  if (dtype != CBS_C128 && dtype != CBS_C64) { set_error("cbs_apply: dtype"); return CBS_EINVAL; }
  if (!apply_supported(h->v, L, dtype, "cbs_apply")) return CBS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const HamView &H = h->v;
  const size_t csz = dtype == CBS_C128 ? sizeof(double2) : sizeof(float2);
  const size_t dbytes = (size_t)n_sys * (H.n_atoms ? H.n_atoms : 1) * H.np4 * L * csz;
  void *scratch = nullptr;
  const size_t sys_bytes = (size_t)n_sys * (sizeof(double2) + sizeof(double));
  CBS_CUDA(cudaMalloc(&scratch, dbytes + sys_bytes + 256));
  double2 *tw = (double2 *)scratch;
  double *Ed = (double *)(tw + n_sys);
  void *D = (char *)scratch + ((sys_bytes + 255) & ~(size_t)255);
  cbs_status s = CBS_OK;
  cudaError_t e = cudaMemcpyAsync(tw, z, (size_t)n_sys * sizeof(double2), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(Ed, E, (size_t)n_sys * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) s = cuda_fail(e, "cbs_apply upload");
  if (s == CBS_OK) {
    if (dtype == CBS_C128)
      s = apply_P<double>(H, n_sys, L, (const double2 *)X, (double2 *)Y, tw, false, Ed, (double2 *)D,
                          nullptr, st);
    else
      s = apply_P<float>(H, n_sys, L, (const float2 *)X, (float2 *)Y, tw, false, Ed, (float2 *)D,
                         nullptr, st);
  }
  // the scratch must outlive the kernels: synchronise the stream before freeing it
  cudaError_t e2 = cudaStreamSynchronize(st);
  cudaFree(scratch);
  if (s == CBS_OK && e2 != cudaSuccess) s = cuda_fail(e2, "cbs_apply");
  return s;
}

extern "C" size_t cbs_apply_workspace_size(const cbs_hamiltonian *h, int n_sys, int L, int dtype) {
  if (!h || n_sys < 1 || L < 1) return 0;
  const HamView &H = h->v;
  const size_t csz = dtype == CBS_C128 ? sizeof(double2) : sizeof(float2);
  return (size_t)n_sys * (H.n_atoms ? H.n_atoms : 1) * H.np4 * L * csz;
}

extern "C" cbs_status cbs_apply_ws(const cbs_hamiltonian *h, int n_sys, const double *z, const double *E,
                                   int L, const void *X, void *Y, int dtype, void *workspace,
                                   size_t workspace_bytes, void *stream) {
  if (!h || !z || !E || !X || !Y || !workspace || n_sys < 1 || L < 1 || L > 512) {
    set_error("cbs_apply_ws: bad argument (need n_sys >= 1, 1 <= L <= 512, non-null pointers)");
    return CBS_EINVAL;
  }
  if (dtype != CBS_C128 && dtype != CBS_C64) { set_error("cbs_apply_ws: dtype"); return CBS_EINVAL; }
  if (!apply_supported(h->v, L, dtype, "cbs_apply_ws")) return CBS_EINVAL;
  if (workspace_bytes < cbs_apply_workspace_size(h, n_sys, L, dtype)) {
    set_error("cbs_apply_ws: workspace smaller than cbs_apply_workspace_size");
    return CBS_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const HamView &H = h->v;
  if (dtype == CBS_C128)
    return apply_P<double>(H, n_sys, L, (const double2 *)X, (double2 *)Y, (const double2 *)z, false, E,
                           (double2 *)workspace, nullptr, st);
  return apply_P<float>(H, n_sys, L, (const float2 *)X, (float2 *)Y, (const double2 *)z, false, E,
                        (float2 *)workspace, nullptr, st);
}

// Launch-shape search for the stencil kernel: every admissible (kernel, x-lines per block)
// is timed with CUDA events on `stream` over a few applies of n_sys systems, and the
// fastest is stored in the handle, where every later apply of that precision uses it.
extern "C" cbs_status cbs_autotune_apply(cbs_hamiltonian *h, int n_sys, int L, int dtype,
                                         void *stream, int *best_py, int *best_pz, int *best_x2,
                                         float *best_ms) {
  if (!h || n_sys < 1 || L < 1 || L > 512) {
    set_error("cbs_autotune_apply: bad argument (need n_sys >= 1, 1 <= L <= 512)");
    return CBS_EINVAL;
  }
  if (dtype != CBS_C128 && dtype != CBS_C64) { set_error("cbs_autotune_apply: dtype"); return CBS_EINVAL; }
  if (dtype == CBS_C128 && L > 256) { set_error("cbs_autotune_apply: complex128 needs L <= 256"); return CBS_EINVAL; }
  HamView &H = h->v;
  const int ti = dtype == CBS_C64 ? 1 : 0;
  const size_t csz = dtype == CBS_C128 ? sizeof(double2) : sizeof(float2);
  const size_t vec = (size_t)n_sys * H.n * L * csz;
  const size_t ws = cbs_apply_workspace_size(h, n_sys, L, dtype);
  const size_t sys_bytes = (size_t)n_sys * (sizeof(double2) + sizeof(double));
  cudaStream_t st = (cudaStream_t)stream;
  char *buf = nullptr;
  const size_t a = (vec + 255) & ~(size_t)255, b = (ws + 255) & ~(size_t)255;
  CBS_CUDA(cudaMalloc(&buf, 2 * a + b + sys_bytes + 256));
  void *X = buf, *Y = buf + a, *D = buf + 2 * a;
  double2 *tw = (double2 *)(buf + 2 * a + b);
  double *Ed = (double *)(tw + n_sys);
  std::vector<double2> hz(n_sys);
  std::vector<double> hE(n_sys, 0.1);
  for (int i = 0; i < n_sys; ++i) {
    const double r = (i % 2) ? 0.5 : 2.0, th = 2.0 * 3.141592653589793 * (i + 0.5) / n_sys;
    hz[i] = make_double2(r * cos(th), r * sin(th));
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cbs_status s = CBS_OK;
  const int keep_py = H.tune_py[ti], keep_pz = H.tune_pz[ti], keep_x2 = H.tune_x2;
  int bp = 0, bz = 0, bx = 0;
  float bms = 0.f;
  auto run = [&]() -> cbs_status {
    if (dtype == CBS_C128)
      return apply_P<double>(H, n_sys, L, (const double2 *)X, (double2 *)Y, tw, false, Ed, (double2 *)D,
                             nullptr, st);
    return apply_P<float>(H, n_sys, L, (const float2 *)X, (float2 *)Y, tw, false, Ed, (float2 *)D,
                          nullptr, st);
  };
  do {
    cudaError_t e = cudaMemsetAsync(X, 0, vec, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tw, hz.data(), n_sys * sizeof(double2), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(Ed, hE.data(), n_sys * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) { s = cuda_fail(e, "cbs_autotune_apply setup"); break; }
    const bool x2_ok = ti == 1 && L % 2 == 0 && H.np4 == 4;
    // complex64 kernels: two columns per thread (1) or one (-1)
    const int variants[2] = {1, -1};
    for (int vi = 0; vi < (x2_ok ? 2 : 1) && s == CBS_OK; ++vi) {
      const int x2 = x2_ok ? variants[vi] : 0;
      const int per_line = (x2_ok && x2 == 1) ? L / 2 : L;
      // the two-columns-per-thread kernel also comes in a 512-thread variant
      const int max_threads = (x2_ok && x2 == 1) ? 512 : 256;
      for (int py = 1; py * per_line <= max_threads && py <= 32 && s == CBS_OK; py *= 2)
      for (int pz = 1; py * pz * per_line <= max_threads && pz <= 16 && s == CBS_OK; pz *= 2) {
        H.tune_py[ti] = py;
        H.tune_pz[ti] = pz;
        H.tune_x2 = x2;
        for (int w = 0; w < 2 && s == CBS_OK; ++w) s = run();
        if (s != CBS_OK) break;
        const int reps = 5;
        e = cudaEventRecord(e0, st);
        for (int r = 0; r < reps && s == CBS_OK && e == cudaSuccess; ++r) s = run();
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) { s = cuda_fail(e, "cbs_autotune_apply timing"); break; }
        ms /= reps;
        if (bp == 0 || ms < bms) { bp = py; bz = pz; bx = x2; bms = ms; }
      }
    }
  } while (0);
  cudaStreamSynchronize(st);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  if (s != CBS_OK || bp == 0) {
    H.tune_py[ti] = keep_py;
    H.tune_pz[ti] = keep_pz;
    H.tune_x2 = keep_x2;
    return s != CBS_OK ? s : CBS_EINVAL;
  }
  H.tune_py[ti] = bp;
  H.tune_pz[ti] = bz;
  H.tune_x2 = ti == 1 ? bx : keep_x2;
  if (best_py) *best_py = bp;
  if (best_pz) *best_pz = bz;
  if (best_x2) *best_x2 = bx;
  if (best_ms) *best_ms = bms;
  return CBS_OK;
}

extern "C" cbs_status cbs_set_apply_shape(cbs_hamiltonian *h, int dtype, int py, int pz, int x2) {
  if (!h || (dtype != CBS_C128 && dtype != CBS_C64) || py < 0 || py > 256 || pz < 0 || pz > 256 ||
      x2 < -1 || x2 > 1) {
    set_error("cbs_set_apply_shape: bad argument");
    return CBS_EINVAL;
  }
  HamView &H = h->v;
  H.tune_py[dtype == CBS_C64 ? 1 : 0] = py;
  H.tune_pz[dtype == CBS_C64 ? 1 : 0] = pz;
  if (dtype == CBS_C64) H.tune_x2 = x2;
  return CBS_OK;
}
