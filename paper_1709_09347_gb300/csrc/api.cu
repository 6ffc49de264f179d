// C-ABI plumbing: error reporting, default options and the batched operator apply.
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <string>

#include "kernels.cuh"

namespace cbs {

static thread_local std::string g_err;
static std::atomic<uint64_t> g_launches{0};

void count_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void uncount_launches(uint64_t n) { g_launches.fetch_sub(n, std::memory_order_relaxed); }
uint64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

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
  o->stream = nullptr;
  return CBS_OK;
}

extern "C" cbs_status cbs_apply(const cbs_hamiltonian *h, int n_sys, const double *z, const double *E,
                                int L, const void *X, void *Y, int dtype, void *stream) {
  if (!h || !z || !E || !X || !Y || n_sys < 1 || L < 1 || L > 1024) {
    set_error("cbs_apply: bad argument (need n_sys >= 1, 1 <= L <= 1024, non-null pointers)");
    return CBS_EINVAL;
  }
  if (dtype != CBS_C128 && dtype != CBS_C64) { set_error("cbs_apply: dtype"); return CBS_EINVAL; }
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
  if (!h || !z || !E || !X || !Y || !workspace || n_sys < 1 || L < 1 || L > 1024) {
    set_error("cbs_apply_ws: bad argument (need n_sys >= 1, 1 <= L <= 1024, non-null pointers)");
    return CBS_EINVAL;
  }
  if (dtype != CBS_C128 && dtype != CBS_C64) { set_error("cbs_apply_ws: dtype"); return CBS_EINVAL; }
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
