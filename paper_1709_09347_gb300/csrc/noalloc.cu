// Operator apply for callers that cannot allocate device memory.
//
// Same computation as cbs_apply (Y = P(z) X for a batch), but the scratch it needs — the
// per-system twists and energies and the projector coefficients D — lives in one
// file-scope device array of fixed size instead of memory obtained from cudaMalloc.  The
// array exists on every GPU that loads this library, for the life of the process.
#include <mutex>

#include "common.cuh"

namespace cbs {

// 32 MiB of scratch per device: enough for the projector coefficients of a few hundred
// systems of the 32x32x16 cell (82 KB per system at L = 32 in complex128).
constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Host code cannot use g_noalloc_scratch as a device address (its name is a host-side
// stand-in), so the address is looked up once per device, with that device current.  With
// CUDA's lazy module loading (the default) that first lookup is also what loads this
// library's device code on the device and reserves the array there.  The cached address
// belongs to the device's primary context: it is stale after a device reset.
constexpr int kMaxDevices = 64;
static void *g_scratch_addr[kMaxDevices] = {};
static std::mutex g_scratch_mu;

static cbs_status scratch_address(void **out) {
  int dev = -1;
  CBS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("cbs_apply_noalloc: device ordinal out of range");
    return CBS_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cbs_apply_noalloc: cudaGetSymbolAddress");
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return CBS_OK;
}

static size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace cbs

using namespace cbs;

extern "C" cbs_status cbs_apply_noalloc(const cbs_hamiltonian *h, int n_sys, const double *z,
                                        const double *E, int L, const void *X, void *Y, int dtype,
                                        void *stream) {
  if (!h || !z || !E || !X || !Y || n_sys < 1 || L < 1 || L > 512) {
    set_error("cbs_apply_noalloc: bad argument (need n_sys >= 1, 1 <= L <= 512, non-null pointers)");
    return CBS_EINVAL;
  }
  if (dtype != CBS_C128 && dtype != CBS_C64) { set_error("cbs_apply_noalloc: dtype"); return CBS_EINVAL; }
  // the same column limits as cbs_apply, checked before anything is queued on the stream
  if (!apply_supported(h->v, L, dtype, "cbs_apply_noalloc")) return CBS_EINVAL;
  const size_t tw_bytes = round256((size_t)n_sys * sizeof(double2));
  const size_t e_bytes = round256((size_t)n_sys * sizeof(double));
  const size_t d_bytes = cbs_apply_workspace_size(h, n_sys, L, dtype);
  if (tw_bytes + e_bytes + d_bytes > kNoAllocScratchBytes) {
    set_error("cbs_apply_noalloc: this n_sys x L needs more than the fixed 32 MiB of scratch; "
              "split the batch, or use cbs_apply / cbs_apply_ws");
    return CBS_EINVAL;
  }
  void *base = nullptr;
  cbs_status s = scratch_address(&base);
  if (s != CBS_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  double2 *tw = (double2 *)base;
  double *Ed = (double *)((char *)base + tw_bytes);
  void *D = (char *)base + tw_bytes + e_bytes;
  // the twists and energies come from host memory; D is fully written by the projector
  // gather before the stencil reads it, so nothing in the array has to start at zero
  CBS_CUDA(cudaMemcpyAsync(tw, z, (size_t)n_sys * sizeof(double2), cudaMemcpyHostToDevice, st));
  CBS_CUDA(cudaMemcpyAsync(Ed, E, (size_t)n_sys * sizeof(double), cudaMemcpyHostToDevice, st));
  const HamView &H = h->v;
  if (dtype == CBS_C128)
    return apply_P<double>(H, n_sys, L, (const double2 *)X, (double2 *)Y, tw, false, Ed, (double2 *)D,
                           nullptr, st);
  return apply_P<float>(H, n_sys, L, (const float2 *)X, (float2 *)Y, tw, false, Ed, (float2 *)D,
                        nullptr, st);
}
