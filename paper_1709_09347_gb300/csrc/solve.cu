// Drivers: the shifted solves (plain FP64 BiCG, or complex64 BiCG with FP64 iterative
// refinement) and the whole method for a list of energies (Algorithm 1 on the ring
// contour of §3.2), plus the host-side result object.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <thread>
#include <vector>

#include "kernels.cuh"

using namespace cbs;

cbs_status cbs_internal_rr(const cbs_hamiltonian *h, double E, const double2 *S, const double2 *Ws,
                           int n, int m, double lambda_min, cudaStream_t st, void **ws_out,
                           int *cnt_out, double2 **lam_out, double2 **Psi_out,
                           std::vector<double2> *lam_all, int *rank_out);

struct cbs_energy_result {
  std::vector<double2> lam, k, vec, lam_all, mu;
  std::vector<double> rho, res_all;
  std::vector<int> iters;
  cbs_stats st;
};

struct cbs_result {
  int n_e = 0;
  int64_t N = 0;
  std::vector<cbs_energy_result> e;
  double ms_solve = 0, ms_moments = 0, ms_extract = 0, ms_total = 0;
  double ms_svd = 0, ms_reduced = 0, ms_vectors = 0;   // parts of ms_extract
  double prof_ms[3] = {0, 0, 0}, prof_launches[3] = {0, 0, 0}, prof_outputs[3] = {0, 0, 0};
};

namespace cbs {

// Stream guard: runs on the caller's stream if given, else on a private non-blocking
// stream (graph capture needs a non-legacy stream).
struct StreamGuard {
  cudaStream_t st = nullptr;
  bool own = false;
  cbs_status open(void *user) {
    if (user) { st = (cudaStream_t)user; return CBS_OK; }
    CBS_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    own = true;
    return CBS_OK;
  }
  ~StreamGuard() {
    if (own && st) cudaStreamDestroy(st);
  }
};

struct DevBuf {
  void *p = nullptr;
  cbs_status alloc(size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      p = nullptr;
      set_error("cudaMalloc failed (" + std::to_string(bytes) + " bytes)");
      return CBS_ENOMEM;
    }
    return CBS_OK;
  }
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  template <typename T> T *as() const { return (T *)p; }
};

#define CBS_TRY(x)                     \
  do {                                 \
    cbs_status _s = (x);               \
    if (_s != CBS_OK) return _s;       \
  } while (0)

__global__ void k_expand_systems(int n_e, int n_int, const double2 *z1, const double *energies,
                                 double2 *zs, double *Es) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n_e * n_int) {
    zs[s] = z1[s % n_int];
    Es[s] = energies[s / n_int];
  }
}

// *flags |= 1 when any of the count complex entries of A is not finite, |= 2 when any has a
// non-zero imaginary part.
__global__ void k_nonfinite(int64_t count, const double2 *A, int *bad) {
  int b = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    b |= !(isfinite(A[i].x) && isfinite(A[i].y));
    b |= (A[i].y != 0.0) << 1;
  }
  const int f = (__syncthreads_or(b & 1) ? 1 : 0) | (__syncthreads_or(b & 2) ? 2 : 0);
  if (f && threadIdx.x == 0) atomicOr(bad, f);
}

// Host-side check of a right-hand-side block on the device: CBS_EINVAL with a message
// when it holds a NaN or an infinity (BiCG on such a block would only spread it).
// *is_real (may be NULL) tells whether every entry is real.
static cbs_status check_finite_block(int64_t count, const double2 *A, const char *who, cudaStream_t st,
                                     bool *is_real = nullptr) {
  DevBuf flag;
  CBS_TRY(flag.alloc(sizeof(int)));
  CBS_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), st));
  k_nonfinite<<<std::min<int64_t>(1024, (count + 255) / 256), 256, 0, st>>>(count, A, flag.as<int>());
  cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  int bad = 0;
  CBS_CUDA(cudaMemcpyAsync(&bad, flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  CBS_CUDA(cudaStreamSynchronize(st));
  if (bad & 1) {
    set_error(std::string(who) + ": the right-hand sides contain a NaN or an infinity");
    return CBS_EINVAL;
  }
  if (is_real) *is_real = !(bad & 2);
  return CBS_OK;
}

__global__ void k_col_norms(int64_t N, int L, const double2 *B, double *out) {
  const int c = threadIdx.x;
  double a = 0;
  for (int64_t i = 0; i < N; ++i) a += cabs2(B[i * L + c]);
  out[c] = sqrt(a);
}

__global__ void k_bnorm_expand(int n2, int L, const double *bn, double *out) {
  const int s = blockIdx.x, c = threadIdx.x;
  if (s < n2) out[(int64_t)s * L + c] = bn[c];
}

__global__ void k_gather_tau(int cnt, const double2 *tau, const int *ridx, double2 *out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < cnt) out[r] = tau[ridx[r]];
}

__global__ void k_scale_rows(int rows, int cols, int64_t ld, const double *sig, double2 *B) {
  const int64_t tot = (int64_t)rows * cols;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx % rows), c = (int)(idx / rows);
    B[r + c * ld] = cscale(B[r + c * ld], 1.0 / sig[r]);
  }
}

// True residual check of solutions Y[2n] against B (shared by all systems):
// maxrel[s][c] = max(||B - P(z)Y||, ||B - P(z)^dagger Y~||)/||B||, colmask = needs work.
struct ResidualCheck {
  DevBuf buf;
  double2 *R = nullptr;
  double2 *D = nullptr;
  double *cn = nullptr, *bn = nullptr, *bn2 = nullptr, *maxrel = nullptr;
  int *colmask = nullptr, *nunc = nullptr;
  int n = 0, L = 0;
  int64_t N = 0;
  cbs_status alloc(const HamView &H, int n_, int L_) {
    n = n_; L = L_; N = H.n;
    const size_t vec = (size_t)2 * n * N * L * sizeof(double2);
    const size_t dsz = (size_t)2 * n * (H.n_atoms ? H.n_atoms : 1) * H.np4 * L * sizeof(double2);
    const size_t small = (size_t)2 * n * 64 * L * sizeof(double) + 3 * (size_t)2 * n * L * sizeof(double) +
                         (size_t)n * L * sizeof(int) + 4096;
    CBS_TRY(buf.alloc(vec + dsz + small + 1024));
    char *b = buf.as<char>();
    auto take = [&](size_t sz) { char *r = b; b += (sz + 255) & ~(size_t)255; return (void *)r; };
    R = (double2 *)take(vec);
    D = (double2 *)take(dsz);
    cn = (double *)take((size_t)2 * n * 64 * L * sizeof(double));
    bn = (double *)take((size_t)L * sizeof(double));
    bn2 = (double *)take((size_t)2 * n * L * sizeof(double));
    maxrel = (double *)take((size_t)n * L * sizeof(double));
    colmask = (int *)take((size_t)n * L * sizeof(int));
    nunc = (int *)take(256);
    return CBS_OK;
  }
  // Y: [2n][N][L]; tw/E: twists [2n] and energies [2n]
  bool profile = false;
  bool have_bn = false;
  double prof_ms = 0, prof_launches = 0, prof_outputs = 0;
  cbs_status run(const HamView &H, const double2 *Y, const double2 *B, const double2 *tw,
                 const double *E, double tol, cudaStream_t st, int *host_unconv) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (profile) {
      CBS_CUDA(cudaEventCreate(&e0));
      CBS_CUDA(cudaEventCreate(&e1));
      CBS_CUDA(cudaEventRecord(e0, st));
    }
    CBS_TRY(apply_P<double>(H, 2 * n, L, Y, R, tw, false, E, D, nullptr, st));
    if (profile) {
      CBS_CUDA(cudaEventRecord(e1, st));
      CBS_CUDA(cudaEventSynchronize(e1));
      float ms = 0;
      CBS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      prof_ms += ms;
      prof_launches += 1;
      prof_outputs += 2.0 * n * (double)N * L;
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
    }
    CBS_TRY(launch_residual(2 * n, N, L, B, 0, B, 0, n, R, cn, st));
    if (!have_bn) {   // the right-hand sides do not change between calls
      k_col_norms<<<1, L, 0, st>>>(N, L, B, bn); cbs::count_launches(1);
      k_bnorm_expand<<<2 * n, L, 0, st>>>(2 * n, L, bn, bn2); cbs::count_launches(1);
      CBS_CUDA(cudaGetLastError());
      have_bn = true;
    }
    CBS_CUDA(cudaMemsetAsync(nunc, 0, sizeof(int), st));
    CBS_TRY(launch_refine_check(n, L, 64, cn, bn2, tol, colmask, nunc, maxrel, st));
    if (host_unconv) {
      CBS_CUDA(cudaMemcpyAsync(host_unconv, nunc, sizeof(int), cudaMemcpyDeviceToHost, st));
      CBS_CUDA(cudaStreamSynchronize(st));
    }
    return CBS_OK;
  }
};

// Shifted solves for n systems; output Y[2n][N][L] (primal then dual), per-column
// iteration counts iters[n][L], flags[n][L], and max true residual maxrel[n][L] (host).
struct ShiftedSolver {
  HamView H;
  int n = 0, L = 0;
  const double2 *zs = nullptr;   // [n] twists of the primal systems (device)
  const double *Es = nullptr;    // [n] energies (device)
  const double2 *B = nullptr;    // [N][L] right-hand sides shared by every system (device)
  DevBuf ybuf;
  double2 *Y = nullptr;      // [2n][N][L] solutions (FP64)
  Bicg<double> b64;
  Bicg<float> b32;
  ResidualCheck rc;
  std::vector<int> iters, flags;
  std::vector<double> maxrel;
  int sweeps = 0;
  bool fp64_continued = false;
  // quadrature points per energy when the systems are energies x points (e-major), for the
  // load-balance rule (0: systems are independent)
  int group = 0;
  double prof_ms[3] = {0, 0, 0}, prof_launches[3] = {0, 0, 0}, prof_outputs[3] = {0, 0, 0};
  // columns that the load-balance rule stopped (flag bit 6) are not refined: clear them in
  // the residual check's mask and recount the columns left
  cbs_status mask_stopped(int *unconv, cudaStream_t st) {
    bool any = false;
    for (int f : flags) any = any || (f & 64);
    if (!any || *unconv == 0) return CBS_OK;
    std::vector<int> m((size_t)n * L);
    CBS_CUDA(cudaMemcpyAsync(m.data(), rc.colmask, m.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
    CBS_CUDA(cudaStreamSynchronize(st));
    int u = 0;
    for (size_t k = 0; k < m.size(); ++k) {
      if (flags[k] & 64) m[k] = 0;
      u += m[k];
    }
    CBS_CUDA(cudaMemcpyAsync(rc.colmask, m.data(), m.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    CBS_CUDA(cudaStreamSynchronize(st));
    *unconv = u;
    return CBS_OK;
  }
  static int stop_need(const cbs_options &o, int n_pt) {
    return o.stop_fraction < 1.0 ? (int)floor(o.stop_fraction * n_pt) : (1 << 30);
  }
  // adds the apply profiles of b64, b32 and the residual checks (and resets them)
  cbs_status collect_profile(cudaStream_t st) {
    double o64 = 0, o32 = 0;
    if (b64.block && b64.profile) CBS_TRY(b64.prof_outputs(st, &o64));
    if (b32.block && b32.profile) CBS_TRY(b32.prof_outputs(st, &o32));
    prof_ms[CBS_C128] += b64.prof_ms + rc.prof_ms;
    prof_launches[CBS_C128] += b64.prof_launches + rc.prof_launches;
    prof_outputs[CBS_C128] += o64 + rc.prof_outputs;
    prof_ms[CBS_C64] += b32.prof_ms;
    prof_launches[CBS_C64] += b32.prof_launches;
    prof_outputs[CBS_C64] += o32;
    b64.prof_ms = b64.prof_launches = b32.prof_ms = b32.prof_launches = 0;
    rc.prof_ms = rc.prof_launches = rc.prof_outputs = 0;
    if (b64.block && b64.sys_apply) CBS_CUDA(cudaMemsetAsync(b64.sys_apply, 0, sizeof(unsigned long long), st));
    if (b32.block && b32.sys_apply) CBS_CUDA(cudaMemsetAsync(b32.sys_apply, 0, sizeof(unsigned long long), st));
    return CBS_OK;
  }

  // device bytes of the per-system solver state (one BiCG per system), per primal system
  static size_t bytes_per_system(const HamView &H, int L, int precision) {
    const size_t v16 = (size_t)H.n * L * 16;
    if (precision == CBS_FP64) return 2 * (4 * v16 + v16) + 2 * v16;   // state + residual check
    return 2 * (4 * v16 / 2) + 2 * v16 + 2 * v16 + 2 * v16;             // f32 state, Y, R, D
  }
  // device bytes per energy of a shifted family of n_pt points: scaled directions and
  // solutions of its 2 n_pt systems, plus the FP64 solutions kept for the moments
  static size_t family_bytes_per_energy(const HamView &H, int n_pt, int L, int precision) {
    const size_t v16 = (size_t)H.n * L * 16;
    const bool fp64 = precision == CBS_FP64;
    const size_t vr = fp64 ? v16 : v16 / 2;
    return (size_t)2 * n_pt * (2 * vr + (fp64 ? 0 : v16));
  }

  MultiShift<double> ms;
  MultiShift<float> ms32;
  DevBuf twbuf;
  ~ShiftedSolver() {
    b64.release();
    b32.release();
    ms.release();
    ms.release_x();
    ms32.release();
    ms32.release_x();
  }

  cbs_status init_stats(int n_, int L_) {
    n = n_; L = L_;
    iters.assign((size_t)n * L, 0);
    flags.assign((size_t)n * L, 0);
    maxrel.assign((size_t)n * L, 0.0);
    return CBS_OK;
  }

  // Per-system BiCG from Y = 0: plain FP64, or complex64 with FP64 reliable updates.
  cbs_status run(const HamView &H_, int n_, int L_, const double2 *zs_, const double *Es_,
                 const double2 *B_, const cbs_options &o, cudaStream_t st) {
    H = H_; zs = zs_; Es = Es_; B = B_;
    init_stats(n_, L_);
    CBS_TRY(rc.alloc(H, n, L));
    rc.profile = o.profile != 0;
    b64.profile = b32.profile = o.profile != 0;
    if (o.precision == CBS_FP64) {
      CBS_TRY(b64.alloc(H, n, L));
      if (group > 0 && o.stop_fraction < 1.0) {
        b64.group = group;
        b64.group_need = stop_need(o, group);
      }
      CBS_TRY(b64.set_systems(zs, Es, st));
      CBS_TRY(b64.init(B, 0, B, 0, nullptr, o.tol, 0.0, st));
      int done = 0;
      CBS_TRY(b64.iterate(o.tol, o.max_iter, o.check_every, st, &done));
      Y = b64.x;
      CBS_TRY(rc.run(H, Y, B, b64.tw, b64.E, o.tol, st, nullptr));
      CBS_CUDA(cudaMemcpyAsync(iters.data(), b64.iters, (size_t)n * L * sizeof(int), cudaMemcpyDeviceToHost, st));
      CBS_CUDA(cudaMemcpyAsync(flags.data(), b64.flags, (size_t)n * L * sizeof(int), cudaMemcpyDeviceToHost, st));
      CBS_CUDA(cudaMemcpyAsync(maxrel.data(), rc.maxrel, (size_t)n * L * sizeof(double), cudaMemcpyDeviceToHost, st));
      CBS_CUDA(cudaStreamSynchronize(st));
      sweeps = 0;
      return collect_profile(st);
    }
    CBS_TRY(ybuf.alloc((size_t)2 * n * H.n * L * sizeof(double2)));
    Y = ybuf.as<double2>();
    CBS_CUDA(cudaMemsetAsync(Y, 0, (size_t)2 * n * H.n * L * sizeof(double2), st));
    return refine(o, st);
  }

  // Continues the solutions Y (already holding a starting guess) until the true residual
  // of every column is below tol: complex64 BiCG with FP64 reliable updates (precision
  // CBS_FP32_REFINE) or FP64 BiCG on the residual equation, for the columns that need it.
  cbs_status refine(const cbs_options &o, cudaStream_t st) {
    if (!rc.R) {
      CBS_TRY(rc.alloc(H, n, L));
      rc.profile = o.profile != 0;
    }
    b64.profile = b32.profile = o.profile != 0;
    std::vector<int> it_tmp((size_t)n * L), fl_tmp((size_t)n * L);
    CBS_TRY(twbuf.alloc((size_t)2 * n * (sizeof(double2) + sizeof(double)) + 256));
    double2 *tw = twbuf.as<double2>();
    double *E2 = (double *)(tw + 2 * n);
    CBS_TRY(launch_twists(n, zs, Es, tw, E2, st));
    int unconv = 0;
    CBS_TRY(rc.run(H, Y, B, tw, E2, o.tol, st, &unconv));
    CBS_TRY(mask_stopped(&unconv, st));
    if (unconv > 0 && o.precision == CBS_FP32_REFINE) {
      // complex64 BiCG with FP64 refinement of the residual (reliable updates):
      //   the complex64 recursion runs until its residual is below inner_tol times the
      //   largest residual norm seen since the last update (or inner_max_iter iterations);
      //   its correction is added to Y in FP64, the true residuals R = B - P(z) Y and
      //   R~ = B - P(z)^dagger Y~ are formed in FP64, and the columns above tol continue
      //   from R (rounded) with their search directions kept.  Stop targets are relative
      //   to the original right-hand side.
      CBS_TRY(b32.alloc(H, n, L));
      CBS_TRY(b32.set_systems(zs, Es, st));
      CBS_TRY(b32.init(rc.R, (int64_t)H.n * L, rc.R + (size_t)n * H.n * L, (int64_t)H.n * L,
                       rc.colmask, 0.25 * o.tol, o.inner_tol, st, rc.bn2));
      std::vector<double> rel((size_t)n * L), best((size_t)n * L, 1e300);
      std::vector<int> need((size_t)n * L), stall((size_t)n * L, 0);
      for (int sw = 0; sw < o.max_sweeps && unconv > 0; ++sw) {
        int done = 0;
        CBS_TRY(b32.iterate(o.tol, o.max_iter, o.check_every, st, &done, o.inner_max_iter));
        CBS_TRY(launch_accumulate((int64_t)2 * n * H.n * L, Y, b32.x, st));
        CBS_TRY(rc.run(H, Y, B, tw, E2, o.tol, st, &unconv));
        ++sweeps;
        if (unconv == 0) break;
        // per column: stagnation of the FP64 true residual means the single-precision
        // recursion no longer makes progress there (loss of bi-orthogonality); such columns
        // leave the complex64 phases and are finished in FP64 below
        CBS_CUDA(cudaMemcpyAsync(rel.data(), rc.maxrel, rel.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        CBS_CUDA(cudaMemcpyAsync(need.data(), rc.colmask, need.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
        CBS_CUDA(cudaStreamSynchronize(st));
        int live = 0;
        for (size_t k = 0; k < rel.size(); ++k) {
          if (!need[k]) continue;
          if (rel[k] < 0.5 * best[k]) { best[k] = rel[k]; stall[k] = 0; }
          else ++stall[k];
          if (stall[k] >= o.stall_sweeps) need[k] = 0;
          live += need[k];
        }
        if (live == 0) break;
        CBS_CUDA(cudaMemcpyAsync(rc.colmask, need.data(), need.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        CBS_TRY(b32.replace(rc.R, rc.colmask, st));
      }
      CBS_CUDA(cudaMemcpyAsync(it_tmp.data(), b32.iters, (size_t)n * L * sizeof(int), cudaMemcpyDeviceToHost, st));
      CBS_CUDA(cudaMemcpyAsync(fl_tmp.data(), b32.flags, (size_t)n * L * sizeof(int), cudaMemcpyDeviceToHost, st));
      CBS_CUDA(cudaStreamSynchronize(st));
      for (size_t k = 0; k < iters.size(); ++k) {
        iters[k] += it_tmp[k];
        flags[k] |= (fl_tmp[k] & 2);
      }
      CBS_TRY(collect_profile(st));
      b32.release();
      if (unconv > 0) {
        CBS_TRY(rc.run(H, Y, B, tw, E2, o.tol, st, &unconv));   // full mask
        CBS_TRY(mask_stopped(&unconv, st));
      }
    }
    if (unconv > 0) {
      // FP64 BiCG for the columns left: P(z) D = R, P(z)^dagger D~ = R~ to tol relative to
      // the original right-hand side, then Y += D
      CBS_TRY(b64.alloc(H, n, L));
      CBS_TRY(b64.set_systems(zs, Es, st));
      CBS_TRY(b64.init(rc.R, (int64_t)H.n * L, rc.R + (size_t)n * H.n * L, (int64_t)H.n * L,
                       rc.colmask, 0.5 * o.tol, 0.0, st, rc.bn2));
      int done = 0;
      CBS_TRY(b64.iterate(o.tol, o.max_iter, o.check_every, st, &done));
      CBS_TRY(launch_accumulate((int64_t)2 * n * H.n * L, Y, b64.x, st));
      CBS_TRY(rc.run(H, Y, B, tw, E2, o.tol, st, &unconv));
      CBS_CUDA(cudaMemcpyAsync(it_tmp.data(), b64.iters, (size_t)n * L * sizeof(int), cudaMemcpyDeviceToHost, st));
      CBS_CUDA(cudaMemcpyAsync(fl_tmp.data(), b64.flags, (size_t)n * L * sizeof(int), cudaMemcpyDeviceToHost, st));
      CBS_CUDA(cudaStreamSynchronize(st));
      for (size_t k = 0; k < iters.size(); ++k) {
        iters[k] += it_tmp[k];
        flags[k] |= (fl_tmp[k] & 2);
      }
      fp64_continued = true;
      CBS_TRY(collect_profile(st));
      b64.release();
    }
    std::vector<int> mask((size_t)n * L);
    CBS_CUDA(cudaMemcpyAsync(maxrel.data(), rc.maxrel, (size_t)n * L * sizeof(double), cudaMemcpyDeviceToHost, st));
    CBS_CUDA(cudaMemcpyAsync(mask.data(), rc.colmask, (size_t)n * L * sizeof(int), cudaMemcpyDeviceToHost, st));
    CBS_CUDA(cudaStreamSynchronize(st));
    for (size_t k = 0; k < mask.size(); ++k)
      if (mask[k] && !(flags[k] & 64)) flags[k] |= 1;
    return CBS_OK;
  }

  // One Krylov sequence per (point, column) for all n_e energies of the batch (systems
  // ordered e * n_pt + j as in zs/Es); seed energy: the highest of the batch.  FP64: the
  // family in FP64.  CBS_FP32_REFINE: the family in complex64 down to family_tol, then the
  // FP64 solutions are refined per energy as in refine().  The per-energy refinement runs
  // on groups of energies sized to the free device memory.
  template <typename R>
  cbs_status run_family(MultiShift<R> &fam, const HamView &H_, int n_e, int n_pt, int L_,
                        const double2 *z1, const double *energies_h, const double2 *zs_,
                        const double *Es_, const double2 *B_, const cbs_options &o, cudaStream_t st) {
    H = H_; zs = zs_; Es = Es_; B = B_;
    init_stats(n_e * n_pt, L_);
    fam.seed.profile = o.profile != 0;
    double E0 = energies_h[0];
    for (int e = 1; e < n_e; ++e) E0 = std::max(E0, energies_h[e]);
    std::vector<double> sig(n_e);
    for (int e = 0; e < n_e; ++e) sig[e] = energies_h[e] - E0;
    const bool mixed = sizeof(R) == sizeof(float);
    const double ftol = mixed ? std::max(o.tol, o.family_tol > 0 ? o.family_tol : 1e-6) : o.tol;
    CBS_TRY(fam.alloc(H, n_pt, n_e, L));
    fam.group_need = stop_need(o, n_pt);
    CBS_TRY(fam.init(z1, E0, sig.data(), B, ftol, st));
    int done = 0;
    CBS_TRY(fam.iterate(o.max_iter, o.check_every, st, &done));
    std::vector<int> fl_tmp((size_t)n * L);
    CBS_CUDA(cudaMemcpyAsync(iters.data(), fam.siters, (size_t)n * L * sizeof(int), cudaMemcpyDeviceToHost, st));
    CBS_CUDA(cudaMemcpyAsync(fl_tmp.data(), fam.sflags, (size_t)n * L * sizeof(int), cudaMemcpyDeviceToHost, st));
    CBS_CUDA(cudaStreamSynchronize(st));
    for (size_t k = 0; k < flags.size(); ++k) flags[k] |= (fl_tmp[k] & (2 | 64));
    double oseed = 0;
    if (o.profile) CBS_TRY(fam.seed.prof_outputs(st, &oseed));
    const int ti = mixed ? CBS_C64 : CBS_C128;
    prof_ms[ti] += fam.seed.prof_ms;
    prof_launches[ti] += fam.seed.prof_launches;
    prof_outputs[ti] += oseed;
    double upd_cols = 0;
    if (o.profile) CBS_TRY(fam.update_columns(st, &upd_cols));
    prof_ms[2] += fam.upd_ms;
    prof_launches[2] += fam.upd_launches;
    prof_outputs[2] += upd_cols * (double)H.n;
    fam.release();
    const size_t vbytes = (size_t)2 * n * H.n * L * sizeof(double2);
    if (mixed) {
      // FP64 solutions from the complex64 ones
      CBS_TRY(ybuf.alloc(vbytes));
      Y = ybuf.as<double2>();
      CBS_CUDA(cudaMemsetAsync(Y, 0, vbytes, st));
      CBS_TRY(launch_accumulate((int64_t)2 * n * H.n * L, Y, (const float2 *)fam.X, st));
      fam.release_x();
    } else {
      Y = (double2 *)fam.X;   // owned by fam until the solver is destroyed
    }
    // per-energy refinement in groups of energies that fit in free memory
    size_t free_b = 0, total_b = 0;
    CBS_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const size_t per_e = (size_t)n_pt * (bytes_per_system(H, L, o.precision) + (size_t)2 * H.n * L * 16) +
                         (size_t)2 * n_pt * (H.n_atoms ? H.n_atoms : 1) * H.np4 * L * 16 * 2;
    const int grp = std::max(1, std::min(n_e, (int)((free_b * 8 / 10) / std::max<size_t>(per_e, 1))));
    const size_t blk = (size_t)H.n * L;
    for (int g0 = 0; g0 < n_e; g0 += grp) {
      const int ge = std::min(grp, n_e - g0);
      ShiftedSolver sub;
      sub.H = H;
      sub.zs = zs + (size_t)g0 * n_pt;
      sub.Es = Es + (size_t)g0 * n_pt;
      sub.B = B;
      sub.init_stats(ge * n_pt, L);
      const size_t sn = (size_t)sub.n;
      for (size_t k = 0; k < sn * L; ++k) sub.flags[k] = flags[(size_t)g0 * n_pt * L + k];
      CBS_TRY(sub.ybuf.alloc(2 * sn * blk * sizeof(double2)));
      sub.Y = sub.ybuf.as<double2>();
      const size_t off = (size_t)g0 * n_pt;
      CBS_CUDA(cudaMemcpyAsync(sub.Y, Y + off * blk, sn * blk * sizeof(double2), cudaMemcpyDeviceToDevice, st));
      CBS_CUDA(cudaMemcpyAsync(sub.Y + sn * blk, Y + ((size_t)n + off) * blk, sn * blk * sizeof(double2),
                               cudaMemcpyDeviceToDevice, st));
      CBS_TRY(sub.refine(o, st));
      CBS_CUDA(cudaMemcpyAsync(Y + off * blk, sub.Y, sn * blk * sizeof(double2), cudaMemcpyDeviceToDevice, st));
      CBS_CUDA(cudaMemcpyAsync(Y + ((size_t)n + off) * blk, sub.Y + sn * blk, sn * blk * sizeof(double2),
                               cudaMemcpyDeviceToDevice, st));
      CBS_CUDA(cudaStreamSynchronize(st));
      for (size_t k = 0; k < sn * L; ++k) {
        iters[off * L + k] += sub.iters[k];
        flags[off * L + k] = sub.flags[k];
        maxrel[off * L + k] = sub.maxrel[k];
      }
      sweeps = std::max(sweeps, sub.sweeps);
      fp64_continued = fp64_continued || sub.fp64_continued;
      for (int t = 0; t < 3; ++t) {
        prof_ms[t] += sub.prof_ms[t];
        prof_launches[t] += sub.prof_launches[t];
        prof_outputs[t] += sub.prof_outputs[t];
      }
    }
    return CBS_OK;
  }
};

static cbs_status check_opts(const cbs_options *opt, cbs_options *o) {
  if (opt) *o = *opt;
  else cbs_options_default(o);
  if (!(o->tol > 0) || !(o->delta > 0) || !(o->rho_max > 0) || o->max_iter < 1 ||
      (o->precision != CBS_FP64 && o->precision != CBS_FP32_REFINE) ||
      (o->extraction != CBS_HANKEL && o->extraction != CBS_RR) || !(o->inner_tol > 0) ||
      o->max_sweeps < 0 || o->inner_max_iter < 1 || o->stall_sweeps < 1 ||
      (o->multi_shift != 0 && o->multi_shift != 1) || o->family_tol < 0 || o->family_tol >= 1 ||
      !(o->stop_fraction > 0 && o->stop_fraction <= 1.0) || o->points_per_wave < 0 ||
      (o->conj_points != 0 && o->conj_points != 1)) {
    set_error("invalid cbs_options");
    return CBS_EINVAL;
  }
  if (o->check_every < 1) o->check_every = 1;
  return CBS_OK;
}

}  // namespace cbs

extern "C" cbs_status cbs_solve_shifted(const cbs_hamiltonian *h, int n_sys, const double *z,
                                        const double *E, int L, const void *B, void *Y, void *Yd,
                                        int *iters, const cbs_options *opt) {
  if (!h || n_sys < 1 || !z || !E || !B || !Y || !Yd || L < 1 || L > 1024) {
    set_error("cbs_solve_shifted: bad argument");
    return CBS_EINVAL;
  }
  cbs_options o;
  CBS_TRY(check_opts(opt, &o));
  StreamGuard sg;
  CBS_TRY(sg.open(o.stream));
  cudaStream_t st = sg.st;
  DevBuf sys;
  CBS_TRY(sys.alloc((size_t)n_sys * (sizeof(double2) + sizeof(double)) + 256));
  double2 *zs = sys.as<double2>();
  double *Es = (double *)(zs + n_sys);
  CBS_CUDA(cudaMemcpyAsync(zs, z, (size_t)n_sys * sizeof(double2), cudaMemcpyHostToDevice, st));
  CBS_CUDA(cudaMemcpyAsync(Es, E, (size_t)n_sys * sizeof(double), cudaMemcpyHostToDevice, st));
  CBS_TRY(check_finite_block((int64_t)h->v.n * L, (const double2 *)B, "cbs_solve_shifted", st));
  ShiftedSolver S;
  CBS_TRY(S.run(h->v, n_sys, L, zs, Es, (const double2 *)B, o, st));
  const size_t blk = (size_t)n_sys * h->v.n * L * sizeof(double2);
  CBS_CUDA(cudaMemcpyAsync(Y, S.Y, blk, cudaMemcpyDeviceToDevice, st));
  CBS_CUDA(cudaMemcpyAsync(Yd, (const char *)S.Y + blk, blk, cudaMemcpyDeviceToDevice, st));
  CBS_CUDA(cudaStreamSynchronize(st));
  if (iters) memcpy(iters, S.iters.data(), S.iters.size() * sizeof(int));
  int fl = 0;
  for (int f : S.flags) fl |= f;
  if (fl & 2) { set_error("BiCG breakdown in some column"); return CBS_EBREAKDOWN; }
  if (fl & 1) { set_error("BiCG did not converge in some column"); return CBS_ENOCONV; }
  return CBS_OK;
}

// ---------------------------------------------------------------------- cbs_solve
static cbs_status solve_impl(const cbs_hamiltonian *h, const double *energies, int n_e,
                             const cbs_contour *ct, int L, int M, const void *V,
                             const cbs_options &o, cudaStream_t st, cbs_result *res) {
  const HamView &H = h->v;
  const int64_t N = H.n;
  const int n_int = ct->n_int;
  const int nLM = L * M;
  res->n_e = n_e;
  res->N = N;
  res->e.resize(n_e);
  cudaEvent_t ev[2];
  CBS_CUDA(cudaEventCreate(&ev[0]));
  CBS_CUDA(cudaEventCreate(&ev[1]));
  struct EvGuard { cudaEvent_t *e; ~EvGuard() { cudaEventDestroy(e[0]); cudaEventDestroy(e[1]); } } evg{ev};
  auto lap = [&](double *acc) -> cbs_status {
    CBS_CUDA(cudaEventRecord(ev[1], st));
    CBS_CUDA(cudaEventSynchronize(ev[1]));
    float ms = 0;
    CBS_CUDA(cudaEventElapsedTime(&ms, ev[0], ev[1]));
    *acc += ms;
    CBS_CUDA(cudaEventRecord(ev[0], st));
    return CBS_OK;
  };
  CBS_CUDA(cudaEventRecord(ev[0], st));

  // right-hand sides on the device
  DevBuf vbuf;
  CBS_TRY(vbuf.alloc((size_t)N * L * sizeof(double2)));
  double2 *dV = vbuf.as<double2>();
  CBS_CUDA(cudaMemcpyAsync(dV, V, (size_t)N * L * sizeof(double2), cudaMemcpyDefault, st));
  bool v_real = false;
  CBS_TRY(check_finite_block((int64_t)N * L, dV, "cbs_solve", st, &v_real));
  // Conjugate points (§3.2 contour, real blocks H0, H+, H- and real E): the outer-circle points
  // come in pairs z_{n_int-1-j} = conj(z_j) (theta -> 2 pi - theta), and so do their dual
  // twists; P(conj z) = conj(P(z)), so with a real V the solutions there are conj(Y_j) and
  // conj(Y~_j).  Only the first n_int/2 points are solved; the moments add the conjugates.
  const bool mirror = o.conj_points && v_real && n_int % 2 == 0;
  const int n_solve = mirror ? n_int / 2 : n_int;
  // contour
  DevBuf cbuf;
  CBS_TRY(cbuf.alloc((size_t)n_int * (4 * M + 1) * sizeof(double2) + (size_t)n_e * sizeof(double) + 512));
  double2 *coef = cbuf.as<double2>();
  double2 *z1 = coef + (size_t)n_int * 4 * M;
  double *dE = (double *)(z1 + n_int);
  CBS_TRY(launch_contour(n_int, M, ct->lambda_min, coef, z1, st));
  CBS_CUDA(cudaMemcpyAsync(dE, energies, (size_t)n_e * sizeof(double), cudaMemcpyHostToDevice, st));

  // energies per batch from free memory
  size_t free_b = 0, total_b = 0;
  CBS_CUDA(cudaMemGetInfo(&free_b, &total_b));
  // Energies per batch (nb) and quadrature points per wave (nw).  A batch's moments S_k,
  // mu_k are accumulated over waves of points, each wave solved and then released, so the
  // solver state scales with nb * nw and only the moments with nb.  Preferred: every point in
  // one wave and as many energies as fit; when not even one energy's points fit at once,
  // all energies (or as many as fit) with as many points per wave as fit.
  const size_t v16 = (size_t)N * L * 16;
  const size_t dsz = (size_t)2 * (H.n_atoms ? H.n_atoms : 1) * H.np4 * L * 16 * 2;
  const size_t per_sys = ShiftedSolver::bytes_per_system(H, L, o.precision) + dsz;
  const size_t extract_e = (size_t)N * nLM * 16 + (size_t)4 * nLM * nLM * 16 * 6;
  auto peak = [&](size_t ne_, size_t nw_) -> size_t {
    const size_t pairs = ne_ * nw_;
    size_t solve;
    if (o.multi_shift) {
      const size_t vr = o.precision == CBS_FP64 ? v16 : v16 / 2;
      const size_t fam = pairs * ShiftedSolver::family_bytes_per_energy(H, 1, L, o.precision) +
                         nw_ * (2 * 4 * vr + dsz);                        // + seed per point
      const size_t ref = pairs * 2 * v16 + nw_ * (per_sys + 2 * v16);   // Y + one energy's refinement
      solve = std::max(fam, ref);
    } else {
      solve = pairs * per_sys;
    }
    return solve + ne_ * extract_e + 2 * pairs * 8 * L * L * 16;
  };
  const size_t usable = free_b * 6 / 10;
  int nb = 0, nw = n_solve;
  if (o.energies_per_batch > 0) nb = std::min(o.energies_per_batch, n_e);
  if (o.points_per_wave > 0) nw = std::min(o.points_per_wave, n_solve);
  if (nb == 0) {
    for (int t = n_e; t >= 1; --t)
      if (peak(t, nw) <= usable) { nb = t; break; }
  }
  if (nb == 0) {                   // not even one energy with these points: waves of points
    nb = o.energies_per_batch > 0 ? nb : n_e;
    if (nb == 0) nb = n_e;
    while (true) {
      int w = 0;
      for (int t = nw; t >= 1; --t)
        if (peak(nb, t) <= usable) { w = t; break; }
      if (w > 0 || nb == 1) { nw = std::max(w, 1); break; }
      nb = (nb + 1) / 2;
    }
  }
  nb = std::max(1, std::min(nb, n_e));

  cbs_status ret = CBS_OK;
  for (int e0 = 0; e0 < n_e; e0 += nb) {
    const int ne = std::min(nb, n_e - e0);
    // per (energy, point, column) statistics of the batch, gathered over the waves
    std::vector<int> b_iters((size_t)ne * n_int * L, 0), b_flags((size_t)ne * n_int * L, 0);
    std::vector<double> b_maxrel((size_t)ne * n_int * L, 0.0);
    int b_sweeps = 0;
    bool b_fp64 = false;
    DevBuf mbuf;
    const int nch = vhy_chunks(N);
    const size_t s_bytes = (size_t)ne * N * nLM * sizeof(double2);
    const size_t mu_bytes = (size_t)ne * 2 * M * L * L * sizeof(double2);
    const size_t part_bytes = (size_t)2 * ne * nw * nch * L * L * sizeof(double2);
    CBS_TRY(mbuf.alloc(s_bytes + mu_bytes + part_bytes + 1024));
    double2 *Sm = mbuf.as<double2>();
    double2 *mu = (double2 *)((char *)Sm + ((s_bytes + 255) & ~(size_t)255));
    double2 *part = (double2 *)((char *)mu + ((mu_bytes + 255) & ~(size_t)255));
    for (int j0 = 0; j0 < n_solve; j0 += nw) {
      const int nwv = std::min(nw, n_solve - j0);
      const int nsys = ne * nwv;
      DevBuf sysb;
      CBS_TRY(sysb.alloc((size_t)nsys * (sizeof(double2) + sizeof(double)) + 256));
      double2 *zs = sysb.as<double2>();
      double *Es = (double *)(zs + nsys);
      k_expand_systems<<<ceil_div(nsys, 128), 128, 0, st>>>(ne, nwv, z1 + j0, dE + e0, zs, Es); cbs::count_launches(1);
      CBS_CUDA(cudaGetLastError());
      // ---- step 1: shifted solves of this wave's points
      ShiftedSolver S;
      S.group = nwv;
      if (o.multi_shift && o.precision == CBS_FP64)
        CBS_TRY(S.run_family(S.ms, H, ne, nwv, L, z1 + j0, energies + e0, zs, Es, dV, o, st));
      else if (o.multi_shift)
        CBS_TRY(S.run_family(S.ms32, H, ne, nwv, L, z1 + j0, energies + e0, zs, Es, dV, o, st));
      else
        CBS_TRY(S.run(H, nsys, L, zs, Es, dV, o, st));
      for (int t = 0; t < 3; ++t) {
        res->prof_ms[t] += S.prof_ms[t];
        res->prof_launches[t] += S.prof_launches[t];
        res->prof_outputs[t] += S.prof_outputs[t];
      }
      for (int e = 0; e < ne; ++e)
        for (int jj = 0; jj < nwv; ++jj)
          for (int c = 0; c < L; ++c) {
            const size_t src = ((size_t)e * nwv + jj) * L + c;
            const size_t dst = ((size_t)e * n_int + j0 + jj) * L + c;
            b_iters[dst] = S.iters[src];
            b_flags[dst] = S.flags[src];
            b_maxrel[dst] = S.maxrel[src];
            if (mirror) {      // the conjugate point's solve is this one's conjugate
              const size_t dm = ((size_t)e * n_int + (n_int - 1 - j0 - jj)) * L + c;
              b_iters[dm] = S.iters[src];
              b_flags[dm] = S.flags[src];
              b_maxrel[dm] = S.maxrel[src];
            }
          }
      b_sweeps = std::max(b_sweeps, S.sweeps);
      b_fp64 = b_fp64 || S.fp64_continued;
      CBS_TRY(lap(&res->ms_solve));
      // ---- step 2: this wave's share of the moments
      CBS_TRY(launch_moments(nsys, ne, nwv, j0, M, N, L, S.Y, coef, Sm, j0 > 0, mirror ? n_int : 0, st));
      CBS_TRY(launch_mu(nsys, ne, nwv, j0, M, N, L, dV, S.Y, coef, part, mu, j0 > 0, mirror ? n_int : 0, v_real, st));
      CBS_TRY(lap(&res->ms_moments));
    }
    // ---- step 3: extraction (Hankel SVD, reduced eigenproblem, vectors, residuals)
    const int n = nLM;   // order of the block Hankel matrices
    const size_t nn = (size_t)n * n;
    DevBuf xbuf;
    CBS_TRY(xbuf.alloc(nn * sizeof(double2) * 9 * ne + (size_t)ne * n * (sizeof(double) + 2 * sizeof(double2) + sizeof(int)) + 4096));
    double2 *T = xbuf.as<double2>();
    double2 *Tl = T + nn * ne, *Aw = Tl + nn * ne, *Ww = Aw + nn * ne, *U = Ww + nn * ne,
            *Ws = U + nn * ne, *C1 = Ws + nn * ne, *Bm = C1 + nn * ne, *Z = Bm + nn * ne;
    double2 *Yc = T;   // T is dead once copied into Aw
    double2 *tau = Z + nn * ne;
    double *sig = (double *)(tau + (size_t)ne * n);
    int *ridx = (int *)(sig + (size_t)ne * n);
    DevBuf sbuf;   // mhat[ne], nring[ne], info_svd[ne], info_eig[ne]
    CBS_TRY(sbuf.alloc((size_t)4 * ne * sizeof(int) + 64));
    int *small = sbuf.as<int>();
    int *mhat = small, *nring = small + ne, *isvd = small + 2 * ne, *ieig = small + 3 * ne;
    CBS_TRY(launch_hankel(ne, L, M, mu, T, Tl, st));
    CBS_CUDA(cudaMemcpyAsync(Aw, T, nn * ne * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    CBS_TRY(launch_svd(ne, n, Aw, Ww, U, Ws, sig, isvd, st));
    CBS_TRY(launch_rank(ne, n, sig, o.delta, mhat, st));
    CBS_TRY(lap(&res->ms_svd));
    const double2 one = make_double2(1, 0), zero = make_double2(0, 0);
    // C1 = T^< W (all n columns), Bm = U^dagger C1, then columns j < m_hat scaled by 1/sigma_j
    if (o.extraction == CBS_HANKEL) {
      CBS_TRY(zgemm(0, 0, n, n, n, one, Tl, n, nn, Ws, n, nn, zero, C1, n, nn, ne, st));
      CBS_TRY(zgemm(2, 0, n, n, n, one, U, n, nn, C1, n, nn, zero, Bm, n, nn, ne, st));
      CBS_TRY(launch_scale(ne, n, n, mhat, sig, Bm, 0, st));
      CBS_TRY(launch_eig(ne, n, mhat, Bm, Z, tau, Yc, nring, ridx, ct->lambda_min, ieig, st));
    } else {
      CBS_CUDA(cudaMemsetAsync(small + ne, 0, (size_t)3 * ne * sizeof(int), st));
    }
    CBS_TRY(lap(&res->ms_reduced));
    std::vector<int> hsmall(4 * ne);
    std::vector<double> hsig((size_t)ne * n);
    std::vector<double2> htau((size_t)ne * n);
    std::vector<double2> hmu((size_t)ne * 2 * M * L * L);
    CBS_CUDA(cudaMemcpyAsync(hsmall.data(), small, 4 * ne * sizeof(int), cudaMemcpyDeviceToHost, st));
    CBS_CUDA(cudaMemcpyAsync(hsig.data(), sig, hsig.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    CBS_CUDA(cudaMemcpyAsync(htau.data(), tau, htau.size() * sizeof(double2), cudaMemcpyDeviceToHost, st));
    CBS_CUDA(cudaMemcpyAsync(hmu.data(), mu, hmu.size() * sizeof(double2), cudaMemcpyDeviceToHost, st));
    CBS_CUDA(cudaStreamSynchronize(st));
    for (int e = 0; e < ne; ++e) {
      cbs_energy_result &R = res->e[e0 + e];
      const double Ee = energies[e0 + e];
      const int m = hsmall[e], cnt = hsmall[ne + e];
      memset(&R.st, 0, sizeof(R.st));
      R.st.rank = m;
      R.st.n_extracted = m;
      R.st.sigma_max = hsig[(size_t)e * n];
      R.st.sigma_cut = m > 0 ? hsig[(size_t)e * n + m - 1] : 0.0;
      R.lam_all.assign(htau.begin() + (size_t)e * n, htau.begin() + (size_t)e * n + m);
      R.res_all.assign(m, NAN);
      R.mu.assign(hmu.begin() + (size_t)e * 2 * M * L * L, hmu.begin() + (size_t)(e + 1) * 2 * M * L * L);
      R.iters.assign((size_t)n_int * L, 0);
      int mx = 0, fl = 0;
      double mr = 0;
      for (int j = 0; j < n_int; ++j)
        for (int c = 0; c < L; ++c) {
          const size_t k = ((size_t)e * n_int + j) * L + c;
          R.iters[(size_t)j * L + c] = b_iters[k];
          mx = std::max(mx, b_iters[k]);
          fl |= b_flags[k];
          mr = std::max(mr, b_maxrel[k]);
        }
      R.st.max_iters = mx;
      R.st.sweeps = b_sweeps;
      R.st.max_solve_residual = mr;
      R.st.flags = (fl & 3) | (m == n ? 4 : 0) | (hsmall[2 * ne + e] ? 8 : 0) | (hsmall[3 * ne + e] ? 16 : 0) |
                   (b_fp64 ? 32 : 0) | (fl & 64);
      if (fl & 2) ret = (ret == CBS_OK ? CBS_EBREAKDOWN : ret);
      else if (fl & 1) ret = (ret == CBS_OK ? CBS_ENOCONV : ret);
      else if (m == n && ret == CBS_OK) ret = CBS_WRANK;
      // residual of every candidate (lambda in the ring), filter, sort, normalise, copy out
      auto finish = [&](int cnt, double2 *Psi, const double2 *twr_src, const int *ring_host) -> cbs_status {
        DevBuf vb;
        const size_t psi_bytes = (size_t)N * cnt * sizeof(double2);
        const size_t dsz = (size_t)(H.n_atoms ? H.n_atoms : 1) * H.np4 * cnt * sizeof(double2);
        CBS_TRY(vb.alloc(psi_bytes + dsz + (size_t)cnt * 256 + 8192));
        char *p = vb.as<char>();
        auto take = [&](size_t sz) { char *r = p; p += (sz + 255) & ~(size_t)255; return (void *)r; };
        double2 *Res = (double2 *)take(psi_bytes);
        double2 *Dd = (double2 *)take(dsz);
        double2 *twr = (double2 *)take((size_t)cnt * sizeof(double2));
        double *stats = (double *)take((size_t)cnt * 4 * sizeof(double));
        double *rho_all = (double *)take((size_t)cnt * sizeof(double));
        int *perm = (int *)take((size_t)cnt * sizeof(int));
        double2 *lam_o = (double2 *)take((size_t)cnt * sizeof(double2));
        double2 *k_o = (double2 *)take((size_t)cnt * sizeof(double2));
        double *rho_o = (double *)take((size_t)cnt * sizeof(double));
        double2 *scale = (double2 *)take((size_t)cnt * sizeof(double2));
        int *nkeep = (int *)take(256);
        double *Ed = (double *)take(256);
        CBS_CUDA(cudaMemcpyAsync(Ed, &Ee, sizeof(double), cudaMemcpyHostToDevice, st));
        CBS_CUDA(cudaMemcpyAsync(twr, twr_src, (size_t)cnt * sizeof(double2), cudaMemcpyDeviceToDevice, st));
        CBS_TRY(apply_P<double>(H, 1, cnt, Psi, Res, twr, true, Ed, Dd, nullptr, st));
        double nHp, nA, nHm;
        cbs_hamiltonian_norms(h, Ee, &nHp, &nA, &nHm);
        const double a_cell = h->hz * H.nz;
        CBS_TRY(launch_filter(N, cnt, twr, Psi, Res, stats, nHp, nA, nHm, o.rho_max, a_cell, rho_all,
                              nkeep, perm, lam_o, k_o, rho_o, scale, st));
        int hk = 0;
        std::vector<double> hrho(cnt);
        CBS_CUDA(cudaMemcpyAsync(&hk, nkeep, sizeof(int), cudaMemcpyDeviceToHost, st));
        CBS_CUDA(cudaMemcpyAsync(hrho.data(), rho_all, cnt * sizeof(double), cudaMemcpyDeviceToHost, st));
        CBS_CUDA(cudaStreamSynchronize(st));
        if (ring_host)
          for (int r = 0; r < cnt; ++r) R.res_all[ring_host[r]] = hrho[r];
        R.st.n_kept = hk;
        R.lam.resize(hk);
        R.k.resize(hk);
        R.rho.resize(hk);
        R.vec.resize((size_t)N * hk);
        if (hk > 0) {
          CBS_TRY(launch_gather_vectors(N, cnt, hk, Psi, perm, scale, Res, st));
          CBS_CUDA(cudaMemcpyAsync(R.lam.data(), lam_o, hk * sizeof(double2), cudaMemcpyDeviceToHost, st));
          CBS_CUDA(cudaMemcpyAsync(R.k.data(), k_o, hk * sizeof(double2), cudaMemcpyDeviceToHost, st));
          CBS_CUDA(cudaMemcpyAsync(R.rho.data(), rho_o, hk * sizeof(double), cudaMemcpyDeviceToHost, st));
          CBS_CUDA(cudaMemcpyAsync(R.vec.data(), Res, (size_t)N * hk * sizeof(double2), cudaMemcpyDeviceToHost, st));
        }
        CBS_CUDA(cudaStreamSynchronize(st));
        return CBS_OK;
      };
      if (o.extraction == CBS_RR) {
        void *rws = nullptr;
        int rcnt = 0, rrank = 0;
        double2 *rlam = nullptr, *rPsi = nullptr;
        std::vector<double2> rall;
        cbs_status rs = m > 0 ? cbs_internal_rr(h, Ee, Sm + (size_t)e * N * n, Ws + nn * e, n, m,
                                                ct->lambda_min, st, &rws, &rcnt, &rlam, &rPsi, &rall,
                                                &rrank)
                              : CBS_OK;
        if (rs == CBS_OK) {
          R.st.rank = rrank;
          R.st.n_extracted = (int)rall.size();
          R.lam_all = rall;
          R.res_all.assign(rall.size(), NAN);
          if (rcnt > 0) rs = finish(rcnt, rPsi, rlam, nullptr);
        }
        cudaStreamSynchronize(st);
        if (rws) cudaFree(rws);
        if (rs != CBS_OK) return rs;
        continue;
      }
      if (cnt == 0) continue;
      {
        // vectors: P1 = Z Yc (m x cnt), rows / sigma, C2 = W_1 P1 (n x cnt), Psi^T = C2^T S^T
        DevBuf vb;
        const size_t psi_bytes = (size_t)N * cnt * sizeof(double2);
        CBS_TRY(vb.alloc(psi_bytes + (size_t)n * cnt * 2 * sizeof(double2) + (size_t)cnt * 64 + 4096));
        char *p = vb.as<char>();
        auto take = [&](size_t sz) { char *r = p; p += (sz + 255) & ~(size_t)255; return (void *)r; };
        double2 *Psi = (double2 *)take(psi_bytes);
        double2 *P1 = (double2 *)take((size_t)n * cnt * sizeof(double2));
        double2 *C2 = (double2 *)take((size_t)n * cnt * sizeof(double2));
        double2 *twr = (double2 *)take((size_t)cnt * sizeof(double2));
        CBS_TRY(zgemm(0, 0, m, cnt, m, one, Z + nn * e, n, 0, Yc + nn * e, n, 0, zero, P1, n, 0, 1, st));
        k_scale_rows<<<64, 256, 0, st>>>(m, cnt, n, sig + (size_t)e * n, P1); cbs::count_launches(1);
        CBS_CUDA(cudaGetLastError());
        CBS_TRY(zgemm(0, 0, n, cnt, m, one, Ws + nn * e, n, 0, P1, n, 0, zero, C2, n, 0, 1, st));
        // Psi (row-major N x cnt) = S (row-major N x n) C2  <=>  Psi^T = C2^T S^T (column-major)
        CBS_TRY(zgemm(1, 0, cnt, (int)N, n, one, C2, n, 0, Sm + (size_t)e * N * n, n, 0, zero, Psi, cnt, 0, 1, st));
        k_gather_tau<<<ceil_div(cnt, 128), 128, 0, st>>>(cnt, tau + (size_t)e * n, ridx + (size_t)e * n, twr); cbs::count_launches(1);
        CBS_CUDA(cudaGetLastError());
        std::vector<int> hridx(cnt);
        CBS_CUDA(cudaMemcpyAsync(hridx.data(), ridx + (size_t)e * n, cnt * sizeof(int), cudaMemcpyDeviceToHost, st));
        CBS_CUDA(cudaStreamSynchronize(st));
        CBS_TRY(finish(cnt, Psi, twr, hridx.data()));
      }
    }
    CBS_TRY(lap(&res->ms_vectors));
  }
  res->ms_extract = res->ms_svd + res->ms_reduced + res->ms_vectors;
  res->ms_total = res->ms_solve + res->ms_moments + res->ms_extract;
  return ret;
}

extern "C" cbs_status cbs_solve(const cbs_hamiltonian *h, const double *energies, int n_e,
                                const cbs_contour *contour, int L, int M, const void *V,
                                const cbs_options *opt, cbs_result **out) {
  if (!out) { set_error("out is NULL"); return CBS_EINVAL; }
  *out = nullptr;
  if (!h || !energies || n_e < 1 || !contour || !V || L < 1 || M < 1 || L * M > 512 || L > 64 ||
      M > 16 || contour->n_int < 1 || !(contour->lambda_min > 0 && contour->lambda_min < 1)) {
    set_error("cbs_solve: bad argument (1 <= L <= 64, 1 <= M <= 16, L*M <= 512, 0 < lambda_min < 1)");
    return CBS_EINVAL;
  }
  for (int e = 0; e < n_e; ++e)
    if (!isfinite(energies[e])) { set_error("energies must be finite"); return CBS_EINVAL; }
  if (cbs_hamiltonian_size(h) > (int64_t)32 * 65535) {
    set_error("cbs_solve: grid larger than 2,097,120 points");
    return CBS_EINVAL;
  }
  cbs_options o;
  CBS_TRY(check_opts(opt, &o));
  if (o.stop_fraction < 1.0 && contour->n_int > 1024) {
    set_error("cbs_solve: stop_fraction < 1 needs n_int <= 1024");
    return CBS_EINVAL;
  }
  StreamGuard sg;
  CBS_TRY(sg.open(o.stream));
  cbs_result *res = new (std::nothrow) cbs_result();
  if (!res) { set_error("host allocation failed"); return CBS_ENOMEM; }
  cbs_status s = solve_impl(h, energies, n_e, contour, L, M, V, o, sg.st, res);
  if (s != CBS_OK && s != CBS_ENOCONV && s != CBS_EBREAKDOWN && s != CBS_WRANK) {
    delete res;
    return s;
  }
  *out = res;
  return s;
}

// Several cells in one call: one host thread and one stream per cell, each running the
// cbs_solve path, so that the cells' work interleaves on the device (one cell's extraction,
// on one SM per energy, runs beside another cell's FP64 solves).
extern "C" cbs_status cbs_solve_cells(const cbs_hamiltonian *const *h, int n_cells, const double *energies,
                                      int n_e, const cbs_contour *contour, int L, int M,
                                      const void *const *V, const cbs_options *opt, cbs_result **out,
                                      cbs_status *cell_status) {
  if (!out) { set_error("out is NULL"); return CBS_EINVAL; }
  if (!h || !V || n_cells < 1 || n_cells > 64) {
    set_error("cbs_solve_cells: bad argument (1 <= n_cells <= 64, h and V non-NULL)");
    return CBS_EINVAL;
  }
  for (int c = 0; c < n_cells; ++c) out[c] = nullptr;
  for (int c = 0; c < n_cells; ++c) {
    if (!h[c] || !V[c]) { set_error("cbs_solve_cells: NULL Hamiltonian or V of a cell"); return CBS_EINVAL; }
    for (int d = 0; d < c; ++d)
      if (h[d] == h[c]) { set_error("cbs_solve_cells: a Hamiltonian handle appears twice"); return CBS_EINVAL; }
  }
  if (opt && opt->stream) {
    set_error("cbs_solve_cells: every cell runs on a stream of its own; opt->stream must be NULL");
    return CBS_EINVAL;
  }
  int dev = 0;
  CBS_CUDA(cudaGetDevice(&dev));
  std::vector<cbs_status> st((size_t)n_cells, CBS_OK);
  std::vector<std::string> err((size_t)n_cells);
  std::vector<std::thread> th;
  th.reserve((size_t)n_cells);
  for (int c = 0; c < n_cells; ++c)
    th.emplace_back([&, c]() {
      const cudaError_t ce = cudaSetDevice(dev);
      if (ce != cudaSuccess) st[c] = cuda_fail(ce, "cudaSetDevice");
      else st[c] = cbs_solve(h[c], energies, n_e, contour, L, M, V[c], opt, &out[c]);
      if (st[c] != CBS_OK) err[c] = cbs_last_error();
    });
  for (auto &t : th) t.join();
  if (cell_status)
    for (int c = 0; c < n_cells; ++c) cell_status[c] = st[c];
  auto soft = [](cbs_status x) { return x == CBS_OK || x == CBS_ENOCONV || x == CBS_EBREAKDOWN || x == CBS_WRANK; };
  for (int c = 0; c < n_cells; ++c)
    if (!soft(st[c])) {
      for (int d = 0; d < n_cells; ++d) {
        cbs_result_free(out[d]);
        out[d] = nullptr;
      }
      set_error("cell " + std::to_string(c) + ": " + err[c]);
      return st[c];
    }
  for (int c = 0; c < n_cells; ++c)
    if (st[c] != CBS_OK) {
      set_error("cell " + std::to_string(c) + ": " + err[c]);
      return st[c];
    }
  return CBS_OK;
}

extern "C" int cbs_result_count(const cbs_result *r, int e) {
  if (!r || e < 0 || e >= r->n_e) return -1;
  return (int)r->e[e].lam.size();
}

extern "C" cbs_status cbs_result_get(const cbs_result *r, int e, double *lambda, double *k,
                                     double *residual, double *vectors) {
  if (!r || e < 0 || e >= r->n_e) { set_error("bad result/energy index"); return CBS_EINVAL; }
  const cbs_energy_result &R = r->e[e];
  if (lambda) memcpy(lambda, R.lam.data(), R.lam.size() * sizeof(double2));
  if (k) memcpy(k, R.k.data(), R.k.size() * sizeof(double2));
  if (residual) memcpy(residual, R.rho.data(), R.rho.size() * sizeof(double));
  if (vectors) memcpy(vectors, R.vec.data(), R.vec.size() * sizeof(double2));
  return CBS_OK;
}

extern "C" cbs_status cbs_result_stats(const cbs_result *r, int e, cbs_stats *st) {
  if (!r || e < 0 || e >= r->n_e || !st) { set_error("bad result/energy index"); return CBS_EINVAL; }
  *st = r->e[e].st;
  return CBS_OK;
}

extern "C" cbs_status cbs_result_all(const cbs_result *r, int e, double *lambda, double *residual) {
  if (!r || e < 0 || e >= r->n_e) { set_error("bad result/energy index"); return CBS_EINVAL; }
  const cbs_energy_result &R = r->e[e];
  if (lambda) memcpy(lambda, R.lam_all.data(), R.lam_all.size() * sizeof(double2));
  if (residual) memcpy(residual, R.res_all.data(), R.res_all.size() * sizeof(double));
  return CBS_OK;
}

extern "C" cbs_status cbs_result_moments(const cbs_result *r, int e, double *mu) {
  if (!r || e < 0 || e >= r->n_e || !mu) { set_error("bad result/energy index"); return CBS_EINVAL; }
  memcpy(mu, r->e[e].mu.data(), r->e[e].mu.size() * sizeof(double2));
  return CBS_OK;
}

extern "C" cbs_status cbs_result_iters(const cbs_result *r, int e, int *iters) {
  if (!r || e < 0 || e >= r->n_e || !iters) { set_error("bad result/energy index"); return CBS_EINVAL; }
  memcpy(iters, r->e[e].iters.data(), r->e[e].iters.size() * sizeof(int));
  return CBS_OK;
}

extern "C" cbs_status cbs_result_extract_timing(const cbs_result *r, double *ms_svd,
                                                double *ms_reduced, double *ms_vectors) {
  if (!r) { set_error("null result"); return CBS_EINVAL; }
  if (ms_svd) *ms_svd = r->ms_svd;
  if (ms_reduced) *ms_reduced = r->ms_reduced;
  if (ms_vectors) *ms_vectors = r->ms_vectors;
  return CBS_OK;
}

extern "C" cbs_status cbs_result_timing(const cbs_result *r, double *ms_solve, double *ms_moments,
                                        double *ms_extract, double *ms_total) {
  if (!r) { set_error("null result"); return CBS_EINVAL; }
  if (ms_solve) *ms_solve = r->ms_solve;
  if (ms_moments) *ms_moments = r->ms_moments;
  if (ms_extract) *ms_extract = r->ms_extract;
  if (ms_total) *ms_total = r->ms_total;
  return CBS_OK;
}

extern "C" cbs_status cbs_result_profile(const cbs_result *r, int dtype, double *ms, double *launches,
                                         double *outputs) {
  if (!r || (dtype != CBS_C128 && dtype != CBS_C64 && dtype != CBS_PROFILE_SHIFT_UPDATE)) {
    set_error("bad result or dtype");
    return CBS_EINVAL;
  }
  if (ms) *ms = r->prof_ms[dtype];
  if (launches) *launches = r->prof_launches[dtype];
  if (outputs) *outputs = r->prof_outputs[dtype];
  return CBS_OK;
}

extern "C" void cbs_result_free(cbs_result *r) { delete r; }

// Ring solves for the objective/adjoint entry point: n systems at the outer-circle points
// and their duals; *Y_out points to [2n][N][L] FP64 solutions owned by *owner (release with
// cbs_internal_ring_release).
cbs_status cbs_internal_ring_solve(const cbs_hamiltonian *h, int n, int L, const double2 *zs,
                                   const double *Es, const double2 *dV, const cbs_options &o,
                                   cudaStream_t st, double2 **Y_out, void **owner) {
  ShiftedSolver *S = new (std::nothrow) ShiftedSolver();
  if (!S) { set_error("host allocation failed"); return CBS_ENOMEM; }
  *owner = S;
  cbs_status s = S->run(h->v, n, L, zs, Es, dV, o, st);
  if (s != CBS_OK) return s;
  *Y_out = S->Y;
  int fl = 0;
  for (int f : S->flags) fl |= f;
  if (fl & 2) { set_error("BiCG breakdown in some column"); return CBS_EBREAKDOWN; }
  if (fl & 1) { set_error("BiCG did not converge in some column"); return CBS_ENOCONV; }
  return CBS_OK;
}

void cbs_internal_ring_release(void *owner) { delete (ShiftedSolver *)owner; }
