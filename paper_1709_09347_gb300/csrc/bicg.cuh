// Batched BiCG for the shifted systems of §3.2 and their duals.
#pragma once

#include "common.cuh"

namespace cbs {

// State for n systems x L columns; the dual of system s is stored as system n + s.
template <typename R>
struct Bicg {
  typedef typename CT<R>::T C;
  HamView H;
  int n = 0, L = 0;
  int64_t N = 0;
  int chunk_pts = 0, n_chunks = 0;
  C *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr;   // [2n][N][L]
  C *D = nullptr;                                             // [2n][n_atoms][n_proj][L]
  double2 *tw = nullptr;                                      // [2n]
  double *E = nullptr;                                        // [2n]
  double2 *rho = nullptr, *alpha = nullptr, *beta = nullptr;  // [n][L]
  double2 *rho_prev = nullptr;                                // [n][L]
  double *tgt = nullptr, *tgtd = nullptr;                     // [n][L] absolute stop targets
  double *rmax = nullptr, *rmaxd = nullptr;                   // [n][L] max ||r|| since (re)start
  double tfac = 0;                                            // relative pause factor
  double *nb = nullptr, *nbd = nullptr;                       // [n][L]
  int *active = nullptr, *iters = nullptr, *flags = nullptr;  // [n][L]
  int *sys_active = nullptr;                                  // [2n]
  int *n_active = nullptr;                                    // [1]
  double *part = nullptr;                                     // [n][n_chunks][L][4]
  void *block = nullptr;
  size_t bytes = 0;
  // profiling of the operator-apply launches (events around each apply inside the graph)
  bool profile = false;
  cudaEvent_t prof_ev[2 * 64] = {};
  int n_prof_ev = 0;
  unsigned long long *sys_apply = nullptr;   // device: active systems summed over applies
  double prof_ms = 0, prof_launches = 0;
  // the captured iteration graph is reused across iterate() calls with the same shape
  cudaGraphExec_t exec = nullptr;
  int exec_max_iter = -1, exec_check_every = -1;
  uint64_t exec_kernels = 0;
  int *h_active = nullptr;                   // pinned host word for the convergence poll

  static size_t bytes_needed(const HamView &H, int n, int L);
  cbs_status alloc(const HamView &H, int n, int L);
  void release();
  // Set twists/energies: primal twist z[s], dual twist 1/conj(z[s]); z, E on device.
  cbs_status set_systems(const double2 *z, const double *Es, cudaStream_t st);
  // Initialise with primal RHS B (stride bstride elements between systems, 0 = shared)
  // and dual RHS Bd; columns with colmask == 0 (if colmask) start inactive.  A column
  // stops when ||r|| <= max(tfac * max||r|| since the (re)start, tfloor ||b||), and the
  // same for the dual (tfac = 0: plain tolerance tfloor).
  cbs_status init(const double2 *B, int64_t bstride, const double2 *Bd, int64_t bdstride,
                  const int *colmask, double tfloor, double tfac, cudaStream_t st,
                  const double *ref_norm = nullptr);
  // Iterate until every column reached its target, broke down or reached max_iter
  // iterations in total; call_cap > 0 bounds the iterations of this call.
  cbs_status iterate(double tol, int max_iter, int check_every, cudaStream_t st,
                     int *host_iters_done, int call_cap = 0);
  // Residual replacement from FP64 true residuals R64 [2n][N][L]; columns with
  // colmask != 0 resume from them.
  cbs_status replace(const double2 *R64, const int *colmask, cudaStream_t st);
  // one iteration (captured into graphs); k indexes the iteration inside the graph
  cbs_status step(double tol, int max_iter, cudaStream_t st, int k);
  // outputs written by the apply launches so far (2 * active systems * N * L)
  cbs_status prof_outputs(cudaStream_t st, double *out);
};

// Elementwise helpers used by the refinement driver.
// R = B - R (in place) for 2n systems, with column norms of the result into part.
cbs_status launch_residual(int n2, int64_t N, int L, const double2 *B, int64_t bstride,
                           const double2 *Bd, int64_t bdstride, int n, double2 *AY,
                           double *colnorm2 /*[2n][L]*/, cudaStream_t st);
// Y[2n] += (double) X32[2n]
cbs_status launch_accumulate(int64_t count, double2 *Y, const float2 *X, cudaStream_t st);
cbs_status launch_accumulate(int64_t count, double2 *Y, const double2 *X, cudaStream_t st);
// X[2n] (type C) copies of Y (double) are not needed; zero fill helper
cbs_status launch_twists(int n, const double2 *z, const double *E, double2 *tw, double *E2,
                         cudaStream_t st);

}  // namespace cbs
