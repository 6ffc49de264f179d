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
  // load-balance rule (§3.3): systems come in groups of `group` quadrature points of one
  // energy (0 = no groups); a group's remaining systems stop once more than group_need of
  // them have stopped
  int group = 0, group_need = 0;

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

// One BiCG Krylov sequence per (quadrature point, column) shared by a family of energies
// (shifted BiCG; not in the paper).  For a fixed twist z, P(z, E_e) = P(z, E_0) + s_e I with
// the real shift s_e = E_e - E_0, so the Krylov spaces of all energies coincide and the
// BiCG residual of energy e is collinear with the seed's: r_e = r / pi_e.  With the seed's
// alpha_k, beta_{k-1} and gamma_k = alpha_k beta_{k-1} / alpha_{k-1} (0 at k = 0):
//     pi_e^{k+1} = (1 + alpha_k s_e) pi_e^k + gamma_k (pi_e^k - pi_e^{k-1}),  pi^0 = pi^{-1} = 1
//     alpha_e = alpha_k pi_e^k / pi_e^{k+1},  beta_e = (pi_e^{k-1} / pi_e^k)^2 beta_{k-1}
//     p_e = r / pi_e^k + beta_e p_e,  x_e += alpha_e p_e
// and for the dual system (P(z, E)^dagger, E real) the same with conjugated coefficients.
// The directions are stored scaled, p^_e = pi_e^k p_e, which turns the update into
// p^_e = r + (pi_e^{k-1}/pi_e^k) beta_{k-1} p^_e and x_e += (alpha_k / pi_e^{k+1}) p^_e.
// Energy e of point j stops when ||r|| / |pi_e| and ||r~|| / |pi_e| are below tol ||b||;
// the seed runs while any of its energies is active.  Outputs X [2n][N][L] with
// n = n_sh * n_pt systems ordered e * n_pt + j (primal), then their duals.
// R = double: the whole family in FP64.  R = float: the seed recursion, the scaled
// directions and the solutions in complex64 (the scalar recurrences for pi, alpha, beta
// stay in FP64); its solutions are accurate to the single-precision level and are refined
// per energy afterwards.
template <typename R>
struct MultiShift {
  typedef typename CT<R>::T C;
  Bicg<R> seed;                           // n_pt seed systems (and duals) at energy E_0
  int n_pt = 0, n_sh = 0, L = 0;
  int64_t N = 0;
  C *X = nullptr;                         // [2n][N][L] solutions (separate allocation)
  C *P = nullptr;                         // [2n][N][L] scaled search directions pi_e p_e
  double2 *pi = nullptr, *pi_prev = nullptr;            // [n][L]
  double2 *cb = nullptr, *ca = nullptr;  // [n][L] this iteration's coefficients
  double2 *alpha_prev = nullptr;          // [n_pt][L]
  double *sigma = nullptr;                // [n_sh] E_e - E_0
  int *sactive = nullptr, *siters = nullptr, *sflags = nullptr;   // [n][L]
  void *block = nullptr, *xblock = nullptr;
  cudaGraphExec_t exec = nullptr;
  int exec_max_iter = -1, exec_check_every = -1;
  uint64_t exec_kernels = 0;
  // profiling of the update kernel (events around each launch inside the graph) and the
  // number of active (energy, point, column) triples it processed
  cudaEvent_t upd_ev[2 * 64] = {};
  int n_upd_ev = 0;
  double upd_ms = 0, upd_launches = 0;
  unsigned long long *upd_cols = nullptr;
  // load-balance rule (§3.3): an energy's remaining points stop once more than group_need
  // of its n_pt points have converged (group_need >= n_pt: off)
  int group_need = 1 << 30;

  static size_t bytes_needed(const HamView &H, int n_pt, int n_sh, int L);
  cbs_status update_columns(cudaStream_t st, double *out);
  // twists z1 [n_pt] (device), shifts sigma_h [n_sh] (host) relative to E0.
  cbs_status alloc(const HamView &H, int n_pt, int n_sh, int L);
  cbs_status init(const double2 *z1, double E0, const double *sigma_h, const double2 *B,
                  double tol, cudaStream_t st);
  cbs_status step(int max_iter, cudaStream_t st, int k);
  cbs_status iterate(int max_iter, int check_every, cudaStream_t st, int *host_iters_done);
  void release();        // everything but X
  void release_x();
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
