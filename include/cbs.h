/*
 * libcbs — complex band structure by the Sakurai-Sugiura contour-integral method,
 * GB300-native (sm_103a).  C ABI.
 *
 * Method (Iwase, Futamura, Imakura, Sakurai, Ono, SC17, arXiv 1709.09347):
 *   A crystal is cut into unit cells along the transport axis z.  Inside one cell the
 *   real-space Kohn-Sham Hamiltonian (central finite-difference Laplacian + local
 *   potential + separable non-local projectors) couples only to the neighbouring
 *   cells (§2, Eq. (2)).  The Bloch ansatz psi_{n+l} = lambda^l psi_n (Eq. (3)) turns
 *   the Kohn-Sham equation into the quadratic eigenvalue problem (Eq. (4))
 *
 *       P(lambda) psi = [ -lambda^{-1} H- + (E - H0) - lambda H+ ] psi = 0,
 *
 *   i.e. P(z) = E - H(z) with H(z) = H0 + z H+ + z^{-1} H- the cell Hamiltonian with a
 *   twisted-periodic boundary along z.  Only lambda in the ring
 *   lambda_min < |lambda| < 1/lambda_min (Eq. (5)) are wanted; they are found with
 *   Algorithm 1 (§3.1) on the two-circle contour of §3.2, whose cost is the batch of
 *   shifted solves P(z_j) Y_j = V and their duals P(z_j)^dagger Y~_j = V (Eq. (9),
 *   (11)), done by BiCG (§3.2).
 *
 * Conventions for every entry point:
 *   - complex numbers are interleaved (re, im) pairs of double (complex128) or float
 *     (complex64);
 *   - grid index i = ix + nx*(iy + ny*iz) (x fastest);
 *   - a block of L vectors over the grid is stored row-major as [N][L] (the L columns
 *     of one grid point are contiguous); a batch of such blocks is [n_sys][N][L];
 *   - every call returns a cbs_status; nothing is thrown across the ABI;
 *     cbs_last_error() returns a message for the calling thread's last failure;
 *   - inputs are caller-owned and never retained; handles are library-owned and
 *     released with the matching *_free call.
 */
#ifndef CBS_H
#define CBS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cbs_hamiltonian cbs_hamiltonian; /* opaque, device-resident */
typedef struct cbs_result cbs_result;           /* opaque, host-resident   */

typedef enum {
  CBS_OK = 0,
  CBS_EINVAL = 1,      /* bad argument or unsupported size                         */
  CBS_ENOMEM = 2,      /* device or host allocation failed                        */
  CBS_ECUDA = 3,       /* a CUDA runtime call failed                               */
  CBS_ENOCONV = 4,     /* some BiCG columns hit max_iter; results are still readable */
  CBS_EBREAKDOWN = 5,  /* BiCG breakdown (rho or (p~, Ap) vanished) in some column  */
  CBS_ETIMEOUT = 6,    /* a bounded device-side wait gave up                        */
  CBS_WRANK = 7        /* warning: numerical rank == L*M, eigenvalues may be missing */
} cbs_status;

/* cbs_options.precision: CBS_FP64 plain FP64 BiCG; CBS_FP32_REFINE complex64 BiCG with FP64
 * reliable updates (residual replacement). */
enum { CBS_FP64 = 0, CBS_FP32_REFINE = 1 };
enum { CBS_HANKEL = 0, CBS_RR = 1 };            /* cbs_options.extraction */
enum { CBS_C128 = 0, CBS_C64 = 1 };             /* element type of vector blocks */

/* Real-space grid of one unit cell: periodic in x and y, coupled to the neighbouring
 * cells along z.  fd_order in {2, 4, 6, 8, 10, 12}: central FD Laplacian of that order
 * (the paper's "nine-point" FD is order 8, §4).  Needs fd_order/2 <= nz. */
typedef struct {
  int nx, ny, nz;
  double hx, hy, hz;
  int fd_order;
} cbs_grid;

/* Separable non-local projectors: V_NL = sum_a sum_{cells n} |beta_{a,n}> h_a <beta_{a,n}|.
 * Support entries of atom a are sup_ptr[a] .. sup_ptr[a+1]-1; entry s is grid point
 * sup_idx[s] of cell 0, covered by the copy of atom a displaced by sup_wrap[s] in
 * {-1,0,+1} cells along z, with projector values sup_val[s*n_proj + mu] (already
 * multiplied by sqrt(dV)).  h is [n_atoms][n_proj][n_proj], symmetric.  A grid point
 * may appear at most once per atom (needs 2 r_c shorter than the cell along z).
 * n_proj <= 8. */
typedef struct {
  int n_atoms, n_proj;
  const int64_t *sup_ptr;
  const int32_t *sup_idx;
  const int8_t *sup_wrap;
  const double *sup_val;
  const double *h;
} cbs_projectors;

/* Two-circle contour of §3.2: radii 1/lambda_min and lambda_min, n_int points each at
 * angles theta_j = 2 pi (j - 1/2) / n_int. */
typedef struct {
  double lambda_min;
  int n_int;
} cbs_contour;

typedef struct {
  double tol;           /* BiCG stop: ||r||/||b|| <= tol and ||r~||/||b~|| <= tol (1e-10) */
  double delta;         /* rank cut: keep sigma_i >= delta * sigma_1 (1e-10)              */
  double rho_max;       /* keep eigenpairs with residual rho <= rho_max (1e-8)           */
  int max_iter;         /* BiCG iterations per column (FP64) / per inner solve (20000)   */
  int precision;        /* CBS_FP64 or CBS_FP32_REFINE (see above)                       */
  int extraction;       /* CBS_HANKEL (Algorithm 1) or CBS_RR (Rayleigh-Ritz)            */
  int check_every;      /* BiCG iterations per CUDA-graph replay between host polls (8)  */
  double inner_tol;     /* complex64 phase ends when ||r|| < inner_tol * max ||r|| since the
                           last FP64 residual update (0.1)                                */
  int max_sweeps;       /* FP64 residual updates (residual replacements) (200)           */
  int inner_max_iter;   /* iteration cap of one complex64 phase (1000)                   */
  int stall_sweeps;     /* updates without halving the FP64 residual before the columns
                           left are finished by FP64 BiCG (12)                             */
  int energies_per_batch; /* energies solved together; 0 = as many as fit (0)            */
  int profile;          /* 1: time every operator-apply launch with CUDA events (0)      */
  int multi_shift;      /* 1: one BiCG Krylov sequence per quadrature point and column
                           serves every energy of a batch, since
                           P(z, E) = P(z, E0) + (E - E0) I (shifted BiCG; not in the paper);
                           columns whose true residual misses tol are then refined per
                           energy from the shifted solution (FP64 BiCG with CBS_FP64; with
                           CBS_FP32_REFINE the family runs in complex64 down to family_tol and
                           the refinement is complex64 BiCG with FP64 reliable updates).
                           0: one BiCG per system (0)                                       */
  void *stream;         /* cudaStream_t to run on; NULL = the library's own stream       */
  double family_tol;    /* CBS_FP32_REFINE with multi_shift: relative residual at which an
                           energy leaves the complex64 family for its refinement
                           (0 = 1e-6; never below tol)                                      */
  double stop_fraction; /* load-balance rule of §3.3: once more than
                           floor(stop_fraction * n_int) quadrature points of an energy have
                           converged, BiCG stops at its other points (their columns get flag
                           bit 6 and are not refined).  Applies to cbs_solve with plain FP64
                           BiCG or with multi_shift.  1.0 = off (1.0; the paper uses 0.5)  */
  int points_per_wave;  /* quadrature points solved together; the moments are accumulated
                           wave by wave, so the solver state of only one wave is held at a
                           time (the rule above then counts the points of one wave).
                           0 = all points when one energy's fit in memory, else as many as
                           fit (0)                                                          */
  int conj_points;      /* 1: when every entry of V is real and n_int is even, solve only the
                           first n_int/2 outer-circle points: the blocks of Eq. (2) are real, so
                           P(conj z) = conj P(z) and the solutions at the conjugate points
                           z_{n_int-1-j} = conj(z_j) (and their duals) are the conjugates of the
                           solved ones (not in the paper).  0: solve every point (1)         */
} cbs_options;

/* Fill *opt with the defaults given above. */
cbs_status cbs_options_default(cbs_options *opt);

/* Build the device-resident Hamiltonian of one unit cell (§2, Eq. (2)).
 * v_loc: host array of N = nx*ny*nz doubles (local potential, Ha).
 * proj: host-side projector table, or NULL for none.
 * Computes the FD weights, uploads V_loc and the projector table (and its transpose:
 * for each grid point the (atom, entry) pairs that cover it), and the Frobenius norms
 * ||H+||_F and ||H-||_F on the device.  Errors: CBS_EINVAL for inconsistent sizes
 * (fd_order/2 > nz, a point covered twice by one atom, wrap outside {-1,0,1}, ...). */
cbs_status cbs_create_hamiltonian(const cbs_grid *grid, const double *v_loc,
                                  const cbs_projectors *proj, cbs_hamiltonian **out);
void cbs_hamiltonian_free(cbs_hamiltonian *h);

/* Replaces the local potential of h (§2: V_loc on the diagonal of H0) in place:
 * v_loc: N doubles, HOST or DEVICE pointer (detected).  The single-precision copy and the
 * Frobenius norms are recomputed on the device; the projector table and launch shapes are
 * kept.  A non-finite value returns CBS_EINVAL and leaves h unchanged.  Synchronises the
 * device; must not run concurrently with other work that uses h.  Lets a caller that
 * differentiates with respect to V_loc (cbs_objective) keep V_loc on the device. */
cbs_status cbs_hamiltonian_set_vloc(cbs_hamiltonian *h, const double *v_loc);

/* N = nx*ny*nz of the cell. */
int64_t cbs_hamiltonian_size(const cbs_hamiltonian *h);

/* ||H+||_F, ||H0 - E||_F, ||H-||_F (Frobenius) for the residual denominator. */
cbs_status cbs_hamiltonian_norms(const cbs_hamiltonian *h, double E, double *n_plus,
                                 double *n_zero, double *n_minus);

/* The QEP matrix applied to a batch (Eq. (4)):  Y[s] = P(z_s) X[s] = E_s X[s] - H(z_s) X[s].
 * z: host array of n_sys complex128 twists; E: host array of n_sys energies.
 * X, Y: DEVICE pointers to [n_sys][N][L] blocks of element type dtype (CBS_C128 or
 * CBS_C64).  1 <= L <= 256 (complex64 with even L: <= 512).  Runs on `stream`
 * (cudaStream_t, NULL = legacy default);
 * scratch is allocated per call and freed after synchronising that stream. */
cbs_status cbs_apply(const cbs_hamiltonian *h, int n_sys, const double *z, const double *E,
                     int L, const void *X, void *Y, int dtype, void *stream);

/* Bytes of device workspace cbs_apply_ws needs for n_sys systems of L columns. */
size_t cbs_apply_workspace_size(const cbs_hamiltonian *h, int n_sys, int L, int dtype);

/* As cbs_apply, with all pointers on the device and caller-provided workspace, so that
 * the call allocates nothing, does not synchronise and can be captured in a CUDA graph:
 * z: DEVICE complex128 [n_sys]; E: DEVICE double [n_sys]; workspace: DEVICE buffer of at
 * least cbs_apply_workspace_size bytes (16-byte aligned), overwritten by the call. */
cbs_status cbs_apply_ws(const cbs_hamiltonian *h, int n_sys, const double *z, const double *E,
                        int L, const void *X, void *Y, int dtype, void *workspace,
                        size_t workspace_bytes, void *stream);

/* As cbs_apply, for callers that must not allocate device memory: code running under an
 * allocator that owns all of the GPU's memory (a framework's memory pool, where a
 * cudaMalloc behind its back can fail or fragment the pool), and latency-bound services
 * that cannot afford cudaMalloc/cudaFree, which synchronise the device and stall other
 * streams.  This call allocates nothing: its scratch (twists, energies and the projector
 * coefficients) is a fixed 32 MiB array compiled into the library, present on every GPU
 * that loads the library's device code until the process exits.  The paper has no
 * counterpart to this entry point.
 * z, E: HOST arrays [n_sys]; X, Y: DEVICE [n_sys][N][L] of type dtype; runs on `stream`
 * and does not synchronise.  L as for cbs_apply, checked before anything is queued.  Sizes
 * whose scratch (about n_sys*L*n_atoms*4*16 bytes in complex128, half that in complex64)
 * exceed the 32 MiB return CBS_EINVAL.  The first call on a device looks up the array's
 * device address (with that device current); under CUDA's lazy module loading (the
 * default) that first call is also when the 32 MiB are reserved on the device, so make it
 * before a memory pool takes the device's free memory, and before any stream capture.  The
 * looked-up address is kept per device ordinal and is invalid after a device reset
 * (cudaDeviceReset).  All calls share the one array: calls whose GPU
 * work overlaps (on different streams or threads) race and must be serialised by the
 * caller. */
cbs_status cbs_apply_noalloc(const cbs_hamiltonian *h, int n_sys, const double *z, const double *E,
                             int L, const void *X, void *Y, int dtype, void *stream);

/* Autotuner for the operator apply (not in the paper, whose code has fixed launch shapes).
 * Times every admissible launch shape of the stencil kernel on n_sys systems of L columns
 * of type dtype (a thread block covers py x-lines of pz grid rows, py, pz powers of two, up
 * to 256 threads; for complex64 with even L and at most 4 projectors, also one versus two
 * columns per thread), with CUDA events on `stream`, a few applies each, and stores the
 * fastest in h:
 * every later apply of that precision through h (cbs_apply*, cbs_solve*, cbs_objective)
 * uses it.  Allocates and frees its own buffers (about 2 n_sys N L elements) and
 * synchronises `stream`.  Outputs (may be NULL): best_py, best_pz (x-lines and rows per
 * block), best_x2 (1 two columns per thread, -1 one, 0 not applicable), best_ms (one
 * apply, milliseconds).
 * Must not run concurrently with other work that uses h.  Every shape computes the same
 * arithmetic per output; the one- and two-column complex64 kernels may differ in the last
 * bit. */
cbs_status cbs_autotune_apply(cbs_hamiltonian *h, int n_sys, int L, int dtype, void *stream,
                              int *best_py, int *best_pz, int *best_x2, float *best_ms);

/* Sets the launch shape that cbs_autotune_apply would store (e.g. one tuned on another
 * handle of the same cell): py x-lines of pz rows per block (0 = default), x2 as best_x2
 * above (complex64 only; ignored for complex128).  A shape that does not fit a launch (py
 * times pz times the threads of one x-line above 256) is ignored at launch time.  Must not
 * run concurrently with other work that uses h. */
cbs_status cbs_set_apply_shape(cbs_hamiltonian *h, int dtype, int py, int pz, int x2);

/* Shifted solves of §3.2 for a batch of n_sys points: BiCG on P(z_s) Y[s] = B and, as
 * its dual, P(z_s)^dagger Yd[s] = B (= P(1/conj z_s) Yd[s] = B).
 * z, E: host arrays [n_sys]; B: DEVICE [N][L] complex128 (shared by all systems);
 * Y, Yd: DEVICE [n_sys][N][L] complex128 outputs; iters: host [n_sys][L] output (may be
 * NULL): per-column iterations (FP64) or total inner iterations (FP32_REFINE).
 * opt->precision selects plain FP64 BiCG or complex64 BiCG with FP64 refinement.
 * Returns CBS_ENOCONV / CBS_EBREAKDOWN if some column failed (outputs still written). */
cbs_status cbs_solve_shifted(const cbs_hamiltonian *h, int n_sys, const double *z,
                             const double *E, int L, const void *B, void *Y, void *Yd,
                             int *iters, const cbs_options *opt);

/* Whole method for a list of energies: contour, shifted solves, moments, Hankel (or
 * Rayleigh-Ritz) extraction, residual check, ring filter and k = -i ln(lambda)/a.
 * energies: host [n_e]; V: [N][L] complex128 right-hand sides, host or device pointer
 * (detected); M = N_mm moments (block Hankel of size L*M).  1 <= L, L*M <= 512.
 * *out receives a result handle also on CBS_ENOCONV / CBS_EBREAKDOWN / CBS_WRANK. */
cbs_status cbs_solve(const cbs_hamiltonian *h, const double *energies, int n_e,
                     const cbs_contour *contour, int L, int M, const void *V,
                     const cbs_options *opt, cbs_result **out);

/* The whole method for several cells of different sizes in one call (the paper distributes
 * supercells and energies over its top and middle parallel layers, §3.3): cell c is solved
 * exactly as cbs_solve(h[c], energies, n_e, contour, L, M, V[c], opt, &out[c]) would, on a
 * stream and a host thread of its own (created by the call, on the calling thread's current
 * device), so the cells' kernels interleave on the GPU; the call returns when every cell is
 * done.  h: [n_cells] distinct handles (1 <= n_cells <= 64), not used by other work meanwhile;
 * V: [n_cells] pointers, V[c] cell c's [N_c][L] complex128 block, host or device as in
 * cbs_solve; opt->stream must be NULL; out: [n_cells] result handles (free each with
 * cbs_result_free); cell_status: [n_cells] per-cell statuses, or NULL.
 * Errors: CBS_EINVAL for bad arguments (nothing is run); if a cell fails with anything other
 * than CBS_ENOCONV / CBS_EBREAKDOWN / CBS_WRANK, every out[c] is freed and NULL and that
 * cell's status is returned (cbs_last_error() names the cell); otherwise the first non-OK
 * status in cell order is returned, with every out[c] readable. */
cbs_status cbs_solve_cells(const cbs_hamiltonian *const *h, int n_cells, const double *energies,
                           int n_e, const cbs_contour *contour, int L, int M,
                           const void *const *V, const cbs_options *opt, cbs_result **out,
                           cbs_status *cell_status);

/* Objective of the ring solves and its gradient (reverse mode, adjoint solves).
 * J = sum_{c=1,2} sum_j c_j^(c) ||Y_j^(c)||_F^2, with Y_j^(c) = P(z_j^(c))^{-1} V the solutions
 * of the shifted systems of §3.2 (Eq. (9)-(11)) at energy E, and real weights
 * c_j^(c) = Re(s_c w_j^(c) sum_{k<M} (z_j^(c))^k), s_1 = +1, s_2 = -1 (the |Y|^2-weighted trace
 * of the moment sum).  If grad_vloc or grad_E is non-NULL, one adjoint BiCG batch gives
 * G = P^{-dagger} Y and
 *   grad_vloc[i] = dJ/dV_loc[i] = sum 2 c Re sum_col conj(G[i,col]) Y[i,col]   (host or device, [N]),
 *   *grad_E      = dJ/dE        = -sum 2 c Re tr(G^dagger Y).
 * The forward solutions are recomputed by every call (nothing is kept between a call that
 * only evaluates J and one that asks for the gradient).  V: [N][L] complex128, host or
 * device.  The adjoint solves run in FP64 to opt->tol. */
cbs_status cbs_objective(const cbs_hamiltonian *h, double E, const cbs_contour *contour, int L,
                         int M, const void *V, const cbs_options *opt, double *J,
                         double *grad_vloc, double *grad_E);

/* Per-energy results.  Eigenpairs are those with lambda_min < |lambda| < 1/lambda_min and
 * residual <= rho_max, sorted by |lambda| then arg(lambda); vectors have unit 2-norm and
 * their largest-modulus entry real positive. */
int cbs_result_count(const cbs_result *r, int e);
/* lambda, k: complex128 [count]; residual: double [count]; vectors: complex128
 * [N][count] (may be NULL).  Caller allocates. */
cbs_status cbs_result_get(const cbs_result *r, int e, double *lambda, double *k,
                          double *residual, double *vectors);

typedef struct {
  int rank;             /* numerical rank m_hat of the Hankel matrix (or of S for RR)  */
  int n_extracted;      /* eigenvalues of the reduced problem                          */
  int n_kept;           /* eigenpairs passing the ring and residual filter             */
  int max_iters;        /* largest BiCG iteration count over the energy's systems      */
  int sweeps;           /* FP64 refinement sweeps (0 for plain FP64)                   */
  int flags;            /* bit 0: not converged, bit 1: breakdown, bit 2: rank saturated,
                           bit 3/4: SVD/eigen-solver iteration limit, bit 5: FP64 continuation,
                           bit 6: some points stopped by the load-balance rule (stop_fraction) */
  double sigma_max, sigma_cut; /* sigma_1 and the smallest kept singular value          */
  double max_solve_residual;   /* max over systems/columns of ||V - P(z)Y||/||V|| (FP64) */
} cbs_stats;
cbs_status cbs_result_stats(const cbs_result *r, int e, cbs_stats *st);

/* All eigenvalues of the reduced problem before filtering, and their residuals.
 * lambda: complex128 [n_extracted], residual: double [n_extracted]. */
cbs_status cbs_result_all(const cbs_result *r, int e, double *lambda, double *residual);

/* The Hankel moments mu_k = V^dagger S_k, k < 2M: complex128 [2M][L][L]. */
cbs_status cbs_result_moments(const cbs_result *r, int e, double *mu);

/* Per-column BiCG iteration counts: int [n_int][L]. */
cbs_status cbs_result_iters(const cbs_result *r, int e, int *iters);

/* Milliseconds spent in setup, solves, moments and extraction by the last cbs_solve. */
cbs_status cbs_result_timing(const cbs_result *r, double *ms_solve, double *ms_moments,
                             double *ms_extract, double *ms_total);

/* The extraction time of cbs_result_timing split into: block Hankel matrices, SVD and rank
 * cut (ms_svd); the reduced eigenproblem (Hankel) or nothing (Rayleigh-Ritz) (ms_reduced);
 * per-energy vectors, Rayleigh-Ritz projection, residuals, filter and copies to the host
 * (ms_vectors).  Milliseconds, summed over the batches of the call. */
cbs_status cbs_result_extract_timing(const cbs_result *r, double *ms_svd, double *ms_reduced,
                                     double *ms_vectors);

/* Operator-apply (stencil + projector) launches of the last cbs_solve with profile = 1:
 * total device milliseconds, number of launches and number of complex outputs written
 * (active systems x N x L summed over launches), for element type dtype (CBS_C128 or
 * CBS_C64).  dtype = CBS_PROFILE_SHIFT_UPDATE instead reports the update kernel of the
 * shifted family (multi_shift = 1): milliseconds, launches and the grid points x active
 * (energy, point, column) triples it updated.  All zero when profiling was off. */
enum { CBS_PROFILE_SHIFT_UPDATE = 2 };
cbs_status cbs_result_profile(const cbs_result *r, int dtype, double *ms, double *launches,
                              double *outputs);

void cbs_result_free(cbs_result *r);

const char *cbs_last_error(void);

/* Number of CUDA kernels this library has launched in this process so far; a CUDA-graph
 * replay counts each of its kernel nodes. */
uint64_t cbs_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* CBS_H */
