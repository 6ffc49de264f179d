// Launchers shared between translation units of libcbs.
#pragma once

#include "bicg.cuh"

namespace cbs {

// moments.cu
cbs_status launch_contour(int n_int, int M, double lambda_min, double2 *coef, double2 *z1,
                          cudaStream_t st);
// moments of the solutions of one wave of quadrature points j0 .. j0 + n_w - 1 (systems
// e * n_w + jj, n = n_e * n_w); accumulate = add to S / mu (later waves); mirror = n_int when
// the conjugate points n_int - 1 - j take conj(Y_j) (real blocks, real V), else 0
cbs_status launch_moments(int n, int n_e, int n_w, int j0, int M, int64_t N, int L, const double2 *Y,
                          const double2 *coef, double2 *S, bool accumulate, int mirror, cudaStream_t st);
int vhy_chunks(int64_t N);
cbs_status launch_mu(int n, int n_e, int n_w, int j0, int M, int64_t N, int L, const double2 *V,
                     const double2 *Y, const double2 *coef, double2 *part, double2 *mu,
                     bool accumulate, int mirror, bool v_real, cudaStream_t st);

// dense.cu
cbs_status launch_hankel(int n_e, int L, int M, const double2 *mu, double2 *T, double2 *Tl,
                         cudaStream_t st);
cbs_status launch_svd(int n_e, int n, double2 *A, double2 *W, double2 *U, double2 *Ws,
                      double *sig, int *info, cudaStream_t st);
cbs_status launch_rank(int n_e, int n, const double *sig, double delta, int *mhat, cudaStream_t st);
cbs_status zgemm(int opa, int opb, int M, int N, int K, double2 alpha, const double2 *A,
                 int64_t lda, int64_t sA, const double2 *B, int64_t ldb, int64_t sB,
                 double2 beta, double2 *C, int64_t ldc, int64_t sC, int batch, cudaStream_t st);
cbs_status launch_scale(int n_e, int rows, int ld, const int *mhat, const double *sig, double2 *B,
                        int rows_scale, cudaStream_t st);
cbs_status launch_eig(int n_e, int ld, const int *mhat, double2 *B, double2 *Z, double2 *tau,
                      double2 *Yc, int *nring, int *ringidx, double lambda_min, int *info,
                      cudaStream_t st, double2 shift = make_double2(0, 0), int shifted = 0);
cbs_status launch_filter(int64_t N, int cnt, const double2 *tau_ring, const double2 *Psi,
                         const double2 *Res, double *stats, double nHp, double nA, double nHm,
                         double rho_max, double a_cell, double *rho_all, int *n_keep, int *perm,
                         double2 *lam_out, double2 *k_out, double *rho_out, double2 *scale_out,
                         cudaStream_t st);
cbs_status launch_gather_vectors(int64_t N, int cnt, int nk, const double2 *Psi, const int *perm,
                                 const double2 *scale, double2 *Out, cudaStream_t st);

// refinement (bicg.cu)
cbs_status launch_refine_check(int n, int L, int nchunks, const double *colnorm2, const double *bnorm,
                               double tol, int *colmask, int *n_unconv, double *maxrel,
                               cudaStream_t st);

}  // namespace cbs
