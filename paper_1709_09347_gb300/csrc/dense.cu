// Small dense FP64 stage of Algorithm 1 (Hankel SVD, rank cut, reduced eigenproblem), on the device.
//
//   T = [mu_{i+j-2}], T^< = [mu_{i+j-1}]  (block Hankel, L*M square)
//   T = U Sigma W^dagger (column-pivoted QR T P = Q R, then one-sided Jacobi on R^dagger),
//   rank m_hat: sigma_i >= delta sigma_1
//   B = U_1^dagger T^< W_1 Sigma_1^{-1},  B phi = tau phi  (Hessenberg + shifted QR),
//   lambda = tau,  psi = S W_1 Sigma_1^{-1} phi,  S = [S_0 ... S_{M-1}].
// followed by the residual check of every in-ring pair and the filter.
//
// One thread block per energy runs each factorisation; matrices are column-major in
// global memory (they fit in L2).  The GEMMs (T^< W_1, U_1^dagger C, the eigenvector
// back-transform and S C) use a tiled complex FP64 GEMM.
#include <math.h>

#include <vector>

#include "kernels.cuh"

namespace cbs {

__device__ __forceinline__ double cabs1(double2 a) { return fabs(a.x) + fabs(a.y); }
__device__ __forceinline__ double cabsd(double2 a) { return hypot(a.x, a.y); }
// Principal square root without cancellation: the larger of |re|, |im| of the root comes
// from sqrt((r + |x|)/2) and the other from y / (2 t).
__device__ __forceinline__ double2 csqrt_d(double2 z) {
  if (z.x == 0.0 && z.y == 0.0) return make_double2(0.0, 0.0);
  const double r = hypot(z.x, z.y);
  const double t = sqrt(0.5 * (r + fabs(z.x)));
  if (z.x >= 0.0) return make_double2(t, z.y / (2.0 * t));
  return make_double2(fabs(z.y) / (2.0 * t), copysign(t, z.y));
}

template <int NT>
__device__ double block_sum(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0;
  if (threadIdx.x < 32) {
    t = (threadIdx.x < NT / 32) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) sh[32] = t;
  }
  __syncthreads();
  return sh[32];
}

// ------------------------------------------------------------------ Hankel
__global__ void k_hankel(int n_e, int L, int M, const double2 *mu, double2 *T, double2 *Tl) {
  const int e = blockIdx.y;
  const int n = L * M;
  const int64_t nn = (int64_t)n * n;
  const double2 *me = mu + (int64_t)e * 2 * M * L * L;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < nn;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int row = (int)(idx % n), col = (int)(idx / n);
    const int bi = row / L, r = row % L, bj = col / L, c = col % L;
    T[e * nn + idx] = me[((int64_t)(bi + bj) * L + r) * L + c];
    Tl[e * nn + idx] = me[((int64_t)(bi + bj + 1) * L + r) * L + c];
  }
}

// ------------------------------------------------------------------ Jacobi SVD
// One-sided (Hestenes) Jacobi on the columns of A (n x n, column-major), accumulating
// the right rotations in W.  A sweep is n2-1 rounds of n2/2 disjoint column pairs
// (round-robin, n2 = n rounded up to even); each round is one launch in which every warp
// of the grid handles one pair of one energy, so a round of all energies spreads over
// the whole GPU (FP64 throughput per SM is small on GB300).  A sweep is captured once
// as a CUDA graph and replayed until no pair of any energy needed a rotation.
// On exit sigma (descending), U = A/sigma and W sorted accordingly.
//
// The Jacobi iteration runs on X = R^dagger of a column-pivoted QR factorisation
// T P = Q R (Householder), the preconditioning of Drmac and Veselic (SIAM J. Matrix Anal.
// Appl. 29, 2008): X has the singular values of T, and its columns are close to
// orthogonal already, so the sweeps needed drop several-fold (each sweep is a round of
// FP64 rotations over both n x n blocks, the cost of this stage).  From X V_x = U_x Sigma:
// T = (Q V_x) Sigma (P U_x)^dagger, i.e. U = Q V_x and W = P U_x.
constexpr int kSvdThreads = 256;

// Column-pivoted Householder QR, one block per energy (A in place: R in the upper
// triangle, zeros below).  Step k takes the remaining column of largest partial norm
// (the first one on ties), then the reflector H_k = I - beta_k v_k v_k^dagger with
// v_k = x + (x_0/|x_0|) ||x|| e_0 on x = A(k:n, k), beta_k = 2 / (v_k^dagger v_k), which
// maps x onto -(x_0/|x_0|) ||x|| e_0; v_k goes to column k of Vh (rows k..n-1).  The partial
// norms are downdated and recomputed from the column once the downdate has cancelled
// more than half the digits (the criterion of LAPACK's xLAQP2).  Q = H_0 H_1 ... H_{n-1}.
constexpr int kQrpThreads = 512;
__global__ void __launch_bounds__(kQrpThreads) k_qrp(int n, double2 *Ab, double2 *Vhb, double *betab,
                                                     int *permb) {
  const int e = blockIdx.x;
  const int64_t nn = (int64_t)n * n;
  double2 *A = Ab + e * nn, *Vh = Vhb + e * nn;
  double *beta = betab + (int64_t)e * n;
  int *perm = permb + (int64_t)e * n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int nwarp = kQrpThreads / 32;
  __shared__ double vn1[512], vn2[512];
  __shared__ int sperm[512];
  __shared__ double red_v[nwarp];
  __shared__ int red_i[nwarp];
  __shared__ int sh_p;
  __shared__ double sh_beta;
  const double tol3z = sqrt(2.220446049250313e-16);
  auto At = [&](int i, int j) -> double2 & { return A[i + (int64_t)j * n]; };
  for (int j = warp; j < n; j += nwarp) {
    double t = 0;
    for (int i = lane; i < n; i += 32) t += cabs2(At(i, j));
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) vn1[j] = vn2[j] = sqrt(t);
  }
  for (int j = tid; j < n; j += kQrpThreads) sperm[j] = j;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    // pivot: largest vn1[j], j >= k, first index on ties
    double bv = -1.0;
    int bi = n;
    for (int j = k + tid; j < n; j += kQrpThreads)
      if (vn1[j] > bv) { bv = vn1[j]; bi = j; }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { red_v[warp] = bv; red_i[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      double v = red_v[0];
      int i0 = red_i[0];
      for (int w = 1; w < nwarp; ++w)
        if (red_v[w] > v || (red_v[w] == v && red_i[w] < i0)) { v = red_v[w]; i0 = red_i[w]; }
      sh_p = i0;
    }
    __syncthreads();
    const int p = sh_p;
    if (p != k) {
      for (int i = tid; i < n; i += kQrpThreads) {
        const double2 t = At(i, k);
        At(i, k) = At(i, p);
        At(i, p) = t;
      }
      if (tid == 0) {
        double t = vn1[k]; vn1[k] = vn1[p]; vn1[p] = t;
        t = vn2[k]; vn2[k] = vn2[p]; vn2[p] = t;
        const int q = sperm[k]; sperm[k] = sperm[p]; sperm[p] = q;
      }
    }
    __syncthreads();
    // reflector of column k (warp 0)
    if (warp == 0) {
      double a2 = 0;
      for (int i = k + lane; i < n; i += 32) a2 += cabs2(At(i, k));
      for (int o = 16; o > 0; o >>= 1) a2 += __shfl_xor_sync(0xffffffffu, a2, o);
      const double2 x0 = At(k, k);
      if (a2 > 0) {
        const double alpha = sqrt(a2), ax0 = cabsd(x0);
        const double2 ph = ax0 > 0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1, 0);
        for (int i = k + lane; i < n; i += 32)
          Vh[i + (int64_t)k * n] = (i == k) ? make_double2(x0.x + ph.x * alpha, x0.y + ph.y * alpha) : At(i, k);
        __syncwarp();
        if (lane == 0) {
          sh_beta = 1.0 / (a2 + alpha * ax0);
          At(k, k) = make_double2(-ph.x * alpha, -ph.y * alpha);
        }
      } else {
        for (int i = k + lane; i < n; i += 32) Vh[i + (int64_t)k * n] = make_double2(0, 0);
        if (lane == 0) sh_beta = 0.0;
      }
      for (int i = k + 1 + lane; i < n; i += 32) At(i, k) = make_double2(0, 0);
      if (lane == 0) beta[k] = sh_beta;
    }
    __syncthreads();
    const double b = sh_beta;
    const double2 *v = Vh + (int64_t)k * n;
    // A(k:n, j) -= beta v (v^dagger A(k:n, j)) for j > k, one warp per column; then the
    // column's partial norm
    for (int j = k + 1 + warp; j < n; j += nwarp) {
      if (b != 0) {
        double sx = 0, sy = 0;
        for (int i = k + lane; i < n; i += 32) {
          const double2 t = cmulc(v[i], At(i, j));   // conj(v_i) a_i
          sx += t.x;
          sy += t.y;
        }
        for (int o = 16; o > 0; o >>= 1) {
          sx += __shfl_xor_sync(0xffffffffu, sx, o);
          sy += __shfl_xor_sync(0xffffffffu, sy, o);
        }
        const double2 sb = make_double2(sx * b, sy * b);
        for (int i = k + lane; i < n; i += 32) At(i, j) = csub(At(i, j), cmul(v[i], sb));
        __syncwarp();
      }
      const double nj = vn1[j];
      if (nj != 0) {
        double t = cabsd(At(k, j)) / nj;
        t = fmax(0.0, (1.0 + t) * (1.0 - t));
        const double r = nj / vn2[j];
        if (t * r * r <= tol3z) {
          double q = 0;
          for (int i = k + 1 + lane; i < n; i += 32) q += cabs2(At(i, j));
          for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
          __syncwarp();
          if (lane == 0) vn1[j] = vn2[j] = sqrt(q);
        } else {
          __syncwarp();
          if (lane == 0) vn1[j] = nj * sqrt(t);
        }
      }
    }
    __syncthreads();
  }
  for (int j = tid; j < n; j += kQrpThreads) perm[j] = sperm[j];
}

// X = R^dagger (lower triangular) from the upper triangle of R
__global__ void k_rdagger(int n, const double2 *Rb, double2 *Xb) {
  const int e = blockIdx.y;
  const int64_t nn = (int64_t)n * n;
  const double2 *R = Rb + e * nn;
  double2 *X = Xb + e * nn;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < nn;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % n), j = (int)(idx / n);
    X[idx] = (j <= i) ? cconj(R[j + (int64_t)i * n]) : make_double2(0, 0);
  }
}

// B <- Q B = H_0 (H_1 (... (H_{n-1} B))), one warp per column of B
__global__ void __launch_bounds__(512) k_apply_q(int n, const double2 *Vhb, const double *betab, double2 *Bb) {
  const int e = blockIdx.y;
  const int64_t nn = (int64_t)n * n;
  const double2 *Vh = Vhb + e * nn;
  const double *beta = betab + (int64_t)e * n;
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= n) return;
  double2 *B = Bb + e * nn + (int64_t)j * n;
  for (int k = n - 1; k >= 0; --k) {
    const double b = beta[k];
    if (b == 0) continue;
    const double2 *v = Vh + (int64_t)k * n;
    double sx = 0, sy = 0;
    for (int i = k + lane; i < n; i += 32) {
      const double2 t = cmulc(v[i], B[i]);
      sx += t.x;
      sy += t.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
      sx += __shfl_xor_sync(0xffffffffu, sx, o);
      sy += __shfl_xor_sync(0xffffffffu, sy, o);
    }
    const double2 sb = make_double2(sx * b, sy * b);
    for (int i = k + lane; i < n; i += 32) B[i] = csub(B[i], cmul(v[i], sb));
    __syncwarp();
  }
}

// Out(perm[i], j) = In(i, j): the row permutation P In
__global__ void k_permute_rows(int n, const int *permb, const double2 *Inb, double2 *Outb) {
  const int e = blockIdx.y;
  const int64_t nn = (int64_t)n * n;
  const int *perm = permb + (int64_t)e * n;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < nn;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % n), j = (int)(idx / n);
    Outb[e * nn + perm[i] + (int64_t)j * n] = Inb[e * nn + idx];
  }
}


__global__ void k_svd_init(int n, double2 *Wb) {
  const int e = blockIdx.y;
  const int64_t nn = (int64_t)n * n;
  double2 *W = Wb + e * nn;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < nn;
       idx += (int64_t)gridDim.x * blockDim.x)
    W[idx] = make_double2((idx % n) == (idx / n) ? 1.0 : 0.0, 0.0);
}

__global__ void __launch_bounds__(kSvdThreads) k_svd_round(int n, int round, double2 *Ab, double2 *Wb,
                                                           double tolj, int *rot) {
  const int e = blockIdx.y;
  const int64_t nn = (int64_t)n * n;
  double2 *A = Ab + e * nn, *W = Wb + e * nn;
  const int lane = threadIdx.x & 31;
  const int pi = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int nn2 = (n + 1) & ~1;
  if (pi >= nn2 / 2) return;
  // circle method: player 0 fixed, the others rotate by `round`
  const int a = pi, b = nn2 - 1 - pi;
  const int p = (a == 0) ? 0 : ((a - 1 + round) % (nn2 - 1)) + 1;
  const int q = (b == 0) ? 0 : ((b - 1 + round) % (nn2 - 1)) + 1;
  if (p >= n || q >= n) return;
  double2 *ap = A + (int64_t)p * n, *aq = A + (int64_t)q * n;
  double al = 0, be = 0, gx = 0, gy = 0;
  for (int i = lane; i < n; i += 32) {
    const double2 u = ap[i], v = aq[i];
    al += cabs2(u);
    be += cabs2(v);
    gx += u.x * v.x + u.y * v.y;   // conj(u) v
    gy += u.x * v.y - u.y * v.x;
  }
  for (int o = 16; o > 0; o >>= 1) {
    al += __shfl_xor_sync(0xffffffffu, al, o);
    be += __shfl_xor_sync(0xffffffffu, be, o);
    gx += __shfl_xor_sync(0xffffffffu, gx, o);
    gy += __shfl_xor_sync(0xffffffffu, gy, o);
  }
  const double g = hypot(gx, gy);
  if (!(g > tolj * sqrt(al * be)) || al == 0.0 || be == 0.0) return;
  // rotation that makes columns p and q orthogonal: with gamma = |g| e^{i phi},
  // zeta = (be - al)/(2|g|), t the smaller root of t^2 + 2 zeta t - 1 = 0,
  // a_p' = c a_p - s e^{-i phi} a_q,  a_q' = s e^{i phi} a_p + c a_q
  const double zeta = (be - al) / (2.0 * g);
  const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
  const double2 sp = make_double2(s * gx / g, s * gy / g);    // s e^{i phi}
  const double2 spc = make_double2(sp.x, -sp.y);              // s e^{-i phi}
  for (int i = lane; i < n; i += 32) {
    const double2 u = ap[i], v = aq[i];
    ap[i] = csub(cscale(u, c), cmul(spc, v));
    aq[i] = cadd(cmul(sp, u), cscale(v, c));
  }
  double2 *wp = W + (int64_t)p * n, *wq = W + (int64_t)q * n;
  for (int i = lane; i < n; i += 32) {
    const double2 u = wp[i], v = wq[i];
    wp[i] = csub(cscale(u, c), cmul(spc, v));
    wq[i] = cadd(cmul(sp, u), cscale(v, c));
  }
  if (lane == 0) atomicAdd(&rot[e], 1);
}

// sigma_j = ||a_j||, sorted descending (ties by index); U = A/sigma, W permuted alike.
__global__ void __launch_bounds__(1024) k_svd_finish(int n, double2 *Ab, const double2 *Wb, double2 *Ub,
                                                     double2 *Wsb, double *sigb) {
  const int e = blockIdx.x;
  const int64_t nn = (int64_t)n * n;
  double2 *A = Ab + e * nn, *U = Ub + e * nn, *Ws = Wsb + e * nn;
  const double2 *W = Wb + e * nn;
  double *sig = sigb + (int64_t)e * n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  __shared__ double s_sig[512];
  __shared__ int rank_of[512];
  for (int j = warp; j < n; j += nwarp) {
    double s2 = 0;
    for (int i = lane; i < n; i += 32) s2 += cabs2(A[(int64_t)j * n + i]);
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    if (lane == 0) s_sig[j] = sqrt(s2);
  }
  __syncthreads();
  for (int j = tid; j < n; j += blockDim.x) {
    const double sj = s_sig[j];
    int r = 0;
    for (int k = 0; k < n; ++k) {
      const double sk = s_sig[k];
      r += (sk > sj) || (sk == sj && k < j);
    }
    rank_of[j] = r;
  }
  __syncthreads();
  for (int j = warp; j < n; j += nwarp) {
    const int r = rank_of[j];
    const double sj = s_sig[j];
    const double inv = sj > 0 ? 1.0 / sj : 0.0;
    for (int i = lane; i < n; i += 32) {
      U[(int64_t)r * n + i] = cscale(A[(int64_t)j * n + i], inv);
      Ws[(int64_t)r * n + i] = W[(int64_t)j * n + i];
    }
  }
  for (int j = tid; j < n; j += blockDim.x) sig[rank_of[j]] = s_sig[j];
}

__global__ void k_rank(int n_e, int n, const double *sig, double delta, int *mhat) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_e) return;
  const double *s = sig + (int64_t)e * n;
  int m = 0;
  if (s[0] > 0)
    for (int i = 0; i < n; ++i) m += (s[i] >= delta * s[0]);
  mhat[e] = m;
}

// ------------------------------------------------------------------ tiled ZGEMM
// C = alpha op(A) op(B) + beta C, column-major; op: 0 = N, 1 = T, 2 = C (conj transpose).
template <int OP>
__device__ __forceinline__ double2 opload(const double2 *A, int64_t ld, int r, int c, int R, int Cc) {
  if (r >= R || c >= Cc) return make_double2(0, 0);
  if (OP == 0) return A[r + (int64_t)c * ld];
  double2 v = A[c + (int64_t)r * ld];
  return OP == 2 ? cconj(v) : v;
}

template <int OPA, int OPB>
__global__ void k_zgemm(int M, int N, int K, double2 alpha, const double2 *A, int64_t lda,
                        int64_t sA, const double2 *B, int64_t ldb, int64_t sB, double2 beta,
                        double2 *C, int64_t ldc, int64_t sC) {
  __shared__ double2 As[16][33];
  __shared__ double2 Bs[16][33];
  const int bz = blockIdx.z;
  A += bz * sA; B += bz * sB; C += bz * sC;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 16 + tx;
  const int m0 = blockIdx.x * 32, n0 = blockIdx.y * 32;
  double2 acc[2][2];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) acc[a][b] = make_double2(0, 0);
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int t = tid; t < 512; t += 256) {
      int mm, kk;
      if (OPA == 0) { mm = t % 32; kk = t / 32; } else { kk = t % 16; mm = t / 16; }
      As[kk][mm] = opload<OPA>(A, lda, m0 + mm, k0 + kk, M, K);
      int nn2, kb;
      if (OPB == 0) { kb = t % 16; nn2 = t / 16; } else { nn2 = t % 32; kb = t / 32; }
      Bs[kb][nn2] = opload<OPB>(B, ldb, k0 + kb, n0 + nn2, K, N);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double2 a0 = As[kk][tx * 2], a1 = As[kk][tx * 2 + 1];
      double2 b0 = Bs[kk][ty * 2], b1 = Bs[kk][ty * 2 + 1];
      acc[0][0] = cfma(a0, b0, acc[0][0]);
      acc[0][1] = cfma(a0, b1, acc[0][1]);
      acc[1][0] = cfma(a1, b0, acc[1][0]);
      acc[1][1] = cfma(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      const int r = m0 + tx * 2 + a, c = n0 + ty * 2 + b;
      if (r < M && c < N) {
        double2 *cp = C + r + (int64_t)c * ldc;
        double2 v = cmul(alpha, acc[a][b]);
        if (beta.x != 0.0 || beta.y != 0.0) v = cfma(beta, *cp, v);
        *cp = v;
      }
    }
}

cbs_status zgemm(int opa, int opb, int M, int N, int K, double2 alpha, const double2 *A,
                 int64_t lda, int64_t sA, const double2 *B, int64_t ldb, int64_t sB,
                 double2 beta, double2 *C, int64_t ldc, int64_t sC, int batch, cudaStream_t st) {
  if (M <= 0 || N <= 0 || batch <= 0) return CBS_OK;
  dim3 blk(16, 16, 1);
  dim3 grd((unsigned)ceil_div(M, 32), (unsigned)ceil_div(N, 32), (unsigned)batch);
#define ZG(a, b) k_zgemm<a, b><<<grd, blk, 0, st>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC)
  if (opa == 0 && opb == 0) ZG(0, 0);
  else if (opa == 0 && opb == 1) ZG(0, 1);
  else if (opa == 0 && opb == 2) ZG(0, 2);
  else if (opa == 1 && opb == 0) ZG(1, 0);
  else if (opa == 2 && opb == 0) ZG(2, 0);
  else if (opa == 1 && opb == 1) ZG(1, 1);
  else { set_error("zgemm: unsupported op pair"); return CBS_EINVAL; }
#undef ZG
  cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  return CBS_OK;
}

// B[:, j] *= 1/sigma_j for j < m (column scaling, B is n x m with leading dim n)
__global__ void k_scale_cols(int n, int ldm, const int *mhat, const double *sig, double2 *B, int rows_scale) {
  const int e = blockIdx.y;
  const int m = mhat[e];
  const int64_t nn = (int64_t)ldm * ldm;
  double2 *Be = B + e * nn;
  const double *s = sig + (int64_t)e * ldm;
  const int64_t tot = (int64_t)n * m;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx % n), c = (int)(idx / n);
    const double inv = 1.0 / s[rows_scale ? r : c];
    Be[r + (int64_t)c * ldm] = cscale(Be[r + (int64_t)c * ldm], inv);
  }
}

// ------------------------------------------------------------------ eigen-solver
// Complex upper-Hessenberg reduction (Householder) and shifted QR to Schur form
// T = Z^dagger B Z, then eigenvectors of T by back substitution for the selected
// eigenvalues (those strictly inside the ring), compacted into Yc (m x n_ring) and
// transformed by Z outside this kernel.
// Complex Givens rotation [c s; -conj(s) c] with c real that maps (x, y) to (r, 0):
// c = |x| / rho, s = (x / |x|) conj(y) / rho, rho = sqrt(|x|^2 + |y|^2).  Computed by one
// thread on the critical path of the QR sweep, so it uses few dependent FP64 operations
// (one reciprocal square root); the scaled form guards tiny or huge entries.
__device__ __forceinline__ void givens(double2 x, double2 y, double &c, double2 &s) {
  const double nx2 = x.x * x.x + x.y * x.y, ny2 = y.x * y.x + y.y * y.y;
  if (ny2 == 0) { c = 1; s = make_double2(0, 0); return; }
  if (nx2 == 0) {
    const double t = rsqrt(ny2);
    c = 0;
    s = make_double2(y.x * t, -y.y * t);
    return;
  }
  double p = nx2 * (nx2 + ny2);
  if (p > 1e-280 && p < 1e280) {
    const double t = rsqrt(p);                          // 1 / (|x| rho)
    c = nx2 * t;
    s = cscale(cmul(x, cconj(y)), t);
    return;
  }
  const double ax = cabsd(x), ay = cabsd(y), rho = hypot(ax, ay);
  c = ax / rho;
  s = cscale(cmul(make_double2(x.x / ax, x.y / ax), cconj(y)), 1.0 / rho);
}

constexpr int kEigThreads = 512;
constexpr int kMaxEigN = 512;   // largest eigenproblem (launch_eig rejects larger)
// shift: 0 selects eigenvalues tau inside the ring; otherwise the eigenvalues are mu of a
// shifted-and-inverted problem, lambda = shift + 1/mu is tested and written back to tau.
__global__ void __launch_bounds__(kEigThreads) k_eig(int ld, const int *mhat, double2 *Bb, double2 *Zb,
                                                     double2 *taub, double2 *Ycb, int *nring,
                                                     int *ringidx, double lambda_min, int *info,
                                                     double2 shift, int shifted) {
  const int e = blockIdx.x;
  const int m = mhat[e];
  const int64_t nn = (int64_t)ld * ld;
  double2 *A = Bb + e * nn, *Z = Zb + e * nn, *Yc = Ycb + e * nn;
  double2 *tau = taub + (int64_t)e * ld;
  int *ridx = ringidx + (int64_t)e * ld;
  const int tid = threadIdx.x, nt = blockDim.x;
  __shared__ double2 v[512];
  __shared__ double shr[40];
  __shared__ int sh_l, sh_hi, sh_act, sh_fail;
  if (m == 0) {
    if (tid == 0) { nring[e] = 0; info[e] = 0; }
    return;
  }
  auto Aat = [&](int i, int j) -> double2 & { return A[i + (int64_t)j * ld]; };
  for (int64_t idx = tid; idx < (int64_t)m * m; idx += nt) {
    const int i = (int)(idx % m), j = (int)(idx / m);
    Z[i + (int64_t)j * ld] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  // ---- Hessenberg reduction
  for (int k = 0; k < m - 2; ++k) {
    double loc = 0;
    for (int i = k + 1 + tid; i < m; i += nt) loc += cabs2(Aat(i, k));
    const double a2 = block_sum<kEigThreads>(loc, shr);
    if (!(a2 > 0)) continue;
    const double alpha = sqrt(a2);
    const double2 x0 = Aat(k + 1, k);
    const double ax0 = cabsd(x0);
    const double2 ph = ax0 > 0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1, 0);
    const double2 v0 = make_double2(x0.x + ph.x * alpha, x0.y + ph.y * alpha);
    const double vhv = 2.0 * (a2 + alpha * ax0);
    const double tau_h = 2.0 / vhv;
    for (int i = k + 1 + tid; i < m; i += nt) v[i] = (i == k + 1) ? v0 : Aat(i, k);
    __syncthreads();
    // left: A[k+1:, k:] -= tau v (v^H A)
    for (int j = k + tid; j < m; j += nt) {
      double2 s = make_double2(0, 0);
      for (int i = k + 1; i < m; ++i) s = cadd(s, cmulc(v[i], Aat(i, j)));
      s = cscale(s, tau_h);
      for (int i = k + 1; i < m; ++i) Aat(i, j) = csub(Aat(i, j), cmul(v[i], s));
    }
    __syncthreads();
    // right: A[:, k+1:] -= tau (A v) v^H ; Z likewise
    for (int i = tid; i < m; i += nt) {
      double2 t = make_double2(0, 0), tz = make_double2(0, 0);
      for (int j = k + 1; j < m; ++j) {
        t = cfma(Aat(i, j), v[j], t);
        tz = cfma(Z[i + (int64_t)j * ld], v[j], tz);
      }
      t = cscale(t, tau_h);
      tz = cscale(tz, tau_h);
      for (int j = k + 1; j < m; ++j) {
        Aat(i, j) = csub(Aat(i, j), cmul(t, cconj(v[j])));
        Z[i + (int64_t)j * ld] = csub(Z[i + (int64_t)j * ld], cmul(tz, cconj(v[j])));
      }
    }
    __syncthreads();
    for (int i = k + 2 + tid; i < m; i += nt) Aat(i, k) = make_double2(0, 0);
    if (tid == 0) Aat(k + 1, k) = make_double2(-ph.x * alpha, -ph.y * alpha);
    __syncthreads();
  }
  // ---- shifted QR (single shift, Wilkinson; exceptional shifts every 10 stalls)
  // Each sweep chases the bulge through the active window [l, hi] only: a rotation updates
  // rows k, k+1 for columns up to hi and columns k, k+1 for rows from l.  The parts outside
  // the window (rows k, k+1 right of hi, columns k, k+1 above l) and the Schur vectors Z are
  // not read by the chase; they receive the sweep's rotations afterwards in one parallel
  // pass, each thread applying them in order to its own column or row (the same operations
  // per element, in the same order).  Every rotation is computed once, by the thread that
  // owns the two entries defining it, and shared through one slot: two block barriers per
  // rotation.  (FP64 on this part runs about 1.6 lanes per clock per SM and a warp
  // instruction costs the same with one active lane as with 32, so redundant per-thread
  // computation of the rotation is what must be avoided.)
  const double eps = 2.220446049250313e-16;
  __shared__ double rot_c[kMaxEigN];
  __shared__ double2 rot_s[kMaxEigN];
  __shared__ double sh_c;
  __shared__ double2 sh_u1, sh_w1;
  __shared__ double2 sh_s;
  __shared__ int sh_defl[kEigThreads / 32];
  if (tid == 0) { sh_hi = m - 1; sh_fail = 0; }
  __syncthreads();
  int its = 0, total = 0;
  while (true) {
    // deflation: the largest l <= hi with a negligible subdiagonal entry (0 if none)
    const int hi0 = sh_hi;
    int best = 0;
    for (int q = 1 + tid; q <= hi0; q += nt) {
      double sc = cabs1(Aat(q - 1, q - 1)) + cabs1(Aat(q, q));
      if (sc == 0) sc = 1e-300;
      if (cabs1(Aat(q, q - 1)) <= eps * sc) best = max(best, q);
    }
    for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((tid & 31) == 0) sh_defl[tid >> 5] = best;
    __syncthreads();
    if (tid == 0) {
      int hi = sh_hi;
      sh_act = 0;
      if (hi < 0) {
        sh_act = -1;
      } else if (hi == 0) {
        tau[0] = Aat(0, 0);
        sh_hi = -1;
      } else {
        int l = 0;
        for (int w = 0; w < nt / 32; ++w) l = max(l, sh_defl[w]);
        if (l > 0) Aat(l, l - 1) = make_double2(0, 0);
        if (l == hi) {
          tau[hi] = Aat(hi, hi);
          sh_hi = hi - 1;
          its = 0;
        } else if (++total > 60 * m) {
          sh_fail = 1;
          sh_act = -1;
        } else {
          ++its;
          double2 mu;
          const double2 d = Aat(hi, hi);
          if (its % 10 == 0) {
            const double sub = cabs1(Aat(hi, hi - 1));
            mu = make_double2(d.x + 0.75 * sub, d.y);
          } else {
            const double2 a = Aat(hi - 1, hi - 1), b = Aat(hi - 1, hi), c = Aat(hi, hi - 1);
            const double2 half = make_double2(0.5 * (a.x - d.x), 0.5 * (a.y - d.y));
            const double2 disc = csqrt_d(cadd(cmul(half, half), cmul(b, c)));
            const double2 mean = make_double2(0.5 * (a.x + d.x), 0.5 * (a.y + d.y));
            const double2 m1 = cadd(mean, disc), m2 = csub(mean, disc);
            mu = (cabs2(csub(m1, d)) <= cabs2(csub(m2, d))) ? m1 : m2;
          }
          sh_l = l;
          sh_act = 1;
          double c0;
          double2 s0;
          givens(csub(Aat(l, l), mu), Aat(l + 1, l), c0, s0);
          sh_c = c0;
          sh_s = s0;
        }
      }
    }
    __syncthreads();
    const int act = sh_act;
    if (act < 0) break;
    if (act == 0) continue;
    const int l = sh_l, hi = sh_hi;
    for (int k = l; k < hi; ++k) {
      const double c = sh_c;
      const double2 sr = sh_s;
      if (tid == 0) { rot_c[k] = c; rot_s[k] = sr; }
      // the leader's entry of row k+2, untouched by this step's row rotation: in flight
      // while the rows are rotated
      double2 w2 = make_double2(0, 0);
      if (tid == 0 && k + 2 <= hi) w2 = Aat(k + 2, k + 1);
      // rows k, k+1 inside the window:  [a; b] <- [c a + s b; -conj(s) a + c b]; the new
      // A(k+1, k) and A(k+1, k+1) also go to the leader through shared memory
      const int j0 = (k == l) ? l : k - 1;
      for (int j = j0 + tid; j <= hi; j += nt) {
        const double2 a = Aat(k, j), b = Aat(k + 1, j);
        const double2 nb = csub(cscale(b, c), cmul(cconj(sr), a));
        Aat(k, j) = cadd(cscale(a, c), cmul(sr, b));
        Aat(k + 1, j) = nb;
        if (j == k) sh_u1 = nb;
        else if (j == k + 1) sh_w1 = nb;
      }
      __syncthreads();
      // columns k, k+1 inside the window:  [u, w] <- [c u + conj(s) w, -s u + c w].
      // Thread 0 (alone in its warp here, so its chain does not wait for a divergent
      // branch) takes rows k+1 and k+2, whose column-k entries define the next rotation;
      // A(k+2, k) is zero before this rotation (the bulge sits one column to the left).
      // Warps 1.. take rows l..k.
      if (tid == 0) {
        if (k > l) Aat(k + 1, k - 1) = make_double2(0, 0);   // the bulge the rotation removed
        const double2 u = sh_u1, w = sh_w1;
        const double2 xn = cadd(cscale(u, c), cmul(cconj(sr), w));
        Aat(k + 1, k) = xn;
        Aat(k + 1, k + 1) = csub(cscale(w, c), cmul(sr, u));
        if (k + 2 <= hi) {
          const double2 yn = cmul(cconj(sr), w2);
          Aat(k + 2, k) = yn;
          Aat(k + 2, k + 1) = cscale(w2, c);
          if (k + 1 < hi) {
            double cn;
            double2 sn;
            givens(xn, yn, cn, sn);
            sh_c = cn;
            sh_s = sn;
          }
        }
      } else if (tid >= 32) {
        for (int i = l + tid - 32; i <= k; i += nt - 32) {
          const double2 u = Aat(i, k), w = Aat(i, k + 1);
          Aat(i, k) = cadd(cscale(u, c), cmul(cconj(sr), w));
          Aat(i, k + 1) = csub(cscale(w, c), cmul(sr, u));
        }
      }
      __syncthreads();
    }
    // deferred: rows k, k+1 right of the window, columns k, k+1 above it, and Z
    for (int j = hi + 1 + tid; j < m; j += nt) {
      double2 a = Aat(l, j);
      for (int k = l; k < hi; ++k) {
        const double c = rot_c[k];
        const double2 sr = rot_s[k];
        const double2 b = Aat(k + 1, j);
        Aat(k, j) = cadd(cscale(a, c), cmul(sr, b));
        a = csub(cscale(b, c), cmul(cconj(sr), a));
      }
      Aat(hi, j) = a;
    }
    for (int i = tid; i < l; i += nt) {
      double2 u = Aat(i, l);
      for (int k = l; k < hi; ++k) {
        const double c = rot_c[k];
        const double2 sr = rot_s[k];
        const double2 w = Aat(i, k + 1);
        Aat(i, k) = cadd(cscale(u, c), cmul(cconj(sr), w));
        u = csub(cscale(w, c), cmul(sr, u));
      }
      Aat(i, hi) = u;
    }
    for (int i = tid; i < m; i += nt) {
      double2 u = Z[i + (int64_t)l * ld];
      for (int k = l; k < hi; ++k) {
        const double c = rot_c[k];
        const double2 sr = rot_s[k];
        const double2 w = Z[i + (int64_t)(k + 1) * ld];
        Z[i + (int64_t)k * ld] = cadd(cscale(u, c), cmul(cconj(sr), w));
        u = csub(cscale(w, c), cmul(sr, u));
      }
      Z[i + (int64_t)hi * ld] = u;
    }
    __syncthreads();
  }
  __syncthreads();
  // ---- select eigenvalues strictly inside the ring
  if (tid == 0) {
    int cnt = 0;
    for (int k = 0; k < m; ++k) {
      double2 lam = tau[k];
      if (shifted) {
        lam = (cabs2(lam) > 0) ? cadd(shift, cdiv(make_double2(1.0, 0.0), lam))
                               : make_double2(INFINITY, INFINITY);
        tau[k] = lam;   // the back substitution below reads the Schur form, not tau
      }
      const double r = cabsd(lam);
      if (!sh_fail && isfinite(r) && r > lambda_min && r < 1.0 / lambda_min) ridx[cnt++] = k;
    }
    nring[e] = cnt;
    info[e] = sh_fail;
  }
  __syncthreads();
  const int cnt = nring[e];
  // ---- eigenvectors of the triangular T for the selected eigenvalues (thread per vector)
  double tnorm = 0;
  for (int64_t idx = tid; idx < (int64_t)m * m; idx += nt) {
    const int i = (int)(idx % m), j = (int)(idx / m);
    if (i <= j) tnorm = fmax(tnorm, cabs1(Aat(i, j)));
  }
  for (int o = 16; o > 0; o >>= 1) tnorm = fmax(tnorm, __shfl_xor_sync(0xffffffffu, tnorm, o));
  __syncthreads();
  if ((tid & 31) == 0) shr[tid >> 5] = tnorm;
  __syncthreads();
  if (tid == 0) {
    double t = 0;
    for (int w = 0; w < nt / 32; ++w) t = fmax(t, shr[w]);
    shr[32] = t;
  }
  __syncthreads();
  const double smin = fmax(eps * shr[32], 1e-300);
  for (int r = tid; r < cnt; r += nt) {
    const int k = ridx[r];
    double2 *y = Yc + (int64_t)r * ld;
    const double2 tkk = Aat(k, k);
    for (int i = k + 1; i < m; ++i) y[i] = make_double2(0, 0);
    y[k] = make_double2(1, 0);
    for (int i = k - 1; i >= 0; --i) {
      double2 sum = Aat(i, k);
      for (int j = i + 1; j < k; ++j) sum = cfma(Aat(i, j), y[j], sum);
      double2 den = csub(Aat(i, i), tkk);
      if (cabs1(den) < smin) den = make_double2(smin, 0);
      double2 yi = cdiv(sum, den);
      y[i] = make_double2(-yi.x, -yi.y);
    }
  }
}

// ------------------------------------------------------------------ residual filter
// Per column r of Psi (N x cnt, row-major [N][cnt]) and Res = P(tau_r) Psi:
// stats[r] = (||psi||^2, ||res||^2, max|psi_i|, index of the first maximum)
__global__ void k_colstats(int64_t N, int cnt, const double2 *Psi, const double2 *Res, double *stats) {
  const int r = blockIdx.x;
  double s1 = 0, s2 = 0, mx = -1;
  int64_t imx = 0;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
    const double2 p = Psi[i * cnt + r], q = Res[i * cnt + r];
    s1 += cabs2(p);
    s2 += cabs2(q);
    const double a = cabs2(p);
    if (a > mx) { mx = a; imx = i; }
  }
  __shared__ double sa[256], sb[256], sm[256];
  __shared__ int64_t si[256];
  sa[threadIdx.x] = s1; sb[threadIdx.x] = s2; sm[threadIdx.x] = mx; si[threadIdx.x] = imx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sa[threadIdx.x] += sa[threadIdx.x + o];
      sb[threadIdx.x] += sb[threadIdx.x + o];
      const double m2 = sm[threadIdx.x + o];
      const int64_t i2 = si[threadIdx.x + o];
      if (m2 > sm[threadIdx.x] || (m2 == sm[threadIdx.x] && i2 < si[threadIdx.x])) {
        sm[threadIdx.x] = m2;
        si[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    stats[r * 4 + 0] = sa[0];
    stats[r * 4 + 1] = sb[0];
    stats[r * 4 + 2] = sm[0];
    stats[r * 4 + 3] = (double)si[0];
  }
}

// rho_r = |tau| ||P(tau) psi|| / (||psi|| (|tau|^2 nHp + |tau| nA + nHm)); keep if rho <= rho_max;
// order kept by (|tau|, arg tau); scale_r = conj(psi_piv)/|psi_piv| / ||psi||.
__global__ void k_filter(int cnt, const double2 *tau_ring, const double *stats, double nHp, double nA,
                         double nHm, double rho_max, double a_cell, const double2 *Psi, int64_t N,
                         double *rho_all, int *n_keep, int *perm, double2 *lam_out, double2 *k_out,
                         double *rho_out, double2 *scale_out) {
  __shared__ int keep[512];
  __shared__ double key1[512], key2[512];
  for (int r = threadIdx.x; r < cnt; r += blockDim.x) {
    const double2 t = tau_ring[r];
    const double at = hypot(t.x, t.y);
    const double num = at * sqrt(stats[r * 4 + 1]);
    const double den = sqrt(stats[r * 4 + 0]) * (at * at * nHp + at * nA + nHm);
    const double rho = num / den;
    rho_all[r] = rho;
    keep[r] = (rho <= rho_max) && isfinite(rho);
    key1[r] = at;
    key2[r] = atan2(t.y, t.x);
  }
  __syncthreads();
  for (int r = threadIdx.x; r < cnt; r += blockDim.x) {
    if (!keep[r]) continue;
    int pos = 0;
    for (int q = 0; q < cnt; ++q) {
      if (!keep[q]) continue;
      const bool before = key1[q] < key1[r] || (key1[q] == key1[r] && (key2[q] < key2[r] ||
                                                (key2[q] == key2[r] && q < r)));
      pos += before;
    }
    perm[pos] = r;
    const double2 t = tau_ring[r];
    lam_out[pos] = t;
    const double at = key1[r];
    k_out[pos] = make_double2(key2[r] / a_cell, -log(at) / a_cell);
    rho_out[pos] = rho_all[r];
    const int64_t piv = (int64_t)stats[r * 4 + 3];
    const double2 pv = Psi[piv * cnt + r];
    const double ap = hypot(pv.x, pv.y);
    const double nrm = sqrt(stats[r * 4 + 0]);
    scale_out[pos] = ap > 0 ? make_double2(pv.x / (ap * nrm), -pv.y / (ap * nrm)) : make_double2(0, 0);
  }
  if (threadIdx.x == 0) {
    int c = 0;
    for (int r = 0; r < cnt; ++r) c += keep[r];
    *n_keep = c;
  }
}

__global__ void k_gather_vectors(int64_t N, int cnt, int nk, const double2 *Psi, const int *perm,
                                 const double2 *scale, double2 *Out) {
  const int64_t tot = N * nk;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / nk;
    const int q = (int)(idx % nk);
    Out[idx] = cmul(Psi[i * cnt + perm[q]], scale[q]);
  }
}

// ------------------------------------------------------------------ launchers
cbs_status launch_hankel(int n_e, int L, int M, const double2 *mu, double2 *T, double2 *Tl,
                         cudaStream_t st) {
  const int64_t nn = (int64_t)L * M * L * M;
  k_hankel<<<dim3((unsigned)ceil_div(nn, 256), (unsigned)n_e, 1), 256, 0, st>>>(n_e, L, M, mu, T, Tl); cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  return CBS_OK;
}

cbs_status launch_svd(int n_e, int n, double2 *A, double2 *W, double2 *U, double2 *Ws,
                      double *sig, int *info, cudaStream_t st) {
  if (n > 512) { set_error("L*M must be <= 512"); return CBS_EINVAL; }
  const double tolj = 1e-14;
  const int max_sweeps = 60;
  const int nn2 = (n + 1) & ~1;
  const int warps = kSvdThreads / 32;
  const int64_t nn = (int64_t)n * n;
  // workspace: reflectors (n x n), beta (n) and the pivot order (n) per energy
  struct Work {
    void *p = nullptr;
    ~Work() { if (p) cudaFree(p); }
  } wk;
  const size_t wbytes = (size_t)nn * n_e * sizeof(double2) + (size_t)n * n_e * (sizeof(double) + sizeof(int)) + 256;
  if (cudaMalloc(&wk.p, wbytes) != cudaSuccess) {
    wk.p = nullptr;
    set_error("cudaMalloc failed (SVD workspace)");
    return CBS_ENOMEM;
  }
  double2 *Vh = (double2 *)wk.p;
  double *beta = (double *)(Vh + nn * n_e);
  int *perm = (int *)(beta + (size_t)n * n_e);
  // T P = Q R in place (A holds R), X = R^dagger into Ws: the matrix the sweeps rotate
  k_qrp<<<n_e, kQrpThreads, 0, st>>>(n, A, Vh, beta, perm);
  cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  k_rdagger<<<dim3(64, (unsigned)n_e, 1), 256, 0, st>>>(n, A, Ws);
  cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  double2 *X = Ws;
  dim3 grd_round((unsigned)ceil_div(nn2 / 2, warps), (unsigned)n_e, 1);
  k_svd_init<<<dim3(64, (unsigned)n_e, 1), 256, 0, st>>>(n, W);
  cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  int *rot = info;   // [n_e] rotation counters of the last sweep, then the info words
  // capture one sweep
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  const uint64_t c0 = thread_launches();
  CBS_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  cudaError_t ce = cudaMemsetAsync(rot, 0, (size_t)n_e * sizeof(int), st);
  for (int r = 0; r < nn2 - 1 && ce == cudaSuccess; ++r) {
    k_svd_round<<<grd_round, kSvdThreads, 0, st>>>(n, r, X, W, tolj, rot);
    cbs::count_launches(1);
    ce = cudaGetLastError();
  }
  cudaError_t ce2 = cudaStreamEndCapture(st, &graph);
  const uint64_t per_sweep = thread_launches() - c0;
  uncount_launches(per_sweep);
  if (ce != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return cuda_fail(ce, "SVD round capture"); }
  if (ce2 != cudaSuccess) return cuda_fail(ce2, "SVD sweep capture");
  ce = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) return cuda_fail(ce, "SVD sweep instantiate");
  std::vector<int> hrot(n_e);
  int sweep = 0;
  cbs_status status = CBS_OK;
  for (; sweep < max_sweeps; ++sweep) {
    ce = cudaGraphLaunch(exec, st);
    count_launches(per_sweep);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(hrot.data(), rot, (size_t)n_e * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) { status = cuda_fail(ce, "SVD sweep"); break; }
    int any = 0;
    for (int v : hrot) any |= (v != 0);
    if (!any) break;
  }
  cudaGraphExecDestroy(exec);
  if (status != CBS_OK) return status;
  // X V_x = U_x Sigma: A <- U_x, U <- V_x (sorted); then U <- Q V_x, Ws <- P U_x
  k_svd_finish<<<n_e, 1024, 0, st>>>(n, X, W, A, U, sig);
  cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  k_apply_q<<<dim3((unsigned)ceil_div(n, 16), (unsigned)n_e, 1), 512, 0, st>>>(n, Vh, beta, U);
  cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  k_permute_rows<<<dim3(64, (unsigned)n_e, 1), 256, 0, st>>>(n, perm, A, Ws);
  cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  // info: 1 if the sweep limit was reached (per energy: its last sweep still rotated)
  std::vector<int> hinfo(n_e);
  for (int e = 0; e < n_e; ++e) hinfo[e] = (sweep >= max_sweeps && hrot[e] != 0) ? 1 : 0;
  CBS_CUDA(cudaMemcpyAsync(info, hinfo.data(), (size_t)n_e * sizeof(int), cudaMemcpyHostToDevice, st));
  CBS_CUDA(cudaStreamSynchronize(st));
  return CBS_OK;
}

cbs_status launch_rank(int n_e, int n, const double *sig, double delta, int *mhat, cudaStream_t st) {
  k_rank<<<ceil_div(n_e, 64), 64, 0, st>>>(n_e, n, sig, delta, mhat); cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  return CBS_OK;
}

cbs_status launch_scale(int n_e, int rows, int ld, const int *mhat, const double *sig, double2 *B,
                        int rows_scale, cudaStream_t st) {
  k_scale_cols<<<dim3(64, (unsigned)n_e, 1), 256, 0, st>>>(rows, ld, mhat, sig, B, rows_scale); cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  return CBS_OK;
}

cbs_status launch_eig(int n_e, int ld, const int *mhat, double2 *B, double2 *Z, double2 *tau,
                      double2 *Yc, int *nring, int *ringidx, double lambda_min, int *info,
                      cudaStream_t st, double2 shift, int shifted) {
  if (ld > 512) { set_error("eigenproblem larger than 512"); return CBS_EINVAL; }
  k_eig<<<n_e, kEigThreads, 0, st>>>(ld, mhat, B, Z, tau, Yc, nring, ringidx, lambda_min, info, shift,
                                     shifted);
  cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  return CBS_OK;
}

cbs_status launch_filter(int64_t N, int cnt, const double2 *tau_ring, const double2 *Psi,
                         const double2 *Res, double *stats, double nHp, double nA, double nHm,
                         double rho_max, double a_cell, double *rho_all, int *n_keep, int *perm,
                         double2 *lam_out, double2 *k_out, double *rho_out, double2 *scale_out,
                         cudaStream_t st) {
  if (cnt <= 0) return CBS_OK;
  if (cnt > 512) { set_error("too many in-ring eigenvalues"); return CBS_EINVAL; }
  k_colstats<<<cnt, 256, 0, st>>>(N, cnt, Psi, Res, stats); cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  k_filter<<<1, 512, 0, st>>>(cnt, tau_ring, stats, nHp, nA, nHm, rho_max, a_cell, Psi, N, rho_all,
                              n_keep, perm, lam_out, k_out, rho_out, scale_out); cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  return CBS_OK;
}

cbs_status launch_gather_vectors(int64_t N, int cnt, int nk, const double2 *Psi, const int *perm,
                                 const double2 *scale, double2 *Out, cudaStream_t st) {
  if (nk <= 0) return CBS_OK;
  k_gather_vectors<<<152 * 4, 256, 0, st>>>(N, cnt, nk, Psi, perm, scale, Out); cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  return CBS_OK;
}

}  // namespace cbs
