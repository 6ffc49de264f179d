// Batched BiCG for the primal systems P(z_s) Y = B and their duals P(z_s)^dagger Y~ = B~.
//
// Paper §3.2: P(lambda)^dagger = P(1/conj lambda) and z^(2) = 1/conj z^(1), so the dual
// of an outer-circle system is the inner-circle system, and BiCG solves both for about
// the cost of one; every right-hand-side column is an independent BiCG run (§3.3, top
// layer).  Per column, with (a, b) = a^dagger b:
//     p = r + beta p,  p~ = r~ + conj(beta) p~                    (beta = 0 at the start)
//     q = P(z) p,      q~ = P(1/conj z) p~,   alpha = (r~, r) / (p~, q)
//     x += alpha p,  r -= alpha q,  x~ += conj(alpha) p~,  r~ -= conj(alpha) q~
//     beta = (r~', r') / (r~, r),  stop when ||r||/||b|| <= tol and ||r~||/||b~|| <= tol.
//
// All systems of a batch advance together; every kernel covers [2n][N][L] (primal
// systems then their duals).  Inner products are reduced in two deterministic levels:
// per-block partial sums over a chunk of grid points, then one thread per (system,
// column) adding the chunks in order.  One iteration = 6 launches (update p, apply,
// (p~, q), alpha, update x/r, beta); `check_every` iterations are captured in a CUDA
// graph and replayed until the device-side count of active systems reaches zero.
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <vector>

#include "bicg.cuh"

#define CBS_TRY_B(x)               \
  do {                             \
    cbs_status _s = (x);           \
    if (_s != CBS_OK) return _s;   \
  } while (0)

namespace cbs {

template <typename R>
__device__ __forceinline__ void block_partials(double (&acc)[4], double *part, int64_t slot) {
  extern __shared__ double red[];  // [py][L][4]
  const int c = threadIdx.x, ly = threadIdx.y, L = blockDim.x, py = blockDim.y;
  for (int k = 0; k < 4; ++k) red[((int64_t)ly * L + c) * 4 + k] = acc[k];
  __syncthreads();
  if (ly == 0) {
    double s[4] = {0, 0, 0, 0};
    for (int y = 0; y < py; ++y)
      for (int k = 0; k < 4; ++k) s[k] += red[((int64_t)y * L + c) * 4 + k];
    for (int k = 0; k < 4; ++k) part[(slot * L + c) * 4 + k] = s[k];
  }
}

template <typename R>
__global__ void k_init(int n, int64_t N, int L, int chunk_pts, int n_chunks, const double2 *B,
                       int64_t bstride, const double2 *Bd, int64_t bdstride,
                       typename CT<R>::T *x, typename CT<R>::T *r, typename CT<R>::T *p,
                       double *part) {
  typedef typename CT<R>::T C;
  const int s = blockIdx.y, chunk = blockIdx.x, c = threadIdx.x, ly = threadIdx.y, py = blockDim.y;
  double acc[4] = {0, 0, 0, 0};
  const int64_t i0 = (int64_t)chunk * chunk_pts;
  const int64_t i1 = min(N, i0 + chunk_pts);
  for (int64_t i = i0 + ly; i < i1; i += py) {
    const int64_t e = ((int64_t)s * N + i) * L + c, ed = ((int64_t)(n + s) * N + i) * L + c;
    C b = from_d<R>(B[(int64_t)s * bstride + i * L + c]);
    C bd = from_d<R>(Bd[(int64_t)s * bdstride + i * L + c]);
    r[e] = b; r[ed] = bd;
    x[e] = mk<R>(0, 0); x[ed] = mk<R>(0, 0);
    p[e] = mk<R>(0, 0); p[ed] = mk<R>(0, 0);
    double2 bdd = to_d(bd), bb = to_d(b);
    acc[0] += bdd.x * bb.x + bdd.y * bb.y;   // conj(bd) * b
    acc[1] += bdd.x * bb.y - bdd.y * bb.x;
    acc[2] += cabs2(bb);
    acc[3] += cabs2(bdd);
  }
  block_partials<R>(acc, part, (int64_t)s * n_chunks + chunk);
}

__global__ void k_reduce_init(int n, int L, int n_chunks, const double *part, double2 *rho,
                              double2 *rho_prev, double2 *beta, double *nb, double *nbd,
                              double *tgt, double *tgtd, double *rmax, double *rmaxd, double tfloor,
                              const double *ref_norm, int *active, int *iters, int *flags,
                              const int *colmask, int *sys_active, int *n_active) {
  const int s = blockIdx.x, c = threadIdx.x;
  const int64_t k = (int64_t)s * L + c;
  double a[4] = {0, 0, 0, 0};
  for (int ch = 0; ch < n_chunks; ++ch)
    for (int q = 0; q < 4; ++q) a[q] += part[(((int64_t)s * n_chunks + ch) * L + c) * 4 + q];
  rho[k] = make_double2(a[0], a[1]);
  rho_prev[k] = make_double2(0, 0);
  beta[k] = make_double2(0, 0);
  nb[k] = sqrt(a[2]);
  nbd[k] = sqrt(a[3]);
  // absolute targets: relative to this right-hand side, or to reference norms
  // ref_norm[2n][L] (primal then dual) when the system solves for a correction
  tgt[k] = tfloor * (ref_norm ? ref_norm[k] : nb[k]);
  tgtd[k] = tfloor * (ref_norm ? ref_norm[(int64_t)n * L + k] : nbd[k]);
  rmax[k] = nb[k];
  rmaxd[k] = nbd[k];
  int act = (colmask ? colmask[k] : 1) && a[2] > 0 && a[3] > 0;
  active[k] = act;
  iters[k] = 0;
  flags[k] = 0;
  int any = __syncthreads_or(act);
  if (c == 0) {
    sys_active[s] = any;
    sys_active[n + s] = any;
    if (any) atomicAdd(n_active, 1);
  }
}

template <typename R>
__global__ void k_update_p(int n, int64_t N, int L, int chunk_pts, const typename CT<R>::T *r,
                           typename CT<R>::T *p, const double2 *beta, const int *active,
                           const int *sys_active) {
  typedef typename CT<R>::T C;
  const int s = blockIdx.y, chunk = blockIdx.x, c = threadIdx.x, ly = threadIdx.y, py = blockDim.y;
  if (!sys_active[s]) return;
  const int64_t k = (int64_t)s * L + c;
  if (!active[k]) return;
  const C b = from_d<R>(beta[k]), bc = cconj(b);
  const int64_t i0 = (int64_t)chunk * chunk_pts;
  const int64_t i1 = min(N, i0 + chunk_pts);
  for (int64_t i = i0 + ly; i < i1; i += py) {
    const int64_t e = ((int64_t)s * N + i) * L + c, ed = ((int64_t)(n + s) * N + i) * L + c;
    p[e] = cfma(b, p[e], r[e]);
    p[ed] = cfma(bc, p[ed], r[ed]);
  }
}

template <typename R>
__global__ void k_dot_pq(int n, int64_t N, int L, int chunk_pts, int n_chunks,
                         const typename CT<R>::T *p, const typename CT<R>::T *q, double *part,
                         const int *sys_active) {
  typedef typename CT<R>::T C;
  const int s = blockIdx.y, chunk = blockIdx.x, c = threadIdx.x, ly = threadIdx.y, py = blockDim.y;
  if (!sys_active[s]) return;
  double acc[4] = {0, 0, 0, 0};
  const int64_t i0 = (int64_t)chunk * chunk_pts;
  const int64_t i1 = min(N, i0 + chunk_pts);
  // (p~, q) decides alpha: its products are formed and summed in FP64 also for complex64
  // vectors (a single-precision sum loses the small inner products of late iterations to
  // cancellation, which stalls the recurrence)
  double ax = 0, ay = 0;
  for (int64_t i = i0 + ly; i < i1; i += py) {
    const double2 pd = to_d(p[((int64_t)(n + s) * N + i) * L + c]);
    const double2 qq = to_d(q[((int64_t)s * N + i) * L + c]);
    ax += pd.x * qq.x + pd.y * qq.y;
    ay += pd.x * qq.y - pd.y * qq.x;
  }
  acc[0] = ax; acc[1] = ay;
  block_partials<R>(acc, part, (int64_t)s * n_chunks + chunk);
}

__global__ void k_reduce_alpha(int n, int L, int n_chunks, const double *part, const double2 *rho,
                               double2 *alpha, int *active, int *flags, const int *sys_active,
                               unsigned long long *sys_apply) {
  const int s = blockIdx.x, c = threadIdx.x;
  if (!sys_active[s]) return;
  if (c == 0 && sys_apply) atomicAdd(sys_apply, 1ull);   // system s went through this apply
  const int64_t k = (int64_t)s * L + c;
  if (!active[k]) { alpha[k] = make_double2(0, 0); return; }
  double gx = 0, gy = 0;
  for (int ch = 0; ch < n_chunks; ++ch) {
    gx += part[(((int64_t)s * n_chunks + ch) * L + c) * 4 + 0];
    gy += part[(((int64_t)s * n_chunks + ch) * L + c) * 4 + 1];
  }
  double2 g = make_double2(gx, gy);
  double g2 = cabs2(g);
  if (!(g2 > 0) || !isfinite(g2)) {
    flags[k] |= 2;
    active[k] = 0;
    alpha[k] = make_double2(0, 0);
    return;
  }
  alpha[k] = cdiv(rho[k], g);
}

template <typename R>
__global__ void k_pass_b(int n, int64_t N, int L, int chunk_pts, int n_chunks,
                         typename CT<R>::T *x, typename CT<R>::T *r, const typename CT<R>::T *p,
                         const typename CT<R>::T *q, const double2 *alpha, const int *active,
                         double *part, const int *sys_active) {
  typedef typename CT<R>::T C;
  const int s = blockIdx.y, chunk = blockIdx.x, c = threadIdx.x, ly = threadIdx.y, py = blockDim.y;
  if (!sys_active[s]) return;
  const int64_t k = (int64_t)s * L + c;
  const bool act = active[k];
  const C a = from_d<R>(alpha[k]), ac = cconj(a);
  const C na = mk<R>(-a.x, -a.y), nac = mk<R>(-a.x, a.y);
  // rho = (r~, r) in FP64 products and sums (it decides beta; see k_dot_pq); the norms,
  // sums of squares without cancellation, in the working precision
  double s0 = 0, s1 = 0;
  R s2 = 0, s3 = 0;
  const int64_t i0 = (int64_t)chunk * chunk_pts;
  const int64_t i1 = min(N, i0 + chunk_pts);
  if (act) {
    for (int64_t i = i0 + ly; i < i1; i += py) {
      const int64_t e = ((int64_t)s * N + i) * L + c, ed = ((int64_t)(n + s) * N + i) * L + c;
      if (x) x[e] = cfma(a, p[e], x[e]);      // no x for the seed of a shifted family
      C rr = cfma(na, q[e], r[e]);
      r[e] = rr;
      if (x) x[ed] = cfma(ac, p[ed], x[ed]);
      C rd = cfma(nac, q[ed], r[ed]);
      r[ed] = rd;
      const double2 r1 = to_d(rr), r2 = to_d(rd);
      s0 += r2.x * r1.x + r2.y * r1.y;
      s1 += r2.x * r1.y - r2.y * r1.x;
      s2 += rr.x * rr.x + rr.y * rr.y;
      s3 += rd.x * rd.x + rd.y * rd.y;
    }
  }
  double acc[4] = {s0, s1, (double)s2, (double)s3};
  block_partials<R>(acc, part, (int64_t)s * n_chunks + chunk);
}

__global__ void k_reduce_beta(int n, int L, int n_chunks, const double *part, double2 *rho,
                              double2 *rho_prev, double2 *beta, const double *tgt,
                              const double *tgtd, double *rmax, double *rmaxd, double tfac,
                              int *active, int *iters, int *flags, int max_iter, int *sys_active,
                              int *n_active) {
  const int s = blockIdx.x, c = threadIdx.x;
  if (!sys_active[s]) return;   // uniform per block
  const int64_t k = (int64_t)s * L + c;
  int act = active[k];
  if (act) {
    double a[4] = {0, 0, 0, 0};
    for (int ch = 0; ch < n_chunks; ++ch)
      for (int q = 0; q < 4; ++q) a[q] += part[(((int64_t)s * n_chunks + ch) * L + c) * 4 + q];
    const int it = iters[k] + 1;
    iters[k] = it;
    const double nr = sqrt(a[2]), nrd = sqrt(a[3]);
    const double2 rn = make_double2(a[0], a[1]);
    const double2 rold = rho[k];
    rho_prev[k] = rold;                  // kept for a later residual replacement
    rho[k] = rn;
    // stop (or pause until the next residual replacement) below max(tfac * the largest
    // residual norm since the last replacement, the absolute target)
    const double mx = fmax(rmax[k], nr), mxd = fmax(rmaxd[k], nrd);
    rmax[k] = mx;
    rmaxd[k] = mxd;
    if (nr <= fmax(tfac * mx, tgt[k]) && nrd <= fmax(tfac * mxd, tgtd[k])) {
      act = 0;
    } else if (!isfinite(nr) || !isfinite(nrd) || !(cabs2(rn) > 0)) {
      flags[k] |= 2;
      act = 0;
    } else if (it >= max_iter) {
      flags[k] |= 1;
      act = 0;
    } else {
      beta[k] = cdiv(rn, rold);
    }
    active[k] = act;
  }
  if (!act) beta[k] = make_double2(0, 0);
  int any = __syncthreads_or(act);
  if (c == 0) {
    sys_active[s] = any;
    sys_active[n + s] = any;
    if (any) atomicAdd(n_active, 1);
  }
}

// Load-balance rule of §3.3 (second stopping rule): the systems of one energy are its
// n_pt quadrature points (systems e * n_pt + j, duals n + s); once more than `need` of them
// have stopped, the others of that energy are stopped too.  A system counts as stopped when
// none of its columns is active; the columns stopped by the rule get flag bit 6.
// One block per energy, one thread per point (n_pt <= 1024).
__global__ void k_group_stop(int n, int n_pt, int L, int need, int *active, int *flags,
                             int *sys_active) {
  const int e = blockIdx.x, j = threadIdx.x;
  const int s = e * n_pt + j;
  const int stopped = j < n_pt ? !sys_active[s] : 0;
  const int count = __syncthreads_count(stopped);
  if (count <= need || j >= n_pt || stopped) return;
  for (int c = 0; c < L; ++c) {
    const int64_t k = (int64_t)s * L + c;
    if (active[k]) { active[k] = 0; flags[k] |= 64; }
  }
  sys_active[s] = 0;
  sys_active[n + s] = 0;
}

// The same rule for a shifted family: for energy e, point j counts as stopped when none of
// its (e, j) columns is active.
__global__ void k_ms_group_stop(int n_pt, int L, int need, int *sactive, int *sflags, int *siters,
                                const int *seed_iters) {
  const int e = blockIdx.x, j = threadIdx.x;
  int live = 0;
  if (j < n_pt)
    for (int c = 0; c < L; ++c) live |= sactive[((int64_t)e * n_pt + j) * L + c];
  const int count = __syncthreads_count(j < n_pt && !live);
  if (count <= need || j >= n_pt || !live) return;
  for (int c = 0; c < L; ++c) {
    const int64_t kk = ((int64_t)e * n_pt + j) * L + c;
    if (sactive[kk]) {
      sactive[kk] = 0;
      sflags[kk] |= 64;
      siters[kk] = seed_iters[(int64_t)j * L + c];
    }
  }
}

// Residual replacement (mixed precision): the recursive residuals of the columns that
// still need work are replaced by the FP64 true residuals R = B - P(z)Y (rounded to the
// working type), the correction x restarts from zero (it has been added to Y), and the
// search directions p, p~ are kept.  Partial sums give rho' = (r~', r'), ||r'||, ||r~'||.
template <typename R>
__global__ void k_replace(int n, int64_t N, int L, int chunk_pts, int n_chunks,
                          const double2 *R64, const int *colmask, typename CT<R>::T *x,
                          typename CT<R>::T *r, double *part) {
  typedef typename CT<R>::T C;
  const int s = blockIdx.y, chunk = blockIdx.x, c = threadIdx.x, ly = threadIdx.y, py = blockDim.y;
  const int64_t k = (int64_t)s * L + c;
  const bool need = colmask[k];
  double acc[4] = {0, 0, 0, 0};
  const int64_t i0 = (int64_t)chunk * chunk_pts;
  const int64_t i1 = min(N, i0 + chunk_pts);
  for (int64_t i = i0 + ly; i < i1; i += py) {
    const int64_t e = ((int64_t)s * N + i) * L + c, ed = ((int64_t)(n + s) * N + i) * L + c;
    x[e] = mk<R>(0, 0);
    x[ed] = mk<R>(0, 0);
    if (need) {
      const C b = from_d<R>(R64[e]), bd = from_d<R>(R64[ed]);
      r[e] = b;
      r[ed] = bd;
      const double2 bb = to_d(b), bdd = to_d(bd);
      acc[0] += bdd.x * bb.x + bdd.y * bb.y;
      acc[1] += bdd.x * bb.y - bdd.y * bb.x;
      acc[2] += cabs2(bb);
      acc[3] += cabs2(bdd);
    }
  }
  block_partials<R>(acc, part, (int64_t)s * n_chunks + chunk);
}

__global__ void k_reduce_replace(int n, int L, int n_chunks, const double *part, double2 *rho,
                                 const double2 *rho_prev, double2 *beta, double *rmax, double *rmaxd,
                                 int *active, const int *colmask, int *sys_active, int *n_active) {
  const int s = blockIdx.x, c = threadIdx.x;
  const int64_t k = (int64_t)s * L + c;
  int act = colmask[k];
  if (act) {
    double a[4] = {0, 0, 0, 0};
    for (int ch = 0; ch < n_chunks; ++ch)
      for (int q = 0; q < 4; ++q) a[q] += part[(((int64_t)s * n_chunks + ch) * L + c) * 4 + q];
    const double2 rn = make_double2(a[0], a[1]);
    const double2 rp = rho_prev[k];
    beta[k] = (cabs2(rp) > 0) ? cdiv(rn, rp) : make_double2(0, 0);
    rho[k] = rn;
    rmax[k] = sqrt(a[2]);
    rmaxd[k] = sqrt(a[3]);
    if (!(cabs2(rn) > 0) || !isfinite(a[2]) || !isfinite(a[3])) { act = 0; beta[k] = make_double2(0, 0); }
  } else {
    beta[k] = make_double2(0, 0);
  }
  active[k] = act;
  int any = __syncthreads_or(act);
  if (c == 0) {
    sys_active[s] = any;
    sys_active[n + s] = any;
    if (any) atomicAdd(n_active, 1);
  }
}

__global__ void k_twists(int n, const double2 *z, const double *E, double2 *tw, double *E2) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) {
    double2 zz = z[s];
    tw[s] = zz;
    tw[n + s] = cdiv(make_double2(1.0, 0.0), cconj(zz));   // 1/conj(z): dual system (§3.2)
    E2[s] = E[s];
    E2[n + s] = E[s];
  }
}

cbs_status launch_twists(int n, const double2 *z, const double *E, double2 *tw, double *E2,
                         cudaStream_t st) {
  k_twists<<<ceil_div(n, 128), 128, 0, st>>>(n, z, E, tw, E2); cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  return CBS_OK;
}

// ---------------------------------------------------------------- Bicg<R> members
static int64_t align256(int64_t b) { return (b + 255) & ~(int64_t)255; }

static void chunking(int64_t N, int L, int *chunk_pts, int *n_chunks) {
  dim3 blk = col_block(L);
  int64_t cp = (N + 127) / 128;                       // at most 128 chunks per system
  int64_t minp = (int64_t)blk.y * 8;
  if (cp < minp) cp = minp;
  cp = ((cp + blk.y - 1) / blk.y) * blk.y;
  *chunk_pts = (int)cp;
  *n_chunks = (int)((N + cp - 1) / cp);
}

template <typename R>
size_t Bicg<R>::bytes_needed(const HamView &H, int n, int L) {
  int cp, nc;
  chunking(H.n, L, &cp, &nc);
  const int64_t vec = (int64_t)2 * n * H.n * L * sizeof(C);
  int64_t b = 4 * align256(vec);
  b += align256((int64_t)2 * n * (H.n_atoms ? H.n_atoms : 1) * H.np4 * L * sizeof(C));
  b += align256((int64_t)2 * n * sizeof(double2)) + align256((int64_t)2 * n * sizeof(double));
  b += 4 * align256((int64_t)n * L * sizeof(double2)) + 6 * align256((int64_t)n * L * sizeof(double));
  b += 3 * align256((int64_t)n * L * sizeof(int)) + align256((int64_t)2 * n * sizeof(int)) + 256;
  b += align256((int64_t)n * nc * L * 4 * sizeof(double)) + 256;
  return (size_t)b;
}

template <typename R>
cbs_status Bicg<R>::alloc(const HamView &H_, int n_, int L_) {
  H = H_; n = n_; L = L_; N = H.n;
  chunking(N, L, &chunk_pts, &n_chunks);
  bytes = bytes_needed(H, n, L);
  cudaError_t e = cudaMalloc(&block, bytes);
  if (e != cudaSuccess) {
    block = nullptr;
    set_error("cudaMalloc of the BiCG state failed (reduce energies_per_batch)");
    return CBS_ENOMEM;
  }
  char *b = (char *)block;
  auto take = [&](int64_t sz) { char *r = b; b += align256(sz); return (void *)r; };
  const int64_t vec = (int64_t)2 * n * N * L * sizeof(C);
  x = (C *)take(vec); r = (C *)take(vec); p = (C *)take(vec); q = (C *)take(vec);
  D = (C *)take((int64_t)2 * n * (H.n_atoms ? H.n_atoms : 1) * H.np4 * L * sizeof(C));
  tw = (double2 *)take((int64_t)2 * n * sizeof(double2));
  E = (double *)take((int64_t)2 * n * sizeof(double));
  rho = (double2 *)take((int64_t)n * L * sizeof(double2));
  alpha = (double2 *)take((int64_t)n * L * sizeof(double2));
  beta = (double2 *)take((int64_t)n * L * sizeof(double2));
  rho_prev = (double2 *)take((int64_t)n * L * sizeof(double2));
  tgt = (double *)take((int64_t)n * L * sizeof(double));
  tgtd = (double *)take((int64_t)n * L * sizeof(double));
  rmax = (double *)take((int64_t)n * L * sizeof(double));
  rmaxd = (double *)take((int64_t)n * L * sizeof(double));
  nb = (double *)take((int64_t)n * L * sizeof(double));
  nbd = (double *)take((int64_t)n * L * sizeof(double));
  active = (int *)take((int64_t)n * L * sizeof(int));
  iters = (int *)take((int64_t)n * L * sizeof(int));
  flags = (int *)take((int64_t)n * L * sizeof(int));
  sys_active = (int *)take((int64_t)2 * n * sizeof(int));
  n_active = (int *)take(256);
  part = (double *)take((int64_t)n * n_chunks * L * 4 * sizeof(double));
  sys_apply = (unsigned long long *)take(256);
  CBS_CUDA(cudaMemset(sys_apply, 0, sizeof(unsigned long long)));
  return CBS_OK;
}

template <typename R>
void Bicg<R>::release() {
  if (block) cudaFree(block);
  block = nullptr;
  for (int k = 0; k < n_prof_ev; ++k) cudaEventDestroy(prof_ev[k]);
  n_prof_ev = 0;
  if (exec) cudaGraphExecDestroy(exec);
  exec = nullptr;
  exec_max_iter = exec_check_every = -1;
  if (h_active) cudaFreeHost(h_active);
  h_active = nullptr;
}

template <typename R>
cbs_status Bicg<R>::prof_outputs(cudaStream_t st, double *out) {
  unsigned long long v = 0;
  CBS_CUDA(cudaMemcpyAsync(&v, sys_apply, sizeof(v), cudaMemcpyDeviceToHost, st));
  CBS_CUDA(cudaStreamSynchronize(st));
  *out = 2.0 * (double)v * (double)N * (double)L;
  return CBS_OK;
}

template <typename R>
cbs_status Bicg<R>::set_systems(const double2 *z, const double *Es, cudaStream_t st) {
  return launch_twists(n, z, Es, tw, E, st);
}

static size_t red_smem(int L) {
  dim3 b = col_block(L);
  return (size_t)b.x * b.y * 4 * sizeof(double);
}

template <typename R>
cbs_status Bicg<R>::init(const double2 *B, int64_t bstride, const double2 *Bd, int64_t bdstride,
                         const int *colmask, double tfloor, double tfac_, cudaStream_t st,
                         const double *ref_norm) {
  tfac = tfac_;
  dim3 blk = col_block(L);
  dim3 grd((unsigned)n_chunks, (unsigned)n, 1);
  k_init<R><<<grd, blk, red_smem(L), st>>>(n, N, L, chunk_pts, n_chunks, B, bstride, Bd, bdstride,
                                          x, r, p, part); cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  CBS_CUDA(cudaMemsetAsync(n_active, 0, sizeof(int), st));
  k_reduce_init<<<n, L, 0, st>>>(n, L, n_chunks, part, rho, rho_prev, beta, nb, nbd, tgt, tgtd, rmax,
                                 rmaxd, tfloor, ref_norm, active, iters, flags, colmask, sys_active,
                                 n_active); cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  return CBS_OK;
}

template <typename R>
cbs_status Bicg<R>::step(double tol, int max_iter, cudaStream_t st, int kk) {
  dim3 blk = col_block(L);
  dim3 grd((unsigned)n_chunks, (unsigned)n, 1);
  k_update_p<R><<<grd, blk, 0, st>>>(n, N, L, chunk_pts, r, p, beta, active, sys_active); cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  const bool prof = profile && kk >= 0 && 2 * kk + 1 < n_prof_ev;
  // recorded as real event nodes of the graph (not capture-dependency markers)
  if (prof) CBS_CUDA(cudaEventRecordWithFlags(prof_ev[2 * kk], st, cudaEventRecordExternal));
  cbs_status s = apply_P<R>(H, 2 * n, L, p, q, tw, false, E, D, sys_active, st);
  if (s != CBS_OK) return s;
  if (prof) CBS_CUDA(cudaEventRecordWithFlags(prof_ev[2 * kk + 1], st, cudaEventRecordExternal));
  k_dot_pq<R><<<grd, blk, red_smem(L), st>>>(n, N, L, chunk_pts, n_chunks, p, q, part, sys_active); cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  k_reduce_alpha<<<n, L, 0, st>>>(n, L, n_chunks, part, rho, alpha, active, flags, sys_active,
                                  sys_apply); cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  k_pass_b<R><<<grd, blk, red_smem(L), st>>>(n, N, L, chunk_pts, n_chunks, x, r, p, q, alpha,
                                             active, part, sys_active); cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  CBS_CUDA(cudaMemsetAsync(n_active, 0, sizeof(int), st));
  k_reduce_beta<<<n, L, 0, st>>>(n, L, n_chunks, part, rho, rho_prev, beta, tgt, tgtd, rmax, rmaxd,
                                 tfac, active, iters, flags, max_iter, sys_active, n_active); cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  if (group > 0 && group_need < group) {
    k_group_stop<<<n / group, ((group + 31) / 32) * 32, 0, st>>>(n, group, L, group_need, active, flags, sys_active);
    cbs::count_launches(1);
    CBS_CUDA(cudaGetLastError());
  }
  return CBS_OK;
}

template <typename R>
cbs_status Bicg<R>::iterate(double tol, int max_iter, int check_every, cudaStream_t st,
                            int *host_iters_done, int call_cap) {
  if (check_every < 1) check_every = 1;
  if (profile && n_prof_ev == 0) {
    const int ne = 2 * (check_every < 64 ? check_every : 64);
    for (int k = 0; k < ne; ++k) CBS_CUDA(cudaEventCreate(&prof_ev[k]));
    n_prof_ev = ne;
  }
  if (!h_active) CBS_CUDA(cudaMallocHost(&h_active, sizeof(int)));
  if (!exec || exec_max_iter != max_iter || exec_check_every != check_every) {
    if (exec) { cudaGraphExecDestroy(exec); exec = nullptr; }
    cudaGraph_t graph = nullptr;
    const uint64_t c0 = thread_launches();
    CBS_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    cbs_status s = CBS_OK;
    for (int k = 0; k < check_every && s == CBS_OK; ++k) s = step(tol, max_iter, st, k);
    cudaError_t ce = cudaStreamEndCapture(st, &graph);
    exec_kernels = thread_launches() - c0;
    uncount_launches(exec_kernels);
    if (s != CBS_OK) { if (graph) cudaGraphDestroy(graph); return s; }
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) { exec = nullptr; return cuda_fail(ce, "cudaGraphInstantiate"); }
    exec_max_iter = max_iter;
    exec_check_every = check_every;
  }
  int done = 0;
  cbs_status s = CBS_OK;
  // every replay advances all still-active columns by check_every iterations; max_iter is
  // also enforced per column on the device, so the loop ends within max_iter/check_every + 1
  int max_replays = max_iter / check_every + 2;
  if (call_cap > 0) max_replays = std::min(max_replays, (call_cap + check_every - 1) / check_every);
  for (int rep = 0; rep < max_replays; ++rep) {
    cudaError_t ce = cudaGraphLaunch(exec, st);
    count_launches(exec_kernels);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(h_active, n_active, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) { s = cuda_fail(ce, "BiCG graph replay"); break; }
    if (profile) {
      for (int k = 0; 2 * k + 1 < n_prof_ev && k < check_every; ++k) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, prof_ev[2 * k], prof_ev[2 * k + 1]) == cudaSuccess) {
          prof_ms += ms;
          prof_launches += 1;
        } else {
          (void)cudaGetLastError();   // do not leave a sticky error for the next check
        }
      }
    }
    done += check_every;
    if (*h_active == 0) break;
  }
  if (host_iters_done) *host_iters_done = done;
  return s;
}

template <typename R>
cbs_status Bicg<R>::replace(const double2 *R64, const int *colmask, cudaStream_t st) {
  dim3 blk = col_block(L);
  dim3 grd((unsigned)n_chunks, (unsigned)n, 1);
  k_replace<R><<<grd, blk, red_smem(L), st>>>(n, N, L, chunk_pts, n_chunks, R64, colmask, x, r, part);
  cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  CBS_CUDA(cudaMemsetAsync(n_active, 0, sizeof(int), st));
  k_reduce_replace<<<n, L, 0, st>>>(n, L, n_chunks, part, rho, rho_prev, beta, rmax, rmaxd, active,
                                    colmask, sys_active, n_active);
  cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  return CBS_OK;
}

template struct Bicg<double>;
template struct Bicg<float>;

// ---------------------------------------------------------------- shifted family (MultiShift)
__global__ void k_ms_init(int n_pt, int n_sh, int L, const int *seed_active, double2 *pi,
                          double2 *pi_prev, double2 *alpha_prev, int *sactive, int *siters,
                          int *sflags) {
  const int j = blockIdx.x, c = threadIdx.x;
  const int64_t k = (int64_t)j * L + c;
  alpha_prev[k] = make_double2(1, 0);
  for (int e = 0; e < n_sh; ++e) {
    const int64_t kk = ((int64_t)e * n_pt + j) * L + c;
    pi[kk] = make_double2(1, 0);
    pi_prev[kk] = make_double2(1, 0);
    sactive[kk] = seed_active[k];
    siters[kk] = 0;
    sflags[kk] = 0;
  }
}

// after alpha_k: pi^{k+1} and the coefficients of this iteration for every energy
__global__ void k_ms_coef(int n_pt, int n_sh, int L, const double *sigma, const double2 *alpha,
                          const double2 *beta, double2 *alpha_prev, double2 *pi, double2 *pi_prev,
                          double2 *cb, double2 *ca, int *sactive, int *sflags,
                          const int *seed_sys_active, unsigned long long *upd_cols) {
  const int j = blockIdx.x, c = threadIdx.x;
  if (!seed_sys_active[j]) return;
  int live = 0;
  const int64_t k = (int64_t)j * L + c;
  const double2 a = alpha[k], b = beta[k], ap = alpha_prev[k];
  const bool first = !(cabs2(b) > 0);
  const double2 g = first ? make_double2(0, 0) : cdiv(cmul(a, b), ap);
  for (int e = 0; e < n_sh; ++e) {
    const int64_t kk = ((int64_t)e * n_pt + j) * L + c;
    if (!sactive[kk]) {
      cb[kk] = ca[kk] = make_double2(0, 0);
      continue;
    }
    const double2 pk = pi[kk], pm = pi_prev[kk];
    const double2 f = make_double2(1.0 + a.x * sigma[e], a.y * sigma[e]);
    const double2 pn = cadd(cmul(f, pk), cmul(g, csub(pk, pm)));
    const double m2 = cabs2(pn);
    if (!(m2 > 0) || !isfinite(m2)) {
      sflags[kk] |= 2;
      sactive[kk] = 0;
      cb[kk] = ca[kk] = make_double2(0, 0);
      continue;
    }
    // the kernel keeps p^_e = pi_e^k p_e: p^_e = r + (pi_e^{k-1} / pi_e^k) beta_{k-1} p^_e,
    // x_e += (alpha_k / pi_e^{k+1}) p^_e  (4 FP64 FMA each per component pair)
    cb[kk] = first ? make_double2(0, 0) : cmul(cdiv(pm, pk), b);
    ca[kk] = cdiv(a, pn);
    pi_prev[kk] = pk;
    pi[kk] = pn;
    ++live;
  }
  alpha_prev[k] = a;
  if (upd_cols) {
    for (int o = 16; o > 0; o >>= 1) live += __shfl_xor_sync(0xffffffffu, live, o);
    if ((c & 31) == 0 && live) atomicAdd(upd_cols, (unsigned long long)live);
  }
}

// p^_e = r + cb p^_e, x_e += ca p^_e (primal; p^_e = pi_e^k p_e, the scaled search
// direction); conjugated coefficients for the dual.  One block per (chunk of points,
// quadrature point); every energy of that point reads the same seed residual chunk.
template <typename R>
__global__ void k_ms_update(int n_pt, int n_sh, int64_t N, int L, int chunk_pts,
                            const typename CT<R>::T *__restrict__ r, typename CT<R>::T *__restrict__ P,
                            typename CT<R>::T *__restrict__ X, const double2 *cb, const double2 *ca,
                            const int *sactive, const int *seed_sys_active) {
  typedef typename CT<R>::T C;
  const int j = blockIdx.y, chunk = blockIdx.x, c = threadIdx.x, ly = threadIdx.y, py = blockDim.y;
  if (!seed_sys_active[j]) return;
  const int64_t n = (int64_t)n_sh * n_pt;
  const int64_t i0 = (int64_t)chunk * chunk_pts;
  const int64_t i1 = min(N, i0 + chunk_pts);
  const C *rp = r + (int64_t)j * N * L, *rd = r + (int64_t)(n_pt + j) * N * L;
  for (int e = 0; e < n_sh; ++e) {
    const int64_t s = (int64_t)e * n_pt + j;
    const int64_t kk = s * L + c;
    if (!sactive[kk]) continue;
    const C b = from_d<R>(cb[kk]), al = from_d<R>(ca[kk]);
    const C bc = cconj(b), alc = cconj(al);
    C *Pp = P + s * N * L, *Xp = X + s * N * L;
    C *Pd = P + (n + s) * N * L, *Xd = X + (n + s) * N * L;
    for (int64_t i = i0 + ly; i < i1; i += py) {
      const int64_t o = i * L + c;
      const C pv = cfma(b, Pp[o], rp[o]);
      Pp[o] = pv;
      Xp[o] = cfma(al, pv, Xp[o]);
      const C pdv = cfma(bc, Pd[o], rd[o]);
      Pd[o] = pdv;
      Xd[o] = cfma(alc, pdv, Xd[o]);
    }
  }
}

// seed reduction after the residual update: new rho, norms; every energy checks
// ||r|| / |pi_e^{k+1}| (and the dual); the seed column runs while one of them is active
__global__ void k_ms_reduce_beta(int n_pt, int n_sh, int L, int n_chunks, const double *part,
                                 double2 *rho, double2 *rho_prev, double2 *beta, const double *tgt,
                                 const double *tgtd, int *active, int *iters, int *flags,
                                 int max_iter, int *sys_active, int *n_active, const double2 *pi,
                                 int *sactive, int *siters, int *sflags) {
  const int j = blockIdx.x, c = threadIdx.x;
  if (!sys_active[j]) return;   // uniform per block
  const int64_t k = (int64_t)j * L + c;
  int act = active[k];
  if (act) {
    double a[4] = {0, 0, 0, 0};
    for (int ch = 0; ch < n_chunks; ++ch)
      for (int q = 0; q < 4; ++q) a[q] += part[(((int64_t)j * n_chunks + ch) * L + c) * 4 + q];
    const int it = iters[k] + 1;
    iters[k] = it;
    const double nr = sqrt(a[2]), nrd = sqrt(a[3]);
    const double2 rn = make_double2(a[0], a[1]);
    const double2 rold = rho[k];
    rho_prev[k] = rold;
    rho[k] = rn;
    int live = 0;
    for (int e = 0; e < n_sh; ++e) {
      const int64_t kk = ((int64_t)e * n_pt + j) * L + c;
      if (!sactive[kk]) continue;
      const double m = sqrt(cabs2(pi[kk]));
      if (nr <= tgt[k] * m && nrd <= tgtd[k] * m) {
        sactive[kk] = 0;
        siters[kk] = it;
      } else {
        live = 1;
      }
    }
    int stop_flag = 0;
    if (!live) act = 0;
    else if (!isfinite(nr) || !isfinite(nrd) || !(cabs2(rn) > 0)) stop_flag = 2;
    else if (it >= max_iter) stop_flag = 1;
    else beta[k] = cdiv(rn, rold);
    if (stop_flag) {
      flags[k] |= stop_flag;
      for (int e = 0; e < n_sh; ++e) {
        const int64_t kk = ((int64_t)e * n_pt + j) * L + c;
        if (!sactive[kk]) continue;
        sactive[kk] = 0;
        siters[kk] = it;
        sflags[kk] |= stop_flag;
      }
      act = 0;
    }
    active[k] = act;
  }
  if (!act) beta[k] = make_double2(0, 0);
  int any = __syncthreads_or(act);
  if (c == 0) {
    sys_active[j] = any;
    sys_active[n_pt + j] = any;
    if (any) atomicAdd(n_active, 1);
  }
}

template <typename R>
size_t MultiShift<R>::bytes_needed(const HamView &H, int n_pt, int n_sh, int L) {
  const int64_t n = (int64_t)n_pt * n_sh;
  int64_t b = align256(2 * n * H.n * L * (int64_t)sizeof(C));                 // P
  b += 4 * align256(n * L * (int64_t)sizeof(double2)) + align256((int64_t)n_pt * L * sizeof(double2));
  b += align256((int64_t)n_sh * sizeof(double)) + 3 * align256(n * L * (int64_t)sizeof(int)) + 512;
  return (size_t)b + Bicg<R>::bytes_needed(H, n_pt, L) +
         (size_t)align256(2 * n * H.n * L * (int64_t)sizeof(C));                // X
}

template <typename R>
cbs_status MultiShift<R>::alloc(const HamView &H, int n_pt_, int n_sh_, int L_) {
  n_pt = n_pt_; n_sh = n_sh_; L = L_; N = H.n;
  CBS_TRY_B(seed.alloc(H, n_pt, L));
  const int64_t n = (int64_t)n_pt * n_sh;
  const int64_t vec = align256(2 * n * N * L * (int64_t)sizeof(C));
  const int64_t bytes = (int64_t)bytes_needed(H, n_pt, n_sh, L) - (int64_t)Bicg<R>::bytes_needed(H, n_pt, L) - vec;
  if (cudaMalloc(&block, bytes) != cudaSuccess) {
    block = nullptr;
    set_error("cudaMalloc of the shifted-family BiCG state failed (reduce energies_per_batch)");
    return CBS_ENOMEM;
  }
  if (cudaMalloc(&xblock, vec) != cudaSuccess) {
    xblock = nullptr;
    set_error("cudaMalloc of the shifted-family solutions failed (reduce energies_per_batch)");
    return CBS_ENOMEM;
  }
  X = (C *)xblock;
  char *b = (char *)block;
  auto take = [&](int64_t sz) { char *r = b; b += align256(sz); return (void *)r; };
  P = (C *)take(2 * n * N * L * (int64_t)sizeof(C));
  pi = (double2 *)take(n * L * (int64_t)sizeof(double2));
  pi_prev = (double2 *)take(n * L * (int64_t)sizeof(double2));
  cb = (double2 *)take(n * L * (int64_t)sizeof(double2));
  ca = (double2 *)take(n * L * (int64_t)sizeof(double2));
  alpha_prev = (double2 *)take((int64_t)n_pt * L * sizeof(double2));
  sigma = (double *)take((int64_t)n_sh * sizeof(double));
  sactive = (int *)take(n * L * (int64_t)sizeof(int));
  siters = (int *)take(n * L * (int64_t)sizeof(int));
  sflags = (int *)take(n * L * (int64_t)sizeof(int));
  upd_cols = (unsigned long long *)take(256);
  CBS_CUDA(cudaMemset(upd_cols, 0, sizeof(unsigned long long)));
  return CBS_OK;
}

template <typename R>
cbs_status MultiShift<R>::update_columns(cudaStream_t st, double *out) {
  unsigned long long v = 0;
  CBS_CUDA(cudaMemcpyAsync(&v, upd_cols, sizeof(v), cudaMemcpyDeviceToHost, st));
  CBS_CUDA(cudaStreamSynchronize(st));
  *out = (double)v;
  return CBS_OK;
}

template <typename R>
void MultiShift<R>::release() {
  seed.release();
  for (int k = 0; k < n_upd_ev; ++k) cudaEventDestroy(upd_ev[k]);
  n_upd_ev = 0;
  if (block) cudaFree(block);
  block = nullptr;
  if (exec) cudaGraphExecDestroy(exec);
  exec = nullptr;
  exec_max_iter = exec_check_every = -1;
}

template <typename R>
void MultiShift<R>::release_x() {
  if (xblock) cudaFree(xblock);
  xblock = nullptr;
  X = nullptr;
}

template <typename R>
cbs_status MultiShift<R>::init(const double2 *z1, double E0, const double *sigma_h, const double2 *B,
                            double tol, cudaStream_t st) {
  std::vector<double> hE(n_pt, E0);
  CBS_CUDA(cudaMemcpyAsync(seed.E, hE.data(), n_pt * sizeof(double), cudaMemcpyHostToDevice, st));
  CBS_TRY_B(seed.set_systems(z1, seed.E, st));   // twists and energies of the seed (and duals)
  CBS_CUDA(cudaMemcpyAsync(sigma, sigma_h, n_sh * sizeof(double), cudaMemcpyHostToDevice, st));
  CBS_CUDA(cudaStreamSynchronize(st));            // hE, sigma_h are host temporaries
  CBS_TRY_B(seed.init(B, 0, B, 0, nullptr, tol, 0.0, st));
  const int64_t n = (int64_t)n_pt * n_sh;
  CBS_CUDA(cudaMemsetAsync(X, 0, 2 * n * N * L * sizeof(C), st));
  CBS_CUDA(cudaMemsetAsync(P, 0, 2 * n * N * L * sizeof(C), st));
  k_ms_init<<<n_pt, L, 0, st>>>(n_pt, n_sh, L, seed.active, pi, pi_prev, alpha_prev, sactive, siters,
                                sflags); cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  return CBS_OK;
}

template <typename R>
cbs_status MultiShift<R>::step(int max_iter, cudaStream_t st, int kk) {
  Bicg<R> &b = seed;
  dim3 blk = col_block(L);
  dim3 grd((unsigned)b.n_chunks, (unsigned)n_pt, 1);
  k_update_p<R><<<grd, blk, 0, st>>>(n_pt, N, L, b.chunk_pts, b.r, b.p, b.beta, b.active, b.sys_active); cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  const bool prof = b.profile && kk >= 0 && 2 * kk + 1 < b.n_prof_ev;
  if (prof) CBS_CUDA(cudaEventRecordWithFlags(b.prof_ev[2 * kk], st, cudaEventRecordExternal));
  cbs_status s = apply_P<R>(b.H, 2 * n_pt, L, b.p, b.q, b.tw, false, b.E, b.D, b.sys_active, st);
  if (s != CBS_OK) return s;
  if (prof) CBS_CUDA(cudaEventRecordWithFlags(b.prof_ev[2 * kk + 1], st, cudaEventRecordExternal));
  k_dot_pq<R><<<grd, blk, red_smem(L), st>>>(n_pt, N, L, b.chunk_pts, b.n_chunks, b.p, b.q, b.part, b.sys_active); cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  k_reduce_alpha<<<n_pt, L, 0, st>>>(n_pt, L, b.n_chunks, b.part, b.rho, b.alpha, b.active, b.flags, b.sys_active,
                                     b.sys_apply); cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  k_ms_coef<<<n_pt, L, 0, st>>>(n_pt, n_sh, L, sigma, b.alpha, b.beta, alpha_prev, pi, pi_prev, cb, ca,
                                sactive, sflags, b.sys_active, b.profile ? upd_cols : nullptr); cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  const bool uprof = b.profile && kk >= 0 && 2 * kk + 1 < n_upd_ev;
  if (uprof) CBS_CUDA(cudaEventRecordWithFlags(upd_ev[2 * kk], st, cudaEventRecordExternal));
  k_ms_update<R><<<grd, blk, 0, st>>>(n_pt, n_sh, N, L, b.chunk_pts, b.r, P, X, cb, ca, sactive, b.sys_active); cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  if (uprof) CBS_CUDA(cudaEventRecordWithFlags(upd_ev[2 * kk + 1], st, cudaEventRecordExternal));
  k_pass_b<R><<<grd, blk, red_smem(L), st>>>(n_pt, N, L, b.chunk_pts, b.n_chunks, nullptr, b.r, b.p, b.q,
                                                  b.alpha, b.active, b.part, b.sys_active); cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  CBS_CUDA(cudaMemsetAsync(b.n_active, 0, sizeof(int), st));
  k_ms_reduce_beta<<<n_pt, L, 0, st>>>(n_pt, n_sh, L, b.n_chunks, b.part, b.rho, b.rho_prev, b.beta, b.tgt, b.tgtd,
                                       b.active, b.iters, b.flags, max_iter, b.sys_active, b.n_active, pi,
                                       sactive, siters, sflags); cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  if (group_need < n_pt) {
    k_ms_group_stop<<<n_sh, ((n_pt + 31) / 32) * 32, 0, st>>>(n_pt, L, group_need, sactive, sflags, siters,
                                                                b.iters);
    cbs::count_launches(1);
    CBS_CUDA(cudaGetLastError());
  }
  return CBS_OK;
}

template <typename R>
cbs_status MultiShift<R>::iterate(int max_iter, int check_every, cudaStream_t st, int *host_iters_done) {
  Bicg<R> &b = seed;
  if (check_every < 1) check_every = 1;
  if (b.profile && b.n_prof_ev == 0) {
    const int ne = 2 * (check_every < 64 ? check_every : 64);
    for (int k = 0; k < ne; ++k) CBS_CUDA(cudaEventCreate(&b.prof_ev[k]));
    b.n_prof_ev = ne;
    for (int k = 0; k < ne; ++k) CBS_CUDA(cudaEventCreate(&upd_ev[k]));
    n_upd_ev = ne;
  }
  if (!b.h_active) CBS_CUDA(cudaMallocHost(&b.h_active, sizeof(int)));
  if (!exec || exec_max_iter != max_iter || exec_check_every != check_every) {
    if (exec) { cudaGraphExecDestroy(exec); exec = nullptr; }
    cudaGraph_t graph = nullptr;
    const uint64_t c0 = thread_launches();
    CBS_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    cbs_status s = CBS_OK;
    for (int k = 0; k < check_every && s == CBS_OK; ++k) s = step(max_iter, st, k);
    cudaError_t ce = cudaStreamEndCapture(st, &graph);
    exec_kernels = thread_launches() - c0;
    uncount_launches(exec_kernels);
    if (s != CBS_OK) { if (graph) cudaGraphDestroy(graph); return s; }
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) { exec = nullptr; return cuda_fail(ce, "cudaGraphInstantiate"); }
    exec_max_iter = max_iter;
    exec_check_every = check_every;
  }
  int done = 0;
  cbs_status s = CBS_OK;
  const int max_replays = max_iter / check_every + 2;
  for (int rep = 0; rep < max_replays; ++rep) {
    cudaError_t ce = cudaGraphLaunch(exec, st);
    count_launches(exec_kernels);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(b.h_active, b.n_active, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) { s = cuda_fail(ce, "shifted-family BiCG graph replay"); break; }
    if (b.profile) {
      for (int k = 0; 2 * k + 1 < b.n_prof_ev && k < check_every; ++k) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, b.prof_ev[2 * k], b.prof_ev[2 * k + 1]) == cudaSuccess) {
          b.prof_ms += ms;
          b.prof_launches += 1;
        } else {
          (void)cudaGetLastError();
        }
        if (2 * k + 1 < n_upd_ev &&
            cudaEventElapsedTime(&ms, upd_ev[2 * k], upd_ev[2 * k + 1]) == cudaSuccess) {
          upd_ms += ms;
          upd_launches += 1;
        } else {
          (void)cudaGetLastError();
        }
      }
    }
    done += check_every;
    if (*b.h_active == 0) break;
  }
  if (host_iters_done) *host_iters_done = done;
  return s;
}

template struct MultiShift<double>;
template struct MultiShift<float>;

// ---------------------------------------------------------------- refinement helpers
// AY holds P(z)Y (primal, systems 0..n-1) and P(z)^dagger Y~ (dual, n..2n-1); replace by
// B - AY and record per-column squared norms.
__global__ void k_residual(int n, int64_t N, int L, const double2 *B, int64_t bstride,
                           const double2 *Bd, int64_t bdstride, double2 *AY, double *colnorm2) {
  const int s2 = blockIdx.y, c = threadIdx.x, ly = threadIdx.y, py = blockDim.y;
  const bool dual = s2 >= n;
  const int s = dual ? s2 - n : s2;
  const double2 *b = dual ? Bd + (int64_t)s * bdstride : B + (int64_t)s * bstride;
  double acc = 0;
  const int64_t per = ((N + gridDim.x - 1) / gridDim.x);
  const int64_t i0 = (int64_t)blockIdx.x * per, i1 = min(N, i0 + per);
  for (int64_t i = i0 + ly; i < i1; i += py) {
    const int64_t e = ((int64_t)s2 * N + i) * L + c;
    double2 v = csub(b[i * L + c], AY[e]);
    AY[e] = v;
    acc += cabs2(v);
  }
  extern __shared__ double red1[];
  red1[ly * L + c] = acc;
  __syncthreads();
  if (ly == 0) {
    double t = 0;
    for (int y = 0; y < py; ++y) t += red1[y * L + c];
    colnorm2[((int64_t)s2 * gridDim.x + blockIdx.x) * L + c] = t;
  }
}

cbs_status launch_residual(int n2, int64_t N, int L, const double2 *B, int64_t bstride,
                           const double2 *Bd, int64_t bdstride, int n, double2 *AY,
                           double *colnorm2, cudaStream_t st) {
  dim3 blk = col_block(L);
  dim3 grd(64, (unsigned)n2, 1);
  k_residual<<<grd, blk, (size_t)blk.x * blk.y * sizeof(double), st>>>(n, N, L, B, bstride, Bd,
                                                                        bdstride, AY, colnorm2); cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  return CBS_OK;
}

__global__ void k_accumulate64(int64_t count, double2 *Y, const double2 *X) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    Y[e] = cadd(Y[e], X[e]);
}

cbs_status launch_accumulate(int64_t count, double2 *Y, const double2 *X, cudaStream_t st) {
  k_accumulate64<<<152 * 8, 256, 0, st>>>(count, Y, X);
  cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  return CBS_OK;
}

__global__ void k_accumulate(int64_t count, double2 *Y, const float2 *X) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    float2 v = X[e];
    double2 y = Y[e];
    Y[e] = make_double2(y.x + (double)v.x, y.y + (double)v.y);
  }
}

cbs_status launch_accumulate(int64_t count, double2 *Y, const float2 *X, cudaStream_t st) {
  k_accumulate<<<152 * 8, 256, 0, st>>>(count, Y, X); cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  return CBS_OK;
}

}  // namespace cbs

namespace cbs {

// colnorm2: [2n][nchunks][L] partial squared norms of the residuals (primal then dual);
// bnorm: [2n][L] right-hand-side norms.  colmask[s][c] = 1 if the column still needs work.
__global__ void k_refine_check(int n, int L, int nchunks, const double *colnorm2, const double *bnorm,
                               double tol, int *colmask, int *n_unconv, double *maxrel) {
  const int s = blockIdx.x, c = threadIdx.x;
  double a = 0, b = 0;
  for (int ch = 0; ch < nchunks; ++ch) {
    a += colnorm2[((int64_t)s * nchunks + ch) * L + c];
    b += colnorm2[((int64_t)(n + s) * nchunks + ch) * L + c];
  }
  const double nb = bnorm[(int64_t)s * L + c], nbd = bnorm[(int64_t)(n + s) * L + c];
  const double rel = nb > 0 ? sqrt(a) / nb : 0.0, reld = nbd > 0 ? sqrt(b) / nbd : 0.0;
  const int need = !(rel <= tol && reld <= tol);
  colmask[(int64_t)s * L + c] = need;
  maxrel[(int64_t)s * L + c] = fmax(rel, reld);
  if (need) atomicAdd(n_unconv, 1);
}

cbs_status launch_refine_check(int n, int L, int nchunks, const double *colnorm2, const double *bnorm,
                               double tol, int *colmask, int *n_unconv, double *maxrel,
                               cudaStream_t st) {
  k_refine_check<<<n, L, 0, st>>>(n, L, nchunks, colnorm2, bnorm, tol, colmask, n_unconv, maxrel); cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  return CBS_OK;
}

}  // namespace cbs
