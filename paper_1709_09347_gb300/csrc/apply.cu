// The QEP matrix applied to blocks of vectors: Y = P(w) X = E X - H(w) X  (Eq. (4)).
//
// H(w) = H0 + w H+ + w^{-1} H- is the cell Hamiltonian with a twisted-periodic boundary
// along z: a finite-difference arm that leaves the cell through the top plane re-enters
// at the bottom multiplied by w, one that leaves through the bottom re-enters at the top
// multiplied by 1/w (Bloch factor of the neighbouring cell, Eq. (3)); x and y are plain
// periodic.  The non-local part is the separable sum over atoms and their copies along
// z, which on cell 0 with Bloch factor w reads
//     H_NL(w) = sum_a F_a(w) h_a F_a(1/w)^T,   F_a(w) = sum_m w^m B_{a,m},
// B_{a,m} the projector values of the copy of atom a displaced by m cells.  It is applied
// in two kernels: a gather D_a = h_a F_a(1/w)^T X (per atom, per column), then a per-point
// scatter-as-gather through the transposed table inside the stencil kernel.
//
// Layout: X, Y are [n_sys][N][L] (columns of a grid point contiguous).  Thread blocks are
// (L, PY): threadIdx.x is the column, threadIdx.y a lane over grid points.
#include "common.cuh"

namespace cbs {

template <typename R> __device__ __forceinline__ const R *vloc_ptr(const HamView &H);
template <> __device__ __forceinline__ const double *vloc_ptr<double>(const HamView &H) { return H.vloc; }
template <> __device__ __forceinline__ const float *vloc_ptr<float>(const HamView &H) { return H.vloc32; }
template <typename R> __device__ __forceinline__ const R *pval_ptr(const HamView &H);
template <> __device__ __forceinline__ const double *pval_ptr<double>(const HamView &H) { return H.sup_val; }
template <> __device__ __forceinline__ const float *pval_ptr<float>(const HamView &H) { return H.sup_val32; }
template <typename R> __device__ __forceinline__ const R *h_ptr(const HamView &H);
template <> __device__ __forceinline__ const double *h_ptr<double>(const HamView &H) { return H.h; }
template <> __device__ __forceinline__ const float *h_ptr<float>(const HamView &H) { return H.h32; }

// D[s][a][mu][c] = sum_nu h_a[mu][nu] sum_{t in a} p_t[nu] w^{-m_t} X[s][i_t][c]
template <typename R, bool PER_COL>
__global__ void k_proj_gather(HamView H, int L, const typename CT<R>::T *__restrict__ X,
                              const double2 *__restrict__ twist,
                              typename CT<R>::T *__restrict__ D, const int *__restrict__ sys_active) {
  typedef typename CT<R>::T C;
  extern __shared__ unsigned char smem_raw[];
  C *red = reinterpret_cast<C *>(smem_raw);  // [PY][n_proj][L]
  const int a = blockIdx.x, s = blockIdx.y;
  const int c = threadIdx.x, ly = threadIdx.y, py = blockDim.y;
  if (sys_active && !sys_active[s]) return;
  const int np = H.n_proj;
  double2 wd = twist[PER_COL ? (int64_t)s * L + c : s];
  double2 wid = cdiv(make_double2(1.0, 0.0), wd);
  C w = from_d<R>(wd), wi = from_d<R>(wid);
  C acc[kMaxProj];
#pragma unroll
  for (int mu = 0; mu < kMaxProj; ++mu) acc[mu] = mk<R>(0, 0);
  const R *pv = pval_ptr<R>(H);
  const int64_t t0 = H.sup_ptr[a], t1 = H.sup_ptr[a + 1];
  const C *Xs = X + (int64_t)s * H.n * L;
  for (int64_t t = t0 + ly; t < t1; t += py) {
    C xv = Xs[(int64_t)H.sup_idx[t] * L + c];
    int m = H.sup_wrap[t];
    C f = (m == 0) ? xv : (m > 0 ? cmul(wi, xv) : cmul(w, xv));   // w^{-m} x
#pragma unroll
    for (int mu = 0; mu < kMaxProj; ++mu)
      if (mu < np) {
        R p = pv[t * np + mu];
        acc[mu].x += p * f.x;
        acc[mu].y += p * f.y;
      }
  }
  for (int mu = 0; mu < np; ++mu) red[((int64_t)ly * np + mu) * L + c] = acc[mu];
  __syncthreads();
  if (ly == 0) {
    C cc[kMaxProj];
    for (int mu = 0; mu < np; ++mu) {
      C sum = mk<R>(0, 0);
      for (int y = 0; y < py; ++y) sum = cadd(sum, red[((int64_t)y * np + mu) * L + c]);
      cc[mu] = sum;
    }
    const R *ha = h_ptr<R>(H) + (int64_t)a * np * np;
    for (int mu = 0; mu < np; ++mu) {
      C d = mk<R>(0, 0);
      for (int nu = 0; nu < np; ++nu) {
        R hv = ha[mu * np + nu];
        d.x += hv * cc[nu].x;
        d.y += hv * cc[nu].y;
      }
      D[(((int64_t)s * H.n_atoms + a) * np + mu) * L + c] = d;
    }
  }
}

__device__ __forceinline__ int wrap_plus(int i, int k, int n) {
  int j = i + k;
  if (j >= n) j -= n;
  if (j >= n) j %= n;
  return j;
}
__device__ __forceinline__ int wrap_minus(int i, int k, int n) {
  int j = i - k;
  if (j < 0) j += n;
  if (j < 0) j = ((j % n) + n) % n;
  return j;
}

constexpr int kApplyPPT = 4;  // grid points per thread

template <typename R, bool PER_COL>
__global__ void k_apply(HamView H, int L, const typename CT<R>::T *__restrict__ X,
                        typename CT<R>::T *__restrict__ Y, const double2 *__restrict__ twist,
                        const double *__restrict__ E, const typename CT<R>::T *__restrict__ D,
                        const int *__restrict__ sys_active) {
  typedef typename CT<R>::T C;
  const int s = blockIdx.y;
  if (sys_active && !sys_active[s]) return;
  const int c = threadIdx.x, ly = threadIdx.y, py = blockDim.y;
  double2 wd = twist[PER_COL ? (int64_t)s * L + c : s];
  double2 wid = cdiv(make_double2(1.0, 0.0), wd);
  const C w = from_d<R>(wd), wi = from_d<R>(wid);
  const R e = (R)E[s];
  const R dk = (R)H.diag_kin;
  R wx[kMaxHalf + 1], wy[kMaxHalf + 1], wz[kMaxHalf + 1];
#pragma unroll
  for (int k = 1; k <= kMaxHalf; ++k) { wx[k] = (R)H.wx[k]; wy[k] = (R)H.wy[k]; wz[k] = (R)H.wz[k]; }
  const R *vl = vloc_ptr<R>(H);
  const R *pv = pval_ptr<R>(H);
  const int np = H.n_proj;
  const int64_t nxy = (int64_t)H.nx * H.ny;
  const C *Xs = X + (int64_t)s * H.n * L;
  C *Ys = Y + (int64_t)s * H.n * L;
  const int64_t base = (int64_t)blockIdx.x * py * kApplyPPT;
  for (int k0 = 0; k0 < kApplyPPT; ++k0) {
    const int64_t i = base + (int64_t)k0 * py + ly;
    if (i >= H.n) break;
    const int ix = (int)(i % H.nx);
    const int iy = (int)((i / H.nx) % H.ny);
    const int iz = (int)(i / nxy);
    const C x0 = Xs[i * L + c];
    const R d = dk + vl[i];
    C acc = mk<R>(d * x0.x, d * x0.y);
    C top = mk<R>(0, 0), bot = mk<R>(0, 0);
    const int64_t rowx = i - ix, rowy = i - (int64_t)iy * H.nx;
#pragma unroll
    for (int k = 1; k <= kMaxHalf; ++k) {
      if (k > H.m) break;
      C a1 = Xs[(rowx + wrap_plus(ix, k, H.nx)) * L + c];
      C a2 = Xs[(rowx + wrap_minus(ix, k, H.nx)) * L + c];
      acc.x += wx[k] * (a1.x + a2.x);
      acc.y += wx[k] * (a1.y + a2.y);
      C b1 = Xs[(rowy + (int64_t)wrap_plus(iy, k, H.ny) * H.nx) * L + c];
      C b2 = Xs[(rowy + (int64_t)wrap_minus(iy, k, H.ny) * H.nx) * L + c];
      acc.x += wy[k] * (b1.x + b2.x);
      acc.y += wy[k] * (b1.y + b2.y);
      int zu = iz + k, zd = iz - k;
      if (zu < H.nz) {
        C u = Xs[(i + k * nxy) * L + c];
        acc.x += wz[k] * u.x; acc.y += wz[k] * u.y;
      } else {
        C u = Xs[(i + (int64_t)(k - H.nz) * nxy) * L + c];
        top.x += wz[k] * u.x; top.y += wz[k] * u.y;
      }
      if (zd >= 0) {
        C u = Xs[(i - k * nxy) * L + c];
        acc.x += wz[k] * u.x; acc.y += wz[k] * u.y;
      } else {
        C u = Xs[(i + (int64_t)(H.nz - k) * nxy) * L + c];
        bot.x += wz[k] * u.x; bot.y += wz[k] * u.y;
      }
    }
    acc = cfma(w, top, acc);
    acc = cfma(wi, bot, acc);
    if (D) {
      const int64_t e0 = H.pt_ptr[i], e1 = H.pt_ptr[i + 1];
      for (int64_t q = e0; q < e1; ++q) {
        const int t = H.pt_ent[q], a = H.pt_atom[q];
        const C *Da = D + (((int64_t)s * H.n_atoms + a) * np) * L + c;
        C v = mk<R>(0, 0);
        for (int mu = 0; mu < np; ++mu) {
          R p = pv[(int64_t)t * np + mu];
          C dv = Da[(int64_t)mu * L];
          v.x += p * dv.x;
          v.y += p * dv.y;
        }
        int m = H.sup_wrap[t];
        if (m == 0) acc = cadd(acc, v);
        else acc = cfma(m > 0 ? w : wi, v, acc);                      // w^{m} v
      }
    }
    Ys[i * L + c] = mk<R>(e * x0.x - acc.x, e * x0.y - acc.y);
  }
}

template <typename R>
cbs_status launch_proj_gather(const HamView &H, int n_sys, int L, const typename CT<R>::T *X,
                              const double2 *twist, bool per_col, typename CT<R>::T *D,
                              const int *sys_active, cudaStream_t st) {
  if (H.n_atoms == 0) return CBS_OK;
  dim3 blk = col_block(L);
  dim3 grd((unsigned)H.n_atoms, (unsigned)n_sys, 1);
  size_t sm = (size_t)blk.y * H.n_proj * L * sizeof(typename CT<R>::T);
  if (sm > 48 * 1024) {
    set_error("projector gather: shared memory per block exceeds 48 KB (reduce L)");
    return CBS_EINVAL;
  }
  if (per_col)
    k_proj_gather<R, true><<<grd, blk, sm, st>>>(H, L, X, twist, D, sys_active);
  else
    k_proj_gather<R, false><<<grd, blk, sm, st>>>(H, L, X, twist, D, sys_active);
  CBS_CUDA(cudaGetLastError());
  return CBS_OK;
}

template <typename R>
cbs_status launch_apply(const HamView &H, int n_sys, int L, const typename CT<R>::T *X,
                        typename CT<R>::T *Y, const double2 *twist, bool per_col,
                        const double *E, const typename CT<R>::T *D, const int *sys_active,
                        cudaStream_t st) {
  dim3 blk = col_block(L);
  dim3 grd((unsigned)ceil_div(H.n, (int64_t)blk.y * kApplyPPT), (unsigned)n_sys, 1);
  const typename CT<R>::T *Dp = H.n_atoms ? D : nullptr;
  if (per_col)
    k_apply<R, true><<<grd, blk, 0, st>>>(H, L, X, Y, twist, E, Dp, sys_active);
  else
    k_apply<R, false><<<grd, blk, 0, st>>>(H, L, X, Y, twist, E, Dp, sys_active);
  CBS_CUDA(cudaGetLastError());
  return CBS_OK;
}

template <typename R>
cbs_status apply_P(const HamView &H, int n_sys, int L, const typename CT<R>::T *X,
                   typename CT<R>::T *Y, const double2 *twist, bool per_col, const double *E,
                   typename CT<R>::T *D, const int *sys_active, cudaStream_t st) {
  cbs_status s = launch_proj_gather<R>(H, n_sys, L, X, twist, per_col, D, sys_active, st);
  if (s != CBS_OK) return s;
  return launch_apply<R>(H, n_sys, L, X, Y, twist, per_col, E, D, sys_active, st);
}

template cbs_status apply_P<double>(const HamView &, int, int, const double2 *, double2 *,
                                    const double2 *, bool, const double *, double2 *,
                                    const int *, cudaStream_t);
template cbs_status apply_P<float>(const HamView &, int, int, const float2 *, float2 *,
                                   const double2 *, bool, const double *, float2 *,
                                   const int *, cudaStream_t);
template cbs_status launch_proj_gather<double>(const HamView &, int, int, const double2 *,
                                               const double2 *, bool, double2 *, const int *,
                                               cudaStream_t);
template cbs_status launch_proj_gather<float>(const HamView &, int, int, const float2 *,
                                              const double2 *, bool, float2 *, const int *,
                                              cudaStream_t);
template cbs_status launch_apply<double>(const HamView &, int, int, const double2 *, double2 *,
                                         const double2 *, bool, const double *,
                                         const double2 *, const int *, cudaStream_t);
template cbs_status launch_apply<float>(const HamView &, int, int, const float2 *, float2 *,
                                        const double2 *, bool, const double *, const float2 *,
                                        const int *, cudaStream_t);

}  // namespace cbs
