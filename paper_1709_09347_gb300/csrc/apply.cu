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
// (L, PY): threadIdx.x is the column; threadIdx.y a lane over support entries (gather)
// or over x (stencil, one block per (x-chunk, y, system), marching along z).
#include "common.cuh"

namespace cbs {

// A system's twist w and its inverse in the working precision.  In complex64 the inverse is
// formed in FP32 from the rounded twist: a complex double division costs ~20 FP64
// instructions per thread, which on this part's narrow FP64 pipe was a visible share of a
// complex64 launch.
__device__ __forceinline__ void twist_pair(double2 wd, double2 &w, double2 &wi) {
  w = wd;
  wi = cdiv(make_double2(1.0, 0.0), wd);
}
__device__ __forceinline__ void twist_pair(double2 wd, float2 &w, float2 &wi) {
  w = make_float2((float)wd.x, (float)wd.y);
  const float r = 1.0f / (w.x * w.x + w.y * w.y);
  wi = make_float2(w.x * r, -w.y * r);
}

__device__ __forceinline__ float4 c2mul(float2 w0, float2 w1, float4 v) {
  const float2 a = cmul(w0, make_float2(v.x, v.y)), b = cmul(w1, make_float2(v.z, v.w));
  return make_float4(a.x, a.y, b.x, b.y);
}

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
template <typename R, bool PER_COL, int NPM>
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
  C w, wi;
  twist_pair(twist[PER_COL ? (int64_t)s * L + c : s], w, wi);
  // one accumulator set per image shift m = 0, +1, -1: the twist w^{-m} is applied once
  // per column at the end instead of once per support entry
  C acc[NPM], accp[NPM], accm[NPM];
#pragma unroll
  for (int mu = 0; mu < NPM; ++mu) acc[mu] = accp[mu] = accm[mu] = mk<R>(0, 0);
  const R *pv = pval_ptr<R>(H);
  const int64_t t0 = H.sup_ptr[a], t1 = H.sup_ptr[a + 1];
  const C *Xs = X + (int64_t)s * H.n * L;
  // four independent support entries per step keep several gathers in flight
  constexpr int U = 4;
  for (int64_t tb = t0 + ly; tb < t1; tb += (int64_t)U * py) {
    C xv[U];
    int mw[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t t = tb + (int64_t)u * py;
      if (t < t1) {
        xv[u] = Xs[(int64_t)H.sup_idx[t] * L + c];
        mw[u] = H.sup_wrap[t];
      } else {
        xv[u] = mk<R>(0, 0);
        mw[u] = 0;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t t = tb + (int64_t)u * py;
      if (t >= t1) break;
      const C f = xv[u];
      if (mw[u] == 0) {
#pragma unroll
        for (int mu = 0; mu < NPM; ++mu)
          if (mu < np) {
            const R p = pv[t * np + mu];
            acc[mu].x = fma(p, f.x, acc[mu].x);
            acc[mu].y = fma(p, f.y, acc[mu].y);
          }
      } else if (mw[u] > 0) {
#pragma unroll
        for (int mu = 0; mu < NPM; ++mu)
          if (mu < np) {
            const R p = pv[t * np + mu];
            accp[mu].x = fma(p, f.x, accp[mu].x);
            accp[mu].y = fma(p, f.y, accp[mu].y);
          }
      } else {
#pragma unroll
        for (int mu = 0; mu < NPM; ++mu)
          if (mu < np) {
            const R p = pv[t * np + mu];
            accm[mu].x = fma(p, f.x, accm[mu].x);
            accm[mu].y = fma(p, f.y, accm[mu].y);
          }
      }
    }
  }
#pragma unroll
  for (int mu = 0; mu < NPM; ++mu)                      // w^{-m} for m = +1, -1
    acc[mu] = cadd(acc[mu], cadd(cmul(wi, accp[mu]), cmul(w, accm[mu])));
#pragma unroll
  for (int mu = 0; mu < NPM; ++mu)
    if (mu < np) red[((int64_t)ly * np + mu) * L + c] = acc[mu];
  __syncthreads();
  if (ly == 0) {
    C cc[NPM];
#pragma unroll
    for (int mu = 0; mu < NPM; ++mu) {
      C sum = mk<R>(0, 0);
      if (mu < np)
        for (int y = 0; y < py; ++y) sum = cadd(sum, red[((int64_t)y * np + mu) * L + c]);
      cc[mu] = sum;
    }
    const R *ha = h_ptr<R>(H) + (int64_t)a * np * np;
#pragma unroll
    for (int mu = 0; mu < NPM; ++mu) {
      if (mu >= np) break;
      C d = mk<R>(0, 0);
#pragma unroll
      for (int nu = 0; nu < NPM; ++nu)
        if (nu < np) {
          R hv = ha[mu * np + nu];
          d.x += hv * cc[nu].x;
          d.y += hv * cc[nu].y;
        }
      D[(((int64_t)s * H.n_atoms + a) * L + c) * H.np4 + mu] = d;
    }
    for (int mu = np; mu < H.np4; ++mu) D[(((int64_t)s * H.n_atoms + a) * L + c) * H.np4 + mu] = mk<R>(0, 0);
  }
}

// Complex64 gather with two columns per thread (16-byte loads):
// D[s][a][c][4] = h_a sum_{t in a} p_t w^{-m_t} X[s][i_t][c], for n_proj <= 4.
template <bool PER_COL>
__global__ void k_proj_gather_c64x2(HamView H, int L, const float4 *__restrict__ X,
                                    const double2 *__restrict__ twist, float2 *__restrict__ D,
                                    const int *__restrict__ sys_active) {
  extern __shared__ float4 red4[];   // [py][4 projectors][L/2] pairs of complex
  const int a = blockIdx.x, s = blockIdx.y;
  const int t = threadIdx.x, ly = threadIdx.y, py = blockDim.y;
  const int L2 = L >> 1;
  if (sys_active && !sys_active[s]) return;
  const double2 wd0 = twist[PER_COL ? (int64_t)s * L + 2 * t : s];
  const double2 wd1 = twist[PER_COL ? (int64_t)s * L + 2 * t + 1 : s];
  float2 w0, w1, wi0, wi1;
  twist_pair(wd0, w0, wi0);
  twist_pair(wd1, w1, wi1);
  float4 acc[4];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) acc[mu] = make_float4(0, 0, 0, 0);
  const int np = H.n_proj;
  const float *pv = H.sup_val32;
  const int64_t t0 = H.sup_ptr[a], t1 = H.sup_ptr[a + 1];
  const float4 *Xs = X + (int64_t)s * H.n * L2;
  constexpr int U = 4;
  for (int64_t tb = t0 + ly; tb < t1; tb += (int64_t)U * py) {
    float4 xv[U];
    int mw[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t tt = tb + (int64_t)u * py;
      if (tt < t1) {
        xv[u] = Xs[(int64_t)H.sup_idx[tt] * L2 + t];
        mw[u] = H.sup_wrap[tt];
      } else {
        xv[u] = make_float4(0, 0, 0, 0);
        mw[u] = 0;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t tt = tb + (int64_t)u * py;
      if (tt >= t1) break;
      float4 f = xv[u];
      if (mw[u] > 0) f = c2mul(wi0, wi1, f);       // w^{-m} x
      else if (mw[u] < 0) f = c2mul(w0, w1, f);
#pragma unroll
      for (int mu = 0; mu < 4; ++mu)
        if (mu < np) {
          const float p = pv[tt * np + mu];
          acc[mu].x += p * f.x; acc[mu].y += p * f.y; acc[mu].z += p * f.z; acc[mu].w += p * f.w;
        }
    }
  }
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) red4[((int64_t)ly * 4 + mu) * L2 + t] = acc[mu];
  __syncthreads();
  if (ly == 0) {
    float4 cc[4];
    for (int mu = 0; mu < 4; ++mu) {
      float4 sum = make_float4(0, 0, 0, 0);
      for (int y = 0; y < py; ++y) {
        const float4 v = red4[((int64_t)y * 4 + mu) * L2 + t];
        sum.x += v.x; sum.y += v.y; sum.z += v.z; sum.w += v.w;
      }
      cc[mu] = sum;
    }
    const float *ha = H.h32 + (int64_t)a * np * np;
    float2 *Da = D + (((int64_t)s * H.n_atoms + a) * L + 2 * t) * 4;   // columns 2t, 2t+1
    for (int mu = 0; mu < 4; ++mu) {
      float4 d = make_float4(0, 0, 0, 0);
      if (mu < np)
        for (int nu = 0; nu < np; ++nu) {
          const float hv = ha[mu * np + nu];
          d.x += hv * cc[nu].x; d.y += hv * cc[nu].y; d.z += hv * cc[nu].z; d.w += hv * cc[nu].w;
        }
      Da[mu] = make_float2(d.x, d.y);
      Da[4 + mu] = make_float2(d.z, d.w);
    }
  }
}

__device__ __forceinline__ int wrap_idx(int j, int n) {
  // j in (-n*kMaxHalf, n*(kMaxHalf+1)): fold into [0, n)
  while (j >= n) j -= n;
  while (j < 0) j += n;
  return j;
}

// z-marching stencil: a thread owns one column c of one (x, y) grid line and walks the
// planes iz = 0..nz-1, keeping the 2*MH+1 planes around iz in registers.  The register
// queue holds the Bloch-extended field psi(p) = w^{floor(p/nz)} X[p mod nz] (Eq. (3)), so
// the twist of arms that cross the cell faces along z is applied once when a plane
// enters the queue.  x and y arms are plain periodic and read through L1/L2 with
// neighbour offsets precomputed once per thread.  Indices inside one system are 32-bit.
template <typename R, bool PER_COL, int MH>
__global__ void __launch_bounds__(256) k_apply_zm(HamView H, int L, const typename CT<R>::T *__restrict__ X,
                                                  typename CT<R>::T *__restrict__ Y,
                                                  const double2 *__restrict__ twist,
                                                  const double *__restrict__ E,
                                                  const typename CT<R>::T *__restrict__ D,
                                                  const int *__restrict__ sys_active) {
  typedef typename CT<R>::T C;
  const int s = blockIdx.z;
  if (sys_active && !sys_active[s]) return;
  const int c = threadIdx.x;
  const int ix = blockIdx.x * blockDim.y + threadIdx.y;
  const int iy = blockIdx.y * blockDim.z + threadIdx.z;   // a block covers blockDim.z rows
  if (ix >= H.nx || iy >= H.ny) return;
  const int nx = H.nx, ny = H.ny, nz = H.nz;
  const int nxy = nx * ny;
  C w, wi;
  twist_pair(twist[PER_COL ? (int64_t)s * L + c : s], w, wi);
  const R ed = (R)(E[s] - H.diag_kin);
  R nwx[MH + 1], nwy[MH + 1], nwz[MH + 1];
  int ox_p[MH + 1], ox_m[MH + 1], oy_p[MH + 1], oy_m[MH + 1];
#pragma unroll
  for (int k = 1; k <= MH; ++k) {
    nwx[k] = (R)-H.wx[k]; nwy[k] = (R)-H.wy[k]; nwz[k] = (R)-H.wz[k];
    ox_p[k] = (wrap_idx(ix + k, nx) - ix) * L;
    ox_m[k] = (wrap_idx(ix - k, nx) - ix) * L;
    oy_p[k] = (wrap_idx(iy + k, ny) - iy) * nx * L;
    oy_m[k] = (wrap_idx(iy - k, ny) - iy) * nx * L;
  }
  const R *vl = vloc_ptr<R>(H);
  const R *pv = pval_ptr<R>(H);
  const int np = H.n_proj;
  const C *Xs = X + (int64_t)s * H.n * L;
  C *Ys = Y + (int64_t)s * H.n * L;
  const int line = iy * nx + ix;           // (x, y) offset inside a plane
  // psi(p) for p in [-nz, 2 nz)
  auto bloch = [&](int p) -> C {
    if (p >= nz) return cmul(w, Xs[((p - nz) * nxy + line) * L + c]);
    if (p < 0) return cmul(wi, Xs[((p + nz) * nxy + line) * L + c]);
    return Xs[(p * nxy + line) * L + c];
  };
  C q[2 * MH + 1];
#pragma unroll
  for (int d = 0; d < 2 * MH; ++d) q[d] = bloch(d - MH);
  for (int iz = 0; iz < nz; ++iz) {
    const int pt = iz * nxy + line;
    int e0 = 0, e1 = 0;
    if (D) { e0 = (int)H.pt_ptr[pt]; e1 = (int)H.pt_ptr[pt + 1]; }   // issued early
    q[2 * MH] = bloch(iz + MH);
    const int b = pt * L + c;
    const C x0 = q[MH];
    // Y = (E - d_i) x0 - sum_k w_k (pair sums) - projector part, accumulated with one
    // FMA per pair and component (the FP64 form is bound by FP64 instruction issue)
    const R dd = ed - vl[pt];
    C acc = mk<R>(dd * x0.x, dd * x0.y);
#pragma unroll
    for (int k = 1; k <= MH; ++k) {
      const C a1 = Xs[b + ox_p[k]], a2 = Xs[b + ox_m[k]];
      const C b1 = Xs[b + oy_p[k]], b2 = Xs[b + oy_m[k]];
      const C z1 = q[MH + k], z2 = q[MH - k];
      acc.x = fma(nwx[k], a1.x + a2.x, acc.x);
      acc.y = fma(nwx[k], a1.y + a2.y, acc.y);
      acc.x = fma(nwy[k], b1.x + b2.x, acc.x);
      acc.y = fma(nwy[k], b1.y + b2.y, acc.y);
      acc.x = fma(nwz[k], z1.x + z2.x, acc.x);
      acc.y = fma(nwz[k], z1.y + z2.y, acc.y);
    }
    if (D) {
      for (int qq = e0; qq < e1; ++qq) {
        const int t = H.pt_ent[qq], a = H.pt_atom[qq];
        const C *Da = D + (((int64_t)s * H.n_atoms + a) * L + c) * H.np4;
        const int m = H.sup_wrap[t];
        if (m == 0) {
          for (int mu = 0; mu < np; ++mu) {
            const R p = -pv[t * np + mu];
            const C dv = Da[mu];
            acc.x = fma(p, dv.x, acc.x);
            acc.y = fma(p, dv.y, acc.y);
          }
        } else {
          C v = mk<R>(0, 0);
          for (int mu = 0; mu < np; ++mu) {
            const R p = pv[t * np + mu];
            const C dv = Da[mu];
            v.x = fma(p, dv.x, v.x);
            v.y = fma(p, dv.y, v.y);
          }
          const C tw = m > 0 ? w : wi;                                  // w^{m} v
          acc = cfma(mk<R>(-tw.x, -tw.y), v, acc);
        }
      }
    }
    Ys[b] = acc;
#pragma unroll
    for (int d = 0; d < 2 * MH; ++d) q[d] = q[d + 1];
  }
}

// Asynchronous 16-byte global -> shared copies (cp.async, bypassing L1), used to keep
// several planes of X in flight per thread.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Planes of X a thread of the complex64 stencil keeps in flight ahead of the one it needs
// (blocks of up to 256 threads; blocks of up to 512 threads keep 2).
constexpr int kApplyPF = 6;
constexpr int kApplyPFBig = 2;

// Complex64 fast path: each thread owns two adjacent columns of one (x, y) line, so every
// load and store is 16 bytes; z arms from the register queue of Bloch-extended values, fed
// from a per-thread ring of kApplyPF planes in shared memory filled by cp.async; the
// projector scatter reads one packed (atom, wrap) word, one float4 of projector values and
// 64 bytes of D per covering entry (D laid out [system][atom][column][4]).  The point's
// scatter-table range and local potential are loaded one plane ahead.  BIG: blocks of up to
// 512 threads (a larger x-y footprint per block, so more of the neighbour loads hit in L1).
template <bool PER_COL, int MH, bool BIG>
__global__ void __launch_bounds__(BIG ? 512 : 256, BIG ? 1 : 2) k_apply_c64x2(HamView H, int L, const float4 *__restrict__ X,
                                                        float4 *__restrict__ Y,
                                                        const double2 *__restrict__ twist,
                                                        const double *__restrict__ E,
                                                        const float4 *__restrict__ D,
                                                        const int *__restrict__ sys_active) {
  constexpr int PF = BIG ? kApplyPFBig : kApplyPF;
  extern __shared__ float4 pf_ring[];   // [PF][threads of the block]
  const int s = blockIdx.z;
  if (sys_active && !sys_active[s]) return;
  const int t = threadIdx.x;                 // column pair
  const int L2 = L >> 1;
  const int ix = blockIdx.x * blockDim.y + threadIdx.y;
  const int iy = blockIdx.y * blockDim.z + threadIdx.z;   // a block covers blockDim.z rows
  if (ix >= H.nx || iy >= H.ny) return;
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nth = blockDim.x * blockDim.y * blockDim.z;
  const int nx = H.nx, ny = H.ny, nz = H.nz, nxy = nx * ny;
  const double2 wd0 = twist[PER_COL ? (int64_t)s * L + 2 * t : s];
  const double2 wd1 = twist[PER_COL ? (int64_t)s * L + 2 * t + 1 : s];
  float2 w0, w1, wi0, wi1;
  twist_pair(wd0, w0, wi0);
  twist_pair(wd1, w1, wi1);
  const float e = (float)E[s];
  const float dk = H.diag_kin32;
  // neighbour offsets in float4 units (x and y periodic); recomputed, not kept in registers
  auto oxp = [&](int k) { return (ix + k < nx ? k : k - nx) * L2; };
  auto oxm = [&](int k) { return (ix - k >= 0 ? -k : nx - k) * L2; };
  auto oyp = [&](int k) { return (iy + k < ny ? k : k - ny) * nx * L2; };
  auto oym = [&](int k) { return (iy - k >= 0 ? -k : ny - k) * nx * L2; };
  const float *vl = H.vloc32;
  const float4 *Xs = X + (int64_t)s * H.n * L2;
  float4 *Ys = Y + (int64_t)s * H.n * L2;
  const float4 *Ds = D + (int64_t)s * H.n_atoms * L * 2 + 4 * t;   // column pair 2t, 2t+1
  const int line = iy * nx + ix;
  // address of this thread's value in plane p of the Bloch-extended field, p in [-nz, 2nz)
  auto src = [&](int p) -> const float4 * {
    const int pw = p >= nz ? p - nz : (p < 0 ? p + nz : p);
    return Xs + (pw * nxy + line) * L2 + t;
  };
  auto bloch = [&](int p) -> float4 {
    const float4 v = *src(p);
    if (p >= nz) return c2mul(w0, w1, v);
    if (p < 0) return c2mul(wi0, wi1, v);
    return v;
  };
  // planes MH .. nz-1+MH enter the queue head one per step; the ring holds the next
  // PF of them (one commit group per plane, empty groups past the last plane)
  const int last = nz - 1 + MH;
#pragma unroll
  for (int k = 0; k < PF; ++k) {
    if (MH + k <= last) cp_async16(&pf_ring[k * nth + tid], src(MH + k));
    cp_async_commit();
  }
  float4 q[2 * MH + 1];
#pragma unroll
  for (int d = 0; d < 2 * MH; ++d) q[d] = bloch(d - MH);
  int e0 = 0, e1 = 0;
  if (D) { e0 = (int)H.pt_ptr[line]; e1 = (int)H.pt_ptr[line + 1]; }
  float vnext = vl[line];
  int slot = 0;
  for (int iz = 0; iz < nz; ++iz) {
    const int pt = iz * nxy + line;
    const int ce0 = e0, ce1 = e1;
    const float vcur = vnext;
    if (iz + 1 < nz) {                       // next plane's table range and potential
      if (D) { e0 = (int)H.pt_ptr[pt + nxy]; e1 = (int)H.pt_ptr[pt + nxy + 1]; }
      vnext = vl[pt + nxy];
    }
    cp_async_wait<PF - 1>();           // plane iz + MH has landed in `slot`
    {
      const float4 v = pf_ring[slot * nth + tid];
      q[2 * MH] = iz + MH >= nz ? c2mul(w0, w1, v) : v;
    }
    const int b = pt * L2 + t;
    const float4 x0 = q[MH];
    const float dd = dk + vcur;
    float4 acc = make_float4(dd * x0.x, dd * x0.y, dd * x0.z, dd * x0.w);
#pragma unroll
    for (int k = 1; k <= MH; ++k) {
      const float4 a1 = Xs[b + oxp(k)], a2 = Xs[b + oxm(k)];
      const float4 b1 = Xs[b + oyp(k)], b2 = Xs[b + oym(k)];
      const float4 z1 = q[MH + k], z2 = q[MH - k];
      const float wx = H.w32[0][k], wy = H.w32[1][k], wz = H.w32[2][k];
      acc.x += wx * (a1.x + a2.x) + wy * (b1.x + b2.x) + wz * (z1.x + z2.x);
      acc.y += wx * (a1.y + a2.y) + wy * (b1.y + b2.y) + wz * (z1.y + z2.y);
      acc.z += wx * (a1.z + a2.z) + wy * (b1.z + b2.z) + wz * (z1.z + z2.z);
      acc.w += wx * (a1.w + a2.w) + wy * (b1.w + b2.w) + wz * (z1.w + z2.w);
    }
    // the queue head has been consumed: refill its slot with plane iz + MH + PF
    if (iz + MH + PF <= last) cp_async16(&pf_ring[slot * nth + tid], src(iz + MH + PF));
    cp_async_commit();
    slot = slot + 1 == PF ? 0 : slot + 1;
    for (int qq = ce0; qq < ce1; ++qq) {
      const int2 aw = H.pt_aw[qq];
      const float4 p = H.pt_p32[qq];
      const float4 *Da = Ds + (int64_t)aw.x * L * 2;
      const float4 d0 = Da[0], d1 = Da[1], d2 = Da[2], d3 = Da[3];
      float4 v;
      v.x = p.x * d0.x + p.y * d0.z + p.z * d1.x + p.w * d1.z;
      v.y = p.x * d0.y + p.y * d0.w + p.z * d1.y + p.w * d1.w;
      v.z = p.x * d2.x + p.y * d2.z + p.z * d3.x + p.w * d3.z;
      v.w = p.x * d2.y + p.y * d2.w + p.z * d3.y + p.w * d3.w;
      if (aw.y > 0) v = c2mul(w0, w1, v);            // w^{m} v
      else if (aw.y < 0) v = c2mul(wi0, wi1, v);
      acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
    }
    Ys[b] = make_float4(e * x0.x - acc.x, e * x0.y - acc.y, e * x0.z - acc.z, e * x0.w - acc.w);
#pragma unroll
    for (int d = 0; d < 2 * MH; ++d) q[d] = q[d + 1];
  }
  cp_async_wait<0>();
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
  if (sizeof(typename CT<R>::T) == sizeof(float2) && L % 2 == 0 && L <= 512 && H.np4 == 4) {
    const int L2 = L / 2;
    int py = 256 / L2;
    if (py < 1) py = 1;
    dim3 b2((unsigned)L2, (unsigned)py, 1);
    const size_t sm2 = (size_t)py * 4 * L2 * sizeof(float4);
    const float4 *X4 = reinterpret_cast<const float4 *>(X);
    float2 *D2 = reinterpret_cast<float2 *>(D);
    if (per_col) k_proj_gather_c64x2<true><<<grd, b2, sm2, st>>>(H, L, X4, twist, D2, sys_active);
    else k_proj_gather_c64x2<false><<<grd, b2, sm2, st>>>(H, L, X4, twist, D2, sys_active);
    cbs::count_launches(1);
    CBS_CUDA(cudaGetLastError());
    return CBS_OK;
  }
  if (H.n_proj <= 4) {
    if (per_col) k_proj_gather<R, true, 4><<<grd, blk, sm, st>>>(H, L, X, twist, D, sys_active);
    else k_proj_gather<R, false, 4><<<grd, blk, sm, st>>>(H, L, X, twist, D, sys_active);
  } else {
    if (per_col) k_proj_gather<R, true, kMaxProj><<<grd, blk, sm, st>>>(H, L, X, twist, D, sys_active);
    else k_proj_gather<R, false, kMaxProj><<<grd, blk, sm, st>>>(H, L, X, twist, D, sys_active);
  }
  cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  return CBS_OK;
}

template <typename R>
cbs_status launch_apply(const HamView &H, int n_sys, int L, const typename CT<R>::T *X,
                        typename CT<R>::T *Y, const double2 *twist, bool per_col,
                        const double *E, const typename CT<R>::T *D, const int *sys_active,
                        cudaStream_t st) {
  if ((int64_t)H.n * L >= ((int64_t)1 << 31)) {
    set_error("apply: N*L must be below 2^31");
    return CBS_EINVAL;
  }
  const typename CT<R>::T *Dp = H.n_atoms ? D : nullptr;
  const int ti = sizeof(typename CT<R>::T) == sizeof(float2) ? 1 : 0;
  // complex64 with an even number of columns and at most 4 projectors: two columns per
  // thread (the only complex64 kernel that takes more than 256 columns)
  if (ti == 1 && L % 2 == 0 && L <= 512 && H.np4 == 4 && (H.tune_x2 >= 0 || L > 256)) {
    const int L2 = L / 2;
    int py = 256 / L2, pz = 1;
    if (H.tune_py[1] > 0 && H.tune_pz[1] > 0 && H.tune_py[1] * H.tune_pz[1] * L2 <= 512) {
      py = H.tune_py[1];
      pz = H.tune_pz[1];
    }
    if (py < 1) py = 1;
    dim3 blk((unsigned)L2, (unsigned)py, (unsigned)pz);
    const bool big = blk.x * blk.y * blk.z > 256;
    dim3 grd((unsigned)ceil_div(H.nx, py), (unsigned)ceil_div(H.ny, pz), (unsigned)n_sys);
    const float4 *X4 = reinterpret_cast<const float4 *>(X);
    float4 *Y4 = reinterpret_cast<float4 *>(Y);
    const float4 *D4 = H.n_atoms ? reinterpret_cast<const float4 *>(D) : nullptr;
    const size_t pf_smem = (size_t)(big ? kApplyPFBig : kApplyPF) * blk.x * blk.y * blk.z * sizeof(float4);
#define FX(MH)                                                                                     \
  do {                                                                                             \
    if (big) {                                                                                     \
      if (per_col) k_apply_c64x2<true, MH, true><<<grd, blk, pf_smem, st>>>(H, L, X4, Y4, twist, E, D4, sys_active); \
      else k_apply_c64x2<false, MH, true><<<grd, blk, pf_smem, st>>>(H, L, X4, Y4, twist, E, D4, sys_active);    \
    } else {                                                                                       \
      if (per_col) k_apply_c64x2<true, MH, false><<<grd, blk, pf_smem, st>>>(H, L, X4, Y4, twist, E, D4, sys_active); \
      else k_apply_c64x2<false, MH, false><<<grd, blk, pf_smem, st>>>(H, L, X4, Y4, twist, E, D4, sys_active);    \
    }                                                                                              \
    cbs::count_launches(1);                                                                        \
  } while (0)
    switch (H.m) {
      case 1: FX(1); break;
      case 2: FX(2); break;
      case 3: FX(3); break;
      case 4: FX(4); break;
      case 5: FX(5); break;
      case 6: FX(6); break;
      default: set_error("apply: FD half-width must be 1..6"); return CBS_EINVAL;
    }
#undef FX
    CBS_CUDA(cudaGetLastError());
    return CBS_OK;
  }
  dim3 blk = col_block(L);
  if (H.tune_py[ti] > 0 && H.tune_pz[ti] > 0 && H.tune_py[ti] * H.tune_pz[ti] * L <= 256) {
    blk.y = (unsigned)H.tune_py[ti];
    blk.z = (unsigned)H.tune_pz[ti];
  }
  if (blk.x * blk.y * blk.z > 256) {
    set_error("apply: at most 256 columns per system (512 in complex64 with even L)");
    return CBS_EINVAL;
  }
  dim3 grd((unsigned)ceil_div(H.nx, blk.y), (unsigned)ceil_div(H.ny, blk.z), (unsigned)n_sys);
#define ZM(MH)                                                                                  \
  do {                                                                                          \
    if (per_col) k_apply_zm<R, true, MH><<<grd, blk, 0, st>>>(H, L, X, Y, twist, E, Dp, sys_active); \
    else k_apply_zm<R, false, MH><<<grd, blk, 0, st>>>(H, L, X, Y, twist, E, Dp, sys_active);   \
    cbs::count_launches(1);                                                                     \
  } while (0)
  switch (H.m) {
    case 1: ZM(1); break;
    case 2: ZM(2); break;
    case 3: ZM(3); break;
    case 4: ZM(4); break;
    case 5: ZM(5); break;
    case 6: ZM(6); break;
    default: set_error("apply: FD half-width must be 1..6"); return CBS_EINVAL;
  }
#undef ZM
  CBS_CUDA(cudaGetLastError());
  return CBS_OK;
}

bool apply_supported(const HamView &H, int L, int dtype, const char *who) {
  const bool ok = L >= 1 && (L <= 256 || (dtype == CBS_C64 && L % 2 == 0 && L <= 512 && H.np4 == 4));
  if (!ok)
    set_error(std::string(who) + ": unsupported number of columns L (complex128: 1..256; complex64: "
              "1..256, or an even L up to 512 when atoms carry at most 4 projectors)");
  return ok;
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
