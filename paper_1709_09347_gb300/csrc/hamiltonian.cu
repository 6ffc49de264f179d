// Cell Hamiltonian set-up (the layout step of the path): FD weights, local potential,
// the projector table and its transpose, and the exact Frobenius norms of H+, H- and the
// pieces of ||H0 - E||_F used by the residual check.
//
// Paper §2, Eq. (2): the cell block H0 = H_{n,n} and the couplings H+ = H_{n,n+1},
// H- = H_{n,n-1} = H+^T of a real-space Hamiltonian (-1/2 FD Laplacian + V_loc +
// separable projectors); §4 uses a nine-point (order 8) central FD Laplacian.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace cbs {

// Central second-derivative weights of order 2m, closed form:
// c_k = 2 (-1)^{k+1} (m!)^2 / (k^2 (m-k)! (m+k)!),  c_0 = -2 sum_k c_k.
static void fd_weights(int order, double *c) {
  int m = order / 2;
  double s = 0.0;
  for (int k = 1; k <= m; ++k) {
    // (m!)^2 / ((m-k)! (m+k)!) = prod_{j=1..k} (m-k+j)/(m+j)
    double r = 1.0;
    for (int j = 1; j <= k; ++j) r *= (double)(m - k + j) / (double)(m + j);
    c[k] = 2.0 * ((k % 2) ? 1.0 : -1.0) * r / ((double)k * k);
    s += c[k];
  }
  c[0] = -2.0 * s;
}

// ------------------------------------------------------------------ Frobenius norms
// One thread per row i.  The row's entries are the merged FD stencil (block l, column j,
// weight) and, for every atom a covering i (entry s), the values (h_a p_s) . p_t at
// columns i_t of all entries t of a, in block l = m_s - m_t.  Entries that coincide in
// (l, j) are summed before squaring, so the result is the exact Frobenius norm.
constexpr int kMaxCover = 64;
constexpr int kMaxSten = 1 + 6 * kMaxHalf;

__global__ void k_frobenius(HamView H, double *part, int *err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double acc[5] = {0, 0, 0, 0, 0};  // off-diag l=0, l=+1, l=-1, diag, diag^2
  if (i < H.n) {
    const int64_t nxy = (int64_t)H.nx * H.ny;
    const int ix = (int)(i % H.nx), iy = (int)((i / H.nx) % H.ny), iz = (int)(i / nxy);
    int sl[kMaxSten];
    int64_t sc[kMaxSten];
    double sw[kMaxSten];
    int ns = 0;
    auto add = [&](int l, int64_t col, double w) {
      for (int q = 0; q < ns; ++q)
        if (sl[q] == l && sc[q] == col) { sw[q] += w; return; }
      sl[ns] = l; sc[ns] = col; sw[ns] = w; ++ns;
    };
    add(0, i, H.diag_kin + H.vloc[i]);
    for (int k = 1; k <= H.m; ++k) {
      for (int sg = -1; sg <= 1; sg += 2) {
        int jx = ((ix + sg * k) % H.nx + H.nx) % H.nx;
        add(0, i - ix + jx, H.wx[k]);
        int jy = ((iy + sg * k) % H.ny + H.ny) % H.ny;
        add(0, i + (int64_t)(jy - iy) * H.nx, H.wy[k]);
        int pz = iz + sg * k;
        int l = pz >= H.nz ? 1 : (pz < 0 ? -1 : 0);
        int jz = pz - l * H.nz;
        add(l, i + (int64_t)(jz - iz) * nxy, H.wz[k]);
      }
    }
    // covering entries of row i
    int ca[kMaxCover], cm[kMaxCover];
    double cq[kMaxCover][kMaxProj];
    int nc = 0;
    const int np = H.n_proj;
    if (H.n_atoms) {
      int64_t e0 = H.pt_ptr[i], e1 = H.pt_ptr[i + 1];
      if (e1 - e0 > kMaxCover) { atomicExch(err, 1); e1 = e0 + kMaxCover; }
      for (int64_t q = e0; q < e1; ++q, ++nc) {
        int t = H.pt_ent[q], a = H.pt_atom[q];
        ca[nc] = a;
        cm[nc] = H.sup_wrap[t];
        const double *ha = H.h + (int64_t)a * np * np;
        for (int mu = 0; mu < np; ++mu) {
          double v = 0;
          for (int nu = 0; nu < np; ++nu) v += ha[mu * np + nu] * H.sup_val[(int64_t)t * np + nu];
          cq[nc][mu] = v;
        }
      }
    }
    // Non-local value at (l, j) from covering entries with index >= from; *earlier is set
    // when a covering entry with index < from also contributes at (l, j).
    auto nl_value = [&](int l, int64_t j, int from, bool *earlier) {
      double v = 0;
      if (earlier) *earlier = false;
      int64_t f0 = H.pt_ptr[j], f1 = H.pt_ptr[j + 1];
      for (int64_t f = f0; f < f1; ++f) {
        int a2 = H.pt_atom[f], u = H.pt_ent[f];
        int mu_w = H.sup_wrap[u];
        for (int q = 0; q < nc; ++q) {
          if (ca[q] != a2 || mu_w != cm[q] - l) continue;
          if (q < from) { if (earlier) *earlier = true; continue; }
          double dot = 0;
          for (int mu = 0; mu < np; ++mu) dot += cq[q][mu] * H.sup_val[(int64_t)u * np + mu];
          v += dot;
        }
      }
      return v;
    };
    for (int q = 0; q < ns; ++q) {
      double val = sw[q] + (nc ? nl_value(sl[q], sc[q], 0, nullptr) : 0.0);
      if (sl[q] == 0 && sc[q] == i) { acc[3] += val; acc[4] += val * val; }
      else acc[sl[q] == 0 ? 0 : (sl[q] == 1 ? 1 : 2)] += val * val;
    }
    for (int q = 0; q < nc; ++q) {
      const int a = ca[q];
      for (int64_t t = H.sup_ptr[a]; t < H.sup_ptr[a + 1]; ++t) {
        const int64_t j = H.sup_idx[t];
        const int l = cm[q] - H.sup_wrap[t];
        if (l < -1 || l > 1) { atomicExch(err, 2); continue; }
        bool in_st = false;
        for (int r = 0; r < ns; ++r)
          if (sl[r] == l && sc[r] == j) { in_st = true; break; }
        if (in_st) continue;
        bool earlier;
        double val = nl_value(l, j, q, &earlier);
        if (earlier) continue;
        acc[l == 0 ? 0 : (l == 1 ? 1 : 2)] += val * val;
      }
    }
  }
  // block reduction
  __shared__ double red[5][256];
  for (int k = 0; k < 5; ++k) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off)
      for (int k = 0; k < 5; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 5; ++k) part[(int64_t)blockIdx.x * 5 + k] = red[k][0];
}

__global__ void k_sum_parts(const double *part, int nparts, double *out) {
  // one block of 5 threads: deterministic serial sums
  int k = threadIdx.x;
  if (k < 5) {
    double s = 0;
    for (int b = 0; b < nparts; ++b) s += part[(int64_t)b * 5 + k];
    out[k] = s;
  }
}

static cbs_status dalloc(cbs_hamiltonian *h, void **p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    set_error("cudaMalloc failed in cbs_create_hamiltonian");
    return CBS_ENOMEM;
  }
  h->allocs[h->n_allocs++] = *p;
  return CBS_OK;
}

template <typename T>
static cbs_status upload(cbs_hamiltonian *h, const T *src, size_t count, const T **dst) {
  void *p = nullptr;
  cbs_status s = dalloc(h, &p, count * sizeof(T));
  if (s != CBS_OK) return s;
  if (count) CBS_CUDA(cudaMemcpy(p, src, count * sizeof(T), cudaMemcpyHostToDevice));
  *dst = (const T *)p;
  return CBS_OK;
}

}  // namespace cbs

using namespace cbs;

extern "C" void cbs_hamiltonian_free(cbs_hamiltonian *h) {
  if (!h) return;
  for (int k = 0; k < h->n_allocs; ++k) cudaFree(h->allocs[k]);
  free(h);
}

extern "C" int64_t cbs_hamiltonian_size(const cbs_hamiltonian *h) { return h ? h->v.n : 0; }

extern "C" cbs_status cbs_hamiltonian_norms(const cbs_hamiltonian *h, double E, double *np_,
                                            double *n0, double *nm) {
  if (!h) { set_error("null hamiltonian"); return CBS_EINVAL; }
  double n = (double)h->v.n;
  double a2 = h->fro_off0 + h->diag_sum2 - 2.0 * E * h->diag_sum + n * E * E;
  if (np_) *np_ = sqrt(h->fro_p2);
  if (n0) *n0 = sqrt(a2 > 0 ? a2 : 0.0);
  if (nm) *nm = sqrt(h->fro_m2);
  return CBS_OK;
}

// Exact Frobenius norms of H+, H- and the pieces of ||H0 - E||_F, on the device.
static cbs_status compute_norms(cbs_hamiltonian *h) {
  HamView &v = h->v;
  // exact Frobenius norms on the device
  const int threads = 128;
  const int nb = ceil_div(v.n, threads);
  double *part = nullptr, *out = nullptr;
  int *err = nullptr;
  CBS_CUDA(cudaMalloc(&part, (size_t)nb * 5 * sizeof(double)));
  CBS_CUDA(cudaMalloc(&out, 5 * sizeof(double) + sizeof(int)));
  err = (int *)(out + 5);
  CBS_CUDA(cudaMemset(err, 0, sizeof(int)));
  k_frobenius<<<nb, threads>>>(v, part, err); cbs::count_launches(1);
  k_sum_parts<<<1, 32>>>(part, nb, out); cbs::count_launches(1);
  double res[5];
  int herr = 0;
  cudaError_t e1 = cudaMemcpy(res, out, sizeof(res), cudaMemcpyDeviceToHost);
  cudaError_t e2 = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(part);
  cudaFree(out);
  if (e1 != cudaSuccess) return cuda_fail(e1, "Frobenius norm kernel");
  if (e2 != cudaSuccess) return cuda_fail(e2, "Frobenius norm kernel");
  if (herr == 1) { set_error("more than 64 atoms cover one grid point"); return CBS_EINVAL; }
  if (herr == 2) { set_error("projector coupling beyond the neighbouring cells"); return CBS_EINVAL; }
  h->fro_off0 = res[0]; h->fro_p2 = res[1]; h->fro_m2 = res[2];
  h->diag_sum = res[3]; h->diag_sum2 = res[4];
  return CBS_OK;
}

static cbs_status create_impl(const cbs_grid *g, const double *v_loc, const cbs_projectors *P,
                              cbs_hamiltonian *h) {
  HamView &v = h->v;
  if (g->nx < 1 || g->ny < 1 || g->nz < 1 || !(g->hx > 0) || !(g->hy > 0) || !(g->hz > 0)) {
    set_error("grid sizes and spacings must be positive");
    return CBS_EINVAL;
  }
  if (g->fd_order < 2 || g->fd_order > 2 * kMaxHalf || g->fd_order % 2) {
    set_error("fd_order must be even, 2..12");
    return CBS_EINVAL;
  }
  const int m = g->fd_order / 2;
  if (m > g->nz) {
    set_error("fd_order/2 must not exceed nz (nearest-cell coupling only)");
    return CBS_EINVAL;
  }
  if (!v_loc) { set_error("v_loc is NULL"); return CBS_EINVAL; }
  v.nx = g->nx; v.ny = g->ny; v.nz = g->nz; v.m = m;
  v.n = (int64_t)g->nx * g->ny * g->nz;
  if (v.n > (int64_t)1 << 31) { set_error("grid larger than 2^31 points"); return CBS_EINVAL; }
  h->hx = g->hx; h->hy = g->hy; h->hz = g->hz; h->fd_order = g->fd_order;
  fd_weights(g->fd_order, h->fd_c);
  v.diag_kin = -0.5 * h->fd_c[0] * (1.0 / (g->hx * g->hx) + 1.0 / (g->hy * g->hy) + 1.0 / (g->hz * g->hz));
  for (int k = 0; k <= kMaxHalf; ++k) {
    double c = (k >= 1 && k <= m) ? h->fd_c[k] : 0.0;
    v.wx[k] = -0.5 * c / (g->hx * g->hx);
    v.wy[k] = -0.5 * c / (g->hy * g->hy);
    v.wz[k] = -0.5 * c / (g->hz * g->hz);
    v.w32[0][k] = (float)v.wx[k];
    v.w32[1][k] = (float)v.wy[k];
    v.w32[2][k] = (float)v.wz[k];
  }
  v.diag_kin32 = (float)v.diag_kin;
  const size_t N = (size_t)v.n;
  for (size_t i = 0; i < N; ++i)
    if (!isfinite(v_loc[i])) { set_error("v_loc contains a non-finite value"); return CBS_EINVAL; }
  cbs_status s = upload(h, v_loc, N, &v.vloc);
  if (s != CBS_OK) return s;
  std::vector<float> v32(v_loc, v_loc + N);
  s = upload(h, v32.data(), N, &v.vloc32);
  if (s != CBS_OK) return s;

  // projectors
  v.n_atoms = 0; v.n_proj = 0; h->nnz = 0; v.np4 = 4;
  std::vector<int64_t> pt_ptr(N + 1, 0);
  if (P && P->n_atoms > 0) {
    if (P->n_proj < 1 || P->n_proj > kMaxProj) { set_error("n_proj must be 1..8"); return CBS_EINVAL; }
    if (!P->sup_ptr || !P->sup_idx || !P->sup_wrap || !P->sup_val || !P->h) {
      set_error("projector table has a NULL array");
      return CBS_EINVAL;
    }
    const int na = P->n_atoms, np = P->n_proj;
    if (P->sup_ptr[0] != 0) { set_error("sup_ptr[0] must be 0"); return CBS_EINVAL; }
    for (int a = 0; a < na; ++a)
      if (P->sup_ptr[a + 1] < P->sup_ptr[a]) { set_error("sup_ptr must be non-decreasing"); return CBS_EINVAL; }
    const int64_t nnz = P->sup_ptr[na];
    if (nnz > INT32_MAX) { set_error("projector table too large"); return CBS_EINVAL; }
    std::vector<int> stamp(N, -1);
    for (int a = 0; a < na; ++a) {
      bool has_m = false, has_p = false;
      for (int64_t t = P->sup_ptr[a]; t < P->sup_ptr[a + 1]; ++t) {
        int32_t i = P->sup_idx[t];
        int w = P->sup_wrap[t];
        if (i < 0 || (size_t)i >= N) { set_error("sup_idx out of range"); return CBS_EINVAL; }
        if (w < -1 || w > 1) { set_error("sup_wrap must be -1, 0 or +1"); return CBS_EINVAL; }
        has_m |= (w == -1); has_p |= (w == 1);
        if (stamp[i] == a) { set_error("a grid point is covered twice by one atom"); return CBS_EINVAL; }
        stamp[i] = a;
        for (int mu = 0; mu < np; ++mu)
          if (!isfinite(P->sup_val[t * np + mu])) { set_error("sup_val not finite"); return CBS_EINVAL; }
        pt_ptr[i + 1]++;
      }
      if (has_m && has_p) {
        set_error("an atom covers points with wraps -1 and +1: support longer than the cell along z");
        return CBS_EINVAL;
      }
      for (int mu = 0; mu < np; ++mu)
        for (int nu = 0; nu < np; ++nu) {
          double x = P->h[((int64_t)a * np + mu) * np + nu], y = P->h[((int64_t)a * np + nu) * np + mu];
          if (!isfinite(x) || fabs(x - y) > 1e-12 * (fabs(x) + fabs(y) + 1e-300)) {
            set_error("h blocks must be finite and symmetric");
            return CBS_EINVAL;
          }
        }
    }
    for (size_t i = 0; i < N; ++i) pt_ptr[i + 1] += pt_ptr[i];
    std::vector<int32_t> pt_ent(nnz), pt_atom(nnz);
    std::vector<int64_t> fill(pt_ptr.begin(), pt_ptr.end() - 1);
    for (int a = 0; a < na; ++a)
      for (int64_t t = P->sup_ptr[a]; t < P->sup_ptr[a + 1]; ++t) {
        int64_t q = fill[P->sup_idx[t]]++;
        pt_ent[q] = (int32_t)t;
        pt_atom[q] = a;
      }
    v.n_atoms = na; v.n_proj = np; h->nnz = nnz;
    if ((s = upload(h, P->sup_ptr, (size_t)na + 1, &v.sup_ptr)) != CBS_OK) return s;
    if ((s = upload(h, P->sup_idx, (size_t)nnz, &v.sup_idx)) != CBS_OK) return s;
    if ((s = upload(h, P->sup_wrap, (size_t)nnz, &v.sup_wrap)) != CBS_OK) return s;
    if ((s = upload(h, P->sup_val, (size_t)nnz * np, &v.sup_val)) != CBS_OK) return s;
    std::vector<float> sv32(P->sup_val, P->sup_val + (size_t)nnz * np);
    if ((s = upload(h, sv32.data(), sv32.size(), &v.sup_val32)) != CBS_OK) return s;
    if ((s = upload(h, P->h, (size_t)na * np * np, &v.h)) != CBS_OK) return s;
    std::vector<float> h32(P->h, P->h + (size_t)na * np * np);
    if ((s = upload(h, h32.data(), h32.size(), &v.h32)) != CBS_OK) return s;
    if ((s = upload(h, pt_ptr.data(), N + 1, &v.pt_ptr)) != CBS_OK) return s;
    if ((s = upload(h, pt_ent.data(), (size_t)nnz, &v.pt_ent)) != CBS_OK) return s;
    if ((s = upload(h, pt_atom.data(), (size_t)nnz, &v.pt_atom)) != CBS_OK) return s;
    // packed per-entry records for the complex64 scatter (point order)
    v.np4 = np <= 4 ? 4 : 8;
    std::vector<int2> aw(nnz);
    std::vector<float4> p4(np <= 4 ? nnz : 0);
    for (int64_t q = 0; q < nnz; ++q) {
      const int t = pt_ent[q];
      aw[q] = make_int2(pt_atom[q], (int)P->sup_wrap[t]);
      if (np <= 4) {
        float pv[4] = {0, 0, 0, 0};
        for (int mu = 0; mu < np; ++mu) pv[mu] = (float)P->sup_val[(int64_t)t * np + mu];
        p4[q] = make_float4(pv[0], pv[1], pv[2], pv[3]);
      }
    }
    if ((s = upload(h, aw.data(), (size_t)nnz, &v.pt_aw)) != CBS_OK) return s;
    if (np <= 4 && (s = upload(h, p4.data(), (size_t)nnz, &v.pt_p32)) != CBS_OK) return s;
  } else {
    if ((s = upload(h, pt_ptr.data(), N + 1, &v.pt_ptr)) != CBS_OK) return s;
  }

  return compute_norms(h);
}

extern "C" cbs_status cbs_create_hamiltonian(const cbs_grid *grid, const double *v_loc,
                                             const cbs_projectors *proj, cbs_hamiltonian **out) {
  if (!grid || !out) { set_error("null argument"); return CBS_EINVAL; }
  *out = nullptr;
  cbs_hamiltonian *h = (cbs_hamiltonian *)calloc(1, sizeof(cbs_hamiltonian));
  if (!h) { set_error("host allocation failed"); return CBS_ENOMEM; }
  cbs_status s = create_impl(grid, v_loc, proj, h);
  if (s != CBS_OK) { cbs_hamiltonian_free(h); return s; }
  *out = h;
  return CBS_OK;
}

namespace cbs {
// V_loc in single precision from the FP64 copy, and a flag if any value is not finite.
__global__ void k_vloc32(int64_t n, const double *v, float *v32, int *bad) {
  int b = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = v[i];
    v32[i] = (float)x;
    b |= !isfinite(x);
  }
  if (__syncthreads_or(b) && threadIdx.x == 0) atomicOr(bad, 1);
}
}  // namespace cbs

extern "C" cbs_status cbs_hamiltonian_set_vloc(cbs_hamiltonian *h, const double *v_loc) {
  if (!h || !v_loc) { set_error("cbs_hamiltonian_set_vloc: null argument"); return CBS_EINVAL; }
  HamView &v = h->v;
  const size_t N = (size_t)v.n;
  int *bad = nullptr;
  double *tmp = nullptr;
  CBS_CUDA(cudaMalloc(&tmp, N * sizeof(double) + 256));
  bad = (int *)((char *)tmp + ((N * sizeof(double) + 127) & ~(size_t)127));
  cbs_status s = CBS_OK;
  cudaError_t e = cudaMemcpy(tmp, v_loc, N * sizeof(double), cudaMemcpyDefault);
  if (e == cudaSuccess) e = cudaMemset(bad, 0, sizeof(int));
  if (e == cudaSuccess) {
    // check into a scratch copy first, so a rejected V_loc leaves the handle unchanged
    k_vloc32<<<std::min<int64_t>(1024, ((int64_t)N + 255) / 256), 256>>>((int64_t)N, tmp,
                                                                         const_cast<float *>(v.vloc32), bad);
    cbs::count_launches(1);
    e = cudaGetLastError();
  }
  int hb = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) s = cuda_fail(e, "cbs_hamiltonian_set_vloc");
  else if (hb) {
    // restore the single-precision copy from the unchanged FP64 one
    k_vloc32<<<std::min<int64_t>(1024, ((int64_t)N + 255) / 256), 256>>>((int64_t)N, v.vloc,
                                                                         const_cast<float *>(v.vloc32), bad);
    cbs::count_launches(1);
    cudaDeviceSynchronize();
    set_error("v_loc contains a non-finite value");
    s = CBS_EINVAL;
  } else {
    e = cudaMemcpy(const_cast<double *>(v.vloc), tmp, N * sizeof(double), cudaMemcpyDeviceToDevice);
    if (e != cudaSuccess) s = cuda_fail(e, "cbs_hamiltonian_set_vloc copy");
  }
  cudaFree(tmp);
  if (s != CBS_OK) return s;
  return compute_norms(h);
}
