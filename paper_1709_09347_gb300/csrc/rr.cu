// Rayleigh-Ritz extraction with a small linearised QEP (not in the paper; an alternative to
// the reduced eigenproblem of Algorithm 1 that uses the same moments).
//
//   Z = S W_1                 (the part of the moment space kept by the Hankel rank cut)
//   Q = orthonormal basis of span(Z)   (two Gram-eigen passes, columns with sigma >= 1e-7 sigma_1)
//   A2 = Q^dagger H+ Q,  A1 = Q^dagger (H0 - E) Q,  A0 = Q^dagger H- Q
//   (lambda^2 A2 + lambda A1 + A0) u = 0, solved through lambda = shift + 1/mu:
//   (mu^2 B0 + mu B1 + A2) u = 0 with B0 = Q(shift) (invertible), B1 = 2 shift A2 + A1,
//   companion [[0, I], [-B0^{-1} A2, -B0^{-1} B1]]; Ritz vectors x = Q u.
// H+ Q, H0 Q, H- Q come from three applies of P(w) with E = 0 at w = 1, -1, i:
// R_w = -P(w)Q|_{E=0} = H0 Q + w H+ Q + w^{-1} H- Q.
#include <math.h>

#include <vector>

#include "kernels.cuh"

#define CBS_TRY_RR(x)                 \
  do {                                \
    cbs_status _s = (x);              \
    if (_s != CBS_OK) return _s;      \
  } while (0)

namespace cbs {

// R[3][N][r] = P(w)Q at w = 1, -1, i with E = 0 (i.e. -H(w)Q); out[0..2] = H0Q, H+Q, H-Q
__global__ void k_rr_blocks(int64_t cnt, const double2 *R, double2 *out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double2 r1 = make_double2(-R[e].x, -R[e].y);                 // H(1) Q
    const double2 rm = make_double2(-R[cnt + e].x, -R[cnt + e].y);     // H(-1) Q
    const double2 ri = make_double2(-R[2 * cnt + e].x, -R[2 * cnt + e].y);  // H(i) Q
    const double2 h0 = cscale(cadd(r1, rm), 0.5);
    const double2 sp = cscale(csub(r1, rm), 0.5);                      // H+Q + H-Q
    const double2 t = csub(ri, h0);                                    // i (H+Q - H-Q)
    const double2 df = make_double2(t.y, -t.x);                        // H+Q - H-Q
    out[e] = h0;
    out[cnt + e] = cscale(cadd(sp, df), 0.5);
    out[2 * cnt + e] = cscale(csub(sp, df), 0.5);
  }
}

__global__ void k_replicate3(int64_t cnt, const double2 *Q, double2 *X3) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = Q[e];
    X3[e] = v;
    X3[cnt + e] = v;
    X3[2 * cnt + e] = v;
  }
}

// rows i of the r x N (column-major, ld r) matrix Qt scaled by inv_sqrt(lambda_i)
__global__ void k_scale_rows_rsqrt(int r, int64_t N, const double *lam, double2 *Qt) {
  const int64_t tot = (int64_t)r * N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % r);
    Qt[e] = cscale(Qt[e], 1.0 / sqrt(lam[i]));
  }
}

// B0 = s^2 A2 + s A1 + A0 - s E I, B1 = 2 s A2 + A1 - E I (A1 = Q^dagger H0 Q here), from the
// transposed products CTk (CTk[j + i r] = Ak(i, j)); LU with partial pivoting of B0 and
// solve for [A2 | B1]; companion C (2r x 2r, column-major) = [[0, I], [-X_A2, -X_B1]].
// Work is r x 3r complex in `work`; info = 1 if a pivot vanished.
constexpr int kLuThreads = 512;
__global__ void __launch_bounds__(kLuThreads) k_rr_companion(int r, const double2 *CT2, const double2 *CT1,
                                                             const double2 *CT0, double E, double2 s,
                                                             double2 *work, double2 *C, int *info) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int ld = r;
  double2 *B = work;                    // r x r  (column-major)
  double2 *Rh = work + (size_t)r * r;   // r x 2r right-hand sides [A2 | B1]
  const double2 s2 = cmul(s, s);
  for (int e = tid; e < r * r; e += nt) {
    const int i = e % r, j = e / r;
    const double2 a2 = CT2[j + (size_t)i * r], a1 = CT1[j + (size_t)i * r], a0 = CT0[j + (size_t)i * r];
    double2 b0 = cadd(cadd(cmul(s2, a2), cmul(s, a1)), a0);
    double2 b1 = cadd(cscale(cmul(s, a2), 2.0), a1);
    if (i == j) {
      b0 = csub(b0, cscale(s, E));     // s (A1 - E I): the -E I part of A1
      b1 = make_double2(b1.x - E, b1.y);
    }
    B[i + (size_t)j * ld] = b0;
    Rh[i + (size_t)j * ld] = a2;
    Rh[i + (size_t)(r + j) * ld] = b1;
  }
  __syncthreads();
  __shared__ int piv;
  __shared__ int bad;
  if (tid == 0) bad = 0;
  for (int k = 0; k < r; ++k) {
    if (tid == 0) {
      int p = k;
      double best = -1;
      for (int i = k; i < r; ++i) {
        const double v = cabs2(B[i + (size_t)k * ld]);
        if (v > best) { best = v; p = i; }
      }
      piv = p;
      if (!(best > 0)) bad = 1;
    }
    __syncthreads();
    if (bad) break;
    const int p = piv;
    if (p != k) {
      for (int j = tid; j < 3 * r; j += nt) {
        double2 *M = j < r ? B + (size_t)j * ld : Rh + (size_t)(j - r) * ld;
        const double2 t = M[k];
        M[k] = M[p];
        M[p] = t;
      }
      __syncthreads();
    }
    // multipliers l_i = B(i,k) / B(k,k), kept in column k
    const double2 d = B[k + (size_t)k * ld];
    for (int i = k + 1 + tid; i < r; i += nt) B[i + (size_t)k * ld] = cdiv(B[i + (size_t)k * ld], d);
    __syncthreads();
    // trailing update over columns j > k of B and all right-hand sides
    for (int j = tid; j < 3 * r; j += nt) {
      if (j < r && j <= k) continue;
      double2 *M = j < r ? B + (size_t)j * ld : Rh + (size_t)(j - r) * ld;
      const double2 mk = M[k];
      for (int i = k + 1; i < r; ++i) M[i] = csub(M[i], cmul(B[i + (size_t)k * ld], mk));
    }
    __syncthreads();
  }
  if (tid == 0) *info = bad;
  if (bad) return;
  // back substitution U x = rhs for every right-hand side (thread per column)
  for (int j = tid; j < 2 * r; j += nt) {
    double2 *x = Rh + (size_t)j * ld;
    for (int i = r - 1; i >= 0; --i) {
      double2 v = x[i];
      for (int q = i + 1; q < r; ++q) v = csub(v, cmul(B[i + (size_t)q * ld], x[q]));
      x[i] = cdiv(v, B[i + (size_t)i * ld]);
    }
  }
  __syncthreads();
  const int n2 = 2 * r;
  for (int e = tid; e < n2 * n2; e += nt) {
    const int i = e % n2, j = e / n2;
    double2 v = make_double2(0, 0);
    if (i < r) v = make_double2((j == r + i) ? 1.0 : 0.0, 0.0);
    else {
      const double2 x = Rh[(i - r) + (size_t)j * ld];   // X_A2 for j < r, X_B1 for j >= r
      v = make_double2(-x.x, -x.y);
    }
    C[i + (size_t)j * n2] = v;
  }
}

}  // namespace cbs

using namespace cbs;

// Rayleigh-Ritz candidates for one energy.  S: [N][n] row-major moments (n = L*M), Ws: the
// n x n right singular vectors of T (column-major, first m columns kept).  On success
// *cnt candidate pairs inside the ring: lam [cnt] and Psi [N][cnt] (device, owned by ws);
// lam_all (host) receives every finite Ritz value.
cbs_status cbs_internal_rr(const cbs_hamiltonian *h, double E, const double2 *S, const double2 *Ws,
                           int n, int m, double lambda_min, cudaStream_t st, void **ws_out,
                           int *cnt_out, double2 **lam_out, double2 **Psi_out,
                           std::vector<double2> *lam_all, int *rank_out) {
  const HamView &H = h->v;
  const int64_t N = H.n;
  *cnt_out = 0;
  *ws_out = nullptr;
  if (m < 1) return CBS_OK;
  const int m0 = m;
  const double2 one = make_double2(1, 0), zero = make_double2(0, 0);
  // workspace
  const size_t Nm = (size_t)N * m0;
  const size_t mm = (size_t)m0 * m0;
  size_t bytes = 0;
  auto add = [&](size_t b) { size_t o = bytes; bytes += (b + 255) & ~(size_t)255; return o; };
  const size_t oZ = add(Nm * 16), oQ = add(Nm * 16), oX3 = add(3 * Nm * 16), oR3 = add(3 * Nm * 16),
               oG = add(mm * 16), oGw = add(mm * 16), oGu = add(mm * 16), oGws = add(mm * 16),
               osig = add(m0 * 8), oinfo = add(64), oCT = add(3 * mm * 16), oLU = add(3 * mm * 16),
               oC = add(4 * mm * 16), oZe = add(4 * mm * 16), otau = add(2 * m0 * 16),
               oYc = add(4 * mm * 16), oring = add(2 * m0 * 4), osm = add(64), oP1 = add(4 * mm * 16),
               oPsi = add((size_t)N * 2 * m0 * 16), oD = add((size_t)3 * (H.n_atoms ? H.n_atoms : 1) * H.np4 * m0 * 16),
               otw = add(256), olam = add(2 * m0 * 16);
  char *base = nullptr;
  if (cudaMalloc(&base, bytes) != cudaSuccess) { set_error("cudaMalloc failed (Rayleigh-Ritz workspace)"); return CBS_ENOMEM; }
  *ws_out = base;
  double2 *Z = (double2 *)(base + oZ), *Q = (double2 *)(base + oQ), *X3 = (double2 *)(base + oX3),
          *R3 = (double2 *)(base + oR3), *G = (double2 *)(base + oG), *Gw = (double2 *)(base + oGw),
          *Gu = (double2 *)(base + oGu), *Gws = (double2 *)(base + oGws), *CT = (double2 *)(base + oCT),
          *LU = (double2 *)(base + oLU), *C = (double2 *)(base + oC), *Ze = (double2 *)(base + oZe),
          *tau = (double2 *)(base + otau), *Yc = (double2 *)(base + oYc), *P1 = (double2 *)(base + oP1),
          *Psi = (double2 *)(base + oPsi), *D = (double2 *)(base + oD), *tw = (double2 *)(base + otw),
          *lam = (double2 *)(base + olam);
  double *sig = (double *)(base + osig);
  int *info = (int *)(base + oinfo), *ring = (int *)(base + oring), *sm = (int *)(base + osm);
  // Z^T (m x N, ld m) = W1^T S^T
  CBS_TRY_RR(zgemm(1, 0, m0, (int)N, n, one, Ws, n, 0, S, n, 0, zero, Z, m0, 0, 1, st));
  // two Gram-eigen passes: Q^T = Lambda^{-1/2} U^dagger Z^T  with  U Lambda U^dagger = conj(Z^dagger Z)
  int r = m0;
  const double2 *src = Z;
  std::vector<double> hs(m0);
  for (int pass = 0; pass < 2; ++pass) {
    CBS_TRY_RR(zgemm(0, 2, r, r, (int)N, one, src, r, 0, src, r, 0, zero, G, r, 0, 1, st));
    CBS_TRY_RR(launch_svd(1, r, G, Gw, Gu, Gws, sig, info, st));
    CBS_CUDA(cudaMemcpyAsync(hs.data(), sig, (size_t)r * sizeof(double), cudaMemcpyDeviceToHost, st));
    CBS_CUDA(cudaStreamSynchronize(st));
    int keep = 0;
    for (int i = 0; i < r; ++i) keep += (hs[i] >= 1e-14 * hs[0] && hs[i] > 0);
    if (pass == 0 && keep > 256) keep = 256;   // companion of size 2r must fit the eigen-solver
    if (keep == 0) return CBS_OK;
    // Q^T (keep x N, ld keep) = Gu[:, :keep]^dagger src
    CBS_TRY_RR(zgemm(2, 0, keep, (int)N, r, one, Gu, r, 0, src, r, 0, zero, Q, keep, 0, 1, st));
    k_scale_rows_rsqrt<<<152 * 4, 256, 0, st>>>(keep, N, sig, Q);
    cbs::count_launches(1);
    CBS_CUDA(cudaGetLastError());
    r = keep;
    if (pass == 0) {
      CBS_CUDA(cudaMemcpyAsync(Z, Q, (size_t)N * r * sizeof(double2), cudaMemcpyDeviceToDevice, st));
      src = Z;
    }
  }
  *rank_out = r;
  // blocks: apply P(w) (E = 0) at w = 1, -1, i to Q ([N][r] row-major = Q^T column-major)
  const int64_t cntQ = N * r;
  k_replicate3<<<152 * 4, 256, 0, st>>>(cntQ, Q, X3);
  cbs::count_launches(1);
  const double2 hw[3] = {make_double2(1, 0), make_double2(-1, 0), make_double2(0, 1)};
  const double hE[3] = {0, 0, 0};
  CBS_CUDA(cudaMemcpyAsync(tw, hw, sizeof(hw), cudaMemcpyHostToDevice, st));
  CBS_CUDA(cudaMemcpyAsync((double *)(tw + 3), hE, sizeof(hE), cudaMemcpyHostToDevice, st));
  CBS_TRY_RR(apply_P<double>(H, 3, r, X3, R3, tw, false, (const double *)(tw + 3), D, nullptr, st));
  k_rr_blocks<<<152 * 4, 256, 0, st>>>(cntQ, R3, X3);   // X3 <- H0Q, H+Q, H-Q
  cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  // CT_l = (Q^dagger X_l)^T = X_l^T conj(Q): zgemm(N, C) on the column-major transposes
  const size_t rr2 = (size_t)r * r;
  CBS_TRY_RR(zgemm(0, 2, r, r, (int)N, one, X3 + cntQ, r, 0, Q, r, 0, zero, CT, r, 0, 1, st));          // A2
  CBS_TRY_RR(zgemm(0, 2, r, r, (int)N, one, X3, r, 0, Q, r, 0, zero, CT + rr2, r, 0, 1, st));          // Q^dagger H0 Q
  CBS_TRY_RR(zgemm(0, 2, r, r, (int)N, one, X3 + 2 * cntQ, r, 0, Q, r, 0, zero, CT + 2 * rr2, r, 0, 1, st));  // A0
  // shift inside the ring, off the unit circle (propagating eigenvalues sit on it)
  const double2 shift = make_double2(0.7 * cos(2.399963), 0.7 * sin(2.399963));
  k_rr_companion<<<1, kLuThreads, 0, st>>>(r, CT, CT + rr2, CT + 2 * rr2, E, shift, LU, C, info);
  cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  int hinfo = 0;
  CBS_CUDA(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st));
  CBS_CUDA(cudaStreamSynchronize(st));
  if (hinfo) { set_error("Rayleigh-Ritz: shifted projected matrix is singular"); return CBS_EBREAKDOWN; }
  const int n2 = 2 * r;
  CBS_CUDA(cudaMemcpyAsync(sm, &n2, sizeof(int), cudaMemcpyHostToDevice, st));
  CBS_TRY_RR(launch_eig(1, n2, sm, C, Ze, tau, Yc, sm + 1, ring, lambda_min, sm + 2, st, shift, 1));
  int hsm[3];
  CBS_CUDA(cudaMemcpyAsync(hsm, sm, sizeof(hsm), cudaMemcpyDeviceToHost, st));
  std::vector<double2> htau(n2);
  CBS_CUDA(cudaMemcpyAsync(htau.data(), tau, n2 * sizeof(double2), cudaMemcpyDeviceToHost, st));
  CBS_CUDA(cudaStreamSynchronize(st));
  lam_all->clear();
  for (int k = 0; k < n2; ++k)
    if (isfinite(htau[k].x) && isfinite(htau[k].y)) lam_all->push_back(htau[k]);
  const int cnt = hsm[1];
  if (cnt == 0 || hsm[2]) return CBS_OK;
  // w = Ze Yc (2r x cnt), u = first r rows; Psi^T (cnt x N) = u^T Q^T
  CBS_TRY_RR(zgemm(0, 0, n2, cnt, n2, one, Ze, n2, 0, Yc, n2, 0, zero, P1, n2, 0, 1, st));
  CBS_TRY_RR(zgemm(1, 0, cnt, (int)N, r, one, P1, n2, 0, Q, r, 0, zero, Psi, cnt, 0, 1, st));
  std::vector<int> hring(cnt);
  CBS_CUDA(cudaMemcpyAsync(hring.data(), ring, cnt * sizeof(int), cudaMemcpyDeviceToHost, st));
  CBS_CUDA(cudaStreamSynchronize(st));
  std::vector<double2> hl(cnt);
  for (int q = 0; q < cnt; ++q) hl[q] = htau[hring[q]];
  CBS_CUDA(cudaMemcpyAsync(lam, hl.data(), cnt * sizeof(double2), cudaMemcpyHostToDevice, st));
  *cnt_out = cnt;
  *lam_out = lam;
  *Psi_out = Psi;
  return CBS_OK;
}
