// Contour quadrature and moment accumulation (Algorithm 1, first step, on the ring of §3.2).
//
//   S_k  = sum_j w_j^(1) (z_j^(1))^k Y_j^(1) - sum_j w_j^(2) (z_j^(2))^k Y_j^(2),  k < M
//   mu_k = V^dagger S_k = sum_j w_j^(1) (z_j^(1))^k G_j - w_j^(2) (z_j^(2))^k G~_j, k < 2M
// with G_j = V^dagger Y_j^(1), G~_j = V^dagger Y_j^(2) (L x L each),
// z_j^(1) = e^{i theta_j} / lambda_min, z_j^(2) = lambda_min e^{i theta_j},
// theta_j = 2 pi (j - 1/2) / N_int, and the trapezoid weights w_j^(c) = z_j^(c) / N_int
// (the printed weight e^{i theta_j}/N_int times the circle's radius, which is what the
// trapezoidal rule for (1/2 pi i) oint dz gives).
#include "kernels.cuh"

namespace cbs {

// coef[j][0][k] = w1_j z1_j^k = z1_j^{k+1}/N, coef[j][1][k] = w2_j z2_j^k, k < 2M;
// z1[j] = z1_j (the primal twist of system j).
__global__ void k_contour(int n_int, int M2, double lambda_min, double2 *coef, double2 *z1) {
  const int j = blockIdx.x;            // 0-based; the paper's j is j + 1
  const int k = threadIdx.x;
  const double frac = (2.0 * j + 1.0) / n_int;   // theta_j / pi
  if (k == 0) {
    double sn, cs;
    sincospi(frac, &sn, &cs);
    z1[j] = make_double2(cs / lambda_min, sn / lambda_min);
  }
  if (k < M2) {
    double sn, cs;
    sincospi(fmod((k + 1.0) * frac, 2.0), &sn, &cs);
    const double r1 = pow(lambda_min, -(double)(k + 1)) / n_int;
    const double r2 = pow(lambda_min, (double)(k + 1)) / n_int;
    coef[((int64_t)j * 2 + 0) * M2 + k] = make_double2(r1 * cs, r1 * sn);
    coef[((int64_t)j * 2 + 1) * M2 + k] = make_double2(r2 * cs, r2 * sn);
  }
}

cbs_status launch_contour(int n_int, int M, double lambda_min, double2 *coef, double2 *z1,
                          cudaStream_t st) {
  k_contour<<<n_int, 64, 0, st>>>(n_int, 2 * M, lambda_min, coef, z1); cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  return CBS_OK;
}

// S[e][i][k][c] for k < M from the n_w primal (system e*n_w + jj) and dual (n + e*n_w + jj)
// solutions stored in Y[2n][N][L], n = n_e * n_w, of quadrature points j = j0 + jj; with
// `accumulate` the wave's sum is added to S (points streamed in waves), else it replaces S.
// mirror > 0: the solutions at the conjugate point j' = mirror - 1 - j (z_j' = conj(z_j),
// same for the dual twists) are conj(Y_j), which holds for real blocks and a real V, and
// enter with their own coefficients.
template <int MM, bool MIR>
__global__ void k_moments(int n, int n_w, int j0, int M, int64_t N, int L, const double2 *__restrict__ Y,
                          const double2 *__restrict__ coef, double2 *__restrict__ S, int accumulate,
                          int mirror) {
  // MIR: a point and its conjugate enter together through
  //   a y + a' conj(y) = (a + a') Re y + i (a - a') Im y,
  // two complex-by-real products instead of two complex ones; the four combined
  // coefficients of each (point, k) are formed once per block in shared memory.
  extern __shared__ double2 mc[];   // [n_w][4][M]: a+a', i(a-a'), -(b+b'), -i(b-b')
  const int e = blockIdx.y, c = threadIdx.x, ly = threadIdx.y, py = blockDim.y;
  const int M2 = 2 * M;
  if (MIR) {
    for (int t = threadIdx.x + threadIdx.y * blockDim.x; t < n_w * M; t += blockDim.x * blockDim.y) {
      const int jj = t / M, k = t % M;
      const int jm = mirror - 1 - j0 - jj;
      const double2 a = coef[((int64_t)(j0 + jj) * 2 + 0) * M2 + k];
      const double2 b = coef[((int64_t)(j0 + jj) * 2 + 1) * M2 + k];
      const double2 am = coef[((int64_t)jm * 2 + 0) * M2 + k];
      const double2 bm = coef[((int64_t)jm * 2 + 1) * M2 + k];
      double2 *q = mc + (int64_t)jj * 4 * M;
      q[k] = make_double2(a.x + am.x, a.y + am.y);
      q[M + k] = make_double2(-(a.y - am.y), a.x - am.x);
      q[2 * M + k] = make_double2(-(b.x + bm.x), -(b.y + bm.y));
      q[3 * M + k] = make_double2(b.y - bm.y, -(b.x - bm.x));
    }
    __syncthreads();
  }
  const int64_t per = (int64_t)py * 4;
  const int64_t i0 = (int64_t)blockIdx.x * per;
  for (int64_t i = i0 + ly; i < min(N, i0 + per); i += py) {
    double2 acc[MM];
    double2 *Se = S + ((int64_t)e * N + i) * M * L;
#pragma unroll
    for (int k = 0; k < MM; ++k)
      acc[k] = (accumulate && k < M) ? Se[(int64_t)k * L + c] : make_double2(0, 0);
    for (int jj = 0; jj < n_w; ++jj) {
      const int64_t s = (int64_t)e * n_w + jj;
      const double2 y1 = Y[(s * N + i) * L + c];
      const double2 y2 = Y[((n + s) * N + i) * L + c];
      if (MIR) {
        const double2 *q = mc + (int64_t)jj * 4 * M;
#pragma unroll
        for (int k = 0; k < MM; ++k)
          if (k < M) {
            const double2 p0 = q[k], p1 = q[M + k], p2 = q[2 * M + k], p3 = q[3 * M + k];
            acc[k].x = fma(p3.x, y2.y, fma(p2.x, y2.x, fma(p1.x, y1.y, fma(p0.x, y1.x, acc[k].x))));
            acc[k].y = fma(p3.y, y2.y, fma(p2.y, y2.x, fma(p1.y, y1.y, fma(p0.y, y1.x, acc[k].y))));
          }
      } else {
        const double2 *a = coef + (int64_t)(j0 + jj) * 2 * M2;
        const double2 *b = a + M2;
#pragma unroll
        for (int k = 0; k < MM; ++k)
          if (k < M) {
            acc[k] = cfma(a[k], y1, acc[k]);
            acc[k] = cfma(make_double2(-b[k].x, -b[k].y), y2, acc[k]);
          }
        if (mirror > 0) {
          const double2 *am = coef + (int64_t)(mirror - 1 - j0 - jj) * 2 * M2;
          const double2 *bm = am + M2;
          const double2 y1c = cconj(y1), y2c = cconj(y2);
#pragma unroll
          for (int k = 0; k < MM; ++k)
            if (k < M) {
              acc[k] = cfma(am[k], y1c, acc[k]);
              acc[k] = cfma(make_double2(-bm[k].x, -bm[k].y), y2c, acc[k]);
            }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < MM; ++k)
      if (k < M) Se[(int64_t)k * L + c] = acc[k];
  }
}

cbs_status launch_moments(int n, int n_e, int n_w, int j0, int M, int64_t N, int L, const double2 *Y,
                          const double2 *coef, double2 *S, bool accumulate, int mirror, cudaStream_t st) {
  dim3 blk = col_block(L);
  dim3 grd((unsigned)ceil_div(N, (int64_t)blk.y * 4), (unsigned)n_e, 1);
  const size_t msm = (size_t)n_w * 4 * M * sizeof(double2);
  const bool mir = mirror > 0 && msm <= 48 * 1024;
  const int acc = accumulate ? 1 : 0;
  if (M <= 8) {
    if (mir) k_moments<8, true><<<grd, blk, msm, st>>>(n, n_w, j0, M, N, L, Y, coef, S, acc, mirror);
    else k_moments<8, false><<<grd, blk, 0, st>>>(n, n_w, j0, M, N, L, Y, coef, S, acc, mirror);
  } else if (M <= 16) {
    if (mir) k_moments<16, true><<<grd, blk, msm, st>>>(n, n_w, j0, M, N, L, Y, coef, S, acc, mirror);
    else k_moments<16, false><<<grd, blk, 0, st>>>(n, n_w, j0, M, N, L, Y, coef, S, acc, mirror);
  } else {
    set_error("M must be <= 16");
    return CBS_EINVAL;
  }
  cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  return CBS_OK;
}

// part[s][chunk][c1][c2] = sum over the chunk's points of conj(V[i][c1]) Y[s][i][c2];
// RV: V is real (its imaginary parts are zero), two real products per term
constexpr int kVhyTile = 16;
template <int NQ, bool RV>
__global__ void k_vhy(int64_t N, int L, int n_chunks, const double2 *__restrict__ V,
                      const double2 *__restrict__ Y, double2 *__restrict__ part) {
  extern __shared__ double2 tile[];   // [kVhyTile][L] of V then of Y
  double2 *tv = tile, *ty = tile + kVhyTile * L;
  const int s = blockIdx.y, chunk = blockIdx.x;
  const int64_t per = (N + n_chunks - 1) / n_chunks;
  const int64_t i0 = (int64_t)chunk * per, i1 = min(N, i0 + per);
  const int LL = L * L;
  double2 acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = make_double2(0, 0);
  const double2 *Ys = Y + (int64_t)s * N * L;
  for (int64_t ib = i0; ib < i1; ib += kVhyTile) {
    const int cnt = (int)min((int64_t)kVhyTile, i1 - ib);
    for (int t = threadIdx.x; t < cnt * L; t += blockDim.x) {
      tv[t] = V[ib * L + t];
      ty[t] = Ys[ib * L + t];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int pidx = threadIdx.x + q * blockDim.x;
      if (pidx < LL) {
        const int c1 = pidx / L, c2 = pidx % L;
        double2 a = acc[q];
        if (RV) {
          for (int t = 0; t < cnt; ++t) {
            const double v = tv[t * L + c1].x;
            const double2 y = ty[t * L + c2];
            a.x = fma(v, y.x, a.x);
            a.y = fma(v, y.y, a.y);
          }
        } else {
          for (int t = 0; t < cnt; ++t) a = cadd(a, cmulc(tv[t * L + c1], ty[t * L + c2]));
        }
        acc[q] = a;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int pidx = threadIdx.x + q * blockDim.x;
    if (pidx < LL) part[((int64_t)s * n_chunks + chunk) * LL + pidx] = acc[q];
  }
}

// mu[e][k][c1][c2] (+)= sum_jj sum_chunks a_{j0+jj,k} G_jj - b_{j0+jj,k} G~_jj over the wave's
// points; mirror > 0: plus the conjugate points' terms, whose G = V^dagger conj(Y_j) is
// conj(G_j) for a real V
__global__ void k_mu(int n, int n_w, int j0, int M2, int L, int n_chunks, const double2 *part,
                     const double2 *coef, double2 *mu, int accumulate, int mirror) {
  const int e = blockIdx.y, k = blockIdx.x;
  const int LL = L * L;
  for (int pidx = threadIdx.x; pidx < LL; pidx += blockDim.x) {
    double2 *out = mu + (((int64_t)e * M2) + k) * LL + pidx;
    double2 acc = accumulate ? *out : make_double2(0, 0);
    for (int jj = 0; jj < n_w; ++jj) {
      const int64_t s = (int64_t)e * n_w + jj;
      double2 g = make_double2(0, 0), gd = make_double2(0, 0);
      for (int ch = 0; ch < n_chunks; ++ch) {
        g = cadd(g, part[(s * n_chunks + ch) * LL + pidx]);
        gd = cadd(gd, part[((n + s) * n_chunks + ch) * LL + pidx]);
      }
      const double2 a = coef[((int64_t)(j0 + jj) * 2 + 0) * M2 + k];
      const double2 b = coef[((int64_t)(j0 + jj) * 2 + 1) * M2 + k];
      acc = cfma(a, g, acc);
      acc = cfma(make_double2(-b.x, -b.y), gd, acc);
      if (mirror > 0) {
        const int jm = mirror - 1 - j0 - jj;
        const double2 am = coef[((int64_t)jm * 2 + 0) * M2 + k];
        const double2 bm = coef[((int64_t)jm * 2 + 1) * M2 + k];
        acc = cfma(am, cconj(g), acc);
        acc = cfma(make_double2(-bm.x, -bm.y), cconj(gd), acc);
      }
    }
    *out = acc;
  }
}

int vhy_chunks(int64_t N) {
  int64_t c = N / 1024;
  if (c < 1) c = 1;
  if (c > 8) c = 8;
  return (int)c;
}

cbs_status launch_mu(int n, int n_e, int n_w, int j0, int M, int64_t N, int L, const double2 *V,
                     const double2 *Y, const double2 *coef, double2 *part, double2 *mu,
                     bool accumulate, int mirror, bool v_real, cudaStream_t st) {
  if (L > 64) {
    set_error("L must be <= 64 for the moment kernel");
    return CBS_EINVAL;
  }
  const int nch = vhy_chunks(N);
  dim3 grd((unsigned)nch, (unsigned)(2 * n), 1);
  const size_t sm = 2 * kVhyTile * L * sizeof(double2);
  if (v_real) {
    if (L * L <= 4 * 256) k_vhy<4, true><<<grd, 256, sm, st>>>(N, L, nch, V, Y, part);
    else if (L * L <= 9 * 256) k_vhy<9, true><<<grd, 256, sm, st>>>(N, L, nch, V, Y, part);
    else k_vhy<16, true><<<grd, 256, sm, st>>>(N, L, nch, V, Y, part);
  } else {
    if (L * L <= 4 * 256) k_vhy<4, false><<<grd, 256, sm, st>>>(N, L, nch, V, Y, part);
    else if (L * L <= 9 * 256) k_vhy<9, false><<<grd, 256, sm, st>>>(N, L, nch, V, Y, part);
    else k_vhy<16, false><<<grd, 256, sm, st>>>(N, L, nch, V, Y, part);
  }
  cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  k_mu<<<dim3((unsigned)(2 * M), (unsigned)n_e, 1), 256, 0, st>>>(n, n_w, j0, 2 * M, L, nch, part,
                                                                 coef, mu, accumulate ? 1 : 0, mirror);
  cbs::count_launches(1);
  CBS_CUDA(cudaGetLastError());
  return CBS_OK;
}

}  // namespace cbs
