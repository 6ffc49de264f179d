// Objective of the ring solves and its reverse-mode gradient (adjoint solves).
//
// J = sum_{c=1,2} sum_j c_j^(c) ||Y_j^(c)||_F^2 with c_j^(c) = Re(s_c w_j^(c) sum_{k<M} (z_j^(c))^k),
// s_1 = +1, s_2 = -1, and Y_j^(c) = P(z_j^(c))^{-1} V the solutions of the shifted systems of
// §3.2 (Eq. (9)-(11)).  With dP = dE I - diag(dV_loc) and G = P^{-dagger} Y:
//   dJ/dV_loc[i] = sum 2 c Re sum_col conj(G[i,col]) Y[i,col],   dJ/dE = -sum 2 c Re tr(G^dagger Y).
// The adjoint systems of both circles are one BiCG batch at the outer-circle points:
//   P(z_j^(1)) G_j^(2) = Y_j^(2)   (primal; P(z^(2))^dagger = P(z^(1)), §3.2)
//   P(z_j^(1))^dagger G_j^(1) = Y_j^(1)   (dual).
// The forward solutions are recomputed on every call; nothing is kept between calls.
#include <math.h>

#include <vector>

#include "kernels.cuh"

namespace cbs {

// c1[j] = Re sum_{k<M} w1_j z1_j^k,  c2[j] = -Re sum_{k<M} w2_j z2_j^k  (coef from k_contour)
__global__ void k_objective_weights(int n_int, int M, const double2 *coef, double *c1, double *c2) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_int) return;
  const int M2 = 2 * M;
  double a = 0, b = 0;
  for (int k = 0; k < M; ++k) {
    a += coef[((int64_t)j * 2 + 0) * M2 + k].x;
    b += coef[((int64_t)j * 2 + 1) * M2 + k].x;
  }
  c1[j] = a;
  c2[j] = -b;
}

// Per grid point: J contribution and, if G, the gradient; block partial sums of J and dJ/dE.
// Y, G: [2n][N][L]; Y[s] = Y1_s, Y[n+s] = Y2_s; G[s] = G2_s, G[n+s] = G1_s.
__global__ void k_objective_points(int n, int64_t N, int L, const double2 *Y, const double2 *G,
                                   const double *c1, const double *c2, double *gV, double *part) {
  double pj = 0, pe = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    double g = 0;
    for (int s = 0; s < n; ++s) {
      const double2 *y1 = Y + ((int64_t)s * N + i) * L, *y2 = Y + ((int64_t)(n + s) * N + i) * L;
      double a1 = 0, a2 = 0, b1 = 0, b2 = 0;
      for (int c = 0; c < L; ++c) {
        const double2 u = y1[c], v = y2[c];
        a1 += cabs2(u);
        a2 += cabs2(v);
        if (G) {
          const double2 g1 = G[((int64_t)(n + s) * N + i) * L + c];
          const double2 g2 = G[((int64_t)s * N + i) * L + c];
          b1 += g1.x * u.x + g1.y * u.y;    // Re conj(G1) Y1
          b2 += g2.x * v.x + g2.y * v.y;    // Re conj(G2) Y2
        }
      }
      pj += c1[s] * a1 + c2[s] * a2;
      g += 2.0 * (c1[s] * b1 + c2[s] * b2);
    }
    if (G) gV[i] = g;
    pe -= g;
  }
  __shared__ double r0[256], r1[256];
  r0[threadIdx.x] = pj;
  r1[threadIdx.x] = pe;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) { r0[threadIdx.x] += r0[threadIdx.x + o]; r1[threadIdx.x] += r1[threadIdx.x + o]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { part[2 * blockIdx.x] = r0[0]; part[2 * blockIdx.x + 1] = r1[0]; }
}

__global__ void k_sum2(const double *part, int nb, double *out) {
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int k = 0; k < nb; ++k) { a += part[2 * k]; b += part[2 * k + 1]; }
    out[0] = a;
    out[1] = b;
  }
}

}  // namespace cbs

using namespace cbs;

// declared in solve.cu
cbs_status cbs_internal_ring_solve(const cbs_hamiltonian *h, int n, int L, const double2 *zs,
                                   const double *Es, const double2 *dV, const cbs_options &o,
                                   cudaStream_t st, double2 **Y_out, void **owner);
void cbs_internal_ring_release(void *owner);

extern "C" cbs_status cbs_objective(const cbs_hamiltonian *h, double E, const cbs_contour *ct, int L,
                                    int M, const void *V, const cbs_options *opt, double *J,
                                    double *grad_vloc, double *grad_E) {
  if (!h || !ct || !V || !J || L < 1 || L > 1024 || M < 1 || M > 16 || ct->n_int < 1 ||
      !(ct->lambda_min > 0 && ct->lambda_min < 1) || !isfinite(E)) {
    set_error("cbs_objective: bad argument");
    return CBS_EINVAL;
  }
  cbs_options o;
  if (opt) o = *opt; else cbs_options_default(&o);
  cudaStream_t st = (cudaStream_t)o.stream;
  bool own_stream = false;
  if (!st) { CBS_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)); own_stream = true; }
  o.stream = st;
  const HamView &H = h->v;
  const int64_t N = H.n;
  const int n = ct->n_int;
  cbs_status s = CBS_OK;
  void *buf = nullptr, *owner = nullptr;
  double2 *Y = nullptr;
  Bicg<double> adj;
  const size_t vbytes = (size_t)N * L * sizeof(double2);
  const int nb = 152 * 2;
  const size_t small = (size_t)n * (4 * M + 1) * sizeof(double2) + 4 * (size_t)n * sizeof(double) + 2 * nb * sizeof(double) + 4096;
  do {
    if (cudaMalloc(&buf, vbytes + small + (size_t)N * sizeof(double)) != cudaSuccess) { set_error("cudaMalloc failed"); s = CBS_ENOMEM; break; }
    double2 *dV = (double2 *)buf;
    double2 *coef = (double2 *)((char *)buf + vbytes);
    double2 *z1 = coef + (size_t)n * 4 * M;
    double *Es = (double *)(z1 + n);
    double *c1 = Es + n, *c2 = c1 + n;
    double *part = c2 + n;
    double *out = part + 2 * nb;
    double *gV = out + 4;
    cudaError_t ce = cudaMemcpyAsync(dV, V, vbytes, cudaMemcpyDefault, st);
    if (ce != cudaSuccess) { s = cuda_fail(ce, "cbs_objective: V upload"); break; }
    if ((s = launch_contour(n, M, ct->lambda_min, coef, z1, st)) != CBS_OK) break;
    std::vector<double> hE(n, E);
    ce = cudaMemcpyAsync(Es, hE.data(), n * sizeof(double), cudaMemcpyHostToDevice, st);
    if (ce != cudaSuccess) { s = cuda_fail(ce, "cbs_objective: energies"); break; }
    k_objective_weights<<<ceil_div(n, 64), 64, 0, st>>>(n, M, coef, c1, c2);
    cbs::count_launches(1);
    // forward: Y (primal outer circle, then its duals = inner circle)
    if ((s = cbs_internal_ring_solve(h, n, L, z1, Es, dV, o, st, &Y, &owner)) != CBS_OK &&
        s != CBS_ENOCONV && s != CBS_EBREAKDOWN)
      break;
    cbs_status fwd = s;
    s = CBS_OK;
    const double2 *G = nullptr;
    if (grad_vloc || grad_E) {
      if ((s = adj.alloc(H, n, L)) != CBS_OK) break;
      if ((s = adj.set_systems(z1, Es, st)) != CBS_OK) break;
      // primal right-hand sides Y2 (systems n..2n-1 of Y), dual right-hand sides Y1
      if ((s = adj.init(Y + (size_t)n * N * L, N * L, Y, N * L, nullptr, o.tol, 0.0, st)) != CBS_OK) break;
      int done = 0;
      if ((s = adj.iterate(o.tol, o.max_iter, o.check_every, st, &done)) != CBS_OK) break;
      G = adj.x;
    }
    k_objective_points<<<nb, 256, 0, st>>>(n, N, L, Y, G, c1, c2, gV, part);
    cbs::count_launches(1);
    k_sum2<<<1, 32, 0, st>>>(part, nb, out);
    cbs::count_launches(1);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) { s = cuda_fail(ce, "cbs_objective kernels"); break; }
    double hout[2];
    ce = cudaMemcpyAsync(hout, out, sizeof(hout), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess && grad_vloc) ce = cudaMemcpyAsync(grad_vloc, gV, (size_t)N * sizeof(double), cudaMemcpyDefault, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) { s = cuda_fail(ce, "cbs_objective: results"); break; }
    *J = hout[0];
    if (grad_E) *grad_E = hout[1];
    if (s == CBS_OK) s = fwd;
  } while (0);
  adj.release();
  if (owner) cbs_internal_ring_release(owner);
  if (buf) { cudaStreamSynchronize(st); cudaFree(buf); }
  if (own_stream) cudaStreamDestroy(st);
  return s;
}
