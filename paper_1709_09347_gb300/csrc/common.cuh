// Shared helpers for libcbs: complex arithmetic on interleaved pairs, error plumbing,
// and the device-side view of the cell Hamiltonian.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/cbs.h"

namespace cbs {

// ---------------------------------------------------------------- complex types
template <typename R> struct CT;
template <> struct CT<double> { typedef double2 T; };
template <> struct CT<float> { typedef float2 T; };

template <typename R> __host__ __device__ __forceinline__ typename CT<R>::T mk(R a, R b) {
  typename CT<R>::T r; r.x = a; r.y = b; return r;
}
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__host__ __device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }
// a += s * b  (s complex)
__host__ __device__ __forceinline__ double2 cfma(double2 s, double2 b, double2 a) {
  a.x = fma(s.x, b.x, a.x); a.x = fma(-s.y, b.y, a.x);
  a.y = fma(s.x, b.y, a.y); a.y = fma(s.y, b.x, a.y);
  return a;
}
__host__ __device__ __forceinline__ float2 cfma(float2 s, float2 b, float2 a) {
  a.x = fmaf(s.x, b.x, a.x); a.x = fmaf(-s.y, b.y, a.x);
  a.y = fmaf(s.x, b.y, a.y); a.y = fmaf(s.y, b.x, a.y);
  return a;
}
__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  // Smith's algorithm (scaled) for a / b
  if (fabs(b.x) >= fabs(b.y)) {
    double r = b.y / b.x, d = b.x + b.y * r;
    return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
  } else {
    double r = b.x / b.y, d = b.y + b.x * r;
    return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
  }
}
__host__ __device__ __forceinline__ double2 to_d(float2 a) { return make_double2(a.x, a.y); }
__host__ __device__ __forceinline__ double2 to_d(double2 a) { return a; }
template <typename R> __host__ __device__ __forceinline__ typename CT<R>::T from_d(double2 a);
template <> __host__ __device__ __forceinline__ double2 from_d<double>(double2 a) { return a; }
template <> __host__ __device__ __forceinline__ float2 from_d<float>(double2 a) {
  return make_float2((float)a.x, (float)a.y);
}

// ---------------------------------------------------------------- Hamiltonian
constexpr int kMaxHalf = 6;   // fd_order <= 12
constexpr int kMaxProj = 8;

// Device view, passed by value to kernels.
struct HamView {
  int nx, ny, nz, m;        // grid and FD half-width
  int64_t n;                // nx*ny*nz
  double diag_kin;          // -1/2 c0 (1/hx^2 + 1/hy^2 + 1/hz^2)
  double wx[kMaxHalf + 1], wy[kMaxHalf + 1], wz[kMaxHalf + 1];  // -1/2 c_k / h^2 (k >= 1)
  float w32[3][kMaxHalf + 1];   // the same weights in single precision (x, y, z)
  float diag_kin32;
  const double *vloc;
  const float *vloc32;
  // projector table and its transpose (grid point -> covering entries)
  int n_atoms, n_proj;
  const int64_t *sup_ptr;   // [n_atoms+1]
  const int32_t *sup_idx;   // [nnz]
  const int8_t *sup_wrap;   // [nnz]
  const double *sup_val;    // [nnz][n_proj]
  const float *sup_val32;
  const double *h;          // [n_atoms][n_proj][n_proj]
  const float *h32;
  const int64_t *pt_ptr;    // [n+1]
  const int32_t *pt_ent;    // [nnz] support entry index
  const int32_t *pt_atom;   // [nnz] atom of that entry
  int np4;                  // projector slots per entry in D and pt_p32: 4 (n_proj <= 4) or 8
  const int2 *pt_aw;        // [nnz] (atom, wrap) of each covering entry, point order
  const float4 *pt_p32;     // [nnz] projector values of the entry, zero-padded to 4 (n_proj <= 4)
  // stencil launch shape chosen by cbs_autotune_apply, per precision ([0] complex128,
  // [1] complex64): a block covers tune_py x-lines of tune_pz rows (0 = default: 256 /
  // threads per line x-lines of one row) and, for complex64, whether the
  // two-columns-per-thread kernel is used (1 = yes, 0 = default, -1 = no)
  int tune_py[2], tune_pz[2];
  int tune_x2;
};

}  // namespace cbs

struct cbs_hamiltonian {
  cbs::HamView v;
  double hx, hy, hz;
  int fd_order;
  int64_t nnz;
  double fd_c[cbs::kMaxHalf + 1];
  // Frobenius pieces: ||H+||^2, ||H-||^2, off-diagonal part of ||H0||^2, sum d_i, sum d_i^2
  double fro_p2, fro_m2, fro_off0, diag_sum, diag_sum2;
  // device allocations owned by the handle
  void *allocs[24];
  int n_allocs;
};

namespace cbs {

// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);
cbs_status cuda_fail(cudaError_t e, const char *what);

// kernel-launch accounting (cbs_kernel_launches)
void count_launches(uint64_t n);
void uncount_launches(uint64_t n);   // kernels recorded into a graph, not run
uint64_t launches_so_far();
uint64_t thread_launches();   // this thread's share of launches_so_far()

#define CBS_STR2(x) #x
#define CBS_STR(x) CBS_STR2(x)
#define CBS_CUDA(call)                                                               \
  do {                                                                               \
    cudaError_t _e = (call);                                                         \
    if (_e != cudaSuccess) return cbs::cuda_fail(_e, __FILE__ ":" CBS_STR(__LINE__) ": " #call); \
  } while (0)

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Thread-block shape for [N][L] blocks: x = columns, y = point lanes.
inline dim3 col_block(int L) {
  int py = 256 / L;
  if (py < 1) py = 1;
  return dim3((unsigned)L, (unsigned)py, 1);
}

// ---------------------------------------------------------------- kernels (launchers)
// apply.cu
template <typename R>
cbs_status launch_proj_gather(const HamView &H, int n_sys, int L, const typename CT<R>::T *X,
                              const double2 *twist, bool per_col, typename CT<R>::T *D,
                              const int *sys_active, cudaStream_t st);
template <typename R>
cbs_status launch_apply(const HamView &H, int n_sys, int L, const typename CT<R>::T *X,
                        typename CT<R>::T *Y, const double2 *twist, bool per_col,
                        const double *E, const typename CT<R>::T *D, const int *sys_active,
                        cudaStream_t st);
// Whether the operator apply supports L columns of element type dtype on this cell:
// complex128 up to 256 columns; complex64 up to 256, or up to 512 with an even L and at
// most 4 projectors (two columns per thread).  Sets the error message when it does not.
bool apply_supported(const HamView &H, int L, int dtype, const char *who);
// Y = P(w) X for n_sys systems; D is scratch of n_sys*n_atoms*np4*L elements
template <typename R>
cbs_status apply_P(const HamView &H, int n_sys, int L, const typename CT<R>::T *X,
                   typename CT<R>::T *Y, const double2 *twist, bool per_col, const double *E,
                   typename CT<R>::T *D, const int *sys_active, cudaStream_t st);

}  // namespace cbs
