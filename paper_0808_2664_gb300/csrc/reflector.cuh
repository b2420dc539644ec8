// Householder reflector generation shared by the leaf and tree-node kernels.
#pragma once

#include <cuda_runtime.h>

#include "tsqr_internal.cuh"

namespace tsqr {

// H = I - tau u u^T with the topmost entry of u equal to one (Section 4, the
// conventional normalisation of Householder vectors).  For x = [alpha; t],
// beta = -sign(alpha) ||x||, tau = (beta - alpha) / beta and
// u = [1; t * scale] with scale = 1 / (alpha - beta); alpha - beta never
// cancels.  A tail that is exactly zero gives tau = 0 (H = I), beta = alpha.
struct Reflector {
  double tau;
  double scale;
  double beta;
};

// ssq is the plain sum of squares of the tail.  When it may have overflowed
// or underflowed (or is zero, which may be an underflow of tiny entries), the
// tail is rescanned with scaling by `rescan`, which returns ||t||_2 computed
// as max|t_i| * sqrt(sum (t_i / max|t_i|)^2), or NaN if some entry is NaN.
template <class Rescan>
__device__ __forceinline__ Reflector make_reflector(double alpha, double ssq, Rescan rescan, int* status) {
  Reflector r;
  const double aa = fabs(alpha);
  double nrm;
  bool zero_tail = false;
  if (ssq >= 1e-290 && ssq <= 1e290 && aa <= 1e145) {
    nrm = sqrt(fma(alpha, alpha, ssq));
  } else {
    const double xn = rescan();
    if (xn == 0.0) {
      zero_tail = true;
      nrm = 0.0;
    } else {
      const double t = fmax(aa, xn);
      const double x = aa / t, y = xn / t;
      nrm = t * sqrt(x * x + y * y);
      if (xn != xn || alpha != alpha) nrm = xn + alpha;  // propagate NaN
    }
  }
  if (zero_tail) {
    r.tau = 0.0;
    r.scale = 0.0;
    r.beta = alpha;
  } else {
    r.beta = alpha >= 0.0 ? -nrm : nrm;
    r.tau = (r.beta - alpha) / r.beta;
    r.scale = 1.0 / (alpha - r.beta);
  }
  if (!isfinite(r.beta) || !isfinite(r.tau) || !isfinite(alpha)) atomicOr(status, kStatusNonfinite);
  return r;
}

// Scaled 2-norm over a strided sequence produced by `get(i)`, i in [0, len).
template <class Get>
__device__ __forceinline__ double scaled_norm(int len, Get get) {
  double mx = 0.0;
  bool nan = false;
  for (int i = 0; i < len; ++i) {
    const double a = fabs(get(i));
    if (a != a) nan = true;
    else if (a > mx) mx = a;
  }
  if (nan) return __longlong_as_double(0x7ff8000000000000ll);
  if (mx == 0.0 || isinf(mx)) return mx;
  double s = 0.0;
  for (int i = 0; i < len; ++i) {
    const double t = get(i) / mx;
    s = fma(t, t, s);
  }
  return mx * sqrt(s);
}

__device__ __forceinline__ int pow2_floor(int x) { return x <= 1 ? 1 : 1 << (31 - __clz(x)); }

// Build the compact-WY T (upper triangular, n x n, column-major ld n, in
// FP64 shared memory) from tau and the strictly upper part of Y^T Y, which
// the caller has stored in Tm(p, j) for p < j.  Forward recurrence of
// Schreiber and Van Loan (cited in Section 2.1):
//   T(j, j) = tau_j,   T(0:j, j) = -tau_j T(0:j, 0:j) (Y(:, 0:j)^T y_j).
// Every thread of the block calls this.
__device__ __forceinline__ void build_t(double* Tm, const double* tau, int n) {
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int p = idx % n, j = idx / n;
    if (p == j) Tm[idx] = tau[j];
    else if (p > j) Tm[idx] = 0.0;
  }
  __syncthreads();
  for (int j = 1; j < n; ++j) {
    double s = 0.0;
    const int p = threadIdx.x;
    if (p < j) {
      for (int q = p; q < j; ++q) s = fma(Tm[p + q * n], Tm[q + j * n], s);
    }
    __syncthreads();
    if (p < j) Tm[p + j * n] = -tau[j] * s;
    __syncthreads();
  }
}

}  // namespace tsqr
