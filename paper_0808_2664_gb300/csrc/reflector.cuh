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
    // With d = alpha - beta (|d| = |alpha| + nrm, no cancellation) and one
    // reciprocal rp = 1 / (beta d): scale = 1/d = beta rp and
    // tau = (beta - alpha)/beta = -d/beta = -d^2 rp.
    r.beta = alpha >= 0.0 ? -nrm : nrm;
    const double d = alpha - r.beta;
    const double bd = r.beta * d;
    if (isfinite(bd) && fabs(bd) > 1e-300) {
      const double rp = 1.0 / bd;
      r.scale = r.beta * rp;
      r.tau = -(d * d) * rp;
    } else {  // beta d over- or underflows: form the two quotients directly
      r.tau = (r.beta - alpha) / r.beta;
      r.scale = 1.0 / d;
    }
  }
  if (!isfinite(r.beta) || !isfinite(r.tau) || !isfinite(alpha)) atomicOr(status, kStatusNonfinite);
  return r;
}

// The same reflector with a shorter chain of dependent FP64 operations, for
// the serial step of each column.  FP64 arithmetic has a long dependent
// latency on this GPU, and IEEE sqrt and division are long sequences of it;
// here 1/||x|| and 1/|alpha - beta| start from FP32 estimates (rsqrtf and a
// fast FP32 reciprocal, about 22 correct bits) and take one third-order
// correction step each, the series (1 - e)^(-1/2) ~ 1 + e/2 + 3e^2/8 with
// e = 1 - x y^2, and (1 - e)^(-1) ~ 1 + e + e^2 with e = 1 - d y (the
// relative error goes from e to O(e^3)), which brings them to a few FP64
// ulps.  Then
//   ||x|| = x2 * (1/||x||),  tau = 1 + |alpha| / ||x||,
//   scale = sign(alpha) / (|alpha| + ||x||),  beta = -sign(alpha) ||x||,
// the formulas of make_reflector rewritten with those two reciprocals.
// Used only where every quantity stays far inside FP32's range (the tail's
// squared norm in [2^-100, 2^100], |alpha| <= 2^50); otherwise, and for
// zero, non-finite or extreme inputs, make_reflector runs.
template <class Rescan>
__device__ __forceinline__ Reflector make_reflector_fast(double alpha, double ssq, Rescan rescan, int* status) {
  const double aa = fabs(alpha);
  if (!(ssq >= 0x1p-100 && ssq <= 0x1p100 && aa <= 0x1p50)) return make_reflector(alpha, ssq, rescan, status);
  const double x2 = fma(alpha, alpha, ssq);
  const double r0 = (double)rsqrtf((float)x2);
  const double e = fma(-(x2 * r0), r0, 1.0);
  const double r = fma(r0 * e, fma(0.375, e, 0.5), r0);  // 1 / ||x||
  const double nrm = x2 * r;
  const double ad = aa + nrm;  // |alpha - beta|
  const double q0 = (double)__fdividef(1.0f, (float)ad);
  const double f = fma(-ad, q0, 1.0);
  const double q = fma(q0 * f, 1.0 + f, q0);  // 1 / |alpha - beta|
  Reflector out;
  out.beta = alpha >= 0.0 ? -nrm : nrm;
  out.scale = alpha >= 0.0 ? q : -q;
  out.tau = fma(aa, r, 1.0);
  return out;
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

// Layout of T while it is built: column-major with leading dimension n + 1,
// so that the lanes of a warp walking along a row of T hit different shared
// memory banks; the doubling workspace pads its b x b blocks likewise.
__host__ __device__ inline int t_ld(int n) { return n + 1; }
__host__ __device__ inline size_t t_work_elems(int n) {
  size_t m = 1;
  for (int b = 1; b < n; b *= 2) {
    const size_t v = (size_t)((n + 2 * b - 1) / (2 * b)) * b * (b + 1);
    if (v > m) m = v;
  }
  return m;
}

// Build the compact-WY T (upper triangular, n x n, shared memory, in the
// product type T) of `count` reflector sets at once, in place: set g has
// its T at Tm0 + g * tm_stride (leading dimension t_ld(n)) and workspace at
// Wt0 + g * wt_stride (t_work_elems(n) entries).  On entry T holds tau on the
// diagonal, the strictly upper part of Y^T Y above it (T(p, q) = y_p^T y_q)
// and zeros below.  Schreiber and Van Loan (cited in Section 2.1) give, for
// two blocks of reflectors, I - Y T Y^T with T = [T1, -T1 (Y1^T Y2) T2; 0,
// T2]; applying that merge to aligned blocks of 1, 2, 4, ... columns builds
// T in log2(n) levels of independent triangular products.  Every thread of
// the block calls this.
template <typename T>
__device__ __forceinline__ void build_t_doubling_many(T* Tm0, size_t tm_stride, T* Wt0, size_t wt_stride, int count,
                                                      int n) {
  const int L = t_ld(n);
  for (int b = 1; b < n; b *= 2) {
    const int npairs = (n + 2 * b - 1) / (2 * b);
    const int bb = b * b, bs = b * (b + 1);
    const int per = npairs * bb;
    // Pass 1: W = Z12 T2 for every pair, W(p - s, q - s - b) at pl + ql (b + 1).
    for (int idx = threadIdx.x; idx < count * per; idx += blockDim.x) {
      const int g = idx / per, r0 = idx - g * per;
      const int pair = r0 / bb, rem = r0 - pair * bb;
      const int pl = rem % b, ql = rem / b;
      const int s = pair * 2 * b, p = s + pl, q = s + b + ql;
      if (q >= n) continue;
      const T* Tm = Tm0 + g * tm_stride;
      T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
      int r = s + b;
      for (; r + 3 <= q; r += 4) {
        a0 = fma(Tm[p + r * L], Tm[r + q * L], a0);
        a1 = fma(Tm[p + (r + 1) * L], Tm[r + 1 + q * L], a1);
        a2 = fma(Tm[p + (r + 2) * L], Tm[r + 2 + q * L], a2);
        a3 = fma(Tm[p + (r + 3) * L], Tm[r + 3 + q * L], a3);
      }
      for (; r <= q; ++r) a0 = fma(Tm[p + r * L], Tm[r + q * L], a0);
      Wt0[g * wt_stride + pair * bs + pl + ql * (b + 1)] = (a0 + a1) + (a2 + a3);
    }
    __syncthreads();
    // Pass 2: T12 = -T1 W; the lanes of a warp share p, so their sums have
    // the same length.
    for (int idx = threadIdx.x; idx < count * per; idx += blockDim.x) {
      const int g = idx / per, r0 = idx - g * per;
      const int pair = r0 / bb, rem = r0 - pair * bb;
      const int ql = rem % b, pl = rem / b;
      const int s = pair * 2 * b, p = s + pl, q = s + b + ql;
      if (q >= n) continue;
      T* Tm = Tm0 + g * tm_stride;
      const T* w = Wt0 + g * wt_stride + pair * bs + ql * (b + 1) - s;
      T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
      int r = p;
      for (; r + 3 < s + b; r += 4) {
        a0 = fma(Tm[p + r * L], w[r], a0);
        a1 = fma(Tm[p + (r + 1) * L], w[r + 1], a1);
        a2 = fma(Tm[p + (r + 2) * L], w[r + 2], a2);
        a3 = fma(Tm[p + (r + 3) * L], w[r + 3], a3);
      }
      for (; r < s + b; ++r) a0 = fma(Tm[p + r * L], w[r], a0);
      Tm[p + q * L] = -((a0 + a1) + (a2 + a3));
    }
    __syncthreads();
  }
}

// One reflector set: T at Tm (leading dimension t_ld(n)), workspace at Wt.
template <typename T>
__device__ __forceinline__ void build_t_doubling(T* Tm, T* Wt, int n) {
  build_t_doubling_many(Tm, 0, Wt, 0, 1, n);
}

}  // namespace tsqr
