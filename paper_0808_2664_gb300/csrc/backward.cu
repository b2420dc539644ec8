// Adjoint of the thin QR A = Q R with diag(R) > 0 (a training-system add-on;
// the paper has no gradient):
//   M  = R dR^T - dQ^T Q,      S = copyltu(M) = tril(M) + tril(M, -1)^T,
//   dA = (dQ + Q S) R^{-T}.
// On the device this is three launches:
//   gram_kernel   G_p = dQ_p^T Q_p for row chunks p (4x4 register tiles);
//   small_kernel  G = sum_p G_p in a fixed order, M, S, Rinv = R^{-1} (column
//                 by column back substitution), and Z = [Rinv^T; S Rinv^T];
//   rows_kernel   dA = [dQ, Q] Z, a row-parallel product with K = 2n,
// which computes (dQ + Q S) R^{-T} = dQ R^{-T} + Q (S R^{-T}).
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/tsqr.h"
#include "tsqr_internal.cuh"

namespace tsqr {
namespace {

constexpr int kGT = 64;      // output tile edge of the Gram and row products
constexpr int kGRows = 32;   // rows staged per pass
constexpr int kBwdThreads = 256;

// Partial Gram matrices: Gp[p] (n x n, ld n) = sum over rows of chunk p of
// dQ(r, :)^T Q(r, :).  Grid: (chunks, tiles_i, tiles_j).
template <typename T>
__global__ void __launch_bounds__(kBwdThreads) gram_kernel(int64_t m, int n, const T* dQ, int64_t lddq, const T* Q,
                                                           int64_t ldq, int64_t chunk, T* Gp) {
  __shared__ T As[kGRows][kGT + 1];
  __shared__ T Bs[kGRows][kGT + 1];
  const int tid = threadIdx.x;
  const int64_t r0 = blockIdx.x * chunk;
  const int64_t r1 = r0 + chunk < m ? r0 + chunk : m;
  const int i0 = blockIdx.y * kGT, j0 = blockIdx.z * kGT;
  const int ti = (tid % 16) * 4, tj = (tid / 16) * 4;
  T acc[4][4] = {};
  for (int64_t rb = r0; rb < r1; rb += kGRows) {
    __syncthreads();
    for (int idx = tid; idx < kGRows * kGT; idx += kBwdThreads) {
      const int rr = idx % kGRows, c = idx / kGRows;
      const int64_t r = rb + rr;
      As[rr][c] = (r < r1 && i0 + c < n) ? dQ[r + (int64_t)(i0 + c) * lddq] : T(0);
      Bs[rr][c] = (r < r1 && j0 + c < n) ? Q[r + (int64_t)(j0 + c) * ldq] : T(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < kGRows; ++rr) {
      T a[4], b[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) a[x] = As[rr][ti + x];
#pragma unroll
      for (int y = 0; y < 4; ++y) b[y] = Bs[rr][tj + y];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
    }
  }
  T* G = Gp + (int64_t)blockIdx.x * n * n;
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int i = i0 + ti + x, j = j0 + tj + y;
      if (i < n && j < n) G[i + (int64_t)j * n] = acc[x][y];
    }
}

// One CTA: the n x n algebra.  Z (2n x n, ld 2n): rows 0..n-1 = Rinv^T,
// rows n..2n-1 = S Rinv^T.  Work buffers in global memory (wk, 3 n x n).
template <typename T>
__global__ void __launch_bounds__(kBwdThreads) small_kernel(int n, int64_t nparts, const T* Gp, const T* R, int64_t ldr,
                                                            const T* dR, int64_t lddr, T* wk, T* Z, int* status) {
  const int tid = threadIdx.x;
  const int64_t nn = (int64_t)n * n;
  T* S = wk;            // n x n
  T* Ri = wk + nn;      // n x n, R^{-1}
  // M = R dR^T - sum_p Gp, then S = copyltu(M).
  for (int64_t idx = tid; idx < nn; idx += kBwdThreads) {
    const int i = (int)(idx % n), j = (int)(idx / n);
    if (i < j) continue;  // only the lower triangle of M is needed
    T g = T(0);
    for (int64_t p = 0; p < nparts; ++p) g += Gp[p * nn + idx];
    T a = T(0);  // (R dR^T)_ij = sum_k R(i, k) dR(j, k), k >= max(i, j) (both upper)
    for (int k = i; k < n; ++k) a = fma(R[i + (int64_t)k * ldr], dR[j + (int64_t)k * lddr], a);
    const T mij = a - g;
    S[i + (int64_t)j * n] = mij;
    S[j + (int64_t)i * n] = mij;
  }
  // Rinv = R^{-1}, one column per thread: R x = e_j by back substitution.
  for (int j = tid; j < n; j += kBwdThreads) {
    for (int i = 0; i < n; ++i) Ri[i + (int64_t)j * n] = T(0);
    const T rjj = R[j + (int64_t)j * ldr];
    if (status && (!(rjj != T(0)) || !isfinite((double)rjj))) atomicOr(status, kStatusNonfinite);
    Ri[j + (int64_t)j * n] = T(1) / rjj;
    for (int i = j - 1; i >= 0; --i) {
      T s = T(0);
      for (int k = i + 1; k <= j; ++k) s = fma(R[i + (int64_t)k * ldr], Ri[k + (int64_t)j * n], s);
      Ri[i + (int64_t)j * n] = -s / R[i + (int64_t)i * ldr];
    }
  }
  __syncthreads();
  // Z(0:n, :) = Rinv^T; Z(n:2n, :) = S Rinv^T, (S Rinv^T)(i, j) = sum_{k >= j} S(i, k) Rinv(j, k).
  const int64_t ldz = 2 * (int64_t)n;
  for (int64_t idx = tid; idx < nn; idx += kBwdThreads) {
    const int i = (int)(idx % n), j = (int)(idx / n);
    Z[i + (int64_t)j * ldz] = Ri[j + (int64_t)i * n];
    T w = T(0);
    for (int k = j; k < n; ++k) w = fma(S[i + (int64_t)k * n], Ri[j + (int64_t)k * n], w);
    Z[n + i + (int64_t)j * ldz] = w;
  }
}

// dA = [dQ, Q] Z for a 64-row x 64-column output tile per CTA; K = 2n.
template <typename T>
__global__ void __launch_bounds__(kBwdThreads) rows_kernel(int64_t m, int n, const T* dQ, int64_t lddq, const T* Q,
                                                           int64_t ldq, const T* Z, T* dA, int64_t ldda) {
  __shared__ T As[kGT][kGRows + 1];  // 64 rows x 32 k
  __shared__ T Bs[kGRows][kGT + 1];  // 32 k x 64 cols
  const int tid = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * kGT;
  const int j0 = blockIdx.y * kGT;
  const int ti = (tid % 16) * 4, tj = (tid / 16) * 4;
  const int64_t ldz = 2 * (int64_t)n;
  T acc[4][4] = {};
  for (int k0 = 0; k0 < 2 * n; k0 += kGRows) {
    __syncthreads();
    for (int idx = tid; idx < kGT * kGRows; idx += kBwdThreads) {
      const int rr = idx % kGT, kk = idx / kGT;
      const int64_t r = r0 + rr;
      const int k = k0 + kk;
      T v = T(0);
      if (r < m && k < 2 * n) v = k < n ? dQ[r + (int64_t)k * lddq] : Q[r + (int64_t)(k - n) * ldq];
      As[rr][kk] = v;
    }
    for (int idx = tid; idx < kGRows * kGT; idx += kBwdThreads) {
      const int kk = idx % kGRows, c = idx / kGRows;
      const int k = k0 + kk;
      Bs[kk][c] = (k < 2 * n && j0 + c < n) ? Z[k + (int64_t)(j0 + c) * ldz] : T(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kGRows; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) a[x] = As[ti + x][kk];
#pragma unroll
      for (int y = 0; y < 4; ++y) b[y] = Bs[kk][tj + y];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
    }
  }
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int64_t r = r0 + ti + x;
      const int j = j0 + tj + y;
      if (r < m && j < n) dA[r + (int64_t)j * ldda] = acc[x][y];
    }
}

template <typename T>
int backward_impl(int64_t m, int64_t n, const T* Q, int64_t ldq, const T* R, int64_t ldr, const T* dQ, int64_t lddq,
                  const T* dR, int64_t lddr, T* dA, int64_t ldda, int* status, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int tiles = (int)((n + kGT - 1) / kGT);
  int64_t parts = 2 * (int64_t)sms / (tiles * tiles);
  if (parts < 1) parts = 1;
  int64_t chunk = (m + parts - 1) / parts;
  chunk = (chunk + kGRows - 1) / kGRows * kGRows;
  parts = (m + chunk - 1) / chunk;
  const int64_t nn = n * n;
  const size_t bytes = sizeof(T) * (size_t)(parts * nn + 3 * nn + 2 * nn);
  void* ws = nullptr;
  if (cudaMallocAsync(&ws, bytes, s) != cudaSuccess) return TSQR_ERR_NOMEM;
  T* Gp = (T*)ws;
  T* wk = Gp + parts * nn;
  T* Z = wk + 3 * nn;
  dim3 g1((unsigned)parts, tiles, tiles);
  gram_kernel<T><<<g1, kBwdThreads, 0, s>>>(m, (int)n, dQ, lddq, Q, ldq, chunk, Gp);
  small_kernel<T><<<1, kBwdThreads, 0, s>>>((int)n, parts, Gp, R, ldr, dR, lddr, wk, Z, status);
  dim3 g3((unsigned)((m + kGT - 1) / kGT), tiles);
  rows_kernel<T><<<g3, kBwdThreads, 0, s>>>(m, (int)n, dQ, lddq, Q, ldq, Z, dA, ldda);
  const cudaError_t e = cudaGetLastError();
  cudaFreeAsync(ws, s);
  return e == cudaSuccess ? TSQR_OK : TSQR_ERR_CUDA;
}

}  // namespace
}  // namespace tsqr

extern "C" int tsqr_qr_backward(int64_t m, int64_t n, int32_t precision, const void* Q, int64_t ldq, const void* R,
                                int64_t ldr, const void* dQ, int64_t lddq, const void* dR, int64_t lddr, void* dA,
                                int64_t ldda, int* status, tsqr_stream_t stream) {
  if (m < 0) return -1;
  if (n < 0 || n > m) return -2;
  if (precision != TSQR_PREC_FP64 && precision != TSQR_PREC_FP32) return -3;
  if (m == 0 || n == 0) return TSQR_OK;
  if (!Q) return -4;
  if (ldq < m) return -5;
  if (!R) return -6;
  if (ldr < n) return -7;
  if (!dQ) return -8;
  if (lddq < m) return -9;
  if (!dR) return -10;
  if (lddr < n) return -11;
  if (!dA) return -12;
  if (ldda < m) return -13;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == TSQR_PREC_FP64)
    return tsqr::backward_impl<double>(m, n, (const double*)Q, ldq, (const double*)R, ldr, (const double*)dQ, lddq,
                                       (const double*)dR, lddr, (double*)dA, ldda, status, s);
  return tsqr::backward_impl<float>(m, n, (const float*)Q, ldq, (const float*)R, ldr, (const float*)dQ, lddq,
                                    (const float*)dR, lddr, (float*)dA, ldda, status, s);
}
