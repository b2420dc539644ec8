// Least squares through TSQR.  Section 1 names the tall-skinny least squares
// problem min ||A x - b||_2 as the first use of TSQR: with A = Q R and the
// square Q kept as its tree of factors, Q^T b splits into the part the
// solution needs and the part orthogonal to range(A),
//     x = R^{-1} (Q^T b)(0:n),     ||A x - b||_2 = ||(Q^T b)(n:m)||_2,
// and the paper notes the R-only variant: factor [A, B] and read the
// solution off its R = [R11, R12; 0, R22] (x = R11^{-1} R12, residual norms
// = column norms of R22).  Both need an upper-triangular solve on the device
// and column norms; Q^T B itself is tsqr_apply_qt.
//
// Kernels:
//   solve_upper_kernel  X = R^{-1} B (n <= 128): one warp per column of B;
//                       lane l holds rows l, l+32, l+64, l+96 in registers;
//                       back substitution with an IEEE division by R(j, j)
//                       and a shuffle broadcast of x_j per step; a zero or
//                       non-finite diagonal entry latches the status word.
//   colnorm_kernel      FP64 sums of squares of rows [r0, m) of each column,
//                       a grid over (row chunks, columns), atomically added;
//   sqrt_kernel         the norms.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/tsqr.h"
#include "tsqr_internal.cuh"

namespace tsqr {
namespace {

constexpr int kSolveWarps = 4;
constexpr int kNormThreads = 256;
constexpr int kNormRows = 8192;  // rows per CTA of the norm kernel

template <typename T>
__global__ void __launch_bounds__(32 * kSolveWarps) solve_upper_kernel(int n, int64_t k, const T* R, int64_t ldr,
                                                                       const T* B, int64_t ldb, T* X, int64_t ldx,
                                                                       int* status) {
  const int lane = threadIdx.x & 31;
  const int64_t col = (int64_t)blockIdx.x * kSolveWarps + (threadIdx.x >> 5);
  if (col >= k) return;
  const T* b = B + col * ldb;
  T v[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int i = lane + 32 * t;
    v[t] = i < n ? b[i] : T(0);
  }
  bool bad = false;
  for (int j = n - 1; j >= 0; --j) {
    const int slot = j >> 5, owner = j & 31;
    T bj = v[0];
#pragma unroll
    for (int t = 1; t < 4; ++t)
      if (slot == t) bj = v[t];
    T xj = T(0);
    if (lane == owner) {
      const T d = R[j + (int64_t)j * ldr];
      if (!(d != T(0)) || !isfinite((double)d)) bad = true;
      xj = bj / d;
    }
    xj = __shfl_sync(0xffffffffu, xj, owner);
    // Row j itself now holds x_j; rows i < j lose R(i, j) x_j.
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int i = lane + 32 * t;
      if (i == j) v[t] = xj;
      else if (i < j) v[t] = fma(-R[i + (int64_t)j * ldr], xj, v[t]);
    }
  }
  T* x = X + col * ldx;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int i = lane + 32 * t;
    if (i < n) x[i] = v[t];
  }
  if (bad && status) atomicOr(status, kStatusNonfinite);
}

template <typename T>
__global__ void __launch_bounds__(kNormThreads) colnorm_kernel(int64_t r0, int64_t m, const T* B, int64_t ldb,
                                                               double* acc) {
  __shared__ double red[kNormThreads / 32];
  const int64_t col = blockIdx.y;
  const int64_t a = r0 + (int64_t)blockIdx.x * kNormRows;
  const int64_t e = a + kNormRows < m ? a + kNormRows : m;
  const T* b = B + col * ldb;
  double s = 0.0;
  for (int64_t i = a + threadIdx.x; i < e; i += kNormThreads) {
    const double x = (double)b[i];
    s = fma(x, x, s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kNormThreads / 32; ++w) t += red[w];
    atomicAdd(acc + col, t);
  }
}

template <typename T>
__global__ void sqrt_kernel(int64_t k, const double* acc, T* out) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < k; j += (int64_t)gridDim.x * blockDim.x)
    out[j] = (T)sqrt(acc[j]);
}

}  // namespace

template <typename T>
cudaError_t launch_solve_upper(int n, int64_t k, const T* R, int64_t ldr, const T* B, int64_t ldb, T* X, int64_t ldx,
                               int* status, cudaStream_t s) {
  if (n <= 0 || k <= 0) return cudaSuccess;
  if (n > kMaxN) return cudaErrorInvalidValue;
  const int64_t blocks = (k + kSolveWarps - 1) / kSolveWarps;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  solve_upper_kernel<T><<<(unsigned)blocks, 32 * kSolveWarps, 0, s>>>(n, k, R, ldr, B, ldb, X, ldx, status);
  return cudaGetLastError();
}

// out[j] = ||B(r0:m, j)||_2 for j < k; acc: k doubles of device workspace.
template <typename T>
cudaError_t launch_column_norms(int64_t r0, int64_t m, int64_t k, const T* B, int64_t ldb, double* acc, T* out,
                                cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double) * k, s);
  if (e != cudaSuccess) return e;
  if (m > r0) {
    const int64_t chunks = (m - r0 + kNormRows - 1) / kNormRows;
    if (chunks > 0x7fffffffLL || k > 65535) return cudaErrorInvalidConfiguration;
    colnorm_kernel<T><<<dim3((unsigned)chunks, (unsigned)k), kNormThreads, 0, s>>>(r0, m, B, ldb, acc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const int64_t blocks = (k + 255) / 256 < 1024 ? (k + 255) / 256 : 1024;
  sqrt_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(k, acc, out);
  return cudaGetLastError();
}

template cudaError_t launch_solve_upper<double>(int, int64_t, const double*, int64_t, const double*, int64_t, double*,
                                                int64_t, int*, cudaStream_t);
template cudaError_t launch_solve_upper<float>(int, int64_t, const float*, int64_t, const float*, int64_t, float*,
                                               int64_t, int*, cudaStream_t);
template cudaError_t launch_column_norms<double>(int64_t, int64_t, int64_t, const double*, int64_t, double*, double*,
                                                 cudaStream_t);
template cudaError_t launch_column_norms<float>(int64_t, int64_t, int64_t, const float*, int64_t, double*, float*,
                                                cudaStream_t);

}  // namespace tsqr

using namespace tsqr;

extern "C" int tsqr_solve_r(int64_t n, int64_t k, int32_t precision, const void* R, int64_t ldr, void* X,
                            int64_t ldx, int* status, tsqr_stream_t stream) {
  if (n < 0) return -1;
  if (k < 0) return -2;
  if (precision != TSQR_PREC_FP64 && precision != TSQR_PREC_FP32) return -3;
  if (n == 0 || k == 0) return TSQR_OK;
  if (n > kMaxN) return TSQR_ERR_UNSUPPORTED;
  if (!R) return -4;
  if (ldr < n) return -5;
  if (!X) return -6;
  if (ldx < n) return -7;
  cudaStream_t s = (cudaStream_t)stream;
  const cudaError_t e =
      precision == TSQR_PREC_FP64
          ? launch_solve_upper<double>((int)n, k, (const double*)R, ldr, (const double*)X, ldx, (double*)X, ldx, status, s)
          : launch_solve_upper<float>((int)n, k, (const float*)R, ldr, (const float*)X, ldx, (float*)X, ldx, status, s);
  return e == cudaSuccess ? TSQR_OK : TSQR_ERR_CUDA;
}

extern "C" int tsqr_column_norms(int64_t m, int64_t k, int32_t precision, const void* B, int64_t ldb, void* norms,
                                 tsqr_stream_t stream) {
  if (m < 0) return -1;
  if (k < 0) return -2;
  if (precision != TSQR_PREC_FP64 && precision != TSQR_PREC_FP32) return -3;
  if (k == 0) return TSQR_OK;
  if (!B && m > 0) return -4;
  if (ldb < (m > 1 ? m : 1)) return -5;
  if (!norms) return -6;
  if (k > 65535) return TSQR_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  double* acc = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&acc, sizeof(double) * k, s);
  if (e != cudaSuccess) return TSQR_ERR_NOMEM;
  e = precision == TSQR_PREC_FP64 ? launch_column_norms<double>(0, m, k, (const double*)B, ldb, acc, (double*)norms, s)
                                  : launch_column_norms<float>(0, m, k, (const float*)B, ldb, acc, (float*)norms, s);
  const cudaError_t ef = cudaFreeAsync(acc, s);
  return e == cudaSuccess && ef == cudaSuccess ? TSQR_OK : TSQR_ERR_CUDA;
}
