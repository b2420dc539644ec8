// Leaf Householder QR of every row block of A (Section 2.1,
// Eq. TSQR_binarytree_1: A_i = Q_i R_i for each block A_i).
//
// One CTA factors one leaf at a time (grid-stride over leaves).  The h x n
// leaf sits in shared memory, column-major with an odd leading dimension so
// that threads walking different columns at the same row hit different banks.
// Per column j the CTA runs four phases separated by barriers:
//   C  thread 0 turns (alpha, ||tail||^2) into (beta, tau, scale);
//   S  the tail of column j is scaled into the Householder vector u_j;
//   A  dot products of u_j with every other column: w_c = u_j^T a_c for c > j
//      (the trailing update) and z_p = y_p^T u_j for p < j (the compact-WY T),
//      rows split into groups whose partial sums meet by warp shuffles;
//   B  a_c -= tau_j w_c u_j for c > j, and the squared norm of the next
//      column's tail, accumulated while it is being updated.
// Work is re-partitioned over all threads in every phase, so the shrinking
// active block keeps the FP64 pipe busy.  Arithmetic: products in T (FP64, or
// FP32 for the mixed form); norms, beta, tau and scale always in FP64.
#include <cuda_runtime.h>

#include "reflector.cuh"
#include "tsqr_internal.cuh"

namespace tsqr {
namespace {

constexpr int kMinRows = 8;

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

template <typename T, int NT>
__global__ void __launch_bounds__(NT) leaf_factor_kernel(LeafFactorArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = a.n;
  const int ld = a.ld_s;
  const int hmax_tile = ld;
  T* S = reinterpret_cast<T*>(smem);
  size_t off = align_up(sizeof(T) * (size_t)n * hmax_tile, 16);
  off = off > sizeof(double) * (size_t)n * n ? off : align_up(sizeof(double) * (size_t)n * n, 16);
  double* part = reinterpret_cast<double*>(smem + off);  // NT partial dot products
  double* nrm_part = part + NT;                           // NT partial squared norms
  double* tau_s = nrm_part + NT;                          // n reflector scalars
  double* Tm = reinterpret_cast<double*>(smem);           // reuses the tile after write-back
  __shared__ double sh_scale;
  __shared__ int sh_nrg;
  const int tid = threadIdx.x;
  const int lane = tid & 31;

  for (int64_t leaf = blockIdx.x; leaf < a.nleaves; leaf += gridDim.x) {
    const int64_t r0 = leaf * a.h;
    const int hl = (leaf == a.nleaves - 1) ? (int)(a.m - r0) : (int)a.h;
    T* Ag = a.A + r0;
    for (int c = 0; c < n; ++c) {
      const T* src = Ag + (int64_t)c * a.lda;
      for (int i = tid; i < hl; i += NT) S[c * ld + i] = src[i];
    }
    __syncthreads();
    {
      double s = 0.0;
      for (int i = 1 + tid; i < hl; i += NT) {
        const double x = (double)S[i];
        s = fma(x, x, s);
      }
      nrm_part[tid] = s;
      if (tid == 0) sh_nrg = NT;
    }
    __syncthreads();

    for (int j = 0; j < n; ++j) {
      // Phase C: reflector scalars for column j.
      if (tid == 0) {
        double ssq = 0.0;
        for (int g = 0; g < sh_nrg; ++g) ssq += nrm_part[g];
        const T* col = S + j * ld;
        const double alpha = (double)col[j];
        const int len = hl - j - 1;
        Reflector r = make_reflector(alpha, ssq,
                                     [&]() { return scaled_norm(len, [&](int i) { return (double)col[j + 1 + i]; }); },
                                     a.status);
        tau_s[j] = r.tau;
        sh_scale = r.scale;
        S[j * ld + j] = (T)r.beta;
      }
      __syncthreads();
      // Phase S: the tail of column j becomes u_j (unit entry implicit).
      {
        const double scale = sh_scale;
        T* col = S + j * ld;
        for (int i = j + 1 + tid; i < hl; i += NT) col[i] = (T)((double)col[i] * scale);
      }
      __syncthreads();
      const int rows = hl - j;  // rows j .. hl-1
      // Phase A: u_j^T a_c for every c != j.
      const int acols = n - 1;
      int rga = 1;
      if (acols > 0) {
        int lim = NT / acols;
        int byrows = rows / kMinRows;
        if (byrows < 1) byrows = 1;
        if (lim > byrows) lim = byrows;
        if (lim > 32) lim = 32;
        rga = pow2_floor(lim < 1 ? 1 : lim);
        int chunk = (rows + rga - 1) / rga;
        chunk |= 1;  // odd stride between the row groups of one warp
        const int slot = tid / rga, g = tid % rga;
        T s = T(0);
        if (slot < acols) {
          const int c = slot < j ? slot : slot + 1;
          const T* u = S + j * ld;
          const T* cc = S + c * ld;
          int i = j + g * chunk;
          const int i1 = min(i + chunk, hl);
          if (i == j && i < i1) {
            s = cc[j];
            ++i;
          }
          for (; i < i1; ++i) s = fma(u[i], cc[i], s);
        }
        // Reduce over the rga row groups of each slot (consecutive lanes).
        for (int o = rga >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (slot < acols && g == 0) part[slot] = (double)s;
        (void)lane;
      }
      __syncthreads();
      // Phase B: z for columns p < j (to the T buffer), updates for c > j.
      if (tid < j) a.Tw[leaf * (int64_t)n * n + tid + (int64_t)j * n] = (T)part[tid];
      const int bcols = n - 1 - j;
      if (bcols > 0) {
        int rgb = NT / bcols;
        int byrows = rows / kMinRows;
        if (byrows < 1) byrows = 1;
        if (rgb > byrows) rgb = byrows;
        if (rgb < 1) rgb = 1;
        const int chunk = (rows + rgb - 1) / rgb;
        const int slot = tid % bcols, g = tid / bcols;
        if (g < rgb) {
          const int c = j + 1 + slot;
          const double w = part[c - 1];
          const T coef = (T)(tau_s[j] * w);
          const T* u = S + j * ld;
          T* cc = S + c * ld;
          int i = j + g * chunk;
          const int i1 = min(i + chunk, hl);
          double ssq = 0.0;
          if (i == j && i < i1) {
            cc[j] -= coef;
            ++i;
          }
          if (slot == 0) {
            for (; i < i1; ++i) {
              const T x = cc[i] - coef * u[i];
              cc[i] = x;
              if (i > j + 1) ssq = fma((double)x, (double)x, ssq);
            }
            nrm_part[g] = ssq;
          } else {
            for (; i < i1; ++i) cc[i] -= coef * u[i];
          }
        }
        if (tid == 0) sh_nrg = rgb;
      }
      __syncthreads();
    }

    // Write back Y (below the diagonal) and R_i (on and above) in place, the
    // leaf R factor to the tree's level-0 items, and tau.
    for (int c = 0; c < n; ++c) {
      T* dst = Ag + (int64_t)c * a.lda;
      for (int i = tid; i < hl; i += NT) dst[i] = S[c * ld + i];
    }
    T* Rl = a.R + leaf * (int64_t)n * n;
    for (int idx = tid; idx < n * n; idx += NT) {
      const int i = idx % n, c = idx / n;
      Rl[idx] = i <= c ? S[c * ld + i] : T(0);
    }
    for (int c = tid; c < n; c += NT) a.tau[leaf * (int64_t)n + c] = (T)tau_s[c];
    __syncthreads();
    // Compact-WY T from the z values stored in the T buffer.
    T* Tg = a.Tw + leaf * (int64_t)n * n;
    for (int idx = tid; idx < n * n; idx += NT) {
      const int p = idx % n, jj = idx / n;
      Tm[idx] = p < jj ? (double)Tg[idx] : 0.0;
    }
    __syncthreads();
    build_t(Tm, tau_s, n);
    for (int idx = tid; idx < n * n; idx += NT) Tg[idx] = (T)Tm[idx];
    __syncthreads();
  }
}

}  // namespace

int leaf_factor_ld(int hmax) { return hmax | 1; }

size_t leaf_factor_smem(int n, int hmax, size_t elem) {
  const int ld = leaf_factor_ld(hmax);
  size_t tile = align_up(elem * (size_t)n * ld, 16);
  const size_t tm = align_up(sizeof(double) * (size_t)n * n, 16);
  if (tm > tile) tile = tm;
  return tile + sizeof(double) * (2 * kLeafThreads + (size_t)n);
}

template <typename T>
cudaError_t launch_leaf_factor(const LeafFactorArgs<T>& a, cudaStream_t s) {
  if (a.nleaves <= 0 || a.n <= 0) return cudaSuccess;
  const int hmax = a.ld_s;
  const size_t smem = leaf_factor_smem(a.n, hmax, sizeof(T));
  auto kern = leaf_factor_kernel<T, kLeafThreads>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kLeafThreads, smem);
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int64_t grid = (int64_t)sms * per_sm;
  if (grid > a.nleaves) grid = a.nleaves;
  kern<<<(unsigned)grid, kLeafThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_leaf_factor<double>(const LeafFactorArgs<double>&, cudaStream_t);
template cudaError_t launch_leaf_factor<float>(const LeafFactorArgs<float>&, cudaStream_t);

}  // namespace tsqr
