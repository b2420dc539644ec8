// Leaf Householder QR of every row block of A (Section 2.1,
// Eq. TSQR_binarytree_1: A_i = Q_i R_i for each block A_i).
//
// One CTA factors one leaf at a time (grid-stride over leaves).  The h x n
// leaf sits in shared memory, column-major with an odd leading dimension so
// that threads walking different columns at the same row hit different
// banks.  The column schedule (leaf_device.cuh): per column, one warp forms
// the reflector while the update warps apply the previous reflector to every
// trailing column fused with that column's dot against the new tail; a short
// coefficient step and a single-column step follow; a separate group of
// warps accumulates Z = strictly-upper(Y^T Y) as the tails become final.
// After the last column the leaf's compact-WY T is built from Z and tau by a
// blocked doubling recurrence.  Arithmetic: products in the storage type T
// (FP64, or FP32 for the mixed form); norms, beta, tau and scale in FP64.
#include <cuda_runtime.h>

#include "leaf_device.cuh"
#include "tsqr_internal.cuh"

namespace tsqr {
namespace {

// FP32 leaves are latency-bound and rely on two or more CTAs per SM to
// overlap their column chains, so their register budget is held to 1024
// threads' worth per SM (64 registers a thread).
template <typename T, int NT, int NMAX>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 1024 / NT : 1) leaf_factor_kernel(LeafFactorArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int64_t nn = (int64_t)a.n * a.n;
  for (int64_t leaf = blockIdx.x; leaf < a.nleaves; leaf += gridDim.x) {
    const int64_t r0 = leaf * a.h;
    const int hl = (leaf == a.nleaves - 1) ? (int)(a.m - r0) : (int)a.h;
    leaf_factor_one<T, NT, NMAX>(a.A + r0, a.lda, hl, a.n, a.ld_s, a.R + leaf * nn, a.tau + leaf * (int64_t)a.n,
                                 a.Tw + leaf * nn, a.status, smem, nullptr, a.Asrc ? a.Asrc + r0 : nullptr,
                                 a.ldsrc);
  }
}

}  // namespace

int leaf_factor_ld(int hmax) { return hmax | 1; }

// Threads per leaf CTA: FP64 leaves use 128 when three tiles share an SM and
// 512 when a tile is so tall that only one CTA fits; FP32 leaves use 256, and
// 512 for tiles above 80 KB (two such CTAs per SM: 384 rows at n = 64 went
// from 12.6 to 11.4 ms at 4,194,304 rows; 256-row tiles lose with 512).
int leaf_factor_threads(int n, int ld, size_t elem) {
  if (leaf_tile_region(n, ld, elem) > (elem == 4 ? 80 : 100) * 1024) return kLeafThreadsBig;
  return elem == 4 ? kLeafThreads32 : kLeafThreads64;
}

size_t leaf_factor_smem(int n, int hmax, size_t elem) {
  const int ld = leaf_factor_ld(hmax);
  return leaf_smem_bytes(n, ld, elem, leaf_factor_threads(n, ld, elem));
}

template <typename T, int NT>
cudaError_t launch_leaf_factor_nt(const LeafFactorArgs<T>& a, cudaStream_t s) {
  const size_t smem = leaf_smem_bytes(a.n, a.ld_s, sizeof(T), NT);
  auto kern = a.n <= 64 ? leaf_factor_kernel<T, NT, 64> : leaf_factor_kernel<T, NT, kMaxN>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int64_t grid = (int64_t)sms * per_sm;
  if (grid > a.nleaves) grid = a.nleaves;
  kern<<<(unsigned)grid, NT, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_leaf_factor(const LeafFactorArgs<T>& a, cudaStream_t s) {
  if (a.nleaves <= 0 || a.n <= 0) return cudaSuccess;
  const int nt = leaf_factor_threads(a.n, a.ld_s, sizeof(T));
  if (nt == kLeafThreadsBig) return launch_leaf_factor_nt<T, kLeafThreadsBig>(a, s);
  return nt == 256 ? launch_leaf_factor_nt<T, 256>(a, s) : launch_leaf_factor_nt<T, 128>(a, s);
}

template cudaError_t launch_leaf_factor<double>(const LeafFactorArgs<double>&, cudaStream_t);
template cudaError_t launch_leaf_factor<float>(const LeafFactorArgs<float>&, cudaStream_t);

}  // namespace tsqr
