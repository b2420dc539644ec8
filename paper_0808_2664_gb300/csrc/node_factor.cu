// Tree-node QR of q stacked upper triangles [R_0; R_1; ...; R_{q-1}]
// (Section 2.1, Eqs. TSQR_binarytree_2 and _3; any arity is valid because the
// map from stacked blocks to their R factor is associative up to signs).
//
// The reflector for column j touches row j of R_0 and rows 0..j of every
// other triangle, so its Householder vector is e_j in the top block and an
// upper-triangular column in each lower block; the zeros below the triangles
// are never stored or touched (Section 2.1, the remark on structured local
// QR; 2n^3/3 flops per binary node, Section 2.2).  The resulting Y of a node
// is the q-1 upper triangles that replaced R_1..R_{q-1}.
//
// One CTA per node, triangles in shared memory.  The same C/A/B phases as
// the leaf kernel run over the "virtual rows" of reflector j: row j of block
// 0 followed by rows 0..j of blocks 1..q-1.
#include <cuda_runtime.h>

#include <algorithm>

#include "node2_device.cuh"
#include "node_device.cuh"
#include "tsqr_internal.cuh"

namespace tsqr {
namespace {

template <typename T, int NT>
__global__ void __launch_bounds__(NT) node_factor_kernel(NodeFactorArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = a.n, q = a.arity;
  const int64_t nn = (int64_t)n * n;
  for (int64_t node = blockIdx.x; node < a.nodes; node += gridDim.x) {
    const int64_t c0 = node * q;
    const int nc = (int)((a.nin - c0) < q ? (a.nin - c0) : q);
    node_factor_one<T, NT, true>(a.Rin + c0 * nn, nc, q, n, a.Rout + node * nn,
                                 a.Y + node * (int64_t)(q - 1) * nn, a.Tw + node * nn, a.tau + node * (int64_t)n,
                                 a.status, smem);
  }
}

// Binary levels: G nodes per CTA (node2_device.cuh), grid-stride over groups.
template <typename T, int NT, int G, int Q>
__global__ void __launch_bounds__(NT) node2_factor_kernel(NodeFactorArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int64_t groups = (a.nodes + G - 1) / G;
  for (int64_t gi = blockIdx.x; gi < groups; gi += gridDim.x)
    node2_factor_group<T, NT, G, Q>(a.Rin, a.nin, a.nodes, gi * G, a.n, a.Rout, a.Y, a.Tw, a.tau, a.status, smem);
}

template <typename T, int NT, int G, int Q>
cudaError_t launch_node2(const NodeFactorArgs<T>& a, int sms, cudaStream_t s) {
  const size_t smem = node2_smem_bytes(a.n, G, sizeof(T), NT, Q);
  auto kern = node2_factor_kernel<T, NT, G, Q>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int64_t groups = (a.nodes + G - 1) / G;
  int64_t grid = (int64_t)sms * per_sm;
  if (grid > groups) grid = groups;
  kern<<<(unsigned)grid, NT, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

// Shared memory of the configuration launch_node_factor picks last (one
// node per CTA), the smallest: the plan only has to know that one fits.
size_t node2_factor_smem_min(int n, int q, size_t elem) { return node2_smem_bytes(n, 1, elem, 256, q); }

template <typename T>
cudaError_t launch_node_factor(const NodeFactorArgs<T>& a, cudaStream_t s) {
  if (a.nodes <= 0 || a.n <= 0) return cudaSuccess;
  int dev = 0, sms = 0, smax = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (a.arity == 2 || a.arity == 4) {
    // Binary wide levels: two nodes per CTA share each serial step (when
    // their tiles fit); narrow binary levels (fewer groups than about two per
    // SM) and arity 4: one node per CTA, three CTAs per SM at n = 64 (measured
    // faster for the four-triangle nodes, whose steps are three times wider).
    // Levels with at most one node per SM run 512-thread CTAs: the same
    // serial steps, twice the warps (and row groups) for the update items.
    const bool narrow = a.nodes <= (int64_t)sms;
    if (a.arity == 2) {
      const bool wide = a.nodes >= 4 * (int64_t)sms;
      if (wide && node2_smem_bytes(a.n, 2, sizeof(T), 256, 2) <= (size_t)smax) return launch_node2<T, 256, 2, 2>(a, sms, s);
      if (narrow && node2_smem_bytes(a.n, 1, sizeof(T), 512, 2) <= (size_t)smax) return launch_node2<T, 512, 1, 2>(a, sms, s);
      return launch_node2<T, 256, 1, 2>(a, sms, s);
    }
    if (narrow && node2_smem_bytes(a.n, 1, sizeof(T), 512, 4) <= (size_t)smax) return launch_node2<T, 512, 1, 4>(a, sms, s);
    return launch_node2<T, 256, 1, 4>(a, sms, s);
  }
  // Arity 8 and 16 (short trees over few leaves, e.g. CAQR panels): the
  // packed lock-step kernel when its triangles fit, else the dense one.
  if ((a.arity == 8 || a.arity == 16) && node2_smem_bytes(a.n, 1, sizeof(T), 256, a.arity) <= (size_t)smax)
    return a.arity == 8 ? launch_node2<T, 256, 1, 8>(a, sms, s) : launch_node2<T, 256, 1, 16>(a, sms, s);
  const size_t smem = node_smem_bytes(a.n, a.arity, sizeof(T), kNodeThreads);
  auto kern = node_factor_kernel<T, kNodeThreads>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kNodeThreads, smem);
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int64_t grid = (int64_t)sms * per_sm;
  if (grid > a.nodes) grid = a.nodes;
  kern<<<(unsigned)grid, kNodeThreads, smem, s>>>(a);
  return cudaGetLastError();
}

size_t node_factor_smem(int n, int q, size_t elem) {
  if (q == 2 || q == 4) return node2_factor_smem_min(n, q, elem);
  const size_t dense = node_smem_bytes(n, q, elem, kNodeThreads);
  if (q == 8 || q == 16) return std::min(node2_factor_smem_min(n, q, elem), dense);
  return dense;
}

template cudaError_t launch_node_factor<double>(const NodeFactorArgs<double>&, cudaStream_t);
template cudaError_t launch_node_factor<float>(const NodeFactorArgs<float>&, cudaStream_t);

}  // namespace tsqr
