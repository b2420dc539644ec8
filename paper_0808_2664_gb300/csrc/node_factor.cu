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
// One CTA per node, triangles in shared memory.  The same C/S/A/B phases as
// the leaf kernel run over the "virtual rows" of reflector j: row j of block
// 0 followed by rows 0..j of blocks 1..q-1.
#include <cuda_runtime.h>

#include "reflector.cuh"
#include "tsqr_internal.cuh"

namespace tsqr {
namespace {

constexpr int kMinRowsNode = 4;

__host__ __device__ inline size_t align_up_n(size_t x, size_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline int node_ld(int n) { return n | 1; }

__host__ __device__ inline size_t node_tile_bytes(int n, int q, size_t elem) {
  size_t tile = align_up_n(elem * (size_t)q * n * node_ld(n), 16);
  const size_t tm = align_up_n(sizeof(double) * ((size_t)n * n + (size_t)n * n / 2 + 1), 16);
  return tile > tm ? tile : tm;
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT) node_factor_kernel(NodeFactorArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = a.n, q = a.arity;
  const int ld = node_ld(n);
  T* S = reinterpret_cast<T*>(smem);
  double* part = reinterpret_cast<double*>(smem + node_tile_bytes(n, q, sizeof(T)));
  double* nrm_part = part + NT;
  double* tau_s = nrm_part + NT;
  double* Tm = reinterpret_cast<double*>(smem);
  double* Wt = Tm + (size_t)n * n;
  __shared__ double sh_scale;
  __shared__ int sh_nrg;
  const int tid = threadIdx.x;
  // Element (i, c) of block b.
  auto at = [&](int b, int c, int i) -> T& { return S[((size_t)b * n + c) * ld + i]; };
  const int64_t nn = (int64_t)n * n;

  for (int64_t node = blockIdx.x; node < a.nodes; node += gridDim.x) {
    const int64_t c0 = node * q;
    const int nc = (int)((a.nin - c0) < q ? (a.nin - c0) : q);
    T* Ro = a.Rout + node * nn;
    T* Yo = a.Y + node * (int64_t)(q - 1) * nn;
    T* To = a.Tw + node * nn;
    T* tauo = a.tau + node * (int64_t)n;
    if (nc == 1) {
      // A lone child passes up unchanged: its Q factor is the identity.
      const T* Ri = a.Rin + c0 * nn;
      for (int64_t idx = tid; idx < nn; idx += NT) {
        Ro[idx] = Ri[idx];
        To[idx] = T(0);
      }
      for (int64_t idx = tid; idx < (int64_t)(q - 1) * nn; idx += NT) Yo[idx] = T(0);
      for (int c = tid; c < n; c += NT) tauo[c] = T(0);
      continue;
    }
    for (int b = 0; b < nc; ++b) {
      const T* Ri = a.Rin + (c0 + b) * nn;
      for (int64_t idx = tid; idx < nn; idx += NT) {
        const int i = (int)(idx % n), c = (int)(idx / n);
        at(b, c, i) = i <= c ? Ri[idx] : T(0);
      }
    }
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int b = 1; b < nc; ++b) {
        const double x = (double)at(b, 0, 0);
        s = fma(x, x, s);
      }
      nrm_part[0] = s;
      sh_nrg = 1;
    }
    __syncthreads();

    for (int j = 0; j < n; ++j) {
      const int jr = j + 1;                  // rows 0..j of each lower block
      const int vrows = 1 + (nc - 1) * jr;   // virtual row 0 is row j of block 0
      if (tid == 0) {
        double ssq = 0.0;
        for (int g = 0; g < sh_nrg; ++g) ssq += nrm_part[g];
        if (j > 0) {
          // Row j of every lower block joins the tail of column j here.
          for (int b = 1; b < nc; ++b) {
            const double x = (double)at(b, j, j);
            ssq = fma(x, x, ssq);
          }
        }
        const double alpha = (double)at(0, j, j);
        Reflector r = make_reflector(
            alpha, ssq,
            [&]() {
              return scaled_norm((nc - 1) * jr, [&](int v) { return (double)at(1 + v / jr, j, v % jr); });
            },
            a.status);
        tau_s[j] = r.tau;
        sh_scale = r.scale;
        at(0, j, j) = (T)r.beta;
      }
      __syncthreads();
      {
        const double scale = sh_scale;
        for (int v = tid; v < (nc - 1) * jr; v += NT) {
          T& x = at(1 + v / jr, j, v % jr);
          x = (T)((double)x * scale);
        }
      }
      __syncthreads();
      // Phase A: dot products of u_j with every other column.
      const int acols = n - 1;
      if (acols > 0) {
        int lim = NT / acols;
        int byrows = vrows / kMinRowsNode;
        if (byrows < 1) byrows = 1;
        if (lim > byrows) lim = byrows;
        if (lim > 32) lim = 32;
        const int rga = pow2_floor(lim < 1 ? 1 : lim);
        const int chunk = (vrows + rga - 1) / rga;
        const int slot = tid / rga, g = tid % rga;
        T s = T(0);
        if (slot < acols) {
          const int c = slot < j ? slot : slot + 1;
          int v = g * chunk;
          const int v1 = min(v + chunk, vrows);
          if (v == 0 && v < v1) {
            s = at(0, c, j);
            ++v;
          }
          if (v < v1) {
            int b = 1 + (v - 1) / jr, i = (v - 1) % jr;
            for (; v < v1; ++v) {
              s = fma(at(b, j, i), at(b, c, i), s);
              if (++i == jr) {
                i = 0;
                ++b;
              }
            }
          }
        }
        for (int o = rga >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (slot < acols && g == 0) part[slot] = (double)s;
      }
      __syncthreads();
      // Phase B: z values for the T factor; trailing updates.
      if (tid < j) To[tid + (int64_t)j * n] = (T)part[tid];
      const int bcols = n - 1 - j;
      if (bcols > 0) {
        int rgb = NT / bcols;
        int byrows = vrows / kMinRowsNode;
        if (byrows < 1) byrows = 1;
        if (rgb > byrows) rgb = byrows;
        if (rgb < 1) rgb = 1;
        const int chunk = (vrows + rgb - 1) / rgb;
        const int slot = tid % bcols, g = tid / bcols;
        if (g < rgb) {
          const int c = j + 1 + slot;
          const T coef = (T)(tau_s[j] * part[c - 1]);
          int v = g * chunk;
          const int v1 = min(v + chunk, vrows);
          double ssq = 0.0;
          if (v == 0 && v < v1) {
            at(0, c, j) -= coef;
            ++v;
          }
          if (v < v1) {
            int b = 1 + (v - 1) / jr, i = (v - 1) % jr;
            for (; v < v1; ++v) {
              T& x = at(b, c, i);
              x -= coef * at(b, j, i);
              if (slot == 0) ssq = fma((double)x, (double)x, ssq);
              if (++i == jr) {
                i = 0;
                ++b;
              }
            }
          }
          if (slot == 0) nrm_part[g] = ssq;
        }
        if (tid == 0) sh_nrg = rgb;
      }
      __syncthreads();
    }

    for (int64_t idx = tid; idx < nn; idx += NT) {
      const int i = (int)(idx % n), c = (int)(idx / n);
      Ro[idx] = i <= c ? at(0, c, i) : T(0);
    }
    for (int b = 1; b < q; ++b) {
      for (int64_t idx = tid; idx < nn; idx += NT) {
        const int i = (int)(idx % n), c = (int)(idx / n);
        Yo[(int64_t)(b - 1) * nn + idx] = (b < nc && i <= c) ? at(b, c, i) : T(0);
      }
    }
    for (int c = tid; c < n; c += NT) tauo[c] = (T)tau_s[c];
    __syncthreads();
    for (int64_t idx = tid; idx < nn; idx += NT) {
      const int p = (int)(idx % n), jj = (int)(idx / n);
      Tm[idx] = p < jj ? (double)To[idx] : (p == jj ? tau_s[p] : 0.0);
    }
    __syncthreads();
    build_t_doubling(Tm, Wt, n);
    for (int64_t idx = tid; idx < nn; idx += NT) To[idx] = (T)Tm[idx];
    __syncthreads();
  }
}

}  // namespace

template <typename T>
cudaError_t launch_node_factor(const NodeFactorArgs<T>& a, cudaStream_t s) {
  if (a.nodes <= 0 || a.n <= 0) return cudaSuccess;
  const size_t smem = node_tile_bytes(a.n, a.arity, sizeof(T)) + sizeof(double) * (2 * kNodeThreads + a.n);
  auto kern = node_factor_kernel<T, kNodeThreads>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kNodeThreads, smem);
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int64_t grid = (int64_t)sms * per_sm;
  if (grid > a.nodes) grid = a.nodes;
  kern<<<(unsigned)grid, kNodeThreads, smem, s>>>(a);
  return cudaGetLastError();
}

size_t node_factor_smem(int n, int q, size_t elem) {
  return node_tile_bytes(n, q, elem) + sizeof(double) * (2 * kNodeThreads + n);
}

template cudaError_t launch_node_factor<double>(const NodeFactorArgs<double>&, cudaStream_t);
template cudaError_t launch_node_factor<float>(const NodeFactorArgs<float>&, cudaStream_t);

}  // namespace tsqr
