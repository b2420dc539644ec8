// Tree-node QR of stacked triangles as a device function, shared by the
// node kernel and the batched persistent kernel.  See node_factor.cu.
#pragma once

#include <cuda_runtime.h>

#include "reflector.cuh"
#include "tsqr_internal.cuh"

namespace tsqr {

constexpr int kMinRowsNode = 4;

__host__ __device__ inline size_t align_up_n(size_t x, size_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline int node_ld(int n) { return (n + 1) | 1; }  // odd, and room for T's t_ld(n)

__host__ __device__ inline size_t node_tile_bytes(int n, int q, size_t elem) {
  const size_t tile = align_up_n(elem * (size_t)q * n * node_ld(n), 16);
  return tile;
}

__host__ __device__ inline size_t node_smem_bytes(int n, int q, size_t elem, int nt) {
  return node_tile_bytes(n, q, elem) + (elem + sizeof(double)) * (size_t)nt + sizeof(double) * (size_t)n;
}

// Factors one node: the nc upper-triangular n x n children stored
// contiguously from Rin (ld n each; read with L1-bypassing loads so that a
// child written by another CTA of the same launch is seen), arity q.  Writes
// the node's R (Ro), its q-1 upper-triangular reflector blocks (Yo), tau
// (tauo) and, when kBuildT, the compact-WY T (To): Z = strictly-upper(Y^T Y)
// summed over the lower blocks using their triangular structure (n^3/6 for
// q = 2), then the doubling merges.  A lone child (nc = 1) passes through with
// an identity Q.  Every thread of the block calls it.
template <typename T, int NT, bool kBuildT>
__device__ void node_factor_one(const T* Rin, int nc, int q, int n, T* Ro, T* Yo, T* To, T* tauo, int* status,
                                unsigned char* smem) {
  const int ld = node_ld(n);
  T* S = reinterpret_cast<T*>(smem);
  // Products (dots, T) in the storage type T; norms and reflector scalars in FP64.
  T* part = reinterpret_cast<T*>(smem + node_tile_bytes(n, q, sizeof(T)));
  double* tau_s = reinterpret_cast<double*>(part + NT) + NT;
  const int tid = threadIdx.x;
  // Element (i, c) of block b.
  auto at = [&](int b, int c, int i) -> T& { return S[((size_t)b * n + c) * ld + i]; };
  const int64_t nn = (int64_t)n * n;
  if (nc == 1) {
    // A lone child passes up unchanged: its Q factor is the identity.
    for (int64_t idx = tid; idx < nn; idx += NT) {
      Ro[idx] = __ldcg(Rin + idx);
      if (kBuildT) To[idx] = T(0);
    }
    for (int64_t idx = tid; idx < (int64_t)(q - 1) * nn; idx += NT) Yo[idx] = T(0);
    for (int c = tid; c < n; c += NT) tauo[c] = T(0);
    return;
  }
  for (int b = 0; b < nc; ++b) {
    const T* Ri = Rin + b * nn;
    for (int64_t idx = tid; idx < nn; idx += NT) {
      const int i = (int)(idx % n), c = (int)(idx / n);
      at(b, c, i) = i <= c ? __ldcg(Ri + idx) : T(0);
    }
  }
  __syncthreads();

  for (int j = 0; j < n; ++j) {
    const int jr = j + 1;                  // rows 0..j of each lower block
    const int vrows = 1 + (nc - 1) * jr;   // virtual row 0 is row j of block 0
    const int tail = (nc - 1) * jr;        // virtual rows 1..vrows-1
    // Phase C: warp 0 sums the squared tail (all lanes, FP64), lane 0 forms
    // the reflector, the warp scales the tail into u_j.
    if (tid < 32) {
      double ssq = 0.0;
      for (int v = tid; v < tail; v += 32) {
        const double x = (double)at(1 + v / jr, j, v % jr);
        ssq = fma(x, x, ssq);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ssq += __shfl_xor_sync(0xffffffffu, ssq, o);
      double scale = 0.0;
      if (tid == 0) {
        const double alpha = (double)at(0, j, j);
        Reflector r = make_reflector_fast(
            alpha, ssq,
            [&]() { return scaled_norm(tail, [&](int v) { return (double)at(1 + v / jr, j, v % jr); }); }, status);
        tau_s[j] = r.tau;
        scale = r.scale;
        at(0, j, j) = (T)r.beta;
      }
      scale = __shfl_sync(0xffffffffu, scale, 0);
      for (int v = tid; v < tail; v += 32) {
        T& x = at(1 + v / jr, j, v % jr);
        x = (T)((double)x * scale);
      }
    }
    __syncthreads();
    // Phase A: w_c = u_j^T a_c for the trailing columns c > j.
    const int acols = n - 1 - j;
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
        const int c = j + 1 + slot;
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
      if (slot < acols && g == 0) part[slot] = s;
    }
    __syncthreads();
    // Phase B: trailing updates a_c -= tau_j w_c u_j.
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
        const T coef = (T)tau_s[j] * part[slot];
        int v = g * chunk;
        const int v1 = min(v + chunk, vrows);
        if (v == 0 && v < v1) {
          at(0, c, j) -= coef;
          ++v;
        }
        if (v < v1) {
          int b = 1 + (v - 1) / jr, i = (v - 1) % jr;
          for (; v < v1; ++v) {
            at(b, c, i) -= coef * at(b, j, i);
            if (++i == jr) {
              i = 0;
              ++b;
            }
          }
        }
      }
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
  if (kBuildT) {
    // T lives in block 0's region (R already written out); the doubling
    // workspace reuses block 1's region once Z no longer needs Y.
    T* Tm = S;  // leading dimension t_ld(n) <= ld
    T* Wt = S + (size_t)n * ld;
    const int L = t_ld(n);
    for (int64_t idx = tid; idx < nn; idx += NT) {  // diagonal and below; Z fills above
      const int p = (int)(idx % n), jj = (int)(idx / n);
      if (p >= jj) Tm[p + (int64_t)jj * L] = p == jj ? (T)tau_s[p] : T(0);
    }
    // Pairs (p, j), p < j, p-major: the lanes of a warp share p, so every
    // lane runs the same (nc - 1)(p + 1)-term sum.
    const int npairs = n * (n - 1) / 2;
    for (int idx = tid; idx < npairs; idx += NT) {
      int p = 0, rem = idx;
      while (rem >= n - 1 - p) {
        rem -= n - 1 - p;
        ++p;
      }
      const int jj = p + 1 + rem;
      T z = T(0);
      for (int b = 1; b < nc; ++b)
        for (int i = 0; i <= p; ++i) z = fma(at(b, p, i), at(b, jj, i), z);
      Tm[p + (int64_t)jj * L] = z;
    }
    __syncthreads();
    build_t_doubling(Tm, Wt, n);
    for (int64_t idx = tid; idx < nn; idx += NT) To[idx] = Tm[idx % n + (idx / n) * L];
    __syncthreads();
  }
}

}  // namespace tsqr
