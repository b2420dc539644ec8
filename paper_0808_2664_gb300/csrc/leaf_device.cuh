// Leaf Householder QR as a device function, shared by the leaf kernel and
// the batched persistent kernel.  See leaf_factor.cu for the algorithm.
#pragma once

#include <cuda_runtime.h>

#include "reflector.cuh"
#include "tsqr_internal.cuh"

namespace tsqr {

constexpr int kLeafMinRows = 8;

__host__ __device__ inline size_t leaf_align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Bytes of the region that holds the leaf tile and, after write-back, the T
// matrix plus the doubling workspace (both in the storage type).
__host__ __device__ inline size_t leaf_tile_region(int n, int ld, size_t elem) {
  const size_t tile = leaf_align_up(elem * (size_t)n * ld, 16);
  const size_t tm = leaf_align_up(elem * ((size_t)n * n + (size_t)n * n / 2 + 1), 16);
  return tile > tm ? tile : tm;
}

// Shared-memory bytes for a leaf of up to ld rows with NT threads.
__host__ __device__ inline size_t leaf_smem_bytes(int n, int ld, size_t elem, int nt) {
  return leaf_tile_region(n, ld, elem) + (elem + sizeof(double)) * (size_t)nt + sizeof(double) * (size_t)n;
}

// Factors one leaf: rows Ag[0..hl) (column stride lda) of an n-column matrix,
// in place (Y below the diagonal, R_i on and above); writes the leaf R (n x n,
// ld n) to Rl, tau to taul and the compact-WY T (n x n) to Tg.  Every thread
// of the block calls it; smem holds leaf_smem_bytes(n, ld, sizeof(T), NT).
template <typename T, int NT, int NMAX>
__device__ void leaf_factor_one(T* Ag, int64_t lda, int hl, int n, int ld, T* Rl, T* taul, T* Tg, int* status,
                                unsigned char* smem) {
  T* S = reinterpret_cast<T*>(smem);
  // Products (dots, Y^T Y, T) run in the storage type T; squared norms and
  // the reflector scalars run in FP64.
  T* part = reinterpret_cast<T*>(smem + leaf_tile_region(n, ld, sizeof(T)));  // NT partial dots
  double* nrm_part = reinterpret_cast<double*>(part + NT);                    // scratch (n coefficients)
  double* tau_s = nrm_part + NT;                                              // n
  T* Tm = reinterpret_cast<T*>(smem);  // n x n, after write-back
  T* Wt = Tm + (size_t)n * n;          // doubling workspace
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  for (int c = 0; c < n; ++c) {
    const T* src = Ag + (int64_t)c * lda;
    for (int i = tid; i < hl; i += NT) S[c * ld + i] = src[i];
  }
  __syncthreads();
  T* coefs = reinterpret_cast<T*>(nrm_part);  // per-column tau * w of the current step

  for (int j = 0; j < n; ++j) {
    T* colj = S + j * ld;
    // Phase C: reflector for column j by one warp, chosen round-robin so the
    // serial step does not always load the same SM sub-partition.  The
    // squared norm of the tail is summed by the whole warp (full lanes).
    if (warp == (j % (NT / 32))) {
      double ssq = 0.0;
      for (int i = j + 1 + lane; i < hl; i += 32) {
        const double x = (double)colj[i];
        ssq = fma(x, x, ssq);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ssq += __shfl_xor_sync(0xffffffffu, ssq, o);
      double scale = 0.0;
      if (lane == 0) {
        const double alpha = (double)colj[j];
        const int len = hl - j - 1;
        Reflector r = make_reflector(
            alpha, ssq, [&]() { return scaled_norm(len, [&](int i) { return (double)colj[j + 1 + i]; }); },
            status);
        tau_s[j] = r.tau;
        scale = r.scale;
        colj[j] = (T)r.beta;
      }
      scale = __shfl_sync(0xffffffffu, scale, 0);
      for (int i = j + 1 + lane; i < hl; i += 32) colj[i] = (T)((double)colj[i] * scale);
    }
    __syncthreads();
    const int acols = n - 1 - j;
    if (acols == 0) break;
    const int rows = hl - j;  // rows j .. hl-1
    int rg = NT / acols;
    {
      int byrows = rows / kLeafMinRows;
      if (byrows < 1) byrows = 1;
      if (rg > byrows) rg = byrows;
      if (rg < 1) rg = 1;
    }
    const int chunk = (rows + rg - 1) / rg;
    const int slot = tid % acols, g = tid / acols;
    const int c = j + 1 + slot;
    const int i0 = j + g * chunk;
    const int i1 = min(i0 + chunk, hl);
    // Phase A: partial dot products u_j^T a_c over this thread's rows.
    if (g < rg) {
      const T* cc = S + c * ld;
      T s = T(0);
      int i = i0;
      if (i == j && i < i1) {
        s = cc[j];
        ++i;
      }
      for (; i < i1; ++i) s = fma(colj[i], cc[i], s);
      part[g * acols + slot] = s;
    }
    __syncthreads();
    // The rg partial sums of each column, once: coef_c = tau_j * w_c.
    if (tid < acols) {
      T w = T(0);
      for (int gg = 0; gg < rg; ++gg) w += part[gg * acols + tid];
      coefs[tid] = (T)tau_s[j] * w;
    }
    __syncthreads();
    // Phase B: a_c -= coef_c u_j.
    if (g < rg) {
      const T coef = coefs[slot];
      T* cc = S + c * ld;
      int i = i0;
      if (i == j && i < i1) {
        cc[j] -= coef;
        ++i;
      }
      for (; i < i1; ++i) cc[i] -= coef * colj[i];
    }
    __syncthreads();
  }
  __syncthreads();

  // Z = strictly-upper(Y^T Y) in registers: 2x2 tiles (P, Q) with P <= Q
  // over the upper triangle of n/2 x n/2 tile blocks, tile t = tid + k*NT.
  const int nb = (n + 1) / 2;
  const int ntiles = nb * (nb + 1) / 2;
  constexpr int kMaxTiles = (NMAX / 2) * (NMAX / 2 + 1) / 2 / NT + 1;
  T zacc[kMaxTiles][4];
  auto yv = [&](int i, int col) -> T {
    if (col >= n || i < col) return T(0);
    return i == col ? T(1) : S[col * ld + i];
  };
#pragma unroll
  for (int k = 0; k < kMaxTiles; ++k) {
    zacc[k][0] = zacc[k][1] = zacc[k][2] = zacc[k][3] = T(0);
    const int t = tid + k * NT;
    if (t < ntiles) {
      // t -> (P, Q) with P <= Q, ordered by Q so that the lanes of a warp
      // loop over nearly the same rows [2Q, hl).
      int Q = 0;
      while ((Q + 1) * (Q + 2) / 2 <= t) ++Q;
      const int P = t - Q * (Q + 1) / 2;
      const int p0 = 2 * P, q0 = 2 * Q;
      T z00 = T(0), z01 = T(0), z10 = T(0), z11 = T(0);
      for (int i = q0; i < hl; ++i) {
        const T a0 = yv(i, p0), a1 = yv(i, p0 + 1);
        const T b0 = yv(i, q0), b1 = yv(i, q0 + 1);
        z00 = fma(a0, b0, z00);
        z01 = fma(a0, b1, z01);
        z10 = fma(a1, b0, z10);
        z11 = fma(a1, b1, z11);
      }
      zacc[k][0] = z00;
      zacc[k][1] = z01;
      zacc[k][2] = z10;
      zacc[k][3] = z11;
    }
  }
  // Write back Y (below the diagonal) and R_i (on and above) in place, the
  // leaf R factor to the tree's level-0 items, and tau.
  for (int cc = 0; cc < n; ++cc) {
    T* dst = Ag + (int64_t)cc * lda;
    for (int i = tid; i < hl; i += NT) dst[i] = S[cc * ld + i];
  }
  for (int idx = tid; idx < n * n; idx += NT) {
    const int i = idx % n, cc = idx / n;
    Rl[idx] = i <= cc ? S[cc * ld + i] : T(0);
  }
  for (int cc = tid; cc < n; cc += NT) taul[cc] = (T)tau_s[cc];
  __syncthreads();
  // Tm = Z above the diagonal, tau on it, zero below.
  for (int idx = tid; idx < n * n; idx += NT) {
    const int p = idx % n, q = idx / n;
    Tm[idx] = p == q ? (T)tau_s[p] : T(0);
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kMaxTiles; ++k) {
    const int t = tid + k * NT;
    if (t < ntiles) {
      int Q = 0;
      while ((Q + 1) * (Q + 2) / 2 <= t) ++Q;
      const int P = t - Q * (Q + 1) / 2;
      const int p0 = 2 * P, q0 = 2 * Q;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int p = p0 + (e >> 1), q = q0 + (e & 1);
        if (p < q && q < n) Tm[p + q * n] = zacc[k][e];
      }
    }
  }
  __syncthreads();
  build_t_doubling(Tm, Wt, n);
  for (int idx = tid; idx < n * n; idx += NT) Tg[idx] = Tm[idx];
  __syncthreads();
}

}  // namespace tsqr
