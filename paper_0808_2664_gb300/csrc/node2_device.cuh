// Tree-node QR of Q stacked triangles, G nodes per CTA in lock step.
//
// A node factors [R_0; R_1; ...; R_{Q-1}] (upper-triangular n x n children)
// with structured Householder QR (Section 2.1, Eqs. TSQR_binarytree_2/_3,
// and the remark on structured local QR): reflector k touches row k of R_0
// and rows 0..k of every other triangle, so its vector is e_k on top and an
// upper-triangular column below in each lower block; nothing below the
// triangles is stored or touched (2n^3/3 flops per eliminated triangle,
// Section 2.2).  The node's Y is the Q-1 upper triangles that replaced
// R_1..R_{Q-1}.
//
// A node has little work per column (at most n^2/2 products) behind a
// serial chain per column (reflector, coefficients), so this kernel
//   * factors G nodes of a tree level together, so that each serial step
//     serves G nodes at once (lane g of warp 0 forms node g's reflector);
//   * uses the leaf kernel's schedule: the reflector of column k is formed
//     by warp 0 while the other warps apply H_{k-1} to every trailing column
//     fused with that column's dot with column k's unscaled tail, and take
//     the entries Z(p, k) = u_p^T u_k of the T factor as extra work items;
//     then, per node, one warp carries column k+1 through H_k (forming its
//     coefficient itself) and sums its squared norm while a second warp
//     turns the other partial dots into coefficients; two barriers per
//     column;
//   * stores the triangles packed (column c of a block holds rows 0..c), so
//     that a node takes n(n+1) values of shared memory.
// Each column is first scaled by a power of two bringing its largest entry
// (over both triangles) to [1/2, 1); Householder QR commutes exactly with
// that, and it keeps the unscaled dot products in range.  Products are in
// the storage type T; squared norms and reflector scalars in FP64.
#pragma once

#include <cuda_runtime.h>

#include "leaf_device.cuh"
#include "reflector.cuh"
#include "tsqr_internal.cuh"

namespace tsqr {

// Row groups per column in the update phase: four for 256 threads, eight
// for the 512-thread form used on narrow levels (shorter per-item chains).
__host__ __device__ constexpr int node2_max_groups(int nt) { return nt >= 512 ? 8 : 4; }
constexpr int kNode2MinRows = 4;    // rows per group at least

__host__ __device__ inline int node2_packed(int n) { return n * (n + 1) / 2; }

// Bytes of one node's compact-WY doubling area: T (leading dimension
// t_ld(n)), then the doubling workspace.
__host__ __device__ inline size_t node2_t_bytes(int n, size_t elem) {
  return leaf_align_up(elem * ((size_t)n * t_ld(n) + t_work_elems(n)), 16);
}

// The region holding G nodes' q packed triangles each, reused for the T builds.
__host__ __device__ inline size_t node2_region_bytes(int n, int G, size_t elem, int q) {
  const size_t data = leaf_align_up(elem * (size_t)q * G * node2_packed(n), 16);
  const size_t tb = node2_t_bytes(n, elem);
  return data > tb ? data : tb;
}

__host__ __device__ inline size_t node2_smem_bytes(int n, int G, size_t elem, int nt, int q) {
  return node2_region_bytes(n, G, elem, q) + leaf_align_up(elem * 3 * (size_t)nt, 8) +
         2 * leaf_align_up(elem * (size_t)G * n, 8) + sizeof(double) * (3 * (size_t)G * n + 32);
}

// Factors nodes node0 .. node0+G-1 of a tree level of arity Q: children
// Rin[Q node + b], b < Q (n x n, ld n, upper part read with L1-bypassing
// loads; missing children read as zeros, which leave the others' R and give
// zero reflector parts), outputs as node_factor_one with kBuildT: R (Ro),
// Y (Q-1 blocks of n x n), tau and, when kBuildT, T (without it Tout is
// unused).  Nodes at or past `nodes` are computed on zeros and not written.
// Every thread of the block calls it.
template <typename T, int NT, int G, int Q, bool kBuildT = true>
__device__ void node2_factor_group(const T* __restrict__ Rin, int64_t nin, int64_t nodes, int64_t node0, int n,
                                   T* Rout, T* Yout, T* Tout, T* tauout, int* status, unsigned char* smem) {
  static_assert(NT / 32 >= 2 * G + 2, "need a reflector warp, two S warps per node and a Z warp");
  // Next-column (S) warps per node: on the 512-thread CTAs of the narrow,
  // latency-bound levels, one per lower triangle when the CTA has the warps
  // (each on its own sub-partition: the FP64 squared norm of a triangle's
  // column per warp); else one for all of them (wide levels, where three
  // CTAs share an SM, lose to the extra warps' repeated coefficient work).
  constexpr int kSW = (NT >= 512 && (NT / 32 - 2 - G) / G >= Q - 1) ? Q - 1 : 1;
  constexpr int kS = G * kSW, kSC = kS + G;  // S warps 1..kS, coefficient warps kS+1..kSC
  static_assert(NT / 32 >= kSC + 2, "need a reflector warp, the S and coefficient warps and a Z warp");
  static_assert(kS < 31, "ssq[0..kS) holds the partial squared norms, ssq[31] the warp-role rotation");
  const int pk = node2_packed(n);
  T* D = reinterpret_cast<T*>(smem);
  unsigned char* aux = smem + node2_region_bytes(n, G, sizeof(T), Q);
  T* part = reinterpret_cast<T*>(aux);  // 3 NT partial dots
  T* coef = reinterpret_cast<T*>(aux + leaf_align_up(sizeof(T) * 3 * NT, 8));  // G n: tau_k w_c
  T* cscl = reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(coef) + leaf_align_up(sizeof(T) * G * n, 8));
  double* tau_s = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(cscl) + leaf_align_up(sizeof(T) * G * n, 8));
  double* sc_s = tau_s + G * n;                         // G n: reflector scales
  int* cexp = reinterpret_cast<int*>(sc_s + G * n);     // G n: column exponents (G n doubles reserved)
  double* ssq = sc_s + 2 * G * n;                       // G kSW: partial squared tail norms
  // Warp roles rotate by the CTA's slot on its SM (thread 0's hardware warp
  // slot, a placement hint shared through shared memory; ssq + 31 is a
  // spare slot), as in the leaf: co-resident CTAs put their single-warp
  // FP64 steps on different sub-partitions.
  {
    int* rot_s = reinterpret_cast<int*>(ssq + 31);
    if (threadIdx.x == 0) {
      unsigned ws;
      asm volatile("mov.u32 %0, %%warpid;" : "=r"(ws));
      *rot_s = (int)((ws / (NT / 32)) & 3u);
    }
    __syncthreads();
  }
  const int tid = (int)(threadIdx.x + 32u * (unsigned)*reinterpret_cast<volatile int*>(ssq + 31)) % NT;
  const int lane = tid & 31, warp = tid >> 5;
  constexpr int kPWarps = NT / 32 - 1;
  const int64_t nn = (int64_t)n * n;
  // Column c of block b (0: R_0, b: R_b) of node g, rows 0..c.
  auto col = [&](int g, int b, int c) -> T* { return D + (size_t)(Q * g + b) * pk + c * (c + 1) / 2; };

  // A lone child (the last node of a level whose count leaves one over)
  // passes up unchanged: its Q factor is the identity.  (Factoring it with
  // zero lower blocks would give the same R but take the scaled-norm path
  // of a zero tail at every column.)
  if (G == 1 && node0 < nodes && (int64_t)Q * node0 + 1 >= nin) {
    const T* src = Rin + (int64_t)Q * node0 * nn;
    for (int64_t idx = tid; idx < nn; idx += NT) {
      Rout[node0 * nn + idx] = __ldcg(src + idx);
      if (kBuildT) Tout[node0 * nn + idx] = T(0);
    }
    for (int64_t idx = tid; idx < (int64_t)(Q - 1) * nn; idx += NT) Yout[node0 * (Q - 1) * nn + idx] = T(0);
    for (int c = tid; c < n; c += NT) tauout[node0 * n + c] = T(0);
    return;
  }

  // Load the children's upper triangles, one warp per (node, column): the
  // triangles' column c (rows 0..c), its largest magnitude, its power-of-two
  // factor applied on the way into shared memory.
  for (int gc = warp; gc < G * n; gc += NT / 32) {
    const int g = gc / n, c = gc - g * n;
    const int64_t node = node0 + g;
    T v[Q][kMaxN / 32];
    unsigned mx = 0u;
#pragma unroll
    for (int b = 0; b < Q; ++b) {
      const int64_t child = (int64_t)Q * node + b;
      const bool has = node < nodes && child < nin;
      const T* src = Rin + child * nn + (int64_t)c * n;
#pragma unroll
      for (int r = 0; r < kMaxN / 32; ++r) {
        const int i = lane + 32 * r;
        v[b][r] = T(0);
        if (i <= c) {
          if (has) v[b][r] = __ldcg(src + i);
          const unsigned bits = sizeof(T) == 8 ? (unsigned)__double2hiint((double)v[b][r]) : __float_as_uint((float)v[b][r]);
          const unsigned m = bits & 0x7fffffffu;
          mx = m > mx ? m : mx;
        }
      }
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    const int ex = column_exp2<T>(mx);
    const T f = pow2_bits<T>(ex);
    if (lane == 0) cexp[gc] = ex;
#pragma unroll
    for (int b = 0; b < Q; ++b) {
      T* d = col(g, b, c);
#pragma unroll
      for (int r = 0; r < kMaxN / 32; ++r) {
        const int i = lane + 32 * r;
        if (i <= c) d[i] = v[b][r] * f;
      }
    }
  }
  __syncthreads();
  if (tid < G) {
    // Column 0's squared tail norm, as the S warps' partial sums: part s
    // of node g over triangles b = 1 + s, 1 + s + kSW, ...
    for (int sw = 0; sw < kSW; ++sw) {
      double x2 = 0.0;
      for (int b = 1 + sw; b < Q; b += kSW) {
        const double x = (double)col(tid, b, 0)[0];
        x2 = fma(x, x, x2);
      }
      ssq[tid * kSW + sw] = x2;
    }
  }
  __syncthreads();

  for (int k = 0; k < n; ++k) {
    const int acols = n - 1 - k;     // trailing columns k+1 .. n-1
    const int npairs = kBuildT ? (k + 1) / 2 : 0;  // Z pairs (p, k-1-p) of column k
    int rg = (32 * kPWarps) / (G * (acols + npairs) > 0 ? G * (acols + npairs) : 1);
    {
      int byrows = (k + 1) / kNode2MinRows;
      if (byrows < 1) byrows = 1;
      if (rg > byrows) rg = byrows;
      if (rg > node2_max_groups(NT)) rg = node2_max_groups(NT);
      if (rg < 1) rg = 1;
    }
    const int ucols = G * acols, zcols = G * npairs;
    const int nu = ucols * rg;
    const int zbase = (nu + 31) / 32 * 32;
    const int nitems = zbase + zcols * rg;
    if (warp == 0) {
      // Reflector k of node g (lane g): alpha = R_0(k, k), tail = R_b(0..k, k), b >= 1.
      if (lane < G) {
        const int g = lane;
        T* ck0 = col(g, 0, k);
        const double alpha = (double)ck0[k];
        double ss = ssq[g * kSW];
        for (int sw = 1; sw < kSW; ++sw) ss += ssq[g * kSW + sw];
        // R_0(k-1, k): H_{k-1}'s unit entry on row k-1 of this column (the
        // S warps all read that entry for their coefficient, so it is
        // updated only now).
        if (k > 0) ck0[k - 1] -= coef[g * n + k];
        Reflector r = make_reflector_fast(
            alpha, ss,
            [&]() { return scaled_norm((Q - 1) * (k + 1), [&](int v) { return (double)col(g, 1 + v / (k + 1), k)[v % (k + 1)]; }); },
            status);
        tau_s[g * n + k] = r.tau;
        sc_s[g * n + k] = r.scale;
        ck0[k] = (T)r.beta;
      }
      __syncwarp();
    } else {
      for (int item = tid - 32; item < nitems; item += 32 * kPWarps) {
        if (item < nu) {
          // H_{k-1} on trailing column c (R_0 row k-1; rows 0..k-1 of every
          // lower block) fused with the partial dot of their rows 0..k with
          // column k's tail.
          const int slot = item % ucols, grp = item / ucols;
          const int g = slot / acols, c = k + 1 + slot % acols;
          T s0 = T(0), s1 = T(0);
          if (k == 0) {
            if (grp == 0)
              for (int b = 1; b < Q; ++b) s0 = fma(col(g, b, 0)[0], col(g, b, c)[0], s0);
          } else {
            const T cf = coef[g * n + c], cs = cscl[g * n + c];
            if (grp == 0) col(g, 0, c)[k - 1] -= cf;  // the unit entry of u_{k-1}: R(k-1, c)
#pragma unroll
            for (int b = 1; b < Q; ++b) {
              T* cc1 = col(g, b, c);
              const T* ak = col(g, b, k);
              const T* up = col(g, b, k - 1);
              int i = grp;
              for (; i + rg < k; i += 2 * rg) {
                const T a0 = fma(-cs, up[i], cc1[i]);
                const T a1 = fma(-cs, up[i + rg], cc1[i + rg]);
                cc1[i] = a0;
                cc1[i + rg] = a1;
                s0 = fma(ak[i], a0, s0);
                s1 = fma(ak[i + rg], a1, s1);
              }
              if (i < k) {
                const T a0 = fma(-cs, up[i], cc1[i]);
                cc1[i] = a0;
                s0 = fma(ak[i], a0, s0);
                i += rg;
              }
              if (i == k) s1 = fma(ak[k], cc1[k], s1);  // row k: not touched by H_{k-1}
            }
          }
          part[grp * ucols + slot] = s0 + s1;
        } else if (kBuildT && item >= zbase) {
          // Z(p, k) and Z(p2, k) with p = t, p2 = k-1-t (one entry when they
          // meet): partial dots of the lower blocks' columns over their rows
          // 0..p and 0..p2.  Pairing a short column with a long one gives
          // every item k+1 rows, walked as one sequence (rows of p, then
          // rows of p2) so that the lanes of a warp run the same count.
          const int zi = item - zbase;
          const int zc = zcols > 0 ? zcols : 1;
          const int slot = zi % zc, grp = zi / zc;
          const int np = npairs > 0 ? npairs : 1;
          const int g = slot / np, t = slot % np;
          const int p = t, p2 = k - 1 - t;
          const int len = p2 > p ? p + p2 + 2 : p + 1;
          T z1 = T(0), z2 = T(0);
#pragma unroll
          for (int b = 1; b < Q; ++b) {
            const T* ak = col(g, b, k);
            const T* x1 = col(g, b, p);
            const T* x2 = col(g, b, p2);
            for (int v = grp; v < len; v += rg) {
              const bool first = v <= p;
              const int i = first ? v : v - p - 1;
              const T acc = fma(ak[i], (first ? x1 : x2)[i], first ? z1 : z2);
              z1 = first ? acc : z1;
              z2 = first ? z2 : acc;
            }
          }
          part[NT + grp * zcols + slot] = z1;
          part[2 * NT + grp * zcols + slot] = z2;
        }
      }
    }
    __syncthreads();
    // S: warp 1 + g takes column k+1 of node g: its coefficient of H_k
    // (every lane forms it from the partial dots), H_k applied to it, and
    // the squared norm of its tail for the next reflector (R_1.. rows
    // 0..k+1).  Warp 1 + G + g forms the coefficients of node g's other
    // trailing columns (lanes over columns) at the same time; the remaining
    // warps take the Z entries of column k.
    if (warp >= 1 && warp <= kSC && acols > 0) {
      const int g = warp <= kS ? (warp - 1) / kSW : warp - 1 - kS;
      const double tk = tau_s[g * n + k], sk = sc_s[g * n + k], ts = tk * sk;
      auto w_of = [&](int j) {
        const int sl = g * acols + j;
        T d0 = T(0), d1 = T(0);
        int gg = 0;
        for (; gg + 1 < rg; gg += 2) {
          d0 += part[gg * ucols + sl];
          d1 += part[(gg + 1) * ucols + sl];
        }
        if (gg < rg) d0 += part[gg * ucols + sl];
        return fma(sk, (double)(d0 + d1), (double)col(g, 0, k + 1 + j)[k]);
      };
      if (warp <= kS) {
        const int sw = (warp - 1) % kSW;
        const double w = w_of(0);
        const T cf1 = (T)(tk * w), cs1 = (T)(ts * w);
        if (sw == 0 && lane == 0) coef[g * n + k + 1] = cf1;  // row k of column k+1: next reflector step
        double ss = 0.0;
        for (int b = 1 + sw; b < Q; b += kSW) {
          T* cc1 = col(g, b, k + 1);
          const T* ak = col(g, b, k);
          for (int i = lane; i <= k + 1; i += 32) {
            T v = cc1[i];
            if (i <= k) {
              v = fma(-cs1, ak[i], v);
              cc1[i] = v;
            }
            ss = fma((double)v, (double)v, ss);
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        if (lane == 0) ssq[g * kSW + sw] = ss;
      } else {
        for (int j = 1 + lane; j < acols; j += 32) {
          const double w = w_of(j);
          coef[g * n + k + 1 + j] = (T)(tk * w);
          cscl[g * n + k + 1 + j] = (T)(ts * w);
        }
      }
    } else if (kBuildT && warp > kSC) {
      for (int zs = tid - 32 * (kSC + 1); zs < zcols; zs += NT - 32 * (kSC + 1)) {
        const int np = npairs > 0 ? npairs : 1;
        const int g = zs / np, t = zs % np;
        T d1 = T(0), d2 = T(0);
        for (int gg = 0; gg < rg; ++gg) {
          d1 += part[NT + gg * zcols + zs];
          d2 += part[2 * NT + gg * zcols + zs];
        }
        const int64_t node = node0 + g;
        if (node < nodes) {
          T* Tg = Tout + node * nn;
          const int p = t, p2 = k - 1 - t;
          const double sk = sc_s[g * n + k];
          Tg[p + k * n] = (T)(sc_s[g * n + p] * sk * (double)d1);
          if (p2 > p) Tg[p2 + k * n] = (T)(sc_s[g * n + p2] * sk * (double)d2);
        }
      }
    }
    __syncthreads();
    if (acols == 0) break;
  }
  // Outputs, one warp per (node, column): R (column factors taken back
  // out), Y_b = s_c * (R_b column c) for b >= 1, zeros below the diagonal;
  // tau.
  for (int gc = warp; gc < G * n; gc += NT / 32) {
    const int g = gc / n, c = gc - g * n;
    const int64_t node = node0 + g;
    if (node < nodes) {
      const T fr = pow2_bits<T>(-cexp[gc]);
      const double sy = sc_s[gc];
      const T* r0 = col(g, 0, c);
      T* ro = Rout + node * nn + (int64_t)c * n;
      for (int i = lane; i < n; i += 32) ro[i] = i <= c ? r0[i] * fr : T(0);
#pragma unroll
      for (int b = 1; b < Q; ++b) {
        const T* rb = col(g, b, c);
        T* yo = Yout + (node * (Q - 1) + (b - 1)) * nn + (int64_t)c * n;
        for (int i = lane; i < n; i += 32) yo[i] = i <= c ? (T)((double)rb[i] * sy) : T(0);
      }
      if (lane == 0) tauout[node * n + c] = (T)tau_s[gc];
    }
  }
  __syncthreads();
  if constexpr (!kBuildT) return;
  // T of each node: Z (from Tout) above the diagonal, tau on it; as many
  // nodes at a time as the region holds.
  const size_t tstride = node2_t_bytes(n, sizeof(T)) / sizeof(T);
  const int per_batch = (int)(node2_region_bytes(n, G, sizeof(T), Q) / node2_t_bytes(n, sizeof(T)));
  for (int g0 = 0; g0 < G; g0 += per_batch) {
    const int cnt = G - g0 < per_batch ? G - g0 : per_batch;
    for (int gq = warp; gq < cnt * n; gq += NT / 32) {
      const int gl = gq / n, q = gq - gl * n, g = g0 + gl;
      const int64_t node = node0 + g;
      T* Tm = D + gl * tstride + (size_t)q * t_ld(n);
      for (int p = lane; p < n; p += 32) {
        T v = T(0);
        if (p == q) v = (T)tau_s[g * n + p];
        else if (p < q && node < nodes) v = Tout[node * nn + (int64_t)q * n + p];
        Tm[p] = v;
      }
    }
    __syncthreads();
    build_t_doubling_many(D, tstride, D + (size_t)n * t_ld(n), tstride, cnt, n);
    for (int gq = warp; gq < cnt * n; gq += NT / 32) {
      const int gl = gq / n, q = gq - gl * n;
      const int64_t node = node0 + g0 + gl;
      if (node < nodes)
        for (int p = lane; p < n; p += 32) Tout[node * nn + (int64_t)q * n + p] = D[gl * tstride + (size_t)q * t_ld(n) + p];
    }
    __syncthreads();
  }
}

}  // namespace tsqr
