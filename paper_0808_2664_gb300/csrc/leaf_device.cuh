// Leaf Householder QR as a device function, shared by the leaf kernel and
// the batched persistent kernel.  See leaf_factor.cu for the algorithm.
#pragma once

#include <cuda_runtime.h>

#include "reflector.cuh"
#include "tsqr_internal.cuh"

namespace tsqr {

constexpr int kLeafMinRows = 8;
constexpr int kLeafMaxGroups = 8;  // row groups per column in the leaf update phase

__host__ __device__ inline size_t leaf_align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Bytes of the region that holds the leaf tile and, after write-back, the T
// matrix plus the doubling workspace (both in the storage type).
__host__ __device__ inline size_t leaf_tile_region(int n, int ld, size_t elem) {
  const size_t tile = leaf_align_up(elem * (size_t)n * ld, 16);
  const size_t tm = leaf_align_up(elem * ((size_t)n * t_ld(n) + t_work_elems(n)), 16);
  return tile > tm ? tile : tm;
}

// Warp groups of a leaf CTA of nt threads: warp 0 (reflectors), the update
// warps, and nt/128 warps for Z = Y^T Y.
__host__ __device__ constexpr int leaf_z_warps(int nt) { return nt / 128; }
__host__ __device__ constexpr int leaf_u_warps(int nt) { return nt / 32 - 1 - leaf_z_warps(nt); }
// Partial-dot slots: the update warps' (one per thread, or one per column),
// then two double-buffered pairs of slices for the Z warps.
__host__ __device__ constexpr int leaf_upart(int nt) { return 32 * leaf_u_warps(nt) > 128 ? 32 * leaf_u_warps(nt) : 128; }
__host__ __device__ constexpr int leaf_zslice(int nt) { return 32 * leaf_z_warps(nt) > 64 ? 32 * leaf_z_warps(nt) : 64; }
__host__ __device__ constexpr int leaf_part_entries(int nt) { return leaf_upart(nt) + 4 * leaf_zslice(nt); }

// Shared-memory bytes for a leaf of up to ld rows with NT threads: the tile
// region, the partial dots, two per-column coefficient vectors, and FP64
// per-column scalars (tau, reflector scale, scaling exponent) plus 128
// per-lane partial norms, the Z group's progress word and the warp-role
// rotation.
__host__ __device__ inline size_t leaf_smem_bytes(int n, int ld, size_t elem, int nt) {
  return leaf_tile_region(n, ld, elem) + leaf_align_up(elem * (size_t)leaf_part_entries(nt), 8) +
         2 * leaf_align_up(elem * (size_t)n, 8) + sizeof(double) * (3 * (size_t)n + 128 + 2);
}

__device__ __forceinline__ void leaf_named_barrier(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Exponent k of the power of two 2^k that brings the largest magnitude of a
// column, given as the high 32 bits of its IEEE pattern with the sign
// cleared, to [1/2, 1), clamped so that 2^k and 2^-k are normal numbers of T.
// Zero, subnormal and non-finite columns get k = 0 (values kept).
template <typename T>
__device__ __forceinline__ int column_exp2(unsigned hi) {
  constexpr bool kF64 = sizeof(T) == 8;
  const int e = kF64 ? (int)(hi >> 20) : (int)(hi >> 23);  // biased exponent
  const int emax = kF64 ? 2047 : 255, bias = kF64 ? 1023 : 127;
  if (e == 0 || e == emax) return 0;
  const int k = -(e - bias + 1);
  const int lo = kF64 ? -1021 : -125, hi_k = kF64 ? 1022 : 126;
  return k < lo ? lo : (k > hi_k ? hi_k : k);
}

// 2^k as a T, built from its bit pattern (k within T's normal exponents).
template <typename T>
__device__ __forceinline__ T pow2_bits(int k) {
  if constexpr (sizeof(T) == 8) return __longlong_as_double((long long)(k + 1023) << 52);
  else return __int_as_float((k + 127) << 23);
}

// Row groups for a phase with `threads` threads per column (or pair) over
// `rows` rows: at least one, and at least kLeafMinRows rows per group.
__device__ __forceinline__ int leaf_groups(int threads, int rows) {
  int byrows = rows / kLeafMinRows;
  if (byrows < 1) byrows = 1;
  int rg = threads < byrows ? threads : byrows;
  return rg < 1 ? 1 : rg;
}

// Factors one leaf: rows Ag[0..hl) (column stride lda) of an n-column matrix,
// in place (Y below the diagonal, R_i on and above); writes the leaf R (n x n,
// ld n) to Rl, tau to taul and, when kWantT, the compact-WY T (n x n) to Tg
// (callers that need only R pass kWantT = false: no Z work, no T, Tg
// unused).  Every thread of the block calls it; smem holds
// leaf_smem_bytes(n, ld, sizeof(T), NT).
//
// Schedule.  Each column is first multiplied by a power of two that brings
// its largest entry to [1/2, 1): Householder QR commutes exactly with such
// column scalings (Q is unchanged, R's columns carry the factors), and it
// keeps every product below in range.  The Householder vector of column k is
// kept unscaled until the end, u_k = [1; s_k a_k(k+1:)] with the reflector's
// scale s_k, so its dot products can be taken before s_k is known.  Step k:
//   P   every trailing column c > k receives H_{k-1} (coefficient tau_{k-1}
//       w_c, with u_{k-1} = s_{k-1} a_{k-1} below its unit entry) and, fused
//       with that update, its partial dot with a_k's tail; meanwhile warp 0
//       alone turns column k's (alpha, ||tail||^2) into (beta, tau_k, s_k);
//   S1  w_c = a_c(k) + s_k (a_k(k+1:)^T a_c(k+1:)) and tau_k w_c per column;
//   S2  column k + 1 alone receives H_k (up to four warps, one per SM
//       sub-partition) and the squared norm of its tail is left per lane,
//       ready for the next step's reflector.
// Three barriers per column among these warps; the bulk of the arithmetic
// (update and dot) is one pass over the trailing block.  A separate group
// of warps takes the products for T's Z = Y^T Y as the tails become final,
// off those barriers (see the loop below).
//
// Stacked form (kStacked, one step of the flat tree of Section 2.1): the
// tile is [Rtop; A_i], the n x n upper-triangular R of the previous step
// (ld n, zeros below the diagonal) over the hl - n rows of Ag.  The same
// column loop factors it: reflector k then touches row k of Rtop and every
// row of A_i (the rows of Rtop below row k stay zero in column k), so the
// Householder vectors are e_k on top and a dense column below; the dense
// part is written to all hl - n rows of Ag and the new R to Rl (which may be
// Rtop: Rtop is read before Rl is written).
//
// As (column stride ldas), when given, is where the leaf's rows are read
// from; Y and R_i are still written to Ag.  A mapped page-locked host
// matrix there lets the leaf load its tile over the host link itself.
template <typename T, int NT, int NMAX, bool kWantT = true, bool kStacked = false>
__device__ void leaf_factor_one(T* Ag, int64_t lda, int hl, int n, int ld, T* Rl, T* taul, T* Tg, int* status,
                                unsigned char* smem, const T* Rtop = nullptr, const T* As = nullptr,
                                int64_t ldas = 0) {
  static_assert(NT >= 128, "the leaf schedule needs at least four warps");
  T* S = reinterpret_cast<T*>(smem);
  unsigned char* aux = smem + leaf_tile_region(n, ld, sizeof(T));
  constexpr int kUPart = leaf_upart(NT), kZSlice = leaf_zslice(NT);
  T* part = reinterpret_cast<T*>(aux);  // update warps' partial dots
  T* zpart = part + kUPart;             // Z warps': [parity][d1 | d2][kZSlice]
  T* coef = reinterpret_cast<T*>(aux + leaf_align_up(sizeof(T) * leaf_part_entries(NT), 8));  // n: tau_k w_c
  T* cscl = reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(coef) + leaf_align_up(sizeof(T) * n, 8));  // n: tau_k w_c s_k
  double* tau_s = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(cscl) + leaf_align_up(sizeof(T) * n, 8));
  double* sc_s = tau_s + n;  // n: reflector scales s_k
  int* cexp = reinterpret_cast<int*>(sc_s + n);  // n: column scaling exponents (n doubles reserved)
  double* wsum = sc_s + 2 * n;  // 128 per-lane partial squared norms (the S2 warps' lanes)
  volatile int* zready = reinterpret_cast<volatile int*>(wsum + 128);  // columns whose tails are final
  T* Tm = reinterpret_cast<T*>(smem);  // n x n (leading dimension t_ld(n)), after write-back
  T* Wt = Tm + (size_t)n * t_ld(n);    // doubling workspace
  // Warp roles rotate by the CTA's position on its SM: the hardware warp
  // slot of thread 0 (a placement hint only) picks a rotation that is
  // shared through shared memory, so the roles stay consistent within the
  // CTA.  Co-resident CTAs then put their reflector warps (and the other
  // single-warp FP64 steps) on different SM sub-partitions, whose FP64 unit
  // an FP64 instruction holds whatever its active lanes.
  {
    int* rot_s = reinterpret_cast<int*>(wsum + 129);
    if (threadIdx.x == 0) {
      unsigned ws;
      asm volatile("mov.u32 %0, %%warpid;" : "=r"(ws));
      *rot_s = (int)((ws / (NT / 32)) & 3u);
    }
    __syncthreads();
  }
  const int tid = (int)(threadIdx.x + 32u * (unsigned)*reinterpret_cast<volatile int*>(wsum + 129)) % NT;
  const int lane = tid & 31, warp = tid >> 5;
  // Z warps (NT/128 when T is wanted): column pairs in FP64, 4 x 4 column
  // blocks in FP32 (see the loop below).
  constexpr bool kZPairs = kWantT && sizeof(T) == 8;
  constexpr bool kZTiles = kWantT && sizeof(T) == 4;
  constexpr int kZWarps = kWantT ? leaf_z_warps(NT) : 0;
  constexpr int kUWarps = NT / 32 - 1 - kZWarps;
  static_assert(32 * kUWarps <= leaf_part_entries(NT), "update partial dots exceed their slots");
  constexpr int kMThreads = 32 * (1 + kUWarps), kZThreads = 32 * kZWarps;
  constexpr int kS2Warps = 1 + kUWarps < 4 ? 1 + kUWarps : 4;  // warps of the single-column phase S2

  // Load the tile: each thread walks the column-major elements e = tid + t NT,
  // several loads in flight.
  const int top = kStacked ? n : 0;  // rows of the tile taken from Rtop
  const T* const Ls = As ? As : Ag;
  const int64_t lls = As ? ldas : lda;
  auto src = [&](int c, int i) -> T {
    if constexpr (kStacked) return i < n ? Rtop[c * n + i] : Ls[(int64_t)c * lls + (i - n)];
    else return Ls[(int64_t)c * lls + i];
  };
  {
    const int total = hl * n;
    int c = tid / hl, i = tid - c * hl;
    const int dc = NT / hl, di = NT - dc * hl;
    int e = tid;
    for (; e + 3 * NT < total; e += 4 * NT) {
      T v[4];
      int cs[4], is[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        cs[u] = c;
        is[u] = i;
        v[u] = src(c, i);
        c += dc;
        i += di;
        if (i >= hl) {
          i -= hl;
          ++c;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) S[cs[u] * ld + is[u]] = v[u];
    }
    for (; e < total; e += NT) {
      S[c * ld + i] = src(c, i);
      c += dc;
      i += di;
      if (i >= hl) {
        i -= hl;
        ++c;
      }
    }
  }
  __syncthreads();
  // Largest magnitude of each column (one warp per column, integer maxima).
  for (int c = warp; c < n; c += NT / 32) {
    const T* col = S + c * ld;
    unsigned mx = 0u;
    for (int i = lane; i < hl; i += 32) {
      const T x = col[i];
      const unsigned bits = sizeof(T) == 8 ? (unsigned)__double2hiint((double)x) : __float_as_uint((float)x);
      const unsigned a = bits & 0x7fffffffu;
      mx = a > mx ? a : mx;
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (lane == 0) cexp[c] = column_exp2<T>(mx);
  }
  __syncthreads();
  // Scale each column by its power of two.
#pragma unroll 4
  for (int c = 0; c < n; ++c) {
    const T f = pow2_bits<T>(cexp[c]);
    T* col = S + c * ld;
    for (int i = tid; i < hl; i += NT) col[i] *= f;
  }
  __syncthreads();
  // Squared norm of column 0's tail, per S2 lane.
  if (warp < kS2Warps) {
    double ss = 0.0;
    for (int i = 1 + tid; i < hl; i += 32 * kS2Warps) {
      const double x = (double)S[i];
      ss = fma(x, x, ss);
    }
    wsum[tid] = ss;
  }
  __syncthreads();

  // Two warp groups run the column loop.  Group M (warp 0 and the update
  // warps) carries the factorisation, with its own barrier.  Group Z takes
  // the dots behind Z = strictly-upper(Y^T Y), needed for T:
  //   Z(p, q) = u_p^T u_q = s_p (a_p(q) + s_q a_p(q+1:)^T a_q(q+1:)),  p < q,
  // the unscaled dot d(p, q) = a_p(q+1:)^T a_q(q+1:) as soon as M reports
  // the tails final: in FP64, column q's dots in pairs (p, p+1) per work
  // item with the group's own barrier, so that Z's work (about a third of
  // the products) fills the FP64 pipe while M waits in its serial
  // per-column steps; in FP32, whole 4 x 4 blocks of d per warp once a
  // block of four columns is final (half a load per product instead of one
  // and a half, less shared-memory traffic beside the latency-bound loop).
  // d goes to Tg and is turned into Z after the loop.
  if (tid == 0) *zready = 0;
  __syncthreads();
  if (warp <= kUWarps) {
    for (int k = 0; k < n; ++k) {
      T* colk = S + k * ld;
      const int acols = n - 1 - k;  // trailing columns k+1 .. n-1
      int rg = acols > 0 ? (32 * kUWarps) / acols : 1;
      rg = leaf_groups(rg < kLeafMaxGroups ? rg : kLeafMaxGroups, hl - k);
      if (warp == 0) {
        // Reflector k, from alpha = a_k(k) and the per-lane squared norms of
        // a_k's tail.  Nothing else reads a_k(k) in this phase.
        double ssq = 0.0;
#pragma unroll
        for (int w = 0; w < kS2Warps; ++w) ssq += wsum[lane + 32 * w];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ssq += __shfl_xor_sync(0xffffffffu, ssq, o);
        if (lane == 0) {
          const double alpha = (double)colk[k];
          const int len = hl - k - 1;
          Reflector r = make_reflector_fast(
              alpha, ssq, [&]() { return scaled_norm(len, [&](int i) { return (double)colk[k + 1 + i]; }); },
              status);
          tau_s[k] = r.tau;
          sc_s[k] = r.scale;
          colk[k] = (T)r.beta;
        }
        __syncwarp();
      } else if (acols > 0) {
        // P: H_{k-1} on column c and the partial dot with a_k's tail, rows
        // interleaved over the rg groups (group g takes rows k-1+g,
        // k-1+g+rg, ...).
        for (int item = tid - 32; item < acols * rg; item += 32 * kUWarps) {
          const int slot = item % acols, g = item / acols;
          const int c = k + 1 + slot;
          T* cc = S + c * ld;
          T s0 = T(0), s1 = T(0);
          if (k == 0) {
            int i = 1 + g;
            for (; i + rg < hl; i += 2 * rg) {
              s0 = fma(colk[i], cc[i], s0);
              s1 = fma(colk[i + rg], cc[i + rg], s1);
            }
            if (i < hl) s0 = fma(colk[i], cc[i], s0);
          } else {
            const T* up = S + (k - 1) * ld;  // a_{k-1}: u_{k-1} = s_{k-1} a_{k-1} below its unit entry
            const T cf = coef[c], cs = cscl[c];
            int i = k - 1 + g;
            if (g == 0) {  // row k-1: the unit entry of u_{k-1}; gives R(k-1, c)
              cc[k - 1] -= cf;
              i += rg;
            }
            if (i == k) {  // row k: updated only (the unit entry of u_k enters in S1)
              cc[k] = fma(-cs, up[k], cc[k]);
              i += rg;
            }
            // Four rows per pass, all loads issued before the stores (the
            // stores may alias later loads as far as the compiler knows);
            // rows alternate between s0 and s1 as in the two-row tail.
            for (; i + 3 * rg < hl; i += 4 * rg) {
              T uv[4], av[4], xv[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                uv[u] = up[i + u * rg];
                av[u] = cc[i + u * rg];
                xv[u] = colk[i + u * rg];
              }
#pragma unroll
              for (int u = 0; u < 4; ++u) av[u] = fma(-cs, uv[u], av[u]);
#pragma unroll
              for (int u = 0; u < 4; ++u) cc[i + u * rg] = av[u];
              s0 = fma(xv[0], av[0], s0);
              s1 = fma(xv[1], av[1], s1);
              s0 = fma(xv[2], av[2], s0);
              s1 = fma(xv[3], av[3], s1);
            }
            for (; i + rg < hl; i += 2 * rg) {
              const T a0 = fma(-cs, up[i], cc[i]);
              const T a1 = fma(-cs, up[i + rg], cc[i + rg]);
              cc[i] = a0;
              cc[i + rg] = a1;
              s0 = fma(colk[i], a0, s0);
              s1 = fma(colk[i + rg], a1, s1);
            }
            if (i < hl) {
              const T a0 = fma(-cs, up[i], cc[i]);
              cc[i] = a0;
              s0 = fma(colk[i], a0, s0);
            }
          }
          part[g * acols + slot] = s0 + s1;
        }
      }
      leaf_named_barrier(1, kMThreads);
      if (acols == 0) break;
      // S1: coefficients of H_k for the trailing columns.
      if (tid < acols) {
        T d0 = T(0), d1 = T(0);
        int gg = 0;
        for (; gg + 1 < rg; gg += 2) {
          d0 += part[gg * acols + tid];
          d1 += part[(gg + 1) * acols + tid];
        }
        if (gg < rg) d0 += part[gg * acols + tid];
        const int cidx = k + 1 + tid;
        const double tk = tau_s[k], sk = sc_s[k], ts = tk * sk;
        const double w = fma(sk, (double)(d0 + d1), (double)S[cidx * ld + k]);
        coef[cidx] = (T)(tk * w);
        cscl[cidx] = (T)(ts * w);
      }
      leaf_named_barrier(1, kMThreads);
      // S2: column k+1 receives H_k; squared norm of its tail below row k+1.
      if (warp < kS2Warps) {
        T* ca = S + (k + 1) * ld;
        const T cf = coef[k + 1], cs = cscl[k + 1];
        double ss = 0.0;
        if (tid == 0) ca[k] -= cf;
        for (int i = k + 1 + tid; i < hl; i += 32 * kS2Warps) {
          const T a = fma(-cs, colk[i], ca[i]);
          ca[i] = a;
          if (i > k + 1) ss = fma((double)a, (double)a, ss);
        }
        wsum[tid] = ss;
      }
      leaf_named_barrier(1, kMThreads);
      if (tid == 0) {
        __threadfence_block();
        *zready = k + 1;  // column k+1's tail is final
      }
    }
  } else if constexpr (kZPairs) {
    const int ztid = tid - kMThreads;
    bool wait_ok = true;
    for (int q = 1; q < n; ++q) {
      if (lane == 0 && wait_ok) {
        int spins = 0;
        while (*zready < q) {
          if (++spins > (1 << 22)) {  // the update warps stopped reporting: give up, flag it
            atomicOr(status, kStatusTimeout);
            wait_ok = false;
            break;
          }
          __nanosleep(64);
        }
        __threadfence_block();
      }
      __syncwarp();
      const int npairs = (q + 1) / 2;
      int rgz = kZThreads / npairs;
      rgz = leaf_groups(rgz < kLeafMaxGroups ? rgz : kLeafMaxGroups, hl - q);
      T* zp = zpart + (q & 1) * 2 * kZSlice;
      const T* xq = S + q * ld;
      for (int item = ztid; item < npairs * rgz; item += kZThreads) {
        const int t = item % npairs, g = item / npairs;
        const int p = 2 * t, p2 = 2 * t + 1 < q ? 2 * t + 1 : 2 * t;
        const T* x1 = S + p * ld;
        const T* x2 = S + p2 * ld;
        T z1 = T(0), z2 = T(0), z3 = T(0), z4 = T(0);
        int i = q + 1 + g;
        for (; i + rgz < hl; i += 2 * rgz) {
          const T v0 = xq[i], v1 = xq[i + rgz];
          z1 = fma(v0, x1[i], z1);
          z2 = fma(v0, x2[i], z2);
          z3 = fma(v1, x1[i + rgz], z3);
          z4 = fma(v1, x2[i + rgz], z4);
        }
        if (i < hl) {
          z1 = fma(xq[i], x1[i], z1);
          z2 = fma(xq[i], x2[i], z2);
        }
        zp[g * npairs + t] = z1 + z3;
        zp[kZSlice + g * npairs + t] = z2 + z4;
      }
      leaf_named_barrier(2, kZThreads);
      for (int t = ztid; t < npairs; t += kZThreads) {
        T d1 = T(0), d2 = T(0);
        for (int g = 0; g < rgz; ++g) {
          d1 += zp[g * npairs + t];
          d2 += zp[kZSlice + g * npairs + t];
        }
        Tg[2 * t + q * n] = d1;
        if (2 * t + 1 < q) Tg[2 * t + 1 + q * n] = d2;
      }
    }
  } else if constexpr (kZTiles) {
    // d = L^T L with L(r, c) = a_c(r) for r > c (the unscaled tails), p < q.
    // Z warp zw takes tiles t = zw, zw + kZWarps, ... in block order (block
    // Q holds t = Q(Q+1)/2 + P, P = 0..Q: columns 4P.., 4Q..) once column
    // min(4Q + 3, n - 1)'s tail is final.  Lane l sums rows r = 4Q + 1 + l
    // (mod 32); the 16 sums are reduce-scattered over the warp, entry s
    // ending in lanes 2s and 2s + 1.
    const int zw = warp - 1 - kUWarps;
    const int nb = (n + 3) / 4;
    bool wait_ok = true;
    int Q = 0, base = 0;
    for (int t = zw; t < nb * (nb + 1) / 2; t += kZWarps) {
      while (base + Q + 1 <= t) {
        base += Q + 1;
        ++Q;
      }
      const int P = t - base;
      const int need = 4 * Q + 3 < n - 1 ? 4 * Q + 3 : n - 1;
      if (lane == 0 && wait_ok) {
        int spins = 0;
        while (*zready < need) {
          if (++spins > (1 << 22)) {  // the update warps stopped reporting: give up, flag it
            atomicOr(status, kStatusTimeout);
            wait_ok = false;
            break;
          }
          __nanosleep(64);
        }
        __threadfence_block();
      }
      __syncwarp();
      int pc[4], qc[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        pc[i] = (4 * P + i < n ? 4 * P + i : n - 1) * ld;
        qc[i] = (4 * Q + i < n ? 4 * Q + i : n - 1) * ld;
      }
      T acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
      int r = 4 * Q + 1 + lane;
      if (r < hl) {  // the only row of this lane that can lie in the block's own rows
        T yp[4], yq[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          yp[i] = S[pc[i] + r];
          yq[i] = r > 4 * Q + i ? S[qc[i] + r] : T(0);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(yp[i], yq[j], acc[i][j]);
        r += 32;
      }
#pragma unroll 2
      for (; r < hl; r += 32) {
        T yp[4], yq[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          yp[i] = S[pc[i] + r];
          yq[i] = S[qc[i] + r];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(yp[i], yq[j], acc[i][j]);
      }
      T v8[8], v4[4], v2[2];
      bool up = lane & 16;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const T lo = acc[u >> 2][u & 3], hi = acc[(u + 8) >> 2][(u + 8) & 3];
        v8[u] = (up ? hi : lo) + __shfl_xor_sync(0xffffffffu, up ? lo : hi, 16);
      }
      up = lane & 8;
#pragma unroll
      for (int u = 0; u < 4; ++u) v4[u] = (up ? v8[u + 4] : v8[u]) + __shfl_xor_sync(0xffffffffu, up ? v8[u] : v8[u + 4], 8);
      up = lane & 4;
#pragma unroll
      for (int u = 0; u < 2; ++u) v2[u] = (up ? v4[u + 2] : v4[u]) + __shfl_xor_sync(0xffffffffu, up ? v4[u] : v4[u + 2], 4);
      up = lane & 2;
      T v = (up ? v2[1] : v2[0]) + __shfl_xor_sync(0xffffffffu, up ? v2[0] : v2[1], 2);
      v += __shfl_xor_sync(0xffffffffu, v, 1);
      const int sl = lane >> 1, p = 4 * P + (sl >> 2), q = 4 * Q + (sl & 3);
      if (!(lane & 1) && p < q && q < n) Tg[p + q * n] = v;
    }
  }
  __syncthreads();
  // Z(p, q) = s_p (a_p(q) + s_q d(p, q)) from the unscaled tails.
  for (int idx = tid; kWantT && idx < n * n; idx += NT) {
    const int p = idx % n, q = idx / n;
    if (p < q) Tg[idx] = (T)(sc_s[p] * ((double)S[p * ld + q] + sc_s[q] * (double)Tg[idx]));
  }
  __syncthreads();
  // Write back the leaf in one pass over its elements (several loads in
  // flight per thread): Householder vectors u_c = s_c a_c below the
  // diagonal, R with the column factors taken out on and above it.
  {
    const int total = hl * n;
    int c = tid / hl, i = tid - c * hl;
    const int dc = NT / hl, di = NT - dc * hl;
    auto final_value = [&](int cc, int ii) -> T {
      const T v = S[cc * ld + ii];
      if (ii <= cc) return v * pow2_bits<T>(-cexp[cc]);
      return sizeof(T) == 8 ? (T)((double)v * sc_s[cc]) : v * (T)sc_s[cc];
    };
    int e = tid;
    for (; e + 3 * NT < total; e += 4 * NT) {
      T v[4];
      int cs[4], is[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        cs[u] = c;
        is[u] = i;
        v[u] = final_value(c, i);
        c += dc;
        i += di;
        if (i >= hl) {
          i -= hl;
          ++c;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (is[u] >= top) Ag[(int64_t)cs[u] * lda + (is[u] - top)] = v[u];
    }
    for (; e < total; e += NT) {
      if (i >= top) Ag[(int64_t)c * lda + (i - top)] = final_value(c, i);
      c += dc;
      i += di;
      if (i >= hl) {
        i -= hl;
        ++c;
      }
    }
  }
  for (int idx = tid; idx < n * n; idx += NT) {
    const int i = idx % n, cc = idx / n;
    Rl[idx] = i <= cc ? S[cc * ld + i] * pow2_bits<T>(-cexp[cc]) : T(0);
  }
  for (int cc = tid; cc < n; cc += NT) taul[cc] = (T)tau_s[cc];
  __syncthreads();
  if constexpr (kWantT) {
    // Tm = Z above the diagonal (from Tg), tau on it, zero below.
    const int L = t_ld(n);
    for (int idx = tid; idx < n * n; idx += NT) {
      const int p = idx % n, q = idx / n;
      Tm[p + q * L] = p == q ? (T)tau_s[p] : (p < q ? Tg[idx] : T(0));
    }
    __syncthreads();
    build_t_doubling(Tm, Wt, n);
    for (int idx = tid; idx < n * n; idx += NT) Tg[idx] = Tm[idx % n + (idx / n) * L];
    __syncthreads();
  }
}

}  // namespace tsqr
