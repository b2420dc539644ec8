// Implicit application of the tree-structured Q (Section 2.1,
// Eq. TSQR_binarytree_4): Q = diag(Q_i) * (tree-node factors) * D.
//
// Every factor is a compact-WY block reflector I - Y T Y^T (Schreiber and Van
// Loan, cited in Section 2.1).  A leaf applies it to its h-row block of C:
//   W = Y^T C,  W <- T^T W (for Q^T) or T W (for Q),  C <- C - Y W.
// A tree node applies it to the q stacked n-row "slots" of C that hold its
// children's R rows; its Y is [I; Y_1; ...; Y_{q-1}] with upper-triangular Y_b.
// The "form" mode computes Q [X; 0] reading only X (the first n rows), which
// is how the thin Q is built top-down without initialising the rest of Q.
#include <cuda_runtime.h>

#include "tsqr_internal.cuh"

namespace tsqr {
namespace {

// Element loop idx = tid, tid + NT, ... < count doing st(idx, ld(idx)),
// with four loads in flight per thread before their stores: a store through
// a pointer the compiler cannot tell apart from the next load's would
// otherwise make every load wait out the one before.
template <int NT, class Ld, class St>
__device__ __forceinline__ void copy4(int tid, int count, Ld ld, St st) {
  int idx = tid;
  for (; idx + 3 * NT < count; idx += 4 * NT) {
    const auto v0 = ld(idx), v1 = ld(idx + NT), v2 = ld(idx + 2 * NT), v3 = ld(idx + 3 * NT);
    st(idx, v0);
    st(idx + NT, v1);
    st(idx + 2 * NT, v2);
    st(idx + 3 * NT, v3);
  }
  for (; idx < count; idx += NT) st(idx, ld(idx));
}


__host__ __device__ inline size_t align16(size_t x) { return (x + 15) / 16 * 16; }

// ---------------------------------------------------------------- leaves --
// Shared memory: Ys [kApplyRows][n+1] (row-major), Cs [kApplyRows][kc+1] (FP32: at
// least [kApplyRows][n+1], the second Y block of phase 3),
// Ws [n][kc] (W, then T-times-W), Ts [n][n] (column-major T).
// Whether a leaf's n x n T fits in the Y and C staging tiles (it is needed
// only after they are done with).
// Bytes of the C staging tile [kApplyRows][kApplyCols + 1]; with FP32 it
// also holds the second 32-row block of Y ([kApplyRows][n + 1]) in phase 3.
__host__ __device__ inline size_t leaf_apply_cs_bytes(int n, size_t elem) {
  const int cols = (elem == 4 && n + 1 > kApplyCols + 1) ? n + 1 : kApplyCols + 1;
  return align16(elem * kApplyRows * (size_t)cols);
}

__host__ __device__ inline bool leaf_apply_t_shared(int n, size_t elem) {
  return elem * (size_t)n * n <= align16(elem * kApplyRows * (n + 1)) + leaf_apply_cs_bytes(n, elem);
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT) leaf_apply_kernel(LeafApplyArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int RB = kApplyRows;
  constexpr int KC = kApplyCols;
  const int n = a.n;
  const int ly = n + 1, lc = KC + 1;
  T* Ys = reinterpret_cast<T*>(smem);
  T* Cs = reinterpret_cast<T*>(smem + align16(sizeof(T) * RB * ly));
  T* Ws = reinterpret_cast<T*>(smem + align16(sizeof(T) * RB * ly) + leaf_apply_cs_bytes(n, sizeof(T)));
  // T is needed only between phases 1 and 3: it reuses the staging area when it fits.
  const bool t_shared = leaf_apply_t_shared(n, sizeof(T));
  T* Ts = t_shared ? Ys : Ws + (size_t)n * KC;
  const int tid = threadIdx.x;

  int64_t unit = blockIdx.x;
  int piece = 0, pieces = 1;
  if (unit >= a.split_from) {
    const int64_t v = unit - a.split_from;
    unit = a.split_from + v / a.split;
    piece = (int)(v % a.split);
    pieces = a.split;
  }
  const int64_t leaf = unit % a.nleaves;
  const int64_t kchunk = (unit / a.nleaves) * KC;
  const int kfull = (int)((a.k - kchunk) < KC ? (a.k - kchunk) : KC);
  const int pw = (kfull + pieces - 1) / pieces;
  const int64_t k0 = kchunk + (int64_t)piece * pw;
  const int kc = kfull - piece * pw < pw ? kfull - piece * pw : pw;
  if (kc <= 0) return;  // an empty piece of a narrow chunk (uniform over the CTA)
  const int64_t r0 = leaf * a.h;
  const int hl = (leaf == a.nleaves - 1) ? (int)(a.m - r0) : (int)a.h;
  const T* Yg = a.Y + r0;
  T* Cg = a.C + r0 + k0 * a.ldc;
  const int mode = a.mode;
  const int rows1 = mode == kApplyForm ? n : hl;  // rows that feed W

  // T of this leaf (column-major n x n).
  const T* Tg = a.Tw + leaf * (int64_t)n * n;
  if (!t_shared)
    for (int idx = tid; idx < n * n; idx += NT) Ts[idx] = Tg[idx];

  // Phase 1: W = Y^T C over rows1 rows; 4x4 register tiles of W.  Tiles
  // are numbered column-tile fastest, so that the lanes of a warp share one
  // or two row tiles p0 and the triangular bounds below (Y(r, p) = 0 for
  // r < p; T triangular) are nearly uniform over the warp and skip the zeros.
  const int tp = (n + 3) / 4, tcn = (kc + 3) / 4;
  const int ntiles = tp * tcn;
  T acc[2][4][4];
#pragma unroll
  for (int t = 0; t < 2; ++t)
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[t][x][y] = T(0);

  // Staging of the next 32-row block of Y and C goes through registers:
  // its global loads are issued before the current block's products.
  constexpr bool kPrefetch = sizeof(T) == 4;  // for FP64 the registers cost more occupancy than the overlap gains
  constexpr int kYPer = kPrefetch ? (RB * kMaxN + NT - 1) / NT : 1, kCPer = kPrefetch ? (RB * KC + NT - 1) / NT : 1;
  T ypre[kYPer], cpre[kCPer];
  auto fetch_y = [&](int rb, int rows) {
#pragma unroll
    for (int j = 0; j < kYPer; ++j) {
      const int idx = tid + j * NT;
      T v = T(0);
      if (idx < RB * n) {
        const int i = idx % RB, p = idx / RB, r = rb + i;
        if (r < rows) v = r < p ? T(0) : (r == p ? T(1) : Yg[r + (int64_t)p * a.ldy]);
      }
      ypre[j] = v;
    }
  };
  auto direct_y = [&](int rb, int rows) {
    copy4<NT>(
        tid, RB * n,
        [&](int idx) {
          const int i = idx % RB, p = idx / RB, r = rb + i;
          T v = T(0);
          if (r < rows) v = r < p ? T(0) : (r == p ? T(1) : Yg[r + (int64_t)p * a.ldy]);
          return v;
        },
        [&](int idx, T v) { Ys[(idx % RB) * ly + idx / RB] = v; });
  };
  auto stage_y = [&]() {
#pragma unroll
    for (int j = 0; j < kYPer; ++j) {
      const int idx = tid + j * NT;
      if (idx < RB * n) Ys[(idx % RB) * ly + idx / RB] = ypre[j];
    }
  };
  auto fetch_c = [&](int rb) {
#pragma unroll
    for (int j = 0; j < kCPer; ++j) {
      const int idx = tid + j * NT;
      const int i = idx % RB, c = idx / RB, r = rb + i;
      cpre[j] = (idx < RB * KC && r < rows1 && c < kc) ? Cg[r + (int64_t)c * a.ldc] : T(0);
    }
  };
  auto stage_c = [&]() {
#pragma unroll
    for (int j = 0; j < kCPer; ++j) {
      const int idx = tid + j * NT;
      if (idx < RB * KC) Cs[(idx % RB) * lc + idx / RB] = cpre[j];
    }
  };
  if (kPrefetch) {
    fetch_y(0, rows1);
    fetch_c(0);
  }
  for (int rb = 0; rb < rows1; rb += RB) {
    __syncthreads();
    if (kPrefetch) {
      stage_y();
      stage_c();
    } else {
      direct_y(rb, rows1);
      copy4<NT>(
          tid, RB * KC,
          [&](int idx) {
            const int i = idx % RB, c = idx / RB, r = rb + i;
            return (r < rows1 && c < kc) ? Cg[r + (int64_t)c * a.ldc] : T(0);
          },
          [&](int idx, T v) { Cs[(idx % RB) * lc + idx / RB] = v; });
    }
    __syncthreads();
    if (kPrefetch && rb + RB < rows1) {
      fetch_y(rb + RB, rows1);
      fetch_c(rb + RB);
    }
    const int rmax = min(RB, rows1 - rb);
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int tile = tid + t * NT;
      if (tile >= ntiles) break;
      const int p0 = (tile / tcn) * 4, c0 = (tile % tcn) * 4;
      for (int i = p0 > rb ? p0 - rb : 0; i < rmax; ++i) {  // rows above p0: zero in Y
        T yv[4], cv[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) yv[x] = (p0 + x < n) ? Ys[i * ly + p0 + x] : T(0);
#pragma unroll
        for (int y = 0; y < 4; ++y) cv[y] = Cs[i * lc + c0 + y];
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[t][x][y] = fma(yv[x], cv[y], acc[t][x][y]);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const int tile = tid + t * NT;
    if (tile >= ntiles) break;
    const int p0 = (tile / tcn) * 4, c0 = (tile % tcn) * 4;
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y)
        if (p0 + x < n && c0 + y < KC) Ws[(p0 + x) * KC + c0 + y] = acc[t][x][y];
  }
  if (t_shared)
    for (int idx = tid; idx < n * n; idx += NT) Ts[idx] = Tg[idx];
  __syncthreads();

  // Phase 2: W <- T^T W (Q^T) or T W (Q, form).
  const bool trans = mode == kApplyQT;
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const int tile = tid + t * NT;
    if (tile >= ntiles) break;
    const int p0 = (tile / tcn) * 4, c0 = (tile % tcn) * 4;
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const int p = p0 + x;
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[t][x][y] = T(0);
      if (p >= n) continue;
      // T^T(p, q) = T(q, p), nonzero for q <= p; T(p, q) nonzero for q >= p.
      const int qa = trans ? 0 : p, qb = trans ? p : n - 1;
      for (int qq = qa; qq <= qb; ++qq) {
        const T tv = trans ? Ts[qq + p * n] : Ts[p + qq * n];
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[t][x][y] = fma(tv, Ws[qq * KC + c0 + y], acc[t][x][y]);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const int tile = tid + t * NT;
    if (tile >= ntiles) break;
    const int p0 = (tile / tcn) * 4, c0 = (tile % tcn) * 4;
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y)
        if (p0 + x < n && c0 + y < KC) Ws[(p0 + x) * KC + c0 + y] = acc[t][x][y];
  }

  // Phase 3: C <- C - Y W  (form: C <- [X; 0] - Y W).
  if constexpr (sizeof(T) == 4) {
    // FP32: 64-row steps, a lane = rows r and r + 32, a warp = 8 contiguous
    // columns, all sixteen dot products at once (W read as two float4 per
    // p, each feeding both rows; the C entries read before any store).  The
    // first 32 rows come through the prefetch registers, the second 32 are
    // staged directly into the C tile (unused here).  Y's zeros above the
    // diagonal and past the leaf are staged, so running both rows' dots to
    // the longer bound adds only exact zeros after each dot's own terms,
    // which are taken in order p = 0, 1, ...
    static_assert(RB == 32 && (NT / 32) * 8 == KC, "phase 3 layout: a warp per 8 columns of a 32-row block");
    T* Ys2 = Cs;
    const int i = tid & 31, c0 = (tid >> 5) * 8;
    fetch_y(0, hl);
    for (int rb = 0; rb < hl; rb += 2 * RB) {
      __syncthreads();
      stage_y();
      copy4<NT>(
          tid, RB * n,
          [&](int idx) {
            const int ii = idx % RB, p = idx / RB, r = rb + RB + ii;
            T v = T(0);
            if (r < hl) v = r < p ? T(0) : (r == p ? T(1) : Yg[r + (int64_t)p * a.ldy]);
            return v;
          },
          [&](int idx, T v) { Ys2[(idx % RB) * ly + idx / RB] = v; });
      __syncthreads();
      if (rb + 2 * RB < hl) fetch_y(rb + 2 * RB, hl);
      const int ra = rb + i, rbb = rb + RB + i;
      if (ra < hl && c0 < kc) {
        const bool two = rbb < hl;
        const int pmax = min(n, (two ? rbb : ra) + 1);  // Y(r, p) = 0 for p > r
        T acc[2][8];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[0][j] = acc[1][j] = T(0);
        const T* ya = Ys + i * ly;
        const T* yb = Ys2 + i * ly;
        for (int p = 0; p < pmax; ++p) {
          const T y0 = ya[p], y1 = yb[p];
          const float4 w0 = *reinterpret_cast<const float4*>(Ws + p * KC + c0);
          const float4 w1 = *reinterpret_cast<const float4*>(Ws + p * KC + c0 + 4);
          acc[0][0] = fma(y0, w0.x, acc[0][0]);
          acc[0][1] = fma(y0, w0.y, acc[0][1]);
          acc[0][2] = fma(y0, w0.z, acc[0][2]);
          acc[0][3] = fma(y0, w0.w, acc[0][3]);
          acc[0][4] = fma(y0, w1.x, acc[0][4]);
          acc[0][5] = fma(y0, w1.y, acc[0][5]);
          acc[0][6] = fma(y0, w1.z, acc[0][6]);
          acc[0][7] = fma(y0, w1.w, acc[0][7]);
          acc[1][0] = fma(y1, w0.x, acc[1][0]);
          acc[1][1] = fma(y1, w0.y, acc[1][1]);
          acc[1][2] = fma(y1, w0.z, acc[1][2]);
          acc[1][3] = fma(y1, w0.w, acc[1][3]);
          acc[1][4] = fma(y1, w1.x, acc[1][4]);
          acc[1][5] = fma(y1, w1.y, acc[1][5]);
          acc[1][6] = fma(y1, w1.z, acc[1][6]);
          acc[1][7] = fma(y1, w1.w, acc[1][7]);
        }
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          const int r = h2 ? rbb : ra;
          if (h2 && !two) break;
          const bool fresh = mode == kApplyForm && r >= n;  // rows below X start from zero
          T* row = Cg + r;
          T old[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) old[j] = (c0 + j < kc && !fresh) ? row[(int64_t)(c0 + j) * a.ldc] : T(0);
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (c0 + j < kc) row[(int64_t)(c0 + j) * a.ldc] = old[j] - acc[h2][j];
        }
      }
    }
    return;
  }
  // FP64: thread = (row, column group).
  constexpr int CG = NT / RB;
  const int i = tid % RB, cg = tid / RB;
  if (kPrefetch) fetch_y(0, hl);
  for (int rb = 0; rb < hl; rb += RB) {
    __syncthreads();
    if (kPrefetch) stage_y();
    else direct_y(rb, hl);
    __syncthreads();
    if (kPrefetch && rb + RB < hl) fetch_y(rb + RB, hl);
    const int r = rb + i;
    if (r < hl) {
      const int pmax = min(n, r + 1);  // Y(r, p) = 0 for p > r
      const bool fresh = mode == kApplyForm && r >= n;  // rows below X start from zero
      T* row = Cg + r;
      // Each column's C entry is read before the previous column's store
      // (the compiler cannot tell the two addresses apart), so its latency
      // overlaps that column's dot product.
      T old = (cg < kc && !fresh) ? row[(int64_t)cg * a.ldc] : T(0);
      for (int c = cg; c < kc; c += CG) {
        const T next = (c + CG < kc && !fresh) ? row[(int64_t)(c + CG) * a.ldc] : T(0);
        T s = T(0);
        for (int p = 0; p < pmax; ++p) s = fma(Ys[i * ly + p], Ws[p * KC + c], s);
        row[(int64_t)c * a.ldc] = old - s;
        old = next;
      }
    }
  }
}

// ----------------------------------------------------------------- nodes --
// Shared memory (column-major tiles, ldn odd): B1 [kc][ldn] holds a lower
// slot while W accumulates and then W' = T^(T) W; B2 [kc][ldn] holds W and
// later Y_b W'; Ys [n][ldn] one lower block of Y, and T ([n][n]) between
// the W accumulation and the Y_b W' products (two CTAs per SM at n = 64 in
// FP64).
template <typename T, int NT>
__global__ void __launch_bounds__(NT) node_apply_kernel(NodeApplyArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int KC = kApplyCols;
  const int n = a.n, q = a.arity;
  const int ldn = n | 1;
  T* B1 = reinterpret_cast<T*>(smem);
  T* B2 = B1 + (size_t)KC * ldn;
  T* Ys = B2 + (size_t)KC * ldn;
  T* Ts = Ys;
  const int tid = threadIdx.x;
  int64_t unit = blockIdx.x;
  int piece = 0, pieces = 1;
  if (unit >= a.split_from) {
    const int64_t v = unit - a.split_from;
    unit = a.split_from + v / a.split;
    piece = (int)(v % a.split);
    pieces = a.split;
  }
  const int64_t node = unit % a.nodes;
  const int64_t c0 = node * q;
  const int nc = (int)((a.nin - c0) < q ? (a.nin - c0) : q);
  if (nc <= 1) return;  // a lone child: identity
  const int64_t kchunk = (unit / a.nodes) * KC;
  const int kfull = (int)((a.k - kchunk) < KC ? (a.k - kchunk) : KC);
  const int kw = KC / pieces;  // columns of this CTA's piece (a power of two)
  const int64_t k0 = kchunk + (int64_t)piece * kw;
  const int kc = kfull - piece * kw < kw ? kfull - piece * kw : kw;
  if (kc <= 0) return;
  const int64_t nn = (int64_t)n * n;
  const T* Yn = a.Y + node * (int64_t)(q - 1) * nn;
  const T* Tg = a.Tw + node * nn;
  const int mode = a.mode;
  const bool trans = mode == kApplyQT;
  auto slot_ptr = [&](int b) -> T* { return a.C + (c0 + b) * a.slot_stride + k0 * a.ldc; };
  auto load_y = [&](int b) {
    const T* Yb = Yn + (int64_t)(b - 1) * nn;
    for (int idx = tid; idx < n * n; idx += NT) {
      const int i = idx % n, p = idx / n;
      Ys[p * ldn + i] = Yb[idx];
    }
  };

  {  // W = C_0 (form: X)
    const T* src = slot_ptr(0);
    for (int idx = tid; idx < n * kc; idx += NT) {
      const int i = idx % n, c = idx / n;
      B2[c * ldn + i] = src[i + (int64_t)c * a.ldc];
    }
  }
  const int PG = NT / kw;  // threads per column: one column per lane, PG rows apart
  const int cc = tid % kw, pg = tid / kw;
  const int nb4 = (n + 3) / 4;  // FP32 phases: blocks of four rows
  if (mode != kApplyForm) {
    // W += Y_b^T C_b; Y_b is upper triangular, so W(p) sums rows i <= p.
    for (int b = 1; b < nc; ++b) {
      __syncthreads();
      const T* src = slot_ptr(b);
      for (int idx = tid; idx < n * kc; idx += NT) {
        const int i = idx % n, c = idx / n;
        B1[c * ldn + i] = src[i + (int64_t)c * a.ldc];
      }
      load_y(b);
      __syncthreads();
      if constexpr (sizeof(T) == 4) {
        // FP32: items (column, four consecutive p), column fastest, so a
        // warp's Y loads are broadcasts; each C_b entry feeds four products.
        // Y_b(i, p) = 0 is stored for i > p, so running i to the block's
        // last p adds only exact zeros after each sum's own terms.
        for (int item = tid; item < kc * nb4; item += NT) {
          const int c = item % kc, p0 = 4 * (item / kc);
          T acc[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[j] = p0 + j < n ? B2[c * ldn + p0 + j] : T(0);
          const int iend = p0 + 4 < n ? p0 + 4 : n;
          for (int i = 0; i < iend; ++i) {
            const T x = B1[c * ldn + i];
#pragma unroll
            for (int j = 0; j < 4; ++j)
              if (p0 + j < n) acc[j] = fma(Ys[(p0 + j) * ldn + i], x, acc[j]);
          }
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (p0 + j < n) B2[c * ldn + p0 + j] = acc[j];
        }
      } else if (cc < kc) {
        for (int p = pg; p < n; p += PG) {
          T s = B2[cc * ldn + p];
          for (int i = 0; i <= p; ++i) s = fma(Ys[p * ldn + i], B1[cc * ldn + i], s);
          B2[cc * ldn + p] = s;
        }
      }
    }
  }
  __syncthreads();
  for (int idx = tid; idx < n * n; idx += NT) Ts[idx] = Tg[idx];
  __syncthreads();
  // W' = T^T W (Q^T) or T W (Q, form), into B1.
  if constexpr (sizeof(T) == 4) {
    // FP32: items (column, four consecutive p) as above; T's zeros below the
    // diagonal are stored, so the extra terms are exact zeros (leading for
    // T W, trailing for T^T W).
    for (int item = tid; item < kc * nb4; item += NT) {
      const int c = item % kc, p0 = 4 * (item / kc);
      T acc[4] = {T(0), T(0), T(0), T(0)};
      if (trans) {
        const int qend = p0 + 4 < n ? p0 + 4 : n;
        for (int qq = 0; qq < qend; ++qq) {
          const T x = B2[c * ldn + qq];
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (p0 + j < n) acc[j] = fma(Ts[qq + (p0 + j) * n], x, acc[j]);
        }
      } else {
        for (int qq = p0; qq < n; ++qq) {
          const T x = B2[c * ldn + qq];
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (p0 + j < n) acc[j] = fma(Ts[(p0 + j) + qq * n], x, acc[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (p0 + j < n) B1[c * ldn + p0 + j] = acc[j];
    }
  } else if (cc < kc) {
    for (int p = pg; p < n; p += PG) {
      T s = T(0);
      if (trans) {
        for (int qq = 0; qq <= p; ++qq) s = fma(Ts[qq + p * n], B2[cc * ldn + qq], s);
      } else {
        for (int qq = p; qq < n; ++qq) s = fma(Ts[p + qq * n], B2[cc * ldn + qq], s);
      }
      B1[cc * ldn + p] = s;
    }
  }
  __syncthreads();
  {  // C_0 <- C_0 - W'  (form: X - W')
    T* dst = slot_ptr(0);
    for (int idx = tid; idx < n * kc; idx += NT) {
      const int i = idx % n, c = idx / n;
      dst[i + (int64_t)c * a.ldc] -= B1[c * ldn + i];
    }
  }
  // C_b <- C_b - Y_b W'  (form: -Y_b W').
  for (int b = 1; b < nc; ++b) {
    __syncthreads();
    load_y(b);
    __syncthreads();
    if constexpr (sizeof(T) == 4) {
      // FP32: items (column, four consecutive rows i); Y_b(i, p) = 0 for
      // p < i is stored, so the leading extra terms are exact zeros.
      for (int item = tid; item < kc * nb4; item += NT) {
        const int c = item % kc, i0 = 4 * (item / kc);
        T acc[4] = {T(0), T(0), T(0), T(0)};
        for (int p = i0; p < n; ++p) {
          const T x = B1[c * ldn + p];
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (i0 + j < n) acc[j] = fma(Ys[p * ldn + i0 + j], x, acc[j]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (i0 + j < n) B2[c * ldn + i0 + j] = acc[j];
      }
    } else if (cc < kc) {
      for (int i = pg; i < n; i += PG) {
        T s = T(0);
        for (int p = i; p < n; ++p) s = fma(Ys[p * ldn + i], B1[cc * ldn + p], s);
        B2[cc * ldn + i] = s;
      }
    }
    __syncthreads();
    T* dst = slot_ptr(b);
    for (int idx = tid; idx < n * kc; idx += NT) {
      const int i = idx % n, c = idx / n;
      T* e = dst + i + (int64_t)c * a.ldc;
      *e = (mode == kApplyForm ? T(0) : *e) - B2[c * ldn + i];
    }
  }
}

// ------------------------------------------------------------ utilities --
template <typename T>
__global__ void sign_fix_kernel(const T* Rroot, int n, T* d, T* Rout, int64_t ldr, bool zero_lower) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n * n; idx += gridDim.x * blockDim.x) {
    const int i = idx % n, c = idx / n;
    const T di = Rroot[i + (int64_t)i * n] < T(0) ? T(-1) : T(1);
    if (i <= c) Rout[i + (int64_t)c * ldr] = di * Rroot[idx];
    else if (zero_lower) Rout[i + (int64_t)c * ldr] = T(0);
    if (c == 0) d[i] = di;
  }
}

template <typename T>
__global__ void scale_rows_kernel(T* C, int64_t ldc, int n, int64_t k, const T* d) {
  const int64_t total = (int64_t)n * k;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % n);
    const int64_t c = idx / n;
    C[i + c * ldc] *= d[i];
  }
}

template <typename T>
__global__ void init_form_kernel(T* Q, int64_t ldq, int n, const T* d) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n * n; idx += gridDim.x * blockDim.x) {
    const int i = idx % n, c = idx / n;
    Q[i + (int64_t)c * ldq] = i == c ? (d ? d[i] : T(1)) : T(0);
  }
}

// Q(0:n, 0:k) = diag(d) X (X n x k, ld ldx): the slot rows that start forming Q X.
template <typename T>
__global__ void init_form_mul_kernel(T* Q, int64_t ldq, int n, int64_t k, const T* d, const T* X, int64_t ldx) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)n * k;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % n);
    const int64_t c = idx / n;
    const T x = X[i + c * ldx];
    Q[i + c * ldq] = d ? d[i] * x : x;
  }
}

template <typename T>
__global__ void copy_upper_kernel(const T* src, int n, T* dst, int64_t ldd) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n * n; idx += gridDim.x * blockDim.x) {
    const int i = idx % n, c = idx / n;
    dst[i + (int64_t)c * ldd] = i <= c ? src[idx] : T(0);
  }
}

inline unsigned small_grid(int64_t work) {
  int64_t g = (work + 255) / 256;
  if (g < 1) g = 1;
  if (g > 4096) g = 4096;
  return (unsigned)g;
}

}  // namespace

size_t leaf_apply_smem(int n, size_t elem) {
  return align16(elem * kApplyRows * (n + 1)) + leaf_apply_cs_bytes(n, elem) +
         elem * (size_t)n * kApplyCols + (leaf_apply_t_shared(n, elem) ? 0 : elem * (size_t)n * n);
}

size_t node_apply_smem(int n, int q, size_t elem) {
  (void)q;
  const int ldn = n | 1;
  return elem * ((size_t)2 * kApplyCols * ldn + (size_t)n * ldn);
}

// Tail split of a grid of equal work units, one per CTA: with S resident
// CTAs, units = w S + f, and the last f units run as a partial wave.  Cut
// into p column pieces they take ceil(p f / S) / p of a wave instead of one
// (each piece costs a little more than its share: Y and T are staged again).
// p goes up to pmax, and to 4 whenever the 4 f pieces all run at once (then
// a piece's lower per-SM efficiency costs nothing).  Returns p (1: no
// split) and the first unit that is split.
template <typename K>
int tail_split(K kern, size_t smem, int64_t units, int pmax, int64_t* split_from) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kApplyThreads, smem);
  const int64_t S = (int64_t)(sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
  const int64_t f = units % S;
  int split = 1;
  double best = 1.0;
  for (int p = 2; f > 0 && p <= 4; p *= 2) {
    if (p > pmax && (int64_t)p * f > S) break;
    const double t = (double)((p * f + S - 1) / S) / p + 0.04 * (p - 1);
    if (t < best) {
      best = t;
      split = p;
    }
  }
  *split_from = split > 1 ? units - f : units;
  return split;
}

template <typename T>
cudaError_t launch_leaf_apply(const LeafApplyArgs<T>& a, cudaStream_t s) {
  if (a.nleaves <= 0 || a.k <= 0 || a.n <= 0) return cudaSuccess;
  const size_t smem = leaf_apply_smem(a.n, sizeof(T));
  auto kern = leaf_apply_kernel<T, kApplyThreads>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t kchunks = (a.k + kApplyCols - 1) / kApplyCols;
  const int64_t units = a.nleaves * kchunks;
  // Quarter pieces (16 columns) in the apply modes only when they all fit in
  // one round: there W = Y^T C runs over all h rows, and 16 columns give it
  // two warps per CTA.
  LeafApplyArgs<T> b = a;
  b.split = tail_split(kern, smem, units, a.mode == kApplyForm ? 4 : 2, &b.split_from);
  const int64_t grid = b.split_from + (units - b.split_from) * b.split;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  kern<<<(unsigned)grid, kApplyThreads, smem, s>>>(b);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_node_apply(const NodeApplyArgs<T>& a, cudaStream_t s) {
  if (a.nodes <= 0 || a.k <= 0 || a.n <= 0) return cudaSuccess;
  const size_t smem = node_apply_smem(a.n, a.arity, sizeof(T));
  auto kern = node_apply_kernel<T, kApplyThreads>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t kchunks = (a.k + kApplyCols - 1) / kApplyCols;
  NodeApplyArgs<T> b = a;
  b.split = tail_split(kern, smem, a.nodes * kchunks, 4, &b.split_from);
  const int64_t grid = b.split_from + (a.nodes * kchunks - b.split_from) * b.split;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  kern<<<(unsigned)grid, kApplyThreads, smem, s>>>(b);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sign_fix(const T* Rroot, int n, T* d, T* Rout, int64_t ldr, bool zero_lower, cudaStream_t s) {
  sign_fix_kernel<T><<<small_grid((int64_t)n * n), 256, 0, s>>>(Rroot, n, d, Rout, ldr, zero_lower);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scale_rows(T* C, int64_t ldc, int n, int64_t k, const T* d, cudaStream_t s) {
  if (k <= 0 || n <= 0) return cudaSuccess;
  scale_rows_kernel<T><<<small_grid((int64_t)n * k), 256, 0, s>>>(C, ldc, n, k, d);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_init_form_mul(T* Q, int64_t ldq, int n, int64_t k, const T* d, const T* X, int64_t ldx,
                                 cudaStream_t s) {
  init_form_mul_kernel<T><<<small_grid((int64_t)n * k), 256, 0, s>>>(Q, ldq, n, k, d, X, ldx);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_init_form(T* Q, int64_t ldq, int n, const T* d, cudaStream_t s) {
  init_form_kernel<T><<<small_grid((int64_t)n * n), 256, 0, s>>>(Q, ldq, n, d);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_copy_upper(const T* src, int n, T* dst, int64_t ldd, cudaStream_t s) {
  copy_upper_kernel<T><<<small_grid((int64_t)n * n), 256, 0, s>>>(src, n, dst, ldd);
  return cudaGetLastError();
}

#define TSQR_INSTANTIATE(T)                                                                          \
  template cudaError_t launch_leaf_apply<T>(const LeafApplyArgs<T>&, cudaStream_t);                  \
  template cudaError_t launch_node_apply<T>(const NodeApplyArgs<T>&, cudaStream_t);                  \
  template cudaError_t launch_sign_fix<T>(const T*, int, T*, T*, int64_t, bool, cudaStream_t);       \
  template cudaError_t launch_scale_rows<T>(T*, int64_t, int, int64_t, const T*, cudaStream_t);      \
  template cudaError_t launch_init_form<T>(T*, int64_t, int, const T*, cudaStream_t);                \
  template cudaError_t launch_init_form_mul<T>(T*, int64_t, int, int64_t, const T*, const T*, int64_t, cudaStream_t); \
  template cudaError_t launch_copy_upper<T>(const T*, int, T*, int64_t, cudaStream_t);
TSQR_INSTANTIATE(double)
TSQR_INSTANTIATE(float)
#undef TSQR_INSTANTIATE

}  // namespace tsqr
