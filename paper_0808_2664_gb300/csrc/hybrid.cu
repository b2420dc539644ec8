// Hybrid reduction tree (Section 2.1): a flat tree inside each CTA, a q-ary
// tree across CTAs.
//
// The leaves are cut into chains of L consecutive leaves, one chain per
// CTA.  Within a chain the flat tree of Section 2.1 runs: the first leaf is
// an ordinary leaf QR, and every later leaf i factors [R; A_i], the chain's
// running R stacked on its rows (the leaf kernel's stacked form), so that
// the chain reads its rows once and produces one R.  The q-ary tree then
// runs over the chains' R factors only: at m = 4,194,304, n = 64 about 150
// chains instead of about 10,000 leaves, four tree levels instead of seven.
//
// Q of a chain step i >= 1 is I - U T_i U^T with U = [I_n; Y_i]: its top
// block acts on the chain's "slot" (the n rows that carry the running R:
// the first n rows of the chain's first leaf), its dense block Y_i on leaf
// i's rows.  Applying it to C (m x k):
//     W = C_slot + Y_i^T C_i,  W' = T_i^T W (Q^T) or T_i W (Q),
//     C_slot -= W',  C_i -= Y_i W'.
// The first leaf is the same step with U = Y_0 (unit lower trapezoidal):
// its top block is the unit lower triangle of Y_0 on the slot rows.  Q^T
// runs the steps in chain order, Q and the thin-Q "form" in reverse; the
// slot stays in shared memory for the whole chain.
#include <cuda_runtime.h>

#include <cstdint>

#include "leaf_device.cuh"
#include "tsqr_internal.cuh"

namespace tsqr {

int leaf_factor_threads(int n, int ld, size_t elem);

namespace {

// FP32 chains, like FP32 leaves, keep two or more CTAs per SM (64 registers).
template <typename T, int NT, int NMAX>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 1024 / NT : 1) chain_factor_kernel(ChainFactorArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int64_t nn = (int64_t)a.n * a.n;
  for (int64_t chain = blockIdx.x; chain < a.nchains; chain += gridDim.x) {
    const int64_t l0 = chain * a.L;
    const int64_t l1 = l0 + a.L < a.nleaves ? l0 + a.L : a.nleaves;
    T* Rc = a.R + chain * nn;
    for (int64_t leaf = l0; leaf < l1; ++leaf) {
      const int64_t r0 = leaf * a.h;
      const int hl = (leaf == a.nleaves - 1) ? (int)(a.m - r0) : (int)a.h;
      if (leaf == l0)
        leaf_factor_one<T, NT, NMAX, true, false>(a.A + r0, a.lda, hl, a.n, a.ld_s, Rc, a.tau + leaf * (int64_t)a.n,
                                                  a.Tw + leaf * nn, a.status, smem);
      else
        leaf_factor_one<T, NT, NMAX, true, true>(a.A + r0, a.lda, a.n + hl, a.n, a.ld_s, Rc,
                                                 a.tau + leaf * (int64_t)a.n, a.Tw + leaf * nn, a.status, smem, Rc);
      __syncthreads();
    }
  }
}

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) / 16 * 16; }

constexpr int kChainRows = 32;  // rows of Y and C staged per pass
constexpr int kChainCols = 32;  // columns of C per CTA
constexpr int kChainThreads = 128;

// Shared memory: Ss [n][KC] slot, Ws [n][KC], Ts [n][n] column-major,
// Ys [RB][n+1] and Cs [RB][KC+1] staging.
template <typename T>
__host__ __device__ inline size_t chain_apply_smem_t(int n) {
  return al16(sizeof(T) * (size_t)n * kChainCols) * 2 + al16(sizeof(T) * (size_t)n * n) +
         al16(sizeof(T) * (size_t)kChainRows * (n + 1)) + al16(sizeof(T) * (size_t)kChainRows * (kChainCols + 1));
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT) chain_apply_kernel(ChainApplyArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int RB = kChainRows, KC = kChainCols;
  const int n = a.n;
  const int ly = n + 1, lc = KC + 1;
  T* Ss = reinterpret_cast<T*>(smem);
  T* Ws = reinterpret_cast<T*>(smem + al16(sizeof(T) * (size_t)n * KC));
  T* Ts = reinterpret_cast<T*>(smem + 2 * al16(sizeof(T) * (size_t)n * KC));
  T* Ys = reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(Ts) + al16(sizeof(T) * (size_t)n * n));
  T* Cs = reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(Ys) + al16(sizeof(T) * (size_t)RB * ly));
  const int tid = threadIdx.x;
  const int64_t chain = blockIdx.x % a.nchains;
  const int64_t k0 = (blockIdx.x / a.nchains) * (int64_t)KC;
  const int kc = (int)((a.k - k0) < KC ? (a.k - k0) : KC);
  if (kc <= 0) return;
  const int64_t l0 = chain * a.L;
  const int64_t l1 = l0 + a.L < a.nleaves ? l0 + a.L : a.nleaves;
  const int64_t slot_row = l0 * a.h;
  const int mode = a.mode;
  const bool trans = mode == kApplyQT;
  const bool form = mode == kApplyForm;
  T* Cslot = a.C + slot_row + k0 * a.ldc;

  // The slot (n x kc) stays here for the whole chain.
  for (int idx = tid; idx < n * KC; idx += NT) {
    const int i = idx % n, c = idx / n;
    Ss[i * KC + c] = c < kc ? Cslot[i + (int64_t)c * a.ldc] : T(0);
  }

  const int tp = (n + 3) / 4, tcn = KC / 4;
  const int ntiles = tp * tcn;
  constexpr int CG = NT / RB;
  const int64_t nsteps = l1 - l0;
  for (int64_t st = 0; st < nsteps; ++st) {
    const int64_t leaf = trans ? l0 + st : l1 - 1 - st;
    const bool first = leaf == l0;
    const int64_t r0 = leaf * a.h;
    const int hl = (leaf == a.nleaves - 1) ? (int)(a.m - r0) : (int)a.h;
    // Dense block: rows [rb0, hl) of the leaf; Y(r, p) read from storage.
    const int rb0 = first ? n : 0;
    const int rows = hl - rb0;
    const T* Yg = a.Y + r0 + rb0;
    T* Cg = a.C + r0 + rb0 + k0 * a.ldc;
    const T* Tg = a.Tw + leaf * (int64_t)n * n;
    const T* Ytop = a.Y + r0;  // first leaf: its unit lower triangle acts on the slot
    __syncthreads();
    for (int idx = tid; idx < n * n; idx += NT) Ts[idx] = Tg[idx];

    // Phase 1: W = U_top^T S + Y^T C over the dense rows (form: C = 0).
    // 4 x 4 register tiles of W, at most two per thread (n <= 128).
    T acc[2][4][4];
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[t][x][y] = T(0);
    if (!form) {
      for (int rb = 0; rb < rows; rb += RB) {
        __syncthreads();
        for (int idx = tid; idx < RB * n; idx += NT) {
          const int i = idx % RB, p = idx / RB, r = rb + i;
          Ys[i * ly + p] = r < rows ? Yg[r + (int64_t)p * a.ldy] : T(0);
        }
        for (int idx = tid; idx < RB * KC; idx += NT) {
          const int i = idx % RB, c = idx / RB, r = rb + i;
          Cs[i * lc + c] = (r < rows && c < kc) ? Cg[r + (int64_t)c * a.ldc] : T(0);
        }
        __syncthreads();
        const int rmax = rows - rb < RB ? rows - rb : RB;
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          const int tile = tid + t * NT;
          if (tile >= ntiles) break;
          const int p0 = (tile / tcn) * 4, c0 = (tile % tcn) * 4;
          for (int i = 0; i < rmax; ++i) {
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
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int tile = tid + t * NT;
      if (tile >= ntiles) break;
      const int p0 = (tile / tcn) * 4, c0 = (tile % tcn) * 4;
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        const int p = p0 + x;
        if (p >= n) continue;
        if (first) {
          // Sum over slot rows i >= p of Y_0(i, p) S(i, c), Y_0(p, p) = 1.
          for (int i = p; i < n; ++i) {
            const T u = i == p ? T(1) : Ytop[i + (int64_t)p * a.ldy];
#pragma unroll
            for (int y = 0; y < 4; ++y) acc[t][x][y] = fma(u, Ss[i * KC + c0 + y], acc[t][x][y]);
          }
        } else {
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[t][x][y] += Ss[p * KC + c0 + y];
        }
#pragma unroll
        for (int y = 0; y < 4; ++y) Ws[p * KC + c0 + y] = acc[t][x][y];
      }
    }
    __syncthreads();

    // Phase 2: W' = T^T W (Q^T) or T W (Q, form).
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
        if (p0 + x < n)
#pragma unroll
          for (int y = 0; y < 4; ++y) Ws[(p0 + x) * KC + c0 + y] = acc[t][x][y];
    }
    __syncthreads();

    // Phase 3a: slot S -= U_top W'.
    for (int idx = tid; idx < n * KC; idx += NT) {
      const int i = idx / KC, c = idx % KC;
      T s;
      if (first) {
        s = Ws[i * KC + c];  // U_top(i, i) = 1
        for (int p = 0; p < i; ++p) s = fma(Ytop[i + (int64_t)p * a.ldy], Ws[p * KC + c], s);
      } else {
        s = Ws[i * KC + c];
      }
      Ss[i * KC + c] -= s;
    }
    // Phase 3b: C -= Y W' over the dense rows (form: C = -Y W').
    const int ii = tid % RB, cg = tid / RB;
    for (int rb = 0; rb < rows; rb += RB) {
      __syncthreads();
      for (int idx = tid; idx < RB * n; idx += NT) {
        const int i = idx % RB, p = idx / RB, r = rb + i;
        Ys[i * ly + p] = r < rows ? Yg[r + (int64_t)p * a.ldy] : T(0);
      }
      __syncthreads();
      const int r = rb + ii;
      if (r < rows) {
        for (int c = cg; c < kc; c += CG) {
          T s = T(0);
          for (int p = 0; p < n; ++p) s = fma(Ys[ii * ly + p], Ws[p * KC + c], s);
          T* dst = Cg + r + (int64_t)c * a.ldc;
          const T old = form ? T(0) : *dst;
          *dst = old - s;
        }
      }
    }
  }
  __syncthreads();
  for (int idx = tid; idx < n * kc; idx += NT) {
    const int i = idx % n, c = idx / n;
    Cslot[i + (int64_t)c * a.ldc] = Ss[i * KC + c];
  }
}

}  // namespace

size_t chain_apply_smem(int n, size_t elem) {
  return elem == 8 ? chain_apply_smem_t<double>(n) : chain_apply_smem_t<float>(n);
}

template <typename T, int NT>
static int chain_resident_nt(int n, int ld) {
  const size_t smem = leaf_smem_bytes(n, ld, sizeof(T), NT);
  auto kern = n <= 64 ? chain_factor_kernel<T, NT, 64> : chain_factor_kernel<T, NT, kMaxN>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem) != cudaSuccess) return 0;
  return sms * per_sm;
}

// CTAs of the chain factor kernel resident at once on the whole GPU (the
// planner makes one chain per resident CTA), 0 if the tile does not fit.
int chain_factor_resident(int n, int ld, size_t elem) {
  const int nt = leaf_factor_threads(n, ld, elem);
  if (elem == 8) {
    if (nt == kLeafThreadsBig) return chain_resident_nt<double, kLeafThreadsBig>(n, ld);
    return nt == 256 ? chain_resident_nt<double, 256>(n, ld) : chain_resident_nt<double, 128>(n, ld);
  }
  if (nt == kLeafThreadsBig) return chain_resident_nt<float, kLeafThreadsBig>(n, ld);
  return nt == 256 ? chain_resident_nt<float, 256>(n, ld) : chain_resident_nt<float, 128>(n, ld);
}

template <typename T, int NT>
static cudaError_t launch_chain_factor_nt(const ChainFactorArgs<T>& a, cudaStream_t s) {
  const size_t smem = leaf_smem_bytes(a.n, a.ld_s, sizeof(T), NT);
  auto kern = a.n <= 64 ? chain_factor_kernel<T, NT, 64> : chain_factor_kernel<T, NT, kMaxN>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int64_t grid = (int64_t)sms * per_sm;
  if (grid > a.nchains) grid = a.nchains;
  kern<<<(unsigned)grid, NT, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_chain_factor(const ChainFactorArgs<T>& a, cudaStream_t s) {
  if (a.nchains <= 0 || a.n <= 0) return cudaSuccess;
  const int nt = leaf_factor_threads(a.n, a.ld_s, sizeof(T));
  if (nt == kLeafThreadsBig) return launch_chain_factor_nt<T, kLeafThreadsBig>(a, s);
  return nt == 256 ? launch_chain_factor_nt<T, 256>(a, s) : launch_chain_factor_nt<T, 128>(a, s);
}

template <typename T>
cudaError_t launch_chain_apply(const ChainApplyArgs<T>& a, cudaStream_t s) {
  if (a.nchains <= 0 || a.k <= 0 || a.n <= 0) return cudaSuccess;
  const size_t smem = chain_apply_smem_t<T>(a.n);
  cudaError_t e = cudaFuncSetAttribute(chain_apply_kernel<T, kChainThreads>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t kchunks = (a.k + kChainCols - 1) / kChainCols;
  const int64_t grid = a.nchains * kchunks;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  chain_apply_kernel<T, kChainThreads><<<(unsigned)grid, kChainThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_chain_factor<double>(const ChainFactorArgs<double>&, cudaStream_t);
template cudaError_t launch_chain_factor<float>(const ChainFactorArgs<float>&, cudaStream_t);
template cudaError_t launch_chain_apply<double>(const ChainApplyArgs<double>&, cudaStream_t);
template cudaError_t launch_chain_apply<float>(const ChainApplyArgs<float>&, cudaStream_t);

}  // namespace tsqr
