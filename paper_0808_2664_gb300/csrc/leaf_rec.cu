// Recursive leaf QR (Elmroth and Gustavson's RGEQR3, which Sections 2.1 and
// 3.3 name as a local QR for TSQR's leaves): to factor columns [c0, c1) of
// the leaf,
//   factor the left half [c0, mid) recursively (its Householder vectors Y_L
//   and compact-WY factor T_L),
//   update the right half A_R <- (I - Y_L T_L Y_L^T)^T A_R,
//   factor the right half [mid, c1) recursively (Y_R, T_R),
//   merge T = [T_L, -T_L (Y_L^T Y_R) T_R; 0, T_R],
// with one column as the base case (its reflector from the FP64 norm of its
// tail).  The updates and the merge are matrix-matrix products, so each
// element of the trailing block passes through them once per recursion
// level (log2 n times) instead of once per column.  The leaf tile stays in
// shared memory (column-major, odd leading dimension); every product
// distributes (output, row group) pairs over the CTA and sums the row groups
// in shared memory.  Products in the storage type; norms, beta, tau in FP64.
// Outputs match the column-by-column leaf kernel's: Householder vectors
// below the diagonal (unit diagonal implicit), R on and above, T (ld n), tau.
#include <cuda_runtime.h>

#include <cstdint>

#include "leaf_device.cuh"
#include "reflector.cuh"
#include "tsqr_internal.cuh"

namespace tsqr {
namespace {

constexpr int kRecThreads = 256;
constexpr int kRecMaxN = 64;

template <typename T>
struct RecSmem {
  T* S;        // tile, ld odd
  T* Tm;       // n x n T, ld n (column-major)
  T* W;        // kRecMaxN / 2 x kRecMaxN / 2 product buffer
  T* W2;       // same size
  T* part;     // kRecThreads partial sums
  double* pd;  // kRecThreads / 32 partial squared norms + scalars
  double* tau; // n
  int* cexp;   // n
};

__host__ __device__ inline size_t rec_al(size_t x) { return (x + 15) / 16 * 16; }

template <typename T>
__host__ __device__ inline size_t rec_smem_bytes(int n, int ld) {
  const int hw = kRecMaxN / 2;
  return rec_al(sizeof(T) * (size_t)n * ld) + rec_al(sizeof(T) * (size_t)n * n) + 2 * rec_al(sizeof(T) * hw * hw) +
         rec_al(sizeof(T) * kRecThreads) + rec_al(sizeof(double) * (kRecThreads / 32 + 8)) +
         rec_al(sizeof(double) * n) + rec_al(sizeof(int) * n);
}

template <typename T>
__device__ RecSmem<T> rec_carve(unsigned char* smem, int n, int ld) {
  const int hw = kRecMaxN / 2;
  RecSmem<T> m;
  unsigned char* p = smem;
  m.S = reinterpret_cast<T*>(p);
  p += rec_al(sizeof(T) * (size_t)n * ld);
  m.Tm = reinterpret_cast<T*>(p);
  p += rec_al(sizeof(T) * (size_t)n * n);
  m.W = reinterpret_cast<T*>(p);
  p += rec_al(sizeof(T) * hw * hw);
  m.W2 = reinterpret_cast<T*>(p);
  p += rec_al(sizeof(T) * hw * hw);
  m.part = reinterpret_cast<T*>(p);
  p += rec_al(sizeof(T) * kRecThreads);
  m.pd = reinterpret_cast<double*>(p);
  p += rec_al(sizeof(double) * (kRecThreads / 32 + 8));
  m.tau = reinterpret_cast<double*>(p);
  p += rec_al(sizeof(double) * n);
  m.cexp = reinterpret_cast<int*>(p);
  return m;
}

// Entry (r, p) of the Householder vectors of column block [c0, c0 + w):
// unit at r = c0 + p, zero above, the stored tail below.
template <typename T>
__device__ __forceinline__ T yval(const T* S, int ld, int c0, int r, int p) {
  const int c = c0 + p;
  return r < c ? T(0) : (r == c ? T(1) : S[c * ld + r]);
}

// W (w x w2, ld w2... row-major [p][q]) = Y(:, cy0 .. cy0+w)^T X(:, cx0 .. cx0+w2)
// over rows [r0, hl), where X is Householder vectors (xhh) or plain tile columns.
template <typename T>
__device__ void rec_gemm_tn(const RecSmem<T>& sm, int ld, int hl, int r0, int cy0, int w, int cx0, int w2, bool xhh,
                            T* W) {
  const int tid = threadIdx.x;
  const int outs = w * w2;
  const int rows = hl - r0;
  if (outs >= kRecThreads / 4) {
    // One thread per output (or several), whole row range.
    for (int o = tid; o < outs; o += kRecThreads) {
      const int p = o / w2, q = o % w2;
      const int rs = r0 > cy0 + p ? r0 : cy0 + p;  // Y is zero above its unit entry
      T a0 = T(0), a1 = T(0);
      int r = rs;
      for (; r + 1 < hl; r += 2) {
        const T x0 = xhh ? yval(sm.S, ld, cx0, r, q) : sm.S[(cx0 + q) * ld + r];
        const T x1 = xhh ? yval(sm.S, ld, cx0, r + 1, q) : sm.S[(cx0 + q) * ld + r + 1];
        a0 = fma(yval(sm.S, ld, cy0, r, p), x0, a0);
        a1 = fma(yval(sm.S, ld, cy0, r + 1, p), x1, a1);
      }
      if (r < hl) a0 = fma(yval(sm.S, ld, cy0, r, p), xhh ? yval(sm.S, ld, cx0, r, q) : sm.S[(cx0 + q) * ld + r], a0);
      W[p * w2 + q] = a0 + a1;
    }
    __syncthreads();
    return;
  }
  // Few outputs: G row groups per output, partial sums, then a sum over groups.
  const int G = kRecThreads / outs;
  if (tid < outs * G) {
    const int o = tid % outs, g = tid / outs;
    const int p = o / w2, q = o % w2;
    T a = T(0);
    for (int r = r0 + g; r < hl; r += G) {
      const T x = xhh ? yval(sm.S, ld, cx0, r, q) : sm.S[(cx0 + q) * ld + r];
      a = fma(yval(sm.S, ld, cy0, r, p), x, a);
    }
    sm.part[tid] = a;
  }
  __syncthreads();
  for (int o = tid; o < outs; o += kRecThreads) {
    T a = T(0);
    for (int g = 0; g < G; ++g) a += sm.part[o + g * outs];
    W[o] = a;
  }
  __syncthreads();
  (void)rows;
}

}  // namespace
}  // namespace tsqr

namespace tsqr {
namespace {

// Base case: the reflector of column c over rows [c, hl).
template <typename T>
__device__ void rec_column(RecSmem<T>& sm, int ld, int hl, int c, int n, int* status) {
  constexpr int NW = kRecThreads / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  T* col = sm.S + c * ld;
  double ss = 0.0;
  for (int r = c + 1 + tid; r < hl; r += kRecThreads) {
    const double x = (double)col[r];
    ss = fma(x, x, ss);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  if (lane == 0) sm.pd[warp] = ss;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < NW; ++w) s += sm.pd[w];
    const double alpha = (double)col[c];
    const int len = hl - c - 1;
    const Reflector rf = make_reflector_fast(
        alpha, s, [&]() { return scaled_norm(len, [&](int i) { return (double)col[c + 1 + i]; }); }, status);
    sm.pd[NW] = rf.scale;
    sm.pd[NW + 1] = rf.beta;
    sm.tau[c] = rf.tau;
    sm.Tm[c + c * n] = (T)rf.tau;
  }
  __syncthreads();
  const double scale = sm.pd[NW];
  for (int r = c + 1 + tid; r < hl; r += kRecThreads) col[r] = (T)((double)col[r] * scale);
  if (tid == 0) col[c] = (T)sm.pd[NW + 1];
  __syncthreads();
}

// A_R <- (I - Y_L T_L Y_L^T)^T A_R: left block [c0, mid), right block [mid, c1), rows [c0, hl).
template <typename T>
__device__ void rec_update(RecSmem<T>& sm, int ld, int hl, int n, int c0, int mid, int c1) {
  const int tid = threadIdx.x;
  const int w = mid - c0, w2 = c1 - mid;
  rec_gemm_tn(sm, ld, hl, c0, c0, w, mid, w2, false, sm.W);  // W = Y_L^T A_R
  for (int o = tid; o < w * w2; o += kRecThreads) {           // W2 = T_L^T W
    const int p = o / w2, q = o % w2;
    T s = T(0);
    for (int pp = 0; pp <= p; ++pp) s = fma(sm.Tm[(c0 + pp) + (c0 + p) * n], sm.W[pp * w2 + q], s);
    sm.W2[o] = s;
  }
  __syncthreads();
  const int rows = hl - c0;
  for (int idx = tid; idx < rows * w2; idx += kRecThreads) {  // A_R -= Y_L W2
    const int i = idx % rows, q = idx / rows, r = c0 + i;
    const int pmax = i + 1 < w ? i + 1 : w;
    T s = T(0);
    for (int p = 0; p < pmax; ++p) s = fma(yval(sm.S, ld, c0, r, p), sm.W2[p * w2 + q], s);
    sm.S[(mid + q) * ld + r] -= s;
  }
  __syncthreads();
}

// T(c0:mid, mid:c1) = -T_L (Y_L^T Y_R) T_R.
template <typename T>
__device__ void rec_merge(RecSmem<T>& sm, int ld, int hl, int n, int c0, int mid, int c1) {
  const int tid = threadIdx.x;
  const int w = mid - c0, w2 = c1 - mid;
  rec_gemm_tn(sm, ld, hl, mid, c0, w, mid, w2, true, sm.W);  // W = Y_L^T Y_R (Y_R is zero above row mid)
  for (int o = tid; o < w * w2; o += kRecThreads) {          // W2 = W T_R
    const int p = o / w2, q = o % w2;
    T s = T(0);
    for (int qq = 0; qq <= q; ++qq) s = fma(sm.W[p * w2 + qq], sm.Tm[(mid + qq) + (mid + q) * n], s);
    sm.W2[o] = s;
  }
  __syncthreads();
  for (int o = tid; o < w * w2; o += kRecThreads) {  // T12 = -T_L W2
    const int p = o / w2, q = o % w2;
    T s = T(0);
    for (int pp = p; pp < w; ++pp) s = fma(sm.Tm[(c0 + p) + (c0 + pp) * n], sm.W2[pp * w2 + q], s);
    sm.Tm[(c0 + p) + (mid + q) * n] = -s;
  }
  __syncthreads();
}

// RGEQR3's recursion on columns [0, n), run as a loop over an explicit stack
// of (c0, c1, stage) frames (stage 0: factor the left half next; 1: update
// the right half and factor it; 2: merge the two T factors), so that the
// kernel needs no call stack.  n <= 64 keeps the depth at most 7.
constexpr int kRecDepth = 8;

template <typename T>
__device__ void rec_factor(RecSmem<T>& sm, int ld, int hl, int n, int* status) {
  int f0[kRecDepth], f1[kRecDepth], fs[kRecDepth];
  int sp = 0;
  f0[0] = 0;
  f1[0] = n;
  fs[0] = 0;
  sp = 1;
  while (sp > 0) {
    const int c0 = f0[sp - 1], c1 = f1[sp - 1], st = fs[sp - 1];
    if (c1 - c0 == 1) {
      rec_column(sm, ld, hl, c0, n, status);
      --sp;
      continue;
    }
    const int mid = c0 + (c1 - c0 + 1) / 2;
    if (st == 2) {
      rec_merge(sm, ld, hl, n, c0, mid, c1);
      --sp;
      continue;
    }
    if (st == 1) rec_update(sm, ld, hl, n, c0, mid, c1);
    fs[sp - 1] = st + 1;
    if (sp == kRecDepth) {  // cannot happen for n <= 64; never overrun the frames
      if (threadIdx.x == 0) atomicOr(status, kStatusTimeout);
      return;
    }
    f0[sp] = st == 0 ? c0 : mid;
    f1[sp] = st == 0 ? mid : c1;
    fs[sp] = 0;
    ++sp;
  }
}

template <typename T>
__global__ void __launch_bounds__(kRecThreads) leaf_rec_kernel(LeafFactorArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = a.n, ld = a.ld_s;
  RecSmem<T> sm = rec_carve<T>(smem, n, ld);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t nn = (int64_t)n * n;
  for (int64_t leaf = blockIdx.x; leaf < a.nleaves; leaf += gridDim.x) {
    const int64_t r0 = leaf * a.h;
    const int hl = (leaf == a.nleaves - 1) ? (int)(a.m - r0) : (int)a.h;
    const T* Ag = a.A + r0;
    for (int idx = tid; idx < hl * n; idx += kRecThreads) {
      const int i = idx % hl, c = idx / hl;
      sm.S[c * ld + i] = Ag[(int64_t)c * a.lda + i];
    }
    for (int idx = tid; idx < n * n; idx += kRecThreads) sm.Tm[idx] = T(0);
    __syncthreads();
    // Each column scaled by the power of two that brings its largest entry
    // to [1/2, 1) (exact; R carries the factors, Q is unchanged).
    for (int c = warp; c < n; c += kRecThreads / 32) {
      unsigned mx = 0u;
      for (int i = lane; i < hl; i += 32) {
        const T x = sm.S[c * ld + i];
        const unsigned bits = sizeof(T) == 8 ? (unsigned)__double2hiint((double)x) : __float_as_uint((float)x);
        const unsigned v = bits & 0x7fffffffu;
        mx = v > mx ? v : mx;
      }
      mx = __reduce_max_sync(0xffffffffu, mx);
      if (lane == 0) sm.cexp[c] = column_exp2<T>(mx);
    }
    __syncthreads();
    for (int idx = tid; idx < hl * n; idx += kRecThreads) {
      const int i = idx % hl, c = idx / hl;
      sm.S[c * ld + i] *= pow2_bits<T>(sm.cexp[c]);
    }
    __syncthreads();
    rec_factor(sm, ld, hl, n, a.status);
    // Write back: vectors below the diagonal, R with the column factors taken out.
    T* Ao = a.A + r0;
    for (int idx = tid; idx < hl * n; idx += kRecThreads) {
      const int i = idx % hl, c = idx / hl;
      const T v = sm.S[c * ld + i];
      Ao[(int64_t)c * a.lda + i] = i <= c ? v * pow2_bits<T>(-sm.cexp[c]) : v;
    }
    T* Rl = a.R + leaf * nn;
    for (int idx = tid; idx < n * n; idx += kRecThreads) {
      const int i = idx % n, c = idx / n;
      Rl[idx] = i <= c ? sm.S[c * ld + i] * pow2_bits<T>(-sm.cexp[c]) : T(0);
    }
    for (int c = tid; c < n; c += kRecThreads) a.tau[leaf * n + c] = (T)sm.tau[c];
    if (a.Tw)
      for (int idx = tid; idx < n * n; idx += kRecThreads) a.Tw[leaf * nn + idx] = sm.Tm[idx];
    __syncthreads();
  }
}

}  // namespace

size_t leaf_rec_smem(int n, int ld, size_t elem) {
  return elem == 8 ? rec_smem_bytes<double>(n, ld) : rec_smem_bytes<float>(n, ld);
}

template <typename T>
cudaError_t launch_leaf_factor_rec(const LeafFactorArgs<T>& a, cudaStream_t s) {
  if (a.nleaves <= 0 || a.n <= 0) return cudaSuccess;
  if (a.n > kRecMaxN) return cudaErrorInvalidValue;
  const size_t smem = rec_smem_bytes<T>(a.n, a.ld_s);
  auto kern = leaf_rec_kernel<T>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRecThreads, smem);
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int64_t grid = (int64_t)sms * per_sm;
  if (grid > a.nleaves) grid = a.nleaves;
  kern<<<(unsigned)grid, kRecThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_leaf_factor_rec<double>(const LeafFactorArgs<double>&, cudaStream_t);
template cudaError_t launch_leaf_factor_rec<float>(const LeafFactorArgs<float>&, cudaStream_t);

}  // namespace tsqr
