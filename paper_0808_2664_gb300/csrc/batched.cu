// Batched uneven TSQR: thousands of independent tall-skinny matrices of
// different m and n factored by ONE persistent kernel launch.
//
// Every matrix gets its own leaf partition and reduction tree (Section 2.1:
// any tree shape gives the same R).  The host flattens all leaves of all
// matrices, then all level-1 nodes, level-2 nodes, ... into one work list;
// resident CTAs claim items in that order from a global counter.  A tree node
// waits (bounded spin) until all its children have signalled completion
// through a per-node counter.  Because items are claimed in list order and
// children always precede their parent, every child of a claimed node is
// already held by a running CTA, so the waits always end.  A wait that
// exceeds its iteration limit sets the timeout bit of the status word and
// the node is skipped instead of hanging the GPU.  The CTA that finishes a
// matrix's root writes the sign-normalised R.
//
// The launch sequence (counter reset + kernel) can be captured once in a
// CUDA graph and replayed.  An autotuner picks the leaf tile size and the
// tree arity by timing candidates on scratch matrices of the batch's shapes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <new>
#include <vector>

#include "../../include/tsqr.h"
#include "leaf_device.cuh"
#include "node2_device.cuh"
#include "node_device.cuh"
#include "tsqr_internal.cuh"

namespace tsqr {
namespace {

constexpr uint32_t kBatchMagic = 0x42545352u;  // "BTSR"
constexpr int kBatchNmax = 64;
constexpr long long kWaitLimit = 1ll << 22;    // spin iterations (x ~256 ns)

template <typename T>
struct BMat {
  T* A;
  int64_t lda;
  T* R;
  int64_t ldr;
  int64_t m;
  int32_t n;
  int32_t q;
  int64_t h;
  int64_t nleaves;
  int32_t levels;
  int32_t ld_s;
  T* leafR;
  T* leafTau;
  T* d;
  int32_t lvl0;  // index of this matrix's level 1 in the level table
  int32_t pad;
};

template <typename T>
struct BLevel {
  T* R;
  T* Y;
  T* tau;
  int64_t items;
  int64_t counter_base;
};

struct BItem {
  int32_t mat;
  int32_t level;  // 0 = leaf
  int64_t idx;
};

template <typename T>
struct BatchArgs {
  const BMat<T>* mats;
  const BLevel<T>* levels;
  const BItem* items;
  int64_t nitems;
  unsigned long long* next;  // claim counter
  int* counters;             // per-node completed-children counts
  int* status;
};

template <typename T>
__device__ void root_finish(const BMat<T>& M, const T* root) {
  const int n = M.n;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx % n, c = idx / n;
    const T di = root[i + (int64_t)i * n] < T(0) ? T(-1) : T(1);
    M.R[i + (int64_t)c * M.ldr] = i <= c ? di * root[idx] : T(0);
    if (c == 0) M.d[i] = di;
  }
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT) batch_kernel(BatchArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long sh_item;
  __shared__ int sh_ok;
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) sh_item = (long long)atomicAdd(a.next, 1ull);
    __syncthreads();
    const long long it = sh_item;
    __syncthreads();
    if (it >= a.nitems) break;
    const BItem w = a.items[it];
    const BMat<T> M = a.mats[w.mat];
    const int n = M.n;
    const int64_t nn = (int64_t)n * n;
    const T* done_r = nullptr;  // R written by this item
    int parent_level = w.level + 1;
    int64_t parent_idx = w.idx / M.q;
    if (w.level == 0) {
      const int64_t r0 = w.idx * M.h;
      const int hl = (w.idx == M.nleaves - 1) ? (int)(M.m - r0) : (int)M.h;
      // R only: no T for the leaves.
      leaf_factor_one<T, NT, kBatchNmax, false>(M.A + r0, M.lda, hl, n, M.ld_s, M.leafR + w.idx * nn,
                                                M.leafTau + w.idx * (int64_t)n, nullptr, a.status, smem);
      done_r = M.leafR + w.idx * nn;
    } else {
      const BLevel<T> L = a.levels[M.lvl0 + w.level - 1];
      const int64_t nin = w.level == 1 ? M.nleaves : a.levels[M.lvl0 + w.level - 2].items;
      const T* Rin = w.level == 1 ? M.leafR : a.levels[M.lvl0 + w.level - 2].R;
      const int64_t c0 = w.idx * M.q;
      const int nc = (int)((nin - c0) < M.q ? (nin - c0) : M.q);
      if (tid == 0) {
        const volatile int* ctr = a.counters + L.counter_base + w.idx;
        long long spins = 0;
        int ok = 1;
        while (*ctr < nc) {
          __nanosleep(256);
          if (++spins > kWaitLimit) {
            atomicOr(a.status, kStatusTimeout);
            ok = 0;
            break;
          }
        }
        __threadfence();
        sh_ok = ok;
      }
      __syncthreads();
      if (sh_ok) {
        // Arity 2 and 4: the lock-step node kernel with one node per CTA and
        // no T; other arities: the general one.
        if (M.q == 2)
          node2_factor_group<T, NT, 1, 2, false>(Rin, nin, L.items, w.idx, n, L.R, L.Y, nullptr, L.tau, a.status,
                                                 smem);
        else if (M.q == 4)
          node2_factor_group<T, NT, 1, 4, false>(Rin, nin, L.items, w.idx, n, L.R, L.Y, nullptr, L.tau, a.status,
                                                 smem);
        else
          node_factor_one<T, NT, false>(Rin + c0 * nn, nc, M.q, n, L.R + w.idx * nn,
                                        L.Y + w.idx * (int64_t)(M.q - 1) * nn, nullptr, L.tau + w.idx * (int64_t)n,
                                        a.status, smem);
      }
      done_r = L.R + w.idx * nn;
    }
    __threadfence();  // this item's R is visible device-wide before the parent is signalled
    __syncthreads();
    if (w.level == M.levels) {
      root_finish(M, done_r);
    } else if (tid == 0) {
      __threadfence();
      const BLevel<T> P = a.levels[M.lvl0 + parent_level - 1];
      atomicAdd(a.counters + P.counter_base + parent_idx, 1);
    }
    __syncthreads();
  }
}

// Fills x[0..count) with values uniform in [-1, 1) from a counter-based hash.
template <typename T>
__global__ void fill_uniform_kernel(T* x, int64_t count, uint64_t seed) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + 0x9e3779b97f4a7c15ull * (uint64_t)(i + 1);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
    x[i] = (T)((double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0);
  }
}

}  // namespace
}  // namespace tsqr

using namespace tsqr;

struct tsqr_batch_s {
  uint32_t magic = kBatchMagic;
  int32_t prec = TSQR_PREC_FP32;
  size_t es = 4;
  int32_t count = 0;
  int32_t tile_kb = 0, arity = 2;
  int64_t nitems = 0;
  size_t ws_bytes = 0, smem = 0;
  unsigned char* ws = nullptr;  // device: workspace + tables + counters
  void* mats = nullptr;
  void* levels = nullptr;
  BItem* items = nullptr;
  unsigned long long* next = nullptr;
  int* counters = nullptr;
  int64_t ncounters = 0;
  int* status = nullptr;
  int grid = 0;
  cudaGraphExec_t graph = nullptr;
  cudaStream_t graph_stream = nullptr;
};

namespace {

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

int64_t pick_h(int64_t n, size_t es, int tile_kb) {
  const int64_t budget = (int64_t)tile_kb * 1024 / (int64_t)es;
  int64_t h = 1;
  while (h * 2 <= budget / n && h * 2 <= 4096) h *= 2;
  if (h < n) h = n;
  return h;
}

int default_tile_kb(size_t es) { return es == 8 ? 68 : 136; }

template <typename T>
int build_batch(tsqr_batch_s* b, const int64_t* m, const int64_t* n, void* const* A, const int64_t* lda,
                void* const* R, const int64_t* ldr, cudaStream_t s) {
  constexpr int NT = sizeof(T) == 8 ? kLeafThreads64 : kLeafThreads32;
  const int cnt = b->count;
  const size_t es = sizeof(T);
  std::vector<BMat<T>> mats(cnt);
  std::vector<BLevel<T>> levels;
  std::vector<std::vector<int64_t>> items_per(cnt);
  size_t smem = 0;
  size_t off = 0;
  int64_t ncounters = 0;
  // Pass 1: plans and workspace offsets (stored as offsets, rebased below).
  for (int i = 0; i < cnt; ++i) {
    BMat<T>& M = mats[i];
    const int64_t mi = m[i], ni = n[i];
    M.m = mi;
    M.n = (int)ni;
    M.q = b->arity;
    M.lda = lda[i];
    M.ldr = ldr[i];
    M.A = (T*)A[i];
    M.R = (T*)R[i];
    int64_t h = pick_h(ni, es, b->tile_kb);
    int64_t nl = (mi + h - 1) / h;
    if (nl > 1 && mi - (nl - 1) * h < ni) --nl;
    const int64_t hmax = nl > 1 ? std::max(mi - (nl - 1) * h, h) : mi;
    M.h = h;
    M.nleaves = nl;
    M.ld_s = leaf_factor_ld((int)hmax);
    smem = std::max(smem, leaf_smem_bytes((int)ni, M.ld_s, es, NT));
    const size_t nnb = (size_t)ni * ni * es, nvb = (size_t)ni * es;
    M.leafR = (T*)off;
    off += al256(nl * nnb);
    M.leafTau = (T*)off;
    off += al256(nl * nvb);
    M.d = (T*)off;
    off += al256(nvb);
    std::vector<int64_t>& its = items_per[i];
    its.push_back(nl);
    while (its.back() > 1) its.push_back((its.back() + b->arity - 1) / b->arity);
    M.levels = (int32_t)its.size() - 1;
    M.lvl0 = (int32_t)levels.size();
    for (int l = 1; l <= M.levels; ++l) {
      BLevel<T> L;
      L.items = its[l];
      L.R = (T*)off;
      off += al256(its[l] * nnb);
      L.Y = (T*)off;
      off += al256(its[l] * (b->arity - 1) * nnb);
      L.tau = (T*)off;
      off += al256(its[l] * nvb);
      L.counter_base = ncounters;
      ncounters += its[l];
      levels.push_back(L);
    }
    if (M.levels > 0)
      smem = std::max(smem, b->arity == 2 || b->arity == 4 ? node2_smem_bytes((int)ni, 1, es, NT, b->arity)
                                                           : node_smem_bytes((int)ni, b->arity, es, NT));
  }
  int dev = 0, smax = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (smem > (size_t)smax) return TSQR_ERR_UNSUPPORTED;
  // Work list: leaves (largest first), then nodes level by level.
  std::vector<BItem> items;
  for (int i = 0; i < cnt; ++i)
    for (int64_t k = 0; k < mats[i].nleaves; ++k) items.push_back({i, 0, k});
  std::stable_sort(items.begin(), items.end(), [&](const BItem& x, const BItem& y) {
    const double cx = (double)mats[x.mat].h * mats[x.mat].n * mats[x.mat].n;
    const double cy = (double)mats[y.mat].h * mats[y.mat].n * mats[y.mat].n;
    return cx > cy;
  });
  int maxlev = 0;
  for (int i = 0; i < cnt; ++i) maxlev = std::max(maxlev, (int)mats[i].levels);
  for (int l = 1; l <= maxlev; ++l) {
    const size_t start = items.size();
    for (int i = 0; i < cnt; ++i)
      if (mats[i].levels >= l)
        for (int64_t k = 0; k < items_per[i][l]; ++k) items.push_back({i, l, k});
    std::stable_sort(items.begin() + start, items.end(),
                     [&](const BItem& x, const BItem& y) { return mats[x.mat].n > mats[y.mat].n; });
  }
  // Tables and counters after the workspace.
  const size_t off_mats = off;
  off += al256(sizeof(BMat<T>) * cnt);
  const size_t off_lv = off;
  off += al256(sizeof(BLevel<T>) * std::max<size_t>(levels.size(), 1));
  const size_t off_items = off;
  off += al256(sizeof(BItem) * items.size());
  const size_t off_next = off;
  off += al256(sizeof(unsigned long long));
  const size_t off_ctr = off;
  off += al256(sizeof(int) * std::max<int64_t>(ncounters, 1));
  const size_t off_status = off;
  off += al256(sizeof(int));
  void* base = nullptr;
  cudaError_t e = cudaMalloc(&base, off);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? TSQR_ERR_NOMEM : TSQR_ERR_CUDA;
  unsigned char* B = (unsigned char*)base;
  auto rebase = [&](T* p) { return (T*)(B + (size_t)p); };
  for (auto& M : mats) {
    M.leafR = rebase(M.leafR);
    M.leafTau = rebase(M.leafTau);
    M.d = rebase(M.d);
  }
  for (auto& L : levels) {
    L.R = rebase(L.R);
    L.Y = rebase(L.Y);
    L.tau = rebase(L.tau);
  }
  b->ws = B;
  b->ws_bytes = off;
  b->mats = B + off_mats;
  b->levels = B + off_lv;
  b->items = (BItem*)(B + off_items);
  b->next = (unsigned long long*)(B + off_next);
  b->counters = (int*)(B + off_ctr);
  b->ncounters = ncounters;
  b->status = (int*)(B + off_status);
  b->nitems = (int64_t)items.size();
  b->smem = smem;
  e = cudaMemcpyAsync(b->mats, mats.data(), sizeof(BMat<T>) * cnt, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !levels.empty())
    e = cudaMemcpyAsync(b->levels, levels.data(), sizeof(BLevel<T>) * levels.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->items, items.data(), sizeof(BItem) * items.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->status, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host tables go out of scope
  if (e != cudaSuccess) return TSQR_ERR_CUDA;
  auto kern = batch_kernel<T, NT>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return TSQR_ERR_CUDA;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
  if (per_sm < 1) return TSQR_ERR_UNSUPPORTED;
  b->grid = sms * per_sm;
  return TSQR_OK;
}

template <typename T>
cudaError_t launch_batch(tsqr_batch_s* b, cudaStream_t s) {
  constexpr int NT = sizeof(T) == 8 ? kLeafThreads64 : kLeafThreads32;
  cudaError_t e = cudaMemsetAsync(b->next, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess && b->ncounters > 0) e = cudaMemsetAsync(b->counters, 0, sizeof(int) * b->ncounters, s);
  if (e != cudaSuccess) return e;
  BatchArgs<T> a;
  a.mats = (const BMat<T>*)b->mats;
  a.levels = (const BLevel<T>*)b->levels;
  a.items = b->items;
  a.nitems = b->nitems;
  a.next = b->next;
  a.counters = b->counters;
  a.status = b->status;
  int64_t grid = b->grid;
  if (grid > b->nitems) grid = b->nitems;
  if (grid < 1) return cudaSuccess;
  batch_kernel<T, NT><<<(unsigned)grid, NT, b->smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_any(tsqr_batch_s* b, cudaStream_t s) {
  return b->prec == TSQR_PREC_FP64 ? launch_batch<double>(b, s) : launch_batch<float>(b, s);
}

void free_batch(tsqr_batch_s* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->ws) cudaFree(b->ws);
  b->graph = nullptr;
  b->ws = nullptr;
}

int create_batch(int32_t count, const int64_t* m, const int64_t* n, void* const* A, const int64_t* lda,
                 void* const* R, const int64_t* ldr, int32_t prec, int tile_kb, int arity, tsqr_batch_s** out,
                 cudaStream_t s) {
  tsqr_batch_s* b = new (std::nothrow) tsqr_batch_s();
  if (!b) return TSQR_ERR_NOMEM;
  b->prec = prec;
  b->es = prec == TSQR_PREC_FP64 ? 8 : 4;
  b->count = count;
  b->tile_kb = tile_kb;
  b->arity = arity;
  const int rc = prec == TSQR_PREC_FP64 ? build_batch<double>(b, m, n, A, lda, R, ldr, s)
                                        : build_batch<float>(b, m, n, A, lda, R, ldr, s);
  if (rc != TSQR_OK) {
    free_batch(b);
    delete b;
    return rc;
  }
  *out = b;
  return TSQR_OK;
}

// Autotuner: times every (tile size, arity) candidate on scratch matrices of
// the batch's shapes (uniform random values; the caller's matrices are not
// touched) and returns the fastest.
int autotune(int32_t count, const int64_t* m, const int64_t* n, int32_t prec, int* best_kb, int* best_q,
             cudaStream_t s) {
  const size_t es = prec == TSQR_PREC_FP64 ? 8 : 4;
  std::vector<size_t> offs(count);
  size_t total = 0;
  for (int i = 0; i < count; ++i) {
    offs[i] = total;
    total += al256((size_t)m[i] * n[i] * es);
  }
  size_t rtotal = 0;
  for (int i = 0; i < count; ++i) rtotal += al256((size_t)n[i] * n[i] * es);
  void *scratch = nullptr, *rscr = nullptr;
  if (cudaMalloc(&scratch, total) != cudaSuccess) return TSQR_ERR_NOMEM;
  if (cudaMalloc(&rscr, rtotal) != cudaSuccess) {
    cudaFree(scratch);
    return TSQR_ERR_NOMEM;
  }
  std::vector<void*> Ap(count), Rp(count);
  std::vector<int64_t> lda(count), ldr(count);
  size_t roff = 0;
  for (int i = 0; i < count; ++i) {
    Ap[i] = (unsigned char*)scratch + offs[i];
    Rp[i] = (unsigned char*)rscr + roff;
    roff += al256((size_t)n[i] * n[i] * es);
    lda[i] = m[i];
    ldr[i] = n[i];
  }
  auto refill = [&]() {
    const int64_t elems = (int64_t)(total / es);
    if (es == 8)
      fill_uniform_kernel<double><<<1024, 256, 0, s>>>((double*)scratch, elems, 12345);
    else
      fill_uniform_kernel<float><<<1024, 256, 0, s>>>((float*)scratch, elems, 12345);
  };
  // Smaller tiles let more leaf CTAs share an SM (the leaf column loop is
  // latency-bound); larger ones make shorter trees.
  const int kbs64[] = {24, 34, 68, 136}, kbs32[] = {34, 48, 68, 136};
  const int qs[] = {2, 4, 8};
  float best = 1e30f;
  *best_kb = default_tile_kb(es);
  *best_q = 2;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int ki = 0; ki < 4; ++ki) {
    for (int qi = 0; qi < 3; ++qi) {
      const int kb = es == 8 ? kbs64[ki] : kbs32[ki];
      tsqr_batch_s* b = nullptr;
      if (create_batch(count, m, n, Ap.data(), lda.data(), Rp.data(), ldr.data(), prec, kb, qs[qi], &b, s) != TSQR_OK)
        continue;
      float t = 0.f;
      for (int rep = 0; rep < 3; ++rep) {
        refill();
        cudaEventRecord(e0, s);
        launch_any(b, s);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) t += ms;  // the first run is a warm-up
      }
      int st = 0;
      cudaMemcpy(&st, b->status, sizeof(int), cudaMemcpyDeviceToHost);
      if (st == 0 && t < best) {
        best = t;
        *best_kb = kb;
        *best_q = qs[qi];
      }
      free_batch(b);
      delete b;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(scratch);
  cudaFree(rscr);
  return best < 1e29f ? TSQR_OK : TSQR_ERR_UNSUPPORTED;
}

}  // namespace

extern "C" {

int tsqr_batch_create(int32_t count, const int64_t* m, const int64_t* n, void* const* A, const int64_t* lda,
                      void* const* R, const int64_t* ldr, int32_t precision, const tsqr_batch_opts_t* opts,
                      tsqr_batch_t* out, tsqr_stream_t stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (!out) return -10;
  *out = nullptr;
  if (count < 1) return -1;
  if (!m) return -2;
  if (!n) return -3;
  if (!A) return -4;
  if (!lda) return -5;
  if (!R) return -6;
  if (!ldr) return -7;
  if (precision != TSQR_PREC_FP64 && precision != TSQR_PREC_FP32) return -8;
  for (int i = 0; i < count; ++i) {
    if (n[i] < 1 || n[i] > kBatchNmax || m[i] < n[i]) return -2;
    if (!A[i] || lda[i] < m[i]) return -4;
    if (!R[i] || ldr[i] < n[i]) return -6;
  }
  int kb = opts && opts->tile_kb > 0 ? opts->tile_kb : default_tile_kb(precision == TSQR_PREC_FP64 ? 8 : 4);
  int q = opts && opts->arity > 0 ? opts->arity : 2;
  if (q < 2 || q > 16) return -9;
  if (opts && opts->autotune) {
    const int rc = autotune(count, m, n, precision, &kb, &q, s);
    if (rc != TSQR_OK) return rc;
  }
  tsqr_batch_s* b = nullptr;
  const int rc = create_batch(count, m, n, A, lda, R, ldr, precision, kb, q, &b, s);
  if (rc != TSQR_OK) return rc;
  *out = b;
  return TSQR_OK;
}

int tsqr_batch_factor(tsqr_batch_t b, tsqr_stream_t stream) {
  if (!b || b->magic != kBatchMagic) return TSQR_ERR_HANDLE;
  const cudaError_t e = launch_any(b, (cudaStream_t)stream);
  return e == cudaSuccess ? TSQR_OK : TSQR_ERR_CUDA;
}

int tsqr_batch_factor_graph(tsqr_batch_t b, tsqr_stream_t stream) {
  if (!b || b->magic != kBatchMagic) return TSQR_ERR_HANDLE;
  cudaStream_t s = (cudaStream_t)stream;
  if (!b->graph) {
    // Capture on a private stream so the caller's stream can be the legacy one.
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return TSQR_ERR_CUDA;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const cudaError_t le = launch_any(b, cs);
      e = cudaStreamEndCapture(cs, &g);
      if (e == cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
      b->graph = nullptr;
      return TSQR_ERR_CUDA;
    }
  }
  return cudaGraphLaunch(b->graph, s) == cudaSuccess ? TSQR_OK : TSQR_ERR_CUDA;
}

int tsqr_batch_info(tsqr_batch_t b, int32_t* tile_kb, int32_t* arity, int64_t* items, int64_t* workspace_bytes) {
  if (!b || b->magic != kBatchMagic) return TSQR_ERR_HANDLE;
  if (tile_kb) *tile_kb = b->tile_kb;
  if (arity) *arity = b->arity;
  if (items) *items = b->nitems;
  if (workspace_bytes) *workspace_bytes = (int64_t)b->ws_bytes;
  return TSQR_OK;
}

int tsqr_batch_sync_status(tsqr_batch_t b, tsqr_stream_t stream) {
  if (!b || b->magic != kBatchMagic) return TSQR_ERR_HANDLE;
  cudaStream_t s = (cudaStream_t)stream;
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, b->status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->status, 0, sizeof(int), s);
  if (e != cudaSuccess) return TSQR_ERR_CUDA;
  if (h & kStatusTimeout) return TSQR_ERR_TIMEOUT;
  if (h & kStatusNonfinite) return TSQR_ERR_NONFINITE;
  return TSQR_OK;
}

int tsqr_batch_destroy(tsqr_batch_t b) {
  if (!b || b->magic != kBatchMagic) return TSQR_ERR_HANDLE;
  b->magic = 0;
  cudaDeviceSynchronize();
  free_batch(b);
  delete b;
  return TSQR_OK;
}

}  // extern "C"
