// C ABI of the TSQR / CAQR library: argument checks, the tree plan, device
// workspace, and the launch sequences of Section 2.1 (TSQR) and Section 3
// (CAQR).  All arithmetic runs in the kernels of leaf_factor.cu,
// node_factor.cu and apply.cu.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "../../include/tsqr.h"
#include "tsqr_internal.cuh"

namespace tsqr {
size_t node_factor_smem(int n, int q, size_t elem);
size_t leaf_rec_smem(int n, int ld, size_t elem);
template <typename T>
cudaError_t launch_leaf_factor_rec(const LeafFactorArgs<T>& a, cudaStream_t s);
size_t leaf_apply_smem(int n, size_t elem);
size_t node_apply_smem(int n, int q, size_t elem);
}  // namespace tsqr

using namespace tsqr;

namespace {

constexpr uint32_t kTsqrMagic = 0x54535152u;  // "TSQR"
constexpr uint32_t kCaqrMagic = 0x43415152u;  // "CAQR"
constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

int max_smem_optin() {
  static int cached = -1;
  if (cached < 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      v = 227 * 1024;
    cached = v;
  }
  return cached;
}

}  // namespace

struct tsqr_q_s {
  uint32_t magic = kTsqrMagic;
  int32_t prec = TSQR_PREC_FP64;
  size_t es = 8;
  int64_t m = 0, n = 0;
  int64_t h = 0, nleaves = 0, hmax = 0;
  int32_t q = 2, levels = 0;
  std::vector<int64_t> items;  // items per level; items[0] = leaves (chains for the hybrid tree)
  // Hybrid / flat tree: chains of L consecutive leaves, each a flat tree in
  // one CTA; the q-ary tree runs over the nchains chain R factors.
  bool hybrid = false;
  bool rec = false;  // recursive (RGEQR3) leaf QR
  int64_t L = 1, nchains = 0;
  int ld_s = 0;  // shared-memory leading dimension of the leaf (or stacked) tile
  // Device workspace (owned unless external).
  unsigned char* ws = nullptr;
  size_t ws_bytes = 0;
  bool owns_ws = true;
  void* leafR = nullptr;
  void* leafTau = nullptr;
  void* leafT = nullptr;
  std::vector<void*> nodeR, nodeY, nodeTau, nodeT;  // index l-1 for level l
  void* d = nullptr;
  int* status = nullptr;
  // The factored matrix (borrowed).
  void* A = nullptr;
  int64_t lda = 0;
  bool factored = false;
  // Stage timing (tracing).
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events[TSQR_NUM_STAGES];
  int64_t launches[TSQR_NUM_STAGES] = {0, 0, 0, 0};
  // Arithmetic of the leaf-block Q^T products (CAQR trailing updates).
  int32_t upd = TSQR_PREC_FP64;
  // Host pipeline (tsqr_factor_form_host): copy stream and per-chunk events,
  // created on first use.
  cudaStream_t copy = nullptr;
  std::vector<cudaEvent_t> ev_in, ev_out;
  cudaEvent_t ev_start = nullptr, ev_done = nullptr;
  // CAQR panels: one event per tree level, recorded as the level's factors
  // are written, and one after the sign fix, so that another stream's Q^T
  // product can take each level as soon as it is factored (empty: none).
  std::vector<cudaEvent_t> ev_level;
};

struct caqr_q_s {
  uint32_t magic = kCaqrMagic;
  int32_t prec = TSQR_PREC_FP64;
  size_t es = 8;
  int64_t m = 0, n = 0, b = 0;
  void* A = nullptr;
  int64_t lda = 0;
  unsigned char* ws = nullptr;
  std::vector<tsqr_q_t> panels;
  int* status = nullptr;  // panel 0's status word
  // Look-ahead: the next panel is factored on `side` while the rest of the
  // trailing matrix is updated on the caller's stream.
  cudaStream_t side = nullptr;
  std::vector<cudaEvent_t> ev_left, ev_fact;
  std::vector<cudaEvent_t> ev_leaf;  // a panel's leaf factors are in (its tree may still run)
  // The FP64 trailing update of a wide panel is issued as two column halves
  // on the caller's stream and on `upd2`, so that one half's latency-bound
  // tree levels overlap the other half's leaf blocks.
  cudaStream_t upd2 = nullptr;
  std::vector<cudaEvent_t> ev_fork, ev_join;
  int32_t upd = TSQR_PREC_FP64;  // trailing-update arithmetic
  // caqr_refactor's panel loop as a CUDA graph, captured for one (A, lda)
  // on a private stream and replayed on the caller's stream.
  cudaStream_t cap = nullptr;
  cudaGraphExec_t graph = nullptr;
  void* graph_A = nullptr;
  int64_t graph_lda = 0;
  bool timing = false;
};

namespace {

bool valid(const tsqr_q_s* q) { return q && q->magic == kTsqrMagic; }

// Records a CUDA event pair around one stage of a call when timing is on.
struct StageTimer {
  tsqr_q_s* q;
  int stage;
  cudaStream_t s;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  StageTimer(const tsqr_q_s* qq, int st, cudaStream_t ss) : q(const_cast<tsqr_q_s*>(qq)), stage(st), s(ss) {
    if (q->timing && cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess)
      cudaEventRecord(e0, s);
  }
  void stop(int64_t nlaunch) {
    q->launches[stage] += nlaunch;
    if (e1) {
      cudaEventRecord(e1, s);
      q->events[stage].emplace_back(e0, e1);
      e0 = e1 = nullptr;
    }
  }
  ~StageTimer() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

void clear_events(tsqr_q_s* q) {
  for (auto& v : q->events) {
    for (auto& p : v) {
      cudaEventDestroy(p.first);
      cudaEventDestroy(p.second);
    }
    v.clear();
  }
  for (auto& l : q->launches) l = 0;
}
bool valid(const caqr_q_s* q) { return q && q->magic == kCaqrMagic; }

int cuda_err(cudaError_t e) { return e == cudaSuccess ? TSQR_OK : (e == cudaErrorMemoryAllocation ? TSQR_ERR_NOMEM : TSQR_ERR_CUDA); }

// Leaf partition (Section 2.1, 1-D block rows; the remainder rule is the
// build's reading of the paper's "m_i >= n"): leaves of h rows, the last one
// takes what is left and is merged into its predecessor when it would have
// fewer than n rows.
int make_plan(tsqr_q_s* q, int64_t m, int64_t n, int32_t prec, const tsqr_opts_t* opts) {
  const int32_t flags = opts ? opts->flags : 0;
  if (flags & ~(TSQR_FLAG_APPLY_BF16X3 | TSQR_FLAG_HYBRID_TREE | TSQR_FLAG_FLAT_TREE | TSQR_FLAG_RECURSIVE_LEAF |
                TSQR_FLAG_APPLY_TF32X3))
    return -4;
  if ((flags & TSQR_FLAG_APPLY_BF16X3) && (flags & TSQR_FLAG_APPLY_TF32X3)) return -4;
  q->prec = prec;
  q->hybrid = (flags & (TSQR_FLAG_HYBRID_TREE | TSQR_FLAG_FLAT_TREE)) != 0;
  q->rec = (flags & TSQR_FLAG_RECURSIVE_LEAF) != 0;
  if (q->rec && (q->hybrid || n > 64)) return TSQR_ERR_UNSUPPORTED;
  // Shared memory of the leaf kernel this plan launches for a tile of `rows` rows.
  auto leaf_smem = [&](int64_t rows) -> int64_t {
    return q->rec ? (int64_t)leaf_rec_smem((int)n, leaf_factor_ld((int)rows), q->es)
                  : (int64_t)leaf_factor_smem((int)n, leaf_factor_ld((int)rows), q->es);
  };
  // Rows of the stacked tile [R; A_i] beyond the leaf's own rows.
  const int64_t top = q->hybrid ? n : 0;
  q->es = prec == TSQR_PREC_FP64 ? 8 : 4;
  q->m = m;
  q->n = n;
  const int64_t smax = max_smem_optin();
  int64_t h = opts && opts->leaf_rows > 0 ? opts->leaf_rows : 0;
  if (h == 0) {
    // Tallest leaf (a multiple of 32 rows, at most 1024) whose n-column tile
    // and working buffers fit in one SM's shared memory (the loop below
    // shrinks it until they do): taller leaves mean fewer tree nodes (the
    // tree's work is about n / (2h) of the leaves') and a smaller n^3 share
    // in forming Q, at one leaf CTA per SM.
    // FP32 leaves stop at 512 rows: beyond that the shorter tree no longer
    // pays for the longer serial leaf (measured at n = 64 and 128); at
    // n <= 64 they stop at 384, whose tile (under 100 KB) lets two CTAs share
    // an SM and overlap their serial column steps (measured at n = 64: 21.2
    // against 22.1 ms for 512 rows).
    h = smax / (int64_t)q->es / n / 32 * 32;
    const int64_t hcap = q->es == 8 ? 1024 : (n <= 64 ? 384 : 512);
    if (h > hcap) h = hcap;
    while (q->rec && h - 32 >= n && leaf_smem(h) > smax) h -= 32;
    h -= top;  // hybrid: the stacked tile [R; A_i] must fit
    if (h < n) h = n;
  }
  if (h < n) return -4;
  const bool auto_h = !(opts && opts->leaf_rows > 0);
  int64_t nl = 0;
  for (;;) {
    nl = (m + h - 1) / h;
    if (nl < 1) nl = 1;
    const int64_t rem = m - (nl - 1) * h;
    if (nl > 1 && rem < n) --nl;
    q->hmax = nl > 1 ? (m - (nl - 1) * h > h ? m - (nl - 1) * h : h) : m;
    // An automatic height shrinks until a merged last leaf still fits.
    if (!auto_h || h - 32 < n || leaf_smem(q->hmax + top) <= smax) break;
    h -= 32;
  }
  q->ld_s = leaf_factor_ld((int)(q->hmax + top));
  q->h = h;
  q->nleaves = nl;
  // Default arity 4 where the four-triangle node fits in shared memory: per
  // eliminated triangle it needs a third less work for T and for applying
  // the node's Q than a binary node, and half the levels.
  if (opts && opts->arity > 0) {
    q->q = opts->arity;
  } else {
    q->q = (int64_t)node_factor_smem((int)n, 4, q->es) <= smax && (int64_t)node_apply_smem((int)n, 4, q->es) <= smax ? 4 : 2;
  }
  if (q->q < 2 || q->q > 16) return -4;
  if (q->hybrid) {
    // One chain per resident CTA of the chain kernel (flat tree: one chain).
    int64_t slots = (flags & TSQR_FLAG_FLAT_TREE) ? 1 : chain_factor_resident((int)n, q->ld_s, q->es);
    if (slots < 1) slots = 1;
    q->L = (nl + slots - 1) / slots;
    q->nchains = (nl + q->L - 1) / q->L;
    q->items.assign(1, q->nchains);
  } else {
    q->L = 1;
    q->nchains = nl;
    q->items.assign(1, nl);
  }
  while (q->items.back() > 1) q->items.push_back((q->items.back() + q->q - 1) / q->q);
  q->levels = (int32_t)q->items.size() - 1;
  if (n > kMaxN) return TSQR_ERR_UNSUPPORTED;
  if (flags & (TSQR_FLAG_APPLY_BF16X3 | TSQR_FLAG_APPLY_TF32X3)) {
    // Leaf stage of Q^T C on the tensor cores: FP32 storage, at most 64
    // reflectors, ordinary leaves.
    if (prec != TSQR_PREC_FP32 || n > kBf16x3MaxN || q->hybrid) return TSQR_ERR_UNSUPPORTED;
    q->upd = (flags & TSQR_FLAG_APPLY_TF32X3) ? TSQR_UPDATE_TF32X3 : TSQR_UPDATE_BF16X3;
  }
  if (leaf_smem(q->hmax + top) > smax) return TSQR_ERR_UNSUPPORTED;
  if ((int64_t)leaf_apply_smem((int)n, q->es) > smax) return TSQR_ERR_UNSUPPORTED;
  if (q->hybrid && (int64_t)chain_apply_smem((int)n, q->es) > smax) return TSQR_ERR_UNSUPPORTED;
  if (q->levels > 0) {
    if ((int64_t)node_factor_smem((int)n, q->q, q->es) > smax) return TSQR_ERR_UNSUPPORTED;
    if ((int64_t)node_apply_smem((int)n, q->q, q->es) > smax) return TSQR_ERR_UNSUPPORTED;
  }
  return TSQR_OK;
}

size_t workspace_bytes(const tsqr_q_s* q) {
  const size_t nn = (size_t)q->n * q->n * q->es, nv = (size_t)q->n * q->es;
  size_t b = 0;
  b += align_up(q->items[0] * nn) + align_up(q->nleaves * nn) + align_up(q->nleaves * nv);
  for (int l = 1; l <= q->levels; ++l) {
    const size_t it = (size_t)q->items[l];
    b += align_up(it * nn) * 2 + align_up(it * (q->q - 1) * nn) + align_up(it * nv);
  }
  b += align_up(nv) + align_up(sizeof(int));
  return b;
}

void bind_workspace(tsqr_q_s* q, unsigned char* base) {
  const size_t nn = (size_t)q->n * q->n * q->es, nv = (size_t)q->n * q->es;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    void* p = base + off;
    off += align_up(bytes);
    return p;
  };
  q->ws = base;
  q->leafR = take(q->items[0] * nn);  // one R per leaf, or per chain
  q->leafT = take(q->nleaves * nn);
  q->leafTau = take(q->nleaves * nv);
  q->nodeR.assign(q->levels, nullptr);
  q->nodeY.assign(q->levels, nullptr);
  q->nodeTau.assign(q->levels, nullptr);
  q->nodeT.assign(q->levels, nullptr);
  for (int l = 1; l <= q->levels; ++l) {
    const size_t it = (size_t)q->items[l];
    q->nodeR[l - 1] = take(it * nn);
    q->nodeT[l - 1] = take(it * nn);
    q->nodeY[l - 1] = take(it * (q->q - 1) * nn);
    q->nodeTau[l - 1] = take(it * nv);
  }
  q->d = take(nv);
  q->status = (int*)take(sizeof(int));
  q->ws_bytes = off;
}

void* root_r(const tsqr_q_s* q) { return q->levels == 0 ? q->leafR : q->nodeR[q->levels - 1]; }

int64_t slot_stride(const tsqr_q_s* q, int level) {
  int64_t s = q->h * q->L;
  for (int l = 1; l < level; ++l) s *= q->q;
  return s;
}

// Rows [leaf_row0(l0), leaf_row0(l1)) hold leaves l0 .. l1-1; the last leaf
// runs to m.
int64_t leaf_row0(const tsqr_q_s* q, int64_t l) { return l >= q->nleaves ? q->m : l * q->h; }

// Leaf QR of leaves [l0, l1) (the same kernel on a sub-range).
template <typename T>
cudaError_t launch_leaf_range(tsqr_q_s* q, T* A, int64_t lda, int64_t l0, int64_t l1, cudaStream_t s,
                              const T* Asrc = nullptr, int64_t ldsrc = 0) {
  const int64_t nn = q->n * q->n, r0 = leaf_row0(q, l0);
  LeafFactorArgs<T> la{};
  la.A = A + r0;
  la.lda = lda;
  la.Asrc = Asrc ? Asrc + r0 : nullptr;  // the recursive leaf reads A only (callers do not pass a source)
  la.ldsrc = ldsrc;
  la.m = leaf_row0(q, l1) - r0;
  la.n = (int)q->n;
  la.h = q->h;
  la.nleaves = l1 - l0;
  la.ld_s = q->ld_s;
  la.R = (T*)q->leafR + l0 * nn;
  la.tau = (T*)q->leafTau + l0 * q->n;
  la.Tw = (T*)q->leafT + l0 * nn;
  la.status = q->status;
  return q->rec ? launch_leaf_factor_rec(la, s) : launch_leaf_factor(la, s);
}

template <typename T>
cudaError_t run_tree_factor(tsqr_q_s* q, T* R, int64_t ldr, bool zero_lower, cudaStream_t s);

template <typename T>
ChainApplyArgs<T> chain_apply_args(const tsqr_q_s* q, int mode, int64_t k, T* C, int64_t ldc) {
  ChainApplyArgs<T> ca{};
  ca.Y = (const T*)q->A;
  ca.ldy = q->lda;
  ca.m = q->m;
  ca.n = (int)q->n;
  ca.h = q->h;
  ca.nleaves = q->nleaves;
  ca.L = q->L;
  ca.nchains = q->nchains;
  ca.Tw = (const T*)q->leafT;
  ca.C = C;
  ca.ldc = ldc;
  ca.k = k;
  ca.mode = mode;
  return ca;
}

template <typename T>
cudaError_t run_factor(tsqr_q_s* q, T* A, int64_t lda, T* R, int64_t ldr, bool zero_lower, cudaStream_t s,
                       cudaEvent_t ev_leaves = nullptr) {
  StageTimer t0(q, TSQR_STAGE_LEAF_FACTOR, s);
  cudaError_t e;
  if (q->hybrid) {
    ChainFactorArgs<T> ca{};
    ca.A = A;
    ca.lda = lda;
    ca.m = q->m;
    ca.n = (int)q->n;
    ca.h = q->h;
    ca.nleaves = q->nleaves;
    ca.L = q->L;
    ca.nchains = q->nchains;
    ca.ld_s = q->ld_s;
    ca.R = (T*)q->leafR;
    ca.tau = (T*)q->leafTau;
    ca.Tw = (T*)q->leafT;
    ca.status = q->status;
    e = launch_chain_factor(ca, s);
  } else {
    e = launch_leaf_range(q, A, lda, 0, q->nleaves, s);
  }
  if (e != cudaSuccess) return e;
  t0.stop(1);
  // The leaf factors (Y, T per leaf) are complete here: a caller may start
  // leaf-level products on another stream while the tree is factored.
  if (ev_leaves && (e = cudaEventRecord(ev_leaves, s)) != cudaSuccess) return e;
  return run_tree_factor(q, R, ldr, zero_lower, s);
}

template <typename T>
cudaError_t run_tree_factor(tsqr_q_s* q, T* R, int64_t ldr, bool zero_lower, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  StageTimer t1(q, TSQR_STAGE_TREE_FACTOR, s);
  for (int l = 1; l <= q->levels; ++l) {
    NodeFactorArgs<T> na{};
    na.Rin = (const T*)(l == 1 ? q->leafR : q->nodeR[l - 2]);
    na.nin = q->items[l - 1];
    na.arity = q->q;
    na.n = (int)q->n;
    na.nodes = q->items[l];
    na.Rout = (T*)q->nodeR[l - 1];
    na.Y = (T*)q->nodeY[l - 1];
    na.tau = (T*)q->nodeTau[l - 1];
    na.Tw = (T*)q->nodeT[l - 1];
    na.status = q->status;
    e = launch_node_factor(na, s);
    if (e != cudaSuccess) return e;
    if (!q->ev_level.empty() && (e = cudaEventRecord(q->ev_level[l - 1], s)) != cudaSuccess) return e;
  }
  e = launch_sign_fix((const T*)root_r(q), (int)q->n, (T*)q->d, R, ldr, zero_lower, s);
  if (e == cudaSuccess && !q->ev_level.empty()) e = cudaEventRecord(q->ev_level[q->levels], s);
  if (e == cudaSuccess) t1.stop(q->levels + 1);
  return e;
}

// Leaf stage of Q C / Q^T C / form on leaves [l0, l1) (rows of C alike).
template <typename T>
LeafApplyArgs<T> leaf_apply_args(const tsqr_q_s* q, int64_t k, T* C, int64_t ldc, int64_t l0, int64_t l1) {
  const int64_t r0 = leaf_row0(q, l0);
  LeafApplyArgs<T> la{};
  la.Y = (const T*)q->A + r0;
  la.ldy = q->lda;
  la.m = leaf_row0(q, l1) - r0;
  la.n = (int)q->n;
  la.h = q->h;
  la.nleaves = l1 - l0;
  la.Tw = (const T*)q->leafT + l0 * q->n * q->n;
  la.C = C + r0;
  la.ldc = ldc;
  la.k = k;
  return la;
}

// Tree stage of forming the thin Q: the root slot starts as diag(d), every
// other row is produced top-down without being read.
template <typename T>
cudaError_t run_tree_form(const tsqr_q_s* q, T* C, int64_t ldc, cudaStream_t s, int64_t k = -1, const T* X = nullptr,
                          int64_t ldx = 0);

template <typename T>
cudaError_t run_apply(const tsqr_q_s* q, int mode, int64_t k, T* C, int64_t ldc, cudaStream_t s, const T* X = nullptr,
                      int64_t ldx = 0, bool wait_tree = false) {
  cudaError_t e = cudaSuccess;
  LeafApplyArgs<T> la = leaf_apply_args(q, k, C, ldc, 0, q->nleaves);
  auto node = [&](int l, int md) {
    NodeApplyArgs<T> na{};
    na.Y = (const T*)q->nodeY[l - 1];
    na.Tw = (const T*)q->nodeT[l - 1];
    na.nin = q->items[l - 1];
    na.arity = q->q;
    na.n = (int)q->n;
    na.nodes = q->items[l];
    na.slot_stride = slot_stride(q, l);
    na.C = C;
    na.ldc = ldc;
    na.k = k;
    na.mode = md;
    return launch_node_apply(na, s);
  };
  auto leaf = [&](int md) {
    StageTimer t(q, TSQR_STAGE_LEAF_APPLY, s);
    la.mode = md;
    cudaError_t r;
    if (q->hybrid) {
      r = launch_chain_apply(chain_apply_args(q, md, k, C, ldc), s);
      if (r == cudaSuccess) t.stop(1);
      return r;
    }
    if constexpr (sizeof(T) == 4) {
      if (md == kApplyQT && (q->upd == TSQR_UPDATE_BF16X3 || q->upd == TSQR_UPDATE_TF32X3))
        r = launch_leaf_update_split3(la, q->upd == TSQR_UPDATE_TF32X3, q->status, s);
      else
        r = launch_leaf_apply(la, s);
    } else {
      r = launch_leaf_apply(la, s);
    }
    if (r == cudaSuccess) t.stop(1);
    return r;
  };
  if (mode == kApplyQT) {
    if ((e = leaf(kApplyQT)) != cudaSuccess) return e;
    // Each tree level needs its node factors: a caller that started this
    // product while the tree was still being factored on another stream
    // (wait_tree) waits for each level's event, then for the sign fix's.
    const bool per_level = wait_tree && (int)q->ev_level.size() == q->levels + 1;
    StageTimer t(q, TSQR_STAGE_TREE_APPLY, s);
    for (int l = 1; l <= q->levels; ++l) {
      if (per_level && (e = cudaStreamWaitEvent(s, q->ev_level[l - 1], 0)) != cudaSuccess) return e;
      if ((e = node(l, kApplyQT)) != cudaSuccess) return e;
    }
    if (per_level && (e = cudaStreamWaitEvent(s, q->ev_level[q->levels], 0)) != cudaSuccess) return e;
    e = launch_scale_rows(C, ldc, (int)q->n, k, (const T*)q->d, s);
    if (e == cudaSuccess) t.stop(q->levels + 1);
    return e;
  }
  if (mode == kApplyQ) {
    {
      StageTimer t(q, TSQR_STAGE_TREE_APPLY, s);
      if ((e = launch_scale_rows(C, ldc, (int)q->n, k, (const T*)q->d, s)) != cudaSuccess) return e;
      for (int l = q->levels; l >= 1; --l)
        if ((e = node(l, kApplyQ)) != cudaSuccess) return e;
      t.stop(q->levels + 1);
    }
    return leaf(kApplyQ);
  }
  if ((e = run_tree_form(q, C, ldc, s, k, X, ldx)) != cudaSuccess) return e;
  return leaf(kApplyForm);
}

// Forms Q [X; 0] (X n x k) when X is given, the thin Q (X = I, k = n) otherwise.
template <typename T>
cudaError_t run_tree_form(const tsqr_q_s* q, T* C, int64_t ldc, cudaStream_t s, int64_t k, const T* X, int64_t ldx) {
  cudaError_t e = cudaSuccess;
  if (k < 0) k = q->n;
  StageTimer t(q, TSQR_STAGE_TREE_APPLY, s);
  e = X ? launch_init_form_mul(C, ldc, (int)q->n, k, (const T*)q->d, X, ldx, s)
        : launch_init_form(C, ldc, (int)q->n, (const T*)q->d, s);
  if (e != cudaSuccess) return e;
  for (int l = q->levels; l >= 1; --l) {
    NodeApplyArgs<T> na{};
    na.Y = (const T*)q->nodeY[l - 1];
    na.Tw = (const T*)q->nodeT[l - 1];
    na.nin = q->items[l - 1];
    na.arity = q->q;
    na.n = (int)q->n;
    na.nodes = q->items[l];
    na.slot_stride = slot_stride(q, l);
    na.C = C;
    na.ldc = ldc;
    na.k = k;
    na.mode = kApplyForm;
    if ((e = launch_node_apply(na, s)) != cudaSuccess) return e;
  }
  t.stop(q->levels + 1);
  return e;
}

// Copies a rows x cols column-major block (the n x n R into a mapped host
// buffer, so that the call queues no copy-engine transfer).
template <typename T>
__global__ void copy_block_kernel(const T* __restrict__ src, int64_t lds, T* __restrict__ dst, int64_t ldd,
                                  int64_t rows, int64_t cols) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / rows, i = e - c * rows;
    dst[c * ldd + i] = src[c * lds + i];
  }
}

// Address at which kernels can reach a page-locked host buffer (allocated
// with cudaHostAlloc or registered); null for pageable memory.
template <typename T>
T* mapped_host(const T* p) {
  cudaPointerAttributes at{};
  if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost && at.devicePointer ? (T*)at.devicePointer : nullptr;
}

// Host-buffer pipeline.  A page-locked A_host is read by the leaf kernel
// itself, over the host link, as it loads each leaf (Y and R_i go to the
// device A); a pageable one arrives in chunks of leaves on the copy stream
// while the compute stream factors the chunks already in.  The tree and the
// tree part of forming Q follow.  With a device Q, Q leaves the device chunk
// by chunk as the form finishes each one; with none, the form kernels store
// Q straight into the page-locked Q_host.  Chunks are whole waves of leaf
// CTAs.  Copy-engine transfers of page-locked memory were measured to stall
// for tens of milliseconds now and then where the SMs' own loads and stores
// to the same buffers did not.
template <typename T>
cudaError_t run_factor_form_host(tsqr_q_s* q, const T* Ah, int64_t ldah, T* Qh, int64_t ldqh, T* Rh, int64_t ldrh,
                                 T* A, int64_t lda, T* Q, int64_t ldq, T* R, int64_t ldr, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  const T* dAh = q->rec ? nullptr : mapped_host(Ah);
  T* dQh = Q ? nullptr : mapped_host(Qh);
  if (!Q && !dQh) return cudaErrorInvalidValue;
  T* dRh = mapped_host(Rh);
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  int64_t chunk = 4 * (int64_t)sms;  // four waves of one-CTA-per-SM leaves
  if (chunk > q->nleaves) chunk = q->nleaves;
  const int64_t nchunks = (q->nleaves + chunk - 1) / chunk;
  const size_t es = sizeof(T);
  const bool copies = !dAh || Q;  // anything on the copy stream
  if (copies) {
    if (!q->copy && (e = cudaStreamCreateWithFlags(&q->copy, cudaStreamNonBlocking)) != cudaSuccess) return e;
    if (!q->ev_start && (e = cudaEventCreateWithFlags(&q->ev_start, cudaEventDisableTiming)) != cudaSuccess) return e;
    if (!q->ev_done && (e = cudaEventCreateWithFlags(&q->ev_done, cudaEventDisableTiming)) != cudaSuccess) return e;
    while ((int64_t)q->ev_in.size() < nchunks) {
      cudaEvent_t a = nullptr, b = nullptr;
      if ((e = cudaEventCreateWithFlags(&a, cudaEventDisableTiming)) != cudaSuccess) return e;
      if ((e = cudaEventCreateWithFlags(&b, cudaEventDisableTiming)) != cudaSuccess) {
        cudaEventDestroy(a);
        return e;
      }
      q->ev_in.push_back(a);
      q->ev_out.push_back(b);
    }
    // The copy stream starts after everything already queued on s.
    if ((e = cudaEventRecord(q->ev_start, s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(q->copy, q->ev_start, 0)) != cudaSuccess) return e;
  }
  if (dAh) {
    StageTimer t0(q, TSQR_STAGE_LEAF_FACTOR, s);
    if ((e = launch_leaf_range(q, A, lda, 0, q->nleaves, s, dAh, ldah)) != cudaSuccess) return e;
    t0.stop(1);
  } else {
    for (int64_t c = 0; c < nchunks; ++c) {
      const int64_t l0 = c * chunk, l1 = l0 + chunk < q->nleaves ? l0 + chunk : q->nleaves;
      const int64_t r0 = leaf_row0(q, l0), r1 = leaf_row0(q, l1);
      if ((e = cudaMemcpy2DAsync(A + r0, lda * es, Ah + r0, ldah * es, (r1 - r0) * es, q->n, cudaMemcpyHostToDevice,
                                 q->copy)) != cudaSuccess)
        return e;
      if ((e = cudaEventRecord(q->ev_in[c], q->copy)) != cudaSuccess) return e;
    }
    StageTimer t0(q, TSQR_STAGE_LEAF_FACTOR, s);
    for (int64_t c = 0; c < nchunks; ++c) {
      const int64_t l0 = c * chunk, l1 = l0 + chunk < q->nleaves ? l0 + chunk : q->nleaves;
      if ((e = cudaStreamWaitEvent(s, q->ev_in[c], 0)) != cudaSuccess) return e;
      if ((e = launch_leaf_range(q, A, lda, l0, l1, s)) != cudaSuccess) return e;
    }
    t0.stop(nchunks);
  }
  if ((e = run_tree_factor(q, R, ldr, true, s)) != cudaSuccess) return e;
  q->A = A;
  q->lda = lda;
  q->factored = true;
  if (dRh) {
    const int64_t nn = q->n * q->n;
    copy_block_kernel<T><<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(R, ldr, dRh, ldrh, q->n, q->n);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  } else if ((e = cudaMemcpy2DAsync(Rh, ldrh * es, R, ldr * es, q->n * es, q->n, cudaMemcpyDeviceToHost, s)) !=
             cudaSuccess) {
    return e;
  }
  if (!Q) {
    // Q straight into Q_host: the same form as tsqr_form_q.
    if ((e = run_apply<T>(q, kApplyForm, q->n, dQh, ldqh, s)) != cudaSuccess) return e;
    if (!copies) return cudaSuccess;
  } else {
    if ((e = run_tree_form(q, Q, ldq, s)) != cudaSuccess) return e;
    StageTimer t(q, TSQR_STAGE_LEAF_APPLY, s);
    for (int64_t c = 0; c < nchunks; ++c) {
      const int64_t l0 = c * chunk, l1 = l0 + chunk < q->nleaves ? l0 + chunk : q->nleaves;
      LeafApplyArgs<T> la = leaf_apply_args(q, q->n, Q, ldq, l0, l1);
      la.mode = kApplyForm;
      if ((e = launch_leaf_apply(la, s)) != cudaSuccess) return e;
      if ((e = cudaEventRecord(q->ev_out[c], s)) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(q->copy, q->ev_out[c], 0)) != cudaSuccess) return e;
      const int64_t r0 = leaf_row0(q, l0), r1 = leaf_row0(q, l1);
      if ((e = cudaMemcpy2DAsync(Qh + r0, ldqh * es, Q + r0, ldq * es, (r1 - r0) * es, q->n, cudaMemcpyDeviceToHost,
                                 q->copy)) != cudaSuccess)
        return e;
    }
    t.stop(nchunks);
  }
  // The call is complete on s once the last copy is.
  if ((e = cudaEventRecord(q->ev_done, q->copy)) != cudaSuccess) return e;
  return cudaStreamWaitEvent(s, q->ev_done, 0);
}

int create_handle(int64_t m, int64_t n, int32_t prec, const tsqr_opts_t* opts, tsqr_q_t* out, unsigned char* external,
                  cudaStream_t s) {
  tsqr_q_s* q = new (std::nothrow) tsqr_q_s();
  if (!q) return TSQR_ERR_NOMEM;
  int rc = make_plan(q, m, n, prec, opts);
  if (rc != TSQR_OK) {
    delete q;
    return rc;
  }
  if (external) {
    q->owns_ws = false;
    bind_workspace(q, external);
  } else {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, workspace_bytes(q));
    if (e != cudaSuccess) {
      delete q;
      return cuda_err(e);
    }
    bind_workspace(q, (unsigned char*)p);
  }
  cudaError_t e = cudaMemsetAsync(q->status, 0, sizeof(int), s);
  if (e != cudaSuccess) {
    if (q->owns_ws) cudaFree(q->ws);
    delete q;
    return cuda_err(e);
  }
  *out = q;
  return TSQR_OK;
}

int refactor(tsqr_q_s* q, void* A, int64_t lda, void* R, int64_t ldr, bool zero_lower, cudaStream_t s,
             cudaEvent_t ev_leaves = nullptr) {
  cudaError_t e;
  if (q->prec == TSQR_PREC_FP64)
    e = run_factor<double>(q, (double*)A, lda, (double*)R, ldr, zero_lower, s, ev_leaves);
  else
    e = run_factor<float>(q, (float*)A, lda, (float*)R, ldr, zero_lower, s, ev_leaves);
  if (e != cudaSuccess) return cuda_err(e);
  q->A = A;
  q->lda = lda;
  q->factored = true;
  return TSQR_OK;
}

int destroy_handle(tsqr_q_s* q) {
  if (!valid(q)) return TSQR_ERR_HANDLE;
  q->magic = 0;
  cudaError_t e = cudaSuccess;
  if (q->owns_ws && q->ws) e = cudaFree(q->ws);
  clear_events(q);
  for (size_t i = 0; i < q->ev_in.size(); ++i) {
    cudaEventDestroy(q->ev_in[i]);
    cudaEventDestroy(q->ev_out[i]);
  }
  for (auto e : q->ev_level)
    if (e) cudaEventDestroy(e);
  if (q->ev_start) cudaEventDestroy(q->ev_start);
  if (q->ev_done) cudaEventDestroy(q->ev_done);
  if (q->copy) cudaStreamDestroy(q->copy);
  delete q;
  return cuda_err(e);
}

int read_status(int* status, cudaStream_t s) {
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), s);
  if (e != cudaSuccess) return cuda_err(e);
  if (h & kStatusTimeout) return TSQR_ERR_TIMEOUT;
  if (h & kStatusNonfinite) return TSQR_ERR_NONFINITE;
  return TSQR_OK;
}

template <typename T>
int factor_common(int64_t m, int64_t n, T* A, int64_t lda, T* R, int64_t ldr, const tsqr_opts_t* opts, tsqr_q_t* q,
                  cudaStream_t s, int32_t prec) {
  if (q) *q = nullptr;
  if (m < 0) return -1;
  if (n < 0 || n > m) return -2;
  if (m > 0 && n > 0 && !A) return -3;
  if (lda < (m > 1 ? m : 1)) return -4;
  if (m > 0 && n > 0 && !R) return -5;
  if (ldr < (n > 1 ? n : 1)) return -6;
  if (m == 0 || n == 0) return TSQR_OK;
  tsqr_q_t h = nullptr;
  int rc = create_handle(m, n, prec, opts, &h, nullptr, s);
  if (rc != TSQR_OK) return rc == -4 ? -7 : rc;
  rc = refactor(h, A, lda, R, ldr, true, s);
  if (rc != TSQR_OK || !q) {
    if (!q) cudaStreamSynchronize(s);
    destroy_handle(h);
    return rc;
  }
  *q = h;
  return TSQR_OK;
}

int apply_common(tsqr_q_s* q, int mode, int64_t k, void* C, int64_t ldc, cudaStream_t s,
                 bool wait_tree = false) {
  if (!valid(q) || !q->factored) return TSQR_ERR_HANDLE;
  if (k < 0) return -2;
  if (k == 0) return TSQR_OK;
  if (!C) return -3;
  if (ldc < q->m) return -4;
  cudaError_t e = q->prec == TSQR_PREC_FP64 ? run_apply<double>(q, mode, k, (double*)C, ldc, s, nullptr, 0, wait_tree)
                                            : run_apply<float>(q, mode, k, (float*)C, ldc, s, nullptr, 0, wait_tree);
  return cuda_err(e);
}

}  // namespace

extern "C" {

int tsqr_factor(int64_t m, int64_t n, double* A, int64_t lda, double* R, int64_t ldr, const tsqr_opts_t* opts,
                tsqr_q_t* q, tsqr_stream_t stream) {
  return factor_common<double>(m, n, A, lda, R, ldr, opts, q, (cudaStream_t)stream, TSQR_PREC_FP64);
}

int tsqr_factor_f32(int64_t m, int64_t n, float* A, int64_t lda, float* R, int64_t ldr, const tsqr_opts_t* opts,
                    tsqr_q_t* q, tsqr_stream_t stream) {
  return factor_common<float>(m, n, A, lda, R, ldr, opts, q, (cudaStream_t)stream, TSQR_PREC_FP32);
}

int tsqr_q_create(int64_t m, int64_t n, int32_t precision, const tsqr_opts_t* opts, tsqr_q_t* q,
                  tsqr_stream_t stream) {
  if (!q) return -5;
  *q = nullptr;
  if (m < 1) return -1;
  if (n < 1 || n > m) return -2;
  if (precision != TSQR_PREC_FP64 && precision != TSQR_PREC_FP32) return -3;
  return create_handle(m, n, precision, opts, q, nullptr, (cudaStream_t)stream);
}

int tsqr_refactor(tsqr_q_t q, void* A, int64_t lda, void* R, int64_t ldr, tsqr_stream_t stream) {
  if (!valid(q)) return TSQR_ERR_HANDLE;
  if (!A) return -2;
  if (lda < q->m) return -3;
  if (!R) return -4;
  if (ldr < q->n) return -5;
  return refactor(q, A, lda, R, ldr, true, (cudaStream_t)stream);
}

int tsqr_apply_qt(tsqr_q_t q, int64_t k, void* C, int64_t ldc, tsqr_stream_t stream) {
  return apply_common(q, kApplyQT, k, C, ldc, (cudaStream_t)stream);
}

int tsqr_apply_q(tsqr_q_t q, int64_t k, void* C, int64_t ldc, tsqr_stream_t stream) {
  return apply_common(q, kApplyQ, k, C, ldc, (cudaStream_t)stream);
}

int tsqr_form_q(tsqr_q_t q, void* Q, int64_t ldq, tsqr_stream_t stream) {
  if (!valid(q) || !q->factored) return TSQR_ERR_HANDLE;
  if (!Q) return -2;
  if (ldq < q->m) return -3;
  if (Q == q->A) return -2;
  cudaError_t e = q->prec == TSQR_PREC_FP64 ? run_apply<double>(q, kApplyForm, q->n, (double*)Q, ldq, (cudaStream_t)stream)
                                            : run_apply<float>(q, kApplyForm, q->n, (float*)Q, ldq, (cudaStream_t)stream);
  return cuda_err(e);
}

int tsqr_form_q_mul(tsqr_q_t q, int64_t k, const void* X, int64_t ldx, void* Q, int64_t ldq, tsqr_stream_t stream) {
  if (!valid(q) || !q->factored) return TSQR_ERR_HANDLE;
  if (k < 0) return -2;
  if (k == 0) return TSQR_OK;
  if (!X) return -3;
  if (ldx < q->n) return -4;
  if (!Q || Q == q->A) return -5;
  if (ldq < q->m) return -6;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = q->prec == TSQR_PREC_FP64
                      ? run_apply<double>(q, kApplyForm, k, (double*)Q, ldq, s, (const double*)X, ldx)
                      : run_apply<float>(q, kApplyForm, k, (float*)Q, ldq, s, (const float*)X, ldx);
  return cuda_err(e);
}

int tsqr_factor_form_host(tsqr_q_t q, const void* A_host, int64_t lda_host, void* Q_host, int64_t ldq_host,
                          void* R_host, int64_t ldr_host, void* A, int64_t lda, void* Q, int64_t ldq, void* R,
                          int64_t ldr, tsqr_stream_t stream) {
  if (!valid(q)) return TSQR_ERR_HANDLE;
  if (q->hybrid) return TSQR_ERR_UNSUPPORTED;  // the copies are pipelined by leaf chunks
  const int64_t m = q->m, n = q->n;
  if (!A_host) return -2;
  if (lda_host < m) return -3;
  if (!Q_host) return -4;
  if (ldq_host < m) return -5;
  if (!R_host) return -6;
  if (ldr_host < n) return -7;
  if (!A) return -8;
  if (lda < m) return -9;
  if (Q == A || (!Q && !mapped_host(static_cast<const char*>(Q_host)))) return -10;
  if (Q && ldq < m) return -11;
  if (!R) return -12;
  if (ldr < n) return -13;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = q->prec == TSQR_PREC_FP64
                      ? run_factor_form_host<double>(q, (const double*)A_host, lda_host, (double*)Q_host, ldq_host,
                                                     (double*)R_host, ldr_host, (double*)A, lda, (double*)Q, ldq,
                                                     (double*)R, ldr, s)
                      : run_factor_form_host<float>(q, (const float*)A_host, lda_host, (float*)Q_host, ldq_host,
                                                    (float*)R_host, ldr_host, (float*)A, lda, (float*)Q, ldq,
                                                    (float*)R, ldr, s);
  return cuda_err(e);
}

int tsqr_sync_status(tsqr_q_t q, tsqr_stream_t stream) {
  if (!valid(q)) return TSQR_ERR_HANDLE;
  return read_status(q->status, (cudaStream_t)stream);
}

int tsqr_q_info(tsqr_q_t q, int64_t* m, int64_t* n, int32_t* precision, int64_t* leaves, int64_t* leaf_rows,
                int32_t* arity, int32_t* levels) {
  if (!valid(q)) return TSQR_ERR_HANDLE;
  if (m) *m = q->m;
  if (n) *n = q->n;
  if (precision) *precision = q->prec;
  if (leaves) *leaves = q->nleaves;
  if (leaf_rows) *leaf_rows = q->h;
  if (arity) *arity = q->q;
  if (levels) *levels = q->levels;
  return TSQR_OK;
}

int tsqr_lstsq(tsqr_q_t q, const void* R, int64_t ldr, int64_t k, void* B, int64_t ldb, void* X, int64_t ldx,
               void* rnorm, tsqr_stream_t stream) {
  if (!valid(q) || !q->factored) return TSQR_ERR_HANDLE;
  if (!R) return -2;
  if (ldr < q->n) return -3;
  if (k < 0) return -4;
  if (k == 0) return TSQR_OK;
  if (!B) return -5;
  if (ldb < q->m) return -6;
  if (!X) return -7;
  if (ldx < q->n) return -8;
  if (rnorm && k > 65535) return TSQR_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  // Q^T B (leaves, tree, signs): rows 0..n-1 = Q_thin^T B, the rest carry the residual.
  int rc = apply_common(q, kApplyQT, k, B, ldb, s);
  if (rc != TSQR_OK) return rc;
  const int n = (int)q->n;
  cudaError_t e = q->prec == TSQR_PREC_FP64
                      ? launch_solve_upper<double>(n, k, (const double*)R, ldr, (const double*)B, ldb, (double*)X, ldx,
                                                   q->status, s)
                      : launch_solve_upper<float>(n, k, (const float*)R, ldr, (const float*)B, ldb, (float*)X, ldx,
                                                  q->status, s);
  if (e != cudaSuccess || !rnorm) return cuda_err(e);
  double* acc = nullptr;
  if ((e = cudaMallocAsync((void**)&acc, sizeof(double) * k, s)) != cudaSuccess) return TSQR_ERR_NOMEM;
  e = q->prec == TSQR_PREC_FP64
          ? launch_column_norms<double>(q->n, q->m, k, (const double*)B, ldb, acc, (double*)rnorm, s)
          : launch_column_norms<float>(q->n, q->m, k, (const float*)B, ldb, acc, (float*)rnorm, s);
  const cudaError_t ef = cudaFreeAsync(acc, s);
  return cuda_err(e != cudaSuccess ? e : ef);
}

int tsqr_q_part(tsqr_q_t q, int32_t what, int32_t level, int64_t index, void* out, tsqr_stream_t stream) {
  if (!valid(q) || !q->factored) return TSQR_ERR_HANDLE;
  if (what < TSQR_PART_R || what > TSQR_PART_Y) return -2;
  if (level < 0 || level > q->levels || (what == TSQR_PART_Y && level == 0)) return -3;
  // Level 0: R per leaf (per chain for the hybrid tree), T and tau per leaf.
  const int64_t count = level == 0 && what != TSQR_PART_R ? q->nleaves : q->items[level];
  if (index < 0 || index >= count) return -4;
  if (!out) return -5;
  const size_t nn = (size_t)q->n * q->n * q->es, nv = (size_t)q->n * q->es;
  const unsigned char* src = nullptr;
  size_t bytes = 0;
  switch (what) {
    case TSQR_PART_R:
      src = (const unsigned char*)(level == 0 ? q->leafR : q->nodeR[level - 1]) + index * nn;
      bytes = nn;
      break;
    case TSQR_PART_T:
      src = (const unsigned char*)(level == 0 ? q->leafT : q->nodeT[level - 1]) + index * nn;
      bytes = nn;
      break;
    case TSQR_PART_TAU:
      src = (const unsigned char*)(level == 0 ? q->leafTau : q->nodeTau[level - 1]) + index * nv;
      bytes = nv;
      break;
    default:
      src = (const unsigned char*)q->nodeY[level - 1] + index * (q->q - 1) * nn;
      bytes = (q->q - 1) * nn;
  }
  return cuda_err(cudaMemcpyAsync(out, src, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
}

int tsqr_q_chains(tsqr_q_t q, int64_t* leaves_per_chain, int64_t* chains) {
  if (!valid(q)) return TSQR_ERR_HANDLE;
  if (leaves_per_chain) *leaves_per_chain = q->L;
  if (chains) *chains = q->nchains;
  return TSQR_OK;
}

int tsqr_q_destroy(tsqr_q_t q) { return destroy_handle(q); }

int tsqr_q_set_timing(tsqr_q_t q, int32_t enable) {
  if (!valid(q)) return TSQR_ERR_HANDLE;
  if (enable) clear_events(q);
  q->timing = enable != 0;
  return TSQR_OK;
}

int tsqr_q_stage_times(tsqr_q_t q, double* ms, int64_t* launches, int32_t count) {
  if (!valid(q)) return TSQR_ERR_HANDLE;
  if (count < 0 || count > TSQR_NUM_STAGES) return -4;
  for (int st = 0; st < count; ++st) {
    double tot = 0.0;
    for (auto& p : q->events[st]) {
      cudaError_t e = cudaEventSynchronize(p.second);
      if (e != cudaSuccess) return cuda_err(e);
      float t = 0.f;
      e = cudaEventElapsedTime(&t, p.first, p.second);
      if (e != cudaSuccess) return cuda_err(e);
      tot += t;
    }
    if (ms) ms[st] = tot;
    if (launches) launches[st] = q->launches[st];
  }
  return TSQR_OK;
}

// ------------------------------------------------------------------ CAQR --

int caqr_q_create(int64_t m, int64_t n, int64_t b, int32_t update_precision, const tsqr_opts_t* opts, caqr_q_t* q,
                  tsqr_stream_t stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (!q) return -6;
  *q = nullptr;
  if (m < 1) return -1;
  if (n < 1 || n > m) return -2;
  if (b < 1) return -3;
  if (update_precision != TSQR_PREC_FP64 && update_precision != TSQR_PREC_FP32 &&
      update_precision != TSQR_UPDATE_BF16X3 && update_precision != TSQR_UPDATE_TF32X3)
    return -4;
  if (opts && opts->flags != 0) return -5;
  caqr_q_s* c = new (std::nothrow) caqr_q_s();
  if (!c) return TSQR_ERR_NOMEM;
  c->m = m;
  c->n = n;
  c->b = b;
  c->prec = update_precision == TSQR_PREC_FP64 ? TSQR_PREC_FP64 : TSQR_PREC_FP32;
  c->es = c->prec == TSQR_PREC_FP64 ? 8 : 4;
  c->upd = update_precision;
  // Plan every panel, then one allocation for all of their workspaces.
  std::vector<tsqr_q_s*> plans;
  size_t total = 0;
  int rc = TSQR_OK;
  for (int64_t j0 = 0; j0 < n && rc == TSQR_OK; j0 += b) {
    const int64_t jb = (n - j0) < b ? (n - j0) : b;
    tsqr_q_s* p = new (std::nothrow) tsqr_q_s();
    if (!p) {
      rc = TSQR_ERR_NOMEM;
      break;
    }
    // Panels take the plain TSQR default (the tallest leaf that fits): the
    // tree part of each trailing update is about n / h of its leaf part.
    // FP32-storage panels: power-of-two leaves of at most kBf16x3MaxLeaf
    // rows (512 at b = 64: two tree levels per 8192-row panel, whose chain
    // of leaf and tree latencies bounds these forms).
    tsqr_opts_t po = opts ? *opts : tsqr_opts_t{0, 0, 0};
    po.flags = 0;  // the trailing-update arithmetic is update_precision
    if (po.leaf_rows == 0 && c->prec == TSQR_PREC_FP32) {
      int64_t h = 1;
      while (h * 2 <= (160 * 1024 / (int64_t)c->es) / jb && h * 2 <= kBf16x3MaxLeaf) h *= 2;
      po.leaf_rows = h < jb ? jb : h;
    }
    rc = make_plan(p, m - j0, jb, c->prec, &po);
    p->upd = update_precision;
    if (rc == -4) rc = -5;
    plans.push_back(p);
    total += workspace_bytes(p);
  }
  void* base = nullptr;
  if (rc == TSQR_OK) rc = cuda_err(cudaMalloc(&base, total));
  if (rc != TSQR_OK) {
    for (auto* p : plans) delete p;
    delete c;
    return rc;
  }
  c->ws = (unsigned char*)base;
  size_t off = 0;
  for (auto* p : plans) {
    p->owns_ws = false;
    bind_workspace(p, c->ws + off);
    off += workspace_bytes(p);
    c->panels.push_back(p);
  }
  c->status = c->panels[0]->status;
  for (auto* p : c->panels) {
    cudaError_t e = cudaMemsetAsync(p->status, 0, sizeof(int), s);
    if (e != cudaSuccess) rc = cuda_err(e);
  }
  // The look-ahead panel runs at the highest stream priority, so that its
  // few leaf CTAs take SMs as the trailing update's CTAs retire instead of
  // queueing behind the whole update.
  if (rc == TSQR_OK) {
    int lo = 0, hi = 0;
    if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess ||
        cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, hi) != cudaSuccess)
      rc = TSQR_ERR_CUDA;
  }
  if (rc == TSQR_OK && cudaStreamCreateWithFlags(&c->upd2, cudaStreamNonBlocking) != cudaSuccess) rc = TSQR_ERR_CUDA;
  c->ev_left.assign(c->panels.size(), nullptr);
  c->ev_fact.assign(c->panels.size(), nullptr);
  c->ev_leaf.assign(c->panels.size(), nullptr);
  c->ev_fork.assign(c->panels.size(), nullptr);
  c->ev_join.assign(c->panels.size(), nullptr);
  for (size_t j = 0; j < c->panels.size() && rc == TSQR_OK; ++j) {
    if (cudaEventCreateWithFlags(&c->ev_left[j], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fact[j], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_leaf[j], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork[j], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join[j], cudaEventDisableTiming) != cudaSuccess)
      rc = TSQR_ERR_CUDA;
    tsqr_q_s* p = c->panels[j];
    p->ev_level.assign(p->levels + 1, nullptr);
    for (auto& e : p->ev_level)
      if (rc == TSQR_OK && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) rc = TSQR_ERR_CUDA;
  }
  if (rc != TSQR_OK) {
    caqr_q_destroy(c);
    return rc;
  }
  *q = c;
  return TSQR_OK;
}

// Column granularity of the two-stream split of a trailing update (a
// multiple of both update kernels' column chunks).
constexpr int64_t kUpdateSplitCols = 128;

// Issues the panel loop on s (the caller's stream, or the capture stream).
static int caqr_issue(caqr_q_t c, void* A, int64_t lda, cudaStream_t s) {
  // Right-looking loop with a look-ahead of one panel (Section 3's panel
  // loop; the overlap is this implementation's): panel j+1's columns get
  // (Q_j D_j)^T first, then panel j+1 is factored on the side stream while
  // the remaining trailing columns are updated on the caller's stream.  The
  // two touch disjoint columns of A.  The leaf stage of panel j+1's update
  // needs only panel j's leaf factors, so (except under stage timing, whose
  // stage times must not overlap) it starts when those are in and runs
  // beside panel j's tree factorisation; its tree stage waits for the tree.
  const bool overlap = !c->timing;
  const size_t np = c->panels.size();
  const size_t es = c->es;
  auto at = [&](int64_t i, int64_t j) -> void* { return (unsigned char*)A + (size_t)(i + j * lda) * es; };
  int rc = refactor(c->panels[0], A, lda, A, lda, false, s);
  if (rc != TSQR_OK) return rc;
  int64_t joined = -1;  // panel whose second update half the caller's stream has not yet waited for
  for (size_t j = 0; j < np; ++j) {
    tsqr_q_s* p = c->panels[j];
    const int64_t j0 = (int64_t)j * c->b;
    const int64_t j1 = j0 + p->n;          // first trailing column
    if (j + 1 == np) break;
    tsqr_q_s* nx = c->panels[j + 1];
    rc = apply_common(p, kApplyQT, nx->n, at(j0, j1), lda, s, overlap && j > 0);
    if (rc != TSQR_OK) return rc;
    if (cudaEventRecord(c->ev_left[j], s) != cudaSuccess) return TSQR_ERR_CUDA;
    if (cudaStreamWaitEvent(c->side, c->ev_left[j], 0) != cudaSuccess) return TSQR_ERR_CUDA;
    void* P = at(j1, j1);
    rc = refactor(nx, P, lda, P, lda, false, c->side, overlap ? c->ev_leaf[j + 1] : nullptr);
    if (rc != TSQR_OK) return rc;
    if (cudaEventRecord(c->ev_fact[j + 1], c->side) != cudaSuccess) return TSQR_ERR_CUDA;
    const int64_t kt = c->n - j1 - nx->n;
    if (kt > 0) {
      // The previous step's second half may have touched any of these columns.
      if (joined >= 0 && cudaStreamWaitEvent(s, c->ev_join[joined], 0) != cudaSuccess) return TSQR_ERR_CUDA;
      joined = -1;
      // FP64 only (its updates bound the loop; the FP32-storage forms are
      // bound by the panel chain, which the split slows a little), and not
      // under stage timing, whose per-stage event times must not overlap.
      const bool split = c->upd == TSQR_PREC_FP64 && !c->timing && kt >= 8 * kUpdateSplitCols;
      const int64_t kt1 = split ? (kt / 2 + kUpdateSplitCols - 1) / kUpdateSplitCols * kUpdateSplitCols : kt;
      if (kt1 < kt) {
        if (cudaEventRecord(c->ev_fork[j], s) != cudaSuccess) return TSQR_ERR_CUDA;
        if (cudaStreamWaitEvent(c->upd2, c->ev_fork[j], 0) != cudaSuccess) return TSQR_ERR_CUDA;
        rc = apply_common(p, kApplyQT, kt - kt1, at(j0, j1 + nx->n + kt1), lda, c->upd2);
        if (rc != TSQR_OK) return rc;
        if (cudaEventRecord(c->ev_join[j], c->upd2) != cudaSuccess) return TSQR_ERR_CUDA;
        joined = (int64_t)j;
      }
      rc = apply_common(p, kApplyQT, kt1, at(j0, j1 + nx->n), lda, s);
      if (rc != TSQR_OK) return rc;
    }
    // Panel j+1's leaf factors (overlap) or its whole factorisation: the
    // next iteration's first product needs the former, its tree stage
    // waits for ev_fact[j + 1] itself.
    if (cudaStreamWaitEvent(s, overlap ? c->ev_leaf[j + 1] : c->ev_fact[j + 1], 0) != cudaSuccess)
      return TSQR_ERR_CUDA;
  }
  // The last panel's tree (its R rows) before the caller's stream goes on.
  if (overlap && np > 1 && cudaStreamWaitEvent(s, c->ev_fact[np - 1], 0) != cudaSuccess) return TSQR_ERR_CUDA;
  if (joined >= 0 && cudaStreamWaitEvent(s, c->ev_join[joined], 0) != cudaSuccess) return TSQR_ERR_CUDA;
  return TSQR_OK;
}

int caqr_refactor(caqr_q_t c, void* A, int64_t lda, tsqr_stream_t stream) {
  if (!valid(c)) return TSQR_ERR_HANDLE;
  if (!A) return -2;
  if (lda < c->m) return -3;
  cudaStream_t s = (cudaStream_t)stream;
  c->A = A;
  c->lda = lda;
  // With stage timing on, the loop runs directly (its events time real
  // launches).  Otherwise the loop (a few thousand launches at n = 8192,
  // whose host-side cost would otherwise pace the late, small panels) is
  // captured once per (A, lda) and replayed as one graph launch.
  if (c->timing) return caqr_issue(c, A, lda, s);
  if (!c->graph || c->graph_A != A || c->graph_lda != lda) {
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
    if (!c->cap && cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) return TSQR_ERR_CUDA;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return TSQR_ERR_CUDA;
    const int rc = caqr_issue(c, A, lda, c->cap);
    const cudaError_t e = cudaStreamEndCapture(c->cap, &g);
    if (rc != TSQR_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return cuda_err(e);
    const cudaError_t ei = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      c->graph = nullptr;
      return cuda_err(ei);
    }
    c->graph_A = A;
    c->graph_lda = lda;
  }
  return cuda_err(cudaGraphLaunch(c->graph, s));
}

static int caqr_factor_any(int64_t m, int64_t n, void* A, int64_t lda, int64_t b, int32_t update_precision,
                           const tsqr_opts_t* opts, caqr_q_t* q, tsqr_stream_t stream) {
  cudaStream_t s = (cudaStream_t)stream;
  caqr_q_t c = nullptr;
  int rc = caqr_q_create(m, n, b, update_precision, opts, &c, stream);
  if (rc != TSQR_OK) return rc == -5 ? -7 : rc;
  // One factorisation: the loop runs directly (a graph would not be reused).
  c->A = A;
  c->lda = lda;
  rc = caqr_issue(c, A, lda, s);
  if (rc != TSQR_OK || !q) {
    cudaStreamSynchronize(s);
    caqr_q_destroy(c);
    return rc;
  }
  *q = c;
  return TSQR_OK;
}

int caqr_factor(int64_t m, int64_t n, double* A, int64_t lda, int64_t b, int32_t update_precision,
                const tsqr_opts_t* opts, caqr_q_t* q, tsqr_stream_t stream) {
  if (q) *q = nullptr;
  if (m < 0) return -1;
  if (n < 0 || n > m) return -2;
  if (m > 0 && n > 0 && !A) return -3;
  if (lda < (m > 1 ? m : 1)) return -4;
  if (b < 1) return -5;
  if (update_precision != TSQR_PREC_FP64) return -6;
  if (m == 0 || n == 0) return TSQR_OK;
  return caqr_factor_any(m, n, A, lda, b, update_precision, opts, q, stream);
}

int caqr_factor_f32(int64_t m, int64_t n, float* A, int64_t lda, int64_t b, int32_t update_precision,
                    const tsqr_opts_t* opts, caqr_q_t* q, tsqr_stream_t stream) {
  if (q) *q = nullptr;
  if (m < 0) return -1;
  if (n < 0 || n > m) return -2;
  if (m > 0 && n > 0 && !A) return -3;
  if (lda < (m > 1 ? m : 1)) return -4;
  if (b < 1) return -5;
  if (update_precision != TSQR_PREC_FP32 && update_precision != TSQR_UPDATE_BF16X3 &&
      update_precision != TSQR_UPDATE_TF32X3)
    return -6;
  if (m == 0 || n == 0) return TSQR_OK;
  return caqr_factor_any(m, n, A, lda, b, update_precision, opts, q, stream);
}

int caqr_apply_qt(caqr_q_t q, int64_t k, void* C, int64_t ldc, tsqr_stream_t stream) {
  if (!valid(q)) return TSQR_ERR_HANDLE;
  if (k < 0) return -2;
  if (k == 0) return TSQR_OK;
  if (!C) return -3;
  if (ldc < q->m) return -4;
  for (size_t j = 0; j < q->panels.size(); ++j) {
    const int64_t j0 = (int64_t)j * q->b;
    int rc = apply_common(q->panels[j], kApplyQT, k, (unsigned char*)C + j0 * q->es, ldc, (cudaStream_t)stream);
    if (rc != TSQR_OK) return rc;
  }
  return TSQR_OK;
}

int caqr_apply_q(caqr_q_t q, int64_t k, void* C, int64_t ldc, tsqr_stream_t stream) {
  if (!valid(q)) return TSQR_ERR_HANDLE;
  if (k < 0) return -2;
  if (k == 0) return TSQR_OK;
  if (!C) return -3;
  if (ldc < q->m) return -4;
  for (size_t j = q->panels.size(); j-- > 0;) {
    const int64_t j0 = (int64_t)j * q->b;
    int rc = apply_common(q->panels[j], kApplyQ, k, (unsigned char*)C + j0 * q->es, ldc, (cudaStream_t)stream);
    if (rc != TSQR_OK) return rc;
  }
  return TSQR_OK;
}

int caqr_form_q(caqr_q_t q, void* Q, int64_t ldq, tsqr_stream_t stream) {
  if (!valid(q)) return TSQR_ERR_HANDLE;
  if (!Q) return -2;
  if (ldq < q->m) return -3;
  if (Q == q->A) return -2;
  cudaStream_t s = (cudaStream_t)stream;
  // Q = Q_0 diag(I, Q_1) diag(I, Q_2) ... [I_n; 0]: start from [I_n; 0] and
  // apply the panels last to first, each to the columns it can reach.
  cudaError_t e = cudaMemset2DAsync(Q, ldq * q->es, 0, q->m * q->es, q->n, s);
  if (e != cudaSuccess) return cuda_err(e);
  e = q->prec == TSQR_PREC_FP64 ? launch_init_form<double>((double*)Q, ldq, (int)q->n, nullptr, s)
                                : launch_init_form<float>((float*)Q, ldq, (int)q->n, nullptr, s);
  if (e != cudaSuccess) return cuda_err(e);
  for (size_t j = q->panels.size(); j-- > 0;) {
    const int64_t j0 = (int64_t)j * q->b;
    int rc = apply_common(q->panels[j], kApplyQ, q->n - j0, (unsigned char*)Q + (size_t)(j0 + j0 * ldq) * q->es, ldq, s);
    if (rc != TSQR_OK) return rc;
  }
  return TSQR_OK;
}

int caqr_q_set_timing(caqr_q_t q, int32_t enable) {
  if (!valid(q)) return TSQR_ERR_HANDLE;
  q->timing = enable != 0;
  for (auto* p : q->panels) tsqr_q_set_timing(p, enable);
  return TSQR_OK;
}

int caqr_q_stage_times(caqr_q_t q, double* ms, int64_t* launches, int32_t count) {
  if (!valid(q)) return TSQR_ERR_HANDLE;
  if (count < 0 || count > TSQR_NUM_STAGES) return -4;
  double tot_ms[TSQR_NUM_STAGES] = {0, 0, 0, 0};
  int64_t tot_l[TSQR_NUM_STAGES] = {0, 0, 0, 0};
  for (auto* p : q->panels) {
    double pm[TSQR_NUM_STAGES];
    int64_t pl[TSQR_NUM_STAGES];
    int rc = tsqr_q_stage_times(p, pm, pl, TSQR_NUM_STAGES);
    if (rc != TSQR_OK) return rc;
    for (int st = 0; st < TSQR_NUM_STAGES; ++st) {
      tot_ms[st] += pm[st];
      tot_l[st] += pl[st];
    }
  }
  for (int st = 0; st < count; ++st) {
    if (ms) ms[st] = tot_ms[st];
    if (launches) launches[st] = tot_l[st];
  }
  return TSQR_OK;
}

int caqr_sync_status(caqr_q_t q, tsqr_stream_t stream) {
  if (!valid(q)) return TSQR_ERR_HANDLE;
  int worst = TSQR_OK;
  for (auto* p : q->panels) {
    int rc = read_status(p->status, (cudaStream_t)stream);
    if (rc != TSQR_OK) worst = rc;
  }
  return worst;
}

int caqr_q_destroy(caqr_q_t q) {
  if (!valid(q)) return TSQR_ERR_HANDLE;
  q->magic = 0;
  if (q->side) {
    cudaStreamSynchronize(q->side);
    cudaStreamDestroy(q->side);
  }
  for (auto e : q->ev_left)
    if (e) cudaEventDestroy(e);
  for (auto e : q->ev_fact)
    if (e) cudaEventDestroy(e);
  for (auto e : q->ev_leaf)
    if (e) cudaEventDestroy(e);
  for (auto e : q->ev_fork)
    if (e) cudaEventDestroy(e);
  for (auto e : q->ev_join)
    if (e) cudaEventDestroy(e);
  if (q->upd2) {
    cudaStreamSynchronize(q->upd2);
    cudaStreamDestroy(q->upd2);
  }
  for (auto* p : q->panels) destroy_handle(p);
  cudaError_t e = q->ws ? cudaFree(q->ws) : cudaSuccess;
  if (q->graph) cudaGraphExecDestroy(q->graph);
  if (q->cap) cudaStreamDestroy(q->cap);
  delete q;
  return cuda_err(e);
}

const char* tsqr_status_string(int code) {
  if (code < 0) return "invalid argument";
  switch (code) {
    case TSQR_OK: return "ok";
    case TSQR_ERR_CUDA: return "CUDA runtime error";
    case TSQR_ERR_NOMEM: return "device allocation failed";
    case TSQR_ERR_TIMEOUT: return "device-side wait timed out";
    case TSQR_ERR_NONFINITE: return "non-finite value in a column norm or pivot";
    case TSQR_ERR_UNSUPPORTED: return "unsupported shape or precision";
    case TSQR_ERR_HANDLE: return "invalid handle";
    case TSQR_ERR_TOO_LARGE: return "problem exceeds the no-allocation entry point's static scratch";
    default: return "unknown status";
  }
}

int tsqr_version(void) { return 100; }

}  // extern "C"
