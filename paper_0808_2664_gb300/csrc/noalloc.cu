// tsqr_factor_r_noalloc: the TSQR R factor with no device allocation.
//
// Some callers cannot call cudaMalloc: code running inside another
// allocator's callback, plugins of frameworks that own all device memory
// through their own pool, or a process whose memory budget is fixed before
// the factorisation is first needed.  This entry point gives them the R
// factor of a tall-skinny FP64 matrix (n <= 64) using only memory that
// exists from the moment the library is loaded: a file-scope device array
// of kScratchBytes (64 MiB), which every GPU that loads the library holds
// until the process exits.  It runs the leaf QR and the binary tree-node QR
// of tsqr_factor in their R-only form (no compact-WY T: no Q is returned),
// with their workspace (leaf R factors, tree-node R and reflector blocks,
// signs, status word) carved out of that array.
//
// Set-up: the array's device address is looked up with cudaGetSymbolAddress
// while the device is current, once per device context (the first call on a
// device, and the first call after that device's context was re-created,
// e.g. after cudaDeviceReset); make that first call before any stream
// capture.  All calls share the one array and it keeps the previous call's
// contents (everything the kernels read is written first within a call; the
// status word is cleared by each call), so calls whose work overlaps on the
// GPU -- on different streams, or from different host threads -- race with
// each other and must be serialised by the caller.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/tsqr.h"
#include "leaf_device.cuh"
#include "node2_device.cuh"
#include "tsqr_internal.cuh"

using namespace tsqr;

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;
constexpr int kMaxLevels = 64;
constexpr size_t kAlignNa = 256;
constexpr int kNaThreads = 128;  // leaf and node CTAs
constexpr int kNaNmax = 64;      // widest matrix served
constexpr size_t kNaTileBytes = 68 * 1024;  // leaf tile budget: leaves of a power-of-two height

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// R-only leaf QR of every leaf (Section 2.1, Eq. TSQR_binarytree_1).
__global__ void __launch_bounds__(kNaThreads) noalloc_leaf_kernel(LeafFactorArgs<double> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int64_t nn = (int64_t)a.n * a.n;
  for (int64_t leaf = blockIdx.x; leaf < a.nleaves; leaf += gridDim.x) {
    const int64_t r0 = leaf * a.h;
    const int hl = (leaf == a.nleaves - 1) ? (int)(a.m - r0) : (int)a.h;
    leaf_factor_one<double, kNaThreads, kNaNmax, false>(a.A + r0, a.lda, hl, a.n, a.ld_s, a.R + leaf * nn,
                                                        a.tau + leaf * (int64_t)a.n, nullptr, a.status, smem);
  }
}

// R-only structured QR of pairs of stacked triangles (Eqs. TSQR_binarytree_2/_3).
__global__ void __launch_bounds__(kNaThreads) noalloc_node_kernel(NodeFactorArgs<double> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  for (int64_t node = blockIdx.x; node < a.nodes; node += gridDim.x)
    node2_factor_group<double, kNaThreads, 1, 2, false>(a.Rin, a.nin, a.nodes, node, a.n, a.Rout, a.Y, nullptr,
                                                        a.tau, a.status, smem);
}

// Device address of the scratch array in the current context, cached per
// device and keyed on the context's unique id, so that a context created
// after cudaDeviceReset looks the address up again.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

std::mutex g_mu;
struct ScratchEntry {
  unsigned long long ctx_id = 0;
  void* ptr = nullptr;
};
ScratchEntry g_scratch[kMaxDevices];
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
bool g_fns_tried = false;

cudaError_t current_context_id(unsigned long long* id) {
  if (!g_fns_tried) {
    g_fns_tried = true;
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", (void**)&g_ctx_get_current, 12000, cudaEnableDefault,
                                         &q1) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess)
      g_ctx_get_current = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", (void**)&g_ctx_get_id, 12000, cudaEnableDefault, &q2) !=
            cudaSuccess ||
        q2 != cudaDriverEntryPointSuccess)
      g_ctx_get_id = nullptr;
  }
  if (!g_ctx_get_current || !g_ctx_get_id) return cudaErrorNotSupported;
  CUcontext ctx = nullptr;
  if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorContextIsDestroyed;
  return g_ctx_get_id(ctx, id) == CUDA_SUCCESS ? cudaSuccess : cudaErrorContextIsDestroyed;
}

cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  // Makes the device's primary context current (a no-op when it already is).
  if ((e = cudaSetDevice(dev)) != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_mu);
  unsigned long long id = 0;
  if ((e = current_context_id(&id)) != cudaSuccess) {
    // Without a context id, look the address up on every call.
    void* p = nullptr;
    if ((e = cudaGetSymbolAddress(&p, g_noalloc_scratch)) != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
  }
  ScratchEntry& s = g_scratch[dev];
  if (!s.ptr || s.ctx_id != id) {
    void* p = nullptr;
    if ((e = cudaGetSymbolAddress(&p, g_noalloc_scratch)) != cudaSuccess) return e;
    s.ptr = p;
    s.ctx_id = id;
  }
  *out = s.ptr;
  return cudaSuccess;
}

size_t al(size_t x) { return (x + kAlignNa - 1) / kAlignNa * kAlignNa; }

}  // namespace

extern "C" int tsqr_factor_r_noalloc(int64_t m, int64_t n, double* A, int64_t lda, double* R, int64_t ldr,
                                     tsqr_stream_t stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (m < 0) return -1;
  if (n < 0 || n > m) return -2;
  if (m > 0 && n > 0 && !A) return -3;
  if (lda < (m > 1 ? m : 1)) return -4;
  if (m > 0 && n > 0 && !R) return -5;
  if (ldr < (n > 1 ? n : 1)) return -6;
  if (m == 0 || n == 0) return TSQR_OK;
  if (n > kNaNmax) return TSQR_ERR_UNSUPPORTED;

  // A fixed plan: leaves of a power-of-two height whose tile fits 68 KB,
  // binary tree.
  int64_t h = 1;
  while (h * 2 <= (int64_t)(kNaTileBytes / 8) / n && h * 2 <= 1024) h *= 2;
  if (h < n) h = n;
  int64_t nl = (m + h - 1) / h;
  if (nl > 1 && m - (nl - 1) * h < n) --nl;
  const int64_t hmax = nl > 1 ? (m - (nl - 1) * h > h ? m - (nl - 1) * h : h) : m;
  const int q = 2;
  int64_t items[kMaxLevels + 1];
  int levels = 0;
  items[0] = nl;
  while (items[levels] > 1) {
    if (levels == kMaxLevels) return TSQR_ERR_UNSUPPORTED;
    items[levels + 1] = (items[levels] + q - 1) / q;
    ++levels;
  }
  int dev = 0, smax = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return TSQR_ERR_CUDA;
  const int ld_s = leaf_factor_ld((int)hmax);
  const size_t leaf_smem = leaf_smem_bytes((int)n, ld_s, 8, kNaThreads);
  const size_t node_smem = node2_smem_bytes((int)n, 1, 8, kNaThreads, q);
  if (leaf_smem > (size_t)smax) return TSQR_ERR_UNSUPPORTED;
  if (levels > 0 && node_smem > (size_t)smax) return TSQR_ERR_UNSUPPORTED;

  // Workspace layout inside the static array; reject problems that do not fit.
  const size_t nn = (size_t)n * n * 8, nv = (size_t)n * 8;
  const size_t off_leafR = 0, off_leafTau = al(nl * nn);
  size_t off = off_leafTau + al(nl * nv);
  size_t offR[kMaxLevels], offY[kMaxLevels], offTau[kMaxLevels];
  for (int l = 1; l <= levels; ++l) {
    const size_t it = (size_t)items[l];
    offR[l - 1] = off;
    off += al(it * nn);
    offY[l - 1] = off;
    off += al(it * (q - 1) * nn);
    offTau[l - 1] = off;
    off += al(it * nv);
  }
  const size_t off_d = off;
  off += al(nv);
  const size_t off_status = off;
  off += al(sizeof(int));
  if (off > kScratchBytes) return TSQR_ERR_TOO_LARGE;

  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return TSQR_ERR_CUDA;
  unsigned char* b = (unsigned char*)base;
  int* status = (int*)(b + off_status);
  if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) return TSQR_ERR_CUDA;

  LeafFactorArgs<double> la{};
  la.A = A;
  la.lda = lda;
  la.m = m;
  la.n = (int)n;
  la.h = h;
  la.nleaves = nl;
  la.ld_s = ld_s;
  la.R = (double*)(b + off_leafR);
  la.tau = (double*)(b + off_leafTau);
  la.Tw = nullptr;
  la.status = status;
  if (cudaFuncSetAttribute(noalloc_leaf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)leaf_smem) !=
      cudaSuccess)
    return TSQR_ERR_CUDA;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, noalloc_leaf_kernel, kNaThreads, leaf_smem) !=
          cudaSuccess ||
      per_sm < 1)
    return TSQR_ERR_CUDA;
  int64_t grid = (int64_t)sms * per_sm;
  if (grid > nl) grid = nl;
  noalloc_leaf_kernel<<<(unsigned)grid, kNaThreads, leaf_smem, s>>>(la);
  if (cudaGetLastError() != cudaSuccess) return TSQR_ERR_CUDA;
  if (levels > 0 && cudaFuncSetAttribute(noalloc_node_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)node_smem) != cudaSuccess)
    return TSQR_ERR_CUDA;
  for (int l = 1; l <= levels; ++l) {
    NodeFactorArgs<double> na{};
    na.Rin = (const double*)(b + (l == 1 ? off_leafR : offR[l - 2]));
    na.nin = items[l - 1];
    na.arity = q;
    na.n = (int)n;
    na.nodes = items[l];
    na.Rout = (double*)(b + offR[l - 1]);
    na.Y = (double*)(b + offY[l - 1]);
    na.tau = (double*)(b + offTau[l - 1]);
    na.Tw = nullptr;
    na.status = status;
    int64_t g = (int64_t)sms * 4;
    if (g > na.nodes) g = na.nodes;
    noalloc_node_kernel<<<(unsigned)g, kNaThreads, node_smem, s>>>(na);
    if (cudaGetLastError() != cudaSuccess) return TSQR_ERR_CUDA;
  }
  const double* root = (const double*)(b + (levels == 0 ? off_leafR : offR[levels - 1]));
  if (launch_sign_fix(root, (int)n, (double*)(b + off_d), R, ldr, true, s) != cudaSuccess) return TSQR_ERR_CUDA;
  return TSQR_OK;
}
