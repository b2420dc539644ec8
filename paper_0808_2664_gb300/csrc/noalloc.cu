// tsqr_factor_r_noalloc: the TSQR R factor with no device allocation.
//
// Some callers cannot call cudaMalloc: code running inside another
// allocator's callback, plugins of frameworks that own all device memory
// through their own pool, or a process whose memory budget is fixed before
// the factorisation is first needed.  This entry point gives them the R
// factor of a tall-skinny FP64 matrix using only memory that exists from the
// moment the library is loaded: a file-scope device array of
// kScratchBytes (64 MiB), which every GPU that loads the library holds until
// the process exits.  It runs the same leaf and tree-node kernels as
// tsqr_factor, with their workspace (leaf R and T factors, tree nodes, signs,
// status word) carved out of that array.  No Q handle is returned.
//
// Set-up: the first call on each device takes the array's device address
// with cudaGetSymbolAddress while that device is current; make that first
// call before any stream capture.  All calls share the one array and it
// keeps the previous call's contents (everything the kernels read is written
// first within a call; the status word is cleared by each call), so calls
// whose work overlaps on the GPU -- on different streams, or from different
// host threads -- race with each other and must be serialised by the caller.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/tsqr.h"
#include "tsqr_internal.cuh"

namespace tsqr {
size_t node_factor_smem(int n, int q, size_t elem);
}  // namespace tsqr

using namespace tsqr;

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;
constexpr int kMaxLevels = 64;
constexpr size_t kAlignNa = 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array for the current device (looked up once per device).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
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
  if (n > kMaxN) return TSQR_ERR_UNSUPPORTED;

  // A fixed plan: leaves of a power-of-two height within 68 KB, binary tree.
  int64_t h = 1;
  while (h * 2 <= (68 * 1024 / 8) / n && h * 2 <= 1024) h *= 2;
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
  int dev = 0, smax = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return TSQR_ERR_CUDA;
  if (leaf_factor_smem((int)n, leaf_factor_ld((int)hmax), 8) > (size_t)smax) return TSQR_ERR_UNSUPPORTED;
  if (levels > 0 && node_factor_smem((int)n, q, 8) > (size_t)smax) return TSQR_ERR_UNSUPPORTED;

  // Workspace layout inside the static array; reject problems that do not fit.
  const size_t nn = (size_t)n * n * 8, nv = (size_t)n * 8;
  size_t off_leafR = 0, off_leafT = al(nl * nn), off_leafTau = off_leafT + al(nl * nn);
  size_t off = off_leafTau + al(nl * nv);
  size_t offR[kMaxLevels], offT[kMaxLevels], offY[kMaxLevels], offTau[kMaxLevels];
  for (int l = 1; l <= levels; ++l) {
    const size_t it = (size_t)items[l];
    offR[l - 1] = off;
    off += al(it * nn);
    offT[l - 1] = off;
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
  la.ld_s = leaf_factor_ld((int)hmax);
  la.R = (double*)(b + off_leafR);
  la.tau = (double*)(b + off_leafTau);
  la.Tw = (double*)(b + off_leafT);
  la.status = status;
  if (launch_leaf_factor(la, s) != cudaSuccess) return TSQR_ERR_CUDA;
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
    na.Tw = (double*)(b + offT[l - 1]);
    na.status = status;
    if (launch_node_factor(na, s) != cudaSuccess) return TSQR_ERR_CUDA;
  }
  const double* root = (const double*)(b + (levels == 0 ? off_leafR : offR[levels - 1]));
  if (launch_sign_fix(root, (int)n, (double*)(b + off_d), R, ldr, true, s) != cudaSuccess) return TSQR_ERR_CUDA;
  return TSQR_OK;
}
