// Entry points of include/tsqr_testing.h: single internal device steps run on
// caller-supplied inputs for the test suite.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../../include/tsqr_testing.h"
#include "reflector.cuh"
#include "tsqr_internal.cuh"

namespace tsqr {
namespace {

__global__ void reflector_test_kernel(int64_t count, const double* alpha, const double* ssq, int fast, double* out,
                                      int* status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const double a = alpha[i], s2 = ssq[i];
    auto rescan = [&]() { return sqrt(s2); };
    const Reflector r = fast ? make_reflector_fast(a, s2, rescan, status) : make_reflector(a, s2, rescan, status);
    out[3 * i] = r.beta;
    out[3 * i + 1] = r.tau;
    out[3 * i + 2] = r.scale;
  }
}

}  // namespace
}  // namespace tsqr

extern "C" int tsqr_test_reflectors(int64_t count, const double* alpha, const double* ssq, int32_t fast, double* out,
                                    tsqr_stream_t stream) {
  if (count < 0) return -1;
  if (count == 0) return TSQR_OK;
  if (!alpha) return -2;
  if (!ssq) return -3;
  if (!out) return -5;
  int* status = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMallocAsync((void**)&status, sizeof(int), s) != cudaSuccess) return TSQR_ERR_NOMEM;
  cudaMemsetAsync(status, 0, sizeof(int), s);
  int64_t blocks = (count + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  tsqr::reflector_test_kernel<<<(unsigned)blocks, 256, 0, s>>>(count, alpha, ssq, fast ? 1 : 0, out, status);
  const cudaError_t e = cudaGetLastError();
  cudaFreeAsync(status, s);
  return e == cudaSuccess ? TSQR_OK : TSQR_ERR_CUDA;
}
