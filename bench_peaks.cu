// Throughput probes for the roofline denominators that MEASURED_PEAKS.json
// does not hold: FP64 FMA, FP32 FMA and FP64 mma.sync m8n8k4 (DMMA) rates,
// each from independent FMA chains over a full grid, timed with CUDA events,
// DFMA and DMMA run side by side (whether they share the FP64 units), and a
// dependent DFMA chain per warp with one or all lanes active.
// The benchmark's FP64 roofline is derived from unit counts and clocks; these
// rates show how close a plain FMA loop gets to it.  Build and run with
// `python bench.py --peaks`, or:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o /tmp/bench_peaks bench_peaks.cu && /tmp/bench_peaks
#include <cstdio>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("CUDA %s @%d\n",cudaGetErrorString(e),__LINE__); return 1;}}while(0)

template<int CH>
__global__ void fma64(double* out, int iters, double a, double b) {
  double x[CH];
  #pragma unroll
  for (int c = 0; c < CH; ++c) x[c] = threadIdx.x * 1e-3 + c;
  for (int i = 0; i < iters; ++i) {
    #pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0; 
  #pragma unroll
  for (int c = 0; c < CH; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
template<int CH>
__global__ void fma32(float* out, int iters, float a, float b) {
  float x[CH];
  #pragma unroll
  for (int c = 0; c < CH; ++c) x[c] = threadIdx.x * 1e-3f + c;
  for (int i = 0; i < iters; ++i) {
    #pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0;
  #pragma unroll
  for (int c = 0; c < CH; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void dmma(double* out, int iters) {
  double a = 1.0 + threadIdx.x * 1e-6, b = 0.5;
  double c[4][2];
  for (int k = 0; k < 4; ++k) { c[k][0] = 0; c[k][1] = 0; }
  for (int i = 0; i < iters; ++i) {
    #pragma unroll
    for (int k = 0; k < 4; ++k)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(c[k][0]), "+d"(c[k][1]) : "d"(a), "d"(b));
  }
  double s = 0; for (int k = 0; k < 4; ++k) s += c[k][0] + c[k][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
// Half of each CTA's warps run FP64 FMA chains and half DMMA chains, each
// half with the work it would do alone: if the two shared no units the pair
// would finish in about half the time of either alone.
__global__ void dfma_dmma(double* out, int iters_f, int iters_m, int fwarps) {
  const int warp = threadIdx.x >> 5;
  double s = 0;
  if (warp < fwarps) {
    double x[8];
    for (int c = 0; c < 8; ++c) x[c] = threadIdx.x * 1e-3 + c;
    for (int i = 0; i < iters_f; ++i) {
      #pragma unroll
      for (int c = 0; c < 8; ++c) x[c] = fma(x[c], 1.0000001, 1e-9);
    }
    for (int c = 0; c < 8; ++c) s += x[c];
  } else {
    double a = 1.0 + threadIdx.x * 1e-6, b = 0.5, c[4][2];
    for (int k = 0; k < 4; ++k) { c[k][0] = 0; c[k][1] = 0; }
    for (int i = 0; i < iters_m; ++i) {
      #pragma unroll
      for (int k = 0; k < 4; ++k)
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                     : "+d"(c[k][0]), "+d"(c[k][1]) : "d"(a), "d"(b));
    }
    for (int k = 0; k < 4; ++k) s += c[k][0] + c[k][1];
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
// A dependent FP64 FMA chain per warp with 1 or 32 active lanes: whether an
// FP64 instruction's cost on its SM sub-partition depends on its lanes.
__global__ void dfma_lanes(double* out, int iters, int lanes) {
  double x = threadIdx.x * 1e-3;
  if ((int)(threadIdx.x & 31) < lanes)
    for (int i = 0; i < iters; ++i) x = fma(x, 1.0000001, 1e-9);
  out[blockIdx.x * blockDim.x + threadIdx.x] = x;
}
int main() {
  int dev = 0; cudaDeviceProp p; CK(cudaGetDeviceProperties(&p, dev));
  printf("name=%s sms=%d cc=%d.%d smem/block optin=%zu l2=%d\n", p.name, p.multiProcessorCount, p.major, p.minor,
         p.sharedMemPerBlockOptin, p.l2CacheSize);
  int sms = p.multiProcessorCount;
  double* d; CK(cudaMalloc(&d, sizeof(double) * sms * 16 * 1024));
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  for (int blocksPerSm : {1, 2, 4, 8}) {
    for (int threads : {128, 256}) {
      int grid = sms * blocksPerSm; int iters = 4096;
      fma64<8><<<grid, threads>>>(d, 16, 1.0000001, 1e-9); CK(cudaDeviceSynchronize());
      cudaEventRecord(e0); fma64<8><<<grid, threads>>>(d, iters, 1.0000001, 1e-9); cudaEventRecord(e1);
      CK(cudaEventSynchronize(e1)); float ms; cudaEventElapsedTime(&ms, e0, e1);
      double fl = 2.0 * 8 * iters * (double)grid * threads;
      printf("fp64 fma: bps=%d thr=%d  %.3f ms  %.3f TFLOP/s\n", blocksPerSm, threads, ms, fl / ms / 1e9);
    }
  }
  for (int blocksPerSm : {2, 4, 8}) {
    int grid = sms * blocksPerSm, threads = 256, iters = 16384;
    fma32<8><<<grid, threads>>>((float*)d, 16, 1.0000001f, 1e-9f); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); fma32<8><<<grid, threads>>>((float*)d, iters, 1.0000001f, 1e-9f); cudaEventRecord(e1);
    CK(cudaEventSynchronize(e1)); float ms; cudaEventElapsedTime(&ms, e0, e1);
    double fl = 2.0 * 8 * iters * (double)grid * threads;
    printf("fp32 fma: bps=%d  %.3f ms  %.3f TFLOP/s\n", blocksPerSm, ms, fl / ms / 1e9);
  }
  for (int blocksPerSm : {1, 2, 4}) {
    int grid = sms * blocksPerSm, threads = 256, iters = 1024;
    dmma<<<grid, threads>>>(d, 8); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); dmma<<<grid, threads>>>(d, iters); cudaEventRecord(e1);
    CK(cudaEventSynchronize(e1)); float ms; cudaEventElapsedTime(&ms, e0, e1);
    double fl = 2.0 * 8 * 8 * 4 * 4.0 * iters * (double)grid * (threads / 32);
    printf("dmma m8n8k4: bps=%d  %.3f ms  %.3f TFLOP/s\n", blocksPerSm, ms, fl / ms / 1e9);
  }
  for (int fw : {8, 0, 4}) {  // all DFMA, all DMMA, half and half (256 threads, one CTA per SM)
    const int grid = sms, threads = 256, itf = 4096, itm = 1024;
    dfma_dmma<<<grid, threads>>>(d, 16, 4, fw); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); dfma_dmma<<<grid, threads>>>(d, itf, itm, fw); cudaEventRecord(e1);
    CK(cudaEventSynchronize(e1)); float ms; cudaEventElapsedTime(&ms, e0, e1);
    const double ff = 2.0 * 8 * itf * 32.0 * fw * grid, fm = 512.0 * 4 * itm * (8 - fw) * (double)grid;
    printf("dfma warps %d + dmma warps %d: %.3f ms  %.3f + %.3f = %.3f TFLOP/s\n", fw, 8 - fw, ms, ff / ms / 1e9,
           fm / ms / 1e9, (ff + fm) / ms / 1e9);
  }
  for (int warps : {4, 8, 16}) {  // warps per SM (one CTA per SM), one dependent chain each
    for (int lanes : {1, 32}) {
      const int grid = sms, threads = 32 * warps, iters = 4096;
      dfma_lanes<<<grid, threads>>>(d, 16, lanes); CK(cudaDeviceSynchronize());
      cudaEventRecord(e0); dfma_lanes<<<grid, threads>>>(d, iters, lanes); cudaEventRecord(e1);
      CK(cudaEventSynchronize(e1)); float ms; cudaEventElapsedTime(&ms, e0, e1);
      printf("dfma chain: %2d warps/SM, %2d active lanes: %.3f ms, %.1f ns per dependent step\n", warps, lanes, ms,
             ms * 1e6 / iters);
    }
  }
  CK(cudaFree(d));
  return 0;
}
