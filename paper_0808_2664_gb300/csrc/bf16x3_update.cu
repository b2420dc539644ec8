// Leaf-block trailing update of CAQR on the 5th-generation tensor cores.
//
// For every leaf i of a panel (n <= 64 reflectors, any height) and a
// 128-column slice of the trailing matrix C (FP32 storage), one CTA computes
//     C_i <- C_i - Y_i (T_i^T (Y_i^T C_i))
// (the leaf phase of Section 3.1's trailing update, Q_i^T in compact-WY
// form).  The two products run on tcgen05.mma (kind::f16, BF16 inputs, FP32
// accumulators in tensor memory).  Each FP32 operand x is split into two
// BF16 terms, hi = bf16(x) and lo = bf16(x - hi), and every product is
// formed as hi*hi + hi*lo + lo*hi ("3xBF16"); the dropped lo*lo term and the
// split residuals leave about 2^-16 relative error per product.
//   1. W^T = C^T Y   M = 128 (columns of C), N = n_pad, K = h in 64-row chunks
//   2. W'^T = W^T T  FP32 on the CUDA cores, one column of C per thread
//   3. D = Y W'      M = 128 rows per tile, N = 128, K = n_pad
//   4. C -= D        epilogue from tensor memory, coalesced stores
// Operands are staged by the CTA's threads into shared memory in the
// no-swizzle K-major core-matrix layout (8 rows x 16 bytes per core matrix);
// one thread issues the MMAs, tcgen05.commit signals an mbarrier, and every
// wait on that mbarrier gives up after a bounded number of polls (latching
// the status word's timeout bit) so the kernel can never hang; tensor memory
// is always released before the CTA exits.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "tsqr_internal.cuh"

namespace tsqr {
namespace {

constexpr int kUN = 128;       // columns of C per CTA (MMA M of step 1, N of step 3)
constexpr int kUThreads = 256; // eight warps; warps w and w+4 share TMEM lane quarter w % 4
constexpr int kUNp = 64;       // reflector count padded to the MMA N / K granularity
constexpr int kTmemCols = 256; // D1 at columns [0, 64), D2 at [64, 192)
constexpr long long kPollLimit = 1ll << 24;

// Shared-memory matrix descriptor (no swizzle): start address, leading byte
// offset (between K-adjacent core matrices), stride byte offset (between
// 8-row groups), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

// Polls the mbarrier for the given phase parity; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (long long i = 0; i < kPollLimit; ++i) {
    uint32_t done = 0;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// One more expected arrival carrying `bytes` of asynchronous copies.
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// 2-D tiled copy global -> shared through the tensor-memory-access engine;
// c0 is the innermost (row) coordinate, completion counted on mbar.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(mbar)
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

struct Bf16x3Args {
  const float* Y;  // factored panel storage: leaf reflectors
  int64_t ldy;
  int64_t m;
  int n;
  int64_t h;
  int64_t nleaves;
  const float* Tw;  // nleaves x (n x n)
  float* C;
  int64_t ldc;
  int64_t k;
  int* status;
  int vec;  // 16-byte loads allowed (C, Y, ldc, ldy, h aligned)
};

// The two split-product forms.  Each FP32 operand x is split into a high
// and a low term of the MMA input type and every product is formed as
// hi*hi + hi*lo + lo*hi:
//   three BF16 products (kind::f16, BF16 A and B): about 2^-16 relative
//   error per product;
//   three TF32 products (kind::tf32): about 2^-21 from the split, below the
//   floor of the tensor cores' FP32 accumulation (about 2^-19 measured).
// Both input types have 16-byte core-matrix rows (8 BF16 or 4 TF32) and 32
// bytes of K per MMA instruction (16 BF16 or 8 TF32), so the descriptors and
// K steps are the same; TF32 tiles take twice the bytes, so its step-1 chunks
// are 32 rows and its step-3 tiles reuse the step-1 region.
// Shared memory map (bytes from a 1024-aligned base): step 1's operand tiles
// are double-buffered ([buffer][hi | lo]) so the next chunk is staged while
// the tensor cores work on the current one; then step 3's Y row tile and W'.
template <bool kTF32>
struct Split3 {
  static constexpr uint32_t ES = kTF32 ? 4 : 2;    // bytes per element
  static constexpr uint32_t EPR = 16 / ES;          // elements per 16-byte core-matrix row
  static constexpr uint32_t KI = kTF32 ? 8 : 16;    // K per MMA instruction
  static constexpr int CHUNK = kTF32 ? 32 : 64;     // leaf rows per step-1 chunk
  static constexpr uint32_t SzA1 = kUN * CHUNK * ES;  // C^T chunk, one term
  static constexpr uint32_t SzB1 = kUNp * CHUNK * ES; // Y chunk, one term
  static constexpr uint32_t SzA3 = 128 * kUNp * ES;   // Y row tile, one term
  static constexpr uint32_t SzB3 = kUN * kUNp * ES;   // W', one term
  static constexpr uint32_t OffA1 = 0;
  static constexpr uint32_t OffB1 = OffA1 + 4 * SzA1;
  static constexpr uint32_t End1 = OffB1 + 4 * SzB1;
  // Raw FP32 chunks of C (CHUNK rows x kUN columns) and Y (CHUNK x kUNp),
  // written by the tensor-memory-access engine, two buffers.
  static constexpr uint32_t RawC = (uint32_t)CHUNK * kUN * 4;
  static constexpr uint32_t RawY = (uint32_t)CHUNK * kUNp * 4;
  static constexpr uint32_t OffRaw = End1;
  static constexpr uint32_t EndRaw = OffRaw + 2 * (RawC + RawY);
  // Step 3's tiles reuse finished step-1 storage: the raw buffers (BF16) or
  // the split tiles and raw buffers (TF32).
  static constexpr uint32_t OffA3 = kTF32 ? 0 : OffRaw;
  static constexpr uint32_t OffB3 = OffA3 + 2 * SzA3;
  static constexpr uint32_t End3 = OffB3 + 2 * SzB3;
  static constexpr uint32_t OffT = EndRaw > End3 ? EndRaw : End3;  // T: 64 x 64 FP32
  // MMA mbarrier (8 B), TMEM address (4 B), two chunk mbarriers (8 B each).
  static constexpr uint32_t OffBar = OffT + kUNp * kUNp * 4;
  static_assert(OffBar + 64 + 1024 <= 227 * 1024, "shared memory of the split-product update");
  static constexpr uint32_t SmemBytes = OffBar + 64 + 1024;    // + alignment slack

  // Byte offset of element (r, k) in a K-major no-swizzle tile with R rows:
  // core matrices of 8 rows x 16 bytes (128 contiguous bytes), R/8 of them
  // per K slab of EPR elements, K slabs one after another.
  static __device__ __forceinline__ uint32_t kmaj(int r, int k, int R) {
    return (uint32_t)(((((uint32_t)k / EPR) * (R >> 3) + (r >> 3)) << 7) + ((r & 7) << 4) + ((uint32_t)k % EPR) * ES);
  }

  // Instruction descriptor: FP32 D; A and B BF16 (1) or TF32 (2); both K-major.
  static __host__ __device__ constexpr uint32_t idesc(int M, int N) {
    return (1u << 4) | ((kTF32 ? 2u : 1u) << 7) | ((kTF32 ? 2u : 1u) << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
  }

  static __device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                             uint32_t accumulate) {
    if constexpr (kTF32) {
      asm volatile(
          "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
          "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
          "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
    } else {
      asm volatile(
          "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
          "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
          "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
    }
  }

  // TF32 rounding of x (round to nearest, ties away), as an FP32 bit pattern.
  static __device__ __forceinline__ uint32_t tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
  }

  // hi and lo terms of one value at byte offset off.
  static __device__ __forceinline__ void store1(unsigned char* hi_base, unsigned char* lo_base, uint32_t off,
                                                float x) {
    if constexpr (kTF32) {
      const uint32_t h = tf32(x);
      const uint32_t l = tf32(x - __uint_as_float(h));
      *reinterpret_cast<uint32_t*>(hi_base + off) = h;
      *reinterpret_cast<uint32_t*>(lo_base + off) = l;
    } else {
      const __nv_bfloat16 h = __float2bfloat16_rn(x);
      const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
      *reinterpret_cast<__nv_bfloat16*>(hi_base + off) = h;
      *reinterpret_cast<__nv_bfloat16*>(lo_base + off) = l;
    }
  }

  // Four consecutive K elements x[0..3] at byte offset off (4 ES-aligned).
  static __device__ __forceinline__ void store4(unsigned char* hi_base, unsigned char* lo_base, uint32_t off,
                                                const float* x) {
    if constexpr (kTF32) {
      uint4 h, l;
      h.x = tf32(x[0]);
      h.y = tf32(x[1]);
      h.z = tf32(x[2]);
      h.w = tf32(x[3]);
      l.x = tf32(x[0] - __uint_as_float(h.x));
      l.y = tf32(x[1] - __uint_as_float(h.y));
      l.z = tf32(x[2] - __uint_as_float(h.z));
      l.w = tf32(x[3] - __uint_as_float(h.w));
      *reinterpret_cast<uint4*>(hi_base + off) = h;
      *reinterpret_cast<uint4*>(lo_base + off) = l;
    } else {
      __nv_bfloat16 h[4], l[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        h[e] = __float2bfloat16_rn(x[e]);
        l[e] = __float2bfloat16_rn(x[e] - __bfloat162float(h[e]));
      }
      *reinterpret_cast<uint2*>(hi_base + off) = *reinterpret_cast<const uint2*>(h);
      *reinterpret_cast<uint2*>(lo_base + off) = *reinterpret_cast<const uint2*>(l);
    }
  }
};

// kTMA: step 1's C and Y chunks arrive through cp.async.bulk.tensor (tmC,
// tmY: maps of C and Y with boxes of CHUNK rows), two chunks ahead of the one
// being converted; otherwise each thread loads its share of the chunk.
template <bool kTF32, bool kTMA>
__global__ void __launch_bounds__(kUThreads, 1)
    split3_update_kernel(Bf16x3Args a, const __grid_constant__ CUtensorMap tmC, const __grid_constant__ CUtensorMap tmY) {
  using S3 = Split3<kTF32>;
  constexpr int kUChunk = S3::CHUNK;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(sm);
  const int tid = threadIdx.x;
  const int quarter = (tid >> 5) & 3;  // TMEM lane quarter this warp may access
  const int half = tid >> 7;           // 0: threads 0..127, 1: threads 128..255
  const int n = a.n;
  const int64_t leaf = blockIdx.x;
  const int64_t k0 = (int64_t)blockIdx.y * kUN;
  const int kc = (int)((a.k - k0) < kUN ? (a.k - k0) : kUN);
  const int64_t r0 = leaf * a.h;
  const int hl = (leaf == a.nleaves - 1) ? (int)(a.m - r0) : (int)a.h;
  const float* Yg = a.Y + r0;
  float* Cg = a.C + r0 + k0 * a.ldc;
  float* Ts = reinterpret_cast<float*>(sm + S3::OffT);
  const uint32_t mbar = sbase + S3::OffBar;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + S3::OffBar + 8);
  const uint32_t mraw = sbase + S3::OffBar + 16;  // chunk buffer b: mraw + 8 b

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    if (kTMA) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mraw) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mraw + 8) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sbase + S3::OffBar + 8),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // T of this leaf, zero-padded to 64 x 64.
  const float* Tg = a.Tw + leaf * (int64_t)n * n;
  for (int idx = tid; idx < kUNp * kUNp; idx += kUThreads) {
    const int p = idx % kUNp, q = idx / kUNp;
    Ts[idx] = (p < n && q < n) ? Tg[p + q * n] : 0.f;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t d1 = tmem, d2 = tmem + kUNp;
  uint32_t commits = 0, waited = 0;  // tcgen05.commit k completes mbarrier phase k
  bool ok = true;
  // Every wait ends with a CTA-wide agreement on `ok`, so that the threads
  // never take different paths around the barriers that follow.
  auto wait_next = [&]() {
    if (mbar_wait(mbar, waited & 1)) {
      ++waited;
    } else {
      ok = false;
      atomicOr(a.status, kStatusTimeout);
    }
    ok = __syncthreads_and(ok) != 0;
  };
  // Raw chunk buffers: copies issued / waited for per buffer (the same on
  // every thread).
  uint32_t raw_issued[2] = {0u, 0u}, raw_done[2] = {0u, 0u};
  auto issue_raw = [&](int ch) {
    const int b = ch & 1;
    if (tid == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(mraw + 8 * b, S3::RawC + S3::RawY);
      const uint32_t dst = sbase + S3::OffRaw + (uint32_t)b * (S3::RawC + S3::RawY);
      const int row = (int)(r0 + (int64_t)ch * kUChunk);
      tma_load_2d(dst, &tmC, row, (int)k0, mraw + 8 * b);
      tma_load_2d(dst + S3::RawC, &tmY, row, 0, mraw + 8 * b);
    }
    ++raw_issued[b];
  };
  // Four rows r..r+3 of column col of a column-major FP32 matrix (rows
  // beyond hl are zero): one 16-byte load when aligned and complete.
  auto load4 = [&](const float* base, int64_t ld, int r, int col, float* x) {
    const float* p = base + r + (int64_t)col * ld;
    if (a.vec && r + 3 < hl) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(p));
      x[0] = v.x, x[1] = v.y, x[2] = v.z, x[3] = v.w;
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) x[e] = (r + e < hl) ? p[e] : 0.f;
    }
  };
  auto mask_y = [&](int r, int p, float* x) {  // unit diagonal, zero above, padding beyond n
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int row = r + e;
      if (p >= n || row >= hl || row < p) x[e] = 0.f;
      else if (row == p) x[e] = 1.f;
    }
  };
  auto stage1 = [&](int ch, int buf) {
    const int rb = ch * kUChunk;
    unsigned char* ahi = sm + S3::OffA1 + (2 * buf) * S3::SzA1;
    unsigned char* bhi = sm + S3::OffB1 + (2 * buf) * S3::SzB1;
    constexpr int kCPer = kUN * (kUChunk / 4) / kUThreads, kYPer = kUNp * (kUChunk / 4) / kUThreads;
    if constexpr (kTMA) {
      // The chunk's raw FP32 tiles ([column][row], CHUNK rows per column)
      // are in buffer ch & 1 once its mbarrier phase completes; rows beyond
      // the leaf are zeroed here (they belong to the next leaf, or are the
      // copy's zero fill past the matrix).
      const int b = ch & 1;
      if (mbar_wait(mraw + 8 * b, raw_done[b] & 1)) {
        ++raw_done[b];
      } else {
        ok = false;
        atomicOr(a.status, kStatusTimeout);
      }
      if (!ok) return;
      const float* rc = reinterpret_cast<const float*>(sm + S3::OffRaw + (uint32_t)b * (S3::RawC + S3::RawY));
      const float* ry = rc + S3::RawC / 4;
#pragma unroll
      for (int t = 0; t < kCPer; ++t) {
        const int idx = tid + t * kUThreads;
        const int quad = idx % (kUChunk / 4), c = idx / (kUChunk / 4);
        const float4 v = *reinterpret_cast<const float4*>(rc + c * kUChunk + 4 * quad);
        float x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (rb + 4 * quad + e >= hl) x[e] = 0.f;
        S3::store4(ahi, ahi + S3::SzA1, S3::kmaj(c, 4 * quad, kUN), x);
      }
#pragma unroll
      for (int t = 0; t < kYPer; ++t) {
        const int idx = tid + t * kUThreads;
        const int quad = idx % (kUChunk / 4), p = idx / (kUChunk / 4);
        const float4 v = *reinterpret_cast<const float4*>(ry + p * kUChunk + 4 * quad);
        float x[4] = {v.x, v.y, v.z, v.w};
        mask_y(rb + 4 * quad, p, x);
        S3::store4(bhi, bhi + S3::SzB1, S3::kmaj(p, 4 * quad, kUNp), x);
      }
    } else {
    // All of this thread's global loads for the chunk are issued before any
    // of them is converted, so that their latencies overlap.
    float xc[kCPer][4], xy[kYPer][4];
#pragma unroll
    for (int t = 0; t < kCPer; ++t) {
      const int idx = tid + t * kUThreads;
      const int quad = idx % (kUChunk / 4), c = idx / (kUChunk / 4);
#pragma unroll
      for (int e = 0; e < 4; ++e) xc[t][e] = 0.f;
      if (c < kc) load4(Cg, a.ldc, rb + 4 * quad, c, xc[t]);
    }
#pragma unroll
    for (int t = 0; t < kYPer; ++t) {
      const int idx = tid + t * kUThreads;
      const int quad = idx % (kUChunk / 4), p = idx / (kUChunk / 4);
#pragma unroll
      for (int e = 0; e < 4; ++e) xy[t][e] = 0.f;
      if (p < n) load4(Yg, a.ldy, rb + 4 * quad, p, xy[t]);
    }
#pragma unroll
    for (int t = 0; t < kCPer; ++t) {
      const int idx = tid + t * kUThreads;
      const int quad = idx % (kUChunk / 4), c = idx / (kUChunk / 4);
      S3::store4(ahi, ahi + S3::SzA1, S3::kmaj(c, 4 * quad, kUN), xc[t]);
    }
#pragma unroll
    for (int t = 0; t < kYPer; ++t) {
      const int idx = tid + t * kUThreads;
      const int quad = idx % (kUChunk / 4), p = idx / (kUChunk / 4);
      mask_y(rb + 4 * quad, p, xy[t]);
      S3::store4(bhi, bhi + S3::SzB1, S3::kmaj(p, 4 * quad, kUNp), xy[t]);
    }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  };
  auto issue1 = [&](int ch, int buf) {
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      constexpr uint32_t id1 = S3::idesc(kUN, kUNp);
      const uint32_t A = sbase + S3::OffA1 + (2 * buf) * S3::SzA1, B = sbase + S3::OffB1 + (2 * buf) * S3::SzB1;
#pragma unroll
      for (int s = 0; s < kUChunk / (int)S3::KI; ++s) {
        const uint32_t aoff = (uint32_t)s * kUN * 32, boff = (uint32_t)s * kUNp * 32;
        const uint64_t ahi = sdesc(A + aoff, kUN * 16, 128), alo = sdesc(A + S3::SzA1 + aoff, kUN * 16, 128);
        const uint64_t bhi = sdesc(B + boff, kUNp * 16, 128), blo = sdesc(B + S3::SzB1 + boff, kUNp * 16, 128);
        S3::mma(d1, ahi, bhi, id1, (ch > 0 || s > 0) ? 1u : 0u);
        S3::mma(d1, ahi, blo, id1, 1u);
        S3::mma(d1, alo, bhi, id1, 1u);
      }
      mma_commit(mbar);
    }
    ++commits;
  };

  // ---- Step 1: W^T = C^T Y over the leaf rows, kUChunk rows per chunk; chunk
  // ch+1 is staged while the MMAs of chunk ch run (and, with kTMA, the raw
  // tiles of chunks ch+1 and ch+2 are in flight meanwhile).
  const int nchunks = (hl + kUChunk - 1) / kUChunk;
  if constexpr (kTMA) {
    issue_raw(0);
    if (nchunks > 1) issue_raw(1);
  }
  stage1(0, 0);
  ok = __syncthreads_and(ok) != 0;
  if (ok) {
    if constexpr (kTMA)
      if (nchunks > 2) issue_raw(2);  // raw buffer 0 is converted
    issue1(0, 0);
  }
  for (int ch = 1; ch < nchunks && ok; ++ch) {
    stage1(ch, ch & 1);  // buffer ch&1 was read by chunk ch-2, already complete
    ok = __syncthreads_and(ok) != 0;
    if (!ok) break;
    if constexpr (kTMA)
      if (ch + 2 < nchunks) issue_raw(ch + 2);  // raw buffer ch&1 is converted
    wait_next();  // chunk ch-1 done
    if (!ok) break;
    issue1(ch, ch & 1);
  }
  if (ok) wait_next();  // last chunk done
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();

  // ---- Step 2: W'^T(c, :) = W^T(c, :) T.  Thread (half, c): column c of C,
  // W' columns q in [32 half, 32 half + 32).
  if (ok) {
    const int c = tid & (kUN - 1);
    float w[kUNp];
#pragma unroll
    for (int q = 0; q < kUNp; q += 16) tmem_ld16(d1 + ((uint32_t)(quarter * 32) << 16) + q, w + q);
    float wp[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) wp[q] = 0.f;
    if (half == 0) {
#pragma unroll
      for (int p = 0; p < 32; ++p)
#pragma unroll
        for (int q = p; q < 32; ++q) wp[q] = fmaf(w[p], Ts[p + q * kUNp], wp[q]);
    } else {
#pragma unroll
      for (int p = 0; p < kUNp; ++p)
#pragma unroll
        for (int q = 0; q < 32; ++q)
          if (p <= q + 32) wp[q] = fmaf(w[p], Ts[p + (q + 32) * kUNp], wp[q]);
    }
#pragma unroll
    for (int q = 0; q < 32; q += 4)
      S3::store4(sm + S3::OffB3, sm + S3::OffB3 + S3::SzB3, S3::kmaj(c, 32 * half + q, kUN), wp + q);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();

  // ---- Steps 3-4: D = Y W' per 128-row tile, then C -= D.
  const int ntiles = (hl + 127) / 128;
  for (int t = 0; t < ntiles && ok; ++t) {
    const int rt = t * 128;
    {
      constexpr int kPer = 32 * kUNp / kUThreads;
      float xt[kPer][4];
#pragma unroll
      for (int t = 0; t < kPer; ++t) {
        const int idx = tid + t * kUThreads;
        const int quad = idx % 32, p = idx / 32;
#pragma unroll
        for (int e = 0; e < 4; ++e) xt[t][e] = 0.f;
        if (p < n) load4(Yg, a.ldy, rt + 4 * quad, p, xt[t]);
      }
#pragma unroll
      for (int t = 0; t < kPer; ++t) {
        const int idx = tid + t * kUThreads;
        const int quad = idx % 32, p = idx / 32;
        mask_y(rt + 4 * quad, p, xt[t]);
#pragma unroll
        for (int e = 0; e < 4; ++e)
          S3::store1(sm + S3::OffA3, sm + S3::OffA3 + S3::SzA3, S3::kmaj(4 * quad + e, p, 128), xt[t][e]);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      constexpr uint32_t id3 = S3::idesc(128, kUN);
#pragma unroll
      for (int s = 0; s < kUNp / (int)S3::KI; ++s) {
        const uint32_t aoff = (uint32_t)s * 128 * 32, boff = (uint32_t)s * kUN * 32;
        const uint64_t ahi = sdesc(sbase + S3::OffA3 + aoff, 128 * 16, 128);
        const uint64_t alo = sdesc(sbase + S3::OffA3 + S3::SzA3 + aoff, 128 * 16, 128);
        const uint64_t bhi = sdesc(sbase + S3::OffB3 + boff, kUN * 16, 128);
        const uint64_t blo = sdesc(sbase + S3::OffB3 + S3::SzB3 + boff, kUN * 16, 128);
        S3::mma(d2, ahi, bhi, id3, s > 0 ? 1u : 0u);
        S3::mma(d2, ahi, blo, id3, 1u);
        S3::mma(d2, alo, bhi, id3, 1u);
      }
      mma_commit(mbar);
    }
    ++commits;
    wait_next();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
      const int row = rt + (tid & 127);  // TMEM lane = row of this tile
#pragma unroll 1
      for (int c0 = 64 * half; c0 < 64 * half + 64; c0 += 16) {
        float d[16];
        tmem_ld16(d2 + ((uint32_t)(quarter * 32) << 16) + c0, d);
        if (row < hl) {
          // All sixteen loads before any store: the compiler cannot tell
          // that the columns' addresses differ, and would otherwise wait
          // out one read-modify-write of C before the next.
          float cv[16];
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int c = c0 + e;
            cv[e] = c < kc ? Cg[row + (int64_t)c * a.ldc] : 0.f;
          }
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int c = c0 + e;
            if (c < kc) Cg[row + (int64_t)c * a.ldc] = cv[e] - d[e];
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  if (!ok && waited < commits) {
    // A commit's phase did not complete in time: give the in-flight MMAs one
    // more bounded wait before tensor memory is released.
    mbar_wait(mbar, waited & 1);
  }
  if constexpr (kTMA) {
    // Copies still in flight after a failed wait land in this CTA's shared
    // memory: wait for them (bounded) before the CTA exits.
#pragma unroll
    for (int b = 0; b < 2; ++b)
      while (raw_done[b] < raw_issued[b]) {
        mbar_wait(mraw + 8 * b, raw_done[b] & 1);
        ++raw_done[b];
      }
  }
  __syncthreads();
  if (tid < 32) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

}  // namespace

// cuTensorMapEncodeTiled from the driver, through the runtime (no link
// against the driver library); null if unavailable.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<EncodeTiledFn>(f);
  }();
  return fn;
}

// Tensor map of a column-major FP32 matrix (rows x cols, leading dimension
// ld elements) with boxes of box_rows x box_cols; reads past the matrix
// return zeros.
static bool make_map(CUtensorMap* map, const float* base, int64_t rows, int64_t cols, int64_t ld, uint32_t box_rows,
                     uint32_t box_cols) {
  const EncodeTiledFn f = encode_tiled();
  if (!f) return false;
  const cuuint64_t gdim[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
  const cuuint64_t gstride[1] = {(cuuint64_t)ld * sizeof(float)};
  const cuuint32_t box[2] = {box_rows, box_cols};
  const cuuint32_t estride[2] = {1, 1};
  return f(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), gdim, gstride, box, estride,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <bool kTF32, bool kTMA>
static cudaError_t launch_split3(const Bf16x3Args& a, const CUtensorMap& tmC, const CUtensorMap& tmY, dim3 grid,
                                 cudaStream_t s) {
  constexpr uint32_t smem = Split3<kTF32>::SmemBytes;
  cudaError_t e = cudaFuncSetAttribute(split3_update_kernel<kTF32, kTMA>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  split3_update_kernel<kTF32, kTMA><<<grid, kUThreads, smem, s>>>(a, tmC, tmY);
  return cudaGetLastError();
}

cudaError_t launch_leaf_update_split3(const LeafApplyArgs<float>& la, bool tf32, int* status, cudaStream_t s) {
  if (la.nleaves <= 0 || la.k <= 0 || la.n <= 0) return cudaSuccess;
  if (la.n > kBf16x3MaxN) return cudaErrorInvalidValue;
  Bf16x3Args a;
  a.Y = la.Y;
  a.ldy = la.ldy;
  a.m = la.m;
  a.n = la.n;
  a.h = la.h;
  a.nleaves = la.nleaves;
  a.Tw = la.Tw;
  a.C = la.C;
  a.ldc = la.ldc;
  a.k = la.k;
  a.status = status;
  a.vec = ((uintptr_t)la.C % 16 == 0 && (uintptr_t)la.Y % 16 == 0 && la.ldc % 4 == 0 && la.ldy % 4 == 0 &&
           la.h % 4 == 0)
              ? 1
              : 0;
  const int64_t kchunks = (la.k + kUN - 1) / kUN;
  if (kchunks > 65535 || la.nleaves > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  dim3 grid((unsigned)la.nleaves, (unsigned)kchunks);
  // The copy engine path needs 16-byte aligned bases and leading dimensions
  // and row coordinates (leaf starts, chunk starts) that are multiples of 4:
  // exactly the conditions of the 16-byte thread loads (a.vec).  Rows stay
  // below 2^31 so that the signed copy coordinates hold them.
  CUtensorMap tmC, tmY;
  std::memset(&tmC, 0, sizeof(tmC));
  std::memset(&tmY, 0, sizeof(tmY));
  const uint32_t chunk = tf32 ? Split3<true>::CHUNK : Split3<false>::CHUNK;
  const bool tma = a.vec && la.m < (int64_t(1) << 31) && la.k < (int64_t(1) << 31) &&
                   make_map(&tmC, la.C, la.m, la.k, la.ldc, chunk, kUN) &&
                   make_map(&tmY, la.Y, la.m, la.n, la.ldy, chunk, kUNp);
  if (tf32)
    return tma ? launch_split3<true, true>(a, tmC, tmY, grid, s) : launch_split3<true, false>(a, tmC, tmY, grid, s);
  return tma ? launch_split3<false, true>(a, tmC, tmY, grid, s) : launch_split3<false, false>(a, tmC, tmY, grid, s);
}

}  // namespace tsqr
