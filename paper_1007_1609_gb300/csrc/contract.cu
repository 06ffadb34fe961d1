// contract.cu -- dense contraction D[m][n] = sum_k A[m][k] * B[n][k] on the
// 5th-generation tensor cores (tcgen05, kind::tf32), used for the LDOS of
// Eq. 17: LDOS[site][E] = sum_n mu_n(site) W[E][n].
//
// Accuracy: each FP32 operand is split into a TF32 head and a TF32 tail
// (x = hi + lo); D accumulates hi*hi + hi*lo + lo*hi in FP32 in tensor
// memory ("3xTF32"), which carries about 21 significant bits per product.
//
// Tiling: a CTA computes a 128 x 128 tile of D.  Per K-block of 32 (128
// bytes of FP32 per row) the CTA stages A_hi, A_lo, B_hi, B_lo (128 rows
// each) in shared memory in the canonical K-major 128-byte-swizzled layout
// (row r at r*128 bytes, 16-byte chunk c at position c ^ (r & 7), tiles
// 1024-byte aligned); one thread issues 4 k-steps x 3 products of
// tcgen05.mma (M = 128, N = 128, K = 8) into a 128-lane x 128-column FP32
// accumulator in tensor memory and commits to an mbarrier.  The tensor
// cores accumulate in FP32 with truncation, so every 8 K-blocks the
// accumulator is drained with tcgen05.ld (each warp its 32-lane quarter)
// into an FP64 tile in shared memory and restarted: the error of the sum
// then grows with 96 accumulations, not with all K/8 * 3 of them.
// Every wait is bounded; on expiry the CTA records an error bit, still
// waits (bounded) for its tensor-core work and frees its tensor memory.
#include <math.h>

#include "internal.h"

namespace cbdg {
namespace {

constexpr int kTileM = 128;
constexpr int kTileN = 128;
constexpr int kFlushBlocks = 8;  // K-blocks per FP32 accumulation group
constexpr int kBlockK = 32;  // FP32 elements per 128-byte row
constexpr int kThreads = 128;
constexpr unsigned kTmemCols = 128;
constexpr unsigned long long kWaitNs = 2000000000ull;

__device__ __forceinline__ unsigned smem_addr(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned it = 0;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255u) == 255u && global_ns() - t0 > kWaitNs) return false;
  }
}

// TF32 head of x (round to nearest, ties away) and the tail x - head, itself
// rounded to TF32.
__device__ __forceinline__ float tf32_round(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Shared-memory matrix descriptor of a K-major, 128-byte-swizzled operand
// tile: start address >> 4 (bits 0-13), leading-dimension byte offset >> 4
// (bits 16-29; not used by swizzled K-major layouts, set to 1), stride byte
// offset >> 4 between 8-row groups (bits 32-45, 1024 bytes), descriptor
// version 1 (bits 46-47), base offset 0, swizzle mode 2 = 128 bytes (bits 61-63).
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr) {
  unsigned long long d = 0;
  d |= static_cast<unsigned long long>((addr & 0x3FFFFu) >> 4);
  d |= static_cast<unsigned long long>(1u) << 16;
  d |= static_cast<unsigned long long>(1024u >> 4) << 32;
  d |= static_cast<unsigned long long>(1u) << 46;
  d |= static_cast<unsigned long long>(2u) << 61;
  return d;
}

// Instruction descriptor, kind::tf32: FP32 accumulator (bits 4-5 = 1), A and
// B TF32 (bits 7-9 = 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 in
// bits 17-22, M >> 4 in bits 24-28.
constexpr unsigned kIdesc = (1u << 4) | (2u << 7) | (2u << 10) |
                            (static_cast<unsigned>(kTileN >> 3) << 17) |
                            (static_cast<unsigned>(kTileM >> 4) << 24);

// Stores 4 consecutive FP32 (one 16-byte chunk, K index 4c..4c+3 of row r)
// into a swizzled tile.
__device__ __forceinline__ void put_chunk(unsigned char *tile, int r, int c, float4 v) {
  *reinterpret_cast<float4 *>(tile + r * 128 + ((c ^ (r & 7)) << 4)) = v;
}

__global__ void __launch_bounds__(kThreads, 1)
    contract_kernel(const float *__restrict__ A, int lda, const float *__restrict__ B, int ldb,
                    float *__restrict__ D, int ldd, int m, int n, int k, unsigned *flags) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned tiles: A_hi, A_lo, B_hi, B_lo (16 KB each), then the
  // FP64 accumulator, column-major [kTileN][kTileM] (conflict-free per row)
  unsigned char *base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  unsigned char *a_hi = base;
  unsigned char *a_lo = a_hi + kTileM * 128;
  unsigned char *b_hi = a_lo + kTileM * 128;
  unsigned char *b_lo = b_hi + kTileN * 128;
  double *acc64 = reinterpret_cast<double *>(b_lo + kTileN * 128);
  __shared__ __align__(8) unsigned long long mbar;
  __shared__ unsigned tmem_slot;
  __shared__ int abort_flag;

  const int t = threadIdx.x;
  const int warp = t >> 5, lane = t & 31;
  const int m0 = blockIdx.x * kTileM, n0 = blockIdx.y * kTileN;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    abort_flag = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const unsigned tmem = tmem_slot;
  for (int idx = t; idx < kTileM * kTileN; idx += kThreads) acc64[idx] = 0.0;

  const int kblocks = (k + kBlockK - 1) / kBlockK;
  int committed = 0;
  for (int kb = 0; kb < kblocks; ++kb) {
    const int k0 = kb * kBlockK;
    // stage: each thread fills 16-byte chunks (row r, chunk c) of the four tiles
    for (int idx = t; idx < kTileM * 8; idx += kThreads) {
      const int r = idx >> 3, c = idx & 7;
      const int gm = m0 + r, gk = k0 + 4 * c;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (gm < m) {
        const float *p = A + static_cast<size_t>(gm) * lda + gk;
        if (gk + 3 < k) v = *reinterpret_cast<const float4 *>(p);
        else {
          float tmp[4] = {0.f, 0.f, 0.f, 0.f};
          for (int j = 0; j < 4; ++j)
            if (gk + j < k) tmp[j] = p[j];
          v = make_float4(tmp[0], tmp[1], tmp[2], tmp[3]);
        }
      }
      const float4 h = make_float4(tf32_round(v.x), tf32_round(v.y), tf32_round(v.z), tf32_round(v.w));
      const float4 l = make_float4(tf32_round(v.x - h.x), tf32_round(v.y - h.y),
                                   tf32_round(v.z - h.z), tf32_round(v.w - h.w));
      put_chunk(a_hi, r, c, h);
      put_chunk(a_lo, r, c, l);
    }
    for (int idx = t; idx < kTileN * 8; idx += kThreads) {
      const int r = idx >> 3, c = idx & 7;
      const int gn = n0 + r, gk = k0 + 4 * c;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (gn < n) {
        const float *p = B + static_cast<size_t>(gn) * ldb + gk;
        if (gk + 3 < k) v = *reinterpret_cast<const float4 *>(p);
        else {
          float tmp[4] = {0.f, 0.f, 0.f, 0.f};
          for (int j = 0; j < 4; ++j)
            if (gk + j < k) tmp[j] = p[j];
          v = make_float4(tmp[0], tmp[1], tmp[2], tmp[3]);
        }
      }
      const float4 h = make_float4(tf32_round(v.x), tf32_round(v.y), tf32_round(v.z), tf32_round(v.w));
      const float4 l = make_float4(tf32_round(v.x - h.x), tf32_round(v.y - h.y),
                                   tf32_round(v.z - h.z), tf32_round(v.w - h.w));
      put_chunk(b_hi, r, c, h);
      put_chunk(b_lo, r, c, l);
    }
    // make the generic-proxy stores visible to the tensor cores (async proxy)
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (t == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const unsigned ah = smem_addr(a_hi), al = smem_addr(a_lo);
      const unsigned bh = smem_addr(b_hi), bl = smem_addr(b_lo);
#pragma unroll
      for (int ks = 0; ks < kBlockK / 8; ++ks) {
        // K = 8 FP32 = 32 bytes per MMA: advance the start address inside the swizzle row
        const unsigned off = ks * 32;
        const unsigned long long dah = smem_desc(ah + off), dal = smem_desc(al + off);
        const unsigned long long dbh = smem_desc(bh + off), dbl = smem_desc(bl + off);
        const unsigned acc0 = (kb % kFlushBlocks > 0 || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(dah), "l"(dbh), "r"(kIdesc), "r"(acc0)
            : "memory");
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(dah), "l"(dbl), "r"(kIdesc), "r"(1u)
            : "memory");
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(dal), "l"(dbh), "r"(kIdesc), "r"(1u)
            : "memory");
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              smem_addr(&mbar))
          : "memory");
    }
    committed = kb + 1;
    // the tiles are rewritten next iteration: wait for the tensor cores to finish reading
    if (!mbar_wait(smem_addr(&mbar), static_cast<unsigned>(kb & 1))) abort_flag = 1;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (abort_flag) break;
    if (kb % kFlushBlocks == kFlushBlocks - 1 || kb == kblocks - 1) {
      // drain the FP32 group sum into the FP64 tile (row = warp*32 + lane)
      const int r = warp * 32 + lane;
      for (int c0 = 0; c0 < kTileN; c0 += 16) {
        unsigned v[16];
        const unsigned taddr = tmem + (static_cast<unsigned>(warp * 32) << 16) + static_cast<unsigned>(c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
              "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
              "=r"(v[14]), "=r"(v[15])
            : "r"(taddr)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
        for (int j = 0; j < 16; ++j) acc64[(c0 + j) * kTileM + r] += static_cast<double>(__uint_as_float(v[j]));
      }
      // the next MMA overwrites the accumulator: order the loads before it
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    }
  }

  if (!abort_flag && kblocks > 0) {
    const int row = m0 + warp * 32 + lane;
    if (row < m) {
      float *out = D + static_cast<size_t>(row) * ldd + n0;
      for (int j = 0; j < kTileN && n0 + j < n; ++j)
        out[j] = static_cast<float>(acc64[j * kTileM + warp * 32 + lane]);
    }
  } else if (abort_flag) {
    if (t == 0) {
      atomicOr(flags, kFlagTimeout);
      // let the committed tensor-core work finish (bounded) before freeing
      mbar_wait(smem_addr(&mbar), static_cast<unsigned>((committed - 1) & 1));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols)
                 : "memory");
  }
}

constexpr size_t kSmem = 1024 + static_cast<size_t>(2 * kTileM + 2 * kTileN) * 128 +
                         static_cast<size_t>(kTileM) * kTileN * sizeof(double);

// error word of the stand-alone contraction entry point
static __device__ unsigned g_contract_flag;

}  // namespace

cudaError_t contract_flag_address(unsigned **out) {
  void *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_contract_flag);
  *out = static_cast<unsigned *>(p);
  return e;
}

cudaError_t launch_contract_tf32x3(const float *A, int lda, const float *B, int ldb, float *D,
                                   int ldd, int m, int n, int k, unsigned *flags, cudaStream_t s) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  static int attr_dev = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (attr_dev != dev) {
    cudaError_t e = cudaFuncSetAttribute(contract_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kSmem));
    if (e != cudaSuccess) return e;
    attr_dev = dev;
  }
  dim3 grid((m + kTileM - 1) / kTileM, (n + kTileN - 1) / kTileN);
  contract_kernel<<<grid, kThreads, kSmem, s>>>(A, lda, B, ldb, D, ldd, m, n, k, flags);
  return cudaGetLastError();
}

}  // namespace cbdg
