// contract.cu -- dense contraction D[m][n] = sum_k A[m][k] * B[n][k] on the
// 5th-generation tensor cores (tcgen05, kind::tf32), used for the LDOS of
// Eq. 17: LDOS[site][E] = sum_n mu_n(site) W[E][n].
//
// Accuracy: each operand is split into a TF32 head and a TF32 tail
// (x = hi + lo, both rounded to nearest); D accumulates hi*hi + hi*lo + lo*hi
// ("3xTF32"), which carries about 21 significant bits per product.  The split
// is done once per operand element, into hi / lo planes [rows][kp] in HBM
// (kp = k rounded up to 32, zero padded), by an HBM-bound pass.
//
// Pipeline (persistent: one CTA per SM walks the 128 x 256 tiles of D, 10 warps):
//   warp 0   TMA producer: per K-block of 16 (64-byte rows) four 2-D tensor
//            copies (A_hi, A_lo 128 rows; B_hi, B_lo 256 rows) with 64-byte
//            swizzle into a 4-stage ring (48 KB per stage), on full[s];
//   warp 1   MMA issuer (one thread): 2 k-steps x 3 products of
//            tcgen05.mma M = 128, N = 256, K = 8 per K-block into a 256-column
//            FP32 accumulator in tensor memory; tcgen05.commit frees the stage.
//            The tensor cores accumulate in FP32 with truncation, so every
//            16 K-blocks (256 terms, "a group") the MMAs switch to the other
//            of two accumulators (512 columns in all);
//   warps 2-9 drain: each warp reads 128 columns of the 32 lanes its id
//            selects (tcgen05.ld), adds them (FP32, round to nearest) to a
//            running sum held in its registers and releases the accumulator,
//            while the tensor cores already fill the other one; after the last
//            group the running sums go to D.
// Tiles are numbered N-tile fastest and CTA c takes tiles c, c + gridDim.x,
// ..., so the CTAs that share an A tile run together and the second read of
// it hits L2; a CTA's copies and MMAs for its next tile start while its
// drain warps still write the previous tile out.
// Every wait is bounded and also gives up when another role has given up;
// on expiry the CTA records an error bit, waits (bounded) for the copies and
// tensor-core work it issued, frees its tensor memory and returns.
#include <cuda.h>
#include <math.h>

#include <algorithm>
#include <mutex>

#include "internal.h"

namespace cbdg {
namespace {

constexpr int kBM = 128;          // rows of A per tile = tensor-memory lanes
constexpr int kBN = 256;          // rows of B per tile = accumulator columns
constexpr int kBK = 16;           // FP32 elements per K-block row (= the swizzle span: 16 -> 64 B, 8 -> 32 B)
constexpr int kRowBytes = kBK * 4;
constexpr int kStages = kBK == 16 ? 4 : 9;   // as many stages as the shared memory holds
constexpr int kGroupBlocks = 256 / kBK;      // K-blocks per FP32 accumulation group (256 terms)
constexpr unsigned kSwizzleMode = kBK == 16 ? 4u : 6u;  // descriptor layout: 64-byte or 32-byte swizzle
static_assert(kBK == 16 || kBK == 8, "K-block rows of 64 or 32 bytes");
constexpr int kThreads = 320;
constexpr int kDrainThreads = 256;
constexpr unsigned kTmemCols = 512;  // two 256-column accumulators
constexpr unsigned kATile = kBM * kRowBytes;
constexpr unsigned kBTile = kBN * kRowBytes;
constexpr unsigned kStageBytes = 2 * kATile + 2 * kBTile;
constexpr size_t kSmem = 1024 + static_cast<size_t>(kStages) * kStageBytes;
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
// Bounded wait: false after kWaitNs, or as soon as another role has set *abort.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, volatile int *abort) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned it = 0;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255u) == 255u && (*abort || global_ns() - t0 > kWaitNs)) return false;
  }
}
// Bounded wait used while tearing down (no early exit on abort).
__device__ __forceinline__ bool mbar_wait_drain(unsigned bar, unsigned parity) {
  const unsigned long long t0 = global_ns();
  for (unsigned it = 0;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255u) == 255u && global_ns() - t0 > kWaitNs) return false;
  }
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tma_load_2d(unsigned dst, const CUtensorMap *map, int x, int y, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_commit(unsigned bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
               : "memory");
}

// Shared-memory matrix descriptor of a K-major, swizzled operand tile as TMA
// writes it (rows of kRowBytes, 8-row swizzle atoms of 8 * kRowBytes):
// start address >> 4 (bits 0-13), leading-dimension byte offset >> 4
// (bits 16-29; unused by swizzled K-major layouts, set to 1), stride byte
// offset >> 4 between 8-row groups (bits 32-45), descriptor version 1
// (bits 46-47), base offset 0, swizzle mode in bits 61-63 (4 = 64 bytes,
// 6 = 32 bytes).
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr) {
  unsigned long long d = 0;
  d |= static_cast<unsigned long long>((addr & 0x3FFFFu) >> 4);
  d |= static_cast<unsigned long long>(1u) << 16;
  d |= static_cast<unsigned long long>((8u * kRowBytes) >> 4) << 32;
  d |= static_cast<unsigned long long>(1u) << 46;
  d |= static_cast<unsigned long long>(kSwizzleMode) << 61;
  return d;
}

// Instruction descriptor, kind::tf32: FP32 accumulator (bits 4-5 = 1), A and
// B TF32 (bits 7-9 = 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 in
// bits 17-22, M >> 4 in bits 24-28.
constexpr unsigned kIdesc = (1u << 4) | (2u << 7) | (2u << 10) |
                            (static_cast<unsigned>(kBN >> 3) << 17) |
                            (static_cast<unsigned>(kBM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(unsigned tmem, unsigned long long a, unsigned long long b,
                                         unsigned accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

// 32 consecutive FP32 columns of this thread's lane.
__device__ __forceinline__ void tmem_ld32(unsigned taddr, float *v) {
  unsigned r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__global__ void __launch_bounds__(kThreads, 1)
    contract_kernel(const __grid_constant__ CUtensorMap tm_ahi, const __grid_constant__ CUtensorMap tm_alo,
                    const __grid_constant__ CUtensorMap tm_bhi, const __grid_constant__ CUtensorMap tm_blo,
                    float *__restrict__ D, int ldd, int m, int n, int kblocks, int tiles, unsigned *flags) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  __shared__ __align__(8) unsigned long long full_bar[kStages], empty_bar[kStages];
  __shared__ __align__(8) unsigned long long accf_bar[2], acce_bar[2], done_bar;
  __shared__ unsigned tmem_slot;
  __shared__ volatile int abort_flag;

  const int t = threadIdx.x;
  const int warp = t >> 5, lane = t & 31;
  const int n_tiles = (n + kBN - 1) / kBN;
  const int groups = (kblocks + kGroupBlocks - 1) / kGroupBlocks;

  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (t == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(smem_addr(&full_bar[s]), 1);
      mbar_init(smem_addr(&empty_bar[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_addr(&accf_bar[b]), 1);
      mbar_init(smem_addr(&acce_bar[b]), kDrainThreads);
    }
    mbar_init(smem_addr(&done_bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    abort_flag = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = tmem_slot;
  // The CTA walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ...; the
  // K-blocks of all its tiles form one stream through the stage ring (it)
  // and the accumulation groups one alternation of the two accumulators
  // (gg), so the next tile's copies and MMAs start while the drain warps
  // still write the previous tile out.
  long long issued = 0;   // producer: K-blocks whose copies were issued
  bool mma_issued = false;

  if (warp == 0) {
    if (lane == 0) {
      long long it = 0;
      for (int tile = blockIdx.x; tile < tiles && !abort_flag; tile += gridDim.x) {
        const int m0 = (tile / n_tiles) * kBM, n0 = (tile % n_tiles) * kBN;
        for (int kb = 0; kb < kblocks && !abort_flag; ++kb, ++it) {
          const int s = static_cast<int>(it % kStages);
          const unsigned u = static_cast<unsigned>(it / kStages);
          // stage s is free once the MMAs of its previous use completed
          if (!mbar_wait(smem_addr(&empty_bar[s]), (u & 1u) ^ 1u, &abort_flag)) {
            abort_flag = 1;
            break;
          }
          const unsigned bar = smem_addr(&full_bar[s]);
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(kStageBytes)
                       : "memory");
          const unsigned st = smem_addr(base + s * kStageBytes);
          const int x = kb * kBK;
          tma_load_2d(st, &tm_ahi, x, m0, bar);
          tma_load_2d(st + kATile, &tm_alo, x, m0, bar);
          tma_load_2d(st + 2 * kATile, &tm_bhi, x, n0, bar);
          tma_load_2d(st + 2 * kATile + kBTile, &tm_blo, x, n0, bar);
          issued = it + 1;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      long long it = 0, gg = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < tiles && ok && !abort_flag; tile += gridDim.x) {
        int kb = 0;
        for (int g = 0; g < groups && !abort_flag; ++g, ++gg) {
          // accumulator b = gg % 2; the drain of group gg - 2 must have read it
          const int b = static_cast<int>(gg & 1);
          const unsigned acc = tmem + static_cast<unsigned>(b * kBN);
          if (gg >= 2 &&
              !mbar_wait(smem_addr(&acce_bar[b]), static_cast<unsigned>(((gg >> 1) - 1) & 1), &abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const int kend = min(kblocks, (g + 1) * kGroupBlocks);
          for (; kb < kend; ++kb, ++it) {
            const int s = static_cast<int>(it % kStages);
            const unsigned u = static_cast<unsigned>(it / kStages);
            if (!mbar_wait(smem_addr(&full_bar[s]), u & 1u, &abort_flag)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const unsigned st = smem_addr(base + s * kStageBytes);
            const unsigned ah = st, al = st + kATile, bh = st + 2 * kATile, bl = bh + kBTile;
#pragma unroll
            for (int ks = 0; ks < kBK / 8; ++ks) {
              // K = 8 FP32 = 32 bytes per MMA: advance the start address inside the 64-byte row
              const unsigned off = ks * 32;
              const unsigned long long dah = smem_desc(ah + off), dal = smem_desc(al + off);
              const unsigned long long dbh = smem_desc(bh + off), dbl = smem_desc(bl + off);
              mma_tf32(acc, dah, dbh, (kb > g * kGroupBlocks || ks > 0) ? 1u : 0u);
              mma_tf32(acc, dah, dbl, 1u);
              mma_tf32(acc, dal, dbh, 1u);
            }
            mma_issued = true;
            tc_commit(smem_addr(&empty_bar[s]));
          }
          if (!ok) break;
          tc_commit(smem_addr(&accf_bar[b]));
        }
      }
      if (!ok) abort_flag = 1;
    }
  } else {
    // drain: tensor-memory lanes 32 * (warp % 4) ..., columns [128 h, 128 h + 128)
    const int q = warp & 3, h = (warp - 2) >> 2;
    const unsigned lanes = static_cast<unsigned>(q * 32) << 16;
    const bool vec_ok = ((ldd & 3) == 0) && ((reinterpret_cast<uintptr_t>(D) & 15) == 0);
    long long gg = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
      const int m0 = (tile / n_tiles) * kBM, n0 = (tile % n_tiles) * kBN;
      const int row = m0 + q * 32 + lane;
      float sum[128];
#pragma unroll
      for (int j = 0; j < 128; ++j) sum[j] = 0.f;
      for (int g = 0; g < groups; ++g, ++gg) {
        const int b = static_cast<int>(gg & 1);
        // warp-uniform outcome: the tensor-memory loads below are warp-collective
        ok = __all_sync(0xffffffffu, mbar_wait(smem_addr(&accf_bar[b]), static_cast<unsigned>((gg >> 1) & 1),
                                               &abort_flag));
        if (!ok) {
          abort_flag = 1;
          break;
        }
        tc_fence_after();
        const unsigned src = tmem + lanes + static_cast<unsigned>(b * kBN + h * 128);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float v[32];
          tmem_ld32(src + c * 32, v);
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
          for (int j = 0; j < 32; ++j) sum[c * 32 + j] = __fadd_rn(sum[c * 32 + j], v[j]);
        }
        tc_fence_before();
        mbar_arrive(smem_addr(&acce_bar[b]));
      }
      if (ok && row < m) {
        float *drow = D + static_cast<size_t>(row) * ldd;
        const int col0 = n0 + h * 128;
        if (vec_ok && col0 + 128 <= n) {
#pragma unroll
          for (int j = 0; j < 128; j += 4)
            *reinterpret_cast<float4 *>(drow + col0 + j) = make_float4(sum[j], sum[j + 1], sum[j + 2], sum[j + 3]);
        } else {
#pragma unroll
          for (int j = 0; j < 128; ++j)
            if (col0 + j < n) drow[col0 + j] = sum[j];
        }
      }
    }
  }

  // teardown: nothing this CTA issued may still be in flight when it exits
  if (warp == 1 && lane == 0 && mma_issued) {
    tc_commit(smem_addr(&done_bar));
    mbar_wait_drain(smem_addr(&done_bar), 0u);
  }
  if (warp == 0 && lane == 0) {
    for (int s = 0; s < kStages && s < issued; ++s) {
      const long long last_it = s + ((issued - 1 - s) / kStages) * kStages;
      mbar_wait_drain(smem_addr(&full_bar[s]), static_cast<unsigned>((last_it / kStages) & 1));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (t == 0 && abort_flag) atomicOr(flags, kFlagTimeout);
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols)
                 : "memory");
  }
}

// TF32 head (round to nearest) of x and the tail, itself rounded to TF32.
__device__ __forceinline__ float tf32_round(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Four consecutive elements of row r starting at column c (c % 4 == 0);
// zero beyond column k.
__device__ __forceinline__ void load4(const float *p, int c, int k, bool vec, float *x) {
  if (vec && c + 3 < k) {
    const float4 v = *reinterpret_cast<const float4 *>(p + c);
    x[0] = v.x, x[1] = v.y, x[2] = v.z, x[3] = v.w;
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) x[j] = c + j < k ? p[c + j] : 0.f;
  }
}
__device__ __forceinline__ void load4(const double *p, int c, int k, bool vec, double *x) {
  if (vec && c + 3 < k) {
    const double2 a = *reinterpret_cast<const double2 *>(p + c), b = *reinterpret_cast<const double2 *>(p + c + 2);
    x[0] = a.x, x[1] = a.y, x[2] = b.x, x[3] = b.y;
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) x[j] = c + j < k ? p[c + j] : 0.0;
  }
}

// hi / lo planes [rows][kp] of src [rows][ld]; one thread per 4 columns.
template <typename T>
__global__ void split_tf32_kernel(int rows, int k, size_t ld, const T *__restrict__ src, int kp,
                                  float *__restrict__ hi, float *__restrict__ lo) {
  const int q4 = kp / 4;
  const bool vec = (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(src) & 15) == 0);
  const size_t total = static_cast<size_t>(rows) * q4;
  for (size_t idx = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
       idx += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int r = static_cast<int>(idx / q4);
    const int c = static_cast<int>(idx - static_cast<size_t>(r) * q4) * 4;
    T x[4];
    load4(src + static_cast<size_t>(r) * ld, c, k, vec, x);
    float h[4], l[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      h[j] = tf32_round(static_cast<float>(x[j]));
      l[j] = tf32_round(static_cast<float>(x[j] - static_cast<T>(h[j])));
    }
    const size_t o = static_cast<size_t>(r) * kp + c;
    *reinterpret_cast<float4 *>(hi + o) = make_float4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<float4 *>(lo + o) = make_float4(l[0], l[1], l[2], l[3]);
  }
}

// Rate probe of the contraction's tensor-core instruction: one CTA per SM
// issues `mmas` back-to-back tcgen05.mma kind::tf32 (M = 128, N = 256, K = 8,
// the shape and descriptors of contract_kernel) from operand tiles resident
// in shared memory into one FP32 accumulator in tensor memory.  No copies,
// no drain: the time of a launch over its 2 M N K flops per MMA is the peak
// the contraction's roofline is quoted against.  The tiles hold zeros (the
// rate does not depend on the values).  The final wait is bounded; on expiry
// the CTA records kFlagTimeout, waits once more (bounded) and frees its
// tensor memory.
constexpr unsigned kPeakCols = 256;
constexpr size_t kPeakSmem = 120 * 1024;  // more than half an SM's shared memory: one CTA per SM
static_assert(kPeakSmem >= 1024 + static_cast<size_t>(kATile) + kBTile, "probe tiles must fit");

__global__ void __launch_bounds__(128, 1) tf32_peak_kernel(long long mmas, unsigned *flags) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  __shared__ __align__(8) unsigned long long done_bar;
  __shared__ unsigned tmem_slot;
  const int t = threadIdx.x, warp = t >> 5;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"(kPeakCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  for (unsigned i = t * 16u; i < kATile + kBTile; i += 128u * 16u)
    *reinterpret_cast<uint4 *>(base + i) = make_uint4(0u, 0u, 0u, 0u);
  // the tensor cores read shared memory through the async proxy
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  if (t == 0) {
    mbar_init(smem_addr(&done_bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = tmem_slot;
  if (t == 0) {
    const unsigned a = smem_addr(base), b = a + kATile;
    for (long long i = 0; i < mmas; ++i) {
      const unsigned off = static_cast<unsigned>(i & 1) * 32u;  // the two K = 8 halves of a 64-byte row
      mma_tf32(tmem, smem_desc(a + off), smem_desc(b + off), i > 0 ? 1u : 0u);
    }
    tc_commit(smem_addr(&done_bar));
    if (!mbar_wait_drain(smem_addr(&done_bar), 0u)) {
      atomicOr(flags, kFlagTimeout);
      mbar_wait_drain(smem_addr(&done_bar), 0u);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kPeakCols)
                 : "memory");
  }
}

// error word of the stand-alone contraction entry point
static __device__ unsigned g_contract_flag;

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                 CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                 CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  });
  return fn;
}

// 2-D tensor map of a [rows][kp] FP32 plane, box kBK x box_rows, 64-byte
// swizzle, zero fill outside the plane.
bool plane_map(CUtensorMap *map, const float *plane, int rows, int kp, int box_rows) {
  EncodeTiled fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(kp), static_cast<cuuint64_t>(rows)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(kp) * sizeof(float)};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(kBK), static_cast<cuuint32_t>(box_rows)};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(plane), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, kBK == 16 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int grid_for(size_t total) {
  return static_cast<int>(std::min<size_t>((total + 255) / 256, 152 * 16));
}

// Library-owned stream-ordered pool for the split planes of the stand-alone
// entry point: freed blocks stay mapped for the next call (no release at
// synchronisation), and the process-wide default pool is left untouched.
cudaError_t scratch_pool(cudaMemPool_t *out) {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    e = cudaMemPoolCreate(&pools[dev], &props);
    if (e != cudaSuccess) return e;
    unsigned long long keep = ~0ull;
    e = cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) return e;
  }
  *out = pools[dev];
  return cudaSuccess;
}

}  // namespace

cudaError_t contract_flag_address(unsigned **out) {
  void *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_contract_flag);
  *out = static_cast<unsigned *>(p);
  return e;
}

int contract_kp(int k) { return (k + 31) / 32 * 32; }

double tf32_peak_flops_per_mma() { return 2.0 * kBM * kBN * 8; }

cudaError_t launch_tf32_peak(int ctas, long long mmas, unsigned *flags, cudaStream_t s) {
  static int attr_dev = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (attr_dev != dev) {
    cudaError_t e = cudaFuncSetAttribute(tf32_peak_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kPeakSmem));
    if (e != cudaSuccess) return e;
    attr_dev = dev;
  }
  tf32_peak_kernel<<<ctas, 128, kPeakSmem, s>>>(mmas, flags);
  return cudaGetLastError();
}

cudaError_t launch_split_tf32(const float *src, size_t ld, int rows, int k, int kp, float *hi, float *lo,
                              cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  split_tf32_kernel<float><<<grid_for(static_cast<size_t>(rows) * kp / 4), 256, 0, s>>>(rows, k, ld, src, kp, hi, lo);
  return cudaGetLastError();
}

cudaError_t launch_split_tf32_f64(const double *src, size_t ld, int rows, int k, int kp, float *hi,
                                  float *lo, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  split_tf32_kernel<double><<<grid_for(static_cast<size_t>(rows) * kp / 4), 256, 0, s>>>(rows, k, ld, src, kp, hi, lo);
  return cudaGetLastError();
}

cudaError_t launch_contract_planes(const float *a_hi, const float *a_lo, const float *b_hi, const float *b_lo,
                                   int kp, float *D, int ldd, int m, int n, unsigned *flags, cudaStream_t s) {
  if (m <= 0 || n <= 0 || kp <= 0) return cudaSuccess;
  static int attr_dev = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (attr_dev != dev) {
    cudaError_t e = cudaFuncSetAttribute(contract_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kSmem));
    if (e != cudaSuccess) return e;
    attr_dev = dev;
  }
  CUtensorMap ahi, alo, bhi, blo;
  if (!plane_map(&ahi, a_hi, m, kp, kBM) || !plane_map(&alo, a_lo, m, kp, kBM) ||
      !plane_map(&bhi, b_hi, n, kp, kBN) || !plane_map(&blo, b_lo, n, kp, kBN))
    return cudaErrorInvalidValue;
  const long long tiles = static_cast<long long>((n + kBN - 1) / kBN) * ((m + kBM - 1) / kBM);
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  // persistent: one CTA per SM (the stage ring fills the shared memory), each walking every
  // gridDim-th tile
  static int sms_dev = -1, sms = 0;
  if (sms_dev != dev) {
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    sms_dev = dev;
  }
  const unsigned grid = static_cast<unsigned>(std::min<long long>(tiles, std::max(1, sms)));
  contract_kernel<<<grid, kThreads, kSmem, s>>>(ahi, alo, bhi, blo, D, ldd, m, n, kp / kBK, static_cast<int>(tiles),
                                                flags);
  return cudaGetLastError();
}

cudaError_t launch_contract_tf32x3(const float *A, int lda, const float *B, int ldb, float *D,
                                   int ldd, int m, int n, int k, unsigned *flags, cudaStream_t s) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  const int kp = contract_kp(k);
  const size_t a_el = static_cast<size_t>(m) * kp, b_el = static_cast<size_t>(n) * kp;
  cudaMemPool_t pool;
  cudaError_t e = scratch_pool(&pool);
  if (e != cudaSuccess) return e;
  void *ws = nullptr;
  e = cudaMallocFromPoolAsync(&ws, 2 * (a_el + b_el) * sizeof(float), pool, s);
  if (e != cudaSuccess) return e;
  float *a_hi = static_cast<float *>(ws), *a_lo = a_hi + a_el, *b_hi = a_lo + a_el, *b_lo = b_hi + b_el;
  e = launch_split_tf32(A, static_cast<size_t>(lda), m, k, kp, a_hi, a_lo, s);
  if (e == cudaSuccess) e = launch_split_tf32(B, static_cast<size_t>(ldb), n, k, kp, b_hi, b_lo, s);
  if (e == cudaSuccess) e = launch_contract_planes(a_hi, a_lo, b_hi, b_lo, kp, D, ldd, m, n, flags, s);
  cudaError_t f = cudaFreeAsync(ws, s);
  return e != cudaSuccess ? e : f;
}

}  // namespace cbdg
