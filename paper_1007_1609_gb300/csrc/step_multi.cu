// step_multi.cu -- K steps of the Chebyshev recursion of Eq. 15 per pass
// over HBM (temporal blocking) for real on-site (s-wave) lattices with open
// edges along y, FP32 vectors.
//
// With (P, Q) = (j_{n-1}, j_n) in HBM, one launch computes j_{n+1} ... j_{n+K}
// and leaves (j_{n+K-1}, j_{n+K}) in (P, Q), plus the fused column sums of
// every level (the same three products as step.cu).  A CTA owns one column
// slab and all lattice rows and sweeps a wavefront g = 0 .. Ly + K - 2: at
// wavefront g, level t (1..K) computes lattice row r = g - t + 1 of j_{n+t}
// from rows r-1, r, r+1 of level t-1 (level 0 = Q, staged by TMA) and row r
// of level t-2 (level -1 = P), so level t runs one row behind level t-1.
// Only P and Q are read from HBM and only levels K-1 and K are written back:
// 4 vector streams per K steps instead of 3 per step.  Rows -1 and Ly do not
// exist (open edges), which is what makes the single wavefront possible.
//
// The pass itself (register windows, TMA staging, bounded waits) is
// mp::multi_pass in multi_pass.cuh; this file launches it once per slab and
// reduces each level's column sums across the CTA in FP64.
#include <algorithm>
#include <type_traits>

#include "multi_pass.cuh"

namespace cbdg {
namespace {

using mp::Kahan;
constexpr int kThreads = mp::kPassThreads;

// LVOUT: per-level outputs, no column sums (the adjoint).  BLK: row blocks
// of a.rows_per_cta lattice rows with recomputed halos, the last two levels
// written out of place to a.lvout[K - 2], a.lvout[K - 1], column sums per
// block (partials [level][block][3][ld]).
template <int W, int K, int D, int MAXX, bool LEAN, bool LVOUT = false, bool BLK = false>
__global__ void __launch_bounds__(kThreads, LVOUT && !BLK && MAXX == 1 ? 2 : 1) step_multi_kernel(StepArgs a) {
  using Sh = mp::PassShape<W, K, D, kThreads, LEAN>;
  constexpr int VEC = Sh::VEC, XSLOTS = Sh::XSLOTS, NB = Sh::NB;
  // FP32 chunk sums flushed into FP64 need four column quads per warp
  constexpr bool kChunk = LEAN && W / VEC == 4;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long bars[NB];
  __shared__ int abort_flag;
  const int t = threadIdx.x;
  const int q = t % Sh::QUADS, xs = t / Sh::QUADS;
  const int nblk = BLK ? (a.Ly + a.rows_per_cta - 1) / a.rows_per_cta : 1;
  const int sl = static_cast<int>(blockIdx.x) / nblk, blk = static_cast<int>(blockIdx.x) % nblk;
  const size_t slab = static_cast<size_t>(sl) * (static_cast<size_t>(2) * a.Lx * a.Ly * W);
  if (t == 0) {
    for (int k = 0; k < NB; ++k)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mp::smem_addr(&bars[k])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    abort_flag = 0;
  }
  __syncthreads();
  using Acc = typename std::conditional<LVOUT && !BLK, mp::NoSum,
                                        typename std::conditional<kChunk, mp::ChunkSum, Kahan>::type>::type;
  using FB = mp::FlushBank<K>;
  Acc accA[K][VEC], accB[K][VEC], accC[K][VEC];
  FB bank;
  bank.clear();
  mp::LevelOut lo{};
  if constexpr (LVOUT) {
#pragma unroll
    for (int l = 0; l < K; ++l) lo.p[l] = a.lvout[l] ? static_cast<float *>(a.lvout[l]) + slab : nullptr;
  }
  const int rb = blk * a.rows_per_cta, re = min(a.Ly, rb + a.rows_per_cta);
  const bool ok = mp::multi_pass<W, K, D, MAXX, kThreads, LEAN, Acc, LVOUT, BLK>(
      static_cast<float *>(a.prev) + slab, static_cast<float *>(const_cast<void *>(a.cur)) + slab,
      static_cast<const float *>(a.params), a.Lx, a.Ly, reinterpret_cast<float *>(smem_raw), bars, 0,
      a.wait_ns, a.stall_tx, &abort_flag, accA, accB, accC, &bank, lo, &a.src, sl * W, rb, re);
  if (!ok) {
    if (t == 0) atomicOr(a.flags, kFlagTimeout);
    return;
  }
  if constexpr (LVOUT && !BLK) return;
  __syncthreads();
  double *red = reinterpret_cast<double *>(smem_raw);
  const size_t c0 = static_cast<size_t>(sl) * W;
  // level lv's sums of this block: partials[((lv * nblk + blk) * 3 + k) * ld + col]
  auto part_at = [&](int lv, int k) { return a.partials + ((static_cast<size_t>(lv) * nblk + blk) * 3 + k) * a.ld; };
  if constexpr (kChunk) {
    // the pass flushed every sum into the warps' FP64 banks: lane l of warp w
    // holds list entries [base(l), base(l) + PER) of column quad l & 3; add the
    // warps in a fixed order -> part_at(lv, k)[col]
    constexpr int NWARP = kThreads / 32;
    const int lane = t & 31, w = t >> 5;
#pragma unroll
    for (int i = 0; i < FB::PER; ++i) red[(w * 4 + (lane & 3)) * FB::NVP + FB::base(lane) + i] = bank.d[i];
    __syncthreads();
    for (int idx = t; idx < K * 3 * W; idx += kThreads) {
      const int lk = idx / W, col = idx - lk * W;  // lk = lv * 3 + k
      const int lv = lk / 3, k = lk - lv * 3;
      const int qd = col / VEC, j = col - qd * VEC;
      double s = 0.0;
      for (int z = 0; z < NWARP; ++z) s += red[(z * 4 + qd) * FB::NVP + lv * 12 + k * 4 + j];
      part_at(lv, k)[c0 + col] = s;
    }
    return;
  } else {
    // per-level column sums -> part_at(lv, k)[col] (fixed order, FP64)
    for (int lv = 0; lv < K; ++lv) {
#pragma unroll
      for (int j = 0; j < VEC; ++j) {
        red[(0 * XSLOTS + xs) * W + q * VEC + j] = accA[lv][j].value();
        red[(1 * XSLOTS + xs) * W + q * VEC + j] = accB[lv][j].value();
        red[(2 * XSLOTS + xs) * W + q * VEC + j] = accC[lv][j].value();
      }
      __syncthreads();
      for (int idx = t; idx < 3 * W; idx += kThreads) {
        const int k = idx / W, col = idx - k * W;
        double s = 0.0;
        for (int z = 0; z < XSLOTS; ++z) s += red[(k * XSLOTS + z) * W + col];
        part_at(lv, k)[c0 + col] = s;
      }
      __syncthreads();
    }
  }
}

constexpr int kMaxDynSmem = 227 * 1024 - 1024;

template <int W, int K, int D, bool LEAN = false>
size_t smem_bytes(int Lx) {
  const size_t ring = mp::PassShape<W, K, D, kThreads, LEAN>::smem_floats(Lx);
  const size_t red = LEAN && W == 16
                          ? static_cast<size_t>(kThreads / 32) * 4 * mp::FlushBank<K>::NVP * sizeof(double) / sizeof(float)
                          : static_cast<size_t>(3) * (kThreads / (W / 4)) * W * sizeof(double) / sizeof(float);
  return std::max(ring, red) * sizeof(float);
}

template <int W, int K, int D, int MAXX, bool LEAN = false, bool LVOUT = false, bool BLK = false>
cudaError_t launch_one(const StepArgs &a, size_t smem, cudaStream_t s) {
  auto k = step_multi_kernel<W, K, D, MAXX, LEAN, LVOUT, BLK>;
  static int attr_dev = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (attr_dev != dev) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
    if (e != cudaSuccess) return e;
    // the per-level-output kernels at one site per thread fit two CTAs per SM
    e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    attr_dev = dev;
  }
  const int nblk = BLK ? (a.Ly + a.rows_per_cta - 1) / a.rows_per_cta : 1;
  k<<<a.ld / W * nblk, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

// Register windows take 24 x K x MAXX registers and the column sums 24 x K,
// so only these shapes are built: one lattice site per thread for K = 2 .. 4,
// two sites per thread for K = 2 (K = 4 spills a few bytes, the rest none),
// and two sites per thread for K = 3 in the LEAN pass (level 0 read from its
// shared-memory ring, parameters through the read-only cache), at depth 1
// and slab width 16 (its rings fill the shared memory at Lx = 128).
constexpr int max_sites_per_thread(int K) { return K == 2 ? 2 : 1; }
constexpr int kLeanK = 3, kLeanW = 16, kLeanD = 1;

template <int W, int K, int D>
cudaError_t dispatch(const StepArgs &a, cudaStream_t s) {
  const int xsl = kThreads / (W / 4);
  const size_t smem = smem_bytes<W, K, D>(a.Lx);
  if (a.Lx <= xsl) return launch_one<W, K, D, 1>(a, smem, s);
  if constexpr (max_sites_per_thread(K) >= 2) {
    if (a.Lx <= 2 * xsl) return launch_one<W, K, D, 2>(a, smem, s);
  }
  return cudaErrorInvalidValue;
}

// K = 3 at two sites per thread: the LEAN pass
cudaError_t dispatch_lean(const StepArgs &a, cudaStream_t s) {
  constexpr int xsl = kThreads / (kLeanW / 4);
  if (a.Lx <= xsl || a.Lx > 2 * xsl) return cudaErrorInvalidValue;
  return launch_one<kLeanW, kLeanK, kLeanD, 2, true>(a, smem_bytes<kLeanW, kLeanK, kLeanD, true>(a.Lx), s);
}

// Row blocks with recomputed halos, two steps per pass: lattices too wide
// for a whole-column pass (rows of up to 2 x 256 sites at slab width 4, 2 x
// 128 at 8), the parameters in the lean pass's ring, Kahan column sums, the
// new vectors out of place.
template <int W>
size_t smem_blocked(int Lx) {
  return smem_bytes<W, 2, 1, true>(Lx);
}

template <int W>
cudaError_t dispatch_blocked(const StepArgs &a, cudaStream_t s) {
  constexpr int xsl = kThreads / (W / 4);
  if (a.Lx <= xsl) return launch_one<W, 2, 1, 1, true, true, true>(a, smem_blocked<W>(a.Lx), s);
  if (a.Lx <= 2 * xsl) return launch_one<W, 2, 1, 2, true, true, true>(a, smem_blocked<W>(a.Lx), s);
  return cudaErrorInvalidValue;
}

// Per-level outputs and no column sums (the adjoint's forward and recomputed
// recursions): slab width 16 at depth 1, K = 2 or 3.
cudaError_t dispatch_lvout(const StepArgs &a, const StepConfig &cfg, int K, cudaStream_t s) {
  constexpr int xsl = kThreads / 4;
  if (cfg.slab_w != 16 || cfg.depth != 1) return cudaErrorInvalidValue;
  if (K == 3 && a.Lx <= xsl) return launch_one<16, 3, 1, 1, false, true>(a, smem_bytes<16, 3, 1>(a.Lx), s);
  if (K == 3 && a.Lx <= 2 * xsl)
    return launch_one<16, 3, 1, 2, true, true>(a, smem_bytes<16, 3, 1, true>(a.Lx), s);
  if (K == 2 && a.Lx <= xsl) return launch_one<16, 2, 1, 1, false, true>(a, smem_bytes<16, 2, 1>(a.Lx), s);
  if (K == 2 && a.Lx <= 2 * xsl) return launch_one<16, 2, 1, 2, false, true>(a, smem_bytes<16, 2, 1>(a.Lx), s);
  return cudaErrorInvalidValue;
}

template <int W, int K>
size_t smem_for(int D, int Lx) {
  return D == 1 ? smem_bytes<W, K, 1>(Lx) : smem_bytes<W, K, 2>(Lx);
}

size_t smem_lookup(int W, int K, int D, int Lx) {
  if (W == 8) {
    if (K == 2) return smem_for<8, 2>(D, Lx);
    if (K == 3) return smem_for<8, 3>(D, Lx);
    if (K == 4) return smem_for<8, 4>(D, Lx);
  } else if (W == 16) {
    if (K == 2) return smem_for<16, 2>(D, Lx);
    if (K == 3) return smem_for<16, 3>(D, Lx);
    if (K == 4) return smem_for<16, 4>(D, Lx);
  }
  return 0;
}

}  // namespace

bool plan_step_multi(int Lx, int Ly, int ld, int want_w, int want_k, int want_depth,
                     StepConfig *cfg, int *k_out) {
  int W = want_w > 0 ? want_w : 16;
  int K = want_k > 0 ? want_k : 2;
  int D = want_depth > 0 ? std::min(want_depth, 2) : 2;
  if (W == kLeanW && K == kLeanK && Ly >= 2 && ld % W == 0 && Lx > kThreads / (W / 4) &&
      Lx <= 2 * (kThreads / (W / 4)) && (want_depth <= 0 || want_depth == kLeanD)) {
    const size_t b = smem_bytes<kLeanW, kLeanK, kLeanD, true>(Lx);
    if (b > static_cast<size_t>(kMaxDynSmem)) return false;
    cfg->slab_w = W;
    cfg->depth = kLeanD;
    cfg->row_split = 1;
    cfg->threads = kThreads;
    cfg->smem = b;
    *k_out = K;
    return true;
  }
  if ((W != 8 && W != 16) || K < 2 || K > 4 || Ly < 2 || ld % W != 0 ||
      Lx > max_sites_per_thread(K) * (kThreads / (W / 4)))
    return false;
  size_t b = smem_lookup(W, K, D, Lx);
  if (want_depth <= 0 && b > static_cast<size_t>(kMaxDynSmem)) b = smem_lookup(W, K, D = 1, Lx);
  if (b == 0 || b > static_cast<size_t>(kMaxDynSmem)) return false;
  cfg->slab_w = W;
  cfg->depth = D;
  cfg->row_split = 1;
  cfg->threads = kThreads;
  cfg->smem = b;
  *k_out = K;
  return true;
}

bool plan_step_multi_blocked(int Lx, int Ly, int ld, int W, StepConfig *cfg) {
  if ((W != 4 && W != 8) || Ly < 2 || ld % W != 0 || Lx > 2 * (kThreads / (W / 4))) return false;
  const size_t b = W == 4 ? smem_blocked<4>(Lx) : smem_blocked<8>(Lx);
  if (b > static_cast<size_t>(kMaxDynSmem)) return false;
  cfg->slab_w = W;
  cfg->depth = 1;
  cfg->threads = kThreads;
  cfg->smem = b;
  cfg->blocked = 1;
  cfg->row_split = choose_row_split(ld / W, Ly, b, kThreads);
  return true;
}

cudaError_t launch_step_multi(const StepArgs &a, const StepConfig &cfg, int K, cudaStream_t s) {
  if (cfg.blocked) {
    if (K != 2 || a.lvout[0] == nullptr || a.lvout[1] == nullptr) return cudaErrorInvalidValue;
    if (cfg.slab_w == 4) return dispatch_blocked<4>(a, s);
    if (cfg.slab_w == 8) return dispatch_blocked<8>(a, s);
    return cudaErrorInvalidValue;
  }
  if (K >= 2 && K <= 4 && a.lvout[K - 1] != nullptr) return dispatch_lvout(a, cfg, K, s);
  if (cfg.slab_w == kLeanW && K == kLeanK && cfg.depth == kLeanD && a.Lx > kThreads / (kLeanW / 4))
    return dispatch_lean(a, s);
#define CBDG_MULTI_CASE(w, k, d) \
  if (cfg.slab_w == w && K == k && cfg.depth == d) return dispatch<w, k, d>(a, s);
  CBDG_MULTI_CASE(8, 2, 1)
  CBDG_MULTI_CASE(8, 2, 2)
  CBDG_MULTI_CASE(8, 3, 1)
  CBDG_MULTI_CASE(8, 3, 2)
  CBDG_MULTI_CASE(8, 4, 1)
  CBDG_MULTI_CASE(8, 4, 2)
  CBDG_MULTI_CASE(16, 2, 1)
  CBDG_MULTI_CASE(16, 2, 2)
  CBDG_MULTI_CASE(16, 3, 1)
  CBDG_MULTI_CASE(16, 3, 2)
  CBDG_MULTI_CASE(16, 4, 1)
  CBDG_MULTI_CASE(16, 4, 2)
#undef CBDG_MULTI_CASE
  return cudaErrorInvalidValue;
}

}  // namespace cbdg
