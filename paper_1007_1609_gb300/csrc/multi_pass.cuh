// multi_pass.cuh -- one pass of K Chebyshev steps (Eq. 15) over a column slab
// held in HBM, for real on-site lattices with open edges along y (FP32).
// Shared by the single-lattice kernel (step_multi.cu) and the ensemble's
// persistent kernel (ensemble.cu).
//
// With (P, Q) = (j_{n-1}, j_n) of one slab ([2N][W], electron rows then hole
// rows per lattice row), the pass computes j_{n+1} ... j_{n+K} and leaves
// (j_{n+K-1}, j_{n+K}) in (P, Q); per thread it accumulates the three column
// sums of every level (|j|^2, <j_{n+t+1}|j_{n+t}>, sum (u'v - v'u)) for its
// VEC columns.  The CTA sweeps a wavefront g = 0 .. Ly + K - 2: level t
// (1..K) computes lattice row g - t + 1 of j_{n+t} from rows r-1, r, r+1 of
// level t-1 (level 0 = Q, staged by TMA) and row r of level t-2 (level -1 =
// P).  A thread's (x, column quad) is fixed, so the rows it needs at its own
// x are rows it computed itself: they stay in registers (a three-row window
// per level, the loop unrolled by three so that window indices are
// compile-time constants); only x +- 1 neighbours pass through shared memory,
// where each level keeps its two most recent rows.  Level t at wavefront g
// reads neighbour rows written at wavefront g - 1, so one CTA barrier per
// wavefront orders everything.  Only P and Q are read from HBM and only
// levels K-1 and K are written back: 4 vector streams per K steps instead of
// 3 per step.  Rows -1 and Ly do not exist (open edges), which is what makes
// the single wavefront possible.
//
// LVOUT: the levels go to vectors of their own instead of (P, Q), which are
// then only read; level t may add a one-element source per column at its
// start site (PassSource) -- the adjoint's forward, recomputed and reverse
// recursions, whose kernel forms no column sums.
//
// BLOCKED (with LVOUT): the CTA owns a block of lattice rows instead of all
// of them and recomputes K - t halo rows of level t on either side, so
// blocks need no exchange; the sums and outputs cover its own rows only.
//
// Staging: TMA bulk copies on mbarriers; load l (rows l of Q and P and the
// parameters of lattice row l) completes on bars[(base + l) % NB] in phase
// ((base + l) / NB) & 1, so consecutive passes on the same barriers continue
// their phases.  Every wait is bounded; on expiry the pass sets *abort_flag,
// thread 0 lets its copies in flight land (bounded) and the pass returns false.
#pragma once

#include <type_traits>

#include "internal.h"

namespace cbdg {
namespace mp {

__device__ __forceinline__ unsigned smem_addr(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void bulk_load(unsigned dst, const void *src, unsigned bytes, unsigned bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
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
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, unsigned long long limit_ns) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned it = 0;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255u) == 255u && global_ns() - t0 > limit_ns) return false;
  }
}

// Kahan accumulation of a1*b1 + a2*b2 with the products and the compensation
// fused into two FMAs (the same arithmetic as the one-step kernel).
struct Kahan {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add2(float a1, float b1, float a2, float b2) {
    const float y = __fmaf_rn(a1, b1, __fmaf_rn(a2, b2, -c));
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// ChunkSum: plain FP32 accumulation of a1*b1 + a2*b2 (two FMAs), used by the
// LEAN pass to fit three levels into the registers.  To keep its error
// independent of the lattice height, the pass flushes it every kFlushRows
// wavefronts (flush_sums below): the partials of the 8 lanes of a warp that
// hold the same columns are added pairwise in FP32 and the result goes into
// FP64, so no FP32 sum spans more than 4 kFlushRows + 3 roundings.
struct ChunkSum {
  float s = 0.f;
  __device__ __forceinline__ void add2(float a1, float b1, float a2, float b2) {
    s = __fmaf_rn(a1, b1, __fmaf_rn(a2, b2, s));
  }
};

// No column sums (passes whose moments nobody reads, e.g. the adjoint's
// forward and recomputed recursions).
struct NoSum {
  __device__ __forceinline__ void add2(float, float, float, float) {}
  __device__ __forceinline__ double value() const { return 0.0; }
};

// Per-level outputs of a pass (LVOUT): level t's rows go to p[t - 1] when it
// is set, and P and Q are only read.
struct LevelOut {
  float *p[4];
};

// Wavefronts between two flushes of ChunkSum accumulators: two iterations of
// the pass's three-wavefront loop.  With two sites per thread a chunk holds at
// most 4 kFlushRows FP32 roundings per lane, then three pairwise additions
// across lanes: relative error (4 kFlushRows + 3) 2^-24 = 27 * 2^-24 of
// sum |terms| for every lattice height.
constexpr int kFlushRows = 6;

// FP64 share of a warp's column sums: after each flush, lane l holds the sums
// of entries [base(l), base(l) + PER) of the zero-padded list of K levels x 3
// products x 4 columns of its column quad (l & 3).
template <int K>
struct FlushBank {
  static constexpr int NV = K * 12, NVP = (NV + 7) / 8 * 8, PER = NVP / 8;
  double d[PER];
  __device__ __forceinline__ void clear() {
#pragma unroll
    for (int i = 0; i < PER; ++i) d[i] = 0.0;
  }
  // first list index held by lane l (lane bits 4, 3, 2 pick halves NVP/2, NVP/4, NVP/8)
  __host__ __device__ static constexpr int base(int lane) {
    return ((lane >> 4) & 1) * (NVP / 2) + ((lane >> 3) & 1) * (NVP / 4) + ((lane >> 2) & 1) * (NVP / 8);
  }
};

// One halving stage of the reduce-scatter over lane bit `mask`: the lane with
// the bit set keeps the upper half of v[0 .. 2H) and receives its partner's
// upper half; the other keeps and receives the lower half.  Result in v[0 .. H).
template <int H>
__device__ __forceinline__ void scatter_stage(float *v, int mask, bool hi) {
#pragma unroll
  for (int i = 0; i < H; ++i) {
    const float send = hi ? v[i] : v[H + i];
    const float keep = hi ? v[H + i] : v[i];
    v[i] = __fadd_rn(keep, __shfl_xor_sync(0xffffffffu, send, mask));
  }
}

// Moves every ChunkSum partial of the calling thread into the warp's FP64
// bank and zeroes it.  All 32 lanes of the warp must call it together; lane
// bits 0-1 select the column quad (4 quads per warp), bits 2-4 the x slot.
template <int K>
__device__ __forceinline__ void flush_sums(ChunkSum (&accA)[K][4], ChunkSum (&accB)[K][4],
                                           ChunkSum (&accC)[K][4], FlushBank<K> &bank) {
  using FB = FlushBank<K>;
  float v[FB::NVP];
#pragma unroll
  for (int l = 0; l < K; ++l)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      v[l * 12 + 0 * 4 + j] = accA[l][j].s;
      v[l * 12 + 1 * 4 + j] = accB[l][j].s;
      v[l * 12 + 2 * 4 + j] = accC[l][j].s;
      accA[l][j].s = accB[l][j].s = accC[l][j].s = 0.f;
    }
#pragma unroll
  for (int i = FB::NV; i < FB::NVP; ++i) v[i] = 0.f;
  const int lane = threadIdx.x & 31;
  scatter_stage<FB::NVP / 2>(v, 16, (lane & 16) != 0);
  scatter_stage<FB::NVP / 4>(v, 8, (lane & 8) != 0);
  scatter_stage<FB::NVP / 8>(v, 4, (lane & 4) != 0);
#pragma unroll
  for (int i = 0; i < FB::PER; ++i) bank.d[i] += static_cast<double>(v[i]);
}

__device__ __forceinline__ float fc(const float4 &v, int j) { return reinterpret_cast<const float *>(&v)[j]; }


__device__ __forceinline__ float4 zero4() { return make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ float4 lds4(const float *p) { return *reinterpret_cast<const float4 *>(p); }

constexpr int kPassThreads = 256;

// LEAN: level 0 (j_n) stays in its shared-memory ring instead of a register
// window, one slot longer (RQ = 4 + D: rows g-2 .. g+2+D), and the stencil
// parameters have a short ring of their own (AR = K + 1 rows: g-K+1 .. g+1,
// row g+1 copied during wavefront g on its own barriers).  That frees 16
// registers per site and row, which is what a third level needs at two sites
// per thread, and the shared memory the third level's rows need.
template <int W, int K, int D, int NT = kPassThreads, bool LEAN = false>
struct PassShape {
  static constexpr int VEC = 4, QUADS = W / VEC, XSLOTS = NT / QUADS;
  static constexpr int RQ = LEAN ? 4 + D : 3 + D;  // j_n ring: rows g-1 (g-2 lean) .. g+2+D
  static constexpr int RP = 3 + D;                 // j_{n-1} ring: rows g-1 .. g+2+D
  static constexpr int RS = RQ;
  static constexpr int AS = LEAN ? 0 : K + 2 + D;  // parameter ring: rows g-K+1 .. g+2+D
  static constexpr int AR = LEAN ? K + 1 : 0;      // LEAN parameter ring: rows g-K+1 .. g+1
  static constexpr int NB = RQ + AR;               // mbarriers (one per staged row in flight)
  // floats of shared memory the pass uses
  static __host__ __device__ size_t smem_floats(int Lx) {
    const size_t rowel = static_cast<size_t>(2) * Lx * W, pel = static_cast<size_t>(Lx) * kParamStride;
    return (RQ + RP + 2 * (K - 1)) * rowel + (AS + AR) * pel;
  }
};

template <int W, int K, int D, int MAXX, int NT = kPassThreads, bool LEAN = false, typename Acc = Kahan,
          bool LVOUT = false, bool BLOCKED = false>
__device__ __forceinline__ bool multi_pass(float *P, float *Q, const float *__restrict__ par, int Lx, int Ly,
                                           float *smem, unsigned long long *bars, long long base,
                                           unsigned long long wait_ns, unsigned stall_tx, int *abort_flag,
                                           Acc (&accA)[K][4], Acc (&accB)[K][4], Acc (&accC)[K][4],
                                           FlushBank<K> *bank = nullptr, LevelOut lo = LevelOut{},
                                           const PassSource *src = nullptr, int col0 = 0, int rb = 0,
                                           int re = -1) {
  static_assert(K <= 4, "LevelOut holds four levels");
  static_assert(!BLOCKED || LVOUT, "a row block writes its levels out of place");
  using Sh = PassShape<W, K, D, NT, LEAN>;
  constexpr bool kFlush = std::is_same<Acc, ChunkSum>::value;
  static_assert(!kFlush || W / 4 == 4, "the chunk flush expects four column quads per warp");
  constexpr int VEC = Sh::VEC, QUADS = Sh::QUADS, XSLOTS = Sh::XSLOTS;
  constexpr int RQ = Sh::RQ, RP = Sh::RP, AS = Sh::AS, AR = Sh::AR;
  static_assert(W % VEC == 0 && NT % QUADS == 0 && K >= 2, "bad shape");
  const int rowel = 2 * Lx * W;
  const int pel = Lx * kParamStride;
  // BLOCKED: the CTA owns lattice rows [rb, re) and computes level t on them
  // and on K - t halo rows either side (none beyond the lattice edges), which
  // it recomputes instead of exchanging; it loads rows r0 .. r0 + NR - 1, and
  // every row index below is relative to r0.  Otherwise it owns all rows.
  if (!BLOCKED || re < 0) re = Ly;
  if (!BLOCKED) rb = 0;
  const int r0 = BLOCKED ? max(0, rb - K) : 0, NR = BLOCKED ? min(Ly, re + K) - r0 : Ly;
  P += static_cast<size_t>(r0) * rowel;
  Q += static_cast<size_t>(r0) * rowel;
  par += static_cast<size_t>(r0) * pel;
  // rows of level t this CTA computes: [clo(t), chi(t))
  auto clo = [&](int t) { return BLOCKED ? max(0, rb - K + t) - r0 : 0; };
  auto chi = [&](int t) { return BLOCKED ? min(Ly, re + K - t) - r0 : Ly; };
  float *sq = smem;                       // [RQ][rowel]  j_n
  float *sp = sq + RQ * rowel;            // [RP][rowel]  j_{n-1}
  float *sl = sp + RP * rowel;            // [K-1][2][rowel] levels 1..K-1
  float *sa = sl + (K - 1) * 2 * rowel;   // [AS][pel], LEAN: [AR][pel]
  const int t = threadIdx.x;
  const int q = t % QUADS, xs = t / QUADS;
  const unsigned row_bytes = rowel * 4u, par_bytes = pel * 4u;
  auto bar_of = [&](int l) { return smem_addr(&bars[(base + l) % RQ]); };
  auto par_of = [&](int l) { return static_cast<unsigned>(((base + l) / RQ) & 1); };
  // LEAN parameter row l: slot and barrier (base + l) % AR, after the RQ row barriers
  auto pbar_of = [&](int l) { return smem_addr(&bars[RQ + (AR > 0 ? (base + l) % AR : 0)]); };
  auto ppar_of = [&](int l) { return static_cast<unsigned>(AR > 0 ? ((base + l) / AR) & 1 : 0); };

  // load l: rows l of j_n and j_{n-1} and the parameters of lattice row l
  auto issue = [&](int l) {
    const unsigned bar = bar_of(l);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar),
                 "r"(2 * row_bytes + (LEAN ? 0u : par_bytes) + (l == 0 ? stall_tx : 0u))
                 : "memory");
    bulk_load(smem_addr(sq + (l % RQ) * rowel), Q + static_cast<size_t>(l) * rowel, row_bytes, bar);
    bulk_load(smem_addr(sp + (l % RP) * rowel), P + static_cast<size_t>(l) * rowel, row_bytes, bar);
    if constexpr (!LEAN)
      bulk_load(smem_addr(sa + (l % AS) * pel), par + static_cast<size_t>(l) * pel, par_bytes, bar);
  };
  // LEAN: parameter row l, copied into its own ring slot
  auto issue_par = [&](int l) {
    const unsigned bar = pbar_of(l);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(par_bytes) : "memory");
    bulk_load(smem_addr(sa + (AR > 0 ? (base + l) % AR : 0) * pel), par + static_cast<size_t>(l) * pel, par_bytes,
              bar);
  };
  int issued = min(NR, 2 + D);
  int pissued = LEAN ? min(NR, 2) : 0;  // rows 0, 1 before the first wavefront
  if (t == 0) {
    for (int l = 0; l < issued; ++l) issue(l);
    for (int l = 0; l < pissued; ++l) issue_par(l);
  }

  const int hb = Lx * W;
  const int off = q * VEC;
  // LVOUT sources: bit j of smask when column col0 + off + j has its start
  // site at one of this thread's x slots (slot s_k, row s_r)
  int smask = 0, s_k[VEC], s_r[VEC], s_i[VEC];
#pragma unroll
  for (int j = 0; j < VEC; ++j) s_k[j] = s_r[j] = s_i[j] = 0;
  if constexpr (LVOUT) {
    if (src != nullptr && src->sites != nullptr) {
#pragma unroll
      for (int j = 0; j < VEC; ++j) {
        const int c = col0 + off + j;
        if (c < src->ncols) {
          const int i = src->sites[c], rx = i % Lx;
          if (rx % XSLOTS == xs) {
            smask |= 1 << j;
            s_k[j] = rx / XSLOTS;
            s_r[j] = i / Lx - r0;
            s_i[j] = i;
          }
        }
      }
    }
  }
  // adds the level-lv sources of this thread's columns whose start site is
  // (slot k, row r)
  auto add_sources = [&](int lv, int r, int k, float4 &un, float4 &vn) {
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      if (((smask >> j) & 1) && s_r[j] == r && s_k[j] == k) {
        const int i = s_i[j];
        const double wv = (src->w ? src->w[i] : 1.0) * (src->u ? src->u[i] : 1.0);
        const double val =
            wv * (src->scale * src->tab[static_cast<size_t>(src->stride) * (col0 + off + j) + src->m0 + src->dm * lv]);
        float *e = reinterpret_cast<float *>(src->part == 0 ? &un : &vn) + j;
        *e = static_cast<float>(static_cast<double>(*e) + val);
      }
    }
  };
  float4 wu[K][3][MAXX], wv[K][3][MAXX];
#pragma unroll
  for (int l = 0; l < K; ++l)
#pragma unroll
    for (int s = 0; s < 3; ++s)
#pragma unroll
      for (int k = 0; k < MAXX; ++k) wu[l][s][k] = wv[l][s][k] = zero4();

  int waited = 0, pwaited = 0;
  bool ok = true;
  if constexpr (!LEAN) {
    ok = mbar_wait(bar_of(0), par_of(0), wait_ns);
    if (ok) {
      waited = 1;
#pragma unroll
      for (int k = 0; k < MAXX; ++k) {
        const int x = xs + k * XSLOTS;
        if (x < Lx) {
          wu[0][0][k] = lds4(sq + x * W + off);
          wv[0][0][k] = lds4(sq + hb + x * W + off);
        }
      }
    }
  }
  const int G = NR + K - 1;
  bool stop = false;
  // Three wavefronts g0 .. g0 + 2 (window slots are compile-time per phase).
  // INNER: every level's row r and the rows r - 1, r + 1 it reads lie inside
  // [0, Ly), so no edge test and no zero fill; FULL: every x slot of every
  // thread holds a lattice site (Lx = MAXX * XSLOTS), so no x test either.
  auto three_waves = [&](const int g0, auto inner_c, auto full_c) {
    constexpr bool INNER = decltype(inner_c)::value, FULL = decltype(full_c)::value;
#pragma unroll
    for (int ph = 0; ph < 3; ++ph) {
      const int g = g0 + ph;
      if (stop || (!INNER && g >= G)) break;
      // rows up to g + 1 must have landed (LEAN: parameter rows up to g)
      for (; ok && waited <= min(g + 1, NR - 1); ++waited)
        if (!mbar_wait(bar_of(waited), par_of(waited), wait_ns))
          ok = false;
      if constexpr (LEAN)
        for (; ok && pwaited <= min(g, NR - 1); ++pwaited)
          if (!mbar_wait(pbar_of(pwaited), ppar_of(pwaited), wait_ns))
            ok = false;
      if (!ok) *abort_flag = 1;
      __syncthreads();
      if (*abort_flag) {
        stop = true;
        break;
      }
      // the slots of rows g - 1 (j_{n-1}) and g - 1 (j_n; LEAN: g - 2) are free:
      // every read of them happened before the barrier
      if (g + 2 + D < NR) {
        if (t == 0) issue(g + 2 + D);
        issued = g + 3 + D;
      }
      // LEAN: the parameter slot of row g - K is free (its last reader, level K,
      // ran at wavefront g - 1): parameter row g + 1 goes there
      if constexpr (LEAN) {
        if (g + 1 < NR && g + 1 >= pissued) {
          if (t == 0) issue_par(g + 1);
          pissued = g + 2;
        }
      }
      // level 0 "computes" row g + 1: its centre enters the window
      if constexpr (!LEAN) {
#pragma unroll
        for (int k = 0; k < MAXX; ++k) {
          const int x = xs + k * XSLOTS;
          float4 nu = zero4(), nv = zero4();
          if ((FULL || x < Lx) && (INNER || g + 1 < NR)) {
            const float *src = sq + ((g + 1) % RQ) * rowel;
            nu = lds4(src + x * W + off);
            nv = lds4(src + hb + x * W + off);
          }
          wu[0][(ph + 1) % 3][k] = nu;
          wv[0][(ph + 1) % 3][k] = nv;
        }
      }
      // LEAN: level 1's j_n row r - 1 at this x (row g - 1) is level 2's
      // j_n row r at this wavefront; kept from level 1's loads
      float4 q_ud[MAXX], q_vd[MAXX];
#pragma unroll
      for (int lv = 1; lv <= K; ++lv) {
        const int r = g - lv + 1;
        const int sm = (ph - lv + 6) % 3, sc = (ph - lv + 7) % 3, su = (ph - lv + 8) % 3;
        // sums and output rows: the block's own rows only
        const bool own = !BLOCKED || (r0 + r >= rb && r0 + r < re);
        if (INNER || (r >= clo(lv) && r < chi(lv))) {
          const float *nb = lv == 1 ? sq + (r % RQ) * rowel : sl + ((lv - 2) * 2 + (r & 1)) * rowel;
          const float *po = sp + (r % RP) * rowel;
          const float *pc = LEAN ? sa + ((base + r) % (AR > 0 ? AR : 1)) * pel : sa + (r % (AS > 0 ? AS : 1)) * pel;
          float *dl = lv < K ? sl + ((lv - 1) * 2 + (r & 1)) * rowel : nullptr;
#pragma unroll
          for (int k = 0; k < MAXX; ++k) {
            const int x = xs + k * XSLOTS;
            if (FULL || x < Lx) {
              const int xl = (x == 0) ? Lx - 1 : x - 1;
              const int xr = (x == Lx - 1) ? 0 : x + 1;
              float4 u, v, uu, vu, ud, vd;
              if (LEAN && lv == 1) {
                // level 0 rows r - 1, r, r + 1 at this x from the j_n ring (zero beyond the edges)
                const float *rc = sq + (r % RQ) * rowel;
                u = lds4(rc + x * W + off);
                v = lds4(rc + hb + x * W + off);
                if (INNER) {
                  const float *rp = sq + ((r + 1) % RQ) * rowel, *rm = sq + ((r - 1) % RQ) * rowel;
                  uu = lds4(rp + x * W + off);
                  vu = lds4(rp + hb + x * W + off);
                  ud = lds4(rm + x * W + off);
                  vd = lds4(rm + hb + x * W + off);
                  q_ud[k] = ud;
                  q_vd[k] = vd;
                } else {
                  uu = vu = ud = vd = zero4();
                  if (r + 1 < NR) {
                    const float *rp = sq + ((r + 1) % RQ) * rowel;
                    uu = lds4(rp + x * W + off);
                    vu = lds4(rp + hb + x * W + off);
                  }
                  if (r >= 1) {
                    const float *rm = sq + ((r - 1) % RQ) * rowel;
                    ud = lds4(rm + x * W + off);
                    vd = lds4(rm + hb + x * W + off);
                  }
                }
              } else {
                u = wu[lv - 1][sc][k], v = wv[lv - 1][sc][k];
                uu = wu[lv - 1][su][k], vu = wv[lv - 1][su][k];
                ud = wu[lv - 1][sm][k], vd = wv[lv - 1][sm][k];
              }
              const float4 ur = lds4(nb + xr * W + off), vr = lds4(nb + hb + xr * W + off);
              const float4 ul = lds4(nb + xl * W + off), vl = lds4(nb + hb + xl * W + off);
              float4 uo, vo;
              if (lv == 1) {
                uo = lds4(po + x * W + off);
                vo = lds4(po + hb + x * W + off);
              } else if (LEAN && lv == 2) {
                // level 0 row r: interior wavefronts kept it from level 1
                if (INNER) {
                  uo = q_ud[k];
                  vo = q_vd[k];
                } else {
                  const float *rc = sq + (r % RQ) * rowel;
                  uo = lds4(rc + x * W + off);
                  vo = lds4(rc + hb + x * W + off);
                }
              } else {
                uo = wu[lv >= 2 ? lv - 2 : 0][sc][k];
                vo = wv[lv >= 2 ? lv - 2 : 0][sc][k];
              }
              const float4 pa = lds4(pc + x * kParamStride), pb = lds4(pc + x * kParamStride + 4);
              const float e = pa.x, d = pa.y, t0 = pa.z, t1 = pa.w, t2 = pb.x, t3 = pb.y;
              float4 un, vn;
#pragma unroll
              for (int j = 0; j < VEC; ++j) {
                const float uj = fc(u, j), vj = fc(v, j);
                const float unj = __fmaf_rn(e, uj, __fmaf_rn(d, vj, -__fmaf_rn(t3, fc(ud, j), __fmaf_rn(t2, fc(uu, j),
                                      __fmaf_rn(t1, fc(ul, j), __fmaf_rn(t0, fc(ur, j), fc(uo, j)))))));
                const float vnj = __fmaf_rn(d, uj, __fmaf_rn(-e, vj, __fmaf_rn(t3, fc(vd, j), __fmaf_rn(t2, fc(vu, j),
                                      __fmaf_rn(t1, fc(vl, j), __fmaf_rn(t0, fc(vr, j), -fc(vo, j)))))));
                reinterpret_cast<float *>(&un)[j] = unj;
                reinterpret_cast<float *>(&vn)[j] = vnj;
                if (own) {
                  accA[lv - 1][j].add2(uj, uj, vj, vj);
                  accB[lv - 1][j].add2(unj, uj, vnj, vj);
                  accC[lv - 1][j].add2(unj, vj, -vnj, uj);
                }
              }
              if constexpr (LVOUT) {
                if (smask != 0) add_sources(lv, r, k, un, vn);
              }
              if (lv < K) {
                wu[lv < K ? lv : 0][sc][k] = un;
                wv[lv < K ? lv : 0][sc][k] = vn;
                *reinterpret_cast<float4 *>(dl + x * W + off) = un;
                *reinterpret_cast<float4 *>(dl + hb + x * W + off) = vn;
              }
              if constexpr (LVOUT) {
                // every level to its own vector, when given; P and Q are only read
                if (own && lo.p[lv - 1] != nullptr) {
                  float *o = lo.p[lv - 1] + static_cast<size_t>(r0 + r) * rowel;
                  __stcs(reinterpret_cast<float4 *>(o + x * W + off), un);
                  __stcs(reinterpret_cast<float4 *>(o + hb + x * W + off), vn);
                }
              } else if (lv == K - 1) {
                // levels K-1 and K become the new (P, Q); their HBM rows are no longer read
                float *o = P + static_cast<size_t>(r) * rowel;
                __stcs(reinterpret_cast<float4 *>(o + x * W + off), un);
                __stcs(reinterpret_cast<float4 *>(o + hb + x * W + off), vn);
              } else if (lv == K) {
                float *o = Q + static_cast<size_t>(r) * rowel;
                __stcs(reinterpret_cast<float4 *>(o + x * W + off), un);
                __stcs(reinterpret_cast<float4 *>(o + hb + x * W + off), vn);
              }
            }
          }
        } else if (!INNER && lv < K) {
          // rows outside [0, Ly) are zero (open edges); a block's rows beyond
          // its halo are never read
#pragma unroll
          for (int k = 0; k < MAXX; ++k) {
            wu[lv < K ? lv : 0][sc][k] = zero4();
            wv[lv < K ? lv : 0][sc][k] = zero4();
          }
        }
      }
    }
  };
  const bool xfull = Lx == MAXX * XSLOTS;
  for (int g0 = 0; g0 < G && !stop; g0 += 3) {
    // wavefronts K .. NR - 2 (a block: 2K - 1 .. NR - 2): level t's row
    // g - t + 1 is one it computes, its neighbours g - t .. g - t + 2 lie
    // inside the rows computed or loaded, and so does row g + 1 (K = 4 keeps
    // the one checked copy: a second copy of its body spills)
    if (K <= 3 && g0 >= (BLOCKED ? 2 * K - 1 : K) && g0 + 2 <= NR - 2) {
      if constexpr (K <= 3) {
        if (xfull) three_waves(g0, std::true_type{}, std::true_type{});
        else three_waves(g0, std::true_type{}, std::false_type{});
      }
    } else {
      three_waves(g0, std::false_type{}, std::false_type{});
    }
    if constexpr (kFlush) {
      // every lane arrives here (stop and G are uniform over the CTA); the
      // last iteration always flushes, so the bank holds the whole sums
      if (!stop && ((g0 / 3) % (kFlushRows / 3) == kFlushRows / 3 - 1 || g0 + 3 >= G))
        flush_sums<K>(accA, accB, accC, *bank);
    }
  }
  if (*abort_flag) {
    if (t == 0) {
      for (int l = waited; l < issued; ++l)
        if (!mbar_wait(bar_of(l), par_of(l), wait_ns)) break;
      for (int l = pwaited; l < pissued; ++l)
        if (!mbar_wait(pbar_of(l), ppar_of(l), wait_ns)) break;
    }
    return false;
  }
  return true;
}

}  // namespace mp
}  // namespace cbdg
