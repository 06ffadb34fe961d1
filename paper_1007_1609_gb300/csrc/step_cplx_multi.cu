// step_cplx_multi.cu -- two steps of the Chebyshev recursion of Eq. 15 per
// pass over HBM (temporal blocking) for general lattices (complex hoppings
// with Peierls phases, optional next-nearest neighbours, on-site or bond
// pairing), FP32 complex vectors, periodic or open edges.
//
// With (P, Q) = (j_{n-1}, j_n) in HBM, one launch computes j_{n+1} into P and
// j_{n+2} into Q (both in place), so that the moment readouts of the one-step
// path (the column sums of on-site pairing, the gathers of bond pairing and
// of chosen targets) see both new vectors.  HBM moves 4 vectors per 2 steps
// instead of 6.  A CTA owns one column slab and all lattice rows and sweeps
// a wavefront g = -1 .. Ly + 1:
//   level 1 computes row g of j_{n+1} for g = -1 .. Ly (rows -1 and Ly are
//           ghosts, the periodic images of rows Ly - 1 and 0, needed by
//           level 2 and never written);
//   level 2 computes row g - 2 of j_{n+2} from level-1 rows g - 3 .. g - 1,
//           all finished before the barrier that opens wavefront g.
// Warps 0-3 compute level 1 and warps 4-7 level 2 (each thread MAXX sites of
// one level, straight-line code the compiler can interleave).
// Every lattice row index is taken modulo Ly, as in the one-step kernel: an
// open y edge has zero hopping and bond amplitude across it, so the wrapped
// rows contribute nothing there.  The rows a periodic sweep needs at its end
// (Q rows 0, 1 and P row 0, the images of rows Ly, Ly + 1) are overwritten
// early in the sweep, so they are copied into shared memory first.
//
// Staging: load k (k = 0 .. Ly + 3, thread 0, TMA bulk copies) brings Q row
// k - 2 (rows >= Ly come from the resident copies instead), the parameters
// of row k - 2 (up to row Ly) and P row k - 2 (rows -1 .. Ly - 1), all on
// barrier k % NB.  At wavefront g loads up to g + 3 must have landed; load k's
// Q slot is last read at wavefront k, its parameter slot at k + 1 and its P
// slot at k - 2, which sizes the three rings.  Every wait is bounded; on
// expiry the CTA records kFlagTimeout, lets its copies in flight land
// (bounded) and returns.
#include <algorithm>

#include "cplx_stencil.cuh"

namespace cbdg {
namespace {

using namespace cx;

__device__ __forceinline__ unsigned saddr(const void *p) { return static_cast<unsigned>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ void minit(unsigned bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mexpect(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bload(unsigned dst, const void *src, unsigned bytes, unsigned bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ bool mtry(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mwait(unsigned bar, unsigned parity, unsigned long long limit_ns) {
  if (mtry(bar, parity)) return true;
  const unsigned long long t0 = gtime();
  for (unsigned it = 0;; ++it) {
    if (mtry(bar, parity)) return true;
    if ((it & 255u) == 255u && gtime() - t0 > limit_ns) return false;
  }
}

struct KahanF {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

constexpr int kThreads = 256;
constexpr int kW = 2;   // complex columns per slab: one float4 per site and part
constexpr int kVC = 2;  // complex elements per float4

// ring sizes (rows) at prefetch depth D
template <int D>
struct Rings {
  static constexpr int RQ = 4 + D, RA = 5 + D, RP = 2 + D, R1 = 4, RES = 3, NB = 5 + D;
};

template <int D>
size_t smem_bytes(int Lx) {
  using R = Rings<D>;
  const size_t rowel = static_cast<size_t>(2) * Lx * kW * 2;
  const size_t pel = static_cast<size_t>(Lx) * kCplxParamStride;
  const size_t ring = ((R::RQ + R::RP + R::R1 + R::RES) * rowel + R::RA * pel) * sizeof(float);
  const size_t red = static_cast<size_t>(2) * 4 * (kThreads / 2) * kW * sizeof(double);  // [2][4][XSLOTS][W]
  return std::max(ring, red);
}

template <int MAXX, int D, bool NNN, bool BOND, bool SUMS>
__global__ void __launch_bounds__(kThreads, 1) step_cplx_multi_kernel(StepArgs a) {
  using R = Rings<D>;
  using V = float4;
  constexpr int QUADS = kW / kVC, GROUP = kThreads / 2, XSLOTS = GROUP / QUADS;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long bars[R::NB];
  __shared__ int abort_flag;
  const int Lx = a.Lx, Ly = a.Ly;
  const int rowel = 2 * Lx * kW * 2;
  const int pel = Lx * kCplxParamStride;
  float *sq = reinterpret_cast<float *>(smem_raw);  // [RQ][rowel] Q rows
  float *sp = sq + R::RQ * rowel;                   // [RP][rowel] P rows
  float *s1 = sp + R::RP * rowel;                   // [R1][rowel] level-1 rows
  float *sr = s1 + R::R1 * rowel;                   // [RES][rowel] Q rows 0, 1, P row 0
  float *sa = sr + R::RES * rowel;                  // [RA][pel] parameter rows
  const int t = threadIdx.x;
  const int grp = t / GROUP;  // 0: level 1, 1: level 2 (warp-uniform)
  const int tl = t % GROUP;
  const int q = tl % QUADS, xs = tl / QUADS;
  const size_t slab = static_cast<size_t>(blockIdx.x) * (static_cast<size_t>(2) * Lx * Ly * kW * 2);
  float *Q = static_cast<float *>(const_cast<void *>(a.cur)) + slab;
  float *P = static_cast<float *>(a.prev) + slab;
  const float *par = static_cast<const float *>(a.params);
  const unsigned row_bytes = static_cast<unsigned>(rowel * sizeof(float));
  const unsigned par_bytes = static_cast<unsigned>(pel * sizeof(float));
  const unsigned long long wait_ns = a.wait_ns;
  auto wrap = [&](int y) { return ((y % Ly) + Ly) % Ly; };

  if (t == 0) {
    for (int k = 0; k < R::NB; ++k) minit(saddr(&bars[k]));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    abort_flag = 0;
  }
  __syncthreads();

  const int nloads = Ly + 4;  // k = 0 .. Ly + 3
  auto issue = [&](int k) {
    const int l = k - 2;
    const bool q_in = l < Ly;                 // rows Ly, Ly + 1: the resident copies
    const bool p_in = l >= -1 && l < Ly;      // P rows -1 .. Ly - 1 (Ly: resident)
    const bool a_in = l <= Ly;                // parameter rows -2 .. Ly
    const unsigned bar = saddr(&bars[k % R::NB]);
    unsigned bytes = (q_in ? row_bytes : 0u) + (p_in ? row_bytes : 0u) + (a_in ? par_bytes : 0u);
    if (k == 0) bytes += 3 * row_bytes + a.stall_tx;  // the resident rows ride on load 0
    mexpect(bar, bytes);
    if (k == 0) {
      bload(saddr(sr + 0 * rowel), Q + static_cast<size_t>(0) * rowel, row_bytes, bar);
      bload(saddr(sr + 1 * rowel), Q + static_cast<size_t>(wrap(1)) * rowel, row_bytes, bar);
      bload(saddr(sr + 2 * rowel), P + static_cast<size_t>(0) * rowel, row_bytes, bar);
    }
    if (q_in) bload(saddr(sq + (k % R::RQ) * rowel), Q + static_cast<size_t>(wrap(l)) * rowel, row_bytes, bar);
    if (p_in) bload(saddr(sp + (k % R::RP) * rowel), P + static_cast<size_t>(wrap(l)) * rowel, row_bytes, bar);
    if (a_in) bload(saddr(sa + (k % R::RA) * pel), par + static_cast<size_t>(wrap(l)) * pel, par_bytes, bar);
  };
  // Q row l (l = -2 .. Ly + 1), P row l (-1 .. Ly), parameter row l (-2 .. Ly), level-1 row l (-1 .. Ly)
  auto qrow = [&](int l) -> const float * { return l >= Ly ? sr + (l - Ly) * rowel : sq + ((l + 2) % R::RQ) * rowel; };
  auto prow = [&](int l) -> const float * { return l >= Ly ? sr + 2 * rowel : sp + ((l + 2) % R::RP) * rowel; };
  auto arow = [&](int l) -> const float * { return sa + ((l + 2) % R::RA) * pel; };
  auto row1 = [&](int l) -> float * { return s1 + ((l + 4) % R::R1) * rowel; };

  // loads 0 .. 2 + D before wavefront -1; wavefront g issues g + 3 + D after its
  // barrier, so load g + 3 (needed at g) was issued at g - D: D >= 1
  static_assert(D >= 1, "the pass waits for load g + 3 before it issues loads at wavefront g");
  int issued = min(nloads, 3 + D);
  if (t == 0)
    for (int k = 0; k < issued; ++k) issue(k);
  int waited = 0;
  bool ok = true;
  KahanF accA[kVC], accB[kVC], accCr[kVC], accCi[kVC];  // this group's level
  const int hb = Lx * kW * 2;
  const int off = q * kVC * 2;

  for (int g = -1; g <= Ly + 1; ++g) {
    // loads up to g + 3 must have landed
    const int need = min(g + 3, nloads - 1);
    for (; ok && waited <= need; ++waited)
      if (!mwait(saddr(&bars[waited % R::NB]), static_cast<unsigned>((waited / R::NB) & 1), wait_ns)) ok = false;
    if (!ok) abort_flag = 1;
    __syncthreads();  // also: level-1 rows of wavefront g - 1 are written, and every read of freed slots is done
    if (abort_flag) break;
    if (g + 3 + D < nloads && g + 3 + D >= issued) {
      if (t == 0) issue(g + 3 + D);
      issued = g + 4 + D;
    }
    auto sums = [&](const V &u, const V &v, const V &un, const V &vn) {
#pragma unroll
      for (int j = 0; j < kVC; ++j) {
        const Cx<float> uj = cget<V, float>(u, j), vj = cget<V, float>(v, j);
        const Cx<float> unj = cget<V, float>(un, j), vnj = cget<V, float>(vn, j);
        accA[j].add(uj.re * uj.re + uj.im * uj.im + vj.re * vj.re + vj.im * vj.im);
        accB[j].add(unj.re * uj.re + unj.im * uj.im + vnj.re * vj.re + vnj.im * vj.im);
        const Cx<float> c = csub(cmul(unj, vj), cmul(vnj, uj));
        accCr[j].add(c.re);
        accCi[j].add(c.im);
      }
    };
    if (grp == 0) {
      // level 1: row g of j_{n+1} from Q rows g-1 .. g+1 and P row g
      if (g <= Ly) {
        const bool real = g >= 0 && g < Ly;
        const float *rm = qrow(g - 1), *rc = qrow(g), *rp = qrow(g + 1), *ro = prow(g);
        const float *py0 = arow(g), *py1 = arow(g - 1);
        float *dst = row1(g);
        float *o = P + static_cast<size_t>(real ? g : 0) * rowel;
#pragma unroll
        for (int k = 0; k < MAXX; ++k) {
          const int x = xs + k * XSLOTS;
          if (x < Lx) {
            const int xl = (x == 0) ? Lx - 1 : x - 1;
            const int xr = (x == Lx - 1) ? 0 : x + 1;
            V u, v, un, vn;
            site_step<float, V, kVC, kW, NNN, BOND, false>(rm, rc, rp, ro, py0, py1, x, xl, xr, off, hb, Lx, u, v,
                                                            un, vn);
            *reinterpret_cast<V *>(dst + x * kW * 2 + off) = un;
            *reinterpret_cast<V *>(dst + hb + x * kW * 2 + off) = vn;
            if (real) {
              __stcs(reinterpret_cast<V *>(o + x * kW * 2 + off), un);
              __stcs(reinterpret_cast<V *>(o + hb + x * kW * 2 + off), vn);
              if (SUMS) sums(u, v, un, vn);
            }
          }
        }
      }
    } else {
      // level 2: row g - 2 of j_{n+2} from level-1 rows g-3 .. g-1 and Q row g-2
      const int r2 = g - 2;
      if (r2 >= 0 && r2 < Ly) {
        const float *rm = row1(r2 - 1), *rc = row1(r2), *rp = row1(r2 + 1), *ro = qrow(r2);
        const float *py0 = arow(r2), *py1 = arow(r2 - 1);
        float *o = Q + static_cast<size_t>(r2) * rowel;
#pragma unroll
        for (int k = 0; k < MAXX; ++k) {
          const int x = xs + k * XSLOTS;
          if (x < Lx) {
            const int xl = (x == 0) ? Lx - 1 : x - 1;
            const int xr = (x == Lx - 1) ? 0 : x + 1;
            V u, v, un, vn;
            site_step<float, V, kVC, kW, NNN, BOND, false>(rm, rc, rp, ro, py0, py1, x, xl, xr, off, hb, Lx, u, v,
                                                            un, vn);
            __stcs(reinterpret_cast<V *>(o + x * kW * 2 + off), un);
            __stcs(reinterpret_cast<V *>(o + hb + x * kW * 2 + off), vn);
            if (SUMS) sums(u, v, un, vn);
          }
        }
      }
    }
  }
  if (abort_flag) {
    if (t == 0) {
      atomicOr(a.flags, kFlagTimeout);
      for (int k = waited; k < issued; ++k)
        if (!mwait(saddr(&bars[k % R::NB]), static_cast<unsigned>((k / R::NB) & 1), wait_ns)) break;
    }
    return;
  }
  if (!SUMS) return;
  __syncthreads();
  // per-level column sums -> partials[(lv * 4 + k) * ld + col] (fixed order, FP64);
  // group lv holds level lv's sums
  double *red = reinterpret_cast<double *>(smem_raw);
  const size_t c0 = static_cast<size_t>(blockIdx.x) * kW;
#pragma unroll
  for (int j = 0; j < kVC; ++j) {
    double *rg = red + static_cast<size_t>(grp) * 4 * XSLOTS * kW;
    rg[(0 * XSLOTS + xs) * kW + q * kVC + j] = accA[j].value();
    rg[(1 * XSLOTS + xs) * kW + q * kVC + j] = accB[j].value();
    rg[(2 * XSLOTS + xs) * kW + q * kVC + j] = accCr[j].value();
    rg[(3 * XSLOTS + xs) * kW + q * kVC + j] = accCi[j].value();
  }
  __syncthreads();
  for (int idx = t; idx < 2 * 4 * kW; idx += kThreads) {
    const int lv = idx / (4 * kW), rem = idx - lv * 4 * kW, k = rem / kW, col = rem - k * kW;
    const double *rg = red + static_cast<size_t>(lv) * 4 * XSLOTS * kW;
    double s = 0.0;
    for (int z = 0; z < XSLOTS; ++z) s += rg[(k * XSLOTS + z) * kW + col];
    a.partials[(static_cast<size_t>(lv) * 4 + k) * a.ld + c0 + col] = s;
  }
}

constexpr int kMaxDynSmem = 227 * 1024 - 1024;

template <int MAXX, int D, bool NNN, bool BOND, bool SUMS>
cudaError_t launch_one(const StepArgs &a, size_t smem, cudaStream_t s) {
  auto k = step_cplx_multi_kernel<MAXX, D, NNN, BOND, SUMS>;
  static int attr_dev = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (attr_dev != dev) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
    if (e != cudaSuccess) return e;
    attr_dev = dev;
  }
  k<<<a.ld / kW, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <int D, bool NNN, bool BOND, bool SUMS>
cudaError_t dispatch_maxx(const StepArgs &a, size_t smem, cudaStream_t s) {
  constexpr int xsl = kThreads / 2 / (kW / kVC);  // threads along x in each level's group
  if (a.Lx <= xsl) return launch_one<1, D, NNN, BOND, SUMS>(a, smem, s);
  if (a.Lx <= 2 * xsl) return launch_one<2, D, NNN, BOND, SUMS>(a, smem, s);
  return cudaErrorInvalidValue;
}

template <int D>
cudaError_t dispatch_kind(const StepArgs &a, size_t smem, int nnn, int bond, cudaStream_t s) {
  if (bond)
    return nnn ? dispatch_maxx<D, true, true, false>(a, smem, s) : dispatch_maxx<D, false, true, false>(a, smem, s);
  return nnn ? dispatch_maxx<D, true, false, true>(a, smem, s) : dispatch_maxx<D, false, false, true>(a, smem, s);
}

}  // namespace

bool plan_step_cplx_multi(int precision, int Lx, int Ly, int ld, StepConfig *cfg) {
  if (precision != 1 || Ly < 3 || Lx < 1 || ld % kW != 0 || Lx > 2 * (kThreads / 2 / (kW / kVC))) return false;
  const int D = 1;
  const size_t b = smem_bytes<1>(Lx);
  if (b > static_cast<size_t>(kMaxDynSmem)) return false;
  cfg->slab_w = kW;
  cfg->depth = D;
  cfg->row_split = 1;
  cfg->threads = kThreads;
  cfg->smem = b;
  return true;
}

cudaError_t launch_step_cplx_multi(int nnn, int bond, const StepArgs &a, const StepConfig &cfg, cudaStream_t s) {
  if (cfg.slab_w != kW || cfg.depth != 1 || a.Ly < 3) return cudaErrorInvalidValue;
  return dispatch_kind<1>(a, cfg.smem, nnn, bond, s);
}

}  // namespace cbdg
