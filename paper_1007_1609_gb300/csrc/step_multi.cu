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
// Staging uses TMA bulk copies on mbarriers with bounded waits, as in step.cu.
// Slab-blocked layout, electron rows then hole rows in each lattice row.
#include <algorithm>

#include "internal.h"

namespace cbdg {
namespace {

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

__device__ __forceinline__ float fc(const float4 &v, int j) { return reinterpret_cast<const float *>(&v)[j]; }

constexpr int kThreads = 256;

__device__ __forceinline__ float4 zero4() { return make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ float4 lds4(const float *p) { return *reinterpret_cast<const float4 *>(p); }

// Thread (x, column quad) is fixed for the whole sweep, so the rows a thread
// needs from the level below at its own x (centre, above, below, and the row
// two levels down) are the rows it computed itself: they stay in registers, in
// a three-row window per level (levels 0 .. K-1), indexed by row mod 3.  Only
// the x +- 1 neighbours come from shared memory, where each level keeps its
// two most recent rows.  Level l at wavefront g computes row g - l + 1, whose
// x-neighbour row of level l - 1 was written at wavefront g - 1, so one CTA
// barrier per wavefront orders all shared-memory traffic.  The wavefront loop
// is unrolled by three so that every window index is a compile-time constant.
template <int W, int K, int D, int MAXX>
__global__ void __launch_bounds__(kThreads, 1) step_multi_kernel(StepArgs a) {
  constexpr int VEC = 4, QUADS = W / VEC, XSLOTS = kThreads / QUADS;
  constexpr int RS = 3 + D;      // j_n / j_{n-1} staging ring: rows g-1 .. g+2+D
  constexpr int AS = K + 2 + D;  // parameter ring: rows g-K+1 .. g+2+D
  constexpr int NB = RS;         // one mbarrier per staged row
  static_assert(W % VEC == 0 && kThreads % QUADS == 0 && K >= 2, "bad shape");

  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long bars[NB];
  __shared__ int abort_flag;
  const int Lx = a.Lx, Ly = a.Ly;
  const int rowel = 2 * Lx * W;
  const int pel = Lx * kParamStride;
  float *sq = reinterpret_cast<float *>(smem_raw);  // [RS][rowel]  j_n
  float *sp = sq + RS * rowel;                       // [RS][rowel]  j_{n-1}
  float *sl = sp + RS * rowel;                       // [K-1][2][rowel] levels 1..K-1
  float *sa = sl + (K - 1) * 2 * rowel;              // [AS][pel]

  const int t = threadIdx.x;
  const int q = t % QUADS, xs = t / QUADS;
  const size_t slab = static_cast<size_t>(blockIdx.x) * (static_cast<size_t>(2) * Lx * Ly * W);
  float *P = static_cast<float *>(a.prev) + slab;
  float *Q = static_cast<float *>(const_cast<void *>(a.cur)) + slab;
  const float *par = static_cast<const float *>(a.params);
  const unsigned row_bytes = rowel * 4u, par_bytes = pel * 4u;
  const unsigned long long wait_ns = a.wait_ns;

  if (t == 0) {
    for (int k = 0; k < NB; ++k)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&bars[k])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    abort_flag = 0;
  }
  __syncthreads();

  // load l: rows l of j_n and j_{n-1} and the parameters of lattice row l
  auto issue = [&](int l) {
    const unsigned bar = smem_addr(&bars[l % NB]);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar),
                 "r"(2 * row_bytes + par_bytes + (l == 0 ? a.stall_tx : 0u))
                 : "memory");
    bulk_load(smem_addr(sq + (l % RS) * rowel), Q + static_cast<size_t>(l) * rowel, row_bytes, bar);
    bulk_load(smem_addr(sp + (l % RS) * rowel), P + static_cast<size_t>(l) * rowel, row_bytes, bar);
    bulk_load(smem_addr(sa + (l % AS) * pel), par + static_cast<size_t>(l) * pel, par_bytes, bar);
  };
  int issued = min(Ly, 2 + D);
  if (t == 0)
    for (int l = 0; l < issued; ++l) issue(l);

  const int hb = Lx * W;
  const int off = q * VEC;
  float4 wu[K][3][MAXX], wv[K][3][MAXX];
#pragma unroll
  for (int l = 0; l < K; ++l)
#pragma unroll
    for (int s = 0; s < 3; ++s)
#pragma unroll
      for (int k = 0; k < MAXX; ++k) wu[l][s][k] = wv[l][s][k] = zero4();
  Kahan accA[K][VEC], accB[K][VEC], accC[K][VEC];

  int waited = 0;
  bool ok = mbar_wait(smem_addr(&bars[0]), 0u, wait_ns);
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
  const int G = Ly + K - 1;
  bool stop = false;
  for (int g0 = 0; g0 < G && !stop; g0 += 3) {
#pragma unroll
    for (int ph = 0; ph < 3; ++ph) {
      const int g = g0 + ph;
      if (stop || g >= G) break;
      // rows up to g + 1 must have landed
      for (; ok && waited <= min(g + 1, Ly - 1); ++waited)
        if (!mbar_wait(smem_addr(&bars[waited % NB]), static_cast<unsigned>((waited / NB) & 1), wait_ns))
          ok = false;
      if (!ok) abort_flag = 1;
      __syncthreads();
      if (abort_flag) {
        stop = true;
        break;
      }
      // the slot of row g - 1 is free: every read of it happened before the barrier
      if (g + 2 + D < Ly) {
        if (t == 0) issue(g + 2 + D);
        issued = g + 3 + D;
      }
      // level 0 "computes" row g + 1: its centre enters the window
#pragma unroll
      for (int k = 0; k < MAXX; ++k) {
        const int x = xs + k * XSLOTS;
        float4 nu = zero4(), nv = zero4();
        if (x < Lx && g + 1 < Ly) {
          const float *src = sq + ((g + 1) % RS) * rowel;
          nu = lds4(src + x * W + off);
          nv = lds4(src + hb + x * W + off);
        }
        wu[0][(ph + 1) % 3][k] = nu;
        wv[0][(ph + 1) % 3][k] = nv;
      }
#pragma unroll
      for (int lv = 1; lv <= K; ++lv) {
        const int r = g - lv + 1;
        const int sm = (ph - lv + 6) % 3, sc = (ph - lv + 7) % 3, su = (ph - lv + 8) % 3;
        if (r >= 0 && r < Ly) {
          const float *nb = lv == 1 ? sq + (r % RS) * rowel : sl + ((lv - 2) * 2 + (r & 1)) * rowel;
          const float *po = sp + (r % RS) * rowel;
          const float *pc = sa + (r % AS) * pel;
          float *dl = lv < K ? sl + ((lv - 1) * 2 + (r & 1)) * rowel : nullptr;
#pragma unroll
          for (int k = 0; k < MAXX; ++k) {
            const int x = xs + k * XSLOTS;
            if (x < Lx) {
              const int xl = (x == 0) ? Lx - 1 : x - 1;
              const int xr = (x == Lx - 1) ? 0 : x + 1;
              const float4 u = wu[lv - 1][sc][k], v = wv[lv - 1][sc][k];
              const float4 uu = wu[lv - 1][su][k], vu = wv[lv - 1][su][k];
              const float4 ud = wu[lv - 1][sm][k], vd = wv[lv - 1][sm][k];
              const float4 ur = lds4(nb + xr * W + off), vr = lds4(nb + hb + xr * W + off);
              const float4 ul = lds4(nb + xl * W + off), vl = lds4(nb + hb + xl * W + off);
              float4 uo, vo;
              if (lv == 1) {
                uo = lds4(po + x * W + off);
                vo = lds4(po + hb + x * W + off);
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
                accA[lv - 1][j].add2(uj, uj, vj, vj);
                accB[lv - 1][j].add2(unj, uj, vnj, vj);
                accC[lv - 1][j].add2(unj, vj, -vnj, uj);
              }
              if (lv < K) {
                wu[lv < K ? lv : 0][sc][k] = un;
                wv[lv < K ? lv : 0][sc][k] = vn;
                *reinterpret_cast<float4 *>(dl + x * W + off) = un;
                *reinterpret_cast<float4 *>(dl + hb + x * W + off) = vn;
              }
              // levels K-1 and K become the new (P, Q); their HBM rows are no longer read
              if (lv == K - 1) {
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
        } else if (lv < K) {
          // rows outside [0, Ly) are zero (open edges)
#pragma unroll
          for (int k = 0; k < MAXX; ++k) {
            wu[lv < K ? lv : 0][sc][k] = zero4();
            wv[lv < K ? lv : 0][sc][k] = zero4();
          }
        }
      }
    }
  }
  if (abort_flag) {
    if (t == 0) {
      atomicOr(a.flags, kFlagTimeout);
      for (int l = waited; l < issued; ++l)
        if (!mbar_wait(smem_addr(&bars[l % NB]), static_cast<unsigned>((l / NB) & 1), wait_ns)) break;
    }
    return;
  }
  __syncthreads();
  // per-level column sums -> partials[(lv * 3 + k) * ld + col] (fixed order, FP64)
  double *red = reinterpret_cast<double *>(smem_raw);
  const size_t c0 = static_cast<size_t>(blockIdx.x) * W;
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
      a.partials[(static_cast<size_t>(lv) * 3 + k) * a.ld + c0 + col] = s;
    }
    __syncthreads();
  }
}

constexpr int kMaxDynSmem = 227 * 1024 - 1024;

template <int W, int K, int D>
size_t smem_bytes(int Lx) {
  const size_t rowel = static_cast<size_t>(2) * Lx * W;
  const size_t pel = static_cast<size_t>(Lx) * kParamStride;
  const size_t ring = (2 * (3 + D) + 2 * (K - 1)) * rowel + (K + 2 + D) * pel;
  const size_t red = static_cast<size_t>(3) * (kThreads / (W / 4)) * W * sizeof(double) / sizeof(float);
  return std::max(ring, red) * sizeof(float);
}

template <int W, int K, int D, int MAXX>
cudaError_t launch_one(const StepArgs &a, size_t smem, cudaStream_t s) {
  auto k = step_multi_kernel<W, K, D, MAXX>;
  static int attr_dev = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (attr_dev != dev) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
    if (e != cudaSuccess) return e;
    attr_dev = dev;
  }
  k<<<a.ld / W, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

// Register windows take 24 x K x MAXX registers and the column sums 24 x K,
// so only these shapes are built: one lattice site per thread for K = 2 .. 4,
// two sites per thread for K = 2 (K = 4 spills a few bytes, the rest none).
constexpr int max_sites_per_thread(int K) { return K == 2 ? 2 : 1; }

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

cudaError_t launch_step_multi(const StepArgs &a, const StepConfig &cfg, int K, cudaStream_t s) {
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
