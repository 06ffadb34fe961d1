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
// of level t-2 (level -1 = P), so level t runs one row behind level t-1 and
// all intermediate levels live in three-row shared-memory rings.  Only P and
// Q are read from HBM and only levels K-1 and K are written back: 4 vector
// streams per K steps instead of 3 per step.  Rows -1 and Ly do not exist
// (open edges), which is what makes the single wavefront possible.
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

struct Kahan {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    float y = __fsub_rn(x, c);
    float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

__device__ __forceinline__ float fc(const float4 &v, int j) { return reinterpret_cast<const float *>(&v)[j]; }

constexpr int kThreads = 256;

template <int W, int K, int D, int MAXX>
__global__ void __launch_bounds__(kThreads, 1) step_multi_kernel(StepArgs a) {
  constexpr int VEC = 4, QUADS = W / VEC, XSLOTS = kThreads / QUADS;
  constexpr int QS = 4 + D;       // Q (level 0) ring: rows g-1 .. g+2+D
  constexpr int PS = 3 + D;       // P (level -1) ring: rows g .. g+2+D
  constexpr int AS = K + 2 + D;   // parameter ring: rows g-K+1 .. g+2+D
  constexpr int NB = AS;          // one mbarrier per load slot (loads are issued per row)
  static_assert(W % VEC == 0 && kThreads % QUADS == 0 && K >= 2, "bad shape");

  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long bars[NB];
  __shared__ int abort_flag;
  const int Lx = a.Lx, Ly = a.Ly;
  const int rowel = 2 * Lx * W;
  const int pel = Lx * kParamStride;
  float *sq = reinterpret_cast<float *>(smem_raw);  // [QS][rowel]
  float *spv = sq + QS * rowel;                      // [PS][rowel]
  float *sr = spv + PS * rowel;                      // [K-1][3][rowel] levels 1..K-1
  float *sa = sr + (K - 1) * 3 * rowel;              // [AS][pel]

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

  // load l: Q, P and parameters of lattice row l (0 <= l < Ly), on bars[l % NB]
  auto issue = [&](int l) {
    const unsigned bar = smem_addr(&bars[l % NB]);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar),
                 "r"(2 * row_bytes + par_bytes + (l == 0 ? a.stall_tx : 0u))
                 : "memory");
    bulk_load(smem_addr(sq + (l % QS) * rowel), Q + static_cast<size_t>(l) * rowel, row_bytes, bar);
    bulk_load(smem_addr(spv + (l % PS) * rowel), P + static_cast<size_t>(l) * rowel, row_bytes, bar);
    bulk_load(smem_addr(sa + (l % AS) * pel), par + static_cast<size_t>(l) * pel, par_bytes, bar);
  };
  int issued = min(Ly, 2 + D);
  if (t == 0)
    for (int l = 0; l < issued; ++l) issue(l);

  Kahan accA[K][VEC], accB[K][VEC], accC[K][VEC];
  int waited = 0;
  bool ok = true;
  const int hb = Lx * W;
  const int off = q * VEC;
  auto row_ptr = [&](int level, int r) -> const float * {  // level >= 0, 0 <= r < Ly
    if (level == 0) return sq + (r % QS) * rowel;
    return sr + ((level - 1) * 3 + (r % 3)) * rowel;
  };

  for (int g = 0; g < Ly + K - 1; ++g) {
    // slots of loads <= g-2 (Q) are free after the barrier that ended wavefront g-1
    if (g + 2 + D < Ly) {
      if (t == 0) issue(g + 2 + D);
      issued = g + 3 + D;
    }
    // rows up to g + 1 must have landed
    for (; ok && waited <= min(g + 1, Ly - 1); ++waited)
      if (!mbar_wait(smem_addr(&bars[waited % NB]), static_cast<unsigned>((waited / NB) & 1), wait_ns)) ok = false;
    if (!ok) abort_flag = 1;
    __syncthreads();
    if (abort_flag) break;
#pragma unroll
    for (int lv = 1; lv <= K; ++lv) {
      const int r = g - lv + 1;
      if (r >= 0 && r < Ly) {
        const float *in_c = row_ptr(lv - 1, r);
        const float *in_m = r > 0 ? row_ptr(lv - 1, r - 1) : nullptr;
        const float *in_p = r + 1 < Ly ? row_ptr(lv - 1, r + 1) : nullptr;
        const float *old = lv == 1 ? spv + (r % PS) * rowel : row_ptr(lv - 2, r);
        const float *pc = sa + (r % AS) * pel;
        float *dst = lv < K ? sr + ((lv - 1) * 3 + (r % 3)) * rowel : nullptr;
#pragma unroll
        for (int k = 0; k < MAXX; ++k) {
          const int x = xs + k * XSLOTS;
          if (x < Lx) {
            const int xl = (x == 0) ? Lx - 1 : x - 1;
            const int xr = (x == Lx - 1) ? 0 : x + 1;
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 u = *reinterpret_cast<const float4 *>(in_c + x * W + off);
            const float4 v = *reinterpret_cast<const float4 *>(in_c + hb + x * W + off);
            const float4 ur = *reinterpret_cast<const float4 *>(in_c + xr * W + off);
            const float4 vr = *reinterpret_cast<const float4 *>(in_c + hb + xr * W + off);
            const float4 ul = *reinterpret_cast<const float4 *>(in_c + xl * W + off);
            const float4 vl = *reinterpret_cast<const float4 *>(in_c + hb + xl * W + off);
            const float4 uu = in_p ? *reinterpret_cast<const float4 *>(in_p + x * W + off) : z;
            const float4 vu = in_p ? *reinterpret_cast<const float4 *>(in_p + hb + x * W + off) : z;
            const float4 ud = in_m ? *reinterpret_cast<const float4 *>(in_m + x * W + off) : z;
            const float4 vd = in_m ? *reinterpret_cast<const float4 *>(in_m + hb + x * W + off) : z;
            const float4 uo = *reinterpret_cast<const float4 *>(old + x * W + off);
            const float4 vo = *reinterpret_cast<const float4 *>(old + hb + x * W + off);
            const float *pp = pc + x * kParamStride;
            const float e = pp[0], d = pp[1], t0 = pp[2], t1 = pp[3], t2 = pp[4], t3 = pp[5];
            float4 un, vn;
#pragma unroll
            for (int j = 0; j < VEC; ++j) {
              const float uj = fc(u, j), vj = fc(v, j);
              const float hu = e * uj + d * vj -
                               (t0 * fc(ur, j) + t1 * fc(ul, j) + t2 * fc(uu, j) + t3 * fc(ud, j));
              const float hv = d * uj - e * vj +
                               (t0 * fc(vr, j) + t1 * fc(vl, j) + t2 * fc(vu, j) + t3 * fc(vd, j));
              const float unj = hu - fc(uo, j), vnj = hv - fc(vo, j);
              reinterpret_cast<float *>(&un)[j] = unj;
              reinterpret_cast<float *>(&vn)[j] = vnj;
              accA[lv - 1][j].add(uj * uj + vj * vj);
              accB[lv - 1][j].add(unj * uj + vnj * vj);
              accC[lv - 1][j].add(unj * vj - vnj * uj);
            }
            if (dst) {
              *reinterpret_cast<float4 *>(dst + x * W + off) = un;
              *reinterpret_cast<float4 *>(dst + hb + x * W + off) = vn;
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
      }
      __syncthreads();  // level lv's row is read by level lv + 1 below
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
  const size_t ring = ((4 + D) + (3 + D) + 3 * (K - 1)) * rowel + (K + 2 + D) * pel;
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

template <int W, int K, int D>
cudaError_t dispatch(const StepArgs &a, cudaStream_t s) {
  const int xsl = kThreads / (W / 4);
  const size_t smem = smem_bytes<W, K, D>(a.Lx);
  if (a.Lx <= xsl) return launch_one<W, K, D, 1>(a, smem, s);
  if (a.Lx <= 2 * xsl) return launch_one<W, K, D, 2>(a, smem, s);
  if (a.Lx <= 4 * xsl) return launch_one<W, K, D, 4>(a, smem, s);
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
  int D = want_depth > 0 ? std::min(want_depth, 2) : 1;
  if ((W != 8 && W != 16) || K < 2 || K > 4 || Ly < 2 || ld % W != 0 || Lx > 4 * kThreads / (W / 4))
    return false;
  const size_t b = smem_lookup(W, K, D, Lx);
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
