// step_cplx.cu -- the Chebyshev recursion step of Eq. 15 for general
// lattices: complex hoppings (Peierls phases), optional next-nearest-neighbour
// hopping and on-site or nearest-neighbour bond pairing (Eq. 2).
//
//   u'_s = (e u + D v - sum_d t_d u_d + sum_{d<4} B_d v_d)_s - u_old     (electron rows)
//   v'_s = (conj(D) u - e v + sum_d conj(t_d) v_d + sum_{d<4} conj(B_d) u_d)_s - v_old (hole rows)
// with e = 2(eps - mu)/a, D = 2 Delta_s/a, t_d = 2 t_{s,d}/a, B_d = 2 Delta_{s,d}/a
// and u_d, v_d the components of the neighbour along direction d.
//
// Vectors are complex (float2 / double2) in the slab-blocked layout of the
// real kernel (rows electron-then-hole inside each lattice row), staged by
// TMA bulk copies on mbarriers with bounded waits.  Parameters (8 complex
// fields per site, field-major inside each lattice row) stay resident in L2:
// the FP32 kernel stages each row with the j_n row of the same lattice row
// (so rows y - 1 and y are on chip together), the FP64 kernel reads them
// through the read-only cache; either way threads on consecutive x read
// consecutive pairs.  H is Hermitian and the bond pairing symmetric, so a
// site stores only its forward hoppings (+x, +y, +x+y, -x+y) and bonds
// (+x, +y); the backward ones are those of the left, lower and diagonal
// neighbours, conjugated for the hoppings:
//   t(i, -x) = conj t(i-x, +x),  t(i, -y) = conj t(i-y, +y),
//   t(i, -x-y) = conj t(i-x-y, +x+y),  t(i, +x-y) = conj t(i+x-y, -x+y),
//   D(i, -x) = D(i-x, +x),  D(i, -y) = D(i-y, +y).
//
// With on-site pairing the doubling identities apply and the kernel fuses
// four column sums (|j_n|^2, Re<j_{n+1}|j_n>, and the complex symplectic sum
// sum_s (u'_s v_s - v'_s u_s)); with bond pairing every moment is read
// directly from the vectors by a gather kernel, and no sums are formed.
#include <algorithm>
#include <cmath>

#include "cplx_stencil.cuh"

namespace cbdg {
namespace {

using namespace cx;

template <typename S>
struct CVec;
template <>
struct CVec<float> {
  using T = float4;            // two complex64
  static constexpr int N = 2;  // complex elements per 16 bytes
};
template <>
struct CVec<double> {
  using T = double2;           // one complex128
  static constexpr int N = 1;
};

__device__ __forceinline__ unsigned smem_addr(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_load(unsigned dst, const void *src, unsigned bytes,
                                          unsigned bar) {
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

template <typename S>
struct Acc {
  S s = 0;
  __device__ __forceinline__ void add(S x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct Acc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    float y = __fsub_rn(x, c);
    float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

template <typename S, int W, int NT, int MAXX, int D, bool NNN, bool BOND, bool SUMS>
__global__ void __launch_bounds__(NT, 1) step_cplx_kernel(StepArgs a) {
  // FP32: parameter rows ride the TMA pipeline with j_n; FP64 (bound by its
  // arithmetic) reads them through the read-only cache.
  constexpr bool PSTAGE = sizeof(S) == 4;
  using V = typename CVec<S>::T;
  constexpr int VC = CVec<S>::N;       // complex elements per 16-byte vector
  constexpr int QUADS = W / VC;        // 16-byte chunks per row segment
  constexpr int XSLOTS = NT / QUADS;
  constexpr int JS = 3 + D;
  constexpr int OS = 2 + D;
  static_assert(W % VC == 0 && NT % QUADS == 0, "bad slab shape");

  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long bars[3 + D];
  __shared__ int abort_flag;
  const int Lx = a.Lx, Ly = a.Ly;
  const int rowel = 2 * Lx * W * 2;    // scalars of one lattice row of a slab (complex)
  S *sj = reinterpret_cast<S *>(smem_raw);
  S *so = sj + JS * rowel;
  const int pel = Lx * kCplxParamStride;  // parameter scalars of one lattice row
  S *sp = so + OS * rowel;                  // [JS][pel] when PSTAGE, slot as the j_n row

  const int t = threadIdx.x;
  const int q = t % QUADS;
  const int xs = t / QUADS;
  const int y0 = blockIdx.y * a.rows_per_cta;
  const int rows = min(a.rows_per_cta, Ly - y0);
  const size_t slab = static_cast<size_t>(blockIdx.x) * (static_cast<size_t>(2) * Lx * Ly * W * 2);
  const S *cur = static_cast<const S *>(a.cur) + slab;
  S *prev = static_cast<S *>(a.prev) + slab;
  S *const dst = a.out ? static_cast<S *>(a.out) + slab : prev;  // j_{n+1} (in place unless out is set)
  const S *par = static_cast<const S *>(a.params);
  const unsigned row_bytes = static_cast<unsigned>(rowel * sizeof(S));
  const unsigned par_bytes = PSTAGE ? static_cast<unsigned>(pel * sizeof(S)) : 0u;
  const unsigned long long kWaitLimitNs = a.wait_ns;

  if (t == 0) {
    for (int k = 0; k < JS; ++k) mbar_init(smem_addr(&bars[k]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    abort_flag = 0;
  }
  __syncthreads();

  auto issue = [&](int k) {
    int y = y0 - 1 + k;
    y = (y < 0) ? y + Ly : (y >= Ly ? y - Ly : y);
    const int r = k - 1;
    const bool with_old = (r >= 0 && r < rows);
    const unsigned bar = smem_addr(&bars[k % JS]);
    mbar_expect_tx(bar, row_bytes + par_bytes + (with_old ? row_bytes : 0u) + (k == 0 ? a.stall_tx : 0u));
    bulk_load(smem_addr(sj + (k % JS) * rowel), cur + static_cast<size_t>(y) * rowel, row_bytes, bar);
    if (PSTAGE)
      bulk_load(smem_addr(sp + (k % JS) * pel), par + static_cast<size_t>(y) * pel, par_bytes, bar);
    if (with_old)
      bulk_load(smem_addr(so + (r % OS) * rowel), prev + static_cast<size_t>(y0 + r) * rowel,
                row_bytes, bar);
  };
  int issued = min(D + 2, rows + 2);
  if (t == 0)
    for (int k = 0; k < D + 2 && k <= rows + 1; ++k) issue(k);

  Acc<S> accA[VC], accB[VC], accCr[VC], accCi[VC];

  int waited = 0;
  bool ok = true;
  for (int i = 0; i < rows; ++i) {
    if (i + 2 + D <= rows + 1) {
      if (t == 0) issue(i + 2 + D);
      issued = i + 3 + D;
    }
    for (; ok && waited <= i + 2; ++waited)
      if (!mbar_wait(smem_addr(&bars[waited % JS]), (waited / JS) & 1u, kWaitLimitNs)) ok = false;
    if (!ok) abort_flag = 1;

    if (ok) {
      const S *rm = sj + (i % JS) * rowel;
      const S *rc = sj + ((i + 1) % JS) * rowel;
      const S *rp = sj + ((i + 2) % JS) * rowel;
      const S *ro = so + (i % OS) * rowel;
      const int y = y0 + i;
      S *out = dst + static_cast<size_t>(y) * rowel;
      const int hb = Lx * W * 2;  // hole rows follow the electron rows (scalars)
      const int off = q * VC * 2;
#pragma unroll
      for (int k = 0; k < MAXX; ++k) {
        const int x = xs + k * XSLOTS;
        if (x < Lx) {
          const int xl = (x == 0) ? Lx - 1 : x - 1;
          const int xr = (x == Lx - 1) ? 0 : x + 1;
          // parameter rows y (own, left neighbour) and y - 1 (lower neighbours)
          const S *py0 = PSTAGE ? sp + ((i + 1) % JS) * pel : par + static_cast<size_t>(y) * pel;
          const S *py1 = PSTAGE ? sp + (i % JS) * pel
                                : par + static_cast<size_t>(y == 0 ? Ly - 1 : y - 1) * pel;
          V u, v, un, vn;
          cx::site_step<S, V, VC, W, NNN, BOND, !PSTAGE>(rm, rc, rp, ro, py0, py1, x, xl, xr, off, hb, Lx, u, v, un,
                                                          vn);
#pragma unroll
          for (int j = 0; j < VC; ++j) {
            const Cx<S> unj = cget<V, S>(un, j);
            const Cx<S> vnj = cget<V, S>(vn, j);
            if (SUMS) {
              const Cx<S> uj = cget<V, S>(u, j), vj = cget<V, S>(v, j);
              accA[j].add(uj.re * uj.re + uj.im * uj.im + vj.re * vj.re + vj.im * vj.im);
              accB[j].add(unj.re * uj.re + unj.im * uj.im + vnj.re * vj.re + vnj.im * vj.im);
              const Cx<S> c = csub(cmul(unj, vj), cmul(vnj, uj));
              accCr[j].add(c.re);
              accCi[j].add(c.im);
            }
          }
          __stcs(reinterpret_cast<V *>(out + x * W * 2 + off), un);
          __stcs(reinterpret_cast<V *>(out + hb + x * W * 2 + off), vn);
        }
      }
    }
    __syncthreads();
    if (abort_flag) break;
  }
  if (abort_flag) {
    if (t == 0) {
      atomicOr(a.flags, kFlagTimeout);
      for (int k = waited; k < issued; ++k)
        if (!mbar_wait(smem_addr(&bars[k % JS]), (k / JS) & 1u, kWaitLimitNs)) break;
    }
    return;
  }
  if (!SUMS) return;
  __syncthreads();
  double *red = reinterpret_cast<double *>(smem_raw);
#pragma unroll
  for (int j = 0; j < VC; ++j) {
    red[(0 * XSLOTS + xs) * W + q * VC + j] = accA[j].value();
    red[(1 * XSLOTS + xs) * W + q * VC + j] = accB[j].value();
    red[(2 * XSLOTS + xs) * W + q * VC + j] = accCr[j].value();
    red[(3 * XSLOTS + xs) * W + q * VC + j] = accCi[j].value();
  }
  __syncthreads();
  const size_t c0 = static_cast<size_t>(blockIdx.x) * W;
  for (int idx = t; idx < 4 * W; idx += NT) {
    const int k = idx / W, col = idx - k * W;
    double s = 0.0;
    for (int z = 0; z < XSLOTS; ++z) s += red[(k * XSLOTS + z) * W + col];
    a.partials[(static_cast<size_t>(blockIdx.y) * 4 + k) * a.ld + c0 + col] = s;
  }
}

constexpr int kThreads = 256;
// FP32 rows of at most kNarrowLx sites at slab width 4 run 128-thread CTAs:
// 64 x slots, so every thread holds a site (256 threads would leave half of
// them idle) and twice the CTAs fit on an SM.
constexpr int kNarrowThreads = 128, kNarrowLx = 64;
constexpr int kMaxDynSmem = 227 * 1024 - 1024;

template <typename S, int W, int D>
size_t smem_bytes(int Lx) {
  constexpr int QUADS = W / CVec<S>::N;
  constexpr int XSLOTS = kThreads / QUADS;
  const size_t rowel = static_cast<size_t>(2) * Lx * W * 2;
  const size_t pel = sizeof(S) == 4 ? static_cast<size_t>(Lx) * kCplxParamStride : 0;
  const size_t ring = (((3 + D) + (2 + D)) * rowel + (3 + D) * pel) * sizeof(S);
  const size_t red = static_cast<size_t>(4) * XSLOTS * W * sizeof(double);
  return std::max(ring, red);
}

template <typename S, int W, int MAXX, int D, bool NNN, bool BOND, bool SUMS, int NT = kThreads>
cudaError_t launch_one(const StepArgs &a, const StepConfig &cfg, cudaStream_t s) {
  auto k = step_cplx_kernel<S, W, NT, MAXX, D, NNN, BOND, SUMS>;
  static int attr_dev = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (attr_dev != dev) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
    if (e != cudaSuccess) return e;
    attr_dev = dev;
  }
  dim3 grid(a.ld / W, cfg.row_split);
  k<<<grid, NT, cfg.smem, s>>>(a);
  return cudaGetLastError();
}

template <typename S, int W, int D, bool NNN, bool BOND, bool SUMS>
cudaError_t dispatch_maxx(const StepArgs &a, const StepConfig &cfg, cudaStream_t s) {
  const int xsl = kThreads / (W / CVec<S>::N);
  if constexpr (sizeof(S) == 4 && W == 4) {
    if (cfg.threads == kNarrowThreads) {
      if (a.Lx > kNarrowLx) return cudaErrorInvalidValue;
      return launch_one<S, W, 1, D, NNN, BOND, SUMS, kNarrowThreads>(a, cfg, s);
    }
  }
  if (cfg.threads != kThreads) return cudaErrorInvalidValue;
  if (a.Lx <= 1 * xsl) return launch_one<S, W, 1, D, NNN, BOND, SUMS>(a, cfg, s);
  if (a.Lx <= 2 * xsl) return launch_one<S, W, 2, D, NNN, BOND, SUMS>(a, cfg, s);
  if (a.Lx <= 4 * xsl) return launch_one<S, W, 4, D, NNN, BOND, SUMS>(a, cfg, s);
  return cudaErrorInvalidValue;
}

template <typename S, int W, int D>
cudaError_t dispatch_kind(const StepArgs &a, const StepConfig &cfg, int nnn, int bond,
                          cudaStream_t s) {
  // bond pairing reads moments directly (no sums); on-site pairing uses the sums
  if (bond) {
    return nnn ? dispatch_maxx<S, W, D, true, true, false>(a, cfg, s)
               : dispatch_maxx<S, W, D, false, true, false>(a, cfg, s);
  }
  return nnn ? dispatch_maxx<S, W, D, true, false, true>(a, cfg, s)
             : dispatch_maxx<S, W, D, false, false, true>(a, cfg, s);
}

template <typename S, int W>
cudaError_t dispatch_depth(const StepArgs &a, const StepConfig &cfg, int nnn, int bond,
                           cudaStream_t s) {
  switch (cfg.depth) {
    case 1: return dispatch_kind<S, W, 1>(a, cfg, nnn, bond, s);
    case 2: return dispatch_kind<S, W, 2>(a, cfg, nnn, bond, s);
    case 3: return dispatch_kind<S, W, 3>(a, cfg, nnn, bond, s);
  }
  return cudaErrorInvalidValue;
}

template <typename S>
size_t smem_dispatch(int W, int D, int Lx) {
  constexpr int V = CVec<S>::N;
#define CBDG_SMEM_CASE(w)                                         \
  case w:                                                         \
    return D == 1   ? smem_bytes<S, w, 1>(Lx)                     \
           : D == 2 ? smem_bytes<S, w, 2>(Lx)                     \
                    : smem_bytes<S, w, 3>(Lx);
  switch (W) {
    CBDG_SMEM_CASE(V)
    CBDG_SMEM_CASE(2 * V)
    CBDG_SMEM_CASE(4 * V)
  }
#undef CBDG_SMEM_CASE
  return 0;
}

template <typename S>
int max_lx(int W) {
  return 4 * kThreads / (W / CVec<S>::N);
}

}  // namespace

int slab_width_default_cplx(int precision) { return precision == 1 ? 4 : 2; }

bool plan_step_cplx(int precision, int Lx, int Ly, int ld, int want_w, int want_split,
                    int want_depth, StepConfig *cfg) {
  const int vc = precision == 1 ? 2 : 1;
  int W = want_w > 0 ? want_w : slab_width_default_cplx(precision);
  const int d0 = want_depth > 0 ? std::min(want_depth, 3) : 2;
  int D = d0;
  auto smem = [&](int w, int d) {
    return precision == 1 ? smem_dispatch<float>(w, d, Lx) : smem_dispatch<double>(w, d, Lx);
  };
  auto lxmax = [&](int w) { return precision == 1 ? max_lx<float>(w) : max_lx<double>(w); };
  auto fits = [&](int w, int d) {
    const size_t b = smem(w, d);
    return b != 0 && b <= kMaxDynSmem && ld % w == 0 && Lx <= lxmax(w);
  };
  while (!fits(W, D)) {
    if (D > 1) {
      D -= 1;
    } else if (W > vc) {
      W /= 2;
      D = d0;
    } else {
      return false;
    }
  }
  const int slabs = ld / W;
  int split = want_split;
  const int threads = precision == 1 && W == 4 && Lx <= kNarrowLx ? kNarrowThreads : kThreads;
  if (split <= 0) split = choose_row_split(slabs, Ly, smem(W, D), threads);
  split = std::max(1, std::min(split, Ly));
  const int rpc = (Ly + split - 1) / split;
  cfg->slab_w = W;
  cfg->depth = D;
  cfg->row_split = (Ly + rpc - 1) / rpc;
  cfg->threads = threads;
  cfg->smem = smem(W, D);
  return true;
}

cudaError_t launch_step_cplx(int precision, int nnn, int bond, const StepArgs &a,
                             const StepConfig &cfg, cudaStream_t s) {
  if (precision == 1) {
    switch (cfg.slab_w) {
      case 2: return dispatch_depth<float, 2>(a, cfg, nnn, bond, s);
      case 4: return dispatch_depth<float, 4>(a, cfg, nnn, bond, s);
      case 8: return dispatch_depth<float, 8>(a, cfg, nnn, bond, s);
    }
  } else {
    switch (cfg.slab_w) {
      case 1: return dispatch_depth<double, 1>(a, cfg, nnn, bond, s);
      case 2: return dispatch_depth<double, 2>(a, cfg, nnn, bond, s);
      case 4: return dispatch_depth<double, 4>(a, cfg, nnn, bond, s);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace cbdg
