// step.cu -- the Chebyshev recursion step of Eq. 15 for real on-site
// (s-wave) lattices, with the moment products fused in.
//
// One launch advances a block of start vectors by one step,
//     j_{n+1} = 2 H~ j_n - j_{n-1}      (written in place over j_{n-1}),
// and emits, per column, the three products that the doubling identities
// turn into four moments (two ee, two eh):
//     A = <j_n|j_n>,  B = <j_{n+1}|j_n>,  C = sum_s (u'_s v_s - v'_s u_s)
// where (u, v) are the electron / hole rows of j_n and (u', v') of j_{n+1}.
//
// Layout (slab-blocked [2N x B]): the B start vectors are cut into slabs of
// W columns and each slab is stored as its own row-major [2N][W] block,
//     element (row r, column b) at (b / W) * 2N*W + r*W + (b % W),
// where the 2N rows are ordered lattice row by lattice row and, inside
// lattice row y, first the Lx electron rows then the Lx hole rows:
//     r(x, y, part) = 2*Lx*y + part*Lx + x      (part 0: electron, 1: hole).
// Lattice row y of one slab is one contiguous 2*Lx*W-element block, which
// streams from HBM as a single run, and a warp reading W-wide segments of
// consecutive x touches consecutive shared-memory words (no bank conflicts).
//
// A CTA owns one slab and a range of lattice rows and marches along y.  A
// pipeline D rows deep stages, per lattice row, the j_n block, the j_{n-1}
// block and the row's parameter records into shared-memory rings (3 + D
// slots for j_n: rows y-1, y, y+1 plus D in flight; 2 + D for j_{n-1}) with
// TMA bulk copies (cp.async.bulk) issued by one thread and completing on one
// mbarrier per slot; every wait is bounded in time and a lost copy sets an
// error flag instead of hanging.  Every element of j_n and j_{n-1} is read from HBM once per step
// and every stencil neighbour comes from shared memory; each Hamiltonian
// parameter is read once per row for all W columns; j_{n+1} is stored
// straight to HBM.  Column sums use Kahan compensation in FP32 (plain FP64
// sums in FP64) and are reduced across the CTA in FP64 in a fixed order:
// deterministic, no atomics.
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace cbdg {
namespace {

template <typename S>
struct Vec;
template <>
struct Vec<float> {
  using T = float4;
  static constexpr int N = 4;
};
template <>
struct Vec<double> {
  using T = double2;
  static constexpr int N = 2;
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
// One bulk copy global -> shared (TMA, untiled), completing on mbarrier bar.
// Addresses 16-byte aligned, bytes a multiple of 16.
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
// Waits for phase `parity` of bar to complete; gives up after ~limit_ns
// (returns false) so that a lost copy can never hang the GPU.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, unsigned long long limit_ns) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned it = 0;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255u) == 255u && global_ns() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// Accumulates a1*b1 + a2*b2: compensated (Kahan) in FP32, with the products
// and the compensation term fused into two FMAs; plain accumulation in FP64.
template <typename S>
struct Acc {
  S s = 0;
  __device__ __forceinline__ void add2(S a1, S b1, S a2, S b2) { s = fma_rn(a1, b1, fma_rn(a2, b2, s)); }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct Acc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add2(float a1, float b1, float a2, float b2) {
    const float y = fma_rn(a1, b1, fma_rn(a2, b2, -c));
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

template <typename V, typename S>
__device__ __forceinline__ S comp(const V &v, int j) {
  return reinterpret_cast<const S *>(&v)[j];
}
template <typename V, typename S>
__device__ __forceinline__ void set_comp(V &v, int j, S x) {
  reinterpret_cast<S *>(&v)[j] = x;
}

// PST: stage each lattice row's parameters with its j_n row (TMA, one ring
// slot per row); without it (wide lattices, whose rings would not fit in
// shared memory) the computed row's parameters are read through the
// read-only cache, where the 32-byte records of a row stay L2-resident.
template <typename S, int W, int NT, int MAXX, int D, bool PST = true>
__global__ void __launch_bounds__(NT, 1) step_real_kernel(StepArgs a) {
  using V = typename Vec<S>::T;
  constexpr int VEC = Vec<S>::N;
  constexpr int QUADS = W / VEC;       // 16-byte chunks per row segment
  constexpr int XSLOTS = NT / QUADS;   // threads along x
  constexpr int JS = 3 + D;            // j_n ring slots
  constexpr int OS = 2 + D;            // j_{n-1} ring slots
  static_assert(W % VEC == 0 && NT % QUADS == 0, "bad slab shape");

  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long bars[3 + D];
  __shared__ int abort_flag;
  const int Lx = a.Lx, Ly = a.Ly;
  const int rowel = 2 * Lx * W;        // elements of one lattice row of a slab
  const int pel = Lx * kParamStride;   // parameter scalars of one lattice row
  S *sj = reinterpret_cast<S *>(smem_raw);
  S *so = sj + JS * rowel;
  S *sp = so + OS * rowel;

  const int t = threadIdx.x;
  const int q = t % QUADS;
  const int xs = t / QUADS;
  const int y0 = blockIdx.y * a.rows_per_cta;
  const int rows = min(a.rows_per_cta, Ly - y0);
  const size_t slab = static_cast<size_t>(blockIdx.x) * (static_cast<size_t>(2) * Lx * Ly * W);
  const S *cur = static_cast<const S *>(a.cur) + slab;
  S *prev = static_cast<S *>(a.prev) + slab;
  S *const dst = a.out ? static_cast<S *>(a.out) + slab : prev;  // j_{n+1}
  const S *par = static_cast<const S *>(a.params);
  const unsigned row_bytes = static_cast<unsigned>(rowel * sizeof(S));
  const unsigned par_bytes = PST ? static_cast<unsigned>(pel * sizeof(S)) : 0u;
  const unsigned long long kWaitLimitNs = a.wait_ns;

  if (t == 0) {
    for (int k = 0; k < JS; ++k) mbar_init(smem_addr(&bars[k]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    abort_flag = 0;
  }
  __syncthreads();

  // Load k (issued by thread 0, one TMA bulk copy per block): j_n and the
  // parameters of lattice row y0 - 1 + k (periodic wrap; an open edge has
  // zero hopping on the wrapped bond), plus j_{n-1} of the computed row
  // y0 + k - 1 when that row belongs to this CTA.  All complete on bars[k % JS].
  auto issue = [&](int k) {
    int y = y0 - 1 + k;
    y = (y < 0) ? y + Ly : (y >= Ly ? y - Ly : y);
    const int r = k - 1;
    const bool with_old = (r >= 0 && r < rows);
    const unsigned bar = smem_addr(&bars[k % JS]);
    mbar_expect_tx(bar, row_bytes + par_bytes + (with_old ? row_bytes : 0u) + (k == 0 ? a.stall_tx : 0u));
    bulk_load(smem_addr(sj + (k % JS) * rowel), cur + static_cast<size_t>(y) * rowel, row_bytes, bar);
    if (PST) bulk_load(smem_addr(sp + (k % JS) * pel), par + static_cast<size_t>(y) * pel, par_bytes, bar);
    if (with_old)
      bulk_load(smem_addr(so + (r % OS) * rowel), prev + static_cast<size_t>(y0 + r) * rowel,
                row_bytes, bar);
  };
  int issued = 0;  // loads issued so far (thread 0's view; loads are issued in order)
  if (t == 0) {
    for (int k = 0; k < D + 2 && k <= rows + 1; ++k) issue(k);
  }
  issued = min(D + 2, rows + 2);

  Acc<S> accA[VEC], accB[VEC], accC[VEC];

  int waited = 0;  // loads this thread has seen complete
  bool ok = true;
  for (int i = 0; i < rows; ++i) {
    // The slots refilled here were last read in iteration i - 1, which every
    // thread has left through the barrier that ends it.
    if (i + 2 + D <= rows + 1) {
      if (t == 0) issue(i + 2 + D);
      issued = i + 3 + D;
    }
    // loads up to i + 2: rows y-1, y, y+1 of j_n and j_{n-1} of y
    for (; ok && waited <= i + 2; ++waited) {
      if (!mbar_wait(smem_addr(&bars[waited % JS]), (waited / JS) & 1u, kWaitLimitNs)) ok = false;
    }
    if (!ok) abort_flag = 1;

    if (ok) {
      const S *rm = sj + (i % JS) * rowel;        // lattice row y - 1
      const S *rc = sj + ((i + 1) % JS) * rowel;  // y
      const S *rp = sj + ((i + 2) % JS) * rowel;  // y + 1
      const S *ro = so + (i % OS) * rowel;        // j_{n-1} of y
      const S *pc = PST ? sp + ((i + 1) % JS) * pel : par + static_cast<size_t>(y0 + i) * pel;
      S *out = dst + static_cast<size_t>(y0 + i) * rowel;
      const int off = q * VEC;
      const int hb = Lx * W;  // hole rows follow the electron rows
#pragma unroll
      for (int k = 0; k < MAXX; ++k) {
        const int x = xs + k * XSLOTS;
        if (x < Lx) {
          const int xl = (x == 0) ? Lx - 1 : x - 1;
          const int xr = (x == Lx - 1) ? 0 : x + 1;
          const V u = *reinterpret_cast<const V *>(rc + x * W + off);
          const V v = *reinterpret_cast<const V *>(rc + hb + x * W + off);
          const V ur = *reinterpret_cast<const V *>(rc + xr * W + off);
          const V vr = *reinterpret_cast<const V *>(rc + hb + xr * W + off);
          const V ul = *reinterpret_cast<const V *>(rc + xl * W + off);
          const V vl = *reinterpret_cast<const V *>(rc + hb + xl * W + off);
          const V uu = *reinterpret_cast<const V *>(rp + x * W + off);
          const V vu = *reinterpret_cast<const V *>(rp + hb + x * W + off);
          const V ud = *reinterpret_cast<const V *>(rm + x * W + off);
          const V vd = *reinterpret_cast<const V *>(rm + hb + x * W + off);
          const V uo = *reinterpret_cast<const V *>(ro + x * W + off);
          const V vo = *reinterpret_cast<const V *>(ro + hb + x * W + off);
          const S *pp = pc + x * kParamStride;
          const S e = PST ? pp[0] : __ldg(pp + 0), d = PST ? pp[1] : __ldg(pp + 1);
          const S t0 = PST ? pp[2] : __ldg(pp + 2), t1 = PST ? pp[3] : __ldg(pp + 3);
          const S t2 = PST ? pp[4] : __ldg(pp + 4), t3 = PST ? pp[5] : __ldg(pp + 5);
          V un, vn;
#pragma unroll
          for (int j = 0; j < VEC; ++j) {
            const S uj = comp<V, S>(u, j), vj = comp<V, S>(v, j);
            // 2 H~ j_n - j_{n-1}:
            //   electron row  (eps-mu) u + Delta v - sum_d t_d u_d - u_old
            //   hole row      Delta u - (eps-mu) v + sum_d t_d v_d - v_old
            // each one chain of six FMAs
            const S unj = fma_rn(e, uj, fma_rn(d, vj, -fma_rn(t3, comp<V, S>(ud, j), fma_rn(t2, comp<V, S>(uu, j),
                              fma_rn(t1, comp<V, S>(ul, j), fma_rn(t0, comp<V, S>(ur, j), comp<V, S>(uo, j)))))));
            const S vnj = fma_rn(d, uj, fma_rn(-e, vj, fma_rn(t3, comp<V, S>(vd, j), fma_rn(t2, comp<V, S>(vu, j),
                              fma_rn(t1, comp<V, S>(vl, j), fma_rn(t0, comp<V, S>(vr, j), -comp<V, S>(vo, j)))))));
            set_comp<V, S>(un, j, unj);
            set_comp<V, S>(vn, j, vnj);
            accA[j].add2(uj, uj, vj, vj);
            accB[j].add2(unj, uj, vnj, vj);
            accC[j].add2(unj, vj, -vnj, uj);
          }
          __stcs(reinterpret_cast<V *>(out + x * W + off), un);
          __stcs(reinterpret_cast<V *>(out + hb + x * W + off), vn);
        }
      }
    }
    __syncthreads();  // ends iteration i: its slots may be refilled
    if (abort_flag) break;
  }
  if (abort_flag) {
    // A copy did not arrive in time: report it, let the copies in flight
    // land (bounded again) so no TMA write targets freed shared memory, and
    // leave without writing partial sums.
    if (t == 0) {
      atomicOr(a.flags, kFlagTimeout);
      for (int k = waited; k < issued; ++k)
        if (!mbar_wait(smem_addr(&bars[k % JS]), (k / JS) & 1u, kWaitLimitNs)) break;
    }
    return;
  }
  __syncthreads();

  // Fixed-order CTA reduction of the column sums, in FP64.
  double *red = reinterpret_cast<double *>(smem_raw);
#pragma unroll
  for (int j = 0; j < VEC; ++j) {
    red[(0 * XSLOTS + xs) * W + q * VEC + j] = accA[j].value();
    red[(1 * XSLOTS + xs) * W + q * VEC + j] = accB[j].value();
    red[(2 * XSLOTS + xs) * W + q * VEC + j] = accC[j].value();
  }
  __syncthreads();
  const size_t c0 = static_cast<size_t>(blockIdx.x) * W;
  for (int idx = t; idx < 3 * W; idx += NT) {
    const int k = idx / W, col = idx - k * W;
    double s = 0.0;
    for (int z = 0; z < XSLOTS; ++z) s += red[(k * XSLOTS + z) * W + col];
    a.partials[(static_cast<size_t>(blockIdx.y) * 3 + k) * a.ld + c0 + col] = s;
  }
}

constexpr int kThreads = 256;
// Dynamic shared memory cap: the 227 KB per-CTA opt-in limit less room for
// the kernel's static mbarriers.
constexpr int kMaxDynSmem = 227 * 1024 - 1024;
constexpr int kUnstagedDepth = 2;  // rows in flight of the unstaged (wide-lattice) variant

template <typename S, int W, int D>
size_t smem_bytes(int Lx) {
  constexpr int QUADS = W / Vec<S>::N;
  constexpr int XSLOTS = kThreads / QUADS;
  const size_t rowel = static_cast<size_t>(2) * Lx * W;
  const size_t ring = ((3 + D) * rowel + (2 + D) * rowel +
                       (3 + D) * static_cast<size_t>(Lx) * kParamStride) * sizeof(S);
  const size_t red = static_cast<size_t>(3) * XSLOTS * W * sizeof(double);
  return std::max(ring, red);
}

template <typename S, int W>
size_t smem_bytes_unstaged(int Lx) {
  constexpr int D = kUnstagedDepth;
  constexpr int QUADS = W / Vec<S>::N;
  constexpr int XSLOTS = kThreads / QUADS;
  const size_t rowel = static_cast<size_t>(2) * Lx * W;
  const size_t ring = ((3 + D) * rowel + (2 + D) * rowel) * sizeof(S);
  const size_t red = static_cast<size_t>(3) * XSLOTS * W * sizeof(double);
  return std::max(ring, red);
}

template <typename S, int W, int MAXX, int D, bool PST = true>
cudaError_t launch_one(const StepArgs &a, const StepConfig &cfg, cudaStream_t s) {
  auto k = step_real_kernel<S, W, kThreads, MAXX, D, PST>;
  static int attr_dev = -1;  // set once per instantiation and device
  int dev = 0;
  cudaGetDevice(&dev);
  if (attr_dev != dev) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
    if (e != cudaSuccess) return e;
    attr_dev = dev;
  }
  dim3 grid(a.ld / W, cfg.row_split);
  k<<<grid, kThreads, cfg.smem, s>>>(a);
  return cudaGetLastError();
}

template <typename S, int W>
int xslots() {
  return kThreads / (W / Vec<S>::N);
}

template <typename S, int W, int D>
cudaError_t dispatch_maxx(const StepArgs &a, const StepConfig &cfg, cudaStream_t s) {
  const int xsl = xslots<S, W>();
  if (!cfg.pstage) {
    // wide lattices only (the staged rings fit up to xsl sites)
    if (a.Lx <= 2 * xsl) return launch_one<S, W, 2, kUnstagedDepth, false>(a, cfg, s);
    if (a.Lx <= 4 * xsl) return launch_one<S, W, 4, kUnstagedDepth, false>(a, cfg, s);
    if (a.Lx <= 8 * xsl) return launch_one<S, W, 8, kUnstagedDepth, false>(a, cfg, s);
    return cudaErrorInvalidValue;
  }
  if (a.Lx <= 1 * xsl) return launch_one<S, W, 1, D>(a, cfg, s);
  if (a.Lx <= 2 * xsl) return launch_one<S, W, 2, D>(a, cfg, s);
  if (a.Lx <= 4 * xsl) return launch_one<S, W, 4, D>(a, cfg, s);
  if (a.Lx <= 8 * xsl) return launch_one<S, W, 8, D>(a, cfg, s);
  return cudaErrorInvalidValue;
}

template <typename S, int W>
cudaError_t dispatch_depth(const StepArgs &a, const StepConfig &cfg, cudaStream_t s) {
  if (!cfg.pstage) return dispatch_maxx<S, W, kUnstagedDepth>(a, cfg, s);
  switch (cfg.depth) {
    case 1: return dispatch_maxx<S, W, 1>(a, cfg, s);
    case 2: return dispatch_maxx<S, W, 2>(a, cfg, s);
    case 3: return dispatch_maxx<S, W, 3>(a, cfg, s);
    case 4: return dispatch_maxx<S, W, 4>(a, cfg, s);
  }
  return cudaErrorInvalidValue;
}

template <typename S>
size_t smem_dispatch(int W, int D, int Lx) {
  constexpr int V = Vec<S>::N;
#define CBDG_SMEM_CASE(w)                                                       \
  case w:                                                                       \
    return D == 1   ? smem_bytes<S, w, 1>(Lx)                                   \
           : D == 2 ? smem_bytes<S, w, 2>(Lx)                                   \
           : D == 3 ? smem_bytes<S, w, 3>(Lx)                                   \
                    : smem_bytes<S, w, 4>(Lx);
  switch (W) {
    CBDG_SMEM_CASE(V)
    CBDG_SMEM_CASE(2 * V)
    CBDG_SMEM_CASE(4 * V)
    CBDG_SMEM_CASE(8 * V)
  }
#undef CBDG_SMEM_CASE
  return 0;
}

template <typename S>
int max_lx(int W) {
  return 8 * kThreads / (W / Vec<S>::N);
}

template <typename S>
size_t smem_unstaged_dispatch(int W, int Lx) {
  constexpr int V = Vec<S>::N;
  switch (W) {
    case V: return smem_bytes_unstaged<S, V>(Lx);
    case 2 * V: return smem_bytes_unstaged<S, 2 * V>(Lx);
    case 4 * V: return smem_bytes_unstaged<S, 4 * V>(Lx);
    case 8 * V: return smem_bytes_unstaged<S, 8 * V>(Lx);
  }
  return 0;
}

}  // namespace

int slab_width_default(int precision) { return precision == 1 ? 16 : 4; }

int choose_row_split(int slabs, int Ly, size_t smem, int threads) {
  int dev = 0;
  cudaGetDevice(&dev);
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int per_sm = static_cast<int>((228 * 1024) / (smem + 1024));
  per_sm = std::max(1, std::min(per_sm, 2048 / threads));
  const int slots = sms * per_sm;
  if (per_sm > 1) {
    // several CTAs per SM share its bandwidth: split only to reach two waves
    int split = 1;
    while (slabs * split < 2 * slots && (Ly + 2 * split - 1) / (2 * split) >= 8) split *= 2;
    return split;
  }
  // One CTA per SM: the CTAs run in ceil(slabs * split / slots) waves, each
  // as long as one CTA's rows -- three vector streams per row, plus two halo
  // rows of j_n and a pipeline fill of a few rows -- so take the split with
  // the least waves x (3 rows + 8), at least 8 rows per CTA, if it beats one
  // CTA per slab by 5% (the model is coarse; splitting re-reads halos).
  auto cost = [&](int n, int rpc) {
    return ((static_cast<long long>(slabs) * n + slots - 1) / slots) * (3LL * rpc + 8);
  };
  const long long whole = cost(1, Ly);
  int best = 1;
  long long best_cost = whole;
  for (int split = 2; split <= Ly; ++split) {
    const int rpc = (Ly + split - 1) / split;
    if (rpc < 8) break;
    const int n = (Ly + rpc - 1) / rpc;
    const long long c = cost(n, rpc);
    if (c < best_cost) {
      best_cost = c;
      best = n;
    }
  }
  return 20 * best_cost <= 19 * whole ? best : 1;
}

bool plan_step_real(int precision, int Lx, int Ly, int ld, int want_w, int want_split,
                    int want_depth, StepConfig *cfg) {
  const int vecn = precision == 1 ? 4 : 2;
  int W = want_w > 0 ? want_w : slab_width_default(precision);
  const int d0 = want_depth > 0 ? std::min(want_depth, 4) : 3;
  int D = d0;
  auto smem = [&](int w, int d) {
    return precision == 1 ? smem_dispatch<float>(w, d, Lx) : smem_dispatch<double>(w, d, Lx);
  };
  auto lxmax = [&](int w) { return precision == 1 ? max_lx<float>(w) : max_lx<double>(w); };
  auto fits = [&](int w, int d) {
    const size_t b = smem(w, d);
    return b != 0 && b <= kMaxDynSmem && ld % w == 0 && Lx <= lxmax(w);
  };
  bool pstage = true;
  while (!fits(W, D)) {
    if (D > 1) {
      D -= 1;
    } else if (W > vecn) {
      W /= 2;
      D = d0;
    } else {
      pstage = false;
      break;
    }
  }
  auto smem_u = [&](int w) {
    return precision == 1 ? smem_unstaged_dispatch<float>(w, Lx) : smem_unstaged_dispatch<double>(w, Lx);
  };
  if (!pstage) {
    // wide lattices (two or more sites per thread): parameters through the
    // read-only cache, smaller rings
    W = want_w > 0 ? want_w : slab_width_default(precision);
    D = kUnstagedDepth;
    while (!(smem_u(W) != 0 && smem_u(W) <= kMaxDynSmem && ld % W == 0 && Lx <= lxmax(W) &&
             Lx > kThreads / (W / vecn))) {
      if (W > vecn) W /= 2;
      else return false;
    }
  }
  const size_t smem_now = pstage ? smem(W, D) : smem_u(W);
  const int slabs = ld / W;
  int split = want_split;
  if (split <= 0) split = choose_row_split(slabs, Ly, smem_now, kThreads);
  split = std::max(1, std::min(split, Ly));
  const int rpc = (Ly + split - 1) / split;
  cfg->slab_w = W;
  cfg->depth = D;
  cfg->row_split = (Ly + rpc - 1) / rpc;
  cfg->threads = kThreads;
  cfg->smem = smem_now;
  cfg->pstage = pstage ? 1 : 0;
  return true;
}

cudaError_t launch_step_real(int precision, const StepArgs &a, const StepConfig &cfg,
                             cudaStream_t s) {
  if (precision == 1) {
    switch (cfg.slab_w) {
      case 4: return dispatch_depth<float, 4>(a, cfg, s);
      case 8: return dispatch_depth<float, 8>(a, cfg, s);
      case 16: return dispatch_depth<float, 16>(a, cfg, s);
      case 32: return dispatch_depth<float, 32>(a, cfg, s);
    }
  } else {
    switch (cfg.slab_w) {
      case 2: return dispatch_depth<double, 2>(a, cfg, s);
      case 4: return dispatch_depth<double, 4>(a, cfg, s);
      case 8: return dispatch_depth<double, 8>(a, cfg, s);
      case 16: return dispatch_depth<double, 16>(a, cfg, s);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace cbdg
