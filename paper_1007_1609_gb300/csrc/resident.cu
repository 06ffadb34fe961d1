// resident.cu -- the whole Chebyshev recursion of Eq. 15 for a small real
// on-site lattice in shared memory: one launch per pass over M moments.
//
// When a column slab's two vectors (2N x W each), the stencil parameters and
// the coefficient table fit in one SM's shared memory, a CTA loads j_0, j_1
// of its slab once and runs every step on chip: j_{n+1} = 2 H~ j_n - j_{n-1}
// written in place over j_{n-1} (a thread owns fixed (site, column) elements
// and reads only its own j_{n-1}), one CTA barrier per step.  The three column
// sums of the doubling identities (A = <j_n|j_n>, B = <j_{n+1}|j_n>,
// C = sum (u'v - v'u)) are reduced per step by warp shuffles and an FP64 sum
// over warps, and folded in FP64 by one thread per column exactly as
// fold_kernel does (moments 2n, 2n+1 of Eqs. 11 and 14, the Delta and n
// accumulators, the |mu| <= 1 check).  In FP64 without moment output the
// fold is linear in A, B, C, so each thread folds its own partial sums into
// FP64 accumulators that are reduced once at the end (the constant terms are
// added by the column's thread), and the full per-step reduction runs only
// every kCheckEvery steps and at the last step for the |mu| <= 1 check (the
// norm of j_n grows monotonically once a is too small); on GB300, where FP64
// runs at 1/64 of the FP32 rate, the shuffle tree of every step would cost as
// much as the stencil.  FP32 without moment output folds linearly too, its
// per-thread shares in compensated FP32 (the coefficients' FP32 copy times
// the FP32 partial sums), so that no single folding thread sits on the
// critical path of every step.  No vector traffic reaches HBM; for the 16 x 16
// lattice a self-consistency iteration becomes one recursion launch.
#include <algorithm>

#include "internal.h"

namespace cbdg {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kCheckEvery = 16;

template <typename S, int VEC>
struct alignas(sizeof(S) * VEC) Pack {
  S v[VEC];
};

// Per-thread share of a linear fold: plain FP64, or compensated FP32.
template <typename S>
struct LinAcc {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct LinAcc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

struct ResidentArgs {
  const void *j0, *j1;  // slab-blocked [ld / W][2N][W] (global), from init_real
  const void *params;   // [N][kParamStride]
  const double *C;      // [M]
  const double *mu1;    // [ld]
  const double2 *dA;    // [ld]
  double *acc_n;        // [ld]
  double2 *acc_d;       // [ld]
  double *mu_ee;        // [ncols][M] or null
  double2 *mu_eh;       // [ncols][M][mom_stride] or null
  int mom_stride;
  unsigned int *flags;
  double tol;
  int Lx, Ly, M, steps, ncols;
};

template <typename S, int W, bool LINEAR>
__global__ void __launch_bounds__(kThreads) resident_kernel(ResidentArgs a) {
  constexpr int VEC = (W * sizeof(S) >= 16) ? 16 / static_cast<int>(sizeof(S)) : W;
  constexpr int QUADS = W / VEC, XS = kThreads / QUADS;
  using P = Pack<S, VEC>;
  const int Lx = a.Lx, Ly = a.Ly, N = Lx * Ly, M = a.M;
  const size_t slab_el = static_cast<size_t>(2) * N * W;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *Cs = reinterpret_cast<double *>(smem_raw);                       // [M]
  double *wred = Cs + M;                                                   // [2][kWarps][3][W]
  S *bp = reinterpret_cast<S *>(wred + 2 * kWarps * 3 * W);                // j_{n-1} -> j_{n+1}
  S *bq = bp + slab_el;                                                    // j_n
  S *par = bq + slab_el;                                                   // [N][kParamStride]
  S *Cf = par + static_cast<size_t>(N) * kParamStride;                     // [M] C in S precision

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int q = t % QUADS, ts = t / QUADS;
  const size_t c0 = static_cast<size_t>(blockIdx.x) * W;
  {
    const S *g0 = static_cast<const S *>(a.j0) + blockIdx.x * slab_el;
    const S *g1 = static_cast<const S *>(a.j1) + blockIdx.x * slab_el;
    for (size_t k = t; k < slab_el; k += kThreads) {
      bp[k] = g0[k];
      bq[k] = g1[k];
    }
    const S *gp = static_cast<const S *>(a.params);
    for (size_t k = t; k < static_cast<size_t>(N) * kParamStride; k += kThreads) par[k] = gp[k];
    for (int k = t; k < M; k += kThreads) {
      Cs[k] = a.C[k];
      Cf[k] = static_cast<S>(a.C[k]);
    }
  }
  // the fold state of column t (threads t < W)
  const int col = static_cast<int>(c0) + t;
  const bool folder = t < W && col < a.ncols;
  double an = 0.0, m1 = 0.0;
  double2 ad = make_double2(0.0, 0.0), da = make_double2(0.0, 0.0);
  if (folder) {
    an = a.acc_n[col];
    ad = a.acc_d[col];
    m1 = a.mu1[col];
    da = a.dA[col];
  }
  bool bad = false;
  LinAcc<S> ln[VEC], ld_[VEC];  // linear fold: this thread's share of acc_n and Re acc_d
  __syncthreads();

  S *prev = bp, *cur = bq;
  const int off = q * VEC, hb = Lx * W;
  for (int n = 1; n <= a.steps; ++n) {
    S pa[VEC], pb[VEC], pc[VEC];
#pragma unroll
    for (int l = 0; l < VEC; ++l) pa[l] = pb[l] = pc[l] = S(0);
    for (int s = ts; s < N; s += XS) {
      const int x = s % Lx, y = s / Lx;
      const int xr = (x + 1 == Lx) ? 0 : x + 1, xl = (x == 0) ? Lx - 1 : x - 1;
      const int yu = (y + 1 == Ly) ? 0 : y + 1, yd = (y == 0) ? Ly - 1 : y - 1;
      // rows: electron 2 Lx y + x, hole + Lx (zero hopping across open edges)
      const int rc = 2 * Lx * y, ru = 2 * Lx * yu, rd = 2 * Lx * yd;
      auto ld = [&](const S *b, int row) { return *reinterpret_cast<const P *>(b + row * W + off); };
      const P u = ld(cur, rc + x), v = ld(cur, rc + x + Lx);
      const P ur = ld(cur, rc + xr), vr = ld(cur, rc + xr + Lx);
      const P ul = ld(cur, rc + xl), vl = ld(cur, rc + xl + Lx);
      const P uu = ld(cur, ru + x), vu = ld(cur, ru + x + Lx);
      const P ud = ld(cur, rd + x), vd = ld(cur, rd + x + Lx);
      const P uo = ld(prev, rc + x), vo = ld(prev, rc + x + Lx);
      const S *pp = par + static_cast<size_t>(s) * kParamStride;
      const S e = pp[0], d = pp[1], t0 = pp[2], t1 = pp[3], t2 = pp[4], t3 = pp[5];
      P un, vn;
#pragma unroll
      for (int l = 0; l < VEC; ++l) {
        const S uj = u.v[l], vj = v.v[l];
        const S unj = fma_rn(e, uj, fma_rn(d, vj, -fma_rn(t3, ud.v[l], fma_rn(t2, uu.v[l],
                                                   fma_rn(t1, ul.v[l], fma_rn(t0, ur.v[l], uo.v[l]))))));
        const S vnj = fma_rn(d, uj, fma_rn(-e, vj, fma_rn(t3, vd.v[l], fma_rn(t2, vu.v[l],
                                                   fma_rn(t1, vl.v[l], fma_rn(t0, vr.v[l], -vo.v[l]))))));
        un.v[l] = unj;
        vn.v[l] = vnj;
        pa[l] = fma_rn(uj, uj, fma_rn(vj, vj, pa[l]));
        pb[l] = fma_rn(unj, uj, fma_rn(vnj, vj, pb[l]));
        pc[l] = fma_rn(unj, vj, fma_rn(-vnj, uj, pc[l]));
      }
      *reinterpret_cast<P *>(prev + (rc + x) * W + off) = un;
      *reinterpret_cast<P *>(prev + (rc + x + Lx) * W + off) = vn;
    }
    (void)hb;
    const int m0 = 2 * n, mo = 2 * n + 1;
    if (LINEAR) {
#pragma unroll
      for (int l = 0; l < VEC; ++l) {
        if (m0 < M) ln[l].add(S(-2) * Cf[m0] * pa[l]);
        if (mo < M) {
          ln[l].add(S(-2) * Cf[mo] * pb[l]);
          ld_[l].add(((n & 1) ? S(2) : S(-2)) * Cf[mo] * pc[l]);
        }
      }
    }
    const bool reduce = !LINEAR || n % kCheckEvery == 0 || n == a.steps;
    if (reduce) {
      // column sums: lanes with the same q hold the same columns
      double *wr = wred + static_cast<size_t>(n & 1) * kWarps * 3 * W + static_cast<size_t>(warp) * 3 * W;
#pragma unroll
      for (int l = 0; l < VEC; ++l) {
        S xa = pa[l], xb = pb[l], xc = pc[l];
#pragma unroll
        for (int o = QUADS; o < 32; o <<= 1) {
          xa += __shfl_xor_sync(0xffffffffu, xa, o);
          xb += __shfl_xor_sync(0xffffffffu, xb, o);
          if (!LINEAR) xc += __shfl_xor_sync(0xffffffffu, xc, o);
        }
        if (lane < QUADS) {
          wr[0 * W + off + l] = static_cast<double>(xa);
          wr[1 * W + off + l] = static_cast<double>(xb);
          wr[2 * W + off + l] = static_cast<double>(xc);
        }
      }
    }
    __syncthreads();  // j_{n+1} complete; this step's warp sums visible
    if (folder && reduce) {
      const double *wb = wred + static_cast<size_t>(n & 1) * kWarps * 3 * W;
      double A = 0.0, B = 0.0, Cc = 0.0;
      for (int w = 0; w < kWarps; ++w) {
        A += wb[(w * 3 + 0) * W + t];
        B += wb[(w * 3 + 1) * W + t];
        Cc += wb[(w * 3 + 2) * W + t];
      }
      const double e0 = 2.0 * A - 1.0;
      const double e1 = 2.0 * B - m1;
      const double sgn = (n & 1) ? 1.0 : -1.0;  // (-1)^(n+1)
      const double2 h1 = make_double2(2.0 * sgn * Cc - da.x, -da.y);
      if (m0 < M) {
        if (!LINEAR) an -= Cs[m0] * e0;
        bad |= fabs(e0) > 1.0 + a.tol;
        if (a.mu_ee) a.mu_ee[static_cast<size_t>(col) * M + m0] = e0;
        if (a.mu_eh) a.mu_eh[(static_cast<size_t>(col) * M + m0) * a.mom_stride] = make_double2(0.0, 0.0);
      }
      if (mo < M) {
        if (!LINEAR) {
          an -= Cs[mo] * e1;
          ad.x += Cs[mo] * h1.x;
          ad.y -= Cs[mo] * h1.y;
        }
        bad |= fabs(e1) > 1.0 + a.tol;
        if (a.mu_ee) a.mu_ee[static_cast<size_t>(col) * M + mo] = e1;
        if (a.mu_eh) a.mu_eh[(static_cast<size_t>(col) * M + mo) * a.mom_stride] = h1;
      }
      if (!(fabs(e0) < 1e300) || !(fabs(e1) < 1e300)) bad = true;  // NaN / inf
    }
    S *tmp = prev;
    prev = cur;
    cur = tmp;
  }
  if (LINEAR) {
    __syncthreads();  // the last check's sums have been read before wred is reused
    // per-column totals of the per-thread shares, then the constant terms:
    //   acc_n += sum_{2n<M} C_2n + mu_1 sum_{2n+1<M} C_2n+1,
    //   acc_d -= (Delta/a) sum_{2n+1<M} C_2n+1 (as in fold_kernel's h1)
    double *wr = wred + static_cast<size_t>(warp) * 3 * W;
#pragma unroll
    for (int l = 0; l < VEC; ++l) {
      double xn = ln[l].value(), xd = ld_[l].value();
#pragma unroll
      for (int o = QUADS; o < 32; o <<= 1) {
        xn += __shfl_xor_sync(0xffffffffu, xn, o);
        xd += __shfl_xor_sync(0xffffffffu, xd, o);
      }
      if (lane < QUADS) {
        wr[0 * W + off + l] = xn;
        wr[1 * W + off + l] = xd;
      }
    }
    __syncthreads();
    if (folder) {
      double sn = 0.0, sd = 0.0, c_even = 0.0, c_odd = 0.0;
      for (int w = 0; w < kWarps; ++w) {
        sn += wred[(w * 3 + 0) * W + t];
        sd += wred[(w * 3 + 1) * W + t];
      }
      for (int n = 1; n <= a.steps; ++n) {
        if (2 * n < M) c_even += Cs[2 * n];
        if (2 * n + 1 < M) c_odd += Cs[2 * n + 1];
      }
      an += sn + c_even + m1 * c_odd;
      ad.x += sd - da.x * c_odd;
      ad.y += da.y * c_odd;
    }
  }
  if (folder) {
    a.acc_n[col] = an;
    a.acc_d[col] = ad;
    if (bad) atomicOr(a.flags, kFlagSpectrum);
  }
}

template <typename S, int W>
size_t smem_bytes(int N, int M) {
  return static_cast<size_t>(M) * 8 + static_cast<size_t>(2) * kWarps * 3 * W * 8 +
         (static_cast<size_t>(4) * N * W + static_cast<size_t>(N) * kParamStride + M) * sizeof(S);
}

constexpr size_t kMaxSmem = 227 * 1024 - 1024;

template <typename S, int W, bool LINEAR>
cudaError_t launch_one(const ResidentArgs &a, int ld, cudaStream_t s) {
  const size_t smem = smem_bytes<S, W>(a.Lx * a.Ly, a.M);
  auto k = resident_kernel<S, W, LINEAR>;
  static int attr_dev = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (attr_dev != dev) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kMaxSmem));
    if (e != cudaSuccess) return e;
    attr_dev = dev;
  }
  k<<<ld / W, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

// Without moment output the fold is linear (see above); with it, per step.
template <typename S, int W>
cudaError_t launch_w(const ResidentArgs &a, int ld, cudaStream_t s) {
  if (!a.mu_ee && !a.mu_eh) return launch_one<S, W, true>(a, ld, s);
  return launch_one<S, W, false>(a, ld, s);
}

size_t smem_for(int precision, int W, int N, int M) {
  if (precision == 1) {
    switch (W) {
      case 1: return smem_bytes<float, 1>(N, M);
      case 2: return smem_bytes<float, 2>(N, M);
      case 4: return smem_bytes<float, 4>(N, M);
    }
  } else {
    switch (W) {
      case 1: return smem_bytes<double, 1>(N, M);
      case 2: return smem_bytes<double, 2>(N, M);
      case 4: return smem_bytes<double, 4>(N, M);
    }
  }
  return 0;
}

}  // namespace

int plan_resident(int precision, int Lx, int Ly, int ncols, int M) {
  // the widest slab that still gives one CTA per SM of 152 (or as close as
  // ncols allows) and fits in shared memory; 0 when no slab width fits
  const int N = Lx * Ly;
  for (int W : {4, 2, 1}) {
    if (W > 1 && (ncols + W - 1) / W < 152) continue;
    const size_t b = smem_for(precision, W, N, M);
    if (b != 0 && b <= kMaxSmem) return W;
  }
  return 0;
}

cudaError_t launch_resident(int precision, int W, int Lx, int Ly, int ld, int ncols, int M, int steps,
                            const void *j0, const void *j1, const void *params, const double *C,
                            const double *mu1, const double2 *dA, double *acc_n, double2 *acc_d,
                            double *mu_ee, double2 *mu_eh, int mom_stride, unsigned int *flags, double tol,
                            cudaStream_t s) {
  ResidentArgs a{j0, j1, params, C, mu1, dA, acc_n, acc_d, mu_ee, mu_eh, mom_stride, flags, tol,
                 Lx, Ly, M, steps, ncols};
  if (precision == 1) {
    switch (W) {
      case 1: return launch_w<float, 1>(a, ld, s);
      case 2: return launch_w<float, 2>(a, ld, s);
      case 4: return launch_w<float, 4>(a, ld, s);
    }
  } else {
    switch (W) {
      case 1: return launch_w<double, 1>(a, ld, s);
      case 2: return launch_w<double, 2>(a, ld, s);
      case 4: return launch_w<double, 4>(a, ld, s);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace cbdg
