// adjoint_cplx.cu -- reverse-mode gradient of one self-consistency map
// Delta_out(eps, t, Delta_in) (Eq. 19 through the recursion of Eq. 15) for
// general lattices: complex hoppings with Peierls phases, next-nearest
// neighbours, on-site or nearest-neighbour bond pairing (Eq. 2), with a and
// the coefficients C_n frozen.
//
// For a real loss L with g = dL/dRe Delta_out + i dL/dIm Delta_out, L changes
// by Re sum_k conj(g_k) dDelta_out,k.  The start column of site i carries
//   on-site: Delta_out,i = (U_i/2) sum_m C_m conj(<h_i|j_m>): source
//            y_m(h_i) = (U_i/2) C_m conj(g_i);
//   bond:    <h_j|j_m> (j = i + d, d < 4) enters Delta_out,(i,d) and
//            Delta_out,(j,d^1) with weight (V/8) C_m each (the symmetrised
//            singlet): y_m(h_j) = (C_m/8) conj(V_{i,d} g_{i,d} + V_{j,d^1} g_{j,d^1}).
// With Phi = Re sum_m <y_m|j_m>, the adjoint vectors follow the recursion of
// the forward step (H~ is Hermitian),
//   lam_m = y_m + 2 H~ lam_{m+1} - lam_{m+2},
// and dPhi = Re sum_rs G_rs dH~_rs with
//   G_rs = sum_{m >= 1} f_m conj(lam_m(r)) j_{m-1}(s),  f_1 = 1, f_m = 2,
// needed only where Eq. 2 has entries.  This file holds the source scatter,
// the pattern-restricted accumulation of G (per site: the on-site block
// e-e, h-h, e-h, h-e; per direction d the hoppings e_i-e_j and h_i-h_j; per
// nearest-neighbour direction with bond pairing e_i-h_j and h_i-e_j; summed
// over the columns of a group in a fixed order, no atomics) and the
// contraction with dH/dparameter, giving complex gradients dL/dRe + i dL/dIm:
//   eps_i:       H_{e_i e_i} = eps - mu, H_{h_i h_i} = -(eps - mu)
//   t_{i,d}:     H_{e_i e_j} = -t, H_{h_i h_j} = conj(t), mirror H_{e_j e_i} =
//                -conj(t), H_{h_j h_i} = t (the mirror entry t_{j,d^1} =
//                conj(t) gets the conjugate gradient)
//   Delta_i:     H_{e_i h_i} = Delta, H_{h_i e_i} = conj(Delta)
//   Delta_{i,d}: H_{e_i h_j} = H_{e_j h_i} = Delta, H_{h_i e_j} = H_{h_j e_i}
//                = conj(Delta) (symmetric; stored on both directed entries).
// Vectors are complex (float2 / double2 pairs) in the slab-blocked layout of
// the step kernels.
#include <algorithm>

#include "internal.h"

namespace cbdg {
namespace {

inline int blocks(long long n, int t) { return static_cast<int>((n + t - 1) / t); }

// Column b's source at moment m: lam(row) += C_m * w.
template <typename S>
__global__ void adjoint_source_cplx_kernel(int Lx, int Ly, int px, int py, int ncols, int W, const int32_t *sites,
                                           int pairing, const double2 *g, const double *cpl, double coupling,
                                           double Cm, S *lam) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= ncols) return;
  const int i = sites[b];
  const size_t rows = 2 * static_cast<size_t>(Lx) * Ly;
  auto add = [&](int site, double wr, double wi) {
    const size_t k = 2 * blocked_index(vector_row(Lx, site, 1), b, rows, W);
    lam[k] = static_cast<S>(static_cast<double>(lam[k]) + Cm * wr);
    lam[k + 1] = static_cast<S>(static_cast<double>(lam[k + 1]) + Cm * wi);
  };
  if (pairing == 0) {
    const double u = 0.5 * (cpl ? cpl[i] : coupling);
    const double2 gi = g[i];
    add(i, u * gi.x, -u * gi.y);
    return;
  }
  for (int d = 0; d < 4; ++d) {
    const int j = neighbour_site(Lx, Ly, px, py, i, d);
    if (j < 0) continue;
    const double v1 = cpl ? cpl[static_cast<size_t>(i) * 4 + d] : coupling;
    const double v2 = cpl ? cpl[static_cast<size_t>(j) * 4 + (d ^ 1)] : coupling;
    const double2 g1 = g[static_cast<size_t>(i) * 4 + d], g2 = g[static_cast<size_t>(j) * 4 + (d ^ 1)];
    const double sr = v1 * g1.x + v2 * g2.x, si = v1 * g1.y + v2 * g2.y;
    add(j, 0.125 * sr, -0.125 * si);
  }
}

// Compensated (FP32) or plain (FP64) sum.
template <typename S>
struct Sum {
  S s = 0;
  __device__ __forceinline__ void add(S x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct Sum<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Sums per site: 0 e-e, 1 h-h, 2 e-h, 3 h-e (on site), 4 + 2d / 5 + 2d the
// hoppings e_i-e_j / h_i-h_j of direction d < nd, 4 + 2 nd + 2d / 5 + 2 nd + 2d
// the bond entries e_i-h_j / h_i-e_j of direction d < 4 (bond pairing).
__host__ __device__ inline int cplx_sums(int nd, int bond) { return 4 + 2 * nd + (bond ? 8 : 0); }

// part[g][site][2 k + {re, im}] += f * sum_{b in group g} conj(lam(r, b)) j(s, b).
// Grid (Ly, groups); group g covers column slabs [g * spg, (g + 1) * spg).
// One thread per (site, column lane); the W lanes of a site are adjacent and
// combine by warp shuffles in FP64.
template <typename S, int W, int NDIR, bool BOND>
__global__ void __launch_bounds__(256) adjoint_accumulate_cplx_kernel(int Lx, int Ly, int px, int py, int ld,
                                                                      int spg, const S *__restrict__ lam,
                                                                      const S *__restrict__ j, double f,
                                                                      double *part) {
  constexpr int KC = 4 + 2 * NDIR + (BOND ? 8 : 0);
  constexpr int XS = 256 / W;
  const int N = Lx * Ly, y = blockIdx.x, g = blockIdx.y;
  const int t = threadIdx.x, lane = t % W, xs = t / W;
  const size_t slab_el = static_cast<size_t>(2) * N * W;  // complex elements of one slab
  const int s0 = g * spg, s1 = min(ld / W, s0 + spg);
  for (int xb = 0; xb < Lx; xb += XS) {  // uniform over the block: every lane reaches the shuffles
    const int x = xb + xs;
    const bool valid = x < Lx;
    const int i = y * Lx + (valid ? x : 0);
    int nb[NDIR];
#pragma unroll
    for (int d = 0; d < NDIR; ++d) nb[d] = valid ? neighbour_site(Lx, Ly, px, py, i, d) : -1;
    Sum<S> re[KC], im[KC];
    if (valid) {
      for (int c = s0; c < s1; ++c) {
        const S *lb = lam + 2 * (c * slab_el), *jb = j + 2 * (c * slab_el);
        auto ld2 = [&](const S *base, int site, int part, S &r, S &m) {
          const size_t k = 2 * (vector_row(Lx, site, part) * W + lane);
          r = base[k];
          m = base[k + 1];
        };
        S ler, lei, lhr, lhi, jer, jei, jhr, jhi;
        ld2(lb, i, 0, ler, lei);
        ld2(lb, i, 1, lhr, lhi);
        ld2(jb, i, 0, jer, jei);
        ld2(jb, i, 1, jhr, jhi);
        // conj(l) * v = (lr vr + li vi) + i (lr vi - li vr)
        auto acc = [&](int k, S lr, S li, S vr, S vi) {
          re[k].add(fma(lr, vr, li * vi));
          im[k].add(fma(lr, vi, -li * vr));
        };
        acc(0, ler, lei, jer, jei);
        acc(1, lhr, lhi, jhr, jhi);
        acc(2, ler, lei, jhr, jhi);
        acc(3, lhr, lhi, jer, jei);
#pragma unroll
        for (int d = 0; d < NDIR; ++d) {
          if (nb[d] < 0) continue;
          S ner, nei, nhr, nhi;
          ld2(jb, nb[d], 0, ner, nei);
          ld2(jb, nb[d], 1, nhr, nhi);
          acc(4 + 2 * d, ler, lei, ner, nei);
          acc(5 + 2 * d, lhr, lhi, nhr, nhi);
          if (BOND && d < 4) {
            acc(4 + 2 * NDIR + 2 * d, ler, lei, nhr, nhi);
            acc(5 + 2 * NDIR + 2 * d, lhr, lhi, ner, nei);
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      double vr = re[k].value(), vi = im[k].value();
#pragma unroll
      for (int o = 1; o < W; o <<= 1) {
        vr += __shfl_xor_sync(0xffffffffu, vr, o);
        vi += __shfl_xor_sync(0xffffffffu, vi, o);
      }
      if (valid && lane == 0) {
        double *pp = part + (static_cast<size_t>(g) * N + i) * 2 * KC + 2 * k;
        pp[0] += f * vr;
        pp[1] += f * vi;
      }
    }
  }
}

// FP32 accumulation with staged rows (slab width 4): one CTA per (lattice
// row y, block of up to kCaXB sites of it, group of column slabs), one thread
// per (site, column).  Per slab, bulk copies (cp.async.bulk on mbarriers)
// bring the lam row y and the j rows y - 1, y, y + 1 (whole rows, electron
// then hole part) into one stage of a kCaStages ring; the sums read every
// neighbour from shared memory.  The sums are plain FP32 over at most
// kCaMaxSpg slabs per launch (relative error below kCaMaxSpg 2^-24 of the sum
// of |terms|), then FP64.
constexpr int kCaW = 4, kCaXB = 64, kCaThreads = kCaW * kCaXB, kCaStages = 3, kCaMaxSpg = 64;
constexpr int kCaSite = kCaW * 2;  // floats of one site's W complex entries

__device__ __forceinline__ unsigned ca_smem_addr(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ bool ca_mbar_wait(unsigned bar, unsigned parity, unsigned long long limit_ns) {
  auto try_once = [&]() {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
  };
  if (try_once()) return true;
  unsigned long long t0;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t0));
  for (unsigned it = 0;; ++it) {
    if (try_once()) return true;
    if ((it & 255u) == 255u) {
      unsigned long long t1;
      asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t1));
      if (t1 - t0 > limit_ns) return false;
    }
  }
}

template <int NDIR, bool BOND>
__global__ void __launch_bounds__(kCaThreads) adjoint_accumulate_cplx_staged_kernel(
    int Lx, int Ly, int px, int py, int ld, int spg, int nxb, const float *__restrict__ lam,
    const float *__restrict__ j, double f, double *part, unsigned long long wait_ns, unsigned *flags) {
  constexpr int KC = 4 + 2 * NDIR + (BOND ? 8 : 0), W = kCaW, R = kCaStages;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long bars[R];
  __shared__ int abort_flag;
  float *sm = reinterpret_cast<float *>(smem_raw);
  const int N = Lx * Ly, y = blockIdx.x / nxb, g = blockIdx.y;
  const int t = threadIdx.x, lane = t % W, x = (blockIdx.x % nxb) * kCaXB + t / W;
  const bool valid = x < Lx;
  const size_t slab_el = static_cast<size_t>(2) * N * kCaSite;  // floats of one slab
  const int rowf = 2 * Lx * kCaSite;                            // floats of one lattice row
  const int s0 = g * spg, ns = min(ld / W, s0 + spg) - s0;
  // staged rows: 0 lam y, 1 j y-1, 2 j y, 3 j y+1 (-1: beyond an open edge)
  const int yrow[4] = {y, y > 0 ? y - 1 : (py ? Ly - 1 : -1), y, y + 1 < Ly ? y + 1 : (py ? 0 : -1)};
  if (t == 0) {
    for (int k = 0; k < R; ++k)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(ca_smem_addr(&bars[k])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    abort_flag = 0;
  }
  __syncthreads();
  const unsigned row_bytes = static_cast<unsigned>(rowf) * 4u;
  const unsigned stage_bytes = row_bytes * (2u + (yrow[1] >= 0 ? 1u : 0u) + (yrow[3] >= 0 ? 1u : 0u));
  auto issue = [&](int i) {
    const int st = i % R;
    const unsigned bar = ca_smem_addr(&bars[st]);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(stage_bytes) : "memory");
    for (int r = 0; r < 4; ++r) {
      if (yrow[r] < 0) continue;
      const float *src = (r == 0 ? lam : j) + static_cast<size_t>(s0 + i) * slab_el + static_cast<size_t>(yrow[r]) * rowf;
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
              ca_smem_addr(sm + (static_cast<size_t>(st) * 4 + r) * rowf)),
          "l"(src), "r"(row_bytes), "r"(bar)
          : "memory");
    }
  };
  int issued = min(ns, R);
  if (t == 0)
    for (int i = 0; i < issued; ++i) issue(i);
  // neighbour d of this thread's site: offset in a stage (row y + dy, site x + dx), -1: none
  int noff[NDIR];
#pragma unroll
  for (int d = 0; d < NDIR; ++d) {
    const int dx = (d == 0 || d == 4 || d == 6) ? 1 : (d == 1 || d == 5 || d == 7) ? -1 : 0;
    const int dy = (d == 2 || d == 4 || d == 7) ? 1 : (d == 3 || d == 5 || d == 6) ? -1 : 0;
    const bool ok = valid && neighbour_site(Lx, Ly, px, py, y * Lx + x, d) >= 0;
    const int nx = (x + dx + Lx) % Lx;
    noff[d] = ok ? (2 + dy) * rowf + nx * kCaSite + 2 * lane : -1;
  }
  float re[KC], im[KC];
#pragma unroll
  for (int k = 0; k < KC; ++k) re[k] = im[k] = 0.f;
  const int own = x * kCaSite + 2 * lane, hp = Lx * kCaSite;  // hole part offset within a row
  int landed = 0;  // slabs whose copies have all landed
  for (int i = 0; i < ns; ++i) {
    const int st = i % R;
    if (!ca_mbar_wait(ca_smem_addr(&bars[st]), static_cast<unsigned>((i / R) & 1), wait_ns)) abort_flag = 1;
    __syncthreads();
    if (abort_flag) break;
    landed = i + 1;
    if (valid) {
      const float *d = sm + static_cast<size_t>(st) * 4 * rowf;
      auto ld2 = [&](int off) { return *reinterpret_cast<const float2 *>(d + off); };
      const float2 le = ld2(own), lh = ld2(own + hp), je = ld2(2 * rowf + own), jh = ld2(2 * rowf + own + hp);
      // conj(l) v = (lr vr + li vi) + i (lr vi - li vr)
      auto acc = [&](int k, float2 l, float2 v) {
        re[k] = fmaf(l.x, v.x, fmaf(l.y, v.y, re[k]));
        im[k] = fmaf(l.x, v.y, fmaf(-l.y, v.x, im[k]));
      };
      acc(0, le, je);
      acc(1, lh, jh);
      acc(2, le, jh);
      acc(3, lh, je);
#pragma unroll
      for (int dd = 0; dd < NDIR; ++dd) {
        if (noff[dd] < 0) continue;
        const float2 ne = ld2(noff[dd]), nh = ld2(noff[dd] + hp);
        acc(4 + 2 * dd, le, ne);
        acc(5 + 2 * dd, lh, nh);
        if (BOND && dd < 4) {
          acc(4 + 2 * NDIR + 2 * dd, le, nh);
          acc(5 + 2 * NDIR + 2 * dd, lh, ne);
        }
      }
    }
    __syncthreads();  // stage st is free
    if (i + R < ns) {
      if (t == 0) issue(i + R);
      issued = i + R + 1;
    }
  }
  if (abort_flag) {
    if (t == 0) {
      atomicOr(flags, kFlagTimeout);
      // let the copies in flight land before the CTA's shared memory goes away
      for (int i = landed; i < issued; ++i)
        if (!ca_mbar_wait(ca_smem_addr(&bars[i % R]), static_cast<unsigned>((i / R) & 1), wait_ns)) break;
    }
    return;
  }
  // combine the W column lanes of each site (adjacent lanes), FP64
#pragma unroll
  for (int k = 0; k < KC; ++k) {
    double vr = re[k], vi = im[k];
#pragma unroll
    for (int o = 1; o < W; o <<= 1) {
      vr += __shfl_xor_sync(0xffffffffu, vr, o);
      vi += __shfl_xor_sync(0xffffffffu, vi, o);
    }
    if (valid && lane == 0) {
      double *pp = part + (static_cast<size_t>(g) * N + static_cast<size_t>(y) * Lx + x) * 2 * KC + 2 * k;
      pp[0] += f * vr;
      pp[1] += f * vi;
    }
  }
}

__global__ void adjoint_final_cplx_kernel(int Lx, int Ly, int px, int py, int nd, int bond, int groups,
                                          const double *part, const double *scal, double *g_eps, double2 *g_hop,
                                          double2 *g_delta) {
  const int N = Lx * Ly;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int KC = cplx_sums(nd, bond);
  const double a = scal[kScalA];
  auto G = [&](int site, int k) {
    double r = 0.0, m = 0.0;
    for (int g = 0; g < groups; ++g) {
      const double *pp = part + (static_cast<size_t>(g) * N + site) * 2 * KC + 2 * k;
      r += pp[0];
      m += pp[1];
    }
    return make_double2(r, m);
  };
  const double2 ee = G(i, 0), hh = G(i, 1);
  if (g_eps) g_eps[i] = (ee.x - hh.x) / a;
  if (!bond && g_delta) {
    const double2 eh = G(i, 2), he = G(i, 3);
    g_delta[i] = make_double2((eh.x + he.x) / a, (he.y - eh.y) / a);
  }
  for (int d = 0; d < nd; ++d) {
    const int j = neighbour_site(Lx, Ly, px, py, i, d);
    if (j < 0) {
      if (g_hop) g_hop[static_cast<size_t>(i) * nd + d] = make_double2(0.0, 0.0);
      if (bond && d < 4 && g_delta) g_delta[static_cast<size_t>(i) * 4 + d] = make_double2(0.0, 0.0);
      continue;
    }
    const int db = d ^ 1;
    if (g_hop) {
      const double2 a1 = G(i, 4 + 2 * d), a2 = G(i, 5 + 2 * d), a3 = G(j, 4 + 2 * db), a4 = G(j, 5 + 2 * db);
      g_hop[static_cast<size_t>(i) * nd + d] =
          make_double2((-a1.x + a2.x - a3.x + a4.x) / a, (a1.y + a2.y - a3.y - a4.y) / a);
    }
    if (bond && d < 4 && g_delta) {
      const double2 b1 = G(i, 4 + 2 * nd + 2 * d), b3 = G(i, 5 + 2 * nd + 2 * d);
      const double2 b2 = G(j, 4 + 2 * nd + 2 * db), b4 = G(j, 5 + 2 * nd + 2 * db);
      g_delta[static_cast<size_t>(i) * 4 + d] =
          make_double2((b1.x + b2.x + b3.x + b4.x) / a, (-b1.y - b2.y + b3.y + b4.y) / a);
    }
  }
}

template <typename S, int W, int NDIR, bool BOND>
cudaError_t accumulate_c(int Lx, int Ly, int px, int py, int ld, int groups, const void *lam, const void *j,
                         double f, double *part, cudaStream_t s) {
  const int slabs = ld / W;
  const int spg = (slabs + groups - 1) / groups;
  adjoint_accumulate_cplx_kernel<S, W, NDIR, BOND><<<dim3(Ly, groups), 256, 0, s>>>(
      Lx, Ly, px, py, ld, spg, static_cast<const S *>(lam), static_cast<const S *>(j), f, part);
  return cudaGetLastError();
}

template <typename S, int W>
cudaError_t accumulate_kind(int Lx, int Ly, int px, int py, int nd, int bond, int ld, int groups, const void *lam,
                            const void *j, double f, double *part, cudaStream_t s) {
  if (nd == 8)
    return bond ? accumulate_c<S, W, 8, true>(Lx, Ly, px, py, ld, groups, lam, j, f, part, s)
                : accumulate_c<S, W, 8, false>(Lx, Ly, px, py, ld, groups, lam, j, f, part, s);
  return bond ? accumulate_c<S, W, 4, true>(Lx, Ly, px, py, ld, groups, lam, j, f, part, s)
              : accumulate_c<S, W, 4, false>(Lx, Ly, px, py, ld, groups, lam, j, f, part, s);
}

size_t cplx_staged_smem(int Lx) { return static_cast<size_t>(kCaStages) * 4 * 2 * Lx * kCaSite * sizeof(float); }
bool cplx_staged(int precision, int Lx, int W) {
  return precision == 1 && W == kCaW && cplx_staged_smem(Lx) <= 200 * 1024;
}

template <int NDIR, bool BOND>
cudaError_t launch_cplx_staged(int Lx, int Ly, int px, int py, int ld, int groups, const void *lam, const void *j,
                               double f, double *part, unsigned long long wait_ns, unsigned *flags, cudaStream_t s) {
  auto k = adjoint_accumulate_cplx_staged_kernel<NDIR, BOND>;
  static int attr_dev = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (attr_dev != dev) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr_dev = dev;
  }
  const int slabs = ld / kCaW, spg = (slabs + groups - 1) / groups, nxb = (Lx + kCaXB - 1) / kCaXB;
  k<<<dim3(Ly * nxb, groups), kCaThreads, cplx_staged_smem(Lx), s>>>(
      Lx, Ly, px, py, ld, spg, nxb, static_cast<const float *>(lam), static_cast<const float *>(j), f, part, wait_ns,
      flags);
  return cudaGetLastError();
}

}  // namespace

int adjoint_cplx_sums(int nd, int bond) { return cplx_sums(nd, bond); }

int adjoint_groups_cplx(int precision, int Lx, int Ly, int ld, int W) {
  if (!cplx_staged(precision, Lx, W)) return adjoint_groups(Ly, ld, W);
  // at most kCaMaxSpg slabs per group (the FP32 sums' error bound); among
  // those, the group count whose CTAs (two resident per SM at 128 registers a
  // thread) run in the fewest waves x slabs per group
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long slots = 2LL * sms;
  const int slabs = std::max(1, ld / W), rows = Ly * ((Lx + kCaXB - 1) / kCaXB);
  const int gmin = (slabs + kCaMaxSpg - 1) / kCaMaxSpg, gmax = std::max(gmin, std::min(slabs, 4 * gmin));
  int best = gmin;
  long long best_cost = -1;
  for (int g = gmin; g <= gmax; ++g) {
    const long long spg = (slabs + g - 1) / g;
    const long long cost = ((static_cast<long long>(rows) * g + slots - 1) / slots) * spg;
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = g;
    }
  }
  return best;
}

cudaError_t launch_adjoint_source_cplx(int precision, int Lx, int Ly, int px, int py, int ncols, int W,
                                       const int32_t *sites, int pairing, const double2 *g, const double *cpl,
                                       double coupling, double Cm, void *lam, cudaStream_t s) {
  if (ncols <= 0) return cudaSuccess;
  if (precision == 1)
    adjoint_source_cplx_kernel<float><<<blocks(ncols, 128), 128, 0, s>>>(
        Lx, Ly, px, py, ncols, W, sites, pairing, g, cpl, coupling, Cm, static_cast<float *>(lam));
  else
    adjoint_source_cplx_kernel<double><<<blocks(ncols, 128), 128, 0, s>>>(
        Lx, Ly, px, py, ncols, W, sites, pairing, g, cpl, coupling, Cm, static_cast<double *>(lam));
  return cudaGetLastError();
}

cudaError_t launch_adjoint_accumulate_cplx(int precision, int Lx, int Ly, int px, int py, int nd, int bond, int ld,
                                           int W, int groups, const void *lam, const void *j, double f, double *part,
                                           unsigned long long wait_ns, unsigned *flags, cudaStream_t s) {
  if (cplx_staged(precision, Lx, W)) {
    if (nd == 8)
      return bond ? launch_cplx_staged<8, true>(Lx, Ly, px, py, ld, groups, lam, j, f, part, wait_ns, flags, s)
                  : launch_cplx_staged<8, false>(Lx, Ly, px, py, ld, groups, lam, j, f, part, wait_ns, flags, s);
    return bond ? launch_cplx_staged<4, true>(Lx, Ly, px, py, ld, groups, lam, j, f, part, wait_ns, flags, s)
                : launch_cplx_staged<4, false>(Lx, Ly, px, py, ld, groups, lam, j, f, part, wait_ns, flags, s);
  }
  if (precision == 1) {
    switch (W) {
      case 1: return accumulate_kind<float, 1>(Lx, Ly, px, py, nd, bond, ld, groups, lam, j, f, part, s);
      case 2: return accumulate_kind<float, 2>(Lx, Ly, px, py, nd, bond, ld, groups, lam, j, f, part, s);
      case 4: return accumulate_kind<float, 4>(Lx, Ly, px, py, nd, bond, ld, groups, lam, j, f, part, s);
      case 8: return accumulate_kind<float, 8>(Lx, Ly, px, py, nd, bond, ld, groups, lam, j, f, part, s);
    }
  } else {
    switch (W) {
      case 1: return accumulate_kind<double, 1>(Lx, Ly, px, py, nd, bond, ld, groups, lam, j, f, part, s);
      case 2: return accumulate_kind<double, 2>(Lx, Ly, px, py, nd, bond, ld, groups, lam, j, f, part, s);
      case 4: return accumulate_kind<double, 4>(Lx, Ly, px, py, nd, bond, ld, groups, lam, j, f, part, s);
    }
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_adjoint_final_cplx(int Lx, int Ly, int px, int py, int nd, int bond, int groups,
                                      const double *part, const double *scal, double *g_eps, double2 *g_hop,
                                      double2 *g_delta, cudaStream_t s) {
  adjoint_final_cplx_kernel<<<blocks(Lx * Ly, 128), 128, 0, s>>>(Lx, Ly, px, py, nd, bond, groups, part, scal, g_eps,
                                                                 g_hop, g_delta);
  return cudaGetLastError();
}

}  // namespace cbdg
