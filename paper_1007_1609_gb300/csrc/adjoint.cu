// adjoint.cu -- reverse-mode gradient of one self-consistency map
// Delta_out(eps, t, Delta_in) (Eq. 19 through Eq. 15), with a and the
// coefficients C_n frozen, for real on-site (s-wave) lattices; and of a loss
// on the LDOS (Eq. 17), whose source sits on the electron row instead:
//     y_m = S[c][m] e_i,  S[c][m] = dL/dmu_m(i) (ldos.cu).
//
// For a start site i the forward recursion j_m = 2 H~ j_{m-1} - j_{m-2}
// (j_1 = H~ j_0, j_0 = e_i) feeds Phi = sum_i w_i (U/2) sum_m C_m <h_i|j_m>,
// w = dL/dDelta_out.  Its adjoint runs backwards,
//     lam_m = y_m + 2 H~ lam_{m+1} - lam_{m+2},   y_m = w_i (U/2) C_m h_i,
// (the same symmetric stencil as the forward step, plus a one-element source
// per column), and the gradient with respect to the matrix entries is
//     dPhi/dH~_rs = sum_columns sum_{m >= 1} f_m lam_m(r) j_{m-1}(s),
// f_1 = 1, f_m = 2 (m >= 2), needed only on the stencil pattern.  The
// vectors j_{m-1} come back segment by segment from checkpoints of
// (j_{kS}, j_{kS+1}) taken every S ~ sqrt(M) steps of the forward pass.
//
// This file holds the kernels: the source scatter, the pattern-restricted
// accumulation (12 sums per site: e-e, h-h, e-h, h-e on site and e-e, h-h
// to each of the 4 neighbours; fixed order, no atomics) and the final
// contraction with dH/dparameter.  The accumulation streams lattice rows of
// the slab-blocked vectors like the recursion kernels: a CTA owns one lattice
// row and a group of column slabs, a thread one site and VEC columns, every
// load is a coalesced 16-byte vector; FP32 vectors are summed in FP32 with
// Kahan compensation, FP64 vectors in FP64, and the column lanes of a site
// are combined by warp shuffles in FP64.
#include <algorithm>

#include "internal.h"

namespace cbdg {
namespace {

inline int blocks(long long n, int t) { return static_cast<int>((n + t - 1) / t); }

template <typename S>
__global__ void adjoint_source_kernel(int Lx, int Ly, int ncols, int W, const int32_t *sites,
                                      const double *w, const double *U_site, double scale_m, S *lam) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= ncols) return;
  const int i = sites[b];
  const size_t rows = 2 * static_cast<size_t>(Lx) * Ly;
  const size_t k = blocked_index(vector_row(Lx, i, 1), b, rows, W);
  const double wi = U_site ? w[i] * U_site[i] : w[i];
  lam[k] = static_cast<S>(static_cast<double>(lam[k]) + wi * scale_m);
}

// LDOS loss: lam(e_i) += src[b * M + m] for column b (start site i)
template <typename S>
__global__ void adjoint_source_table_kernel(int Lx, int Ly, int ncols, int W, const int32_t *sites,
                                            const double *src, int M, int m, S *lam) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= ncols) return;
  const int i = sites[b];
  const size_t rows = 2 * static_cast<size_t>(Lx) * Ly;
  const size_t k = blocked_index(vector_row(Lx, i, 0), b, rows, W);
  lam[k] = static_cast<S>(static_cast<double>(lam[k]) + src[static_cast<size_t>(b) * M + m]);
}

template <typename S>
struct SumOf {
  S s = 0;
  __device__ __forceinline__ void add(S x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct SumOf<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

template <typename S, int VEC>
struct alignas(sizeof(S) * VEC) Pack {
  S v[VEC];
};

// part[g][site][12] += f * sum_{b in group g} lam(r, b) j(s, b) on the pattern.
// Grid (Ly, groups); group g covers column slabs [g * spg, (g + 1) * spg).
template <typename S, int W>
__global__ void __launch_bounds__(256) adjoint_accumulate_kernel(int Lx, int Ly, int px, int py, int ld,
                                                                 int spg, const S *__restrict__ lam,
                                                                 const S *__restrict__ j, double f,
                                                                 double *part) {
  constexpr int VEC = (W * sizeof(S) >= 16) ? 16 / static_cast<int>(sizeof(S)) : W;
  constexpr int QUADS = W / VEC, XSLOTS = 256 / QUADS;
  using P = Pack<S, VEC>;
  const int N = Lx * Ly, y = blockIdx.x, g = blockIdx.y;
  const int t = threadIdx.x, q = t % QUADS, xs = t / QUADS;
  const size_t slab_el = static_cast<size_t>(2) * N * W;
  const int s0 = g * spg, s1 = min(ld / W, s0 + spg);
  const int off = q * VEC;
  for (int xb = 0; xb < Lx; xb += XSLOTS) {  // warp-uniform: the shuffles below need every lane
    const int x = xb + xs;
    const bool valid = x < Lx;
    int nx[4], ny[4];
    bool has[4];
    {
      const int DX[4] = {1, -1, 0, 0}, DY[4] = {0, 0, 1, -1};
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        int a = x + DX[d], b = y + DY[d];
        bool ok = valid;
        if (a < 0 || a >= Lx) {
          ok = ok && px != 0;
          a = (a + Lx) % Lx;
        }
        if (b < 0 || b >= Ly) {
          ok = ok && py != 0;
          b = (b + Ly) % Ly;
        }
        nx[d] = a;
        ny[d] = b;
        has[d] = ok;
      }
    }
    SumOf<S> acc[12];
    if (valid) {
      for (int c = s0; c < s1; ++c) {
        const S *lb = lam + c * slab_el, *jb = j + c * slab_el;
        const size_t re = static_cast<size_t>(2 * Lx * y + x) * W + off, rh = re + static_cast<size_t>(Lx) * W;
        const P le = *reinterpret_cast<const P *>(lb + re), lh = *reinterpret_cast<const P *>(lb + rh);
        const P je = *reinterpret_cast<const P *>(jb + re), jh = *reinterpret_cast<const P *>(jb + rh);
        // FP32: the VEC lane products of a sum first (cheap), then one
        // compensated add; FP64 (bound by its FMA rate): one FMA per product
        auto dot = [&](int k, const P &a, const P &b) {
          if constexpr (sizeof(S) == 8) {
#pragma unroll
            for (int l = 0; l < VEC; ++l) acc[k].s = fma(a.v[l], b.v[l], acc[k].s);
          } else {
            S p = a.v[0] * b.v[0];
#pragma unroll
            for (int l = 1; l < VEC; ++l) p = fmaf(a.v[l], b.v[l], p);
            acc[k].add(p);
          }
        };
        // every load of the slab first (one memory round trip per slab): a
        // missing neighbour reads the site itself and is not summed
        P de[4], dh[4];
#pragma unroll
        for (int d = 0; d < 4; ++d) {
          const size_t ne = has[d] ? static_cast<size_t>(2 * Lx * ny[d] + nx[d]) * W + off : re;
          de[d] = *reinterpret_cast<const P *>(jb + ne);
          dh[d] = *reinterpret_cast<const P *>(jb + ne + static_cast<size_t>(Lx) * W);
        }
        dot(0, le, je);
        dot(1, lh, jh);
        dot(2, le, jh);
        dot(3, lh, je);
#pragma unroll
        for (int d = 0; d < 4; ++d) {
          if (!has[d]) continue;
          dot(4 + d, le, de[d]);
          dot(8 + d, lh, dh[d]);
        }
      }
    }
    // combine the QUADS column lanes of each site (adjacent lanes), FP64
    double tot[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      double v = acc[k].value();
#pragma unroll
      for (int o = 1; o < QUADS; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      tot[k] = v;
    }
    if (valid && q == 0) {
      double *pp = part + (static_cast<size_t>(g) * N + static_cast<size_t>(y) * Lx + x) * 12;
#pragma unroll
      for (int k = 0; k < 12; ++k) pp[k] += f * tot[k];
    }
  }
}

// FP32 accumulation with staged rows: one CTA per (lattice row y, group of
// column slabs); per slab, bulk copies (cp.async.bulk on mbarriers) bring
// the lam row y and the j rows y-1, y, y+1 of that slab into one stage of a
// kAccStages ring, the copies of the next slabs in flight while the sums of
// this one read every neighbour from shared memory.  MAXX x slots per thread
// (Lx <= 64 MAXX); same sums, order and compensation as the unstaged kernel.
constexpr int kAccStages = 2, kAccThreads = 256, kAccW = 16;

__device__ __forceinline__ unsigned acc_smem_addr(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ bool acc_mbar_wait(unsigned bar, unsigned parity, unsigned long long limit_ns) {
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

template <int MAXX>
__global__ void __launch_bounds__(kAccThreads) adjoint_accumulate_staged_kernel(
    int Lx, int Ly, int px, int py, int ld, int spg, const float *__restrict__ lam, const float *__restrict__ j,
    double f, double *part, unsigned long long wait_ns, unsigned *flags) {
  constexpr int W = kAccW, VEC = 4, QUADS = W / VEC, XSLOTS = kAccThreads / QUADS, R = kAccStages;
  using P = Pack<float, VEC>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long bars[R];
  __shared__ int abort_flag;
  const int N = Lx * Ly, y = blockIdx.x, g = blockIdx.y;
  const int t = threadIdx.x, q = t % QUADS, xs = t / QUADS, off = q * VEC;
  const size_t slab_el = static_cast<size_t>(2) * N * W;
  const int rowel = 2 * Lx * W;  // floats of one lattice row: electron then hole part
  const int s0 = g * spg, ns = min(ld / W, s0 + spg) - s0;
  // rows y - 1 and y + 1 (-1: beyond an open edge)
  const int ym = y > 0 ? y - 1 : (py ? Ly - 1 : -1), yp = y + 1 < Ly ? y + 1 : (py ? 0 : -1);
  float *sm = reinterpret_cast<float *>(smem_raw);  // [R][4][rowel]: lam y, j y-1, j y, j y+1
  if (t == 0) {
    for (int k = 0; k < R; ++k)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(acc_smem_addr(&bars[k])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    abort_flag = 0;
  }
  __syncthreads();
  const unsigned row_bytes = static_cast<unsigned>(rowel) * 4u;
  auto copy = [&](float *dst, const float *src, unsigned bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            acc_smem_addr(dst)),
        "l"(src), "r"(row_bytes), "r"(bar)
        : "memory");
  };
  auto issue = [&](int i) {
    const int st = i % R;
    const unsigned bar = acc_smem_addr(&bars[st]);
    const unsigned n_rows = 2u + (ym >= 0 ? 1u : 0u) + (yp >= 0 ? 1u : 0u);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(n_rows * row_bytes)
                 : "memory");
    const float *lb = lam + (s0 + i) * slab_el, *jb = j + (s0 + i) * slab_el;
    float *d = sm + static_cast<size_t>(st) * 4 * rowel;
    copy(d, lb + static_cast<size_t>(y) * rowel, bar);
    copy(d + 2 * rowel, jb + static_cast<size_t>(y) * rowel, bar);
    if (ym >= 0) copy(d + rowel, jb + static_cast<size_t>(ym) * rowel, bar);
    if (yp >= 0) copy(d + 3 * rowel, jb + static_cast<size_t>(yp) * rowel, bar);
  };
  int issued = min(ns, R);
  if (t == 0)
    for (int i = 0; i < issued; ++i) issue(i);
  // neighbours along x of each x slot (-1: beyond an open edge)
  int xl[MAXX], xr[MAXX];
#pragma unroll
  for (int k = 0; k < MAXX; ++k) {
    const int x = xs + k * XSLOTS;
    xl[k] = x > 0 ? x - 1 : (px ? Lx - 1 : -1);
    xr[k] = x + 1 < Lx ? x + 1 : (px ? 0 : -1);
  }
  SumOf<float> acc[MAXX][12];
  auto dot = [](SumOf<float> &a, const P &u, const P &v) {
    float p = u.v[0] * v.v[0];
#pragma unroll
    for (int l = 1; l < VEC; ++l) p = fmaf(u.v[l], v.v[l], p);
    a.add(p);
  };
  const int hb = Lx * W;
  int landed = 0;  // slabs whose copies have all landed
  for (int i = 0; i < ns; ++i) {
    const int st = i % R;
    if (!acc_mbar_wait(acc_smem_addr(&bars[st]), static_cast<unsigned>((i / R) & 1), wait_ns)) abort_flag = 1;
    __syncthreads();
    if (abort_flag) break;
    landed = i + 1;
    const float *d = sm + static_cast<size_t>(st) * 4 * rowel;
    const float *sl = d, *jm = d + rowel, *jc = d + 2 * rowel, *jp = d + 3 * rowel;
#pragma unroll
    for (int k = 0; k < MAXX; ++k) {
      const int x = xs + k * XSLOTS;
      if (x >= Lx) continue;
      const int e = x * W + off;
      const P le = *reinterpret_cast<const P *>(sl + e), lh = *reinterpret_cast<const P *>(sl + hb + e);
      const P je = *reinterpret_cast<const P *>(jc + e), jh = *reinterpret_cast<const P *>(jc + hb + e);
      dot(acc[k][0], le, je);
      dot(acc[k][1], lh, jh);
      dot(acc[k][2], le, jh);
      dot(acc[k][3], lh, je);
      // directions +x, -x, +y, -y
      if (xr[k] >= 0) {
        const int n = xr[k] * W + off;
        dot(acc[k][4], le, *reinterpret_cast<const P *>(jc + n));
        dot(acc[k][8], lh, *reinterpret_cast<const P *>(jc + hb + n));
      }
      if (xl[k] >= 0) {
        const int n = xl[k] * W + off;
        dot(acc[k][5], le, *reinterpret_cast<const P *>(jc + n));
        dot(acc[k][9], lh, *reinterpret_cast<const P *>(jc + hb + n));
      }
      if (yp >= 0) {
        dot(acc[k][6], le, *reinterpret_cast<const P *>(jp + e));
        dot(acc[k][10], lh, *reinterpret_cast<const P *>(jp + hb + e));
      }
      if (ym >= 0) {
        dot(acc[k][7], le, *reinterpret_cast<const P *>(jm + e));
        dot(acc[k][11], lh, *reinterpret_cast<const P *>(jm + hb + e));
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
        if (!acc_mbar_wait(acc_smem_addr(&bars[i % R]), static_cast<unsigned>((i / R) & 1), wait_ns)) break;
    }
    return;
  }
  // combine the QUADS column lanes of each site (adjacent lanes), FP64
#pragma unroll
  for (int k = 0; k < MAXX; ++k) {
    const int x = xs + k * XSLOTS;
    double tot[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      double v = acc[k][c].value();
#pragma unroll
      for (int o = 1; o < QUADS; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      tot[c] = v;
    }
    if (x < Lx && q == 0) {
      double *pp = part + (static_cast<size_t>(g) * N + static_cast<size_t>(y) * Lx + x) * 12;
#pragma unroll
      for (int c = 0; c < 12; ++c) pp[c] += f * tot[c];
    }
  }
}

// One damped step of the fixed-point adjoint lam = g + J^T lam (J = dF/dDelta_in):
//   lam <- (1 - mix) lam + mix (g + J^T lam),  J^T lam = gd from the last adjoint run;
// w (the next run's weights) <- lam; max |lam_new - lam| into scal[kScalMaxDiffBits]
// (non-negative doubles order like their bit patterns).
__global__ void fixed_point_update_kernel(int N, double mix, const double *g, const double *gd, double *lam,
                                          double *w, double *scal) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double next = (1.0 - mix) * lam[i] + mix * (g[i] + gd[i]);
  const double diff = fabs(next - lam[i]);
  atomicMax(reinterpret_cast<unsigned long long *>(scal + kScalMaxDiffBits),
            static_cast<unsigned long long>(__double_as_longlong(isfinite(diff) ? diff : 1e300)));
  lam[i] = next;
  w[i] = next;
}

// dL/deps_i = (G_ee - G_hh)/a, dL/dDelta_i = (G_eh + G_he)/a,
// dL/dt_b = (-G_{e_i e_j} - G_{e_j e_i} + G_{h_i h_j} + G_{h_j h_i})/a for the
// undirected bond b = (i, i+d), stored on both directed entries.
__global__ void adjoint_final_kernel(int Lx, int Ly, int px, int py, int groups, const double *part,
                                     const double *scal, double *g_eps, double *g_hop,
                                     double *g_delta) {
  const int N = Lx * Ly;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double a = scal[kScalA];
  auto G = [&](int site, int k) {
    double s = 0.0;
    for (int g = 0; g < groups; ++g) s += part[(static_cast<size_t>(g) * N + site) * 12 + k];
    return s;
  };
  if (g_eps) g_eps[i] = (G(i, 0) - G(i, 1)) / a;
  if (g_delta) g_delta[i] = (G(i, 2) + G(i, 3)) / a;
  if (g_hop) {
    const int x = i % Lx, y = i / Lx;
    const int DX[4] = {1, -1, 0, 0}, DY[4] = {0, 0, 1, -1};
    for (int d = 0; d < 4; ++d) {
      int nx = x + DX[d], ny = y + DY[d];
      bool ok = true;
      if (nx < 0 || nx >= Lx) {
        ok = px != 0;
        nx = (nx + Lx) % Lx;
      }
      if (ny < 0 || ny >= Ly) {
        ok = ok && py != 0;
        ny = (ny + Ly) % Ly;
      }
      double v = 0.0;
      if (ok) {
        const int jn = nx + Lx * ny, db = d ^ 1;
        // pairwise sums are commutative, so both directed entries get the same bits
        v = ((G(i, 8 + d) + G(jn, 8 + db)) - (G(i, 4 + d) + G(jn, 4 + db))) / a;
      }
      g_hop[static_cast<size_t>(i) * 4 + d] = v;
    }
  }
}

}  // namespace

cudaError_t launch_adjoint_source(int precision, int Lx, int Ly, int ncols, int W,
                                  const int32_t *sites, const double *w, const double *U_site,
                                  double scale_m, void *lam, cudaStream_t s) {
  if (ncols <= 0) return cudaSuccess;
  if (precision == 1)
    adjoint_source_kernel<float><<<blocks(ncols, 128), 128, 0, s>>>(Lx, Ly, ncols, W, sites, w, U_site,
                                                                    scale_m, static_cast<float *>(lam));
  else
    adjoint_source_kernel<double><<<blocks(ncols, 128), 128, 0, s>>>(Lx, Ly, ncols, W, sites, w, U_site,
                                                                     scale_m, static_cast<double *>(lam));
  return cudaGetLastError();
}

cudaError_t launch_adjoint_source_table(int precision, int Lx, int Ly, int ncols, int W, const int32_t *sites,
                                        const double *src, int M, int m, void *lam, cudaStream_t s) {
  if (ncols <= 0) return cudaSuccess;
  if (precision == 1)
    adjoint_source_table_kernel<float><<<blocks(ncols, 128), 128, 0, s>>>(Lx, Ly, ncols, W, sites, src, M, m,
                                                                          static_cast<float *>(lam));
  else
    adjoint_source_table_kernel<double><<<blocks(ncols, 128), 128, 0, s>>>(Lx, Ly, ncols, W, sites, src, M, m,
                                                                           static_cast<double *>(lam));
  return cudaGetLastError();
}

int adjoint_groups(int Ly, int ld, int W) {
  // about 8 CTAs per SM of 152 (several resident per SM, so an uneven last
  // round costs little), at least 8 slabs per group
  const int slabs = std::max(1, ld / W);
  const int want = std::max(1, (8 * 152 + Ly - 1) / Ly);
  return std::max(1, std::min(want, slabs / 8));
}

template <typename S, int W>
cudaError_t accumulate_w(int Lx, int Ly, int px, int py, int ld, int groups, const void *lam, const void *j,
                         double f, double *part, cudaStream_t s) {
  const int slabs = ld / W;
  const int spg = (slabs + groups - 1) / groups;
  dim3 grid(Ly, groups);
  adjoint_accumulate_kernel<S, W><<<grid, 256, 0, s>>>(Lx, Ly, px, py, ld, spg, static_cast<const S *>(lam),
                                                      static_cast<const S *>(j), f, part);
  return cudaGetLastError();
}

template <typename S>
cudaError_t accumulate_s(int Lx, int Ly, int px, int py, int ld, int W, int groups, const void *lam,
                         const void *j, double f, double *part, cudaStream_t s) {
  switch (W) {
    case 1: return accumulate_w<S, 1>(Lx, Ly, px, py, ld, groups, lam, j, f, part, s);
    case 2: return accumulate_w<S, 2>(Lx, Ly, px, py, ld, groups, lam, j, f, part, s);
    case 4: return accumulate_w<S, 4>(Lx, Ly, px, py, ld, groups, lam, j, f, part, s);
    case 8: return accumulate_w<S, 8>(Lx, Ly, px, py, ld, groups, lam, j, f, part, s);
    case 16: return accumulate_w<S, 16>(Lx, Ly, px, py, ld, groups, lam, j, f, part, s);
    case 32: return accumulate_w<S, 32>(Lx, Ly, px, py, ld, groups, lam, j, f, part, s);
  }
  return cudaErrorInvalidValue;
}

namespace {
bool accumulate_staged(int precision, int Lx, int W) {
  return precision == 1 && W == kAccW && Lx <= 2 * (kAccThreads / (kAccW / 4));
}
size_t staged_smem(int Lx) { return static_cast<size_t>(kAccStages) * 4 * 2 * Lx * kAccW * sizeof(float); }

template <int MAXX>
cudaError_t launch_staged(int Lx, int Ly, int px, int py, int ld, int groups, const void *lam, const void *j,
                          double f, double *part, unsigned long long wait_ns, unsigned *flags, cudaStream_t s) {
  auto k = adjoint_accumulate_staged_kernel<MAXX>;
  static int attr_dev = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (attr_dev != dev) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024 - 1024);
    if (e != cudaSuccess) return e;
    attr_dev = dev;
  }
  const int slabs = ld / kAccW, spg = (slabs + groups - 1) / groups;
  k<<<dim3(Ly, groups), kAccThreads, staged_smem(Lx), s>>>(Lx, Ly, px, py, ld, spg, static_cast<const float *>(lam),
                                                         static_cast<const float *>(j), f, part, wait_ns, flags);
  return cudaGetLastError();
}
}  // namespace

int adjoint_groups_real(int precision, int Lx, int Ly, int ld, int W) {
  if (!accumulate_staged(precision, Lx, W)) return adjoint_groups(Ly, ld, W);
  // staged CTAs: about two waves of the resident CTAs, at least 4 slabs per group
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = std::max(1, std::min(8, static_cast<int>((228 * 1024) / (staged_smem(Lx) + 1024))));
  const int slabs = std::max(1, ld / W);
  return std::max(1, std::min(slabs / 4, (2 * sms * per_sm) / Ly));
}

cudaError_t launch_adjoint_accumulate(int precision, int Lx, int Ly, int px, int py, int ld, int W,
                                      int groups, const void *lam, const void *j, double f,
                                      double *part, unsigned long long wait_ns, unsigned *flags,
                                      cudaStream_t s) {
  if (accumulate_staged(precision, Lx, W)) {
    if (Lx <= kAccThreads / (kAccW / 4))
      return launch_staged<1>(Lx, Ly, px, py, ld, groups, lam, j, f, part, wait_ns, flags, s);
    return launch_staged<2>(Lx, Ly, px, py, ld, groups, lam, j, f, part, wait_ns, flags, s);
  }
  return precision == 1 ? accumulate_s<float>(Lx, Ly, px, py, ld, W, groups, lam, j, f, part, s)
                        : accumulate_s<double>(Lx, Ly, px, py, ld, W, groups, lam, j, f, part, s);
}

cudaError_t launch_fixed_point_update(int N, double mix, const double *g, const double *gd, double *lam,
                                      double *w, double *scal, cudaStream_t s) {
  fixed_point_update_kernel<<<blocks(N, 256), 256, 0, s>>>(N, mix, g, gd, lam, w, scal);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_final(int Lx, int Ly, int px, int py, int groups, const double *part,
                                 const double *scal, double *g_eps, double *g_hop, double *g_delta,
                                 cudaStream_t s) {
  adjoint_final_kernel<<<blocks(Lx * Ly, 128), 128, 0, s>>>(Lx, Ly, px, py, groups, part, scal, g_eps,
                                                            g_hop, g_delta);
  return cudaGetLastError();
}

}  // namespace cbdg
