// ensemble.cu -- many independent disorder realisations of uneven lattice
// size, each iterated to self-consistency (paragraph after Eq. 20), with one
// persistent recursion launch per iteration and the iteration captured once
// as a CUDA graph and replayed.
//
// Work items are (sample, column slab of W start vectors), ordered largest
// sample first and handed out through an atomic counter.  A CTA owns an item
// from j_0 to the last moment: its two vectors live in a per-CTA scratch
// block (slab-blocked [2N][W], electron rows then hole rows per lattice row),
// three steps per pass (the lean mp::multi_pass) while three remain, the
// rest one step at a time; every pass marches the lattice rows with TMA bulk
// copies on mbarriers (the same pipeline as step.cu), and the step
// dependencies stay inside the CTA,
// so no grid-wide synchronisation is needed.  Moments are folded per column
// in FP64 as they appear (doubling identities of the real s-wave case), and
// the item ends with Delta_out and n of its W sites.  Per-sample Gershgorin
// rescale, Fermi coefficients (Chebyshev recurrence over K quadrature nodes),
// parameters, mixing and convergence run as small batched kernels around it.
// Converged samples are skipped by every kernel.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/cbdg.h"
#include "internal.h"
#include "multi_pass.cuh"

using namespace cbdg;

namespace {

constexpr int kEnsW = 16;        // start vectors per item (FP32: four 16-byte chunks)
constexpr int kEnsThreads = 256;
constexpr int kEnsD = 3;         // rows staged ahead
constexpr int kEnsJS = 3 + kEnsD;
constexpr int kEnsOS = 2 + kEnsD;
constexpr int kCoefThreads = 256;
constexpr unsigned long long kWaitNs = 2000000000ull;

struct EnsArgs {
  int n_samples, n_items, M, K;
  double T, mix, tol, U;
  const int *Lx, *Ly;               // [n_samples]
  const long long *site_off;        // [n_samples + 1]
  const int *item_sample, *item_slab;
  const float *params;              // [total sites][8]
  const double *C;                  // [n_samples][M]
  const double *scal;               // [n_samples][kScalars]
  const int *converged;             // [n_samples]
  const double *eps;                // [total sites]
  const double2 *hop, *delta;       // [total][4], [total]
  double mu;
  float *scratch;                   // [gridDim][2][scratch_per_buf]
  long long scratch_per_buf;        // floats per vector buffer of one CTA
  double2 *dout;                    // [total]
  double *nout;                     // [total]
  unsigned *queue;                  // item counter
  unsigned *flags;
  int multi;                        // 1: three steps per pass (mp::multi_pass, lean) while three remain
};

__device__ __forceinline__ unsigned smem_addr(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
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
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned it = 0;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255u) == 255u && global_ns() - t0 > kWaitNs) return false;
  }
}
__device__ __forceinline__ void bulk_load(unsigned dst, const void *src, unsigned bytes, unsigned bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
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

__device__ __forceinline__ float fcomp(const float4 &v, int j) {
  return reinterpret_cast<const float *>(&v)[j];
}

// NT threads (256): one or two lattice sites per thread, Lx <= 128.  (384
// threads with one site each up to Lx = 96 measured slower on the 256-lattice
// ensemble: 7.04 s against 6.79 s per iteration; the passes over its short
// rows are bound by per-wavefront latency, not by the uneven site split.)
template <int MAXX, int NT>
__global__ void __launch_bounds__(NT, 1) ensemble_recursion_kernel(EnsArgs a) {
  constexpr int W = kEnsW, VEC = 4, QUADS = W / VEC, XSLOTS = NT / QUADS;
  constexpr int JS = kEnsJS, OS = kEnsOS, D = kEnsD;
  using Lean = mp::PassShape<W, 3, 1, NT, true>;  // the three-step pass
  using FB = mp::FlushBank<3>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long bars[JS];         // the one-step march
  __shared__ __align__(8) unsigned long long pbars[Lean::NB];  // the three-step pass
  __shared__ int abort_flag;
  __shared__ int item_s;
  // per-thread column sums, [3][XSLOTS][W], in the ring's space: written and
  // read only between passes, when no staged row is live
  auto red = reinterpret_cast<double (*)[XSLOTS][W]>(smem_raw);
  __shared__ double accn[W], accd[W], m1s[W], dAs[W];

  const int t = threadIdx.x;
  const int q = t % QUADS, xs = t / QUADS;
  float *bufA = a.scratch + static_cast<size_t>(blockIdx.x) * 2 * a.scratch_per_buf;
  float *bufB = bufA + a.scratch_per_buf;

  if (t == 0) {
    for (int k = 0; k < JS; ++k)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&bars[k])) : "memory");
    for (int k = 0; k < Lean::NB; ++k)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&pbars[k])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    abort_flag = 0;
  }
  __syncthreads();

  long long G = 0;   // march loads issued by this CTA so far (slot = G % JS, parity = (G / JS) & 1)
  long long Gp = 0;  // rows the three-step passes staged so far (their barriers' phase base)
  for (;;) {
    if (t == 0) item_s = static_cast<int>(atomicAdd(a.queue, 1u));
    __syncthreads();
    const int item = item_s;
    __syncthreads();
    if (item >= a.n_items || abort_flag) break;
    const int s = a.item_sample[item];
    if (a.converged[s]) continue;
    const int Lx = a.Lx[s], Ly = a.Ly[s], N = Lx * Ly;
    const int c0 = a.item_slab[item] * W;
    const int cols = min(W, N - c0);
    const long long so = a.site_off[s];
    const int rowel = 2 * Lx * W, pel = Lx * kParamStride;
    const size_t vec_el = static_cast<size_t>(Ly) * rowel;
    const float *par = a.params + so * kParamStride;
    const double am = a.scal[s * kScalars + kScalA];
    const double *C = a.C + static_cast<size_t>(s) * a.M;
    float *sj = reinterpret_cast<float *>(smem_raw);
    float *so_ = sj + JS * rowel;
    float *sp = so_ + OS * rowel;

    // j_0 = e_i (bufA), j_1 = H~ e_i (bufB) for the item's columns
    for (size_t k = t; k < vec_el; k += NT) {
      bufA[k] = 0.f;
      bufB[k] = 0.f;
    }
    __syncthreads();
    if (t < cols) {
      const int b = t, i = c0 + b;
      const int x = i % Lx, y = i / Lx;
      const double m1 = (a.eps[so + i] - a.mu) / am;
      const double dl = a.delta[so + i].x;
      bufA[blocked_index(vector_row(Lx, i, 0), b, 2 * static_cast<size_t>(N), W)] = 1.f;
      bufB[blocked_index(vector_row(Lx, i, 0), b, 2 * static_cast<size_t>(N), W)] = static_cast<float>(m1);
      bufB[blocked_index(vector_row(Lx, i, 1), b, 2 * static_cast<size_t>(N), W)] = static_cast<float>(dl / am);
      const int DX[4] = {1, -1, 0, 0}, DY[4] = {0, 0, 1, -1};
      for (int d = 0; d < 4; ++d) {
        const int nx = x + DX[d], ny = y + DY[d];
        if (nx < 0 || nx >= Lx || ny < 0 || ny >= Ly) continue;  // open edges
        const int j = nx + Lx * ny;
        bufB[blocked_index(vector_row(Lx, j, 0), b, 2 * static_cast<size_t>(N), W)] =
            static_cast<float>(-a.hop[(so + i) * 4 + d].x / am);
      }
      m1s[b] = m1;
      dAs[b] = dl / am;
      accn[b] = -(C[0] + C[1] * m1);
      accd[b] = C[1] * dl / am;
    } else if (t < W) {
      m1s[t] = dAs[t] = accn[t] = accd[t] = 0.0;
    }
    asm volatile("fence.proxy.async;\n" ::: "memory");
    __syncthreads();

    const int steps = (a.M + 1) / 2 - 1;
    float *cur = bufB, *prev = bufA;
    // column t's sums of step n (|j_n|^2, <j_{n+1}|j_n>, symplectic) -> moments 2n, 2n+1 -> fold
    auto fold = [&](int n, double A, double B, double Cs) {
      const int m0 = 2 * n, m1 = 2 * n + 1;
      const double e0 = 2.0 * A - 1.0, e1 = 2.0 * B - m1s[t];
      const double sgn = (n & 1) ? 1.0 : -1.0;
      const double h1 = 2.0 * sgn * Cs - dAs[t];
      if (m0 < a.M) accn[t] -= C[m0] * e0;
      if (m1 < a.M) {
        accn[t] -= C[m1] * e1;
        accd[t] += C[m1] * h1;
      }
      if (!(fabs(e0) <= 1.0 + 1e-4) || !(fabs(e1) <= 1.0 + 1e-4)) atomicOr(a.flags, kFlagSpectrum);
    };
    // fixed-order FP64 column sums of one step -> fold
    auto reduce_fold = [&](int n, auto &sA, auto &sB, auto &sC) {
#pragma unroll
      for (int j = 0; j < VEC; ++j) {
        red[0][xs][q * VEC + j] = sA[j].value();
        red[1][xs][q * VEC + j] = sB[j].value();
        red[2][xs][q * VEC + j] = sC[j].value();
      }
      __syncthreads();
      if (t < cols) {
        double A = 0.0, B = 0.0, Cs = 0.0;
        for (int z = 0; z < XSLOTS; ++z) {
          A += red[0][z][t];
          B += red[1][z][t];
          Cs += red[2][z][t];
        }
        fold(n, A, B, Cs);
      }
      __syncthreads();
    };
    // the three-step pass's sums are in the warps' FP64 banks: lane l of warp
    // w holds list entries [base(l), base(l) + PER) of column quad l & 3; add
    // the warps in a fixed order and fold steps n, n + 1, n + 2
    auto reduce_fold_bank = [&](int n, const FB &bank) {
      double *rb = reinterpret_cast<double *>(smem_raw);
      const int lane = t & 31, w = t >> 5;
#pragma unroll
      for (int i = 0; i < FB::PER; ++i) rb[(w * 4 + (lane & 3)) * FB::NVP + FB::base(lane) + i] = bank.d[i];
      __syncthreads();
      if (t < cols) {
        const int qd = t / VEC, j = t % VEC;
        for (int lv = 0; lv < 3; ++lv) {
          double A = 0.0, B = 0.0, Cs = 0.0;
          for (int z = 0; z < NT / 32; ++z) {
            const double *r = rb + (z * 4 + qd) * FB::NVP + lv * 12 + j;
            A += r[0];
            B += r[4];
            Cs += r[8];
          }
          fold(n + lv, A, B, Cs);
        }
      }
      __syncthreads();
    };
    int n = 1;
    if (a.multi && Ly >= 2) {
      // three steps per pass over the item's vectors (the lean pass: FP32
      // column sums flushed into FP64 every few rows); (prev, cur) end as
      // (j_{n+2}, j_{n+3})
      for (; n + 2 <= steps && !abort_flag; n += 3) {
        mp::ChunkSum pA[3][VEC], pB[3][VEC], pC[3][VEC];
        FB bank;
        bank.clear();
        if (!mp::multi_pass<W, 3, 1, MAXX, NT, true, mp::ChunkSum>(prev, cur, par, Lx, Ly,
                                                                   reinterpret_cast<float *>(smem_raw), pbars, Gp,
                                                                   kWaitNs, 0u, &abort_flag, pA, pB, pC, &bank))
          break;
        Gp += Ly;
        // the new rows were stored by this thread; the next pass reads them through TMA
        asm volatile("fence.proxy.async;\n" ::: "memory");
        reduce_fold_bank(n, bank);
      }
    }
    for (; n <= steps && !abort_flag; ++n) {
      const int rows = Ly;
      const unsigned row_bytes = rowel * 4u, par_bytes = pel * 4u;
      auto issue = [&](int k) {
        int y = k - 1;
        y = (y < 0) ? y + Ly : (y >= Ly ? y - Ly : y);
        const long long g = G + k;
        const int slot = static_cast<int>(g % JS);
        const int r = k - 1;
        const bool with_old = (r >= 0 && r < rows);
        const unsigned bar = smem_addr(&bars[slot]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar),
                     "r"(row_bytes + par_bytes + (with_old ? row_bytes : 0u))
                     : "memory");
        bulk_load(smem_addr(sj + slot * rowel), cur + static_cast<size_t>(y) * rowel, row_bytes, bar);
        bulk_load(smem_addr(sp + slot * pel), par + static_cast<size_t>(y) * pel, par_bytes, bar);
        if (with_old)
          bulk_load(smem_addr(so_ + (r % OS) * rowel), prev + static_cast<size_t>(r) * rowel, row_bytes, bar);
      };
      if (t == 0)
        for (int k = 0; k < D + 2 && k <= rows + 1; ++k) issue(k);
      Kahan accA[VEC], accB[VEC], accC[VEC];
      int waited = 0, issued = min(D + 2, rows + 2);
      bool ok = true;
      for (int i = 0; i < rows; ++i) {
        if (i + 2 + D <= rows + 1) {
          if (t == 0) issue(i + 2 + D);
          issued = i + 3 + D;
        }
        for (; ok && waited <= i + 2; ++waited) {
          const long long g = G + waited;
          if (!mbar_wait(smem_addr(&bars[g % JS]), static_cast<unsigned>((g / JS) & 1))) ok = false;
        }
        if (!ok) abort_flag = 1;
        if (ok) {
          const float *rm = sj + static_cast<int>((G + i) % JS) * rowel;
          const float *rc = sj + static_cast<int>((G + i + 1) % JS) * rowel;
          const float *rp = sj + static_cast<int>((G + i + 2) % JS) * rowel;
          const float *ro = so_ + (i % OS) * rowel;
          const float *pc = sp + static_cast<int>((G + i + 1) % JS) * pel;
          float *out = prev + static_cast<size_t>(i) * rowel;
          const int hb = Lx * W, off = q * VEC;
#pragma unroll
          for (int k = 0; k < MAXX; ++k) {
            const int x = xs + k * XSLOTS;
            if (x < Lx) {
              const int xl = (x == 0) ? Lx - 1 : x - 1;
              const int xr = (x == Lx - 1) ? 0 : x + 1;
              const float4 u = *reinterpret_cast<const float4 *>(rc + x * W + off);
              const float4 v = *reinterpret_cast<const float4 *>(rc + hb + x * W + off);
              const float4 ur = *reinterpret_cast<const float4 *>(rc + xr * W + off);
              const float4 vr = *reinterpret_cast<const float4 *>(rc + hb + xr * W + off);
              const float4 ul = *reinterpret_cast<const float4 *>(rc + xl * W + off);
              const float4 vl = *reinterpret_cast<const float4 *>(rc + hb + xl * W + off);
              const float4 uu = *reinterpret_cast<const float4 *>(rp + x * W + off);
              const float4 vu = *reinterpret_cast<const float4 *>(rp + hb + x * W + off);
              const float4 ud = *reinterpret_cast<const float4 *>(rm + x * W + off);
              const float4 vd = *reinterpret_cast<const float4 *>(rm + hb + x * W + off);
              const float4 uo = *reinterpret_cast<const float4 *>(ro + x * W + off);
              const float4 vo = *reinterpret_cast<const float4 *>(ro + hb + x * W + off);
              const float *pp = pc + x * kParamStride;
              const float e = pp[0], d = pp[1], t0 = pp[2], t1 = pp[3], t2 = pp[4], t3 = pp[5];
              float4 un, vn;
#pragma unroll
              for (int j = 0; j < VEC; ++j) {
                const float uj = fcomp(u, j), vj = fcomp(v, j);
                const float hu = e * uj + d * vj -
                                 (t0 * fcomp(ur, j) + t1 * fcomp(ul, j) + t2 * fcomp(uu, j) + t3 * fcomp(ud, j));
                const float hv = d * uj - e * vj +
                                 (t0 * fcomp(vr, j) + t1 * fcomp(vl, j) + t2 * fcomp(vu, j) + t3 * fcomp(vd, j));
                const float unj = hu - fcomp(uo, j), vnj = hv - fcomp(vo, j);
                reinterpret_cast<float *>(&un)[j] = unj;
                reinterpret_cast<float *>(&vn)[j] = vnj;
                accA[j].add(uj * uj + vj * vj);
                accB[j].add(unj * uj + vnj * vj);
                accC[j].add(unj * vj - vnj * uj);
              }
              *reinterpret_cast<float4 *>(out + x * W + off) = un;
              *reinterpret_cast<float4 *>(out + hb + x * W + off) = vn;
            }
          }
        }
        __syncthreads();
        if (abort_flag) break;
      }
      if (abort_flag) {
        // let the copies in flight land (bounded) before the CTA leaves
        if (t == 0)
          for (int k = waited; k < issued; ++k) {
            const long long g = G + k;
            if (!mbar_wait(smem_addr(&bars[g % JS]), static_cast<unsigned>((g / JS) & 1))) break;
          }
        break;
      }
      G += rows + 2;
      // the new vector is read by the next step through TMA (async proxy)
      asm volatile("fence.proxy.async;\n" ::: "memory");
      reduce_fold(n, accA, accB, accC);
      float *tmp = cur;
      cur = prev;
      prev = tmp;
    }
    if (t < cols && !abort_flag) {
      a.dout[so + c0 + t] = make_double2(0.5 * a.U * accd[t], 0.0);
      a.nout[so + c0 + t] = 1.0 + accn[t];
    }
    __syncthreads();
  }
  if (abort_flag && t == 0) atomicOr(a.flags, kFlagTimeout);
}

// Per-sample Gershgorin bound (block y = sample).
__global__ void ens_gershgorin_kernel(const int *Lx, const int *Ly, const long long *site_off,
                                      const int *converged, const double *eps, double mu,
                                      const double2 *hop, const double2 *delta, double *scal) {
  const int s = blockIdx.y;
  if (converged[s]) return;
  const int N = Lx[s] * Ly[s];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const long long g = site_off[s] + i;
  double sum = fabs(eps[g] - mu) + hypot(delta[g].x, delta[g].y);
  for (int d = 0; d < 4; ++d) sum += hypot(hop[g * 4 + d].x, hop[g * 4 + d].y);
  atomicMax(reinterpret_cast<unsigned long long *>(scal + s * kScalars + kScalBoundBits),
            static_cast<unsigned long long>(__double_as_longlong(sum)));
}

__global__ void ens_rescale_kernel(int n, double margin, const int *converged, double *scal) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n || converged[s]) return;
  const double b = __longlong_as_double(static_cast<long long>(
      reinterpret_cast<unsigned long long *>(scal + s * kScalars)[kScalBoundBits]));
  scal[s * kScalars + kScalA] = margin * b;
}

// Block partials of the odd c_n = (2/K) sum_{k < K/2} f_k T_n(x_k),
// x_k = cos(pi (k+1/2)/K) (tanh is odd and the nodes symmetric, so the even
// c_n vanish and the other half of the nodes repeats the first), with the odd
// T_n(x_k) from the two-step recurrence T_{n+2} = 2 T_2 T_n - T_{n-2} (FP64)
// for each node.  grid (node blocks, sample); part[s][block][i], n = 2i + 1.
__global__ void ens_coef_partial_kernel(int M, int K, double T, const int *converged,
                                        const double *scal, double *part) {
  const int s = blockIdx.y;
  if (converged[s]) return;
  extern __shared__ double wsum[];  // [warps][M / 2]
  const int n_odd = M / 2;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double a = scal[s * kScalars + kScalA];
  double x = 0.0, f = 0.0;
  if (k < K / 2) {
    x = cospi((2.0 * k + 1.0) / (2.0 * K));
    f = (T > 0.0) ? tanh(a * x / (2.0 * T)) : (x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0));
  }
  const double t2 = 2.0 * (2.0 * x * x - 1.0);
  double tm2 = x, tn = x;  // T_{-1} = T_1 = x
  for (int i = 0; i < n_odd; ++i) {
    double v = f * tn;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) wsum[warp * n_odd + i] = v;
    const double tp = fma(t2, tn, -tm2);
    tm2 = tn;
    tn = tp;
  }
  __syncthreads();
  const int warps = blockDim.x >> 5;
  for (int i = threadIdx.x; i < n_odd; i += blockDim.x) {
    double v = 0.0;
    for (int w = 0; w < warps; ++w) v += wsum[w * n_odd + i];
    part[(static_cast<size_t>(s) * gridDim.x + blockIdx.x) * n_odd + i] = v;
  }
}

// C[s][n] = g_n (2 - delta_n0) c_n, c_n = (2/K) sum_blocks part for odd n, 0
// for even n (Jackson g_n).
__global__ void ens_coef_final_kernel(int n_samples, int M, int K, int nblocks,
                                      const int *converged, const double *part, double *C) {
  const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= static_cast<long long>(n_samples) * M) return;
  const int s = static_cast<int>(idx / M), n = static_cast<int>(idx % M);
  if (converged[s]) return;
  const int n_odd = M / 2;
  double c = 0.0;
  if (n & 1) {
    for (int b = 0; b < nblocks; ++b) c += part[(static_cast<size_t>(s) * nblocks + b) * n_odd + (n - 1) / 2];
    c = 2.0 * c / K;
  }
  const double q = 1.0 / (M + 1.0);
  const double g = ((M - n + 1) * cospi(n * q) + sinpi(n * q) * cospi(q) / sinpi(q)) / (M + 1.0);
  C[idx] = g * (n == 0 ? 1.0 : 2.0) * c;
}

__global__ void ens_params_kernel(const int *Lx, const int *Ly, const long long *site_off,
                                  const int *converged, const double *eps, double mu,
                                  const double2 *hop, const double2 *delta, const double *scal,
                                  float *p) {
  const int s = blockIdx.y;
  if (converged[s]) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Lx[s] * Ly[s]) return;
  const long long g = site_off[s] + i;
  const double s2 = 2.0 / scal[s * kScalars + kScalA];
  float *r = p + g * kParamStride;
  r[0] = static_cast<float>(s2 * (eps[g] - mu));
  r[1] = static_cast<float>(s2 * delta[g].x);
  for (int d = 0; d < 4; ++d) r[2 + d] = static_cast<float>(s2 * hop[g * 4 + d].x);
  r[6] = r[7] = 0.f;
}

__global__ void ens_mix_kernel(const int *Lx, const int *Ly, const long long *site_off,
                               const int *converged, double mix, const double2 *dout,
                               double2 *delta, double *scal) {
  const int s = blockIdx.y;
  if (converged[s]) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Lx[s] * Ly[s]) return;
  const long long g = site_off[s] + i;
  const double2 o = dout[g], d = delta[g];
  const double dx = o.x - d.x, dy = o.y - d.y;
  delta[g] = make_double2(d.x + mix * dx, d.y + mix * dy);
  atomicMax(reinterpret_cast<unsigned long long *>(scal + s * kScalars + kScalMaxDiffBits),
            static_cast<unsigned long long>(__double_as_longlong(sqrt(dx * dx + dy * dy))));
}

// Marks samples whose max |Delta_out - Delta| fell below tol; counts the rest.
__global__ void ens_converge_kernel(int n, double tol, const double *scal, int *converged,
                                    int *iters, double *last_diff, unsigned *remaining) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n || converged[s]) return;
  const double d = __longlong_as_double(static_cast<long long>(
      reinterpret_cast<const unsigned long long *>(scal + s * kScalars)[kScalMaxDiffBits]));
  iters[s] += 1;
  last_diff[s] = d;
  if (d < tol) converged[s] = 1;
  else atomicAdd(remaining, 1u);
}

__global__ void ens_reset_kernel(int n, const int *converged, double *scal) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n || converged[s]) return;
  reinterpret_cast<unsigned long long *>(scal + s * kScalars)[kScalBoundBits] = 0ull;
  reinterpret_cast<unsigned long long *>(scal + s * kScalars)[kScalMaxDiffBits] = 0ull;
}

inline int blocks(long long n, int t) { return static_cast<int>((n + t - 1) / t); }

}  // namespace

// ---------------------------------------------------------------- host side

struct cbdg_ensemble {
  int device = 0;
  cudaStream_t stream = nullptr;
  int n = 0, Lmax = 0, Nmax = 0;
  long long total = 0;
  double mu = 0.0, U = 0.0;
  int K = 16384;
  std::vector<int> hLx, hLy;
  std::vector<long long> hoff;
  void *d_Lx = nullptr, *d_Ly = nullptr, *d_off = nullptr, *d_items_s = nullptr, *d_items_c = nullptr;
  void *d_eps = nullptr, *d_hop = nullptr, *d_delta = nullptr, *d_params = nullptr, *d_C = nullptr;
  void *d_part = nullptr, *d_scal = nullptr, *d_conv = nullptr, *d_iters = nullptr, *d_last = nullptr;
  void *d_scratch = nullptr, *d_dout = nullptr, *d_nout = nullptr, *d_small = nullptr;
  int n_items = 0, grid = 0;
  long long scratch_per_buf = 0;
  size_t smem = 0;
  int multi = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  double g_T = -1, g_mix = -1, g_tol = -1;
  int g_M = -1;
};

namespace {

cbdg_status efail(cbdg_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  cbdg_internal_set_error(buf);
  return st;
}

#define ECK(call)                                                                                \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess)                                                                       \
      return efail(e_ == cudaErrorMemoryAllocation ? CBDG_ERR_OOM : CBDG_ERR_CUDA, "%s: %s", #call, \
                   cudaGetErrorString(e_));                                                      \
  } while (0)

size_t ens_smem(int Lmax) {
  const size_t rowel = static_cast<size_t>(2) * Lmax * kEnsW;
  return ((kEnsJS + kEnsOS) * rowel + kEnsJS * static_cast<size_t>(Lmax) * kParamStride) * sizeof(float);
}
// shared memory of the three-step (lean) pass and of its FP64 sums' reduction
size_t ens_multi_smem(int Lmax) {
  const size_t bank = static_cast<size_t>(kEnsThreads / 32) * 4 * mp::FlushBank<3>::NVP * sizeof(double);
  return std::max(mp::PassShape<kEnsW, 3, 1, kEnsThreads, true>::smem_floats(Lmax) * sizeof(float), bank);
}
// the per-thread column sums [3][XSLOTS][W] doubles share the ring's space
size_t ens_red_smem(int Lmax);
constexpr size_t kEnsDynLimit = 220 * 1024;

template <int MAXX, int NT>
cudaError_t launch_ens(const EnsArgs &a, int grid, size_t smem, cudaStream_t s) {
  ensemble_recursion_kernel<MAXX, NT><<<grid, NT, smem, s>>>(a);
  return cudaGetLastError();
}

// Kernel shape for the widest lattice.
int ens_threads(int) { return kEnsThreads; }
int ens_maxx(int Lmax) { return (Lmax + 63) / 64; }
size_t ens_red_smem(int Lmax) {
  return static_cast<size_t>(3) * (ens_threads(Lmax) / (kEnsW / 4)) * kEnsW * sizeof(double);
}

cudaError_t set_ens_attr(int Lmax, size_t smem) {
  const int attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if (ens_maxx(Lmax) == 1)
    return cudaFuncSetAttribute(ensemble_recursion_kernel<1, kEnsThreads>, (cudaFuncAttribute)attr, static_cast<int>(smem));
  return cudaFuncSetAttribute(ensemble_recursion_kernel<2, kEnsThreads>, (cudaFuncAttribute)attr, static_cast<int>(smem));
}

cudaError_t launch_ens_for(int Lmax, const EnsArgs &a, int grid, size_t smem, cudaStream_t s) {
  return ens_maxx(Lmax) == 1 ? launch_ens<1, kEnsThreads>(a, grid, smem, s) : launch_ens<2, kEnsThreads>(a, grid, smem, s);
}

// Records the launch sequence of one self-consistency iteration on e->stream.
cudaError_t enqueue_iteration(cbdg_ensemble *e, double T, int M, double mix, double tol) {
  cudaStream_t s = e->stream;
  int *conv = static_cast<int *>(e->d_conv);
  double *scal = static_cast<double *>(e->d_scal);
  unsigned *small = static_cast<unsigned *>(e->d_small);  // [0] queue, [1] remaining, [2] flags
  cudaError_t err;
  ens_reset_kernel<<<blocks(e->n, 128), 128, 0, s>>>(e->n, conv, scal);
  dim3 gs(blocks(e->Nmax, 256), e->n);
  ens_gershgorin_kernel<<<gs, 256, 0, s>>>(static_cast<int *>(e->d_Lx), static_cast<int *>(e->d_Ly),
                                           static_cast<long long *>(e->d_off), conv,
                                           static_cast<double *>(e->d_eps), e->mu,
                                           static_cast<double2 *>(e->d_hop),
                                           static_cast<double2 *>(e->d_delta), scal);
  ens_rescale_kernel<<<blocks(e->n, 128), 128, 0, s>>>(e->n, 1.1, conv, scal);
  const int nb = std::max(1, blocks(e->K / 2, kCoefThreads));
  dim3 gc(nb, e->n);
  ens_coef_partial_kernel<<<gc, kCoefThreads, (kCoefThreads / 32) * std::max(1, M / 2) * sizeof(double), s>>>(
      M, e->K, T, conv, scal, static_cast<double *>(e->d_part));
  ens_coef_final_kernel<<<blocks(static_cast<long long>(e->n) * M, 256), 256, 0, s>>>(
      e->n, M, e->K, nb, conv, static_cast<double *>(e->d_part), static_cast<double *>(e->d_C));
  ens_params_kernel<<<gs, 256, 0, s>>>(static_cast<int *>(e->d_Lx), static_cast<int *>(e->d_Ly),
                                       static_cast<long long *>(e->d_off), conv,
                                       static_cast<double *>(e->d_eps), e->mu,
                                       static_cast<double2 *>(e->d_hop),
                                       static_cast<double2 *>(e->d_delta), scal,
                                       static_cast<float *>(e->d_params));
  if ((err = cudaMemsetAsync(small, 0, 2 * sizeof(unsigned), s)) != cudaSuccess) return err;
  EnsArgs a;
  a.n_samples = e->n;
  a.n_items = e->n_items;
  a.M = M;
  a.K = e->K;
  a.T = T;
  a.mix = mix;
  a.tol = tol;
  a.U = e->U;
  a.Lx = static_cast<int *>(e->d_Lx);
  a.Ly = static_cast<int *>(e->d_Ly);
  a.site_off = static_cast<long long *>(e->d_off);
  a.item_sample = static_cast<int *>(e->d_items_s);
  a.item_slab = static_cast<int *>(e->d_items_c);
  a.params = static_cast<float *>(e->d_params);
  a.C = static_cast<double *>(e->d_C);
  a.scal = scal;
  a.converged = conv;
  a.eps = static_cast<double *>(e->d_eps);
  a.hop = static_cast<double2 *>(e->d_hop);
  a.delta = static_cast<double2 *>(e->d_delta);
  a.mu = e->mu;
  a.scratch = static_cast<float *>(e->d_scratch);
  a.scratch_per_buf = e->scratch_per_buf;
  a.dout = static_cast<double2 *>(e->d_dout);
  a.nout = static_cast<double *>(e->d_nout);
  a.queue = small;
  a.flags = small + 2;
  a.multi = e->multi;
  err = launch_ens_for(e->Lmax, a, e->grid, e->smem, s);
  if (err != cudaSuccess) return err;
  ens_mix_kernel<<<gs, 256, 0, s>>>(static_cast<int *>(e->d_Lx), static_cast<int *>(e->d_Ly),
                                    static_cast<long long *>(e->d_off), conv, mix,
                                    static_cast<double2 *>(e->d_dout), static_cast<double2 *>(e->d_delta),
                                    scal);
  ens_converge_kernel<<<blocks(e->n, 128), 128, 0, s>>>(e->n, tol, scal, conv,
                                                        static_cast<int *>(e->d_iters),
                                                        static_cast<double *>(e->d_last), small + 1);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

cbdg_status cbdg_build_ensemble(const cbdg_lattice_desc *descs, int32_t n, cbdg_stream stream,
                                cbdg_ensemble **out) {
  if (!descs || !out || n < 1) return efail(CBDG_ERR_INVALID_ARG, "need n >= 1 descriptors");
  *out = nullptr;
  // each member is validated by the single-lattice builder's rules
  for (int s = 0; s < n; ++s) {
    const cbdg_lattice_desc &d = descs[s];
    if (d.precision != CBDG_FP32_MIXED || d.pairing != CBDG_ONSITE_U || d.n_dirs != 4 || d.complex_field)
      return efail(CBDG_ERR_UNSUPPORTED,
                   "ensembles take real on-site pairing, 4 directions, FP32 recursion (sample %d)", s);
    if (d.periodic_x || d.periodic_y)
      return efail(CBDG_ERR_UNSUPPORTED, "ensemble lattices have open edges (sample %d)", s);
    if (d.mu != descs[0].mu || d.coupling != descs[0].coupling)
      return efail(CBDG_ERR_INVALID_ARG, "ensemble members share mu and U (sample %d)", s);
    cbdg_lattice *probe = nullptr;
    cbdg_status st = cbdg_build_lattice(&d, stream, &probe);  // validation
    if (st != CBDG_OK) return st;
    cbdg_destroy(probe);
  }
  cbdg_ensemble *e = new (std::nothrow) cbdg_ensemble();
  if (!e) return efail(CBDG_ERR_OOM, "host allocation failed");
  cudaGetDevice(&e->device);
  e->stream = reinterpret_cast<cudaStream_t>(stream);
  e->n = n;
  e->mu = descs[0].mu;
  e->U = descs[0].coupling;
  e->hoff.assign(n + 1, 0);
  for (int s = 0; s < n; ++s) {
    e->hLx.push_back(descs[s].Lx);
    e->hLy.push_back(descs[s].Ly);
    e->hoff[s + 1] = e->hoff[s] + static_cast<long long>(descs[s].Lx) * descs[s].Ly;
    e->Lmax = std::max(e->Lmax, descs[s].Lx);
    e->Nmax = std::max(e->Nmax, descs[s].Lx * descs[s].Ly);
  }
  e->total = e->hoff[n];
  auto bail = [&](cbdg_status st) {
    cbdg_ensemble_destroy(e);
    return st;
  };
  if (e->Lmax > 128) return bail(efail(CBDG_ERR_UNSUPPORTED, "ensemble lattices must have Lx <= 128"));
  e->smem = std::max(ens_smem(e->Lmax), ens_red_smem(e->Lmax));
  if (e->smem > kEnsDynLimit) return bail(efail(CBDG_ERR_UNSUPPORTED, "ensemble lattice rows too long"));
  e->multi = ens_multi_smem(e->Lmax) <= kEnsDynLimit ? 1 : 0;
  if (e->multi) e->smem = std::max(e->smem, ens_multi_smem(e->Lmax));
  // items: (sample, slab) ordered by sample size, largest first
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return e->hLx[x] * e->hLy[x] > e->hLx[y] * e->hLy[y];
  });
  std::vector<int> is, ic;
  for (int s : order) {
    const int N = e->hLx[s] * e->hLy[s];
    for (int c = 0; c * kEnsW < N; ++c) {
      is.push_back(s);
      ic.push_back(c);
    }
  }
  e->n_items = static_cast<int>(is.size());
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, e->device);
  e->grid = std::min(sms, e->n_items);
  e->scratch_per_buf = static_cast<long long>(2) * e->Nmax * kEnsW;
  auto dalloc = [&](void **p, size_t bytes) { return cudaMalloc(p, std::max<size_t>(bytes, 16)); };
  cudaError_t err;
#define EALLOC(ptr, bytes)                                               \
  if ((err = dalloc(&(ptr), (bytes))) != cudaSuccess) {                  \
    cudaGetLastError();                                                  \
    return bail(efail(CBDG_ERR_OOM, "ensemble allocation failed"));      \
  }
  EALLOC(e->d_Lx, n * sizeof(int));
  EALLOC(e->d_Ly, n * sizeof(int));
  EALLOC(e->d_off, (n + 1) * sizeof(long long));
  EALLOC(e->d_items_s, e->n_items * sizeof(int));
  EALLOC(e->d_items_c, e->n_items * sizeof(int));
  EALLOC(e->d_eps, e->total * sizeof(double));
  EALLOC(e->d_hop, e->total * 4 * sizeof(double2));
  EALLOC(e->d_delta, e->total * sizeof(double2));
  EALLOC(e->d_params, e->total * kParamStride * sizeof(float));
  EALLOC(e->d_scal, static_cast<size_t>(n) * kScalars * sizeof(double));
  EALLOC(e->d_conv, n * sizeof(int));
  EALLOC(e->d_iters, n * sizeof(int));
  EALLOC(e->d_last, n * sizeof(double));
  EALLOC(e->d_scratch, static_cast<size_t>(e->grid) * 2 * e->scratch_per_buf * sizeof(float));
  EALLOC(e->d_dout, e->total * sizeof(double2));
  EALLOC(e->d_nout, e->total * sizeof(double));
  EALLOC(e->d_small, 4 * sizeof(unsigned));
#undef EALLOC
  // upload (descriptor arrays may be host or device memory)
  for (int s = 0; s < n; ++s) {
    const long long o = e->hoff[s], N = e->hoff[s + 1] - o;
    if ((err = cudaMemcpy(static_cast<double *>(e->d_eps) + o, descs[s].eps, N * sizeof(double), cudaMemcpyDefault)) != cudaSuccess ||
        (err = cudaMemcpy(static_cast<double2 *>(e->d_hop) + o * 4, descs[s].hop, N * 4 * sizeof(double2), cudaMemcpyDefault)) != cudaSuccess ||
        (err = cudaMemcpy(static_cast<double2 *>(e->d_delta) + o, descs[s].delta0, N * sizeof(double2), cudaMemcpyDefault)) != cudaSuccess)
      return bail(efail(CBDG_ERR_CUDA, "ensemble upload: %s", cudaGetErrorString(err)));
  }
  if ((err = cudaMemcpy(e->d_Lx, e->hLx.data(), n * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (err = cudaMemcpy(e->d_Ly, e->hLy.data(), n * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (err = cudaMemcpy(e->d_off, e->hoff.data(), (n + 1) * sizeof(long long), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (err = cudaMemcpy(e->d_items_s, is.data(), is.size() * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (err = cudaMemcpy(e->d_items_c, ic.data(), ic.size() * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (err = cudaMemset(e->d_conv, 0, n * sizeof(int))) != cudaSuccess ||
      (err = cudaMemset(e->d_iters, 0, n * sizeof(int))) != cudaSuccess ||
      (err = cudaMemset(e->d_last, 0, n * sizeof(double))) != cudaSuccess ||
      (err = cudaMemset(e->d_scal, 0, static_cast<size_t>(n) * kScalars * sizeof(double))) != cudaSuccess ||
      (err = set_ens_attr(e->Lmax, e->smem)) != cudaSuccess)
    return bail(efail(CBDG_ERR_CUDA, "ensemble setup: %s", cudaGetErrorString(err)));
  *out = e;
  return CBDG_OK;
}

cbdg_status cbdg_ensemble_destroy(cbdg_ensemble *e) {
  if (!e) return CBDG_OK;
  cudaSetDevice(e->device);
  if (e->stream) cudaStreamSynchronize(e->stream);
  else cudaDeviceSynchronize();
  if (e->exec) cudaGraphExecDestroy(e->exec);
  if (e->graph) cudaGraphDestroy(e->graph);
  void *ptrs[] = {e->d_Lx, e->d_Ly, e->d_off, e->d_items_s, e->d_items_c, e->d_eps, e->d_hop,
                  e->d_delta, e->d_params, e->d_C, e->d_part, e->d_scal, e->d_conv, e->d_iters,
                  e->d_last, e->d_scratch, e->d_dout, e->d_nout, e->d_small};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  delete e;
  return CBDG_OK;
}

cbdg_status cbdg_ensemble_scf(cbdg_ensemble *e, double T, int32_t M, double mix, double tol,
                              int32_t max_iter, int32_t *iters_out, int32_t *converged_mask) {
  if (!e) return efail(CBDG_ERR_INVALID_ARG, "ensemble is NULL");
  if (!(T >= 0.0) || M < 2 || !(mix > 0.0 && mix <= 1.0) || !(tol >= 0.0) || max_iter < 0)
    return efail(CBDG_ERR_INVALID_ARG, "bad SCF arguments");
  ECK(cudaSetDevice(e->device));
  const int nb = (e->K + kCoefThreads - 1) / kCoefThreads;
  if (e->g_M != M) {
    if (e->d_C) cudaFree(e->d_C);
    if (e->d_part) cudaFree(e->d_part);
    e->d_C = e->d_part = nullptr;
    ECK(cudaMalloc(&e->d_C, static_cast<size_t>(e->n) * M * sizeof(double)));
    ECK(cudaMalloc(&e->d_part, static_cast<size_t>(e->n) * nb * M * sizeof(double)));
    if ((kCoefThreads / 32) * M * sizeof(double) > 48 * 1024)
      ECK(cudaFuncSetAttribute(ens_coef_partial_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               static_cast<int>((kCoefThreads / 32) * M * sizeof(double))));
  }
  if (!e->exec || e->g_T != T || e->g_M != M || e->g_mix != mix || e->g_tol != tol) {
    if (e->exec) cudaGraphExecDestroy(e->exec);
    if (e->graph) cudaGraphDestroy(e->graph);
    e->exec = nullptr;
    e->graph = nullptr;
    cudaStream_t cap = nullptr;
    ECK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaStream_t keep = e->stream;
    e->stream = cap;
    cudaError_t err = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (err == cudaSuccess) {
      err = enqueue_iteration(e, T, M, mix, tol);
      cudaGraph_t g = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(cap, &g);
      if (err == cudaSuccess) err = e2;
      e->graph = g;
    }
    e->stream = keep;
    cudaStreamDestroy(cap);
    if (err != cudaSuccess) return efail(CBDG_ERR_CUDA, "capturing the SCF iteration: %s", cudaGetErrorString(err));
    ECK(cudaGraphInstantiate(&e->exec, e->graph, 0));
    e->g_T = T;
    e->g_M = M;
    e->g_mix = mix;
    e->g_tol = tol;
  }
  unsigned *small = static_cast<unsigned *>(e->d_small);
  ECK(cudaMemsetAsync(small + 2, 0, sizeof(unsigned), e->stream));
  int it = 0;
  unsigned remaining = 1, flags = 0;
  while (it < max_iter && remaining > 0) {
    ECK(cudaGraphLaunch(e->exec, e->stream));
    ECK(cudaMemcpyAsync(&remaining, small + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, e->stream));
    ECK(cudaMemcpyAsync(&flags, small + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, e->stream));
    ECK(cudaStreamSynchronize(e->stream));
    ++it;
    if (flags & kFlagTimeout) return efail(CBDG_ERR_CUDA, "the ensemble kernel gave up waiting for a staged copy");
    if (flags & kFlagSpectrum) return efail(CBDG_ERR_SPECTRUM, "a Chebyshev moment exceeded 1 in magnitude");
  }
  std::vector<int> conv(e->n), iters(e->n);
  ECK(cudaMemcpy(conv.data(), e->d_conv, e->n * sizeof(int), cudaMemcpyDeviceToHost));
  ECK(cudaMemcpy(iters.data(), e->d_iters, e->n * sizeof(int), cudaMemcpyDeviceToHost));
  if (iters_out) *iters_out = it;
  if (converged_mask)
    for (int s = 0; s < e->n; ++s) converged_mask[s] = conv[s];
  return remaining > 0 ? efail(CBDG_ERR_NOT_CONVERGED, "%u samples not converged after %d iterations",
                               remaining, it)
                       : CBDG_OK;
}

cbdg_status cbdg_ensemble_get_delta(cbdg_ensemble *e, int32_t sample, cbdg_complex *delta) {
  if (!e || !delta || sample < 0 || sample >= e->n) return efail(CBDG_ERR_INVALID_ARG, "bad arguments");
  ECK(cudaSetDevice(e->device));
  const long long o = e->hoff[sample], N = e->hoff[sample + 1] - o;
  ECK(cudaMemcpy(delta, static_cast<double2 *>(e->d_delta) + o, N * sizeof(double2), cudaMemcpyDefault));
  return CBDG_OK;
}

cbdg_status cbdg_ensemble_set_option(cbdg_ensemble *e, int32_t option, int64_t value) {
  if (!e) return efail(CBDG_ERR_INVALID_ARG, "ensemble is NULL");
  if (option == CBDG_OPT_QUADRATURE_NODES) {
    if (value < 32 || value > (1 << 22)) return efail(CBDG_ERR_INVALID_ARG, "K out of range");
    e->K = static_cast<int>(value);
    e->g_M = -1;  // reallocate partials and re-capture
    return CBDG_OK;
  }
  return efail(CBDG_ERR_INVALID_ARG, "unsupported ensemble option %d", option);
}

}  // extern "C"
