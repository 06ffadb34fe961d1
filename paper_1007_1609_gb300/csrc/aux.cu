// aux.cu -- the O(N) and O(M) kernels around the recursion: Gershgorin
// rescale, damped Fermi-function coefficients, stencil parameters, the
// j_0 / j_1 start of Eq. 15, the per-step moment fold, the order-parameter
// scatter and the self-consistency mix.  All in FP64.
#include <math.h>

#include <algorithm>

#include "internal.h"

namespace cbdg {
namespace {

__device__ __forceinline__ unsigned long long ordered_bits(double v) {
  // non-negative doubles order like their bit patterns
  return static_cast<unsigned long long>(__double_as_longlong(v));
}

__device__ __forceinline__ double cabs2(double2 z) { return sqrt(z.x * z.x + z.y * z.y); }

// Gershgorin bound of Eq. 2: both rows of site i carry
// |eps_i - mu| + |Delta_i| + sum_d |t_{i,d}| (+ sum_d |Delta_{i,d}| for bonds).
// Hoppings and bond pairings across open edges are stored as zero.
__global__ void gershgorin_kernel(int N, int n_dirs, int pairing, const double *eps, double mu,
                                  const double2 *hop, const double2 *delta, double *scal) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double s = fabs(eps[i] - mu);
  for (int d = 0; d < n_dirs; ++d) s += cabs2(hop[static_cast<size_t>(i) * n_dirs + d]);
  if (pairing == 0) {
    s += cabs2(delta[i]);
  } else {
    for (int d = 0; d < 4; ++d) s += cabs2(delta[static_cast<size_t>(i) * 4 + d]);
  }
  atomicMax(reinterpret_cast<unsigned long long *>(scal + kScalBoundBits), ordered_bits(s));
}

__global__ void set_rescale_kernel(double margin, double *scal) {
  const double bound = __longlong_as_double(
      static_cast<long long>(reinterpret_cast<unsigned long long *>(scal)[kScalBoundBits]));
  scal[kScalA] = margin * bound;
}

// f_k = tanh(a cos(th_k) / 2T), th_k = pi (k + 1/2) / K  (sign(x) at T = 0).
// Coefficients of Eqs. 6-7 for the Fermi factor tanh(a x / 2T) by a K-node
// Gauss-Chebyshev sum,
//   c_n = (1/K) sum_k f_k T_n(x_k),  x_k = cos(pi (2k+1) / 2K),
//   C_n = g_n (2 - delta_n0) c_n.
// tanh is odd and the nodes are symmetric (x_{K-1-k} = -x_k, T_n(-x) =
// (-1)^n T_n(x)), so c_n = 0 for even n and, for odd n,
//   c_n = (2/K) sum_{k < K/2} f_k T_n(x_k)
// (for odd K the middle node x = 0 has f = 0).  Odd T_n come from the
// two-step recurrence T_{n+2} = 2 T_2(x) T_n - T_{n-2} (one FMA per term; the
// FP64 rounding error grows like the number of terms inside a chunk of
// kCoefChunk odd moments started from directly evaluated T_{n0}, T_{n0-2}).
// kCoefNodes nodes per thread: per n a thread sums its nodes, a warp-shuffle
// sum follows, the warps of a block are summed in a fixed order into
// part[node block][i] (n = 2i + 1); a second kernel sums the node blocks.
constexpr int kCoefThreads = 256, kCoefChunk = 128, kCoefNodes = 1;  // nodes per thread (more blocks: FP64-bound)

// cos(n pi (2k+1) / 2K) with the exact integer reduction of the argument.
__device__ __forceinline__ double cheb_node_cos(long long n, int k, int K) {
  const long long period = 4LL * K;
  const long long r = (((n % period) + period) % period) * (2LL * k + 1) % period;
  return cospi(static_cast<double>(r) / (2.0 * K));
}

// Grid (node blocks over k < K/2, chunks of odd n): block (b, c) sums nodes
// [b * kCoefNodes * 256, (b + 1) * kCoefNodes * 256) for the odd n = 2i + 1,
// i in chunk c, starting the recurrence from T_{n0} and T_{n0-2} evaluated
// directly.
__global__ void __launch_bounds__(kCoefThreads) coef_partial_kernel(int M, int K, double T, const double *scal,
                                                                    double *part) {
  __shared__ double wsum[kCoefThreads / 32][kCoefChunk];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_odd = M / 2;  // odd n < M
  const int i0 = blockIdx.y * kCoefChunk, nc = min(kCoefChunk, n_odd - i0);
  const int n0 = 2 * i0 + 1;
  const int half = K / 2;
  const double a = scal[kScalA];
  double t2[kCoefNodes], f[kCoefNodes], tm2[kCoefNodes], tn[kCoefNodes];
#pragma unroll
  for (int j = 0; j < kCoefNodes; ++j) {
    const int k = (blockIdx.x * kCoefNodes + j) * kCoefThreads + threadIdx.x;
    t2[j] = f[j] = tm2[j] = tn[j] = 0.0;
    if (k < half) {
      const double x = cospi((2.0 * k + 1.0) / (2.0 * K));
      f[j] = (T > 0.0) ? tanh(a * x / (2.0 * T)) : (x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0));
      t2[j] = 2.0 * cheb_node_cos(2, k, K);
      tn[j] = cheb_node_cos(n0, k, K);
      tm2[j] = cheb_node_cos(n0 - 2, k, K);
    }
  }
  for (int i = 0; i < nc; ++i) {
    double v = 0.0;
#pragma unroll
    for (int j = 0; j < kCoefNodes; ++j) {
      v = fma(f[j], tn[j], v);
      const double tp = fma(t2[j], tn[j], -tm2[j]);
      tm2[j] = tn[j];
      tn[j] = tp;
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) wsum[warp][i] = v;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    double v = 0.0;
    for (int w = 0; w < kCoefThreads / 32; ++w) v += wsum[w][i];
    part[static_cast<size_t>(blockIdx.x) * n_odd + i0 + i] = v;
  }
}

__global__ void coef_final_kernel(int M, int K, int nblocks, int kernel, double lambda, const double *part,
                                  double *C) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= M) return;
  const int n_odd = M / 2;
  double c = 0.0;
  if (n & 1) {
    for (int b = 0; b < nblocks; ++b) c += part[static_cast<size_t>(b) * n_odd + (n - 1) / 2];
    c = 2.0 * c / K;
  }
  double g;
  if (kernel == 0) {  // Jackson
    const double q = 1.0 / (M + 1.0);
    g = ((M - n + 1) * cospi(n * q) + sinpi(n * q) * cospi(q) / sinpi(q)) / (M + 1.0);
  } else {  // Lorentz, Eq. 16
    g = sinh(lambda * (1.0 - static_cast<double>(n) / M)) / sinh(lambda);
  }
  C[n] = g * (n == 0 ? 1.0 : 2.0) * c;
}

template <typename S>
__global__ void params_real_kernel(int N, const double *eps, double mu, const double2 *hop,
                                   const double2 *delta, const double *scal, S *p) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double s2 = 2.0 / scal[kScalA];
  S *r = p + static_cast<size_t>(i) * kParamStride;
  r[0] = static_cast<S>(s2 * (eps[i] - mu));
  r[1] = static_cast<S>(s2 * delta[i].x);
  for (int d = 0; d < 4; ++d) r[2 + d] = static_cast<S>(s2 * hop[static_cast<size_t>(i) * 4 + d].x);
  r[6] = 0;
  r[7] = 0;
}

__device__ __forceinline__ int neighbour(int Lx, int Ly, int px, int py, int x, int y, int dx,
                                         int dy) {
  int nx = x + dx, ny = y + dy;
  if (nx < 0 || nx >= Lx) {
    if (!px) return -1;
    nx = (nx + Lx) % Lx;
  }
  if (ny < 0 || ny >= Ly) {
    if (!py) return -1;
    ny = (ny + Ly) % Ly;
  }
  return nx + Lx * ny;
}

// j_0 = e_i and j_1 = H~ e_i for each column (buffers pre-zeroed), plus the
// per-column constants of the doubling identities and the n = 0, 1 terms of
// the fold: mu_0 = 1, mu_1 = (eps_i - mu)/a, <h_i|e_i> = 0,
// <h_i|H~|e_i> = conj(Delta_i)/a.
template <typename S>
__global__ void init_real_kernel(int Lx, int Ly, int px, int py, int ncols, int W,
                                 const int32_t *sites, const double *eps, double mu,
                                 const double2 *hop, const double2 *delta, const double *scal,
                                 const double *C, int M, S *j0, S *j1, double *mu1, double2 *dA,
                                 double *acc_n, double2 *acc_d, double *mu_ee, double2 *mu_eh,
                                 int mom_stride) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= ncols) return;
  const double a = scal[kScalA];
  const int i = sites[b];
  const int x = i % Lx, y = i / Lx;
  const size_t rows = 2 * static_cast<size_t>(Lx) * Ly;
  const double m1 = (eps[i] - mu) / a;
  const double2 dl = delta[i];
  j0[blocked_index(vector_row(Lx, i, 0), b, rows, W)] = static_cast<S>(1);
  j1[blocked_index(vector_row(Lx, i, 0), b, rows, W)] = static_cast<S>(m1);
  j1[blocked_index(vector_row(Lx, i, 1), b, rows, W)] = static_cast<S>(dl.x / a);
  const int DX[4] = {1, -1, 0, 0}, DY[4] = {0, 0, 1, -1};
  for (int d = 0; d < 4; ++d) {
    const int j = neighbour(Lx, Ly, px, py, x, y, DX[d], DY[d]);
    if (j < 0) continue;
    // H_{e_j e_i} = -t_{j -> i} = -conj(t_{i -> j})
    j1[blocked_index(vector_row(Lx, j, 0), b, rows, W)] =
        static_cast<S>(-hop[static_cast<size_t>(i) * 4 + d].x / a);
  }
  mu1[b] = m1;
  dA[b] = make_double2(dl.x / a, -dl.y / a);  // conj(Delta_i)/a
  acc_n[b] = -(C[0] * 1.0 + C[1] * m1);
  acc_d[b] = make_double2(C[1] * dl.x / a, C[1] * dl.y / a);  // C_1 conj(conj(Delta)/a)
  if (mu_ee) {
    mu_ee[static_cast<size_t>(b) * M + 0] = 1.0;
    mu_ee[static_cast<size_t>(b) * M + 1] = m1;
  }
  if (mu_eh) {
    mu_eh[(static_cast<size_t>(b) * M + 0) * mom_stride] = make_double2(0.0, 0.0);
    mu_eh[(static_cast<size_t>(b) * M + 1) * mom_stride] = make_double2(dl.x / a, -dl.y / a);
  }
}

// Doubling identities (T_{2n} = 2 T_n^2 - 1, T_{2n+1} = 2 T_{n+1} T_n - T_1)
// and the particle-hole identity T_n(H~) h_i = (-1)^n S T_n(H~) e_i with
// S(u, v) = (-v*, u*), which holds for symmetric pairing:
//   mu_2n      = 2 <j_n|j_n> - 1
//   mu_2n+1    = 2 <j_{n+1}|j_n> - mu_1
//   mu^eh_2n   = 0
//   mu^eh_2n+1 = 2 (-1)^(n+1) sum_s (u'_s v_s - v'_s u_s) - conj(Delta_i)/a
// then the fold acc_n -= C_m mu_m, acc_d += C_m conj(mu^eh_m).
// Steps n .. n + levels - 1 in order (a multi-step pass leaves one [3][ld]
// block of sums per level, row_split = 1); the same arithmetic, in the same
// order, as one launch per step.
__global__ void fold_kernel(int n0, int levels, int M, int ncols, int ld, int row_split,
                            const double *partials, const double *C, const double *mu1,
                            const double2 *dA, double *acc_n, double2 *acc_d, double *mu_ee,
                            double2 *mu_eh, int mom_stride, unsigned int *flags, double tol) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= ncols) return;
  double an = acc_n[b];
  double2 ad = acc_d[b];
  bool bad = false;
  for (int lv = 0; lv < levels; ++lv) {
  const int n = n0 + lv;
  const double *part = partials + static_cast<size_t>(lv) * row_split * 3 * ld;
  double A = 0.0, B = 0.0, Cs = 0.0;
  for (int s = 0; s < row_split; ++s) {
    A += part[(static_cast<size_t>(s) * 3 + 0) * ld + b];
    B += part[(static_cast<size_t>(s) * 3 + 1) * ld + b];
    Cs += part[(static_cast<size_t>(s) * 3 + 2) * ld + b];
  }
  const int m0 = 2 * n, m1 = 2 * n + 1;
  const double e0 = 2.0 * A - 1.0;
  const double e1 = 2.0 * B - mu1[b];
  const double sgn = (n & 1) ? 1.0 : -1.0;  // (-1)^(n+1)
  const double2 da = dA[b];
  const double2 h1 = make_double2(2.0 * sgn * Cs - da.x, -da.y);
  if (m0 < M) {
    an -= C[m0] * e0;
    bad |= fabs(e0) > 1.0 + tol;
    if (mu_ee) mu_ee[static_cast<size_t>(b) * M + m0] = e0;
    if (mu_eh) mu_eh[(static_cast<size_t>(b) * M + m0) * mom_stride] = make_double2(0.0, 0.0);
  }
  if (m1 < M) {
    an -= C[m1] * e1;
    ad.x += C[m1] * h1.x;
    ad.y -= C[m1] * h1.y;
    bad |= fabs(e1) > 1.0 + tol;
    if (mu_ee) mu_ee[static_cast<size_t>(b) * M + m1] = e1;
    if (mu_eh) mu_eh[(static_cast<size_t>(b) * M + m1) * mom_stride] = h1;
  }
  if (!(fabs(e0) < 1e300) || !(fabs(e1) < 1e300)) bad = true;  // NaN / inf
  }
  acc_n[b] = an;
  acc_d[b] = ad;
  if (bad) atomicOr(flags, kFlagSpectrum);
}

// Delta_i = (U_i/2) acc_d, n_i = 1 + acc_n for the column's start site
// (U_i = U_site[i], or the lattice's U when U_site is NULL).
__global__ void finalize_onsite_kernel(int ncols, const int32_t *sites, double U_all, const double *U_site,
                                       const double *acc_n, const double2 *acc_d, double2 *dout,
                                       double *nout) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= ncols) return;
  const int i = sites[b];
  const double U = U_site ? U_site[i] : U_all;
  const double2 ad = acc_d[b];
  if (dout) dout[i] = make_double2(0.5 * U * ad.x, 0.5 * U * ad.y);
  if (nout) nout[i] = 1.0 + acc_n[b];
}

// dst[k] = (src[k], 0)
__global__ void real_to_complex_kernel(int n, const double *src, double2 *dst) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) dst[k] = make_double2(src[k], 0.0);
}

// Symmetry reduction: every site takes Delta_out and n of its orbit's
// representative (rep[rep[i]] == rep[i], so representatives are only read).
__global__ void orbit_fill_kernel(int N, const int32_t *rep, double2 *dout, double *nout) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int r = rep[i];
  if (r == i) return;
  if (dout) dout[i] = dout[r];
  if (nout) nout[i] = nout[r];
}

// Delta <- Delta + mix (Delta_out - Delta); max |Delta_out - Delta| by atomicMax.
__global__ void mix_kernel(int n, double mix, const double2 *dout, double2 *delta, double *scal) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double2 o = dout[i], d = delta[i];
  const double2 diff = make_double2(o.x - d.x, o.y - d.y);
  delta[i] = make_double2(d.x + mix * diff.x, d.y + mix * diff.y);
  atomicMax(reinterpret_cast<unsigned long long *>(scal + kScalMaxDiffBits),
            ordered_bits(cabs2(diff)));
}

inline int blocks(long long n, int t) { return static_cast<int>((n + t - 1) / t); }

}  // namespace

cudaError_t launch_gershgorin(int N, int n_dirs, int pairing, int, int, int, int,
                              const double *eps, double mu, const double2 *hop,
                              const double2 *delta, double margin, double *scal, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(scal + kScalBoundBits, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  if (N > 0) gershgorin_kernel<<<blocks(N, 256), 256, 0, s>>>(N, n_dirs, pairing, eps, mu, hop, delta, scal);
  set_rescale_kernel<<<1, 1, 0, s>>>(margin, scal);
  return cudaGetLastError();
}

size_t coefficient_work(int M, int K) {
  return static_cast<size_t>(std::max(1, blocks(K / 2, kCoefThreads * kCoefNodes))) *
         static_cast<size_t>(std::max(1, M / 2));
}

cudaError_t launch_coefficients(int M, int K, double T, int kernel, double lambda,
                                const double *scal, double *work, double *C, cudaStream_t s) {
  const int nb = blocks(K / 2, kCoefThreads * kCoefNodes);
  if (nb > 0 && M / 2 > 0)
    coef_partial_kernel<<<dim3(nb, blocks(M / 2, kCoefChunk)), kCoefThreads, 0, s>>>(M, K, T, scal, work);
  coef_final_kernel<<<blocks(M, 128), 128, 0, s>>>(M, K, M / 2 > 0 ? nb : 0, kernel, lambda, work, C);
  return cudaGetLastError();
}

cudaError_t launch_params_real(int precision, int N, const double *eps, double mu,
                               const double2 *hop, const double2 *delta, const double *scal,
                               void *params, cudaStream_t s) {
  if (precision == 1)
    params_real_kernel<float><<<blocks(N, 256), 256, 0, s>>>(N, eps, mu, hop, delta, scal,
                                                             static_cast<float *>(params));
  else
    params_real_kernel<double><<<blocks(N, 256), 256, 0, s>>>(N, eps, mu, hop, delta, scal,
                                                              static_cast<double *>(params));
  return cudaGetLastError();
}

cudaError_t launch_init_real(int precision, int Lx, int Ly, int px, int py, int ncols, int W,
                             const int32_t *sites, const double *eps, double mu,
                             const double2 *hop, const double2 *delta, const double *scal,
                             const double *C, int M, void *j0, void *j1, double *mu1,
                             double2 *dA, double *acc_n, double2 *acc_d, double *mu_ee,
                             double2 *mu_eh, int mom_stride, cudaStream_t s) {
  if (ncols <= 0) return cudaSuccess;
  if (precision == 1)
    init_real_kernel<float><<<blocks(ncols, 128), 128, 0, s>>>(
        Lx, Ly, px, py, ncols, W, sites, eps, mu, hop, delta, scal, C, M,
        static_cast<float *>(j0), static_cast<float *>(j1), mu1, dA, acc_n, acc_d, mu_ee, mu_eh,
        mom_stride);
  else
    init_real_kernel<double><<<blocks(ncols, 128), 128, 0, s>>>(
        Lx, Ly, px, py, ncols, W, sites, eps, mu, hop, delta, scal, C, M,
        static_cast<double *>(j0), static_cast<double *>(j1), mu1, dA, acc_n, acc_d, mu_ee, mu_eh,
        mom_stride);
  return cudaGetLastError();
}

cudaError_t launch_fold(int n, int M, int ncols, int ld, int row_split, const double *partials,
                        const double *C, const double *mu1, const double2 *dA, double *acc_n,
                        double2 *acc_d, double *mu_ee, double2 *mu_eh, int mom_stride,
                        unsigned int *flags, double tol, cudaStream_t s, int levels) {
  if (ncols <= 0) return cudaSuccess;
  fold_kernel<<<blocks(ncols, 256), 256, 0, s>>>(n, levels, M, ncols, ld, row_split, partials, C, mu1, dA,
                                                 acc_n, acc_d, mu_ee, mu_eh, mom_stride, flags, tol);
  return cudaGetLastError();
}

cudaError_t launch_finalize_onsite(int ncols, const int32_t *sites, double U, const double *U_site,
                                   const double *acc_n, const double2 *acc_d, double2 *dout,
                                   double *nout, cudaStream_t s) {
  if (ncols <= 0) return cudaSuccess;
  finalize_onsite_kernel<<<blocks(ncols, 256), 256, 0, s>>>(ncols, sites, U, U_site, acc_n, acc_d, dout,
                                                            nout);
  return cudaGetLastError();
}

cudaError_t launch_real_to_complex(int n, const double *src, double2 *dst, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  real_to_complex_kernel<<<blocks(n, 256), 256, 0, s>>>(n, src, dst);
  return cudaGetLastError();
}

cudaError_t launch_orbit_fill(int N, const int32_t *rep, double2 *dout, double *nout, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  orbit_fill_kernel<<<blocks(N, 256), 256, 0, s>>>(N, rep, dout, nout);
  return cudaGetLastError();
}

cudaError_t launch_mix(int n, double mix, const double2 *dout, double2 *delta, double *scal,
                       cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(scal + kScalMaxDiffBits, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  if (n > 0) mix_kernel<<<blocks(n, 256), 256, 0, s>>>(n, mix, dout, delta, scal);
  return cudaGetLastError();
}

cudaError_t launch_ldos_eval(int, int, int, double, const double *, const double *, int,
                             const double *, float *, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace cbdg
