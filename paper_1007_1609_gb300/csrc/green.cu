// green.cu -- the direct recursion of Eq. 15 read at chosen target sites.
//
//   * target_gather_kernel: nonlocal Chebyshev moments <e_t|j_m>, <h_t|j_m>
//     of the start vector j_0 = e_i (a^{11}_m(t, i), a^{12}_m(t, i) of Eqs. 11
//     and coeff2 times 1 + delta_m0), and the current fold
//     K_{i,d} = sum_m C_m <e_{i+d}|j_m>;
//   * bond_current_kernel: J_{i->i+d} of Eq. 20 from K (both spins);
//   * green_weights_kernel + green_contract_kernel: the retarded Green's
//     function of gf1 at chosen energies, a complex contraction of the
//     moments with a per-energy weight table.
#include <math.h>

#include "internal.h"

namespace cbdg {
namespace {

inline int blocks(long long n, int t) { return static_cast<int>((n + t - 1) / t); }

// Moment m of every (column b, target t) from j_m (slab-blocked layout):
//   a_e[(b*M + m)*n_t + t] = <e_tgt|j_m>,  a_h[...] = <h_tgt|j_m>,
//   acc[b*n_t + t] += C_m <e_tgt|j_m>,
// tgt = targets[t], or with targets == NULL the neighbour of sites[b] along
// direction t (nothing is read across an open edge).  The index runs over
// columns fastest: a warp reads consecutive columns of one vector row.
// |<x|T_m(H~)|e_i>| <= 1 while the spectrum of H~ lies in [-1, 1]; a larger
// value (or a NaN) raises kFlagSpectrum.
template <typename S>
__global__ void target_gather_kernel(int m, int M, int Lx, int Ly, int px, int py, int ncols, int W,
                                     const int32_t *sites, int n_t, const int32_t *targets,
                                     const S *j, const double *C, double2 *acc, double2 *a_e,
                                     double2 *a_h, unsigned int *flags, double tol) {
  const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= static_cast<long long>(n_t) * ncols) return;
  const int t = static_cast<int>(idx / ncols);
  const int b = static_cast<int>(idx % ncols);
  const int tgt = targets ? targets[t] : neighbour_site(Lx, Ly, px, py, sites[b], t);
  double2 e = make_double2(0.0, 0.0), h = make_double2(0.0, 0.0);
  if (tgt >= 0) {
    const size_t rows = 2 * static_cast<size_t>(Lx) * Ly;
    const size_t ke = blocked_index(vector_row(Lx, tgt, 0), b, rows, W);
    e = make_double2(static_cast<double>(j[2 * ke]), static_cast<double>(j[2 * ke + 1]));
    if (a_h) {
      const size_t kh = blocked_index(vector_row(Lx, tgt, 1), b, rows, W);
      h = make_double2(static_cast<double>(j[2 * kh]), static_cast<double>(j[2 * kh + 1]));
    }
  }
  const size_t o = (static_cast<size_t>(b) * M + m) * n_t + t;
  if (a_e) a_e[o] = e;
  if (a_h) a_h[o] = h;
  if (acc) {
    double2 s = acc[static_cast<size_t>(b) * n_t + t];
    const double c = C[m];
    s.x = fma(c, e.x, s.x);
    s.y = fma(c, e.y, s.y);
    acc[static_cast<size_t>(b) * n_t + t] = s;
  }
  const double bound = 1.0 + tol;
  if (!(e.x * e.x + e.y * e.y <= bound * bound) || !(h.x * h.x + h.y * h.y <= bound * bound))
    atomicOr(flags, kFlagSpectrum);
}

// J[i*n_dirs + d] = -2 Im[t_{i,d} K_{i,d}]: 2 Im[t_ij <c+_i c_j>] per spin with
// <c+_{i,up} c_{j,up}> = -(1/2) K_{i,d}, times 2 for the equal spin-down
// current (particle-hole symmetry); 0 across an open edge.  K is indexed by
// site (all N sites were start vectors, in order).
__global__ void bond_current_kernel(int N, int n_dirs, int Lx, int Ly, int px, int py,
                                    const double2 *hop, const double2 *K, double *J) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N * n_dirs) return;
  const int i = idx / n_dirs, d = idx % n_dirs;
  double r = 0.0;
  if (neighbour_site(Lx, Ly, px, py, i, d) >= 0) {
    const double2 t = hop[idx], k = K[idx];
    r = -2.0 * (t.x * k.y + t.y * k.x);
  }
  J[idx] = r;
}

// W[e][n] = (-2i / (a sqrt(1 - x^2))) g_n / (1 + delta_n0) exp(-i n arccos x),
// x = E_e / a, g_n the Jackson (kernel 0) or Lorentz (kernel 1, Eq. 16) kernel.
__global__ void green_weights_kernel(int n_E, int M, int kernel, double lambda,
                                     const double *energies, const double *scal, double2 *W) {
  const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= static_cast<long long>(n_E) * M) return;
  const int e = static_cast<int>(idx / M);
  const int n = static_cast<int>(idx % M);
  const double a = scal[kScalA];
  const double x = energies[e] / a;
  double g;
  if (kernel == 0) {
    const double q = 1.0 / (M + 1.0);
    g = ((M - n + 1) * cospi(n * q) + sinpi(n * q) * cospi(q) / sinpi(q)) / (M + 1.0);
  } else {
    g = sinh(lambda * (1.0 - static_cast<double>(n) / M)) / sinh(lambda);
  }
  const double w = g * (n == 0 ? 0.5 : 1.0) * 2.0 / (a * sqrt(1.0 - x * x));
  double s, c;
  sincos(n * acos(x), &s, &c);
  // -i w (c - i s) = -w s - i w c
  W[idx] = make_double2(-w * s, -w * c);
}

// G[(c*n_t + t)*n_E + e] = sum_n mom[(c*M + n)*n_t + t] W[e][n]  (complex).
// A CTA owns 16 targets x 64 energies of one start site; each thread keeps
// four energies of one target and the moment chunks of 32 pass through
// shared memory.
constexpr int kGT = 16, kGE = 64, kGN = 32;

__global__ void __launch_bounds__(256) green_contract_kernel(int n_sites, int n_t, int M, int n_E,
                                                             const double2 *mom, const double2 *W,
                                                             double2 *G) {
  __shared__ double2 sm[kGN][kGT];
  __shared__ double2 sw[kGE][kGN + 1];
  const int tiles_t = (n_t + kGT - 1) / kGT, tiles_e = (n_E + kGE - 1) / kGE;
  long long tile = blockIdx.x;
  const int te = static_cast<int>(tile % tiles_e);
  tile /= tiles_e;
  const int tt = static_cast<int>(tile % tiles_t);
  const int c = static_cast<int>(tile / tiles_t);
  if (c >= n_sites) return;
  const int tx = threadIdx.x % kGT, ty = threadIdx.x / kGT;
  const int t0 = tt * kGT, e0 = te * kGE;
  double2 acc[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) acc[k] = make_double2(0.0, 0.0);
  for (int n0 = 0; n0 < M; n0 += kGN) {
    for (int q = threadIdx.x; q < kGN * kGT; q += blockDim.x) {
      const int n = n0 + q / kGT, t = t0 + q % kGT;
      sm[q / kGT][q % kGT] =
          (n < M && t < n_t) ? mom[(static_cast<size_t>(c) * M + n) * n_t + t] : make_double2(0.0, 0.0);
    }
    for (int q = threadIdx.x; q < kGE * kGN; q += blockDim.x) {
      const int e = e0 + q / kGN, n = n0 + q % kGN;
      sw[q / kGN][q % kGN] = (e < n_E && n < M) ? W[static_cast<size_t>(e) * M + n] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int n = 0; n < kGN; ++n) {
      const double2 a = sm[n][tx];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const double2 w = sw[ty + 16 * k][n];
        acc[k].x = fma(a.x, w.x, fma(-a.y, w.y, acc[k].x));
        acc[k].y = fma(a.x, w.y, fma(a.y, w.x, acc[k].y));
      }
    }
    __syncthreads();
  }
  const int t = t0 + tx;
  if (t >= n_t) return;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int e = e0 + ty + 16 * k;
    if (e < n_E) G[(static_cast<size_t>(c) * n_t + t) * n_E + e] = acc[k];
  }
}

}  // namespace

cudaError_t launch_target_gather(int precision, int m, int M, int Lx, int Ly, int px, int py, int ncols,
                                 int W, const int32_t *sites, int n_t, const int32_t *targets,
                                 const void *j, const double *C, double2 *acc, double2 *a_e,
                                 double2 *a_h, unsigned int *flags, double tol, cudaStream_t s) {
  const long long n = static_cast<long long>(n_t) * ncols;
  if (n <= 0) return cudaSuccess;
  if (precision == 1)
    target_gather_kernel<float><<<blocks(n, 256), 256, 0, s>>>(m, M, Lx, Ly, px, py, ncols, W, sites, n_t,
                                                               targets, static_cast<const float *>(j), C,
                                                               acc, a_e, a_h, flags, tol);
  else
    target_gather_kernel<double><<<blocks(n, 256), 256, 0, s>>>(m, M, Lx, Ly, px, py, ncols, W, sites, n_t,
                                                                targets, static_cast<const double *>(j), C,
                                                                acc, a_e, a_h, flags, tol);
  return cudaGetLastError();
}

cudaError_t launch_bond_currents(int N, int n_dirs, int Lx, int Ly, int px, int py, const double2 *hop,
                                 const double2 *K, double *J, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  bond_current_kernel<<<blocks(static_cast<long long>(N) * n_dirs, 256), 256, 0, s>>>(N, n_dirs, Lx, Ly, px,
                                                                                      py, hop, K, J);
  return cudaGetLastError();
}

cudaError_t launch_green_weights(int n_E, int M, int kernel, double lambda, const double *energies,
                                 const double *scal, double2 *W, cudaStream_t s) {
  const long long n = static_cast<long long>(n_E) * M;
  if (n <= 0) return cudaSuccess;
  green_weights_kernel<<<blocks(n, 256), 256, 0, s>>>(n_E, M, kernel, lambda, energies, scal, W);
  return cudaGetLastError();
}

cudaError_t launch_green_contract(int n_sites, int n_t, int M, int n_E, const double2 *mom,
                                  const double2 *W, double2 *G, cudaStream_t s) {
  const long long tiles = static_cast<long long>(n_sites) * ((n_t + kGT - 1) / kGT) * ((n_E + kGE - 1) / kGE);
  if (tiles <= 0) return cudaSuccess;
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  green_contract_kernel<<<static_cast<unsigned>(tiles), 256, 0, s>>>(n_sites, n_t, M, n_E, mom, W, G);
  return cudaGetLastError();
}

}  // namespace cbdg
