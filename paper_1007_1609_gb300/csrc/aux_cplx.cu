// aux_cplx.cu -- parameters, start vectors, moment folds and the bond
// order parameter for the general (complex / next-nearest / bond-pairing)
// recursion of step_cplx.cu.  FP64 throughout except the vectors.
#include <math.h>

#include "internal.h"

namespace cbdg {
namespace {

inline int blocks(long long n, int t) { return static_cast<int>((n + t - 1) / t); }

// Field-major parameters: complex field k of site (x, y) at
// ((y * kCplxFields + k) * Lx + x) * 2:  kCpE 2(eps - mu)/a, kCpDelta 2 Delta_i/a
// (on-site pairing), kCpHop + k 2 t_{i,d}/a for the forward directions
// d = 0, 2, 4, 7, kCpBond + k 2 Delta_{i,d}/a for d = 0, 2 (bond pairing);
// the rest 0.
template <typename S>
__global__ void params_cplx_kernel(int N, int Lx, int n_dirs, int pairing, const double *eps, double mu,
                                   const double2 *hop, const double2 *delta, const double *scal,
                                   S *p) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double s2 = 2.0 / scal[kScalA];
  const int x = i % Lx, y = i / Lx;
  auto f = [&](int k, double re, double im) {
    S *q = p + ((static_cast<size_t>(y) * kCplxFields + k) * Lx + x) * 2;
    q[0] = static_cast<S>(re);
    q[1] = static_cast<S>(im);
  };
  for (int k = 0; k < kCplxFields; ++k) f(k, 0.0, 0.0);
  f(kCpE, s2 * (eps[i] - mu), 0.0);
  if (pairing == 0) {
    f(kCpDelta, s2 * delta[i].x, s2 * delta[i].y);
  } else {
    // forward bonds +x (direction 0) and +y (direction 2)
    const double2 bx = delta[static_cast<size_t>(i) * 4 + 0], by = delta[static_cast<size_t>(i) * 4 + 2];
    f(kCpBond + 0, s2 * bx.x, s2 * bx.y);
    f(kCpBond + 1, s2 * by.x, s2 * by.y);
  }
  // forward hoppings +x, +y (directions 0, 2) and, with next-nearest
  // neighbours, +x+y, -x+y (directions 4, 7)
  const int fwd[4] = {0, 2, 4, 7};
  for (int k = 0; k < 4; ++k) {
    if (fwd[k] >= n_dirs) continue;
    const double2 t = hop[static_cast<size_t>(i) * n_dirs + fwd[k]];
    f(kCpHop + k, s2 * t.x, s2 * t.y);
  }
}

template <typename S>
__device__ __forceinline__ void put(S *v, size_t rows, int W, int Lx, int site, int part, int b,
                                    double re, double im) {
  const size_t k = blocked_index(vector_row(Lx, site, part), b, rows, W);
  v[2 * k] = static_cast<S>(re);
  v[2 * k + 1] = static_cast<S>(im);
}

// j_0 = e_i, j_1 = H~ e_i (buffers pre-zeroed):
//   <e_i|j_1> = (eps_i - mu)/a, <h_i|j_1> = conj(Delta_i)/a,
//   <e_j|j_1> = -conj(t_{i,d})/a and, for bond pairing, <h_j|j_1> = conj(Delta_{i,d})/a
// for every neighbour j = i + d.  With on-site pairing also the constants of
// the doubling identities and the n = 0, 1 fold terms.
template <typename S>
__global__ void init_cplx_kernel(int Lx, int Ly, int px, int py, int n_dirs, int pairing,
                                 int ncols, int W, const int32_t *sites, const double *eps,
                                 double mu, const double2 *hop, const double2 *delta,
                                 const double *scal, const double *C, int M, S *j0, S *j1,
                                 double *mu1, double2 *dA, double *acc_n, double2 *acc_d,
                                 double *mu_ee, double2 *mu_eh, int mom_stride) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= ncols) return;
  const double a = scal[kScalA];
  const size_t rows = 2 * static_cast<size_t>(Lx) * Ly;
  const int i = sites[b];
  const double m1 = (eps[i] - mu) / a;
  put(j0, rows, W, Lx, i, 0, b, 1.0, 0.0);
  put(j1, rows, W, Lx, i, 0, b, m1, 0.0);
  double2 dl = make_double2(0.0, 0.0);
  if (pairing == 0) {
    dl = delta[i];
    put(j1, rows, W, Lx, i, 1, b, dl.x / a, -dl.y / a);
  }
  for (int d = 0; d < n_dirs; ++d) {
    const int j = neighbour_site(Lx, Ly, px, py, i, d);
    if (j < 0) continue;
    const double2 t = hop[static_cast<size_t>(i) * n_dirs + d];
    put(j1, rows, W, Lx, j, 0, b, -t.x / a, t.y / a);
    if (pairing == 1 && d < 4) {
      const double2 bd = delta[static_cast<size_t>(i) * 4 + d];
      put(j1, rows, W, Lx, j, 1, b, bd.x / a, -bd.y / a);
    }
  }
  if (pairing == 0) {
    mu1[b] = m1;
    dA[b] = make_double2(dl.x / a, -dl.y / a);
    acc_n[b] = -(C[0] * 1.0 + C[1] * m1);
    acc_d[b] = make_double2(C[1] * dl.x / a, C[1] * dl.y / a);
    if (mu_ee) {
      mu_ee[static_cast<size_t>(b) * M + 0] = 1.0;
      mu_ee[static_cast<size_t>(b) * M + 1] = m1;
    }
    if (mu_eh) {
      mu_eh[(static_cast<size_t>(b) * M + 0) * mom_stride] = make_double2(0.0, 0.0);
      mu_eh[(static_cast<size_t>(b) * M + 1) * mom_stride] = make_double2(dl.x / a, -dl.y / a);
    }
  }
}

// Doubling fold for complex vectors (sums: |j_n|^2, Re<j_{n+1}|j_n>, symplectic re, im).
__global__ void fold_cplx_kernel(int n, int M, int ncols, int ld, int row_split,
                                 const double *partials, const double *C, const double *mu1,
                                 const double2 *dA, double *acc_n, double2 *acc_d, double *mu_ee,
                                 double2 *mu_eh, int mom_stride, unsigned int *flags, double tol) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= ncols) return;
  double A = 0.0, B = 0.0, Cr = 0.0, Ci = 0.0;
  for (int s = 0; s < row_split; ++s) {
    const double *p = partials + static_cast<size_t>(s) * 4 * ld;
    A += p[0 * ld + b];
    B += p[1 * ld + b];
    Cr += p[2 * ld + b];
    Ci += p[3 * ld + b];
  }
  const int m0 = 2 * n, m1 = 2 * n + 1;
  const double e0 = 2.0 * A - 1.0;
  const double e1 = 2.0 * B - mu1[b];
  const double sgn = (n & 1) ? 1.0 : -1.0;
  const double2 da = dA[b];
  const double2 h1 = make_double2(2.0 * sgn * Cr - da.x, 2.0 * sgn * Ci - da.y);
  double an = acc_n[b];
  double2 ad = acc_d[b];
  bool bad = false;
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
  if (!(fabs(e0) < 1e300) || !(fabs(e1) < 1e300)) bad = true;
  acc_n[b] = an;
  acc_d[b] = ad;
  if (bad) atomicOr(flags, kFlagSpectrum);
}

// Direct readout of moment m from vector j_m (bond pairing):
//   mu_ee = Re <e_i|j_m>, mu_eh[0] = <h_i|j_m>, mu_eh[1+d] = <h_{i+d}|j_m>,
// and the fold  acc_n -= C_m mu_ee,  acc_b[d] += C_m conj(mu_eh[1+d]).
template <typename S>
__global__ void gather_kernel(int m, int M, int Lx, int Ly, int px, int py, int ncols, int W,
                              const int32_t *sites, const S *j, const double *C, double *acc_n,
                              double2 *acc_b, double *mu_ee, double2 *mu_eh,
                              unsigned int *flags, double tol) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= ncols) return;
  const size_t rows = 2 * static_cast<size_t>(Lx) * Ly;
  const int i = sites[b];
  auto get = [&](int site, int part) {
    const size_t k = blocked_index(vector_row(Lx, site, part), b, rows, W);
    return make_double2(static_cast<double>(j[2 * k]), static_cast<double>(j[2 * k + 1]));
  };
  const double2 ee = get(i, 0);
  const double2 hh = get(i, 1);
  const double cm = C[m];
  acc_n[b] -= cm * ee.x;
  if (mu_ee) mu_ee[static_cast<size_t>(b) * M + m] = ee.x;
  if (mu_eh) mu_eh[(static_cast<size_t>(b) * M + m) * 5] = hh;
  for (int d = 0; d < 4; ++d) {
    const int jn = neighbour_site(Lx, Ly, px, py, i, d);
    const double2 h = jn >= 0 ? get(jn, 1) : make_double2(0.0, 0.0);
    double2 ab = acc_b[static_cast<size_t>(b) * 4 + d];
    ab.x += cm * h.x;
    ab.y -= cm * h.y;
    acc_b[static_cast<size_t>(b) * 4 + d] = ab;
    if (mu_eh) mu_eh[(static_cast<size_t>(b) * M + m) * 5 + 1 + d] = h;
  }
  if (!(fabs(ee.x) <= 1.0 + tol)) atomicOr(flags, kFlagSpectrum);
}

// Delta_{i,d} = (V_{i,d}/8) (acc_b[i][d] + acc_b[i+d][d^1]),  n_i = 1 + acc_n[i]
// (accumulators indexed by site; every site was a start vector; V_{i,d} =
// V_site[4i + d], or the lattice's V when V_site is NULL).
__global__ void finalize_bond_kernel(int N, int Lx, int Ly, int px, int py, double V_all,
                                     const double *V_site, const double *acc_n, const double2 *acc_b,
                                     double2 *dout, double *nout) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  for (int d = 0; d < 4; ++d) {
    const int j = neighbour_site(Lx, Ly, px, py, i, d);
    double2 r = make_double2(0.0, 0.0);
    if (j >= 0) {
      const double V = V_site ? V_site[static_cast<size_t>(i) * 4 + d] : V_all;
      const double2 f = acc_b[static_cast<size_t>(i) * 4 + d];
      const double2 g = acc_b[static_cast<size_t>(j) * 4 + (d ^ 1)];
      r = make_double2(0.125 * V * (f.x + g.x), 0.125 * V * (f.y + g.y));
    }
    if (dout) dout[static_cast<size_t>(i) * 4 + d] = r;
  }
  if (nout) nout[i] = 1.0 + acc_n[i];
}

}  // namespace

cudaError_t launch_params_cplx(int precision, int N, int Lx, int n_dirs, int pairing, const double *eps,
                               double mu, const double2 *hop, const double2 *delta,
                               const double *scal, void *params, cudaStream_t s) {
  if (precision == 1)
    params_cplx_kernel<float><<<blocks(N, 128), 128, 0, s>>>(N, Lx, n_dirs, pairing, eps, mu, hop, delta,
                                                             scal, static_cast<float *>(params));
  else
    params_cplx_kernel<double><<<blocks(N, 128), 128, 0, s>>>(N, Lx, n_dirs, pairing, eps, mu, hop,
                                                              delta, scal, static_cast<double *>(params));
  return cudaGetLastError();
}

cudaError_t launch_init_cplx(int precision, int Lx, int Ly, int px, int py, int n_dirs, int pairing,
                             int ncols, int W, const int32_t *sites, const double *eps, double mu,
                             const double2 *hop, const double2 *delta, const double *scal,
                             const double *C, int M, void *j0, void *j1, double *mu1, double2 *dA,
                             double *acc_n, double2 *acc_d, double *mu_ee, double2 *mu_eh,
                             int mom_stride, cudaStream_t s) {
  if (ncols <= 0) return cudaSuccess;
  if (precision == 1)
    init_cplx_kernel<float><<<blocks(ncols, 128), 128, 0, s>>>(
        Lx, Ly, px, py, n_dirs, pairing, ncols, W, sites, eps, mu, hop, delta, scal, C, M,
        static_cast<float *>(j0), static_cast<float *>(j1), mu1, dA, acc_n, acc_d, mu_ee, mu_eh,
        mom_stride);
  else
    init_cplx_kernel<double><<<blocks(ncols, 128), 128, 0, s>>>(
        Lx, Ly, px, py, n_dirs, pairing, ncols, W, sites, eps, mu, hop, delta, scal, C, M,
        static_cast<double *>(j0), static_cast<double *>(j1), mu1, dA, acc_n, acc_d, mu_ee, mu_eh,
        mom_stride);
  return cudaGetLastError();
}

cudaError_t launch_fold_cplx(int n, int M, int ncols, int ld, int row_split, const double *partials,
                             const double *C, const double *mu1, const double2 *dA, double *acc_n,
                             double2 *acc_d, double *mu_ee, double2 *mu_eh, int mom_stride,
                             unsigned int *flags, double tol, cudaStream_t s) {
  if (ncols <= 0) return cudaSuccess;
  fold_cplx_kernel<<<blocks(ncols, 256), 256, 0, s>>>(n, M, ncols, ld, row_split, partials, C, mu1,
                                                      dA, acc_n, acc_d, mu_ee, mu_eh, mom_stride,
                                                      flags, tol);
  return cudaGetLastError();
}

cudaError_t launch_gather(int precision, int m, int M, int Lx, int Ly, int px, int py, int ncols,
                          int W, const int32_t *sites, const void *j, const double *C,
                          double *acc_n, double2 *acc_b, double *mu_ee, double2 *mu_eh,
                          unsigned int *flags, double tol, cudaStream_t s) {
  if (ncols <= 0) return cudaSuccess;
  if (precision == 1)
    gather_kernel<float><<<blocks(ncols, 128), 128, 0, s>>>(m, M, Lx, Ly, px, py, ncols, W, sites,
                                                            static_cast<const float *>(j), C, acc_n,
                                                            acc_b, mu_ee, mu_eh, flags, tol);
  else
    gather_kernel<double><<<blocks(ncols, 128), 128, 0, s>>>(m, M, Lx, Ly, px, py, ncols, W, sites,
                                                             static_cast<const double *>(j), C, acc_n,
                                                             acc_b, mu_ee, mu_eh, flags, tol);
  return cudaGetLastError();
}

cudaError_t launch_finalize_bond(int N, int Lx, int Ly, int px, int py, double V, const double *V_site,
                                 const double *acc_n, const double2 *acc_b, double2 *dout,
                                 double *nout, cudaStream_t s) {
  finalize_bond_kernel<<<blocks(N, 256), 256, 0, s>>>(N, Lx, Ly, px, py, V, V_site, acc_n, acc_b, dout,
                                                      nout);
  return cudaGetLastError();
}

}  // namespace cbdg
