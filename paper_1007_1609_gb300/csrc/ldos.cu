// ldos.cu -- the LDOS weight table of Eq. 17 with the expansion of Eq. 10,
//   W[e][n] = g_n (2 - delta_n0) T_n(E_e / a) / (pi a sqrt(1 - (E_e/a)^2)),
// built in FP64 and stored as the TF32 head / tail planes that the
// tensor-core contraction LDOS[site][e] = sum_n mu_n(site) W[e][n] reads
// (K-major, row stride kp = M rounded up to 32, zero padded).
//
// The adjoint of that contraction (a loss on the LDOS): with
// G[c][e] = dL/dLDOS(E_e, site c), the loss's derivative with respect to the
// moment mu_n(site c) is S[c][n] = sum_e G[c][e] W[e][n], formed here in FP64
// (the table W in FP64, then one thread per (c, n)); S is the source of the
// reverse recursion in adjoint.cu.
#include <math.h>

#include "internal.h"

namespace cbdg {
namespace {

inline int blocks(long long n, int t) { return static_cast<int>((n + t - 1) / t); }

__device__ __forceinline__ float tf32_rna(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// W[e][n] of Eq. 17 for n < M at x = E / a (Jackson or Lorentz g_n).
__device__ __forceinline__ double ldos_weight(int n, int M, int kernel, double lambda, double x, double a) {
  double g;
  if (kernel == 0) {
    const double q = 1.0 / (M + 1.0);
    g = ((M - n + 1) * cospi(n * q) + sinpi(n * q) * cospi(q) / sinpi(q)) / (M + 1.0);
  } else {
    g = sinh(lambda * (1.0 - static_cast<double>(n) / M)) / sinh(lambda);
  }
  const double th = acos(x);
  const double tn = cos(n * th);
  return g * (n == 0 ? 1.0 : 2.0) * tn / (M_PI * a * sqrt(1.0 - x * x));
}

__global__ void ldos_weights_kernel(int n_E, int M, int ld, int kernel, double lambda,
                                    const double *energies, const double *scal, float *w_hi, float *w_lo) {
  const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= static_cast<long long>(n_E) * ld) return;
  const int e = static_cast<int>(idx / ld);
  const int n = static_cast<int>(idx % ld);
  double w = 0.0;
  if (n < M) {
    const double a = scal[kScalA];
    w = ldos_weight(n, M, kernel, lambda, energies[e] / a, a);
  }
  const float h = tf32_rna(static_cast<float>(w));
  w_hi[static_cast<size_t>(e) * ld + n] = h;
  w_lo[static_cast<size_t>(e) * ld + n] = tf32_rna(static_cast<float>(w - static_cast<double>(h)));
}

// W[e][n], FP64, [n_E][M]
__global__ void ldos_weights_f64_kernel(int n_E, int M, int kernel, double lambda, const double *energies,
                                        const double *scal, double *W) {
  const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= static_cast<long long>(n_E) * M) return;
  const int e = static_cast<int>(idx / M), n = static_cast<int>(idx % M);
  const double a = scal[kScalA];
  W[idx] = ldos_weight(n, M, kernel, lambda, energies[e] / a, a);
}

// S[c][n] = sum_e G[c][e] W[e][n]; consecutive threads take consecutive n of
// one c (coalesced reads of W, one broadcast value of G per e).
__global__ void ldos_source_kernel(int n_sites, int n_E, int M, const double *__restrict__ G,
                                   const double *__restrict__ W, double *__restrict__ S) {
  const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= static_cast<long long>(n_sites) * M) return;
  const int c = static_cast<int>(idx / M), n = static_cast<int>(idx % M);
  const double *g = G + static_cast<size_t>(c) * n_E;
  double s = 0.0;
  for (int e = 0; e < n_E; ++e) s = fma(g[e], W[static_cast<size_t>(e) * M + n], s);
  S[idx] = s;
}

}  // namespace

cudaError_t launch_ldos_source(int n_sites, int n_E, int M, int kernel, double lambda, const double *energies,
                               const double *scal, const double *G, double *W, double *S, cudaStream_t s) {
  if (n_sites <= 0 || M <= 0) return cudaSuccess;
  ldos_weights_f64_kernel<<<blocks(static_cast<long long>(n_E) * M, 256), 256, 0, s>>>(n_E, M, kernel, lambda,
                                                                                        energies, scal, W);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ldos_source_kernel<<<blocks(static_cast<long long>(n_sites) * M, 256), 256, 0, s>>>(n_sites, n_E, M, G, W, S);
  return cudaGetLastError();
}

cudaError_t launch_ldos_weights(int n_E, int M, int ld, int kernel, double lambda,
                                const double *energies, const double *scal, float *w_hi, float *w_lo,
                                cudaStream_t s) {
  if (n_E <= 0) return cudaSuccess;
  ldos_weights_kernel<<<blocks(static_cast<long long>(n_E) * ld, 256), 256, 0, s>>>(n_E, M, ld, kernel, lambda,
                                                                                     energies, scal, w_hi, w_lo);
  return cudaGetLastError();
}

}  // namespace cbdg
