// ldos.cu -- the LDOS weight table of Eq. 17 with the expansion of Eq. 10,
//   W[e][n] = g_n (2 - delta_n0) T_n(E_e / a) / (pi a sqrt(1 - (E_e/a)^2)),
// built in FP64 and stored in FP32 for the tensor-core contraction
// LDOS[site][e] = sum_n mu_n(site) W[e][n], and the FP64 -> FP32 copy of
// the moments.  Both operands are K-major (n contiguous) with a row stride
// padded to a multiple of 4 so that 16-byte loads stay aligned.
#include <math.h>

#include "internal.h"

namespace cbdg {
namespace {

inline int blocks(long long n, int t) { return static_cast<int>((n + t - 1) / t); }

__global__ void ldos_weights_kernel(int n_E, int M, int ld, int kernel, double lambda,
                                    const double *energies, const double *scal, float *W) {
  const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= static_cast<long long>(n_E) * ld) return;
  const int e = static_cast<int>(idx / ld);
  const int n = static_cast<int>(idx % ld);
  float w = 0.f;
  if (n < M) {
    const double a = scal[kScalA];
    const double x = energies[e] / a;
    double g;
    if (kernel == 0) {
      const double q = 1.0 / (M + 1.0);
      g = ((M - n + 1) * cospi(n * q) + sinpi(n * q) * cospi(q) / sinpi(q)) / (M + 1.0);
    } else {
      g = sinh(lambda * (1.0 - static_cast<double>(n) / M)) / sinh(lambda);
    }
    const double th = acos(x);
    const double tn = cos(n * th);
    w = static_cast<float>(g * (n == 0 ? 1.0 : 2.0) * tn / (M_PI * a * sqrt(1.0 - x * x)));
  }
  W[static_cast<size_t>(e) * ld + n] = w;
}

__global__ void moments_to_f32_kernel(int rows, int M, int ld, const double *mu, float *out) {
  const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= static_cast<long long>(rows) * ld) return;
  const int r = static_cast<int>(idx / ld);
  const int n = static_cast<int>(idx % ld);
  out[static_cast<size_t>(r) * ld + n] = n < M ? static_cast<float>(mu[static_cast<size_t>(r) * M + n]) : 0.f;
}

}  // namespace

cudaError_t launch_ldos_weights(int n_E, int M, int ld, int kernel, double lambda,
                                const double *energies, const double *scal, float *W,
                                cudaStream_t s) {
  if (n_E <= 0) return cudaSuccess;
  ldos_weights_kernel<<<blocks(static_cast<long long>(n_E) * ld, 256), 256, 0, s>>>(n_E, M, ld, kernel, lambda, energies, scal, W);
  return cudaGetLastError();
}

cudaError_t launch_moments_to_f32(int rows, int M, int ld, const double *mu, float *out,
                                  cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  moments_to_f32_kernel<<<blocks(static_cast<long long>(rows) * ld, 256), 256, 0, s>>>(rows, M, ld, mu, out);
  return cudaGetLastError();
}

}  // namespace cbdg
