// adjoint.cu -- reverse-mode gradient of one self-consistency map
// Delta_out(eps, t, Delta_in) (Eq. 19 through Eq. 15), with a and the
// coefficients C_n frozen, for real on-site (s-wave) lattices.
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
// accumulation (one thread per (site, column group), 12 FP64 sums per site:
// e-e, h-h, e-h, h-e on site and e-e, h-h to each of the 4 neighbours; fixed
// order, no atomics) and the final contraction with dH/dparameter.
#include "internal.h"

namespace cbdg {
namespace {

inline int blocks(long long n, int t) { return static_cast<int>((n + t - 1) / t); }

template <typename S>
__global__ void adjoint_source_kernel(int Lx, int Ly, int ncols, int W, const int32_t *sites,
                                      const double *w, double scale_m, S *lam) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= ncols) return;
  const int i = sites[b];
  const size_t rows = 2 * static_cast<size_t>(Lx) * Ly;
  const size_t k = blocked_index(vector_row(Lx, i, 1), b, rows, W);
  lam[k] = static_cast<S>(static_cast<double>(lam[k]) + w[i] * scale_m);
}

// part[g][site][12] += f * sum_{b in group g} lam(r, b) j(s, b) on the pattern.
template <typename S>
__global__ void adjoint_accumulate_kernel(int Lx, int Ly, int px, int py, int ld, int W,
                                          int cols_per_group, const S *lam, const S *j, double f,
                                          double *part) {
  const int N = Lx * Ly;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int g = blockIdx.y;
  if (i >= N) return;
  const int x = i % Lx, y = i / Lx;
  const size_t rows = 2 * static_cast<size_t>(N);
  const int DX[4] = {1, -1, 0, 0}, DY[4] = {0, 0, 1, -1};
  int nb[4];
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
    nb[d] = ok ? nx + Lx * ny : -1;
  }
  const size_t re = vector_row(Lx, i, 0), rh = vector_row(Lx, i, 1);
  double acc[12];
  for (int k = 0; k < 12; ++k) acc[k] = 0.0;
  const int b0 = g * cols_per_group, b1 = min(ld, b0 + cols_per_group);
  for (int b = b0; b < b1; ++b) {
    const double le = lam[blocked_index(re, b, rows, W)], lh = lam[blocked_index(rh, b, rows, W)];
    const double je = j[blocked_index(re, b, rows, W)], jh = j[blocked_index(rh, b, rows, W)];
    acc[0] += le * je;
    acc[1] += lh * jh;
    acc[2] += le * jh;
    acc[3] += lh * je;
    for (int d = 0; d < 4; ++d) {
      if (nb[d] < 0) continue;
      acc[4 + d] += le * static_cast<double>(j[blocked_index(vector_row(Lx, nb[d], 0), b, rows, W)]);
      acc[8 + d] += lh * static_cast<double>(j[blocked_index(vector_row(Lx, nb[d], 1), b, rows, W)]);
    }
  }
  double *p = part + (static_cast<size_t>(g) * N + i) * 12;
  for (int k = 0; k < 12; ++k) p[k] += f * acc[k];
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
        v = (-G(i, 4 + d) - G(jn, 4 + db) + G(i, 8 + d) + G(jn, 8 + db)) / a;
      }
      g_hop[static_cast<size_t>(i) * 4 + d] = v;
    }
  }
}

}  // namespace

cudaError_t launch_adjoint_source(int precision, int Lx, int Ly, int ncols, int W,
                                  const int32_t *sites, const double *w, double scale_m, void *lam,
                                  cudaStream_t s) {
  if (ncols <= 0) return cudaSuccess;
  if (precision == 1)
    adjoint_source_kernel<float><<<blocks(ncols, 128), 128, 0, s>>>(Lx, Ly, ncols, W, sites, w, scale_m,
                                                                    static_cast<float *>(lam));
  else
    adjoint_source_kernel<double><<<blocks(ncols, 128), 128, 0, s>>>(Lx, Ly, ncols, W, sites, w, scale_m,
                                                                     static_cast<double *>(lam));
  return cudaGetLastError();
}

cudaError_t launch_adjoint_accumulate(int precision, int Lx, int Ly, int px, int py, int ld, int W,
                                      int groups, const void *lam, const void *j, double f,
                                      double *part, cudaStream_t s) {
  const int N = Lx * Ly;
  const int cpg = (ld + groups - 1) / groups;
  dim3 grid(blocks(N, 128), groups);
  if (precision == 1)
    adjoint_accumulate_kernel<float><<<grid, 128, 0, s>>>(Lx, Ly, px, py, ld, W, cpg,
                                                          static_cast<const float *>(lam),
                                                          static_cast<const float *>(j), f, part);
  else
    adjoint_accumulate_kernel<double><<<grid, 128, 0, s>>>(Lx, Ly, px, py, ld, W, cpg,
                                                           static_cast<const double *>(lam),
                                                           static_cast<const double *>(j), f, part);
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
