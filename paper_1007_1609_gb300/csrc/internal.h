// internal.h -- declarations shared by the translation units of libcbdg.
// Not part of the public ABI (include/cbdg.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cbdg {

// Parameter record per site in the step precision S, 8 scalars (32 B for
// float, 64 B for double), pre-multiplied by 2/a so that one stencil
// application yields 2 H~ j:
//   [0] 2 (eps - mu)/a   [1] 2 Delta/a   [2..5] 2 t_{s,d}/a (d = 0..3)   [6,7] 0
constexpr int kParamStride = 8;
// General (complex / next-nearest / bond) parameters: 8 complex fields per
// site, stored field-major inside each lattice row, field f of site (x, y)
// (real, imaginary) at
//   params[((y * kCplxFields + f) * Lx + x) * 2 + {0, 1}]
// so that a lattice row is one contiguous block of kCplxParamStride * Lx
// scalars and threads on consecutive x read consecutive pairs.  Only the
// forward half of the Hermitian hoppings and of the symmetric bond pairing is
// stored (the backward half is the neighbour's, see step_cplx.cu).  Fields:
//   [0] (2(eps-mu)/a, 0)  [1] 2 Delta_i/a
//   [2..5] 2 t_{i,d}/a for d = +x, +y, +x+y, -x+y
//   [6, 7] 2 Delta_{i,d}/a for d = +x, +y
constexpr int kCplxFields = 8;
constexpr int kCplxParamStride = 2 * kCplxFields;
constexpr int kCpE = 0, kCpDelta = 1, kCpHop = 2, kCpBond = 6;

// Arguments of one recursion step j_{n+1} = 2 H~ j_n - j_{n-1} over a block
// of ld start vectors.  Vectors use the slab-blocked layout: column slab
// c = b / W is a row-major [2N][W] block at offset c * 2N * W, so element
// (row r, column b) sits at (b / W) * 2N*W + r*W + (b % W).  Rows go lattice
// row by lattice row; inside lattice row y the Lx electron rows come first,
// then the Lx hole rows (vector_row below).
// One-element sources of a multi-step pass with per-level outputs (the
// adjoint's reverse recursion, lam_m = y_m + 2 H~ lam_{m+1} - lam_{m+2}):
// level t adds to column c, at the electron (part 0) or hole (part 1) row of
// its start site i = sites[c], the value
//     w[i] u[i] (scale tab[stride c + m]),   m = m0 + dm t,
// with w, u taken as 1 where null.  sites == nullptr: no sources.
struct PassSource {
  const int32_t *sites = nullptr;
  int ncols = 0;  // columns with a start site (the rest are padding)
  const double *w = nullptr;
  const double *u = nullptr;
  const double *tab = nullptr;
  int stride = 0;
  double scale = 1.0;
  int m0 = 0, dm = -1;
  int part = 1;
};

struct StepArgs {
  const void *cur;      // j_n
  void *prev;           // j_{n-1} on entry, j_{n+1} on exit (in place)
  const void *params;   // [N][kParamStride] scalars of the step precision
  double *partials;     // [row_split][3][ld]: sum |j_n|^2, <j_{n+1}|j_n>, symplectic
  unsigned int *flags;  // error bits (kFlagTimeout when a staged copy never arrived)
  unsigned long long wait_ns;  // limit of every wait on a staged copy
  unsigned stall_tx;    // test hook: extra bytes the first staged row expects (never arrive)
  int Lx, Ly;
  int ld;               // columns (a multiple of the slab width)
  int rows_per_cta;     // lattice rows per CTA along y
  void *out = nullptr;  // one-step kernels: j_{n+1} goes here when set (prev is kept)
  // multi-step kernels: when lvout[K-1] is set, level t (j_{n+t}) goes to
  // lvout[t-1] where that is set, (prev, cur) are only read and no column
  // sums are formed
  void *lvout[4] = {nullptr, nullptr, nullptr, nullptr};
  PassSource src;       // sources of the per-level-output passes
};

struct StepConfig {
  int slab_w;           // columns per CTA (W)
  int depth;            // lattice rows staged ahead (D)
  int row_split;        // CTAs per column slab along y
  int threads;
  size_t smem;
  int pstage = 1;       // real one-step kernel: 0 = parameters through the read-only cache (wide lattices)
  int blocked = 0;      // multi-step pass over row blocks of row_split lattice rows, out of place
};

// Storage row of the electron (part 0) or hole (part 1) component of site s.
__host__ __device__ inline size_t vector_row(int Lx, size_t s, int part) {
  return 2 * static_cast<size_t>(Lx) * (s / Lx) + static_cast<size_t>(part) * Lx + (s % Lx);
}

// Offset of element (row r, column b) in the slab-blocked layout.
__host__ __device__ inline size_t blocked_index(size_t r, size_t b, size_t rows, int W) {
  return (b / W) * rows * W + r * W + (b % W);
}

// Neighbour of site s = x + Lx*y along direction d (0:+x 1:-x 2:+y 3:-y
// 4:+x+y 5:-x-y 6:+x-y 7:-x+y), or -1 where an open edge cuts the bond.
__host__ __device__ inline int neighbour_site(int Lx, int Ly, int px, int py, int s, int d) {
  const int dx = (d == 0 || d == 4 || d == 6) ? 1 : (d == 1 || d == 5 || d == 7) ? -1 : 0;
  const int dy = (d == 2 || d == 4 || d == 7) ? 1 : (d == 3 || d == 5 || d == 6) ? -1 : 0;
  int x = s % Lx + dx, y = s / Lx + dy;
  if (x < 0 || x >= Lx) {
    if (!px) return -1;
    x = (x + Lx) % Lx;
  }
  if (y < 0 || y >= Ly) {
    if (!py) return -1;
    y = (y + Ly) % Ly;
  }
  return x + Lx * y;
}

// Recursion step for real on-site (s-wave) lattices with nearest-neighbour
// hopping.  precision 0: double, 1: float.
cudaError_t launch_step_real(int precision, const StepArgs &a, const StepConfig &cfg,
                             cudaStream_t s);
// Fills cfg for the given shape; returns false if no instantiation fits.
bool plan_step_real(int precision, int Lx, int Ly, int ld, int want_w, int want_split,
                    int want_depth, StepConfig *cfg);
int slab_width_default(int precision);
// Lattice-row split of the one-step kernels: CTAs per column slab, chosen
// from the SM count and how many CTAs of `smem` bytes fit on an SM.
int choose_row_split(int slabs, int Ly, size_t smem, int threads);

// K recursion steps per pass (temporal blocking) for real on-site FP32
// lattices with open y edges; one CTA per slab (row split 1).  Partial sums
// are [K][3][ld].  plan_step_multi returns false when the shape has no
// instantiation or the rings do not fit in shared memory.
bool plan_step_multi(int Lx, int Ly, int ld, int want_w, int want_k, int want_depth,
                     StepConfig *cfg, int *k_out);
// Two steps per pass over row blocks with recomputed halos (real FP32, open
// y edges, slab width 4 or 8): for lattices too wide for the whole-column
// pass.  Fills cfg (row_split = blocks per slab); false if it does not fit.
bool plan_step_multi_blocked(int Lx, int Ly, int ld, int W, StepConfig *cfg);
cudaError_t launch_step_multi(const StepArgs &a, const StepConfig &cfg, int K, cudaStream_t s);

// Whole recursion in shared memory for small real on-site lattices
// (resident.cu): plan_resident returns the slab width (1, 2 or 4) or 0 when
// the lattice does not fit; launch_resident runs steps 1..steps with the
// folds of fold_kernel on j_0, j_1 written by init_real at that width.
int plan_resident(int precision, int Lx, int Ly, int ncols, int M);
cudaError_t launch_resident(int precision, int W, int Lx, int Ly, int ld, int ncols, int M, int steps,
                            const void *j0, const void *j1, const void *params, const double *C,
                            const double *mu1, const double2 *dA, double *acc_n, double2 *acc_d,
                            double *mu_ee, double2 *mu_eh, int mom_stride, unsigned int *flags, double tol,
                            cudaStream_t s);

// Recursion step for the general lattice (complex vectors; nnn: 8 hopping
// directions; bond: nearest-neighbour pairing, which skips the column sums).
// The partial sums, when formed, are [row_split][4][ld].
cudaError_t launch_step_cplx(int precision, int nnn, int bond, const StepArgs &a,
                             const StepConfig &cfg, cudaStream_t s);
bool plan_step_cplx(int precision, int Lx, int Ly, int ld, int want_w, int want_split,
                    int want_depth, StepConfig *cfg);
// Two steps per pass over the vectors for the general lattice (FP32 complex,
// step_cplx_multi.cu): j_{n+1} into prev, j_{n+2} into cur, both in place;
// with on-site pairing the column sums of both steps in partials [2][4][ld].
// Slab width 2, one CTA per slab; returns false when the shape does not fit.
bool plan_step_cplx_multi(int precision, int Lx, int Ly, int ld, StepConfig *cfg);
cudaError_t launch_step_cplx_multi(int nnn, int bond, const StepArgs &a, const StepConfig &cfg, cudaStream_t s);
int slab_width_default_cplx(int precision);
cudaError_t launch_params_cplx(int precision, int N, int Lx, int n_dirs, int pairing, const double *eps,
                               double mu, const double2 *hop, const double2 *delta,
                               const double *scal, void *params, cudaStream_t s);
cudaError_t launch_init_cplx(int precision, int Lx, int Ly, int px, int py, int n_dirs, int pairing,
                             int ncols, int W, const int32_t *sites, const double *eps, double mu,
                             const double2 *hop, const double2 *delta, const double *scal,
                             const double *C, int M, void *j0, void *j1, double *mu1, double2 *dA,
                             double *acc_n, double2 *acc_d, double *mu_ee, double2 *mu_eh,
                             int mom_stride, cudaStream_t s);
cudaError_t launch_fold_cplx(int n, int M, int ncols, int ld, int row_split, const double *partials,
                             const double *C, const double *mu1, const double2 *dA, double *acc_n,
                             double2 *acc_d, double *mu_ee, double2 *mu_eh, int mom_stride,
                             unsigned int *flags, double tol, cudaStream_t s);
cudaError_t launch_gather(int precision, int m, int M, int Lx, int Ly, int px, int py, int ncols,
                          int W, const int32_t *sites, const void *j, const double *C,
                          double *acc_n, double2 *acc_b, double *mu_ee, double2 *mu_eh,
                          unsigned int *flags, double tol, cudaStream_t s);
// V_site (may be NULL): a coupling per bond [N*4] in place of V.
cudaError_t launch_finalize_bond(int N, int Lx, int Ly, int px, int py, double V, const double *V_site,
                                 const double *acc_n, const double2 *acc_b, double2 *dout,
                                 double *nout, cudaStream_t s);

// ---- nonlocal readout, bond currents, Green's function (green.cu) -----------
// Moment m at every (column, target) of j_m; targets == NULL: the neighbours
// of each column's start site along directions 0..n_t-1.  Any output may be NULL.
cudaError_t launch_target_gather(int precision, int m, int M, int Lx, int Ly, int px, int py, int ncols,
                                 int W, const int32_t *sites, int n_t, const int32_t *targets,
                                 const void *j, const double *C, double2 *acc, double2 *a_e,
                                 double2 *a_h, unsigned int *flags, double tol, cudaStream_t s);
cudaError_t launch_bond_currents(int N, int n_dirs, int Lx, int Ly, int px, int py, const double2 *hop,
                                 const double2 *K, double *J, cudaStream_t s);
cudaError_t launch_green_weights(int n_E, int M, int kernel, double lambda, const double *energies,
                                 const double *scal, double2 *W, cudaStream_t s);
cudaError_t launch_green_contract(int n_sites, int n_t, int M, int n_E, const double2 *mom,
                                  const double2 *W, double2 *G, cudaStream_t s);

// ---- auxiliary kernels (aux.cu) -------------------------------------------
cudaError_t launch_gershgorin(int N, int n_dirs, int pairing, int Lx, int Ly, int px, int py,
                              const double *eps, double mu, const double2 *hop,
                              const double2 *delta, double margin, double *scal, cudaStream_t s);
// Coefficient table C[M] (Eqs. 6-7 with the kernel of Eq. 16 or Jackson);
// work holds coefficient_work(M, K) doubles.
size_t coefficient_work(int M, int K);
cudaError_t launch_coefficients(int M, int K, double T, int kernel, double lambda,
                                const double *scal, double *work, double *C, cudaStream_t s);
cudaError_t launch_params_real(int precision, int N, const double *eps, double mu,
                               const double2 *hop, const double2 *delta, const double *scal,
                               void *params, cudaStream_t s);
cudaError_t launch_init_real(int precision, int Lx, int Ly, int px, int py, int ncols, int W,
                             const int32_t *sites, const double *eps, double mu,
                             const double2 *hop, const double2 *delta, const double *scal,
                             const double *C, int M, void *j0, void *j1, double *mu1,
                             double2 *dA, double *acc_n, double2 *acc_d, double *mu_ee,
                             double2 *mu_eh, int mom_stride, cudaStream_t s);
// levels > 1: steps n .. n + levels - 1 of a multi-step pass, partials [levels][3][ld].
cudaError_t launch_fold(int n, int M, int ncols, int ld, int row_split, const double *partials,
                        const double *C, const double *mu1, const double2 *dA, double *acc_n,
                        double2 *acc_d, double *mu_ee, double2 *mu_eh, int mom_stride,
                        unsigned int *flags, double tol, cudaStream_t s, int levels = 1);
// U_site (may be NULL): a coupling per site [N] in place of U.
cudaError_t launch_finalize_onsite(int ncols, const int32_t *sites, double U, const double *U_site,
                                   const double *acc_n, const double2 *acc_d, double2 *dout,
                                   double *nout, cudaStream_t s);
cudaError_t launch_mix(int n, double mix, const double2 *dout, double2 *delta, double *scal,
                       cudaStream_t s);
// dst[k] = (src[k], 0), k < n.
cudaError_t launch_real_to_complex(int n, const double *src, double2 *dst, cudaStream_t s);
// dout[i], nout[i] <- dout[rep[i]], nout[rep[i]] for every non-representative i.
cudaError_t launch_orbit_fill(int N, const int32_t *rep, double2 *dout, double *nout, cudaStream_t s);
cudaError_t launch_ldos_eval(int n_sites, int M, int kernel, double lambda, const double *mu_ee,
                             const double *energies, int n_E, const double *scal, float *ldos,
                             cudaStream_t s);

// Device scalars block (double[kScalars]).
enum {
  kScalBoundBits = 0,   // Gershgorin bound, as ordered bits (atomicMax)
  kScalA = 1,           // a = 1.1 * bound
  kScalMaxDiffBits = 2, // max |Delta_out - Delta|, as ordered bits
  kScalars = 4
};
// Error flags (unsigned int bits).
enum { kFlagSpectrum = 1u, kFlagTimeout = 2u };

// Dense D[m][n] = sum_k A[m][k] B[n][k] on tcgen05 tensor cores with the
// 3xTF32 split (contract.cu).  launch_contract_tf32x3 splits FP32 operands
// into TF32 hi / lo planes [rows][kp] (kp = contract_kp(k), zero padded) in
// stream-ordered scratch and contracts them; callers that build operands
// themselves write the planes directly (launch_split_tf32*) and call
// launch_contract_planes.
cudaError_t launch_contract_tf32x3(const float *A, int lda, const float *B, int ldb, float *D,
                                   int ldd, int m, int n, int k, unsigned *flags, cudaStream_t s);
int contract_kp(int k);
cudaError_t launch_split_tf32(const float *src, size_t ld, int rows, int k, int kp, float *hi, float *lo,
                              cudaStream_t s);
cudaError_t launch_split_tf32_f64(const double *src, size_t ld, int rows, int k, int kp, float *hi,
                                  float *lo, cudaStream_t s);
cudaError_t launch_contract_planes(const float *a_hi, const float *a_lo, const float *b_hi, const float *b_lo,
                                   int kp, float *D, int ldd, int m, int n, unsigned *flags, cudaStream_t s);
// Adjoint of one self-consistency map (adjoint.cu).
// lam(h_i) += w_i u_i scale_m, u_i = U_site[i] (or 1 when U_site is NULL).
cudaError_t launch_adjoint_source(int precision, int Lx, int Ly, int ncols, int W,
                                  const int32_t *sites, const double *w, const double *U_site,
                                  double scale_m, void *lam, cudaStream_t s);
// lam(e_i) += src[b * M + m] for column b (start site i = sites[b]).
cudaError_t launch_adjoint_source_table(int precision, int Lx, int Ly, int ncols, int W, const int32_t *sites,
                                        const double *src, int M, int m, void *lam, cudaStream_t s);
// Source table of the LDOS-loss adjoint: W [n_E][M] (work) = the FP64 weights
// of Eq. 17, S [n_sites][M] = G [n_sites][n_E] . W.
cudaError_t launch_ldos_source(int n_sites, int n_E, int M, int kernel, double lambda, const double *energies,
                               const double *scal, const double *G, double *W, double *S, cudaStream_t s);
// Column groups of the accumulation for ld columns at slab width W on Ly rows.
int adjoint_groups(int Ly, int ld, int W);
// column-slab groups of launch_adjoint_accumulate (the FP32 kernel with staged
// rows, slab width 16, Lx <= 128, sizes its own grid)
int adjoint_groups_real(int precision, int Lx, int Ly, int ld, int W);
cudaError_t launch_adjoint_accumulate(int precision, int Lx, int Ly, int px, int py, int ld, int W,
                                      int groups, const void *lam, const void *j, double f,
                                      double *part, unsigned long long wait_ns, unsigned *flags,
                                      cudaStream_t s);
cudaError_t launch_fixed_point_update(int N, double mix, const double *g, const double *gd, double *lam,
                                      double *w, double *scal, cudaStream_t s);
cudaError_t launch_adjoint_final(int Lx, int Ly, int px, int py, int groups, const double *part,
                                 const double *scal, double *g_eps, double *g_hop, double *g_delta,
                                 cudaStream_t s);

// Rate probe of tcgen05.mma kind::tf32 at the contraction's shape (M = 128,
// N = 256, K = 8): `ctas` CTAs (one per SM) issue `mmas` MMAs each.
cudaError_t launch_tf32_peak(int ctas, long long mmas, unsigned *flags, cudaStream_t s);
double tf32_peak_flops_per_mma();

// Adjoint of the map for general lattices (adjoint_cplx.cu): complex vectors,
// nd = 4 or 8 hopping directions, bond = nearest-neighbour pairing.
// Sums per site of the accumulation (part is [groups][N][2 * sums]).
int adjoint_cplx_sums(int nd, int bond);
// lam(h_*) += Cm * (source weight of g) for every column (see adjoint_cplx.cu).
cudaError_t launch_adjoint_source_cplx(int precision, int Lx, int Ly, int px, int py, int ncols, int W,
                                       const int32_t *sites, int pairing, const double2 *g, const double *cpl,
                                       double coupling, double Cm, void *lam, cudaStream_t s);
// column-slab groups of launch_adjoint_accumulate_cplx (the FP32 kernel with
// staged rows, slab width 4, sizes its own grid)
int adjoint_groups_cplx(int precision, int Lx, int Ly, int ld, int W);
cudaError_t launch_adjoint_accumulate_cplx(int precision, int Lx, int Ly, int px, int py, int nd, int bond, int ld,
                                           int W, int groups, const void *lam, const void *j, double f, double *part,
                                           unsigned long long wait_ns, unsigned *flags, cudaStream_t s);
// g_eps [N] real; g_hop [N * nd], g_delta [N] or [N * 4] complex (dL/dRe + i dL/dIm).
cudaError_t launch_adjoint_final_cplx(int Lx, int Ly, int px, int py, int nd, int bond, int groups,
                                      const double *part, const double *scal, double *g_eps, double2 *g_hop,
                                      double2 *g_delta, cudaStream_t s);

// Device address of the stand-alone contraction's error word (this device).
cudaError_t contract_flag_address(unsigned **out);
// LDOS weights of Eq. 17 as TF32 head / tail planes [n_E][ld].
cudaError_t launch_ldos_weights(int n_E, int M, int ld, int kernel, double lambda,
                                const double *energies, const double *scal, float *w_hi, float *w_lo,
                                cudaStream_t s);

}  // namespace cbdg

// Records msg as the calling thread's cbdg_last_error() text.
void cbdg_internal_set_error(const char *msg);
