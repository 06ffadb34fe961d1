/*
 * cbdg.h -- C ABI of libcbdg, a GB300 (sm_103a) implementation of the hot
 * path of the Chebyshev-Bogoliubov-de Gennes method (Covaci, Peeters,
 * Berciu, arXiv:1007.1609).
 *
 * The problem (Eq. 2): a square lattice of N = Lx*Ly sites with on-site
 * energies eps_i, chemical potential mu, hoppings t_ij (Peierls phases
 * included) and pairing Delta_i (on-site, s-wave) or Delta_ij (nearest-
 * neighbour bonds, d-wave).  The Nambu basis interleaves, per site s, the
 * electron row 2s (c_{s,up}) and the hole row 2s+1 (c^dagger_{s,down}).
 *
 * Conventions shared by every call:
 *   - Directions d: 0:+x 1:-x 2:+y 3:-y 4:+x+y 5:-x-y 6:+x-y 7:-x+y.
 *     hop[s*n_dirs + d] is t_ij for the bond from s to its neighbour along d;
 *     it enters H_{e_i e_j} = -t_ij and H_{h_i h_j} = conj(t_ij) (Eq. 2).
 *   - Spectral rescale (paragraph after Eq. 8): H~ = H / a with
 *     a = 1.1 * max_r sum_s |H_rs| (Gershgorin), b = 0.  a is recomputed
 *     from the current Delta by every call that needs it.
 *   - Array arguments may point to host memory or to device memory of the
 *     device that was current at cbdg_build_lattice; the library detects
 *     which (cudaPointerGetAttributes).  Host arrays are copied through the
 *     lattice's stream.  The caller owns every array it passes; the library
 *     never frees or keeps caller memory beyond the call.
 *   - Every call returns a cbdg_status and never aborts or exits.  On an
 *     error, cbdg_last_error() (per thread) describes it.  Compute calls are
 *     synchronous with respect to the host: results are complete when the
 *     call returns.
 *   - Complex numbers are cbdg_complex {re, im} (layout of C99 double
 *     complex, numpy complex128 and CUDA double2).
 */
#ifndef CBDG_H
#define CBDG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t cbdg_status;
enum {
  CBDG_OK = 0,
  CBDG_ERR_INVALID_ARG = 1,   /* bad size, enum, pointer, non-finite or non-Hermitian input */
  CBDG_ERR_CUDA = 2,          /* a CUDA runtime call failed */
  CBDG_ERR_OOM = 3,           /* device allocation failed */
  CBDG_ERR_SPECTRUM = 4,      /* a moment exceeded 1 in magnitude: a too small */
  CBDG_ERR_NOT_CONVERGED = 5, /* self-consistency did not reach its tolerance */
  CBDG_ERR_UNSUPPORTED = 6    /* valid input that the library has no kernel for */
};

enum { CBDG_ONSITE_U = 0, CBDG_BOND_V = 1 };        /* pairing channel */
enum { CBDG_FP64 = 0, CBDG_FP32_MIXED = 1 };        /* recursion precision */
enum { CBDG_JACKSON = 0, CBDG_LORENTZ = 1 };        /* damping kernel */

typedef struct {
  double re, im;
} cbdg_complex;

typedef struct cbdg_lattice cbdg_lattice;
typedef struct CUstream_st *cbdg_stream; /* a cudaStream_t; NULL = legacy default stream */

/* Lattice description (Eq. 2 and the Peierls phases below it). */
typedef struct {
  int32_t Lx, Ly;                /* lattice sides, >= 1; a periodic side must be >= 3 */
  int32_t periodic_x, periodic_y;/* 0: open edge, 1: periodic */
  const double *eps;             /* [N] on-site energies epsilon_i */
  double mu;                     /* chemical potential */
  int32_t n_dirs;                /* 4 (nearest) or 8 (plus next-nearest) */
  const cbdg_complex *hop;       /* [N*n_dirs] t_ij; must be 0 across an open edge and
                                    satisfy hop[j*n_dirs + (d^1)] == conj(hop[i*n_dirs + d]) */
  int32_t pairing;               /* CBDG_ONSITE_U or CBDG_BOND_V */
  double coupling;               /* U (on-site) or V (bond), attractive for > 0 */
  const cbdg_complex *delta0;    /* [N] Delta_i, or [N*4] Delta_{i,d} (d = 0..3) with
                                    Delta_{j,d^1} == Delta_{i,d} (singlet) */
  int32_t precision;             /* CBDG_FP64 or CBDG_FP32_MIXED */
  int32_t complex_field;         /* 0: hop and Delta real (real vectors), 1: complex */
} cbdg_lattice_desc;

/* Builds a lattice on the current CUDA device and copies the description
 * into library-owned device memory (Eq. 2).  All descriptor arrays are read
 * during the call only.  *out receives an opaque handle; release it with
 * cbdg_destroy.  Errors: INVALID_ARG for any violated constraint above,
 * UNSUPPORTED for combinations the library has no kernel for, OOM, CUDA. */
cbdg_status cbdg_build_lattice(const cbdg_lattice_desc *desc, cbdg_stream stream,
                               cbdg_lattice **out);

/* Releases a lattice and all its device memory.  NULL is accepted. */
cbdg_status cbdg_destroy(cbdg_lattice *lat);

/* Chebyshev moments of the rescaled Hamiltonian (Eqs. 11, 14, 15):
 * for each start site i = sites[c], c < n_sites, and n < M,
 *   mu_ee[c*M + n]            = <e_i | T_n(H~) | e_i>
 *   mu_eh[(c*M + n)*n_eh + 0] = <h_i | T_n(H~) | e_i>
 *   bond pairing (n_eh = 5):  mu_eh[(c*M + n)*5 + 1 + d] = <h_{i+d} | T_n(H~) | e_i>,
 *                             d = 0..3, zero across an open edge.
 * n_eh is 1 for on-site pairing.  The moments are unnormalised (mu_0 = 1);
 * the 1/(1 + delta_n0) of Eq. 11 is left to the caller.  Either output may
 * be NULL.  M >= 2.  sites may repeat.  Errors: INVALID_ARG, SPECTRUM, OOM,
 * CUDA. */
cbdg_status cbdg_moments(cbdg_lattice *lat, const int32_t *sites, int32_t n_sites, int32_t M,
                         double *mu_ee, cbdg_complex *mu_eh);

/* Order parameter and density from the current Delta (Eqs. 18-19, read as
 * expectation values of tanh(H/2T) through its kernel-damped Chebyshev
 * series with M terms):
 *   Delta_i     = (U/2) sum_n C_n conj(<h_i|T_n(H~)|e_i>)                 (on-site)
 *   Delta_{i,d} = (V/8) sum_n C_n conj(<h_{i+d}|T_n|e_i> + <h_i|T_n|e_{i+d}>)  (bond)
 *   n_i         = 1 - sum_n C_n <e_i|T_n(H~)|e_i>
 * with C_n = g_n (2 - delta_n0) c_n, c_n the Chebyshev coefficients of
 * tanh(a x / 2T) and g_n the Jackson kernel or the Lorentz kernel of Eq. 16
 * (parameter lambda).  All N sites are start vectors.  delta_out is [N] or
 * [N*4] (may be NULL); n_out is [N] (may be NULL).  T >= 0 (T = 0 means the
 * sign function).  Delta is not modified.  Errors: INVALID_ARG, SPECTRUM,
 * OOM, CUDA. */
cbdg_status cbdg_order_parameter(cbdg_lattice *lat, double T, int32_t kernel, double lambda,
                                 int32_t M, cbdg_complex *delta_out, double *n_out);

/* Up-spin local density of states of Eq. 17 with the expansion of Eq. 10,
 * per unit energy, at absolute energies E (|E| < a):
 *   ldos[c*n_E + e] = [g_0 mu_0 + 2 sum_{n>=1} g_n mu_n(i) T_n(E/a)] / (pi a sqrt(1-(E/a)^2))
 * for i = sites[c], g_n the Jackson or Lorentz (lambda) kernel.  The
 * moments come from the recursion; the sum over n is a dense
 * [n_sites x M] . [M x n_E] contraction on the tensor cores
 * (cbdg_contract_tf32x3).  Errors: INVALID_ARG (also for |E| >= a),
 * SPECTRUM, OOM, CUDA. */
cbdg_status cbdg_ldos(cbdg_lattice *lat, const int32_t *sites, int32_t n_sites, int32_t M,
                      int32_t kernel, double lambda, const double *energies, int32_t n_E,
                      float *ldos);

/* Nonlocal Chebyshev moments: one direct recursion (Eq. 15) per start site
 * i = sites[c], j_0 = e_i (the |c^dagger_{i,up}> of Eq. 15), read at every
 * target site t = targets[k] (the paragraph after Eq. 15: one recursion gives
 * G^{1 alpha}_{t i} for all t and alpha):
 *   a11[(c*M + n)*n_targets + k] = <e_t | T_n(H~) | e_i>   (a^{11}_n(t, i) (1 + delta_n0), Eq. 11)
 *   a12[(c*M + n)*n_targets + k] = <h_t | T_n(H~) | e_i>   (a^{12}_n(t, i) (1 + delta_n0), Eq. coeff2)
 * for n < M.  Any lattice kind (the recursion runs on complex vectors; a
 * real lattice gets complex copies of its parameters).  Arrays host or
 * device; sites and targets may repeat; either output may be NULL.  M >= 2.
 * Errors: INVALID_ARG (also an index outside 0..N-1), SPECTRUM (a moment
 * above 1 in magnitude), OOM, CUDA. */
cbdg_status cbdg_green_moments(cbdg_lattice *lat, const int32_t *sites, int32_t n_sites,
                               const int32_t *targets, int32_t n_targets, int32_t M,
                               cbdg_complex *a11, cbdg_complex *a12);

/* Retarded Green's functions of Eq. gf1 (imaginary part Eq. imag2, real part
 * Eq. real1) at absolute energies E (|E| < a) from the moments of
 * cbdg_green_moments:
 *   G11[(c*n_targets + k)*n_E + e] = (1/a) (-2i / sqrt(1 - x^2))
 *                                    sum_n g_n a11_n / (1 + delta_n0) exp(-i n arccos x),  x = E_e/a,
 * and G12 likewise from a12, g_n the Jackson kernel or the Lorentz kernel of
 * Eq. 16 (lambda; broadening lambda/M in arccos x).  G11 at t = i is
 * -pi times the LDOS of Eq. 17 in its imaginary part.  The sum over n is a
 * complex FP64 contraction [M] x [M x n_E] per (site, target).  Arrays host
 * or device; either output may be NULL.  Errors: INVALID_ARG (also for
 * |E| >= a), SPECTRUM, OOM, CUDA. */
cbdg_status cbdg_green_function(cbdg_lattice *lat, const int32_t *sites, int32_t n_sites,
                                const int32_t *targets, int32_t n_targets, int32_t M, int32_t kernel,
                                double lambda, const double *energies, int32_t n_E, cbdg_complex *G11,
                                cbdg_complex *G12);

/* Bond currents of Eq. 20, read as the continuity equation of the hopping
 * term of Eq. 2 (particle current, e = hbar = 1), summed over both spins:
 *   J[i*n_dirs + d] = sum_s 2 Im[t_{i,d} <c^dagger_{i,s} c_{j,s}>],  j = i + d,
 * with the density matrix of the kernel-damped series of the Fermi function
 * f(E) = [1 - tanh(E/2T)]/2 (the C_n of cbdg_order_parameter):
 *   <c^dagger_{i,up} c_{j,up}> = -(1/2) sum_n C_n <e_j|T_n(H~)|e_i>   (i != j)
 * and the equal spin-down term (particle-hole symmetry of Eq. 2).  J is the
 * current from i to its neighbour along d (directions as in hop), 0 across an
 * open edge; J_{i->j} = -J_{j->i}.  All N sites are start vectors (M - 2
 * recursion steps each).  J host or device, [N*n_dirs].  Any lattice kind (a
 * real lattice, with real t and Delta, carries none up to round-off).
 * Errors: INVALID_ARG, SPECTRUM, OOM, CUDA. */
cbdg_status cbdg_bond_currents(cbdg_lattice *lat, double T, int32_t M, int32_t kernel, double lambda,
                               double *J);

/* Dense contraction behind cbdg_ldos, on the tensor cores (tcgen05,
 * kind::tf32) with each operand split into TF32 head and tail (3 products,
 * about 21 significant bits; FP32 accumulation, re-based every 256 terms of
 * the k sum so that the tensor cores' truncating accumulation stays short):
 *   D[i*ldd + j] = sum_{l<k} A[i*lda + l] * B[j*ldb + l],  i < m, j < n.
 * A, B, D are device pointers on the current device; lda, ldb >= k,
 * ldd >= n.  The split planes live in a library-owned stream-ordered pool
 * (2 (m + n) kp floats, kp = cbdg_contract_kp(k)).  Runs on `stream` and
 * returns after completion.  Errors: INVALID_ARG, OOM, CUDA. */
cbdg_status cbdg_contract_tf32x3(const float *A, int32_t lda, const float *B, int32_t ldb, float *D,
                                 int32_t ldd, int32_t m, int32_t n, int32_t k, cbdg_stream stream);

/* Row length of the split planes for a contraction over k terms: k rounded
 * up to 32 (one 128-byte K-block).  Returns 0 for k <= 0. */
int32_t cbdg_contract_kp(int32_t k);

/* Splits src [rows][ld] (device, FP32, ld >= k) into TF32 planes hi and lo
 * [rows][kp], kp = cbdg_contract_kp(k): hi = TF32(x) and lo = TF32(x - hi),
 * both rounded to nearest, zero for columns k .. kp-1.  hi and lo are device
 * pointers, 16-byte aligned.  For an operand reused across contractions
 * (e.g. a weight table), split it once.  Runs on `stream`, returns without
 * waiting.  Errors: INVALID_ARG, CUDA. */
cbdg_status cbdg_split_tf32(const float *src, int32_t ld, int32_t rows, int32_t k, float *hi, float *lo,
                            cbdg_stream stream);

/* cbdg_contract_tf32x3 on operands already split by cbdg_split_tf32:
 * a_hi, a_lo [m][kp] and b_hi, b_lo [n][kp] (device, 16-byte aligned, kp a
 * positive multiple of 32); D as above.  Runs on `stream` and returns after
 * completion.  Errors: INVALID_ARG, CUDA. */
cbdg_status cbdg_contract_tf32x3_planes(const float *a_hi, const float *a_lo, const float *b_hi,
                                        const float *b_lo, int32_t kp, float *D, int32_t ldd, int32_t m,
                                        int32_t n, cbdg_stream stream);

/* One self-consistency iteration (paragraph after Eq. 20) with the Jackson
 * kernel: computes Delta_out from the current Delta as cbdg_order_parameter
 * does, then Delta <- Delta + mix (Delta_out - Delta).  *max_abs_ddelta
 * (host pointer, may be NULL) receives max_i |Delta_out,i - Delta_i| taken
 * before mixing.  0 < mix <= 1.  Errors: INVALID_ARG, SPECTRUM, OOM, CUDA. */
cbdg_status cbdg_scf_step(cbdg_lattice *lat, double T, int32_t M, double mix,
                          double *max_abs_ddelta);

/* Reverse-mode gradient of one self-consistency map Delta_out(eps, t, Delta_in)
 * (Eq. 19 through the recursion of Eq. 15) for every lattice kind (real or
 * complex Peierls hoppings, next-nearest neighbours, on-site or bond
 * pairing), with the rescale a and the coefficients C_n frozen at their
 * values for the current Delta (a Gershgorin value, or the fixed one).
 * Given dL_ddelta_out [nd] = dL/dRe Delta_out + i dL/dIm Delta_out
 * (nd = N, or N*4 for bond pairing; host or device), writes
 *   dL_deps[i]                = dL/deps_i (real)
 *   dL_dhop[i*n_dirs + d]     = dL/dRe t + i dL/dIm t for t = t_{i,d}, the
 *                               hopping of Eq. 2 with its Peierls phase; t
 *                               and its Hermitian mirror t_{j,d^1} = conj(t)
 *                               move together, so the mirror entry holds the
 *                               conjugate (0 across an open edge)
 *   dL_ddelta_in[k]           = dL/dRe Delta_k + i dL/dIm Delta_k of the input
 *                               Delta (on-site [N], or bond [N*4] with
 *                               Delta_{j,d^1} = Delta_{i,d} moving together)
 * Any output may be NULL; outputs are host or device arrays.  Real lattices
 * run the real recursion (imaginary parts 0), general ones complex vectors.
 * The forward recursion runs without doubling, keeps checkpoints of
 * (j_{kS}, j_{kS+1}) every S = ceil(sqrt(M)) steps and recomputes each
 * segment during the reverse sweep
 *   lam_m = y_m + 2 H~ lam_{m+1} - lam_{m+2},
 * with the source y_m = (U_i/2) C_m conj(g_i) h_i (on-site) or
 * (C_m/8) conj(V_{i,d} g_{i,d} + V_{j,d^1} g_{j,d^1}) h_j on each bond.
 * Errors: INVALID_ARG, OOM, CUDA.  Not in the paper (it has no
 * derivatives); added for gradient-based inverse design on Delta. */
cbdg_status cbdg_order_parameter_backward(cbdg_lattice *lat, double T, int32_t M,
                                          const cbdg_complex *dL_ddelta_out, double *dL_deps,
                                          cbdg_complex *dL_dhop, cbdg_complex *dL_ddelta_in);

/* Reverse-mode gradient of a loss on the up-spin LDOS of Eq. 17 (the
 * expansion of Eq. 10, as cbdg_ldos computes it) at the listed sites, for
 * real on-site pairing with 4 directions, with the rescale a frozen at its
 * value for the current Delta.  With G[c*n_E + e] = dL/dLDOS(E_e, sites[c])
 * (dL_dldos, [n_sites*n_E] doubles, host or device), the derivative of L
 * with respect to the moment mu_m(i_c) = <e_i|T_m(H~)|e_i> is
 *   s_{c,m} = sum_e G[c,e] g_m (2 - delta_m0) T_m(E_e/a) / (pi a sqrt(1 - (E_e/a)^2))
 * (formed in FP64 on the GPU), and the reverse recursion of
 * cbdg_order_parameter_backward runs over the listed start sites with the
 * source y_m = s_{c,m} e_i on the electron row.  Outputs (any may be NULL),
 * as in cbdg_order_parameter_backward:
 *   dL_deps [N], dL_dhop [N*4] (undirected bonds, stored on both directed
 *   entries), dL_ddelta [N] (dL/dDelta_i).
 * sites [n_sites] and energies [n_E] (|E| < a) are host or device arrays;
 * kernel / lambda as for cbdg_ldos.  Errors: INVALID_ARG (bad lists, energy
 * outside the band, non-finite host dL_dldos), UNSUPPORTED (complex or bond
 * lattices), OOM, CUDA.  Not in the paper (it has no derivatives). */
cbdg_status cbdg_ldos_backward(cbdg_lattice *lat, const int32_t *sites, int32_t n_sites, int32_t M,
                               int32_t kernel, double lambda, const double *energies, int32_t n_E,
                               const double *dL_dldos, double *dL_deps, double *dL_dhop, double *dL_ddelta);

/* Gradient of a loss L(Delta*) on the self-consistent order parameter
 * Delta* = F(Delta*; eps, t) (the fixed point of cbdg_scf_step, with a and the
 * coefficients frozen as in cbdg_order_parameter_backward), through the fixed
 * point rather than one map: by the implicit function theorem
 *   dL/dtheta = lam^T dF/dtheta,  lam = dL/dDelta* + (dF/dDelta_in)^T lam,
 * solved by the damped iteration lam <- (1 - mix) lam + mix (dL/dDelta* +
 * (dF/dDelta_in)^T lam), each product one run of the adjoint of
 * cbdg_order_parameter_backward, until max_i |d lam_i| < tol (at most
 * max_iter runs; it converges when the mixed self-consistency loop does).
 * The lattice's current Delta must be the converged Delta*.  dL_ddelta [N]
 * (real part used); outputs dL_deps [N], dL_dhop [N*4] as in
 * cbdg_order_parameter_backward (may be NULL); iterations may be NULL.
 * Real on-site lattices only.  Errors: INVALID_ARG, UNSUPPORTED,
 * NOT_CONVERGED (outputs hold the last lam's gradients), OOM, CUDA.  Not in
 * the paper. */
cbdg_status cbdg_fixed_point_backward(cbdg_lattice *lat, double T, int32_t M, double mix,
                                      const cbdg_complex *dL_ddelta, double tol, int32_t max_iter,
                                      double *dL_deps, double *dL_dhop, int32_t *iterations);

/* Copies the lattice's current Delta ([N] or [N*4]) out, or replaces it.  A
 * new bond Delta must be symmetric (Delta_{j,d^1} == Delta_{i,d}) and 0
 * across open edges, like delta0 (the recursion reads each bond from one end);
 * otherwise INVALID_ARG. */
cbdg_status cbdg_get_delta(cbdg_lattice *lat, cbdg_complex *delta);
cbdg_status cbdg_set_delta(cbdg_lattice *lat, const cbdg_complex *delta);

/* Replaces the scalar coupling of the descriptor by one coupling per Delta
 * entry: coupling[i] = U_i for on-site pairing ([N]), coupling[4i + d] =
 * V_{i,d} for bond pairing ([N*4], symmetric: V_{j,d^1} == V_{i,d}; entries
 * across an open edge are ignored).  Eq. 19 then reads Delta_i = (U_i/2) ...
 * (and Delta_{i,d} = (V_{i,d}/8) ...) in cbdg_order_parameter, cbdg_scf_step
 * and the gradients; U_i = 0 marks a normal-metal site (the S/N and S/N/S
 * junctions of the paper's examples).  NULL restores the scalar.  Host or
 * device array, read during the call.  Errors: INVALID_ARG (not finite, not
 * symmetric), OOM, CUDA.  Not in the ensemble API. */
cbdg_status cbdg_set_coupling(cbdg_lattice *lat, const double *coupling);

/* Replaces the on-site energies eps [N] and/or the hoppings hop [N*n_dirs]
 * (Eq. 2; the same layout and rules as in the descriptor: zero across open
 * edges, Hermitian pairs, real unless complex_field) of an existing lattice;
 * NULL keeps the current array.  Host or device arrays, read during the
 * call; an invalid array changes nothing.  Lets a caller that iterates on
 * parameters (an optimiser, an autograd loop) reuse one lattice and its
 * buffers.  Errors: INVALID_ARG, CUDA. */
cbdg_status cbdg_set_hamiltonian(cbdg_lattice *lat, const double *eps, const cbdg_complex *hop);

/* Start-vector symmetry reduction.  rep [N] (host or device) maps every
 * site to the representative of its orbit under a symmetry of the
 * Hamiltonian and of the current and future Delta that the CALLER guarantees,
 * e.g. the translations along a periodic direction of a lattice without
 * disorder (rep[x + Lx*y] = Lx*y).  cbdg_order_parameter and cbdg_scf_step
 * then run one recursion per distinct representative and give every site of
 * an orbit its representative's Delta_out and n: each grid point's Green's
 * function is computed separately (the paragraph after Eq. 20), and
 * equivalent points have the same one.  Needs rep[rep[i]] == rep[i]; NULL
 * restores every site as a start vector.  On-site pairing only (a bond fold
 * reads the recursion of both ends).  Other calls (moments, LDOS, adjoints)
 * are unaffected.  Errors: INVALID_ARG, UNSUPPORTED, CUDA. */
cbdg_status cbdg_set_symmetry(cbdg_lattice *lat, const int32_t *rep);

/* The rescale factor a used by the most recent compute call (0 before any). */
cbdg_status cbdg_get_rescale(cbdg_lattice *lat, double *a);

/* lambda of the Lorentz kernel (Eq. 16, g_n = sinh(lambda (1 - n/M)) /
 * sinh(lambda)) that broadens every level by `broadening` (an energy, in the
 * units of t) at the band centre: the kernel's width is lambda / M in the
 * rescaled energy (the paragraph after Eq. 16), so lambda = broadening * M / a
 * with the rescale a that the next compute call will use for the current
 * Delta (1.1 x the Gershgorin bound, or the fixed rescale option), computed
 * on the GPU by this call.  *lambda is a host double.  Errors: INVALID_ARG
 * (broadening <= 0 or not finite, M < 2), SPECTRUM (a <= 0), CUDA. */
cbdg_status cbdg_lorentz_lambda(cbdg_lattice *lat, double broadening, int32_t M, double *lambda);

/* Tuning and instrumentation options (cbdg_set_option / cbdg_get_option). */
enum {
  CBDG_OPT_QUADRATURE_NODES = 0, /* K of the Gauss-Chebyshev sum for c_n; default 65536 */
  CBDG_OPT_COLUMN_CHUNK = 1,     /* start vectors per recursion pass; 0 = automatic */
  CBDG_OPT_PROFILE = 2,          /* 1: time every recursion-step launch with CUDA events */
  CBDG_OPT_SLAB_WIDTH = 3,       /* columns per CTA of the recursion kernel (power of two,
                                    at most 32; the planner narrows it to what fits);
                                    0 = automatic */
  CBDG_OPT_ROW_SPLIT = 4,        /* CTAs per column slab along y; 0 = automatic */
  CBDG_OPT_WORKSPACE_MB = 5,     /* cap on the recursion vectors' memory; 0 = automatic */
  CBDG_OPT_RESCALE_MILLI = 6,    /* a = (value/1000) * Gershgorin bound; default 1100 (1.1).
                                    Below 1000 the spectrum may leave [-1, 1] and calls
                                    then fail with CBDG_ERR_SPECTRUM */
  CBDG_OPT_PIPELINE_DEPTH = 7,   /* lattice rows the recursion kernel stages ahead (1..4);
                                    0 = automatic */
  CBDG_OPT_FIXED_RESCALE_PICO = 8, /* > 0: use a = value * 1e-12 instead of the Gershgorin
                                    rescale (frozen a, e.g. for finite differences);
                                    0 = Gershgorin (default) */
  CBDG_OPT_WAIT_LIMIT_MS = 9,    /* limit of every wait of the recursion kernels on a staged
                                    copy (default 2000); on expiry the call returns
                                    CBDG_ERR_CUDA and the lattice stays usable */
  CBDG_OPT_TEST_STALL_COPY = 10, /* test hook for failure detection: 1 makes the first staged
                                    row of each recursion CTA wait for 16 bytes that never
                                    arrive, so the wait runs out; 0 (default) off */
  CBDG_OPT_AUTOTUNE = 11,        /* 1: time candidate tiles (slab width, depth, row split) on
                                    the first pass of each lattice shape and keep the fastest
                                    (cached per process); 0 (default): static plan */
  CBDG_OPT_TEMPORAL_STEPS = 12,  /* recursion steps K per pass over the vectors (temporal
                                    blocking), 1..4, for real on-site FP32 lattices with open
                                    y edges: one pass reads j_(n-1), j_n and writes
                                    j_(n+K-1), j_(n+K); 1 = one step per pass; 0 (default) =
                                    3 where each thread holds one lattice site (Lx <= 256 /
                                    (W / 4)) and at slab width 16 up to Lx = 128 (the lean
                                    pass), else 2.  Shapes the multi-step kernel does not
                                    serve run one step per pass: periodic y, FP64, slab
                                    widths other than 8 and 16, Lx above 64 at slab width
                                    16 (128 for K = 2, and for K = 3 at pipeline depth 1,
                                    the lean pass), above 128 at slab width 8 (256 for
                                    K = 2), and rings that do not fit in shared memory;
                                    except that K = 2 requested explicitly on a lattice
                                    128 < Lx <= 512 at slab width 4 or 8 runs the two-step
                                    pass over row blocks (each block recomputes its halo
                                    rows, the new vectors are written to two more vector
                                    buffers: four vectors of workspace instead of two).
                                    General lattices (complex FP32 vectors: Peierls
                                    hoppings, t', bond pairing; periodic or open): K >= 2
                                    selects the two-step pass (slab width 2, Lx <= 256,
                                    Ly >= 3, the default tile); 0 (default) keeps one step
                                    per pass there, which measured faster */
  CBDG_OPT_GRAPH = 13,           /* 1 (default): cbdg_scf_step captures its iteration as a
                                    CUDA graph on the second call with the same (T, M, mix)
                                    and replays it afterwards (not while profiling,
                                    autotuning, with a fixed rescale or the stall hook); any
                                    option change or buffer reallocation drops the graph;
                                    0: always launch directly */
  CBDG_OPT_RESIDENT = 14         /* 1 (default): real on-site lattices whose two vectors per
                                    column slab, stencil parameters and coefficient table
                                    fit in one SM's shared memory (about 2300 sites in FP64,
                                    4700 in FP32) run the whole recursion on chip, one
                                    launch per pass (unless a tile option, autotuning or the
                                    stall hook is set); 0: the streamed kernels */
};
/* Read-only (cbdg_get_option): the tile of the last recursion pass, packed as
 * slab width | depth << 16 | row split << 32. */
enum { CBDG_INFO_LAST_TILE = 100 };
/* Read-only: recursion steps per pass (K) used by the last pass. */
enum { CBDG_INFO_LAST_TEMPORAL = 101 };
cbdg_status cbdg_set_option(cbdg_lattice *lat, int32_t option, int64_t value);
cbdg_status cbdg_get_option(cbdg_lattice *lat, int32_t option, int64_t *value);

/* Accumulated device time of the recursion-step kernel since the last reset
 * (CBDG_OPT_PROFILE must be on): total milliseconds, number of launches and
 * algorithmic bytes (read j_n, read j_{n-1}, write j_{n+1}) summed over the
 * launches.  reset != 0 clears the counters after reading. */
cbdg_status cbdg_profile_read(cbdg_lattice *lat, double *step_ms, int64_t *step_launches,
                              double *step_bytes, int32_t reset);

/* Ensembles: many independent lattices (disorder realisations of uneven
 * size) iterated to self-consistency together.  Every member: real on-site
 * pairing, 4 directions, open edges, CBDG_FP32_MIXED, sides <= 128, and one
 * shared mu and U.  Each iteration is one persistent launch over (sample,
 * 16-column slab) work items plus small batched kernels (rescale, Fermi
 * coefficients by K-node quadrature, parameters, mixing, convergence),
 * captured once as a CUDA graph and replayed.  Not in the paper: a batching
 * layer over its self-consistency loop (paragraph after Eq. 20). */
typedef struct cbdg_ensemble cbdg_ensemble;
cbdg_status cbdg_build_ensemble(const cbdg_lattice_desc *descs, int32_t n, cbdg_stream stream,
                                cbdg_ensemble **out);
cbdg_status cbdg_ensemble_destroy(cbdg_ensemble *ens);
/* Runs up to max_iter iterations (Jackson kernel, M moments, linear mixing
 * `mix`); a sample stops once max_i |Delta_out - Delta| < tol (the mix of
 * that iteration is applied).  *iters_out = iterations run; converged_mask
 * [n] (host) = 1 for converged samples.  Returns CBDG_ERR_NOT_CONVERGED if
 * any sample is left, with all outputs filled. */
cbdg_status cbdg_ensemble_scf(cbdg_ensemble *ens, double T, int32_t M, double mix, double tol,
                              int32_t max_iter, int32_t *iters_out, int32_t *converged_mask);
/* Copies sample `sample`'s current Delta ([N], host or device) out. */
cbdg_status cbdg_ensemble_get_delta(cbdg_ensemble *ens, int32_t sample, cbdg_complex *delta);
/* CBDG_OPT_QUADRATURE_NODES only (default 16384). */
cbdg_status cbdg_ensemble_set_option(cbdg_ensemble *ens, int32_t option, int64_t value);

/* Number of CUDA kernels the library has launched for this lattice since the
 * last reset (reset != 0 clears the counter after reading). */
cbdg_status cbdg_launch_count(cbdg_lattice *lat, int64_t *launches, int32_t reset);

/* Moments of cbdg_moments (same definitions, outputs and tolerances) for
 * callers that cannot allocate device memory while they run -- for example a
 * host program that works inside a fixed, pre-planned memory budget, or a
 * plug-in inside another framework whose allocator owns the GPU's memory --
 * and so cannot build a lattice handle (which allocates).  The paper has no
 * counterpart; this is a deployment variant.
 *   desc:    as for cbdg_build_lattice, but eps, hop and delta0 must be
 *            DEVICE pointers; inputs are not checked for finiteness or
 *            Hermiticity (invalid values give meaningless moments, or
 *            CBDG_ERR_SPECTRUM).  Real on-site pairing with n_dirs = 4 only.
 *   sites:   device array of n_sites start sites; a site outside [0, N) is
 *            detected on the GPU, never indexed, and makes the call return
 *            CBDG_ERR_INVALID_ARG (the outputs are then not valid).
 *            mu_ee [n_sites*M] and mu_eh [n_sites*M] (n_eh = 1) are device
 *            outputs, either may be NULL.
 *   stream:  the stream all work is queued on; the call returns after it
 *            has finished.
 * Every intermediate lives in one fixed 64 MiB device array reserved when
 * the library is loaded (on each GPU that loads it, until the process
 * exits); nothing is allocated.  Lattices whose single column slab does not
 * fit are rejected with CBDG_ERR_INVALID_ARG; more start sites are handled
 * in chunks.  The recursion runs one CTA per column slab with no row split,
 * so few start sites use few SMs: the call trades throughput for its fixed
 * footprint.  The first call on a device looks up the array's device
 * address (once per device, with that device current) and caches it: make
 * that first call before any stream capture, and do not call again after a
 * cudaDeviceReset in the same process.  All calls share the array and a call
 * resets what it needs, but calls whose GPU work overlaps (other streams or
 * threads) race on it: serialise them. */
cbdg_status cbdg_moments_noalloc(const cbdg_lattice_desc *desc, const int32_t *sites,
                                 int32_t n_sites, int32_t M, double *mu_ee, cbdg_complex *mu_eh,
                                 cbdg_stream stream);

/* Arithmetic peaks of the current GPU, measured by the library's own
 * microbenchmarks: the denominators of the rooflines of the arithmetic-bound
 * kernels (the FP64 recursion, the FP64 Green's-function contraction, the
 * 3xTF32 LDOS contraction).  Not in the paper (it reports no timings).
 *   kind: CBDG_PEAK_FP64_FMA / CBDG_PEAK_FP32_FMA -- 8 (FP64) or 16 (FP32)
 *         independent FMA chains per thread, 8 CTAs of 256 threads per SM,
 *         `work` FMAs per chain; CBDG_PEAK_TF32_MMA -- one CTA per SM issuing `work`
 *         tcgen05.mma kind::tf32 of M = 128, N = 256, K = 8 (the LDOS
 *         contraction's instruction) from shared memory into tensor memory.
 *   work: 1 .. 2^40.  *flops (host) receives the flops of the launch
 *         (2 per FMA, 2 M N K per MMA).
 * Queues one launch on `stream` and returns without waiting: the caller
 * times it (CUDA events).  cbdg_peak_status waits for the stream and
 * reports CBDG_ERR_CUDA if the tensor-core probe's bounded final wait ran
 * out.  Errors: INVALID_ARG, CUDA. */
enum { CBDG_PEAK_FP64_FMA = 0, CBDG_PEAK_FP32_FMA = 1, CBDG_PEAK_TF32_MMA = 2 };
cbdg_status cbdg_measure_peak(int32_t kind, int64_t work, cbdg_stream stream, double *flops);
cbdg_status cbdg_peak_status(cbdg_stream stream);

/* Per-thread description of the last error; never NULL. */
const char *cbdg_last_error(void);

/* Library version string. */
const char *cbdg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CBDG_H */
