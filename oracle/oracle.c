/*
 * oracle.c -- plain, slow, FP64 reference implementation of the
 * Chebyshev-Bogoliubov-de Gennes (CBdG) method (Covaci, Peeters, Berciu,
 * arXiv:1007.1609).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * execute this file: only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark use it.  It shares no code, header, table or
 * constant with the CUDA library; it is written from the paper's equations.
 *
 * Every function computes a plain definition:
 *   - H is an explicit CSR matrix (double complex) built entry by entry from
 *     Eq. 2 (hamil2); the basis interleaves electron and hole rows per site:
 *     row 2s is c_{s,up}, row 2s+1 is c^dagger_{s,down}.
 *   - a = 1.1 * max_r sum_s |H_rs| (Gershgorin), b = 0: the rescale of the
 *     paragraph after Eq. 8 with symmetric bounds.
 *   - moments by the DIRECT recursion of Eq. 15 (ref2): j_0 = e_i,
 *     j_1 = H~ j_0, j_{n+1} = 2 H~ j_n - j_{n-1}; a_n = <alpha|j_n>.  No
 *     doubling and no particle-hole shortcut.
 *   - kernels: Jackson (the Weisse et al. KPM review the paper cites for its
 *     kernel polynomials) and Lorentz, Eq. 16.
 *   - Fermi-function coefficients by Gauss-Chebyshev quadrature, a direct
 *     O(M K) sum.
 *   - order parameter, density, LDOS: Eqs. 17-19 read as expectation values
 *     of the truncated, kernel-damped Chebyshev series of tanh(H/2T).
 *   - a cyclic Jacobi eigensolver for dense Hermitian matrices (Golub and
 *     Van Loan, the symmetric Jacobi method with a phase rotation for the
 *     complex off-diagonal), used only as an independent exact check.
 *   - reverse-mode gradients, storing every j_n: of one self-consistency
 *     map (a loss on Delta_out; real lattices, and general ones with complex
 *     hoppings, next-nearest neighbours and bond pairing) and of a loss on
 *     the LDOS, a frozen.
 *   - nonlocal moments <alpha_t|T_n|e_i> at chosen target sites, the
 *     Green's function of gf1 built from them, and the bond currents of
 *     Eq. 20 from the one-body density matrix f(H).
 *
 * OpenMP parallelises over start sites (the paper's "trivially parallel"
 * axis, paragraph after Eq. 20) and over coefficient indices.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* ------------------------------------------------------------------------ */
/* Lattice description (oracle's own; mirrors the paper's Eq. 2 symbols).   */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t Lx, Ly;
  int32_t periodic_x, periodic_y;
  int32_t n_dirs;      /* 4: nearest neighbours; 8: plus next-nearest       */
  const double *eps;   /* [N] on-site potential epsilon_i                    */
  double mu;           /* chemical potential                                 */
  const cplx *hop;     /* [N*n_dirs] t_ij for the bond from i along dir d    */
  int32_t pairing;     /* 0: on-site Delta_i; 1: nearest-neighbour Delta_ij  */
  double coupling;     /* U (on-site) or V (bond)                            */
  const cplx *delta;   /* [N] (on-site) or [N*4] (bond)                      */
  const double *coupling_site; /* NULL, or a coupling per Delta entry ([N] U_i
                                  or [N*4] V_{i,d}) that replaces `coupling`  */
} orc_lattice;

/* The coupling of Delta entry k (site i, or bond (i, d) at k = 4i + d). */
static double coupling_of(const orc_lattice *L, size_t k) {
  return L->coupling_site ? L->coupling_site[k] : L->coupling;
}

/* Direction d -> lattice offset.  0:+x 1:-x 2:+y 3:-y 4:+x+y 5:-x-y 6:+x-y
 * 7:-x+y.  Opposite directions are d and d^1. */
static const int DX[8] = {+1, -1, 0, 0, +1, -1, +1, -1};
static const int DY[8] = {0, 0, +1, -1, +1, -1, -1, +1};

/* Neighbour of site s along d, or -1 when an open edge cuts the bond. */
int orc_neighbour(const orc_lattice *L, int s, int d) {
  int x = s % L->Lx, y = s / L->Lx;
  int nx = x + DX[d], ny = y + DY[d];
  if (nx < 0 || nx >= L->Lx) {
    if (!L->periodic_x) return -1;
    nx = (nx + L->Lx) % L->Lx;
  }
  if (ny < 0 || ny >= L->Ly) {
    if (!L->periodic_y) return -1;
    ny = (ny + L->Ly) % L->Ly;
  }
  return nx + L->Lx * ny;
}

/* ------------------------------------------------------------------------ */
/* Explicit CSR Hamiltonian, Eq. 2.                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
  int n;        /* 2N */
  int *rowptr;  /* [n+1] */
  int *col;     /* [nnz] */
  cplx *val;    /* [nnz] */
} orc_csr;

/* Add v at (r,c) into a row buffer, merging duplicates (so that for any
 * geometry the CSR holds the plain matrix element). */
static void row_add(int *cols, cplx *vals, int *cnt, int c, cplx v) {
  for (int k = 0; k < *cnt; ++k)
    if (cols[k] == c) { vals[k] += v; return; }
  cols[*cnt] = c;
  vals[*cnt] = v;
  (*cnt)++;
}

/* Build H of Eq. 2:
 *   site block  [[eps_i - mu, Delta_i], [conj(Delta_i), -eps_i + mu]]
 *   bond block  [[-t_ij, Delta_ij], [conj(Delta_ij), conj(t_ij)]]  (i != j)
 * with e_i = row 2i, h_i = row 2i+1. */
static orc_csr build_csr(const orc_lattice *L) {
  int N = L->Lx * L->Ly;
  int n = 2 * N;
  int maxrow = 2 + 2 * L->n_dirs;
  orc_csr H;
  H.n = n;
  H.rowptr = (int *)malloc(sizeof(int) * (n + 1));
  H.col = (int *)malloc(sizeof(int) * (size_t)n * maxrow);
  H.val = (cplx *)malloc(sizeof(cplx) * (size_t)n * maxrow);
  int nnz = 0;
  int cols[32];
  cplx vals[32];
  for (int i = 0; i < N; ++i) {
    for (int part = 0; part < 2; ++part) { /* 0: electron row, 1: hole row */
      int cnt = 0;
      double xi = L->eps[i] - L->mu;
      if (part == 0) {
        row_add(cols, vals, &cnt, 2 * i, xi);
        if (L->pairing == 0) row_add(cols, vals, &cnt, 2 * i + 1, L->delta[i]);
      } else {
        if (L->pairing == 0) row_add(cols, vals, &cnt, 2 * i, conj(L->delta[i]));
        row_add(cols, vals, &cnt, 2 * i + 1, -xi);
      }
      for (int d = 0; d < L->n_dirs; ++d) {
        int j = orc_neighbour(L, i, d);
        if (j < 0) continue;
        cplx t = L->hop[(size_t)i * L->n_dirs + d];
        if (part == 0) {
          row_add(cols, vals, &cnt, 2 * j, -t);
          if (L->pairing == 1 && d < 4)
            row_add(cols, vals, &cnt, 2 * j + 1, L->delta[(size_t)i * 4 + d]);
        } else {
          row_add(cols, vals, &cnt, 2 * j + 1, conj(t));
          if (L->pairing == 1 && d < 4)
            row_add(cols, vals, &cnt, 2 * j, conj(L->delta[(size_t)i * 4 + d]));
        }
      }
      int r = 2 * i + part;
      H.rowptr[r] = nnz;
      for (int k = 0; k < cnt; ++k) {
        H.col[nnz] = cols[k];
        H.val[nnz] = vals[k];
        nnz++;
      }
    }
  }
  H.rowptr[n] = nnz;
  return H;
}

static void free_csr(orc_csr *H) {
  free(H->rowptr);
  free(H->col);
  free(H->val);
}

/* Dense H (row-major, 2N x 2N) for exact diagonalisation. */
int orc_dense_hamiltonian(const orc_lattice *L, cplx *out) {
  orc_csr H = build_csr(L);
  memset(out, 0, sizeof(cplx) * (size_t)H.n * H.n);
  for (int r = 0; r < H.n; ++r)
    for (int k = H.rowptr[r]; k < H.rowptr[r + 1]; ++k)
      out[(size_t)r * H.n + H.col[k]] += H.val[k];
  free_csr(&H);
  return 0;
}

/* Gershgorin bound max_r sum_s |H_rs| over the plain matrix elements. */
double orc_gershgorin(const orc_lattice *L) {
  orc_csr H = build_csr(L);
  double best = 0.0;
  for (int r = 0; r < H.n; ++r) {
    double s = 0.0;
    for (int k = H.rowptr[r]; k < H.rowptr[r + 1]; ++k) s += cabs(H.val[k]);
    if (s > best) best = s;
  }
  free_csr(&H);
  return best;
}

/* y = (alpha/a) H x + beta * z   (z may alias y). */
static void csr_step(const orc_csr *H, double scale, const cplx *x, double beta,
                     const cplx *z, cplx *y) {
  for (int r = 0; r < H->n; ++r) {
    cplx acc = 0.0;
    for (int k = H->rowptr[r]; k < H->rowptr[r + 1]; ++k) acc += H->val[k] * x[H->col[k]];
    y[r] = scale * acc + beta * z[r];
  }
}

/* ------------------------------------------------------------------------ */
/* Kernels and coefficients.                                                 */
/* ------------------------------------------------------------------------ */

/* Jackson kernel, M terms:
 *   g_n = [(M-n+1) cos(pi n/(M+1)) + sin(pi n/(M+1)) cot(pi/(M+1))]/(M+1). */
void orc_jackson(int M, double *g) {
  double q = M_PI / (M + 1);
  for (int n = 0; n < M; ++n)
    g[n] = ((M - n + 1) * cos(q * n) + sin(q * n) * cos(q) / sin(q)) / (M + 1);
}

/* Lorentz kernel of Eq. 16: g_n = sinh[lambda (1 - n/M)] / sinh(lambda). */
void orc_lorentz(int M, double lambda, double *g) {
  for (int n = 0; n < M; ++n) g[n] = sinh(lambda * (1.0 - (double)n / M)) / sinh(lambda);
}

/* Chebyshev coefficients of f(x) = tanh(a x / 2T) on [-1,1], in the
 * normalisation of the expansion after the introduction of the KPM
 * (f = sum_n (2 - delta_n0) c_n T_n):
 *   c_n = (1/pi) int_{-1}^{1} f(x) T_n(x) / sqrt(1-x^2) dx,
 * evaluated by K-node Gauss-Chebyshev quadrature
 *   c_n = (1/K) sum_k f(cos th_k) cos(n th_k),  th_k = pi (k + 1/2) / K.
 * At T == 0 the function is sign(x). */
void orc_tanh_coefficients(int M, int K, double a, double T, double *c) {
  double *f = (double *)malloc(sizeof(double) * K);
  for (int k = 0; k < K; ++k) {
    double x = cos(M_PI * (k + 0.5) / K);
    f[k] = (T > 0.0) ? tanh(a * x / (2.0 * T)) : (x > 0 ? 1.0 : (x < 0 ? -1.0 : 0.0));
  }
#pragma omp parallel for schedule(dynamic, 4)
  for (int n = 0; n < M; ++n) {
    double s = 0.0;
    for (int k = 0; k < K; ++k) s += f[k] * cos(n * M_PI * (k + 0.5) / K);
    c[n] = s / K;
  }
  free(f);
}

/* C_n = g_n (2 - delta_n0) c_n: the damped expansion coefficients of
 * tanh(a x / 2T), F_M(x) = sum_n C_n T_n(x). kernel 0 = Jackson, 1 = Lorentz. */
void orc_fold_coefficients(int M, int K, double a, double T, int kernel, double lambda,
                           double *C) {
  double *g = (double *)malloc(sizeof(double) * M);
  if (kernel == 0) orc_jackson(M, g);
  else orc_lorentz(M, lambda, g);
  orc_tanh_coefficients(M, K, a, T, C);
  for (int n = 0; n < M; ++n) C[n] *= g[n] * (n == 0 ? 1.0 : 2.0);
  free(g);
}

/* ------------------------------------------------------------------------ */
/* Moments by the direct recursion, Eq. 15.                                  */
/* ------------------------------------------------------------------------ */

/* For each start site i = sites[c]:
 *   mu_ee[c*M + n] = <e_i | T_n(H/a) | e_i>         (a^{11}_n (1+delta_n0), Eq. 11)
 *   mu_eh[(c*M + n)*n_eh + 0] = <h_i | T_n(H/a) | e_i>   (a^{12} numerator, Eq. 14)
 *   bond pairing adds, for d = 0..3, <h_{i+d} | T_n(H/a) | e_i> at index 1+d
 *   (zero where an open edge cuts the bond).
 * n_eh = 1 for on-site pairing and 5 for bond pairing. */
int orc_moments(const orc_lattice *L, double a, const int32_t *sites, int n_sites, int M,
                double *mu_ee, cplx *mu_eh) {
  orc_csr H = build_csr(L);
  int n = H.n;
  int n_eh = (L->pairing == 1) ? 5 : 1;
#pragma omp parallel
  {
    cplx *jprev = (cplx *)malloc(sizeof(cplx) * n);
    cplx *jcur = (cplx *)malloc(sizeof(cplx) * n);
#pragma omp for schedule(dynamic, 1)
    for (int c = 0; c < n_sites; ++c) {
      int i = sites[c];
      int nb[4];
      for (int d = 0; d < 4; ++d) nb[d] = orc_neighbour(L, i, d);
      memset(jprev, 0, sizeof(cplx) * n);
      jprev[2 * i] = 1.0; /* j_0 = e_i */
      for (int m = 0; m < M; ++m) {
        cplx *jn;
        if (m == 0) {
          jn = jprev;
        } else if (m == 1) {
          csr_step(&H, 1.0 / a, jprev, 0.0, jprev, jcur); /* j_1 = H~ j_0 */
          jn = jcur;
        } else {
          /* j_{m} = 2 H~ j_{m-1} - j_{m-2}: jcur holds j_{m-1}, jprev j_{m-2} */
          csr_step(&H, 2.0 / a, jcur, -1.0, jprev, jprev);
          cplx *t = jprev;
          jprev = jcur;
          jcur = t;
          jn = jcur;
        }
        mu_ee[(size_t)c * M + m] = creal(jn[2 * i]);
        cplx *out = mu_eh + ((size_t)c * M + m) * n_eh;
        out[0] = jn[2 * i + 1];
        if (n_eh == 5)
          for (int d = 0; d < 4; ++d) out[1 + d] = (nb[d] >= 0) ? jn[2 * nb[d] + 1] : 0.0;
      }
    }
    free(jprev);
    free(jcur);
  }
  free_csr(&H);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Observables.                                                              */
/* ------------------------------------------------------------------------ */

/* Order parameter and density from the damped series of tanh(H/2T):
 *  on-site (Eq. 19 with i = j, as the expectation U <c_{i,up} c_{i,down}>):
 *     Delta_i = (U/2) sum_n C_n conj(<h_i|T_n|e_i>)
 *  bond, along d = 0..3 (symmetrised singlet):
 *     Delta_{i,d} = (V/8) sum_n C_n conj(<h_{i+d}|T_n|e_i> + <h_i|T_n|e_{i+d}>)
 *  density (Eq. 18 with N_up = N_down):
 *     n_i = 1 - sum_n C_n <e_i|T_n|e_i>.
 * All N sites are start vectors.  delta_out is [N] or [N*4]. */
int orc_order_parameter(const orc_lattice *L, double a, double T, int M, int K, int kernel,
                        double lambda, cplx *delta_out, double *n_out) {
  int N = L->Lx * L->Ly;
  int n_eh = (L->pairing == 1) ? 5 : 1;
  double *C = (double *)malloc(sizeof(double) * M);
  orc_fold_coefficients(M, K, a, T, kernel, lambda, C);
  int32_t *sites = (int32_t *)malloc(sizeof(int32_t) * N);
  for (int i = 0; i < N; ++i) sites[i] = i;
  double *mu_ee = (double *)malloc(sizeof(double) * (size_t)N * M);
  cplx *mu_eh = (cplx *)malloc(sizeof(cplx) * (size_t)N * M * n_eh);
  orc_moments(L, a, sites, N, M, mu_ee, mu_eh);
  for (int i = 0; i < N; ++i) {
    double nn = 1.0;
    for (int m = 0; m < M; ++m) nn -= C[m] * mu_ee[(size_t)i * M + m];
    if (n_out) n_out[i] = nn;
    if (L->pairing == 0) {
      cplx s = 0.0;
      for (int m = 0; m < M; ++m) s += C[m] * conj(mu_eh[(size_t)i * M + m]);
      delta_out[i] = 0.5 * coupling_of(L, i) * s;
    } else {
      for (int d = 0; d < 4; ++d) {
        int j = orc_neighbour(L, i, d);
        if (j < 0) {
          delta_out[(size_t)i * 4 + d] = 0.0;
          continue;
        }
        int dback = d ^ 1;
        cplx s = 0.0;
        for (int m = 0; m < M; ++m) {
          cplx fwd = mu_eh[((size_t)i * M + m) * 5 + 1 + d];     /* <h_j|T_n|e_i> */
          cplx bwd = mu_eh[((size_t)j * M + m) * 5 + 1 + dback]; /* <h_i|T_n|e_j> */
          s += C[m] * conj(fwd + bwd);
        }
        delta_out[(size_t)i * 4 + d] = 0.125 * coupling_of(L, (size_t)i * 4 + d) * s;
      }
    }
  }
  free(C);
  free(sites);
  free(mu_ee);
  free(mu_eh);
  return 0;
}

/* The on-site order parameter and density of orc_order_parameter restricted
 * to the start sites listed in sites[0..n_sites) (on-site pairing only):
 * Delta_i = (U/2) sum_n C_n conj(<h_i|T_n|e_i>), n_i = 1 - sum_n C_n <e_i|T_n|e_i>.
 * delta_out and n_out are [n_sites]. */
int orc_order_parameter_sites(const orc_lattice *L, double a, double T, int M, int K, int kernel,
                              double lambda, const int32_t *sites, int n_sites, cplx *delta_out,
                              double *n_out) {
  if (L->pairing != 0) return -1;
  double *C = (double *)malloc(sizeof(double) * M);
  orc_fold_coefficients(M, K, a, T, kernel, lambda, C);
  double *mu_ee = (double *)malloc(sizeof(double) * (size_t)n_sites * M);
  cplx *mu_eh = (cplx *)malloc(sizeof(cplx) * (size_t)n_sites * M);
  orc_moments(L, a, sites, n_sites, M, mu_ee, mu_eh);
  for (int c = 0; c < n_sites; ++c) {
    double nn = 1.0;
    cplx s = 0.0;
    for (int m = 0; m < M; ++m) {
      nn -= C[m] * mu_ee[(size_t)c * M + m];
      s += C[m] * conj(mu_eh[(size_t)c * M + m]);
    }
    if (n_out) n_out[c] = nn;
    delta_out[c] = 0.5 * coupling_of(L, sites[c]) * s;
  }
  free(C);
  free(mu_ee);
  free(mu_eh);
  return 0;
}

/* Bond order parameter of orc_order_parameter restricted to the sites listed
 * in sites[0..n_sites): for each listed i and d = 0..3,
 *   Delta_{i,d} = (V/8) sum_n C_n conj(<h_{i+d}|T_n|e_i> + <h_i|T_n|e_{i+d}>),
 * from the moments of start vectors e_i and e_{i+d}; n_i as before.
 * delta_out is [n_sites*4], n_out [n_sites].  Bond pairing only. */
int orc_order_parameter_bonds(const orc_lattice *L, double a, double T, int M, int K, int kernel,
                              double lambda, const int32_t *sites, int n_sites, cplx *delta_out,
                              double *n_out) {
  if (L->pairing != 1) return -1;
  double *C = (double *)malloc(sizeof(double) * M);
  orc_fold_coefficients(M, K, a, T, kernel, lambda, C);
  int nall = 5 * n_sites;
  int32_t *all = (int32_t *)malloc(sizeof(int32_t) * nall);
  for (int c = 0; c < n_sites; ++c) {
    all[5 * c] = sites[c];
    for (int d = 0; d < 4; ++d) {
      int j = orc_neighbour(L, sites[c], d);
      all[5 * c + 1 + d] = j >= 0 ? j : sites[c];
    }
  }
  double *mu_ee = (double *)malloc(sizeof(double) * (size_t)nall * M);
  cplx *mu_eh = (cplx *)malloc(sizeof(cplx) * (size_t)nall * M * 5);
  orc_moments(L, a, all, nall, M, mu_ee, mu_eh);
  for (int c = 0; c < n_sites; ++c) {
    double nn = 1.0;
    for (int m = 0; m < M; ++m) nn -= C[m] * mu_ee[(size_t)(5 * c) * M + m];
    if (n_out) n_out[c] = nn;
    for (int d = 0; d < 4; ++d) {
      if (orc_neighbour(L, sites[c], d) < 0) {
        delta_out[(size_t)c * 4 + d] = 0.0;
        continue;
      }
      cplx s = 0.0;
      for (int m = 0; m < M; ++m) {
        cplx fwd = mu_eh[((size_t)(5 * c) * M + m) * 5 + 1 + d];
        cplx bwd = mu_eh[((size_t)(5 * c + 1 + d) * M + m) * 5 + 1 + (d ^ 1)];
        s += C[m] * conj(fwd + bwd);
      }
      delta_out[(size_t)c * 4 + d] = 0.125 * coupling_of(L, (size_t)sites[c] * 4 + d) * s;
    }
  }
  free(C);
  free(all);
  free(mu_ee);
  free(mu_eh);
  return 0;
}

/* Up-spin LDOS of Eq. 17 from the expansion of Eq. 10, per unit energy, from
 * given moments mu_ee [n_sites*M]:
 *   N(E, i) = [g_0 mu_0 + 2 sum_{n>=1} g_n mu_n T_n(E/a)] / (pi a sqrt(1-(E/a)^2)).
 * ldos is [n_sites * n_E]. */
int orc_ldos_from_moments(const double *mu_ee, int n_sites, int M, double a, int kernel,
                          double lambda, const double *energies, int n_E, double *ldos) {
  double *g = (double *)malloc(sizeof(double) * M);
  if (kernel == 0) orc_jackson(M, g);
  else orc_lorentz(M, lambda, g);
  for (int c = 0; c < n_sites; ++c) {
    for (int e = 0; e < n_E; ++e) {
      double x = energies[e] / a;
      double th = acos(x);
      double s = g[0] * mu_ee[(size_t)c * M];
      for (int m = 1; m < M; ++m) s += 2.0 * g[m] * mu_ee[(size_t)c * M + m] * cos(m * th);
      ldos[(size_t)c * n_E + e] = s / (M_PI * a * sqrt(1.0 - x * x));
    }
  }
  free(g);
  return 0;
}

/* The LDOS at the listed start sites: moments by the direct recursion, then
 * orc_ldos_from_moments. */
int orc_ldos(const orc_lattice *L, double a, const int32_t *sites, int n_sites, int M,
             int kernel, double lambda, const double *energies, int n_E, double *ldos) {
  int n_eh = (L->pairing == 1) ? 5 : 1;
  double *mu_ee = (double *)malloc(sizeof(double) * (size_t)n_sites * M);
  cplx *mu_eh = (cplx *)malloc(sizeof(cplx) * (size_t)n_sites * M * n_eh);
  orc_moments(L, a, sites, n_sites, M, mu_ee, mu_eh);
  orc_ldos_from_moments(mu_ee, n_sites, M, a, kernel, lambda, energies, n_E, ldos);
  free(mu_ee);
  free(mu_eh);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Nonlocal Green's functions (Eqs. 11-15, gf1) and bond currents (Eq. 20).   */
/* ------------------------------------------------------------------------ */

/* The direct recursion of Eq. 15 from the basis vector of row start_row:
 * out[m*n_rows + r] = <row rows[r] | T_m(H/a) | start_row> for m < M, 0 for
 * rows[r] < 0.  jprev, jcur are work vectors of H->n entries. */
static void chebyshev_rows(const orc_csr *H, double a, int start_row, int M, const int *rows,
                           int n_rows, cplx *out, cplx *jprev, cplx *jcur) {
  memset(jprev, 0, sizeof(cplx) * H->n);
  jprev[start_row] = 1.0;
  for (int m = 0; m < M; ++m) {
    cplx *jn;
    if (m == 0) {
      jn = jprev;
    } else if (m == 1) {
      csr_step(H, 1.0 / a, jprev, 0.0, jprev, jcur);
      jn = jcur;
    } else {
      csr_step(H, 2.0 / a, jcur, -1.0, jprev, jprev);
      cplx *t = jprev;
      jprev = jcur;
      jcur = t;
      jn = jcur;
    }
    for (int r = 0; r < n_rows; ++r) out[(size_t)m * n_rows + r] = rows[r] >= 0 ? jn[rows[r]] : 0.0;
  }
}

/* One direct recursion (Eq. 15) per start vector, j_0 = e_i (start_part 0,
 * the |c^dagger_{i,up}> of Eq. 15) or j_0 = h_i (start_part 1), i = sites[c];
 * every moment is read at every listed target site:
 *   a_e[(c*M + n)*n_t + t] = <e_{targets[t]} | T_n(H/a) | j_0>
 *   a_h[(c*M + n)*n_t + t] = <h_{targets[t]} | T_n(H/a) | j_0>
 * With start_part 0 these are a^{11}_n(t, i) and a^{12}_n(t, i) of Eqs. 11
 * and coeff2 times (1 + delta_n0): one recursion gives G^{1 alpha}_{t i} for
 * all t and alpha (the paragraph after Eq. 15).  Either output may be NULL. */
int orc_green_moments(const orc_lattice *L, double a, int start_part, const int32_t *sites,
                      int n_sites, const int32_t *targets, int n_t, int M, cplx *a_e, cplx *a_h) {
  orc_csr H = build_csr(L);
  int *rows = (int *)malloc(sizeof(int) * 2 * (n_t > 0 ? n_t : 1));
  for (int t = 0; t < n_t; ++t) {
    rows[t] = 2 * targets[t];
    rows[n_t + t] = 2 * targets[t] + 1;
  }
#pragma omp parallel
  {
    cplx *jprev = (cplx *)malloc(sizeof(cplx) * H.n);
    cplx *jcur = (cplx *)malloc(sizeof(cplx) * H.n);
    cplx *out = (cplx *)malloc(sizeof(cplx) * (size_t)M * 2 * (n_t > 0 ? n_t : 1));
#pragma omp for schedule(dynamic, 1)
    for (int c = 0; c < n_sites; ++c) {
      chebyshev_rows(&H, a, 2 * sites[c] + start_part, M, rows, 2 * n_t, out, jprev, jcur);
      for (int m = 0; m < M; ++m)
        for (int t = 0; t < n_t; ++t) {
          size_t o = ((size_t)c * M + m) * n_t + t;
          if (a_e) a_e[o] = out[(size_t)m * 2 * n_t + t];
          if (a_h) a_h[o] = out[(size_t)m * 2 * n_t + n_t + t];
        }
    }
    free(jprev);
    free(jcur);
    free(out);
  }
  free(rows);
  free_csr(&H);
  return 0;
}

/* Retarded Green's function of gf1 from moments of the rescaled H~ = H/a:
 *   G(E) = (1/a) (-2i / sqrt(1 - x^2)) sum_n g_n mom_n / (1 + delta_n0) exp(-i n arccos x),
 * x = E/a, g_n the Jackson (kernel 0) or Lorentz (kernel 1, Eq. 16) kernel;
 * its imaginary part is Eq. imag2 and its real part Eq. real1.  mom is laid
 * out as orc_green_moments writes it, [(c*M + n)*n_t + t]; G is
 * [(c*n_t + t)*n_E + e].  Energies must satisfy |E| < a. */
int orc_green_function(const cplx *mom, int n_sites, int n_t, int M, double a, int kernel,
                       double lambda, const double *energies, int n_E, cplx *G) {
  double *g = (double *)malloc(sizeof(double) * M);
  if (kernel == 0) orc_jackson(M, g);
  else orc_lorentz(M, lambda, g);
  for (int c = 0; c < n_sites; ++c)
    for (int t = 0; t < n_t; ++t)
      for (int e = 0; e < n_E; ++e) {
        double x = energies[e] / a;
        double th = acos(x);
        cplx s = 0.0;
        for (int m = 0; m < M; ++m) {
          cplx am = mom[((size_t)c * M + m) * n_t + t] * g[m] / (m == 0 ? 2.0 : 1.0);
          s += am * cexp(-I * (double)m * th);
        }
        G[((size_t)c * n_t + t) * n_E + e] = -2.0 * I * s / (sqrt(1.0 - x * x) * a);
      }
  free(g);
  return 0;
}

/* Particle current along every bond with hopping (Eq. 20, read as the
 * lattice continuity equation of the hopping term of Eq. 2 with e = hbar = 1):
 *   J^s_{i->j} = 2 Im[ t_ij <c^dagger_{i s} c_{j s}> ],   j = i + d,
 * the one-body density matrix taken from the damped series of
 * f(E) = [1 - tanh(E/2T)]/2 in the Nambu basis (i != j):
 *   spin up:   <c^dag_{i,up} c_{j,up}> = <e_j|f(H)|e_i> = -(1/2) sum_n C_n <e_j|T_n|e_i>
 *   spin down: <c^dag_{i,dn} c_{j,dn}> = -<h_i|f(H)|h_j> = (1/2) conj(sum_n C_n <h_j|T_n|h_i>)
 * spin selects the start vectors: 0 (up) starts from e_i, 1 (down) from h_i.
 * The start sites are sites[0..n_sites), or all N in order when sites is
 * NULL.  J is [n_sites*n_dirs]; J[c*n_dirs + d] is the current from
 * i = sites[c] to i + d, 0 where an open edge cuts the bond. */
int orc_bond_currents(const orc_lattice *L, double a, double T, int M, int K, int kernel,
                      double lambda, int spin, const int32_t *sites, int n_sites, double *J) {
  int nd = L->n_dirs;
  if (!sites) n_sites = L->Lx * L->Ly;
  double *C = (double *)malloc(sizeof(double) * M);
  orc_fold_coefficients(M, K, a, T, kernel, lambda, C);
  orc_csr H = build_csr(L);
#pragma omp parallel
  {
    cplx *jprev = (cplx *)malloc(sizeof(cplx) * H.n);
    cplx *jcur = (cplx *)malloc(sizeof(cplx) * H.n);
    cplx *out = (cplx *)malloc(sizeof(cplx) * (size_t)M * nd);
    int rows[8];
#pragma omp for schedule(dynamic, 1)
    for (int c = 0; c < n_sites; ++c) {
      int i = sites ? sites[c] : c;
      for (int d = 0; d < nd; ++d) {
        int j = orc_neighbour(L, i, d);
        rows[d] = j >= 0 ? 2 * j + spin : -1;
      }
      chebyshev_rows(&H, a, 2 * i + spin, M, rows, nd, out, jprev, jcur);
      for (int d = 0; d < nd; ++d) {
        cplx k = 0.0;
        for (int m = 0; m < M; ++m) k += C[m] * out[(size_t)m * nd + d];
        cplx rho = (spin == 0) ? -0.5 * k : 0.5 * conj(k);
        J[(size_t)c * nd + d] = rows[d] >= 0 ? 2.0 * cimag(L->hop[(size_t)i * nd + d] * rho) : 0.0;
      }
    }
    free(jprev);
    free(jcur);
    free(out);
  }
  free_csr(&H);
  free(C);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Self-consistency (paragraph after Eq. 20).                                */
/* ------------------------------------------------------------------------ */

/* Runs up to max_iter iterations of
 *   a   = 1.1 * Gershgorin bound of H(Delta)
 *   Dout = order parameter from H(Delta)
 *   Delta <- Delta + mix (Dout - Delta)
 * stopping early once max |Dout - Delta| < tol (tol <= 0: never).
 * delta_io holds the starting guess and receives the final mixed Delta;
 * history[k] receives max|Dout - Delta| of iteration k.  Returns the number
 * of iterations run. */
int orc_scf(orc_lattice *L, double T, int M, int K, double mix, double tol, int max_iter,
            cplx *delta_io, double *history, double *n_out) {
  int N = L->Lx * L->Ly;
  int nd = (L->pairing == 1) ? 4 * N : N;
  cplx *dout = (cplx *)malloc(sizeof(cplx) * nd);
  const cplx *saved = L->delta;
  L->delta = delta_io;
  int it;
  for (it = 0; it < max_iter; ++it) {
    double a = 1.1 * orc_gershgorin(L);
    orc_order_parameter(L, a, T, M, K, 0, 0.0, dout, n_out);
    double dmax = 0.0;
    for (int k = 0; k < nd; ++k) {
      double e = cabs(dout[k] - delta_io[k]);
      if (e > dmax) dmax = e;
    }
    for (int k = 0; k < nd; ++k) delta_io[k] += mix * (dout[k] - delta_io[k]);
    if (history) history[it] = dmax;
    if (tol > 0.0 && dmax < tol) {
      it++;
      break;
    }
  }
  L->delta = saved;
  free(dout);
  return it;
}

/* ------------------------------------------------------------------------ */
/* Exact diagonalisation: cyclic Jacobi for a dense Hermitian matrix.        */
/* ------------------------------------------------------------------------ */

/* A (n x n, row-major, Hermitian) is destroyed; w receives the eigenvalues
 * (unsorted) and V (row-major) the eigenvectors as columns: A_in V = V diag(w).
 * Each rotation zeroes A[p][q]: a diagonal phase makes the pivot real, then
 * the real symmetric 2x2 Jacobi rotation with t = tan(theta) of smaller
 * magnitude is applied.  Sweeps until the off-diagonal Frobenius norm falls
 * below tol times the full norm.  Returns the number of sweeps. */
int orc_jacobi_eigh(int n, cplx *A, double *w, cplx *V, double tol, int max_sweeps) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[(size_t)i * n + j] = (i == j) ? 1.0 : 0.0;
  double full = 0.0;
  for (size_t k = 0; k < (size_t)n * n; ++k) full += creal(A[k] * conj(A[k]));
  full = sqrt(full);
  int sweep;
  for (sweep = 0; sweep < max_sweeps; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += 2.0 * creal(A[(size_t)p * n + q] * conj(A[(size_t)p * n + q]));
    off = sqrt(off);
    if (off <= tol * full) break;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        cplx apq = A[(size_t)p * n + q];
        double r = cabs(apq);
        if (r == 0.0) continue;
        cplx ph = apq / r; /* e^{i phi} */
        double app = creal(A[(size_t)p * n + p]), aqq = creal(A[(size_t)q * n + q]);
        double tau = (aqq - app) / (2.0 * r);
        double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        /* J restricted to (p,q): [[ph c, ph s], [-s, c]] */
        cplx Jpp = ph * c, Jpq = ph * s, Jqp = -s, Jqq = c;
        for (int k = 0; k < n; ++k) { /* A <- A J (columns p, q) */
          cplx akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = akp * Jpp + akq * Jqp;
          A[(size_t)k * n + q] = akp * Jpq + akq * Jqq;
        }
        for (int k = 0; k < n; ++k) { /* A <- J^H A (rows p, q) */
          cplx apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = conj(Jpp) * apk + conj(Jqp) * aqk;
          A[(size_t)q * n + k] = conj(Jpq) * apk + conj(Jqq) * aqk;
        }
        A[(size_t)p * n + q] = 0.0;
        A[(size_t)q * n + p] = 0.0;
        A[(size_t)p * n + p] = creal(A[(size_t)p * n + p]);
        A[(size_t)q * n + q] = creal(A[(size_t)q * n + q]);
        for (int k = 0; k < n; ++k) { /* V <- V J */
          cplx vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = vkp * Jpp + vkq * Jqp;
          V[(size_t)k * n + q] = vkp * Jpq + vkq * Jqq;
        }
      }
    }
  }
  for (int i = 0; i < n; ++i) w[i] = creal(A[(size_t)i * n + i]);
  return sweep;
}

/* ------------------------------------------------------------------------ */
/* Reverse-mode gradient of one self-consistency map (a and C_n frozen).     */
/* ------------------------------------------------------------------------ */

/* Reverse mode of the direct recursion for ONE start column e_i (real
 * lattice): stores j_0 .. j_{M-1} in J [M*n], runs the adjoint recursion
 *   lam_m = src[m] u + (2/a) H lam_{m+1} - lam_{m+2}   (m = M-1 .. 1),
 * where u is the basis vector of row src_row, for the output
 * sum_{m>=1} src[m] <u|j_m>, and adds the matrix gradient
 * dOut/dH~_{rs} = sum_{m>=1} f_m lam_m(r) j_{m-1}(s) (f_1 = 1, f_m = 2) at
 * every CSR position of H into Gl.  lam is [(M+2)*n], tmp [n]. */
static void column_reverse_mode(const orc_csr *H, int n, int i, int M, double a, int src_row,
                                const double *src, double *J, double *lam, double *tmp, double *Gl) {
  /* forward, storing every j_m (real) */
  memset(J, 0, sizeof(double) * n);
  J[2 * i] = 1.0;
  for (int m = 1; m < M; ++m) {
    double *jm = J + (size_t)m * n, *j1 = J + (size_t)(m - 1) * n;
    double *j2 = (m >= 2) ? J + (size_t)(m - 2) * n : NULL;
    double s = (m == 1) ? 1.0 / a : 2.0 / a;
    for (int r = 0; r < n; ++r) {
      double acc = 0.0;
      for (int k = H->rowptr[r]; k < H->rowptr[r + 1]; ++k) acc += creal(H->val[k]) * j1[H->col[k]];
      jm[r] = s * acc - (j2 ? j2[r] : 0.0);
    }
  }
  memset(lam, 0, sizeof(double) * (size_t)n * (M + 2));
  for (int m = M - 1; m >= 1; --m) {
    double *lm = lam + (size_t)m * n, *l1 = lam + (size_t)(m + 1) * n, *l2 = lam + (size_t)(m + 2) * n;
    /* lam_m = y_m + (2/a) H l1 - l2, where the step producing j_{m+1} is
     * j_{m+1} = (2/a)H j_m - j_{m-1} for m >= 1 (and j_1 = (1/a) H j_0). */
    for (int r = 0; r < n; ++r) {
      double acc = 0.0;
      for (int k = H->rowptr[r]; k < H->rowptr[r + 1]; ++k) acc += creal(H->val[k]) * l1[H->col[k]];
      tmp[r] = (m + 1 < M ? (2.0 / a) * acc : 0.0) - (m + 2 < M ? l2[r] : 0.0);
    }
    for (int r = 0; r < n; ++r) lm[r] = tmp[r];
    lm[src_row] += src[m];
  }
  /* dL/dH~ contributions: step m (m>=2): j_m = 2 H~ j_{m-1} - j_{m-2}
   *   -> 2 lam_m (x) j_{m-1};  step 1: j_1 = H~ j_0 -> lam_1 (x) j_0.
   * Stored per CSR entry (r,s): sum lam(r) j(s). */
  for (int m = 1; m < M; ++m) {
    double f = (m == 1) ? 1.0 : 2.0;
    double *lm = lam + (size_t)m * n, *jp = J + (size_t)(m - 1) * n;
    for (int r = 0; r < n; ++r) {
      double lr = f * lm[r];
      if (lr == 0.0) continue;
      for (int k = H->rowptr[r]; k < H->rowptr[r + 1]; ++k) Gl[k] += lr * jp[H->col[k]];
    }
  }
}

/* Contracts the matrix gradient G = dL/dH~ (per CSR position of H) with
 * dH~/dparameter (H~ = H/a, Eq. 2):
 *   g_eps[i]        = dL/d eps_i          (H_{e_i e_i} = eps - mu, H_{h_i h_i} = -(eps - mu))
 *   g_hop[i*nd + d] = dL/d t_{i,d}, treating t_{i,d} and its mirror
 *                     t_{i+d,d^1} as ONE real parameter (the undirected bond;
 *                     H_{e_i e_j} = -t, H_{h_i h_j} = +t for both directed
 *                     copies); the value is stored on both directed entries
 *   g_delta[i]      = dL/d Delta_i        (H_{e_i h_i} = H_{h_i e_i} = Delta_i). */
static void matrix_gradient_to_params(const orc_lattice *L, const orc_csr *H, const double *G, double a,
                                      double *g_eps, double *g_hop, double *g_delta) {
  int N = L->Lx * L->Ly;
  int nd = L->n_dirs;
  for (int i = 0; i < N; ++i) {
    double ge = 0.0, gd = 0.0;
    for (int part = 0; part < 2; ++part) {
      int r = 2 * i + part;
      for (int k = H->rowptr[r]; k < H->rowptr[r + 1]; ++k) {
        int c = H->col[k];
        if (c == 2 * i && part == 0) ge += G[k];          /* H_{e_i e_i} = eps - mu */
        if (c == 2 * i + 1 && part == 1) ge -= G[k];      /* H_{h_i h_i} = -(eps - mu) */
        if (c == 2 * i + 1 && part == 0) gd += G[k];      /* H_{e_i h_i} = Delta_i */
        if (c == 2 * i && part == 1) gd += G[k];          /* H_{h_i e_i} = Delta_i */
      }
    }
    g_eps[i] = ge / a;
    g_delta[i] = gd / a;
  }
  for (int i = 0; i < N; ++i) {
    for (int d = 0; d < nd; ++d) {
      int j = orc_neighbour(L, i, d);
      double g = 0.0;
      if (j >= 0) {
        for (int part = 0; part < 2; ++part) {
          for (int side = 0; side < 2; ++side) {
            int r = side == 0 ? 2 * i + part : 2 * j + part;
            int cc = side == 0 ? 2 * j + part : 2 * i + part;
            for (int k = H->rowptr[r]; k < H->rowptr[r + 1]; ++k)
              if (H->col[k] == cc) g += (part == 0 ? -1.0 : 1.0) * G[k];
          }
        }
      }
      g_hop[(size_t)i * nd + d] = g / a;
    }
  }
}

/* Reverse mode over the listed start columns: column c (start site
 * sites[c]) contributes sum_{m>=1} src[c*M + m] <row(c)|j_m>, row(c) =
 * 2 sites[c] + src_part (0: electron row e_i, 1: hole row h_i).  The matrix
 * gradient is summed over columns (per-thread copies, added in thread order)
 * and contracted with dH/dparam. */
static void reverse_mode(const orc_lattice *L, double a, const int32_t *sites, int n_cols, int M, int src_part,
                         const double *src, double *g_eps, double *g_hop, double *g_delta) {
  int N = L->Lx * L->Ly;
  int n = 2 * N;
  orc_csr H = build_csr(L);
  int nnz = H.rowptr[n];
  double *G = (double *)calloc(nnz, sizeof(double));
  int nthreads = 1;
#ifdef _OPENMP
  nthreads = omp_get_max_threads();
#endif
  double *Gt = (double *)calloc((size_t)nnz * nthreads, sizeof(double));
#pragma omp parallel
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    double *Gl = Gt + (size_t)nnz * tid;
    double *J = (double *)malloc(sizeof(double) * (size_t)n * M);
    double *lam = (double *)malloc(sizeof(double) * (size_t)n * (M + 2));
    double *tmp = (double *)malloc(sizeof(double) * n);
#pragma omp for schedule(dynamic, 1)
    for (int c = 0; c < n_cols; ++c)
      column_reverse_mode(&H, n, sites[c], M, a, 2 * sites[c] + src_part, src + (size_t)c * M, J, lam, tmp, Gl);
    free(J);
    free(lam);
    free(tmp);
  }
  for (int t = 0; t < nthreads; ++t)
    for (int k = 0; k < nnz; ++k) G[k] += Gt[(size_t)nnz * t + k];
  free(Gt);
  matrix_gradient_to_params(L, &H, G, a, g_eps, g_hop, g_delta);
  free(G);
  free_csr(&H);
}

/* Real on-site s-wave lattices only (real eps, real hoppings, real Delta).
 * Forward: Dout_i = (U/2) sum_{n<M} C_n <h_i|T_n(H/a)|e_i> for every site.
 * Given w_i = dL/dDout_i, returns g_eps, g_hop, g_delta as described at
 * matrix_gradient_to_params (g_delta = dL/d Delta_in).  For every column
 * the full sequence j_0..j_{M-1} is stored and the adjoint recursion
 * lam_n = y_n + 2 H~ lam_{n+1} - lam_{n+2}, y_n = w_i (U_i/2) C_n h_i, runs
 * backwards (column_reverse_mode). */
int orc_scf_map_gradient(const orc_lattice *L, double a, const double *C, int M,
                         const double *w, double *g_eps, double *g_hop, double *g_delta) {
  int N = L->Lx * L->Ly;
  int32_t *sites = (int32_t *)malloc(sizeof(int32_t) * N);
  double *src = (double *)malloc(sizeof(double) * (size_t)N * M);
  for (int i = 0; i < N; ++i) {
    sites[i] = i;
    double wi = w[i] * 0.5 * coupling_of(L, i);
    for (int m = 0; m < M; ++m) src[(size_t)i * M + m] = wi * C[m];
  }
  reverse_mode(L, a, sites, N, M, 1, src, g_eps, g_hop, g_delta);
  free(sites);
  free(src);
  return 0;
}

/* Reverse-mode gradient of a loss on the up-spin LDOS of Eq. 17 (with the
 * expansion of Eq. 10) at the listed start sites, a frozen.  Real on-site
 * s-wave lattices only.  The forward map is orc_ldos:
 *   N(E_e, i_c) = sum_m w_m(E_e) mu_m(i_c),  mu_m(i) = <e_i|T_m(H/a)|e_i>,
 *   w_m(E) = (2 - delta_m0) g_m T_m(E/a) / (pi a sqrt(1 - (E/a)^2)),
 * so with G[c*n_E + e] = dL/dN(E_e, i_c) the output is
 * sum_c sum_{m>=1} s_{c,m} <e_{i_c}|j_m> with s_{c,m} = sum_e G[c,e] w_m(E_e)
 * (mu_0 = 1 carries no parameter), and the gradient follows by reverse
 * mode exactly as for the self-consistency map, with the source on the
 * electron row.  Returns g_eps, g_hop, g_delta as described at
 * matrix_gradient_to_params. */
int orc_ldos_gradient(const orc_lattice *L, double a, const int32_t *sites, int n_sites, int M, int kernel,
                      double lambda, const double *energies, int n_E, const double *dL_dldos, double *g_eps,
                      double *g_hop, double *g_delta) {
  double *g = (double *)malloc(sizeof(double) * M);
  if (kernel == 0) orc_jackson(M, g);
  else orc_lorentz(M, lambda, g);
  double *src = (double *)calloc((size_t)n_sites * M, sizeof(double));
  for (int c = 0; c < n_sites; ++c) {
    for (int m = 1; m < M; ++m) {
      double s = 0.0;
      for (int e = 0; e < n_E; ++e) {
        double x = energies[e] / a;
        double w = 2.0 * g[m] * cos(m * acos(x)) / (M_PI * a * sqrt(1.0 - x * x));
        s += dL_dldos[(size_t)c * n_E + e] * w;
      }
      src[(size_t)c * M + m] = s;
    }
  }
  reverse_mode(L, a, sites, n_sites, M, 0, src, g_eps, g_hop, g_delta);
  free(g);
  free(src);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Reverse mode for general lattices: complex hoppings (Peierls phases),     */
/* next-nearest neighbours, on-site or bond pairing (a and C_n frozen).      */
/* ------------------------------------------------------------------------ */

/* Forward map: Delta_out = orc_order_parameter (Eq. 19 through the direct
 * recursion of Eq. 15).  For a real loss L with g[k] = dL/dRe Delta_out,k
 * + i dL/dIm Delta_out,k ([N] on-site, [N*4] bond), L changes by
 * Re sum_k conj(g_k) dDelta_out,k.  Column i (start vector e_i) carries
 *   on-site:  Delta_out,i = (U_i/2) sum_m C_m conj(<h_i|j_m>), so the
 *             source is y_m(h_i) = (U_i/2) C_m conj(g_i);
 *   bond:     <h_j|j_m> (j = i + d, d < 4) enters Delta_out,(i,d) and
 *             Delta_out,(j,d^1) with weight (V/8) C_m each (the
 *             symmetrised singlet of the order-parameter routine), so
 *             y_m(h_j) = (C_m/8) conj(V_{i,d} g_{i,d} + V_{j,d^1} g_{j,d^1}).
 * With Phi = Re sum_m <y_m|j_m> the adjoint recursion is
 *   lam_m = y_m + 2 H~ lam_{m+1} - lam_{m+2}   (H~ Hermitian),
 * and dPhi = Re sum_rs G_rs dH~_rs with G_rs = sum_{m>=1} f_m conj(lam_m(r)) j_{m-1}(s)
 * (f_1 = 1, f_m = 2).  Parameters, from the entries of Eq. 2 that each one
 * sets (H~ = H/a), as complex gradients dL/dRe + i dL/dIm:
 *   eps_i:        H_{e_i e_i} = eps - mu, H_{h_i h_i} = -(eps - mu)  (real)
 *   t = t_{i,d}:  H_{e_i e_j} = -t, H_{h_i h_j} = conj(t), and its mirror
 *                 H_{e_j e_i} = -conj(t), H_{h_j h_i} = t; g_hop[i,d] is
 *                 the gradient with respect to t_{i,d}, g_hop[j,d^1] with
 *                 respect to t_{j,d^1} = conj(t), i.e. its conjugate
 *   Delta_i:      H_{e_i h_i} = Delta, H_{h_i e_i} = conj(Delta)
 *   Delta_{i,d}:  H_{e_i h_j} = H_{e_j h_i} = Delta, H_{h_i e_j} = H_{h_j e_i}
 *                 = conj(Delta) (symmetric), stored on both directed entries.
 * Every j_m of a column is stored (no checkpoints).  g_hop [N*n_dirs],
 * g_delta [N] or [N*4]. */

/* G at the CSR position of (r, c), or 0 when the entry is not stored. */
static cplx g_at(const orc_csr *H, const cplx *G, int r, int c) {
  for (int k = H->rowptr[r]; k < H->rowptr[r + 1]; ++k)
    if (H->col[k] == c) return G[k];
  return 0.0;
}

int orc_map_gradient_general(const orc_lattice *L, double a, const double *C, int M, const cplx *g,
                             double *g_eps, cplx *g_hop, cplx *g_delta) {
  int N = L->Lx * L->Ly;
  int n = 2 * N;
  int nd = L->n_dirs;
  orc_csr H = build_csr(L);
  int nnz = H.rowptr[n];
  cplx *G = (cplx *)calloc(nnz, sizeof(cplx));
  int nthreads = 1;
#ifdef _OPENMP
  nthreads = omp_get_max_threads();
#endif
  cplx *Gt = (cplx *)calloc((size_t)nnz * nthreads, sizeof(cplx));
#pragma omp parallel
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    cplx *Gl = Gt + (size_t)nnz * tid;
    cplx *J = (cplx *)malloc(sizeof(cplx) * (size_t)n * M);
    cplx *lam = (cplx *)malloc(sizeof(cplx) * (size_t)n * (M + 2));
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * n);
#pragma omp for schedule(dynamic, 1)
    for (int i = 0; i < N; ++i) {
      /* forward: j_0 = e_i, j_1 = H~ j_0, j_m = 2 H~ j_{m-1} - j_{m-2} */
      memset(J, 0, sizeof(cplx) * n);
      J[2 * i] = 1.0;
      for (int m = 1; m < M; ++m) {
        cplx *jm = J + (size_t)m * n, *j1 = J + (size_t)(m - 1) * n;
        cplx *j2 = (m >= 2) ? J + (size_t)(m - 2) * n : NULL;
        double sc = (m == 1) ? 1.0 / a : 2.0 / a;
        for (int r = 0; r < n; ++r) {
          cplx acc = 0.0;
          for (int k = H.rowptr[r]; k < H.rowptr[r + 1]; ++k) acc += H.val[k] * j1[H.col[k]];
          jm[r] = sc * acc - (j2 ? j2[r] : 0.0);
        }
      }
      /* source rows and weights of this column: y_m(row) = C_m * w_row */
      int srow[4];
      cplx sw[4];
      int ns = 0;
      if (L->pairing == 0) {
        srow[ns] = 2 * i + 1;
        sw[ns++] = 0.5 * coupling_of(L, i) * conj(g[i]);
      } else {
        for (int d = 0; d < 4; ++d) {
          int j = orc_neighbour(L, i, d);
          if (j < 0) continue;
          srow[ns] = 2 * j + 1;
          sw[ns++] = 0.125 * conj(coupling_of(L, (size_t)i * 4 + d) * g[(size_t)i * 4 + d] +
                                  coupling_of(L, (size_t)j * 4 + (d ^ 1)) * g[(size_t)j * 4 + (d ^ 1)]);
        }
      }
      memset(lam, 0, sizeof(cplx) * (size_t)n * (M + 2));
      for (int m = M - 1; m >= 1; --m) {
        cplx *lm = lam + (size_t)m * n, *l1 = lam + (size_t)(m + 1) * n, *l2 = lam + (size_t)(m + 2) * n;
        for (int r = 0; r < n; ++r) {
          cplx acc = 0.0;
          for (int k = H.rowptr[r]; k < H.rowptr[r + 1]; ++k) acc += H.val[k] * l1[H.col[k]];
          tmp[r] = (m + 1 < M ? (2.0 / a) * acc : 0.0) - (m + 2 < M ? l2[r] : 0.0);
        }
        for (int r = 0; r < n; ++r) lm[r] = tmp[r];
        for (int q = 0; q < ns; ++q) lm[srow[q]] += C[m] * sw[q];
      }
      for (int m = 1; m < M; ++m) {
        double f = (m == 1) ? 1.0 : 2.0;
        cplx *lm = lam + (size_t)m * n, *jp = J + (size_t)(m - 1) * n;
        for (int r = 0; r < n; ++r) {
          cplx lr = f * conj(lm[r]);
          if (lr == 0.0) continue;
          for (int k = H.rowptr[r]; k < H.rowptr[r + 1]; ++k) Gl[k] += lr * jp[H.col[k]];
        }
      }
    }
    free(J);
    free(lam);
    free(tmp);
  }
  for (int t = 0; t < nthreads; ++t)
    for (int k = 0; k < nnz; ++k) G[k] += Gt[(size_t)nnz * t + k];
  free(Gt);
  for (int i = 0; i < N; ++i) {
    int e = 2 * i, h = 2 * i + 1;
    g_eps[i] = creal(g_at(&H, G, e, e) - g_at(&H, G, h, h)) / a;
    if (L->pairing == 0) {
      cplx geh = g_at(&H, G, e, h), ghe = g_at(&H, G, h, e);
      g_delta[i] = (creal(geh + ghe) + I * (cimag(ghe) - cimag(geh))) / a;
    }
    for (int d = 0; d < nd; ++d) {
      int j = orc_neighbour(L, i, d);
      if (j < 0) {
        g_hop[(size_t)i * nd + d] = 0.0;
        if (L->pairing == 1 && d < 4) g_delta[(size_t)i * 4 + d] = 0.0;
        continue;
      }
      int ej = 2 * j, hj = 2 * j + 1;
      cplx a1 = g_at(&H, G, e, ej), a2 = g_at(&H, G, h, hj), a3 = g_at(&H, G, ej, e), a4 = g_at(&H, G, hj, h);
      double gr = creal(-a1 + a2 - a3 + a4), gi = cimag(a1) + cimag(a2) - cimag(a3) - cimag(a4);
      g_hop[(size_t)i * nd + d] = (gr + I * gi) / a;
      if (L->pairing == 1 && d < 4) {
        cplx b1 = g_at(&H, G, e, hj), b2 = g_at(&H, G, ej, h), b3 = g_at(&H, G, h, ej), b4 = g_at(&H, G, hj, e);
        double dr = creal(b1 + b2 + b3 + b4), di = -cimag(b1) - cimag(b2) + cimag(b3) + cimag(b4);
        g_delta[(size_t)i * 4 + d] = (dr + I * di) / a;
      }
    }
  }
  free(G);
  free_csr(&H);
  return 0;
}

/* Thread count the oracle runs with (for the CPU-baseline record). */
int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
