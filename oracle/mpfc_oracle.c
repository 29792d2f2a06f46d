/*
 * mpfc_oracle.c -- plain, slow FP64 CPU oracle of the MPFC convex-splitting schemes
 * and their nonlinear FAS multigrid solver.  Built twice from this one source: serial,
 * and with OpenMP over the host cores, which parallelises only loops over independent
 * cells and keeps every reduction serial, so the two builds give identical bits.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or calls
 * this file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header or constant with the CUDA path.
 *
 * Paper: Baskaran, Zhou, Hu, Wang, Wise, Lowengrub, "Energy stable and efficient
 * finite-difference nonlinear multigrid schemes for the modified phase field
 * crystal equation" (arXiv:1208.2643).
 *
 * Grid functions are m x n cell-centred arrays stored row-major, f[j*m + i], with
 * i the x index (0..m-1) and j the y index (0..n-1).  The ghost ring of App. A is
 * not stored: periodic boundary conditions (App. A, (A.8)-(A.9)) are applied by
 * wrapping indices.  orc_set_boundary(1) switches every following call to the mixed
 * conditions of Sec. 4.5: periodic in x, homogeneous Neumann in y with the ghost rule
 * of App. A, (A.7): phi_{i,0} = phi_{i,1}, phi_{i,n+1} = phi_{i,n}, i.e. a ghost row
 * holds the value of the boundary row next to it.
 *
 * Readings of points the paper leaves open:
 *  - smoother: red-black ordering, red = (i+j) even first; one local Newton
 *    linearisation of the cubic per cell visit (App. B.1 offers Newton or Picard;
 *    Picard is kept as an option); the cell update may be under-relaxed,
 *    u <- u + omega (x - u).  omega = 1 is the smoother exactly as printed; for
 *    intermediate time steps that smoother amplifies the smoothest error modes
 *    (spectral radius of one red-black sweep above 1) and the V-cycle stalls,
 *    which omega = 0.8 cures;
 *  - App. B.2 smoother, first equation: the neighbour coefficient is read as
 *    sM/(h^2(beta+2/s)) (the printed factor 4 contradicts the operator N^(1));
 *    third equation: kappa^{k+1,l+1} read as kappa^{l+1};
 *  - FAS transfers (the paper defers to Trottenberg et al.): restriction is the
 *    2x2 cell average, prolongation the cell-centred bilinear (9,3,3,1)/16 stencil,
 *    coarse source S_c = N_c(R u) + R(S - N(u)); scheme 2 uses phi^k_c = R phi^k;
 *  - coarsest level (a few cells per side): dense Newton on all 3*m*n unknowns,
 *    Gaussian elimination with partial pivoting;
 *  - stopping rule: scaled residual sqrt(sum_{c,i,j} r_c^2 / (3mn)) <= tol;
 *  - pinning (Sec. 4.6, second-order scheme only): the unknown mu is the pinned
 *    potential mu~ = mu + 2 (phi^{k+1/2} - phihat) W, W the weight; with
 *    phi^{k+1/2} = (phi + phi^k)/2 this moves W phi into row 2 of N, a pointwise
 *    linear term (gam -> gam + W_ij), and W (phi^k - 2 phihat) into S2; coarse
 *    levels use the 2x2 average of W (standard FAS restriction);
 *  - Neumann rows (Sec. 4.5 says only that the solver is easily adapted): explicit
 *    stencils read the ghost row as the boundary row (A.7); in the smoother's cell
 *    system the ghost is the unknown itself, so it leaves the neighbour sum and the
 *    diagonal count drops from 4 to 3 (exact elimination of the ghost); the
 *    transfers and the coarsest solve use the same ghost rule on every level.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAX_LEVELS 16

/* All-cores build (compiled with -fopenmp; the serial build ignores the pragmas):
 * only loops whose iterations write disjoint cells and read nothing another iteration
 * writes run in parallel -- the cells of one colour in a smoothing half sweep, the
 * cells of an operator application, of a source, of a transfer.  Every reduction (the
 * residual norm) stays serial in the serial order, so both builds give the same bits.
 * Grids below ORC_OMP_CELLS cells stay serial (thread start-up would dominate). */
#define ORC_OMP_CELLS 4096

/* Threads of the parallel loops (OpenMP build); returns the number in use, 1 in the
 * serial build. */
int orc_set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
  return omp_get_max_threads();
#else
  (void)nthreads;
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Parameters                                                               */
/* ------------------------------------------------------------------------ */
typedef struct {
  int m, n;          /* cells in x and y on the finest grid                    */
  double h;          /* finest spacing, L_x = m h, L_y = n h (App. A)           */
  double M;          /* mobility                                                */
  double eps;        /* alpha = 1 - eps (Sec. 2, (2.1))                          */
  double beta;       /* damping                                                 */
  double s;          /* time step                                               */
  int nu1, nu2;      /* pre/post smoothing sweeps (l_max of App. B)             */
  int newton;        /* 1: local Newton linearisation, 0: local Picard          */
  int coarse_cells;  /* coarsen while the coarse grid keeps >= this many cells
                        per side and both sides stay even                        */
  double omega;      /* relaxation of the cell update; 1 = the paper's smoother */
  int model;         /* 0: MPFC (2), the damped wave equation; 1: PFC (1), the
                        parabolic special case d_t phi = M Delta mu (Sec. 1)      */
} orc_params;

/* Scheme constants of the FAS operator N (App. B.1 / B.2).
 *   c     coefficient of Delta_h mu in N^(1): sM/(beta+1/s) or sM/(beta+2/s)
 *   gam   linear coefficient in N^(2):        alpha        or alpha/2
 *   theta coefficient of Delta_h phi in N^(3): 1           or 1/2           */
typedef struct { double c, gam, theta; int scheme; double omega; } orc_consts;

static orc_consts consts_of(const orc_params* p, int scheme) {
  orc_consts k;
  double alpha = 1.0 - p->eps;
  k.scheme = scheme;
  k.omega = p->omega;
  if (scheme == 1) {
    k.c = p->s * p->M / (p->beta + 1.0 / p->s);
    k.gam = alpha;
    k.theta = 1.0;
  } else {
    k.c = p->s * p->M / (p->beta + 2.0 / p->s);
    k.gam = 0.5 * alpha;
    k.theta = 0.5;
  }
  /* PFC, (phi^{k+1} - phi^k)/s = M Delta_h mu with the same mu as the MPFC schemes:
   * row 1 of N reads phi - s M Delta_h mu */
  if (p->model == 1) k.c = p->s * p->M;
  return k;
}

/* ------------------------------------------------------------------------ */
/* Grid helpers (App. A)                                                    */
/* ------------------------------------------------------------------------ */
static int g_ny_neumann = 0;   /* 0: periodic in y (A.9); 1: homogeneous Neumann in y (A.7) */

void orc_set_boundary(int ny_neumann) { g_ny_neumann = ny_neumann ? 1 : 0; }
int orc_get_boundary(void) { return g_ny_neumann; }

static int wrap(int i, int m) { return (i % m + m) % m; }

/* Stored row that holds row j (j = -1 and j = n are the ghost rows). */
static int yrow(int j, int n) {
  if (!g_ny_neumann) return wrap(j, n);
  return j < 0 ? 0 : (j >= n ? n - 1 : j);
}

/* Whether row j is a ghost row under the Neumann rule. */
static int y_is_ghost(int j, int n) { return g_ny_neumann && (j < 0 || j >= n); }

static double at(const double* f, int m, int n, int i, int j) {
  return f[yrow(j, n) * m + wrap(i, m)];
}

/* Sum of the four face neighbours, ghost values by the boundary rule. */
static double nb_sum(const double* f, int m, int n, int i, int j) {
  return at(f, m, n, i - 1, j) + at(f, m, n, i + 1, j) + at(f, m, n, i, j - 1) + at(f, m, n, i, j + 1);
}

/* Sum over the face neighbours that are not ghost cells, and their number. */
static double real_nb_sum(const double* f, int m, int n, int i, int j, int* count) {
  double s = at(f, m, n, i - 1, j) + at(f, m, n, i + 1, j);
  int c = 2;
  if (!y_is_ghost(j - 1, n)) { s += at(f, m, n, i, j - 1); ++c; }
  if (!y_is_ghost(j + 1, n)) { s += at(f, m, n, i, j + 1); ++c; }
  *count = c;
  return s;
}

/* Standard five-point discrete Laplacian Delta_h (App. A) with the ghost
 * values of the boundary rule (periodic (A.8)-(A.9), or (A.7) in y). */
void orc_laplacian(int m, int n, double h, const double* f, double* out) {
#pragma omp parallel for schedule(static) if (m * n >= ORC_OMP_CELLS)
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < m; ++i)
      out[j * m + i] = (nb_sum(f, m, n, i, j) - 4.0 * f[j * m + i]) / (h * h);
}

/* Nonlinear term g of N^(2) and its derivative.
 *   scheme 1 (App. B.1): g(phi) = phi^3.
 *   scheme 2 (App. B.2): g(phi) = (1/2) chi(phi, phik) (phi + phik),
 *     chi(a,b) = (a^2 + b^2)/2 (Sec. 3.2). */
static double g_of(int scheme, double phi, double phik) {
  if (scheme == 1) return phi * phi * phi;
  return 0.5 * (0.5 * (phi * phi + phik * phik)) * (phi + phik);
}
static double dg_of(int scheme, double phi, double phik) {
  if (scheme == 1) return 3.0 * phi * phi;
  /* d/dphi [ (phi^2+phik^2)(phi+phik)/4 ] = (2 phi (phi+phik) + phi^2 + phik^2)/4 */
  return 0.25 * (2.0 * phi * (phi + phik) + phi * phi + phik * phik);
}

/* ------------------------------------------------------------------------ */
/* FAS operator N and source S                                              */
/* ------------------------------------------------------------------------ */
/* N(u), u = (phi, mu, kappa):  App. B.1 (scheme 1) and App. B.2 (scheme 2).
 *   N1 = phi   - c Delta_h mu
 *   N2 = mu    - g(phi) - gam phi - Delta_h kappa
 *   N3 = kappa - theta Delta_h phi
 * phik is only read for scheme 2. */
/* W (nullable): pinning weight on this grid (Sec. 4.6); row 2 then reads
 *   N2 = mu - g(phi) - (gam + W) phi - Delta_h kappa. */
static void apply_N_w(int scheme, double c, double gam, double theta, int m, int n, double h,
                      const double* phi, const double* mu, const double* kappa, const double* phik,
                      const double* W, double* N1, double* N2, double* N3) {
  double* lmu = malloc(sizeof(double) * m * n);
  double* lka = malloc(sizeof(double) * m * n);
  double* lph = malloc(sizeof(double) * m * n);
  orc_laplacian(m, n, h, mu, lmu);
  orc_laplacian(m, n, h, kappa, lka);
  orc_laplacian(m, n, h, phi, lph);
#pragma omp parallel for schedule(static) if (m * n >= ORC_OMP_CELLS)
  for (int k = 0; k < m * n; ++k) {
    double pk = (scheme == 2) ? phik[k] : 0.0;
    N1[k] = phi[k] - c * lmu[k];
    N2[k] = mu[k] - g_of(scheme, phi[k], pk) - gam * phi[k] - lka[k];
    if (W) N2[k] -= W[k] * phi[k];
    N3[k] = kappa[k] - theta * lph[k];
  }
  free(lmu); free(lka); free(lph);
}

void orc_apply_N(int scheme, double c, double gam, double theta, int m, int n, double h,
                 const double* phi, const double* mu, const double* kappa, const double* phik,
                 double* N1, double* N2, double* N3) {
  apply_N_w(scheme, c, gam, theta, m, n, h, phi, mu, kappa, phik, NULL, N1, N2, N3);
}

/* Source S.
 * Scheme 1 (App. B.1): S1 = phik + psik/(beta+1/s), S2 = 2 Delta_h phik, S3 = 0.
 * PFC (either scheme): S1 = phik (no velocity term).
 * Scheme 2 (App. B.2): S1 = phik + 2 psik/(beta+2/s),
 *   S2 = (alpha/2) phik + 2 Delta_h phitilde, phitilde = (3 phik - phikm1)/2,
 *   S3 = (1/2) Delta_h phik. */
/* Pinned source (Sec. 4.6, scheme 2): S2 additionally gets W (phi^k - 2 phihat), the
 * part of 2 W (phi^{k+1/2} - phihat) that does not involve the unknown. */
static void source_w(int scheme, const orc_params* p, const double* phik, const double* phikm1,
                     const double* psik, const double* W, const double* phihat, double* S1, double* S2,
                     double* S3);

void orc_source(int scheme, const orc_params* p, const double* phik, const double* phikm1,
                const double* psik, double* S1, double* S2, double* S3) {
  source_w(scheme, p, phik, phikm1, psik, NULL, NULL, S1, S2, S3);
}

static void source_w(int scheme, const orc_params* p, const double* phik, const double* phikm1,
                     const double* psik, const double* W, const double* phihat, double* S1, double* S2,
                     double* S3) {
  int m = p->m, n = p->n, N = m * n;
  double alpha = 1.0 - p->eps;
  double* lap = malloc(sizeof(double) * N);
  if (scheme == 1) {
    orc_laplacian(m, n, p->h, phik, lap);
#pragma omp parallel for schedule(static) if (N >= ORC_OMP_CELLS)
    for (int k = 0; k < N; ++k) {
      S1[k] = phik[k] + (p->model == 1 ? 0.0 : psik[k] / (p->beta + 1.0 / p->s));
      S2[k] = 2.0 * lap[k];
      S3[k] = 0.0;
    }
  } else {
    double* tl = malloc(sizeof(double) * N);
    double* lap_t = malloc(sizeof(double) * N);
    for (int k = 0; k < N; ++k) tl[k] = 0.5 * (3.0 * phik[k] - phikm1[k]);
    orc_laplacian(m, n, p->h, tl, lap_t);
    orc_laplacian(m, n, p->h, phik, lap);
#pragma omp parallel for schedule(static) if (N >= ORC_OMP_CELLS)
    for (int k = 0; k < N; ++k) {
      S1[k] = phik[k] + (p->model == 1 ? 0.0 : 2.0 * psik[k] / (p->beta + 2.0 / p->s));
      S2[k] = 0.5 * alpha * phik[k] + 2.0 * lap_t[k];
      if (W) S2[k] += W[k] * (phik[k] - 2.0 * phihat[k]);
      S3[k] = 0.5 * lap[k];
    }
    free(tl); free(lap_t);
  }
  free(lap);
}

/* ------------------------------------------------------------------------ */
/* Smoother (App. B.1 / B.2): nonlinear red-black block Gauss-Seidel        */
/* ------------------------------------------------------------------------ */
/* Cramer's rule for the 3x3 cell system  A x = r  (App. B: "we solve for the
 * unknowns ... using Cramer's rule").  A is row-major. */
static double det3(const double* A) {
  return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
         A[2] * (A[3] * A[7] - A[4] * A[6]);
}
void orc_cramer3(const double* A, const double* r, double* x) {
  double D = det3(A);
  for (int col = 0; col < 3; ++col) {
    double B[9];
    memcpy(B, A, sizeof(B));
    for (int row = 0; row < 3; ++row) B[row * 3 + col] = r[row];
    x[col] = det3(B) / D;
  }
}

/* One visit of cell (i,j): builds the cell's 3x3 linearised system from the
 * smoothing scheme of App. B and replaces (phi, mu, kappa) at that cell.
 *   eq 1: phi + (d c/h^2) mu                    = S1 + (c/h^2) sum_nb mu
 *   eq 2: -(gam + q) phi + mu + (d/h^2) kappa   = S2 + e + (1/h^2) sum_nb kappa
 *   eq 3: (d theta/h^2) phi + kappa             = S3 + (theta/h^2) sum_nb phi
 * where sum_nb runs over the d face neighbours that are not ghost cells (d = 4,
 * or 3 next to a Neumann boundary, whose ghost is the cell's own unknown)
 * with the cubic linearised about the current value p = phi_ij:
 *   Newton: g(phi) ~ g(p) + g'(p)(phi - p)  ->  q = g'(p),  e = g(p) - g'(p) p
 *   Picard, scheme 1: phi^3 ~ p^2 phi        ->  q = p^2,    e = 0
 *   Picard, scheme 2: g ~ chi(p,phik)(phi+phik)/2
 *                                            ->  q = chi/2,  e = chi phik / 2  */
static void visit_cell(const orc_consts* k, int newton, int m, int n, double h, int i, int j,
                       double* phi, double* mu, double* kappa, const double* S1, const double* S2,
                       const double* S3, const double* phik, const double* W) {
  int id = j * m + i;
  double h2 = h * h;
  double p = phi[id];
  double pk = (k->scheme == 2) ? phik[id] : 0.0;
  double q, e;
  if (newton) {
    q = dg_of(k->scheme, p, pk);
    e = g_of(k->scheme, p, pk) - q * p;
  } else if (k->scheme == 1) {
    q = p * p;
    e = 0.0;
  } else {
    double chi = 0.5 * (p * p + pk * pk);
    q = 0.5 * chi;
    e = 0.5 * chi * pk;
  }
  int d;
  double smu = real_nb_sum(mu, m, n, i, j, &d);
  double ska = real_nb_sum(kappa, m, n, i, j, &d);
  double sph = real_nb_sum(phi, m, n, i, j, &d);
  double w = W ? W[id] : 0.0;   /* pinning weight: a pointwise linear term of row 2 */
  double A[9] = {1.0, d * k->c / h2, 0.0,
                 -(k->gam + w + q), 1.0, d / h2,
                 d * k->theta / h2, 0.0, 1.0};
  double r[3] = {S1[id] + k->c / h2 * smu,
                 S2[id] + e + ska / h2,
                 S3[id] + k->theta / h2 * sph};
  double x[3];
  orc_cramer3(A, r, x);
  /* relaxed update u <- u + omega (x - u); omega = 1 is the plain update */
  phi[id] = p + k->omega * (x[0] - p);
  mu[id] = mu[id] + k->omega * (x[1] - mu[id]);
  kappa[id] = kappa[id] + k->omega * (x[2] - kappa[id]);
}

/* sweeps full red-black passes: red cells ((i+j) even) first, then black. */
static void smooth_w(int scheme, double c, double gam, double theta, int newton, double omega, int sweeps, int m,
                     int n, double h, double* phi, double* mu, double* kappa, const double* S1, const double* S2,
                     const double* S3, const double* phik, const double* W) {
  orc_consts k = {c, gam, theta, scheme, omega};
  for (int sw = 0; sw < sweeps; ++sw)
    for (int color = 0; color < 2; ++color) {
      /* the cells of one colour only read the other colour's values: any order */
#pragma omp parallel for schedule(static) if (m * n >= ORC_OMP_CELLS)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < m; ++i)
          if (((i + j) & 1) == color)
            visit_cell(&k, newton, m, n, h, i, j, phi, mu, kappa, S1, S2, S3, phik, W);
    }
}

void orc_smooth(int scheme, double c, double gam, double theta, int newton, double omega, int sweeps, int m,
                int n, double h, double* phi, double* mu, double* kappa, const double* S1, const double* S2,
                const double* S3, const double* phik) {
  smooth_w(scheme, c, gam, theta, newton, omega, sweeps, m, n, h, phi, mu, kappa, S1, S2, S3, phik, NULL);
}

/* ------------------------------------------------------------------------ */
/* FAS transfers (standard FAS V-cycle, App. B; readings in the header)      */
/* ------------------------------------------------------------------------ */
/* Restriction: coarse cell = average of its 2x2 fine children. */
void orc_restrict(int mc, int nc, const double* fine, double* coarse) {
  int mf = 2 * mc;
#pragma omp parallel for schedule(static) if (4 * mc * nc >= ORC_OMP_CELLS)
  for (int J = 0; J < nc; ++J)
    for (int I = 0; I < mc; ++I)
      coarse[J * mc + I] = 0.25 * (fine[(2 * J) * mf + 2 * I] + fine[(2 * J) * mf + 2 * I + 1] +
                                   fine[(2 * J + 1) * mf + 2 * I] + fine[(2 * J + 1) * mf + 2 * I + 1]);
}

/* Prolongation (added into fine): cell-centred bilinear interpolation.  A fine
 * cell lies a quarter coarse spacing from its parent's centre, towards the
 * neighbour at di = -1 for even i and di = +1 for odd i (likewise dj);
 * weights 9/16 (parent), 3/16, 3/16 (face neighbours), 1/16 (diagonal). */
void orc_prolong_add(int mc, int nc, const double* coarse, double* fine) {
  int mf = 2 * mc, nf = 2 * nc;
#pragma omp parallel for schedule(static) if (mf * nf >= ORC_OMP_CELLS)
  for (int j = 0; j < nf; ++j)
    for (int i = 0; i < mf; ++i) {
      int I = i / 2, J = j / 2;
      int di = (i % 2 == 0) ? -1 : 1, dj = (j % 2 == 0) ? -1 : 1;
      double v = 9.0 * at(coarse, mc, nc, I, J) + 3.0 * at(coarse, mc, nc, I + di, J) +
                 3.0 * at(coarse, mc, nc, I, J + dj) + 1.0 * at(coarse, mc, nc, I + di, J + dj);
      fine[j * mf + i] += v / 16.0;
    }
}

/* ------------------------------------------------------------------------ */
/* Coarsest level: dense Newton on all 3*m*n unknowns                       */
/* ------------------------------------------------------------------------ */
/* Solve A x = b (A is N x N row-major, overwritten) by Gaussian elimination
 * with partial pivoting.  Returns 0, or -1 on a zero pivot. */
int orc_gauss_solve(int N, double* A, double* b, double* x) {
  for (int col = 0; col < N; ++col) {
    int piv = col;
    for (int r = col + 1; r < N; ++r)
      if (fabs(A[r * N + col]) > fabs(A[piv * N + col])) piv = r;
    if (A[piv * N + col] == 0.0) return -1;
    if (piv != col) {
      for (int c2 = 0; c2 < N; ++c2) {
        double t = A[col * N + c2]; A[col * N + c2] = A[piv * N + c2]; A[piv * N + c2] = t;
      }
      double t = b[col]; b[col] = b[piv]; b[piv] = t;
    }
    for (int r = col + 1; r < N; ++r) {
      double f = A[r * N + col] / A[col * N + col];
      if (f == 0.0) continue;
      for (int c2 = col; c2 < N; ++c2) A[r * N + c2] -= f * A[col * N + c2];
      b[r] -= f * b[col];
    }
  }
  for (int r = N - 1; r >= 0; --r) {
    double acc = b[r];
    for (int c2 = r + 1; c2 < N; ++c2) acc -= A[r * N + c2] * x[c2];
    x[r] = acc / A[r * N + r];
  }
  return 0;
}

/* Newton's method for N(u) = S on a small grid.  Unknown ordering:
 * [phi (m n), mu (m n), kappa (m n)].  Jacobian blocks, with L the matrix of
 * Delta_h and D = diag(gam + g'(phi)):
 *   [ I       -c L   0  ]
 *   [ -D       I    -L  ]
 *   [ -theta L 0     I  ]
 * Iterates until the update is below 1e-15 (1 + |u|_inf), then takes one
 * more iteration; at most 60 iterations.  Returns the iteration count. */
static int coarse_newton_w(int scheme, double c, double gam, double theta, int m, int n, double h,
                           double* phi, double* mu, double* kappa, const double* S1, const double* S2,
                           const double* S3, const double* phik, const double* W) {
  int G = m * n, N = 3 * G;
  double* A = malloc(sizeof(double) * N * N);
  double* b = malloc(sizeof(double) * N);
  double* x = malloc(sizeof(double) * N);
  double* N1 = malloc(sizeof(double) * G);
  double* N2 = malloc(sizeof(double) * G);
  double* N3 = malloc(sizeof(double) * G);
  double h2 = h * h;
  int it, extra = -1;
  for (it = 0; it < 60; ++it) {
    apply_N_w(scheme, c, gam, theta, m, n, h, phi, mu, kappa, phik, W, N1, N2, N3);
    for (int k = 0; k < G; ++k) {
      b[k] = S1[k] - N1[k];
      b[G + k] = S2[k] - N2[k];
      b[2 * G + k] = S3[k] - N3[k];
    }
    memset(A, 0, sizeof(double) * N * N);
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < m; ++i) {
        int r = j * m + i;
        /* a ghost neighbour is the boundary cell itself (yrow), which folds it into the diagonal */
        int nbr[4] = {j * m + wrap(i - 1, m), j * m + wrap(i + 1, m), yrow(j - 1, n) * m + i,
                      yrow(j + 1, n) * m + i};
        double pk = (scheme == 2) ? phik[r] : 0.0;
        /* row block 1: phi - c Lap mu */
        A[r * N + r] += 1.0;
        A[r * N + G + r] += 4.0 * c / h2;
        for (int t = 0; t < 4; ++t) A[r * N + G + nbr[t]] -= c / h2;
        /* row block 2: mu - g(phi) - gam phi - Lap kappa */
        A[(G + r) * N + r] += -(gam + (W ? W[r] : 0.0) + dg_of(scheme, phi[r], pk));
        A[(G + r) * N + G + r] += 1.0;
        A[(G + r) * N + 2 * G + r] += 4.0 / h2;
        for (int t = 0; t < 4; ++t) A[(G + r) * N + 2 * G + nbr[t]] -= 1.0 / h2;
        /* row block 3: kappa - theta Lap phi */
        A[(2 * G + r) * N + 2 * G + r] += 1.0;
        A[(2 * G + r) * N + r] += 4.0 * theta / h2;
        for (int t = 0; t < 4; ++t) A[(2 * G + r) * N + nbr[t]] -= theta / h2;
      }
    if (orc_gauss_solve(N, A, b, x) != 0) break;
    double dmax = 0.0, umax = 0.0;
    for (int k = 0; k < G; ++k) {
      phi[k] += x[k];
      mu[k] += x[G + k];
      kappa[k] += x[2 * G + k];
      double d = fmax(fabs(x[k]), fmax(fabs(x[G + k]), fabs(x[2 * G + k])));
      double u = fmax(fabs(phi[k]), fmax(fabs(mu[k]), fabs(kappa[k])));
      if (d > dmax) dmax = d;
      if (u > umax) umax = u;
    }
    if (extra >= 0) break;
    if (dmax <= 1e-15 * (1.0 + umax)) extra = it;
  }
  free(A); free(b); free(x); free(N1); free(N2); free(N3);
  return it + 1;
}

int orc_coarse_newton(int scheme, double c, double gam, double theta, int m, int n, double h,
                      double* phi, double* mu, double* kappa, const double* S1, const double* S2,
                      const double* S3, const double* phik) {
  return coarse_newton_w(scheme, c, gam, theta, m, n, h, phi, mu, kappa, S1, S2, S3, phik, NULL);
}

/* ------------------------------------------------------------------------ */
/* Level hierarchy and the FAS V-cycle                                      */
/* ------------------------------------------------------------------------ */
typedef struct {
  int m, n;
  double h;
  double *phi, *mu, *kappa;   /* u                                   */
  double *S1, *S2, *S3;       /* source (tau-corrected on coarse)    */
  double *r1, *r2, *r3;       /* residual scratch                    */
  double *b1, *b2, *b3;       /* R u_f saved for the correction      */
  double* phik;               /* phi^k on this level (scheme 2)      */
  double* W;                  /* pinning weight (NULL: no pinning)   */
} orc_level;

typedef struct {
  orc_params p;
  int nlev;
  orc_level lev[ORC_MAX_LEVELS];
  double *phik, *phikm1, *psik;   /* time-level state (Sec. 3)          */
  double* phihat;                 /* pinning target (Sec. 4.6), finest grid */
  long step_index;
} orc_ctx;

static double* zalloc(int count) { return calloc((size_t)count, sizeof(double)); }

/* Number of levels: halve while both sides stay even and the coarse grid
 * keeps at least coarse_cells cells per side. */
int orc_num_levels(int m, int n, int coarse_cells) {
  int L = 1;
  while (L < ORC_MAX_LEVELS && m % 2 == 0 && n % 2 == 0 && m / 2 >= coarse_cells && n / 2 >= coarse_cells &&
         (m / 2) % 2 == 0 && (n / 2) % 2 == 0) {
    m /= 2;
    n /= 2;
    ++L;
  }
  return L;
}

orc_ctx* orc_create(const orc_params* p) {
  if (p->m < 2 || p->n < 2 || p->m % 2 || p->n % 2) return NULL;
  orc_ctx* ctx = calloc(1, sizeof(orc_ctx));
  ctx->p = *p;
  ctx->nlev = orc_num_levels(p->m, p->n, p->coarse_cells);
  int m = p->m, n = p->n;
  double h = p->h;
  for (int l = 0; l < ctx->nlev; ++l) {
    orc_level* L = &ctx->lev[l];
    int G = m * n;
    L->m = m; L->n = n; L->h = h;
    L->phi = zalloc(G); L->mu = zalloc(G); L->kappa = zalloc(G);
    L->S1 = zalloc(G); L->S2 = zalloc(G); L->S3 = zalloc(G);
    L->r1 = zalloc(G); L->r2 = zalloc(G); L->r3 = zalloc(G);
    L->b1 = zalloc(G); L->b2 = zalloc(G); L->b3 = zalloc(G);
    L->phik = zalloc(G);
    m /= 2; n /= 2; h *= 2.0;
  }
  ctx->phik = zalloc(p->m * p->n);
  ctx->phikm1 = zalloc(p->m * p->n);
  ctx->psik = zalloc(p->m * p->n);
  return ctx;
}

void orc_destroy(orc_ctx* ctx) {
  if (!ctx) return;
  for (int l = 0; l < ctx->nlev; ++l) {
    orc_level* L = &ctx->lev[l];
    free(L->phi); free(L->mu); free(L->kappa); free(L->S1); free(L->S2); free(L->S3);
    free(L->r1); free(L->r2); free(L->r3); free(L->b1); free(L->b2); free(L->b3); free(L->phik);
    free(L->W);
  }
  free(ctx->phik); free(ctx->phikm1); free(ctx->psik); free(ctx->phihat);
  free(ctx);
}

int orc_levels(const orc_ctx* ctx) { return ctx->nlev; }

/* Pinning of Sec. 4.6: weight W >= 0 and target phihat on the finest grid (copied);
 * coarse levels get the 2x2 averages of W.  weight NULL switches pinning off. */
void orc_set_pinning(orc_ctx* ctx, const double* weight, const double* target) {
  for (int l = 0; l < ctx->nlev; ++l) { free(ctx->lev[l].W); ctx->lev[l].W = NULL; }
  free(ctx->phihat);
  ctx->phihat = NULL;
  if (!weight) return;
  int G = ctx->p.m * ctx->p.n;
  ctx->phihat = zalloc(G);
  memcpy(ctx->phihat, target, sizeof(double) * G);
  ctx->lev[0].W = zalloc(G);
  memcpy(ctx->lev[0].W, weight, sizeof(double) * G);
  for (int l = 1; l < ctx->nlev; ++l) {
    ctx->lev[l].W = zalloc(ctx->lev[l].m * ctx->lev[l].n);
    orc_restrict(ctx->lev[l].m, ctx->lev[l].n, ctx->lev[l - 1].W, ctx->lev[l].W);
  }
}

static void level_residual(const orc_consts* k, orc_level* L) {
  int G = L->m * L->n;
  apply_N_w(k->scheme, k->c, k->gam, k->theta, L->m, L->n, L->h, L->phi, L->mu, L->kappa, L->phik, L->W,
            L->r1, L->r2, L->r3);
#pragma omp parallel for schedule(static) if (G >= ORC_OMP_CELLS)
  for (int i = 0; i < G; ++i) {
    L->r1[i] = L->S1[i] - L->r1[i];
    L->r2[i] = L->S2[i] - L->r2[i];
    L->r3[i] = L->S3[i] - L->r3[i];
  }
}

/* Scaled residual norm sqrt( sum_c sum_ij r_c^2 / (3 m n) ). */
static double scaled_norm(const orc_level* L) {
  int G = L->m * L->n;
  double acc = 0.0;
  for (int i = 0; i < G; ++i) acc += L->r1[i] * L->r1[i] + L->r2[i] * L->r2[i] + L->r3[i] * L->r3[i];
  return sqrt(acc / (3.0 * G));
}

/* One FAS V-cycle on level l (standard FAS, App. B; Trottenberg et al.):
 * pre-smooth, restrict u and the residual, tau-corrected coarse source,
 * recurse (or solve exactly on the coarsest level), correct with the
 * prolongated coarse change, post-smooth. */
static void vcycle(orc_ctx* ctx, const orc_consts* k, int l) {
  orc_level* F = &ctx->lev[l];
  const orc_params* p = &ctx->p;
  if (l == ctx->nlev - 1) {
    coarse_newton_w(k->scheme, k->c, k->gam, k->theta, F->m, F->n, F->h, F->phi, F->mu, F->kappa, F->S1,
                    F->S2, F->S3, F->phik, F->W);
    return;
  }
  orc_level* C = &ctx->lev[l + 1];
  int Gc = C->m * C->n;
  smooth_w(k->scheme, k->c, k->gam, k->theta, p->newton, k->omega, p->nu1, F->m, F->n, F->h, F->phi, F->mu, F->kappa,
           F->S1, F->S2, F->S3, F->phik, F->W);
  level_residual(k, F);
  orc_restrict(C->m, C->n, F->phi, C->phi);
  orc_restrict(C->m, C->n, F->mu, C->mu);
  orc_restrict(C->m, C->n, F->kappa, C->kappa);
  memcpy(C->b1, C->phi, sizeof(double) * Gc);
  memcpy(C->b2, C->mu, sizeof(double) * Gc);
  memcpy(C->b3, C->kappa, sizeof(double) * Gc);
  /* S_c = N_c(R u) + R r */
  apply_N_w(k->scheme, k->c, k->gam, k->theta, C->m, C->n, C->h, C->phi, C->mu, C->kappa, C->phik, C->W, C->S1,
            C->S2, C->S3);
  orc_restrict(C->m, C->n, F->r1, C->r1);
  orc_restrict(C->m, C->n, F->r2, C->r2);
  orc_restrict(C->m, C->n, F->r3, C->r3);
  for (int i = 0; i < Gc; ++i) {
    C->S1[i] += C->r1[i];
    C->S2[i] += C->r2[i];
    C->S3[i] += C->r3[i];
  }
  vcycle(ctx, k, l + 1);
  /* u_f += P (u_c - R u_f) */
  for (int i = 0; i < Gc; ++i) {
    C->b1[i] = C->phi[i] - C->b1[i];
    C->b2[i] = C->mu[i] - C->b2[i];
    C->b3[i] = C->kappa[i] - C->b3[i];
  }
  orc_prolong_add(C->m, C->n, C->b1, F->phi);
  orc_prolong_add(C->m, C->n, C->b2, F->mu);
  orc_prolong_add(C->m, C->n, C->b3, F->kappa);
  smooth_w(k->scheme, k->c, k->gam, k->theta, p->newton, k->omega, p->nu2, F->m, F->n, F->h, F->phi, F->mu, F->kappa,
           F->S1, F->S2, F->S3, F->phik, F->W);
}

/* ------------------------------------------------------------------------ */
/* Time stepping (Sec. 3.1, 3.2)                                            */
/* ------------------------------------------------------------------------ */
/* State (phi^k, phi^{k-1}, psi^k).  NULL phi_prev means phi^{-1} = phi^0 and
 * NULL psi means psi^0 = 0 (Sec. 3.2: the start-up rule). */
void orc_set_state(orc_ctx* ctx, const double* phi, const double* phi_prev, const double* psi) {
  int G = ctx->p.m * ctx->p.n;
  memcpy(ctx->phik, phi, sizeof(double) * G);
  memcpy(ctx->phikm1, phi_prev ? phi_prev : phi, sizeof(double) * G);
  if (psi) memcpy(ctx->psik, psi, sizeof(double) * G);
  else memset(ctx->psik, 0, sizeof(double) * G);
  ctx->step_index = 0;
}

void orc_get_state(const orc_ctx* ctx, double* phi, double* phi_prev, double* psi) {
  int G = ctx->p.m * ctx->p.n;
  if (phi) memcpy(phi, ctx->phik, sizeof(double) * G);
  if (phi_prev) memcpy(phi_prev, ctx->phikm1, sizeof(double) * G);
  if (psi) memcpy(psi, ctx->psik, sizeof(double) * G);
}

/* Copies out the finest-level unknowns u = (phi, mu, kappa) of the last solve. */
void orc_get_u(const orc_ctx* ctx, double* phi, double* mu, double* kappa) {
  const orc_level* L = &ctx->lev[0];
  int G = L->m * L->n;
  if (phi) memcpy(phi, L->phi, sizeof(double) * G);
  if (mu) memcpy(mu, L->mu, sizeof(double) * G);
  if (kappa) memcpy(kappa, L->kappa, sizeof(double) * G);
}

typedef struct {
  int cycles;
  int status;          /* 0 ok, 1 not converged, 2 diverged */
  double res0, res;
} orc_info;

/* Initial guess (the paper does not fix one):
 *   guess 0: phi0 = phi^k; guess 1: phi0 = 2 phi^k - phi^{k-1}; guess 2: phi0 given.
 * mu and kappa are then chosen so that N2 = S2 and N3 = S3 hold exactly:
 *   kappa0 = S3 + theta Delta_h phi0,  mu0 = S2 + g(phi0) + gam phi0 + Delta_h kappa0. */
static void initial_guess(orc_ctx* ctx, const orc_consts* k, int guess, const double* phi0_in) {
  orc_level* L = &ctx->lev[0];
  int G = L->m * L->n;

  double* lap = zalloc(G);
  for (int i = 0; i < G; ++i) {
    if (guess == 0) L->phi[i] = ctx->phik[i];
    else if (guess == 1) L->phi[i] = 2.0 * ctx->phik[i] - ctx->phikm1[i];
    else L->phi[i] = phi0_in[i];
  }
  orc_laplacian(L->m, L->n, L->h, L->phi, lap);
  for (int i = 0; i < G; ++i) L->kappa[i] = L->S3[i] + k->theta * lap[i];
  orc_laplacian(L->m, L->n, L->h, L->kappa, lap);
#pragma omp parallel for schedule(static) if (G >= ORC_OMP_CELLS)
  for (int i = 0; i < G; ++i) {
    double pk = (k->scheme == 2) ? L->phik[i] : 0.0;
    L->mu[i] = L->S2[i] + g_of(k->scheme, L->phi[i], pk) + k->gam * L->phi[i] + lap[i];
    if (L->W) L->mu[i] += L->W[i] * L->phi[i];
  }
  free(lap);
}

/* One time step of scheme 1 (Sec. 3.1) or scheme 2 (Sec. 3.2):
 * build S, solve N(u) = S by FAS V-cycles until the scaled residual is at or
 * below tol (or exactly fixed_cycles cycles when fixed_cycles > 0), then
 * psi^{k+1} = (phi - phi^k)/s (scheme 1, (3.9)) or
 * psi^{k+1} = (2/s)(phi - phi^k) - psi^k (scheme 2, (3.15)).
 * On failure the state is left unchanged.  res_hist (nullable) receives the
 * scaled residual after each cycle (max_cycles entries). */
int orc_step(orc_ctx* ctx, int scheme, int guess, const double* phi0_in, double tol, int max_cycles,
             int fixed_cycles, orc_info* info, double* res_hist) {
  const orc_params* p = &ctx->p;
  orc_consts k = consts_of(p, scheme);
  orc_level* L0 = &ctx->lev[0];
  int G = p->m * p->n;
  if ((scheme != 1 && scheme != 2) || guess < 0 || guess > 2 || (guess == 2 && !phi0_in)) return -1;
  if (L0->W && scheme != 2) return -1;   /* pinning is defined for the second-order scheme (Sec. 4.6) */
  source_w(scheme, p, ctx->phik, ctx->phikm1, ctx->psik, L0->W, ctx->phihat, L0->S1, L0->S2, L0->S3);
  memcpy(L0->phik, ctx->phik, sizeof(double) * G);
  for (int l = 1; l < ctx->nlev; ++l)
    orc_restrict(ctx->lev[l].m, ctx->lev[l].n, ctx->lev[l - 1].phik, ctx->lev[l].phik);
  initial_guess(ctx, &k, guess, phi0_in);
  level_residual(&k, L0);
  double res0 = scaled_norm(L0), res = res0;
  int cycles = 0, status = 0;
  int limit = fixed_cycles > 0 ? fixed_cycles : max_cycles;
  while (cycles < limit && (fixed_cycles > 0 || res > tol)) {
    vcycle(ctx, &k, 0);
    level_residual(&k, L0);
    res = scaled_norm(L0);
    if (res_hist) res_hist[cycles] = res;
    ++cycles;
    if (!(res == res) || isinf(res) || res > 1e10 * fmax(res0, tol)) { status = 2; break; }
  }
  if (status == 0 && fixed_cycles <= 0 && res > tol) status = 1;
  if (info) { info->cycles = cycles; info->status = status; info->res0 = res0; info->res = res; }
  if (status != 0) return status;
  for (int i = 0; i < G; ++i) {
    double phinew = L0->phi[i];
    /* MPFC: (3.9) / (3.15); PFC has no velocity unknown, psi keeps (phi^{k+1} - phi^k)/s */
    double psinew = (scheme == 1 || p->model == 1) ? (phinew - ctx->phik[i]) / p->s
                                                  : 2.0 / p->s * (phinew - ctx->phik[i]) - ctx->psik[i];
    ctx->psik[i] = psinew;
    ctx->phikm1[i] = ctx->phik[i];
    ctx->phik[i] = phinew;
  }
  ctx->step_index += 1;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Level-operator entry points (used by kernel-by-kernel parity tests)      */
/* ------------------------------------------------------------------------ */
/* Constants of N for a scheme: c, gam, theta (App. B.1 / B.2). */
void orc_scheme_consts(const orc_params* p, int scheme, double* c, double* gam, double* theta) {
  orc_consts k = consts_of(p, scheme);
  *c = k.c; *gam = k.gam; *theta = k.theta;
}

/* r = S - N(u) on one grid. */
void orc_residual(int scheme, double c, double gam, double theta, int m, int n, double h, const double* phi,
                  const double* mu, const double* kappa, const double* S1, const double* S2, const double* S3,
                  const double* phik, double* r1, double* r2, double* r3) {
  orc_apply_N(scheme, c, gam, theta, m, n, h, phi, mu, kappa, phik, r1, r2, r3);
  for (int i = 0; i < m * n; ++i) {
    r1[i] = S1[i] - r1[i];
    r2[i] = S2[i] - r2[i];
    r3[i] = S3[i] - r3[i];
  }
}

/* Runs V-cycles on a standalone problem N(u) = S on the finest grid of ctx,
 * starting from the given u (in/out) with the given S and phik.  Stops at
 * tol or after max_cycles.  Returns the number of cycles; *res_out gets the
 * final scaled residual. */
int orc_solve(orc_ctx* ctx, int scheme, double* phi, double* mu, double* kappa, const double* S1,
              const double* S2, const double* S3, const double* phik, double tol, int max_cycles,
              double* res_hist, double* res_out) {
  orc_consts k = consts_of(&ctx->p, scheme);
  orc_level* L0 = &ctx->lev[0];
  int G = L0->m * L0->n;
  memcpy(L0->phi, phi, sizeof(double) * G);
  memcpy(L0->mu, mu, sizeof(double) * G);
  memcpy(L0->kappa, kappa, sizeof(double) * G);
  memcpy(L0->S1, S1, sizeof(double) * G);
  memcpy(L0->S2, S2, sizeof(double) * G);
  memcpy(L0->S3, S3, sizeof(double) * G);
  if (phik) memcpy(L0->phik, phik, sizeof(double) * G);
  else memset(L0->phik, 0, sizeof(double) * G);
  for (int l = 1; l < ctx->nlev; ++l)
    orc_restrict(ctx->lev[l].m, ctx->lev[l].n, ctx->lev[l - 1].phik, ctx->lev[l].phik);
  level_residual(&k, L0);
  double res = scaled_norm(L0);
  int cycles = 0;
  while (cycles < max_cycles && res > tol) {
    vcycle(ctx, &k, 0);
    level_residual(&k, L0);
    res = scaled_norm(L0);
    if (res_hist) res_hist[cycles] = res;
    ++cycles;
  }
  memcpy(phi, L0->phi, sizeof(double) * G);
  memcpy(mu, L0->mu, sizeof(double) * G);
  memcpy(kappa, L0->kappa, sizeof(double) * G);
  if (res_out) *res_out = res;
  return cycles;
}

/* Level operators with a pinning weight W on the grid (Sec. 4.6), for the kernel
 * parity tests. */
void orc_apply_N_pinned(int scheme, double c, double gam, double theta, int m, int n, double h,
                        const double* phi, const double* mu, const double* kappa, const double* phik,
                        const double* W, double* N1, double* N2, double* N3) {
  apply_N_w(scheme, c, gam, theta, m, n, h, phi, mu, kappa, phik, W, N1, N2, N3);
}

void orc_smooth_pinned(int scheme, double c, double gam, double theta, int newton, double omega, int sweeps, int m,
                       int n, double h, double* phi, double* mu, double* kappa, const double* S1, const double* S2,
                       const double* S3, const double* phik, const double* W) {
  smooth_w(scheme, c, gam, theta, newton, omega, sweeps, m, n, h, phi, mu, kappa, S1, S2, S3, phik, W);
}

int orc_coarse_newton_pinned(int scheme, double c, double gam, double theta, int m, int n, double h,
                             double* phi, double* mu, double* kappa, const double* S1, const double* S2,
                             const double* S3, const double* phik, const double* W) {
  return coarse_newton_w(scheme, c, gam, theta, m, n, h, phi, mu, kappa, S1, S2, S3, phik, W);
}

void orc_source_pinned(int scheme, const orc_params* p, const double* phik, const double* phikm1,
                       const double* psik, const double* W, const double* phihat, double* S1, double* S2,
                       double* S3) {
  source_w(scheme, p, phik, phikm1, psik, W, phihat, S1, S2, S3);
}
