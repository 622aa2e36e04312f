/*
 * isis_oracle.c -- plain, slow FP64 CPU oracle for the ISIS scalar-field
 * multigrid solve (Llinares, Mota & Winther 2013, arXiv:1307.6748).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  The CUDA library never
 * links, includes or calls it, and it shares no code with it.
 *
 * Everything here is written from the paper's equations, in the paper's
 * order, with no blocking, fusion or reordering:
 *   - 7-point Laplacian ............................ Sect. 3.1, Eq. (disc_lap)
 *   - Poisson source (3/2) Om H0^2 delta / a ....... Sect. 1, Eq. (eqs_general_1)
 *   - FAS: L(phi) = Sigma, coarse Sigma ............ Sect. 3.2
 *   - implicit (Newton) Gauss-Seidel update ........ Sect. 3.2
 *   - canonical derivative dL/dphi ................. Sect. 3.3
 *   - non-canonical flux form, face b .............. Sect. 3.4, Eq. (disc_non_canonical)
 *   - non-canonical derivative ..................... Sect. 3.4, Eq. (dbeq)
 *   - symmetron equation ........................... Sect. 4.1, Eq. (symmetron_dimensionles)
 *   - Hu-Sawicki f(R) in u, f_R = -a^-2 e^u ........ Sect. 4.2
 *   - CIC density estimate ......................... Sect. 5.1
 *   - fifth forces ................................. Sect. 4.1 Eq. (symmetron_geodesics_tilde_chi),
 *                                                    Sect. 4.2 (f(R) geodesic)
 *
 * Readings where the paper is silent or garbled (each also listed in the
 * design notes):
 *   R1  restriction R = mean of the 8 children (cell-centred full weighting);
 *       prolongation P = cell-centred trilinear (3/4, 1/4 per axis).
 *   R2  coarse source Sigma_H = L_H(R phi_h) + R[Sigma_h - L_h(phi_h)]
 *       (Sect. 3.2's expression read with eps = L - Sigma).
 *   R3  FAS correction phi_h += P(phi_H - R phi_h).
 *   R4  Eq. (dbeq): the db/du terms carry a factor 1/2 (the exact derivative
 *       of the face average b_f = (b + b_nb)/2); Eq. (disc_non_canonical)
 *       is divided by h^2.
 *   R5  red cells ((i+j+k) even) first, then black; V(nu1,nu2) cycles;
 *       coarsest level solved by dense Newton with LU (partial pivoting),
 *       stop when max|dx| <= 1e-13 max(1, max|phi|), at most 50 steps.
 *   R6  convergence: RMS of L(phi) - Sigma on the finest grid <= tol * ref,
 *       ref = RMS of L(phi_bg) for the uniform background field phi_bg, in
 *       closed form (symmetron A s chi_bg RMS(eta-1); f(R) K1 RMS(eta-1);
 *       Poisson KP RMS(eta - <eta>)); ref = initial residual when that is 0.
 *   R7  Poisson gauge: the source uses eta - mean(eta); after every cycle
 *       the mean of Phi is removed; the coarsest Jacobian is
 *       J - (6/h^2)(1 1^T)/n and the Newton update is projected to zero mean.
 *   R8  CIC: cell centres at i+1/2 in cell units; weight 1-t to cell
 *       floor(x-1/2), t to the next, periodic wrap.
 *   R9  gradients: 2-point central differences at cells, interpolated to
 *       particles with the same CIC weights.
 *   R10 lengths in Mpc/h with c = 1, so H0 = 1/2997.92458 (Mpc/h)^-1.
 *
 * Grid: periodic N^3, cell (i,j,k) stored at (i*N + j)*N + k, h = box/N.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOCONV -2
#define ORC_ENAN -3
#define ORC_ENOMEM -5

enum { ORC_POISSON = 0, ORC_SYMMETRON = 1, ORC_FOFR = 2, ORC_CHAMELEON = 3 };

/* Problem description handed in from Python (ctypes mirror). */
typedef struct {
  int model;     /* ORC_POISSON, ORC_SYMMETRON, ORC_FOFR or ORC_CHAMELEON */
  int N;         /* finest grid size per dimension */
  double box;    /* box side in Mpc/h */
  double a;      /* expansion factor */
  double Omega_m, Omega_L, H0;
  double lambda0, beta, a_ssb; /* symmetron, Sect. 4.1 */
  int n;                       /* Hu-Sawicki exponent, Sect. 4.2 */
  double fR0_abs;              /* |f_R0| */
  double cham_n;               /* chameleon exponent (> -1), Sect. 6's chameleon equation */
} orc_problem;

typedef struct {
  int cycles;
  int coarse_newton_max; /* largest number of coarsest Newton steps seen */
  double res0, ref, res_final;
  double hist[256];
} orc_info;

/* Per-model constants of the source term. */
typedef struct {
  int model;
  double A, s;          /* symmetron: A = a^2/(2 lambda0^2), s = (a_SSB/a)^3 */
  double K1, K2, K3;    /* f(R): S(u) = K1(eta-1) - K2 e^{-u/(n+1)} + K3 */
  double np1;           /* n + 1 */
  double KP, eta_mean;  /* Poisson: S = KP (eta - mean eta) */
} orc_coef;

typedef struct {
  int N;
  double h;
  double *eta, *phi, *phi0, *sigma, *res; /* sigma == NULL on the finest level */
} orc_level;

static size_t IDX(int N, int i, int j, int k) {
  return ((size_t)i * N + j) * N + k;
}
static int WRAP(int i, int N) { return (i % N + N) % N; }

/* ------------------------------------------------------------------ */
/* Model source terms                                                  */
/* ------------------------------------------------------------------ */

static void make_coef(const orc_problem* p, const double* eta_fine, orc_coef* c) {
  memset(c, 0, sizeof(*c));
  c->model = p->model;
  double a = p->a, H02 = p->H0 * p->H0;
  if (p->model == ORC_SYMMETRON) {
    /* Eq. (symmetron_dimensionles): lap chi = a^2/(2 lambda0^2) [ (a_SSB/a)^3 eta chi - chi + chi^3 ] */
    c->A = a * a / (2.0 * p->lambda0 * p->lambda0);
    c->s = pow(p->a_ssb / a, 3.0);
  } else if (p->model == ORC_FOFR) {
    /* Sect. 4.2, the equation for u (f_R = -a^-2 e^u, b = e^u):
       div(e^u grad u) = Om a H0^2 (eta - 1)
                         - Om a^4 H0^2 (1 + 4 OL/Om) (|fR0| a^2)^{1/(n+1)} e^{-u/(n+1)}
                         + Om a H0^2 (1 + 4 a^3 OL/Om)                                  */
    double r = p->Omega_L / p->Omega_m;
    c->np1 = p->n + 1.0;
    c->K1 = p->Omega_m * a * H02;
    c->K2 = p->Omega_m * pow(a, 4.0) * H02 * (1.0 + 4.0 * r) * pow(p->fR0_abs * a * a, 1.0 / c->np1);
    c->K3 = p->Omega_m * a * H02 * (1.0 + 4.0 * a * a * a * r);
  } else if (p->model == ORC_CHAMELEON) {
    /* The chameleon equation of Sect. 6, lap phi = -M^{4+n} phi^{-(1+n)} + beta rho / M_pl, taken as a
       free source S (Sect. 2) in comoving units (lap -> a^2 lap) with rho = rho_m0 a^-3 eta and
       phi = phi_0 psi, phi_0 the minimum at a = 1, eta = 1:
           lap psi = A_c [a^-3 eta - psi^{-(1+n)}],  A_c = a^2 / ((1+n) lambda0^2),
       lambda0 the range (inverse mass) of the field in the background today.  In u = ln psi,
       lap psi = div(e^u grad u): the non-canonical operator of Sect. 3.4 with b = e^u and
           S(u) = K1 (eta - 1) - K2 e^{-u/np1} + K3,  K1 = K3 = A_c a^-3, K2 = A_c, np1 = 1/(1+n),
       the form of the Hu-Sawicki source, so every f(R) step below serves it unchanged. */
    double Ac = a * a / ((1.0 + p->cham_n) * p->lambda0 * p->lambda0);
    c->model = ORC_FOFR;
    c->np1 = 1.0 / (1.0 + p->cham_n);
    c->K1 = Ac / (a * a * a);
    c->K2 = Ac;
    c->K3 = c->K1;
  } else {
    /* Sect. 3.1: lap Phi = (3/2) Om H0^2 delta / a, delta = eta - 1 with its mean removed (R7) */
    c->KP = 1.5 * p->Omega_m * H02 / a;
    if (eta_fine) { /* a refinement patch passes NULL and sets the domain mean itself */
      double sum = 0.0;
      size_t n3 = (size_t)p->N * p->N * p->N;
      for (size_t q = 0; q < n3; ++q) sum += eta_fine[q];
      c->eta_mean = sum / (double)n3;
    }
  }
}

/* S(phi, eta) and dS/dphi for the canonical models, written so that
   L = lap(phi) - S (Sect. 3.2). */
static double source(const orc_coef* c, double phi, double eta) {
  if (c->model == ORC_SYMMETRON) return c->A * ((c->s * eta - 1.0) * phi + phi * phi * phi);
  if (c->model == ORC_FOFR) return c->K1 * (eta - 1.0) - c->K2 * exp(-phi / c->np1) + c->K3;
  return c->KP * (eta - c->eta_mean);
}
static double dsource(const orc_coef* c, double phi, double eta) {
  if (c->model == ORC_SYMMETRON) return c->A * (c->s * eta - 1.0 + 3.0 * phi * phi);
  if (c->model == ORC_FOFR) return c->K2 / c->np1 * exp(-phi / c->np1);
  (void)eta;
  return 0.0;
}

/* ------------------------------------------------------------------ */
/* Discrete operator L and its diagonal derivative                     */
/* ------------------------------------------------------------------ */

static const int DI[6] = {+1, -1, 0, 0, 0, 0};
static const int DJ[6] = {0, 0, +1, -1, 0, 0};
static const int DK[6] = {0, 0, 0, 0, +1, -1};

static double nbval(const double* f, int N, int i, int j, int k, int d) {
  return f[IDX(N, WRAP(i + DI[d], N), WRAP(j + DJ[d], N), WRAP(k + DK[d], N))];
}

/* L(phi) at cell (i,j,k). */
static double op_L(const orc_coef* c, const orc_level* L, const double* phi, int i, int j, int k) {
  int N = L->N;
  double h2 = L->h * L->h;
  double u = phi[IDX(N, i, j, k)];
  double eta = L->eta[IDX(N, i, j, k)];
  if (c->model == ORC_FOFR) {
    /* Eq. (disc_non_canonical) / h^2 with b = e^u and face values from Sect. 3.4 */
    double bu = exp(u), div = 0.0;
    for (int d = 0; d < 6; ++d) {
      double un = nbval(phi, N, i, j, k, d);
      double bf = 0.5 * (bu + exp(un));
      div += bf * (un - u);
    }
    return div / h2 - source(c, u, eta);
  }
  /* Eq. (disc_lap) */
  double sum = 0.0;
  for (int d = 0; d < 6; ++d) sum += nbval(phi, N, i, j, k, d);
  return (sum - 6.0 * u) / h2 - source(c, u, eta);
}

/* dL/dphi at cell (i,j,k) (Sect. 3.3 for the canonical models, Eq. (dbeq) with R4 for f(R)). */
static double op_dL(const orc_coef* c, const orc_level* L, const double* phi, int i, int j, int k) {
  int N = L->N;
  double h2 = L->h * L->h;
  double u = phi[IDX(N, i, j, k)];
  double eta = L->eta[IDX(N, i, j, k)];
  if (c->model == ORC_FOFR) {
    double bu = exp(u), acc = 0.0;
    for (int d = 0; d < 6; ++d) {
      double un = nbval(phi, N, i, j, k, d);
      double bf = 0.5 * (bu + exp(un));
      acc += -bf + 0.5 * bu * (un - u);
    }
    return acc / h2 - dsource(c, u, eta);
  }
  return -6.0 / h2 - dsource(c, u, eta);
}

/* ------------------------------------------------------------------ */
/* Smoother, residual, transfers                                       */
/* ------------------------------------------------------------------ */

/* One red-black Newton-Gauss-Seidel sweep (Sect. 3.2):
   phi <- phi - (L(phi) - Sigma) / (dL/dphi), red cells first. */
static void smooth(const orc_coef* c, orc_level* L) {
  int N = L->N;
  for (int color = 0; color < 2; ++color) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j)
        for (int k = 0; k < N; ++k) {
          if (((i + j + k) & 1) != color) continue;
          size_t q = IDX(N, i, j, k);
          double sig = L->sigma ? L->sigma[q] : 0.0;
          double F = op_L(c, L, L->phi, i, j, k) - sig;
          double dF = op_dL(c, L, L->phi, i, j, k);
          L->phi[q] = L->phi[q] - F / dF;
        }
  }
}

/* res = Sigma - L(phi) */
static void residual(const orc_coef* c, orc_level* L) {
  int N = L->N;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j)
      for (int k = 0; k < N; ++k) {
        size_t q = IDX(N, i, j, k);
        double sig = L->sigma ? L->sigma[q] : 0.0;
        L->res[q] = sig - op_L(c, L, L->phi, i, j, k);
      }
}

/* R1: coarse value = mean of its 8 children. */
static void restrict_mean(int NH, const double* fine, double* coarse) {
  int Nf = 2 * NH;
#pragma omp parallel for schedule(static)
  for (int I = 0; I < NH; ++I)
    for (int J = 0; J < NH; ++J)
      for (int K = 0; K < NH; ++K) {
        double s = 0.0;
        for (int di = 0; di < 2; ++di)
          for (int dj = 0; dj < 2; ++dj)
            for (int dk = 0; dk < 2; ++dk) s += fine[IDX(Nf, 2 * I + di, 2 * J + dj, 2 * K + dk)];
        coarse[IDX(NH, I, J, K)] = s / 8.0;
      }
}

/* R1: cell-centred trilinear interpolation, fine += P(coarse_delta).
   The fine cell 2I+d sits at coarse coordinate I + 1/4 (d=0) or I + 3/4
   (d=1): weight 3/4 on coarse I and 1/4 on I-1 (d=0) or I+1 (d=1). */
static void prolong_add(int NH, const double* cdelta, double* fine) {
  int Nf = 2 * NH;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < Nf; ++i)
    for (int j = 0; j < Nf; ++j)
      for (int k = 0; k < Nf; ++k) {
        int ci[2], cj[2], ck[2];
        double wi[2] = {0.75, 0.25}, wj[2] = {0.75, 0.25}, wk[2] = {0.75, 0.25};
        ci[0] = i / 2; ci[1] = WRAP(i / 2 + ((i & 1) ? 1 : -1), NH);
        cj[0] = j / 2; cj[1] = WRAP(j / 2 + ((j & 1) ? 1 : -1), NH);
        ck[0] = k / 2; ck[1] = WRAP(k / 2 + ((k & 1) ? 1 : -1), NH);
        double v = 0.0;
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b)
            for (int d = 0; d < 2; ++d) v += wi[a] * wj[b] * wk[d] * cdelta[IDX(NH, ci[a], cj[b], ck[d])];
        fine[IDX(Nf, i, j, k)] += v;
      }
}

/* RMS of (L(phi) - Sigma) over a level; deterministic (plane partial sums
   added in plane order).  Returns NaN if any value is not finite. */
static double rms_residual(const orc_coef* c, orc_level* L) {
  int N = L->N;
  double* part = (double*)calloc((size_t)N, sizeof(double));
#pragma omp parallel for schedule(static)
  for (int i = 0; i < N; ++i) {
    double s = 0.0;
    for (int j = 0; j < N; ++j)
      for (int k = 0; k < N; ++k) {
        size_t q = IDX(N, i, j, k);
        double sig = L->sigma ? L->sigma[q] : 0.0;
        double F = op_L(c, L, L->phi, i, j, k) - sig;
        s += F * F;
      }
    part[i] = s;
  }
  double tot = 0.0;
  for (int i = 0; i < N; ++i) tot += part[i];
  free(part);
  return sqrt(tot / ((double)N * N * N));
}

/* ------------------------------------------------------------------ */
/* Coarsest level: dense Newton with the exact Jacobian (R5)           */
/* ------------------------------------------------------------------ */

/* LU with partial pivoting (first maximum on ties), then solve A x = b.
   A is n x n row-major and is overwritten.  Returns 0, or -1 if singular. */
static int lu_solve(int n, double* A, double* b) {
  for (int kk = 0; kk < n; ++kk) {
    int piv = kk;
    double best = fabs(A[(size_t)kk * n + kk]);
    for (int r = kk + 1; r < n; ++r)
      if (fabs(A[(size_t)r * n + kk]) > best) { best = fabs(A[(size_t)r * n + kk]); piv = r; }
    if (!(best > 0.0)) return -1;
    if (piv != kk) {
      for (int cc = 0; cc < n; ++cc) {
        double t = A[(size_t)kk * n + cc]; A[(size_t)kk * n + cc] = A[(size_t)piv * n + cc]; A[(size_t)piv * n + cc] = t;
      }
      double t = b[kk]; b[kk] = b[piv]; b[piv] = t;
    }
    for (int r = kk + 1; r < n; ++r) {
      double m = A[(size_t)r * n + kk] / A[(size_t)kk * n + kk];
      A[(size_t)r * n + kk] = m;
      for (int cc = kk + 1; cc < n; ++cc) A[(size_t)r * n + cc] -= m * A[(size_t)kk * n + cc];
      b[r] -= m * b[kk];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = b[r];
    for (int cc = r + 1; cc < n; ++cc) s -= A[(size_t)r * n + cc] * b[cc];
    b[r] = s / A[(size_t)r * n + r];
  }
  return 0;
}

/* Exact Jacobian of F(phi) = L(phi) - Sigma on the level (dense, n x n). */
static void jacobian(const orc_coef* c, const orc_level* L, double* J) {
  int N = L->N, n = N * N * N;
  double h2 = L->h * L->h;
  memset(J, 0, sizeof(double) * (size_t)n * n);
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j)
      for (int k = 0; k < N; ++k) {
        size_t row = IDX(N, i, j, k);
        double u = L->phi[row], eta = L->eta[row];
        if (c->model == ORC_FOFR) {
          double bu = exp(u);
          double diag = -dsource(c, u, eta);
          for (int d = 0; d < 6; ++d) {
            size_t col = IDX(N, WRAP(i + DI[d], N), WRAP(j + DJ[d], N), WRAP(k + DK[d], N));
            double un = L->phi[col], bn = exp(un);
            double bf = 0.5 * (bu + bn);
            diag += (-bf + 0.5 * bu * (un - u)) / h2;
            J[row * n + col] += (bf + 0.5 * bn * (un - u)) / h2;
          }
          J[row * n + row] += diag;
        } else {
          J[row * n + row] += -6.0 / h2 - dsource(c, u, eta);
          for (int d = 0; d < 6; ++d) {
            size_t col = IDX(N, WRAP(i + DI[d], N), WRAP(j + DJ[d], N), WRAP(k + DK[d], N));
            J[row * n + col] += 1.0 / h2;
          }
        }
      }
  if (c->model == ORC_POISSON) {
    /* R7: remove the null space of the periodic Laplacian */
    double shift = 6.0 / h2 / (double)n;
    for (size_t q = 0; q < (size_t)n * n; ++q) J[q] -= shift;
  }
}

static int coarse_newton(const orc_coef* c, orc_level* L, int* steps) {
  int N = L->N, n = N * N * N;
  double* J = (double*)malloc(sizeof(double) * (size_t)n * n);
  double* F = (double*)malloc(sizeof(double) * (size_t)n);
  if (!J || !F) { free(J); free(F); return ORC_ENOMEM; }
  /* ENOCONV unless a step meets the stop rule within 50 steps */
  int st = ORC_ENOCONV, it;
  for (it = 0; it < 50; ++it) {
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j)
        for (int k = 0; k < N; ++k) {
          size_t q = IDX(N, i, j, k);
          F[q] = -(op_L(c, L, L->phi, i, j, k) - L->sigma[q]);
        }
    jacobian(c, L, J);
    if (lu_solve(n, J, F) != 0) { st = ORC_ENAN; break; }
    if (c->model == ORC_POISSON) {
      double m = 0.0;
      for (int q = 0; q < n; ++q) m += F[q];
      m /= (double)n;
      for (int q = 0; q < n; ++q) F[q] -= m;
    }
    double dmax = 0.0, pmax = 0.0;
    for (int q = 0; q < n; ++q) {
      L->phi[q] += F[q];
      if (fabs(F[q]) > dmax) dmax = fabs(F[q]);
      if (fabs(L->phi[q]) > pmax) pmax = fabs(L->phi[q]);
    }
    if (!isfinite(dmax)) { st = ORC_ENAN; break; }
    if (dmax <= 1e-13 * (pmax > 1.0 ? pmax : 1.0)) { st = ORC_OK; ++it; break; }
  }
  if (steps) *steps = it;
  free(J);
  free(F);
  return st;
}

/* ------------------------------------------------------------------ */
/* FAS V-cycle (Sect. 3.2)                                             */
/* ------------------------------------------------------------------ */

typedef struct {
  orc_coef coef;
  int nlev;
  orc_level lev[16];
  int nu1, nu2;
  int coarse_steps_max;
} orc_hier;

static int vcycle(orc_hier* H, int l) {
  orc_level* L = &H->lev[l];
  if (l == H->nlev - 1) {
    int steps = 0;
    int st = coarse_newton(&H->coef, L, &steps);
    if (steps > H->coarse_steps_max) H->coarse_steps_max = steps;
    return st;
  }
  orc_level* C = &H->lev[l + 1];
  size_t nc = (size_t)C->N * C->N * C->N;
  for (int s = 0; s < H->nu1; ++s) smooth(&H->coef, L);
  /* R2: Sigma_H = L_H(R phi) + R[Sigma - L(phi)] */
  residual(&H->coef, L);
  restrict_mean(C->N, L->phi, C->phi);
  memcpy(C->phi0, C->phi, nc * sizeof(double));
  restrict_mean(C->N, L->res, C->sigma);
  for (int i = 0; i < C->N; ++i)
    for (int j = 0; j < C->N; ++j)
      for (int k = 0; k < C->N; ++k) C->sigma[IDX(C->N, i, j, k)] += op_L(&H->coef, C, C->phi, i, j, k);
  int st = vcycle(H, l + 1);
  if (st != ORC_OK) return st;
  /* R3: phi_h += P(phi_H - R phi_h) */
  for (size_t q = 0; q < nc; ++q) C->phi0[q] = C->phi[q] - C->phi0[q];
  prolong_add(C->N, C->phi0, L->phi);
  for (int s = 0; s < H->nu2; ++s) smooth(&H->coef, L);
  return ORC_OK;
}

static void remove_mean(int N, double* f) {
  size_t n3 = (size_t)N * N * N;
  double s = 0.0;
  for (size_t q = 0; q < n3; ++q) s += f[q];
  s /= (double)n3;
  for (size_t q = 0; q < n3; ++q) f[q] -= s;
}

static void free_hier(orc_hier* H) {
  for (int l = 0; l < H->nlev; ++l) {
    if (l > 0) { free(H->lev[l].eta); free(H->lev[l].phi); free(H->lev[l].sigma); }
    free(H->lev[l].phi0);
    free(H->lev[l].res);
  }
}

/* Build the level hierarchy: the finest level aliases eta/phi. */
static int build_hier(orc_hier* H, const orc_problem* p, double* eta, double* phi, int nu1, int nu2, int ncoarse) {
  memset(H, 0, sizeof(*H));
  make_coef(p, eta, &H->coef);
  H->nu1 = nu1;
  H->nu2 = nu2;
  int N = p->N, l = 0;
  while (1) {
    orc_level* L = &H->lev[l];
    size_t n3 = (size_t)N * N * N;
    L->N = N;
    L->h = p->box / N;
    if (l == 0) { L->eta = eta; L->phi = phi; L->sigma = NULL; }
    else {
      L->eta = (double*)malloc(n3 * sizeof(double));
      L->phi = (double*)malloc(n3 * sizeof(double));
      L->sigma = (double*)calloc(n3, sizeof(double));
      if (!L->eta || !L->phi || !L->sigma) { H->nlev = l + 1; free_hier(H); return ORC_ENOMEM; }
      restrict_mean(N, H->lev[l - 1].eta, L->eta);
    }
    L->phi0 = (double*)malloc(n3 * sizeof(double));
    L->res = (double*)malloc(n3 * sizeof(double));
    ++l;
    H->nlev = l;
    if (!L->phi0 || !L->res) { free_hier(H); return ORC_ENOMEM; }
    if (N <= ncoarse || N % 2 != 0 || l == 16) break;
    N /= 2;
  }
  return ORC_OK;
}

/* Background field of R6 and the reference residual. */
static double background(const orc_problem* p, const orc_coef* c) {
  if (p->model == ORC_SYMMETRON) {
    double v = 1.0 - c->s;
    return v > 0.0 ? sqrt(v) : 0.0;
  }
  if (c->model == ORC_FOFR) {
    /* uniform eta = 1 root of S(u) = 0: e^{u/(n+1)} = K2/K3 */
    return c->np1 * log(c->K2 / c->K3);
  }
  return 0.0;
}

static int valid(const orc_problem* p) {
  if (p->N < 2 || (p->N & (p->N - 1)) != 0) return 0;
  if (!(p->a > 0.0) || !(p->box > 0.0)) return 0;
  if (p->model < 0 || p->model > 3) return 0;
  if (p->model == ORC_CHAMELEON && (!(p->lambda0 > 0.0) || !(p->cham_n > -1.0) || !(p->cham_n <= 8.0))) return 0;
  if (p->model == ORC_SYMMETRON && !(p->lambda0 > 0.0)) return 0;
  if (p->model == ORC_FOFR && (!(p->fR0_abs > 0.0) || p->n < 1)) return 0;
  return 1;
}

/* Full FAS solve (Sect. 3.2) from the guess in phi (overwritten). */
int orc_solve(const orc_problem* p, const double* eta_in, double* phi, double tol, int nu1, int nu2, int ncoarse,
              int max_cycles, orc_info* info) {
  if (!valid(p) || ncoarse < 2 || max_cycles < 0 || max_cycles > 256) return ORC_EINVAL;
  size_t n3 = (size_t)p->N * p->N * p->N;
  double* eta = (double*)malloc(n3 * sizeof(double));
  if (!eta) return ORC_ENOMEM;
  memcpy(eta, eta_in, n3 * sizeof(double));
  orc_hier H;
  int st = build_hier(&H, p, eta, phi, nu1, nu2, ncoarse);
  if (st != ORC_OK) { free(eta); return st; }
  memset(info, 0, sizeof(*info));

  /* R6: reference residual = RMS of L(phi_bg), the background field's
     residual, in closed form: for a uniform field the Laplacian vanishes and
     S(phi_bg, eta) - S(phi_bg, eta_ref) is the coefficient times (eta - eta_ref). */
  {
    double eref = (p->model == ORC_POISSON) ? H.coef.eta_mean : 1.0;
    double sum2 = 0.0;
    for (size_t q = 0; q < n3; ++q) sum2 += (eta[q] - eref) * (eta[q] - eref);
    double scale;
    if (p->model == ORC_SYMMETRON) scale = H.coef.A * H.coef.s * background(p, &H.coef);
    else if (H.coef.model == ORC_FOFR) scale = H.coef.K1;
    else scale = H.coef.KP;
    info->ref = scale * sqrt(sum2 / (double)n3);
  }

  double res = rms_residual(&H.coef, &H.lev[0]);
  info->res0 = res;
  if (!(info->ref > 0.0)) info->ref = res; /* uniform density: relative to the initial residual */
  double target = tol * info->ref;
  info->res_final = res;
  if (!isfinite(res)) st = ORC_ENAN;
  else if (res <= target) st = ORC_OK;
  else {
    st = ORC_ENOCONV;
    for (int cyc = 0; cyc < max_cycles; ++cyc) {
      int vs = vcycle(&H, 0);
      if (p->model == ORC_POISSON) remove_mean(p->N, phi);
      res = rms_residual(&H.coef, &H.lev[0]);
      info->hist[cyc] = res;
      info->cycles = cyc + 1;
      info->res_final = res;
      if (vs != ORC_OK) { st = vs; break; }
      if (!isfinite(res)) { st = ORC_ENAN; break; }
      if (res <= target) { st = ORC_OK; break; }
    }
  }
  info->coarse_newton_max = H.coarse_steps_max;
  free_hier(&H);
  free(eta);
  return st;
}

/* ------------------------------------------------------------------ */
/* Exposed pieces for unit pins                                        */
/* ------------------------------------------------------------------ */

/* out = L(phi) - Sigma on one grid of size p->N (sigma may be NULL). */
int orc_residual(const orc_problem* p, const double* eta, const double* phi, const double* sigma, double* out) {
  if (!valid(p)) return ORC_EINVAL;
  orc_coef c;
  make_coef(p, eta, &c);
  orc_level L = {p->N, p->box / p->N, (double*)eta, (double*)phi, NULL, (double*)sigma, NULL};
  int N = p->N;
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j)
      for (int k = 0; k < N; ++k)
        out[IDX(N, i, j, k)] = op_L(&c, &L, phi, i, j, k) - (sigma ? sigma[IDX(N, i, j, k)] : 0.0);
  return ORC_OK;
}

/* out = dL/dphi (diagonal) on one grid. */
int orc_dL(const orc_problem* p, const double* eta, const double* phi, double* out) {
  if (!valid(p)) return ORC_EINVAL;
  orc_coef c;
  make_coef(p, eta, &c);
  orc_level L = {p->N, p->box / p->N, (double*)eta, (double*)phi, NULL, NULL, NULL};
  int N = p->N;
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j)
      for (int k = 0; k < N; ++k) out[IDX(N, i, j, k)] = op_dL(&c, &L, phi, i, j, k);
  return ORC_OK;
}

/* One red-black sweep in place (sigma may be NULL). */
int orc_smooth(const orc_problem* p, const double* eta, double* phi, const double* sigma) {
  if (!valid(p)) return ORC_EINVAL;
  orc_coef c;
  make_coef(p, eta, &c);
  orc_level L = {p->N, p->box / p->N, (double*)eta, phi, NULL, (double*)sigma, NULL};
  smooth(&c, &L);
  return ORC_OK;
}

void orc_restrict(int NH, const double* fine, double* coarse) { restrict_mean(NH, fine, coarse); }
void orc_prolong_add(int NH, const double* cdelta, double* fine) { prolong_add(NH, cdelta, fine); }

/* The dense Jacobian of the coarsest solve, dF_r/dphi_c (row-major n x n, n = N^3), at phi; for pins.
   Poisson's carries the shift -(6/h^2)/n in every entry that removes the periodic Laplacian's null space. */
int orc_jacobian(const orc_problem* p, const double* eta, const double* phi, double* J) {
  if (!valid(p)) return ORC_EINVAL;
  orc_coef c;
  make_coef(p, eta, &c);
  orc_level L = {p->N, p->box / p->N, (double*)eta, (double*)phi, NULL, NULL, NULL};
  jacobian(&c, &L, J);
  return ORC_OK;
}

/* RMS of L(phi) - Sigma over one grid, the norm of the convergence test; for pins. */
double orc_rms_residual(const orc_problem* p, const double* eta, const double* phi, const double* sigma) {
  if (!valid(p)) return NAN;
  orc_coef c;
  make_coef(p, eta, &c);
  orc_level L = {p->N, p->box / p->N, (double*)eta, (double*)phi, NULL, (double*)sigma, NULL};
  return rms_residual(&c, &L);
}

/* Dense-Newton solve of L(phi) = Sigma on one (small) grid; for pins. */
int orc_dense_newton(const orc_problem* p, const double* eta, double* phi, const double* sigma, int* steps) {
  if (!valid(p)) return ORC_EINVAL;
  size_t n3 = (size_t)p->N * p->N * p->N;
  orc_coef c;
  make_coef(p, eta, &c);
  double* sg = (double*)calloc(n3, sizeof(double));
  if (sigma) memcpy(sg, sigma, n3 * sizeof(double));
  orc_level L = {p->N, p->box / p->N, (double*)eta, phi, NULL, sg, NULL};
  int st = coarse_newton(&c, &L, steps);
  free(sg);
  return st;
}

/* ------------------------------------------------------------------ */
/* CIC density estimate (Sect. 5.1) and forces (Sects. 4.1, 4.2)      */
/* ------------------------------------------------------------------ */

/* R8: the two cells and weights along one axis for a coordinate x in cell units. */
static void cic_axis(double x, int N, int* i0, int* i1, double* w0, double* w1) {
  double xs = x - 0.5;
  double f = floor(xs);
  double t = xs - f;
  *i0 = WRAP((int)f, N);
  *i1 = WRAP((int)f + 1, N);
  *w0 = 1.0 - t;
  *w1 = t;
}

/* eta = (sum of CIC weights) / nbar, nbar = npart / N^3. Positions in cell units. */
int orc_cic_deposit(int N, int64_t np, const float* x, const float* y, const float* z, double* eta) {
  if (N < 1 || np < 1) return ORC_EINVAL;
  size_t n3 = (size_t)N * N * N;
  memset(eta, 0, n3 * sizeof(double));
  for (int64_t q = 0; q < np; ++q) {
    int ix[2], iy[2], iz[2];
    double wx[2], wy[2], wz[2];
    cic_axis(x[q], N, &ix[0], &ix[1], &wx[0], &wx[1]);
    cic_axis(y[q], N, &iy[0], &iy[1], &wy[0], &wy[1]);
    cic_axis(z[q], N, &iz[0], &iz[1], &wz[0], &wz[1]);
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b)
        for (int d = 0; d < 2; ++d) eta[IDX(N, ix[a], iy[b], iz[d])] += wx[a] * wy[b] * wz[d];
  }
  double nbar = (double)np / (double)n3;
  for (size_t q = 0; q < n3; ++q) eta[q] /= nbar;
  return ORC_OK;
}

/* Central-difference gradient of f at every cell (R9): g[3][N^3]. */
int orc_gradient(int N, double box, const double* f, double* gx, double* gy, double* gz) {
  double h = box / N;
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j)
      for (int k = 0; k < N; ++k) {
        size_t q = IDX(N, i, j, k);
        gx[q] = (f[IDX(N, WRAP(i + 1, N), j, k)] - f[IDX(N, WRAP(i - 1, N), j, k)]) / (2.0 * h);
        gy[q] = (f[IDX(N, i, WRAP(j + 1, N), k)] - f[IDX(N, i, WRAP(j - 1, N), k)]) / (2.0 * h);
        gz[q] = (f[IDX(N, i, j, WRAP(k + 1, N))] - f[IDX(N, i, j, WRAP(k - 1, N))]) / (2.0 * h);
      }
  return ORC_OK;
}

/* Acceleration d^2x/dtau^2 at each particle (super-comoving units):
     g = -[ grad Phi~ + F5 ],  Phi~ = a^2 Phi,
     symmetron F5 = 6 Om H0^2 (beta lambda0)^2 / a_SSB^3 chi~ grad chi~, chi~ = a chi
                    (Eq. (symmetron_geodesics_tilde_chi)),
     f(R)      F5 = (1/2) e^u grad u (Sect. 4.2).
   Phi and/or phi may be NULL to leave that term out.  Grid values of the
   force are formed at the cells, then CIC-interpolated (R9). */
int orc_fifth_force(const orc_problem* p, const double* Phi, const double* phi, int64_t np, const float* x,
                    const float* y, const float* z, double* gx, double* gy, double* gz) {
  if (!valid(p)) return ORC_EINVAL;
  int N = p->N;
  size_t n3 = (size_t)N * N * N;
  double h = p->box / N, a = p->a;
  double* f[3];
  for (int d = 0; d < 3; ++d) f[d] = (double*)calloc(n3, sizeof(double));
  double* g[3];
  for (int d = 0; d < 3; ++d) g[d] = (double*)malloc(n3 * sizeof(double));
  if (Phi) {
    orc_gradient(N, p->box, Phi, g[0], g[1], g[2]);
    for (int d = 0; d < 3; ++d)
      for (size_t q = 0; q < n3; ++q) f[d][q] += a * a * g[d][q];
  }
  if (phi && p->model != ORC_POISSON) {
    orc_gradient(N, p->box, phi, g[0], g[1], g[2]);
    double Cs = 6.0 * p->Omega_m * p->H0 * p->H0 * pow(p->beta * p->lambda0, 2.0) / pow(p->a_ssb, 3.0);
    /* chameleon: beta phi_0 / M_pl = 3 (1+n) beta^2 Om H0^2 lambda0^2, from the mass of the field at the
       background minimum today, m0^2 = (1+n) beta rho_m0 / (M_pl phi_0) = 1/lambda0^2, rho_m0 = 3 Om H0^2 M_pl^2 */
    double Cc = 3.0 * (1.0 + p->cham_n) * pow(p->beta, 2.0) * p->Omega_m * p->H0 * p->H0 * pow(p->lambda0, 2.0);
    for (size_t q = 0; q < n3; ++q) {
      double pref;
      if (p->model == ORC_SYMMETRON) pref = Cs * (a * phi[q]) * a; /* chi~ grad chi~ = a chi * a grad chi */
      else if (p->model == ORC_CHAMELEON) pref = a * a * Cc * exp(phi[q]); /* a^2 grad ln A, ln A = beta phi / M_pl */
      else pref = 0.5 * exp(phi[q]);
      for (int d = 0; d < 3; ++d) f[d][q] += pref * g[d][q];
    }
  }
  (void)h;
  for (int64_t q = 0; q < np; ++q) {
    int ix[2], iy[2], iz[2];
    double wx[2], wy[2], wz[2];
    cic_axis(x[q], N, &ix[0], &ix[1], &wx[0], &wx[1]);
    cic_axis(y[q], N, &iy[0], &iy[1], &wy[0], &wy[1]);
    cic_axis(z[q], N, &iz[0], &iz[1], &wz[0], &wz[1]);
    double acc[3] = {0, 0, 0};
    for (int aa = 0; aa < 2; ++aa)
      for (int b = 0; b < 2; ++b)
        for (int d = 0; d < 2; ++d) {
          double w = wx[aa] * wy[b] * wz[d];
          size_t c = IDX(N, ix[aa], iy[b], iz[d]);
          for (int e = 0; e < 3; ++e) acc[e] += w * f[e][c];
        }
    gx[q] = -acc[0];
    gy[q] = -acc[1];
    gz[q] = -acc[2];
  }
  for (int d = 0; d < 3; ++d) { free(f[d]); free(g[d]); }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Refinement patches: masks and ghost values (Sect. 3.3.1, 3.4.1)     */
/* ------------------------------------------------------------------ */
/*
 * A patch is a box of n[0] x n[1] x n[2] cells of its parent grid, origin o[],
 * refined by two: its finest level has 2n cells per axis and h = h_parent / 2
 * = box / (N 2^level).  flags[] (one per parent cell of the box, same order)
 * marks the refined parent cells, whose 8 children exist.  Readings:
 *   P1 mask: children of flagged cells m = +1, the others m = -1 (they do not
 *      exist); every coarser level of the patch's multigrid takes m = R(m)
 *      (Sect. 3.4.1), except its outer layer of cells, which stays m = -1 (it
 *      lies outside the box's refined part; flags on the box's outer layer of
 *      parent cells must be 0, which makes this hold on the finest level too).
 *      Cells with m > 0 are the unknowns; the others keep their values.
 *   P2 the cells that do not exist on the finest level hold u^Int, the
 *      cell-centred trilinear interpolation (R1's P) of the parent field;
 *      coarser levels take all values from R (full-approximation restriction).
 *   P3 the ghost value of a neighbour nb with m_nb <= 0 of an unknown c is
 *      Eq. (ueq): u^G = u_nb + (m_nb / m_c)(u_c - u_c^Pre), where u_nb is the
 *      neighbour's value (u^Int or its value before the iterations) and
 *      u_c^Pre the value of c when the smoothing phase (nu sweeps) began.
 *      Residuals take u^Pre = u, so u^G = u_nb.  f(R): b^G = e^{u^G} and
 *      c^G = db/du = e^{u^G} (the consistent choice of Sect. 3.4.1).
 *   P4 dL/du_c gains, for every masked neighbour, the derivative through u^G
 *      (Sect. 3.4.1): (m_nb/m_c)/h^2 (canonical), (m_nb/m_c)[(c^G/2)(u^G - u_c)
 *      + b_f]/h^2 (f(R), with the factor 1/2 of the face mean as in R4).
 *   P5 FAS on the patch levels: the residual (zero off the unknowns) and u are
 *      restricted with R; Sigma_H = L_H(R u) + R r at the coarse unknowns; the
 *      correction P(u_H - R u) is added at the fine unknowns, with a zero
 *      correction for coarse cells outside the box.
 *   P6 levels: halve while every dimension is even and the smallest is >= 8;
 *      the coarsest level gets 16 red-black sweeps (the paper is silent; the
 *      patch V-cycles converge at the same rate with 8, 16 or 64).
 *   P7 convergence: RMS of L(u) - Sigma over the finest unknowns <= tol * ref,
 *      ref = R6's closed form over the same cells.
 */

typedef struct {
  int n[3];         /* patch box in parent cells */
  int o[3];         /* its origin in parent cells */
  int pn[3];        /* parent grid dimensions */
  int periodic;     /* 1: the parent is the periodic domain grid */
  int level;        /* refinement level >= 1 of the patch */
  double eta_mean;  /* Poisson: the domain's mean density */
} orc_patch;

typedef struct {
  int n[3];
  double h;
  double *m, *eta, *u, *u0, *sig, *res, *pre;
} orc_plevel;

typedef struct {
  orc_coef coef;
  int nlev;
  orc_plevel lev[16];
  int nu1, nu2;
} orc_phier;

static size_t PIDX(const int* n, int i, int j, int k) { return ((size_t)i * n[1] + j) * n[2] + k; }
static size_t PSIZE(const int* n) { return (size_t)n[0] * n[1] * n[2]; }

/* P3: value of neighbour d seen by the unknown q, and its mask ratio (0 for an unknown). */
static double patch_nb(const orc_plevel* L, size_t q, int i, int j, int k, int d, double* mu) {
  size_t qn = PIDX(L->n, i + DI[d], j + DJ[d], k + DK[d]);
  double mn = L->m[qn];
  if (mn > 0.0) { *mu = 0.0; return L->u[qn]; }
  *mu = mn / L->m[q];
  return L->u[qn] + (*mu) * (L->u[q] - L->pre[q]);
}

/* L(u) at the unknown (i,j,k) (Eq. (gen_lap) in its general form, Eq. (disc_non_canonical)) and
   dL/du (Sect. 3.3, Eq. (dbeq) with R4, plus P4). */
static void patch_op(const orc_coef* c, const orc_plevel* L, int i, int j, int k, double* Lv, double* dL) {
  size_t q = PIDX(L->n, i, j, k);
  double h2 = L->h * L->h, u = L->u[q], eta = L->eta[q];
  double acc = 0.0, dacc = 0.0;
  if (c->model == ORC_FOFR) {
    double bu = exp(u);
    for (int d = 0; d < 6; ++d) {
      double mu, un = patch_nb(L, q, i, j, k, d, &mu);
      double bn = exp(un), bf = 0.5 * (bu + bn);
      acc += bf * (un - u);
      dacc += -bf + 0.5 * bu * (un - u);
      dacc += mu * (0.5 * bn * (un - u) + bf);
    }
  } else {
    for (int d = 0; d < 6; ++d) {
      double mu, un = patch_nb(L, q, i, j, k, d, &mu);
      acc += un;
      dacc += mu;
    }
    acc -= 6.0 * u;
    dacc -= 6.0;
  }
  *Lv = acc / h2 - source(c, u, eta);
  *dL = dacc / h2 - dsource(c, u, eta);
}

/* One red-black Newton-Gauss-Seidel sweep over the unknowns (Sect. 3.2). */
static void patch_sweep(const orc_coef* c, orc_plevel* L) {
  for (int color = 0; color < 2; ++color) {
#pragma omp parallel for schedule(static)
    for (int i = 1; i < L->n[0] - 1; ++i)
      for (int j = 1; j < L->n[1] - 1; ++j)
        for (int k = 1; k < L->n[2] - 1; ++k) {
          if (((i + j + k) & 1) != color) continue;
          size_t q = PIDX(L->n, i, j, k);
          if (!(L->m[q] > 0.0)) continue;
          double Lv, dL;
          patch_op(c, L, i, j, k, &Lv, &dL);
          double sig = L->sig ? L->sig[q] : 0.0;
          L->u[q] = L->u[q] - (Lv - sig) / dL;
        }
  }
}

/* A smoothing phase: u^Pre fixed at its start (P3), then nsweep sweeps. */
static void patch_phase(const orc_coef* c, orc_plevel* L, int nsweep) {
  memcpy(L->pre, L->u, PSIZE(L->n) * sizeof(double));
  for (int s = 0; s < nsweep; ++s) patch_sweep(c, L);
}

/* res = Sigma - L(u) at the unknowns, 0 elsewhere (u^Pre = u). */
static void patch_residual(const orc_coef* c, orc_plevel* L) {
  memcpy(L->pre, L->u, PSIZE(L->n) * sizeof(double));
  size_t n3 = PSIZE(L->n);
  memset(L->res, 0, n3 * sizeof(double));
#pragma omp parallel for schedule(static)
  for (int i = 1; i < L->n[0] - 1; ++i)
    for (int j = 1; j < L->n[1] - 1; ++j)
      for (int k = 1; k < L->n[2] - 1; ++k) {
        size_t q = PIDX(L->n, i, j, k);
        if (!(L->m[q] > 0.0)) continue;
        double Lv, dL;
        patch_op(c, L, i, j, k, &Lv, &dL);
        L->res[q] = (L->sig ? L->sig[q] : 0.0) - Lv;
      }
}

/* P7: RMS of the residual over the unknowns, and their number. */
static double patch_rms(const orc_coef* c, orc_plevel* L, size_t* count) {
  patch_residual(c, L);
  double s = 0.0;
  size_t cnt = 0, n3 = PSIZE(L->n);
  for (size_t q = 0; q < n3; ++q)
    if (L->m[q] > 0.0) { s += L->res[q] * L->res[q]; ++cnt; }
  if (count) *count = cnt;
  return cnt ? sqrt(s / (double)cnt) : 0.0;
}

/* R1 on a box: coarse = mean of the 8 children. */
static void patch_restrict(const int* nc, const double* fine, double* coarse) {
  int nf[3] = {2 * nc[0], 2 * nc[1], 2 * nc[2]};
  for (int I = 0; I < nc[0]; ++I)
    for (int J = 0; J < nc[1]; ++J)
      for (int K = 0; K < nc[2]; ++K) {
        double s = 0.0;
        for (int di = 0; di < 2; ++di)
          for (int dj = 0; dj < 2; ++dj)
            for (int dk = 0; dk < 2; ++dk) s += fine[PIDX(nf, 2 * I + di, 2 * J + dj, 2 * K + dk)];
        coarse[PIDX(nc, I, J, K)] = s / 8.0;
      }
}

/* P5: fine unknowns += P(cdelta), coarse cells outside the box contributing 0. */
static void patch_prolong_add(const orc_plevel* C, const double* cdelta, orc_plevel* L) {
  for (int i = 0; i < L->n[0]; ++i)
    for (int j = 0; j < L->n[1]; ++j)
      for (int k = 0; k < L->n[2]; ++k) {
        size_t q = PIDX(L->n, i, j, k);
        if (!(L->m[q] > 0.0)) continue;
        int ci[2] = {i / 2, i / 2 + ((i & 1) ? 1 : -1)};
        int cj[2] = {j / 2, j / 2 + ((j & 1) ? 1 : -1)};
        int ck[2] = {k / 2, k / 2 + ((k & 1) ? 1 : -1)};
        double w[2] = {0.75, 0.25}, v = 0.0;
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b)
            for (int d = 0; d < 2; ++d) {
              if (ci[a] < 0 || ci[a] >= C->n[0] || cj[b] < 0 || cj[b] >= C->n[1] || ck[d] < 0 || ck[d] >= C->n[2])
                continue;
              v += w[a] * w[b] * w[d] * cdelta[PIDX(C->n, ci[a], cj[b], ck[d])];
            }
        L->u[q] += v;
      }
}

/* P2: u^Int of every cell of the finest patch level from the parent field. */
static void patch_interp(const orc_patch* P, const double* parent, const int* nf, double* out) {
  for (int i = 0; i < nf[0]; ++i)
    for (int j = 0; j < nf[1]; ++j)
      for (int k = 0; k < nf[2]; ++k) {
        int f[3] = {i, j, k}, pc[3][2];
        for (int a = 0; a < 3; ++a) {
          pc[a][0] = P->o[a] + f[a] / 2;
          pc[a][1] = pc[a][0] + ((f[a] & 1) ? 1 : -1);
          if (P->periodic) { pc[a][0] = WRAP(pc[a][0], P->pn[a]); pc[a][1] = WRAP(pc[a][1], P->pn[a]); }
        }
        double w[2] = {0.75, 0.25}, v = 0.0;
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b)
            for (int d = 0; d < 2; ++d) v += w[a] * w[b] * w[d] * parent[PIDX(P->pn, pc[0][a], pc[1][b], pc[2][d])];
        out[PIDX(nf, i, j, k)] = v;
      }
}

static void patch_vcycle(orc_phier* H, int l) {
  orc_plevel* L = &H->lev[l];
  if (l == H->nlev - 1) { patch_phase(&H->coef, L, 16); return; }
  orc_plevel* C = &H->lev[l + 1];
  size_t nc = PSIZE(C->n);
  patch_phase(&H->coef, L, H->nu1);
  patch_residual(&H->coef, L);
  patch_restrict(C->n, L->u, C->u);
  memcpy(C->u0, C->u, nc * sizeof(double));
  patch_restrict(C->n, L->res, C->sig);
  memcpy(C->pre, C->u, nc * sizeof(double));
  for (int i = 1; i < C->n[0] - 1; ++i)
    for (int j = 1; j < C->n[1] - 1; ++j)
      for (int k = 1; k < C->n[2] - 1; ++k) {
        size_t q = PIDX(C->n, i, j, k);
        if (!(C->m[q] > 0.0)) continue;
        double Lv, dL;
        patch_op(&H->coef, C, i, j, k, &Lv, &dL);
        C->sig[q] += Lv;
      }
  patch_vcycle(H, l + 1);
  for (size_t q = 0; q < nc; ++q) C->u0[q] = C->u[q] - C->u0[q];
  patch_prolong_add(C, C->u0, L);
  patch_phase(&H->coef, L, H->nu2);
}

static void free_phier(orc_phier* H) {
  for (int l = 0; l < H->nlev; ++l) {
    orc_plevel* L = &H->lev[l];
    free(L->m); free(L->eta); free(L->u0); free(L->res); free(L->pre);
    if (l > 0) { free(L->u); free(L->sig); }
  }
}

static int patch_valid(const orc_problem* p, const orc_patch* P, const uint8_t* flags) {
  if (!valid(p) || P->level < 1 || P->level > 12) return 0;
  for (int a = 0; a < 3; ++a) {
    if (P->n[a] < 4 || (P->n[a] & 1) || P->pn[a] < 1) return 0;
    if (P->periodic) {
      if (P->pn[a] != p->N || P->n[a] > P->pn[a]) return 0;
    } else if (P->o[a] < 1 || P->o[a] + P->n[a] + 1 > P->pn[a]) {
      return 0;
    }
  }
  for (int i = 0; i < P->n[0]; ++i)
    for (int j = 0; j < P->n[1]; ++j)
      for (int k = 0; k < P->n[2]; ++k) {
        int edge = i == 0 || j == 0 || k == 0 || i == P->n[0] - 1 || j == P->n[1] - 1 || k == P->n[2] - 1;
        if (edge && flags[PIDX(P->n, i, j, k)]) return 0;
      }
  return 1;
}

/* Solve the patch (Sect. 3.3.1, 3.4.1; P1-P7).  parent: the parent field (P->pn dims); flags: refined
   parent cells of the box; eta: density of the finest patch level (2n dims); u: the finest patch level,
   in: the guess at the unknowns when init == 0 (init == 1: start from u^Int), out: the solution (cells
   that are not unknowns hold u^Int). */
int orc_patch_solve(const orc_problem* p, const orc_patch* P, const double* parent, const uint8_t* flags,
                    const double* eta, double* u, double tol, int nu1, int nu2, int max_cycles, int init,
                    orc_info* info) {
  if (!patch_valid(p, P, flags) || max_cycles < 0 || max_cycles > 256 || nu1 < 0 || nu2 < 0) return ORC_EINVAL;
  orc_phier H;
  memset(&H, 0, sizeof(H));
  make_coef(p, NULL, &H.coef);
  H.coef.eta_mean = P->eta_mean;
  H.nu1 = nu1;
  H.nu2 = nu2;
  int n[3] = {2 * P->n[0], 2 * P->n[1], 2 * P->n[2]};
  double h = p->box / ((double)p->N * (double)(1 << P->level));
  for (int l = 0;; ++l) {
    orc_plevel* L = &H.lev[l];
    size_t n3 = PSIZE(n);
    memcpy(L->n, n, sizeof(n));
    L->h = h;
    L->m = (double*)malloc(n3 * sizeof(double));
    L->eta = (double*)malloc(n3 * sizeof(double));
    L->u0 = (double*)malloc(n3 * sizeof(double));
    L->res = (double*)malloc(n3 * sizeof(double));
    L->pre = (double*)malloc(n3 * sizeof(double));
    if (l == 0) { L->u = u; L->sig = NULL; }
    else { L->u = (double*)malloc(n3 * sizeof(double)); L->sig = (double*)calloc(n3, sizeof(double)); }
    H.nlev = l + 1;
    if (!L->m || !L->eta || !L->u0 || !L->res || !L->pre || !L->u || (l > 0 && !L->sig)) {
      free_phier(&H);
      return ORC_ENOMEM;
    }
    if (l == 0) {
      /* P1 */
      for (int i = 0; i < n[0]; ++i)
        for (int j = 0; j < n[1]; ++j)
          for (int k = 0; k < n[2]; ++k)
            L->m[PIDX(n, i, j, k)] = flags[PIDX(P->n, i / 2, j / 2, k / 2)] ? 1.0 : -1.0;
      memcpy(L->eta, eta, n3 * sizeof(double));
    } else {
      patch_restrict(n, H.lev[l - 1].m, L->m);
      patch_restrict(n, H.lev[l - 1].eta, L->eta);
      for (int i = 0; i < n[0]; ++i)
        for (int j = 0; j < n[1]; ++j)
          for (int k = 0; k < n[2]; ++k)
            if (i == 0 || j == 0 || k == 0 || i == n[0] - 1 || j == n[1] - 1 || k == n[2] - 1)
              L->m[PIDX(n, i, j, k)] = -1.0;
    }
    int mn = n[0] < n[1] ? n[0] : n[1];
    if (n[2] < mn) mn = n[2];
    if ((n[0] & 1) || (n[1] & 1) || (n[2] & 1) || mn < 8 || l == 15) break;
    n[0] /= 2; n[1] /= 2; n[2] /= 2;
    h *= 2.0;
  }
  orc_plevel* F = &H.lev[0];
  size_t nf3 = PSIZE(F->n);
  /* P2: u^Int where the cells do not exist (and everywhere for init == 1) */
  patch_interp(P, parent, F->n, F->u0);
  for (size_t q = 0; q < nf3; ++q)
    if (init == 1 || !(F->m[q] > 0.0)) u[q] = F->u0[q];
  memset(info, 0, sizeof(*info));
  /* P7: R6's reference over the unknowns */
  {
    double eref = (p->model == ORC_POISSON) ? P->eta_mean : 1.0, s2 = 0.0;
    size_t cnt = 0;
    for (size_t q = 0; q < nf3; ++q)
      if (F->m[q] > 0.0) { s2 += (eta[q] - eref) * (eta[q] - eref); ++cnt; }
    double scale;
    if (p->model == ORC_SYMMETRON) scale = H.coef.A * H.coef.s * background(p, &H.coef);
    else if (H.coef.model == ORC_FOFR) scale = H.coef.K1;
    else scale = H.coef.KP;
    info->ref = cnt ? scale * sqrt(s2 / (double)cnt) : 0.0;
  }
  size_t cnt = 0;
  double res = patch_rms(&H.coef, F, &cnt);
  info->res0 = res;
  if (!(info->ref > 0.0)) info->ref = res;
  info->res_final = res;
  int st;
  if (cnt == 0 || res <= tol * info->ref) st = ORC_OK;
  else if (!isfinite(res)) st = ORC_ENAN;
  else {
    st = ORC_ENOCONV;
    for (int cyc = 0; cyc < max_cycles; ++cyc) {
      patch_vcycle(&H, 0);
      res = patch_rms(&H.coef, F, NULL);
      info->hist[cyc] = res;
      info->cycles = cyc + 1;
      info->res_final = res;
      if (!isfinite(res)) { st = ORC_ENAN; break; }
      if (res <= tol * info->ref) { st = ORC_OK; break; }
    }
  }
  free_phier(&H);
  return st;
}

/* For pins: L(u) - Sigma and dL/du at the unknowns of one patch level with mask m (0 elsewhere), u^Pre =
   pre.  Cells with m > 0 must not lie on the outer layer of the box. */
int orc_patch_eval(const orc_problem* p, const int* n, double h, const double* m, const double* eta,
                   const double* u, const double* pre, const double* sig, double eta_mean, double* F, double* dF) {
  if (!valid(p)) return ORC_EINVAL;
  orc_coef c;
  make_coef(p, NULL, &c);
  c.eta_mean = eta_mean;
  orc_plevel L;
  memset(&L, 0, sizeof(L));
  memcpy(L.n, n, 3 * sizeof(int));
  L.h = h;
  L.m = (double*)m; L.eta = (double*)eta; L.u = (double*)u; L.pre = (double*)pre; L.sig = (double*)sig;
  size_t n3 = PSIZE(n);
  for (size_t q = 0; q < n3; ++q) { F[q] = 0.0; dF[q] = 0.0; }
  for (int i = 0; i < n[0]; ++i)
    for (int j = 0; j < n[1]; ++j)
      for (int k = 0; k < n[2]; ++k) {
        size_t q = PIDX(n, i, j, k);
        if (!(m[q] > 0.0)) continue;
        if (i == 0 || j == 0 || k == 0 || i == n[0] - 1 || j == n[1] - 1 || k == n[2] - 1) return ORC_EINVAL;
        double Lv, dL;
        patch_op(&c, &L, i, j, k, &Lv, &dL);
        F[q] = Lv - (sig ? sig[q] : 0.0);
        dF[q] = dL;
      }
  return ORC_OK;
}

/* fine += P(cdelta) at the fine cells with m > 0 of a patch level (P5), coarse cells outside the box
   contributing 0; nc: coarse dims (the fine level has 2 nc).  Exposed for the pins. */
int orc_patch_prolong_add(const int* nc, const double* cdelta, const double* m_fine, double* fine) {
  if (nc[0] < 1 || nc[1] < 1 || nc[2] < 1) return ORC_EINVAL;
  orc_plevel C, L;
  memset(&C, 0, sizeof(C));
  memset(&L, 0, sizeof(L));
  for (int a = 0; a < 3; ++a) {
    C.n[a] = nc[a];
    L.n[a] = 2 * nc[a];
  }
  L.m = (double*)m_fine;
  L.u = fine;
  patch_prolong_add(&C, cdelta, &L);
  return ORC_OK;
}
