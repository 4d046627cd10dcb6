/*
 * CPU FP64 oracle for the geometric-multigrid-preconditioned CG solve of
 * -div(k grad phi) = f (Eq. 2) on a vertex-centred structured grid of the
 * unit cube with zero Dirichlet boundary values.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU library computes.  Only the test suite, the
 * package smoke check and the benchmark's CPU-baseline leg load it.  It
 * shares no code, header or table with the CUDA library.
 *
 * Everything is IEEE binary64, compiled with -ffp-contract=off so that no
 * fused multiply-add changes the rounding.  The operator is an assembled CSR
 * matrix on every level; restriction, prolongation, smoother and Krylov
 * recurrences are plain loops; the coarsest level is a dense Cholesky
 * factorisation.  Loops over rows run under OpenMP (each row is independent,
 * so the result does not depend on the thread count); every dot product is a
 * sequential sum in index order.
 *
 * Passages followed (section / equation / algorithm of the paper):
 *   operator              Eq. 1 (Ax = b) with A from Eq. 2, a 7-point
 *                         finite-difference stencil (Sec. 4.1, "Disc. A": at
 *                         most 7 non-zeros per row); the variable-coefficient
 *                         face rule is this library's reading (harmonic mean
 *                         of the 4 cells sharing an edge)
 *   coarse operators      re-discretised on every level (Sec. 1, Sec. 4.3)
 *   two-level cycle       Algorithm 1, applied recursively (V-cycle, Fig. 1)
 *   level components      Sec. 2.1.1 (operator, smoother, R, P, coarse LU)
 *   smoother              Chebyshev preconditioned with Jacobi (Sec. 4.3)
 *   coarse solve          exact factorisation of the coarsest operator
 *                         (Sec. 1; Sec. 3.3.1)
 *   outer Krylov method   CG (Sec. 2.1), stopped when the residual 2-norm is
 *                         reduced by a factor rtol (Sec. 4.2, Sec. 4.3)
 *
 * Layout of every array passed in or out: full vertex grid including the
 * boundary, C order [z][y][x] with x fastest.  Cells are (Nz-1)(Ny-1)(Nx-1),
 * indexed by their lower corner.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_LEVELS 24
#define ORC_MAX_COARSE 4096

typedef struct {
  int Nx, Ny, Nz;      /* vertices per axis, boundary included */
  int nx, ny, nz;      /* interior unknowns per axis */
  long n;              /* nx*ny*nz */
  double hx, hy, hz;   /* grid spacing, unit cube */
  double *kc;          /* cell conductivity */
  long *rowptr;        /* CSR over interior unknowns */
  int *col;
  double *val;
  double *diag;
  double *b, *x, *r, *s, *d, *t; /* work vectors (interior numbering) */
  int face_rule;
  double alpha, beta;  /* Chebyshev interval for D^-1 A on this level */
  int sum_order;       /* 0: every sum in index order; 1: the second fixed order
                          (pairwise dot products, CSR rows summed from the last
                          stored entry to the first) */
} olevel;

typedef struct {
  int L;
  olevel lv[ORC_MAX_LEVELS];
  int nu_pre, nu_post, degree;
  double alpha, beta;  /* Chebyshev interval for D^-1 A */
  int smoother;        /* 0 Chebyshev-Jacobi, 1 Richardson-Jacobi */
  double omega;        /* Richardson damping */
  int nc;              /* unknowns on the coarsest level */
  int coarse_rule;     /* 0 arithmetic, 1 geometric, 2 harmonic mean of children */
  int face_rule;       /* edge k: 0 harmonic, 1 arithmetic mean of the 4 cells */
  int galerkin;        /* coarse operators: 0 re-discretised, 1 Galerkin R A P */
  int eig_mode;        /* Chebyshev interval: 0 fixed / Gershgorin, 1 Lanczos estimate */
  int coarse_mode;     /* coarsest solve: 0 Cholesky, 1 GMRES with Jacobi to coarse_rtol */
  double coarse_rtol;
  int coarse_maxit;
  double *Ac, *Lc;     /* dense coarsest operator and its Cholesky factor */
} ohier;

/* ---------------------------------------------------------------- indexing */
static inline long uidx(const olevel *L, int i, int j, int k) {
  return ((long)k * L->ny + j) * L->nx + i; /* interior coordinates */
}
static inline long fidx(const olevel *L, int I, int J, int K) {
  return ((long)K * L->Ny + J) * L->Nx + I; /* full-grid coordinates */
}
static inline double kcell(const olevel *L, int ci, int cj, int ck) {
  return L->kc[((long)ck * (L->Ny - 1) + cj) * (L->Nx - 1) + ci];
}
static inline int interior(const olevel *L, int I, int J, int K) {
  return I >= 1 && I <= L->Nx - 2 && J >= 1 && J <= L->Ny - 2 && K >= 1 && K <= L->Nz - 2;
}

/* Edge coefficient: mean of the four cells that share the edge leaving
 * full-grid node (I,J,K) in the +axis direction (axis 0 = x, 1 = y, 2 = z).
 * Harmonic mean 4 / sum(1/k_c) by default; arithmetic mean sum(k_c)/4 when
 * the level was built with the arithmetic face rule. */
static double kedge(const olevel *L, int axis, int I, int J, int K) {
  double s = 0.0, t = 0.0;
  for (int a = -1; a <= 0; ++a)
    for (int b = -1; b <= 0; ++b) {
      double kc;
      if (axis == 0) kc = kcell(L, I, J + a, K + b);
      else if (axis == 1) kc = kcell(L, I + a, J, K + b);
      else kc = kcell(L, I + a, J + b, K);
      s += 1.0 / kc;
      t += kc;
    }
  return L->face_rule ? t / 4.0 : 4.0 / s;
}

static void to_interior(const olevel *L, const double *full, double *u) {
#pragma omp parallel for schedule(static)
  for (int k = 0; k < L->nz; ++k)
    for (int j = 0; j < L->ny; ++j)
      for (int i = 0; i < L->nx; ++i) u[uidx(L, i, j, k)] = full[fidx(L, i + 1, j + 1, k + 1)];
}

static void to_full(const olevel *L, const double *u, double *full) {
  long N = (long)L->Nx * L->Ny * L->Nz;
  memset(full, 0, sizeof(double) * N);
#pragma omp parallel for schedule(static)
  for (int k = 0; k < L->nz; ++k)
    for (int j = 0; j < L->ny; ++j)
      for (int i = 0; i < L->nx; ++i) full[fidx(L, i + 1, j + 1, k + 1)] = u[uidx(L, i, j, k)];
}

/* ------------------------------------------------------------ assembly */
/* Row p of A: (A x)_p = sum over the 6 neighbours q of h_a^-2 k_pq (x_p - x_q),
 * with x_q = 0 on the Dirichlet boundary.  Entries in increasing column order. */
static int assemble(olevel *L) {
  long n = L->n;
  L->rowptr = (long *)malloc(sizeof(long) * (n + 1));
  L->col = (int *)malloc(sizeof(int) * n * 7);
  L->val = (double *)malloc(sizeof(double) * n * 7);
  L->diag = (double *)malloc(sizeof(double) * n);
  if (!L->rowptr || !L->col || !L->val || !L->diag) return -1;
  const double ih2[3] = {1.0 / (L->hx * L->hx), 1.0 / (L->hy * L->hy), 1.0 / (L->hz * L->hz)};
  /* Each row has up to 7 entries; rows are laid out with stride 7 first and
   * compacted afterwards so the row loop can run in parallel. */
  int *cnt = (int *)malloc(sizeof(int) * n);
#pragma omp parallel for schedule(static)
  for (int k = 0; k < L->nz; ++k)
    for (int j = 0; j < L->ny; ++j)
      for (int i = 0; i < L->nx; ++i) {
        long p = uidx(L, i, j, k);
        int I = i + 1, J = j + 1, K = k + 1;
        /* neighbour offsets in increasing column order: -z,-y,-x,+x,+y,+z */
        const int off[6][3] = {{0, 0, -1}, {0, -1, 0}, {-1, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
        const int ax[6] = {2, 1, 0, 0, 1, 2};
        double c[6], dsum = 0.0;
        for (int e = 0; e < 6; ++e) {
          int a = ax[e];
          int lo = off[e][a] < 0; /* edge goes from the neighbour to p */
          int EI = lo ? I + off[e][0] : I, EJ = lo ? J + off[e][1] : J, EK = lo ? K + off[e][2] : K;
          c[e] = ih2[a] * kedge(L, a, EI, EJ, EK);
          dsum += c[e];
        }
        long base = p * 7;
        int m = 0;
        for (int e = 0; e < 3; ++e) {
          int QI = I + off[e][0], QJ = J + off[e][1], QK = K + off[e][2];
          if (interior(L, QI, QJ, QK)) {
            L->col[base + m] = (int)uidx(L, QI - 1, QJ - 1, QK - 1);
            L->val[base + m] = -c[e];
            ++m;
          }
        }
        L->col[base + m] = (int)p;
        L->val[base + m] = dsum;
        ++m;
        for (int e = 3; e < 6; ++e) {
          int QI = I + off[e][0], QJ = J + off[e][1], QK = K + off[e][2];
          if (interior(L, QI, QJ, QK)) {
            L->col[base + m] = (int)uidx(L, QI - 1, QJ - 1, QK - 1);
            L->val[base + m] = -c[e];
            ++m;
          }
        }
        cnt[p] = m;
        L->diag[p] = dsum;
      }
  L->rowptr[0] = 0;
  for (long p = 0; p < n; ++p) L->rowptr[p + 1] = L->rowptr[p] + cnt[p];
  /* compact in place: rows only move towards lower addresses */
  for (long p = 0; p < n; ++p) {
    long src = p * 7, dst = L->rowptr[p];
    for (int m = 0; m < cnt[p]; ++m) {
      L->col[dst + m] = L->col[src + m];
      L->val[dst + m] = L->val[src + m];
    }
  }
  free(cnt);
  return 0;
}

/* y = A x.  Each row is summed in increasing column order, or (second
 * summation order) in decreasing column order. */
static void spmv(const olevel *L, const double *x, double *y) {
  if (L->sum_order == 1) {
#pragma omp parallel for schedule(static)
    for (long p = 0; p < L->n; ++p) {
      double s = 0.0;
      for (long q = L->rowptr[p + 1] - 1; q >= L->rowptr[p]; --q) s += L->val[q] * x[L->col[q]];
      y[p] = s;
    }
    return;
  }
#pragma omp parallel for schedule(static)
  for (long p = 0; p < L->n; ++p) {
    double s = 0.0;
    for (long q = L->rowptr[p]; q < L->rowptr[p + 1]; ++q) s += L->val[q] * x[L->col[q]];
    y[p] = s;
  }
}

/* Pairwise (cascade) sum of a[i] b[i]: halves summed recursively, runs of at
 * most 8 products summed in index order.  Its rounding error is bounded by
 * about (log2(n) + 8) u sum |a_i b_i| instead of the n u of the sequential
 * sum; used only as the second summation order. */
static double dot_pairwise(long n, const double *a, const double *b) {
  if (n <= 8) {
    double s = 0.0;
    for (long i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
  }
  const long h = n / 2;
  return dot_pairwise(h, a, b) + dot_pairwise(n - h, a + h, b + h);
}

/* a . b over n entries: a sequential sum in index order, or the pairwise sum
 * when the level runs the second summation order. */
static double dot(const olevel *L, long n, const double *a, const double *b) {
  if (L->sum_order == 1) return dot_pairwise(n, a, b);
  double s = 0.0;
  for (long i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* ------------------------------------------------------------ transfers */
/* Full weighting R = P^T / 8: per axis weights (1/4, 1/2, 1/4) around the
 * fine node coincident with the coarse node; all 27 fine nodes are interior. */
static void restrict_fw(const olevel *F, const olevel *C, const double *rf, double *bc) {
  static const double w[3] = {0.25, 0.5, 0.25};
#pragma omp parallel for schedule(static)
  for (int k = 0; k < C->nz; ++k)
    for (int j = 0; j < C->ny; ++j)
      for (int i = 0; i < C->nx; ++i) {
        /* coarse interior (i,j,k) is fine interior (2i+1, 2j+1, 2k+1) */
        double s = 0.0;
        for (int c = -1; c <= 1; ++c)
          for (int b = -1; b <= 1; ++b)
            for (int a = -1; a <= 1; ++a)
              s += w[a + 1] * w[b + 1] * w[c + 1] * rf[uidx(F, 2 * i + 1 + a, 2 * j + 1 + b, 2 * k + 1 + c)];
        bc[uidx(C, i, j, k)] = s;
      }
}

/* Trilinear interpolation P: along each axis a fine node with even full
 * coordinate coincides with a coarse node (weight 1); an odd one takes half of
 * each of its two coarse neighbours.  Coarse boundary values are zero. */
static double pw(int F, int Cc) {
  int d = F - 2 * Cc;
  return d == 0 ? 1.0 : (d == 1 || d == -1) ? 0.5 : 0.0;
}
static void prolong_add(const olevel *F, const olevel *C, const double *ec, double *xf) {
#pragma omp parallel for schedule(static)
  for (int k = 0; k < F->nz; ++k)
    for (int j = 0; j < F->ny; ++j)
      for (int i = 0; i < F->nx; ++i) {
        int I = i + 1, J = j + 1, K = k + 1; /* fine full coordinates */
        double s = 0.0;
        for (int CK = K / 2; CK <= (K + 1) / 2; ++CK)
          for (int CJ = J / 2; CJ <= (J + 1) / 2; ++CJ)
            for (int CI = I / 2; CI <= (I + 1) / 2; ++CI) {
              if (!interior(C, CI, CJ, CK)) continue;
              double wgt = pw(I, CI) * pw(J, CJ) * pw(K, CK);
              if (wgt != 0.0) s += wgt * ec[uidx(C, CI - 1, CJ - 1, CK - 1)];
            }
        xf[uidx(F, i, j, k)] += s;
      }
}

/* ------------------------------------------------------------ Galerkin */
/* Galerkin coarse operator A_c = R A_f P with R = P^T / 8 (the paper's runs
 * use Galerkin coarse operators, Sec. 4.3 and Sec. 5), entry by entry from
 * the definition (A_c)_IJ = sum_{i,j} R_Ii (A_f)_ij P_jJ: for each coarse row
 * I, the 27 fine rows i of R's stencil, each stored entry a_ij of fine row i,
 * and the coarse interior nodes J that interpolate to fine node j.  J - I
 * lies in {-1,0,1}^3, so rows have at most 27 entries (increasing column
 * order).  The diagonal is kept in diag. */
static int galerkin(const olevel *F, olevel *C) {
  long n = C->n;
  C->rowptr = (long *)malloc(sizeof(long) * (n + 1));
  C->col = (int *)malloc(sizeof(int) * n * 27);
  C->val = (double *)malloc(sizeof(double) * n * 27);
  C->diag = (double *)malloc(sizeof(double) * n);
  int *cnt = (int *)malloc(sizeof(int) * n);
  if (!C->rowptr || !C->col || !C->val || !C->diag || !cnt) {
    free(cnt);
    return -1;
  }
#pragma omp parallel for schedule(static)
  for (int ck = 0; ck < C->nz; ++ck)
    for (int cj = 0; cj < C->ny; ++cj)
      for (int ci = 0; ci < C->nx; ++ci) {
        const int I0 = ci + 1, J0 = cj + 1, K0 = ck + 1; /* coarse full coordinates */
        double acc[27];
        for (int e = 0; e < 27; ++e) acc[e] = 0.0;
        for (int c = -1; c <= 1; ++c)
          for (int b = -1; b <= 1; ++b)
            for (int a = -1; a <= 1; ++a) {
              const int fI = 2 * I0 + a, fJ = 2 * J0 + b, fK = 2 * K0 + c; /* fine full coordinates of i */
              const double rI = pw(fI, I0) * pw(fJ, J0) * pw(fK, K0) / 8.0;
              const long i = uidx(F, fI - 1, fJ - 1, fK - 1);
              for (long q = F->rowptr[i]; q < F->rowptr[i + 1]; ++q) {
                const long jl = F->col[q];
                const int jI = (int)(jl % F->nx) + 1, jJ = (int)((jl / F->nx) % F->ny) + 1,
                          jK = (int)(jl / ((long)F->nx * F->ny)) + 1;
                for (int CK = jK / 2; CK <= (jK + 1) / 2; ++CK)
                  for (int CJ = jJ / 2; CJ <= (jJ + 1) / 2; ++CJ)
                    for (int CI = jI / 2; CI <= (jI + 1) / 2; ++CI) {
                      if (!interior(C, CI, CJ, CK)) continue;
                      const double pj = pw(jI, CI) * pw(jJ, CJ) * pw(jK, CK);
                      if (pj == 0.0) continue;
                      acc[((CK - K0 + 1) * 3 + (CJ - J0 + 1)) * 3 + (CI - I0 + 1)] += rI * F->val[q] * pj;
                    }
              }
            }
        const long p = uidx(C, ci, cj, ck);
        long base = p * 27;
        int m = 0;
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              if (!interior(C, I0 + dx, J0 + dy, K0 + dz)) continue;
              C->col[base + m] = (int)uidx(C, ci + dx, cj + dy, ck + dz);
              C->val[base + m] = acc[((dz + 1) * 3 + (dy + 1)) * 3 + (dx + 1)];
              ++m;
            }
        cnt[p] = m;
        C->diag[p] = acc[13];
      }
  C->rowptr[0] = 0;
  for (long p = 0; p < n; ++p) C->rowptr[p + 1] = C->rowptr[p] + cnt[p];
  for (long p = 0; p < n; ++p) {
    long src = p * 27, dst = C->rowptr[p];
    for (int m = 0; m < cnt[p]; ++m) {
      C->col[dst + m] = C->col[src + m];
      C->val[dst + m] = C->val[src + m];
    }
  }
  free(cnt);
  return 0;
}

/* Gershgorin bound of D^-1 A: max over rows of sum_j |a_ij| / a_ii. */
static double gershgorin(const olevel *L) {
  double g = 0.0;
  for (long p = 0; p < L->n; ++p) {
    double s = 0.0;
    for (long q = L->rowptr[p]; q < L->rowptr[p + 1]; ++q) s += fabs(L->val[q]);
    if (s / L->diag[p] > g) g = s / L->diag[p];
  }
  return g;
}

/* ------------------------------------------------------------ eigen-estimate */
/* Counter-based uniform numbers in [0,1): Vigna's SplitMix64 finaliser,
 * u(seed, stream, idx) = (sm(sm(seed ^ stream << 56) ^ idx) >> 11) 2^-53. */
static uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static double uniform01(uint64_t seed, uint64_t stream, uint64_t idx) {
  return (double)(splitmix64(splitmix64(seed ^ (stream << 56)) ^ idx) >> 11) * (1.0 / 9007199254740992.0);
}
#define ORC_EIG_SEED 20160424ull
#define ORC_EIG_STEPS 10

/* Number of eigenvalues of the symmetric tridiagonal (d, e) below x (Sturm
 * sequence of the LDL^T pivots). */
static int sturm_below(int m, const double *d, const double *e, double x) {
  int c = 0;
  double q = 1.0;
  for (int i = 0; i < m; ++i) {
    q = d[i] - x - (i > 0 ? e[i - 1] * e[i - 1] / q : 0.0);
    if (q == 0.0) q = -1e-300;
    if (q < 0.0) ++c;
  }
  return c;
}

/* Largest eigenvalue of D^-1 A on a level, estimated by CG with the Jacobi
 * preconditioner for ORC_EIG_STEPS steps from a seeded random right-hand side
 * (entries u - 1/2, stream 3, index = interior point number) and a zero guess.
 * The CG coefficients give the Lanczos tridiagonal matrix of the
 * preconditioned operator (Saad, Iterative Methods, Sec. 6.7.3):
 * T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1}, T_{j,j+1} = sqrt(beta_j)/alpha_j;
 * its largest eigenvalue by bisection. */
static double lanczos_lmax(olevel *L) {
  const long n = L->n;
  double *r = L->r, *z = L->s, *p = L->d, *q = L->t;
  double al[ORC_EIG_STEPS], be[ORC_EIG_STEPS], d[ORC_EIG_STEPS], e[ORC_EIG_STEPS];
  for (long i = 0; i < n; ++i) r[i] = uniform01(ORC_EIG_SEED, 3, (uint64_t)i) - 0.5;
  for (long i = 0; i < n; ++i) z[i] = r[i] / L->diag[i];
  memcpy(p, z, sizeof(double) * n);
  double rz = dot(L, n, r, z);
  int m = 0;
  for (int j = 0; j < ORC_EIG_STEPS && (long)j < n; ++j) {
    spmv(L, p, q);
    const double pq = dot(L, n, p, q);
    if (!(pq > 0.0) || !(rz > 0.0)) break;
    al[j] = rz / pq;
    for (long i = 0; i < n; ++i) r[i] -= al[j] * q[i];
    for (long i = 0; i < n; ++i) z[i] = r[i] / L->diag[i];
    const double rz_new = dot(L, n, r, z);
    be[j] = rz_new / rz;
    for (long i = 0; i < n; ++i) p[i] = z[i] + be[j] * p[i];
    rz = rz_new;
    m = j + 1;
  }
  if (m == 0) return 2.0;
  for (int j = 0; j < m; ++j) {
    d[j] = 1.0 / al[j] + (j > 0 ? be[j - 1] / al[j - 1] : 0.0);
    if (j + 1 < m) e[j] = sqrt(be[j]) / al[j];
  }
  double lo = d[0], hi = d[0];
  for (int j = 0; j < m; ++j) {
    const double rad = (j > 0 ? fabs(e[j - 1]) : 0.0) + (j + 1 < m ? fabs(e[j]) : 0.0);
    if (d[j] - rad < lo) lo = d[j] - rad;
    if (d[j] + rad > hi) hi = d[j] + rad;
  }
  for (int it = 0; it < 200; ++it) { /* largest: count below x is m - 1 */
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_below(m, d, e, mid) >= m) hi = mid;
    else lo = mid;
  }
  return hi;
}

/* ------------------------------------------------------------ smoother */
/* One sweep of degree-m Chebyshev iteration for D^-1 A on [alpha, beta]
 * (preconditioned Chebyshev recurrence, Saad, Iterative Methods for Sparse
 * Linear Systems, Alg. 12.1): theta = (beta+alpha)/2, delta = (beta-alpha)/2,
 * sigma = theta/delta, rho_0 = 1/sigma, s = D^-1(b - A x), d = s/theta; then
 * m times: x += d and, unless last, s = D^-1(b - A x),
 * rho_j = 1/(2 sigma - rho_{j-1}), d = rho_j rho_{j-1} d + (2 rho_j/delta) s. */
static void cheby_sweep(const ohier *H, olevel *L, const double *b, double *x, int zero_guess) {
  const double theta = 0.5 * (L->beta + L->alpha), delta = 0.5 * (L->beta - L->alpha);
  const double sigma = theta / delta;
  double rho_prev = 1.0 / sigma;
  long n = L->n;
  double *s = L->s, *d = L->d, *t = L->t;
  if (zero_guess) {
#pragma omp parallel for schedule(static)
    for (long p = 0; p < n; ++p) s[p] = b[p] / L->diag[p];
  } else {
    spmv(L, x, t);
#pragma omp parallel for schedule(static)
    for (long p = 0; p < n; ++p) s[p] = (b[p] - t[p]) / L->diag[p];
  }
#pragma omp parallel for schedule(static)
  for (long p = 0; p < n; ++p) d[p] = s[p] / theta;
  for (int j = 1; j <= H->degree; ++j) {
#pragma omp parallel for schedule(static)
    for (long p = 0; p < n; ++p) x[p] += d[p];
    if (j < H->degree) {
      spmv(L, x, t);
      double rho = 1.0 / (2.0 * sigma - rho_prev);
      double c1 = rho * rho_prev, c2 = 2.0 * rho / delta;
#pragma omp parallel for schedule(static)
      for (long p = 0; p < n; ++p) {
        double sp = (b[p] - t[p]) / L->diag[p];
        d[p] = c1 * d[p] + c2 * sp;
      }
      rho_prev = rho;
    }
  }
}

/* One Richardson iteration preconditioned with Jacobi, the classical
 * fixed-point smoother of Sec. 2.1.1 (Sec. 5 runs eight of them per level):
 * x += omega D^-1 (b - A x).  From a zero guess the residual is b. */
static void richardson_sweep(const ohier *H, olevel *L, const double *b, double *x, int zero_guess) {
  const long n = L->n;
  double *t = L->t;
  if (zero_guess) {
#pragma omp parallel for schedule(static)
    for (long p = 0; p < n; ++p) x[p] = H->omega * (b[p] / L->diag[p]);
    return;
  }
  spmv(L, x, t);
#pragma omp parallel for schedule(static)
  for (long p = 0; p < n; ++p) x[p] += H->omega * ((b[p] - t[p]) / L->diag[p]);
}

static void smooth_sweep(const ohier *H, olevel *L, const double *b, double *x, int zero_guess) {
  if (H->smoother == 1) richardson_sweep(H, L, b, x, zero_guess);
  else cheby_sweep(H, L, b, x, zero_guess);
}

/* ------------------------------------------------------------ coarse solve */
static int build_coarse(ohier *H) {
  olevel *L = &H->lv[H->L - 1];
  int n = (int)L->n;
  H->nc = n;
  H->Ac = (double *)calloc((size_t)n * n, sizeof(double));
  H->Lc = (double *)calloc((size_t)n * n, sizeof(double));
  if (!H->Ac || !H->Lc) return -1;
  for (int p = 0; p < n; ++p)
    for (long q = L->rowptr[p]; q < L->rowptr[p + 1]; ++q) H->Ac[(size_t)p * n + L->col[q]] = L->val[q];
  /* Cholesky A = L L^T, column by column (textbook Cholesky-Crout order). */
  double *A = H->Ac, *C = H->Lc;
  for (int j = 0; j < n; ++j) {
    double s = A[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) s -= C[(size_t)j * n + k] * C[(size_t)j * n + k];
    if (!(s > 0.0)) return -2; /* not positive definite */
    double ljj = sqrt(s);
    C[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double t = A[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) t -= C[(size_t)i * n + k] * C[(size_t)j * n + k];
      C[(size_t)i * n + j] = t / ljj;
    }
  }
  return 0;
}

/* Inexact coarsest solve (the "truncated" coarse solve of Sec. 5): GMRES
 * preconditioned on the right with Jacobi (the diagonal of A_L), classical
 * Gram-Schmidt, Givens rotations, from x = 0, stopped when the rotated
 * residual norm falls to coarse_rtol times ||b|| or after coarse_maxit steps. */
static void coarse_gmres(const ohier *H, const double *b, double *x) {
  const int n = H->nc, m = H->coarse_maxit;
  const double *A = H->Ac;
  double *V = (double *)calloc((size_t)(m + 1) * n, sizeof(double));
  double *Hs = (double *)calloc((size_t)(m + 1) * m, sizeof(double));
  double *w = (double *)malloc(sizeof(double) * n), *z = (double *)malloc(sizeof(double) * n);
  double *g = (double *)calloc(m + 1, sizeof(double)), *cs = (double *)malloc(sizeof(double) * m);
  double *sn = (double *)malloc(sizeof(double) * m), *y = (double *)malloc(sizeof(double) * m);
  for (int i = 0; i < n; ++i) x[i] = 0.0;
  double beta = 0.0;
  for (int i = 0; i < n; ++i) beta += b[i] * b[i];
  beta = sqrt(beta);
  int jj = 0;
  if (beta > 0.0) {
    for (int i = 0; i < n; ++i) V[i] = b[i] / beta;
    g[0] = beta;
    for (int j = 0; j < m; ++j) {
      for (int i = 0; i < n; ++i) z[i] = V[(size_t)j * n + i] / A[(size_t)i * n + i];
      for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += A[(size_t)i * n + k] * z[k];
        w[i] = s;
      }
      for (int i = 0; i <= j; ++i) {
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += w[k] * V[(size_t)i * n + k];
        Hs[(size_t)i * m + j] = s;
      }
      for (int i = 0; i <= j; ++i)
        for (int k = 0; k < n; ++k) w[k] -= Hs[(size_t)i * m + j] * V[(size_t)i * n + k];
      double hn = 0.0;
      for (int k = 0; k < n; ++k) hn += w[k] * w[k];
      hn = sqrt(hn);
      Hs[(size_t)(j + 1) * m + j] = hn;
      if (hn > 0.0)
        for (int k = 0; k < n; ++k) V[(size_t)(j + 1) * n + k] = w[k] / hn;
      for (int i = 0; i < j; ++i) {
        const double a = Hs[(size_t)i * m + j], c = Hs[(size_t)(i + 1) * m + j];
        Hs[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
        Hs[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
      }
      const double a = Hs[(size_t)j * m + j], c = Hs[(size_t)(j + 1) * m + j];
      const double d = sqrt(a * a + c * c);
      if (!(d > 0.0)) break;
      cs[j] = a / d;
      sn[j] = c / d;
      Hs[(size_t)j * m + j] = d;
      Hs[(size_t)(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      jj = j + 1;
      if (fabs(g[j + 1]) <= H->coarse_rtol * beta || hn == 0.0) break;
    }
    for (int i = jj - 1; i >= 0; --i) {
      double s = g[i];
      for (int k = i + 1; k < jj; ++k) s -= Hs[(size_t)i * m + k] * y[k];
      y[i] = s / Hs[(size_t)i * m + i];
    }
    for (int i = 0; i < n; ++i) { /* x = D^-1 V y */
      double s = 0.0;
      for (int k = 0; k < jj; ++k) s += y[k] * V[(size_t)k * n + i];
      x[i] = s / A[(size_t)i * n + i];
    }
  }
  free(V); free(Hs); free(w); free(z); free(g); free(cs); free(sn); free(y);
}

static void coarse_solve(const ohier *H, const double *b, double *x) {
  if (H->coarse_mode == 1) {
    coarse_gmres(H, b, x);
    return;
  }
  int n = H->nc;
  const double *C = H->Lc;
  for (int i = 0; i < n; ++i) { /* L y = b */
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= C[(size_t)i * n + k] * x[k];
    x[i] = s / C[(size_t)i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) { /* L^T x = y */
    double s = x[i];
    for (int k = i + 1; k < n; ++k) s -= C[(size_t)k * n + i] * x[k];
    x[i] = s / C[(size_t)i * n + i];
  }
}

/* ------------------------------------------------------------ V-cycle */
/* Algorithm 1 applied recursively with a zero initial guess on every level:
 * pre-smooth, restrict the residual, solve for the coarse correction (the
 * next level's cycle, or the exact factorisation on the coarsest level),
 * prolongate and add it, post-smooth. */
static void vcycle(ohier *H, int l, const double *b, double *x) {
  olevel *L = &H->lv[l];
  if (l == H->L - 1) {
    coarse_solve(H, b, x);
    return;
  }
  olevel *C = &H->lv[l + 1];
  memset(x, 0, sizeof(double) * L->n);
  for (int s = 0; s < H->nu_pre; ++s) smooth_sweep(H, L, b, x, s == 0);
  spmv(L, x, L->r);
#pragma omp parallel for schedule(static)
  for (long p = 0; p < L->n; ++p) L->r[p] = b[p] - L->r[p];
  restrict_fw(L, C, L->r, C->b);
  vcycle(H, l + 1, C->b, C->x);
  prolong_add(L, C, C->x, x);
  for (int s = 0; s < H->nu_post; ++s) smooth_sweep(H, L, b, x, 0);
}

/* ------------------------------------------------------------ public API */
void orc_free(void *hh);

/* coarse_op 0: re-discretised coarse operators (cell k averaged by
 * coarse_rule); 1: Galerkin R A P.  The Chebyshev interval of a level is
 * [eig_lo_frac beta, beta] with beta = eig_hi on re-discretised levels (their
 * Gershgorin bound is 2) and the level's Gershgorin bound of D^-1 A on
 * Galerkin levels. */
void *orc_create_opt(int Nx, int Ny, int Nz, const double *kc, int levels, int nu_pre, int nu_post,
                     int degree, double eig_lo_frac, double eig_hi, int coarse_rule, int face_rule,
                     int coarse_op) {
  if (levels < 1 || levels > ORC_MAX_LEVELS || degree < 1 || nu_pre < 0 || nu_post < 0) return NULL;
  if (coarse_rule < 0 || coarse_rule > 2 || face_rule < 0 || face_rule > 1) return NULL;
  if (coarse_op < 0 || coarse_op > 1) return NULL;
  ohier *H = (ohier *)calloc(1, sizeof(ohier));
  if (!H) return NULL;
  H->L = levels;
  H->nu_pre = nu_pre;
  H->nu_post = nu_post;
  H->degree = degree;
  H->beta = eig_hi;
  H->omega = 6.0 / 7.0;
  H->alpha = eig_lo_frac * eig_hi;
  H->coarse_rule = coarse_rule;
  H->face_rule = face_rule;
  H->galerkin = coarse_op;
  int N[3] = {Nx, Ny, Nz};
  for (int l = 0; l < levels; ++l) {
    olevel *L = &H->lv[l];
    if (N[0] < 3 || N[1] < 3 || N[2] < 3) goto fail;
    L->Nx = N[0]; L->Ny = N[1]; L->Nz = N[2];
    L->nx = N[0] - 2; L->ny = N[1] - 2; L->nz = N[2] - 2;
    L->n = (long)L->nx * L->ny * L->nz;
    L->hx = 1.0 / (N[0] - 1); L->hy = 1.0 / (N[1] - 1); L->hz = 1.0 / (N[2] - 1);
    L->face_rule = face_rule;
    long ncell = (long)(N[0] - 1) * (N[1] - 1) * (N[2] - 1);
    L->kc = (double *)malloc(sizeof(double) * ncell);
    if (!L->kc) goto fail;
    if (l == 0) {
      for (long c = 0; c < ncell; ++c) {
        if (!(kc[c] > 0.0) || !isfinite(kc[c])) goto fail;
        L->kc[c] = kc[c];
      }
    } else {
      /* re-discretised coarse level: cell k is a mean of its 8 children
       * (arithmetic by default; the paper does not state the rule) */
      const olevel *F = &H->lv[l - 1];
      const int rule = H->coarse_rule;
#pragma omp parallel for schedule(static)
      for (int ck = 0; ck < N[2] - 1; ++ck)
        for (int cj = 0; cj < N[1] - 1; ++cj)
          for (int ci = 0; ci < N[0] - 1; ++ci) {
            double s = 0.0;
            for (int c = 0; c < 2; ++c)
              for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a) {
                  double kv = kcell(F, 2 * ci + a, 2 * cj + b, 2 * ck + c);
                  s += rule == 0 ? kv : rule == 1 ? log(kv) : 1.0 / kv;
                }
            double m = rule == 0 ? s / 8.0 : rule == 1 ? exp(s / 8.0) : 8.0 / s;
            L->kc[((long)ck * (N[1] - 1) + cj) * (N[0] - 1) + ci] = m;
          }
    }
    if (l > 0 && H->galerkin) {
      if (galerkin(&H->lv[l - 1], L)) goto fail;
      L->beta = gershgorin(L);
    } else {
      if (assemble(L)) goto fail;
      L->beta = eig_hi;
    }
    L->alpha = eig_lo_frac * L->beta;
    long n = L->n;
    L->b = (double *)calloc(n, sizeof(double));
    L->x = (double *)calloc(n, sizeof(double));
    L->r = (double *)calloc(n, sizeof(double));
    L->s = (double *)calloc(n, sizeof(double));
    L->d = (double *)calloc(n, sizeof(double));
    L->t = (double *)calloc(n, sizeof(double));
    if (!L->b || !L->x || !L->r || !L->s || !L->d || !L->t) goto fail;
    if (l + 1 < levels) {
      for (int a = 0; a < 3; ++a) {
        if ((N[a] - 1) % 2) goto fail;
        N[a] = (N[a] - 1) / 2 + 1;
      }
    }
  }
  if (H->lv[levels - 1].n > ORC_MAX_COARSE) goto fail;
  if (build_coarse(H)) goto fail;
  return H;
fail:
  orc_free(H);
  return NULL;
}

void *orc_create(int Nx, int Ny, int Nz, const double *kc, int levels, int nu_pre, int nu_post,
                 int degree, double eig_lo_frac, double eig_hi, int coarse_rule, int face_rule) {
  return orc_create_opt(Nx, Ny, Nz, kc, levels, nu_pre, nu_post, degree, eig_lo_frac, eig_hi, coarse_rule,
                        face_rule, 0);
}

/* Coarsest solve: mode 0 the Cholesky factorisation; mode 1 GMRES with the
 * Jacobi preconditioner to rtol, at most maxit steps (an inexact solve: the
 * preconditioner is then no longer a fixed linear operator, and the outer
 * method should be flexible GMRES). */
int orc_set_coarse(void *hh, int mode, double rtol, int maxit) {
  ohier *H = (ohier *)hh;
  if (!H || mode < 0 || mode > 1 || !(rtol > 0.0) || maxit < 1) return -1;
  H->coarse_mode = mode;
  H->coarse_rtol = rtol;
  H->coarse_maxit = maxit;
  return 0;
}

/* Upper end of level l's Chebyshev interval. */
/* Summation order of every level's dot products and operator rows: 0 (the
 * default) sums in index order; 1 sums dot products pairwise and operator
 * rows from the last stored entry to the first.  Both are fixed orders of the
 * same arithmetic; running a solve under each measures how far rounding order
 * alone moves its iterates (test infrastructure for the parity tolerances). */
int orc_set_sum_order(void *hh, int order) {
  ohier *H = (ohier *)hh;
  if (order < 0 || order > 1) return -1;
  for (int l = 0; l < H->L; ++l) H->lv[l].sum_order = order;
  return 0;
}

/* a . b over n entries in the finest level's summation order. */
double orc_dot(void *hh, long n, const double *a, const double *b) {
  return dot(&((ohier *)hh)->lv[0], n, a, b);
}

double orc_level_beta(void *hh, int l) { return ((ohier *)hh)->lv[l].beta; }
double orc_level_alpha(void *hh, int l) { return ((ohier *)hh)->lv[l].alpha; }

/* Chebyshev intervals: mode 0 keeps [eig_lo_frac beta, beta] with beta =
 * eig_hi (Gershgorin on Galerkin levels); mode 1 sets
 * [eig_lo_frac lambda, safety lambda] per level from the Lanczos estimate
 * lambda of the largest eigenvalue of D^-1 A (the PETSc default is an
 * estimate of this kind with the interval [0.1 lambda, 1.1 lambda]). */
int orc_set_eig_mode(void *hh, int mode, double safety) {
  ohier *H = (ohier *)hh;
  if (!H || mode < 0 || mode > 1 || !(safety > 0.0)) return -1;
  const double lo_frac = H->alpha / H->beta;
  H->eig_mode = mode;
  for (int l = 0; l < H->L; ++l) {
    olevel *L = &H->lv[l];
    if (mode == 1) {
      const double lm = lanczos_lmax(L);
      L->beta = safety * lm;
      L->alpha = lo_frac * lm;
    } else {
      L->beta = (l > 0 && H->galerkin) ? gershgorin(L) : H->beta;
      L->alpha = lo_frac * L->beta;
    }
  }
  return 0;
}

/* Largest-eigenvalue estimate of level l (the Lanczos procedure above). */
double orc_level_lanczos(void *hh, int l) { return lanczos_lmax(&((ohier *)hh)->lv[l]); }

void orc_free(void *hh) {
  ohier *H = (ohier *)hh;
  if (!H) return;
  for (int l = 0; l < ORC_MAX_LEVELS; ++l) {
    olevel *L = &H->lv[l];
    free(L->kc); free(L->rowptr); free(L->col); free(L->val); free(L->diag);
    free(L->b); free(L->x); free(L->r); free(L->s); free(L->d); free(L->t);
  }
  free(H->Ac);
  free(H->Lc);
  free(H);
}

int orc_num_levels(void *hh) { return ((ohier *)hh)->L; }

void orc_level_dims(void *hh, int l, int *N3) {
  olevel *L = &((ohier *)hh)->lv[l];
  N3[0] = L->Nx; N3[1] = L->Ny; N3[2] = L->Nz;
}

long orc_nnz(void *hh, int l) {
  olevel *L = &((ohier *)hh)->lv[l];
  return L->rowptr[L->n];
}

void orc_csr(void *hh, int l, long *rowptr, int *col, double *val) {
  olevel *L = &((ohier *)hh)->lv[l];
  memcpy(rowptr, L->rowptr, sizeof(long) * (L->n + 1));
  memcpy(col, L->col, sizeof(int) * L->rowptr[L->n]);
  memcpy(val, L->val, sizeof(double) * L->rowptr[L->n]);
}

void orc_cells(void *hh, int l, double *kc) {
  olevel *L = &((ohier *)hh)->lv[l];
  memcpy(kc, L->kc, sizeof(double) * (long)(L->Nx - 1) * (L->Ny - 1) * (L->Nz - 1));
}

int orc_coarse_n(void *hh) { return ((ohier *)hh)->nc; }

void orc_coarse_dense(void *hh, double *A, double *Lf) {
  ohier *H = (ohier *)hh;
  memcpy(A, H->Ac, sizeof(double) * H->nc * H->nc);
  memcpy(Lf, H->Lc, sizeof(double) * H->nc * H->nc);
}

/* y = A_l x on full-grid arrays of level l (boundary of y set to 0). */
void orc_apply(void *hh, int l, const double *xf, double *yf) {
  olevel *L = &((ohier *)hh)->lv[l];
  to_interior(L, xf, L->x);
  spmv(L, L->x, L->t);
  to_full(L, L->t, yf);
}

/* One smoother sweep on level l; x is read unless zero_guess. */
void orc_smooth(void *hh, int l, const double *bf, double *xf, int zero_guess) {
  ohier *H = (ohier *)hh;
  olevel *L = &H->lv[l];
  double *b = (double *)malloc(sizeof(double) * L->n), *x = (double *)calloc(L->n, sizeof(double));
  to_interior(L, bf, b);
  if (!zero_guess) to_interior(L, xf, x);
  smooth_sweep(H, L, b, x, zero_guess);
  to_full(L, x, xf);
  free(b);
  free(x);
}

/* Flexible GMRES(m) preconditioned on the right by the V-cycle (Saad,
 * Iterative Methods for Sparse Linear Systems, Alg. 9.6), the outer Krylov
 * method of the paper's Sec. 5 runs.  The Arnoldi basis is orthogonalised by
 * classical Gram-Schmidt (all coefficients from the same vector, no second
 * pass); the least-squares problem is reduced by Givens rotations; the
 * iteration stops when the rotated residual norm |g_{j+1}| <= rtol ||b||, or
 * after maxit steps, and restarts from the true residual every m steps.
 * x starts at zero.  Returns the iterations done (-1: breakdown). */
int orc_fgmres(void *hh, const double *ff, double *xf, double rtol, int maxit, int m, double *hist, double *out) {
  ohier *H = (ohier *)hh;
  olevel *L = &H->lv[0];
  const long n = L->n;
  if (m < 1) return -1;
  double *b = (double *)malloc(sizeof(double) * n), *x = (double *)calloc(n, sizeof(double));
  double *r = (double *)malloc(sizeof(double) * n), *w = (double *)malloc(sizeof(double) * n);
  double *V = (double *)malloc(sizeof(double) * n * (m + 1)), *Z = (double *)malloc(sizeof(double) * n * m);
  double *Hs = (double *)calloc((size_t)(m + 1) * m, sizeof(double));
  double *cs = (double *)malloc(sizeof(double) * m), *sn = (double *)malloc(sizeof(double) * m);
  double *g = (double *)malloc(sizeof(double) * (m + 1)), *y = (double *)malloc(sizeof(double) * m);
  to_interior(L, ff, b);
  const double bnorm = sqrt(dot(L, n, b, b));
  int it = 0, status = 0;
  double rnorm = bnorm;
  if (hist) hist[0] = bnorm > 0 ? 1.0 : 0.0;
  while (bnorm > 0.0) {
    spmv(L, x, w); /* restart from the true residual */
    for (long i = 0; i < n; ++i) r[i] = b[i] - w[i];
    const double beta = sqrt(dot(L, n, r, r));
    rnorm = beta;
    if (beta <= rtol * bnorm || it >= maxit) break;
    for (long i = 0; i < n; ++i) V[i] = r[i] / beta;
    for (int i = 0; i <= m; ++i) g[i] = 0.0;
    g[0] = beta;
    int jj = 0, done = 0;
    for (int j = 0; j < m; ++j) {
      double *vj = V + (size_t)j * n, *zj = Z + (size_t)j * n;
      vcycle(H, 0, vj, zj);
      spmv(L, zj, w);
      for (int i = 0; i <= j; ++i) Hs[(size_t)i * m + j] = dot(L, n, w, V + (size_t)i * n);
      for (int i = 0; i <= j; ++i) {
        const double hij = Hs[(size_t)i * m + j];
        const double *vi = V + (size_t)i * n;
        for (long q = 0; q < n; ++q) w[q] -= hij * vi[q];
      }
      const double hn = sqrt(dot(L, n, w, w));
      Hs[(size_t)(j + 1) * m + j] = hn;
      if (hn > 0.0)
        for (long q = 0; q < n; ++q) V[(size_t)(j + 1) * n + q] = w[q] / hn;
      for (int i = 0; i < j; ++i) { /* earlier rotations on column j */
        const double a = Hs[(size_t)i * m + j], c = Hs[(size_t)(i + 1) * m + j];
        Hs[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
        Hs[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
      }
      const double a = Hs[(size_t)j * m + j], c = Hs[(size_t)(j + 1) * m + j];
      const double d = sqrt(a * a + c * c);
      if (!(d > 0.0)) { status = -1; done = 1; break; }
      cs[j] = a / d;
      sn[j] = c / d;
      Hs[(size_t)j * m + j] = d;
      Hs[(size_t)(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++it;
      jj = j + 1;
      rnorm = fabs(g[j + 1]);
      if (hist) hist[it] = rnorm / bnorm;
      if (rnorm <= rtol * bnorm || it >= maxit || hn == 0.0) { done = 1; break; }
    }
    for (int i = jj - 1; i >= 0; --i) { /* R y = g, then x += Z y */
      double s = g[i];
      for (int k = i + 1; k < jj; ++k) s -= Hs[(size_t)i * m + k] * y[k];
      y[i] = s / Hs[(size_t)i * m + i];
    }
    for (int i = 0; i < jj; ++i) {
      const double *zi = Z + (size_t)i * n;
      for (long q = 0; q < n; ++q) x[q] += y[i] * zi[q];
    }
    if (done) break;
  }
  spmv(L, x, w);
  for (long i = 0; i < n; ++i) w[i] = b[i] - w[i];
  if (out) {
    out[0] = bnorm > 0 ? rnorm / bnorm : 0.0;
    out[1] = bnorm > 0 ? sqrt(dot(L, n, w, w)) / bnorm : 0.0;
    out[2] = bnorm;
  }
  to_full(L, x, xf);
  free(b); free(x); free(r); free(w); free(V); free(Z); free(Hs); free(cs); free(sn); free(g); free(y);
  return status < 0 ? -1 : it;
}

/* Smoother choice: 0 Chebyshev-Jacobi (default), 1 Richardson-Jacobi with
 * damping omega (one iteration per sweep). */
int orc_set_smoother(void *hh, int smoother, double omega) {
  ohier *H = (ohier *)hh;
  if (!H || smoother < 0 || smoother > 1 || !(omega > 0.0)) return -1;
  H->smoother = smoother;
  H->omega = omega;
  return 0;
}

/* bc = R (b - A x) from level l to level l+1. */
void orc_residual_restrict(void *hh, int l, const double *bf, const double *xf, double *bcf) {
  ohier *H = (ohier *)hh;
  olevel *L = &H->lv[l], *C = &H->lv[l + 1];
  double *b = (double *)malloc(sizeof(double) * L->n);
  to_interior(L, bf, b);
  to_interior(L, xf, L->x);
  spmv(L, L->x, L->t);
  for (long p = 0; p < L->n; ++p) L->r[p] = b[p] - L->t[p];
  restrict_fw(L, C, L->r, C->t);
  to_full(C, C->t, bcf);
  free(b);
}

/* x += P ec from level l+1 to level l. */
void orc_prolong_add(void *hh, int l, const double *ecf, double *xf) {
  ohier *H = (ohier *)hh;
  olevel *L = &H->lv[l], *C = &H->lv[l + 1];
  to_interior(C, ecf, C->t);
  to_interior(L, xf, L->x);
  prolong_add(L, C, C->t, L->x);
  to_full(L, L->x, xf);
}

/* x = A_L^-1 b on the coarsest level. */
void orc_coarse_solve(void *hh, const double *bf, double *xf) {
  ohier *H = (ohier *)hh;
  olevel *L = &H->lv[H->L - 1];
  to_interior(L, bf, L->b);
  coarse_solve(H, L->b, L->x);
  to_full(L, L->x, xf);
}

/* z = M^-1 r: one V-cycle from level l0 with zero initial guess. */
void orc_vcycle(void *hh, int l0, const double *rf, double *zf) {
  ohier *H = (ohier *)hh;
  olevel *L = &H->lv[l0];
  double *r = (double *)malloc(sizeof(double) * L->n), *z = (double *)malloc(sizeof(double) * L->n);
  to_interior(L, rf, r);
  vcycle(H, l0, r, z);
  to_full(L, z, zf);
  free(r);
  free(z);
}

/* Preconditioned CG on level 0 (Hestenes-Stiefel recurrences).  x0 = 0 unless
 * nonzero_guess.  Stops when the recurrence residual satisfies
 * ||r_k||_2 <= rtol ||b||_2 or after maxit iterations.  flexible selects the
 * Polak-Ribiere beta = r_{k+1}.(z_{k+1} - z_k) / rho_k, otherwise the
 * Fletcher-Reeves beta = rho_{k+1}/rho_k.  hist (maxit+1 entries, may be NULL)
 * receives ||r_k||/||b||.  out[0] = final recurrence relative residual,
 * out[1] = true relative residual ||b - A x||/||b||, out[2] = ||b||.
 * Returns the iteration count, or -1 on breakdown (p.Ap <= 0). */
int orc_pcg(void *hh, const double *ff, double *xf, double rtol, int maxit, int flexible,
            int nonzero_guess, double *hist, double *out) {
  ohier *H = (ohier *)hh;
  olevel *L = &H->lv[0];
  long n = L->n;
  double *b = (double *)malloc(sizeof(double) * n), *x = (double *)calloc(n, sizeof(double));
  double *r = (double *)malloc(sizeof(double) * n), *z = (double *)malloc(sizeof(double) * n);
  double *zo = (double *)malloc(sizeof(double) * n), *p = (double *)malloc(sizeof(double) * n);
  double *q = (double *)malloc(sizeof(double) * n);
  to_interior(L, ff, b);
  if (nonzero_guess) to_interior(L, xf, x);
  double bnorm = sqrt(dot(L, n, b, b));
  spmv(L, x, q);
  for (long i = 0; i < n; ++i) r[i] = b[i] - q[i];
  double rnorm = sqrt(dot(L, n, r, r));
  int it = 0, status = 0;
  if (hist) hist[0] = bnorm > 0 ? rnorm / bnorm : 0.0;
  if (bnorm == 0.0 || rnorm <= rtol * bnorm) goto done;
  vcycle(H, 0, r, z);
  memcpy(p, z, sizeof(double) * n);
  double rho = dot(L, n, r, z);
  for (it = 1; it <= maxit; ++it) {
    spmv(L, p, q);
    double pq = dot(L, n, p, q);
    if (!(pq > 0.0)) { status = -1; break; }
    double alpha = rho / pq;
    for (long i = 0; i < n; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * q[i];
    }
    rnorm = sqrt(dot(L, n, r, r));
    if (hist) hist[it] = rnorm / bnorm;
    if (rnorm <= rtol * bnorm) break;
    if (it == maxit) break;
    if (flexible) memcpy(zo, z, sizeof(double) * n);
    vcycle(H, 0, r, z);
    double rho_new = dot(L, n, r, z);
    double beta = flexible ? (rho_new - dot(L, n, r, zo)) / rho : rho_new / rho;
    for (long i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    rho = rho_new;
  }
  if (it > maxit) it = maxit;
done:
  spmv(L, x, q);
  for (long i = 0; i < n; ++i) q[i] = b[i] - q[i];
  if (out) {
    out[0] = bnorm > 0 ? rnorm / bnorm : 0.0;
    out[1] = bnorm > 0 ? sqrt(dot(L, n, q, q)) / bnorm : 0.0;
    out[2] = bnorm;
  }
  to_full(L, x, xf);
  free(b); free(x); free(r); free(z); free(zo); free(p); free(q);
  return status ? status : it;
}

/* Gradient of a loss L(phi) with respect to the natural log of each finest
 * cell's k, given phi = A^-1 f and the adjoint lambda = A^-1 dL/dphi:
 *   dL/dk_e       = -h_a^-2 (lambda_p - lambda_q)(phi_p - phi_q)  for edge e=(p,q)
 *   dk_e/dln k_c  = k_e^2 / (4 k_c)        (k_e harmonic mean of 4 cells)
 *                 = k_c / 4                (k_e arithmetic mean of 4 cells)
 *   dL/dln k_c    = sum over the 12 edges of cell c.
 * Edges with both ends on the boundary contribute nothing. */
void orc_gradient(void *hh, const double *phi, const double *lam, double *grad) {
  ohier *H = (ohier *)hh;
  olevel *L = &H->lv[0];
  const double ih2[3] = {1.0 / (L->hx * L->hx), 1.0 / (L->hy * L->hy), 1.0 / (L->hz * L->hz)};
#pragma omp parallel for schedule(static)
  for (int ck = 0; ck < L->Nz - 1; ++ck)
    for (int cj = 0; cj < L->Ny - 1; ++cj)
      for (int ci = 0; ci < L->Nx - 1; ++ci) {
        double kcv = kcell(L, ci, cj, ck), g = 0.0;
        for (int axis = 0; axis < 3; ++axis)
          for (int u = 0; u < 2; ++u)
            for (int v = 0; v < 2; ++v) {
              int P0[3], P1[3];
              if (axis == 0) { P0[0] = ci; P0[1] = cj + u; P0[2] = ck + v; }
              else if (axis == 1) { P0[0] = ci + u; P0[1] = cj; P0[2] = ck + v; }
              else { P0[0] = ci + u; P0[1] = cj + v; P0[2] = ck; }
              P1[0] = P0[0]; P1[1] = P0[1]; P1[2] = P0[2];
              P1[axis] += 1;
              int in0 = interior(L, P0[0], P0[1], P0[2]), in1 = interior(L, P1[0], P1[1], P1[2]);
              if (!in0 && !in1) continue;
              double l0 = in0 ? lam[fidx(L, P0[0], P0[1], P0[2])] : 0.0;
              double l1 = in1 ? lam[fidx(L, P1[0], P1[1], P1[2])] : 0.0;
              double f0 = in0 ? phi[fidx(L, P0[0], P0[1], P0[2])] : 0.0;
              double f1 = in1 ? phi[fidx(L, P1[0], P1[1], P1[2])] : 0.0;
              double ke = kedge(L, axis, P0[0], P0[1], P0[2]);
              double dLdke = -ih2[axis] * (l0 - l1) * (f0 - f1);
              g += dLdke * (L->face_rule ? kcv / 4.0 : ke * ke / (4.0 * kcv));
            }
        grad[((long)ck * (L->Ny - 1) + cj) * (L->Nx - 1) + ci] = g;
      }
}
