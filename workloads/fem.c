/*
 * Seeded synthetic finite-element workloads for the R-tree multilevel solver.
 *
 * This file builds the linear systems the solver is applied to: the Poisson
 * model problem -div(kappa grad u) = f on the unit square/cube with u = 0 on
 * the boundary (Section 2, eqs. (poisson), (weakform), (discweakform)),
 * discretised by continuous Q_p Lagrange elements (Section 2.1) on a
 * structured N^d mesh whose interior vertices may be randomly perturbed.
 * It holds none of the multilevel method's arithmetic: no partitioning,
 * no transfer operators, no smoother, no Krylov iteration.  Both the
 * CPU oracle and the GPU library consume what it produces.
 *
 * Conventions
 *   - support points: Gauss-Lobatto-Legendre (GLL) nodes of each cell,
 *     mapped by the cell's multilinear (Q1) geometry map;
 *   - global nodes lexicographic on the (N p + 1)^d grid, x fastest;
 *   - Dirichlet rows/columns eliminated: only free (interior) nodes are
 *     unknowns, numbered lexicographically on the (N p - 1)^d interior grid;
 *   - quadrature: tensor Gauss-Legendre with p+1 points per direction;
 *   - cells are assembled in 2^d parity colours so that the OpenMP sum is
 *     deterministic; local matrices are filled for a <= b and mirrored, so the
 *     assembled matrix is bitwise symmetric;
 *   - random numbers: splitmix64 (Steele, Lea, Flood 2014), doubles in [0,1)
 *     from the top 53 bits.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define FEM_MAXP 8
#define FEM_MAXD 3

static uint64_t sm64_next(uint64_t* s) {
  uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static double sm64_unit(uint64_t* s) { return (double)(sm64_next(s) >> 11) * (1.0 / 9007199254740992.0); }

/* Legendre polynomial P_n and derivative at x in [-1,1] (three-term recurrence). */
static void legendre(int n, double x, double* P, double* dP) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int k = 2; k <= n; ++k) { double pk = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k; p0 = p1; p1 = pk; }
  *P = p1;
  *dP = (fabs(x) < 1.0) ? n * (x * p1 - p0) / (x * x - 1.0) : 0.5 * n * (n + 1) * (x > 0 ? 1.0 : ((n % 2) ? 1.0 : -1.0));
}

/* Gauss-Legendre nodes/weights on [0,1], m points (Newton on P_m). */
static void gauss_legendre01(int m, double* x, double* w) {
  for (int i = 0; i < m; ++i) {
    double t = cos(M_PI * (i + 0.75) / (m + 0.5)), P, dP;
    for (int it = 0; it < 100; ++it) { legendre(m, t, &P, &dP); double dt = P / dP; t -= dt; if (fabs(dt) < 1e-16) break; }
    legendre(m, t, &P, &dP);
    x[m - 1 - i] = 0.5 * (t + 1.0);
    w[m - 1 - i] = 1.0 / ((1.0 - t * t) * dP * dP);   /* = (2/((1-t^2)P'^2)) / 2 on [0,1] */
  }
}

/* GLL nodes on [0,1], p+1 points: endpoints and roots of P_p' (Newton on P_p'). */
static void gll01(int p, double* x) {
  x[0] = 0.0; x[p] = 1.0;
  for (int i = 1; i < p; ++i) {
    /* initial guess: Chebyshev-Gauss-Lobatto point, then Newton on q = P_p' using q' from the ODE */
    double t = -cos(M_PI * i / p), P, dP;
    for (int it = 0; it < 100; ++it) {
      legendre(p, t, &P, &dP);
      double d2P = (2.0 * t * dP - p * (p + 1.0) * P) / (1.0 - t * t);
      double dt = dP / d2P; t -= dt;
      if (fabs(dt) < 1e-16) break;
    }
    x[i] = 0.5 * (t + 1.0);
  }
}

/* 1-D Lagrange basis on nodes z[0..p]: values and derivatives at t. */
static void lagrange1d(int p, const double* z, double t, double* L, double* dL) {
  for (int a = 0; a <= p; ++a) {
    double v = 1.0, dv = 0.0;
    for (int k = 0; k <= p; ++k) {
      if (k == a) continue;
      double f = (t - z[k]) / (z[a] - z[k]);
      dv = dv * f + v / (z[a] - z[k]);
      v *= f;
    }
    L[a] = v; dL[a] = dv;
  }
}

typedef struct {
  int dim, N, p;
  int nodes1d;          /* N p + 1 */
  int free1d;           /* N p - 1 */
  double* vert;         /* (N+1)^d * d vertex coordinates */
  double gll[FEM_MAXP + 1];
  int nkappa;           /* number of Fourier modes in log kappa (0: kappa = 1) */
  double kwave[64][3], kphase[64], kamp;
  int rhs_kind;         /* 0: manufactured sine, 1: f = 1 */
} fem_mesh;

static double kappa_at(const fem_mesh* m, const double* x) {
  if (m->nkappa == 0) return 1.0;
  double g = 0.0;
  for (int k = 0; k < m->nkappa; ++k) {
    double ph = m->kphase[k];
    for (int a = 0; a < m->dim; ++a) ph += 2.0 * M_PI * m->kwave[k][a] * x[a];
    g += m->kamp * cos(ph);
  }
  return exp(g);
}

static double rhs_at(const fem_mesh* m, const double* x) {
  if (m->rhs_kind == 1) return 1.0;
  double v = m->dim * M_PI * M_PI;
  for (int a = 0; a < m->dim; ++a) v *= sin(M_PI * x[a]);
  return v;
}

/* multilinear cell map at reference point xi in [0,1]^d: position and Jacobian J[r][c] = dx_r/dxi_c */
static void cell_map(const fem_mesh* m, const int* c, const double* xi, double* x, double J[FEM_MAXD][FEM_MAXD]) {
  int d = m->dim, nv = 1 << d, V = m->N + 1;
  for (int r = 0; r < d; ++r) { x[r] = 0.0; for (int s = 0; s < d; ++s) J[r][s] = 0.0; }
  for (int v = 0; v < nv; ++v) {
    int vi = 0, stride = 1;
    double w = 1.0, dw[FEM_MAXD];
    for (int a = 0; a < d; ++a) {
      int bit = (v >> a) & 1;
      vi += (c[a] + bit) * stride; stride *= V;
    }
    for (int a = 0; a < d; ++a) {
      int bit = (v >> a) & 1;
      double f = bit ? xi[a] : 1.0 - xi[a];
      w *= f;
    }
    for (int s = 0; s < d; ++s) {
      double g = 1.0;
      for (int a = 0; a < d; ++a) {
        int bit = (v >> a) & 1;
        g *= (a == s) ? (bit ? 1.0 : -1.0) : (bit ? xi[a] : 1.0 - xi[a]);
      }
      dw[s] = g;
    }
    const double* X = m->vert + (size_t)vi * d;
    for (int r = 0; r < d; ++r) {
      x[r] += w * X[r];
      for (int s = 0; s < d; ++s) J[r][s] += dw[s] * X[r];
    }
  }
}

static double inv_det(int d, double J[FEM_MAXD][FEM_MAXD], double Ji[FEM_MAXD][FEM_MAXD]) {
  if (d == 2) {
    double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    Ji[0][0] = J[1][1] / det; Ji[0][1] = -J[0][1] / det; Ji[1][0] = -J[1][0] / det; Ji[1][1] = J[0][0] / det;
    return det;
  }
  double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
               J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  return det;
}

/* free index of a global node multi-index, or -1 on the boundary */
static int64_t free_index(const fem_mesh* m, const int* I) {
  int64_t f = 0, stride = 1;
  for (int a = 0; a < m->dim; ++a) {
    if (I[a] <= 0 || I[a] >= m->nodes1d - 1) return -1;
    f += (int64_t)(I[a] - 1) * stride; stride *= m->free1d;
  }
  return f;
}

/* 1-D coupling range of node i restricted to free nodes: [lo, lo+len) */
static void range1d(const fem_mesh* m, int i, int* lo, int* len) {
  int p = m->p, a, b;
  if (i % p == 0) { a = i - p; b = i + p; } else { a = p * (i / p); b = a + p; }
  if (a < 1) a = 1;
  if (b > m->nodes1d - 2) b = m->nodes1d - 2;
  *lo = a; *len = b - a + 1;
}

/* ------------------------------------------------------------------ API */

/* Sizes of the free system: returns n (free nodes) and nnz through pointers. */
int fem_sizes(int dim, int N, int p, int64_t* n_out, int64_t* nnz_out) {
  if (dim < 2 || dim > 3 || N < 1 || p < 1 || p > FEM_MAXP) return 1;
  fem_mesh m; memset(&m, 0, sizeof m);
  m.dim = dim; m.N = N; m.p = p; m.nodes1d = N * p + 1; m.free1d = N * p - 1;
  if (m.free1d < 1) { *n_out = 0; *nnz_out = 0; return 0; }
  int64_t n1 = m.free1d, nnz1 = 0;
  for (int i = 1; i <= m.free1d; ++i) { int lo, len; range1d(&m, i, &lo, &len); nnz1 += len; }
  int64_t n = 1, nnz = 1;
  for (int a = 0; a < dim; ++a) { n *= n1; nnz *= nnz1; }
  *n_out = n; *nnz_out = nnz;
  return 0;
}

/*
 * Assemble the free system.  Outputs (caller-allocated):
 *   coords[n*dim], rowptr[n+1], colidx[nnz], vals[nnz], rhs[n], uex[n] (exact
 *   manufactured solution at the free support points; zeros when rhs_kind=1).
 * perturb: interior vertices move by U(-perturb*h, perturb*h) per component.
 * nkappa: number of random Fourier modes in g = log kappa (unit variance);
 *   0 gives kappa = 1.
 */
int fem_assemble(int dim, int N, int p, double perturb, uint64_t seed, int nkappa, int rhs_kind,
                 double* coords, int64_t* rowptr, int32_t* colidx, double* vals, double* rhs, double* uex) {
  if (dim < 2 || dim > 3 || N < 1 || p < 1 || p > FEM_MAXP || nkappa < 0 || nkappa > 64) return 1;
  fem_mesh m; memset(&m, 0, sizeof m);
  m.dim = dim; m.N = N; m.p = p; m.nodes1d = N * p + 1; m.free1d = N * p - 1;
  m.rhs_kind = rhs_kind; m.nkappa = nkappa;
  gll01(p, m.gll);
  int V = N + 1; int64_t nvert = 1; for (int a = 0; a < dim; ++a) nvert *= V;
  m.vert = (double*)malloc(sizeof(double) * nvert * dim);
  if (!m.vert) return 2;
  uint64_t st = seed;
  double h = 1.0 / N;
  for (int64_t v = 0; v < nvert; ++v) {
    int64_t t = v; int interior = 1; int I[FEM_MAXD];
    for (int a = 0; a < dim; ++a) { I[a] = (int)(t % V); t /= V; if (I[a] == 0 || I[a] == N) interior = 0; }
    for (int a = 0; a < dim; ++a) m.vert[v * dim + a] = I[a] * h;
    if (interior && perturb > 0.0)
      for (int a = 0; a < dim; ++a) m.vert[v * dim + a] += (2.0 * sm64_unit(&st) - 1.0) * perturb * h;
  }
  if (nkappa > 0) {
    uint64_t ks = seed ^ 0x6b617070615f6d6fULL;
    m.kamp = sqrt(2.0 / nkappa);   /* Var g = nkappa * amp^2 / 2 = 1 */
    for (int k = 0; k < nkappa; ++k) {
      int nz;
      do {
        nz = 0;
        for (int a = 0; a < 3; ++a) { m.kwave[k][a] = (a < dim) ? (double)((int)(sm64_unit(&ks) * 9.0) - 4) : 0.0; nz |= (m.kwave[k][a] != 0.0); }
      } while (!nz);
      m.kphase[k] = 2.0 * M_PI * sm64_unit(&ks);
    }
  }
  int64_t n, nnz;
  fem_sizes(dim, N, p, &n, &nnz);
  int F = m.free1d;
  /* row pointers and column indices: tensor products of 1-D ranges, ascending */
  rowptr[0] = 0;
  for (int64_t f = 0; f < n; ++f) {
    int64_t t = f; int64_t len = 1;
    for (int a = 0; a < dim; ++a) { int i = (int)(t % F) + 1; t /= F; int lo, l; range1d(&m, i, &lo, &l); len *= l; }
    rowptr[f + 1] = rowptr[f] + len;
  }
  #pragma omp parallel for schedule(static)
  for (int64_t f = 0; f < n; ++f) {
    int64_t t = f; int lo[FEM_MAXD] = {0, 0, 0}, l[FEM_MAXD] = {1, 1, 1};
    for (int a = 0; a < dim; ++a) { int i = (int)(t % F) + 1; t /= F; range1d(&m, i, &lo[a], &l[a]); }
    int64_t k = rowptr[f];
    for (int c2 = 0; c2 < (dim == 3 ? l[2] : 1); ++c2)
      for (int c1 = 0; c1 < l[1]; ++c1)
        for (int c0 = 0; c0 < l[0]; ++c0) {
          int64_t col = (lo[0] + c0 - 1) + (int64_t)F * ((lo[1] + c1 - 1) + (int64_t)F * (dim == 3 ? (lo[2] + c2 - 1) : 0));
          colidx[k++] = (int32_t)col;
        }
  }
  memset(vals, 0, sizeof(double) * nnz);
  memset(rhs, 0, sizeof(double) * n);
  /* quadrature and 1-D basis tables */
  int q1 = p + 1, nb1 = p + 1;
  double gx[FEM_MAXP + 1], gw[FEM_MAXP + 1], L[FEM_MAXP + 1][FEM_MAXP + 1], dL[FEM_MAXP + 1][FEM_MAXP + 1];
  gauss_legendre01(q1, gx, gw);
  for (int q = 0; q < q1; ++q) lagrange1d(p, m.gll, gx[q], L[q], dL[q]);
  int nb = 1, nq = 1; for (int a = 0; a < dim; ++a) { nb *= nb1; nq *= q1; }
  int ncell_side = N; int64_t ncell = 1; for (int a = 0; a < dim; ++a) ncell *= ncell_side;
  for (int color = 0; color < (1 << dim); ++color) {
    #pragma omp parallel
    {
      double* K = (double*)malloc(sizeof(double) * nb * nb);
      double* Bq = (double*)malloc(sizeof(double) * nb * FEM_MAXD);
      double* Cq = (double*)malloc(sizeof(double) * nb * FEM_MAXD);
      double* Fl = (double*)malloc(sizeof(double) * nb);
      double* phi = (double*)malloc(sizeof(double) * nb);
      int64_t* gid = (int64_t*)malloc(sizeof(int64_t) * nb);
      int (*gI)[FEM_MAXD] = malloc(sizeof(int[FEM_MAXD]) * nb);
      #pragma omp for schedule(dynamic, 16)
      for (int64_t cidx = 0; cidx < ncell; ++cidx) {
        int c[FEM_MAXD] = {0, 0, 0}; int64_t t = cidx; int col = 0;
        for (int a = 0; a < dim; ++a) { c[a] = (int)(t % N); t /= N; col |= (c[a] & 1) << a; }
        if (col != color) continue;
        memset(K, 0, sizeof(double) * nb * nb); memset(Fl, 0, sizeof(double) * nb);
        for (int la = 0; la < nb; ++la) {
          int tt = la; int I[FEM_MAXD] = {0, 0, 0};
          for (int a = 0; a < dim; ++a) { I[a] = c[a] * p + tt % nb1; tt /= nb1; gI[la][a] = I[a]; }
          gid[la] = free_index(&m, I);
        }
        for (int q = 0; q < nq; ++q) {
          int qi[FEM_MAXD] = {0, 0, 0}; int tt = q; double xi[FEM_MAXD], w = 1.0;
          for (int a = 0; a < dim; ++a) { qi[a] = tt % q1; tt /= q1; xi[a] = gx[qi[a]]; w *= gw[qi[a]]; }
          double x[FEM_MAXD], J[FEM_MAXD][FEM_MAXD], Ji[FEM_MAXD][FEM_MAXD];
          cell_map(&m, c, xi, x, J);
          double det = inv_det(dim, J, Ji);
          double kap = kappa_at(&m, x);
          double G[FEM_MAXD][FEM_MAXD];
          for (int r = 0; r < dim; ++r)
            for (int s = 0; s < dim; ++s) {
              double g = 0.0;
              for (int k = 0; k < dim; ++k) g += Ji[r][k] * Ji[s][k];
              G[r][s] = g * w * det * kap;
            }
          for (int la = 0; la < nb; ++la) {
            int tt2 = la; int ai[FEM_MAXD] = {0, 0, 0};
            for (int a = 0; a < dim; ++a) { ai[a] = tt2 % nb1; tt2 /= nb1; }
            double v = 1.0;
            for (int a = 0; a < dim; ++a) v *= L[qi[a]][ai[a]];
            phi[la] = v;
            for (int s = 0; s < dim; ++s) {
              double g = 1.0;
              for (int a = 0; a < dim; ++a) g *= (a == s) ? dL[qi[a]][ai[a]] : L[qi[a]][ai[a]];
              Bq[la * FEM_MAXD + s] = g;
            }
            for (int r = 0; r < dim; ++r) {
              double g = 0.0;
              for (int s = 0; s < dim; ++s) g += G[r][s] * Bq[la * FEM_MAXD + s];
              Cq[la * FEM_MAXD + r] = g;
            }
          }
          double fq = rhs_at(&m, x) * w * det;
          for (int la = 0; la < nb; ++la) {
            Fl[la] += fq * phi[la];
            for (int lb = la; lb < nb; ++lb) {
              double s = 0.0;
              for (int r = 0; r < dim; ++r) s += Cq[la * FEM_MAXD + r] * Bq[lb * FEM_MAXD + r];
              K[la * nb + lb] += s;
            }
          }
        }
        for (int la = 0; la < nb; ++la)
          for (int lb = 0; lb < la; ++lb) K[la * nb + lb] = K[lb * nb + la];
        for (int la = 0; la < nb; ++la) {
          int64_t gi = gid[la];
          if (gi < 0) continue;
          rhs[gi] += Fl[la];
          int lo[FEM_MAXD] = {0, 0, 0}, l[FEM_MAXD] = {1, 1, 1};
          for (int a = 0; a < dim; ++a) range1d(&m, gI[la][a], &lo[a], &l[a]);
          for (int lb = 0; lb < nb; ++lb) {
            if (gid[lb] < 0) continue;
            int64_t off = 0, str = 1;
            for (int a = 0; a < dim; ++a) { off += (gI[lb][a] - lo[a]) * str; str *= l[a]; }
            vals[rowptr[gi] + off] += K[la * nb + lb];
          }
        }
      }
      free(K); free(Bq); free(Cq); free(Fl); free(phi); free(gid); free(gI);
    }
  }
  /* support-point coordinates of free nodes, exact solution */
  #pragma omp parallel for schedule(static)
  for (int64_t f = 0; f < n; ++f) {
    int64_t t = f; int I[FEM_MAXD] = {0, 0, 0}, c[FEM_MAXD] = {0, 0, 0}; double xi[FEM_MAXD] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) {
      I[a] = (int)(t % F) + 1; t /= F;
      c[a] = I[a] / p; if (c[a] >= N) c[a] = N - 1;
      xi[a] = m.gll[I[a] - c[a] * p];
    }
    double x[FEM_MAXD], J[FEM_MAXD][FEM_MAXD];
    cell_map(&m, c, xi, x, J);
    double u = 1.0;
    for (int a = 0; a < dim; ++a) { coords[f * dim + a] = x[a]; u *= sin(M_PI * x[a]); }
    uex[f] = (rhs_kind == 0) ? u : 0.0;
  }
  free(m.vert);
  return 0;
}

/*
 * L2 error || u_h - u_exact || of a free-node coefficient vector for the
 * manufactured solution u = prod sin(pi x_a), integrated with a tensor
 * Gauss-Legendre rule of p+3 points per direction on each mapped cell.
 * The mesh is regenerated from (dim, N, p, perturb, seed).
 */
double fem_l2_error(int dim, int N, int p, double perturb, uint64_t seed, const double* u_free) {
  fem_mesh m; memset(&m, 0, sizeof m);
  m.dim = dim; m.N = N; m.p = p; m.nodes1d = N * p + 1; m.free1d = N * p - 1;
  gll01(p, m.gll);
  int V = N + 1; int64_t nvert = 1; for (int a = 0; a < dim; ++a) nvert *= V;
  m.vert = (double*)malloc(sizeof(double) * nvert * dim);
  uint64_t st = seed; double h = 1.0 / N;
  for (int64_t v = 0; v < nvert; ++v) {
    int64_t t = v; int interior = 1; int I[FEM_MAXD];
    for (int a = 0; a < dim; ++a) { I[a] = (int)(t % V); t /= V; if (I[a] == 0 || I[a] == N) interior = 0; }
    for (int a = 0; a < dim; ++a) m.vert[v * dim + a] = I[a] * h;
    if (interior && perturb > 0.0)
      for (int a = 0; a < dim; ++a) m.vert[v * dim + a] += (2.0 * sm64_unit(&st) - 1.0) * perturb * h;
  }
  int q1 = p + 3, nb1 = p + 1;
  double gx[FEM_MAXP + 4], gw[FEM_MAXP + 4], L[FEM_MAXP + 4][FEM_MAXP + 1], dL[FEM_MAXP + 4][FEM_MAXP + 1];
  gauss_legendre01(q1, gx, gw);
  for (int q = 0; q < q1; ++q) lagrange1d(p, m.gll, gx[q], L[q], dL[q]);
  int nb = 1, nq = 1; for (int a = 0; a < dim; ++a) { nb *= nb1; nq *= q1; }
  int64_t ncell = 1; for (int a = 0; a < dim; ++a) ncell *= N;
  double err2 = 0.0;
  #pragma omp parallel for reduction(+ : err2) schedule(static)
  for (int64_t cidx = 0; cidx < ncell; ++cidx) {
    int c[FEM_MAXD] = {0, 0, 0}; int64_t t = cidx;
    for (int a = 0; a < dim; ++a) { c[a] = (int)(t % N); t /= N; }
    for (int q = 0; q < nq; ++q) {
      int qi[FEM_MAXD] = {0, 0, 0}; int tt = q; double xi[FEM_MAXD], w = 1.0;
      for (int a = 0; a < dim; ++a) { qi[a] = tt % q1; tt /= q1; xi[a] = gx[qi[a]]; w *= gw[qi[a]]; }
      double x[FEM_MAXD], J[FEM_MAXD][FEM_MAXD], Ji[FEM_MAXD][FEM_MAXD];
      cell_map(&m, c, xi, x, J);
      double det = inv_det(dim, J, Ji);
      double uh = 0.0;
      for (int la = 0; la < nb; ++la) {
        int tt2 = la; int I[FEM_MAXD] = {0, 0, 0}; double v = 1.0;
        for (int a = 0; a < dim; ++a) { int ai = tt2 % nb1; tt2 /= nb1; I[a] = c[a] * p + ai; v *= L[qi[a]][ai]; }
        int64_t gi = free_index(&m, I);
        if (gi >= 0) uh += v * u_free[gi];
      }
      double u = 1.0;
      for (int a = 0; a < dim; ++a) u *= sin(M_PI * x[a]);
      err2 += (uh - u) * (uh - u) * w * det;
    }
  }
  free(m.vert);
  return sqrt(err2);
}

/* GLL nodes on [0,1] (exported for tests of this generator). */
void fem_gll01(int p, double* x) { gll01(p, x); }

/* ================================================================== P_p simplices
 *
 * Continuous P_p Lagrange elements on the Kuhn (Freudenthal) triangulation of the structured
 * mesh: every cell [c, c+1]^d (in cell units) is split into d! simplices, one per permutation
 * pi of the axes, with vertices v_0 = 0 and v_k = v_{k-1} + e_{pi(k-1)}; the splitting is the
 * same in every cell, so the triangulation is conforming.  Each simplex is the affine image of
 * the reference simplex {xi >= 0, sum xi <= 1} under its (possibly perturbed) vertices.  The
 * nodes of P_p are the barycentric lattice points alpha/p, |alpha| <= p; in lattice units a
 * node of the simplex in cell c sits at c p + sum_k alpha_k (v_k - v_0), so the nodes of all
 * simplices are exactly the (N p + 1)^d grid, numbered and eliminated as for Q_p.  Node
 * positions are the affine images (straight-sided simplices).
 * Basis: the monomials xi^beta, |beta| <= p, combined by the inverse Vandermonde matrix of the
 * lattice nodes.  Quadrature: collapsed (Duffy) Gauss-Legendre rules, q points per direction.
 * Assembly runs over the simplices in a fixed order on one thread, upper triangle mirrored, so
 * the matrix is bitwise symmetric and deterministic.
 */
#define SX_MAXNB 35   /* C(p+d, d) for p <= 4, d <= 3 */

typedef struct {
  int d, p, nb;
  int alpha[SX_MAXNB][FEM_MAXD];   /* lattice nodes (and monomial exponents, same set) */
  double C[SX_MAXNB][SX_MAXNB];    /* phi_a = sum_m C[m][a] xi^beta_m */
} sx_basis;

static int sx_lattice(int d, int p, int (*al)[FEM_MAXD]) {
  int n = 0;
  for (int k = 0; k <= (d == 3 ? p : 0); ++k)
    for (int j = 0; j <= p - k; ++j)
      for (int i = 0; i <= p - k - j; ++i) {
        al[n][0] = i; al[n][1] = j; al[n][2] = (d == 3) ? k : 0;
        ++n;
      }
  return n;
}

static double sx_mono(int d, const int* beta, const double* xi) {
  double v = 1.0;
  for (int a = 0; a < d; ++a)
    for (int e = 0; e < beta[a]; ++e) v *= xi[a];
  return v;
}

/* d/dxi_k of xi^beta */
static double sx_dmono(int d, const int* beta, const double* xi, int k) {
  if (beta[k] == 0) return 0.0;
  double v = (double)beta[k];
  for (int a = 0; a < d; ++a) {
    int e = beta[a] - (a == k ? 1 : 0);
    for (int t = 0; t < e; ++t) v *= xi[a];
  }
  return v;
}

/* inverse Vandermonde by Gauss-Jordan elimination with partial pivoting; 0 on success */
static int sx_build(sx_basis* B, int d, int p) {
  B->d = d; B->p = p;
  B->nb = sx_lattice(d, p, B->alpha);
  int n = B->nb;
  double V[SX_MAXNB][2 * SX_MAXNB];
  for (int r = 0; r < n; ++r) {
    double xi[FEM_MAXD];
    for (int a = 0; a < d; ++a) xi[a] = (double)B->alpha[r][a] / p;
    for (int m = 0; m < n; ++m) V[r][m] = sx_mono(d, B->alpha[m], xi);
    for (int m = 0; m < n; ++m) V[r][n + m] = (r == m) ? 1.0 : 0.0;
  }
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r) if (fabs(V[r][c]) > fabs(V[piv][c])) piv = r;
    if (fabs(V[piv][c]) < 1e-14) return 1;
    if (piv != c) for (int m = 0; m < 2 * n; ++m) { double t = V[c][m]; V[c][m] = V[piv][m]; V[piv][m] = t; }
    double s = 1.0 / V[c][c];
    for (int m = 0; m < 2 * n; ++m) V[c][m] *= s;
    for (int r = 0; r < n; ++r) {
      if (r == c || V[r][c] == 0.0) continue;
      double f = V[r][c];
      for (int m = 0; m < 2 * n; ++m) V[r][m] -= f * V[c][m];
    }
  }
  /* V (node x monomial) times C = I  =>  C = V^-1 (monomial x node) */
  for (int m = 0; m < n; ++m)
    for (int a = 0; a < n; ++a) B->C[m][a] = V[m][n + a];
  return 0;
}

/* collapsed Gauss rule on the reference simplex: q^d points; returns the count */
static int sx_quad(int d, int q, double (*xq)[FEM_MAXD], double* wq) {
  double gx[FEM_MAXP + 8], gw[FEM_MAXP + 8];
  gauss_legendre01(q, gx, gw);
  int n = 0;
  if (d == 2) {
    for (int i = 0; i < q; ++i)
      for (int j = 0; j < q; ++j) {
        double u = gx[i], v = gx[j];
        xq[n][0] = u; xq[n][1] = v * (1.0 - u); xq[n][2] = 0.0;
        wq[n] = gw[i] * gw[j] * (1.0 - u);
        ++n;
      }
  } else {
    for (int i = 0; i < q; ++i)
      for (int j = 0; j < q; ++j)
        for (int k = 0; k < q; ++k) {
          double u = gx[i], v = gx[j], w = gx[k];
          xq[n][0] = u; xq[n][1] = v * (1.0 - u); xq[n][2] = w * (1.0 - u) * (1.0 - v);
          wq[n] = gw[i] * gw[j] * gw[k] * (1.0 - u) * (1.0 - u) * (1.0 - v);
          ++n;
        }
  }
  return n;
}

/* the d! Kuhn simplices of the unit cube: vertex offsets kv[s][0..d][axis] */
static int sx_kuhn(int d, int (*kv)[FEM_MAXD + 1][FEM_MAXD]) {
  int perm3[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  int perm2[2][3] = {{0, 1, 0}, {1, 0, 0}};
  int ns = (d == 3) ? 6 : 2;
  for (int s = 0; s < ns; ++s) {
    const int* pi = (d == 3) ? perm3[s] : perm2[s];
    for (int a = 0; a < FEM_MAXD; ++a) kv[s][0][a] = 0;
    for (int k = 1; k <= d; ++k) {
      for (int a = 0; a < FEM_MAXD; ++a) kv[s][k][a] = kv[s][k - 1][a];
      kv[s][k][pi[k - 1]] += 1;
    }
  }
  return ns;
}

static void sx_mesh(fem_mesh* m, int dim, int N, int p, double perturb, uint64_t seed) {
  memset(m, 0, sizeof *m);
  m->dim = dim; m->N = N; m->p = p; m->nodes1d = N * p + 1; m->free1d = N * p - 1;
  int V = N + 1; int64_t nvert = 1; for (int a = 0; a < dim; ++a) nvert *= V;
  m->vert = (double*)malloc(sizeof(double) * nvert * dim);
  uint64_t st = seed;
  double h = 1.0 / N;
  for (int64_t v = 0; v < nvert; ++v) {
    int64_t t = v; int interior = 1; int I[FEM_MAXD];
    for (int a = 0; a < dim; ++a) { I[a] = (int)(t % V); t /= V; if (I[a] == 0 || I[a] == N) interior = 0; }
    for (int a = 0; a < dim; ++a) m->vert[v * dim + a] = I[a] * h;
    if (interior && perturb > 0.0)
      for (int a = 0; a < dim; ++a) m->vert[v * dim + a] += (2.0 * sm64_unit(&st) - 1.0) * perturb * h;
  }
}

static const double* sx_vertex(const fem_mesh* m, const int* c, const int* off) {
  int64_t vi = 0, stride = 1;
  for (int a = 0; a < m->dim; ++a) { vi += (int64_t)(c[a] + off[a]) * stride; stride *= (m->N + 1); }
  return m->vert + vi * m->dim;
}

typedef struct { int64_t row, col; } sx_pair;
static int sx_pair_cmp(const void* x, const void* y) {
  const sx_pair* a = (const sx_pair*)x; const sx_pair* b = (const sx_pair*)y;
  if (a->row != b->row) return a->row < b->row ? -1 : 1;
  if (a->col != b->col) return a->col < b->col ? -1 : 1;
  return 0;
}

/* visit every simplex: cell c, simplex s, its node multi-indices gI[nb][d] and free ids gid[nb] */
#define SX_FOR_SIMPLICES(m, ns, kv, B, ...)                                                     \
  do {                                                                                          \
    int64_t ncell_ = 1; for (int a_ = 0; a_ < (m)->dim; ++a_) ncell_ *= (m)->N;                 \
    for (int64_t cidx_ = 0; cidx_ < ncell_; ++cidx_) {                                          \
      int c[FEM_MAXD] = {0, 0, 0}; int64_t t_ = cidx_;                                          \
      for (int a_ = 0; a_ < (m)->dim; ++a_) { c[a_] = (int)(t_ % (m)->N); t_ /= (m)->N; }        \
      for (int s = 0; s < (ns); ++s) {                                                          \
        int gI[SX_MAXNB][FEM_MAXD]; int64_t gid[SX_MAXNB];                                      \
        for (int la = 0; la < (B).nb; ++la) {                                                   \
          for (int a_ = 0; a_ < (m)->dim; ++a_) {                                               \
            int v_ = c[a_] * (m)->p;                                                            \
            for (int k_ = 1; k_ <= (m)->dim; ++k_) v_ += (B).alpha[la][k_ - 1] * ((kv)[s][k_][a_] - (kv)[s][0][a_]); \
            gI[la][a_] = v_;                                                                    \
          }                                                                                     \
          gid[la] = free_index((m), gI[la]);                                                    \
        }                                                                                       \
        __VA_ARGS__                                                                             \
      }                                                                                         \
    }                                                                                           \
  } while (0)

/* Sizes of the free P_p system (n free nodes, nnz of the coupling pattern). */
int fem_simplex_sizes(int dim, int N, int p, int64_t* n_out, int64_t* nnz_out) {
  if (dim < 2 || dim > 3 || N < 1 || p < 1 || p > (dim == 3 ? 3 : 4)) return 1;
  fem_mesh m; memset(&m, 0, sizeof m);
  m.dim = dim; m.N = N; m.p = p; m.nodes1d = N * p + 1; m.free1d = N * p - 1;
  sx_basis B;
  if (sx_build(&B, dim, p)) return 3;
  int kv[6][FEM_MAXD + 1][FEM_MAXD];
  int ns = sx_kuhn(dim, kv);
  int64_t n = 1; for (int a = 0; a < dim; ++a) n *= (m.free1d > 0 ? m.free1d : 0);
  int64_t ncell = 1; for (int a = 0; a < dim; ++a) ncell *= N;
  int64_t cap = ncell * ns * B.nb * B.nb, np = 0;
  sx_pair* P = (sx_pair*)malloc(sizeof(sx_pair) * (cap > 0 ? cap : 1));
  if (!P) return 2;
  SX_FOR_SIMPLICES(&m, ns, kv, B, {
    for (int la = 0; la < B.nb; ++la) {
      if (gid[la] < 0) continue;
      for (int lb = 0; lb < B.nb; ++lb)
        if (gid[lb] >= 0) { P[np].row = gid[la]; P[np].col = gid[lb]; ++np; }
    }
  });
  qsort(P, (size_t)np, sizeof(sx_pair), sx_pair_cmp);
  int64_t nnz = 0;
  for (int64_t k = 0; k < np; ++k)
    if (k == 0 || sx_pair_cmp(&P[k], &P[k - 1]) != 0) ++nnz;
  free(P);
  *n_out = n; *nnz_out = nnz;
  return 0;
}

/*
 * Assemble the free P_p system on the Kuhn triangulation (outputs as fem_assemble; kappa = 1).
 * perturb: interior vertices move by U(-perturb*h, perturb*h) per component (same generator
 * and order as the Q_p meshes).  rhs_kind 0: manufactured u = prod sin(pi x_a); 1: f = 1.
 */
int fem_simplex_assemble(int dim, int N, int p, double perturb, uint64_t seed, int rhs_kind, double* coords,
                         int64_t* rowptr, int32_t* colidx, double* vals, double* rhs, double* uex) {
  int64_t n, nnz;
  int rc = fem_simplex_sizes(dim, N, p, &n, &nnz);
  if (rc) return rc;
  fem_mesh m;
  sx_mesh(&m, dim, N, p, perturb, seed);
  if (!m.vert) return 2;
  m.rhs_kind = rhs_kind;
  sx_basis B;
  sx_build(&B, dim, p);
  int kv[6][FEM_MAXD + 1][FEM_MAXD];
  int ns = sx_kuhn(dim, kv);
  /* pattern: sorted unique (row, col) pairs of nodes sharing a simplex */
  int64_t ncell = 1; for (int a = 0; a < dim; ++a) ncell *= N;
  int64_t cap = ncell * ns * B.nb * B.nb, np = 0;
  sx_pair* P = (sx_pair*)malloc(sizeof(sx_pair) * (cap > 0 ? cap : 1));
  if (!P) { free(m.vert); return 2; }
  SX_FOR_SIMPLICES(&m, ns, kv, B, {
    for (int la = 0; la < B.nb; ++la) {
      if (gid[la] < 0) continue;
      for (int lb = 0; lb < B.nb; ++lb)
        if (gid[lb] >= 0) { P[np].row = gid[la]; P[np].col = gid[lb]; ++np; }
    }
  });
  qsort(P, (size_t)np, sizeof(sx_pair), sx_pair_cmp);
  for (int64_t f = 0; f <= n; ++f) rowptr[f] = 0;
  int64_t k = 0;
  for (int64_t t = 0; t < np; ++t) {
    if (t > 0 && sx_pair_cmp(&P[t], &P[t - 1]) == 0) continue;
    colidx[k++] = (int32_t)P[t].col;
    rowptr[P[t].row + 1] += 1;
  }
  free(P);
  for (int64_t f = 0; f < n; ++f) rowptr[f + 1] += rowptr[f];
  memset(vals, 0, sizeof(double) * nnz);
  memset(rhs, 0, sizeof(double) * n);
  for (int64_t f = 0; f < n; ++f) { coords[f * dim] = NAN; }
  /* quadrature tables on the reference simplex */
  int q = p + 2;
  static double xq[(FEM_MAXP + 8) * (FEM_MAXP + 8) * (FEM_MAXP + 8)][FEM_MAXD];
  static double wq[(FEM_MAXP + 8) * (FEM_MAXP + 8) * (FEM_MAXP + 8)];
  int nq = sx_quad(dim, q, xq, wq);
  double* phi = (double*)malloc(sizeof(double) * nq * B.nb);
  double* dphi = (double*)malloc(sizeof(double) * nq * B.nb * FEM_MAXD);
  for (int iq = 0; iq < nq; ++iq)
    for (int la = 0; la < B.nb; ++la) {
      double v = 0.0, g[FEM_MAXD] = {0, 0, 0};
      for (int mo = 0; mo < B.nb; ++mo) {
        v += B.C[mo][la] * sx_mono(dim, B.alpha[mo], xq[iq]);
        for (int kk = 0; kk < dim; ++kk) g[kk] += B.C[mo][la] * sx_dmono(dim, B.alpha[mo], xq[iq], kk);
      }
      phi[iq * B.nb + la] = v;
      for (int kk = 0; kk < dim; ++kk) dphi[(iq * B.nb + la) * FEM_MAXD + kk] = g[kk];
    }
  double K[SX_MAXNB][SX_MAXNB], Fl[SX_MAXNB];
  SX_FOR_SIMPLICES(&m, ns, kv, B, {
    /* affine map: x = X0 + J xi, J[r][k] = X_k[r] - X0[r] */
    const double* X0 = sx_vertex(&m, c, kv[s][0]);
    double J[FEM_MAXD][FEM_MAXD] = {{0}}, Ji[FEM_MAXD][FEM_MAXD];
    for (int kk = 1; kk <= dim; ++kk) {
      const double* Xk = sx_vertex(&m, c, kv[s][kk]);
      for (int r = 0; r < dim; ++r) J[r][kk - 1] = Xk[r] - X0[r];
    }
    double det = fabs(inv_det(dim, J, Ji));
    memset(K, 0, sizeof K); memset(Fl, 0, sizeof Fl);
    for (int iq = 0; iq < nq; ++iq) {
      double x[FEM_MAXD];
      for (int r = 0; r < dim; ++r) { x[r] = X0[r]; for (int kk = 0; kk < dim; ++kk) x[r] += J[r][kk] * xq[iq][kk]; }
      double w = wq[iq] * det;
      double gx[SX_MAXNB][FEM_MAXD];   /* physical gradients: grad_x = Ji^T grad_xi */
      for (int la = 0; la < B.nb; ++la)
        for (int r = 0; r < dim; ++r) {
          double g = 0.0;
          for (int kk = 0; kk < dim; ++kk) g += Ji[kk][r] * dphi[(iq * B.nb + la) * FEM_MAXD + kk];
          gx[la][r] = g;
        }
      double fq = rhs_at(&m, x) * w;
      for (int la = 0; la < B.nb; ++la) {
        Fl[la] += fq * phi[iq * B.nb + la];
        for (int lb = la; lb < B.nb; ++lb) {
          double sdot = 0.0;
          for (int r = 0; r < dim; ++r) sdot += gx[la][r] * gx[lb][r];
          K[la][lb] += sdot * w;
        }
      }
    }
    for (int la = 0; la < B.nb; ++la)
      for (int lb = 0; lb < la; ++lb) K[la][lb] = K[lb][la];
    for (int la = 0; la < B.nb; ++la) {
      int64_t gi = gid[la];
      if (gi < 0) continue;
      rhs[gi] += Fl[la];
      if (isnan(coords[gi * dim])) {   /* the node's position: the affine image of its lattice point */
        for (int r = 0; r < dim; ++r) {
          double v = X0[r];
          for (int kk = 0; kk < dim; ++kk) v += J[r][kk] * ((double)B.alpha[la][kk] / p);
          coords[gi * dim + r] = v;
        }
      }
      for (int lb = 0; lb < B.nb; ++lb) {
        int64_t gj = gid[lb];
        if (gj < 0) continue;
        int64_t lo = rowptr[gi], hi = rowptr[gi + 1] - 1;   /* binary search of column gj */
        while (lo < hi) { int64_t mid = (lo + hi) / 2; if (colidx[mid] < gj) lo = mid + 1; else hi = mid; }
        vals[lo] += K[la][lb];
      }
    }
  });
  for (int64_t f = 0; f < n; ++f) {
    double u = 1.0;
    for (int a = 0; a < dim; ++a) u *= sin(M_PI * coords[f * dim + a]);
    uex[f] = (rhs_kind == 0) ? u : 0.0;
  }
  free(phi); free(dphi); free(m.vert);
  return 0;
}

/* L2 error of a free-node coefficient vector against u = prod sin(pi x_a) (rule with q = p + 3). */
double fem_simplex_l2_error(int dim, int N, int p, double perturb, uint64_t seed, const double* u_free) {
  fem_mesh m;
  sx_mesh(&m, dim, N, p, perturb, seed);
  sx_basis B;
  if (sx_build(&B, dim, p)) { free(m.vert); return NAN; }
  int kv[6][FEM_MAXD + 1][FEM_MAXD];
  int ns = sx_kuhn(dim, kv);
  static double xq[(FEM_MAXP + 8) * (FEM_MAXP + 8) * (FEM_MAXP + 8)][FEM_MAXD];
  static double wq[(FEM_MAXP + 8) * (FEM_MAXP + 8) * (FEM_MAXP + 8)];
  int nq = sx_quad(dim, p + 3, xq, wq);
  double err2 = 0.0;
  SX_FOR_SIMPLICES(&m, ns, kv, B, {
    const double* X0 = sx_vertex(&m, c, kv[s][0]);
    double J[FEM_MAXD][FEM_MAXD] = {{0}}, Ji[FEM_MAXD][FEM_MAXD];
    for (int kk = 1; kk <= dim; ++kk) {
      const double* Xk = sx_vertex(&m, c, kv[s][kk]);
      for (int r = 0; r < dim; ++r) J[r][kk - 1] = Xk[r] - X0[r];
    }
    double det = fabs(inv_det(dim, J, Ji));
    for (int iq = 0; iq < nq; ++iq) {
      double x[FEM_MAXD], uh = 0.0, u = 1.0;
      for (int r = 0; r < dim; ++r) { x[r] = X0[r]; for (int kk = 0; kk < dim; ++kk) x[r] += J[r][kk] * xq[iq][kk]; }
      for (int la = 0; la < B.nb; ++la) {
        if (gid[la] < 0) continue;
        double v = 0.0;
        for (int mo = 0; mo < B.nb; ++mo) v += B.C[mo][la] * sx_mono(dim, B.alpha[mo], xq[iq]);
        uh += v * u_free[gid[la]];
      }
      for (int a = 0; a < dim; ++a) u *= sin(M_PI * x[a]);
      err2 += (uh - u) * (uh - u) * wq[iq] * det;
    }
  });
  free(m.vert);
  return sqrt(err2);
}
