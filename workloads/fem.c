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
