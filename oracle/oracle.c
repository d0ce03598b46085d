/*
 * oracle.c -- plain FP64 CPU oracle for the matrix-free Poisson element
 * operator (AxLocal, CEED BK5) of Cao, Sun, Zhang, Li, "Towards a Higher
 * Roofline for Matrix-Vector Multiplication in Matrix-Free HOSFEM"
 * (arXiv 2504.07042), and for the steps around it (gather-scatter, CG).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code with the CUDA library.
 *
 * Every routine is the plain definition the paper states, written for
 * readability, not speed: no blocking, no fusion, no reordering beyond the
 * paper's own loops.  Element loops are OpenMP-parallel (each element is an
 * independent problem, Algorithm 1's e-loop), nothing else is.
 *
 * Conventions (all from Sec. 2):
 *   N1 = N+1, n3 = N1^3.
 *   Node [i,j,k] of an element is entry i + j*N1 + k*N1^2 (Algorithm 1 text).
 *   Reference coordinates of node [i,j,k]: (r,s,t) = (xi_i, xi_j, xi_k).
 *   Vertex matrix V (8x3, row-major) in the Kronecker order of Eq. 8:
 *     vertex index v = a + 2b + 4c, where a/b/c pick (1-r,1+r)/(1-s,1+s)/(1-t,1+t).
 *   Jacobian J[c][d] = d x_c / d ref_d (Eq. 5), stored row-major J[3*c+d].
 *   Geometric factors per node, 7 values in the order
 *     g00 g01 g02 g11 g12 g22 gwj  (Eq. 3 / Eq. 7), stored [E][7][n3].
 *
 * Parity status: every exported function is pinned by tests in
 * tests/test_oracle_*.py (see the header of each test module).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ------------------------------------------------------------------------
 * GLL constants (Table 1).
 *   L_N: Legendre polynomial, evaluated by Bonnet's recurrence
 *        (n+1) L_{n+1} = (2n+1) x L_n - n L_{n-1}.
 *   GLL points: zeros of (1-x^2) L_N'(x), i.e. -1, +1 and the N-1 roots of
 *        L_N', found by Newton's method in long double.
 *   Weights: w_i = 2 / (N (N+1) L_N(xi_i)^2).
 *   D[i][j] = pi_j'(xi_i): the textbook closed form of the derivative of the
 *        GLL Lagrange basis at the nodes,
 *          D[i][j] = L_N(xi_i) / (L_N(xi_j) (xi_i - xi_j)),   i != j,
 *          D[0][0] = -N(N+1)/4,  D[N][N] = +N(N+1)/4,  D[i][i] = 0 otherwise.
 * ---------------------------------------------------------------------- */
static void legendre_ld(int N, long double x, long double *L, long double *dL) {
  long double p0 = 1.0L, p1 = x, dp0 = 0.0L, dp1 = 1.0L;
  if (N == 0) { *L = 1.0L; *dL = 0.0L; return; }
  for (int n = 1; n < N; ++n) {
    long double p2 = ((2 * n + 1) * x * p1 - n * p0) / (n + 1);
    /* derivative of the recurrence: (n+1) L'_{n+1} = (2n+1)(L_n + x L'_n) - n L'_{n-1} */
    long double dp2 = ((2 * n + 1) * (p1 + x * dp1) - n * dp0) / (n + 1);
    p0 = p1; p1 = p2; dp0 = dp1; dp1 = dp2;
  }
  *L = p1; *dL = dp1;
}

int orc_gll(int N, double *xi, double *w, double *D) {
  if (N < 1 || N > 64) return 1;
  const int N1 = N + 1;
  long double x[65];
  x[0] = -1.0L; x[N] = 1.0L;
  for (int i = 1; i < N; ++i) {
    /* initial guess: Chebyshev-Gauss-Lobatto point; Newton on f = L_N' with
       f' = L_N'' from the Legendre equation (1-x^2) L'' = 2x L' - N(N+1) L */
    long double z = -cosl(3.14159265358979323846264338327950288L * i / N);
    for (int it = 0; it < 100; ++it) {
      long double L, dL;
      legendre_ld(N, z, &L, &dL);
      long double d2L = (2.0L * z * dL - (long double)N * (N + 1) * L) / (1.0L - z * z);
      long double dz = dL / d2L;
      z -= dz;
      if (fabsl(dz) < 1e-30L) break;
    }
    x[i] = z;
  }
  long double LN[65];
  for (int i = 0; i < N1; ++i) {
    long double L, dL;
    legendre_ld(N, x[i], &L, &dL);
    LN[i] = L;
  }
  for (int i = 0; i < N1; ++i) {
    xi[i] = (double)x[i];
    w[i] = (double)(2.0L / ((long double)N * (N + 1) * LN[i] * LN[i]));
  }
  for (int i = 0; i < N1; ++i)
    for (int j = 0; j < N1; ++j) {
      long double d;
      if (i != j) d = LN[i] / (LN[j] * (x[i] - x[j]));
      else if (i == 0) d = -(long double)N * (N + 1) / 4.0L;
      else if (i == N) d = (long double)N * (N + 1) / 4.0L;
      else d = 0.0L;
      D[i * N1 + j] = (double)d;
    }
  return 0;
}

/* ------------------------------------------------------------------------
 * Trilinear map (Eq. 8) and its Jacobian (Eq. 9), evaluated literally:
 * Kronecker rows of length 8 times the 8x3 vertex matrix, times 1/8.
 * This is the 144-flop direct form that Sec. 3.3 calls impractical for a
 * kernel; it is the definition, so the oracle uses it.
 * ---------------------------------------------------------------------- */
static void kron3(const double c2[2], const double c1[2], const double c0[2], double out[8]) {
  /* (c2) (x) (c1) (x) (c0): entry index 4*p + 2*q + m */
  for (int p = 0; p < 2; ++p)
    for (int q = 0; q < 2; ++q)
      for (int m = 0; m < 2; ++m) out[4 * p + 2 * q + m] = c2[p] * c1[q] * c0[m];
}

void orc_trilinear_map(const double *V, double r, double s, double t, double X[3]) {
  const double tv[2] = {1.0 - t, 1.0 + t}, sv[2] = {1.0 - s, 1.0 + s}, rv[2] = {1.0 - r, 1.0 + r};
  double row[8];
  kron3(tv, sv, rv, row);
  for (int c = 0; c < 3; ++c) {
    double acc = 0.0;
    for (int v = 0; v < 8; ++v) acc += row[v] * V[3 * v + c];
    X[c] = acc / 8.0;
  }
}

void orc_jacobian_trilinear(const double *V, double r, double s, double t, double J[9]) {
  const double tv[2] = {1.0 - t, 1.0 + t}, sv[2] = {1.0 - s, 1.0 + s}, rv[2] = {1.0 - r, 1.0 + r};
  const double dv[2] = {-1.0, 1.0};
  double row[3][8];
  kron3(tv, sv, dv, row[0]); /* d/dr */
  kron3(tv, dv, rv, row[1]); /* d/ds */
  kron3(dv, sv, rv, row[2]); /* d/dt */
  for (int d = 0; d < 3; ++d)
    for (int c = 0; c < 3; ++c) {
      double acc = 0.0;
      for (int v = 0; v < 8; ++v) acc += row[d][v] * V[3 * v + c];
      J[3 * c + d] = acc / 8.0; /* transpose: column d holds d Phi / d ref_d */
    }
}

/* ------------------------------------------------------------------------
 * Geometric factors of one node (Eq. 7):
 *   G = W |J| J^{-1} J^{-T}  (symmetric 3x3; six entries)  and  gwj = W |J|,
 * with W = w_i w_j w_k.  J^{-1} by the textbook cofactor formula.
 * Returns det J.
 * ---------------------------------------------------------------------- */
double orc_factors_from_jacobian(const double J[9], double W, double g[7]) {
  const double a = J[0], b = J[1], c = J[2], d = J[3], e = J[4], f = J[5], gg = J[6], h = J[7], k = J[8];
  const double det = a * (e * k - f * h) - b * (d * k - f * gg) + c * (d * h - e * gg);
  double inv[9];
  inv[0] = (e * k - f * h) / det;
  inv[1] = (c * h - b * k) / det;
  inv[2] = (b * f - c * e) / det;
  inv[3] = (f * gg - d * k) / det;
  inv[4] = (a * k - c * gg) / det;
  inv[5] = (c * d - a * f) / det;
  inv[6] = (d * h - e * gg) / det;
  inv[7] = (b * gg - a * h) / det;
  inv[8] = (a * e - b * d) / det;
  double M[9]; /* J^{-1} J^{-T} */
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < 3; ++q) {
      double acc = 0.0;
      for (int m = 0; m < 3; ++m) acc += inv[3 * p + m] * inv[3 * q + m];
      M[3 * p + q] = acc;
    }
  const double s = W * det;
  g[0] = s * M[0]; g[1] = s * M[1]; g[2] = s * M[2];
  g[3] = s * M[4]; g[4] = s * M[5]; g[5] = s * M[8];
  g[6] = s;
  return det;
}

/* Factors of the n3 nodes of one element from its vertices, J from Eq. 9. */
static int64_t factors_eq9_one(int N1, const double *xi, const double *w, const double *Ve, double *Ge) {
  const int n3 = N1 * N1 * N1;
  int64_t bad = 0;
  for (int k = 0; k < N1; ++k)
    for (int j = 0; j < N1; ++j)
      for (int i = 0; i < N1; ++i) {
        const int l = i + j * N1 + k * N1 * N1;
        double J[9], g[7];
        orc_jacobian_trilinear(Ve, xi[i], xi[j], xi[k], J);
        double det = orc_factors_from_jacobian(J, w[i] * w[j] * w[k], g);
        if (!(det > 0.0)) ++bad;
        for (int q = 0; q < 7; ++q) Ge[(int64_t)q * n3 + l] = g[q];
      }
  return bad;
}

/* Factors of all nodes of E trilinear elements, [E][7][n3].
 * Returns the number of nodes with det J <= 0, or -1 for a bad N. */
int64_t orc_factors_eq9(int64_t E, int N, const double *V, double *G) {
  const int N1 = N + 1, n3 = N1 * N1 * N1;
  double xi[65], w[65], D[65 * 65];
  if (orc_gll(N, xi, w, D)) return -1;
  int64_t bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
  for (int64_t e = 0; e < E; ++e) bad += factors_eq9_one(N1, xi, w, V + 24 * e, G + (int64_t)7 * n3 * e);
  return bad;
}

/* Nodal coordinates Phi(xi_i, xi_j, xi_k) of every node (Eq. 8), [E][3][n3]. */
int orc_nodal_coords(int64_t E, int N, const double *V, double *XYZ) {
  const int N1 = N + 1, n3 = N1 * N1 * N1;
  double xi[65], w[65], D[65 * 65];
  if (orc_gll(N, xi, w, D)) return 1;
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < E; ++e)
    for (int k = 0; k < N1; ++k)
      for (int j = 0; j < N1; ++j)
        for (int i = 0; i < N1; ++i) {
          double X[3];
          orc_trilinear_map(V + 24 * e, xi[i], xi[j], xi[k], X);
          for (int c = 0; c < 3; ++c) XYZ[(int64_t)(3 * e + c) * n3 + i + j * N1 + k * N1 * N1] = X[c];
        }
  return 0;
}

/* Standard discrete Jacobian (Sec. 3.2): apply the discrete gradient D of
 * Table 1 to each coordinate vector, read entry [i,j,k] of the nine results,
 * then Eq. 7.  Independent route to the same factors for trilinear maps
 * (degree 1 <= N, so the discrete derivative is exact).  Returns bad-node count. */
int64_t orc_factors_discrete(int64_t E, int N, const double *V, double *G) {
  const int N1 = N + 1, n3 = N1 * N1 * N1;
  double xi[65], w[65], D[65 * 65];
  if (orc_gll(N, xi, w, D)) return -1;
  double *XYZ = (double *)malloc(sizeof(double) * 3 * n3 * (size_t)E);
  if (!XYZ) return -1;
  orc_nodal_coords(E, N, V, XYZ);
  int64_t bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
  for (int64_t e = 0; e < E; ++e) {
    double *Ge = G + (int64_t)7 * n3 * e;
    for (int k = 0; k < N1; ++k)
      for (int j = 0; j < N1; ++j)
        for (int i = 0; i < N1; ++i) {
          double J[9], g[7];
          for (int c = 0; c < 3; ++c) {
            const double *xc = XYZ + (int64_t)(3 * e + c) * n3;
            double dr = 0, ds = 0, dt = 0;
            for (int n = 0; n < N1; ++n) {
              dr += D[i * N1 + n] * xc[n + j * N1 + k * N1 * N1];
              ds += D[j * N1 + n] * xc[i + n * N1 + k * N1 * N1];
              dt += D[k * N1 + n] * xc[i + j * N1 + n * N1 * N1];
            }
            J[3 * c + 0] = dr; J[3 * c + 1] = ds; J[3 * c + 2] = dt;
          }
          const int l = i + j * N1 + k * N1 * N1;
          double det = orc_factors_from_jacobian(J, w[i] * w[j] * w[k], g);
          if (!(det > 0.0)) ++bad;
          for (int q = 0; q < 7; ++q) Ge[(int64_t)q * n3 + l] = g[q];
        }
  }
  free(XYZ);
  return bad;
}

/* ------------------------------------------------------------------------
 * AxLocal, Algorithm 1, Poisson case (lambda0 = 1, lambda1 = 0: Eq. 3 drops
 * Lambda0, Lambda1 and G_wj).  Two passes over the nodes with the r, s, t
 * temporaries, exactly as the algorithm is written.
 * G is [E][7][n3] (only the first six factors are read).
 * ---------------------------------------------------------------------- */
static void axlocal_one(int N1, const double *D, const double *g, const double *x, double *y,
                        double *r, double *s, double *t) {
  const int n3 = N1 * N1 * N1;
  for (int k = 0; k < N1; ++k)
    for (int j = 0; j < N1; ++j)
      for (int i = 0; i < N1; ++i) {
        const int l = i + j * N1 + k * N1 * N1;
        const double g00 = g[0 * n3 + l], g01 = g[1 * n3 + l], g02 = g[2 * n3 + l];
        const double g11 = g[3 * n3 + l], g12 = g[4 * n3 + l], g22 = g[5 * n3 + l];
        double x0 = 0, x1 = 0, x2 = 0;
        for (int n = 0; n < N1; ++n) {
          x0 += D[i * N1 + n] * x[n + j * N1 + k * N1 * N1];
          x1 += D[j * N1 + n] * x[i + n * N1 + k * N1 * N1];
          x2 += D[k * N1 + n] * x[i + j * N1 + n * N1 * N1];
        }
        r[l] = g00 * x0 + g01 * x1 + g02 * x2;
        s[l] = g01 * x0 + g11 * x1 + g12 * x2;
        t[l] = g02 * x0 + g12 * x1 + g22 * x2;
      }
  for (int k = 0; k < N1; ++k)
    for (int j = 0; j < N1; ++j)
      for (int i = 0; i < N1; ++i) {
        double y0 = 0, y1 = 0, y2 = 0;
        for (int n = 0; n < N1; ++n) {
          y0 += D[n * N1 + i] * r[n + j * N1 + k * N1 * N1];
          y1 += D[n * N1 + j] * s[i + n * N1 + k * N1 * N1];
          y2 += D[n * N1 + k] * t[i + j * N1 + n * N1 * N1];
        }
        y[i + j * N1 + k * N1 * N1] = y0 + y1 + y2;
      }
}

int orc_axlocal(int64_t E, int N, const double *G, const double *X, double *Y) {
  const int N1 = N + 1, n3 = N1 * N1 * N1;
  double xi[65], w[65], D[65 * 65];
  if (orc_gll(N, xi, w, D)) return 1;
  int fail = 0;
#pragma omp parallel reduction(| : fail)
  {
    double *tmp = (double *)malloc(sizeof(double) * 3 * n3);
    if (!tmp) fail = 1;
    else {
#pragma omp for schedule(static)
      for (int64_t e = 0; e < E; ++e)
        axlocal_one(N1, D, G + (int64_t)7 * n3 * e, X + (int64_t)n3 * e, Y + (int64_t)n3 * e, tmp,
                    tmp + n3, tmp + 2 * n3);
      free(tmp);
    }
  }
  return fail;
}

/* AxLocal straight from vertices: per element, factors from Eq. 9 + Eq. 7,
 * then Algorithm 1.  Same arithmetic as orc_factors_eq9 + orc_axlocal, with
 * the factors held per element instead of for the whole mesh (this is what
 * the CPU baseline times).  Returns the bad-node count, or -1. */
int64_t orc_axlocal_vertices(int64_t E, int N, const double *V, const double *X, double *Y) {
  const int N1 = N + 1, n3 = N1 * N1 * N1;
  double xi[65], w[65], D[65 * 65];
  if (orc_gll(N, xi, w, D)) return -1;
  int64_t bad = 0;
  int fail = 0;
#pragma omp parallel reduction(+ : bad) reduction(| : fail)
  {
    double *tmp = (double *)malloc(sizeof(double) * 10 * n3);
    if (!tmp) fail = 1;
    else {
#pragma omp for schedule(static)
      for (int64_t e = 0; e < E; ++e) {
        double *g = tmp + 3 * n3;
        bad += factors_eq9_one(N1, xi, w, V + 24 * e, g);
        axlocal_one(N1, D, g, X + (int64_t)n3 * e, Y + (int64_t)n3 * e, tmp, tmp + n3, tmp + 2 * n3);
      }
      free(tmp);
    }
  }
  return fail ? -1 : bad;
}

/* ------------------------------------------------------------------------
 * Gather-scatter (Eq. 1): Y <- Q Q^T Y for the binary global-to-local matrix
 * Q[e*n3 + l][gid] = 1.  Q^T sums the local copies of every global node,
 * Q copies the sum back.  Plain serial loops.
 * ---------------------------------------------------------------------- */
int orc_gs(int64_t nlocal, const int64_t *gid, int64_t n_global, double *Y) {
  double *acc = (double *)calloc((size_t)n_global, sizeof(double));
  if (!acc) return 1;
  for (int64_t m = 0; m < nlocal; ++m) {
    if (gid[m] < 0 || gid[m] >= n_global) { free(acc); return 2; }
    acc[gid[m]] += Y[m];
  }
  for (int64_t m = 0; m < nlocal; ++m) Y[m] = acc[gid[m]];
  free(acc);
  return 0;
}

/* Q^T y (assembled global vector) and Q u (local copies). */
int orc_gather(int64_t nlocal, const int64_t *gid, int64_t n_global, const double *Yl, double *yg) {
  for (int64_t g = 0; g < n_global; ++g) yg[g] = 0.0;
  for (int64_t m = 0; m < nlocal; ++m) {
    if (gid[m] < 0 || gid[m] >= n_global) return 2;
    yg[gid[m]] += Yl[m];
  }
  return 0;
}

int orc_scatter(int64_t nlocal, const int64_t *gid, int64_t n_global, const double *ug, double *Ul) {
  for (int64_t m = 0; m < nlocal; ++m) {
    if (gid[m] < 0 || gid[m] >= n_global) return 2;
    Ul[m] = ug[gid[m]];
  }
  return 0;
}

/* ------------------------------------------------------------------------
 * Diagonal of every element matrix: diag[e][l] = e_l^T A^(e) e_l, by applying
 * Algorithm 1 to each unit vector (the definition; O(n3^2) per element, for
 * small meshes only).
 * ---------------------------------------------------------------------- */
int orc_diag(int64_t E, int N, const double *G, double *diag) {
  const int N1 = N + 1, n3 = N1 * N1 * N1;
  double xi[65], w[65], D[65 * 65];
  if (orc_gll(N, xi, w, D)) return 1;
  int fail = 0;
#pragma omp parallel reduction(| : fail)
  {
    double *tmp = (double *)malloc(sizeof(double) * 5 * n3);
    if (!tmp) fail = 1;
    else {
#pragma omp for schedule(static)
      for (int64_t e = 0; e < E; ++e) {
        double *x = tmp + 3 * n3, *y = tmp + 4 * n3;
        for (int l = 0; l < n3; ++l) x[l] = 0.0;
        for (int l = 0; l < n3; ++l) {
          x[l] = 1.0;
          axlocal_one(N1, D, G + (int64_t)7 * n3 * e, x, y, tmp, tmp + n3, tmp + 2 * n3);
          diag[(int64_t)n3 * e + l] = y[l];
          x[l] = 0.0;
        }
      }
      free(tmp);
    }
  }
  return fail;
}

/* ------------------------------------------------------------------------
 * Preconditioned conjugate gradients (textbook PCG, e.g. Saad, "Iterative
 * Methods for Sparse Linear Systems", Alg. 9.1) for the assembled Poisson
 * system A = Q^T blkdiag(A^(e)) Q of Eq. 1, with homogeneous Dirichlet
 * conditions imposed by masking: rows and columns of masked global nodes are
 * removed (their entries of x, r, p are held at zero).
 *   b, x: [n_global]; x is the initial guess on entry (masked entries ignored).
 *   diag_global: NULL for plain CG, else the assembled diagonal (Jacobi).
 *   Stops when ||r||_2 <= rtol ||b||_2 (b masked) or after maxit iterations.
 * Returns 0 when converged, 1 when maxit was reached, -1 on error.
 * ---------------------------------------------------------------------- */
static void apply_assembled(int64_t E, int N, const double *G, const int64_t *gid, int64_t n_global,
                            const unsigned char *mask, const double *p, double *w, double *Ul, double *Yl) {
  const int64_t nl = E * (int64_t)(N + 1) * (N + 1) * (N + 1);
  orc_scatter(nl, gid, n_global, p, Ul);
  orc_axlocal(E, N, G, Ul, Yl);
  orc_gather(nl, gid, n_global, Yl, w);
  if (mask)
    for (int64_t g = 0; g < n_global; ++g)
      if (mask[g]) w[g] = 0.0;
}

static double dotv(int64_t n, const double *a, const double *b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

int orc_pcg(int64_t E, int N, const double *G, const int64_t *gid, int64_t n_global, const unsigned char *mask,
            const double *b_in, double *x, const double *diag_global, double rtol, int maxit, int *iters,
            double *relres) {
  const int64_t nl = E * (int64_t)(N + 1) * (N + 1) * (N + 1);
  double *b = (double *)malloc(sizeof(double) * n_global);
  double *r = (double *)malloc(sizeof(double) * n_global);
  double *z = (double *)malloc(sizeof(double) * n_global);
  double *p = (double *)malloc(sizeof(double) * n_global);
  double *w = (double *)malloc(sizeof(double) * n_global);
  double *Ul = (double *)malloc(sizeof(double) * nl);
  double *Yl = (double *)malloc(sizeof(double) * nl);
  int status = -1;
  if (!b || !r || !z || !p || !w || !Ul || !Yl) goto done;
  for (int64_t g = 0; g < n_global; ++g) {
    const int m = mask && mask[g];
    b[g] = m ? 0.0 : b_in[g];
    if (m) x[g] = 0.0;
  }
  {
    const double bnorm = sqrt(dotv(n_global, b, b));
    apply_assembled(E, N, G, gid, n_global, mask, x, w, Ul, Yl);
    for (int64_t g = 0; g < n_global; ++g) r[g] = b[g] - w[g];
    for (int64_t g = 0; g < n_global; ++g) z[g] = diag_global ? r[g] / diag_global[g] : r[g];
    if (mask)
      for (int64_t g = 0; g < n_global; ++g)
        if (mask[g]) z[g] = 0.0;
    for (int64_t g = 0; g < n_global; ++g) p[g] = z[g];
    double rz = dotv(n_global, r, z);
    double rnorm = sqrt(dotv(n_global, r, r));
    int it = 0;
    status = 1;
    if (bnorm == 0.0 || rnorm <= rtol * bnorm) status = 0;
    while (status == 1 && it < maxit) {
      apply_assembled(E, N, G, gid, n_global, mask, p, w, Ul, Yl);
      const double alpha = rz / dotv(n_global, p, w);
      for (int64_t g = 0; g < n_global; ++g) {
        x[g] += alpha * p[g];
        r[g] -= alpha * w[g];
      }
      ++it;
      rnorm = sqrt(dotv(n_global, r, r));
      if (rnorm <= rtol * bnorm) {
        status = 0;
        break;
      }
      for (int64_t g = 0; g < n_global; ++g) z[g] = diag_global ? r[g] / diag_global[g] : r[g];
      if (mask)
        for (int64_t g = 0; g < n_global; ++g)
          if (mask[g]) z[g] = 0.0;
      const double rz_new = dotv(n_global, r, z);
      const double beta = rz_new / rz;
      rz = rz_new;
      for (int64_t g = 0; g < n_global; ++g) p[g] = z[g] + beta * p[g];
    }
    *iters = it;
    *relres = bnorm > 0.0 ? rnorm / bnorm : 0.0;
  }
done:
  free(b); free(r); free(z); free(p); free(w); free(Ul); free(Yl);
  return status;
}
