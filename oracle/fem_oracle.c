/*
 * fem_oracle.c -- plain FP64 CPU oracle for low-order finite element
 * integration (Knepley & Terrel, "Finite Element Integration on GPUs").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only the test suite, the smoke check and the CPU baseline
 * leg of the benchmark use it.  It shares no code, header or table with the
 * CUDA library.
 *
 * What it computes, and how (deliberately slow and direct):
 *   * Element matrices by DIRECT QUADRATURE of the weak forms, never through
 *     the tensor decomposition A = G:K of Eq. 1 / Eq. 6:
 *       - Laplacian, Eqs. 3-5:  A_ij = sum_q w_q |J| c_e  grad(phi_i).grad(phi_j)
 *       - elasticity, Eq. 10 with the 1/4 of Eq. 14 / Eq. 24, i.e. the form
 *         eps(v):eps(u):  A_IJ = sum_q w_q |J| c_e  eps(Phi_I):eps(Phi_J)
 *       - c_e is a per-element constant coefficient (the piecewise-constant
 *         case of the coefficient of Eq. 20); c_e = 1 when none is given.
 *       - or, for the P1 coefficient of Eqs. 20-23, c(xi) = sum_k w_k lambda_k(xi)
 *         evaluated at every quadrature point from the element's vertex
 *         values w_k (orc_integrate_w1); the Laplacian forms only.
 *   * Non-affine (isoparametric) elements, Eqs. 16-19 (orc_integrate_iso): the
 *     element has quadratic geometry (its vertices and edge-midpoint nodes);
 *     J^{-1} is projected onto P1 by its values at the vertices, J^{-1}(xi) =
 *     sum_k lambda_k(xi) J^{-1}(vertex k), and |J| is taken out of the
 *     integral as |det J| at the element centroid (Eq. 17), so
 *       A_ij = |J_c| c_e int_ref sum_a (J^{-1}(xi)^T grad_ref phi_i)_a (J^{-1}(xi)^T grad_ref phi_j)_a.
 *   * Physical gradients grad(phi) = J^{-T} grad_ref(phi) (the chain rule of
 *     Eq. 5, d xi_mu / d x_alpha = (J^{-1})_{mu alpha} as in Eq. 8) obtained
 *     by an LU solve with partial pivoting in FP64.
 *   * The reference simplex has vertices 0, e_1, ..., e_d and the affine map
 *     x(xi) = x_0 + sum_mu xi_mu (x_{mu+1} - x_0), so
 *     J_{alpha mu} = x_{mu+1,alpha} - x_{0,alpha}.  |J| = |det J|.
 *   * Quadrature: Gauss-Legendre points on [0,1] (roots found by Newton's
 *     method on the Legendre recurrence) collapsed onto the simplex by the
 *     Duffy map.  q points per direction integrate degree 2q-3 (tet) exactly
 *     in the collapsed direction; q = 3 covers every form here.
 *   * The coupling block of a multiphysics pair (Sec. 6: coupled systems
 *     broken into blocks), B_{i,(c,j)} = int_T c_e phi_i d psi_j / d x_c with
 *     phi the P1 scalar basis and psi the P1 or P2 basis of each component of
 *     a vector field (orc_integrate_div): by the same quadrature and LU solve.
 *   * The reverse mode (vector-Jacobian product) is derived by hand from the
 *     same quadrature steps, in the opposite order -- for the affine forms,
 *     the P1 coefficient, the coupling block and the non-affine elements
 *     (orc_integrate_iso_vjp: gradients of the vertices, of the edge nodes and
 *     of the per-element coefficient).
 *
 * Conventions shared with the library (they are conventions, not arithmetic):
 *   P1 basis lambda_0 = 1 - sum xi, lambda_k = xi_k.  P2 basis: vertex
 *   functions lambda_i (2 lambda_i - 1), i = 0..d, then edge functions
 *   4 lambda_i lambda_j over edges in lexicographic order.  Vector DOF index
 *   is c * n_basis + i (component-major).  Output A is [E][n][n] row-major.
 *   An element with det J == 0 gets A = 0 and flag bit 2; a connectivity
 *   index outside [0, V) gets A = 0 and flag bit 1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_LAPLACE_P1 0
#define ORC_LAPLACE_P2 1
#define ORC_ELASTIC_P1 2

#define ORC_FLAG_CONN 1
#define ORC_FLAG_DEGENERATE 2

#define ORC_MAXQ 8
#define ORC_MAXPTS (ORC_MAXQ * ORC_MAXQ * ORC_MAXQ)
#define ORC_MAXB 10 /* P2 on a tet */
#define ORC_MAXN 12 /* elasticity on a tet: 4 basis x 3 components */

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Quadrature                                                               */
/* ------------------------------------------------------------------------ */

/* Legendre polynomial P_q(t) and its derivative on [-1,1] by the three-term
 * recurrence (k+1) P_{k+1} = (2k+1) t P_k - k P_{k-1}. */
static void legendre(int q, double t, double* p, double* dp) {
  double p0 = 1.0, p1 = t;
  if (q == 0) { *p = 1.0; *dp = 0.0; return; }
  for (int k = 1; k < q; ++k) {
    double p2 = ((2.0 * k + 1.0) * t * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  *p = p1;
  *dp = q * (t * p1 - p0) / (t * t - 1.0);
}

/* q-point Gauss-Legendre rule mapped to [0,1]; weights sum to 1. */
int orc_gauss_legendre01(int q, double* x, double* w) {
  if (q < 1 || q > ORC_MAXQ) return -1;
  for (int i = 0; i < q; ++i) {
    double t = cos(M_PI * (i + 0.75) / (q + 0.5)); /* initial guess */
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(q, t, &p, &dp);
      double dt = p / dp;
      t -= dt;
      if (fabs(dt) < 1e-16) break;
    }
    double p, dp;
    legendre(q, t, &p, &dp);
    x[i] = 0.5 * (1.0 - t);
    w[i] = 1.0 / ((1.0 - t * t) * dp * dp); /* 2/((1-t^2)P'^2), halved for [0,1] */
  }
  return 0;
}

/* Duffy-collapsed rule on the reference simplex {xi >= 0, sum xi <= 1}.
 * Triangle: xi = (u, v(1-u)),                 weight (1-u).
 * Tet:      xi = (u, v(1-u), s(1-u)(1-v)),    weight (1-u)^2 (1-v).
 * Returns the number of points (q^dim); weights sum to 1/d!. */
int orc_simplex_rule(int dim, int q, double* pts, double* wts) {
  double x[ORC_MAXQ], w[ORC_MAXQ];
  if (dim < 2 || dim > 3) return -1;
  if (orc_gauss_legendre01(q, x, w) != 0) return -1;
  int n = 0;
  if (dim == 2) {
    for (int a = 0; a < q; ++a)
      for (int b = 0; b < q; ++b) {
        double u = x[a], v = x[b];
        pts[2 * n + 0] = u;
        pts[2 * n + 1] = v * (1.0 - u);
        wts[n] = w[a] * w[b] * (1.0 - u);
        ++n;
      }
  } else {
    for (int a = 0; a < q; ++a)
      for (int b = 0; b < q; ++b)
        for (int c = 0; c < q; ++c) {
          double u = x[a], v = x[b], s = x[c];
          pts[3 * n + 0] = u;
          pts[3 * n + 1] = v * (1.0 - u);
          pts[3 * n + 2] = s * (1.0 - u) * (1.0 - v);
          wts[n] = w[a] * w[b] * w[c] * (1.0 - u) * (1.0 - u) * (1.0 - v);
          ++n;
        }
  }
  return n;
}

/* ------------------------------------------------------------------------ */
/* Reference basis                                                          */
/* ------------------------------------------------------------------------ */

int orc_n_basis(int dim, int degree) {
  if (degree == 1) return dim + 1;
  if (degree == 2) return (dim + 1) * (dim + 2) / 2;
  return -1;
}

/* Barycentric coordinates lambda_k(xi) and their (constant) reference
 * gradients dlam[k][mu]. */
static void barycentric(int dim, const double* xi, double* lam, double dlam[4][3]) {
  double s = 0.0;
  for (int mu = 0; mu < dim; ++mu) s += xi[mu];
  lam[0] = 1.0 - s;
  for (int mu = 0; mu < dim; ++mu) dlam[0][mu] = -1.0;
  for (int k = 1; k <= dim; ++k) {
    lam[k] = xi[k - 1];
    for (int mu = 0; mu < dim; ++mu) dlam[k][mu] = (mu == k - 1) ? 1.0 : 0.0;
  }
}

/* Values phi[i] and reference gradients grad[i][mu] of the P1 or P2 basis at xi. */
int orc_basis(int dim, int degree, const double* xi, double* phi, double* grad) {
  double lam[4], dlam[4][3];
  barycentric(dim, xi, lam, dlam);
  int nv = dim + 1;
  if (degree == 1) {
    for (int i = 0; i < nv; ++i) {
      phi[i] = lam[i];
      for (int mu = 0; mu < dim; ++mu) grad[i * dim + mu] = dlam[i][mu];
    }
    return nv;
  }
  if (degree != 2) return -1;
  int n = 0;
  for (int i = 0; i < nv; ++i, ++n) { /* vertex functions lambda_i (2 lambda_i - 1) */
    phi[n] = lam[i] * (2.0 * lam[i] - 1.0);
    for (int mu = 0; mu < dim; ++mu) grad[n * dim + mu] = (4.0 * lam[i] - 1.0) * dlam[i][mu];
  }
  for (int i = 0; i < nv; ++i) /* edge functions 4 lambda_i lambda_j, i < j, lexicographic */
    for (int j = i + 1; j < nv; ++j, ++n) {
      phi[n] = 4.0 * lam[i] * lam[j];
      for (int mu = 0; mu < dim; ++mu)
        grad[n * dim + mu] = 4.0 * (lam[j] * dlam[i][mu] + lam[i] * dlam[j][mu]);
    }
  return n;
}

/* ------------------------------------------------------------------------ */
/* Small dense FP64 linear algebra: LU with partial pivoting                */
/* ------------------------------------------------------------------------ */

typedef struct {
  int n;
  double lu[3][3];
  int piv[3];
  double det;
} lu3;

static void lu_factor(int n, const double M[3][3], lu3* f) {
  f->n = n;
  memcpy(f->lu, M, sizeof(f->lu));
  double det = 1.0;
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int r = k + 1; r < n; ++r)
      if (fabs(f->lu[r][k]) > fabs(f->lu[p][k])) p = r;
    f->piv[k] = p;
    if (p != k) {
      for (int c = 0; c < n; ++c) {
        double t = f->lu[k][c];
        f->lu[k][c] = f->lu[p][c];
        f->lu[p][c] = t;
      }
      det = -det;
    }
    det *= f->lu[k][k];
    if (f->lu[k][k] == 0.0) continue;
    for (int r = k + 1; r < n; ++r) {
      f->lu[r][k] /= f->lu[k][k];
      for (int c = k + 1; c < n; ++c) f->lu[r][c] -= f->lu[r][k] * f->lu[k][c];
    }
  }
  f->det = det;
}

/* Solve M x = b in place (M factored in f as P M = L U, nonsingular).  The
 * factorisation swapped whole rows, multipliers included, so every row
 * interchange is applied to b first, then L y = P b, then U x = y. */
static void lu_solve(const lu3* f, double* b) {
  int n = f->n;
  for (int k = 0; k < n; ++k) {
    int p = f->piv[k];
    if (p != k) {
      double t = b[k];
      b[k] = b[p];
      b[p] = t;
    }
  }
  for (int k = 0; k < n; ++k)
    for (int r = k + 1; r < n; ++r) b[r] -= f->lu[r][k] * b[k];
  for (int k = n - 1; k >= 0; --k) {
    for (int c = k + 1; c < n; ++c) b[k] -= f->lu[k][c] * b[c];
    b[k] /= f->lu[k][k];
  }
}

/* ------------------------------------------------------------------------ */
/* One element                                                              */
/* ------------------------------------------------------------------------ */

static int form_degree(int form) { return form == ORC_LAPLACE_P2 ? 2 : 1; }
static int form_ncomp(int form, int dim) { return form == ORC_ELASTIC_P1 ? dim : 1; }

int orc_form_n(int form, int dim) {
  if (form < 0 || form > 2 || dim < 2 || dim > 3) return -1;
  return orc_n_basis(dim, form_degree(form)) * form_ncomp(form, dim);
}

/* Jacobian J[alpha][mu] = X[mu+1][alpha] - X[0][alpha]. */
static void jacobian(int dim, const double* X, double J[3][3]) {
  memset(J, 0, sizeof(double) * 9);
  for (int a = 0; a < dim; ++a)
    for (int mu = 0; mu < dim; ++mu) J[a][mu] = X[(mu + 1) * dim + a] - X[a];
}

/* Physical gradients at one quadrature point: solve J^T g_i = grad_ref(phi_i). */
static void physical_gradients(int dim, const lu3* fJt, int nb, const double* gref,
                               double g[ORC_MAXB][3]) {
  for (int i = 0; i < nb; ++i) {
    double b[3] = {0, 0, 0};
    for (int mu = 0; mu < dim; ++mu) b[mu] = gref[i * dim + mu];
    lu_solve(fJt, b);
    for (int a = 0; a < 3; ++a) g[i][a] = (a < dim) ? b[a] : 0.0;
  }
}

/* Symmetric gradient of the vector basis function Phi_I = phi_i e_c:
 * (grad Phi)_{ab} = delta_{ac} g_i[b], eps = (grad Phi + grad Phi^T) / 2. */
static void sym_grad(int dim, int c, const double* gi, double eps[3][3]) {
  for (int a = 0; a < dim; ++a)
    for (int b = 0; b < dim; ++b)
      eps[a][b] = 0.5 * ((a == c ? gi[b] : 0.0) + (b == c ? gi[a] : 0.0));
}

static double ddot_mat(int dim, double x[3][3], double y[3][3]) {
  double s = 0.0;
  for (int a = 0; a < dim; ++a)
    for (int b = 0; b < dim; ++b) s += x[a][b] * y[a][b];
  return s;
}

/* Element matrix of one element with vertex coordinates X[(dim+1)*dim], by
 * q^dim-point quadrature, with the coefficient either the constant coef
 * (wv == NULL) or the P1 function sum_k wv[k] lambda_k (wv = its d+1 vertex
 * values).  Returns 0, or ORC_FLAG_DEGENERATE (A zeroed) when det J == 0.
 * detJ_out (may be NULL) receives det J. */
static int element_matrix(int dim, int form, const double* X, double coef, const double* wv, int q, double* A,
                          double* detJ_out) {
  int n = orc_form_n(form, dim);
  if (n < 0) return -1;
  int deg = form_degree(form), nb = orc_n_basis(dim, deg), nc = form_ncomp(form, dim);
  memset(A, 0, sizeof(double) * n * n);
  double J[3][3], Jt[3][3];
  jacobian(dim, X, J);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) Jt[a][b] = J[b][a];
  lu3 fJt;
  lu_factor(dim, Jt, &fJt); /* det(J^T) = det(J) */
  if (detJ_out) *detJ_out = fJt.det;
  if (fJt.det == 0.0) return ORC_FLAG_DEGENERATE;
  double absdet = fabs(fJt.det);

  double pts[ORC_MAXPTS * 3], wts[ORC_MAXPTS];
  int np = orc_simplex_rule(dim, q, pts, wts);
  if (np < 0) return -1;
  for (int p = 0; p < np; ++p) {
    double phi[ORC_MAXB], gref[ORC_MAXB * 3], g[ORC_MAXB][3];
    orc_basis(dim, deg, pts + p * dim, phi, gref);
    physical_gradients(dim, &fJt, nb, gref, g);
    double c = coef;
    if (wv) { /* barycentrics of the point: lambda_0 = 1 - sum xi, lambda_k = xi_k */
      const double* xi = pts + p * dim;
      double l0 = 1.0;
      c = 0.0;
      for (int k = 1; k <= dim; ++k) {
        c += wv[k] * xi[k - 1];
        l0 -= xi[k - 1];
      }
      c += wv[0] * l0;
    }
    double scale = wts[p] * absdet * c;
    if (form != ORC_ELASTIC_P1) {
      for (int i = 0; i < nb; ++i)
        for (int j = 0; j < nb; ++j) {
          double s = 0.0;
          for (int a = 0; a < dim; ++a) s += g[i][a] * g[j][a];
          A[i * n + j] += scale * s;
        }
    } else {
      double eps[ORC_MAXN][3][3];
      for (int cc = 0; cc < nc; ++cc)
        for (int i = 0; i < nb; ++i) sym_grad(dim, cc, g[i], eps[cc * nb + i]);
      for (int I = 0; I < n; ++I)
        for (int K = 0; K < n; ++K) A[I * n + K] += scale * ddot_mat(dim, eps[I], eps[K]);
    }
  }
  return 0;
}

/* Element matrix with a per-element constant coefficient coef. */
int orc_element_matrix(int dim, int form, const double* X, double coef, int q, double* A,
                       double* detJ_out) {
  return element_matrix(dim, form, X, coef, NULL, q, A, detJ_out);
}

/* Element matrix of a Laplacian form with the P1 coefficient of vertex values
 * wv[0..dim] (Eqs. 20-23). */
int orc_element_matrix_w1(int dim, int form, const double* X, const double* wv, int q, double* A,
                          double* detJ_out) {
  if (form == ORC_ELASTIC_P1 || !wv) return -1;
  return element_matrix(dim, form, X, 1.0, wv, q, A, detJ_out);
}

/* Jacobian J[alpha][mu] = d x_alpha / d xi_mu of the quadratic geometry map
 * x(xi) = sum_a node_a psi_a(xi) at the reference point xi (nodes: vertices,
 * then edge midpoints in the P2 order). */
static void iso_jacobian(int dim, const double* nodes, const double* xi, double J[3][3]) {
  double psi[ORC_MAXB], gpsi[ORC_MAXB * 3];
  int nn = orc_basis(dim, 2, xi, psi, gpsi);
  memset(J, 0, sizeof(double) * 9);
  for (int a = 0; a < nn; ++a)
    for (int al = 0; al < dim; ++al)
      for (int mu = 0; mu < dim; ++mu) J[al][mu] += nodes[a * dim + al] * gpsi[a * dim + mu];
}

static double det3(int dim, double J[3][3]) {
  if (dim == 2) return J[0][0] * J[1][1] - J[0][1] * J[1][0];
  return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
         J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

/* Element matrix of a Laplacian form on a non-affine element (Eqs. 16-19):
 * X[(dim+1)*dim] vertices, Mid[n_edges*dim] edge-midpoint nodes (P2 edge
 * order), per-element coefficient coef.  Returns 0, or ORC_FLAG_DEGENERATE (A
 * zeroed) when J is singular at a vertex or at the centroid. */
int orc_element_matrix_iso(int dim, int form, const double* X, const double* Mid, double coef, int q, double* A,
                           double* detc_out) {
  if (form == ORC_ELASTIC_P1) return -1;
  int n = orc_form_n(form, dim);
  if (n < 0) return -1;
  int deg = form_degree(form), nb = orc_n_basis(dim, deg), nv = dim + 1;
  int ne = dim == 2 ? 3 : 6;
  memset(A, 0, sizeof(double) * n * n);
  double nodes[ORC_MAXB * 3];
  for (int k = 0; k < nv * dim; ++k) nodes[k] = X[k];
  for (int k = 0; k < ne * dim; ++k) nodes[nv * dim + k] = Mid[k];
  /* J^{-1} at the vertices: Jinv_k[mu][alpha] = (J(vertex k)^{-1})[mu][alpha] */
  double Jinv[4][3][3];
  for (int k = 0; k < nv; ++k) {
    double xi[3] = {0, 0, 0};
    if (k > 0) xi[k - 1] = 1.0;
    double J[3][3];
    iso_jacobian(dim, nodes, xi, J);
    lu3 f;
    lu_factor(dim, J, &f);
    if (f.det == 0.0) {
      if (detc_out) *detc_out = 0.0;
      return ORC_FLAG_DEGENERATE;
    }
    for (int al = 0; al < dim; ++al) {
      double b[3] = {0, 0, 0};
      b[al] = 1.0;
      lu_solve(&f, b); /* J b = e_alpha: b is column alpha of J^{-1}, b[mu] = (J^{-1})[mu][alpha] */
      for (int mu = 0; mu < dim; ++mu) Jinv[k][mu][al] = b[mu];
    }
  }
  double xc[3] = {0, 0, 0};
  for (int mu = 0; mu < dim; ++mu) xc[mu] = 1.0 / nv;
  double Jc[3][3];
  iso_jacobian(dim, nodes, xc, Jc);
  double detc = det3(dim, Jc);
  if (detc_out) *detc_out = detc;
  if (detc == 0.0) return ORC_FLAG_DEGENERATE;
  double absdet = fabs(detc);
  double pts[ORC_MAXPTS * 3], wts[ORC_MAXPTS];
  int np = orc_simplex_rule(dim, q, pts, wts);
  if (np < 0) return -1;
  for (int p = 0; p < np; ++p) {
    const double* xi = pts + p * dim;
    double lam[4];
    lam[0] = 1.0;
    for (int k = 1; k <= dim; ++k) {
      lam[k] = xi[k - 1];
      lam[0] -= xi[k - 1];
    }
    double Ji[3][3] = {{0}};
    for (int k = 0; k < nv; ++k)
      for (int mu = 0; mu < dim; ++mu)
        for (int al = 0; al < dim; ++al) Ji[mu][al] += lam[k] * Jinv[k][mu][al];
    double phi[ORC_MAXB], gref[ORC_MAXB * 3], g[ORC_MAXB][3];
    orc_basis(dim, deg, xi, phi, gref);
    for (int i = 0; i < nb; ++i)
      for (int al = 0; al < 3; ++al) {
        double s = 0.0;
        if (al < dim)
          for (int mu = 0; mu < dim; ++mu) s += Ji[mu][al] * gref[i * dim + mu];
        g[i][al] = s;
      }
    double scale = wts[p] * absdet * coef;
    for (int i = 0; i < nb; ++i)
      for (int j = 0; j < nb; ++j) {
        double s = 0.0;
        for (int a = 0; a < dim; ++a) s += g[i][a] * g[j][a];
        A[i * n + j] += scale * s;
      }
  }
  return 0;
}

/* Reverse mode of orc_element_matrix: given Abar = dL/dA, returns
 * Xbar[(dim+1)*dim] = dL/dX and *cbar = dL/dcoef.  Derivation, per quadrature
 * point with s = |det J|, c = coef:
 *   Laplacian   A_ij  += w s c g_i.g_j
 *               gbar_i += w s c sum_j (Abar_ij + Abar_ji) g_j
 *   elasticity  A_IK  += w s c eps_I:eps_K
 *               epsbar_I = w s c sum_K (Abar_IK + Abar_KI) eps_K
 *               gbar_i[m] += (epsbar_I[c][m] + epsbar_I[m][c]) / 2   for I = (c, i)
 *   both        sbar  += w c sum Abar .* (integrand),  cbar += w s sum Abar .* (integrand)
 * then with B = J^{-1} (g_i = B^T gref_i):
 *   Bbar[mu][a] += sum_i gref_i[mu] gbar_i[a]
 *   Jbar = -B^T Bbar B^T + sbar s B^T           (d|det J|/dJ = |det J| J^{-T})
 *   Xbar[mu+1][a] = Jbar[a][mu],  Xbar[0][a] = -sum_mu Jbar[a][mu]. */
int orc_element_vjp(int dim, int form, const double* X, double coef, int q, const double* Abar,
                    double* Xbar, double* cbar) {
  int n = orc_form_n(form, dim);
  if (n < 0) return -1;
  int deg = form_degree(form), nb = orc_n_basis(dim, deg), nc = form_ncomp(form, dim);
  int nv = dim + 1;
  for (int k = 0; k < nv * dim; ++k) Xbar[k] = 0.0;
  *cbar = 0.0;
  double J[3][3], Jt[3][3];
  jacobian(dim, X, J);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) Jt[a][b] = J[b][a];
  lu3 fJt;
  lu_factor(dim, Jt, &fJt);
  if (fJt.det == 0.0) return ORC_FLAG_DEGENERATE;
  double s = fabs(fJt.det);

  /* B = J^{-1}: column k of B solves J b = e_k; J = (J^T)^T so use J's own LU. */
  lu3 fJ;
  lu_factor(dim, J, &fJ);
  double B[3][3] = {{0}};
  for (int k = 0; k < dim; ++k) {
    double e[3] = {0, 0, 0};
    e[k] = 1.0;
    lu_solve(&fJ, e);
    for (int r = 0; r < dim; ++r) B[r][k] = e[r];
  }

  double pts[ORC_MAXPTS * 3], wts[ORC_MAXPTS];
  int np = orc_simplex_rule(dim, q, pts, wts);
  double sbar = 0.0, Bbar[3][3] = {{0}};
  for (int p = 0; p < np; ++p) {
    double phi[ORC_MAXB], gref[ORC_MAXB * 3], g[ORC_MAXB][3], gbar[ORC_MAXB][3];
    orc_basis(dim, deg, pts + p * dim, phi, gref);
    physical_gradients(dim, &fJt, nb, gref, g);
    memset(gbar, 0, sizeof(gbar));
    double wq = wts[p];
    if (form != ORC_ELASTIC_P1) {
      for (int i = 0; i < nb; ++i)
        for (int j = 0; j < nb; ++j) {
          double gg = 0.0;
          for (int a = 0; a < dim; ++a) gg += g[i][a] * g[j][a];
          double ab = Abar[i * n + j];
          sbar += wq * coef * ab * gg;
          *cbar += wq * s * ab * gg;
          double sym = Abar[i * n + j] + Abar[j * n + i];
          for (int a = 0; a < dim; ++a) gbar[i][a] += wq * s * coef * sym * g[j][a];
        }
    } else {
      double eps[ORC_MAXN][3][3], epsbar[ORC_MAXN][3][3];
      memset(epsbar, 0, sizeof(epsbar));
      for (int c = 0; c < nc; ++c)
        for (int i = 0; i < nb; ++i) sym_grad(dim, c, g[i], eps[c * nb + i]);
      for (int I = 0; I < n; ++I)
        for (int K = 0; K < n; ++K) {
          double ee = ddot_mat(dim, eps[I], eps[K]);
          double ab = Abar[I * n + K];
          sbar += wq * coef * ab * ee;
          *cbar += wq * s * ab * ee;
          double sym = Abar[I * n + K] + Abar[K * n + I];
          for (int a = 0; a < dim; ++a)
            for (int b = 0; b < dim; ++b) epsbar[I][a][b] += wq * s * coef * sym * eps[K][a][b];
        }
      for (int c = 0; c < nc; ++c)
        for (int i = 0; i < nb; ++i)
          for (int m = 0; m < dim; ++m)
            gbar[i][m] += 0.5 * (epsbar[c * nb + i][c][m] + epsbar[c * nb + i][m][c]);
    }
    for (int i = 0; i < nb; ++i)
      for (int mu = 0; mu < dim; ++mu)
        for (int a = 0; a < dim; ++a) Bbar[mu][a] += gref[i * dim + mu] * gbar[i][a];
  }
  /* Jbar = -B^T Bbar B^T + sbar s B^T */
  double Jbar[3][3] = {{0}};
  for (int a = 0; a < dim; ++a)
    for (int mu = 0; mu < dim; ++mu) {
      double acc = 0.0;
      for (int k = 0; k < dim; ++k)
        for (int l = 0; l < dim; ++l) acc += B[k][a] * Bbar[k][l] * B[mu][l];
      Jbar[a][mu] = -acc + sbar * s * B[mu][a];
    }
  for (int a = 0; a < dim; ++a) {
    double col = 0.0;
    for (int mu = 0; mu < dim; ++mu) {
      Xbar[(mu + 1) * dim + a] = Jbar[a][mu];
      col += Jbar[a][mu];
    }
    Xbar[a] = -col;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Whole meshes                                                             */
/* ------------------------------------------------------------------------ */

static int gather(int dim, int64_t n_vert, const int32_t* conn_e, const double* coords,
                  double* X) {
  for (int k = 0; k <= dim; ++k) {
    int64_t v = conn_e[k];
    if (v < 0 || v >= n_vert) return ORC_FLAG_CONN;
    for (int a = 0; a < dim; ++a) X[k * dim + a] = coords[v * dim + a];
  }
  return 0;
}

/* A[e] for every element (A is [E][n][n] FP64).  coef may be NULL (= 1).
 * flags (may be NULL) receives per-element flag bits.  Returns the OR of the flags. */
int orc_integrate(int dim, int form, int64_t n_elem, int64_t n_vert, const int32_t* conn,
                  const double* coords, const double* coef, int q, double* A, int32_t* flags,
                  double* detJ, int nthreads) {
  int n = orc_form_n(form, dim);
  if (n < 0) return -1;
  int any = 0;
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(static) num_threads(nthreads) reduction(| : any)
  for (int64_t e = 0; e < n_elem; ++e) {
    double X[12];
    double* Ae = A + e * (int64_t)n * n;
    int f = gather(dim, n_vert, conn + e * (dim + 1), coords, X);
    double det = 0.0;
    if (f == 0) {
      f = orc_element_matrix(dim, form, X, coef ? coef[e] : 1.0, q, Ae, &det);
    } else {
      memset(Ae, 0, sizeof(double) * n * n);
    }
    if (flags) flags[e] = f;
    if (detJ) detJ[e] = det;
    any |= f;
  }
  return any;
}

/* A[e] for every element of a Laplacian form with the P1 coefficient whose
 * vertex values are wvert [V] (Eqs. 20-23).  Flags as in orc_integrate. */
int orc_integrate_w1(int dim, int form, int64_t n_elem, int64_t n_vert, const int32_t* conn,
                     const double* coords, const double* wvert, int q, double* A, int32_t* flags,
                     int nthreads) {
  int n = orc_form_n(form, dim);
  if (n < 0 || form == ORC_ELASTIC_P1 || !wvert) return -1;
  int any = 0;
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(static) num_threads(nthreads) reduction(| : any)
  for (int64_t e = 0; e < n_elem; ++e) {
    double X[12], wv[4];
    double* Ae = A + e * (int64_t)n * n;
    const int32_t* ce = conn + e * (dim + 1);
    int f = gather(dim, n_vert, ce, coords, X);
    if (f == 0) {
      for (int k = 0; k <= dim; ++k) wv[k] = wvert[ce[k]];
      f = element_matrix(dim, form, X, 1.0, wv, q, Ae, NULL);
    } else {
      memset(Ae, 0, sizeof(double) * n * n);
    }
    if (flags) flags[e] = f;
    any |= f;
  }
  return any;
}

/* A[e] for every element of a Laplacian form on non-affine elements: mid
 * [E][n_edges][dim] holds each element's edge-midpoint nodes.  Flags as in
 * orc_integrate. */
int orc_integrate_iso(int dim, int form, int64_t n_elem, int64_t n_vert, const int32_t* conn, const double* coords,
                      const double* mid, const double* coef, int q, double* A, int32_t* flags, int nthreads) {
  int n = orc_form_n(form, dim);
  if (n < 0 || form == ORC_ELASTIC_P1) return -1;
  int ne = dim == 2 ? 3 : 6;
  int any = 0;
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(static) num_threads(nthreads) reduction(| : any)
  for (int64_t e = 0; e < n_elem; ++e) {
    double X[12];
    double* Ae = A + e * (int64_t)n * n;
    int f = gather(dim, n_vert, conn + e * (dim + 1), coords, X);
    if (f == 0) {
      f = orc_element_matrix_iso(dim, form, X, mid + e * (int64_t)ne * dim, coef ? coef[e] : 1.0, q, Ae, NULL);
    } else {
      memset(Ae, 0, sizeof(double) * n * n);
    }
    if (flags) flags[e] = f;
    any |= f;
  }
  return any;
}

/* Reverse mode of orc_element_matrix_iso (Eqs. 16-19), derived by hand from
 * its steps taken backwards.  Given Abar = dL/dA [n][n]:
 *   1. at every quadrature point p the forward adds s_p g_i.g_j into A_ij with
 *      s_p = w_p |det J_c| coef and g_i = Ji(xi_p)^T grad_ref phi_i, so
 *        d|det J_c| += w_p coef sum_ij Abar_ij g_i.g_j,  dcoef likewise,
 *        gbar_i = s_p sum_j (Abar_ij + Abar_ji) g_j,
 *        Jibar(xi_p)[mu][al] = sum_i gbar_i[al] grad_ref phi_i[mu];
 *   2. Ji(xi) = sum_k lambda_k(xi) Jinv_k, so Jinvbar_k += lambda_k(xi_p) Jibar;
 *   3. Jinv_k = J_k^{-1} (J_k = J at vertex k): Jbar_k = -Jinv_k^T Jinvbar_k Jinv_k^T;
 *   4. |det J_c|: Jbar_c = sign(det J_c) d|det J_c| cof(J_c), cof = det J^{-T};
 *   5. J(xi) = sum_a node_a grad psi_a(xi)^T: nodebar_a[al] =
 *        sum_k sum_mu Jbar_k[al][mu] dpsi_a/dxi_mu(vertex k)
 *        + sum_mu Jbar_c[al][mu] dpsi_a/dxi_mu(centroid).
 * Xbar [(dim+1)*dim] gets the vertex nodes' gradients, Midbar [n_edges*dim]
 * the edge nodes', *cbar the coefficient's (may be NULL).  Returns as
 * orc_element_matrix_iso; a degenerate element leaves the outputs zero. */
int orc_element_vjp_iso(int dim, int form, const double* X, const double* Mid, double coef, int q,
                        const double* Abar, double* Xbar, double* Midbar, double* cbar) {
  if (form == ORC_ELASTIC_P1) return -1;
  int n = orc_form_n(form, dim);
  if (n < 0) return -1;
  int deg = form_degree(form), nb = orc_n_basis(dim, deg), nv = dim + 1;
  int ne = dim == 2 ? 3 : 6, nn = nv + ne;
  for (int k = 0; k < nv * dim; ++k) Xbar[k] = 0.0;
  for (int k = 0; k < ne * dim; ++k) Midbar[k] = 0.0;
  if (cbar) *cbar = 0.0;
  double nodes[ORC_MAXB * 3];
  for (int k = 0; k < nv * dim; ++k) nodes[k] = X[k];
  for (int k = 0; k < ne * dim; ++k) nodes[nv * dim + k] = Mid[k];
  double Jinv[4][3][3];
  for (int k = 0; k < nv; ++k) {
    double xi[3] = {0, 0, 0};
    if (k > 0) xi[k - 1] = 1.0;
    double J[3][3];
    iso_jacobian(dim, nodes, xi, J);
    lu3 f;
    lu_factor(dim, J, &f);
    if (f.det == 0.0) return ORC_FLAG_DEGENERATE;
    for (int al = 0; al < dim; ++al) {
      double b[3] = {0, 0, 0};
      b[al] = 1.0;
      lu_solve(&f, b);
      for (int mu = 0; mu < dim; ++mu) Jinv[k][mu][al] = b[mu];
    }
  }
  double xc[3] = {0, 0, 0};
  for (int mu = 0; mu < dim; ++mu) xc[mu] = 1.0 / nv;
  double Jc[3][3];
  iso_jacobian(dim, nodes, xc, Jc);
  double detc = det3(dim, Jc);
  if (detc == 0.0) return ORC_FLAG_DEGENERATE;
  double absdet = fabs(detc);
  double pts[ORC_MAXPTS * 3], wts[ORC_MAXPTS];
  int np = orc_simplex_rule(dim, q, pts, wts);
  if (np < 0) return -1;
  /* steps 1-2 */
  double Jinvbar[4][3][3];
  memset(Jinvbar, 0, sizeof(Jinvbar));
  double absdet_bar = 0.0, coef_bar = 0.0;
  for (int p = 0; p < np; ++p) {
    const double* xi = pts + p * dim;
    double lam[4];
    lam[0] = 1.0;
    for (int k = 1; k <= dim; ++k) {
      lam[k] = xi[k - 1];
      lam[0] -= xi[k - 1];
    }
    double Ji[3][3] = {{0}};
    for (int k = 0; k < nv; ++k)
      for (int mu = 0; mu < dim; ++mu)
        for (int al = 0; al < dim; ++al) Ji[mu][al] += lam[k] * Jinv[k][mu][al];
    double phi[ORC_MAXB], gref[ORC_MAXB * 3], g[ORC_MAXB][3];
    orc_basis(dim, deg, xi, phi, gref);
    for (int i = 0; i < nb; ++i)
      for (int al = 0; al < dim; ++al) {
        double s = 0.0;
        for (int mu = 0; mu < dim; ++mu) s += Ji[mu][al] * gref[i * dim + mu];
        g[i][al] = s;
      }
    double quad = 0.0; /* sum_ij Abar_ij g_i.g_j */
    for (int i = 0; i < nb; ++i)
      for (int j = 0; j < nb; ++j) {
        double s = 0.0;
        for (int a = 0; a < dim; ++a) s += g[i][a] * g[j][a];
        quad += Abar[i * n + j] * s;
      }
    absdet_bar += wts[p] * coef * quad;
    coef_bar += wts[p] * absdet * quad;
    double sp = wts[p] * absdet * coef;
    double gbar[ORC_MAXB][3];
    for (int i = 0; i < nb; ++i)
      for (int a = 0; a < dim; ++a) {
        double s = 0.0;
        for (int j = 0; j < nb; ++j) s += (Abar[i * n + j] + Abar[j * n + i]) * g[j][a];
        gbar[i][a] = sp * s;
      }
    double Jibar[3][3] = {{0}};
    for (int mu = 0; mu < dim; ++mu)
      for (int al = 0; al < dim; ++al) {
        double s = 0.0;
        for (int i = 0; i < nb; ++i) s += gbar[i][al] * gref[i * dim + mu];
        Jibar[mu][al] = s;
      }
    for (int k = 0; k < nv; ++k)
      for (int mu = 0; mu < dim; ++mu)
        for (int al = 0; al < dim; ++al) Jinvbar[k][mu][al] += lam[k] * Jibar[mu][al];
  }
  if (cbar) *cbar = coef_bar;
  /* step 3: Jbar_k[al][mu] = -sum_{nu,be} Jinv_k[nu][al] Jinvbar_k[nu][be] Jinv_k[mu][be] */
  double Jbar[5][3][3];
  memset(Jbar, 0, sizeof(Jbar));
  for (int k = 0; k < nv; ++k)
    for (int al = 0; al < dim; ++al)
      for (int mu = 0; mu < dim; ++mu) {
        double s = 0.0;
        for (int nu = 0; nu < dim; ++nu)
          for (int be = 0; be < dim; ++be) s += Jinv[k][nu][al] * Jinvbar[k][nu][be] * Jinv[k][mu][be];
        Jbar[k][al][mu] = -s;
      }
  /* step 4: cofactor of J_c by minors */
  double sgn = detc > 0.0 ? 1.0 : -1.0;
  for (int al = 0; al < dim; ++al)
    for (int mu = 0; mu < dim; ++mu) {
      double cof;
      if (dim == 2) {
        cof = (al == mu ? Jc[1 - al][1 - mu] : -Jc[1 - al][1 - mu]);
      } else {
        int r0 = (al + 1) % 3, r1 = (al + 2) % 3, c0 = (mu + 1) % 3, c1 = (mu + 2) % 3;
        cof = Jc[r0][c0] * Jc[r1][c1] - Jc[r0][c1] * Jc[r1][c0];
      }
      Jbar[nv][al][mu] = sgn * absdet_bar * cof;
    }
  /* step 5 */
  for (int k = 0; k <= nv; ++k) {
    double xi[3] = {0, 0, 0};
    if (k == nv) {
      for (int mu = 0; mu < dim; ++mu) xi[mu] = 1.0 / nv;
    } else if (k > 0) {
      xi[k - 1] = 1.0;
    }
    double psi[ORC_MAXB], gpsi[ORC_MAXB * 3];
    orc_basis(dim, 2, xi, psi, gpsi);
    for (int a = 0; a < nn; ++a)
      for (int al = 0; al < dim; ++al) {
        double s = 0.0;
        for (int mu = 0; mu < dim; ++mu) s += Jbar[k][al][mu] * gpsi[a * dim + mu];
        if (a < nv)
          Xbar[a * dim + al] += s;
        else
          Midbar[(a - nv) * dim + al] += s;
      }
  }
  return 0;
}

/* Reverse mode of orc_integrate_iso over a mesh: given Abar [E][n][n],
 * dcoords [V][dim] (overwritten; per-vertex sums in element order), dmid
 * [E][n_edges][dim] (overwritten) and dcoef [E] (may be NULL).  Flagged
 * elements contribute nothing. */
int orc_integrate_iso_vjp(int dim, int form, int64_t n_elem, int64_t n_vert, const int32_t* conn,
                          const double* coords, const double* mid, const double* coef, int q, const double* Abar,
                          double* dcoords, double* dmid, double* dcoef, int nthreads) {
  int n = orc_form_n(form, dim);
  if (n < 0 || form == ORC_ELASTIC_P1) return -1;
  int nv = dim + 1, ne = dim == 2 ? 3 : 6;
  double* xbar = (double*)malloc(sizeof(double) * (size_t)(n_elem > 0 ? n_elem : 1) * nv * dim);
  int32_t* fl = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_elem > 0 ? n_elem : 1));
  if (!xbar || !fl) {
    free(xbar);
    free(fl);
    return -2;
  }
  if (nthreads < 1) nthreads = 1;
  int any = 0;
#pragma omp parallel for schedule(static) num_threads(nthreads) reduction(| : any)
  for (int64_t e = 0; e < n_elem; ++e) {
    double X[12], cb = 0.0;
    double* xb = xbar + e * nv * dim;
    double* mb = dmid + e * (int64_t)ne * dim;
    int f = gather(dim, n_vert, conn + e * nv, coords, X);
    if (f == 0)
      f = orc_element_vjp_iso(dim, form, X, mid + e * (int64_t)ne * dim, coef ? coef[e] : 1.0, q,
                              Abar + e * (int64_t)n * n, xb, mb, &cb);
    if (f != 0) {
      for (int k = 0; k < nv * dim; ++k) xb[k] = 0.0;
      for (int k = 0; k < ne * dim; ++k) mb[k] = 0.0;
      cb = 0.0;
    }
    fl[e] = f;
    if (dcoef) dcoef[e] = cb;
    any |= f;
  }
  for (int64_t k = 0; k < n_vert * dim; ++k) dcoords[k] = 0.0;
  for (int64_t e = 0; e < n_elem; ++e) {
    if (fl[e] & ORC_FLAG_CONN) continue;
    for (int k = 0; k < nv; ++k) {
      int64_t v = conn[e * nv + k];
      for (int a = 0; a < dim; ++a) dcoords[v * dim + a] += xbar[(e * nv + k) * dim + a];
    }
  }
  free(xbar);
  free(fl);
  return any;
}

/* Reverse mode over a mesh: given Abar [E][n][n], writes dcoords [V][dim]
 * (overwritten; per-vertex sums taken in element order, FP64) and dcoef [E]
 * (may be NULL).  Flagged elements contribute nothing. */
int orc_integrate_vjp(int dim, int form, int64_t n_elem, int64_t n_vert, const int32_t* conn,
                      const double* coords, const double* coef, int q, const double* Abar,
                      double* dcoords, double* dcoef, int nthreads) {
  int n = orc_form_n(form, dim);
  if (n < 0) return -1;
  int nv = dim + 1;
  double* xbar = (double*)malloc(sizeof(double) * (size_t)n_elem * nv * dim);
  int32_t* fl = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_elem > 0 ? n_elem : 1));
  if (!xbar || !fl) {
    free(xbar);
    free(fl);
    return -2;
  }
  if (nthreads < 1) nthreads = 1;
  int any = 0;
#pragma omp parallel for schedule(static) num_threads(nthreads) reduction(| : any)
  for (int64_t e = 0; e < n_elem; ++e) {
    double X[12], cb = 0.0;
    double* xb = xbar + e * nv * dim;
    int f = gather(dim, n_vert, conn + e * nv, coords, X);
    if (f == 0)
      f = orc_element_vjp(dim, form, X, coef ? coef[e] : 1.0, q, Abar + e * (int64_t)n * n, xb,
                          &cb);
    if (f != 0) {
      for (int k = 0; k < nv * dim; ++k) xb[k] = 0.0;
      cb = 0.0;
    }
    fl[e] = f;
    if (dcoef) dcoef[e] = cb;
    any |= f;
  }
  for (int64_t k = 0; k < n_vert * dim; ++k) dcoords[k] = 0.0;
  for (int64_t e = 0; e < n_elem; ++e) {
    if (fl[e] & ORC_FLAG_CONN) continue;
    for (int k = 0; k < nv; ++k) {
      int64_t v = conn[e * nv + k];
      for (int a = 0; a < dim; ++a) dcoords[v * dim + a] += xbar[(e * nv + k) * dim + a];
    }
  }
  free(xbar);
  free(fl);
  return any;
}

/* ------------------------------------------------------------------------ */
/* Coupling block of a multiphysics system                                  */
/* ------------------------------------------------------------------------ */
/* Sec. 6 plans systems of equations from multiphysics problems, with the weak
 * form broken into blocks; the off-diagonal block of a pair (scalar field q,
 * vector field v) is the bilinear form int q div v, whose analytic tensor
 * holds a basis function times a basis-function derivative (Eq. 1 and the
 * closing remark of Sec. 3.1).  Here, by direct quadrature:
 *   B_{i,(c,j)} = int_T coef phi_i d psi_j / d x_c
 * phi the P1 scalar basis (rows i = 0..d), psi the P`vdeg` basis of each
 * component c of the vector field (columns c * nbv + j, component-major).
 * B is [(d+1)][d * nbv] row-major.  Returns 0 or ORC_FLAG_DEGENERATE (B
 * zeroed) when det J == 0. */
int orc_element_matrix_div(int dim, int vdeg, const double* X, double coef, int q, double* B, double* detJ_out) {
  int nq = dim + 1, nbv = orc_n_basis(dim, vdeg);
  if (nbv < 0 || dim < 2 || dim > 3) return -1;
  int ncol = dim * nbv;
  memset(B, 0, sizeof(double) * nq * ncol);
  double J[3][3], Jt[3][3];
  jacobian(dim, X, J);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) Jt[a][b] = J[b][a];
  lu3 fJt;
  lu_factor(dim, Jt, &fJt);
  if (detJ_out) *detJ_out = fJt.det;
  if (fJt.det == 0.0) return ORC_FLAG_DEGENERATE;
  double absdet = fabs(fJt.det);
  double pts[ORC_MAXPTS * 3], wts[ORC_MAXPTS];
  int np = orc_simplex_rule(dim, q, pts, wts);
  if (np < 0) return -1;
  for (int p = 0; p < np; ++p) {
    double phi[ORC_MAXB], gphi[ORC_MAXB * 3], psi[ORC_MAXB], gref[ORC_MAXB * 3], g[ORC_MAXB][3];
    orc_basis(dim, 1, pts + p * dim, phi, gphi);
    orc_basis(dim, vdeg, pts + p * dim, psi, gref);
    physical_gradients(dim, &fJt, nbv, gref, g);
    double scale = wts[p] * absdet * coef;
    for (int i = 0; i < nq; ++i)
      for (int c = 0; c < dim; ++c)
        for (int j = 0; j < nbv; ++j) B[i * ncol + c * nbv + j] += scale * phi[i] * g[j][c];
  }
  return 0;
}

/* Reverse mode of orc_element_matrix_div: given Bbar = dL/dB, returns Xbar =
 * dL/dX [(d+1)*d] and *cbar = dL/dcoef.  Per quadrature point, with s =
 * |det J|, c = coef and the integrand I = sum Bbar_{i,(a,j)} phi_i g_j[a]:
 *   gbar_j[a] += w s c sum_i Bbar_{i,(a,j)} phi_i,   sbar += w c I,   cbar += w s I
 * and then, as in orc_element_vjp, with B = J^{-1}:
 *   Bbar[mu][a] += sum_j gref_j[mu] gbar_j[a],   Jbar = -B^T Bbar B^T + sbar s B^T. */
int orc_element_vjp_div(int dim, int vdeg, const double* X, double coef, int q, const double* Bbar_in, double* Xbar,
                        double* cbar) {
  int nq = dim + 1, nbv = orc_n_basis(dim, vdeg);
  if (nbv < 0 || dim < 2 || dim > 3) return -1;
  int ncol = dim * nbv, nv = dim + 1;
  for (int k = 0; k < nv * dim; ++k) Xbar[k] = 0.0;
  *cbar = 0.0;
  double J[3][3], Jt[3][3];
  jacobian(dim, X, J);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) Jt[a][b] = J[b][a];
  lu3 fJt;
  lu_factor(dim, Jt, &fJt);
  if (fJt.det == 0.0) return ORC_FLAG_DEGENERATE;
  double s = fabs(fJt.det);
  lu3 fJ;
  lu_factor(dim, J, &fJ);
  double Binv[3][3] = {{0}};
  for (int k = 0; k < dim; ++k) {
    double e[3] = {0, 0, 0};
    e[k] = 1.0;
    lu_solve(&fJ, e);
    for (int r = 0; r < dim; ++r) Binv[r][k] = e[r];
  }
  double pts[ORC_MAXPTS * 3], wts[ORC_MAXPTS];
  int np = orc_simplex_rule(dim, q, pts, wts);
  if (np < 0) return -1;
  double sbar = 0.0, Mbar[3][3] = {{0}};
  for (int p = 0; p < np; ++p) {
    double phi[ORC_MAXB], gphi[ORC_MAXB * 3], psi[ORC_MAXB], gref[ORC_MAXB * 3], g[ORC_MAXB][3];
    double gbar[ORC_MAXB][3];
    orc_basis(dim, 1, pts + p * dim, phi, gphi);
    orc_basis(dim, vdeg, pts + p * dim, psi, gref);
    physical_gradients(dim, &fJt, nbv, gref, g);
    memset(gbar, 0, sizeof(gbar));
    double wq = wts[p], integrand = 0.0;
    for (int i = 0; i < nq; ++i)
      for (int a = 0; a < dim; ++a)
        for (int j = 0; j < nbv; ++j) {
          double bb = Bbar_in[i * ncol + a * nbv + j];
          integrand += bb * phi[i] * g[j][a];
          gbar[j][a] += wq * s * coef * bb * phi[i];
        }
    sbar += wq * coef * integrand;
    *cbar += wq * s * integrand;
    for (int j = 0; j < nbv; ++j)
      for (int mu = 0; mu < dim; ++mu)
        for (int a = 0; a < dim; ++a) Mbar[mu][a] += gref[j * dim + mu] * gbar[j][a];
  }
  double Jbar[3][3] = {{0}};
  for (int a = 0; a < dim; ++a)
    for (int mu = 0; mu < dim; ++mu) {
      double acc = 0.0;
      for (int k = 0; k < dim; ++k)
        for (int l = 0; l < dim; ++l) acc += Binv[k][a] * Mbar[k][l] * Binv[mu][l];
      Jbar[a][mu] = -acc + sbar * s * Binv[mu][a];
    }
  for (int a = 0; a < dim; ++a) {
    double col = 0.0;
    for (int mu = 0; mu < dim; ++mu) {
      Xbar[(mu + 1) * dim + a] = Jbar[a][mu];
      col += Jbar[a][mu];
    }
    Xbar[a] = -col;
  }
  return 0;
}

/* B[e] [(d+1)][d * nbv] for every element (coef may be NULL = 1); flags as in
 * orc_integrate. */
int orc_integrate_div(int dim, int vdeg, int64_t n_elem, int64_t n_vert, const int32_t* conn, const double* coords,
                      const double* coef, int q, double* B, int32_t* flags, int nthreads) {
  int nbv = orc_n_basis(dim, vdeg);
  if (nbv < 0 || dim < 2 || dim > 3) return -1;
  int64_t nb = (int64_t)(dim + 1) * dim * nbv;
  int any = 0;
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(static) num_threads(nthreads) reduction(| : any)
  for (int64_t e = 0; e < n_elem; ++e) {
    double X[12];
    double* Be = B + e * nb;
    int f = gather(dim, n_vert, conn + e * (dim + 1), coords, X);
    if (f == 0) {
      f = orc_element_matrix_div(dim, vdeg, X, coef ? coef[e] : 1.0, q, Be, NULL);
    } else {
      memset(Be, 0, sizeof(double) * nb);
    }
    if (flags) flags[e] = f;
    any |= f;
  }
  return any;
}

/* Reverse mode of orc_integrate_div over a mesh: Bbar [E][(d+1)][d * nbv] ->
 * dcoords [V][d] (overwritten; per-vertex sums in element order) and dcoef
 * [E] (may be NULL).  Flagged elements contribute nothing. */
int orc_integrate_div_vjp(int dim, int vdeg, int64_t n_elem, int64_t n_vert, const int32_t* conn,
                          const double* coords, const double* coef, int q, const double* Bbar, double* dcoords,
                          double* dcoef, int nthreads) {
  int nbv = orc_n_basis(dim, vdeg);
  if (nbv < 0 || dim < 2 || dim > 3) return -1;
  int64_t nb = (int64_t)(dim + 1) * dim * nbv;
  int nv = dim + 1;
  double* xbar = (double*)malloc(sizeof(double) * (size_t)(n_elem > 0 ? n_elem : 1) * nv * dim);
  int32_t* fl = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_elem > 0 ? n_elem : 1));
  if (!xbar || !fl) {
    free(xbar);
    free(fl);
    return -2;
  }
  if (nthreads < 1) nthreads = 1;
  int any = 0;
#pragma omp parallel for schedule(static) num_threads(nthreads) reduction(| : any)
  for (int64_t e = 0; e < n_elem; ++e) {
    double X[12], cb = 0.0;
    double* xb = xbar + e * nv * dim;
    int f = gather(dim, n_vert, conn + e * nv, coords, X);
    if (f == 0) f = orc_element_vjp_div(dim, vdeg, X, coef ? coef[e] : 1.0, q, Bbar + e * nb, xb, &cb);
    if (f != 0) {
      for (int k = 0; k < nv * dim; ++k) xb[k] = 0.0;
      cb = 0.0;
    }
    fl[e] = f;
    if (dcoef) dcoef[e] = cb;
    any |= f;
  }
  for (int64_t k = 0; k < n_vert * dim; ++k) dcoords[k] = 0.0;
  for (int64_t e = 0; e < n_elem; ++e) {
    if (fl[e] & ORC_FLAG_CONN) continue;
    for (int k = 0; k < nv; ++k) {
      int64_t v = conn[e * nv + k];
      for (int a = 0; a < dim; ++a) dcoords[v * dim + a] += xbar[(e * nv + k) * dim + a];
    }
  }
  free(xbar);
  free(fl);
  return any;
}

/* ------------------------------------------------------------------------ */
/* Reverse mode of the P1-coefficient Laplacian (Eqs. 20-23)               */
/* ------------------------------------------------------------------------ */
/* Reverse mode of orc_element_matrix_w1: given Abar = dL/dA, returns Xbar =
 * dL/dX [(d+1)*d] and wbar[d+1] = dL/dw_k for the vertex values w_k of the
 * coefficient c(xi) = sum_k w_k lambda_k(xi).  Per quadrature point, with
 * s = |det J| and I = sum_ij Abar_ij g_i.g_j:
 *   wbar_k += w_q s lambda_k I,   sbar += w_q c I,
 *   gbar_i += w_q s c sum_j (Abar_ij + Abar_ji) g_j
 * then, as in orc_element_vjp, with B = J^{-1}:
 *   Bbar[mu][a] += sum_i gref_i[mu] gbar_i[a],   Jbar = -B^T Bbar B^T + sbar s B^T. */
int orc_element_vjp_w1(int dim, int form, const double* X, const double* wv, int q, const double* Abar,
                       double* Xbar, double* wbar) {
  if (form == ORC_ELASTIC_P1 || !wv) return -1;
  int n = orc_form_n(form, dim);
  if (n < 0) return -1;
  int deg = form_degree(form), nb = orc_n_basis(dim, deg), nv = dim + 1;
  for (int k = 0; k < nv * dim; ++k) Xbar[k] = 0.0;
  for (int k = 0; k < nv; ++k) wbar[k] = 0.0;
  double J[3][3], Jt[3][3];
  jacobian(dim, X, J);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) Jt[a][b] = J[b][a];
  lu3 fJt;
  lu_factor(dim, Jt, &fJt);
  if (fJt.det == 0.0) return ORC_FLAG_DEGENERATE;
  double s = fabs(fJt.det);
  lu3 fJ;
  lu_factor(dim, J, &fJ);
  double B[3][3] = {{0}};
  for (int k = 0; k < dim; ++k) {
    double e[3] = {0, 0, 0};
    e[k] = 1.0;
    lu_solve(&fJ, e);
    for (int r = 0; r < dim; ++r) B[r][k] = e[r];
  }
  double pts[ORC_MAXPTS * 3], wts[ORC_MAXPTS];
  int np = orc_simplex_rule(dim, q, pts, wts);
  if (np < 0) return -1;
  double sbar = 0.0, Bbar[3][3] = {{0}};
  for (int p = 0; p < np; ++p) {
    const double* xi = pts + p * dim;
    double lam[4];
    lam[0] = 1.0;
    for (int k = 1; k <= dim; ++k) {
      lam[k] = xi[k - 1];
      lam[0] -= xi[k - 1];
    }
    double c = 0.0;
    for (int k = 0; k < nv; ++k) c += wv[k] * lam[k];
    double phi[ORC_MAXB], gref[ORC_MAXB * 3], g[ORC_MAXB][3], gbar[ORC_MAXB][3];
    orc_basis(dim, deg, xi, phi, gref);
    physical_gradients(dim, &fJt, nb, gref, g);
    memset(gbar, 0, sizeof(gbar));
    double wq = wts[p], integrand = 0.0;
    for (int i = 0; i < nb; ++i)
      for (int j = 0; j < nb; ++j) {
        double gg = 0.0;
        for (int a = 0; a < dim; ++a) gg += g[i][a] * g[j][a];
        integrand += Abar[i * n + j] * gg;
        double sym = Abar[i * n + j] + Abar[j * n + i];
        for (int a = 0; a < dim; ++a) gbar[i][a] += wq * s * c * sym * g[j][a];
      }
    sbar += wq * c * integrand;
    for (int k = 0; k < nv; ++k) wbar[k] += wq * s * lam[k] * integrand;
    for (int i = 0; i < nb; ++i)
      for (int mu = 0; mu < dim; ++mu)
        for (int a = 0; a < dim; ++a) Bbar[mu][a] += gref[i * dim + mu] * gbar[i][a];
  }
  double Jbar[3][3] = {{0}};
  for (int a = 0; a < dim; ++a)
    for (int mu = 0; mu < dim; ++mu) {
      double acc = 0.0;
      for (int k = 0; k < dim; ++k)
        for (int l = 0; l < dim; ++l) acc += B[k][a] * Bbar[k][l] * B[mu][l];
      Jbar[a][mu] = -acc + sbar * s * B[mu][a];
    }
  for (int a = 0; a < dim; ++a) {
    double col = 0.0;
    for (int mu = 0; mu < dim; ++mu) {
      Xbar[(mu + 1) * dim + a] = Jbar[a][mu];
      col += Jbar[a][mu];
    }
    Xbar[a] = -col;
  }
  return 0;
}

/* Reverse mode of orc_integrate_w1 over a mesh: Abar [E][n][n] -> dcoords
 * [V][d] and dwvert [V] (both overwritten; per-vertex sums in element order).
 * Flagged elements contribute nothing. */
int orc_integrate_w1_vjp(int dim, int form, int64_t n_elem, int64_t n_vert, const int32_t* conn,
                         const double* coords, const double* wvert, int q, const double* Abar, double* dcoords,
                         double* dwvert, int nthreads) {
  int n = orc_form_n(form, dim);
  if (n < 0 || form == ORC_ELASTIC_P1 || !wvert) return -1;
  int nv = dim + 1;
  double* xbar = (double*)malloc(sizeof(double) * (size_t)(n_elem > 0 ? n_elem : 1) * nv * dim);
  double* wb = (double*)malloc(sizeof(double) * (size_t)(n_elem > 0 ? n_elem : 1) * nv);
  int32_t* fl = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_elem > 0 ? n_elem : 1));
  if (!xbar || !wb || !fl) {
    free(xbar);
    free(wb);
    free(fl);
    return -2;
  }
  if (nthreads < 1) nthreads = 1;
  int any = 0;
#pragma omp parallel for schedule(static) num_threads(nthreads) reduction(| : any)
  for (int64_t e = 0; e < n_elem; ++e) {
    double X[12], wv[4];
    const int32_t* ce = conn + e * nv;
    double* xb = xbar + e * nv * dim;
    double* w = wb + e * nv;
    int f = gather(dim, n_vert, ce, coords, X);
    if (f == 0) {
      for (int k = 0; k < nv; ++k) wv[k] = wvert[ce[k]];
      f = orc_element_vjp_w1(dim, form, X, wv, q, Abar + e * (int64_t)n * n, xb, w);
    }
    if (f != 0) {
      for (int k = 0; k < nv * dim; ++k) xb[k] = 0.0;
      for (int k = 0; k < nv; ++k) w[k] = 0.0;
    }
    fl[e] = f;
    any |= f;
  }
  for (int64_t k = 0; k < n_vert * dim; ++k) dcoords[k] = 0.0;
  for (int64_t k = 0; k < n_vert; ++k) dwvert[k] = 0.0;
  for (int64_t e = 0; e < n_elem; ++e) {
    if (fl[e] & ORC_FLAG_CONN) continue;
    for (int k = 0; k < nv; ++k) {
      int64_t v = conn[e * nv + k];
      for (int a = 0; a < dim; ++a) dcoords[v * dim + a] += xbar[(e * nv + k) * dim + a];
      dwvert[v] += wb[e * nv + k];
    }
  }
  free(xbar);
  free(wb);
  free(fl);
  return any;
}
