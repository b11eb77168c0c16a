/*
 * lfem_oracle.c -- plain, slow, FP64 reference for isoparametric FE assembly.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header or table with the CUDA library; nothing here is used by the product
 * path.
 *
 * Structure follows the paper's element-by-element ("naive") assembly
 * (Sec. 3.3): precompute reference quantities, then for every element and
 * every quadrature point build the local matrices and add them into the
 * global sparse matrix.  Definitions:
 *   - Lagrange P1/P2 basis on the reference simplex (Eq. F_map requires the
 *     Lagrange property phi_j(x_i) = delta_ij; the printed P2 formulas of
 *     Eq. form_functions_s2dp2 are read as the Lagrange P2 basis
 *     lambda_a (2 lambda_a - 1), 4 lambda_i lambda_j).
 *   - Element map F(xi) = sum_a x_a phi_a(xi)          (Eq. F_map)
 *   - Integral transform with |det DF|               (Eq. basic integral formula)
 *     surfaces d=2,n=3: |dF/dxi1 x dF/dxi2| (the listing's vecnorm of the
 *     cross product, Sec. 3.4); bulk d=n: |det J|; curves d=1: |dF/dxi|.
 *   - Tangential gradient  grad_E phi = C_E^T grad^ phi with
 *     C_E = L_E^{-1}, L_E = [d1F, d2F, d1F x d2F]      (Eqs. surf grad - pre,
 *     jacobian_inv; the columns follow the listing of Sec. 3.4); bulk:
 *     C_E = J^{-1}; curves in R^2: L = [t, t_perp]; curves in R^3: t/|t|^2.
 *   - Local matrices by quadrature                  (Eqs. reference_quadrature_mass,
 *     reference_quadrature_stiffness); coefficient-weighted mass uses the
 *     given quadrature-point weights c_{e,q} (the pattern of the non-linear
 *     terms of Sec. 5.2).
 *   - Global matrices: sum over elements (Eqs. M matrix, A matrix), every
 *     structural pair (E[e,a], E[e,b]) kept, duplicates summed as sparse()
 *     does (Sec. 3.3).  Contributions to one slot are added in increasing
 *     (e, a, b) with Neumaier-compensated FP64 sums.
 *   - Adjoint (not in the paper): closed forms of d s and d(s G^{-1}) for the
 *     metric G = J^T J, see oracle_adjoint.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORACLE_MUTATION
#define ORACLE_MUTATION 0 /* >0 only in tests that plant a known mistake */
#endif

#define MAXREF 35
#define MAXD 3

static int n_ref(int dim, int order) {
  if (order == 1) return dim + 1;
  if (order == 2) return (dim + 1) * (dim + 2) / 2;
  /* orders 3, 4: C(p + d, d) */
  if (order == 3 || order == 4) {
    if (dim == 1) return order + 1;
    if (dim == 2) return (order + 1) * (order + 2) / 2;
    return (order + 1) * (order + 2) * (order + 3) / 6;
  }
  return -1;
}

/* Edge node (i, j) of the P2 element for local index dim+1+k. */
static const int EDGES1[1][2] = {{0, 1}};
static const int EDGES2[3][2] = {{0, 1}, {1, 2}, {2, 0}};
static const int EDGES3[6][2] = {{0, 1}, {1, 2}, {2, 0}, {0, 3}, {1, 3}, {2, 3}};

static const int (*edge_list(int dim))[2] {
  return dim == 1 ? EDGES1 : (dim == 2 ? EDGES2 : EDGES3);
}

/*
 * Orders p = 3, 4: the Lagrange basis of the nodes
 * lambda = alpha / p, |alpha| = p, written in barycentric coordinates as
 *   phi_alpha = prod_i l_{alpha_i}(lambda_i),  l_k(t) = prod_{j<k} (p t - j) / (j + 1),
 * which is 1 at its own node and 0 at every other (l_k vanishes at t = j/p,
 * j < k).  Node order: corners; then, edge by edge in the P2 edge order
 * (i, j), the p - 1 nodes alpha = (p - k) e_i + k e_j, k = 1..p-1 (from corner
 * i towards j); then the triangle's interior nodes (every alpha_i >= 1) in
 * increasing (alpha_1, alpha_2).  Tetrahedra: after the edges, the face
 * nodes face by face in the order (0,1,2), (0,1,3), (0,2,3), (1,2,3), each
 * face (i, j, l) with its nodes alpha_i, alpha_j, alpha_l >= 1 in increasing
 * (alpha_j, alpha_l); then the interior nodes (all four >= 1) in increasing
 * (alpha_1, alpha_2, alpha_3).
 */
static int node_multi_indices(int dim, int p, int (*al)[MAXD + 1]) {
  int cnt = 0;
  for (int i = 0; i <= dim; ++i) {
    for (int c = 0; c <= dim; ++c) al[cnt][c] = 0;
    al[cnt++][i] = p;
  }
  const int(*ed)[2] = edge_list(dim);
  const int ne = dim == 1 ? 1 : (dim == 2 ? 3 : 6);
  for (int k = 0; k < ne; ++k)
    for (int t = 1; t < p; ++t) {
      for (int c = 0; c <= dim; ++c) al[cnt][c] = 0;
      al[cnt][ed[k][0]] = p - t;
      al[cnt][ed[k][1]] = t;
      ++cnt;
    }
  if (dim == 2)
    for (int a1 = 1; a1 < p; ++a1)
      for (int a2 = 1; a1 + a2 < p; ++a2) {
        al[cnt][0] = p - a1 - a2;
        al[cnt][1] = a1;
        al[cnt][2] = a2;
        ++cnt;
      }
  if (dim == 3) {
#if ORACLE_MUTATION == 9
    static const int FACES3[4][3] = {{0, 1, 2}, {0, 2, 3}, {0, 1, 3}, {1, 2, 3}}; /* planted: face order */
#else
    static const int FACES3[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};
#endif
    for (int f = 0; f < 4; ++f)
      for (int aj = 1; aj < p; ++aj)
        for (int al2 = 1; aj + al2 < p; ++al2) {
          for (int c = 0; c <= dim; ++c) al[cnt][c] = 0;
          al[cnt][FACES3[f][0]] = p - aj - al2;
          al[cnt][FACES3[f][1]] = aj;
          al[cnt][FACES3[f][2]] = al2;
          ++cnt;
        }
    for (int a1 = 1; a1 < p; ++a1)
      for (int a2 = 1; a1 + a2 < p; ++a2)
        for (int a3 = 1; a1 + a2 + a3 < p; ++a3) {
          al[cnt][0] = p - a1 - a2 - a3;
          al[cnt][1] = a1;
          al[cnt][2] = a2;
          al[cnt][3] = a3;
          ++cnt;
        }
  }
  return cnt;
}

/* l_k(t) and its derivative for the order-p Lagrange factors. */
static void lag_factor(int p, int k, double t, double* v, double* dv) {
  double val = 1.0, der = 0.0;
  for (int j = 0; j < k; ++j) {
    const double f = (p * t - j) / (j + 1), df = (double)p / (j + 1);
#if ORACLE_MUTATION == 10
    der = der * f + val * df * 0.5; /* planted: half of the product rule's new term */
#else
    der = der * f + val * df;
#endif
    val *= f;
  }
  *v = val;
  *dv = der;
}

static void basis_high(int dim, int p, const double* lam, double dlam[][MAXD], double* phi, double dphi[][MAXD]) {
  int al[MAXREF][MAXD + 1];
  const int ref = node_multi_indices(dim, p, al);
  for (int a = 0; a < ref; ++a) {
    double v[MAXD + 1], dv[MAXD + 1];
    for (int i = 0; i <= dim; ++i) lag_factor(p, al[a][i], lam[i], &v[i], &dv[i]);
    double prod = 1.0;
    for (int i = 0; i <= dim; ++i) prod *= v[i];
    phi[a] = prod;
    for (int m = 0; m < dim; ++m) {
      double g = 0.0;
      for (int i = 0; i <= dim; ++i) {
        double rest = dv[i] * dlam[i][m];
        for (int l = 0; l <= dim; ++l)
          if (l != i) rest *= v[l];
        g += rest;
      }
      dphi[a][m] = g;
    }
  }
}

/* Basis values phi[a] and reference gradients dphi[a][m] at reference point xi. */
static void basis(int dim, int order, const double* xi, double* phi, double dphi[][MAXD]) {
  double lam[MAXD + 1], dlam[MAXD + 1][MAXD];
  double s = 0.0;
  for (int m = 0; m < dim; ++m) s += xi[m];
  lam[0] = 1.0 - s;
  for (int m = 0; m < dim; ++m) lam[m + 1] = xi[m];
  for (int i = 0; i <= dim; ++i)
    for (int m = 0; m < dim; ++m) dlam[i][m] = (i == 0) ? -1.0 : (i == m + 1 ? 1.0 : 0.0);

  if (order == 1) {
    for (int a = 0; a <= dim; ++a) {
      phi[a] = lam[a];
      for (int m = 0; m < dim; ++m) dphi[a][m] = dlam[a][m];
    }
    return;
  }
  if (order >= 3) {
    basis_high(dim, order, lam, dlam, phi, dphi);
    return;
  }
  for (int a = 0; a <= dim; ++a) {
    phi[a] = lam[a] * (2.0 * lam[a] - 1.0);
    for (int m = 0; m < dim; ++m) dphi[a][m] = (4.0 * lam[a] - 1.0) * dlam[a][m];
  }
  const int(*ed)[2] = edge_list(dim);
  int ne = n_ref(dim, 2) - (dim + 1);
  for (int k = 0; k < ne; ++k) {
    int i = ed[k][0], j = ed[k][1];
#if ORACLE_MUTATION == 2
    if (k == 0 && ne > 1) { i = ed[1][0]; j = ed[1][1]; } /* planted: wrong edge-node order */
#endif
    double f = 4.0;
#if ORACLE_MUTATION == 1
    f = 2.0; /* planted: wrong edge-bubble scaling */
#endif
    phi[dim + 1 + k] = f * lam[i] * lam[j];
    for (int m = 0; m < dim; ++m) dphi[dim + 1 + k][m] = f * (lam[i] * dlam[j][m] + lam[j] * dlam[i][m]);
  }
}

int oracle_tabulate(int dim, int order, int nq, const double* xi, double* phi, double* dphi) {
  int ref = n_ref(dim, order);
  if (ref < 0 || dim < 1 || dim > 3) return 1;
  for (int q = 0; q < nq; ++q) {
    double dp[MAXREF][MAXD];
    basis(dim, order, xi + q * dim, phi + q * ref, dp);
    for (int a = 0; a < ref; ++a)
      for (int m = 0; m < dim; ++m) dphi[(q * ref + a) * dim + m] = dp[a][m];
  }
  return 0;
}

/* Inverse of an n x n matrix (n <= 3), row-major; returns the determinant. */
static double inv_small(int n, const double* A, double* Ai) {
  if (n == 1) {
    Ai[0] = 1.0 / A[0];
    return A[0];
  }
  if (n == 2) {
    double det = A[0] * A[3] - A[1] * A[2];
    Ai[0] = A[3] / det;
    Ai[1] = -A[1] / det;
    Ai[2] = -A[2] / det;
    Ai[3] = A[0] / det;
    return det;
  }
  double c00 = A[4] * A[8] - A[5] * A[7];
  double c01 = A[5] * A[6] - A[3] * A[8];
  double c02 = A[3] * A[7] - A[4] * A[6];
  double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
  Ai[0] = c00 / det;
  Ai[1] = (A[2] * A[7] - A[1] * A[8]) / det;
  Ai[2] = (A[1] * A[5] - A[2] * A[4]) / det;
  Ai[3] = c01 / det;
  Ai[4] = (A[0] * A[8] - A[2] * A[6]) / det;
  Ai[5] = (A[2] * A[3] - A[0] * A[5]) / det;
  Ai[6] = c02 / det;
  Ai[7] = (A[1] * A[6] - A[0] * A[7]) / det;
  Ai[8] = (A[0] * A[4] - A[1] * A[3]) / det;
  return det;
}

typedef struct {
  double J[MAXD][MAXD]; /* J[i][m] = d x_i / d xi_m, i < n, m < d */
  double s;             /* surface / volume element |det DF| */
  double grad[MAXREF][MAXD]; /* tangential gradients grad_E phi_a in R^n */
  double phi[MAXREF];
  double dphi[MAXREF][MAXD];
} qp_geom;

/* Geometry at one quadrature point of one element (Sec. 3.2). */
static void element_qp(int dim, int order, int n, const double* X /*[ref][n]*/, const double* xi,
                       qp_geom* g) {
  int ref = n_ref(dim, order);
  basis(dim, order, xi, g->phi, g->dphi);
  for (int i = 0; i < n; ++i)
    for (int m = 0; m < dim; ++m) {
      double acc = 0.0;
      for (int a = 0; a < ref; ++a) acc += X[a * n + i] * g->dphi[a][m];
      g->J[i][m] = acc;
    }
  if (dim == n) {
    /* bulk: C_E = J^{-1}, grad phi = J^{-T} grad^ phi */
    double Jm[9], Ji[9];
    for (int i = 0; i < n; ++i)
      for (int m = 0; m < n; ++m) Jm[i * n + m] = g->J[i][m];
    double det = inv_small(n, Jm, Ji);
    g->s = fabs(det);
    for (int a = 0; a < ref; ++a)
      for (int i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int m = 0; m < n; ++m) acc += Ji[m * n + i] * g->dphi[a][m]; /* (J^{-T})_{im} = Ji[m][i] */
#if ORACLE_MUTATION == 4
        acc = 0.0;
        for (int m = 0; m < n; ++m) acc += Ji[i * n + m] * g->dphi[a][m]; /* planted: J^{-1} for J^{-T} */
#endif
        g->grad[a][i] = acc;
      }
    return;
  }
  if (dim == 2 && n == 3) {
    /* L = [t1, t2, t1 x t2] (columns), C = L^{-1}, grad = C^T (d1 phi, d2 phi, 0) */
    double t1[3] = {g->J[0][0], g->J[1][0], g->J[2][0]};
    double t2[3] = {g->J[0][1], g->J[1][1], g->J[2][1]};
    double L3[3] = {t1[1] * t2[2] - t1[2] * t2[1], t1[2] * t2[0] - t1[0] * t2[2], t1[0] * t2[1] - t1[1] * t2[0]};
    g->s = sqrt(L3[0] * L3[0] + L3[1] * L3[1] + L3[2] * L3[2]);
#if ORACLE_MUTATION == 3
    g->s = sqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]) * sqrt(t2[0] * t2[0] + t2[1] * t2[1] + t2[2] * t2[2]);
#endif
    double L[9], C[9];
    for (int i = 0; i < 3; ++i) {
      L[i * 3 + 0] = t1[i];
      L[i * 3 + 1] = t2[i];
      L[i * 3 + 2] = L3[i];
    }
    inv_small(3, L, C);
    for (int a = 0; a < ref; ++a) {
      double gh[3] = {g->dphi[a][0], g->dphi[a][1], 0.0};
      for (int i = 0; i < 3; ++i) g->grad[a][i] = C[0 * 3 + i] * gh[0] + C[1 * 3 + i] * gh[1] + C[2 * 3 + i] * gh[2];
    }
    return;
  }
  if (dim == 1 && n == 2) {
    /* L = [t, t_perp], grad = L^{-T} (phi', 0) */
    double t[2] = {g->J[0][0], g->J[1][0]};
    g->s = sqrt(t[0] * t[0] + t[1] * t[1]);
    double L[4] = {t[0], -t[1], t[1], t[0]}, C[4];
    inv_small(2, L, C);
    for (int a = 0; a < ref; ++a)
      for (int i = 0; i < 2; ++i) g->grad[a][i] = C[0 * 2 + i] * g->dphi[a][0];
    return;
  }
  if (dim == 1 && n == 3) {
    double t[3] = {g->J[0][0], g->J[1][0], g->J[2][0]};
    double tt = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    g->s = sqrt(tt);
    for (int a = 0; a < ref; ++a)
      for (int i = 0; i < 3; ++i) g->grad[a][i] = t[i] * g->dphi[a][0] / tt;
    return;
  }
  g->s = NAN;
}

static int check_combo(int dim, int order, int n) {
  if (dim < 1 || dim > 3 || n < dim || n > 3) return 1;
  if (order < 1 || order > 4) return 1;
  if (dim == 2 && n == 3) return 0;
  if (dim == n) return 0;
  if (dim == 1) return 0;
  return 1;
}

static void gather(const double* coords, int n, const int32_t* conn, int ref, int64_t e, double* X) {
  for (int a = 0; a < ref; ++a) {
    int64_t v = conn[e * ref + a];
    for (int i = 0; i < n; ++i) X[a * n + i] = coords[v * n + i];
  }
}

/* Physical quadrature points x_q = F_E(xi_q) (Eq. F_map): out [nE][nq][n]. */
int oracle_eval_points(const double* coords, int n, const int32_t* conn, int64_t nE, int dim, int order,
                       int nq, const double* xi, double* out) {
  int ref = n_ref(dim, order);
  if (check_combo(dim, order, n)) return 1;
  double X[MAXREF * MAXD];
  for (int64_t e = 0; e < nE; ++e) {
    gather(coords, n, conn, ref, e, X);
    for (int q = 0; q < nq; ++q) {
      double phi[MAXREF], dp[MAXREF][MAXD];
      basis(dim, order, xi + q * dim, phi, dp);
      for (int i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int a = 0; a < ref; ++a) acc += phi[a] * X[a * n + i];
        out[(e * nq + q) * n + i] = acc;
      }
    }
  }
  return 0;
}

/* Per-quadrature-point geometry: J [nE][nq][n][d], s [nE][nq], Ginv [nE][nq][d][d]. */
int oracle_geometry(const double* coords, int n, const int32_t* conn, int64_t nE, int dim, int order, int nq,
                    const double* xi, double* Jout, double* sout, double* Ginv_out) {
  int ref = n_ref(dim, order);
  if (check_combo(dim, order, n)) return 1;
  double X[MAXREF * MAXD];
  for (int64_t e = 0; e < nE; ++e) {
    gather(coords, n, conn, ref, e, X);
    for (int q = 0; q < nq; ++q) {
      qp_geom g;
      element_qp(dim, order, n, X, xi + q * dim, &g);
      int64_t b = e * nq + q;
      if (sout) sout[b] = g.s;
      if (Jout)
        for (int i = 0; i < n; ++i)
          for (int m = 0; m < dim; ++m) Jout[(b * n + i) * dim + m] = g.J[i][m];
      if (Ginv_out) {
        double G[9], Gi[9];
        for (int m = 0; m < dim; ++m)
          for (int k = 0; k < dim; ++k) {
            double acc = 0.0;
            for (int i = 0; i < n; ++i) acc += g.J[i][m] * g.J[i][k];
            G[m * dim + k] = acc;
          }
        inv_small(dim, G, Gi);
        for (int m = 0; m < dim * dim; ++m) Ginv_out[b * dim * dim + m] = Gi[m];
      }
    }
  }
  return 0;
}

/* Local matrices of one element, full ref x ref (Eqs. reference_quadrature_*). */
static void local_matrices(int dim, int order, int n, const double* X, int nq, const double* xi, const double* w,
                           const double* coef_e, double* Ml, double* Al, double* Cl) {
  int ref = n_ref(dim, order);
  for (int k = 0; k < ref * ref; ++k) Ml[k] = Al[k] = Cl[k] = 0.0;
  for (int q = 0; q < nq; ++q) {
    qp_geom g;
    element_qp(dim, order, n, X, xi + q * dim, &g);
    double ws = w[q] * g.s;
#if ORACLE_MUTATION == 5
    ws = g.s; /* planted: quadrature weight dropped */
#endif
    double c = coef_e ? coef_e[q] : 0.0;
    for (int a = 0; a < ref; ++a)
      for (int b = 0; b < ref; ++b) {
        double dot = 0.0;
        for (int i = 0; i < n; ++i) dot += g.grad[a][i] * g.grad[b][i];
        Ml[a * ref + b] += ws * g.phi[a] * g.phi[b];
        Al[a * ref + b] += ws * dot;
        Cl[a * ref + b] += ws * c * g.phi[a] * g.phi[b];
      }
  }
}

/* Local matrices for every element: out [nE][ref][ref] each (NULL to skip). */
int oracle_local(const double* coords, int n, const int32_t* conn, int64_t nE, int dim, int order, int nq,
                 const double* xi, const double* w, const double* coef, double* Mout, double* Aout, double* Cout) {
  int ref = n_ref(dim, order);
  if (check_combo(dim, order, n)) return 1;
  double X[MAXREF * MAXD], Ml[MAXREF * MAXREF], Al[MAXREF * MAXREF], Cl[MAXREF * MAXREF];
  for (int64_t e = 0; e < nE; ++e) {
    gather(coords, n, conn, ref, e, X);
    local_matrices(dim, order, n, X, nq, xi, w, coef ? coef + e * nq : NULL, Ml, Al, Cl);
    for (int k = 0; k < ref * ref; ++k) {
      if (Mout) Mout[e * ref * ref + k] = Ml[k];
      if (Aout) Aout[e * ref * ref + k] = Al[k];
      if (Cout) Cout[e * ref * ref + k] = Cl[k];
    }
  }
  return 0;
}

/* Slot of (row, col) in a CSR pattern with ascending columns; -1 if absent. */
static int64_t find_slot(const int64_t* row_ptr, const int32_t* col_idx, int64_t row, int32_t col) {
  int64_t lo = row_ptr[row], hi = row_ptr[row + 1];
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (col_idx[mid] < col) lo = mid + 1;
    else hi = mid;
  }
  if (lo < row_ptr[row + 1] && col_idx[lo] == col) return lo;
  return -1;
}

static void neumaier_add(double* sum, double* comp, double x) {
  double t = *sum + x;
  if (fabs(*sum) >= fabs(x)) *comp += (*sum - t) + x;
  else *comp += (x - t) + *sum;
  *sum = t;
}

/*
 * Global assembly into a given CSR pattern (Eqs. M matrix, A matrix).
 * M/A/MC: [nnz] outputs (NULL to skip).  coef: [nE][nq] or NULL (then MC = 0).
 * Returns 0, or 2 if a pair has no slot in the pattern.
 */
int oracle_assemble(const double* coords, int n, const int32_t* conn, int64_t nE, int dim, int order, int nq,
                    const double* xi, const double* w, const double* coef, const int64_t* row_ptr,
                    const int32_t* col_idx, int64_t nnz, double* M, double* A, double* MC) {
  int ref = n_ref(dim, order);
  if (check_combo(dim, order, n)) return 1;
  double* acc = (double*)calloc((size_t)nnz * 6, sizeof(double));
  if (!acc) return 3;
  double X[MAXREF * MAXD], Ml[MAXREF * MAXREF], Al[MAXREF * MAXREF], Cl[MAXREF * MAXREF];
  int rc = 0;
  for (int64_t e = 0; e < nE && !rc; ++e) {
    gather(coords, n, conn, ref, e, X);
    local_matrices(dim, order, n, X, nq, xi, w, coef ? coef + e * nq : NULL, Ml, Al, Cl);
    for (int a = 0; a < ref; ++a)
      for (int b = 0; b < ref; ++b) {
        int64_t s = find_slot(row_ptr, col_idx, conn[e * ref + a], conn[e * ref + b]);
        if (s < 0) {
          rc = 2;
          break;
        }
        neumaier_add(&acc[6 * s + 0], &acc[6 * s + 1], Ml[a * ref + b]);
        neumaier_add(&acc[6 * s + 2], &acc[6 * s + 3], Al[a * ref + b]);
        neumaier_add(&acc[6 * s + 4], &acc[6 * s + 5], Cl[a * ref + b]);
      }
  }
  for (int64_t s = 0; s < nnz; ++s) {
    if (M) M[s] = acc[6 * s + 0] + acc[6 * s + 1];
    if (A) A[s] = acc[6 * s + 2] + acc[6 * s + 3];
    if (MC) MC[s] = acc[6 * s + 4] + acc[6 * s + 5];
  }
  free(acc);
  return rc;
}

/*
 * Adjoint of L = sum_s (gM[s] M[s] + gA[s] A[s] + gMC[s] MC[s]) with respect to
 * the node coordinates (and the quadrature-point coefficient).
 *
 * Per element and quadrature point, with G = J^T J, s = sqrt(det G):
 *   Gbar_ab          = g[slot(E[a], E[b])]  (all a, b)
 *   m_q              = sum_ab (GbarM_ab + c_q GbarC_ab) phi_a phi_b
 *   K_q              = sym( sum_ab GbarA_ab grad^phi_a grad^phi_b^T )     (d x d)
 *   L_e              = sum_q w_q ( s m_q + s <K_q, G^{-1}> )
 *   ds               = s <J G^{-1}, dJ>
 *   d(s G^{-1})      = s [ <J G^{-1}, dJ> G^{-1} - G^{-1}(dJ^T J + J^T dJ) G^{-1} ]
 *   dL/dJ_q          = w_q s [ (m_q + <K_q, G^{-1}>) J G^{-1} - 2 J G^{-1} K_q G^{-1} ]
 *   dL/dx_{E[k]}    += dL/dJ_q grad^phi_k(xi_q)
 *   dL/dc_{e,q}      = w_q s sum_ab GbarC_ab phi_a phi_b
 * g_coords [N][n] is overwritten; g_coef [nE][nq] may be NULL.
 */
int oracle_adjoint(const double* coords, int n, const int32_t* conn, int64_t nE, int64_t n_nodes, int dim,
                   int order, int nq, const double* xi, const double* w, const double* coef,
                   const int64_t* row_ptr, const int32_t* col_idx, const double* gM, const double* gA,
                   const double* gMC, double* g_coords, double* g_coef) {
  int ref = n_ref(dim, order);
  if (check_combo(dim, order, n)) return 1;
  double* acc = (double*)calloc((size_t)n_nodes * n * 2, sizeof(double));
  if (!acc) return 3;
  double X[MAXREF * MAXD];
  double GM[MAXREF * MAXREF], GA[MAXREF * MAXREF], GC[MAXREF * MAXREF];
  int rc = 0;
  for (int64_t e = 0; e < nE && !rc; ++e) {
    gather(coords, n, conn, ref, e, X);
    for (int a = 0; a < ref; ++a)
      for (int b = 0; b < ref; ++b) {
        int64_t s = find_slot(row_ptr, col_idx, conn[e * ref + a], conn[e * ref + b]);
        if (s < 0) {
          rc = 2;
          break;
        }
        GM[a * ref + b] = gM ? gM[s] : 0.0;
        GA[a * ref + b] = gA ? gA[s] : 0.0;
        GC[a * ref + b] = gMC ? gMC[s] : 0.0;
      }
    double ge[MAXREF][MAXD];
    memset(ge, 0, sizeof(ge));
    for (int q = 0; q < nq; ++q) {
      qp_geom g;
      element_qp(dim, order, n, X, xi + q * dim, &g);
      double G[9], Gi[9];
      for (int m = 0; m < dim; ++m)
        for (int k = 0; k < dim; ++k) {
          double t = 0.0;
          for (int i = 0; i < n; ++i) t += g.J[i][m] * g.J[i][k];
          G[m * dim + k] = t;
        }
      inv_small(dim, G, Gi);
      double s = g.s;
      double c = coef ? coef[e * nq + q] : 0.0;
      double mq = 0.0, mc = 0.0, K[9] = {0};
      for (int a = 0; a < ref; ++a)
        for (int b = 0; b < ref; ++b) {
          double pp = g.phi[a] * g.phi[b];
          mq += (GM[a * ref + b] + c * GC[a * ref + b]) * pp;
          mc += GC[a * ref + b] * pp;
          for (int m = 0; m < dim; ++m)
            for (int k = 0; k < dim; ++k) K[m * dim + k] += GA[a * ref + b] * g.dphi[a][m] * g.dphi[b][k];
        }
      double Ks[9];
      for (int m = 0; m < dim; ++m)
        for (int k = 0; k < dim; ++k) Ks[m * dim + k] = 0.5 * (K[m * dim + k] + K[k * dim + m]);
      double KG = 0.0;
      for (int m = 0; m < dim * dim; ++m) KG += Ks[m] * Gi[m];
      /* JGi = J G^{-1} (n x d); B = G^{-1} K G^{-1} (d x d) */
      double JGi[MAXD][MAXD], T[9], B[9];
      for (int i = 0; i < n; ++i)
        for (int k = 0; k < dim; ++k) {
          double t = 0.0;
          for (int m = 0; m < dim; ++m) t += g.J[i][m] * Gi[m * dim + k];
          JGi[i][k] = t;
        }
      for (int m = 0; m < dim; ++m)
        for (int k = 0; k < dim; ++k) {
          double t = 0.0;
          for (int l = 0; l < dim; ++l) t += Gi[m * dim + l] * Ks[l * dim + k];
          T[m * dim + k] = t;
        }
      for (int m = 0; m < dim; ++m)
        for (int k = 0; k < dim; ++k) {
          double t = 0.0;
          for (int l = 0; l < dim; ++l) t += T[m * dim + l] * Gi[l * dim + k];
          B[m * dim + k] = t;
        }
      double two = 2.0;
#if ORACLE_MUTATION == 6
      two = 1.0; /* planted: factor of the symmetric metric variation dropped */
#endif
      double dLdJ[MAXD][MAXD];
      for (int i = 0; i < n; ++i)
        for (int k = 0; k < dim; ++k) {
          double JB = 0.0;
          for (int m = 0; m < dim; ++m) JB += g.J[i][m] * B[m * dim + k];
          dLdJ[i][k] = w[q] * s * ((mq + KG) * JGi[i][k] - two * JB);
        }
      for (int a = 0; a < ref; ++a)
        for (int i = 0; i < n; ++i) {
          double t = 0.0;
          for (int k = 0; k < dim; ++k) t += dLdJ[i][k] * g.dphi[a][k];
          ge[a][i] += t;
        }
      if (g_coef) g_coef[e * nq + q] = w[q] * s * mc;
    }
    for (int a = 0; a < ref; ++a) {
      int64_t v = conn[e * ref + a];
      for (int i = 0; i < n; ++i) neumaier_add(&acc[2 * (v * n + i)], &acc[2 * (v * n + i) + 1], ge[a][i]);
    }
  }
  for (int64_t k = 0; k < n_nodes * n; ++k) g_coords[k] = acc[2 * k] + acc[2 * k + 1];
  free(acc);
  return rc;
}

/*
 * Load vector (Sec. 2, the load vector of the Poisson problem): b_j =
 * integral over Gamma_h of f_h phi_j, with f_h = sum_i f_i phi_i the
 * interpolant of the nodal values f (so b = M f).  Per element and quadrature
 * point: f_q = sum_b f_{E[b]} phi_b, local b_a += w_q s_q f_q phi_a; the local
 * vectors are added into b in increasing (e, a) with Neumaier sums.
 * b [n_nodes] is overwritten.
 */
int oracle_load(const double* coords, int n, const int32_t* conn, int64_t nE, int64_t n_nodes, int dim, int order,
                int nq, const double* xi, const double* w, const double* f, double* b) {
  int ref = n_ref(dim, order);
  if (check_combo(dim, order, n)) return 1;
  double* acc = (double*)calloc((size_t)n_nodes * 2, sizeof(double));
  if (!acc) return 3;
  double X[MAXREF * MAXD];
  for (int64_t e = 0; e < nE; ++e) {
    gather(coords, n, conn, ref, e, X);
    double loc[MAXREF] = {0};
    for (int q = 0; q < nq; ++q) {
      qp_geom g;
      element_qp(dim, order, n, X, xi + q * dim, &g);
      double fq = 0.0;
      for (int a = 0; a < ref; ++a) fq += f[conn[e * ref + a]] * g.phi[a];
      double sq = g.s;
#if ORACLE_MUTATION == 7
      sq = 1.0; /* planted: surface element dropped */
#endif
      for (int a = 0; a < ref; ++a) loc[a] += w[q] * sq * fq * g.phi[a];
    }
    for (int a = 0; a < ref; ++a) {
      int64_t v = conn[e * ref + a];
      neumaier_add(&acc[2 * v], &acc[2 * v + 1], loc[a]);
    }
  }
  for (int64_t v = 0; v < n_nodes; ++v) b[v] = acc[2 * v] + acc[2 * v + 1];
  free(acc);
  return 0;
}

/*
 * Non-linear vectors of the mean curvature flow system (Sec. 5.1, after
 * Kovacs-Li-Lubich): with u = (nu, H) given at the nodes ([n_nodes][4]),
 * nu_h and H_h their interpolants and alpha^2 = |grad_Gamma_h nu_h|^2 (the
 * Frobenius norm of the tangential gradient of the normal field),
 *   f1[k][j] = integral of alpha^2 (nu_h)_k phi_j   (k = 0, 1, 2)
 *   f2[j]    = integral of alpha^2 H_h phi_j,
 * written to out[k * n_nodes + j] (k = 0..2) and out[3 * n_nodes + j].  The
 * tangential gradient is the oracle's C_E^T grad^ phi (as for the stiffness).
 * Surfaces (dim 2 in R^3) only.
 */
int oracle_kll(const double* coords, const int32_t* conn, int64_t nE, int64_t n_nodes, int order, int nq,
               const double* xi, const double* w, const double* u, double* out) {
  const int dim = 2, n = 3;
  int ref = n_ref(dim, order);
  if (check_combo(dim, order, n)) return 1;
  double* acc = (double*)calloc((size_t)n_nodes * 8, sizeof(double));
  if (!acc) return 3;
  double X[MAXREF * MAXD];
  for (int64_t e = 0; e < nE; ++e) {
    gather(coords, n, conn, ref, e, X);
    double loc[MAXREF][4];
    memset(loc, 0, sizeof(loc));
    for (int q = 0; q < nq; ++q) {
      qp_geom g;
      element_qp(dim, order, n, X, xi + q * dim, &g);
      double val[4] = {0, 0, 0, 0};     /* nu_h (3), H_h at the point */
      double gnu[3][3] = {{0}};         /* gnu[k][i] = i-th component of grad_Gamma (nu_h)_k */
      for (int b = 0; b < ref; ++b) {
        const double* ub = u + (int64_t)conn[e * ref + b] * 4;
        for (int k = 0; k < 4; ++k) val[k] += ub[k] * g.phi[b];
        for (int k = 0; k < 3; ++k)
          for (int i = 0; i < 3; ++i) {
#if ORACLE_MUTATION == 8
            gnu[k][i] += ub[k] * (i < dim ? g.dphi[b][i] : 0.0); /* planted: reference gradient */
#else
            gnu[k][i] += ub[k] * g.grad[b][i];
#endif
          }
      }
      double alpha2 = 0.0;
      for (int k = 0; k < 3; ++k)
        for (int i = 0; i < 3; ++i) alpha2 += gnu[k][i] * gnu[k][i];
      for (int a = 0; a < ref; ++a)
        for (int k = 0; k < 4; ++k) loc[a][k] += w[q] * g.s * alpha2 * val[k] * g.phi[a];
    }
    for (int a = 0; a < ref; ++a) {
      int64_t v = conn[e * ref + a];
      for (int k = 0; k < 4; ++k) neumaier_add(&acc[(k * n_nodes + v) * 2], &acc[(k * n_nodes + v) * 2 + 1], loc[a][k]);
    }
  }
  for (int64_t i = 0; i < 4 * n_nodes; ++i) out[i] = acc[2 * i] + acc[2 * i + 1];
  free(acc);
  return 0;
}

int oracle_mutation_id(void) { return ORACLE_MUTATION; }

/*
 * The same global assembly on every host core (the timed CPU baseline), with
 * the result bit-identical to oracle_assemble: elements are taken in chunks;
 * the chunk's local matrices are computed element-parallel into a buffer,
 * then each thread adds them row by row -- for a row i, its incident
 * elements of the chunk in increasing e, for each the local rows a with
 * conn[e][a] = i in increasing a, each local column b in increasing b -- so
 * that every slot receives its contributions in the single-thread order
 * (e, a, b), with the same Neumaier sums.  nthreads <= 0: all threads OpenMP
 * offers.  Returns the codes of oracle_assemble, or 3 if out of memory.
 */
int oracle_assemble_threads(const double* coords, int n, const int32_t* conn, int64_t nE, int64_t n_nodes, int dim,
                            int order, int nq, const double* xi, const double* w, const double* coef,
                            const int64_t* row_ptr, const int32_t* col_idx, int64_t nnz, double* M, double* A,
                            double* MC, int nthreads) {
  int ref = n_ref(dim, order);
  if (check_combo(dim, order, n)) return 1;
  const int64_t chunk = 65536;
  const int64_t rr = (int64_t)ref * ref;
  double* acc = (double*)calloc((size_t)nnz * 6, sizeof(double));
  double* loc = (double*)malloc(sizeof(double) * (size_t)(chunk < nE ? chunk : (nE > 0 ? nE : 1)) * rr * 3);
  int64_t* inc_ptr = (int64_t*)calloc((size_t)n_nodes + 1, sizeof(int64_t));
  int64_t* inc = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nE * ref > 0 ? nE * ref : 1));
  int64_t* fill = (int64_t*)calloc((size_t)n_nodes + 1, sizeof(int64_t));
  int rc = 0;
  if (!acc || !loc || !inc_ptr || !inc || !fill) rc = 3;
  /* node -> incidences (e * ref + a), ascending in e then a: a counting sort */
  if (!rc) {
    for (int64_t k = 0; k < nE * ref; ++k) {
      if (conn[k] < 0 || conn[k] >= n_nodes) {
        rc = 2;
        break;
      }
      ++inc_ptr[conn[k] + 1];
    }
  }
  if (!rc) {
    for (int64_t i = 0; i < n_nodes; ++i) inc_ptr[i + 1] += inc_ptr[i];
    for (int64_t k = 0; k < nE * ref; ++k) inc[inc_ptr[conn[k]] + fill[conn[k]]++] = k;
  }
  if (nthreads > 0) omp_set_num_threads(nthreads);
  /* per row, the next incidence not yet added */
  for (int64_t i = 0; i < n_nodes && !rc; ++i) fill[i] = inc_ptr[i];
  for (int64_t c0 = 0; c0 < nE && !rc; c0 += chunk) {
    const int64_t c1 = c0 + chunk < nE ? c0 + chunk : nE;
#pragma omp parallel for schedule(static)
    for (int64_t e = c0; e < c1; ++e) {
      double X[MAXREF * MAXD];
      double* Ml = loc + (e - c0) * rr * 3;
      gather(coords, n, conn, ref, e, X);
      local_matrices(dim, order, n, X, nq, xi, w, coef ? coef + e * nq : NULL, Ml, Ml + rr, Ml + 2 * rr);
    }
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1024) reduction(| : bad)
    for (int64_t i = 0; i < n_nodes; ++i) {
      int64_t k = fill[i];
      for (; k < inc_ptr[i + 1] && inc[k] / ref < c1; ++k) {
        const int64_t e = inc[k] / ref;
        const int a = (int)(inc[k] % ref);
        const double* Ml = loc + (e - c0) * rr * 3;
        for (int b = 0; b < ref; ++b) {
          int64_t s = find_slot(row_ptr, col_idx, i, conn[e * ref + b]);
          if (s < 0) {
            bad = 1;
            continue;
          }
          neumaier_add(&acc[6 * s + 0], &acc[6 * s + 1], Ml[a * ref + b]);
          neumaier_add(&acc[6 * s + 2], &acc[6 * s + 3], Ml[rr + a * ref + b]);
          neumaier_add(&acc[6 * s + 4], &acc[6 * s + 5], Ml[2 * rr + a * ref + b]);
        }
      }
      fill[i] = k;
    }
    if (bad) rc = 2;
  }
  if (!rc) {
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < nnz; ++s) {
      if (M) M[s] = acc[6 * s + 0] + acc[6 * s + 1];
      if (A) A[s] = acc[6 * s + 2] + acc[6 * s + 3];
      if (MC) MC[s] = acc[6 * s + 4] + acc[6 * s + 5];
    }
  }
  free(acc);
  free(loc);
  free(inc_ptr);
  free(inc);
  free(fill);
  return rc;
}

/* Threads the all-core assembly uses by default. */
int oracle_max_threads(void) { return omp_get_max_threads(); }
