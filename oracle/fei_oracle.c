/*
 * fei_oracle.c -- plain FP64 CPU oracle for element integration on
 * higher-order prisms (Kruzel & Banas, "Vectorized OpenCL implementation of
 * numerical integration for higher order finite elements").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this file.  It is used by the test-suite, by the smoke check and
 * by the CPU-baseline leg of the benchmark, and it shares no code, header,
 * table or constant with the CUDA path.
 *
 * What it computes (Sec. 2, Eq. (1) / Eq. (2), generalised to the
 * convection-diffusion-reaction form):
 *
 *   A_e[i][j] = sum_q w_q det J(xi_q) * ( grad phi_i . K_q grad phi_j
 *                                       + phi_i  b_q . grad phi_j
 *                                       + c_q phi_i phi_j )
 *   b_e[i]    = sum_q w_q det J(xi_q) * f_q phi_i
 *
 * with grad phi = J^{-T} grad_ref phi (chain rule of the change of variables
 * x(xi), Sec. 2), i = test function (row), j = trial function (column).
 * The loops follow Algorithm 1: element -> quadrature point -> i -> j -> k,
 * with the integration-point loop outside the shape-function loops (Sec. 2.1).
 *
 * Readings where the paper is silent (each is one fixed convention):
 *  - reference prism: triangle {xi1, xi2 >= 0, xi1 + xi2 <= 1} x [-1, 1]
 *    (volume 1);
 *  - basis: orthonormal Dubiner triangle polynomials times normalised
 *    Legendre polynomials in zeta ("complete triangle basis x 1D functions",
 *    Table 1 and the text beside it); N_sh = (p+1)^2 (p+2)/2 (Table 1);
 *  - basis order: index = k * T_p + t(m, n), T_p = (p+1)(p+2)/2, k the zeta
 *    degree, t running over total degree d = m + n ascending, then n
 *    ascending inside d;
 *  - quadrature: Duffy-collapsed Gauss-Legendre, (p+1) points per direction,
 *    q = (iz * (p+1) + iv) * (p+1) + iu, xi1 = (1+u)(1-v)/4, xi2 = (1+v)/2,
 *    zeta = z, w = w_u w_v (1-v)/8 * w_z;
 *  - geometry: bilinear prism (Sec. 4), bottom vertices 0,1,2 at zeta = -1,
 *    top vertex a+3 above vertex a;
 *  - det J <= 0 at any point, or a non-finite input, flags the element and
 *    its outputs are zero.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define FO_OK 0
#define FO_ERR_INVALID_ARG 1
#define FO_ERR_INVALID_DEGREE 2
#define FO_ERR_NEGATIVE_JACOBIAN 3
#define FO_ERR_NONFINITE 4

#define FO_PMAX 7
#define FO_PI 3.14159265358979323846

int fo_nsh(int p) { return (p + 1) * (p + 1) * (p + 2) / 2; }
int fo_nq(int p) { return (p + 1) * (p + 1) * (p + 1); }
static int fo_ntri(int p) { return (p + 1) * (p + 2) / 2; }

/* ------------------------------------------------------------------ */
/* 1D polynomials                                                      */
/* ------------------------------------------------------------------ */

/* Legendre P_n(x) by the three-term recurrence; P'_n by the identity
 * P'_{k+1} = P'_{k-1} + (2k+1) P_k. */
static void legendre(int n, double x, double *P, double *dP) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (n == 0) {
    *P = 1.0;
    *dP = 0.0;
    return;
  }
  for (int k = 1; k < n; ++k) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    double d2 = d0 + (2.0 * k + 1.0) * p1;
    p0 = p1;
    p1 = p2;
    d0 = d1;
    d1 = d2;
  }
  *P = p1;
  *dP = d1;
}

/* Jacobi P_n^{(a,b)}(x) by the standard three-term recurrence. */
static double jacobi(int n, double a, double b, double x) {
  if (n < 0) return 0.0;
  double p0 = 1.0;
  if (n == 0) return p0;
  double p1 = 0.5 * ((a - b) + (a + b + 2.0) * x);
  for (int k = 1; k < n; ++k) {
    double s = 2.0 * k + a + b;
    double a1 = 2.0 * (k + 1.0) * (k + a + b + 1.0) * s;
    double a2 = (s + 1.0) * (a * a - b * b);
    double a3 = s * (s + 1.0) * (s + 2.0);
    double a4 = 2.0 * (k + a) * (k + b) * (s + 2.0);
    double p2 = ((a2 + a3 * x) * p1 - a4 * p0) / a1;
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

/* d/dx P_n^{(a,b)}(x) = (n+a+b+1)/2 P_{n-1}^{(a+1,b+1)}(x). */
static double jacobi_deriv(int n, double a, double b, double x) {
  if (n == 0) return 0.0;
  return 0.5 * (n + a + b + 1.0) * jacobi(n - 1, a + 1.0, b + 1.0, x);
}

/* n-point Gauss-Legendre rule on [-1, 1]: Newton iteration on P_n from the
 * Chebyshev-like initial guesses, weights 2 / ((1 - x^2) P_n'(x)^2).
 * Nodes ascending. */
int fo_gauss_legendre(int n, double *x, double *w) {
  if (n < 1 || !x || !w) return FO_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    double t = cos(FO_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(n, t, &P, &dP);
      double dt = P / dP;
      t -= dt;
      if (fabs(dt) < 1e-16) break;
    }
    double P, dP;
    legendre(n, t, &P, &dP);
    x[n - 1 - i] = t;
    w[n - 1 - i] = 2.0 / ((1.0 - t * t) * dP * dP);
  }
  return FO_OK;
}

/* Duffy-collapsed Gauss-Legendre rule on the reference prism:
 * pts[q] = (xi1, xi2, zeta, w), q = (iz*(p+1) + iv)*(p+1) + iu. */
int fo_quadrature(int p, double *pts) {
  if (p < 1 || p > FO_PMAX) return FO_ERR_INVALID_DEGREE;
  if (!pts) return FO_ERR_INVALID_ARG;
  int n = p + 1;
  double x[FO_PMAX + 1], w[FO_PMAX + 1];
  fo_gauss_legendre(n, x, w);
  for (int iz = 0; iz < n; ++iz)
    for (int iv = 0; iv < n; ++iv)
      for (int iu = 0; iu < n; ++iu) {
        int q = (iz * n + iv) * n + iu;
        double u = x[iu], v = x[iv];
        pts[4 * q + 0] = 0.25 * (1.0 + u) * (1.0 - v);
        pts[4 * q + 1] = 0.5 * (1.0 + v);
        pts[4 * q + 2] = x[iz];
        pts[4 * q + 3] = w[iu] * w[iv] * (1.0 - v) / 8.0 * w[iz];
      }
  return FO_OK;
}

/* ------------------------------------------------------------------ */
/* Shape functions on the reference prism                             */
/* ------------------------------------------------------------------ */

/* Orthonormal Dubiner polynomial psi_mn on the unit right triangle and its
 * gradient (d/dxi1, d/dxi2).  psi_mn = c_mn P_m(eta1) (1-xi2)^m
 * P_n^{(2m+1,0)}(eta2), eta2 = 2 xi2 - 1, eta1 = 2 xi1/(1-xi2) - 1,
 * c_mn = sqrt(2 (2m+1) (m+n+1)) so that the integral of psi^2 over the
 * triangle is 1. */
static void dubiner(int m, int n, double xi1, double xi2, double *val,
                    double *d1, double *d2) {
  double c = sqrt(2.0 * (2.0 * m + 1.0) * (m + n + 1.0));
  double om = 1.0 - xi2;
  double eta2 = 2.0 * xi2 - 1.0;
  double eta1 = (om > 1e-300) ? 2.0 * xi1 / om - 1.0 : -1.0;
  double A, dA;
  legendre(m, eta1, &A, &dA);
  double Q = jacobi(n, 2.0 * m + 1.0, 0.0, eta2);
  double dQ = jacobi_deriv(n, 2.0 * m + 1.0, 0.0, eta2);
  double om_m = pow(om, m);
  double om_m1 = (m >= 1) ? pow(om, m - 1) : 0.0;
  *val = c * A * om_m * Q;
  *d1 = c * 2.0 * dA * om_m1 * Q;
  *d2 = c * (dA * (1.0 + eta1) * om_m1 * Q +
             A * (-(double)m * om_m1 * Q + 2.0 * om_m * dQ));
}

/* All N_sh prism shape functions at one reference point: phi[i] and
 * dphi[3*i + l] = d phi_i / d(xi1, xi2, zeta)_l. */
int fo_basis(int p, double xi1, double xi2, double zeta, double *phi,
             double *dphi) {
  if (p < 1 || p > FO_PMAX) return FO_ERR_INVALID_DEGREE;
  int T = fo_ntri(p);
  double tv[64], t1[64], t2[64];
  int t = 0;
  for (int d = 0; d <= p; ++d)
    for (int n = 0; n <= d; ++n) {
      int m = d - n;
      dubiner(m, n, xi1, xi2, &tv[t], &t1[t], &t2[t]);
      ++t;
    }
  for (int k = 0; k <= p; ++k) {
    double P, dP;
    legendre(k, zeta, &P, &dP);
    double s = sqrt((2.0 * k + 1.0) / 2.0);
    double L = s * P, dL = s * dP;
    for (int tt = 0; tt < T; ++tt) {
      int i = k * T + tt;
      phi[i] = tv[tt] * L;
      dphi[3 * i + 0] = t1[tt] * L;
      dphi[3 * i + 1] = t2[tt] * L;
      dphi[3 * i + 2] = tv[tt] * dL;
    }
  }
  return FO_OK;
}

/* Tabulate the basis at the quadrature points of degree p. */
int fo_tabulate(int p, double *pts, double *phi, double *dphi) {
  int rc = fo_quadrature(p, pts);
  if (rc) return rc;
  int nq = fo_nq(p), nsh = fo_nsh(p);
  for (int q = 0; q < nq; ++q)
    fo_basis(p, pts[4 * q], pts[4 * q + 1], pts[4 * q + 2], phi + (size_t)q * nsh,
             dphi + (size_t)q * nsh * 3);
  return FO_OK;
}

/* ------------------------------------------------------------------ */
/* Geometry: bilinear prism map x(xi) = sum_a X_a N_a(xi)              */
/* ------------------------------------------------------------------ */

/* Reference gradients of the six vertex functions
 * N_a = lambda_a (1-zeta)/2, N_{a+3} = lambda_a (1+zeta)/2,
 * lambda = (1 - xi1 - xi2, xi1, xi2). */
static void vertex_grads(double xi1, double xi2, double zeta, double g[6][3]) {
  double lam[3] = {1.0 - xi1 - xi2, xi1, xi2};
  double dl[3][2] = {{-1.0, -1.0}, {1.0, 0.0}, {0.0, 1.0}};
  for (int a = 0; a < 3; ++a) {
    g[a][0] = dl[a][0] * 0.5 * (1.0 - zeta);
    g[a][1] = dl[a][1] * 0.5 * (1.0 - zeta);
    g[a][2] = -0.5 * lam[a];
    g[a + 3][0] = dl[a][0] * 0.5 * (1.0 + zeta);
    g[a + 3][1] = dl[a][1] * 0.5 * (1.0 + zeta);
    g[a + 3][2] = 0.5 * lam[a];
  }
}

/* J[k][l] = d x_k / d xi_l; det J; R = J^{-1} by the adjugate. */
static void jacobian(const double *X, const double g[6][3], double J[3][3],
                     double *det, double R[3][3]) {
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) {
      double s = 0.0;
      for (int a = 0; a < 6; ++a) s += X[3 * a + k] * g[a][l];
      J[k][l] = s;
    }
  double d = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
             J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
             J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  *det = d;
  R[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / d;
  R[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / d;
  R[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / d;
  R[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / d;
  R[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / d;
  R[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / d;
  R[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / d;
  R[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / d;
  R[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / d;
}

/* ------------------------------------------------------------------ */
/* Batch description                                                   */
/* ------------------------------------------------------------------ */

typedef struct {
  int64_t n_elem;
  const double *geom;   /* [n][6][3] */
  const int32_t *degree; /* [n] or NULL */
  int uniform_p;
  int per_qp;           /* 0: coefficients per element, 1: per point */
  const double *K, *b, *c, *f;
  const int64_t *A_off, *b_off, *q_off; /* [n+1] or NULL */
  /* forward outputs */
  double *A, *bv;
  int32_t *status;
  /* backward inputs / outputs */
  const double *gA, *gb;
  double *g_geom, *gK, *gbc, *gc, *gf;
} fo_batch;

typedef struct {
  int nq, nsh;
  double *pts, *phi, *dphi;
} fo_table;

static fo_table g_tab[FO_PMAX + 1];
static pthread_once_t g_once = PTHREAD_ONCE_INIT;

static void build_tables(void) {
  for (int p = 1; p <= FO_PMAX; ++p) {
    fo_table *t = &g_tab[p];
    t->nq = fo_nq(p);
    t->nsh = fo_nsh(p);
    t->pts = (double *)malloc(sizeof(double) * 4 * t->nq);
    t->phi = (double *)malloc(sizeof(double) * t->nq * t->nsh);
    t->dphi = (double *)malloc(sizeof(double) * t->nq * t->nsh * 3);
    fo_tabulate(p, t->pts, t->phi, t->dphi);
  }
}

static int elem_degree(const fo_batch *B, int64_t e) {
  return B->degree ? B->degree[e] : B->uniform_p;
}
static int64_t A_offset(const fo_batch *B, int64_t e, int nsh) {
  return B->A_off ? B->A_off[e] : e * (int64_t)nsh * nsh;
}
static int64_t b_offset(const fo_batch *B, int64_t e, int nsh) {
  return B->b_off ? B->b_off[e] : e * (int64_t)nsh;
}
/* index of the coefficient record of element e at point q */
static int64_t coef_index(const fo_batch *B, int64_t e, int q, int nq) {
  if (!B->per_qp) return e;
  return (B->q_off ? B->q_off[e] : e * (int64_t)nq) + q;
}

static int finite_inputs(const fo_batch *B, int64_t e, int nq) {
  for (int i = 0; i < 18; ++i)
    if (!isfinite(B->geom[18 * e + i])) return 0;
  int npts = B->per_qp ? nq : 1;
  for (int q = 0; q < npts; ++q) {
    int64_t r = coef_index(B, e, q, nq);
    for (int i = 0; i < 9; ++i)
      if (!isfinite(B->K[9 * r + i])) return 0;
    for (int i = 0; i < 3; ++i)
      if (!isfinite(B->b[3 * r + i])) return 0;
    if (!isfinite(B->c[r]) || !isfinite(B->f[r])) return 0;
  }
  return 1;
}

/* ------------------------------------------------------------------ */
/* Forward: Algorithm 1 for one element                                */
/* ------------------------------------------------------------------ */

static void integrate_element(const fo_batch *B, int64_t e, double *gx) {
  int p = elem_degree(B, e);
  const fo_table *T = &g_tab[p];
  int nq = T->nq, nsh = T->nsh;
  double *A = B->A + A_offset(B, e, nsh);
  double *bv = B->bv + b_offset(B, e, nsh);
  const double *X = B->geom + 18 * e;
  /* step 4: initialise the element matrix */
  memset(A, 0, sizeof(double) * nsh * nsh);
  memset(bv, 0, sizeof(double) * nsh);
  int32_t st = FO_OK;
  if (!finite_inputs(B, e, nq)) st = FO_ERR_NONFINITE;
  for (int q = 0; q < nq && st == FO_OK; ++q) {
    /* step 6: shape functions and reference derivatives at xi_q */
    const double *phi = T->phi + (size_t)q * nsh;
    const double *dphi = T->dphi + (size_t)q * nsh * 3;
    double xi1 = T->pts[4 * q], xi2 = T->pts[4 * q + 1];
    double zeta = T->pts[4 * q + 2], w = T->pts[4 * q + 3];
    /* step 7: Jacobian, determinant, inverse */
    double g[6][3], J[3][3], R[3][3], det;
    vertex_grads(xi1, xi2, zeta, g);
    jacobian(X, g, J, &det, R);
    if (!isfinite(det)) {
      st = FO_ERR_NONFINITE;
      break;
    }
    if (det <= 0.0) {
      st = FO_ERR_NEGATIVE_JACOBIAN;
      break;
    }
    /* step 8: physical derivatives, grad phi = J^{-T} grad_ref phi */
    for (int j = 0; j < nsh; ++j)
      for (int k = 0; k < 3; ++k) {
        double s = 0.0;
        for (int l = 0; l < 3; ++l) s += R[l][k] * dphi[3 * j + l];
        gx[3 * j + k] = s;
      }
    int64_t r = coef_index(B, e, q, nq);
    const double *K = B->K + 9 * r, *bb = B->b + 3 * r;
    double c = B->c[r], f = B->f[r];
    double s = w * det;
    /* steps 9-13: the double loop over shape functions */
    for (int i = 0; i < nsh; ++i) {
      for (int j = 0; j < nsh; ++j) {
        double diff = 0.0;
        for (int k = 0; k < 3; ++k)
          for (int l = 0; l < 3; ++l) diff += gx[3 * i + k] * K[3 * k + l] * gx[3 * j + l];
        double conv = 0.0;
        for (int k = 0; k < 3; ++k) conv += bb[k] * gx[3 * j + k];
        A[(size_t)i * nsh + j] += s * (diff + phi[i] * conv + c * phi[i] * phi[j]);
      }
      bv[i] += s * f * phi[i];
    }
  }
  if (st != FO_OK) {
    memset(A, 0, sizeof(double) * nsh * nsh);
    memset(bv, 0, sizeof(double) * nsh);
  }
  if (B->status) B->status[e] = st;
}

/* ------------------------------------------------------------------ */
/* Backward: hand-derived reverse pass of the forward above            */
/* ------------------------------------------------------------------ */
/*
 * L = sum_ij gA_ij A_ij + sum_i gb_i b_i.  Per point, with s = w det J,
 * P_i = grad phi_i (physical), R = J^{-1}:
 *   dL/dc   = s sum_ij gA_ij phi_i phi_j
 *   dL/db   = s sum_ij gA_ij phi_i P_j
 *   dL/dK   = s sum_ij gA_ij P_i P_j^T
 *   dL/df   = s sum_i gb_i phi_i
 *   dL/ds   = sum_ij gA_ij (P_i.K P_j + phi_i b.P_j + c phi_i phi_j)
 *             + f sum_i gb_i phi_i
 *   dL/dP_m = s ( sum_j gA_mj K P_j + sum_i gA_im K^T P_i
 *                 + (sum_i gA_im phi_i) b )
 *   dL/dR   = sum_m grad_ref phi_m (dL/dP_m)^T          (P_m = R^T g_m)
 *   dL/dJ   = (dL/ds) s R^T - R^T (dL/dR) R^T   (d det = det tr(R dJ),
 *                                                dR = -R dJ R)
 *   dL/dX_a = sum_l (dL/dJ)[:, l] dN_a/dxi_l     (J = sum_a X_a grad N_a^T)
 * Coefficients per element sum the per-point gradients.  Per-point
 * coefficient values are held fixed when differentiating by X.
 */
static void backward_element(const fo_batch *B, int64_t e, double *gx,
                             double *gP) {
  int p = elem_degree(B, e);
  const fo_table *T = &g_tab[p];
  int nq = T->nq, nsh = T->nsh;
  const double *gA = B->gA + A_offset(B, e, nsh);
  const double *gb = B->gb + b_offset(B, e, nsh);
  const double *X = B->geom + 18 * e;
  double *gX = B->g_geom + 18 * e;
  memset(gX, 0, sizeof(double) * 18);
  int npts = B->per_qp ? nq : 1;
  for (int q = 0; q < npts; ++q) {
    int64_t r = coef_index(B, e, q, nq);
    memset(B->gK + 9 * r, 0, sizeof(double) * 9);
    memset(B->gbc + 3 * r, 0, sizeof(double) * 3);
    B->gc[r] = 0.0;
    B->gf[r] = 0.0;
  }
  if (!finite_inputs(B, e, nq)) return;
  for (int q = 0; q < nq; ++q) {
    const double *phi = T->phi + (size_t)q * nsh;
    const double *dphi = T->dphi + (size_t)q * nsh * 3;
    double xi1 = T->pts[4 * q], xi2 = T->pts[4 * q + 1];
    double zeta = T->pts[4 * q + 2], w = T->pts[4 * q + 3];
    double g[6][3], J[3][3], R[3][3], det;
    vertex_grads(xi1, xi2, zeta, g);
    jacobian(X, g, J, &det, R);
    if (!(det > 0.0) || !isfinite(det)) {
      memset(gX, 0, sizeof(double) * 18);
      return;
    }
    for (int j = 0; j < nsh; ++j)
      for (int k = 0; k < 3; ++k) {
        double s = 0.0;
        for (int l = 0; l < 3; ++l) s += R[l][k] * dphi[3 * j + l];
        gx[3 * j + k] = s;
      }
    int64_t r = coef_index(B, e, q, nq);
    const double *K = B->K + 9 * r, *bb = B->b + 3 * r;
    double c = B->c[r], f = B->f[r];
    double s = w * det;
    double gc = 0.0, gbq[3] = {0, 0, 0}, gK[3][3] = {{0}}, gf = 0.0, gs = 0.0;
    for (int m = 0; m < nsh; ++m) gP[3 * m] = gP[3 * m + 1] = gP[3 * m + 2] = 0.0;
    for (int i = 0; i < nsh; ++i) {
      for (int j = 0; j < nsh; ++j) {
        double a = gA[(size_t)i * nsh + j];
        const double *Pi = gx + 3 * i, *Pj = gx + 3 * j;
        double KPj[3], KtPi[3];
        for (int k = 0; k < 3; ++k) {
          KPj[k] = K[3 * k] * Pj[0] + K[3 * k + 1] * Pj[1] + K[3 * k + 2] * Pj[2];
          KtPi[k] = K[k] * Pi[0] + K[3 + k] * Pi[1] + K[6 + k] * Pi[2];
        }
        double diff = Pi[0] * KPj[0] + Pi[1] * KPj[1] + Pi[2] * KPj[2];
        double conv = bb[0] * Pj[0] + bb[1] * Pj[1] + bb[2] * Pj[2];
        gs += a * (diff + phi[i] * conv + c * phi[i] * phi[j]);
        gc += a * phi[i] * phi[j];
        for (int k = 0; k < 3; ++k) {
          gbq[k] += a * phi[i] * Pj[k];
          for (int l = 0; l < 3; ++l) gK[k][l] += a * Pi[k] * Pj[l];
          gP[3 * i + k] += s * a * KPj[k];
          gP[3 * j + k] += s * a * KtPi[k];
          gP[3 * j + k] += s * a * phi[i] * bb[k];
        }
      }
      gs += gb[i] * f * phi[i];
      gf += gb[i] * phi[i];
    }
    B->gc[r] += s * gc;
    B->gf[r] += s * gf;
    for (int k = 0; k < 3; ++k) {
      B->gbc[3 * r + k] += s * gbq[k];
      for (int l = 0; l < 3; ++l) B->gK[9 * r + 3 * k + l] += s * gK[k][l];
    }
    /* dL/dR[l][k] = sum_m dphi_m,l gP_m,k */
    double gR[3][3] = {{0}};
    for (int m = 0; m < nsh; ++m)
      for (int l = 0; l < 3; ++l)
        for (int k = 0; k < 3; ++k) gR[l][k] += dphi[3 * m + l] * gP[3 * m + k];
    /* dL/dJ = gs s R^T - R^T gR R^T */
    double gJ[3][3];
    for (int k = 0; k < 3; ++k)
      for (int l = 0; l < 3; ++l) {
        double t = 0.0;
        for (int a = 0; a < 3; ++a)
          for (int bq = 0; bq < 3; ++bq) t += R[a][k] * gR[a][bq] * R[l][bq];
        gJ[k][l] = gs * s * R[l][k] - t;
      }
    for (int a = 0; a < 6; ++a)
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) gX[3 * a + k] += gJ[k][l] * g[a][l];
  }
}

/* ------------------------------------------------------------------ */
/* Threaded drivers                                                    */
/* ------------------------------------------------------------------ */

typedef struct {
  const fo_batch *B;
  int64_t e0, e1;
  int backward;
} fo_job;

static void *run_job(void *arg) {
  fo_job *j = (fo_job *)arg;
  double *gx = (double *)malloc(sizeof(double) * 3 * 288);
  double *gP = (double *)malloc(sizeof(double) * 3 * 288);
  for (int64_t e = j->e0; e < j->e1; ++e) {
    if (j->backward)
      backward_element(j->B, e, gx, gP);
    else
      integrate_element(j->B, e, gx);
  }
  free(gx);
  free(gP);
  return NULL;
}

static int run_batch(const fo_batch *B, int nthreads, int backward) {
  pthread_once(&g_once, build_tables);
  if (B->n_elem < 0 || !B->geom || !B->K || !B->b || !B->c || !B->f)
    return FO_ERR_INVALID_ARG;
  for (int64_t e = 0; e < B->n_elem; ++e) {
    int p = elem_degree(B, e);
    if (p < 1 || p > FO_PMAX) return FO_ERR_INVALID_DEGREE;
  }
  if (nthreads <= 0) nthreads = (int)sysconf(_SC_NPROCESSORS_ONLN);
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if ((int64_t)nthreads > B->n_elem) nthreads = (int)(B->n_elem > 0 ? B->n_elem : 1);
  pthread_t th[256];
  fo_job jobs[256];
  int64_t chunk = (B->n_elem + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].B = B;
    jobs[t].e0 = t * chunk < B->n_elem ? t * chunk : B->n_elem;
    jobs[t].e1 = (t + 1) * chunk < B->n_elem ? (t + 1) * chunk : B->n_elem;
    jobs[t].backward = backward;
    if (t == 0) continue;
    pthread_create(&th[t], NULL, run_job, &jobs[t]);
  }
  run_job(&jobs[0]);
  for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
  return FO_OK;
}

/* Forward: A_e and b_e for a batch (offset arrays may be NULL for a uniform
 * degree, contiguous layout). */
int fo_integrate(int64_t n_elem, const double *geom, const int32_t *degree,
                 int uniform_p, int per_qp, const double *K, const double *b,
                 const double *c, const double *f, const int64_t *A_off,
                 const int64_t *b_off, const int64_t *q_off, double *A,
                 double *bv, int32_t *status, int nthreads) {
  fo_batch B;
  memset(&B, 0, sizeof(B));
  B.n_elem = n_elem;
  B.geom = geom;
  B.degree = degree;
  B.uniform_p = uniform_p;
  B.per_qp = per_qp;
  B.K = K;
  B.b = b;
  B.c = c;
  B.f = f;
  B.A_off = A_off;
  B.b_off = b_off;
  B.q_off = q_off;
  B.A = A;
  B.bv = bv;
  B.status = status;
  if (!A || !bv) return FO_ERR_INVALID_ARG;
  return run_batch(&B, nthreads, 0);
}

/* Backward: gradients of L = <gA, A> + <gb, b> with respect to the vertex
 * coordinates and the coefficients (same layout as the inputs). */
int fo_integrate_backward(int64_t n_elem, const double *geom,
                          const int32_t *degree, int uniform_p, int per_qp,
                          const double *K, const double *b, const double *c,
                          const double *f, const int64_t *A_off,
                          const int64_t *b_off, const int64_t *q_off,
                          const double *gA, const double *gb, double *g_geom,
                          double *gK, double *gbc, double *gc, double *gf,
                          int nthreads) {
  fo_batch B;
  memset(&B, 0, sizeof(B));
  B.n_elem = n_elem;
  B.geom = geom;
  B.degree = degree;
  B.uniform_p = uniform_p;
  B.per_qp = per_qp;
  B.K = K;
  B.b = b;
  B.c = c;
  B.f = f;
  B.A_off = A_off;
  B.b_off = b_off;
  B.q_off = q_off;
  B.gA = gA;
  B.gb = gb;
  B.g_geom = g_geom;
  B.gK = gK;
  B.gbc = gbc;
  B.gc = gc;
  B.gf = gf;
  if (!gA || !gb || !g_geom || !gK || !gbc || !gc || !gf) return FO_ERR_INVALID_ARG;
  return run_batch(&B, nthreads, 1);
}
