// fei_reference.cu -- per-degree reference data, tabulated on the GPU in FP64.
//
// Sec. 2.2: quadrature data and the values of the shape functions and their
// reference derivatives are identical for all elements of one type and
// degree, so they are computed once and kept resident (the paper's "SR"
// variant; Table 2 gives their sizes).  Everything here is computed by
// kernels; the host only allocates and launches.
//
// Basis (Table 1 and its text: complete triangle basis times 1D functions in
// the vertical direction): phi_{t,k}(xi, zeta) = psi_t(xi1, xi2) L_k(zeta),
// psi the orthonormal Dubiner polynomials of the unit right triangle, L_k
// the Legendre polynomials normalised on [-1, 1].  psi_{m,n} is evaluated as
//   psi_{m,n} = c_{mn} S_m(a, b) P_n^{(2m+1,0)}(2 xi2 - 1),
//   a = 2 xi1 + xi2 - 1, b = 1 - xi2, S_m(a, b) = b^m P_m(a / b),
// with S_m from the homogeneous ("scaled") Legendre recurrence, so no
// division by 1 - xi2 occurs.  c_{mn} = sqrt(2 (2m+1) (m+n+1)).
#include <math.h>

#include <cstdlib>

#include "fei_internal.cuh"

namespace fei {
namespace {

// Newton's method for the n Gauss-Legendre nodes on [-1, 1] (ascending),
// starting from Tricomi's asymptotic approximation, with
// P_n'(x) = n (x P_n - P_{n-1}) / (x^2 - 1); w = 2 / ((1 - x^2) P_n'^2).
__global__ void gauss_legendre_kernel(int n, double *znode) {
  int i = threadIdx.x;
  if (i >= n) return;
  int r = n - i;  // 1-based index of the root in descending order
  double x = (1.0 - 1.0 / (8.0 * n * n) + 1.0 / (8.0 * n * n * n)) *
             cos(M_PI * (4.0 * r - 1.0) / (4.0 * n + 2.0));
  double dPn = 1.0;
  for (int it = 0; it < 60; ++it) {
    double pm = 1.0, pc = x;
    for (int k = 1; k < n; ++k) {
      double pn = ((2.0 * k + 1.0) * x * pc - k * pm) / (k + 1.0);
      pm = pc;
      pc = pn;
    }
    dPn = n * (x * pc - pm) / (x * x - 1.0);
    double dx = pc / dPn;
    x -= dx;
    if (fabs(dx) <= 4e-16 * fabs(x) + 1e-300) {
      // one more evaluation at the converged x for the weight
      pm = 1.0;
      pc = x;
      for (int k = 1; k < n; ++k) {
        double pn = ((2.0 * k + 1.0) * x * pc - k * pm) / (k + 1.0);
        pm = pc;
        pc = pn;
      }
      dPn = n * (x * pc - pm) / (x * x - 1.0);
      break;
    }
  }
  znode[2 * i + 0] = x;
  znode[2 * i + 1] = 2.0 / ((1.0 - x * x) * dPn * dPn);
}

// Collapsed triangle nodes from the 1D nodes: xi1 = (1+u)(1-v)/4,
// xi2 = (1+v)/2, w = w_u w_v (1-v)/8; t = iv*(p+1) + iu.
__global__ void triangle_nodes_kernel(int n, const double *znode, double *tnode) {
  int t = threadIdx.x;
  if (t >= n * n) return;
  int iv = t / n, iu = t % n;
  double u = znode[2 * iu], wu = znode[2 * iu + 1];
  double v = znode[2 * iv], wv = znode[2 * iv + 1];
  tnode[4 * t + 0] = 0.25 * (1.0 + u) * (1.0 - v);
  tnode[4 * t + 1] = 0.5 * (1.0 + v);
  tnode[4 * t + 2] = wu * wv * (1.0 - v) * 0.125;
  tnode[4 * t + 3] = 0.0;
}

// Dubiner psi_{m,n} and its gradient at (xi1, xi2).
__device__ void dubiner_eval(int m, int n, double xi1, double xi2, double &v, double &d1,
                             double &d2) {
  const double a = 2.0 * xi1 + xi2 - 1.0, b = 1.0 - xi2;
  // scaled Legendre S_m(a, b) and its partial derivatives in a and b
  double S0 = 1.0, Sa0 = 0.0, Sb0 = 0.0;
  double S = 1.0, Sa = 0.0, Sb = 0.0;
  if (m >= 1) {
    S = a;
    Sa = 1.0;
    Sb = 0.0;
    for (int k = 1; k < m; ++k) {
      const double kk = k, c1 = 2.0 * kk + 1.0, inv = 1.0 / (kk + 1.0);
      double Sn = (c1 * a * S - kk * b * b * S0) * inv;
      double San = (c1 * (S + a * Sa) - kk * b * b * Sa0) * inv;
      double Sbn = (c1 * a * Sb - kk * (2.0 * b * S0 + b * b * Sb0)) * inv;
      S0 = S;
      Sa0 = Sa;
      Sb0 = Sb;
      S = Sn;
      Sa = San;
      Sb = Sbn;
    }
  }
  // Jacobi P_n^{(alpha,0)}(y), y = 2 xi2 - 1, and d/dy from the
  // differentiated three-term recurrence
  const double al = 2.0 * m + 1.0, y = 2.0 * xi2 - 1.0;
  double Q0 = 1.0, dQ0 = 0.0, Q = 1.0, dQ = 0.0;
  if (n >= 1) {
    Q = 0.5 * (al + (al + 2.0) * y);
    dQ = 0.5 * (al + 2.0);
    for (int k = 1; k < n; ++k) {
      const double s = 2.0 * k + al;
      const double a1 = 2.0 * (k + 1.0) * (k + al + 1.0) * s;
      const double a2 = (s + 1.0) * al * al;
      const double a3 = s * (s + 1.0) * (s + 2.0);
      const double a4 = 2.0 * (k + al) * k * (s + 2.0);
      double Qn = ((a2 + a3 * y) * Q - a4 * Q0) / a1;
      double dQn = ((a2 + a3 * y) * dQ + a3 * Q - a4 * dQ0) / a1;
      Q0 = Q;
      dQ0 = dQ;
      Q = Qn;
      dQ = dQn;
    }
  }
  const double c = sqrt(2.0 * (2.0 * m + 1.0) * (m + n + 1.0));
  v = c * S * Q;
  d1 = c * 2.0 * Sa * Q;
  d2 = c * ((Sa - Sb) * Q + 2.0 * S * dQ);
}

// Normalised Legendre L_k(z) = sqrt(k + 1/2) P_k(z) and its derivative,
// with P'_{k+1} = (k+1) P_k + z P'_k.
__device__ void legendre_norm_eval(int k, double z, double &L, double &dL) {
  double pm = 1.0, pc = 1.0, dc = 0.0;
  if (k >= 1) {
    pc = z;
    dc = 1.0;
    for (int j = 1; j < k; ++j) {
      double pn = ((2.0 * j + 1.0) * z * pc - j * pm) / (j + 1.0);
      double dn = (j + 1.0) * pc + z * dc;
      pm = pc;
      pc = pn;
      dc = dn;
    }
  }
  const double s = sqrt(k + 0.5);
  L = s * pc;
  dL = s * dc;
}

// One thread per (point q, shape function i).
__global__ void tabulate_kernel(int p, const double *znode, const double *tnode, double *pts,
                                double *G64, float *G32, float *G32T) {
  const int nsh = nsh_of(p), nq = nq_of(p), T = ntri_of(p), n1 = p + 1;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nq * nsh) return;
  const int q = idx / nsh, i = idx % nsh;
  const int iz = q / (n1 * n1), t = q % (n1 * n1);
  const double xi1 = tnode[4 * t], xi2 = tnode[4 * t + 1], wt = tnode[4 * t + 2];
  const double z = znode[2 * iz], wz = znode[2 * iz + 1];
  if (i == 0) {
    pts[4 * q + 0] = xi1;
    pts[4 * q + 1] = xi2;
    pts[4 * q + 2] = z;
    pts[4 * q + 3] = wt * wz;
  }
  const int k = i / T, tt = i % T;
  int d = 0;
  while ((d + 1) * (d + 2) / 2 <= tt) ++d;
  const int n = tt - d * (d + 1) / 2, m = d - n;
  double v, d1, d2, L, dL;
  dubiner_eval(m, n, xi1, xi2, v, d1, d2);
  legendre_norm_eval(k, z, L, dL);
  const double g[4] = {v * L, d1 * L, d2 * L, v * dL};
  for (int a = 0; a < 4; ++a) {
    G64[(size_t)(q * 4 + a) * nsh + i] = g[a];
    G32[(size_t)(q * 4 + a) * nsh + i] = (float)g[a];
    G32T[((size_t)q * nsh + i) * 4 + a] = (float)g[a];
  }
}

}  // namespace
}  // namespace fei

using namespace fei;

extern "C" fei_status fei_reference_create(int p, fei_reference_t *out) {
  const Range range_("fei_reference_create");
  if (!out) return set_error(FEI_ERR_INVALID_ARG, "fei_reference_create: out is NULL");
  *out = nullptr;
  if (p < 1 || p > kPMax)
    return set_error(FEI_ERR_INVALID_DEGREE, "fei_reference_create: degree %d outside 1..%d", p, kPMax);
  fei_reference *r = (fei_reference *)calloc(1, sizeof(fei_reference));
  if (!r) return set_error(FEI_ERR_OOM, "fei_reference_create: host allocation failed");
  r->p = p;
  r->nsh = nsh_of(p);
  r->nq = nq_of(p);
  cudaError_t e = cudaGetDevice(&r->device);
  if (e != cudaSuccess) {
    free(r);
    return cuda_error(e, "cudaGetDevice");
  }
  const int n1 = p + 1;
  size_t bytes[6] = {sizeof(double) * 4 * r->nq, sizeof(double) * 4 * r->nq * r->nsh,
                     sizeof(float) * 4 * r->nq * r->nsh, sizeof(double) * 2 * n1,
                     sizeof(double) * 4 * n1 * n1, sizeof(float) * 4 * r->nq * r->nsh};
  void **ptrs[6] = {(void **)&r->pts, (void **)&r->G64, (void **)&r->G32, (void **)&r->znode,
                    (void **)&r->tnode, (void **)&r->G32T};
  for (int k = 0; k < 6; ++k) {
    e = cudaMalloc(ptrs[k], bytes[k]);
    if (e != cudaSuccess) {
      fei_reference_destroy(r);
      return e == cudaErrorMemoryAllocation ? set_error(FEI_ERR_OOM, "fei_reference_create: cudaMalloc")
                                            : cuda_error(e, "cudaMalloc");
    }
  }
  cudaStream_t s;
  e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    fei_reference_destroy(r);
    return cuda_error(e, "cudaStreamCreate");
  }
  gauss_legendre_kernel<<<1, 32, 0, s>>>(n1, r->znode);
  triangle_nodes_kernel<<<1, 64, 0, s>>>(n1, r->znode, r->tnode);
  const int total = r->nq * r->nsh;
  tabulate_kernel<<<(total + 255) / 256, 256, 0, s>>>(p, r->znode, r->tnode, r->pts, r->G64, r->G32, r->G32T);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  if (e != cudaSuccess) {
    fei_reference_destroy(r);
    return cuda_error(e, "reference tabulation kernels");
  }
  if (p >= 3) {
    fei_status st = build_tc_image(r);
    if (st == FEI_OK) st = build_sf_tables(r);
    if (st != FEI_OK) {
      fei_reference_destroy(r);
      return st;
    }
  }
  *out = r;
  return FEI_OK;
}

extern "C" fei_status fei_reference_destroy(fei_reference_t r) {
  if (!r) return FEI_OK;
  free_tc_image(r);
  free_sf_tables(r);
  cudaFree(r->pts);
  cudaFree(r->G64);
  cudaFree(r->G32);
  cudaFree(r->znode);
  cudaFree(r->tnode);
  cudaFree(r->G32T);
  free(r);
  return FEI_OK;
}

extern "C" fei_status fei_reference_info(fei_reference_t r, int *p, int *nsh, int *nq) {
  if (!r) return set_error(FEI_ERR_INVALID_ARG, "fei_reference_info: NULL handle");
  if (p) *p = r->p;
  if (nsh) *nsh = r->nsh;
  if (nq) *nq = r->nq;
  return FEI_OK;
}

extern "C" fei_status fei_reference_copy_table(fei_reference_t r, double *pts, double *G) {
  if (!r) return set_error(FEI_ERR_INVALID_ARG, "fei_reference_copy_table: NULL handle");
  if (pts) FEI_CUDA_TRY(cudaMemcpy(pts, r->pts, sizeof(double) * 4 * r->nq, cudaMemcpyDeviceToHost), "cudaMemcpy pts");
  if (G)
    FEI_CUDA_TRY(cudaMemcpy(G, r->G64, sizeof(double) * 4 * r->nq * r->nsh, cudaMemcpyDeviceToHost), "cudaMemcpy G");
  return FEI_OK;
}
