// fei_sf.cu -- sum-factorised element integration on the CUDA cores
// (FEI_SF_FP32, p >= 3).
//
// The paper points to sum factorisation as the way to cut the O(p^9) cost
// of the double loop for high orders (Sec. 1.2-1.3, the special integration
// it cites for p >= 4-5) and contrasts shape functions recomputed per
// element (SC) with tables read (SR, Sec. 4).  On the prism with the
// Duffy-collapsed rule both the basis and the rule are tensor products in
// the collapsed coordinates (u, v, zeta): with
//   xi1 = (1+u)(1-v)/4, xi2 = (1+v)/2,
//   phi_{(m,n),k} = A_m(u) B_mn(v) L_k(zeta),
//   A_m = P_m (Legendre), B_mn = c_mn ((1-v)/2)^m P_n^{(2m+1,0)}(v),
//   L_k = sqrt((2k+1)/2) P_k, c_mn = sqrt(2 (2m+1)(m+n+1)),
// (the Dubiner product of the reference tables), and the reference
// gradient has separable terms:
//   d/dxi1   = A'(u) [4 B/(1-v)] L,
//   d/dxi2   = [(1+u) A'(u)] [2 B/(1-v)] L + A(u) [2 B'(v)] L,
//   d/dzeta  = A(u) B(v) L'.
// So a component a of G is a sum of one or two terms U_a(u) V_a(v) Z_a(z),
// and A_e[i][j] = sum_q sum_ab G_a(q,i) Dt_q[a][b] G_b(q,j) becomes, per
// pair of terms (alpha of a, beta of b), a sum over u, then v, then zeta:
//   X1[iv][iz][m][m']   = sum_iu U_alpha(iu,m) U_beta(iu,m') Dt_ab(iz,iv,iu)
//   Y[zz][iz][t][t']   += sum_iv V_alpha(iv,t) V_beta(iv,t') X1[iv][iz][m(t)][m(t')]
//   A[(k,t),(k',t')]    = sum_zz sum_iz Z_alpha(iz,k) Z_beta(iz,k') Y[zz][iz][t][t']
// where the last sum is grouped by the pair of zeta factors zz (L or L' on
// each side), so it runs 4 times instead of once per term pair (21).  At
// p = 7 this is about 5.7 M multiply-adds per element against 41 M for the
// dense contraction (8 N_sh^2 N_q / 2).
//
// One thread block per element (persistent over elements): the point
// operators Dt of every point as in the FEI_FP32 path (FP64 node columns
// and w det J, FP32 adjugate and operator), the 21 term pairs in turn
// (stage 1 over all threads, stage 2 with each thread accumulating its own
// (t, t') pairs in registers), then stage 3 with each thread forming the
// (k, k') block of its (t, t') pairs.  FP32 throughout the sums.  The load
// vector is factorised the same way.  The 1D factor tables are tabulated
// once per degree (FP64, stored FP32) and checked against the library's 3D
// reference table when the reference is created; a degree whose check
// fails has no sum-factorised path (FEI_ERR_UNSUPPORTED).
#include <math.h>
#include <string.h>

#include <type_traits>

#include "fei_geom.cuh"
#include "fei_internal.cuh"

namespace fei {

namespace {

// The term pairs (alpha, beta): U, V, Z kinds of alpha, then of beta, and
// the index of Dt_ab in the point operator (fei_geom.cuh), sorted by the
// pair of zeta kinds zz = 2 Z_alpha + Z_beta.  Kinds: U0 = A, U1 = A',
// U2 = (1+u) A'; V0 = B, V1 = 4B/(1-v), V2 = 2B/(1-v), V3 = 2B'; Z0 = L,
// Z1 = L'.  Components: 0 = {U0 V0 Z0}, 1 = {U1 V1 Z0}, 2 = {U2 V2 Z0,
// U0 V3 Z0}, 3 = {U0 V0 Z1}; Dt_a0 = 0 for a >= 1.
struct SfPair {
  int ua, va, za, ub, vb, zb, d;
};
constexpr int kPairs = 21;
__constant__ SfPair c_pairs[kPairs] = {
    {0, 0, 0, 0, 0, 0, 0},   // a=0 b=0
    {0, 0, 0, 1, 1, 0, 1},   // a=0 b=1
    {0, 0, 0, 2, 2, 0, 2},   // a=0 b=2
    {0, 0, 0, 0, 3, 0, 2},   // a=0 b=2
    {1, 1, 0, 1, 1, 0, 4},   // a=1 b=1
    {1, 1, 0, 2, 2, 0, 5},   // a=1 b=2
    {1, 1, 0, 0, 3, 0, 5},   // a=1 b=2
    {2, 2, 0, 1, 1, 0, 7},   // a=2 b=1
    {0, 3, 0, 1, 1, 0, 7},   // a=2 b=1
    {2, 2, 0, 2, 2, 0, 8},   // a=2 b=2
    {2, 2, 0, 0, 3, 0, 8},   // a=2 b=2
    {0, 3, 0, 2, 2, 0, 8},   // a=2 b=2
    {0, 3, 0, 0, 3, 0, 8},   // a=2 b=2
    {0, 0, 0, 0, 0, 1, 3},   // a=0 b=3
    {1, 1, 0, 0, 0, 1, 6},   // a=1 b=3
    {2, 2, 0, 0, 0, 1, 9},   // a=2 b=3
    {0, 3, 0, 0, 0, 1, 9},   // a=2 b=3
    {0, 0, 1, 1, 1, 0, 10},  // a=3 b=1
    {0, 0, 1, 2, 2, 0, 11},  // a=3 b=2
    {0, 0, 1, 0, 3, 0, 11},  // a=3 b=2
    {0, 0, 1, 0, 0, 1, 12},  // a=3 b=3
};

// ---------------------------------------------------------------------------
// 1D factor tables
// ---------------------------------------------------------------------------
// Layout (FP64 while tabulated, FP32 for the kernel), M = p+1, T = the
// triangle functions (total degree ascending, then n ascending):
//   U[3][M iu][M m], V[4][M iv][T t], Z[2][M k][M iz], mt[T] (m of t).
__host__ __device__ constexpr int sf_tab_size(int p) {
  return 3 * (p + 1) * (p + 1) + 4 * (p + 1) * ((p + 1) * (p + 2) / 2) + 2 * (p + 1) * (p + 1) +
         (p + 1) * (p + 2) / 2;
}

// Legendre P_0..P_n and derivatives at x.
__device__ void legendre_all(int n, double x, double *P, double *dP) {
  P[0] = 1.0;
  dP[0] = 0.0;
  if (n >= 1) {
    P[1] = x;
    dP[1] = 1.0;
  }
  for (int k = 1; k < n; ++k) {
    P[k + 1] = ((2 * k + 1) * x * P[k] - k * P[k - 1]) / (k + 1);
    dP[k + 1] = dP[k - 1] + (2 * k + 1) * P[k];
  }
}

// Jacobi P_n^{(al, 0)}(x) by the three-term recurrence.
__device__ double jacobi(int n, double al, double x) {
  if (n == 0) return 1.0;
  double pm = 1.0, pc = 0.5 * ((al + 2.0) * x + al);
  for (int k = 2; k <= n; ++k) {
    const double a1 = 2.0 * k * (k + al) * (2.0 * k + al - 2.0);
    const double a2 = (2.0 * k + al - 1.0) * (al * al);
    const double a3 = (2.0 * k + al - 2.0) * (2.0 * k + al - 1.0) * (2.0 * k + al);
    const double a4 = 2.0 * (k + al - 1.0) * (k - 1.0) * (2.0 * k + al);
    const double pn = ((a2 + a3 * x) * pc - a4 * pm) / a1;
    pm = pc;
    pc = pn;
  }
  return pc;
}
// d/dx P_n^{(al, 0)} = (n + al + 1) / 2 P_{n-1}^{(al + 1, 1)}; the (al+1, 1)
// polynomial by the general three-term recurrence.
__device__ double jacobi_deriv(int n, double al, double x) {
  if (n == 0) return 0.0;
  const double a = al + 1.0, b = 1.0;
  const int m = n - 1;
  double pm = 1.0, pc = 0.5 * ((a + b + 2.0) * x + (a - b));
  if (m == 0) pc = 1.0;
  for (int k = 2; k <= m; ++k) {
    const double s = 2.0 * k + a + b;
    const double a1 = 2.0 * k * (k + a + b) * (s - 2.0);
    const double a2 = (s - 1.0) * (a * a - b * b);
    const double a3 = (s - 2.0) * (s - 1.0) * s;
    const double a4 = 2.0 * (k + a - 1.0) * (k + b - 1.0) * s;
    const double pn = ((a2 + a3 * x) * pc - a4 * pm) / a1;
    pm = pc;
    pc = pn;
  }
  return 0.5 * (n + al + 1.0) * pc;
}

// One thread: every table entry (FP64) from the 1D Gauss-Legendre nodes.
__global__ void sf_tables_kernel(int p, const double *znode, double *tab) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int M = p + 1, T = (p + 1) * (p + 2) / 2;
  double *U = tab, *V = U + 3 * M * M, *Z = V + 4 * M * T, *mt = Z + 2 * M * M;
  double P[8], dP[8];
  for (int i = 0; i < M; ++i) {
    const double x = znode[2 * i];
    legendre_all(p, x, P, dP);
    for (int m = 0; m < M; ++m) {
      U[(0 * M + i) * M + m] = P[m];
      U[(1 * M + i) * M + m] = dP[m];
      U[(2 * M + i) * M + m] = (1.0 + x) * dP[m];
    }
    for (int k = 0; k < M; ++k) {
      const double nk = sqrt((2.0 * k + 1.0) / 2.0);
      Z[(0 * M + k) * M + i] = nk * P[k];
      Z[(1 * M + k) * M + i] = nk * dP[k];
    }
    int t = 0;
    for (int d = 0; d <= p; ++d)
      for (int n = 0; n <= d; ++n, ++t) {
        const int m = d - n;
        const double c = sqrt(2.0 * (2 * m + 1) * (m + n + 1));
        const double h = 0.5 * (1.0 - x);
        const double hm = pow(h, m), jn = jacobi(n, 2.0 * m + 1.0, x), djn = jacobi_deriv(n, 2.0 * m + 1.0, x);
        const double B = c * hm * jn;
        const double dB = c * (m > 0 ? -0.5 * m * pow(h, m - 1) * jn : 0.0) + c * hm * djn;
        V[(0 * M + i) * T + t] = B;
        V[(1 * M + i) * T + t] = 4.0 * B / (1.0 - x);
        V[(2 * M + i) * T + t] = 2.0 * B / (1.0 - x);
        V[(3 * M + i) * T + t] = 2.0 * dB;
        if (i == 0) mt[t] = m;
      }
  }
}

// max |G(from the factors) - G64| over the whole reference table, and max
// |G64|, as the bits of non-negative doubles (atomicMax orders them).
__global__ void sf_check_kernel(int p, const double *tab, const double *G64, unsigned long long *out) {
  const int M = p + 1, T = (p + 1) * (p + 2) / 2, nsh = T * M, nq = M * M * M;
  const double *U = tab, *V = U + 3 * M * M, *Z = V + 4 * M * T, *mt = Z + 2 * M * M;
  double dmax = 0.0, gmax = 0.0;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nq * nsh; idx += gridDim.x * blockDim.x) {
    const int q = idx / nsh, i = idx % nsh;
    const int iz = q / (M * M), iv = (q / M) % M, iu = q % M;
    const int k = i / T, t = i % T, m = (int)mt[t];
    const double A = U[iu * M + m], A1 = U[(M + iu) * M + m], A2 = U[(2 * M + iu) * M + m];
    const double B = V[iv * T + t], B1 = V[(M + iv) * T + t], B2 = V[(2 * M + iv) * T + t],
                 B3 = V[(3 * M + iv) * T + t];
    const double L = Z[k * M + iz], L1 = Z[(M + k) * M + iz];
    const double g[4] = {A * B * L, A1 * B1 * L, A2 * B2 * L + A * B3 * L, A * B * L1};
    for (int a = 0; a < 4; ++a) {
      const double ref = G64[(size_t)(4 * q + a) * nsh + i];
      dmax = fmax(dmax, fabs(g[a] - ref));
      gmax = fmax(gmax, fabs(ref));
    }
  }
  atomicMax(&out[0], (unsigned long long)__double_as_longlong(dmax));
  atomicMax(&out[1], (unsigned long long)__double_as_longlong(gmax));
}

__global__ void to_float_kernel(const double *x, int n, float *y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = (float)x[i];
}

// ---------------------------------------------------------------------------
// The kernel
// ---------------------------------------------------------------------------
template <int P>
struct SfCfg {
  static constexpr int M = P + 1, T = (P + 1) * (P + 2) / 2, NSH = nsh_of(P), NQ = nq_of(P), NT2 = M * M;
  static constexpr int MZ = (M + 3) / 4 * 4;  // iz extent of X1, padded for 16-byte loads
  static constexpr int NTH = P >= 5 ? 512 : 256;
  static constexpr int TT = T * T;
  static constexpr int NPR = (TT + NTH - 1) / NTH;  // (t, t') pairs per thread
  static constexpr int TAB = sf_tab_size(P);
  // dynamic shared memory (floats): tables, Dt [13][NQ], F [NQ],
  // X1 [M iv][M m][M m'][MZ iz], Y [4 zz][M iz][T*T]
  static constexpr int O_DT = (TAB + 3) / 4 * 4;
  static constexpr int O_F = O_DT + 13 * NQ;
  static constexpr int O_X1 = (O_F + NQ + 3) / 4 * 4;  // 16-byte aligned
  static constexpr int O_Y = O_X1 + M * M * M * MZ;
  static constexpr int FLOATS = O_Y + 4 * M * TT;
  static constexpr int DYN_SMEM = FLOATS * 4;
};

// Element data in FP64 and its FP32 copies (the FEI_FP32 path's point
// operator: FP64 columns and w det J, FP32 adjugate).
template <int P>
struct SfElem {
  using C = SfCfg<P>;
  double X[18], ev[21], cd[14];
  double zn3w[C::M][3], tc3w[C::NT2][3];
  float zc1f[C::M][3], zc2f[C::M][3], zn3f[C::M][3], zwf[C::M];
  float tc3f[C::NT2][3], twf[C::NT2];
  int status;
};

template <int P>
__global__ void __launch_bounds__(SfCfg<P>::NTH, 1) sf_forward_kernel(FwdArgs a, const float *gtab) {
  using C = SfCfg<P>;
  constexpr int M = C::M, MZ = C::MZ, T = C::T, NSH = C::NSH, NQ = C::NQ, NT2 = C::NT2, NTH = C::NTH, TT = C::TT;
  extern __shared__ __align__(16) float sm[];
  __shared__ SfElem<P> E;
  const float *U = sm, *V = sm + 3 * M * M, *Z = V + 4 * M * T, *mtf = Z + 2 * M * M;
  float *Dt = sm + C::O_DT, *Fq = sm + C::O_F, *X1 = sm + C::O_X1, *Y = sm + C::O_Y;
  const int tid = threadIdx.x;
  for (int i = tid; i < C::TAB; i += NTH) sm[i] = gtab[i];
  const int64_t items = a.count ? (int64_t)(*a.count) : a.n_work;

  for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
    const int64_t e = a.list ? (int64_t)a.list[item] : item;
    if (tid == 0) E.status = 0;
    __syncthreads();
    // geometry, per-element coefficients, status
    bool ok = true, sym = true;
    if (tid < 18) {
      E.X[tid] = a.geom[18 * e + tid];
      ok = finite64(E.X[tid]);
    }
    if (a.coef_mode == FEI_COEF_PER_ELEMENT && tid == 32) {
      ok = [&] {
        bool f = true;
        for (int k = 0; k < 9; ++k) f &= finite64(E.cd[k] = a.K[9 * e + k]);
        for (int k = 0; k < 3; ++k) f &= finite64(E.cd[9 + k] = a.b[3 * e + k]);
        f &= finite64(E.cd[12] = a.c[e]);
        f &= finite64(E.cd[13] = a.f[e]);
        return f;
      }();
      sym = !a.upper || coef_symmetric(E.cd, E.cd + 9);
    }
    if (!ok) atomicMax(&E.status, FEI_ERR_NONFINITE);
    if (!sym) atomicMax(&E.status, FEI_ERR_INVALID_ARG);
    __syncthreads();
    if (tid == 0) elem_vectors(E.X, E.ev);
    __syncthreads();
    // FP64 node columns: vertical nodes (c1, c2, n3) and triangle nodes (c3)
    if (tid < M) {
      const double z = a.znode[2 * tid], wz = a.znode[2 * tid + 1];
      double c1[3], c2[3], n3[3];
      znode_columns(E.ev, z, c1, c2, n3);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        E.zc1f[tid][k] = (float)c1[k];
        E.zc2f[tid][k] = (float)c2[k];
        E.zn3f[tid][k] = (float)n3[k];
        E.zn3w[tid][k] = wz * n3[k];
      }
      E.zwf[tid] = (float)wz;
    } else if (tid >= 32 && tid < 32 + NT2) {
      const int t = tid - 32;
      const double wt = a.tnode[4 * t + 2];
      double c3[3];
      tnode_column(E.ev, a.tnode[4 * t], a.tnode[4 * t + 1], c3);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        E.tc3f[t][k] = (float)c3[k];
        E.tc3w[t][k] = wt * c3[k];
      }
      E.twf[t] = (float)wt;
    }
    __syncthreads();
    // the point operators of every point (Dt by component, w det J f)
    for (int q = tid; q < NQ; q += NTH) {
      const int iz = q / NT2, t = q - iz * NT2;
      double cq[14];
      const double *cp = E.cd;
      int pst = 0;
      if (a.coef_mode == FEI_COEF_PER_POINT) {
        const int64_t r = (a.q_off ? a.q_off[e] : e * (int64_t)NQ) + q;
        bool f = true;
        for (int k = 0; k < 9; ++k) f &= finite64(cq[k] = a.K[9 * r + k]);
        for (int k = 0; k < 3; ++k) f &= finite64(cq[9 + k] = a.b[3 * r + k]);
        f &= finite64(cq[12] = a.c[r]);
        f &= finite64(cq[13] = a.f[r]);
        if (!f) pst = FEI_ERR_NONFINITE;
        else if (a.upper && !coef_symmetric(cq, cq + 9)) pst = FEI_ERR_INVALID_ARG;
        cp = cq;
      }
      float K[9], b[3];
#pragma unroll
      for (int k = 0; k < 9; ++k) K[k] = (float)cp[k];
#pragma unroll
      for (int k = 0; k < 3; ++k) b[k] = (float)cp[9 + k];
      const double s = dot3(E.zn3w[iz], E.tc3w[t]);  // w det J in FP64
      const float sf = (float)s, wf = E.zwf[iz] * E.twf[t];
      float a0[3], a1[3], D[16];
      cross3(E.zc2f[iz], E.tc3f[t], a0);
      cross3(E.tc3f[t], E.zc1f[iz], a1);
      dt_from_adj<float>(a0, a1, E.zn3f[iz], wf, sf, wf * wf / sf, K, b, (float)cp[12], (float)cp[13], D);
#pragma unroll
      for (int k = 0; k < 13; ++k) Dt[k * NQ + q] = D[k];
      Fq[q] = D[13];
      pst = merge_status(pst, point_status(s));
      if (pst) atomicMax(&E.status, pst);
    }
    __syncthreads();
    const int st = E.status;
    // load vector, factorised: F1[iz][iv][m] = sum_iu A(iu,m) F,
    // F2[iz][t] = sum_iv B(iv,t) F1[..][m(t)], b[k T + t] = sum_iz L(k,iz) F2
    {
      float *F1 = X1, *F2 = X1 + M * M * M;
      for (int o = tid; o < M * M * M; o += NTH) {
        const int iz = o / (M * M), iv = (o / M) % M, m = o % M;
        float acc = 0.f;
#pragma unroll
        for (int iu = 0; iu < M; ++iu) acc = fmaf(U[iu * M + m], Fq[(iz * M + iv) * M + iu], acc);
        F1[o] = acc;
      }
      __syncthreads();
      for (int o = tid; o < M * T; o += NTH) {
        const int iz = o / T, t = o % T, m = (int)mtf[t];
        float acc = 0.f;
#pragma unroll
        for (int iv = 0; iv < M; ++iv) acc = fmaf(V[iv * T + t], F1[(iz * M + iv) * M + m], acc);
        F2[o] = acc;
      }
      __syncthreads();
      float *bout = reinterpret_cast<float *>(a.bv) + out_b(a, item, e, NSH);
      for (int i = tid; i < NSH; i += NTH) {
        const int k = i / T, t = i % T;
        float acc = 0.f;
#pragma unroll
        for (int iz = 0; iz < M; ++iz) acc = fmaf(Z[k * M + iz], F2[iz * T + t], acc);
        bout[i] = st ? 0.f : acc;
      }
      __syncthreads();
    }
    // stages 1 and 2 over the term pairs; each thread accumulates the Y of
    // its own (t, t') pairs pr = tid + j NTH in registers and writes them
    // when the zeta pair zz changes
    float acc[C::NPR][M];
#pragma unroll
    for (int j = 0; j < C::NPR; ++j)
#pragma unroll
      for (int iz = 0; iz < M; ++iz) acc[j][iz] = 0.f;
    for (int ip = 0; ip < kPairs; ++ip) {
      const SfPair pr = c_pairs[ip];
      const float *Ua = U + pr.ua * M * M, *Ub = U + pr.ub * M * M;
      const float *Va = V + pr.va * M * T, *Vb = V + pr.vb * M * T;
      const float *Dd = Dt + pr.d * NQ;
      // stage 1: thread o = (iv, m, m') forms X1[iv][m][m'][0..M-1 (iz)]
      for (int o = tid; o < M * M * M; o += NTH) {
        const int iv = o / (M * M), m = (o / M) % M, m2 = o % M;
        float cu[M];
#pragma unroll
        for (int iu = 0; iu < M; ++iu) cu[iu] = Ua[iu * M + m] * Ub[iu * M + m2];
        float x[MZ];
#pragma unroll
        for (int iz = 0; iz < MZ; ++iz) {
          x[iz] = 0.f;
          if (iz < M) {
#pragma unroll
            for (int iu = 0; iu < M; ++iu) x[iz] = fmaf(cu[iu], Dd[(iz * M + iv) * M + iu], x[iz]);
          }
        }
        float4 *dst = reinterpret_cast<float4 *>(X1 + o * MZ);
#pragma unroll
        for (int c = 0; c < MZ / 4; ++c) dst[c] = make_float4(x[4 * c], x[4 * c + 1], x[4 * c + 2], x[4 * c + 3]);
      }
      __syncthreads();
      // stage 2: Y[iz][t][t'] += sum_iv Va(iv,t) Vb(iv,t') X1[iv][m(t)][m(t')][iz]
#pragma unroll
      for (int j = 0; j < C::NPR; ++j) {
        const int pq = tid + j * NTH;
        if (pq < TT) {
          const int t = pq / T, t2 = pq - t * T;
          const int mm = (int)mtf[t] * M + (int)mtf[t2];
#pragma unroll
          for (int iv = 0; iv < M; ++iv) {
            const float cv = Va[iv * T + t] * Vb[iv * T + t2];
            const float4 *src = reinterpret_cast<const float4 *>(X1 + (iv * M * M + mm) * MZ);
#pragma unroll
            for (int c = 0; c < MZ / 4; ++c) {
              const float4 v = src[c];
              const float xv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
              for (int r = 0; r < 4; ++r)
                if (4 * c + r < M) acc[j][4 * c + r] = fmaf(cv, xv[r], acc[j][4 * c + r]);
            }
          }
        }
      }
      const int zz = 2 * pr.za + pr.zb;
      if (ip == kPairs - 1 || 2 * c_pairs[ip + 1].za + c_pairs[ip + 1].zb != zz) {
#pragma unroll
        for (int j = 0; j < C::NPR; ++j) {
          const int pq = tid + j * NTH;
          if (pq < TT) {
#pragma unroll
            for (int iz = 0; iz < M; ++iz) {
              Y[(zz * M + iz) * TT + pq] = acc[j][iz];
              acc[j][iz] = 0.f;
            }
          }
        }
      }
      __syncthreads();
    }
    // stage 3: each thread the (k, k') block of its (t, t') pairs (its own
    // Y values), A[(k T + t), (k' T + t')] = sum_zz sum_iz Za(k,iz) Y Zb(k',iz)
    float *Aout = reinterpret_cast<float *>(a.A) + out_a(a, item, e, NSH);
#pragma unroll 1
    for (int j = 0; j < C::NPR; ++j) {
      const int pq = tid + j * NTH;
      if (pq >= TT) break;
      const int t = pq / T, t2 = pq - t * T;
      float blk[M][M];
#pragma unroll
      for (int k = 0; k < M; ++k)
#pragma unroll
        for (int k2 = 0; k2 < M; ++k2) blk[k][k2] = 0.f;
#pragma unroll
      for (int zz = 0; zz < 4; ++zz) {
        const float *Za = Z + (zz >> 1) * M * M, *Zb = Z + (zz & 1) * M * M;
#pragma unroll
        for (int iz = 0; iz < M; ++iz) {
          const float y = Y[(zz * M + iz) * TT + pq];
          float zb[M];
#pragma unroll
          for (int k2 = 0; k2 < M; ++k2) zb[k2] = Zb[k2 * M + iz];
#pragma unroll
          for (int k = 0; k < M; ++k) {
            const float ay = Za[k * M + iz] * y;
#pragma unroll
            for (int k2 = 0; k2 < M; ++k2) blk[k][k2] = fmaf(ay, zb[k2], blk[k][k2]);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < M; ++k) {
        const int row = k * T + t;
#pragma unroll
        for (int k2 = 0; k2 < M; ++k2) {
          const int col = k2 * T + t2;
          if (!a.upper || col >= row) Aout[a_pos(row, col, NSH, a.upper)] = st ? 0.f : blk[k][k2];
        }
      }
    }
    if (tid == 0) a.status[e] = st;
    __syncthreads();
  }
}

template <int P>
fei_status launch_sf(const fei_reference *ref, const FwdArgs &a, int64_t grid_work, cudaStream_t s,
                     int64_t grid_cap) {
  using C = SfCfg<P>;
  static_assert(sizeof(SfElem<P>) + C::DYN_SMEM <= 232448, "shared memory of one block (227 KB)");
  if (!ref->sf) return set_error(FEI_ERR_UNSUPPORTED, "no sum-factorised tables for degree %d", P);
  FEI_CUDA_TRY(cudaFuncSetAttribute(sf_forward_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::DYN_SMEM),
               "cudaFuncSetAttribute(sf_forward)");
  int dev, sms, per_sm = 1;
  FEI_CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
  FEI_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");
  FEI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sf_forward_kernel<P>, C::NTH, C::DYN_SMEM),
               "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if (per_sm < 1) per_sm = 1;
  int64_t blocks = grid_cap > 0 ? grid_cap : (int64_t)sms * per_sm;
  if (!a.count && blocks > grid_work) blocks = grid_work;
  if (blocks < 1) blocks = 1;
  sf_forward_kernel<P><<<(unsigned)blocks, C::NTH, C::DYN_SMEM, s>>>(a, ref->sf);
  FEI_CUDA_TRY(cudaGetLastError(), "sf_forward_kernel launch");
  return FEI_OK;
}

}  // namespace

fei_status build_sf_tables(fei_reference *r) {
  r->sf = nullptr;
  if (r->p < 3) return FEI_OK;
  const int n = sf_tab_size(r->p);
  double *t64 = nullptr;
  unsigned long long *dd = nullptr;
  cudaError_t e = cudaMalloc(&t64, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc(&dd, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(dd, 0, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) {
    sf_tables_kernel<<<1, 32>>>(r->p, r->znode, t64);
    sf_check_kernel<<<64, 256>>>(r->p, t64, r->G64, dd);
    e = cudaGetLastError();
  }
  unsigned long long h[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(h, dd, sizeof(h), cudaMemcpyDeviceToHost);
  float *t32 = nullptr;
  if (e == cudaSuccess) {
    double dmax, gmax;
    memcpy(&dmax, &h[0], 8);
    memcpy(&gmax, &h[1], 8);
    // the factors must reproduce the reference table (same basis, same
    // ordering, same signs) to FP64 rounding; otherwise no sum-factorised
    // path for this degree
    if (dmax <= 1e-12 * gmax) {
      e = cudaMalloc(&t32, sizeof(float) * n);
      if (e == cudaSuccess) {
        to_float_kernel<<<8, 256>>>(t64, n, t32);
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
  }
  if (t64) cudaFree(t64);
  if (dd) cudaFree(dd);
  if (e != cudaSuccess) {
    if (t32) cudaFree(t32);
    return cuda_error(e, "sum-factorisation tables");
  }
  r->sf = t32;
  return FEI_OK;
}

void free_sf_tables(fei_reference *r) {
  if (r->sf) cudaFree(r->sf);
  r->sf = nullptr;
}

fei_status launch_sf_forward(int p, const fei_reference *ref, const FwdArgs &a, int64_t grid_work, cudaStream_t s,
                             int64_t grid_cap) {
  if (grid_work <= 0) return FEI_OK;
  switch (p) {
    case 3: return launch_sf<3>(ref, a, grid_work, s, grid_cap);
    case 4: return launch_sf<4>(ref, a, grid_work, s, grid_cap);
    case 5: return launch_sf<5>(ref, a, grid_work, s, grid_cap);
    case 6: return launch_sf<6>(ref, a, grid_work, s, grid_cap);
    case 7: return launch_sf<7>(ref, a, grid_work, s, grid_cap);
  }
  return set_error(FEI_ERR_UNSUPPORTED, "sum-factorised path for degree %d", p);
}

}  // namespace fei
