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
// One thread block per element, persistent over elements: 512 threads and
// one block per SM at p = 6, 7 (the shared memory of one element), 256
// threads and three blocks per SM at p <= 5, where several elements in
// flight hide the latency of each one's short stages.  Setup: the
// element record is fetched one element ahead into registers; each node
// thread forms its own Jacobian columns in FP64 from the vertices; the
// point operators Dt of every point as in the FEI_FP32 path (FP64 w det J,
// FP32 adjugate and operator).  Then the 21 term pairs in turn: stage 1
// over all threads (one X1 chunk, the M values of zeta, per thread), stage
// 2 with each thread accumulating a fixed block of (t, t') pairs that share
// (m(t), m(t')), so that one X1 chunk serves the whole block and
// neighbouring threads read the same chunk; the block's sums stay in
// registers until the zeta pair changes.  Stage 3 with each thread forming
// the (k, k') block of its (t, t') pairs.  FP32 throughout the sums.  The
// load vector is factorised the same way.  The 1D factor tables are
// tabulated once per degree (FP64, stored FP32) and checked against the
// library's 3D reference table when the reference is created; a degree
// whose check fails has no sum-factorised path (FEI_ERR_UNSUPPORTED).
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
// Layout while tabulated (FP64), M = p+1, T = the triangle functions
// (total degree ascending, then n ascending):
//   U[3][M iu][M m], V[4][M iv][T t], Z[2][M k][M iz], mt[T] (m of t).
__host__ __device__ constexpr int sf_tab_size(int p) {
  return 3 * (p + 1) * (p + 1) + 4 * (p + 1) * ((p + 1) * (p + 2) / 2) + 2 * (p + 1) * (p + 1) +
         (p + 1) * (p + 2) / 2;
}
// The kernel's FP32 copy, with the node index of U and Z innermost and
// padded to MZ = M rounded up to 4 (16-byte loads; pads are zero):
//   UT[3][M m][MZ iu], V[4][M iv][T t], ZT[2][M iz][MZ k], mt[T].
__host__ __device__ constexpr int sf_mz(int p) { return (p + 4) / 4 * 4; }
__host__ __device__ constexpr int sf_ktab_size(int p) {
  return 3 * (p + 1) * sf_mz(p) + 4 * (p + 1) * ((p + 1) * (p + 2) / 2) + 2 * (p + 1) * sf_mz(p) +
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

// The FP64 tables rounded to FP32 in the kernel's layout.
__global__ void pack_tables_kernel(int p, const double *t64, float *t32) {
  const int M = p + 1, MZ = sf_mz(p), T = (p + 1) * (p + 2) / 2;
  const double *U = t64, *V = U + 3 * M * M, *Z = V + 4 * M * T, *mt = Z + 2 * M * M;
  float *UT = t32, *V32 = UT + 3 * M * MZ, *ZT = V32 + 4 * M * T, *mt32 = ZT + 2 * M * MZ;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < sf_ktab_size(p); i += gridDim.x * blockDim.x) {
    if (i < 3 * M * MZ) {
      const int kind = i / (M * MZ), m = (i / MZ) % M, iu = i % MZ;
      UT[i] = iu < M ? (float)U[(kind * M + iu) * M + m] : 0.f;
    } else if (i < 3 * M * MZ + 4 * M * T) {
      const int j = i - 3 * M * MZ;
      V32[j] = (float)V[j];
    } else if (i < 3 * M * MZ + 4 * M * T + 2 * M * MZ) {
      const int j = i - 3 * M * MZ - 4 * M * T;
      const int kind = j / (M * MZ), iz = (j / MZ) % M, k = j % MZ;
      ZT[j] = k < M ? (float)Z[(kind * M + k) * M + iz] : 0.f;
    } else {
      const int j = i - 3 * M * MZ - 4 * M * T - 2 * M * MZ;
      mt32[j] = (float)mt[j];
    }
  }
}

// ---------------------------------------------------------------------------
// The kernel
// ---------------------------------------------------------------------------
template <int P>
struct SfCfg {
  static constexpr int M = P + 1, T = (P + 1) * (P + 2) / 2, NSH = nsh_of(P), NQ = nq_of(P), NT2 = M * M;
  static constexpr int MZ = sf_mz(P);  // a node index padded for 16-byte loads
  static constexpr int NTH = P >= 7 ? 512 : P == 6 ? 416 : 256;
  // blocks per SM the register budget is set for: several small elements
  // in flight per SM hide the latency of each one's short stages
  static constexpr int MINB = P <= 5 ? 3 : 1;
  static constexpr int TT = T * T;
  static constexpr int NPR = (TT + NTH - 1) / NTH;  // stage-3 (t, t') pairs per thread
  // stage 2: each thread a BR x BC block of (t, t') pairs sharing (m(t), m(t'))
  static constexpr int BR = P >= 6 ? 2 : 1, BC = P >= 5 ? 2 : 1;
  static constexpr int NBLK = [] {
    int a = 0, b = 0;
    for (int m = 0; m < M; ++m) a += (M - m + BR - 1) / BR, b += (M - m + BC - 1) / BC;
    return a * b;
  }();
  static constexpr int TAB = sf_ktab_size(P);
  static constexpr int NQP = M * M * MZ;  // points with the u index padded
  // dynamic shared memory (floats): tables, Dt [13][M iz][M iv][MZ iu],
  // F [NQ], X1 [M iv][M m][M m'][MZ iz] (16-byte halves swizzled), Y [4 zz][M iz][T*T]
  static constexpr int O_DT = (TAB + 3) / 4 * 4;
  static constexpr int O_F = O_DT + 13 * NQP;
  static constexpr int O_X1 = (O_F + NQ + 3) / 4 * 4;  // 16-byte aligned
  static constexpr int O_Y = O_X1 + M * M * M * MZ;
  static constexpr int FLOATS = O_Y + 4 * M * TT;
  static constexpr int DYN_SMEM = FLOATS * 4;
  static_assert(NBLK <= NTH, "one stage-2 block per thread");
  static_assert(32 + NT2 <= NTH, "one thread per triangle node");
};

// Element data in FP64 and its FP32 copies (the FEI_FP32 path's point
// operator: FP64 columns and w det J, FP32 adjugate).
template <int P>
struct SfElem {
  using C = SfCfg<P>;
  double X[18], cd[14];
  float cdf[14];  // the per-element coefficients rounded once
  double zn3w[C::M][3], tc3w[C::NT2][3];
  float zc1f[C::M][3], zc2f[C::M][3], zn3f[C::M][3], zwf[C::M];
  float tc3f[C::NT2][3], twf[C::NT2];
  int status;
};

// Position of 16-byte half c of X1 chunk ch (MZ floats): with two halves,
// swapped when bit 2 of the chunk index is set, so that the eight chunks a
// quarter-warp touches fall in distinct banks.
template <int MZ>
__device__ __forceinline__ int x1_half(int ch, int c) {
  return MZ == 8 ? c ^ ((ch >> 2) & 1) : c;
}

// Index of the triangle function (m, n): total degree ascending, then n.
__device__ __forceinline__ int tri_index(int m, int n) { return (m + n) * (m + n + 1) / 2 + n; }

// Columns c1, c2 and n3 = c1 x c2 at the vertical node z from the vertex
// coordinates (the element vectors A1, B1, A2, B2 of fei_geom.cuh formed
// by each node thread for itself), FP64.
__device__ __forceinline__ void z_columns_from_vertices(const double *X, double z, double *c1, double *c2,
                                                        double *n3) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double e1p = X[3 + k] - X[k], e1q = X[12 + k] - X[9 + k];
    const double e2p = X[6 + k] - X[k], e2q = X[15 + k] - X[9 + k];
    c1[k] = fma(z, 0.5 * (e1q - e1p), 0.5 * (e1p + e1q));
    c2[k] = fma(z, 0.5 * (e2q - e2p), 0.5 * (e2p + e2q));
  }
  cross3(c1, c2, n3);
}
// Column c3 at the triangle node (xi1, xi2) (element vectors C, D1, D2).
__device__ __forceinline__ void t_column_from_vertices(const double *X, double xi1, double xi2, double *c3) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double v0 = X[9 + k] - X[k], v1 = X[12 + k] - X[3 + k], v2 = X[15 + k] - X[6 + k];
    c3[k] = fma(xi2, 0.5 * (v2 - v0), fma(xi1, 0.5 * (v1 - v0), 0.5 * v0));
  }
}

template <int P>
__global__ void __launch_bounds__(SfCfg<P>::NTH, SfCfg<P>::MINB) sf_forward_kernel(FwdArgs a, const float *gtab) {
  using C = SfCfg<P>;
  constexpr int M = C::M, MZ = C::MZ, T = C::T, NSH = C::NSH, NQ = C::NQ, NT2 = C::NT2, NTH = C::NTH, TT = C::TT;
  constexpr int BR = C::BR, BC = C::BC;
  extern __shared__ __align__(16) float sm[];
  __shared__ SfElem<P> E;
  const float *UT = sm, *V = sm + 3 * M * MZ, *ZT = V + 4 * M * T, *mtf = ZT + 2 * M * MZ;
  float *Dt = sm + C::O_DT, *Fq = sm + C::O_F, *X1 = sm + C::O_X1, *Y = sm + C::O_Y;
  const int tid = threadIdx.x;
  for (int i = tid; i < C::TAB; i += NTH) sm[i] = gtab[i];
  for (int i = tid; i < 13 * C::NQP; i += NTH) Dt[i] = 0.f;  // the pads (u >= M) stay zero
  const int64_t items = a.count ? (int64_t)(*a.count) : a.n_work;

  // the nodes of this thread (constant over elements): vertical node tid
  // (tid < M), triangle node tid - 32 (32 <= tid < 32 + NT2)
  double nz = 0.0, nwz = 0.0, nx1 = 0.0, nx2 = 0.0, nwt = 0.0;
  if (tid < M) {
    nz = a.znode[2 * tid];
    nwz = a.znode[2 * tid + 1];
  } else if (tid >= 32 && tid < 32 + NT2) {
    nx1 = a.tnode[4 * (tid - 32)];
    nx2 = a.tnode[4 * (tid - 32) + 1];
    nwt = a.tnode[4 * (tid - 32) + 2];
  }
  // the stage-2 block of this thread (constant over elements): BR x BC
  // pairs (t, t') with m(t) = mA, m(t') = mB, blocks ordered by (mA, mB) so
  // that neighbouring threads read the same X1 rows; a ragged block repeats
  // a valid pair (computed, not stored: vmask)
  int tA[BR], tB[BC], mm = 0, vmask = 0;
#pragma unroll
  for (int r = 0; r < BR; ++r) tA[r] = 0;
#pragma unroll
  for (int c = 0; c < BC; ++c) tB[c] = 0;
  {
    int base = 0;
    for (int mA = 0; mA < M; ++mA)
      for (int mB = 0; mB < M; ++mB) {
        const int na = (M - mA + BR - 1) / BR, nb = (M - mB + BC - 1) / BC;
        if (tid >= base && tid < base + na * nb) {
          const int ia = (tid - base) / nb, ib = (tid - base) % nb;
#pragma unroll
          for (int r = 0; r < BR; ++r) {
            const int n = ia * BR + r;
            tA[r] = tri_index(mA, n < M - mA ? n : M - 1 - mA);
#pragma unroll
            for (int c = 0; c < BC; ++c) {
              const int n2 = ib * BC + c;
              if (n < M - mA && n2 < M - mB) vmask |= 1 << (r * BC + c);
            }
          }
#pragma unroll
          for (int c = 0; c < BC; ++c) {
            const int n2 = ib * BC + c;
            tB[c] = tri_index(mB, n2 < M - mB ? n2 : M - 1 - mB);
          }
          mm = mA * M + mB;
        }
        base += na * nb;
      }
  }

  // this thread's share of work item it's record: a vertex coordinate
  // (threads 0..17) or a per-element coefficient (threads 18..31)
  auto fetch = [&](int64_t it) -> double {
    if (it >= items || tid >= 32) return 0.0;
    const int64_t e = a.list ? (int64_t)a.list[it] : it;
    if (tid < 18) return a.geom[18 * e + tid];
    if (a.coef_mode != FEI_COEF_PER_ELEMENT) return 0.0;
    const int j = tid - 18;
    return j < 9 ? a.K[9 * e + j] : j < 12 ? a.b[3 * e + j - 9] : j == 12 ? a.c[e] : a.f[e];
  };
  double rec = fetch(blockIdx.x);

  for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
    const int64_t e = a.list ? (int64_t)a.list[item] : item;
    // the element record into shared memory; the next one's loads issued
    if (tid == 0) E.status = 0;
    if (tid < 18) E.X[tid] = rec;
    else if (tid < 32) {
      E.cd[tid - 18] = rec;
      E.cdf[tid - 18] = (float)rec;
    }
    const bool ok = tid >= 32 || (tid >= 18 && a.coef_mode != FEI_COEF_PER_ELEMENT) || finite64(rec);
    rec = fetch(item + gridDim.x);
    __syncthreads();
    if (!ok) atomicMax(&E.status, FEI_ERR_NONFINITE);
    if (tid == 32 && a.coef_mode == FEI_COEF_PER_ELEMENT && a.upper && !coef_symmetric(E.cd, E.cd + 9))
      atomicMax(&E.status, FEI_ERR_INVALID_ARG);
    // FP64 node columns: vertical nodes (c1, c2, n3) and triangle nodes (c3)
    if (tid < M) {
      double c1[3], c2[3], n3[3];
      z_columns_from_vertices(E.X, nz, c1, c2, n3);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        E.zc1f[tid][k] = (float)c1[k];
        E.zc2f[tid][k] = (float)c2[k];
        E.zn3f[tid][k] = (float)n3[k];
        E.zn3w[tid][k] = nwz * n3[k];
      }
      E.zwf[tid] = (float)nwz;
    } else if (tid >= 32 && tid < 32 + NT2) {
      const int t = tid - 32;
      double c3[3];
      t_column_from_vertices(E.X, nx1, nx2, c3);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        E.tc3f[t][k] = (float)c3[k];
        E.tc3w[t][k] = nwt * c3[k];
      }
      E.twf[t] = (float)nwt;
    }
    __syncthreads();
    // the point operators of every point (Dt by component, w det J f)
    for (int q = tid; q < NQ; q += NTH) {
      const int iz = q / NT2, t = q - iz * NT2;
      double cq[14];
      float K[9], b[3], cf, ff;
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
#pragma unroll
        for (int k = 0; k < 9; ++k) K[k] = (float)cq[k];
#pragma unroll
        for (int k = 0; k < 3; ++k) b[k] = (float)cq[9 + k];
        cf = (float)cq[12];
        ff = (float)cq[13];
      } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) K[k] = E.cdf[k];
#pragma unroll
        for (int k = 0; k < 3; ++k) b[k] = E.cdf[9 + k];
        cf = E.cdf[12];
        ff = E.cdf[13];
      }
      const double s = dot3(E.zn3w[iz], E.tc3w[t]);  // w det J in FP64
      const float sf = (float)s, wf = E.zwf[iz] * E.twf[t];
      float a0[3], a1[3], D[16];
      cross3(E.zc2f[iz], E.tc3f[t], a0);
      cross3(E.tc3f[t], E.zc1f[iz], a1);
      dt_from_adj<float>(a0, a1, E.zn3f[iz], wf, sf, wf * wf / sf, K, b, cf, ff, D);
#pragma unroll
      for (int k = 0; k < 13; ++k) Dt[k * C::NQP + (q / M) * MZ + q % M] = D[k];
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
        for (int iu = 0; iu < M; ++iu) acc = fmaf(UT[m * MZ + iu], Fq[(iz * M + iv) * M + iu], acc);
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
        for (int iz = 0; iz < M; ++iz) acc = fmaf(ZT[iz * MZ + k], F2[iz * T + t], acc);
        bout[i] = st ? 0.f : acc;
      }
      __syncthreads();
    }
    // stages 1 and 2 over the term pairs; each thread accumulates the Y of
    // its stage-2 block in registers and writes them when the zeta pair zz
    // changes
    float acc[BR][BC][M];
#pragma unroll
    for (int r = 0; r < BR; ++r)
#pragma unroll
      for (int c = 0; c < BC; ++c)
#pragma unroll
        for (int iz = 0; iz < M; ++iz) acc[r][c][iz] = 0.f;
    for (int ip = 0; ip < kPairs; ++ip) {
      const SfPair pr = c_pairs[ip];
      const float *Ua = UT + pr.ua * M * MZ, *Ub = UT + pr.ub * M * MZ;
      const float *Va = V + pr.va * M * T, *Vb = V + pr.vb * M * T;
      const float *Dd = Dt + pr.d * C::NQP;
      // stage 1: thread o = (iv, m, m') forms X1 chunk o (the M values of iz)
      for (int o = tid; o < M * M * M; o += NTH) {
        const int iv = o / (M * M), m = (o / M) % M, m2 = o % M;
        float cu[MZ];  // Ua(iu, m) Ub(iu, m')
#pragma unroll
        for (int c = 0; c < MZ / 4; ++c) {
          const float4 ua = reinterpret_cast<const float4 *>(Ua + m * MZ)[c];
          const float4 ub = reinterpret_cast<const float4 *>(Ub + m2 * MZ)[c];
          cu[4 * c] = ua.x * ub.x;
          cu[4 * c + 1] = ua.y * ub.y;
          cu[4 * c + 2] = ua.z * ub.z;
          cu[4 * c + 3] = ua.w * ub.w;
        }
        float x[MZ];
#pragma unroll
        for (int iz = 0; iz < MZ; ++iz) {
          x[iz] = 0.f;
          if (iz < M) {
            const float4 *row = reinterpret_cast<const float4 *>(Dd + (iz * M + iv) * MZ);
#pragma unroll
            for (int c = 0; c < MZ / 4; ++c) {
              const float4 d = row[c];
              const float dv[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
              for (int r = 0; r < 4; ++r)
                if (4 * c + r < M) x[iz] = fmaf(cu[4 * c + r], dv[r], x[iz]);
            }
          }
        }
        float4 *dst = reinterpret_cast<float4 *>(X1 + o * MZ);
#pragma unroll
        for (int c = 0; c < MZ / 4; ++c)
          dst[x1_half<MZ>(o, c)] = make_float4(x[4 * c], x[4 * c + 1], x[4 * c + 2], x[4 * c + 3]);
      }
      __syncthreads();
      // stage 2: Y[iz][t][t'] += sum_iv Va(iv,t) Vb(iv,t') X1[iv][m(t)][m(t')][iz]
      if (vmask) {
#pragma unroll
        for (int iv = 0; iv < M; ++iv) {
          const int ch = iv * M * M + mm;
          const float4 *src = reinterpret_cast<const float4 *>(X1 + ch * MZ);
          float x[MZ];
#pragma unroll
          for (int c = 0; c < MZ / 4; ++c) {
            const float4 v = src[x1_half<MZ>(ch, c)];
            x[4 * c] = v.x, x[4 * c + 1] = v.y, x[4 * c + 2] = v.z, x[4 * c + 3] = v.w;
          }
          float va[BR], vb[BC];
#pragma unroll
          for (int r = 0; r < BR; ++r) va[r] = Va[iv * T + tA[r]];
#pragma unroll
          for (int c = 0; c < BC; ++c) vb[c] = Vb[iv * T + tB[c]];
#pragma unroll
          for (int r = 0; r < BR; ++r)
#pragma unroll
            for (int c = 0; c < BC; ++c) {
              const float cv = va[r] * vb[c];
#pragma unroll
              for (int iz = 0; iz < M; ++iz) acc[r][c][iz] = fmaf(cv, x[iz], acc[r][c][iz]);
            }
        }
      }
      const int zz = 2 * pr.za + pr.zb;
      if (ip == kPairs - 1 || 2 * c_pairs[ip + 1].za + c_pairs[ip + 1].zb != zz) {
#pragma unroll
        for (int r = 0; r < BR; ++r)
#pragma unroll
          for (int c = 0; c < BC; ++c) {
            if ((vmask >> (r * BC + c)) & 1) {
              float *yp = Y + zz * M * TT + tA[r] * T + tB[c];
#pragma unroll
              for (int iz = 0; iz < M; ++iz) yp[iz * TT] = acc[r][c][iz];
            }
#pragma unroll
            for (int iz = 0; iz < M; ++iz) acc[r][c][iz] = 0.f;
          }
      }
      __syncthreads();
    }
    // stage 3: thread tid the (k, k') blocks of pairs pq = tid + j NTH,
    // A[(k T + t), (k' T + t')] = sum_zz sum_iz Za(k,iz) Y Zb(k',iz)
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
#pragma unroll 1
      for (int zz = 0; zz < 4; ++zz) {
        const float *Za = ZT + (zz >> 1) * M * MZ, *Zb = ZT + (zz & 1) * M * MZ;
#pragma unroll
        for (int iz = 0; iz < M; ++iz) {
          const float y = Y[(zz * M + iz) * TT + pq];
          float za[MZ], zb[MZ];
#pragma unroll
          for (int c = 0; c < MZ / 4; ++c) {
            const float4 va = reinterpret_cast<const float4 *>(Za + iz * MZ)[c];
            const float4 vb = reinterpret_cast<const float4 *>(Zb + iz * MZ)[c];
            za[4 * c] = va.x, za[4 * c + 1] = va.y, za[4 * c + 2] = va.z, za[4 * c + 3] = va.w;
            zb[4 * c] = vb.x, zb[4 * c + 1] = vb.y, zb[4 * c + 2] = vb.z, zb[4 * c + 3] = vb.w;
          }
#pragma unroll
          for (int k = 0; k < M; ++k) {
            const float ay = za[k] * y;
#pragma unroll
            for (int k2 = 0; k2 < M; ++k2) blk[k][k2] = fmaf(ay, zb[k2], blk[k][k2]);
          }
        }
      }
      if (!a.upper) {
        // A_e[k T + t][k' T + t'] at a constant offset from A_e[t][t']
        float *o = Aout + t * NSH + t2;
#pragma unroll
        for (int k = 0; k < M; ++k)
#pragma unroll
          for (int k2 = 0; k2 < M; ++k2)
            o[k * T * NSH + k2 * T] = st ? 0.f : blk[k][k2];
      } else {
#pragma unroll
        for (int k = 0; k < M; ++k) {
          const int row = k * T + t;
#pragma unroll
          for (int k2 = 0; k2 < M; ++k2) {
            const int col = k2 * T + t2;
            if (col >= row)
              Aout[a_pos(row, col, NSH, true)] = st ? 0.f : blk[k][k2];
          }
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
  const int n = sf_tab_size(r->p), nk = sf_ktab_size(r->p);
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
      e = cudaMalloc(&t32, sizeof(float) * nk);
      if (e == cudaSuccess) {
        pack_tables_kernel<<<8, 256>>>(r->p, t64, t32);
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
