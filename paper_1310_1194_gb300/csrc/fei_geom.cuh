// fei_geom.cuh -- geometry of the bilinear prism and the point operator.
//
// Geometry (Sec. 4, the geometrically bilinear prism; Algorithm 1 step 7):
// with bottom vertices P_a = X_a and top vertices Q_a = X_{a+3} (a = 0,1,2),
//   x(xi, zeta) = sum_a lambda_a(xi) [ (1-zeta)/2 P_a + (1+zeta)/2 Q_a ],
// the Jacobian columns are
//   c1 = dx/dxi1  = A1 + zeta B1,      c2 = dx/dxi2 = A2 + zeta B2,
//   c3 = dx/dzeta = C + xi1 D1 + xi2 D2,
// A1 = ((P1-P0) + (Q1-Q0))/2, B1 = ((Q1-Q0) - (P1-P0))/2 (same with 2),
// C = (Q0-P0)/2, D1 = ((Q1-P1) - (Q0-P0))/2, D2 = ((Q2-P2) - (Q0-P0))/2.
// So c1, c2 depend only on the vertical node and c3 only on the triangle
// node; det J = (c1 x c2) . c3 and J^{-1} has rows
//   adj_0 = c2 x c3, adj_1 = c3 x c1, adj_2 = c1 x c2, divided by det J.
// The element vectors are differences of vertex coordinates and are always
// formed in FP64 (this is where FP32 would lose the most: |x| ~ 1, h ~ 1/50).
//
// Point operator (Eq. (2) with the general weak form): with
// T = blockdiag(1, J^{-T}) and D = [[c, b^T], [0, K]] (row = test
// component (value, d/dx), column = trial component),
//   Dt_q = w det J  T^T D T
//        = [[ w det J c,  w (adj_l . b) ], [ 0, (w/det J) adj_l K adj_m^T ]],
// and A_e[i][j] = sum_q sum_{a,b} G[q][a][i] Dt_q[a][b] G[q][b][j] with
// G[q] = (phi, dphi/dxi1, dphi/dxi2, dphi/dzeta).  Layout of Dt in memory:
//   [0] = Dt00, [1..3] = Dt0l, [4..12] = Dt_lm (row-major l, m),
//   [13] = w det J f (load-vector weight), [14] = w det J, [15] unused.
#pragma once

#include <math.h>
#include <string.h>

#include "fei_internal.cuh"

namespace fei {

__device__ __forceinline__ void elem_vectors(const double *X, double *ev) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double p0 = X[0 + k], p1 = X[3 + k], p2 = X[6 + k];
    const double q0 = X[9 + k], q1 = X[12 + k], q2 = X[15 + k];
    const double e1p = p1 - p0, e1q = q1 - q0, e2p = p2 - p0, e2q = q2 - q0;
    const double v0 = q0 - p0, v1 = q1 - p1, v2 = q2 - p2;
    ev[0 + k] = 0.5 * (e1p + e1q);   // A1
    ev[3 + k] = 0.5 * (e1q - e1p);   // B1
    ev[6 + k] = 0.5 * (e2p + e2q);   // A2
    ev[9 + k] = 0.5 * (e2q - e2p);   // B2
    ev[12 + k] = 0.5 * v0;           // C
    ev[15 + k] = 0.5 * (v1 - v0);    // D1
    ev[18 + k] = 0.5 * (v2 - v0);    // D2
  }
}

template <typename T>
__device__ __forceinline__ void cross3(const T *a, const T *b, T *r) {
  r[0] = a[1] * b[2] - a[2] * b[1];
  r[1] = a[2] * b[0] - a[0] * b[2];
  r[2] = a[0] * b[1] - a[1] * b[0];
}

template <typename T>
__device__ __forceinline__ T dot3(const T *a, const T *b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// Vertical-node quantities: c1, c2 and n3 = c1 x c2 (FP64).
__device__ __forceinline__ void znode_columns(const double *ev, double z, double *c1, double *c2,
                                              double *n3) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    c1[k] = fma(z, ev[3 + k], ev[0 + k]);
    c2[k] = fma(z, ev[9 + k], ev[6 + k]);
  }
  cross3(c1, c2, n3);
}

// Triangle-node quantity: c3 (FP64).
__device__ __forceinline__ void tnode_column(const double *ev, double xi1, double xi2, double *c3) {
#pragma unroll
  for (int k = 0; k < 3; ++k) c3[k] = fma(xi2, ev[18 + k], fma(xi1, ev[15 + k], ev[12 + k]));
}

// Dt from adjugate rows, w, s = w det J and the coefficients, in type T.
// winv_det = w / det J.
template <typename T>
__device__ __forceinline__ void dt_from_adj(const T *a0, const T *a1, const T *a2, T w, T s,
                                            T winv_det, const T *K, const T *b, T c, T f, T *D) {
  const T *adj[3] = {a0, a1, a2};
  D[0] = s * c;
#pragma unroll
  for (int l = 0; l < 3; ++l) D[1 + l] = w * dot3(adj[l], b);
  T Ka[3][3];  // Ka[m] = K adj_m^T
#pragma unroll
  for (int m = 0; m < 3; ++m)
#pragma unroll
    for (int r = 0; r < 3; ++r) Ka[m][r] = K[3 * r + 0] * adj[m][0] + K[3 * r + 1] * adj[m][1] + K[3 * r + 2] * adj[m][2];
#pragma unroll
  for (int l = 0; l < 3; ++l)
#pragma unroll
    for (int m = 0; m < 3; ++m) D[4 + 3 * l + m] = winv_det * dot3(adj[l], Ka[m]);
  D[13] = s * f;
  D[14] = s;
  D[15] = T(0);
}

// Double-FP32 arithmetic (w det J on the FP32-class paths, reading the
// FP64 node sums once per node and forming each point's value in FP32
// pipes; one FP64 instruction costs tens of FP32 ones on this part).
// An FP64 value as an unevaluated sum of two FP32 values, hi = rn(x) and
// lo = rn(x - hi): 48 significant bits, enough for products and sums whose
// FP32 rounding is taken once at the end.
__device__ __forceinline__ float2 split_f64(double x) {
  const float hi = (float)x;
  return make_float2(hi, (float)(x - (double)hi));
}
// a.x b.x + a.y b.x + a.x b.y (the lo * lo term is below 2^-46 relative)
// as (product, error) with the error of the leading product exact (FMA)
__device__ __forceinline__ float2 mul_ff(float2 a, float2 b) {
  const float p = a.x * b.x;
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  return make_float2(p, e);
}
// sum of two (value, error) pairs, the rounding error of the leading sum
// kept exactly (Knuth's two-sum)
__device__ __forceinline__ float2 add_ff(float2 a, float2 b) {
  const float s = a.x + b.x;
  const float bb = s - a.x;
  const float err = (a.x - (s - bb)) + (b.x - bb);
  return make_float2(s, err + a.y + b.y);
}
// a.x + a.y as (s, e): s the FP32 sum, e its exact rounding error (two-sum),
// so that s carries the leading bits again after a cancellation
__device__ __forceinline__ float2 norm_ff(float2 a) {
  const float s = a.x + a.y;
  const float bb = s - a.x;
  const float e = (a.x - (s - bb)) + (a.y - bb);
  return make_float2(s, e);
}
__device__ __forceinline__ float2 neg_ff(float2 a) { return make_float2(-a.x, -a.y); }
// An FP64 value as hi + lo in FP32 from its bit fields, integer operations
// only: hi = x with the significand cut to 24 bits (exact), lo = the next
// 29 bits rounded to 24, so hi + lo = x to 2^-47 relative.  in_range is false
// (and the pair meaningless) outside 2^-60 <= |x| < 2^60, except x = +-0.
__host__ __device__ inline float2 split_f64_bits(double x, bool *in_range) {
  unsigned long long b;
  memcpy(&b, &x, 8);
  const unsigned h = (unsigned)(b >> 32), l = (unsigned)b;
  const int E = (int)((h >> 20) & 0x7ffu) - 1023;
  const unsigned sgn = h & 0x80000000u;
  if ((b << 1) == 0ull) {
    *in_range = true;
    return make_float2(0.f, 0.f);
  }
  *in_range = E >= -60 && E < 60;
  const int ef = *in_range ? E + 127 : 127;
  const unsigned hb = sgn | ((unsigned)ef << 23) | ((h & 0xfffffu) << 3) | (l >> 29), sb = (unsigned)ef << 23;
  float hi, scale;
  memcpy(&hi, &hb, 4);
  memcpy(&scale, &sb, 4);
  // m[28:0] 2^(E - 52): the 29 low bits as an integer (rounded to 24),
  // scaled by 2^-52 and 2^E (both exact)
  const float lo = (float)(l & 0x1fffffffu) * 2.220446049250313e-16f * scale;
  return make_float2(hi, sgn ? -lo : lo);
}
// FP64 -> FP32 rounded to nearest (ties to even) from the bit fields, for
// a finite x whose FP32 result is normal or overflows; other magnitudes
// take the conversion instruction (which runs on the FP64 pipe).
__host__ __device__ inline float f64_to_f32_bits(double x) {
  unsigned long long b;
  memcpy(&b, &x, 8);
  const unsigned h = (unsigned)(b >> 32), l = (unsigned)b;
  const int e = (int)((h >> 20) & 0x7ffu) - 1023 + 127;
  if (e < 1 || e > 254) return (float)x;
  unsigned r = (h & 0x80000000u) | ((unsigned)e << 23) | ((h & 0xfffffu) << 3) | (l >> 29);
  const unsigned rest = l & 0x1fffffffu;  // the 29 bits cut off
  r += (rest > 0x10000000u || (rest == 0x10000000u && (r & 1u))) ? 1u : 0u;  // a carry raises the exponent
  float f;
  memcpy(&f, &r, 4);
  return f;
}
// Finite test on the exponent bits of an FP64 value (integer pipe: FP64
// compares run at the FP64 rate, which is low on this part).
__device__ __forceinline__ bool finite64(double x) {
  return ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff;
}

// Status of one point from s = w det J: 0 ok, 3 det <= 0, 4 non-finite.
__device__ __forceinline__ int point_status(double s) {
  if (!finite64(s)) return FEI_ERR_NONFINITE;
  if (!(s > 0.0)) return FEI_ERR_NEGATIVE_JACOBIAN;
  return 0;
}

__device__ __forceinline__ int merge_status(int a, int b) {
  // NONFINITE takes precedence over NEGATIVE_JACOBIAN, which takes
  // precedence over INVALID_ARG (a non-symmetric record in the upper layout)
  if (a == FEI_ERR_NONFINITE || b == FEI_ERR_NONFINITE) return FEI_ERR_NONFINITE;
  return a > b ? a : b;
}

}  // namespace fei
