// fei_backward.cu -- reverse pass of the element integration.
//
// L = <gA, A> + <gb, b>.  With A_e = sum_q G_q^T Dt_q G_q (fei_geom.cuh):
//   dL/dDt_q[a][b] = (G_q gA G_q^T)[a][b] = sum_i G[q][a][i] W[i][(q,b)],
//   W = gA G^T  (N_sh x 4 N_q, the same contraction size as the forward),
//   dL/d(w det J f)_q = sum_i gb_i phi_i(q).
// The Jacobian is recomputed at every point (never stored) and the chain
// from dL/dDt to the coefficients, to the adjugate rows and det J, to the
// Jacobian columns c1, c2, c3, to the element vectors and finally to the 18
// vertex coordinates runs in FP64:
//   Dt00 = w det c, Dt0l = w adj_l.b, Dt_lm = (w/det) adj_l K adj_m^T,
//   adj_0 = c2 x c3, adj_1 = c3 x c1, adj_2 = c1 x c2, det = adj_2 . c3,
//   c1 = A1 + zeta B1, c2 = A2 + zeta B2, c3 = C + xi1 D1 + xi2 D2.
// One thread block per element; rows of gA are processed in blocks of 32 and
// points in chunks of 8, with dL/dDt accumulated in shared memory.
#include <type_traits>

#include "fei_geom.cuh"
#include "fei_internal.cuh"

namespace fei {
namespace {

template <typename T>
__device__ __forceinline__ const T *gtab_b(const BwdArgs &a);
template <>
__device__ __forceinline__ const double *gtab_b<double>(const BwdArgs &a) { return a.G64; }
template <>
__device__ __forceinline__ const float *gtab_b<float>(const BwdArgs &a) { return a.G32; }

// W = gA G^T is computed in tiles of BI rows x KC columns (QC points x 4),
// TM x TN outputs per thread; the operand rows are stored with a padded
// stride NSHP (a multiple of 4, plus 4) so that the 16-byte loads of the
// threads of a warp fall into distinct banks.
template <typename T, int P, bool Q = false>
struct BwdCfg {
  static constexpr bool F32 = std::is_same<T, float>::value;
  static constexpr int NSH = nsh_of(P), NQ = nq_of(P), NZ = P + 1, NT = (P + 1) * (P + 1);
  static constexpr int BI = F32 ? 64 : 32, QC = F32 ? 16 : 8, KC = 4 * QC;
  static constexpr int TM = BI / 16, TN = KC / 16;  // outputs per thread (16 x 16 threads)
  static constexpr int NSHP = F32 ? (NSH + 3) / 4 * 4 + 4 : NSH;
  // dynamic shared memory layout (bytes); the quadratic-loss adjoint (Q)
  // needs only u (in the gA area) and the per-point results
  static constexpr size_t OFF_GA = 0;                                        // T [BI][NSHP] (Q: u [NSH])
  static constexpr size_t OFF_GC = OFF_GA + (Q ? sizeof(T) * ((NSH + 3) / 4 * 4) : sizeof(T) * BI * NSHP);
  static constexpr size_t OFF_W = OFF_GC + (Q ? 0 : sizeof(T) * KC * NSHP);  // T [BI][KC]
  static constexpr size_t OFF_GD = OFF_W + (Q ? 0 : sizeof(T) * BI * KC);    // T [NQ][16]
  static constexpr size_t OFF_GSF = OFF_GD + sizeof(T) * NQ * 16;            // T [NQ]
  static constexpr size_t OFF_END = ((OFF_GSF + sizeof(T) * NQ + 15) / 16) * 16;
  // the sums over points reuse the dynamic area: per warp 35 values x 32
  // lanes (rows padded to 33) in FP64
  static constexpr size_t RED_BYTES = F32 ? sizeof(float) * 35 * 256 : sizeof(double) * 8 * 35 * 33;
  static constexpr size_t SMEM = OFF_END > RED_BYTES ? OFF_END : RED_BYTES;
};

struct BwdStatic {
  double X[18];
  double ev[21];
  double cd[14];
  double zc1[8][3], zc2[8][3], zn3[8][3], zz[8], zw[8];
  double tc3[64][3], txi[64][2], tw[64];
  double gev[21];   // gradient of the element vectors
  double gcoef[14]; // per-element coefficient gradient
  int status;
};
// FP32 path: node tables of the block (once) and per element the FP32
// element vectors, node columns and node sums of det J (FP32 pairs), the
// coefficients in FP32 and the element-vector gradients as FP32 pairs
struct BwdTablesF32 {
  float2 ttab2[64][3];  // (w_t, w_t xi1, w_t xi2) as FP32 hi + lo
  float ttabf[64][3];   // (w_t, xi1, xi2)
  float2 ztab2[8][2];   // (zeta, w_z) as FP32 hi + lo
  float ztabf[8][2];    // (zeta, w_z)
  float evf[21];
  float cdf[14];
  float zc1f[8][3], zc2f[8][3], zn3f[8][3];
  float2 zabg[8][3];    // w_z (n3.C, n3.D1, n3.D2)
  float tc3f[64][3];
  float2 gev2[21];
  // for single roundings of c3, w and det J: the element vectors and the
  // node sums (n3.C, n3.D1, n3.D2) as FP32 pairs, xi1, xi2 as pairs
  float2 ev2[21];
  float2 zsum[8][3];
  float2 txi2[64][2];
};
// the block's static shared data: the FP32 tables only in FP32 kernels (the
// FP64 kernel at p = 7 needs the room for its dynamic area)
template <bool F32>
struct BwdShared : BwdStatic {};
template <>
struct BwdShared<true> : BwdStatic, BwdTablesF32 {};

__device__ __forceinline__ int point_status_f(float s) {
  if (!(fabsf(s) <= 3.402823466e38f)) return FEI_ERR_NONFINITE;
  if (!(s > 0.f)) return FEI_ERR_NEGATIVE_JACOBIAN;
  return 0;
}

// FP32 path, warp 0: the element vectors (lanes 0-20, component k = j % 3 of
// vector j / 3) and the vertical-node quantities (lanes 3 iz + k: c1, c2,
// n3 = c1 x c2 and w_z (n3.C, n3.D1, n3.D2)).  The vertex differences in
// FP64 (two independent subtractions), split from their bit fields into
// FP32 pairs, the rest in double-FP32 arithmetic: a dependent FP64
// instruction takes hundreds of cycles on this part, an FP32 one a few.
// Differences outside 2^-60 <= |d| < 2^60 (other than 0) take the same
// steps in FP64.
template <int P>
__device__ __forceinline__ void bwd_elem_setup_f32(BwdShared<true> &sm, int lane) {
  constexpr int NZ = P + 1;
  const double x = lane < 18 ? sm.X[lane] : 0.0;
  const int v = lane < 21 ? lane / 3 : 0, kv = lane < 21 ? lane % 3 : 0;
  // vertices (a, b, c, d) of vector v, 3 bits each, 12 bits per vector:
  //   A1 (1,0,4,3)  B1 (4,3,1,0)  A2 (2,0,5,3)  B2 (5,3,2,0)
  //   C  (3,0,0,0)  D1 (4,1,3,0)  D2 (5,2,3,0)
  // each (X_a - X_b) +- (X_c - X_d), halved
  constexpr unsigned long long kTab =
      (0x223ull << 0) | (0x8C8ull << 12) | (0x42Bull << 24) | (0xAD0ull << 36) | (0x600ull << 48);
  constexpr unsigned long long kTab2 = (0x858ull << 0) | (0xA98ull << 12);  // D1, D2
  constexpr unsigned kNeg = 0x6Au;  // B1, B2, D1, D2 subtract
  const unsigned tv = (unsigned)((v < 5 ? kTab >> (12 * v) : kTab2 >> (12 * (v - 5))) & 0xFFFu);
  const int la = 3 * ((tv >> 9) & 7u) + kv, lb = 3 * ((tv >> 6) & 7u) + kv;
  const int lc = 3 * ((tv >> 3) & 7u) + kv, ld = 3 * (tv & 7u) + kv;
  const bool subtract = (kNeg >> v) & 1u;
  const bool act = lane < 3 * NZ;
  const int iz = act ? lane / 3 : 0, k = act ? lane % 3 : 0;
  const int g0 = lane - k, l1 = g0 + (k + 1) % 3, l2 = g0 + (k + 2) % 3;
  const double xa = __shfl_sync(0xffffffffu, x, la), xb = __shfl_sync(0xffffffffu, x, lb);
  const double xc = __shfl_sync(0xffffffffu, x, lc), xd = __shfl_sync(0xffffffffu, x, ld);
  const double t1 = xa - xb, t2 = xc - xd;
  bool r1 = true, r2 = true;
  const float2 t1s = split_f64_bits(t1, &r1), t2s = split_f64_bits(t2, &r2);
  float evf;
  if (__all_sync(0xffffffffu, lane >= 21 || (r1 && r2))) {
    auto shfl2 = [](float2 q, int src) {
      return make_float2(__shfl_sync(0xffffffffu, q.x, src), __shfl_sync(0xffffffffu, q.y, src));
    };
    float2 ev = norm_ff(add_ff(t1s, subtract ? neg_ff(t2s) : t2s));
    ev = make_float2(0.5f * ev.x, 0.5f * ev.y);
    evf = ev.x;
    const float2 z2 = sm.ztab2[iz][0], wz2 = sm.ztab2[iz][1];
    const float2 c1 = norm_ff(add_ff(shfl2(ev, k), mul_ff(z2, shfl2(ev, 3 + k))));
    const float2 c2 = norm_ff(add_ff(shfl2(ev, 6 + k), mul_ff(z2, shfl2(ev, 9 + k))));
    const float2 c1a = shfl2(c1, l1), c1b = shfl2(c1, l2), c2a = shfl2(c2, l1), c2b = shfl2(c2, l2);
    const float2 n3 = norm_ff(add_ff(mul_ff(c1a, c2b), neg_ff(mul_ff(c1b, c2a))));
    float2 ab = mul_ff(n3, shfl2(ev, 12 + k));
    float2 bb = mul_ff(n3, shfl2(ev, 15 + k));
    float2 gb = mul_ff(n3, shfl2(ev, 18 + k));
    ab = norm_ff(add_ff(ab, add_ff(shfl2(ab, l1), shfl2(ab, l2))));
    bb = norm_ff(add_ff(bb, add_ff(shfl2(bb, l1), shfl2(bb, l2))));
    gb = norm_ff(add_ff(gb, add_ff(shfl2(gb, l1), shfl2(gb, l2))));
    if (lane < 21) sm.ev2[lane] = ev;
    if (act) {
      const float2 sk = k == 0 ? ab : k == 1 ? bb : gb;
      sm.zsum[iz][k] = sk;
      sm.zabg[iz][k] = norm_ff(mul_ff(wz2, sk));
      sm.zc1f[iz][k] = c1.x;
      sm.zc2f[iz][k] = c2.x;
      sm.zn3f[iz][k] = n3.x;
    }
  } else {
    const double ev = 0.5 * (subtract ? t1 - t2 : t1 + t2);
    evf = (float)ev;
    const double z = sm.zz[iz], wz = sm.zw[iz];
    const double c1 = fma(z, __shfl_sync(0xffffffffu, ev, 3 + k), __shfl_sync(0xffffffffu, ev, k));
    const double c2 = fma(z, __shfl_sync(0xffffffffu, ev, 9 + k), __shfl_sync(0xffffffffu, ev, 6 + k));
    const double c1a = __shfl_sync(0xffffffffu, c1, l1), c1b = __shfl_sync(0xffffffffu, c1, l2);
    const double c2a = __shfl_sync(0xffffffffu, c2, l1), c2b = __shfl_sync(0xffffffffu, c2, l2);
    const double n3 = c1a * c2b - c1b * c2a;
    double ab = n3 * __shfl_sync(0xffffffffu, ev, 12 + k);
    double bb = n3 * __shfl_sync(0xffffffffu, ev, 15 + k);
    double gb = n3 * __shfl_sync(0xffffffffu, ev, 18 + k);
    ab += __shfl_sync(0xffffffffu, ab, l1) + __shfl_sync(0xffffffffu, ab, l2);
    bb += __shfl_sync(0xffffffffu, bb, l1) + __shfl_sync(0xffffffffu, bb, l2);
    gb += __shfl_sync(0xffffffffu, gb, l1) + __shfl_sync(0xffffffffu, gb, l2);
    if (lane < 21) sm.ev2[lane] = split_f64(ev);
    if (act) {
      const double sk = k == 0 ? ab : k == 1 ? bb : gb;
      sm.zsum[iz][k] = split_f64(sk);
      sm.zabg[iz][k] = split_f64(wz * sk);
      sm.zc1f[iz][k] = (float)c1;
      sm.zc2f[iz][k] = (float)c2;
      sm.zn3f[iz][k] = (float)n3;
    }
  }
  if (lane < 21) sm.evf[lane] = evf;
}

__device__ __forceinline__ bool load_coef_b(const BwdArgs &a, int64_t r, double *cd) {
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    cd[k] = a.K[9 * r + k];
    ok &= finite64(cd[k]);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    cd[9 + k] = a.b[3 * r + k];
    ok &= finite64(cd[9 + k]);
  }
  cd[12] = a.c[r];
  cd[13] = a.f[r];
  ok &= finite64(cd[12]) && finite64(cd[13]);
  return ok;
}

// An FP32 value as FP64, exactly, by moving its fields (normal numbers;
// zero, subnormals, infinities and NaN through the conversion instruction):
// integer work instead of this part's slow FP64 pipe.
__device__ __forceinline__ double f32_to_f64(float x) {
  const uint32_t u = __float_as_uint(x), ex = (u >> 23) & 0xffu;
  if (ex == 0u || ex == 0xffu) return (double)x;
  const uint32_t hi = (u & 0x80000000u) | ((ex + 896u) << 20) | ((u & 0x7fffffu) >> 3);
  return __hiloint2double((int)hi, (int)((u & 7u) << 29));
}
// (s, e) with s + e = a + b exactly (Knuth's two-sum), FP32.
__device__ __forceinline__ float2 two_sum_f(float a, float b) {
  const float s = a + b, bb = s - a;
  return make_float2(s, (a - (s - bb)) + (b - bb));
}
// x + y for unevaluated FP32 pairs (hi, lo), normalised.
__device__ __forceinline__ float2 add_pair_f(float2 x, float2 y) {
  const float2 s = two_sum_f(x.x, y.x);
  const float lo = s.y + x.y + y.y;
  const float hi = s.x + lo;
  return make_float2(hi, lo - (hi - s.x));
}

// The chain of the FP32 adjoint to the coefficients and the vertices, one
// thread per point (two at p >= 6), from dL/dDt (gD) and dL/d(w det J f)
// (gsf) of every point.  det J and w det J come from the FP64 node columns;
// the rest runs in FP32 (the contraction that produced gD is FP32 too).
// The sums over points of the 21 element-vector and 14 coefficient
// gradients: each thread adds its points' terms in FP32, then the 256
// partial sums of each value are added as unevaluated FP32 pairs
// (two-sum, 2^-44 relative), in a fixed order, and stored in sm as FP64.
template <int P>
__device__ __forceinline__ void chain_f32(const BwdArgs &a, BwdShared<true> &sm, const float *gD, const float *gsf,
                                          int64_t qoff, float *red) {
  constexpr int NQ = nq_of(P), NT = (P + 1) * (P + 1);
  const int tid = threadIdx.x;
  float acc[35];
#pragma unroll
  for (int k = 0; k < 35; ++k) acc[k] = 0.f;
  int pst = 0;
  const bool perq = a.coef_mode == FEI_COEF_PER_POINT;
  for (int q = tid; q < NQ; q += 256) {
    const int iz = q / NT, t = q - iz * NT;
    // w det J = w_t (a + xi1 b + xi2 g) from the node sums in double-FP32,
    // rounded once
    const float2 wp = mul_ff(sm.ztab2[iz][1], sm.ttab2[t][0]);
    const float w = wp.x + wp.y;
    const float2 sd = add_ff(add_ff(mul_ff(sm.ttab2[t][0], sm.zabg[iz][0]), mul_ff(sm.ttab2[t][1], sm.zabg[iz][1])),
                             mul_ff(sm.ttab2[t][2], sm.zabg[iz][2]));
    const float s = sd.x + sd.y;
    // det J = a + xi1 b + xi2 g from the node sums, rounded once
    const float2 dd = add_ff(add_ff(sm.zsum[iz][0], mul_ff(sm.txi2[t][0], sm.zsum[iz][1])),
                             mul_ff(sm.txi2[t][1], sm.zsum[iz][2]));
    const float det = dd.x + dd.y;
    pst = merge_status(pst, point_status_f(s));
    // coefficients in FP32 (converted from the bit fields)
    float cf[14];
    if (perq) {
      double cq[14];
      if (!load_coef_b(a, qoff + q, cq)) pst = FEI_ERR_NONFINITE;
#pragma unroll
      for (int k = 0; k < 14; ++k) cf[k] = f64_to_f32_bits(cq[k]);
    } else {
#pragma unroll
      for (int k = 0; k < 14; ++k) cf[k] = sm.cdf[k];
    }
    float K[9], bvec[3];
#pragma unroll
    for (int k = 0; k < 9; ++k) K[k] = cf[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) bvec[k] = cf[9 + k];
    const float cc = cf[12], ff = cf[13];
    float adj[3][3], cx1[3], cx2[3], cx3[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      cx1[k] = sm.zc1f[iz][k];
      cx2[k] = sm.zc2f[iz][k];
      cx3[k] = sm.tc3f[t][k];
      adj[2][k] = sm.zn3f[iz][k];
    }
    cross3(cx2, cx3, adj[0]);
    cross3(cx3, cx1, adj[1]);
    const float gD00 = gD[q * 16 + 0];
    float gD0[3], gDm[3][3];
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      gD0[l] = gD[q * 16 + 1 + l];
#pragma unroll
      for (int m = 0; m < 3; ++m) gDm[l][m] = gD[q * 16 + 4 * (l + 1) + (m + 1)];
    }
    const float gs = gsf[q];
    const float wd = w / det, wdd = wd / det;
    float Ka[3][3], Kta[3][3];
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        Ka[m][r] = K[3 * r] * adj[m][0] + K[3 * r + 1] * adj[m][1] + K[3 * r + 2] * adj[m][2];
        Kta[m][r] = K[r] * adj[m][0] + K[3 + r] * adj[m][1] + K[6 + r] * adj[m][2];
      }
    float U[3][3], V[3][3], Tm[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        U[r][k] = gDm[r][0] * Ka[0][k] + gDm[r][1] * Ka[1][k] + gDm[r][2] * Ka[2][k];
        V[r][k] = gDm[0][r] * Kta[0][k] + gDm[1][r] * Kta[1][k] + gDm[2][r] * Kta[2][k];
        Tm[r][k] = gDm[r][0] * adj[0][k] + gDm[r][1] * adj[1][k] + gDm[r][2] * adj[2][k];
      }
    // coefficient gradients at this point: dL/dK = (w / det) adj^T gDm adj,
    // dL/db = w adj^T gD0, dL/dc = w det gD00, dL/df = w det gs
    float gco[14];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        gco[3 * r + c] = wd * (adj[0][r] * Tm[0][c] + adj[1][r] * Tm[1][c] + adj[2][r] * Tm[2][c]);
#pragma unroll
    for (int k = 0; k < 3; ++k) gco[9 + k] = w * (gD0[0] * adj[0][k] + gD0[1] * adj[1][k] + gD0[2] * adj[2][k]);
    gco[12] = s * gD00;
    gco[13] = s * gs;
    if (perq) {
      const int64_t r = qoff + q;
#pragma unroll
      for (int k = 0; k < 9; ++k) a.gK[9 * r + k] = f32_to_f64(gco[k]);
#pragma unroll
      for (int k = 0; k < 3; ++k) a.gbc[3 * r + k] = f32_to_f64(gco[9 + k]);
      a.gc[r] = f32_to_f64(gco[12]);
      a.gf[r] = f32_to_f64(gco[13]);
    } else {
#pragma unroll
      for (int k = 0; k < 14; ++k) acc[21 + k] += gco[k];
    }
    // through det J and the adjugate rows: with the quadratic form
    // sum_lm gDm[l][m] adj_l K adj_m^T = sum_{l,r} adj[l][r] U[l][r]
    float quad = 0.f;
#pragma unroll
    for (int l = 0; l < 3; ++l) quad += adj[l][0] * U[l][0] + adj[l][1] * U[l][1] + adj[l][2] * U[l][2];
    const float gdet = w * (cc * gD00 + ff * gs) - wdd * quad;
    float gadj[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int k = 0; k < 3; ++k) gadj[r][k] = w * gD0[r] * bvec[k] + wd * (U[r][k] + V[r][k]);
    float gc1[3] = {0, 0, 0}, gc2[3] = {0, 0, 0}, gc3[3], tmp[3], gn3[3];
    cross3(cx3, gadj[0], gc2);  // adj0 = c2 x c3
    cross3(gadj[0], cx2, gc3);
    cross3(cx1, gadj[1], tmp);  // adj1 = c3 x c1
#pragma unroll
    for (int k = 0; k < 3; ++k) gc3[k] += tmp[k];
    cross3(gadj[1], cx3, gc1);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      gn3[k] = gadj[2][k] + gdet * cx3[k];  // adj2 = n3, det = n3 . c3
      gc3[k] += gdet * adj[2][k];
    }
    cross3(cx2, gn3, tmp);  // n3 = c1 x c2
#pragma unroll
    for (int k = 0; k < 3; ++k) gc1[k] += tmp[k];
    cross3(gn3, cx1, tmp);
#pragma unroll
    for (int k = 0; k < 3; ++k) gc2[k] += tmp[k];
    const float z = sm.ztabf[iz][0], x1 = sm.ttabf[t][1], x2 = sm.ttabf[t][2];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      acc[0 + k] += gc1[k];
      acc[3 + k] += z * gc1[k];
      acc[6 + k] += gc2[k];
      acc[9 + k] += z * gc2[k];
      acc[12 + k] += gc3[k];
      acc[15 + k] += x1 * gc3[k];
      acc[18 + k] += x2 * gc3[k];
    }
  }
  if (pst) atomicMax(&sm.status, pst);
  __syncthreads();  // every point's dL/dDt has been read: the area is free
  // red [35][256]: each thread's partial sums
#pragma unroll
  for (int k = 0; k < 35; ++k) red[k * 256 + tid] = acc[k];
  __syncthreads();
  // value k = pass * 32 + tid / 8: eight lanes add 32 partials each as
  // FP32 pairs, then combine across the eight lanes (fixed order)
  const int nval = a.coef_mode == FEI_COEF_PER_ELEMENT ? 35 : 21;
  for (int pass = 0; pass < 2; ++pass) {
    const int k = pass * 32 + (tid >> 3), sub = tid & 7;
    float2 v = make_float2(0.f, 0.f);
    if (k < nval) {
      for (int j = 0; j < 32; ++j) v = add_pair_f(v, make_float2(red[k * 256 + sub + 8 * j], 0.f));
    }
#pragma unroll
    for (int off = 4; off >= 1; off >>= 1) {
      const float2 o = make_float2(__shfl_xor_sync(0xffffffffu, v.x, off), __shfl_xor_sync(0xffffffffu, v.y, off));
      v = add_pair_f(v, o);
    }
    if (k < nval && sub == 0) {
      const double d = f32_to_f64(v.x) + f32_to_f64(v.y);
      if (k < 21) {
        sm.gev[k] = d;
        sm.gev2[k] = v;
      } else {
        sm.gcoef[k - 21] = d;
      }
    }
  }
  __syncthreads();
}

template <typename T, int P, bool Q>
__global__ void __launch_bounds__(256, 2) cc_backward_kernel(BwdArgs a) {
  using C = BwdCfg<T, P, Q>;
  constexpr int NSH = C::NSH, NQ = C::NQ, NT = C::NT, BI = C::BI, QC = C::QC, KC = C::KC, NSHP = C::NSHP;
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ BwdShared<C::F32> sm;
  T *gAs = reinterpret_cast<T *>(dsm + C::OFF_GA);
  T *Gc = reinterpret_cast<T *>(dsm + C::OFF_GC);
  T *Wc = reinterpret_cast<T *>(dsm + C::OFF_W);
  T *gD = reinterpret_cast<T *>(dsm + C::OFF_GD);
  T *gsf = reinterpret_cast<T *>(dsm + C::OFF_GSF);
  const int tid = threadIdx.x;
  const T *Gg = gtab_b<T>(a);
  const T *gAg = reinterpret_cast<const T *>(a.gA);
  const T *gbg = reinterpret_cast<const T *>(a.gb);
  const int64_t items = a.count ? (int64_t)(*a.count) : a.n_work;
  // node tables of the degree, once per block (FP64 node data; the FP32
  // path's FP32 copies and pairs)
  for (int t = tid; t < NT; t += 256) {
    const double x1 = a.tnode[4 * t], x2 = a.tnode[4 * t + 1], wt = a.tnode[4 * t + 2];
    sm.txi[t][0] = x1;
    sm.txi[t][1] = x2;
    sm.tw[t] = wt;
    if constexpr (C::F32) {
      sm.ttab2[t][0] = split_f64(wt);
      sm.ttab2[t][1] = split_f64(wt * x1);
      sm.ttab2[t][2] = split_f64(wt * x2);
      sm.txi2[t][0] = split_f64(x1);
      sm.txi2[t][1] = split_f64(x2);
      sm.ttabf[t][0] = (float)wt;
      sm.ttabf[t][1] = (float)x1;
      sm.ttabf[t][2] = (float)x2;
    }
  }
  for (int z = tid; z < C::NZ; z += 256) {
    const double zz = a.znode[2 * z], zw = a.znode[2 * z + 1];
    sm.zz[z] = zz;
    sm.zw[z] = zw;
    if constexpr (C::F32) {
      sm.ztab2[z][0] = split_f64(zz);
      sm.ztab2[z][1] = split_f64(zw);
      sm.ztabf[z][0] = (float)zz;
      sm.ztabf[z][1] = (float)zw;
    }
  }
  __syncthreads();

  for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
    const int64_t e = a.list ? (int64_t)a.list[item] : a.e0 + item;
    const int64_t aoff = a.A_off ? a.A_off[e] : e * (int64_t)(NSH * NSH);
    const int64_t boff = a.b_off ? a.b_off[e] : e * (int64_t)NSH;
    const int64_t qoff = a.q_off ? a.q_off[e] : e * (int64_t)NQ;
    if (tid == 0) sm.status = 0;
    if (tid < 21) sm.gev[tid] = 0.0;
    if (tid >= 32 && tid < 46) sm.gcoef[tid - 32] = 0.0;
    __syncthreads();
    bool ok = true;
    if (tid < 18) {
      sm.X[tid] = a.geom[18 * e + tid];
      ok = finite64(sm.X[tid]);
    }
    if (a.coef_mode == FEI_COEF_PER_ELEMENT && tid == 32) ok = load_coef_b(a, e, sm.cd);
    if (!ok) sm.status = FEI_ERR_NONFINITE;
    __syncthreads();
    if constexpr (C::F32) {
      // element vectors and vertical-node data (warp 0, double-FP32), the
      // per-element coefficients in FP32; then the triangle-node columns
      // c3 = C + xi1 D1 + xi2 D2 in double-FP32, rounded once
      if (tid < 32) bwd_elem_setup_f32<P>(sm, tid);
      else if (tid < 46 && a.coef_mode == FEI_COEF_PER_ELEMENT) sm.cdf[tid - 32] = f64_to_f32_bits(sm.cd[tid - 32]);
      __syncthreads();
      for (int j = tid; j < 3 * NT; j += 256) {
        const int t = j / 3, k = j - 3 * t;
        const float2 c3 = add_ff(add_ff(sm.ev2[12 + k], mul_ff(sm.txi2[t][0], sm.ev2[15 + k])),
                                 mul_ff(sm.txi2[t][1], sm.ev2[18 + k]));
        sm.tc3f[t][k] = c3.x + c3.y;
      }
    } else {
      if (tid == 0) elem_vectors(sm.X, sm.ev);
      __syncthreads();
      if (tid < C::NZ) {
        znode_columns(sm.ev, sm.zz[tid], sm.zc1[tid], sm.zc2[tid], sm.zn3[tid]);
      } else if (tid >= 32 && tid < 32 + NT) {
        const int t = tid - 32;
        tnode_column(sm.ev, sm.txi[t][0], sm.txi[t][1], sm.tc3[t]);
      }
    }
    if constexpr (Q) {
      // L_e = u^T A_e u - u^T b_e: with v_q = G_q u (4 values per point),
      // dL/dDt_q = v_q v_q^T and dL/d(w det f)_q = -v_q[0] (row 0 of G_q
      // is phi), so gA = u u^T is never formed.  One warp per point.
      T *us = gAs;
      for (int i = tid; i < NSH; i += 256) {
        if constexpr (C::F32) us[i] = f64_to_f32_bits(a.u[boff + i]);
        else us[i] = a.u[boff + i];
      }
      __syncthreads();
      const int warp = tid >> 5, lane = tid & 31;
      constexpr int NI = (NSH + 31) / 32;  // table entries per lane and row
      T ul[NI];
#pragma unroll
      for (int k = 0; k < NI; ++k) ul[k] = lane + 32 * k < NSH ? us[lane + 32 * k] : T(0);
      for (int q = warp; q < NQ; q += 8) {
        // the four rows of G_q: every load issued before the first use
        T g[4][NI];
#pragma unroll
        for (int aa = 0; aa < 4; ++aa) {
          const T *row = Gg + (size_t)(4 * q + aa) * NSH;
#pragma unroll
          for (int k = 0; k < NI; ++k) g[aa][k] = lane + 32 * k < NSH ? row[lane + 32 * k] : T(0);
        }
        T v[4];
#pragma unroll
        for (int aa = 0; aa < 4; ++aa) {
          T s = T(0);
#pragma unroll
          for (int k = 0; k < NI; ++k) s += g[aa][k] * ul[k];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
          v[aa] = s;
        }
        if (lane < 16) gD[q * 16 + lane] = v[lane >> 2] * v[lane & 3];
        if (lane == 0) gsf[q] = -v[0];
      }
      __syncthreads();
    }
    if constexpr (!Q) {
    // zero the dL/dDt accumulators (or take them from the tensor-core
    // adjoint); dL/d(w det f) per point
    const bool pre = C::F32 && a.gDpre != nullptr;
    if (pre) {
      const float *src = a.gDpre + (size_t)item * NQ * 16;
      for (int k = tid; k < NQ * 16; k += 256) gD[k] = (T)src[k];
    } else {
      for (int k = tid; k < NQ * 16; k += 256) gD[k] = T(0);
    }
    for (int q = tid; q < NQ; q += 256) {
      T s = T(0);
      for (int i = 0; i < NSH; ++i) s += gbg[boff + i] * Gg[(size_t)(4 * q) * NSH + i];
      gsf[q] = s;
    }
    __syncthreads();

    // dL/dDt_q = G_q gA G_q^T, row block by row block
    for (int r0 = 0; r0 < (pre ? 0 : NSH); r0 += BI) {
      for (int k = tid; k < BI * NSHP; k += 256) {
        const int ii = k / NSHP, j = k - ii * NSHP;
        gAs[k] = (r0 + ii < NSH && j < NSH) ? gAg[aoff + (int64_t)(r0 + ii) * NSH + j] : T(0);
      }
      for (int q0 = 0; q0 < NQ; q0 += QC) {
        for (int k = tid; k < KC * NSHP; k += 256) {
          const int kk = k / NSHP, j = k - kk * NSHP;
          const int q = q0 + kk / 4;
          Gc[k] = (q < NQ && j < NSH) ? Gg[(size_t)(4 * q0 + kk) * NSH + j] : T(0);
        }
        __syncthreads();
        // W[ii][kk] = sum_j gA[r0+ii][j] G[(q0,kk)][j]; thread (ty, tx) owns
        // rows ty + 16 r and columns tx + 16 c (r < TM, c < TN)
        {
          const int ty = tid >> 4, tx = tid & 15;
          T acc[C::TM][C::TN];
#pragma unroll
          for (int r = 0; r < C::TM; ++r)
#pragma unroll
            for (int c = 0; c < C::TN; ++c) acc[r][c] = T(0);
          if constexpr (C::F32) {
#pragma unroll 2
            for (int j = 0; j < NSHP; j += 4) {
              float4 av[C::TM], bv[C::TN];
#pragma unroll
              for (int r = 0; r < C::TM; ++r) av[r] = *reinterpret_cast<const float4 *>(&gAs[(ty + 16 * r) * NSHP + j]);
#pragma unroll
              for (int c = 0; c < C::TN; ++c) bv[c] = *reinterpret_cast<const float4 *>(&Gc[(tx + 16 * c) * NSHP + j]);
#pragma unroll
              for (int r = 0; r < C::TM; ++r)
#pragma unroll
                for (int c = 0; c < C::TN; ++c) {
                  acc[r][c] = fmaf(av[r].x, bv[c].x, acc[r][c]);
                  acc[r][c] = fmaf(av[r].y, bv[c].y, acc[r][c]);
                  acc[r][c] = fmaf(av[r].z, bv[c].z, acc[r][c]);
                  acc[r][c] = fmaf(av[r].w, bv[c].w, acc[r][c]);
                }
            }
          } else {
#pragma unroll 4
            for (int j = 0; j < NSH; ++j) {
              T av[C::TM], bv[C::TN];
#pragma unroll
              for (int r = 0; r < C::TM; ++r) av[r] = gAs[(ty + 16 * r) * NSHP + j];
#pragma unroll
              for (int c = 0; c < C::TN; ++c) bv[c] = Gc[(tx + 16 * c) * NSHP + j];
#pragma unroll
              for (int r = 0; r < C::TM; ++r)
#pragma unroll
                for (int c = 0; c < C::TN; ++c) acc[r][c] += av[r] * bv[c];
            }
          }
#pragma unroll
          for (int r = 0; r < C::TM; ++r)
#pragma unroll
            for (int c = 0; c < C::TN; ++c) Wc[(ty + 16 * r) * KC + tx + 16 * c] = acc[r][c];
        }
        __syncthreads();
        // gD[q][a][b] += sum_ii G[q][a][r0+ii] W[ii][(q,b)]
        for (int task = tid; task < QC * 16; task += 256) {
          const int qq = task >> 4, ab = task & 15, aa = ab >> 2, bb = ab & 3;
          const int q = q0 + qq;
          if (q < NQ) {
            T sacc = T(0);
            const int lim = (NSH - r0 < BI) ? NSH - r0 : BI;
            for (int ii = 0; ii < lim; ++ii) sacc += Gc[(4 * qq + aa) * NSHP + r0 + ii] * Wc[ii * KC + 4 * qq + bb];
            gD[q * 16 + ab] += sacc;
          }
        }
        __syncthreads();
      }
    }

    }  // !Q

    if constexpr (C::F32) {
      chain_f32<P>(a, sm, gD, gsf, qoff, reinterpret_cast<float *>(dsm));
    } else {
    // The chain to the coefficients and the vertices, one thread per point.
    // det J, w det J, w / det J and the sums over points are FP64; the 3 x 3
    // products that carry dL/dDt through the adjugate run in the contraction's
    // type CT (FP64 for FEI_FP64, FP32 for FEI_FP32, whose dL/dDt is FP32 already)
    using CT = T;
    double gev[21];
#pragma unroll
    for (int k = 0; k < 21; ++k) gev[k] = 0.0;
    double gco[14];
#pragma unroll
    for (int k = 0; k < 14; ++k) gco[k] = 0.0;
    int pst = 0;
    for (int q = tid; q < NQ; q += 256) {
      const int iz = q / NT, t = q - iz * NT;
      const double *c1 = sm.zc1[iz], *c2 = sm.zc2[iz], *n3 = sm.zn3[iz], *c3 = sm.tc3[t];
      const double w = sm.zw[iz] * sm.tw[t];
      const double det = dot3(n3, c3);
      pst = merge_status(pst, point_status(w * det));
      double cq[14];
      const double *cp = sm.cd;
      if (a.coef_mode == FEI_COEF_PER_POINT) {
        if (!load_coef_b(a, qoff + q, cq)) pst = FEI_ERR_NONFINITE;
        cp = cq;
      }
      CT K[9], bvec[3];
#pragma unroll
      for (int k = 0; k < 9; ++k) K[k] = (CT)cp[k];
#pragma unroll
      for (int k = 0; k < 3; ++k) bvec[k] = (CT)cp[9 + k];
      const double cc = cp[12], ff = cp[13];
      CT adj[3][3], cx1[3], cx2[3], cx3[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        cx1[k] = (CT)c1[k];
        cx2[k] = (CT)c2[k];
        cx3[k] = (CT)c3[k];
        adj[2][k] = (CT)n3[k];
      }
      cross3(cx2, cx3, adj[0]);
      cross3(cx3, cx1, adj[1]);
      const double gD00 = (double)gD[q * 16 + 0];
      CT gD0[3], gDm[3][3];
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        gD0[l] = gD[q * 16 + 1 + l];
#pragma unroll
        for (int m = 0; m < 3; ++m) gDm[l][m] = gD[q * 16 + 4 * (l + 1) + (m + 1)];
      }
      const double gs = (double)gsf[q];
      const double s = w * det, wd = w / det;
      const CT wc = (CT)w, wdc = (CT)wd;
      // K adj_m^T and K^T adj_m per adjugate row m, and the products
      // U = gDm Ka, V = gDm^T Kta, T = gDm adj (3 x 3 each)
      CT Ka[3][3], Kta[3][3];
#pragma unroll
      for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          Ka[m][r] = K[3 * r] * adj[m][0] + K[3 * r + 1] * adj[m][1] + K[3 * r + 2] * adj[m][2];
          Kta[m][r] = K[r] * adj[m][0] + K[3 + r] * adj[m][1] + K[6 + r] * adj[m][2];
        }
      CT U[3][3], V[3][3], Tm[3][3];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          U[r][k] = gDm[r][0] * Ka[0][k] + gDm[r][1] * Ka[1][k] + gDm[r][2] * Ka[2][k];
          V[r][k] = gDm[0][r] * Kta[0][k] + gDm[1][r] * Kta[1][k] + gDm[2][r] * Kta[2][k];
          Tm[r][k] = gDm[r][0] * adj[0][k] + gDm[r][1] * adj[1][k] + gDm[r][2] * adj[2][k];
        }
      // coefficient gradients at this point: dL/dK = (w / det) adj^T gDm adj,
      // dL/db = w adj^T gD0, dL/dc = w det gD00, dL/df = w det gs
      CT gKq[9], gbq[3];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          gKq[3 * r + c] = wdc * (adj[0][r] * Tm[0][c] + adj[1][r] * Tm[1][c] + adj[2][r] * Tm[2][c]);
#pragma unroll
      for (int k = 0; k < 3; ++k) gbq[k] = wc * (gD0[0] * adj[0][k] + gD0[1] * adj[1][k] + gD0[2] * adj[2][k]);
      const double gcq = s * gD00, gfq = s * gs;
      if (a.coef_mode == FEI_COEF_PER_POINT) {
        const int64_t r = qoff + q;
#pragma unroll
        for (int k = 0; k < 9; ++k) a.gK[9 * r + k] = gKq[k];
#pragma unroll
        for (int k = 0; k < 3; ++k) a.gbc[3 * r + k] = gbq[k];
        a.gc[r] = gcq;
        a.gf[r] = gfq;
      } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) gco[k] += gKq[k];
#pragma unroll
        for (int k = 0; k < 3; ++k) gco[9 + k] += gbq[k];
        gco[12] += gcq;
        gco[13] += gfq;
      }
      // through det J and the adjugate rows: with the quadratic form
      // sum_lm gDm[l][m] adj_l K adj_m^T = sum_{l,r} adj[l][r] U[l][r]
      CT quad = CT(0);
#pragma unroll
      for (int l = 0; l < 3; ++l) quad += adj[l][0] * U[l][0] + adj[l][1] * U[l][1] + adj[l][2] * U[l][2];
      const double gdet = w * (cc * gD00 + ff * gs) - wd / det * (double)quad;
      const CT gdetc = (CT)gdet;
      CT gadj[3][3];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) gadj[r][k] = wc * gD0[r] * bvec[k] + wdc * (U[r][k] + V[r][k]);
      CT gc1[3] = {0, 0, 0}, gc2[3] = {0, 0, 0}, gc3[3], tmp[3], gn3[3];
      cross3(cx3, gadj[0], gc2);   // adj0 = c2 x c3
      cross3(gadj[0], cx2, gc3);
      cross3(cx1, gadj[1], tmp);   // adj1 = c3 x c1
#pragma unroll
      for (int k = 0; k < 3; ++k) gc3[k] += tmp[k];
      cross3(gadj[1], cx3, gc1);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        gn3[k] = gadj[2][k] + gdetc * cx3[k];  // adj2 = n3, det = n3 . c3
        gc3[k] += gdetc * adj[2][k];
      }
      cross3(cx2, gn3, tmp);       // n3 = c1 x c2
#pragma unroll
      for (int k = 0; k < 3; ++k) gc1[k] += tmp[k];
      cross3(gn3, cx1, tmp);
#pragma unroll
      for (int k = 0; k < 3; ++k) gc2[k] += tmp[k];
      const double z = sm.zz[iz], x1 = sm.txi[t][0], x2 = sm.txi[t][1];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        gev[0 + k] += gc1[k];
        gev[3 + k] += z * gc1[k];
        gev[6 + k] += gc2[k];
        gev[9 + k] += z * gc2[k];
        gev[12 + k] += gc3[k];
        gev[15 + k] += x1 * gc3[k];
        gev[18 + k] += x2 * gc3[k];
      }
    }
    if (pst) atomicMax(&sm.status, pst);
    // sums over the points: every lane stores its 35 partial sums, then lane
    // k of the warp adds up value k over the 32 lanes (a 32-term FP64 sum per
    // value, instead of a 5-level shuffle tree for each of the 35 values)
    __syncthreads();  // every point's dL/dDt has been read: the area is free
    {
      const int lane = tid & 31;
      double *red = reinterpret_cast<double *>(dsm) + (tid >> 5) * (35 * 33);
#pragma unroll
      for (int k = 0; k < 21; ++k) red[k * 33 + lane] = gev[k];
#pragma unroll
      for (int k = 0; k < 14; ++k) red[(21 + k) * 33 + lane] = gco[k];
      __syncwarp();
      for (int k = lane; k < 35; k += 32) {
        if (k >= 21 && a.coef_mode != FEI_COEF_PER_ELEMENT) continue;
        double v = 0.0;
#pragma unroll 8
        for (int l = 0; l < 32; ++l) v += red[k * 33 + l];
        red[k * 33 + 32] = v;  // this warp's sum, in the row's spare slot
      }
    }
    __syncthreads();
    // the warps' sums added in warp order: a fixed order, so the gradients
    // are the same bit for bit from run to run
    if (tid < 35 && (tid < 21 || a.coef_mode == FEI_COEF_PER_ELEMENT)) {
      const double *red0 = reinterpret_cast<const double *>(dsm);
      double v = 0.0;
#pragma unroll
      for (int w = 0; w < 256 / 32; ++w) v += red0[w * (35 * 33) + tid * 33 + 32];
      if (tid < 21) sm.gev[tid] = v;
      else sm.gcoef[tid - 21] = v;
    }
    __syncthreads();
    }
    const int st = sm.status;
    // element vectors -> vertices (transpose of elem_vectors)
    if constexpr (C::F32) {
     if (tid < 18) {
      // vertex component (vertex tid / 3, coordinate tid % 3) from the
      // element-vector gradients as FP32 pairs: signed sums of up to 7
      // terms (rows of the transpose), halved
      const int vx = tid / 3, k = tid - 3 * vx;
      // signs of (A1, B1, A2, B2, C, D1, D2) for P0, P1, P2, Q0, Q1, Q2,
      // two bits each (0: none, 1: +, 2: -)
      const unsigned sg = vx == 0 ? 0x1666u : vx == 1 ? 0x809u : vx == 2 ? 0x2090u : vx == 3 ? 0x29AAu
                          : vx == 4 ? 0x405u : 0x1050u;
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int c = 0; c < 7; ++c) {
        const unsigned b = (sg >> (2 * c)) & 3u;
        if (b) {
          const float2 g = sm.gev2[3 * c + k];
          acc = add_pair_f(acc, b == 1u ? g : make_float2(-g.x, -g.y));
        }
      }
      const double val = 0.5 * (f32_to_f64(acc.x) + f32_to_f64(acc.y));
      a.g_geom[18 * e + 3 * vx + k] = st ? 0.0 : val;
     }
    } else if (tid < 3) {
      const int k = tid;
      const double *g = sm.gev;
      const double gA1 = g[0 + k], gB1 = g[3 + k], gA2 = g[6 + k], gB2 = g[9 + k];
      const double gC = g[12 + k], gD1 = g[15 + k], gD2 = g[18 + k];
      double gP0 = 0.5 * (-gA1 + gB1 - gA2 + gB2 - gC + gD1 + gD2);
      double gQ0 = 0.5 * (-gA1 - gB1 - gA2 - gB2 + gC - gD1 - gD2);
      double gP1 = 0.5 * (gA1 - gB1 - gD1);
      double gQ1 = 0.5 * (gA1 + gB1 + gD1);
      double gP2 = 0.5 * (gA2 - gB2 - gD2);
      double gQ2 = 0.5 * (gA2 + gB2 + gD2);
      double *out = a.g_geom + 18 * e;
      out[0 + k] = st ? 0.0 : gP0;
      out[3 + k] = st ? 0.0 : gP1;
      out[6 + k] = st ? 0.0 : gP2;
      out[9 + k] = st ? 0.0 : gQ0;
      out[12 + k] = st ? 0.0 : gQ1;
      out[15 + k] = st ? 0.0 : gQ2;
    }
    if (a.coef_mode == FEI_COEF_PER_ELEMENT && tid >= 32 && tid < 46) {
      const int k = tid - 32;
      const double v = st ? 0.0 : sm.gcoef[k];
      if (k < 9) a.gK[9 * e + k] = v;
      else if (k < 12) a.gbc[3 * e + (k - 9)] = v;
      else if (k == 12) a.gc[e] = v;
      else a.gf[e] = v;
    }
    if (a.coef_mode == FEI_COEF_PER_POINT && st) {
      // flagged element: overwrite the per-point gradients with zeros
      for (int q = tid; q < NQ; q += 256) {
        const int64_t r = qoff + q;
        for (int k = 0; k < 9; ++k) a.gK[9 * r + k] = 0.0;
        for (int k = 0; k < 3; ++k) a.gbc[3 * r + k] = 0.0;
        a.gc[r] = 0.0;
        a.gf[r] = 0.0;
      }
    }
    __syncthreads();
  }
}

template <typename T, int P, bool Q>
fei_status launch_bwd(const BwdArgs &a, int64_t grid_work, cudaStream_t s) {
  using C = BwdCfg<T, P, Q>;
  static_assert(sizeof(BwdShared<C::F32>) + C::SMEM <= 232448, "shared memory of one block (227 KB)");
  FEI_CUDA_TRY(cudaFuncSetAttribute(cc_backward_kernel<T, P, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)C::SMEM),
               "cudaFuncSetAttribute(cc_backward)");
  int64_t blocks = grid_work;
  if (a.count) blocks = blocks < 152 * 4 ? blocks : 152 * 4;
  if (blocks > 2147483647LL) blocks = 2147483647LL;
  if (blocks < 1) blocks = 1;
  cc_backward_kernel<T, P, Q><<<(unsigned)blocks, 256, C::SMEM, s>>>(a);
  FEI_CUDA_TRY(cudaGetLastError(), "cc_backward_kernel launch");
  return FEI_OK;
}

template <typename T, bool Q>
fei_status launch_bwd_typed(int p, const BwdArgs &a, int64_t grid_work, cudaStream_t s) {
  switch (p) {
    case 1: return launch_bwd<T, 1, Q>(a, grid_work, s);
    case 2: return launch_bwd<T, 2, Q>(a, grid_work, s);
    case 3: return launch_bwd<T, 3, Q>(a, grid_work, s);
    case 4: return launch_bwd<T, 4, Q>(a, grid_work, s);
    case 5: return launch_bwd<T, 5, Q>(a, grid_work, s);
    case 6: return launch_bwd<T, 6, Q>(a, grid_work, s);
    case 7: return launch_bwd<T, 7, Q>(a, grid_work, s);
  }
  return set_error(FEI_ERR_INVALID_DEGREE, "degree %d outside 1..7", p);
}

}  // namespace

fei_status launch_cc_backward(int p, bool fp64, const BwdArgs &a, int64_t grid_work, cudaStream_t s,
                              bool quadratic) {
  if (grid_work <= 0) return FEI_OK;
  if (quadratic)
    return fp64 ? launch_bwd_typed<double, true>(p, a, grid_work, s)
                : launch_bwd_typed<float, true>(p, a, grid_work, s);
  return fp64 ? launch_bwd_typed<double, false>(p, a, grid_work, s)
              : launch_bwd_typed<float, false>(p, a, grid_work, s);
}

}  // namespace fei
