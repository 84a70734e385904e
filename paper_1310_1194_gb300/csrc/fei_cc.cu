// fei_cc.cu -- element integration on the CUDA cores (FP64 and FP32 paths).
//
// Algorithm 1 of the paper with its loop over points outside the loops over
// shape functions (Sec. 2.1), arranged for a GPU thread block:
//   * the element's geometry is read once (step 2) and its Jacobian columns
//     are formed once per vertical node and once per triangle node;
//   * the points are processed in chunks; per chunk the block forms the
//     point operators Dt_q (steps 7-8, fei_geom.cuh), then the operand
//     H'[q][b][i] = sum_a Dt_q[a][b] G[q][a][i] for its rows and stages the
//     reference table G[q][b][j] for its columns in shared memory;
//   * the double loop over shape functions (steps 9-13) becomes a
//     register-tiled contraction A[i][j] += sum_{q,b} H'[q][b][i] G[q][b][j]
//     over the 4 N_q dimension.
// For high p the element matrix is split into square blocks handled by
// separate thread blocks, the GPU counterpart of the paper's "parts" of the
// stiffness matrix (Sec. 4, Table 4): each block repeats the per-point work.
//
// FEI_FP64: everything in FP64.  FEI_FP32: the element vectors, the
// Jacobian columns at the nodes and w det J at every point in FP64; the
// adjugate rows, the point operator and the contraction in FP32.
#include <type_traits>

#include "fei_geom.cuh"
#include "fei_internal.cuh"

namespace fei {
namespace {

template <typename T>
__device__ __forceinline__ const T *gtab(const FwdArgs &a);
template <>
__device__ __forceinline__ const double *gtab<double>(const FwdArgs &a) { return a.G64; }
template <>
__device__ __forceinline__ const float *gtab<float>(const FwdArgs &a) { return a.G32; }

__device__ __forceinline__ int64_t n_items(const FwdArgs &a) {
  return a.count ? (int64_t)(*a.count) : a.n_work;
}

// Loads the 14 coefficient values of record r (K 9, b 3, c, f) and reports
// whether all are finite.
__device__ __forceinline__ bool load_coef(const FwdArgs &a, int64_t r, double *cd) {
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

// Point operator directly from the element vectors, FP64 (the FEI_FP64
// path at p <= 2).
__device__ __forceinline__ int point_direct64(const double *ev, const double *pt, const double *cd, double *D) {
  double c1[3], c2[3], n3[3], c3[3];
  znode_columns(ev, pt[2], c1, c2, n3);
  tnode_column(ev, pt[0], pt[1], c3);
  const double w = pt[3];
  const double det = dot3(n3, c3);
  const double s = w * det;
  double a0[3], a1[3];
  cross3(c2, c3, a0);
  cross3(c3, c1, a1);
  dt_from_adj<double>(a0, a1, n3, w, s, w / det, cd, cd + 9, cd[12], cd[13], D);
  return point_status(s);
}

// ---------------------------------------------------------------------------
// Low degree (p <= 2): EPW elements per warp (p = 1: four elements of 8
// points, p = 2: one of 27), so that every lane takes a point; lanes then
// run over the entries of the A_e.  The FP64 path forms each point's
// Jacobian in FP64.  The FP32 path keeps FP64 to what reading its inputs
// needs: the element vectors, and per vertical node the FP64 sums
// alpha, beta, gamma of det J = alpha + xi1 beta + xi2 gamma (split into
// FP32 pairs); each point's w det J is then formed in double-FP32
// arithmetic and rounded once, and the columns and adjugate are FP32.  At
// p = 1 that is about 200 FP64 instructions per element instead of about
// 500 with per-point FP64 columns (this part's FP64 rate binds there).
// ---------------------------------------------------------------------------

// One component (j = vector * 3 + axis) of the element vectors A1, B1, A2,
// B2, C, D1, D2 from the bottom (P) and top (Q) vertices, FP64:
// 0.5 ((X_a - X_b) + s (X_c - X_d)) with the vertices a, b, c, d and the
// sign s of each vector picked by integer selects, so that lanes holding
// different vectors run the same FP64 instructions (a branch per vector
// would run every branch's FP64 work in every lane of the warp).
__device__ __forceinline__ double elem_vec_comp(const double *X, int j) {
  const int v = j / 3, k = j - 3 * v;
  // a | b << 4 | c << 8 | d << 12 | (s + 1) << 16, vertices P0..P2 = 0..2,
  // Q0..Q2 = 3..5: A1 = (P1-P0) + (Q1-Q0), B1 = (Q1-Q0) - (P1-P0),
  // A2 = (P2-P0) + (Q2-Q0), B2 = (Q2-Q0) - (P2-P0), C = Q0-P0,
  // D1 = (Q1-P1) - (Q0-P0), D2 = (Q2-P2) - (Q0-P0), each halved
  const int code = v == 0 ? (1 | 0 << 4 | 4 << 8 | 3 << 12 | 2 << 16)
                   : v == 1 ? (4 | 3 << 4 | 1 << 8 | 0 << 12 | 0 << 16)
                   : v == 2 ? (2 | 0 << 4 | 5 << 8 | 3 << 12 | 2 << 16)
                   : v == 3 ? (5 | 3 << 4 | 2 << 8 | 0 << 12 | 0 << 16)
                   : v == 4 ? (3 | 0 << 4 | 0 << 8 | 0 << 12 | 1 << 16)
                   : v == 5 ? (4 | 1 << 4 | 3 << 8 | 0 << 12 | 0 << 16)
                            : (5 | 2 << 4 | 3 << 8 | 0 << 12 | 0 << 16);
  const double xa = X[3 * (code & 15) + k], xb = X[3 * ((code >> 4) & 15) + k];
  const double xc = X[3 * ((code >> 8) & 15) + k], xd = X[3 * ((code >> 12) & 15) + k];
  const int sg = code >> 16;  // s + 1
  const long long t = __double_as_longlong(xc - xd);
  // s (X_c - X_d) by the sign bit (s = -1) or zero (s = 0): integer work
  const double st = sg == 1 ? 0.0 : __longlong_as_double(sg == 0 ? t ^ (1LL << 63) : t);
  return 0.5 * ((xa - xb) + st);
}

template <typename T, int P>
struct SmallCfg {
  static constexpr int NSH = nsh_of(P), NQ = nq_of(P), K4 = 4 * NQ;
  static constexpr int M = P + 1, NT = (P + 1) * (P + 1);
  static constexpr bool F64 = std::is_same<T, double>::value;
  static constexpr int EPW = 32 / NQ;  // elements per warp
  static constexpr int WPB = F64 ? 4 : 8;
  // FP32 path, floats per slot: per vertical node w_z (alpha, beta, gamma)
  // as FP32 pairs [M][6], evf[21], cdf[14], the FP32 columns c1, c2, n3 [M][9]
  static constexpr int XF = F64 ? 0 : M * 6 + 21 + 14 + M * 9;
  static_assert((sizeof(double) * (18 + 21 + 14) + sizeof(T) * (NQ * 16 + K4 * NSH)) % 8 == 0,
                "the FP32 pairs start 8-byte aligned");
  // per element slot: X[18], ev[21], cd[14] (FP64), D[NQ][16], H[K4][NSH] (T),
  // the FP32 extras, status
  static constexpr int SLOT_BYTES =
      ((sizeof(double) * (18 + 21 + 14) + sizeof(T) * (NQ * 16 + K4 * NSH) + 4 * XF + 16 + 15) / 16) * 16;
  static constexpr int WARP_BYTES = EPW * SLOT_BYTES;
  static constexpr int SMEM = ((sizeof(T) * K4 * NSH + 15) / 16) * 16 + WPB * WARP_BYTES;
};

template <typename T, int P>
__global__ void __launch_bounds__(SmallCfg<T, P>::WPB * 32) cc_small_kernel(FwdArgs a) {
  using C = SmallCfg<T, P>;
  constexpr int NSH = C::NSH, NQ = C::NQ, K4 = C::K4, EPW = C::EPW, M = C::M, NT = C::NT;
  constexpr bool F64 = C::F64;
  static_assert(NQ <= 32, "one point per lane");
  // FP32 path: node tables of the degree, once per block (triangle node:
  // w_t, w_t xi1, w_t xi2 as FP32 pairs, and w_t, xi1, xi2; vertical node:
  // zeta and w_z)
  __shared__ float2 ttab[NT][3];
  __shared__ float ttabf[NT][3], zf[M], zwf[M];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *Gs = reinterpret_cast<T *>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char *wb = smem_raw + ((sizeof(T) * K4 * NSH + 15) / 16) * 16 + warp * C::WARP_BYTES;
  auto Xs = [&](int sl) { return reinterpret_cast<double *>(wb + sl * C::SLOT_BYTES); };
  auto evs = [&](int sl) { return Xs(sl) + 18; };
  auto cds = [&](int sl) { return Xs(sl) + 39; };
  auto Ds = [&](int sl) { return reinterpret_cast<T *>(Xs(sl) + 53); };
  auto Hs = [&](int sl) { return Ds(sl) + NQ * 16; };
  // FP32 extras: the FP32 pairs first (Fx is 8-byte aligned: the slot is
  // 16-byte aligned and every array before it a multiple of 8 bytes), then
  // evf, cdf, zc
  auto Fx = [&](int sl) { return reinterpret_cast<float *>(Hs(sl) + K4 * NSH); };
  auto zabs = [&](int sl) { return reinterpret_cast<float2 *>(Fx(sl)); };
  auto evfs = [&](int sl) { return Fx(sl) + 6 * M; };
  auto cdfs = [&](int sl) { return Fx(sl) + 6 * M + 21; };
  auto zcs = [&](int sl) { return Fx(sl) + 6 * M + 35; };
  auto Ss = [&](int sl) { return reinterpret_cast<int *>(Fx(sl) + C::XF); };

  const T *G = gtab<T>(a);
  for (int k = threadIdx.x; k < K4 * NSH; k += blockDim.x) Gs[k] = G[k];
  if constexpr (!F64) {
    for (int t = threadIdx.x; t < NT; t += blockDim.x) {
      const double x1 = a.tnode[4 * t], x2 = a.tnode[4 * t + 1], wt = a.tnode[4 * t + 2];
      ttab[t][0] = split_f64(wt);
      ttab[t][1] = split_f64(wt * x1);
      ttab[t][2] = split_f64(wt * x2);
      ttabf[t][0] = (float)wt;
      ttabf[t][1] = (float)x1;
      ttabf[t][2] = (float)x2;
    }
    for (int iz = threadIdx.x; iz < M; iz += blockDim.x) {
      zf[iz] = (float)a.znode[2 * iz];
      zwf[iz] = (float)a.znode[2 * iz + 1];
    }
  }
  __syncthreads();

  const int64_t items = n_items(a);
  const int64_t nwarps = (int64_t)gridDim.x * C::WPB;
  for (int64_t item0 = ((int64_t)blockIdx.x * C::WPB + warp) * EPW; item0 < items; item0 += nwarps * EPW) {
    const int nel = items - item0 < EPW ? (int)(items - item0) : EPW;
    // geometry and coefficients of the warp's elements, spread over lanes
    for (int idx = lane; idx < nel * 32; idx += 32) {
      const int sl = idx >> 5, k = idx & 31;
      const int64_t e = a.list ? (int64_t)a.list[item0 + sl] : item0 + sl;
      bool ok = true;
      if (k < 18) {
        const double x = a.geom[18 * e + k];
        Xs(sl)[k] = x;
        ok = finite64(x);
      } else if (a.coef_mode == FEI_COEF_PER_ELEMENT) {
        const int c = k - 18;
        const double x = c < 9 ? a.K[9 * e + c] : c < 12 ? a.b[3 * e + (c - 9)] : c == 12 ? a.c[e] : a.f[e];
        cds(sl)[c] = x;
        if constexpr (!F64) cdfs(sl)[c] = (float)x;
        ok = finite64(x);
      }
      // lanes of one element are one aligned group of 32: the whole warp
      const unsigned bad = __ballot_sync(0xffffffffu, !ok);
      // upper layout: K symmetric (K01 = K10, K02 = K20, K12 = K21: lanes
      // 19/21, 20/24, 23/25) and b = 0 (lanes 27-29), per-element records
      bool sym = true;
      if (a.upper && a.coef_mode == FEI_COEF_PER_ELEMENT) {
        const double xk = k >= 18 ? cds(sl)[k - 18] : 0.0;
        const int c = k - 18;
        const int partner = c == 1 ? 21 : c == 3 ? 19 : c == 2 ? 24 : c == 6 ? 20 : c == 5 ? 25 : c == 7 ? 23 : k;
        const double xp = __shfl_sync(0xffffffffu, xk, partner);
        sym = (c >= 9 && c <= 11) ? xk == 0.0 : xk == xp;
      }
      const unsigned nonsym = __ballot_sync(0xffffffffu, !sym);
      if (k == 0) Ss(sl)[0] = bad ? 2 * FEI_ERR_NONFINITE : (nonsym ? FEI_ERR_INVALID_ARG : 0);
    }
    __syncwarp();
    // element vectors, one component per lane (FP64)
    for (int idx = lane; idx < nel * 21; idx += 32) {
      const int sl = idx / 21, j = idx - sl * 21;
      const double v = elem_vec_comp(Xs(sl), j);
      evs(sl)[j] = v;
      if constexpr (!F64) evfs(sl)[j] = (float)v;
    }
    __syncwarp();
    if constexpr (!F64) {
      // per vertical node, three lanes (one per axis k): FP64 n3 = c1 x c2
      // and w_z (n3.C, n3.D1, n3.D2) as FP32 pairs; the FP32 columns c1, c2
      // and n3 from the FP32 vectors
      {
        const bool act = lane < nel * M * 3;
        const int sl = act ? lane / (3 * M) : 0, rem = act ? lane - sl * 3 * M : 0;
        const int iz = rem / 3, k = rem - 3 * iz;
        const int g0 = lane - k, l1 = g0 + (k + 1) % 3, l2 = g0 + (k + 2) % 3;
        const double *ev = evs(sl);
        const double z = a.znode[2 * iz], wz = a.znode[2 * iz + 1];
        const double c1 = fma(z, ev[3 + k], ev[k]), c2 = fma(z, ev[9 + k], ev[6 + k]);
        const double c1a = __shfl_sync(0xffffffffu, c1, l1), c1b = __shfl_sync(0xffffffffu, c1, l2);
        const double c2a = __shfl_sync(0xffffffffu, c2, l1), c2b = __shfl_sync(0xffffffffu, c2, l2);
        const double n3 = c1a * c2b - c1b * c2a;  // (c1 x c2)_k
        double al = n3 * ev[12 + k], be = n3 * ev[15 + k], ga = n3 * ev[18 + k];
        al += __shfl_sync(0xffffffffu, al, l1) + __shfl_sync(0xffffffffu, al, l2);
        be += __shfl_sync(0xffffffffu, be, l1) + __shfl_sync(0xffffffffu, be, l2);
        ga += __shfl_sync(0xffffffffu, ga, l1) + __shfl_sync(0xffffffffu, ga, l2);
        const float *evf = evfs(sl);
        const float f1 = fmaf(zf[iz], evf[3 + k], evf[k]), f2 = fmaf(zf[iz], evf[9 + k], evf[6 + k]);
        const float f1a = __shfl_sync(0xffffffffu, f1, l1), f1b = __shfl_sync(0xffffffffu, f1, l2);
        const float f2a = __shfl_sync(0xffffffffu, f2, l1), f2b = __shfl_sync(0xffffffffu, f2, l2);
        if (act) {
          // lane k of the node keeps value k of (alpha, beta, gamma)
          zabs(sl)[3 * iz + k] = split_f64(wz * (k == 0 ? al : k == 1 ? be : ga));
          float *zc = zcs(sl) + 9 * iz;
          zc[k] = f1;
          zc[3 + k] = f2;
          zc[6 + k] = f1a * f2b - f1b * f2a;
        }
      }
      __syncwarp();
    }
    // point operators: lane = (element slot, point)
    const int psl = lane / NQ, q = lane - psl * NQ;
    int pst = 0;
    if (psl < nel) {
      const int64_t e = a.list ? (int64_t)a.list[item0 + psl] : item0 + psl;
      // quadrature point from the node tables: q = iz*(p+1)^2 + t
      const int iz = q / NT, t = q % NT;
      double cq[14];
      if (a.coef_mode == FEI_COEF_PER_POINT) {
        const int64_t r = (a.q_off ? a.q_off[e] : e * (int64_t)NQ) + q;
        if (!load_coef(a, r, cq)) pst = FEI_ERR_NONFINITE;
        else if (a.upper && !coef_symmetric(cq, cq + 9)) pst = FEI_ERR_INVALID_ARG;
      }
      const bool perq = a.coef_mode == FEI_COEF_PER_POINT;
      if constexpr (F64) {
        const double ptv[4] = {a.tnode[4 * t], a.tnode[4 * t + 1], a.znode[2 * iz],
                               a.tnode[4 * t + 2] * a.znode[2 * iz + 1]};
        pst = merge_status(pst, point_direct64(evs(psl), ptv, perq ? cq : cds(psl), Ds(psl) + 16 * q));
      } else {
        const float *evf = evfs(psl), *zc = zcs(psl) + 9 * iz;
        const float2 *zab = zabs(psl) + 3 * iz;
        // w det J in double-FP32, rounded once
        const float2 sd = add_ff(add_ff(mul_ff(ttab[t][0], zab[0]), mul_ff(ttab[t][1], zab[1])),
                                 mul_ff(ttab[t][2], zab[2]));
        const float sf = sd.x + sd.y;
        const int sst = !(fabsf(sf) <= 3.402823466e38f) ? FEI_ERR_NONFINITE
                        : !(sf > 0.f)                    ? FEI_ERR_NEGATIVE_JACOBIAN
                                                         : 0;
        float c3[3], a0[3], a1[3], K[9], b[3], cf, ff;
#pragma unroll
        for (int k = 0; k < 3; ++k) c3[k] = fmaf(ttabf[t][2], evf[18 + k], fmaf(ttabf[t][1], evf[15 + k], evf[12 + k]));
        cross3(zc + 3, c3, a0);
        cross3(c3, zc, a1);
        if (perq) {
#pragma unroll
          for (int k = 0; k < 9; ++k) K[k] = (float)cq[k];
#pragma unroll
          for (int k = 0; k < 3; ++k) b[k] = (float)cq[9 + k];
          cf = (float)cq[12];
          ff = (float)cq[13];
        } else {
          const float *cdf = cdfs(psl);
#pragma unroll
          for (int k = 0; k < 9; ++k) K[k] = cdf[k];
#pragma unroll
          for (int k = 0; k < 3; ++k) b[k] = cdf[9 + k];
          cf = cdf[12];
          ff = cdf[13];
        }
        const float wf = ttabf[t][0] * zwf[iz];
        dt_from_adj<float>(a0, a1, zc + 6, wf, sf, wf * wf / sf, K, b, cf, ff, Ds(psl) + 16 * q);
        pst = merge_status(pst, sst);
      }
      if (pst) atomicMax(Ss(psl), pst == FEI_ERR_NONFINITE ? 2 * FEI_ERR_NONFINITE : pst);
    }
    __syncwarp();
    // H[(q, b)][i] = sum_a Dt_q[a][b] G[q][a][i], per element
    for (int idx = lane; idx < nel * NQ * NSH; idx += 32) {
      const int sl = idx / (NQ * NSH), rem = idx - sl * (NQ * NSH);
      const int qq = rem / NSH, i = rem - qq * NSH;
      const T *Dq = Ds(sl) + 16 * qq;
      T *H = Hs(sl);
      const T g0 = Gs[(4 * qq + 0) * NSH + i], g1 = Gs[(4 * qq + 1) * NSH + i];
      const T g2 = Gs[(4 * qq + 2) * NSH + i], g3 = Gs[(4 * qq + 3) * NSH + i];
      H[(4 * qq + 0) * NSH + i] = Dq[0] * g0;
#pragma unroll
      for (int m = 0; m < 3; ++m)
        H[(4 * qq + 1 + m) * NSH + i] = Dq[1 + m] * g0 + Dq[4 + m] * g1 + Dq[7 + m] * g2 + Dq[10 + m] * g3;
    }
    __syncwarp();
    // A_e = H^T G and b_e, lanes over (element, entry)
    for (int idx = lane; idx < nel * NSH * NSH; idx += 32) {
      const int sl = idx / (NSH * NSH), ij = idx - sl * (NSH * NSH);
      const int i = ij / NSH, j = ij - i * NSH;
      const int64_t e = a.list ? (int64_t)a.list[item0 + sl] : item0 + sl;
      const int64_t aoff = out_a(a, item0 + sl, e, NSH);
      if (a.upper && j < i) continue;  // the upper layout keeps j >= i
      const T *H = Hs(sl);
      T acc = T(0);
#pragma unroll 4
      for (int k = 0; k < K4; ++k) acc += H[k * NSH + i] * Gs[k * NSH + j];
      reinterpret_cast<T *>(a.A)[aoff + a_pos(i, j, NSH, a.upper)] = Ss(sl)[0] ? T(0) : acc;
    }
    for (int idx = lane; idx < nel * NSH; idx += 32) {
      const int sl = idx / NSH, i = idx - sl * NSH;
      const int64_t e = a.list ? (int64_t)a.list[item0 + sl] : item0 + sl;
      const int64_t boff = out_b(a, item0 + sl, e, NSH);
      const T *D = Ds(sl);
      T acc = T(0);
      for (int qq = 0; qq < NQ; ++qq) acc += D[16 * qq + 13] * Gs[(4 * qq) * NSH + i];
      reinterpret_cast<T *>(a.bv)[boff + i] = Ss(sl)[0] ? T(0) : acc;
    }
    for (int sl = lane; sl < nel; sl += 32) {
      const int64_t e = a.list ? (int64_t)a.list[item0 + sl] : item0 + sl;
      const int v = Ss(sl)[0];
      // NONFINITE is recorded as 2 * NONFINITE so that it wins the max
      a.status[e] = v == 2 * FEI_ERR_NONFINITE ? FEI_ERR_NONFINITE : v;
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// p = 1, FP32 path: one thread per element.  A p = 1 element is small (6
// shape functions, 8 points, 36 entries), so a thread keeps A_e and b_e in
// registers and runs the points in turn.  With one element per lane, every
// FP64 instruction of the setup (element vectors, the vertical-node sums
// of det J) serves 32 elements: this part's FP64 rate is what binds p = 1,
// and a warp shared by four elements ran most of that work on a few lanes.
// ---------------------------------------------------------------------------
constexpr int kP1Threads = 128;

// The two p = 1 kernels below (one thread per element for large batches,
// eight lanes per element for small ones) give the same bits: their
// FP64 node sums and their sums over points run in one fixed order of
// rounded operations (the host-memory entry cuts a batch into chunks of
// any size and must equal the device entry bit for bit).
//
// w_z (n3.C, n3.D1, n3.D2) of a vertical node as FP32 pairs, from the
// columns' components c1[k], c2[k] and C, D1, D2 (FP64): n3_k and its
// products p_k rounded one by one, value v summed as (p_v + p_v+1) + p_v+2.
__device__ __forceinline__ double p1_node_sum(const double *n3, const double *w, int v) {
  const double a = __dmul_rn(n3[v], w[v]), b = __dmul_rn(n3[(v + 1) % 3], w[(v + 1) % 3]);
  const double c = __dmul_rn(n3[(v + 2) % 3], w[(v + 2) % 3]);
  return __dadd_rn(__dadd_rn(a, b), c);
}
__device__ __forceinline__ double p1_cross_comp(double a1, double a2, double b1, double b2) {
  return __dsub_rn(__dmul_rn(a1, b2), __dmul_rn(a2, b1));  // a1 b2 - a2 b1
}
// One point's contribution to A_e (36 values, row-major) and b_e (6):
// G_q^T Dt_q G_q and (w det J f) G_q0, every operation rounded in turn.
__device__ __forceinline__ void p1_point_contrib(const float *D, const float *G, float *c) {
  constexpr int NSH = 6;
#pragma unroll
  for (int i = 0; i < NSH; ++i) {
    const float g0 = G[i], g1 = G[NSH + i], g2 = G[2 * NSH + i], g3 = G[3 * NSH + i];
    const float h0 = __fmul_rn(D[0], g0);
    const float h1 = __fmaf_rn(D[10], g3, __fmaf_rn(D[7], g2, __fmaf_rn(D[4], g1, __fmul_rn(D[1], g0))));
    const float h2 = __fmaf_rn(D[11], g3, __fmaf_rn(D[8], g2, __fmaf_rn(D[5], g1, __fmul_rn(D[2], g0))));
    const float h3 = __fmaf_rn(D[12], g3, __fmaf_rn(D[9], g2, __fmaf_rn(D[6], g1, __fmul_rn(D[3], g0))));
#pragma unroll
    for (int j = 0; j < NSH; ++j)
      c[i * NSH + j] = __fmaf_rn(h3, G[3 * NSH + j],
                                 __fmaf_rn(h2, G[2 * NSH + j], __fmaf_rn(h1, G[NSH + j], __fmul_rn(h0, G[j]))));
    c[NSH * NSH + i] = __fmul_rn(D[13], g0);
  }
}

__global__ void __launch_bounds__(kP1Threads, 3) cc_p1_kernel(FwdArgs a) {
  constexpr int NSH = 6, NQ = 8, M = 2, NT = 4;
  __shared__ float Gs[4 * NQ * NSH];  // G32 [q][a][i]
  __shared__ float2 ttab[NT][3];      // w_t, w_t xi1, w_t xi2 as FP32 pairs
  __shared__ float ttabf[NT][3];      // w_t, xi1, xi2
  __shared__ float zf[M], zwf[M];
  __shared__ double zd[M], zwd[M];
  for (int k = threadIdx.x; k < 4 * NQ * NSH; k += blockDim.x) Gs[k] = a.G32[k];
  if (threadIdx.x < NT) {
    const int t = threadIdx.x;
    const double x1 = a.tnode[4 * t], x2 = a.tnode[4 * t + 1], wt = a.tnode[4 * t + 2];
    ttab[t][0] = split_f64(wt);
    ttab[t][1] = split_f64(wt * x1);
    ttab[t][2] = split_f64(wt * x2);
    ttabf[t][0] = (float)wt;
    ttabf[t][1] = (float)x1;
    ttabf[t][2] = (float)x2;
  } else if (threadIdx.x >= 32 && threadIdx.x < 32 + M) {
    const int iz = threadIdx.x - 32;
    zd[iz] = a.znode[2 * iz];
    zwd[iz] = a.znode[2 * iz + 1];
    zf[iz] = (float)zd[iz];
    zwf[iz] = (float)zwd[iz];
  }
  __syncthreads();
  const int64_t items = n_items(a);
  for (int64_t item = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; item < items;
       item += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = a.list ? (int64_t)a.list[item] : item;
    bool ok = true, sym = true;
    float ev32[21];   // element vectors rounded once
    float2 zab[M][3];  // per vertical node w_z (n3.C, n3.D1, n3.D2), FP32 pairs
    {
      double X[18], ev[21];
#pragma unroll
      for (int k = 0; k < 18; ++k) {
        X[k] = a.geom[18 * e + k];
        ok &= finite64(X[k]);
      }
      elem_vectors(X, ev);
#pragma unroll
      for (int k = 0; k < 21; ++k) ev32[k] = (float)ev[k];
#pragma unroll
      for (int iz = 0; iz < M; ++iz) {
        double c1[3], c2[3], n3[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          c1[k] = fma(zd[iz], ev[3 + k], ev[k]);
          c2[k] = fma(zd[iz], ev[9 + k], ev[6 + k]);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k)
          n3[k] = p1_cross_comp(c1[(k + 1) % 3], c1[(k + 2) % 3], c2[(k + 1) % 3], c2[(k + 2) % 3]);
        zab[iz][0] = split_f64(__dmul_rn(zwd[iz], p1_node_sum(n3, ev + 12, 0)));
        zab[iz][1] = split_f64(__dmul_rn(zwd[iz], p1_node_sum(n3, ev + 15, 1)));
        zab[iz][2] = split_f64(__dmul_rn(zwd[iz], p1_node_sum(n3, ev + 18, 2)));
      }
    }
    // FP32 columns c1, c2 and n3 per vertical node
    float zc[M][9];
#pragma unroll
    for (int iz = 0; iz < M; ++iz) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        zc[iz][k] = fmaf(zf[iz], ev32[3 + k], ev32[k]);
        zc[iz][3 + k] = fmaf(zf[iz], ev32[9 + k], ev32[6 + k]);
      }
      cross3(zc[iz], zc[iz] + 3, zc[iz] + 6);
    }
    float cf[14];
    const bool perq = a.coef_mode == FEI_COEF_PER_POINT;
    if (!perq) {
      double cd[14];
      ok &= load_coef(a, e, cd);
      sym = !a.upper || coef_symmetric(cd, cd + 9);
#pragma unroll
      for (int k = 0; k < 14; ++k) cf[k] = (float)cd[k];
    }
    int st = !ok ? FEI_ERR_NONFINITE : (!sym ? FEI_ERR_INVALID_ARG : 0);
    float A[NSH][NSH], bv[NSH];
#pragma unroll
    for (int i = 0; i < NSH; ++i) {
      bv[i] = 0.f;
#pragma unroll
      for (int j = 0; j < NSH; ++j) A[i][j] = 0.f;
    }
#pragma unroll
    for (int iz = 0; iz < M; ++iz)
#pragma unroll 1
    for (int t = 0; t < NT; ++t) {
      const int q = iz * NT + t;
      if (perq) {
        double cd[14];
        const int64_t r = (a.q_off ? a.q_off[e] : e * (int64_t)NQ) + q;
        int pst = 0;
        if (!load_coef(a, r, cd)) pst = FEI_ERR_NONFINITE;
        else if (a.upper && !coef_symmetric(cd, cd + 9)) pst = FEI_ERR_INVALID_ARG;
        st = merge_status(st, pst);
#pragma unroll
        for (int k = 0; k < 14; ++k) cf[k] = (float)cd[k];
      }
      // w det J in double-FP32, rounded once
      const float2 sd = add_ff(add_ff(mul_ff(ttab[t][0], zab[iz][0]), mul_ff(ttab[t][1], zab[iz][1])),
                               mul_ff(ttab[t][2], zab[iz][2]));
      const float sf = sd.x + sd.y;
      st = merge_status(st, !(fabsf(sf) <= 3.402823466e38f) ? FEI_ERR_NONFINITE
                            : !(sf > 0.f)                    ? FEI_ERR_NEGATIVE_JACOBIAN
                                                             : 0);
      float c3[3], a0[3], a1[3], D[16];
#pragma unroll
      for (int k = 0; k < 3; ++k)
        c3[k] = fmaf(ttabf[t][2], ev32[18 + k], fmaf(ttabf[t][1], ev32[15 + k], ev32[12 + k]));
      cross3(zc[iz] + 3, c3, a0);
      cross3(c3, zc[iz], a1);
      const float wf = ttabf[t][0] * zwf[iz];
      dt_from_adj<float>(a0, a1, zc[iz] + 6, wf, sf, wf * wf / sf, cf, cf + 9, cf[12], cf[13], D);
      // A_e += G_q^T Dt_q G_q, b_e += (w det J f) G_q0
      float c[NSH * NSH + NSH];
      p1_point_contrib(D, Gs + q * 4 * NSH, c);
#pragma unroll
      for (int i = 0; i < NSH; ++i) {
#pragma unroll
        for (int j = 0; j < NSH; ++j) A[i][j] = __fadd_rn(A[i][j], c[i * NSH + j]);
        bv[i] = __fadd_rn(bv[i], c[NSH * NSH + i]);
      }
    }
    float *Ao = reinterpret_cast<float *>(a.A) + out_a(a, item, e, NSH);
#pragma unroll
    for (int i = 0; i < NSH; ++i)
#pragma unroll
      for (int j = 0; j < NSH; ++j)
        if (!a.upper || j >= i) Ao[a_pos(i, j, NSH, a.upper)] = st ? 0.f : A[i][j];
    float *bo = reinterpret_cast<float *>(a.bv) + out_b(a, item, e, NSH);
#pragma unroll
    for (int i = 0; i < NSH; ++i) bo[i] = st ? 0.f : bv[i];
    a.status[e] = st;
  }
}

// p = 1, FP32 path, small batches: eight lanes per element (one per
// point), so that a batch that fills only part of the GPU (4096 prisms:
// 32 blocks of the kernel above) is not bound by one thread walking its
// eight points in turn.  The FP64 work is spread over the lanes (three
// element-vector components per lane, three lanes per vertical node for
// the node sums), each lane forms its point's contribution to A_e and b_e
// in registers, and a butterfly over the eight lanes adds them up.
__global__ void __launch_bounds__(kP1Threads) cc_p1_small_kernel(FwdArgs a) {
  constexpr int NSH = 6, NQ = 8, M = 2, NT = 4;
  __shared__ float Gs[4 * NQ * NSH];  // G32 [q][a][i]
  __shared__ float2 ttab[NT][3];
  __shared__ float ttabf[NT][3];
  __shared__ float zf[M], zwf[M];
  __shared__ double zd[M], zwd[M];
  for (int k = threadIdx.x; k < 4 * NQ * NSH; k += blockDim.x) Gs[k] = a.G32[k];
  if (threadIdx.x < NT) {
    const int t = threadIdx.x;
    const double x1 = a.tnode[4 * t], x2 = a.tnode[4 * t + 1], wt = a.tnode[4 * t + 2];
    ttab[t][0] = split_f64(wt);
    ttab[t][1] = split_f64(wt * x1);
    ttab[t][2] = split_f64(wt * x2);
    ttabf[t][0] = (float)wt;
    ttabf[t][1] = (float)x1;
    ttabf[t][2] = (float)x2;
  } else if (threadIdx.x >= 32 && threadIdx.x < 32 + M) {
    const int iz = threadIdx.x - 32;
    zd[iz] = a.znode[2 * iz];
    zwd[iz] = a.znode[2 * iz + 1];
    zf[iz] = (float)zd[iz];
    zwf[iz] = (float)zwd[iz];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane & 7, gbase = lane & 24;
  const int64_t items = n_items(a);
  const int64_t groups = (int64_t)gridDim.x * (blockDim.x / 8);
  // every lane of the warp runs every iteration (the shuffles need the
  // whole warp); a group past the end computes on a clamped element and
  // stores nothing
  const int64_t first = (int64_t)blockIdx.x * (blockDim.x / 8) + (threadIdx.x >> 3);
  const int64_t warp_first = first - (lane >> 3);
  for (int64_t it0 = warp_first; it0 < items; it0 += groups) {
    const int64_t item = it0 + (lane >> 3);
    const bool live = item < items;
    const int64_t e = live ? (a.list ? (int64_t)a.list[item] : item) : (a.list ? (int64_t)a.list[0] : 0);
    // vertices: lane g checks coordinates g, g + 8, g + 16 (the group's AND
    // below); the element-vector components g, g + 8, g + 16 read theirs
    // from global memory (the group's 144 bytes, cached), in FP64
    const double *X = a.geom + 18 * e;
    bool ok = finite64(X[g]) && finite64(X[g + 8]) && (g >= 2 || finite64(X[g + 16]));
    double evm[3];
    float evfm[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int j = g + 8 * r;
      evm[r] = elem_vec_comp(X, j < 21 ? j : 20);
      evfm[r] = (float)evm[r];
    }
    float ev32[21];
#pragma unroll
    for (int j = 0; j < 21; ++j) ev32[j] = __shfl_sync(0xffffffffu, evfm[j / 8], gbase + (j & 7));
    auto ev64 = [&](int j) { return __shfl_sync(0xffffffffu, evm[j / 8], gbase + (j & 7)); };
    // node sums: lanes 0..5 of the group, three per vertical node
    float2 zab[M][3];
    {
      const int iz = g < 3 ? 0 : 1, k = g < 6 ? g - 3 * iz : 0;
      const int l1 = gbase + 3 * iz + (k + 1) % 3, l2 = gbase + 3 * iz + (k + 2) % 3;
      // components k of A1, B1, A2, B2, C, D1, D2 (the shuffles run in all lanes)
      double e0 = ev64(0), e1 = ev64(1), e2 = ev64(2), e3 = ev64(3), e4 = ev64(4), e5 = ev64(5);
      double e6 = ev64(6), e7 = ev64(7), e8 = ev64(8), e9 = ev64(9), e10 = ev64(10), e11 = ev64(11);
      double e12 = ev64(12), e13 = ev64(13), e14 = ev64(14), e15 = ev64(15), e16 = ev64(16), e17 = ev64(17);
      double e18 = ev64(18), e19 = ev64(19), e20 = ev64(20);
      const double A1 = k == 0 ? e0 : k == 1 ? e1 : e2, B1 = k == 0 ? e3 : k == 1 ? e4 : e5;
      const double A2 = k == 0 ? e6 : k == 1 ? e7 : e8, B2 = k == 0 ? e9 : k == 1 ? e10 : e11;
      const double Cc = k == 0 ? e12 : k == 1 ? e13 : e14, D1 = k == 0 ? e15 : k == 1 ? e16 : e17;
      const double D2 = k == 0 ? e18 : k == 1 ? e19 : e20;
      const double z = zd[iz], wz = zwd[iz];
      const double c1 = fma(z, B1, A1), c2 = fma(z, B2, A2);
      const double c1a = __shfl_sync(0xffffffffu, c1, l1), c1b = __shfl_sync(0xffffffffu, c1, l2);
      const double c2a = __shfl_sync(0xffffffffu, c2, l1), c2b = __shfl_sync(0xffffffffu, c2, l2);
      const double n3 = p1_cross_comp(c1a, c1b, c2a, c2b);
      // lane k of the node keeps value k, summed as (p_k + p_k+1) + p_k+2
      const double pa = __dmul_rn(n3, Cc), pb = __dmul_rn(n3, D1), pc = __dmul_rn(n3, D2);
      const double s_al = __dadd_rn(__dadd_rn(pa, __shfl_sync(0xffffffffu, pa, l1)), __shfl_sync(0xffffffffu, pa, l2));
      const double s_be = __dadd_rn(__dadd_rn(pb, __shfl_sync(0xffffffffu, pb, l1)), __shfl_sync(0xffffffffu, pb, l2));
      const double s_ga = __dadd_rn(__dadd_rn(pc, __shfl_sync(0xffffffffu, pc, l1)), __shfl_sync(0xffffffffu, pc, l2));
      const float2 mine = split_f64(__dmul_rn(wz, k == 0 ? s_al : k == 1 ? s_be : s_ga));
#pragma unroll
      for (int n = 0; n < M; ++n)
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          zab[n][v].x = __shfl_sync(0xffffffffu, mine.x, gbase + 3 * n + v);
          zab[n][v].y = __shfl_sync(0xffffffffu, mine.y, gbase + 3 * n + v);
        }
    }
    // coefficients: components g and g + 8 per lane, shared in FP32
    float cf[14];
    const bool perq = a.coef_mode == FEI_COEF_PER_POINT;
    bool sym = true;
    if (!perq) {
      float cm[2];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int c = g + 8 * r;
        double x = 0.0;
        if (c < 14) x = c < 9 ? a.K[9 * e + c] : c < 12 ? a.b[3 * e + c - 9] : c == 12 ? a.c[e] : a.f[e];
        ok &= finite64(x);
        cm[r] = (float)x;
      }
#pragma unroll
      for (int c = 0; c < 14; ++c) cf[c] = __shfl_sync(0xffffffffu, cm[c / 8], gbase + (c & 7));
      if (a.upper) {
        // K symmetric and b = 0, compared in FP64 (as the other kernels)
        const double k01 = a.K[9 * e + 1], k10 = a.K[9 * e + 3], k02 = a.K[9 * e + 2], k20 = a.K[9 * e + 6];
        const double k12 = a.K[9 * e + 5], k21 = a.K[9 * e + 7];
        sym = k01 == k10 && k02 == k20 && k12 == k21 && a.b[3 * e] == 0.0 && a.b[3 * e + 1] == 0.0 &&
              a.b[3 * e + 2] == 0.0;
      }
    }
    // the point of this lane
    const int q = g, iz = q / NT, t = q - iz * NT;
    int st = 0;
    if (perq) {
      double cd[14];
      const int64_t r = (a.q_off ? a.q_off[e] : e * (int64_t)NQ) + q;
      if (!load_coef(a, r, cd)) st = FEI_ERR_NONFINITE;
      else if (a.upper && !coef_symmetric(cd, cd + 9)) st = FEI_ERR_INVALID_ARG;
#pragma unroll
      for (int k = 0; k < 14; ++k) cf[k] = (float)cd[k];
    }
    const float2 *zq = iz ? zab[1] : zab[0];
    const float2 sd = add_ff(add_ff(mul_ff(ttab[t][0], zq[0]), mul_ff(ttab[t][1], zq[1])), mul_ff(ttab[t][2], zq[2]));
    const float sf = sd.x + sd.y;
    st = merge_status(st, !(fabsf(sf) <= 3.402823466e38f) ? FEI_ERR_NONFINITE
                          : !(sf > 0.f)                    ? FEI_ERR_NEGATIVE_JACOBIAN
                                                           : 0);
    float zc[9];
    {
      const float zz = zf[iz];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        zc[k] = fmaf(zz, ev32[3 + k], ev32[k]);
        zc[3 + k] = fmaf(zz, ev32[9 + k], ev32[6 + k]);
      }
      cross3(zc, zc + 3, zc + 6);
    }
    float c3[3], a0[3], a1[3], D[16];
#pragma unroll
    for (int k = 0; k < 3; ++k) c3[k] = fmaf(ttabf[t][2], ev32[18 + k], fmaf(ttabf[t][1], ev32[15 + k], ev32[12 + k]));
    cross3(zc + 3, c3, a0);
    cross3(c3, zc, a1);
    const float wf = ttabf[t][0] * zwf[iz];
    dt_from_adj<float>(a0, a1, zc + 6, wf, sf, wf * wf / sf, cf, cf + 9, cf[12], cf[13], D);
    float c[NSH * NSH + NSH];  // this point's G_q^T Dt_q G_q, then its share of b
    p1_point_contrib(D, Gs + q * 4 * NSH, c);
    // the sums over the group's points in point order (q = lane), as the
    // one-thread kernel adds them
    float A[NSH * NSH + NSH];
#pragma unroll
    for (int v = 0; v < NSH * NSH + NSH; ++v) A[v] = 0.f;
#pragma unroll
    for (int qq = 0; qq < NQ; ++qq)
#pragma unroll
      for (int v = 0; v < NSH * NSH + NSH; ++v) A[v] = __fadd_rn(A[v], __shfl_sync(0xffffffffu, c[v], gbase + qq));
    int code = st == FEI_ERR_NONFINITE ? 2 * FEI_ERR_NONFINITE : st;
    if (!ok) code = 2 * FEI_ERR_NONFINITE;  // any lane's coordinate or coefficient
    else if (!sym && code == 0) code = FEI_ERR_INVALID_ARG;
#pragma unroll
    for (int off = 4; off >= 1; off >>= 1) code = max(code, __shfl_xor_sync(0xffffffffu, code, off));
    const int fst = code == 2 * FEI_ERR_NONFINITE ? FEI_ERR_NONFINITE : code;
    if (live) {
      float *Ao = reinterpret_cast<float *>(a.A) + out_a(a, item, e, NSH);
      float *bo = reinterpret_cast<float *>(a.bv) + out_b(a, item, e, NSH);
#pragma unroll
      for (int v = 0; v < NSH * NSH + NSH; ++v) {
        if ((v & 7) != g) continue;
        if (v < NSH * NSH) {
          const int i = v / NSH, j = v - i * NSH;
          if (!a.upper || j >= i) Ao[a_pos(i, j, NSH, a.upper)] = fst ? 0.f : A[v];
        } else {
          bo[v - NSH * NSH] = fst ? 0.f : A[v];
        }
      }
      if (g == 0) a.status[e] = fst;
    }
  }
}

// Below this many elements the batch fills little of the GPU with one
// thread per element, and eight lanes per element finish sooner.
constexpr int64_t kP1SmallBatch = 16384;

fei_status launch_p1(const FwdArgs &a, int64_t grid_work, cudaStream_t s, int64_t grid_cap) {
  if (!a.count && grid_work <= kP1SmallBatch) {
    int64_t blocks = (grid_work * 8 + kP1Threads - 1) / kP1Threads;
    if (grid_cap > 0 && blocks > grid_cap) blocks = grid_cap;
    cc_p1_small_kernel<<<(unsigned)blocks, kP1Threads, 0, s>>>(a);
    FEI_CUDA_TRY(cudaGetLastError(), "cc_p1_small_kernel launch");
    return FEI_OK;
  }
  int64_t blocks = (grid_work + kP1Threads - 1) / kP1Threads;
  const int64_t cap = grid_cap > 0 ? grid_cap : (a.count ? 152 * 8 : 0);
  if (cap > 0 && blocks > cap) blocks = cap;
  if (blocks > 2147483647LL) blocks = 2147483647LL;
  if (blocks < 1) blocks = 1;
  cc_p1_kernel<<<(unsigned)blocks, kP1Threads, 0, s>>>(a);
  FEI_CUDA_TRY(cudaGetLastError(), "cc_p1_kernel launch");
  return FEI_OK;
}

// ---------------------------------------------------------------------------
// Higher degree (p >= 3): one thread block per (element, row block, column
// block), 16x16 threads, RM x RM register tile per thread.
// ---------------------------------------------------------------------------

template <typename T, int P>
struct TileCfg {
  static constexpr int NSH = nsh_of(P), NQ = nq_of(P), NZ = P + 1, NT = (P + 1) * (P + 1);
  static constexpr int RM = (P == 3) ? 3 : (P == 4) ? 5 : (P == 5) ? 8 : (P == 6) ? 7 : 6;
  static constexpr int BM = 16 * RM;
  static constexpr int NB = (NSH + BM - 1) / BM;
  static constexpr int QC = std::is_same<T, double>::value ? 4 : 8;
  static constexpr int KC = 4 * QC;
};

template <typename T, int P>
struct TileSmem {
  using C = TileCfg<T, P>;
  double X[18];
  double ev[21];
  double cd[14];
  // FP64 node data
  double zc1[C::NZ][3], zc2[C::NZ][3], zn3[C::NZ][3], zw[C::NZ];
  double tc3[C::NT][3], tw[C::NT];
  // FP32 node data (FP32 path): columns rounded once, w-scaled FP64 for s
  float zc1f[C::NZ][3], zc2f[C::NZ][3], zn3f[C::NZ][3], zwf[C::NZ];
  float tc3f[C::NT][3], twf[C::NT];
  double zn3w[C::NZ][3], tc3w[C::NT][3];
  T D[C::QC][16];
  T H[C::KC][C::BM];
  T G[C::KC][C::BM];
  int status;
};

template <typename T, int P>
__global__ void __launch_bounds__(256) cc_tile_kernel(FwdArgs a) {
  using C = TileCfg<T, P>;
  constexpr int NSH = C::NSH, NQ = C::NQ, NT = C::NT, BM = C::BM, NB = C::NB, RM = C::RM;
  constexpr int QC = C::QC, KC = C::KC;
  constexpr bool F64 = std::is_same<T, double>::value;
  __shared__ __align__(16) TileSmem<T, P> sm;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const T *Gg = gtab<T>(a);
  const int64_t jobs = n_items(a) * (NB * NB);

  for (int64_t job = blockIdx.x; job < jobs; job += gridDim.x) {
    const int64_t item = job / (NB * NB);
    const int rb = (int)((job / NB) % NB), cb = (int)(job % NB);
    const int64_t e = a.list ? (int64_t)a.list[item] : item;
    if (tid == 0) sm.status = 0;
    __syncthreads();
    // step 2: geometry (and per-element coefficients)
    bool ok = true;
    if (tid < 18) {
      sm.X[tid] = a.geom[18 * e + tid];
      ok = finite64(sm.X[tid]);
    }
    bool sym = true;
    if (a.coef_mode == FEI_COEF_PER_ELEMENT && tid == 32) {
      ok = load_coef(a, e, sm.cd);
      sym = !a.upper || coef_symmetric(sm.cd, sm.cd + 9);
    }
    if (!ok) sm.status = FEI_ERR_NONFINITE;
    __syncthreads();
    if (!sym) atomicMax(&sm.status, FEI_ERR_INVALID_ARG);
    __syncthreads();
    if (tid == 0) elem_vectors(sm.X, sm.ev);
    __syncthreads();
    // Jacobian columns at the vertical and triangle nodes (FP64)
    if (tid < C::NZ) {
      const double z = a.znode[2 * tid], wz = a.znode[2 * tid + 1];
      znode_columns(sm.ev, z, sm.zc1[tid], sm.zc2[tid], sm.zn3[tid]);
      sm.zw[tid] = wz;
      if constexpr (!F64) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          sm.zc1f[tid][k] = (float)sm.zc1[tid][k];
          sm.zc2f[tid][k] = (float)sm.zc2[tid][k];
          sm.zn3f[tid][k] = (float)sm.zn3[tid][k];
          sm.zn3w[tid][k] = wz * sm.zn3[tid][k];
        }
        sm.zwf[tid] = (float)wz;
      }
    } else if (tid >= 32 && tid < 32 + NT) {
      const int t = tid - 32;
      const double wt = a.tnode[4 * t + 2];
      tnode_column(sm.ev, a.tnode[4 * t], a.tnode[4 * t + 1], sm.tc3[t]);
      sm.tw[t] = wt;
      if constexpr (!F64) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          sm.tc3f[t][k] = (float)sm.tc3[t][k];
          sm.tc3w[t][k] = wt * sm.tc3[t][k];
        }
        sm.twf[t] = (float)wt;
      }
    }
    __syncthreads();

    T acc[RM][RM];
#pragma unroll
    for (int r = 0; r < RM; ++r)
#pragma unroll
      for (int c = 0; c < RM; ++c) acc[r][c] = T(0);
    T bacc = T(0);
    const int brow = rb * BM + tid;  // load-vector row of this thread (cb == 0)

    for (int q0 = 0; q0 < NQ; q0 += QC) {
      // steps 7-8: point operators of this chunk
      if (tid < QC) {
        const int q = q0 + tid;
        T *D = sm.D[tid];
        if (q < NQ) {
          const int iz = q / NT, t = q - iz * NT;
          double cq[14];
          const double *cp = sm.cd;
          int pst = 0;
          if (a.coef_mode == FEI_COEF_PER_POINT) {
            const int64_t r = (a.q_off ? a.q_off[e] : e * (int64_t)NQ) + q;
            if (!load_coef(a, r, cq)) pst = FEI_ERR_NONFINITE;
            else if (a.upper && !coef_symmetric(cq, cq + 9)) pst = FEI_ERR_INVALID_ARG;
            cp = cq;
          }
          T K[9], b[3];
#pragma unroll
          for (int k = 0; k < 9; ++k) K[k] = (T)cp[k];
#pragma unroll
          for (int k = 0; k < 3; ++k) b[k] = (T)cp[9 + k];
          double s;
          if constexpr (F64) {
            const double w = sm.zw[iz] * sm.tw[t];
            const double det = dot3(sm.zn3[iz], sm.tc3[t]);
            s = w * det;
            double a0[3], a1[3];
            cross3(sm.zc2[iz], sm.tc3[t], a0);
            cross3(sm.tc3[t], sm.zc1[iz], a1);
            dt_from_adj<double>(a0, a1, sm.zn3[iz], w, s, w / det, K, b, cp[12], cp[13], D);
          } else {
            s = dot3(sm.zn3w[iz], sm.tc3w[t]);  // w det J in FP64
            const float sf = (float)s, wf = sm.zwf[iz] * sm.twf[t];
            float a0[3], a1[3];
            cross3(sm.zc2f[iz], sm.tc3f[t], a0);
            cross3(sm.tc3f[t], sm.zc1f[iz], a1);
            dt_from_adj<float>(a0, a1, sm.zn3f[iz], wf, sf, wf * wf / sf, K, b, (float)cp[12],
                               (float)cp[13], D);
          }
          pst = merge_status(pst, point_status(s));
          if (pst) atomicMax(&sm.status, pst);  // NONFINITE (4) > NEGATIVE_JACOBIAN (3)
        } else {
#pragma unroll
          for (int k = 0; k < 16; ++k) D[k] = T(0);
        }
      }
      __syncthreads();
      // operand H' for this block's rows and the table for its columns
      for (int idx = tid; idx < QC * BM; idx += 256) {
        const int qq = idx / BM, ii = idx - qq * BM;
        const int q = q0 + qq, i = rb * BM + ii, j = cb * BM + ii;
        const T *D = sm.D[qq];
        T h0 = T(0), h1 = T(0), h2 = T(0), h3 = T(0);
        if (q < NQ && i < NSH) {
          const T g0 = Gg[(size_t)(4 * q + 0) * NSH + i], g1 = Gg[(size_t)(4 * q + 1) * NSH + i];
          const T g2 = Gg[(size_t)(4 * q + 2) * NSH + i], g3 = Gg[(size_t)(4 * q + 3) * NSH + i];
          h0 = D[0] * g0;
          h1 = D[1] * g0 + D[4] * g1 + D[7] * g2 + D[10] * g3;
          h2 = D[2] * g0 + D[5] * g1 + D[8] * g2 + D[11] * g3;
          h3 = D[3] * g0 + D[6] * g1 + D[9] * g2 + D[12] * g3;
        }
        sm.H[4 * qq + 0][ii] = h0;
        sm.H[4 * qq + 1][ii] = h1;
        sm.H[4 * qq + 2][ii] = h2;
        sm.H[4 * qq + 3][ii] = h3;
#pragma unroll
        for (int c = 0; c < 4; ++c)
          sm.G[4 * qq + c][ii] = (q < NQ && j < NSH) ? Gg[(size_t)(4 * q + c) * NSH + j] : T(0);
      }
      if (cb == 0 && tid < BM && brow < NSH) {
        for (int qq = 0; qq < QC && q0 + qq < NQ; ++qq)
          bacc += sm.D[qq][13] * Gg[(size_t)(4 * (q0 + qq)) * NSH + brow];
      }
      __syncthreads();
      // steps 9-13: the double loop over shape functions as a register tile
#pragma unroll 4
      for (int k = 0; k < KC; ++k) {
        T av[RM], bvv[RM];
#pragma unroll
        for (int r = 0; r < RM; ++r) av[r] = sm.H[k][ty + 16 * r];
#pragma unroll
        for (int c = 0; c < RM; ++c) bvv[c] = sm.G[k][tx + 16 * c];
#pragma unroll
        for (int r = 0; r < RM; ++r)
#pragma unroll
          for (int c = 0; c < RM; ++c) acc[r][c] += av[r] * bvv[c];
      }
      __syncthreads();
    }
    const int st = sm.status;
    const int64_t aoff = out_a(a, item, e, NSH);
    T *A = reinterpret_cast<T *>(a.A) + aoff;
#pragma unroll
    for (int r = 0; r < RM; ++r) {
      const int i = rb * BM + ty + 16 * r;
#pragma unroll
      for (int c = 0; c < RM; ++c) {
        const int j = cb * BM + tx + 16 * c;
        if (i < NSH && j < NSH && (!a.upper || j >= i)) A[a_pos(i, j, NSH, a.upper)] = st ? T(0) : acc[r][c];
      }
    }
    if (cb == 0 && tid < BM && brow < NSH) {
      const int64_t boff = out_b(a, item, e, NSH);
      reinterpret_cast<T *>(a.bv)[boff + brow] = st ? T(0) : bacc;
    }
    if (tid == 0 && rb == 0 && cb == 0) a.status[e] = st;
    __syncthreads();
  }
}

template <typename T, int P>
fei_status launch_small(const FwdArgs &a, int64_t grid_work, cudaStream_t s, int64_t grid_cap) {
  using C = SmallCfg<T, P>;
  FEI_CUDA_TRY(cudaFuncSetAttribute(cc_small_kernel<T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM),
               "cudaFuncSetAttribute(cc_small)");
  int64_t blocks = (grid_work + C::WPB * C::EPW - 1) / (C::WPB * C::EPW);
  const int64_t cap = grid_cap > 0 ? grid_cap : (a.count ? 152 * 4 : 0);
  if (cap > 0 && blocks > cap) blocks = cap;
  if (blocks > 2147483647LL) blocks = 2147483647LL;
  if (blocks < 1) blocks = 1;
  cc_small_kernel<T, P><<<(unsigned)blocks, C::WPB * 32, C::SMEM, s>>>(a);
  FEI_CUDA_TRY(cudaGetLastError(), "cc_small_kernel launch");
  return FEI_OK;
}

template <typename T, int P>
fei_status launch_tile(const FwdArgs &a, int64_t grid_work, cudaStream_t s, int64_t grid_cap) {
  using C = TileCfg<T, P>;
  int64_t blocks = grid_work * C::NB * C::NB;
  const int64_t cap = grid_cap > 0 ? grid_cap : (a.count ? 152 * 8 : 0);
  if (cap > 0 && blocks > cap) blocks = cap;
  if (blocks > 2147483647LL) blocks = 2147483647LL;
  if (blocks < 1) blocks = 1;
  cc_tile_kernel<T, P><<<(unsigned)blocks, 256, 0, s>>>(a);
  FEI_CUDA_TRY(cudaGetLastError(), "cc_tile_kernel launch");
  return FEI_OK;
}

template <typename T>
fei_status launch_typed(int p, const FwdArgs &a, int64_t grid_work, cudaStream_t s, int64_t cap) {
  switch (p) {
    case 1:
      if constexpr (std::is_same<T, float>::value) return launch_p1(a, grid_work, s, cap);
      return launch_small<T, 1>(a, grid_work, s, cap);
    case 2: return launch_small<T, 2>(a, grid_work, s, cap);
    case 3: return launch_tile<T, 3>(a, grid_work, s, cap);
    case 4: return launch_tile<T, 4>(a, grid_work, s, cap);
    case 5: return launch_tile<T, 5>(a, grid_work, s, cap);
    case 6: return launch_tile<T, 6>(a, grid_work, s, cap);
    case 7: return launch_tile<T, 7>(a, grid_work, s, cap);
  }
  return set_error(FEI_ERR_INVALID_DEGREE, "degree %d outside 1..7", p);
}

}  // namespace

fei_status launch_cc_forward(int p, bool fp64, const FwdArgs &a, int64_t grid_work, cudaStream_t s,
                             int64_t grid_cap) {
  if (grid_work <= 0) return FEI_OK;
  return fp64 ? launch_typed<double>(p, a, grid_work, s, grid_cap)
              : launch_typed<float>(p, a, grid_work, s, grid_cap);
}

}  // namespace fei
