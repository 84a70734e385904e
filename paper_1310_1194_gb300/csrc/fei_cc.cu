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
    ok &= isfinite(cd[k]);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    cd[9 + k] = a.b[3 * r + k];
    ok &= isfinite(cd[9 + k]);
  }
  cd[12] = a.c[r];
  cd[13] = a.f[r];
  ok &= isfinite(cd[12]) && isfinite(cd[13]);
  return ok;
}

// Point operator directly from the element vectors (no node caching).
template <typename T>
__device__ __forceinline__ int point_direct(const double *ev, const double *pt, const double *cd,
                                            T *D) {
  double c1[3], c2[3], n3[3], c3[3];
  znode_columns(ev, pt[2], c1, c2, n3);
  tnode_column(ev, pt[0], pt[1], c3);
  const double w = pt[3];
  const double det = dot3(n3, c3);
  const double s = w * det;
  T K[9], b[3];
#pragma unroll
  for (int k = 0; k < 9; ++k) K[k] = (T)cd[k];
#pragma unroll
  for (int k = 0; k < 3; ++k) b[k] = (T)cd[9 + k];
  if constexpr (std::is_same<T, double>::value) {
    double a0[3], a1[3];
    cross3(c2, c3, a0);
    cross3(c3, c1, a1);
    dt_from_adj<double>(a0, a1, n3, w, s, w / det, K, b, cd[12], cd[13], D);
  } else {
    float f1[3], f2[3], f3[3], fn[3], a0[3], a1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      f1[k] = (float)c1[k];
      f2[k] = (float)c2[k];
      f3[k] = (float)c3[k];
      fn[k] = (float)n3[k];
    }
    cross3(f2, f3, a0);
    cross3(f3, f1, a1);
    const float wf = (float)w, sf = (float)s;
    dt_from_adj<float>(a0, a1, fn, wf, sf, wf * wf / sf, K, b, (float)cd[12], (float)cd[13], D);
  }
  return point_status(s);
}

// ---------------------------------------------------------------------------
// Low degree (p <= 2): one warp per element, lanes over the entries of A_e.
// ---------------------------------------------------------------------------

template <typename T, int P>
struct SmallCfg {
  static constexpr int NSH = nsh_of(P), NQ = nq_of(P), K4 = 4 * NQ;
  static constexpr int WPB = std::is_same<T, double>::value ? 4 : 8;
  static constexpr int WARP_BYTES =
      ((sizeof(double) * (18 + 21 + 14) + sizeof(T) * (NQ * 16 + K4 * NSH) + 16 + 15) / 16) * 16;
  static constexpr int SMEM = sizeof(T) * K4 * NSH + WPB * WARP_BYTES + 16;
};

template <typename T, int P>
__global__ void __launch_bounds__(SmallCfg<T, P>::WPB * 32) cc_small_kernel(FwdArgs a) {
  using C = SmallCfg<T, P>;
  constexpr int NSH = C::NSH, NQ = C::NQ, K4 = C::K4;
  static_assert(NQ <= 32, "one point per lane");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *Gs = reinterpret_cast<T *>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char *wb = smem_raw + ((sizeof(T) * K4 * NSH + 15) / 16) * 16 + warp * C::WARP_BYTES;
  double *X = reinterpret_cast<double *>(wb);
  double *ev = X + 18;
  double *cd = ev + 21;
  T *D = reinterpret_cast<T *>(cd + 14);
  T *H = D + NQ * 16;

  const T *G = gtab<T>(a);
  for (int k = threadIdx.x; k < K4 * NSH; k += blockDim.x) Gs[k] = G[k];
  __syncthreads();

  const int64_t items = n_items(a);
  for (int64_t item = (int64_t)blockIdx.x * C::WPB + warp; item < items;
       item += (int64_t)gridDim.x * C::WPB) {
    const int64_t e = a.list ? (int64_t)a.list[item] : item;
    bool ok = true;
    if (lane < 18) {
      X[lane] = a.geom[18 * e + lane];
      ok = isfinite(X[lane]);
    }
    if (a.coef_mode == FEI_COEF_PER_ELEMENT && lane == 0) ok &= load_coef(a, e, cd);
    int st = __any_sync(0xffffffffu, !ok) ? FEI_ERR_NONFINITE : 0;
    __syncwarp();
    if (lane == 0) elem_vectors(X, ev);
    __syncwarp();
    int pst = 0;
    if (lane < NQ) {
      double ptv[4];
      // quadrature point from the node tables: q = iz*(p+1)^2 + t
      const int iz = lane / ((P + 1) * (P + 1)), t = lane % ((P + 1) * (P + 1));
      ptv[0] = a.tnode[4 * t];
      ptv[1] = a.tnode[4 * t + 1];
      ptv[2] = a.znode[2 * iz];
      ptv[3] = a.tnode[4 * t + 2] * a.znode[2 * iz + 1];
      double cq[14];
      const double *cp = cd;
      if (a.coef_mode == FEI_COEF_PER_POINT) {
        const int64_t r = (a.q_off ? a.q_off[e] : e * (int64_t)NQ) + lane;
        if (!load_coef(a, r, cq)) pst = FEI_ERR_NONFINITE;
        cp = cq;
      }
      pst = merge_status(pst, point_direct<T>(ev, ptv, cp, D + 16 * lane));
    }
    // warp-wide status with NONFINITE precedence
    if (__any_sync(0xffffffffu, pst == FEI_ERR_NONFINITE)) st = FEI_ERR_NONFINITE;
    else if (!st && __any_sync(0xffffffffu, pst == FEI_ERR_NEGATIVE_JACOBIAN)) st = FEI_ERR_NEGATIVE_JACOBIAN;
    __syncwarp();
    for (int idx = lane; idx < NQ * NSH; idx += 32) {
      const int q = idx / NSH, i = idx - q * NSH;
      const T *Dq = D + 16 * q;
      const T g0 = Gs[(4 * q + 0) * NSH + i], g1 = Gs[(4 * q + 1) * NSH + i];
      const T g2 = Gs[(4 * q + 2) * NSH + i], g3 = Gs[(4 * q + 3) * NSH + i];
      H[(4 * q + 0) * NSH + i] = Dq[0] * g0;
#pragma unroll
      for (int m = 0; m < 3; ++m)
        H[(4 * q + 1 + m) * NSH + i] = Dq[1 + m] * g0 + Dq[4 + m] * g1 + Dq[7 + m] * g2 + Dq[10 + m] * g3;
    }
    __syncwarp();
    const int64_t aoff = a.A_off ? a.A_off[e] : e * (int64_t)(NSH * NSH);
    const int64_t boff = a.b_off ? a.b_off[e] : e * (int64_t)NSH;
    T *A = reinterpret_cast<T *>(a.A) + aoff;
    T *bv = reinterpret_cast<T *>(a.bv) + boff;
    for (int idx = lane; idx < NSH * NSH; idx += 32) {
      const int i = idx / NSH, j = idx - i * NSH;
      T acc = T(0);
#pragma unroll 4
      for (int k = 0; k < K4; ++k) acc += H[k * NSH + i] * Gs[k * NSH + j];
      A[idx] = st ? T(0) : acc;
    }
    for (int i = lane; i < NSH; i += 32) {
      T acc = T(0);
      for (int q = 0; q < NQ; ++q) acc += D[16 * q + 13] * Gs[(4 * q) * NSH + i];
      bv[i] = st ? T(0) : acc;
    }
    if (lane == 0) a.status[e] = st;
    __syncwarp();
  }
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
      ok = isfinite(sm.X[tid]);
    }
    if (a.coef_mode == FEI_COEF_PER_ELEMENT && tid == 32) ok = load_coef(a, e, sm.cd);
    if (!ok) sm.status = FEI_ERR_NONFINITE;
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
    const int64_t aoff = a.A_off ? a.A_off[e] : e * (int64_t)(NSH * NSH);
    T *A = reinterpret_cast<T *>(a.A) + aoff;
#pragma unroll
    for (int r = 0; r < RM; ++r) {
      const int i = rb * BM + ty + 16 * r;
#pragma unroll
      for (int c = 0; c < RM; ++c) {
        const int j = cb * BM + tx + 16 * c;
        if (i < NSH && j < NSH) A[(size_t)i * NSH + j] = st ? T(0) : acc[r][c];
      }
    }
    if (cb == 0 && tid < BM && brow < NSH) {
      const int64_t boff = a.b_off ? a.b_off[e] : e * (int64_t)NSH;
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
  int64_t blocks = (grid_work + C::WPB - 1) / C::WPB;
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
    case 1: return launch_small<T, 1>(a, grid_work, s, cap);
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
