// fei_internal.cuh -- shared declarations of the libfei CUDA sources.
//
// Layout of the device reference data of one degree p (N_sh shape
// functions, N_q = (p+1)^3 points, Sec. 2.2 / Table 2):
//   pts   double [N_q][4]        (xi1, xi2, zeta, w)
//   G64   double [N_q][4][N_sh]  row 0 = phi, rows 1..3 = d phi / d(xi1, xi2, zeta)
//   G32   float  [N_q][4][N_sh]  the same rounded to FP32
//   G32T  float  [N_q][N_sh][4]  the same, components adjacent (one 16-byte
//                                load per point and shape function)
//   znode double [p+1][2]        (zeta, w_zeta)        vertical Gauss nodes
//   tnode double [(p+1)^2][4]    (xi1, xi2, w_tri, 0)  collapsed triangle nodes
//   point q = iz * (p+1)^2 + t, t = iv * (p+1) + iu, w_q = w_tri[t] w_zeta[iz].
//   tc    the tensor-core B operand images and paired tables (fei_tc.cu).
//   sf    FP32 1D factor tables of the sum-factorised path (fei_sf.cu).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "../../include/fei.h"

namespace fei {

constexpr int kPMax = 7;

__host__ __device__ constexpr int nsh_of(int p) { return (p + 1) * (p + 1) * (p + 2) / 2; }
__host__ __device__ constexpr int nq_of(int p) { return (p + 1) * (p + 1) * (p + 1); }
__host__ __device__ constexpr int ntri_of(int p) { return (p + 1) * (p + 2) / 2; }

struct TcImage;  // tensor-core operand image, fei_tc.cu

}  // namespace fei

struct fei_reference {
  int p, nsh, nq;
  int device;
  double *pts;
  double *G64;
  float *G32;
  double *znode;
  double *tnode;
  float *G32T;       // [N_q][N_sh][4] the FP32 table with the 4 components adjacent
  fei::TcImage *tc;  // null until built (degree >= 3)
  float *sf;         // 1D factor tables of the sum-factorised path (degree >= 3), or null
};

namespace fei {

// Arguments of every forward kernel.  A "work item" is one element; with a
// bucket list the work items are list[0 .. *count) (device count), else
// elements 0 .. n_work.
struct FwdArgs {
  int64_t n_work;
  const int32_t *count;  // device, or null
  const int32_t *list;   // device, or null
  const double *geom;
  int coef_mode;
  const double *K, *b, *c, *f;
  const int64_t *A_off, *b_off, *q_off;
  // with A_off and b_off null: 1 = work item k's outputs at k N_sh^2 and
  // k N_sh (a list written contiguously in list order), 0 = at e N_sh^2 and
  // e N_sh for element e
  int out_by_item;
  // 1: A_e as its upper triangle (FEI_A_UPPER), N_sh (N_sh + 1) / 2 values
  int upper;
  void *A;
  void *bv;
  int32_t *status;
  const double *G64;
  const float *G32;
  const double *znode;
  const double *tnode;
  const float *G32T;
};

// Values of one A_e: N_sh^2, or N_sh (N_sh + 1) / 2 in the upper layout.
__host__ __device__ __forceinline__ int64_t a_size(int64_t s, bool upper) { return upper ? s * (s + 1) / 2 : s * s; }
// Position of A_e[i][j] (j >= i in the upper layout) in the element's values.
__host__ __device__ __forceinline__ int64_t a_pos(int i, int j, int s, bool upper) {
  return upper ? (int64_t)i * s - (int64_t)i * (i + 1) / 2 + j : (int64_t)i * s + j;
}
// Start of work item k (element e) in A and in b (s = N_sh).
__device__ __forceinline__ int64_t out_a(const FwdArgs &a, int64_t k, int64_t e, int64_t s) {
  return a.A_off ? a.A_off[e] : (a.out_by_item ? k : e) * a_size(s, a.upper);
}
// FEI_A_UPPER needs a symmetric weak form: b = 0 and K = K^T exactly in
// every coefficient record (K row-major [3][3], b [3], FP64).
__device__ __forceinline__ bool coef_symmetric(const double *K, const double *b) {
  return K[1] == K[3] && K[2] == K[6] && K[5] == K[7] && b[0] == 0.0 && b[1] == 0.0 && b[2] == 0.0;
}
__device__ __forceinline__ int64_t out_b(const FwdArgs &a, int64_t k, int64_t e, int64_t s) {
  return a.b_off ? a.b_off[e] : (a.out_by_item ? k : e) * s;
}

struct BwdArgs {
  int64_t n_work;
  const int32_t *count;
  const int32_t *list;
  const double *geom;
  int coef_mode;
  const double *K, *b, *c, *f;
  const int64_t *A_off, *b_off, *q_off;
  const void *gA;
  const void *gb;
  const double *u;  // quadratic-loss adjoint: u_e at b_off[e] (else unused)
  // general adjoint with dL/dDt precomputed (FEI_FP32 chain only): gDpre
  // [n_work][N_q][16] for the work items, element e0 + item (no list)
  const float *gDpre;
  int64_t e0;
  double *g_geom;
  double *gK, *gbc, *gc, *gf;
  const double *G64;
  const float *G32;
  const double *znode;
  const double *tnode;
};

// Error reporting (fei_api.cu).
fei_status set_error(fei_status st, const char *fmt, ...);
fei_status cuda_error(cudaError_t e, const char *what);

// Argument checks and forward dispatch (fei_api.cu).  check_refs fills
// by_p[p] with the handle of degree p (or null); fill_fwd sets the
// arguments of a forward launch over the whole batch (no list).
fei_status check_refs(const fei_reference_t *refs, int nrefs, int dev, const fei_reference **by_p);
fei_status check_batch(const fei_batch *b);
void fill_fwd(FwdArgs &a, const fei_batch *b, const fei_reference *r, void *A, void *bv, int32_t *st);
fei_status launch_forward(int p, fei_precision prec, const fei_reference *r, const FwdArgs &a, int64_t grid_work,
                          cudaStream_t s);
// FEI_DEBUG set (and not "0") in the environment: every launch is followed
// by a wait on its stream and an error check, so that a failing kernel is
// reported by the call that launched it, under its name.  Skipped while the
// stream is being captured into a CUDA graph.  Off: returns FEI_OK at once.
bool debug_enabled();
fei_status debug_check(cudaStream_t s, const char *what);

// The forward of fei_integrate on checked arguments (by_p from check_refs),
// with the bucketing scratch given: counts int32 [8] and lists int32
// [7][cap], cap >= n_elem (both unused for a uniform degree).
fei_status integrate_scratch(const fei_reference *const *by_p, const fei_batch *batch, fei_precision prec,
                             void *A_out, void *b_out, int32_t *elem_status, int32_t *counts, int32_t *lists,
                             int64_t cap, cudaStream_t s);

// Kernel launchers (each returns FEI_OK or an error already recorded).
// grid_cap: largest grid (blocks) of the grid-stride kernels, 0 = default
// (all work items for a known count, 152 x 4 or 152 x 8 for a device count)
fei_status launch_cc_forward(int p, bool fp64, const FwdArgs &a, int64_t grid_work, cudaStream_t s,
                             int64_t grid_cap = 0);
// quadratic = true: the adjoint of L = sum_e u_e^T A_e u_e - u_e^T b_e
// (gA_e = u_e u_e^T and gb_e = -u_e never formed; a.u holds u)
fei_status launch_cc_backward(int p, bool fp64, const BwdArgs &a, int64_t grid_work, cudaStream_t s,
                              bool quadratic = false);
// The tensor-core precisions (split fp16 or split TF32 operands).
inline bool tc_precision(fei_precision prec) { return prec == FEI_TC_F16X3 || prec == FEI_TC_3XTF32; }
inline bool valid_precision(fei_precision prec) {
  return prec == FEI_FP64 || prec == FEI_FP32 || tc_precision(prec) || prec == FEI_SF_FP32 || prec == FEI_AUTO;
}
// The kernels of the forward: CUDA-core (fei_cc.cu), tensor-core
// (fei_tc.cu) and sum-factorised (fei_sf.cu).  The tensor-core and
// sum-factorised kernels run degrees >= 3; lower degrees of those
// precisions run the FEI_FP32 CUDA-core kernels.
enum KernelKind { KERNEL_CC = 0, KERNEL_TC = 1, KERNEL_SF = 2 };
// The kernel of degree p under prec on a direct call, and the precision it
// runs in (FEI_AUTO resolved per degree).
inline KernelKind direct_kernel(fei_precision prec, int p, fei_precision *run) {
  if (prec == FEI_AUTO) prec = p <= 2 ? FEI_FP32 : p <= 4 ? FEI_TC_F16X3 : FEI_SF_FP32;
  *run = prec;
  if (p >= 3 && tc_precision(prec)) return KERNEL_TC;
  if (p >= 3 && prec == FEI_SF_FP32) return KERNEL_SF;
  return KERNEL_CC;
}
fei_status launch_sf_forward(int p, const fei_reference *ref, const FwdArgs &a, int64_t grid_work, cudaStream_t s,
                             int64_t grid_cap = 0);
fei_status build_sf_tables(fei_reference *ref);
void free_sf_tables(fei_reference *ref);
// variant: 0 .. tc_variant_count(p, prec) - 1 (warp-role variants of one
// kernel); prec: FEI_TC_F16X3 or FEI_TC_3XTF32
fei_status launch_tc_forward(int p, const fei_reference *ref, const FwdArgs &a, int64_t grid_work,
                             cudaStream_t s, int variant, fei_precision prec);
int tc_variant_count(int p, fei_precision prec);
// Tensor-core adjoint (fei_tc.cu, p = 3..5, uniform degree): gD [count][N_q]
// [16] = dL/dDt_q of the elements e0 .. e0 + count - 1, from gA (FP32, at
// A_off[e] or e N_sh^2) with W^T = G gA^T on the tensor cores (split fp16).
bool tc_adjoint_ready(const fei_reference *ref);  // degree 3..5 and its image built
fei_status launch_tc_adjoint(int p, const fei_reference *ref, const float *gA, const int64_t *A_off, int64_t e0,
                             int64_t count, float *gD, cudaStream_t s);
fei_status build_tc_image(fei_reference *ref);
void free_tc_image(fei_reference *ref);

}  // namespace fei

namespace fei {

// NVTX range over a host entry point: visible in a profiler's timeline,
// a no-op when no tool is attached (NVTX v3, header only).
struct Range {
  explicit Range(const char *name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range &) = delete;
  Range &operator=(const Range &) = delete;
};

}  // namespace fei

#define FEI_CUDA_TRY(call, what)                               \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return ::fei::cuda_error(e_, what); \
  } while (0)
