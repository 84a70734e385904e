// fei_api.cu -- the C ABI entry points: validation, dispatch, bucketing.
//
// The batch of Algorithm 1 ("for ielem = 1 to nr_elems_in_subset") is a set
// of independent elements (Sec. 2: integration is embarrassingly parallel).
// Elements of one degree share the reference tables (Sec. 2.2: "elements
// are grouped into sets of elements with the same type and degree"), so a
// mixed-degree batch is first bucketed by degree on the device (a counting
// pass with one atomic per element), then one persistent kernel per degree
// walks its bucket.  Every element still writes to its own offsets, so the
// processing order does not change any output bit.
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>

#include "fei_internal.cuh"

namespace fei {

static thread_local char g_err[512] = "no error";

fei_status set_error(fei_status st, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

fei_status cuda_error(cudaError_t e, const char *what) {
  return set_error(e == cudaErrorMemoryAllocation ? FEI_ERR_OOM : FEI_ERR_CUDA, "%s: %s (%s)", what,
                   cudaGetErrorName(e), cudaGetErrorString(e));
}

namespace {

// Bucket workspace of one device: counts[8] and lists[7][capacity].
struct Workspace {
  int32_t *counts = nullptr;
  int32_t *lists = nullptr;
  int64_t capacity = 0;
};
std::mutex g_ws_mutex;
Workspace g_ws[64];

fei_status workspace_for(int dev, int64_t n, Workspace **out) {
  if (dev < 0 || dev >= 64) return set_error(FEI_ERR_UNSUPPORTED, "device ordinal %d", dev);
  std::lock_guard<std::mutex> lock(g_ws_mutex);
  Workspace &w = g_ws[dev];
  if (w.capacity < n) {
    if (w.counts) cudaFree(w.counts);
    if (w.lists) cudaFree(w.lists);
    w.counts = nullptr;
    w.lists = nullptr;
    w.capacity = 0;
    FEI_CUDA_TRY(cudaMalloc(&w.counts, sizeof(int32_t) * 8), "cudaMalloc(bucket counts)");
    FEI_CUDA_TRY(cudaMalloc(&w.lists, sizeof(int32_t) * 7 * (size_t)n), "cudaMalloc(bucket lists)");
    w.capacity = n;
  }
  *out = &w;
  return FEI_OK;
}

// One atomic per element into the bucket of its degree; elements whose
// degree has no reference (avail bit clear) or lies outside 1..7 get
// FEI_ERR_INVALID_DEGREE in their status and no bucket.
__global__ void bucket_kernel(const int32_t *degree, int64_t n, unsigned avail, int32_t *counts,
                              int32_t *lists, int64_t cap, int32_t *status) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int p = degree[e];
    if (p >= 1 && p <= kPMax && ((avail >> p) & 1u)) {
      const int pos = atomicAdd(&counts[p], 1);
      lists[(int64_t)(p - 1) * cap + pos] = (int32_t)e;
    } else if (status) {
      status[e] = FEI_ERR_INVALID_DEGREE;
    }
  }
}

// Single-block exclusive scan of N_sh^2, N_sh and N_q over the degrees.
__global__ void __launch_bounds__(1024) offsets_kernel(const int32_t *degree, int64_t n, int upper, int64_t *Ao,
                                                        int64_t *bo, int64_t *qo, int32_t *bad) {
  __shared__ int64_t sA[1024], sb[1024], sq[1024];
  __shared__ int32_t sbad;
  const int t = threadIdx.x, T = blockDim.x;
  if (t == 0) sbad = 0;
  const int64_t chunk = (n + T - 1) / T;
  const int64_t e0 = t * chunk, e1 = (e0 + chunk < n) ? e0 + chunk : n;
  int64_t a = 0, b = 0, q = 0;
  int nbad = 0;
  for (int64_t e = e0; e < e1; ++e) {
    int p = degree[e];
    if (p < 1 || p > kPMax) {
      ++nbad;
      p = 0;
      continue;
    }
    const int64_t s = nsh_of(p);
    a += a_size(s, upper);
    b += s;
    q += nq_of(p);
  }
  sA[t] = a;
  sb[t] = b;
  sq[t] = q;
  __syncthreads();
  if (nbad) atomicAdd(&sbad, nbad);
  // Hillis-Steele inclusive scan over the per-thread sums
  for (int off = 1; off < T; off <<= 1) {
    int64_t va = 0, vb = 0, vq = 0;
    if (t >= off) {
      va = sA[t - off];
      vb = sb[t - off];
      vq = sq[t - off];
    }
    __syncthreads();
    sA[t] += va;
    sb[t] += vb;
    sq[t] += vq;
    __syncthreads();
  }
  a = sA[t] - a;
  b = sb[t] - b;
  q = sq[t] - q;
  for (int64_t e = e0; e < e1; ++e) {
    if (Ao) Ao[e] = a;
    if (bo) bo[e] = b;
    if (qo) qo[e] = q;
    const int p = degree[e];
    if (p >= 1 && p <= kPMax) {
      const int64_t s = nsh_of(p);
      a += a_size(s, upper);
      b += s;
      q += nq_of(p);
    }
  }
  if (t == T - 1) {
    if (Ao) Ao[n] = sA[t];
    if (bo) bo[n] = sb[t];
    if (qo) qo[n] = sq[t];
  }
  __syncthreads();
  if (t == 0 && bad) *bad = sbad;
}

}  // namespace

// Argument checks and the per-degree forward launch, shared with the
// assembly entry points (fei_assembly.cu).
fei_status check_refs(const fei_reference_t *refs, int nrefs, int dev, const fei_reference **by_p) {
  if (!refs || nrefs < 1) return set_error(FEI_ERR_INVALID_ARG, "refs is NULL or nrefs < 1");
  for (int p = 0; p <= kPMax; ++p) by_p[p] = nullptr;
  for (int k = 0; k < nrefs; ++k) {
    const fei_reference *r = refs[k];
    if (!r) return set_error(FEI_ERR_INVALID_ARG, "refs[%d] is NULL", k);
    if (r->device != dev)
      return set_error(FEI_ERR_INVALID_ARG, "refs[%d] was created on device %d, current device is %d", k,
                       r->device, dev);
    by_p[r->p] = r;
  }
  return FEI_OK;
}

fei_status check_batch(const fei_batch *b) {
  if (!b) return set_error(FEI_ERR_INVALID_ARG, "batch is NULL");
  if (b->n_elem < 0 || b->n_elem > 2147483647LL)
    return set_error(FEI_ERR_INVALID_ARG, "n_elem %lld outside 0..2^31-1", (long long)b->n_elem);
  if (b->n_elem == 0) return FEI_OK;
  if (!b->geom || !b->K || !b->b || !b->c || !b->f)
    return set_error(FEI_ERR_INVALID_ARG, "batch geometry/coefficient pointer is NULL");
  if (b->coef_mode != FEI_COEF_PER_ELEMENT && b->coef_mode != FEI_COEF_PER_POINT)
    return set_error(FEI_ERR_INVALID_ARG, "coef_mode %d", b->coef_mode);
  if (b->a_layout != FEI_A_FULL && b->a_layout != FEI_A_UPPER)
    return set_error(FEI_ERR_INVALID_ARG, "a_layout %d", b->a_layout);
  if (b->degree) {
    if (!b->A_offset || !b->b_offset || (b->coef_mode == FEI_COEF_PER_POINT && !b->q_offset))
      return set_error(FEI_ERR_INVALID_ARG, "a degree array needs A_offset, b_offset (and q_offset per point)");
  } else if (b->uniform_degree < 1 || b->uniform_degree > kPMax) {
    return set_error(FEI_ERR_INVALID_DEGREE, "uniform_degree %d outside 1..7", b->uniform_degree);
  }
  return FEI_OK;
}

void fill_fwd(FwdArgs &a, const fei_batch *b, const fei_reference *r, void *A, void *bv, int32_t *st) {
  memset(&a, 0, sizeof(a));
  a.n_work = b->n_elem;
  a.geom = b->geom;
  a.coef_mode = b->coef_mode;
  a.K = b->K;
  a.b = b->b;
  a.c = b->c;
  a.f = b->f;
  a.A_off = b->A_offset;
  a.b_off = b->b_offset;
  a.q_off = b->q_offset;
  a.upper = b->a_layout == FEI_A_UPPER;
  a.A = A;
  a.bv = bv;
  a.status = st;
  a.G64 = r->G64;
  a.G32 = r->G32;
  a.znode = r->znode;
  a.tnode = r->tnode;
  a.G32T = r->G32T;
}

fei_status launch_forward(int p, fei_precision prec, const fei_reference *r, const FwdArgs &a,
                          int64_t grid_work, cudaStream_t s) {
  fei_precision run;
  const KernelKind k = direct_kernel(prec, p, &run);
  const fei_status st = k == KERNEL_TC   ? launch_tc_forward(p, r, a, grid_work, s, 0, run)
                        : k == KERNEL_SF ? launch_sf_forward(p, r, a, grid_work, s)
                                         : launch_cc_forward(p, run == FEI_FP64, a, grid_work, s);
  return st ? st : debug_check(s, "forward kernel");
}

bool debug_enabled() {
  static const bool on = [] {
    const char *v = getenv("FEI_DEBUG");
    return v != nullptr && *v != '\0' && strcmp(v, "0") != 0;
  }();
  return on;
}

fei_status debug_check(cudaStream_t s, const char *what) {
  if (!debug_enabled()) return FEI_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  FEI_CUDA_TRY(cudaStreamIsCapturing(s, &cs), "cudaStreamIsCapturing");
  if (cs != cudaStreamCaptureStatusNone) return FEI_OK;
  FEI_CUDA_TRY(cudaGetLastError(), what);
  FEI_CUDA_TRY(cudaStreamSynchronize(s), what);
  return FEI_OK;
}

}  // namespace fei

using namespace fei;

extern "C" const char *fei_last_error_string(void) { return g_err; }

namespace fei {
namespace {

// Rank of a status for the summary: NONFINITE > NEGATIVE_JACOBIAN > other
// nonzero codes > OK.
__device__ __forceinline__ int status_rank(int st) {
  return st == FEI_ERR_NONFINITE ? 3 : st == FEI_ERR_NEGATIVE_JACOBIAN ? 2 : st != 0 ? 1 : 0;
}

// summary[0] = worst status, summary[1] = count of nonzero statuses; one
// block, so no second pass and no host work.
__global__ void __launch_bounds__(1024) status_summary_kernel(const int32_t *st, int64_t n, int32_t *summary) {
  __shared__ int s_rank, s_code, s_count;
  if (threadIdx.x == 0) {
    s_rank = 0;
    s_code = 0;
    s_count = 0;
  }
  __syncthreads();
  int best_rank = 0, best_code = 0, count = 0;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
    const int v = st[e];
    const int r = status_rank(v);
    if (r > best_rank || (r == best_rank && v > best_code)) {
      best_rank = r;
      best_code = v;
    }
    count += v != 0;
  }
  atomicAdd(&s_count, count);
  atomicMax(&s_rank, best_rank);
  __syncthreads();
  if (best_rank == s_rank) atomicMax(&s_code, best_code);
  __syncthreads();
  if (threadIdx.x == 0) {
    summary[0] = s_code;
    summary[1] = s_count;
  }
}

}  // namespace
}  // namespace fei

extern "C" fei_status fei_status_summary(const int32_t *elem_status, int64_t n_elem, int32_t *summary,
                                         fei_stream_t stream) {
  if (n_elem < 0) return set_error(FEI_ERR_INVALID_ARG, "fei_status_summary: n_elem < 0");
  if (!summary) {
    if (n_elem == 0) return FEI_OK;
    return set_error(FEI_ERR_INVALID_ARG, "fei_status_summary: summary is NULL");
  }
  if (!elem_status && n_elem > 0) return set_error(FEI_ERR_INVALID_ARG, "fei_status_summary: elem_status is NULL");
  status_summary_kernel<<<1, 1024, 0, (cudaStream_t)stream>>>(elem_status, n_elem, summary);
  FEI_CUDA_TRY(cudaGetLastError(), "status_summary_kernel launch");
  return FEI_OK;
}

namespace fei {
namespace {

// The summary word fei_sync_status reads back: [worst, count] per device
// (a __device__ array exists once on every device), written by the summary
// kernel; calls on one device are serialised by the mutex.
static __device__ int32_t g_sync_summary[2];
std::mutex g_sync_mutex[64];
int32_t *g_sync_ptr[64];

}  // namespace
}  // namespace fei

extern "C" fei_status fei_sync_status(const int32_t *elem_status, int64_t n_elem, int32_t *worst, int64_t *count,
                                      fei_stream_t stream) {
  const Range range_("fei_sync_status");
  if (n_elem < 0) return set_error(FEI_ERR_INVALID_ARG, "fei_sync_status: n_elem < 0");
  if (!worst || !count) return set_error(FEI_ERR_INVALID_ARG, "fei_sync_status: worst and count are required");
  if (!elem_status && n_elem > 0) return set_error(FEI_ERR_INVALID_ARG, "fei_sync_status: elem_status is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if (n_elem == 0) {
    FEI_CUDA_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    *worst = 0;
    *count = 0;
    return FEI_OK;
  }
  int dev;
  FEI_CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev < 0 || dev >= 64) return set_error(FEI_ERR_UNSUPPORTED, "device ordinal %d", dev);
  std::lock_guard<std::mutex> lock(g_sync_mutex[dev]);
  if (!g_sync_ptr[dev]) {
    void *ptr = nullptr;
    FEI_CUDA_TRY(cudaGetSymbolAddress(&ptr, g_sync_summary), "cudaGetSymbolAddress(status summary)");
    g_sync_ptr[dev] = static_cast<int32_t *>(ptr);
  }
  status_summary_kernel<<<1, 1024, 0, s>>>(elem_status, n_elem, g_sync_ptr[dev]);
  FEI_CUDA_TRY(cudaGetLastError(), "status_summary_kernel launch");
  int32_t h[2] = {0, 0};
  FEI_CUDA_TRY(cudaMemcpyAsync(h, g_sync_ptr[dev], sizeof(h), cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync(summary)");
  FEI_CUDA_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  *worst = h[0];
  *count = h[1];
  return FEI_OK;
}

namespace fei {
namespace {
fei_status plan_offsets(const char *who, const int32_t *degree, int64_t n_elem, int upper, int64_t *A_offset,
                        int64_t *b_offset, int64_t *q_offset, int32_t *bad_count, fei_stream_t stream) {
  if (!degree && n_elem > 0) return set_error(FEI_ERR_INVALID_ARG, "%s: degree is NULL", who);
  if (n_elem < 0) return set_error(FEI_ERR_INVALID_ARG, "%s: n_elem < 0", who);
  if (!A_offset && !b_offset && !q_offset && !bad_count) return FEI_OK;
  offsets_kernel<<<1, 1024, 0, (cudaStream_t)stream>>>(degree, n_elem, upper, A_offset, b_offset, q_offset,
                                                        bad_count);
  FEI_CUDA_TRY(cudaGetLastError(), "offsets_kernel launch");
  return FEI_OK;
}
}  // namespace
}  // namespace fei

extern "C" fei_status fei_plan_offsets(const int32_t *degree, int64_t n_elem, int64_t *A_offset,
                                       int64_t *b_offset, int64_t *q_offset, int32_t *bad_count,
                                       fei_stream_t stream) {
  return plan_offsets("fei_plan_offsets", degree, n_elem, 0, A_offset, b_offset, q_offset, bad_count, stream);
}

extern "C" fei_status fei_plan_offsets_upper(const int32_t *degree, int64_t n_elem, int64_t *A_offset,
                                             int64_t *b_offset, int64_t *q_offset, int32_t *bad_count,
                                             fei_stream_t stream) {
  return plan_offsets("fei_plan_offsets_upper", degree, n_elem, 1, A_offset, b_offset, q_offset, bad_count,
                      stream);
}

namespace fei {

fei_status integrate_scratch(const fei_reference *const *by_p, const fei_batch *batch, fei_precision prec,
                             void *A_out, void *b_out, int32_t *elem_status, int32_t *counts, int32_t *lists,
                             int64_t cap, cudaStream_t s) {
  if (!batch->degree) {
    const int p = batch->uniform_degree;
    if (!by_p[p]) return set_error(FEI_ERR_INVALID_DEGREE, "no reference for degree %d", p);
    FwdArgs a;
    fill_fwd(a, batch, by_p[p], A_out, b_out, elem_status);
    return launch_forward(p, prec, by_p[p], a, batch->n_elem, s);
  }
  unsigned avail = 0;
  for (int p = 1; p <= kPMax; ++p)
    if (by_p[p]) avail |= 1u << p;
  FEI_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(int32_t) * 8, s), "cudaMemsetAsync(bucket counts)");
  int64_t blocks = (batch->n_elem + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  bucket_kernel<<<(unsigned)blocks, 256, 0, s>>>(batch->degree, batch->n_elem, avail, counts, lists, cap,
                                                  elem_status);
  FEI_CUDA_TRY(cudaGetLastError(), "bucket_kernel launch");
  fei_status st0 = debug_check(s, "bucket_kernel");
  if (st0) return st0;
  for (int p = 1; p <= kPMax; ++p) {
    if (!by_p[p]) continue;
    FwdArgs a;
    fill_fwd(a, batch, by_p[p], A_out, b_out, elem_status);
    a.count = counts + p;
    a.list = lists + (int64_t)(p - 1) * cap;
    const fei_status st = launch_forward(p, prec, by_p[p], a, batch->n_elem, s);
    if (st) return st;
  }
  return FEI_OK;
}

}  // namespace fei

extern "C" fei_status fei_integrate(const fei_reference_t *refs, int nrefs, const fei_batch *batch,
                                    fei_precision prec, void *A_out, void *b_out, int32_t *elem_status,
                                    fei_stream_t stream) {
  const Range range_("fei_integrate");
  fei_status st = check_batch(batch);
  if (st) return st;
  if (!valid_precision(prec))
    return set_error(FEI_ERR_INVALID_ARG, "precision %d", (int)prec);
  if (batch->n_elem == 0) return FEI_OK;
  if (!A_out || !b_out || !elem_status) return set_error(FEI_ERR_INVALID_ARG, "A_out, b_out and elem_status are required");
  int dev;
  FEI_CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
  const fei_reference *by_p[kPMax + 1];
  st = check_refs(refs, nrefs, dev, by_p);
  if (st) return st;
  Workspace *ws = nullptr;
  if (batch->degree) {
    st = workspace_for(dev, batch->n_elem, &ws);
    if (st) return st;
  }
  return integrate_scratch(by_p, batch, prec, A_out, b_out, elem_status, ws ? ws->counts : nullptr,
                           ws ? ws->lists : nullptr, ws ? ws->capacity : 0, (cudaStream_t)stream);
}

namespace fei {
namespace {

// Shared by the general adjoint (gA, gb given) and the quadratic-loss
// adjoint (u given, gA = u u^T and gb = -u implied).
// elements per launch pair of the tensor-core adjoint (its scratch: 64 N_q
// bytes per element, 14 MB per 1024 elements at p = 5); FEI_ADJOINT_CHUNK
// in the environment (a positive integer) overrides it
int64_t adjoint_chunk() {
  const char *v = getenv("FEI_ADJOINT_CHUNK");
  const long long c = v ? atoll(v) : 0;
  return c > 0 ? (int64_t)c : 8192;
}

fei_status backward_impl(const char *who, const fei_reference_t *refs, int nrefs, const fei_batch *batch,
                         fei_precision prec, const void *gA, const void *gb, const double *u, double *g_geom,
                         const fei_coef_grad *g_coef, fei_stream_t stream) {
  const Range range_(who);
  const bool quad = u != nullptr;
  fei_status st = check_batch(batch);
  if (st) return st;
  if (!valid_precision(prec)) return set_error(FEI_ERR_INVALID_ARG, "%s: precision %d", who, (int)prec);
  // FEI_TC_F16X3 (and FEI_AUTO): W on the tensor cores for a uniform degree
  // 3..5 and the general adjoint; every other case of a precision other
  // than FEI_FP64 runs the FEI_FP32 adjoint
  const bool want_tc = prec == FEI_TC_F16X3 || prec == FEI_AUTO;
  if (batch->a_layout != FEI_A_FULL)
    return set_error(FEI_ERR_UNSUPPORTED, "%s: the adjoint takes the full A_e layout", who);
  if (batch->n_elem == 0) return FEI_OK;
  if ((!quad && (!gA || !gb)) || !g_geom || !g_coef || !g_coef->K || !g_coef->b || !g_coef->c || !g_coef->f)
    return set_error(FEI_ERR_INVALID_ARG, "%s: NULL gradient pointer", who);
  int dev;
  FEI_CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
  const fei_reference *by_p[kPMax + 1];
  st = check_refs(refs, nrefs, dev, by_p);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  BwdArgs a;
  memset(&a, 0, sizeof(a));
  a.n_work = batch->n_elem;
  a.geom = batch->geom;
  a.coef_mode = batch->coef_mode;
  a.K = batch->K;
  a.b = batch->b;
  a.c = batch->c;
  a.f = batch->f;
  a.A_off = batch->A_offset;
  a.b_off = batch->b_offset;
  a.q_off = batch->q_offset;
  a.gA = gA;
  a.gb = gb;
  a.u = u;
  a.g_geom = g_geom;
  a.gK = g_coef->K;
  a.gbc = g_coef->b;
  a.gc = g_coef->c;
  a.gf = g_coef->f;
  if (!batch->degree) {
    const int p = batch->uniform_degree;
    const fei_reference *r = by_p[p];
    if (!r) return set_error(FEI_ERR_INVALID_DEGREE, "no reference for degree %d", p);
    a.G64 = r->G64;
    a.G32 = r->G32;
    a.znode = r->znode;
    a.tnode = r->tnode;
    if (want_tc && !quad && tc_adjoint_ready(r)) {
      // dL/dDt of a chunk of elements on the tensor cores into a scratch
      // array (stream-ordered allocation), then the FP32 chain reads it
      const int64_t n = batch->n_elem, cmax = adjoint_chunk(), chunk = n < cmax ? n : cmax;
      float *gDs = nullptr;
      FEI_CUDA_TRY(cudaMallocAsync((void **)&gDs, sizeof(float) * (size_t)chunk * r->nq * 16, s),
                   "cudaMallocAsync(adjoint scratch)");
      for (int64_t e0 = 0; e0 < n && !st; e0 += chunk) {
        const int64_t cnt = n - e0 < chunk ? n - e0 : chunk;
        st = launch_tc_adjoint(p, r, reinterpret_cast<const float *>(gA), batch->A_offset, e0, cnt, gDs, s);
        if (!st) st = debug_check(s, "tensor-core adjoint kernel");
        if (st) break;
        BwdArgs ac = a;
        ac.n_work = cnt;
        ac.e0 = e0;
        ac.gDpre = gDs;
        st = launch_cc_backward(p, false, ac, cnt, s, false);
        if (!st) st = debug_check(s, "backward kernel");
      }
      const cudaError_t fe = cudaFreeAsync(gDs, s);
      if (st) return st;
      FEI_CUDA_TRY(fe, "cudaFreeAsync(adjoint scratch)");
      return FEI_OK;
    }
    st = launch_cc_backward(p, prec == FEI_FP64, a, batch->n_elem, s, quad);
    return st ? st : debug_check(s, "backward kernel");
  }
  Workspace *ws;
  st = workspace_for(dev, batch->n_elem, &ws);
  if (st) return st;
  unsigned avail = 0;
  for (int p = 1; p <= kPMax; ++p)
    if (by_p[p]) avail |= 1u << p;
  // the backward has no status output; elements of a degree without a
  // reference are skipped (their gradients are left untouched)
  FEI_CUDA_TRY(cudaMemsetAsync(ws->counts, 0, sizeof(int32_t) * 8, s), "cudaMemsetAsync(bucket counts)");
  int64_t blocks = (batch->n_elem + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  bucket_kernel<<<(unsigned)blocks, 256, 0, s>>>(batch->degree, batch->n_elem, avail, ws->counts, ws->lists,
                                                  ws->capacity, nullptr);
  FEI_CUDA_TRY(cudaGetLastError(), "bucket_kernel launch");
  for (int p = 1; p <= kPMax; ++p) {
    const fei_reference *r = by_p[p];
    if (!r) continue;
    BwdArgs ap = a;
    ap.G64 = r->G64;
    ap.G32 = r->G32;
    ap.znode = r->znode;
    ap.tnode = r->tnode;
    ap.count = ws->counts + p;
    ap.list = ws->lists + (int64_t)(p - 1) * ws->capacity;
    st = launch_cc_backward(p, prec == FEI_FP64, ap, batch->n_elem, s, quad);
    if (!st) st = debug_check(s, "backward kernel");
    if (st) return st;
  }
  return FEI_OK;
}

}  // namespace
}  // namespace fei

extern "C" fei_status fei_integrate_backward(const fei_reference_t *refs, int nrefs, const fei_batch *batch,
                                             fei_precision prec, const void *gA, const void *gb,
                                             double *g_geom, const fei_coef_grad *g_coef,
                                             fei_stream_t stream) {
  if (!gA || !gb) {
    if (batch && batch->n_elem == 0) return FEI_OK;
    return set_error(FEI_ERR_INVALID_ARG, "fei_integrate_backward: NULL gradient pointer");
  }
  return backward_impl("fei_integrate_backward", refs, nrefs, batch, prec, gA, gb, nullptr, g_geom, g_coef,
                       stream);
}

extern "C" fei_status fei_integrate_backward_quadratic(const fei_reference_t *refs, int nrefs,
                                                       const fei_batch *batch, fei_precision prec,
                                                       const double *u, double *g_geom,
                                                       const fei_coef_grad *g_coef, fei_stream_t stream) {
  if (!u) {
    if (batch && batch->n_elem == 0) return FEI_OK;
    return set_error(FEI_ERR_INVALID_ARG, "fei_integrate_backward_quadratic: u is NULL");
  }
  return backward_impl("fei_integrate_backward_quadratic", refs, nrefs, batch, prec, nullptr, nullptr, u, g_geom,
                       g_coef, stream);
}
