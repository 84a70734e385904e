// fei_noalloc.cu -- fei_integrate_noalloc: the mixed-degree forward pass
// with its bucketing scratch in a fixed device array instead of memory that
// the library allocates.
//
// fei_integrate sorts a batch with a degree array into per-degree element
// lists before it launches one kernel per degree; those lists and their
// counts are scratch memory, which fei_integrate allocates (once per device,
// grown on demand) with cudaMalloc.  Some callers cannot let a library call
// cudaMalloc: code that runs while a stream is being captured into a CUDA
// graph (an allocation there is not allowed), code that must never block
// the device (cudaMalloc can synchronise), and applications whose device
// memory is owned by a pool or budget the library must not bypass.  This
// entry point serves them: its scratch is the file-scope array below,
// reserved on every GPU that loads the library until the process exits, and
// it calls no allocating routine at all.
//
// Limits and sharing:
//  - at most FEI_NOALLOC_MAX_ELEM elements per call (larger batches are
//    rejected with FEI_ERR_INVALID_ARG);
//  - every call on a device uses the same array and leaves its contents
//    behind; the call clears the per-degree counts itself before bucketing,
//    but two calls whose work overlaps on the GPU (different streams without
//    ordering between them) race on the array and give wrong results;
//  - the first call on a device looks up the array's device address
//    (cudaGetSymbolAddress) -- make that first call before any stream
//    capture begins.
#include <string.h>

#include <mutex>

#include "fei_internal.cuh"

namespace fei {
namespace {

constexpr int64_t kNoAllocMax = FEI_NOALLOC_MAX_ELEM;

// counts[8] followed by 7 lists of kNoAllocMax element ids (one per degree).
static __device__ __align__(256) int32_t g_noalloc_scratch[8 + 7 * kNoAllocMax];

std::mutex g_na_mutex;
int32_t *g_na_ptr[64];

// The host-side name g_noalloc_scratch is not a device address; look the
// address up once per device, with that device current.
fei_status scratch_ptr(int dev, int32_t **out) {
  if (dev < 0 || dev >= 64) return set_error(FEI_ERR_UNSUPPORTED, "device ordinal %d", dev);
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void *p = nullptr;
    FEI_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress(no-alloc scratch)");
    g_na_ptr[dev] = static_cast<int32_t *>(p);
  }
  *out = g_na_ptr[dev];
  return FEI_OK;
}

// Same bucketing as the allocating path: one atomic per element into the
// list of its degree; degrees without a reference are marked.
__global__ void noalloc_bucket_kernel(const int32_t *degree, int64_t n, unsigned avail, int32_t *counts,
                                      int32_t *lists, int64_t cap, int32_t *status) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int p = degree[e];
    if (p >= 1 && p <= kPMax && ((avail >> p) & 1u)) {
      const int pos = atomicAdd(&counts[p], 1);
      lists[(int64_t)(p - 1) * cap + pos] = (int32_t)e;
    } else {
      status[e] = FEI_ERR_INVALID_DEGREE;
    }
  }
}

__global__ void noalloc_clear_counts(int32_t *counts) {
  if (threadIdx.x < 8) counts[threadIdx.x] = 0;
}

fei_status launch_one(int p, fei_precision prec, const fei_reference *r, const FwdArgs &a, int64_t grid_work,
                      cudaStream_t s) {
  const fei_status st = (prec == FEI_TC_F16X3 && p >= 3) ? launch_tc_forward(p, r, a, grid_work, s)
                                                          : launch_cc_forward(p, prec == FEI_FP64, a, grid_work, s);
  return st ? st : debug_check(s, "forward kernel");
}

}  // namespace
}  // namespace fei

using namespace fei;

extern "C" fei_status fei_integrate_noalloc(const fei_reference_t *refs, int nrefs, const fei_batch *batch,
                                            fei_precision prec, void *A_out, void *b_out, int32_t *elem_status,
                                            fei_stream_t stream) {
  const Range range_("fei_integrate_noalloc");
  if (!batch) return set_error(FEI_ERR_INVALID_ARG, "fei_integrate_noalloc: batch is NULL");
  if (batch->n_elem < 0) return set_error(FEI_ERR_INVALID_ARG, "fei_integrate_noalloc: n_elem < 0");
  if (batch->n_elem > kNoAllocMax)
    return set_error(FEI_ERR_INVALID_ARG,
                     "fei_integrate_noalloc: %lld elements exceed the fixed scratch capacity of %lld "
                     "(FEI_NOALLOC_MAX_ELEM); split the batch or use fei_integrate",
                     (long long)batch->n_elem, (long long)kNoAllocMax);
  if (prec != FEI_FP64 && prec != FEI_FP32 && prec != FEI_TC_F16X3)
    return set_error(FEI_ERR_INVALID_ARG, "fei_integrate_noalloc: precision %d", (int)prec);
  if (batch->n_elem == 0) return FEI_OK;
  if (!batch->geom || !batch->K || !batch->b || !batch->c || !batch->f || !A_out || !b_out || !elem_status)
    return set_error(FEI_ERR_INVALID_ARG, "fei_integrate_noalloc: NULL input or output pointer");
  if (batch->coef_mode != FEI_COEF_PER_ELEMENT && batch->coef_mode != FEI_COEF_PER_POINT)
    return set_error(FEI_ERR_INVALID_ARG, "fei_integrate_noalloc: coef_mode %d", batch->coef_mode);
  if (!batch->degree)  // a uniform-degree batch needs no scratch at all
    return fei_integrate(refs, nrefs, batch, prec, A_out, b_out, elem_status, stream);
  if (!batch->A_offset || !batch->b_offset || (batch->coef_mode == FEI_COEF_PER_POINT && !batch->q_offset))
    return set_error(FEI_ERR_INVALID_ARG, "fei_integrate_noalloc: a degree array needs A_offset, b_offset (and q_offset per point)");
  if (!refs || nrefs < 1) return set_error(FEI_ERR_INVALID_ARG, "fei_integrate_noalloc: refs is NULL or nrefs < 1");
  int dev;
  FEI_CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
  const fei_reference *by_p[kPMax + 1] = {nullptr};
  for (int k = 0; k < nrefs; ++k) {
    if (!refs[k]) return set_error(FEI_ERR_INVALID_ARG, "fei_integrate_noalloc: refs[%d] is NULL", k);
    if (refs[k]->device != dev)
      return set_error(FEI_ERR_INVALID_ARG, "fei_integrate_noalloc: refs[%d] belongs to device %d", k, refs[k]->device);
    by_p[refs[k]->p] = refs[k];
  }
  int32_t *scratch;
  fei_status st = scratch_ptr(dev, &scratch);
  if (st) return st;
  int32_t *counts = scratch, *lists = scratch + 8;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned avail = 0;
  for (int p = 1; p <= kPMax; ++p)
    if (by_p[p]) avail |= 1u << p;
  // the array keeps the previous call's counts: clear them first
  noalloc_clear_counts<<<1, 32, 0, s>>>(counts);
  FEI_CUDA_TRY(cudaGetLastError(), "noalloc_clear_counts launch");
  int64_t blocks = (batch->n_elem + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  noalloc_bucket_kernel<<<(unsigned)blocks, 256, 0, s>>>(batch->degree, batch->n_elem, avail, counts, lists,
                                                          kNoAllocMax, elem_status);
  FEI_CUDA_TRY(cudaGetLastError(), "noalloc_bucket_kernel launch");
  for (int p = 1; p <= kPMax; ++p) {
    const fei_reference *r = by_p[p];
    if (!r) continue;
    FwdArgs a;
    memset(&a, 0, sizeof(a));
    a.n_work = batch->n_elem;
    a.count = counts + p;
    a.list = lists + (int64_t)(p - 1) * kNoAllocMax;
    a.geom = batch->geom;
    a.coef_mode = batch->coef_mode;
    a.K = batch->K;
    a.b = batch->b;
    a.c = batch->c;
    a.f = batch->f;
    a.A_off = batch->A_offset;
    a.b_off = batch->b_offset;
    a.q_off = batch->q_offset;
    a.A = A_out;
    a.bv = b_out;
    a.status = elem_status;
    a.G64 = r->G64;
    a.G32 = r->G32;
    a.znode = r->znode;
    a.tnode = r->tnode;
    a.G32T = r->G32T;
    st = launch_one(p, prec, r, a, batch->n_elem, s);
    if (st) return st;
  }
  return FEI_OK;
}
