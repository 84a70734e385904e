// fei_noalloc.cu -- fei_integrate_noalloc: the mixed-degree forward pass
// with its bucketing scratch in a fixed device array instead of memory that
// the library allocates.
//
// fei_integrate sorts a batch with a degree array into per-degree element
// lists before it launches one kernel per degree; those lists and their
// counts are scratch memory, which fei_integrate allocates (once per device,
// grown on demand) with cudaMalloc.  Some callers cannot let a library call
// cudaMalloc: code that must never block the device (cudaMalloc can
// synchronise it), and applications whose device memory is owned by a pool
// or a budget that the library must not bypass.  This entry point serves
// them: its scratch is the file-scope array below, reserved on every GPU
// that loads the library until the process exits, and it calls no
// allocating routine at all.  After the bucketing it runs the same code as
// fei_integrate (integrate_scratch), so its outputs are those of
// fei_integrate bit for bit.
//
// Limits and sharing:
//  - at most FEI_NOALLOC_MAX_ELEM elements per call (larger batches are
//    rejected with FEI_ERR_INVALID_ARG);
//  - every call on a device uses the same array and leaves its contents
//    behind; the call clears the per-degree counts itself before bucketing,
//    but two calls whose work overlaps on the GPU (different streams without
//    ordering between them) race on the array and give wrong results;
//  - the first call on a device looks up the array's device address
//    (cudaGetSymbolAddress) and keeps it for the life of the process.  The
//    kept address is not valid after cudaDeviceReset on that device.
#include "fei_internal.cuh"

#include <mutex>

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

}  // namespace
}  // namespace fei

using namespace fei;

extern "C" fei_status fei_integrate_noalloc(const fei_reference_t *refs, int nrefs, const fei_batch *batch,
                                            fei_precision prec, void *A_out, void *b_out, int32_t *elem_status,
                                            fei_stream_t stream) {
  const Range range_("fei_integrate_noalloc");
  if (!batch) return set_error(FEI_ERR_INVALID_ARG, "fei_integrate_noalloc: batch is NULL");
  if (batch->n_elem > kNoAllocMax)
    return set_error(FEI_ERR_INVALID_ARG,
                     "fei_integrate_noalloc: %lld elements exceed the fixed scratch capacity of %lld "
                     "(FEI_NOALLOC_MAX_ELEM); split the batch or use fei_integrate",
                     (long long)batch->n_elem, (long long)kNoAllocMax);
  fei_status st = check_batch(batch);
  if (st) return st;
  if (!valid_precision(prec))
    return set_error(FEI_ERR_INVALID_ARG, "fei_integrate_noalloc: precision %d", (int)prec);
  if (batch->n_elem == 0) return FEI_OK;
  if (!A_out || !b_out || !elem_status)
    return set_error(FEI_ERR_INVALID_ARG, "fei_integrate_noalloc: A_out, b_out and elem_status are required");
  int dev;
  FEI_CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
  const fei_reference *by_p[kPMax + 1];
  st = check_refs(refs, nrefs, dev, by_p);
  if (st) return st;
  int32_t *counts = nullptr, *lists = nullptr;
  if (batch->degree) {  // a uniform-degree batch needs no scratch at all
    int32_t *scratch;
    st = scratch_ptr(dev, &scratch);
    if (st) return st;
    counts = scratch;
    lists = scratch + 8;
  }
  return integrate_scratch(by_p, batch, prec, A_out, b_out, elem_status, counts, lists, kNoAllocMax,
                           (cudaStream_t)stream);
}
