// fei_pipeline.cu -- integration of a batch held in host memory.
//
// The batch is cut into chunks of consecutive elements whose inputs and
// outputs fit one device slot.  Each chunk is copied in on an upload
// stream, integrated (the kernels of fei_integrate, with the bucketing
// scratch of the slot) on the caller's stream and copied out
// on a download stream, with two input slots and two output slots, so that
// the download of chunk k overlaps the integration of chunk k + 1 and the
// upload of chunk k + 2.  Outputs are packed in element order (the layout
// of fei_plan_offsets), on the host exactly as fei_integrate would have
// written them on the device.
#include <cstring>
#include <vector>

#include "fei_internal.cuh"

using namespace fei;

namespace {

constexpr int kSlots = 2;
constexpr int64_t kMinSlotBytes = int64_t(1) << 20;
constexpr int64_t kDefaultSlotBytes = int64_t(256) << 20;
constexpr int64_t kGeomBytes = 18 * sizeof(double);
constexpr int64_t kRecordBytes = 14 * sizeof(double);  // K 9, b 3, c 1, f 1

struct InSlot {
  double *geom = nullptr, *K = nullptr, *b = nullptr, *c = nullptr, *f = nullptr;
  int32_t *degree = nullptr;
  int64_t *A_off = nullptr, *b_off = nullptr, *q_off = nullptr;
  int32_t *bad = nullptr;
  int32_t *counts = nullptr, *lists = nullptr;  // the chunk's degree buckets (own scratch)
  cudaEvent_t ready = nullptr;     // inputs of the slot's chunk uploaded
  cudaEvent_t consumed = nullptr;  // the chunk's integration has run
};

struct OutSlot {
  void *A = nullptr, *bv = nullptr;
  int32_t *status = nullptr;
  cudaEvent_t drained = nullptr;  // the chunk's outputs downloaded
};

struct Chunk {
  int64_t e0, e1;  // elements [e0, e1)
  int64_t q0, q1;  // coefficient records [q0, q1)
  int64_t a0, a1;  // scalars of A
  int64_t b0, b1;  // scalars of b
};

}  // namespace

struct fei_pipeline {
  int device = -1;
  fei_precision prec = FEI_FP32;
  const fei_reference *by_p[kPMax + 1] = {};
  int64_t slot_bytes = 0;
  int64_t max_elem = 0, max_rec = 0, max_a = 0, max_b = 0;  // per chunk
  InSlot in[kSlots];
  OutSlot out[kSlots];
  cudaStream_t up = nullptr, down = nullptr;
  cudaEvent_t start = nullptr, up_done = nullptr, done = nullptr;
  int next = 0;  // slot of the next chunk (carried across calls)
  std::vector<int64_t> aoff, boff, qoff;
  std::vector<Chunk> chunks;
};

namespace {

void release(fei_pipeline *pl) {
  for (int k = 0; k < kSlots; ++k) {
    InSlot &i = pl->in[k];
    for (void *ptr : {(void *)i.geom, (void *)i.K, (void *)i.b, (void *)i.c, (void *)i.f, (void *)i.degree,
                      (void *)i.A_off, (void *)i.b_off, (void *)i.q_off, (void *)i.bad, (void *)i.counts,
                      (void *)i.lists})
      if (ptr) cudaFree(ptr);
    if (i.ready) cudaEventDestroy(i.ready);
    if (i.consumed) cudaEventDestroy(i.consumed);
    OutSlot &o = pl->out[k];
    for (void *ptr : {o.A, o.bv, (void *)o.status})
      if (ptr) cudaFree(ptr);
    if (o.drained) cudaEventDestroy(o.drained);
  }
  if (pl->up) cudaStreamDestroy(pl->up);
  if (pl->down) cudaStreamDestroy(pl->down);
  if (pl->start) cudaEventDestroy(pl->start);
  if (pl->done) cudaEventDestroy(pl->done);
  if (pl->up_done) cudaEventDestroy(pl->up_done);
  delete pl;
}

fei_status dmalloc(void **ptr, int64_t bytes, const char *what) {
  const cudaError_t e = cudaMalloc(ptr, (size_t)bytes);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return set_error(FEI_ERR_OOM, "fei_pipeline_create: cudaMalloc(%s, %lld bytes)", what, (long long)bytes);
  }
  return e == cudaSuccess ? FEI_OK : cuda_error(e, what);
}

fei_status allocate(fei_pipeline *pl) {
  const int64_t dt = pl->prec == FEI_FP64 ? 8 : 4;
  pl->max_a = pl->slot_bytes / dt;
  pl->max_b = pl->max_a / 6 + 1;  // N_sh >= 6, so sum N_sh <= sum N_sh^2 / 6
  pl->max_elem = pl->slot_bytes / kGeomBytes;
  if (pl->max_elem > 2147483647LL) pl->max_elem = 2147483647LL;
  pl->max_rec = pl->slot_bytes / kRecordBytes;
  fei_status st;
  for (int k = 0; k < kSlots; ++k) {
    InSlot &i = pl->in[k];
    const int64_t ne = pl->max_elem, nr = pl->max_rec;
    if ((st = dmalloc((void **)&i.geom, ne * kGeomBytes, "pipeline geometry"))) return st;
    if ((st = dmalloc((void **)&i.K, nr * 9 * 8, "pipeline K"))) return st;
    if ((st = dmalloc((void **)&i.b, nr * 3 * 8, "pipeline b"))) return st;
    if ((st = dmalloc((void **)&i.c, nr * 8, "pipeline c"))) return st;
    if ((st = dmalloc((void **)&i.f, nr * 8, "pipeline f"))) return st;
    if ((st = dmalloc((void **)&i.degree, ne * 4, "pipeline degrees"))) return st;
    if ((st = dmalloc((void **)&i.A_off, (ne + 1) * 8, "pipeline A offsets"))) return st;
    if ((st = dmalloc((void **)&i.b_off, (ne + 1) * 8, "pipeline b offsets"))) return st;
    if ((st = dmalloc((void **)&i.q_off, (ne + 1) * 8, "pipeline point offsets"))) return st;
    if ((st = dmalloc((void **)&i.bad, 4, "pipeline bad count"))) return st;
    if ((st = dmalloc((void **)&i.counts, 8 * 4, "pipeline bucket counts"))) return st;
    if ((st = dmalloc((void **)&i.lists, 7 * ne * 4, "pipeline bucket lists"))) return st;
    FEI_CUDA_TRY(cudaEventCreateWithFlags(&i.ready, cudaEventDisableTiming), "cudaEventCreate");
    FEI_CUDA_TRY(cudaEventCreateWithFlags(&i.consumed, cudaEventDisableTiming), "cudaEventCreate");
    OutSlot &o = pl->out[k];
    if ((st = dmalloc(&o.A, pl->max_a * dt, "pipeline A"))) return st;
    if ((st = dmalloc(&o.bv, pl->max_b * dt, "pipeline b_e"))) return st;
    if ((st = dmalloc((void **)&o.status, ne * 4, "pipeline status"))) return st;
    FEI_CUDA_TRY(cudaEventCreateWithFlags(&o.drained, cudaEventDisableTiming), "cudaEventCreate");
  }
  FEI_CUDA_TRY(cudaStreamCreateWithFlags(&pl->up, cudaStreamNonBlocking), "cudaStreamCreate(upload)");
  FEI_CUDA_TRY(cudaStreamCreateWithFlags(&pl->down, cudaStreamNonBlocking), "cudaStreamCreate(download)");
  FEI_CUDA_TRY(cudaEventCreateWithFlags(&pl->start, cudaEventDisableTiming), "cudaEventCreate");
  FEI_CUDA_TRY(cudaEventCreateWithFlags(&pl->done, cudaEventDisableTiming), "cudaEventCreate");
  FEI_CUDA_TRY(cudaEventCreateWithFlags(&pl->up_done, cudaEventDisableTiming), "cudaEventCreate");
  return FEI_OK;
}

fei_status copy_in(void *dst, const void *src, int64_t bytes, cudaStream_t s) {
  if (bytes <= 0) return FEI_OK;
  FEI_CUDA_TRY(cudaMemcpyAsync(dst, src, (size_t)bytes, cudaMemcpyHostToDevice, s), "cudaMemcpyAsync(upload)");
  return FEI_OK;
}

fei_status copy_out(void *dst, const void *src, int64_t bytes, cudaStream_t s) {
  if (bytes <= 0) return FEI_OK;
  FEI_CUDA_TRY(cudaMemcpyAsync(dst, src, (size_t)bytes, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync(download)");
  return FEI_OK;
}

// Packed offsets of the whole batch on the host (degrees outside 1..7 take
// no room, as in fei_plan_offsets) and the chunks that fit one slot.
fei_status plan_chunks(fei_pipeline *pl, const fei_batch *hb) {
  const int64_t n = hb->n_elem;
  const bool upper = hb->a_layout == FEI_A_UPPER;
  const bool per_point = hb->coef_mode == FEI_COEF_PER_POINT;
  pl->chunks.clear();
  if (hb->degree) {
    pl->aoff.resize(n + 1);
    pl->boff.resize(n + 1);
    pl->qoff.resize(n + 1);
    int64_t a = 0, b = 0, q = 0;  // q: per-point records (unused per element)
    for (int64_t e = 0; e < n; ++e) {
      pl->aoff[e] = a;
      pl->boff[e] = b;
      pl->qoff[e] = q;
      const int p = hb->degree[e];
      if (p >= 1 && p <= kPMax) {
        const int64_t s = nsh_of(p);
        a += a_size(s, upper);
        b += s;
        q += nq_of(p);
      }
    }
    pl->aoff[n] = a;
    pl->boff[n] = b;
    pl->qoff[n] = q;
  }
  auto A_at = [&](int64_t e) -> int64_t {
    if (hb->degree) return pl->aoff[e];
    return e * a_size(nsh_of(hb->uniform_degree), upper);
  };
  auto b_at = [&](int64_t e) -> int64_t { return hb->degree ? pl->boff[e] : e * nsh_of(hb->uniform_degree); };
  auto q_at = [&](int64_t e) -> int64_t {
    if (!per_point) return e;
    return hb->degree ? pl->qoff[e] : e * nq_of(hb->uniform_degree);
  };
  int64_t e0 = 0;
  while (e0 < n) {
    // largest e1 with every per-chunk size within the slot (binary search:
    // all four sizes grow with e1)
    int64_t lo = e0 + 1, hi = (n - e0 > pl->max_elem) ? e0 + pl->max_elem : n;
    auto fits = [&](int64_t e1) {
      return A_at(e1) - A_at(e0) <= pl->max_a && b_at(e1) - b_at(e0) <= pl->max_b &&
             q_at(e1) - q_at(e0) <= pl->max_rec;
    };
    if (!fits(lo)) return set_error(FEI_ERR_INVALID_ARG, "fei_integrate_host: element %lld does not fit a slot",
                                    (long long)e0);
    while (lo < hi) {
      const int64_t mid = lo + (hi - lo + 1) / 2;
      if (fits(mid)) lo = mid;
      else hi = mid - 1;
    }
    pl->chunks.push_back({e0, lo, q_at(e0), q_at(lo), A_at(e0), A_at(lo), b_at(e0), b_at(lo)});
    e0 = lo;
  }
  return FEI_OK;
}

}  // namespace

extern "C" fei_status fei_pipeline_create(const fei_reference_t *refs, int nrefs, fei_precision prec,
                                          int64_t slot_bytes, fei_pipeline_t *out) {
  if (!out) return set_error(FEI_ERR_INVALID_ARG, "fei_pipeline_create: out is NULL");
  *out = nullptr;
  if (!valid_precision(prec))
    return set_error(FEI_ERR_INVALID_ARG, "fei_pipeline_create: precision %d", (int)prec);
  if (!refs || nrefs < 1) return set_error(FEI_ERR_INVALID_ARG, "fei_pipeline_create: refs is NULL or nrefs < 1");
  if (slot_bytes == 0) slot_bytes = kDefaultSlotBytes;
  if (slot_bytes < kMinSlotBytes || slot_bytes > (int64_t(1) << 40))
    return set_error(FEI_ERR_INVALID_ARG, "fei_pipeline_create: slot_bytes %lld outside 1 MiB .. 1 TiB",
                     (long long)slot_bytes);
  int dev;
  FEI_CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
  const fei_reference *by_p[kPMax + 1];
  fei_status st = check_refs(refs, nrefs, dev, by_p);
  if (st) return st;
  fei_pipeline *pl = new fei_pipeline;
  pl->device = dev;
  pl->prec = prec;
  for (int p = 0; p <= kPMax; ++p) pl->by_p[p] = by_p[p];
  pl->slot_bytes = slot_bytes;
  st = allocate(pl);
  if (st) {
    release(pl);
    return st;
  }
  *out = pl;
  return FEI_OK;
}

extern "C" fei_status fei_pipeline_destroy(fei_pipeline_t pl) {
  if (!pl) return FEI_OK;
  int dev;
  FEI_CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
  const int own = pl->device;
  if (dev != own) FEI_CUDA_TRY(cudaSetDevice(own), "cudaSetDevice");
  // outstanding copies and integrations may still use the slots
  cudaStreamSynchronize(pl->up);
  cudaStreamSynchronize(pl->down);
  for (int k = 0; k < kSlots; ++k) cudaEventSynchronize(pl->in[k].consumed);
  release(pl);
  if (dev != own) cudaSetDevice(dev);
  return FEI_OK;
}

extern "C" fei_status fei_pipeline_info(fei_pipeline_t pl, int64_t *slot_bytes, int64_t *max_elem) {
  if (!pl) return set_error(FEI_ERR_INVALID_ARG, "fei_pipeline_info: pipeline is NULL");
  if (slot_bytes) *slot_bytes = pl->slot_bytes;
  if (max_elem) *max_elem = pl->max_elem;
  return FEI_OK;
}

namespace {

// Enqueues the chunks of pl->chunks (see fei_integrate_host).
fei_status enqueue_chunks(fei_pipeline *pl, const fei_batch *hb, void *A_host, void *b_host, int32_t *status_host,
                          cudaStream_t s) {
  const int64_t dt = pl->prec == FEI_FP64 ? 8 : 4;
  const bool mixed = hb->degree != nullptr;
  const bool per_point = hb->coef_mode == FEI_COEF_PER_POINT;
  fei_status st;
  for (const Chunk &ch : pl->chunks) {
    const int k = pl->next;
    pl->next = (pl->next + 1) % kSlots;
    InSlot &in = pl->in[k];
    OutSlot &out = pl->out[k];
    const int64_t ne = ch.e1 - ch.e0, nr = ch.q1 - ch.q0;
    // upload, once the slot's previous chunk has been integrated
    FEI_CUDA_TRY(cudaStreamWaitEvent(pl->up, in.consumed, 0), "cudaStreamWaitEvent");
    if ((st = copy_in(in.geom, hb->geom + ch.e0 * 18, ne * kGeomBytes, pl->up))) return st;
    if ((st = copy_in(in.K, hb->K + ch.q0 * 9, nr * 72, pl->up))) return st;
    if ((st = copy_in(in.b, hb->b + ch.q0 * 3, nr * 24, pl->up))) return st;
    if ((st = copy_in(in.c, hb->c + ch.q0, nr * 8, pl->up))) return st;
    if ((st = copy_in(in.f, hb->f + ch.q0, nr * 8, pl->up))) return st;
    if (mixed && (st = copy_in(in.degree, hb->degree + ch.e0, ne * 4, pl->up))) return st;
    FEI_CUDA_TRY(cudaEventRecord(in.ready, pl->up), "cudaEventRecord");
    // integrate on the caller's stream, once the output slot has drained
    FEI_CUDA_TRY(cudaStreamWaitEvent(s, in.ready, 0), "cudaStreamWaitEvent");
    FEI_CUDA_TRY(cudaStreamWaitEvent(s, out.drained, 0), "cudaStreamWaitEvent");
    fei_batch db;
    memset(&db, 0, sizeof(db));
    db.n_elem = ne;
    db.geom = in.geom;
    db.uniform_degree = hb->uniform_degree;
    db.coef_mode = hb->coef_mode;
    db.a_layout = hb->a_layout;
    db.K = in.K;
    db.b = in.b;
    db.c = in.c;
    db.f = in.f;
    if (mixed) {
      db.degree = in.degree;
      st = (hb->a_layout == FEI_A_UPPER ? fei_plan_offsets_upper : fei_plan_offsets)(
          in.degree, ne, in.A_off, in.b_off, per_point ? in.q_off : nullptr, in.bad, (fei_stream_t)s);
      if (st) return st;
      db.A_offset = in.A_off;
      db.b_offset = in.b_off;
      db.q_offset = per_point ? in.q_off : nullptr;
    }
    st = integrate_scratch(pl->by_p, &db, pl->prec, out.A, out.bv, out.status, in.counts, in.lists,
                           pl->max_elem, s);
    if (st) return st;
    FEI_CUDA_TRY(cudaEventRecord(in.consumed, s), "cudaEventRecord");
    // download
    FEI_CUDA_TRY(cudaStreamWaitEvent(pl->down, in.consumed, 0), "cudaStreamWaitEvent");
    if ((st = copy_out((char *)A_host + ch.a0 * dt, out.A, (ch.a1 - ch.a0) * dt, pl->down))) return st;
    if ((st = copy_out((char *)b_host + ch.b0 * dt, out.bv, (ch.b1 - ch.b0) * dt, pl->down))) return st;
    if ((st = copy_out(status_host + ch.e0, out.status, ne * 4, pl->down))) return st;
    FEI_CUDA_TRY(cudaEventRecord(out.drained, pl->down), "cudaEventRecord");
  }
  return FEI_OK;
}

}  // namespace

extern "C" fei_status fei_integrate_host(fei_pipeline_t pl, const fei_batch *hb, void *A_host, void *b_host,
                                         int32_t *status_host, int64_t *n_chunks, fei_stream_t stream) {
  const Range range_("fei_integrate_host");
  if (!pl) return set_error(FEI_ERR_INVALID_ARG, "fei_integrate_host: pipeline is NULL");
  if (!hb) return set_error(FEI_ERR_INVALID_ARG, "fei_integrate_host: batch is NULL");
  if (hb->A_offset || hb->b_offset || hb->q_offset)
    return set_error(FEI_ERR_INVALID_ARG, "fei_integrate_host: outputs are packed in element order; "
                                          "A_offset, b_offset and q_offset must be NULL");
  // the checks of fei_integrate, with the offsets the pipeline makes itself
  fei_batch probe = *hb;
  if (hb->degree) {
    static const int64_t dummy = 0;
    probe.A_offset = probe.b_offset = probe.q_offset = &dummy;
  }
  fei_status st = check_batch(&probe);
  if (st) return st;
  if (n_chunks) *n_chunks = 0;
  if (hb->n_elem == 0) return FEI_OK;
  if (!A_host || !b_host || !status_host)
    return set_error(FEI_ERR_INVALID_ARG, "fei_integrate_host: A_host, b_host and status_host are required");
  int dev;
  FEI_CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev != pl->device)
    return set_error(FEI_ERR_INVALID_ARG, "fei_integrate_host: pipeline was created on device %d, current is %d",
                     pl->device, dev);
  st = plan_chunks(pl, hb);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  // work enqueued on the caller's stream before this call comes first
  FEI_CUDA_TRY(cudaEventRecord(pl->start, s), "cudaEventRecord");
  FEI_CUDA_TRY(cudaStreamWaitEvent(pl->up, pl->start, 0), "cudaStreamWaitEvent");
  st = enqueue_chunks(pl, hb, A_host, b_host, status_host, s);
  // the caller's stream completes after the last upload and download, also
  // when enqueueing failed part-way (what was enqueued still runs)
  cudaError_t e = cudaEventRecord(pl->up_done, pl->up);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, pl->up_done, 0);
  if (e == cudaSuccess) e = cudaEventRecord(pl->done, pl->down);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, pl->done, 0);
  if (st) return st;
  if (e != cudaSuccess) return cuda_error(e, "fei_integrate_host: joining the copy streams");
  if (n_chunks) *n_chunks = (int64_t)pl->chunks.size();
  return FEI_OK;
}
