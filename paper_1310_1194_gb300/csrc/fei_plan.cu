// fei_plan.cu -- plans: a mixed-degree batch as one CUDA graph, with the
// kernel shape of every degree chosen by measurement.
//
// Elements of one degree share the reference tables (Sec. 2.2: elements
// are grouped by type and degree so that the tables stay in fast memory),
// so a mixed batch runs as: clear the bucket counts, bucket the elements by
// degree (one atomic per element), then one persistent kernel per degree
// that walks its bucket.  A plan owns the bucket scratch (allocated once, at
// creation) and, per degree, the kernel variant and grid that its
// autotuner measured fastest on a real batch.  fei_plan_execute captures the
// whole sequence into a CUDA graph on the first call with a given set of
// pointers and replays it afterwards, so a repeated batch costs one graph
// launch and no host work per degree.
//
// Candidates per degree (what fei_plan_tune times):
//   tensor-core paths (p >= 3, FEI_TC_F16X3, FEI_TC_3XTF32): the warp-role variants of the
//     tcgen05 kernel (8 or 16 producer warps), one CTA per SM;
//   sum-factorised path (p >= 3, FEI_SF_FP32): as many blocks as fit on the
//     SMs, or one per SM;
//   FEI_AUTO at p >= 3: both of the above (FEI_TC_F16X3 variants and the
//     sum-factorised kernel), so the fastest kernel within the 1e-6 bar wins;
//   CUDA-core paths (FEI_FP64, FEI_FP32, and p <= 2 under the other precisions): the
//     grid of the grid-stride kernel, 2, 4, 8 or 16 blocks per SM.
// Every candidate computes the same quantities; variants differ only in the
// order of a few FP32 additions (load-vector partial sums), so results stay
// within the path's tolerance whichever candidate a plan picks.
#include <string.h>

#include "fei_internal.cuh"

struct fei_plan {
  int device;
  fei_precision prec;
  int64_t max_elem;
  const fei_reference *by_p[fei::kPMax + 1];
  unsigned avail;
  int32_t *counts;  // [8]
  int32_t *lists;   // [7][max_elem]
  int variant[fei::kPMax + 1];
  int64_t grid_cap[fei::kPMax + 1];
  float tuned_ms[fei::kPMax + 1];
  // graph of the last argument set
  bool has_graph;
  cudaGraphExec_t exec;
  fei_batch key_batch;
  void *key_A, *key_b;
  int32_t *key_st;
};

namespace fei {
namespace {

// The kernel of degree p for a plan's variant number, and its precision.
// Variants: the tensor-core warp-role variants 0 .. tc_variant_count - 1;
// under FEI_AUTO at p >= 3 one more, the sum-factorised kernel; else 0.
KernelKind plan_kernel(fei_precision prec, int p, int variant, fei_precision *run) {
  if (prec == FEI_AUTO && p >= 3) {
    *run = variant < tc_variant_count(p, FEI_TC_F16X3) ? FEI_TC_F16X3 : FEI_SF_FP32;
    return *run == FEI_TC_F16X3 ? KERNEL_TC : KERNEL_SF;
  }
  return direct_kernel(prec, p, run);
}
int n_variants(fei_precision prec, int p) {
  fei_precision run;
  if (prec == FEI_AUTO && p >= 3) return tc_variant_count(p, FEI_TC_F16X3) + 1;
  return direct_kernel(prec, p, &run) == KERNEL_TC ? tc_variant_count(p, run) : 1;
}
// The variant a plan starts from (before any tuning).
int default_variant(fei_precision prec, int p) {
  return (prec == FEI_AUTO && p >= 5) ? tc_variant_count(p, FEI_TC_F16X3) : 0;
}

// The batch a graph was captured for, field by field (not the padding).
bool same_batch(const fei_batch &x, const fei_batch &y) {
  return x.n_elem == y.n_elem && x.geom == y.geom && x.degree == y.degree && x.uniform_degree == y.uniform_degree &&
         x.coef_mode == y.coef_mode && x.K == y.K && x.b == y.b && x.c == y.c && x.f == y.f &&
         x.A_offset == y.A_offset && x.b_offset == y.b_offset && x.q_offset == y.q_offset &&
         x.a_layout == y.a_layout;
}

// Candidates of degree p: every tensor-core variant (grid: one CTA per
// SM), the sum-factorised kernel with as many blocks as fit or one per SM,
// the CUDA-core kernels with 2, 4, 8 or 16 blocks per SM.
int n_candidates(fei_precision prec, int p) {
  fei_precision run;
  const KernelKind k = plan_kernel(prec, p, 0, &run);
  if (prec == FEI_AUTO && p >= 3) return tc_variant_count(p, FEI_TC_F16X3) + 2;
  return k == KERNEL_TC ? tc_variant_count(p, run) : k == KERNEL_SF ? 2 : 4;
}

// Candidate c of degree p as (variant, grid cap).
void candidate(fei_precision prec, int p, int c, int *variant, int64_t *grid_cap) {
  fei_precision run;
  const int ntc = (prec == FEI_AUTO && p >= 3) ? tc_variant_count(p, FEI_TC_F16X3) : 0;
  const KernelKind k = plan_kernel(prec, p, c, &run);
  if (k == KERNEL_TC) {
    *variant = c;
    *grid_cap = 0;
  } else if (k == KERNEL_SF) {
    *variant = ntc;
    *grid_cap = c == ntc ? 0 : 152;
  } else {
    static const int per_sm[4] = {2, 4, 8, 16};
    *variant = 0;
    *grid_cap = 152 * per_sm[c];
  }
}

void fill_args(FwdArgs &a, const fei_batch *b, const fei_reference *r, void *A, void *bv, int32_t *st) {
  memset(&a, 0, sizeof(a));
  a.n_work = b->n_elem;
  a.geom = b->geom;
  a.coef_mode = b->coef_mode;
  a.K = b->K;
  a.b = b->b;
  a.c = b->c;
  a.f = b->f;
  a.A_off = b->A_offset;
  a.upper = b->a_layout == FEI_A_UPPER;
  a.b_off = b->b_offset;
  a.q_off = b->q_offset;
  a.A = A;
  a.bv = bv;
  a.status = st;
  a.G64 = r->G64;
  a.G32 = r->G32;
  a.znode = r->znode;
  a.tnode = r->tnode;
  a.G32T = r->G32T;
}

fei_status launch_degree(const fei_plan *pl, int p, int variant, int64_t grid_cap, const fei_batch *b, void *A,
                         void *bv, int32_t *st, bool bucketed, cudaStream_t s) {
  const fei_reference *r = pl->by_p[p];
  FwdArgs a;
  fill_args(a, b, r, A, bv, st);
  if (bucketed) {
    a.count = pl->counts + p;
    a.list = pl->lists + (int64_t)(p - 1) * pl->max_elem;
  }
  fei_precision run;
  const KernelKind k = plan_kernel(pl->prec, p, variant, &run);
  const fei_status ls = k == KERNEL_TC   ? launch_tc_forward(p, r, a, b->n_elem, s, variant, run)
                        : k == KERNEL_SF ? launch_sf_forward(p, r, a, b->n_elem, s, grid_cap)
                                         : launch_cc_forward(p, run == FEI_FP64, a, b->n_elem, s, grid_cap);
  return ls ? ls : debug_check(s, "forward kernel");
}

__global__ void plan_bucket_kernel(const int32_t *degree, int64_t n, unsigned avail, int32_t *counts,
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

fei_status enqueue_bucketing(const fei_plan *pl, const fei_batch *b, int32_t *st, cudaStream_t s) {
  FEI_CUDA_TRY(cudaMemsetAsync(pl->counts, 0, sizeof(int32_t) * 8, s), "cudaMemsetAsync(plan counts)");
  int64_t blocks = (b->n_elem + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  plan_bucket_kernel<<<(unsigned)blocks, 256, 0, s>>>(b->degree, b->n_elem, pl->avail, pl->counts, pl->lists,
                                                       pl->max_elem, st);
  FEI_CUDA_TRY(cudaGetLastError(), "plan_bucket_kernel launch");
  return FEI_OK;
}

// The whole batch with the plan's current choices.
fei_status enqueue_all(const fei_plan *pl, const fei_batch *b, void *A, void *bv, int32_t *st, cudaStream_t s) {
  if (!b->degree) {
    const int p = b->uniform_degree;
    return launch_degree(pl, p, pl->variant[p], pl->grid_cap[p], b, A, bv, st, false, s);
  }
  fei_status e = enqueue_bucketing(pl, b, st, s);
  if (e) return e;
  for (int p = 1; p <= kPMax; ++p) {
    if (!pl->by_p[p]) continue;
    e = launch_degree(pl, p, pl->variant[p], pl->grid_cap[p], b, A, bv, st, true, s);
    if (e) return e;
  }
  return FEI_OK;
}

fei_status check_call(const fei_plan *pl, const fei_batch *b, void *A, void *bv, int32_t *st) {
  if (!pl) return set_error(FEI_ERR_INVALID_ARG, "plan is NULL");
  if (!b) return set_error(FEI_ERR_INVALID_ARG, "batch is NULL");
  if (b->n_elem < 0) return set_error(FEI_ERR_INVALID_ARG, "n_elem < 0");
  if (b->n_elem == 0) return FEI_OK;
  if (b->degree && b->n_elem > pl->max_elem)
    return set_error(FEI_ERR_INVALID_ARG, "%lld elements exceed the plan's max_elem %lld", (long long)b->n_elem,
                     (long long)pl->max_elem);
  if (!b->geom || !b->K || !b->b || !b->c || !b->f || !A || !bv || !st)
    return set_error(FEI_ERR_INVALID_ARG, "NULL input or output pointer");
  if (b->coef_mode != FEI_COEF_PER_ELEMENT && b->coef_mode != FEI_COEF_PER_POINT)
    return set_error(FEI_ERR_INVALID_ARG, "coef_mode %d", b->coef_mode);
  if (b->degree) {
    if (!b->A_offset || !b->b_offset || (b->coef_mode == FEI_COEF_PER_POINT && !b->q_offset))
      return set_error(FEI_ERR_INVALID_ARG, "a degree array needs A_offset, b_offset (and q_offset per point)");
  } else {
    const int p = b->uniform_degree;
    if (p < 1 || p > kPMax) return set_error(FEI_ERR_INVALID_DEGREE, "uniform_degree %d outside 1..7", p);
    if (!pl->by_p[p]) return set_error(FEI_ERR_INVALID_DEGREE, "the plan has no reference for degree %d", p);
  }
  int dev;
  FEI_CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev != pl->device) return set_error(FEI_ERR_INVALID_ARG, "plan belongs to device %d, current is %d", pl->device, dev);
  return FEI_OK;
}

void drop_graph(fei_plan *pl) {
  if (pl->has_graph) cudaGraphExecDestroy(pl->exec);
  pl->has_graph = false;
}

}  // namespace
}  // namespace fei

using namespace fei;

extern "C" fei_status fei_plan_create(const fei_reference_t *refs, int nrefs, int64_t max_elem, fei_precision prec,
                                      fei_plan_t *out) {
  if (!out) return set_error(FEI_ERR_INVALID_ARG, "fei_plan_create: out is NULL");
  *out = nullptr;
  if (!refs || nrefs < 1) return set_error(FEI_ERR_INVALID_ARG, "fei_plan_create: refs is NULL or nrefs < 1");
  if (max_elem < 0 || max_elem > 2147483647LL)
    return set_error(FEI_ERR_INVALID_ARG, "fei_plan_create: max_elem %lld outside 0..2^31-1", (long long)max_elem);
  if (!valid_precision(prec))
    return set_error(FEI_ERR_INVALID_ARG, "fei_plan_create: precision %d", (int)prec);
  for (int k = 0; k < nrefs; ++k)
    if (!refs[k]) return set_error(FEI_ERR_INVALID_ARG, "fei_plan_create: refs[%d] is NULL", k);
  int dev;
  FEI_CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
  fei_plan *pl = new fei_plan();
  memset(pl, 0, sizeof(*pl));
  pl->device = dev;
  pl->prec = prec;
  pl->max_elem = max_elem;
  for (int k = 0; k < nrefs; ++k) {
    if (refs[k]->device != dev) {
      delete pl;
      return set_error(FEI_ERR_INVALID_ARG, "fei_plan_create: refs[%d] belongs to device %d", k, refs[k]->device);
    }
    pl->by_p[refs[k]->p] = refs[k];
    pl->avail |= 1u << refs[k]->p;
  }
  for (int p = 1; p <= kPMax; ++p) {
    pl->variant[p] = pl->by_p[p] ? default_variant(prec, p) : 0;
    pl->grid_cap[p] = 0;
    pl->tuned_ms[p] = -1.f;
  }
  cudaError_t e = cudaMalloc(&pl->counts, sizeof(int32_t) * 8);
  if (e == cudaSuccess && max_elem > 0) e = cudaMalloc(&pl->lists, sizeof(int32_t) * 7 * (size_t)max_elem);
  if (e != cudaSuccess) {
    if (pl->counts) cudaFree(pl->counts);
    delete pl;
    return cuda_error(e, "fei_plan_create: scratch");
  }
  *out = pl;
  return FEI_OK;
}

extern "C" fei_status fei_plan_destroy(fei_plan_t plan) {
  if (!plan) return FEI_OK;
  drop_graph(plan);
  if (plan->counts) cudaFree(plan->counts);
  if (plan->lists) cudaFree(plan->lists);
  delete plan;
  return FEI_OK;
}

extern "C" fei_status fei_plan_tune(fei_plan_t plan, const fei_batch *batch, void *A_out, void *b_out,
                                    int32_t *elem_status, fei_stream_t stream) {
  const Range range_("fei_plan_tune");
  fei_status st = check_call(plan, batch, A_out, b_out, elem_status);
  if (st || batch->n_elem == 0) return st;
  cudaStream_t s = (cudaStream_t)stream;
  int32_t counts[8] = {0};
  bool bucketed = batch->degree != nullptr;
  if (bucketed) {
    st = enqueue_bucketing(plan, batch, elem_status, s);
    if (st) return st;
    FEI_CUDA_TRY(cudaMemcpyAsync(counts, plan->counts, sizeof(counts), cudaMemcpyDeviceToHost, s),
                 "cudaMemcpyAsync(plan counts)");
    FEI_CUDA_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  } else {
    counts[batch->uniform_degree] = (int32_t)batch->n_elem;
  }
  cudaEvent_t e0, e1;
  FEI_CUDA_TRY(cudaEventCreate(&e0), "cudaEventCreate");
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_error(ce, "cudaEventCreate");
  }
  for (int p = 1; p <= kPMax && !st; ++p) {
    if (!plan->by_p[p] || counts[p] == 0) continue;
    float best = 3.0e38f;
    for (int c = 0; c < n_candidates(plan->prec, p) && !st; ++c) {
      int variant;
      int64_t cap;
      candidate(plan->prec, p, c, &variant, &cap);
      // one untimed run, then the best of two timed runs
      float t_best = 3.0e38f;
      for (int rep = 0; rep < 3 && !st; ++rep) {
        cudaEventRecord(e0, s);
        st = launch_degree(plan, p, variant, cap, batch, A_out, b_out, elem_status, bucketed, s);
        cudaEventRecord(e1, s);
        if (st) break;
        ce = cudaEventSynchronize(e1);
        if (ce != cudaSuccess) {
          st = cuda_error(ce, "cudaEventSynchronize");
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < t_best) t_best = ms;
      }
      if (!st && t_best < best) {
        best = t_best;
        plan->variant[p] = variant;
        plan->grid_cap[p] = cap;
        plan->tuned_ms[p] = t_best;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  drop_graph(plan);  // the choices changed
  return st;
}

extern "C" fei_status fei_plan_execute(fei_plan_t plan, const fei_batch *batch, void *A_out, void *b_out,
                                       int32_t *elem_status, fei_stream_t stream) {
  const Range range_("fei_plan_execute");
  fei_status st = check_call(plan, batch, A_out, b_out, elem_status);
  if (st || batch->n_elem == 0) return st;
  cudaStream_t s = (cudaStream_t)stream;
  // the legacy default stream cannot be captured: launch directly
  if (s == nullptr || s == cudaStreamLegacy) return enqueue_all(plan, batch, A_out, b_out, elem_status, s);
  const bool same = plan->has_graph && same_batch(plan->key_batch, *batch) &&
                    plan->key_A == A_out && plan->key_b == b_out && plan->key_st == elem_status;
  if (!same) {
    FEI_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    st = enqueue_all(plan, batch, A_out, b_out, elem_status, s);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(s, &graph);
    if (st) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (ce != cudaSuccess) return cuda_error(ce, "cudaStreamEndCapture");
    bool updated = false;
    if (plan->has_graph) {
      cudaGraphExecUpdateResultInfo info;
      updated = cudaGraphExecUpdate(plan->exec, graph, &info) == cudaSuccess;
      if (!updated) {
        (void)cudaGetLastError();
        drop_graph(plan);
      }
    }
    if (!updated) {
      const cudaError_t ie = cudaGraphInstantiate(&plan->exec, graph, 0);
      if (ie != cudaSuccess) {
        cudaGraphDestroy(graph);
        return cuda_error(ie, "cudaGraphInstantiate");
      }
      plan->has_graph = true;
    }
    cudaGraphDestroy(graph);
    plan->key_batch = *batch;
    plan->key_A = A_out;
    plan->key_b = b_out;
    plan->key_st = elem_status;
  }
  FEI_CUDA_TRY(cudaGraphLaunch(plan->exec, s), "cudaGraphLaunch");
  return FEI_OK;
}

extern "C" fei_status fei_plan_choice(fei_plan_t plan, int p, int *variant, int64_t *grid_cap, float *tuned_ms) {
  if (!plan) return set_error(FEI_ERR_INVALID_ARG, "fei_plan_choice: plan is NULL");
  if (p < 1 || p > kPMax) return set_error(FEI_ERR_INVALID_DEGREE, "fei_plan_choice: degree %d", p);
  if (variant) *variant = plan->variant[p];
  if (grid_cap) *grid_cap = plan->grid_cap[p];
  if (tuned_ms) *tuned_ms = plan->tuned_ms[p];
  return FEI_OK;
}

extern "C" fei_status fei_plan_kernel(fei_plan_t plan, int p, int *kernel) {
  if (!plan || !kernel) return set_error(FEI_ERR_INVALID_ARG, "fei_plan_kernel: NULL plan or kernel");
  if (p < 1 || p > kPMax) return set_error(FEI_ERR_INVALID_DEGREE, "fei_plan_kernel: degree %d", p);
  fei_precision run;
  *kernel = (int)plan_kernel(plan->prec, p, plan->variant[p], &run);
  return FEI_OK;
}

extern "C" fei_status fei_plan_set_choice(fei_plan_t plan, int p, int variant, int64_t grid_cap) {
  if (!plan) return set_error(FEI_ERR_INVALID_ARG, "fei_plan_set_choice: plan is NULL");
  if (p < 1 || p > kPMax) return set_error(FEI_ERR_INVALID_DEGREE, "fei_plan_set_choice: degree %d", p);
  const int nv = n_variants(plan->prec, p);
  if (variant < 0 || variant >= nv)
    return set_error(FEI_ERR_INVALID_ARG, "fei_plan_set_choice: variant %d for degree %d", variant, p);
  if (grid_cap < 0 || grid_cap > 2147483647LL)
    return set_error(FEI_ERR_INVALID_ARG, "fei_plan_set_choice: grid cap %lld", (long long)grid_cap);
  plan->variant[p] = variant;
  plan->grid_cap[p] = grid_cap;
  plan->tuned_ms[p] = -1.f;
  drop_graph(plan);  // the next execute captures with the new choice
  return FEI_OK;
}

