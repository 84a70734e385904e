// fei_assembly.cu -- colour-by-colour assembly of element matrices into a
// global CSR matrix, the step that follows integration (Sec. 2).
//
// A global entry (r, c) is the sum of A_e[i][j] over the elements e whose
// local basis functions i and j carry the global numbers r and c; that sum
// is what makes assembly a dependent step.  Colouring the elements so that
// two elements sharing a global function never have the same colour removes
// the dependencies (Sec. 2): the elements of one colour touch disjoint rows,
// so one launch per colour adds them without atomics.
//
// Host part (fei_assembly_create), from the element-to-global map l2g:
//   1. global function -> elements incidence;
//   2. greedy colouring in element order: e takes the smallest colour not
//      held by an earlier element that shares a global function with it;
//   3. CSR pattern: row r lists, sorted, the global functions of all the
//      elements that contain r;
//   4. scatter map: for entry (i, j) of element e, the place of l2g_e[j] in
//      row l2g_e[i], counted from the row's start (uint16);
//   5. chunks for the fused path: elements sorted by (colour, degree) and
//      split so that a chunk's element matrices fit in a scratch buffer
//      that stays in the L2 (129 MB).
// Device part: a block per element adds its N_sh^2 entries at
// row_ptr[l2g_i] + off and its load vector at rhs[l2g_i].
// fei_integrate_assemble integrates one chunk into the scratch and
// assembles it right away, so the element matrices are read back from L2
// instead of making a round trip through HBM.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "fei_internal.cuh"

struct fei_assembly {
  int64_t n_elem, n_dof, nnz, n_entries;
  int32_t n_colours;
  int uniform_degree;  // 0 when degrees differ per element
  bool host_only;
  int device;
  std::vector<int32_t> degree_h;
  std::vector<int32_t> colour_h;
  std::vector<int64_t> row_ptr_h;  // kept only in host-only mode
  std::vector<int32_t> col_idx_h;
  std::vector<int64_t> colour_start;  // [n_colours + 1] into elems (sorted by colour, degree)
  struct Chunk {
    int32_t colour, degree;
    int64_t start, n, a_len, b_len;
  };
  std::vector<Chunk> chunks;
  int64_t max_chunk_a, max_chunk_b;
  // device
  int64_t *row_ptr;
  int32_t *col_idx;
  int64_t *l2g;
  int64_t *loff;  // start of element e in l2g and in b (sum of N_sh before e)
  int64_t *moff;  // start of element e in A and in the scatter map (sum of N_sh^2)
  uint16_t *off;
  int32_t *degree;
  int32_t *elems;        // elements sorted by (colour, degree)
  int32_t *chunk_count;  // [chunks] element count of each chunk (the forward's device count)
  int64_t *scr_aoff, *scr_boff;  // start of element e in its chunk's scratch
  void *scratch_A, *scratch_b;
  size_t scratch_A_bytes, scratch_b_bytes;
};

namespace fei {
namespace {

constexpr int64_t kChunkBytes = 48ll << 20;  // FP32 element matrices of one chunk

template <typename T>
__global__ void assemble_kernel(const int32_t *elems, int64_t n, const int32_t *degree, const T *A,
                                const int64_t *aoff, const T *bv, const int64_t *boff, const int64_t *l2g,
                                const int64_t *loff, const int64_t *moff, const uint16_t *off,
                                const int64_t *row_ptr, T *values, T *rhs) {
  __shared__ int64_t rstart[nsh_of(kPMax)];
  for (int64_t k = blockIdx.x; k < n; k += gridDim.x) {
    const int e = elems[k];
    const int s = nsh_of(degree[e]);
    const int64_t *g = l2g + loff[e];
    __syncthreads();  // the previous element's row starts are no longer read
    for (int i = threadIdx.x; i < s; i += blockDim.x) {
      rstart[i] = row_ptr[g[i]];
      rhs[g[i]] += bv[boff[e] + i];
    }
    __syncthreads();
    const T *Ae = A + aoff[e];
    const uint16_t *oe = off + moff[e];
    for (int idx = threadIdx.x; idx < s * s; idx += blockDim.x) {
      const int i = idx / s;
      values[rstart[i] + oe[idx]] += Ae[idx];
    }
  }
}

template <typename T>
fei_status launch_assemble(const fei_assembly *as, const int32_t *elems, int64_t n, const void *A,
                           const int64_t *aoff, const void *bv, const int64_t *boff, void *values, void *rhs,
                           cudaStream_t s) {
  if (n <= 0) return FEI_OK;
  const int64_t blocks = n < 152 * 16 ? n : 152 * 16;
  assemble_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(elems, n, as->degree, (const T *)A, aoff, (const T *)bv,
                                                      boff, as->l2g, as->loff, as->moff, as->off, as->row_ptr,
                                                      (T *)values, (T *)rhs);
  FEI_CUDA_TRY(cudaGetLastError(), "assemble_kernel launch");
  return FEI_OK;
}

void free_device(fei_assembly *as) {
  cudaFree(as->row_ptr);
  cudaFree(as->col_idx);
  cudaFree(as->l2g);
  cudaFree(as->loff);
  cudaFree(as->moff);
  cudaFree(as->off);
  cudaFree(as->degree);
  cudaFree(as->elems);
  cudaFree(as->chunk_count);
  cudaFree(as->scr_aoff);
  cudaFree(as->scr_boff);
  cudaFree(as->scratch_A);
  cudaFree(as->scratch_b);
}

template <typename T>
fei_status upload(T **dst, const T *src, size_t count) {
  *dst = nullptr;
  if (count == 0) return FEI_OK;
  cudaError_t e = cudaMalloc(dst, sizeof(T) * count);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return set_error(FEI_ERR_OOM, "fei_assembly_create: cudaMalloc of %zu bytes", sizeof(T) * count);
  }
  if (e != cudaSuccess) return cuda_error(e, "cudaMalloc");
  FEI_CUDA_TRY(cudaMemcpy(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice), "cudaMemcpy (assembly)");
  return FEI_OK;
}

// Everything of steps 1-5 on the host; uploads unless host_only.
fei_status build(fei_assembly *as, const int64_t *l2g) {
  const int64_t n = as->n_elem, nd = as->n_dof;
  std::vector<int64_t> loff(n + 1), moff(n + 1);
  loff[0] = moff[0] = 0;
  for (int64_t e = 0; e < n; ++e) {
    const int64_t s = nsh_of(as->degree_h[e]);
    loff[e + 1] = loff[e] + s;
    moff[e + 1] = moff[e] + s * s;
  }
  as->n_entries = moff[n];
  // map values in range and distinct within an element
  std::vector<int64_t> stamp(nd, -1);
  for (int64_t e = 0; e < n; ++e)
    for (int64_t k = loff[e]; k < loff[e + 1]; ++k) {
      const int64_t d = l2g[k];
      if (d < 0 || d >= nd)
        return set_error(FEI_ERR_INVALID_ARG, "l2g of element %lld holds %lld, outside 0..n_dof-1", (long long)e,
                         (long long)d);
      if (stamp[d] == e)
        return set_error(FEI_ERR_INVALID_ARG, "l2g of element %lld holds %lld twice", (long long)e, (long long)d);
      stamp[d] = e;
    }
  // 1. incidence
  std::vector<int64_t> inc_ptr(nd + 1, 0);
  for (int64_t k = 0; k < loff[n]; ++k) ++inc_ptr[l2g[k] + 1];
  for (int64_t d = 0; d < nd; ++d) inc_ptr[d + 1] += inc_ptr[d];
  std::vector<int32_t> inc(loff[n]);
  {
    std::vector<int64_t> fill(inc_ptr.begin(), inc_ptr.end() - 1);
    for (int64_t e = 0; e < n; ++e)
      for (int64_t k = loff[e]; k < loff[e + 1]; ++k) inc[fill[l2g[k]]++] = (int32_t)e;
  }
  // 2. greedy colouring
  as->colour_h.assign(n, -1);
  std::vector<int64_t> seen;  // seen[c] == e: colour c is taken by a neighbour of e
  for (int64_t e = 0; e < n; ++e) {
    for (int64_t k = loff[e]; k < loff[e + 1]; ++k) {
      const int64_t d = l2g[k];
      for (int64_t t = inc_ptr[d]; t < inc_ptr[d + 1]; ++t) {
        const int32_t c2 = as->colour_h[inc[t]];
        if (c2 >= 0) seen[c2] = e;
      }
    }
    int32_t c = 0;
    while (c < (int32_t)seen.size() && seen[c] == e) ++c;
    if (c == (int32_t)seen.size()) seen.push_back(-1);
    as->colour_h[e] = c;
  }
  as->n_colours = (int32_t)seen.size();
  // 3. pattern.  Each element's functions sorted, with the rank of local j.
  std::vector<int64_t> sorted(l2g, l2g + loff[n]);
  std::vector<uint16_t> rank(loff[n]);
  for (int64_t e = 0; e < n; ++e) {
    std::sort(sorted.begin() + loff[e], sorted.begin() + loff[e + 1]);
    for (int64_t k = loff[e]; k < loff[e + 1]; ++k)
      rank[k] = (uint16_t)(std::lower_bound(sorted.begin() + loff[e], sorted.begin() + loff[e + 1], l2g[k]) -
                           (sorted.begin() + loff[e]));
  }
  std::vector<int64_t> row_ptr(nd + 1, 0);
  std::fill(stamp.begin(), stamp.end(), -1);
  for (int64_t d = 0; d < nd; ++d) {
    int64_t len = 0;
    if (inc_ptr[d + 1] - inc_ptr[d] == 1) {
      const int32_t e = inc[inc_ptr[d]];
      len = loff[e + 1] - loff[e];
    } else {
      for (int64_t t = inc_ptr[d]; t < inc_ptr[d + 1]; ++t) {
        const int32_t e = inc[t];
        for (int64_t k = loff[e]; k < loff[e + 1]; ++k)
          if (stamp[l2g[k]] != d) {
            stamp[l2g[k]] = d;
            ++len;
          }
      }
    }
    if (len > 65535)
      return set_error(FEI_ERR_UNSUPPORTED, "row %lld has %lld nonzeros (at most 65535)", (long long)d, (long long)len);
    row_ptr[d + 1] = row_ptr[d] + len;
  }
  as->nnz = row_ptr[nd];
  std::vector<int32_t> col_idx;
  try {
    col_idx.resize(as->nnz);
  } catch (const std::bad_alloc &) {
    return set_error(FEI_ERR_OOM, "fei_assembly_create: host pattern of %lld entries", (long long)as->nnz);
  }
  std::fill(stamp.begin(), stamp.end(), -1);
  std::vector<int64_t> tmp;
  for (int64_t d = 0; d < nd; ++d) {
    int32_t *dst = col_idx.data() + row_ptr[d];
    if (inc_ptr[d + 1] - inc_ptr[d] == 1) {
      const int32_t e = inc[inc_ptr[d]];
      for (int64_t k = loff[e]; k < loff[e + 1]; ++k) *dst++ = (int32_t)sorted[k];
    } else {
      tmp.clear();
      for (int64_t t = inc_ptr[d]; t < inc_ptr[d + 1]; ++t) {
        const int32_t e = inc[t];
        for (int64_t k = loff[e]; k < loff[e + 1]; ++k)
          if (stamp[l2g[k]] != d) {
            stamp[l2g[k]] = d;
            tmp.push_back(l2g[k]);
          }
      }
      std::sort(tmp.begin(), tmp.end());
      for (const int64_t c : tmp) *dst++ = (int32_t)c;
    }
  }
  // 4. scatter map
  std::vector<uint16_t> off;
  try {
    off.resize(moff[n]);
  } catch (const std::bad_alloc &) {
    return set_error(FEI_ERR_OOM, "fei_assembly_create: host scatter map of %lld entries", (long long)moff[n]);
  }
  for (int64_t e = 0; e < n; ++e) {
    const int64_t s = loff[e + 1] - loff[e];
    for (int64_t i = 0; i < s; ++i) {
      const int64_t r = l2g[loff[e] + i];
      uint16_t *o = off.data() + moff[e] + i * s;
      if (inc_ptr[r + 1] - inc_ptr[r] == 1) {
        for (int64_t j = 0; j < s; ++j) o[j] = rank[loff[e] + j];
      } else {
        const int32_t *b = col_idx.data() + row_ptr[r], *end = col_idx.data() + row_ptr[r + 1];
        for (int64_t j = 0; j < s; ++j) o[j] = (uint16_t)(std::lower_bound(b, end, (int32_t)l2g[loff[e] + j]) - b);
      }
    }
  }
  // 5. elements by (colour, degree), colour ranges, chunks
  std::vector<int32_t> elems(n);
  for (int64_t e = 0; e < n; ++e) elems[e] = (int32_t)e;
  std::stable_sort(elems.begin(), elems.end(), [&](int32_t x, int32_t y) {
    return as->colour_h[x] != as->colour_h[y] ? as->colour_h[x] < as->colour_h[y]
                                              : as->degree_h[x] < as->degree_h[y];
  });
  as->colour_start.assign(as->n_colours + 1, 0);
  for (int64_t e = 0; e < n; ++e) ++as->colour_start[as->colour_h[e] + 1];
  for (int32_t c = 0; c < as->n_colours; ++c) as->colour_start[c + 1] += as->colour_start[c];
  std::vector<int64_t> scr_aoff(n), scr_boff(n);
  as->chunks.clear();
  as->max_chunk_a = as->max_chunk_b = 0;
  for (int64_t k = 0; k < n;) {
    const int32_t e0 = elems[k], c = as->colour_h[e0], p = as->degree_h[e0];
    const int64_t s = nsh_of(p);
    // enough elements for a few tiles per SM, and no more than the L2 budget
    // allows beyond that
    int64_t cap = kChunkBytes / (4 * s * s);
    const int64_t tiles_min = 8ll * 152 * 128 / s;
    if (cap < tiles_min) cap = tiles_min;
    fei_assembly::Chunk ch{c, p, k, 0, 0, 0};
    while (k < n && ch.n < cap && as->colour_h[elems[k]] == c && as->degree_h[elems[k]] == p) {
      scr_aoff[elems[k]] = ch.a_len;
      scr_boff[elems[k]] = ch.b_len;
      ch.a_len += s * s;
      ch.b_len += s;
      ++ch.n;
      ++k;
    }
    as->max_chunk_a = std::max(as->max_chunk_a, ch.a_len);
    as->max_chunk_b = std::max(as->max_chunk_b, ch.b_len);
    as->chunks.push_back(ch);
  }
  if (as->host_only) {
    as->row_ptr_h.swap(row_ptr);
    as->col_idx_h.swap(col_idx);
    return FEI_OK;
  }
  std::vector<int32_t> ccount(as->chunks.size());
  for (size_t i = 0; i < as->chunks.size(); ++i) ccount[i] = (int32_t)as->chunks[i].n;
  fei_status st;
  if ((st = upload(&as->row_ptr, row_ptr.data(), row_ptr.size()))) return st;
  if ((st = upload(&as->col_idx, col_idx.data(), col_idx.size()))) return st;
  if ((st = upload(&as->l2g, l2g, (size_t)loff[n]))) return st;
  if ((st = upload(&as->loff, loff.data(), loff.size()))) return st;
  if ((st = upload(&as->moff, moff.data(), moff.size()))) return st;
  if ((st = upload(&as->off, off.data(), off.size()))) return st;
  if ((st = upload(&as->degree, as->degree_h.data(), as->degree_h.size()))) return st;
  if ((st = upload(&as->elems, elems.data(), elems.size()))) return st;
  if ((st = upload(&as->chunk_count, ccount.data(), ccount.size()))) return st;
  if ((st = upload(&as->scr_aoff, scr_aoff.data(), scr_aoff.size()))) return st;
  if ((st = upload(&as->scr_boff, scr_boff.data(), scr_boff.size()))) return st;
  return FEI_OK;
}

fei_status value_type(fei_precision prec, size_t *bytes) {
  if (prec == FEI_FP64) *bytes = 8;
  else if (prec == FEI_FP32 || prec == FEI_TC_F16X3) *bytes = 4;
  else return set_error(FEI_ERR_INVALID_ARG, "precision %d", (int)prec);
  return FEI_OK;
}

fei_status check_device(const fei_assembly *as) {
  if (!as) return set_error(FEI_ERR_INVALID_ARG, "assembly is NULL");
  if (as->host_only) return set_error(FEI_ERR_INVALID_ARG, "a host-only assembly has no device data");
  int dev;
  FEI_CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev != as->device)
    return set_error(FEI_ERR_INVALID_ARG, "assembly was created on device %d, current device is %d", as->device, dev);
  return FEI_OK;
}

}  // namespace
}  // namespace fei

using namespace fei;

extern "C" fei_status fei_assembly_create(int64_t n_elem, const int32_t *degree, int32_t uniform_degree,
                                          const int64_t *l2g, int64_t n_dof, int32_t flags, fei_assembly_t *out) {
  if (!out) return set_error(FEI_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n_elem < 1 || n_elem > 2147483647LL)
    return set_error(FEI_ERR_INVALID_ARG, "n_elem %lld outside 1..2^31-1", (long long)n_elem);
  if (n_dof < 1 || n_dof > 2147483647LL)
    return set_error(FEI_ERR_INVALID_ARG, "n_dof %lld outside 1..2^31-1", (long long)n_dof);
  if (!l2g) return set_error(FEI_ERR_INVALID_ARG, "l2g is NULL");
  if (flags & ~FEI_ASSEMBLY_HOST_ONLY) return set_error(FEI_ERR_INVALID_ARG, "flags %d", flags);
  if (!degree && (uniform_degree < 1 || uniform_degree > kPMax))
    return set_error(FEI_ERR_INVALID_DEGREE, "uniform_degree %d outside 1..7", uniform_degree);
  fei_assembly *as = new (std::nothrow) fei_assembly();
  if (!as) return set_error(FEI_ERR_OOM, "fei_assembly_create: host allocation");
  as->n_elem = n_elem;
  as->n_dof = n_dof;
  as->host_only = (flags & FEI_ASSEMBLY_HOST_ONLY) != 0;
  as->uniform_degree = degree ? 0 : uniform_degree;
  as->device = -1;
  fei_status st = FEI_OK;
  try {
    as->degree_h.resize(n_elem);
  } catch (const std::bad_alloc &) {
    delete as;
    return set_error(FEI_ERR_OOM, "fei_assembly_create: host allocation");
  }
  for (int64_t e = 0; e < n_elem; ++e) {
    const int32_t p = degree ? degree[e] : uniform_degree;
    if (p < 1 || p > kPMax) {
      delete as;
      return set_error(FEI_ERR_INVALID_DEGREE, "degree[%lld] = %d outside 1..7", (long long)e, p);
    }
    as->degree_h[e] = p;
  }
  if (!as->host_only) {
    cudaError_t e = cudaGetDevice(&as->device);
    if (e != cudaSuccess) {
      delete as;
      return cuda_error(e, "cudaGetDevice");
    }
  }
  try {
    st = build(as, l2g);
  } catch (const std::bad_alloc &) {
    st = set_error(FEI_ERR_OOM, "fei_assembly_create: host allocation");
  }
  if (st) {
    if (!as->host_only) free_device(as);
    delete as;
    return st;
  }
  *out = as;
  return FEI_OK;
}

extern "C" fei_status fei_assembly_destroy(fei_assembly_t as) {
  if (!as) return FEI_OK;
  if (!as->host_only) free_device(as);
  delete as;
  return FEI_OK;
}

extern "C" fei_status fei_assembly_info(fei_assembly_t as, int64_t *n_dof, int64_t *nnz, int32_t *n_colours,
                                        int32_t *n_chunks) {
  if (!as) return set_error(FEI_ERR_INVALID_ARG, "assembly is NULL");
  if (n_dof) *n_dof = as->n_dof;
  if (nnz) *nnz = as->nnz;
  if (n_colours) *n_colours = as->n_colours;
  if (n_chunks) *n_chunks = (int32_t)as->chunks.size();
  return FEI_OK;
}

extern "C" fei_status fei_assembly_pattern(fei_assembly_t as, int64_t *row_ptr, int32_t *col_idx,
                                           int32_t *colour) {
  if (!as) return set_error(FEI_ERR_INVALID_ARG, "assembly is NULL");
  if (colour) memcpy(colour, as->colour_h.data(), sizeof(int32_t) * as->n_elem);
  if (as->host_only) {
    if (row_ptr) memcpy(row_ptr, as->row_ptr_h.data(), sizeof(int64_t) * (as->n_dof + 1));
    if (col_idx) memcpy(col_idx, as->col_idx_h.data(), sizeof(int32_t) * as->nnz);
    return FEI_OK;
  }
  if (row_ptr)
    FEI_CUDA_TRY(cudaMemcpy(row_ptr, as->row_ptr, sizeof(int64_t) * (as->n_dof + 1), cudaMemcpyDeviceToHost),
                 "cudaMemcpy (row_ptr)");
  if (col_idx && as->nnz)
    FEI_CUDA_TRY(cudaMemcpy(col_idx, as->col_idx, sizeof(int32_t) * as->nnz, cudaMemcpyDeviceToHost),
                 "cudaMemcpy (col_idx)");
  return FEI_OK;
}

extern "C" fei_status fei_assemble(fei_assembly_t as, fei_precision prec, const void *A, const void *b,
                                   void *values, void *rhs, fei_stream_t stream) {
  fei_status st = check_device(as);
  if (st) return st;
  size_t vb;
  if ((st = value_type(prec, &vb))) return st;
  if (!A || !b || !values || !rhs) return set_error(FEI_ERR_INVALID_ARG, "A, b, values and rhs are required");
  cudaStream_t s = (cudaStream_t)stream;
  FEI_CUDA_TRY(cudaMemsetAsync(values, 0, vb * as->nnz, s), "cudaMemsetAsync(values)");
  FEI_CUDA_TRY(cudaMemsetAsync(rhs, 0, vb * as->n_dof, s), "cudaMemsetAsync(rhs)");
  for (int32_t c = 0; c < as->n_colours; ++c) {
    const int64_t k0 = as->colour_start[c], k1 = as->colour_start[c + 1];
    st = vb == 8 ? launch_assemble<double>(as, as->elems + k0, k1 - k0, A, as->moff, b, as->loff, values, rhs, s)
                 : launch_assemble<float>(as, as->elems + k0, k1 - k0, A, as->moff, b, as->loff, values, rhs, s);
    if (st) return st;
  }
  return FEI_OK;
}

extern "C" fei_status fei_integrate_assemble(fei_assembly_t as, const fei_reference_t *refs, int nrefs,
                                             const fei_batch *batch, fei_precision prec, void *values, void *rhs,
                                             int32_t *elem_status, fei_stream_t stream) {
  fei_status st = check_device(as);
  if (st) return st;
  if (!batch) return set_error(FEI_ERR_INVALID_ARG, "batch is NULL");
  // the element outputs go to the scratch: the batch's A_offset and b_offset
  // are not used (the natural layout stands in for the checks)
  fei_batch bt = *batch;
  bt.A_offset = as->moff;
  bt.b_offset = as->loff;
  batch = &bt;
  if ((st = check_batch(batch))) return st;
  size_t vb;
  if ((st = value_type(prec, &vb))) return st;
  if (batch->n_elem != as->n_elem)
    return set_error(FEI_ERR_INVALID_ARG, "batch has %lld elements, the assembly %lld", (long long)batch->n_elem,
                     (long long)as->n_elem);
  if ((batch->degree == nullptr) != (as->uniform_degree != 0) ||
      (!batch->degree && batch->uniform_degree != as->uniform_degree))
    return set_error(FEI_ERR_INVALID_ARG, "batch degrees differ from the assembly's");
  if (!values || !rhs || !elem_status) return set_error(FEI_ERR_INVALID_ARG, "values, rhs and elem_status are required");
  const fei_reference *by_p[kPMax + 1];
  if ((st = check_refs(refs, nrefs, as->device, by_p))) return st;
  for (const auto &ch : as->chunks)
    if (!by_p[ch.degree]) return set_error(FEI_ERR_INVALID_DEGREE, "no reference for degree %d", ch.degree);
  // scratch for the largest chunk (FP64 size, so that any precision fits)
  const size_t need_a = 8 * (size_t)as->max_chunk_a, need_b = 8 * (size_t)as->max_chunk_b;
  if (as->scratch_A_bytes < need_a) {
    cudaFree(as->scratch_A);
    as->scratch_A = nullptr;
    as->scratch_A_bytes = 0;
    cudaError_t e = cudaMalloc(&as->scratch_A, need_a);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? set_error(FEI_ERR_OOM, "assembly scratch") : cuda_error(e, "cudaMalloc");
    as->scratch_A_bytes = need_a;
  }
  if (as->scratch_b_bytes < need_b) {
    cudaFree(as->scratch_b);
    as->scratch_b = nullptr;
    as->scratch_b_bytes = 0;
    cudaError_t e = cudaMalloc(&as->scratch_b, need_b);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? set_error(FEI_ERR_OOM, "assembly scratch") : cuda_error(e, "cudaMalloc");
    as->scratch_b_bytes = need_b;
  }
  cudaStream_t s = (cudaStream_t)stream;
  FEI_CUDA_TRY(cudaMemsetAsync(values, 0, vb * as->nnz, s), "cudaMemsetAsync(values)");
  FEI_CUDA_TRY(cudaMemsetAsync(rhs, 0, vb * as->n_dof, s), "cudaMemsetAsync(rhs)");
  for (size_t ci = 0; ci < as->chunks.size(); ++ci) {
    const auto &ch = as->chunks[ci];
    const fei_reference *r = by_p[ch.degree];
    FwdArgs a;
    fill_fwd(a, batch, r, as->scratch_A, as->scratch_b, elem_status);
    a.n_work = ch.n;
    a.count = as->chunk_count + ci;
    a.list = as->elems + ch.start;
    a.A_off = as->scr_aoff;
    a.b_off = as->scr_boff;
    if ((st = launch_forward(ch.degree, prec, r, a, ch.n, s))) return st;
    st = vb == 8 ? launch_assemble<double>(as, a.list, ch.n, as->scratch_A, as->scr_aoff, as->scratch_b, as->scr_boff,
                                           values, rhs, s)
                 : launch_assemble<float>(as, a.list, ch.n, as->scratch_A, as->scr_aoff, as->scratch_b, as->scr_boff,
                                          values, rhs, s);
    if (st) return st;
  }
  return FEI_OK;
}
