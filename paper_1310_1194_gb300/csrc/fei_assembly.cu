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
//   4. scatter map.  A row that only one element touches ("private") holds
//      exactly that element's functions, sorted, so entry (i, j) goes to the
//      rank of l2g_e[j] among them, the same for every private row of the
//      element: one uint16 rank per local function.  A shared row needs its
//      own offsets: for each shared local row i, the place of every l2g_e[j]
//      in row l2g_e[i] (uint16), reached through a per-row slot;
//   5. elements sorted by (degree, colour): the runs of equal (degree,
//      colour) are the assembly launches, in that order, for both entry
//      points (so both add the contributions of a shared entry in the same
//      order); for the fused path, the elements of one degree split into
//      chunks where a chunk's element matrices would pass a size cap.
// Device part (fei_assemble): the shared rows are cleared, then a block
// per element stores its entries of private rows (the only contribution
// they get) and adds those of shared rows, one launch per (degree, colour)
// run.  fei_integrate_assemble integrates the batch chunk by chunk into one
// scratch buffer (one forward launch per chunk, all colours of a degree
// together) and assembles each chunk from it run by run, so that a batch
// never needs memory for all of its element matrices at once.
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
  std::vector<int64_t> run_start;  // runs of equal (degree, colour) in elems: [runs + 1]
  std::vector<int32_t> run_degree;  // [runs]
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
  int64_t *moff;     // start of element e in A (sum of N_sh^2)
  uint16_t *rank;    // [loff layout] rank of l2g_e[j] among the element's functions
  int16_t *slot;     // [loff layout] shared-row slot of local row i, -1 = private
  int64_t *shptr;    // [n_elem] start of element e's shared-row offsets in shoff
  uint16_t *shoff;   // per shared row: the N_sh places of the element's columns
  int32_t *shrows;   // global rows touched by several elements (cleared first)
  int64_t n_shrows;
  int32_t *elems;        // elements sorted by (colour, degree)
  int32_t *chunk_count;  // [chunks] element count of each chunk (the forward's device count)
  int64_t *scr_aoff, *scr_boff;  // start of element e in its chunk's scratch
  // fused path: two scratch buffers (chunk k uses buffer k % 2), the stream
  // that assembles while the caller's stream integrates the next chunk, and
  // the events that order the two
  // fused path: the chunk scratch (element matrices and vectors), allocated
  // on first use
  void *scratch_A, *scratch_b;
  size_t scratch_A_bytes, scratch_b_bytes;
};

namespace fei {
namespace {

constexpr int64_t kChunkBytes = 256ll << 20;  // cap of one chunk's FP32 element matrices

template <typename T>
__global__ void clear_rows_kernel(const int32_t *rows, int64_t n, const int64_t *row_ptr, T *values) {
  for (int64_t k = blockIdx.x; k < n; k += gridDim.x) {
    const int64_t r0 = row_ptr[rows[k]], r1 = row_ptr[rows[k] + 1];
    for (int64_t t = r0 + threadIdx.x; t < r1; t += blockDim.x) values[t] = T(0);
  }
}

// One run of elements of a single degree (s functions each) that share no
// global function: work unit u is rows [rb part, rb part + rb) of element
// k = u / units_per_element (a warp per row, lanes over columns), so that a
// run of few large elements still fills the GPU.
template <typename T>
__global__ void assemble_kernel(const int32_t *elems, int64_t n, int s, int rb, const T *A, const int64_t *aoff,
                                const T *bv, const int64_t *boff, const int64_t *l2g, const int64_t *loff,
                                const uint16_t *rank, const int16_t *slot, const int64_t *shptr,
                                const uint16_t *shoff, const int64_t *row_ptr, T *values, T *rhs) {
  __shared__ int64_t rstart[nsh_of(kPMax)];
  __shared__ int16_t sl[nsh_of(kPMax)];
  __shared__ uint16_t rk[nsh_of(kPMax)];
  const int upe = (s + rb - 1) / rb;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int64_t u = blockIdx.x; u < n * upe; u += gridDim.x) {
    const int64_t k = u / upe;
    const int i0 = (int)(u - k * upe) * rb;
    const int nr = s - i0 < rb ? s - i0 : rb;
    const int e = elems[k];
    const int64_t lo = loff[e];
    __syncthreads();  // the previous unit's row data are no longer read
    for (int j = threadIdx.x; j < s; j += blockDim.x) rk[j] = rank[lo + j];
    for (int t = threadIdx.x; t < nr; t += blockDim.x) {
      const int64_t g = l2g[lo + i0 + t];
      rstart[t] = row_ptr[g];
      sl[t] = slot[lo + i0 + t];
      rhs[g] += bv[boff[e] + i0 + t];
    }
    __syncthreads();
    const T *Ae = A + aoff[e];
    const uint16_t *so = shoff + shptr[e];
    for (int t = warp; t < nr; t += nw) {
      const int i = i0 + t, q = sl[t];
      const int64_t base = rstart[t];
      const T *Ai = Ae + (int64_t)i * s;
      if (q < 0) {
        for (int j = lane; j < s; j += 32) values[base + rk[j]] = Ai[j];  // a private row: its only contribution
      } else {
        const uint16_t *o = so + q * s;
        for (int j = lane; j < s; j += 32) values[base + o[j]] += Ai[j];
      }
    }
  }
}

// elems[0 .. n): one run (one degree p)
template <typename T>
fei_status launch_assemble(const fei_assembly *as, int p, const int32_t *elems, int64_t n, const void *A,
                           const int64_t *aoff, const void *bv, const int64_t *boff, void *values, void *rhs,
                           cudaStream_t s) {
  if (n <= 0) return FEI_OK;
  const int sh = nsh_of(p);
  // rows per work unit: whole elements when the run has enough of them,
  // else split so that the run gives about 8 units per SM (at least 32 rows)
  int64_t rb = (n * sh + 152 * 8 - 1) / (152 * 8);
  rb = rb < 32 ? 32 : (rb > sh ? sh : rb);
  const int64_t units = n * ((sh + rb - 1) / rb);
  const int64_t blocks = units < 152 * 16 ? units : 152 * 16;
  assemble_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(elems, n, sh, (int)rb, (const T *)A, aoff, (const T *)bv, boff,
                                                      as->l2g, as->loff, as->rank, as->slot, as->shptr, as->shoff,
                                                      as->row_ptr, (T *)values, (T *)rhs);
  FEI_CUDA_TRY(cudaGetLastError(), "assemble_kernel launch");
  return debug_check(s, "assemble_kernel");
}

// values of the shared rows and the whole rhs set to zero (private rows are
// stored, not added, by the assembly)
fei_status clear_outputs(const fei_assembly *as, size_t vb, void *values, void *rhs, cudaStream_t s) {
  FEI_CUDA_TRY(cudaMemsetAsync(rhs, 0, vb * as->n_dof, s), "cudaMemsetAsync(rhs)");
  if (as->n_shrows == 0) return FEI_OK;
  const int64_t blocks = as->n_shrows < 152 * 16 ? as->n_shrows : 152 * 16;
  if (vb == 8)
    clear_rows_kernel<double><<<(unsigned)blocks, 256, 0, s>>>(as->shrows, as->n_shrows, as->row_ptr, (double *)values);
  else
    clear_rows_kernel<float><<<(unsigned)blocks, 256, 0, s>>>(as->shrows, as->n_shrows, as->row_ptr, (float *)values);
  FEI_CUDA_TRY(cudaGetLastError(), "clear_rows_kernel launch");
  return debug_check(s, "clear_rows_kernel");
}

void free_device(fei_assembly *as) {
  cudaFree(as->row_ptr);
  cudaFree(as->col_idx);
  cudaFree(as->l2g);
  cudaFree(as->loff);
  cudaFree(as->moff);
  cudaFree(as->rank);
  cudaFree(as->slot);
  cudaFree(as->shptr);
  cudaFree(as->shoff);
  cudaFree(as->shrows);
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
  // 4. scatter map: ranks (computed above), slots of shared rows and
  // their offsets, and the list of shared rows
  std::vector<int16_t> slot(loff[n], -1);
  std::vector<int64_t> shptr(n + 1, 0);
  for (int64_t e = 0; e < n; ++e) {
    const int64_t s = loff[e + 1] - loff[e];
    int64_t q = 0;
    for (int64_t i = 0; i < s; ++i) {
      const int64_t r = l2g[loff[e] + i];
      if (inc_ptr[r + 1] - inc_ptr[r] > 1) slot[loff[e] + i] = (int16_t)q++;
    }
    shptr[e + 1] = shptr[e] + q * s;
  }
  std::vector<uint16_t> shoff(shptr[n]);
  for (int64_t e = 0; e < n; ++e) {
    const int64_t s = loff[e + 1] - loff[e];
    for (int64_t i = 0; i < s; ++i) {
      const int16_t q = slot[loff[e] + i];
      if (q < 0) continue;
      const int64_t r = l2g[loff[e] + i];
      const int32_t *b = col_idx.data() + row_ptr[r], *end = col_idx.data() + row_ptr[r + 1];
      uint16_t *o = shoff.data() + shptr[e] + q * s;
      for (int64_t j = 0; j < s; ++j) o[j] = (uint16_t)(std::lower_bound(b, end, (int32_t)l2g[loff[e] + j]) - b);
    }
  }
  std::vector<int32_t> shrows;
  for (int64_t d = 0; d < nd; ++d)
    if (inc_ptr[d + 1] - inc_ptr[d] > 1) shrows.push_back((int32_t)d);
  as->n_shrows = (int64_t)shrows.size();
  // 5. elements by (degree, colour), runs, chunks
  std::vector<int32_t> elems(n);
  for (int64_t e = 0; e < n; ++e) elems[e] = (int32_t)e;
  std::stable_sort(elems.begin(), elems.end(), [&](int32_t x, int32_t y) {
    return as->degree_h[x] != as->degree_h[y] ? as->degree_h[x] < as->degree_h[y]
                                              : as->colour_h[x] < as->colour_h[y];
  });
  as->run_start.assign(1, 0);
  as->run_degree.clear();
  for (int64_t k = 1; k <= n; ++k)
    if (k == n || as->degree_h[elems[k]] != as->degree_h[elems[k - 1]] ||
        as->colour_h[elems[k]] != as->colour_h[elems[k - 1]]) {
      as->run_degree.push_back(as->degree_h[elems[k - 1]]);
      as->run_start.push_back(k);
    }
  std::vector<int64_t> scr_aoff(n), scr_boff(n);
  as->chunks.clear();
  as->max_chunk_a = as->max_chunk_b = 0;
  for (int64_t k = 0; k < n;) {
    const int32_t e0 = elems[k], c = as->colour_h[e0], p = as->degree_h[e0];
    const int64_t s = nsh_of(p);
    // all elements of a degree unless their matrices pass the cap (the
    // forward kernels want large launches), and at least a few tiles per SM
    int64_t cap = kChunkBytes / (4 * s * s);
    const int64_t tiles_min = 8ll * 152 * 128 / s;
    if (cap < tiles_min) cap = tiles_min;
    fei_assembly::Chunk ch{c, p, k, 0, 0, 0};
    while (k < n && ch.n < cap && as->degree_h[elems[k]] == p) {
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
  if ((st = upload(&as->rank, rank.data(), rank.size()))) return st;
  if ((st = upload(&as->slot, slot.data(), slot.size()))) return st;
  if ((st = upload(&as->shptr, shptr.data(), shptr.size()))) return st;
  if ((st = upload(&as->shoff, shoff.data(), shoff.size()))) return st;
  if ((st = upload(&as->shrows, shrows.data(), shrows.size()))) return st;
  if ((st = upload(&as->elems, elems.data(), elems.size()))) return st;
  if ((st = upload(&as->chunk_count, ccount.data(), ccount.size()))) return st;

  if ((st = upload(&as->scr_aoff, scr_aoff.data(), scr_aoff.size()))) return st;
  if ((st = upload(&as->scr_boff, scr_boff.data(), scr_boff.size()))) return st;
  return FEI_OK;
}

fei_status value_type(fei_precision prec, size_t *bytes) {
  if (prec == FEI_FP64) *bytes = 8;
  else if (valid_precision(prec)) *bytes = 4;
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
  const Range range_("fei_assemble");
  fei_status st = check_device(as);
  if (st) return st;
  size_t vb;
  if ((st = value_type(prec, &vb))) return st;
  if (!A || !b || !values || !rhs) return set_error(FEI_ERR_INVALID_ARG, "A, b, values and rhs are required");
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = clear_outputs(as, vb, values, rhs, s))) return st;
  for (size_t r = 0; r + 1 < as->run_start.size(); ++r) {
    const int64_t k0 = as->run_start[r], k1 = as->run_start[r + 1];
    const int p = as->run_degree[r];
    st = vb == 8 ? launch_assemble<double>(as, p, as->elems + k0, k1 - k0, A, as->moff, b, as->loff, values, rhs, s)
                 : launch_assemble<float>(as, p, as->elems + k0, k1 - k0, A, as->moff, b, as->loff, values, rhs, s);
    if (st) return st;
  }
  return FEI_OK;
}

extern "C" fei_status fei_integrate_assemble(fei_assembly_t as, const fei_reference_t *refs, int nrefs,
                                             const fei_batch *batch, fei_precision prec, void *values, void *rhs,
                                             int32_t *elem_status, fei_stream_t stream) {
  const Range range_("fei_integrate_assemble");
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
  if (batch->a_layout != FEI_A_FULL)
    return set_error(FEI_ERR_UNSUPPORTED, "fei_integrate_assemble: assembly takes the full A_e layout");
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
  // the chunk scratch (FP64 size, so that any precision fits), on first use
  const size_t need_a = 8 * (size_t)as->max_chunk_a, need_b = 8 * (size_t)as->max_chunk_b;
  if (as->scratch_A_bytes < need_a || as->scratch_b_bytes < need_b) {
    cudaFree(as->scratch_A);
    cudaFree(as->scratch_b);
    as->scratch_A = as->scratch_b = nullptr;
    as->scratch_A_bytes = as->scratch_b_bytes = 0;
    cudaError_t e = cudaMalloc(&as->scratch_A, need_a);
    if (e == cudaSuccess) e = cudaMalloc(&as->scratch_b, need_b);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? set_error(FEI_ERR_OOM, "assembly scratch") : cuda_error(e, "cudaMalloc");
    }
    as->scratch_A_bytes = need_a;
    as->scratch_b_bytes = need_b;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = clear_outputs(as, vb, values, rhs, s))) return st;
  // chunk by chunk, in (colour, degree) order: integrate into the scratch,
  // then assemble from it (the next chunk's forward follows on the stream)
  for (size_t ci = 0; ci < as->chunks.size(); ++ci) {
    const auto &ch = as->chunks[ci];
    const fei_reference *r = by_p[ch.degree];
    FwdArgs a;
    fill_fwd(a, batch, r, as->scratch_A, as->scratch_b, elem_status);
    a.n_work = ch.n;
    a.count = as->chunk_count + ci;
    a.list = as->elems + ch.start;
    a.A_off = nullptr;
    a.b_off = nullptr;
    a.out_by_item = 1;  // the chunk's matrices in list order: scr_aoff / scr_boff
    if ((st = launch_forward(ch.degree, prec, r, a, ch.n, s))) return st;
    // the chunk's part of each (degree, colour) run, one launch each
    const int64_t c0 = ch.start, c1 = ch.start + ch.n;
    const size_t r0 = std::upper_bound(as->run_start.begin(), as->run_start.end(), c0) - as->run_start.begin() - 1;
    for (size_t rr = r0; rr + 1 < as->run_start.size() && as->run_start[rr] < c1; ++rr) {
      const int64_t k0 = std::max(as->run_start[rr], c0), k1 = std::min(as->run_start[rr + 1], c1);
      st = vb == 8 ? launch_assemble<double>(as, ch.degree, as->elems + k0, k1 - k0, as->scratch_A, as->scr_aoff,
                                             as->scratch_b, as->scr_boff, values, rhs, s)
                   : launch_assemble<float>(as, ch.degree, as->elems + k0, k1 - k0, as->scratch_A, as->scr_aoff,
                                            as->scratch_b, as->scr_boff, values, rhs, s);
      if (st) return st;
    }
  }
  return FEI_OK;
}
