/*
 * fei.h -- C ABI of the GB300 element-integration library (libfei.so).
 *
 * The library computes, for a batch of bilinear prismatic finite elements of
 * degree p = 1..7, the element stiffness matrices and load vectors of the
 * weak form
 *
 *     a(u, v) = int  grad v . K grad u  +  v b . grad u  +  c u v,
 *     l(v)    = int  f v,
 *
 * by the standard quadrature of Sec. 2 (Eq. (1) generalised, Eq. (2)):
 *
 *     A_e[i][j] = sum_q w_q det J(xi_q) ( grad phi_i . K_q grad phi_j
 *                                        + phi_i b_q . grad phi_j
 *                                        + c_q phi_i phi_j )
 *     b_e[i]    = sum_q w_q det J(xi_q) f_q phi_i
 *
 * i = test function (row), j = trial function (column), grad phi = J^{-T}
 * grad_ref phi.  Basis: orthonormal Dubiner triangle polynomials times
 * normalised Legendre polynomials in zeta (Table 1: N_sh = (p+1)^2 (p+2)/2),
 * index = k * (p+1)(p+2)/2 + t, k the zeta degree, t over triangle total
 * degree d = m + n ascending then n ascending.  Quadrature: Duffy-collapsed
 * Gauss-Legendre with (p+1)^3 points, point q = (iz*(p+1) + iv)*(p+1) + iu,
 * xi1 = (1+u)(1-v)/4, xi2 = (1+v)/2, zeta = z, w = w_u w_v (1-v)/8 w_z.
 * Reference prism: {xi1, xi2 >= 0, xi1 + xi2 <= 1} x [-1, 1].  Geometry
 * (Sec. 4, bilinear prism): vertices 0, 1, 2 span the bottom triangle at
 * zeta = -1 (counter-clockwise seen from the top), vertex a+3 lies above a.
 *
 * Conventions for every entry point:
 *  - "device" pointers are CUDA device (or managed) memory of the current
 *    device; "host" pointers are ordinary host memory.
 *  - All work is enqueued on the given stream (NULL = legacy default stream)
 *    and is asynchronous unless stated; a return of FEI_OK only means the
 *    work was enqueued.
 *  - The caller owns every buffer it passes; the library never frees them
 *    and keeps no pointer to them after the call returns.
 *  - Failures return a status code; fei_last_error_string() (thread-local)
 *    describes the last failure of the calling thread.  Nothing in the
 *    library aborts the process or traps on the GPU.
 */
#ifndef FEI_H_
#define FEI_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same object as cudaStream_t. */
typedef struct CUstream_st *fei_stream_t;

typedef enum {
  FEI_OK = 0,
  FEI_ERR_INVALID_ARG = 1,       /* null pointer, bad size, bad enum      */
  FEI_ERR_INVALID_DEGREE = 2,    /* p outside 1..7, or no reference for p */
  FEI_ERR_NEGATIVE_JACOBIAN = 3, /* per element: det J <= 0 at a point    */
  FEI_ERR_NONFINITE = 4,         /* per element: NaN/Inf input or det J   */
  FEI_ERR_CUDA = 5,              /* a CUDA runtime call failed            */
  FEI_ERR_TIMEOUT = 6,           /* a bounded device wait gave up         */
  FEI_ERR_UNSUPPORTED = 7,       /* combination not implemented           */
  FEI_ERR_OOM = 8                /* device allocation failed              */
} fei_status;

typedef enum {
  /* Everything in FP64 on the CUDA cores: the plain FP64 GPU path. */
  FEI_FP64 = 0,
  /* FP64 Jacobian columns and w det J; FP32 point operator, FP32
   * contraction on the CUDA cores.  Output FP32. */
  FEI_FP32 = 1,
  /* As FEI_FP32 for the geometry and point operator; the contraction runs
   * on the tcgen05 tensor cores with each operand split into fp16 hi + lo
   * (3 products: hi*hi + hi*lo + lo*hi) and FP32 accumulation in TMEM
   * (operands scaled by powers of two into fp16 range).  Degrees 1 and 2
   * fall back to the FEI_FP32 kernels.  Output FP32. */
  FEI_TC_F16X3 = 2,
  /* As FEI_TC_F16X3 with each operand split into TF32 hi + lo
   * (tcgen05.mma kind::tf32, 3 products, FP32 accumulation): the FP32
   * exponent range needs no scaling, at half the fp16 tensor rate.  The
   * paper computes in single precision (Sec. 4); split bf16 is not offered:
   * bf16's 8 significant bits need three pieces and six products for the
   * same accuracy.  Degrees 1 and 2 fall back to FEI_FP32.  Output FP32. */
  FEI_TC_3XTF32 = 3,
  /* Sum factorisation on the CUDA cores (degrees >= 3): the basis and the
   * collapsed rule are tensor products in (u, v, zeta), so each component
   * of the reference gradient is a sum of one or two products of 1D
   * factors and the sum over points runs as three short sums, u then v
   * then zeta, over the 21 pairs of gradient terms (about 7x fewer
   * multiply-adds than the dense contraction at p = 7).  Geometry and
   * point operator as FEI_FP32, the sums in FP32.  Degrees 1 and 2 fall
   * back to FEI_FP32.  Output FP32. */
  FEI_SF_FP32 = 4,
  /* Per degree, the fastest kernel among those measured within 1e-6 of
   * the FP64 oracle (relative Frobenius norm per element): the FEI_FP32
   * kernels for p <= 2, the FEI_TC_F16X3 kernel for p = 3, 4 and the
   * sum-factorised kernel for p = 5..7 on a direct call; a plan's tuner
   * times the tensor-core variants and the sum-factorised kernel at every
   * p >= 3 and keeps the fastest.  Output FP32. */
  FEI_AUTO = 5
} fei_precision;

typedef enum {
  FEI_COEF_PER_ELEMENT = 0, /* one (K, b, c, f) record per element        */
  FEI_COEF_PER_POINT = 1    /* one record per quadrature point            */
} fei_coef_mode;

/* Layout of each A_e in A_out.  FEI_A_FULL: N_sh x N_sh row-major.
 * FEI_A_UPPER: for a symmetric weak form (b = 0 and K symmetric, so that
 * A_e = A_e^T: the Laplacian-type term of Sec. 2, Eq. (1), plus reaction),
 * only the upper triangle, row by row: row i holds A_e[i][i..N_sh-1], so
 * A_e[i][j] (j >= i) is at i N_sh - i (i+1) / 2 + j and an element takes
 * N_sh (N_sh + 1) / 2 values.  Every coefficient record of an element must
 * have b = 0 and K[k][l] == K[l][k] exactly; an element that does not is
 * flagged FEI_ERR_INVALID_ARG (outputs zero). */
typedef enum {
  FEI_A_FULL = 0,
  FEI_A_UPPER = 1
} fei_a_layout;

/* Opaque per-degree reference data (quadrature, basis tables, tensor-core
 * operand images), resident on the device where it was created. */
typedef struct fei_reference *fei_reference_t;

/* A batch of elements.  All pointers are device pointers (host pointers for
 * fei_integrate_host).
 *  geom      double [n_elem][6][3]  vertex coordinates (layout above).
 *  degree    int32  [n_elem] per-element degree, or NULL: every element has
 *            degree uniform_degree.
 *  coef_mode fei_coef_mode.
 *  K, b, c, f  double [n_rec][3][3], [n_rec][3], [n_rec], [n_rec]; n_rec =
 *            n_elem (per element) or the total number of points (per point,
 *            element e's records start at q_offset[e], point order as above).
 *            K is used as given (row k, column l multiplies d/dx_l of the
 *            trial function in the k-th component); it need not be symmetric.
 *            The library cannot see the arrays' lengths: the caller owns
 *            them and must pass n_rec records (a shorter array is read past
 *            its end; the Python binding refuses one).
 *  A_offset, b_offset, q_offset  int64 [n_elem + 1] start of element e in
 *            A_out (scalars), b_out, and the per-point records; NULL means
 *            the contiguous layout of a uniform degree (e*S, e*N_sh,
 *            e*N_q with S = N_sh^2, or N_sh (N_sh + 1) / 2 for FEI_A_UPPER).
 *            Required when degree != NULL (see fei_plan_offsets).
 *  a_layout  fei_a_layout of A_out (0 = FEI_A_FULL). */
typedef struct {
  int64_t n_elem;
  const double *geom;
  const int32_t *degree;
  int32_t uniform_degree;
  int32_t coef_mode;
  const double *K;
  const double *b;
  const double *c;
  const double *f;
  const int64_t *A_offset;
  const int64_t *b_offset;
  const int64_t *q_offset;
  int32_t a_layout;
} fei_batch;

/* Gradient outputs of fei_integrate_backward, same layouts as the inputs
 * (device pointers, all required). */
typedef struct {
  double *K;
  double *b;
  double *c;
  double *f;
} fei_coef_grad;

/* --------------------------------------------------------------------- */

/* Tabulate the reference data of degree p (Sec. 2.2: quadrature data and
 * shape functions are the same for every element of one type and degree,
 * so they are computed once and kept in fast memory; Table 2 sizes).
 * Runs FP64 kernels on the current device and waits for them.
 * p outside 1..7 -> FEI_ERR_INVALID_DEGREE; out == NULL -> INVALID_ARG.
 * The handle is owned by the caller and released with
 * fei_reference_destroy; it may be shared by threads for reading. */
fei_status fei_reference_create(int p, fei_reference_t *out);
fei_status fei_reference_destroy(fei_reference_t ref);
/* Query degree, N_sh and N_q of a handle (host pointers, any may be NULL). */
fei_status fei_reference_info(fei_reference_t ref, int *p, int *nsh, int *nq);
/* Copy the FP64 reference table to host memory (Table 2 rows 1-2 and 4):
 * pts [N_q][4] = (xi1, xi2, zeta, w), G [N_q][4][N_sh] = phi, dphi/dxi1,
 * dphi/dxi2, dphi/dzeta.  Either pointer may be NULL.  Synchronous. */
fei_status fei_reference_copy_table(fei_reference_t ref, double *pts, double *G);

/* Forward integration (Algorithm 1; the loops over points and shape
 * functions of Sec. 2.1 run in the kernels).
 *  refs/nrefs  host array of handles; the one whose degree matches each
 *              element is used (INVALID_DEGREE if one is missing).
 *  batch       host pointer to the batch description (device data).
 *  A_out       device [sum N_sh^2] output, FP64 for FEI_FP64, FP32 else,
 *              row-major A_e (row i = test function) at A_offset[e].
 *  b_out       device [sum N_sh] output, same precision, at b_offset[e].
 *  elem_status device int32 [n_elem] (required): 0, or
 *              FEI_ERR_NEGATIVE_JACOBIAN / FEI_ERR_NONFINITE for an element
 *              whose outputs are then zero (NONFINITE takes precedence).
 * Uniform-degree batches use no scratch memory.  A batch with a degree
 * array needs a bucketing workspace, which this call allocates on first
 * use per device and keeps; use a plan (below) to allocate up front.
 * Every call with a degree array on one device uses that one workspace:
 * issue such calls on one stream (calls on different streams may overlap
 * on the GPU and race on it), or use plans or pipelines, which own their
 * scratch. */
fei_status fei_integrate(const fei_reference_t *refs, int nrefs,
                         const fei_batch *batch, fei_precision prec,
                         void *A_out, void *b_out, int32_t *elem_status,
                         fei_stream_t stream);

/* Reverse pass: given gA (same layout/precision as A_out) and gb, writes
 * (overwrites) the gradient of L = <gA, A> + <gb, b> with respect to the
 * vertex coordinates g_geom [n_elem][6][3] (FP64) and the coefficients
 * (g_coef, same layout and mode as the inputs, FP64).  Per-point
 * coefficient values are held fixed when differentiating by the geometry.
 * Jacobians are recomputed, not stored.  Precision: FEI_FP64 (all FP64);
 * FEI_FP32 (the contraction W = gA G^T in FP32 on the CUDA cores, the chain
 * in FP32 with det J from FP64 node sums); FEI_TC_F16X3 or FEI_AUTO with a
 * uniform degree 3..5: dL/dDt_q = G_q gA G_q^T with W^T = G gA^T on the
 * tensor cores (each gA row split into fp16 hi + lo with its own
 * power-of-two scale, three products per K slice) and the FP32 chain, in
 * chunks of 8192 elements (FEI_ADJOINT_CHUNK in the environment overrides
 * it) with 64 N_q bytes of scratch per element allocated stream-ordered on
 * the stream; every other precision and case runs as FEI_FP32.  gA and gb
 * are FP32 for every precision but FEI_FP64.
 * Elements with a nonzero elem_status from the forward get zero gradients
 * (this call recomputes the status itself).  batch->a_layout must be
 * FEI_A_FULL (FEI_ERR_UNSUPPORTED otherwise). */
fei_status fei_integrate_backward(const fei_reference_t *refs, int nrefs,
                                  const fei_batch *batch, fei_precision prec,
                                  const void *gA, const void *gb,
                                  double *g_geom, const fei_coef_grad *g_coef,
                                  fei_stream_t stream);

/* Adjoint of the quadratic loss L = sum_e u_e^T A_e u_e - u_e^T b_e (the
 * energy of a field u; not in the paper): the gradients fei_integrate_backward
 * gives for gA_e = u_e u_e^T and gb_e = -u_e, computed without forming gA.
 * With v_q = G_q u_e (value and reference gradient of the field at point q),
 * dL/dDt_q = v_q v_q^T and dL/d(w det J f)_q = -v_q[0], so the cost per
 * element is O(N_sh N_q) instead of O(N_sh^2 N_q).
 *  u  device double [b_total]: u_e at b_offset[e] (the layout of b_out).
 * Other arguments, outputs, precisions and errors as for
 * fei_integrate_backward (FEI_FP32: v_q in FP32, the Jacobian chain in
 * FP64). */
fei_status fei_integrate_backward_quadratic(const fei_reference_t *refs, int nrefs,
                                            const fei_batch *batch, fei_precision prec,
                                            const double *u, double *g_geom,
                                            const fei_coef_grad *g_coef,
                                            fei_stream_t stream);

/* Contiguous offsets for a degree array (device pointers): A_offset,
 * b_offset, q_offset [n_elem + 1] (any may be NULL).  Also validates the
 * degrees: an element with p outside 1..7 sets *bad_count (device int32,
 * may be NULL) nonzero.  Runs on the stream, asynchronous. */
fei_status fei_plan_offsets(const int32_t *degree, int64_t n_elem,
                            int64_t *A_offset, int64_t *b_offset,
                            int64_t *q_offset, int32_t *bad_count,
                            fei_stream_t stream);
/* The same for A_out in the FEI_A_UPPER layout: A_offset advances by
 * N_sh (N_sh + 1) / 2 per element. */
fei_status fei_plan_offsets_upper(const int32_t *degree, int64_t n_elem,
                                  int64_t *A_offset, int64_t *b_offset,
                                  int64_t *q_offset, int32_t *bad_count,
                                  fei_stream_t stream);

/* --------------------------------------------------------------------- */
/* Plans: a mixed-degree batch as one CUDA graph, with the kernel shape of
 * every degree chosen by measurement.  Elements are grouped by degree so
 * that each degree's tables stay resident (Sec. 2.2); a plan owns the
 * grouping scratch, per degree a kernel variant and grid (defaults, or the
 * fastest measured by fei_plan_tune), and the CUDA graph of its last
 * argument set. */
typedef struct fei_plan *fei_plan_t;

/* refs/nrefs as for fei_integrate (host array, handles of the current
 * device; the plan keeps pointers to them: destroy the plan first).
 * max_elem: largest n_elem of a batch with a degree array (the scratch,
 * 4 * (8 + 7 * max_elem) bytes of device memory, is allocated here and never
 * again).  prec: as for fei_integrate.  Errors: INVALID_ARG (NULL pointers,
 * max_elem outside 0..2^31-1, bad precision, a handle of another device),
 * CUDA/OOM. */
fei_status fei_plan_create(const fei_reference_t *refs, int nrefs, int64_t max_elem,
                           fei_precision prec, fei_plan_t *out);
fei_status fei_plan_destroy(fei_plan_t plan);

/* Same arguments, outputs and statuses as fei_integrate.  The first call
 * with a given (batch contents, A_out, b_out, elem_status) captures the
 * grouping kernel and one kernel per degree into a CUDA graph on `stream`
 * and launches it; later calls with the same pointers replay the graph
 * (one cudaGraphLaunch); different pointers re-capture (updating the
 * graph in place when possible).  The legacy default stream (NULL) cannot
 * be captured: there the kernels are launched directly.  No device memory
 * is allocated.  Calls on one plan must not overlap on the GPU (they share
 * its scratch) and must come from one host thread at a time. */
fei_status fei_plan_execute(fei_plan_t plan, const fei_batch *batch, void *A_out,
                            void *b_out, int32_t *elem_status, fei_stream_t stream);

/* Autotuner: runs every candidate kernel shape of every degree present in
 * `batch` on that degree's elements (writing the same outputs a normal call
 * writes), times each with CUDA events (best of two after one warm-up run)
 * and keeps the fastest per degree.  Candidates: the tensor-core kernel's
 * warp-role variants (p >= 3 under the tensor-core precisions), the
 * sum-factorised kernel with as many blocks as fit or one per SM (p >= 3
 * under FEI_SF_FP32), both of these under FEI_AUTO, or 2/4/8/16 blocks per
 * SM for the CUDA-core kernels.  Synchronous (waits for the stream). */
fei_status fei_plan_tune(fei_plan_t plan, const fei_batch *batch, void *A_out,
                         void *b_out, int32_t *elem_status, fei_stream_t stream);

/* The plan's choice for degree p (host pointers, any may be NULL):
 * variant index, grid cap in blocks (0 = the kernel's default) and the
 * time fei_plan_tune measured for that degree (ms, -1 if not tuned).
 * Variants of degree p >= 3: the tensor-core kernel's warp-role variants
 * 0 .. count - 1 (count: 2 or more, fixed per degree and precision); under
 * FEI_AUTO the variant equal to that count is the sum-factorised kernel. */
fei_status fei_plan_choice(fei_plan_t plan, int p, int *variant, int64_t *grid_cap,
                           float *tuned_ms);

/* Sets the choice for degree p, e.g. one that fei_plan_tune measured in an
 * earlier process on the same GPU model (the tuning cache persisted by the
 * caller).  variant: as fei_plan_choice reports it (0 where a degree has a
 * single kernel); grid_cap: blocks, 0 = the kernel's default.  The plan's graph is recaptured on the next
 * fei_plan_execute.  Errors: INVALID_ARG, INVALID_DEGREE. */
fei_status fei_plan_set_choice(fei_plan_t plan, int p, int variant, int64_t grid_cap);

/* The kernel the plan's current choice runs for degree p (host pointer):
 * 0 the CUDA-core kernels, 1 the tensor-core kernel, 2 the sum-factorised
 * kernel.  Errors: INVALID_ARG (NULL plan or kernel), INVALID_DEGREE. */
fei_status fei_plan_kernel(fei_plan_t plan, int p, int *kernel);

/* Batch-level summary of the per-element statuses (device int32
 * [n_elem], as written by fei_integrate): summary (device int32 [2])
 * receives the worst status (FEI_ERR_NONFINITE over
 * FEI_ERR_NEGATIVE_JACOBIAN over any other nonzero code over FEI_OK) and the
 * number of flagged elements.  Asynchronous on the stream; read summary
 * after the stream has reached this point.  elem_status or summary NULL ->
 * INVALID_ARG (summary may be NULL only when n_elem is 0). */
fei_status fei_status_summary(const int32_t *elem_status, int64_t n_elem, int32_t *summary,
                              fei_stream_t stream);

/* Host-side read of the status summary (the boundary's per-batch error
 * report; Sec. 2 leaves failures unspecified, this library flags them per
 * element): reduces elem_status (device int32 [n_elem], as written by
 * fei_integrate or a plan) on `stream` to the worst status (same order as
 * fei_status_summary) and the number of flagged elements, waits for the
 * stream (so every call enqueued on it before has finished) and writes both
 * to the HOST pointers worst and count.  n_elem == 0 waits for the stream and
 * reports (0, 0).  The reduction goes through a summary word inside libfei
 * (no allocation); calls on one device are serialised.  Errors: INVALID_ARG
 * (NULL pointers, n_elem < 0), CUDA (including a failed kernel earlier on
 * the stream, reported by the wait).  Synchronous. */
fei_status fei_sync_status(const int32_t *elem_status, int64_t n_elem, int32_t *worst, int64_t *count,
                           fei_stream_t stream);

/* Largest batch fei_integrate_noalloc accepts. */
#define FEI_NOALLOC_MAX_ELEM 262144

/* fei_integrate without any device allocation (the paper has no
 * counterpart; this serves callers that cannot allocate).  fei_integrate
 * allocates scratch with cudaMalloc for a batch with a degree array (the
 * per-degree element lists).  Callers that cannot have a library allocate
 * -- code that must never block the device (cudaMalloc can synchronise
 * it), applications whose device memory belongs to a pool or budget the
 * library must not bypass -- call this instead.  Same arguments, layout,
 * outputs and statuses as fei_integrate, and the same values bit for bit;
 * the scratch is a fixed device array inside libfei (4 * (8 + 7 *
 * FEI_NOALLOC_MAX_ELEM) bytes, about 7.3 MB, reserved on every GPU that
 * loads the library until the process exits); no cudaMalloc, cudaFree or
 * allocating routine is called.  n_elem > FEI_NOALLOC_MAX_ELEM ->
 * FEI_ERR_INVALID_ARG.  Every call on a device shares that array and
 * leaves its contents behind (the call clears the counts it needs); calls
 * whose work overlaps on the GPU race on it, so order them on one stream.
 * The first call on a device with a degree array looks the array's address
 * up (cudaGetSymbolAddress) and keeps it for later calls; the kept address
 * does not survive cudaDeviceReset. */
fei_status fei_integrate_noalloc(const fei_reference_t *refs, int nrefs,
                                 const fei_batch *batch, fei_precision prec,
                                 void *A_out, void *b_out, int32_t *elem_status,
                                 fei_stream_t stream);

/* ---- Assembly into a global CSR matrix (Sec. 2) -------------------------
 * After integration, entry (r, c) of the global matrix is the sum of
 * A_e[i][j] over the elements e whose local functions i and j carry the
 * global numbers r = l2g_e[i] and c = l2g_e[j]; the global load vector
 * gathers b_e[i] at l2g_e[i].  Elements that share a global function
 * depend on each other; a colouring in which such elements never share a
 * colour removes the dependency (Sec. 2), so each colour is added by one
 * launch without atomics. */
typedef struct fei_assembly *fei_assembly_t;

/* fei_assembly_create flag: build the pattern and colouring on the host
 * only (no device memory, no CUDA call); fei_assembly_info and
 * fei_assembly_pattern work, the assemble calls refuse the handle. */
#define FEI_ASSEMBLY_HOST_ONLY 1

/* Builds, on the host, the CSR pattern, a greedy colouring of the elements
 * and the scatter map, and copies them to the current device.
 *  n_elem            number of elements (1..2^31-1).
 *  degree            HOST int32 [n_elem] degrees, or NULL: every element has
 *                    uniform_degree (1..7).
 *  l2g               HOST int64, element e's N_sh(p_e) global numbers at
 *                    the element's load-vector offset (the layout of b_out
 *                    of fei_integrate: sum of N_sh over earlier elements).
 *                    Values in 0..n_dof-1, distinct within an element.
 *  n_dof             global functions (rows), 1..2^31-1.
 *  flags             0 or FEI_ASSEMBLY_HOST_ONLY.
 * The pattern holds, in row r, the sorted global numbers of every element
 * that contains r; a row may hold at most 65535 entries.  Errors:
 * INVALID_ARG (NULL pointers, sizes, l2g out of range or repeated within an
 * element), INVALID_DEGREE, UNSUPPORTED (a row over 65535 entries), OOM,
 * CUDA.  Synchronous; the handle owns all its memory. */
fei_status fei_assembly_create(int64_t n_elem, const int32_t *degree, int32_t uniform_degree,
                               const int64_t *l2g, int64_t n_dof, int32_t flags,
                               fei_assembly_t *out);
fei_status fei_assembly_destroy(fei_assembly_t as);

/* Sizes (host pointers, any may be NULL): rows, stored entries, colours,
 * and chunks of the fused path. */
fei_status fei_assembly_info(fei_assembly_t as, int64_t *n_dof, int64_t *nnz, int32_t *n_colours,
                             int32_t *n_chunks);

/* Copies the pattern and the colouring to HOST arrays (any may be NULL):
 * row_ptr int64 [n_dof + 1], col_idx int32 [nnz], colour int32 [n_elem].
 * Synchronous. */
fei_status fei_assembly_pattern(fei_assembly_t as, int64_t *row_ptr, int32_t *col_idx, int32_t *colour);

/* values (device [nnz]) = the assembled matrix and rhs (device [n_dof]) =
 * the assembled load vector, from element matrices and vectors in the
 * layout fei_integrate writes for the batch the handle describes (A_offset
 * and b_offset of fei_plan_offsets, or the contiguous uniform layout).
 * Types follow prec: double for FEI_FP64, float otherwise.  Both outputs are
 * overwritten.  One launch per run of elements of equal (degree, colour),
 * in that order, so the sum of each entry runs in a fixed order (the same
 * as in fei_integrate_assemble).  Asynchronous on the stream. */
fei_status fei_assemble(fei_assembly_t as, fei_precision prec, const void *A, const void *b,
                        void *values, void *rhs, fei_stream_t stream);

/* Integration and assembly fused: the handle's elements, grouped by degree
 * into chunks (all elements of a degree unless their FP32 element matrices
 * pass 256 MB), are integrated chunk by chunk into a scratch buffer that
 * the library allocates on first use (kept with the handle), and each
 * chunk is assembled from there, run by (degree, colour) run, before the
 * next, so a batch never needs memory for all of its element matrices.
 * batch: as for fei_integrate, with the
 * handle's element count and degrees (a degree array if and only if the
 * handle was created with one, holding the same degrees); its A_offset and
 * b_offset are not used (no element output).  values, rhs: as for
 * fei_assemble; elem_status: as for
 * fei_integrate (device int32 [n_elem]).  Calls on one handle must not
 * overlap on the GPU (they share the scratch).  Asynchronous on the stream
 * (the first call allocates). */
fei_status fei_integrate_assemble(fei_assembly_t as, const fei_reference_t *refs, int nrefs,
                                  const fei_batch *batch, fei_precision prec, void *values,
                                  void *rhs, int32_t *elem_status, fei_stream_t stream);

/* ---- Host-memory batches --------------------------------------------
 * Integration of a batch whose inputs and outputs live in host memory.
 * The batch is cut into chunks of consecutive elements that fit one device
 * slot; each chunk is uploaded on the pipeline's upload stream, integrated
 * with fei_integrate on the caller's stream and downloaded on the
 * pipeline's download stream.  Two input and two output slots let the
 * download of one chunk overlap the integration of the next and the upload
 * of the one after.  Element matrices and vectors are those of
 * fei_integrate (same kernels, same values, bit for bit).
 *
 * fei_pipeline_create: refs / nrefs as for fei_integrate (the handles must
 * outlive the pipeline); prec as for fei_integrate; slot_bytes = the size
 * of one slot's A_e output (0: 256 MiB; 1 MiB .. 1 TiB, else
 * FEI_ERR_INVALID_ARG).  Allocates two input slots (geometry for
 * slot_bytes / 144 elements, coefficient records for slot_bytes / 112
 * records, degrees and offsets) and two output slots (A_e, b_e, status) on
 * the current device, about 7 x slot_bytes in all, and two streams.
 * Allocation failure -> FEI_ERR_OOM.  The handle belongs to the caller and
 * is used by one host thread at a time. */
typedef struct fei_pipeline *fei_pipeline_t;
fei_status fei_pipeline_create(const fei_reference_t *refs, int nrefs, fei_precision prec,
                               int64_t slot_bytes, fei_pipeline_t *out);
/* Waits for the pipeline's outstanding copies, then frees it.  NULL is a
 * no-op. */
fei_status fei_pipeline_destroy(fei_pipeline_t pipeline);
/* Slot size in bytes and the largest number of elements of one chunk. */
fei_status fei_pipeline_info(fei_pipeline_t pipeline, int64_t *slot_bytes, int64_t *max_elem);

/* batch: a fei_batch whose pointers (geom, degree, K, b, c, f) are HOST
 * pointers, with the same layouts as for fei_integrate; A_offset, b_offset
 * and q_offset must be NULL (FEI_ERR_INVALID_ARG otherwise): the outputs
 * are packed in element order, element e's A_e at the sum of N_sh^2 over
 * the elements before it (its b_e likewise, the per-point records at the
 * sum of N_q), degrees outside 1..7 taking no room -- the layout of
 * fei_plan_offsets.  A_host, b_host: host arrays of that total size (FP64
 * for FEI_FP64, FP32 otherwise); status_host: int32 [n_elem], the
 * per-element status of fei_integrate.  *n_chunks (may be NULL) receives
 * the number of chunks.  Asynchronous: the call returns once every copy
 * and launch is enqueued; the outputs are complete when the work enqueued
 * on `stream` so far has completed, and work enqueued on `stream` before
 * the call runs first.  The host arrays must stay valid until then.  Page-
 * locked host memory (cudaHostAlloc, cudaHostRegister) lets the copies
 * overlap; pageable memory works, with copies that block the calling
 * thread.  An element larger than a slot -> FEI_ERR_INVALID_ARG. */
fei_status fei_integrate_host(fei_pipeline_t pipeline, const fei_batch *batch, void *A_host,
                              void *b_host, int32_t *status_host, int64_t *n_chunks,
                              fei_stream_t stream);

/* Fault injection for tests: the time limit of the tensor-core forward's
 * pipeline waits on the current device, in nanoseconds (0 restores the
 * default, 2 s).  A block whose wait runs out raises an abort flag, marks
 * the elements of its remaining tiles FEI_ERR_TIMEOUT, lets its in-flight
 * tensor-core work and copies finish, frees its tensor memory and returns:
 * nothing traps and the context stays usable.  A tiny limit makes a launch
 * report FEI_ERR_TIMEOUT without any fault.  Synchronous. */
fei_status fei_debug_set_wait_limit(uint64_t ns);

/* Thread-local description of the last failure of the calling thread. */
const char *fei_last_error_string(void);

#ifdef __cplusplus
}
#endif

#endif /* FEI_H_ */
