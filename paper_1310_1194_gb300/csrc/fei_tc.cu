// fei_tc.cu -- the contraction on the 5th-generation tensor cores (p >= 3).
//
// The double loop over shape functions of Algorithm 1 (steps 9-13, "the
// dominant cost", Sec. 2.2) is, for every element e, the product
//     A_e = H'_e^T G,   H'_e[(q,b)][i] = sum_a Dt_q[a][b] G[q][a][i],
// over the K = 4 N_q dimension (q = point, b = value / 3 derivatives).  G is
// the same for every element of one degree (Sec. 2.2), so the batch is ONE
// GEMM: the rows (e, i) of all elements are stacked along M in tiles of
// 128 rows that run across element boundaries, N = N_sh (the shared G), and
// K = 4 N_q.  This is the GPU counterpart of the paper's vectorisation over
// the entries of A_e (Algorithm 2 "DD", four consecutive j per float4): here
// one tcgen05.mma produces a 128 x N tile.
//
// Precision (FEI_TC_F16X3).  Each operand x is split into two fp16 numbers
// hi = rn(x), lo = rn(x - hi); hi*hi + hi*lo + lo*hi is x*y to about 2^-21
// relative.  To keep fp16 in range, G is scaled by 2^tau (per degree) and
// H'_e by 2^sigma_e (per element), chosen from the bound
// max |H'| <= max_{q,b} sum_a |Dt[a][b]| max |G| (itself bounded from the
// norms of the Jacobian columns, tc_bound), so every operand value is at
// most 2^14; the accumulator holds A_e 2^(sigma_e + tau) and the epilogue
// scales back exactly.  The tensor core adds into its FP32 accumulator with truncation,
// so a long chain of MMAs drifts by about half an ulp of the accumulator per
// instruction; to keep the error independent of K, each K chunk (and N half)
// accumulates into a fresh partial buffer in tensor memory, and the epilogue
// warps add the partial into a running FP32 sum with round-to-nearest
// ("promotion") while the MMAs fill the next partial buffer.  The point
// operators are formed as in the FEI_FP32 path: element vectors, the
// vertical-node cross products and the node sums of det J in FP64; w det J
// at each point from those FP64 sums in double-FP32 arithmetic (error-free
// to about 2^-44 before its single rounding to FP32), which needs no FP64
// instruction per point (FP64 is slow per instruction on this part).
//
// Operand A in tensor memory (p <= 5).  The producers write H' hi/lo with
// tcgen05.st into tensor-memory columns and the MMAs read A from there
// (tcgen05.mma [d], [a], b-desc), so that shared memory carries only the B
// operand to the tensor core and no A tile is stored to it: at p = 4 the
// A tiles were about 40 % of the shared-memory traffic, which bound the
// kernel.  At p = 6, 7 the accumulators fill tensor memory and A stays in
// shared memory.
//
// One thread block per SM walks a contiguous range of 128-row tiles;
// nothing synchronises the whole block between tiles.  Roles (warp = 32
// threads):
//   warp 0       TMEM owner; lane 0 streams the pre-swizzled B operand (the
//                split G image) and, for p <= 4, the chunk's rows of the
//                FP32 table into shared memory with cp.async.bulk;
//   warp 1       lane 0 issues tcgen05.mma (M = 128, N = N_pad or 2 halves);
//   next warps   point operators: per tile, the elements not seen before
//                (one warp per element for its FP64 node data, its inputs
//                fetched during the previous tile; then w det J, status and
//                operand bound at every point over all these warps), their
//                scales and the row data; per K chunk, the point operators
//                of its points into a ring that runs ahead of the producers;
//   producers    per K chunk, H' for the 128 rows from the FP32 table (from
//                the stage for p <= 4, else through L2) with packed FP32
//                FMAs on pairs of consecutive points; split into hi/lo (the
//                residual by one mixed-precision FMA per value), written to
//                tensor memory (a thread per row and a few point pairs,
//                p <= 5) or in the swizzled K-major shared-memory layout (a
//                thread per point pair and a few rows, p = 6, 7); and the
//                partial load vectors;
//   last 4 warps epilogue: promotion of every partial accumulator, then
//                scaling and stores of A_e (bulk copies of staged rows for
//                a contiguous layout at p <= 4), b_e and the statuses.
// All hand-offs are mbarriers; every wait is bounded by a time limit after
// which the block raises an abort flag, marks its remaining elements with
// FEI_ERR_TIMEOUT, drains its MMAs, frees its TMEM and exits.
#include <cuda_fp16.h>
#include <math.h>
#include <string.h>

#include "fei_geom.cuh"
#include "fei_internal.cuh"

namespace fei {

// The operands of one split kind (0: fp16 hi/lo of G 2^tau, 1: TF32 hi/lo
// of G), chunked by that kind's points per chunk.
struct TcOperands {
  // B image [NCHUNK][2 (hi, lo)][NPAD][ROWB bytes], each [NPAD][ROWB] block
  // in the ROWB-byte swizzled K-major layout
  unsigned char *img;
  // the FP32 table by chunk and point pair: [NCHUNK][2][PP][GST] float4,
  // half h of pair (q, q+1) and shape i = (G_2h(q), G_2h(q+1), G_2h+1(q),
  // G_2h+1(q+1)), G_b = phi, dphi/dxi1, dphi/dxi2, dphi/dzeta; zero past
  // N_q and N_sh (GST >= N_sh is the row stride)
  float *gp;
  int nchunk;
};
struct TcImage {
  TcOperands k[2];
  int npad, rowb, tau;
  // adjoint A operand (p = 3..5): G 2^tau by rows (q, b), K = j, split into
  // fp16 hi/lo, [M tile][K chunk][hi, lo][128 rows][64 bytes] swizzled
  unsigned char *aimg;
  // the FP32 table for the adjoint epilogue: [N_q][N_pad] float4 (G of the
  // four components a at (q, i)), zero for i >= N_sh
  float4 *gq4p;
};

namespace {

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s per wait
// The limit of the pipeline waits (mbar_wait), per device: kWaitLimitNs,
// or what fei_debug_set_wait_limit set for fault-injection tests.  The
// drain of in-flight MMAs before an aborted block frees its tensor memory
// always uses kWaitLimitNs.
__device__ uint64_t g_wait_limit_ns = kWaitLimitNs;

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
// try_wait that lets the thread sleep until the phase completes or about
// 0.5 ms pass (the hardware wakes it when the phase completes, so a waiting
// warp neither spins nor misses the completion)
__device__ __forceinline__ bool mbar_try_wait_sleep(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity), "r"(500000u)
      : "memory");
  return ok != 0;
}
// Bounded wait: false (and the abort flag raised) after g_wait_limit_ns, or
// as soon as another role raised the flag (checked between sleeps).
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, volatile int *abort_flag) {
  if (mbar_try_wait(a, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    if (mbar_try_wait_sleep(a, parity)) return true;
    if (*abort_flag) return false;
    if (global_ns() - t0 > g_wait_limit_ns) {
      *abort_flag = 1;
      return false;
    }
  }
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// 8-byte asynchronous copy global -> shared (cp.async, both 8-byte aligned);
// complete for this thread after cp_async_wait_all
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// shared -> global bulk copy (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_s2g(void *dst, uint32_t src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// wait until the bulk copies of this thread have read their source
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// wait until the bulk copies of this thread have completed
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// MMAs and commits are executed by the whole warp and issued by one
// elected lane (elect.sync elects the lowest active lane, the same lane each
// time, so that its commits track all of these MMAs).  A warp-uniform MMA
// loop lets the compiler keep the operands in uniform registers; a loop in
// lane 0 alone moved them from per-thread registers at every MMA and, next
// to warps busy with FP32 work, issued one MMA per 3-10 tensor-pipe times.
// KD = 0: kind::f16 (fp16 A and B), KD = 1: kind::tf32.  A and B from
// shared memory by descriptor.
template <int KD>
__device__ __forceinline__ void tc_mma_ss_w(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (KD == 0)
    asm volatile(
        "{\n .reg .pred p, e;\n setp.ne.b32 p, %4, 0;\n elect.sync _|e, 0xffffffff;\n"
        " @e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p, e;\n setp.ne.b32 p, %4, 0;\n elect.sync _|e, 0xffffffff;\n"
        " @e tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void tc_commit_w(uint32_t mbar) {
  asm volatile(
      "{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n"
      " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n" ::"r"(mbar)
      : "memory");
}
// x rounded to TF32 (10 fraction bits, nearest, ties away), as FP32 bits
__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
// A from tensor memory (a = TMEM address of the 128-row A slice: lane =
// row; two consecutive fp16 K values, or one TF32 value, per 32-bit column),
// B from shared memory by descriptor.
template <int KD>
__device__ __forceinline__ void tc_mma_ts_w(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (KD == 0)
    asm volatile(
        "{\n .reg .pred p, e;\n setp.ne.b32 p, %4, 0;\n elect.sync _|e, 0xffffffff;\n"
        " @e tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
        "r"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p, e;\n setp.ne.b32 p, %4, 0;\n elect.sync _|e, 0xffffffff;\n"
        " @e tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
        "r"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
// 16 bytes to shared memory at a shared-window address
__device__ __forceinline__ void st_shared_v4(uint32_t addr, const uint32_t *v) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3])
               : "memory");
}
// 32 lanes x 8 columns of 32-bit values from registers (thread t = lane t)
__device__ __forceinline__ void tmem_st8u(uint32_t taddr, const uint32_t *v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr), "r"(v[0]),
               "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
               : "memory");
}
__device__ __forceinline__ void named_bar(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
// 32 lanes x 16 columns of 32-bit values; thread t owns its lane's columns.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float *v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
      "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
      "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// Issue-only variants (no wait): the caller waits once for a batch.
__device__ __forceinline__ void tmem_ld16_nw(uint32_t taddr, uint32_t *r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

__device__ __forceinline__ float exp2i(int k) {  // exact 2^k for |k| < 126
  return __int_as_float((127 + k) << 23);
}

// ---------------------------------------------------------------------------
// Configuration
// ---------------------------------------------------------------------------
// ROWB = bytes of one swizzled operand row = K values per chunk * 2 (fp16):
// 128 (128-byte swizzle, 16 points per chunk) or 64 (64-byte swizzle,
// 8 points per chunk, used for p = 7 to leave room for three stages).
// V selects a variant of the warp roles (the autotuner of a plan times
// them): 0 = 8 producer warps, 1 = 16 producer warps with half the points
// each (more warps in flight, fewer registers per thread).
template <int P, int V = 0, int KD = 0>
struct TcCfg {
  static constexpr int NSH = nsh_of(P), NQ = nq_of(P), NZ = P + 1, NT = (P + 1) * (P + 1);
  static constexpr int NPAD = P == 6 ? 224 : (NSH + 15) / 16 * 16;
  static constexpr int NHALF = P >= 6 ? 2 : 1;
  static constexpr int NMMA = NPAD / NHALF;  // N of one MMA = one partial buffer
  static constexpr int ROWB = P == 7 ? 64 : 128;
  // KD = 0: split fp16 operands (2 bytes, K = 16 per MMA); KD = 1: split
  // TF32 operands (4 bytes, K = 8 per MMA)
  static constexpr int EB = KD ? 4 : 2;
  static constexpr int KMMA = KD ? 8 : 16;
  static constexpr int KCH = ROWB / EB;       // K values per chunk
  static constexpr int PPC = KCH / 4;         // points per chunk
  static constexpr int KSL = KCH / KMMA;      // MMA K slices per chunk
  static constexpr int NCHUNK = (NQ + PPC - 1) / PPC;
  // chunks per promotion unit: a partial accumulator collects 4 K slices
  // (12 MMAs) before the epilogue adds it into the running sum
  static constexpr int UC = KSL == 2 ? 2 : 1;
  // partial accumulators the MMAs fill in turn while the epilogue promotes
  // the previous ones: three where tensor memory leaves room (p <= 4), so
  // that the MMAs do not wait for the promotion of the one before
  static constexpr int NPART = (P <= 4) ? 3 : 2;
  // running sum: columns [0, RT) in TMEM after the partial buffers, the
  // rest (RREG columns) in registers of the epilogue threads
  static constexpr int RT = (512 - NPART * NMMA) < NPAD ? (512 - NPART * NMMA) : NPAD;
  static constexpr int RREG = NPAD - RT;
  // TS: the A operand (H' split into hi/lo) lives in tensor memory, written
  // by the producers with tcgen05.st and read by the MMA from there, so the
  // MMA reads only B from shared memory and the producers store nothing to
  // it (p <= 5, where the accumulators leave room).  Per stage KCH columns:
  // KCH/2 of hi (two fp16 per column) then KCH/2 of lo, from column ABASE.
  static constexpr bool TS = P <= 5;
  static constexpr int ACC_COLS = NPART * NMMA + RT;
  static constexpr int RSUM = NPART * NMMA;  // first column of the running sum
  static constexpr int ABASE = TS ? (ACC_COLS + 31) / 32 * 32 : 0;
  static constexpr int ACOLS = KCH * EB / 2;  // hi then lo, 32-bit columns
  static constexpr int AHALF = ACOLS / 2;
  static constexpr int VPC = 4 / EB;  // operand values per 32-bit column
  static constexpr int TMEM_COLS = TS ? 512 : (3 * NPAD <= 256 ? 256 : 512);
  static constexpr int EMAX = (128 + NSH - 1) / NSH + 1;  // elements a tile can touch
  static constexpr int NSLOT = EMAX + 1;  // element slots: a tile's elements plus the one it shares
  static constexpr int NDW = P == 7 ? 2 : P == 6 || P == 5 ? 4 : V == 1 ? 6 : 8;  // point-operator warps
  static constexpr int NPW = V == 1 ? 16 : 8;  // producer warps
  static constexpr int NEW = 4;  // epilogue warps
  static constexpr int W_DW = 2, W_PW = W_DW + NDW, W_EW = W_PW + NPW;
  static constexpr int NTHREADS = (2 + NDW + NPW + NEW) * 32;
  // GS: the chunk's rows of the FP32 table (PPC points x GST x 16 bytes)
  // travel with the B operand into the stage (copy engine), so the
  // producers read them from shared memory instead of L2 (p <= 4, where
  // they fit beside two stages)
  static constexpr bool GS = P <= 4;
  // producer layout, PP = pairs of consecutive points per chunk (a pair is
  // one 16-byte chunk of an operand row).  With the table chunk in shared
  // memory (GS): lane = pp + PP rg, a warp covers RW consecutive rows in RG
  // row groups.  Otherwise a warp works on one pair (WPP warps per pair) for
  // RWP consecutive rows, lanes over consecutive rows, so that the table
  // reads from L2 are contiguous.  RPT = rows per thread.
  static constexpr int PP = PPC / 2, RG = 32 / PP, RW = 128 / NPW;
  static constexpr int WPP = NPW / PP, RWP = 128 / WPP;
  static constexpr int RPT = GS ? RW / RG : RWP / 32;
  // row stride of the paired table: odd with GS, so that the 8 pairs of a
  // row group fall into different 16-byte bank groups of shared memory
  static constexpr int GST = GS ? (NSH | 1) : NSH;
  // chunks of point operators ahead, and per round (one wait and one pass
  // of the point-operator warps for several chunks): at p = 4 a whole tile
  // (8 chunks) per round on a 16-chunk ring, 4.3 % faster than rounds of 4
  static constexpr int DRING = P == 4 ? 16 : 8;
  static constexpr int DB = P == 4 ? 8 : 4;
  static constexpr int A_BYTES = 128 * ROWB;
  static constexpr int B_BYTES = NPAD * ROWB;
  static constexpr int G_BYTES = GS ? PPC * GST * 16 : 0;
  static constexpr int G_AREA = (G_BYTES + 1023) / 1024 * 1024;
  static constexpr bool BS = P <= 4;  // bulk stores of staged rows (shared-memory budget)
  static constexpr int STAGE_BYTES = (TS ? 0 : 2 * A_BYTES) + 2 * B_BYTES + G_AREA;
  static constexpr int STAGES = P == 7 ? 3 : (TS && ABASE + 3 * ACOLS <= 512 ? 3 : 2);
  // TS producer layout: PQ warps per TMEM lane quarter, each thread one row
  // (its lane) and PPW consecutive point pairs of the chunk
  static constexpr int PQ = NPW / 4, PPW = PP / PQ;
  // load-vector partials per row (one per producer thread that covers it)
  static constexpr int BSN = TS ? PQ : PP;
  static constexpr int DYN_SMEM = STAGES * STAGE_BYTES + 1024;
  static_assert(NMMA % 16 == 0 && NMMA <= 256, "MMA N");
  static_assert(RT % 16 == 0 && RREG % 16 == 0 && RT >= 0, "running-sum split");
  static_assert(NPART * NMMA + RT <= TMEM_COLS, "tensor memory");
  static_assert(!TS || (ABASE + STAGES * ACOLS <= TMEM_COLS && PP % PQ == 0 && (PPW * 4) % 8 == 0 &&
                        STAGE_BYTES % 1024 == 0),
                "tensor-memory A operand");
  static_assert(PPC % 2 == 0 && (GS ? 32 % PP == 0 && RW % RG == 0 : NPW % PP == 0 && RWP % 32 == 0) && RPT >= 1,
                "producer layout");
  static_assert(STAGES > UC, "a promotion unit must leave a stage for the producers");
  static_assert(BSN <= PP, "load-vector partials");
  static_assert(DRING >= 2 * DB, "the operator ring holds two rounds");
  static_assert(NEW == 4, "four consecutive epilogue warps cover the four TMEM lane quarters");
};

template <int P>
struct TcElem {
  using C = TcCfg<P>;
  float evf[21];          // element vectors A1, B1, A2, B2, C, D1, D2, rounded once to FP32
  alignas(16) float cf[16];  // the per-element coefficients rounded once to FP32 (14 used)
  float cn[3];            // their norms in the scale bound: sqrt(||K||_1 ||K||_inf), |b|, |c|
  float2 zabg[C::NZ][3];  // w_z (n3.C, n3.D1, n3.D2) per vertical node: FP64 as FP32 hi + lo
  float zc1f[C::NZ][3], zc2f[C::NZ][3], zn3f[C::NZ][3];
  float tc3f[C::NT][3];
  float zn[C::NZ][3];  // |c1|, |c2|, |c1 x c2| per vertical node (FP32)
  float tn[C::NT];     // |c3| per triangle node
  int64_t e, aoff, boff, qoff;
  int status;
  int mbits;   // float bits of max_{q,b} sum_a |Dt[a][b]|
  float up;    // 2^sigma (applied to Dt before H')
  float down;  // 2^-(sigma + tau)
};

// Per-tile row data handed from the point-operator warps to the producers
// (load vector, statuses) and to the epilogue (stores of A_e).
struct TcMeta {
  int64_t row_off[128];   // start of the row in A_out (minus its first column), -1 past the end
  int16_t row_lo[128];    // first column stored (the row index in the upper layout, else 0)
  int64_t row_boff[128];  // position of the row in b_out
  int32_t row_eid[128];   // element id of the row's element at its first row, else -1
  float row_down[128];    // exact scale back of the row's element
  int row_status[128];    // status of the row's element (nonzero: write zeros)
};

template <int P, int V, int KD>
struct TcAux {
  using C = TcCfg<P, V, KD>;
  uint64_t full[C::STAGES];   // producers wrote A of the stage
  uint64_t bfull[C::STAGES];  // B of the stage landed
  uint64_t empty[C::STAGES];  // MMAs of the stage completed
  // GS: the table rows of a stage have their own hand-off, released by the
  // producers once they have read them, so that the next chunk's rows are
  // copied while the MMAs of this one still run.  gfull also takes the
  // commit of the MMAs of the chunk S before (the A columns free), so the
  // producers wait on one barrier for both; the copy warp stands in for
  // that commit at the first use of a stage.
  uint64_t gfull[C::STAGES];   // table rows of the stage landed, A columns free
  uint64_t gempty[C::STAGES];  // producers done with the table rows
  uint64_t dfull[C::DRING];   // point operators of a chunk ready
  uint64_t dempty[C::DRING];  // producers done with them
  uint64_t part_full[3];      // partial accumulator ready for promotion
  uint64_t promo_done[3];     // partial accumulator promoted (free again)
  uint64_t meta_full[2];
  uint64_t meta_empty[2];
  uint64_t bsum_full[2];      // producers' load-vector partials of a tile
  uint64_t drain;
  uint32_t tmem_base;
  int abort_flag;
  int dsnap;
  TcElem<P> el[C::NSLOT];    // element k lives in slot k % NSLOT
  float sp[C::NSLOT][C::NQ];  // w det J per point (FP32, from FP64)
  float2 ttab[C::NT][3];     // (w_t, w_t xi1, w_t xi2) per triangle node: FP64 as FP32 hi + lo
  float ttabf[C::NT][3];     // (w_t, xi1, xi2) in FP32
  float ztabf[C::NZ][2];     // (zeta, w_z) in FP32
  float2 ztab2[C::NZ][2];    // (zeta, w_z) as FP32 hi + lo
  // inputs of the next tile's first new element of each point-operator warp
  // (copied with cp.async while the current tile is processed)
  double pf_buf[C::NDW][32];
  // point operators of a chunk, [tile-relative element][k'][point pair]:
  // float4 k' of pair (q, q+1) is (c_2k'(q), c_2k'(q+1), c_2k'+1(q),
  // c_2k'+1(q+1)) for the 14 values c_0..c_13 of a point (Dt by rows, then
  // w det J f), i.e. the pairs the producers feed to packed FP32 FMAs;
  // consecutive pairs are consecutive 16-byte words (broadcast loads); one
  // word of padding per element, so that a warp whose rows span two
  // elements reads their words from different banks
  float4 Dc[C::DRING][C::EMAX][7 * C::PP + 1];
  TcMeta meta[2];
  float bsum[2][C::PP][128];
  alignas(16) float stg[C::NEW][32][17];  // epilogue transpose staging
  // BS: for a contiguous output layout (p <= 4), each epilogue warp stages
  // 16 of its rows of A_e here and stores them with one bulk copy
  alignas(16) float rows16[C::BS ? C::NEW : 1][C::BS ? 16 * C::NSH : 4];
};

// Per-point coefficient record r (K 9, b 3, c, f) rounded to FP32; returns
// whether all 14 values are finite (tested on the FP64 bits).
__device__ __forceinline__ bool load_coef_tc(const FwdArgs &a, int64_t r, float *cf, bool *sym = nullptr) {
  double cd[14];
#pragma unroll
  for (int k = 0; k < 9; ++k) cd[k] = a.K[9 * r + k];
#pragma unroll
  for (int k = 0; k < 3; ++k) cd[9 + k] = a.b[3 * r + k];
  cd[12] = a.c[r];
  cd[13] = a.f[r];
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 14; ++k) {
    ok &= finite64(cd[k]);
    cf[k] = (float)cd[k];
  }
  if (sym) *sym = coef_symmetric(cd, cd + 9);
  return ok;
}

// FP32 point operator of element slot E at point q from the node tables;
// sf = w det J (formed in FP64, rounded once); cf = coefficients in FP32.
template <int P, class AX>
__device__ __forceinline__ void tc_point(const TcElem<P> &E, const AX &ax, const float *cf, int q, float sf,
                                         float *D) {
  using C = TcCfg<P>;
  const int iz = q / C::NT, t = q - iz * C::NT;
  float a0[3], a1[3];
  cross3(E.zc2f[iz], E.tc3f[t], a0);
  cross3(E.tc3f[t], E.zc1f[iz], a1);
  const float wf = ax.ztabf[iz][1] * ax.ttabf[t][0];
  dt_from_adj<float>(a0, a1, E.zn3f[iz], wf, sf, wf * wf / sf, cf, cf + 9, cf[12], cf[13], D);
}
__device__ __forceinline__ float norm3f(const float *v) { return sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]); }
// Upper bound of max_b sum_a |Dt[a][b]| at one point, from norms only:
// |adj_0| <= |c2||c3|, |adj_1| <= |c3||c1|, |adj_2| = |c1 x c2|, so
//   sum_a |Dt[a][0]| = s |c|,
//   sum_a |Dt[a][m]| <= w |adj_m| |b| + (w / det J) |adj_m| ||K||_2 sum_l |adj_l|,
// with w / det J = w^2 / s and ||K||_2 <= sqrt(||K||_1 ||K||_inf).  It sets
// the element's power-of-two operand scale, which only has to keep the fp16
// operands in range; an over-estimate costs at most a few bits of headroom.
template <int P, class AX>
__device__ __forceinline__ float tc_bound(const TcElem<P> &E, const AX &ax, const float *cn, int iz, int t,
                                          float sf) {
  const float w = ax.ztabf[iz][1] * ax.ttabf[t][0];
  const float n3 = E.tn[t];
  const float a0 = E.zn[iz][1] * n3, a1 = n3 * E.zn[iz][0], a2 = E.zn[iz][2];
  const float amax = fmaxf(fmaxf(a0, a1), a2), asum = a0 + a1 + a2;
  // cn: the coefficient norms (coef_norms).  w / sf only sets a power-of-two scale with two bits of headroom in fp16
  // range, so the fast division (error of a few ulp) is enough
  return fmaxf(sf * cn[2], w * amax * (cn[1] + __fdividef(w, sf) * cn[0] * asum));
}
// The coefficient norms of the bound: sqrt(||K||_1 ||K||_inf) >= ||K||_2,
// |b| and |c|, from the 14 FP32 coefficient values.
__device__ __forceinline__ void coef_norms(const float *cf, float *cn) {
  float r1 = 0.f, ri = 0.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    r1 = fmaxf(r1, fabsf(cf[k]) + fabsf(cf[3 + k]) + fabsf(cf[6 + k]));
    ri = fmaxf(ri, fabsf(cf[3 * k]) + fabsf(cf[3 * k + 1]) + fabsf(cf[3 * k + 2]));
  }
  cn[0] = sqrtf(r1 * ri);
  cn[1] = norm3f(cf + 9);
  cn[2] = fabsf(cf[12]);
}
// Shared-memory matrix descriptor of a K-major operand with ROWB-byte rows
// in the ROWB-byte swizzle layout; 8-row groups 8 * ROWB bytes apart.
template <int ROWB>
__device__ __forceinline__ uint64_t sw_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);    // start address
  d |= (uint64_t)1 << 16;                      // leading byte offset (unused)
  d |= (uint64_t)((8 * ROWB) >> 4) << 32;      // stride byte offset
  d |= (uint64_t)1 << 46;                      // descriptor version
  d |= (uint64_t)(ROWB == 128 ? 2 : 4) << 61;  // 128- or 64-byte swizzle
  return d;
}
// Byte offset of 16-byte chunk c of row r in a swizzled operand tile whose
// base is 1024-byte aligned: the chunk index is XORed with address bits
// [9:7] (128-byte rows) or [8:7] (64-byte rows).
template <int ROWB>
__host__ __device__ __forceinline__ uint32_t sw_off(int r, int c) {
  const int x = ROWB == 128 ? (r & 7) : ((r >> 1) & 3);
  return (uint32_t)(r * ROWB + ((c ^ x) << 4));
}
// x - hi for the two values of a split: hi holds rn_f16(x0) (low half) and
// rn_f16(x1) (high half).  One mixed-precision FMA per value, hi * (-1) + x
// with the fp16 operand widened exactly; the difference is exact in FP32
// (hi is x rounded to 11 significant bits).
__device__ __forceinline__ float2 split_residual(__half2 hi, float x0, float x1) {
  uint32_t h;
  memcpy(&h, &hi, 4);
  float r0, r1;
  asm("{\n .reg .f16 a, b, m;\n mov.b32 {a, b}, %2;\n mov.b16 m, 0xBC00;\n"
      " fma.rn.f32.f16 %0, a, m, %3;\n fma.rn.f32.f16 %1, b, m, %4;\n}"
      : "=f"(r0), "=f"(r1)
      : "r"(h), "f"(x0), "f"(x1));
  return make_float2(r0, r1);
}
// Instruction descriptor: FP32 D; A and B K-major, both fp16 (kind::f16,
// type code 0) or both TF32 (kind::tf32, type code 2); N and M.
__host__ __device__ constexpr uint32_t idesc_mma(int M, int N, int KD) {
  return (1u << 4) | ((KD ? 2u : 0u) << 7) | ((KD ? 2u : 0u) << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

template <int P, int V, int KD>
__global__ void __launch_bounds__(TcCfg<P, V, KD>::NTHREADS, 1)
    tc_forward_kernel(FwdArgs a, const unsigned char *img, const float4 *gp, int tau) {
  using C = TcCfg<P, V, KD>;
  constexpr int NSH = C::NSH, NQ = C::NQ, NT = C::NT, NZ = C::NZ, S = C::STAGES, NCH = C::NCHUNK;
  constexpr int NP = C::NPW * 32, ND = C::NDW * 32, PPC = C::PPC, ROWB = C::ROWB, DR = C::DRING;
  extern __shared__ __align__(1024) unsigned char dsm_raw[];
  __shared__ TcAux<P, V, KD> ax;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t dbase = (smem_u32(dsm_raw) + 1023u) & ~1023u;
  auto stageA = [&](int s, int piece) { return dbase + s * C::STAGE_BYTES + piece * C::A_BYTES; };
  constexpr int AST = C::TS ? 0 : 2 * C::A_BYTES;  // A tiles of a stage in shared memory (SS only)
  auto stageB = [&](int s) { return dbase + s * C::STAGE_BYTES + AST; };
  auto stageG = [&](int s) { return dbase + s * C::STAGE_BYTES + AST + 2 * C::B_BYTES; };
  volatile int *abort_flag = &ax.abort_flag;

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&ax.full[s]), C::NPW);
      mbar_init(smem_u32(&ax.bfull[s]), 1);
      mbar_init(smem_u32(&ax.empty[s]), 1);
      mbar_init(smem_u32(&ax.gfull[s]), 2);
      mbar_init(smem_u32(&ax.gempty[s]), C::NPW);
    }
    for (int k = 0; k < DR; ++k) {
      mbar_init(smem_u32(&ax.dfull[k]), 1);
      mbar_init(smem_u32(&ax.dempty[k]), C::NPW);
    }
    for (int k = 0; k < C::NPART; ++k) {
      mbar_init(smem_u32(&ax.part_full[k]), 1);
      mbar_init(smem_u32(&ax.promo_done[k]), C::NEW);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(smem_u32(&ax.meta_full[k]), 1);
      mbar_init(smem_u32(&ax.meta_empty[k]), C::NEW);
      mbar_init(smem_u32(&ax.bsum_full[k]), C::NPW);
    }
    mbar_init(smem_u32(&ax.drain), 1);
    ax.abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ax.tmem_base)),
                 "r"(C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // quadrature node tables of this degree, once per block
  for (int t = tid; t < NT; t += blockDim.x) {
    const double x1 = a.tnode[4 * t], x2 = a.tnode[4 * t + 1], wt = a.tnode[4 * t + 2];
    ax.ttab[t][0] = split_f64(wt);
    ax.ttab[t][1] = split_f64(wt * x1);
    ax.ttab[t][2] = split_f64(wt * x2);
    ax.ttabf[t][0] = (float)wt;
    ax.ttabf[t][1] = (float)x1;
    ax.ttabf[t][2] = (float)x2;
  }
  for (int z = tid; z < NZ; z += blockDim.x) {
    ax.ztabf[z][0] = (float)a.znode[2 * z];
    ax.ztabf[z][1] = (float)a.znode[2 * z + 1];
    ax.ztab2[z][0] = split_f64(a.znode[2 * z]);
    ax.ztab2[z][1] = split_f64(a.znode[2 * z + 1]);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ax.tmem_base;

  const int64_t items = a.count ? (int64_t)(*a.count) : a.n_work;
  const int64_t rows_total = items * NSH;
  const int64_t tiles = (rows_total + 127) / 128;
  // this block's tiles: a contiguous range (consecutive tiles share elements)
  const int64_t t_per = tiles / gridDim.x, t_extra = tiles % gridDim.x;
  const int64_t t_begin = blockIdx.x * t_per + (blockIdx.x < t_extra ? blockIdx.x : t_extra);
  const int64_t t_end = t_begin + t_per + (blockIdx.x < t_extra ? 1 : 0);

  if (warp >= C::W_DW && warp < C::W_PW) {
    // ======================================================== point operators
    // Per tile: set up the elements not seen before (geometry, FP64 node
    // columns, w det J at every point, the scale), then the row data; per
    // chunk: the point operators of its points (pre-scaled by 2^sigma) into
    // a ring that runs ahead of the producers.  A block walks consecutive
    // tiles, so an element split between two tiles is set up once.
    const int td = tid - C::W_DW * 32;  // 0 .. ND-1
    int it = 0;
    int64_t kdone = -1;  // elements 0 .. kdone of this block are set up
    // the inputs of the element this warp sets up first in the next tile,
    // loaded while the current tile's point operators are formed (lanes
    // 0-17 a vertex coordinate, 18-31 a per-element coefficient)
    int64_t pf_k = -1;
    double *const pf_slot = &ax.pf_buf[warp - C::W_DW][lane];
    // this lane's input of work item k (null: none)
    auto input_ptr = [&](int64_t k) -> const double * {
      const int64_t e = a.list ? (int64_t)a.list[k] : k;
      if (lane < 18) return a.geom + 18 * e + lane;
      if (a.coef_mode != FEI_COEF_PER_ELEMENT) return nullptr;
      const int j = lane - 18;
      return j < 9 ? a.K + 9 * e + j : j < 12 ? a.b + 3 * e + (j - 9) : j == 12 ? a.c + e : a.f + e;
    };
    auto fetch_input = [&](int64_t k) {
      const double *src = input_ptr(k);
      return src ? *src : 0.0;
    };
    for (int64_t tile = t_begin; tile < t_end; ++tile, ++it) {
      // the point-operator warps leave together (they share named barriers)
      if (td == 0) ax.dsnap = *abort_flag;
      named_bar(2, ND);
      if (ax.dsnap) break;
      const int64_t r0 = tile * 128;
      const int64_t k0 = r0 / NSH;
      int64_t k1 = (r0 + 127) / NSH;
      if (k1 > items - 1) k1 = items - 1;
      const int nel = (int)(k1 - k0 + 1);
      const int64_t kn0 = kdone + 1 > k0 ? kdone + 1 : k0;  // first new element
      const int nnew = (int)(k1 - kn0 + 1);
      kdone = k1;
      auto slot_of = [&](int64_t k) { return (int)(k % C::NSLOT); };
      // Set-up of the new elements, one warp per element with lanes in
      // parallel and only warp-level synchronisation between its steps, so
      // that the elements of a tile are set up at the same time and no step
      // waits for the whole group (FP64 is slow per instruction on this
      // part, and a step of a few FP64 operations per element is mostly
      // latency).
      for (int i = warp - C::W_DW; i < nnew; i += C::NDW) {
        const int sl = slot_of(kn0 + i);
        TcElem<P> &E = ax.el[sl];
        const int64_t e = a.list ? (int64_t)a.list[kn0 + i] : kn0 + i;
        // geometry (lanes 0-17) and per-element coefficients (lanes 18-31),
        // prefetched during the previous tile when this warp knew the element
        double x;
        if (pf_k == kn0 + i) {
          cp_async_wait_all();
          x = *pf_slot;
        } else {
          x = fetch_input(kn0 + i);
        }
        const bool ok = __all_sync(0xffffffffu, finite64(x));
        // upper layout: a symmetric K (K01 = K10, K02 = K20, K12 = K21: lanes
        // 19/21, 20/24, 23/25) and b = 0 (lanes 27-29) in the element's record
        // (compared on the bits, +0 and -0 equal)
        bool sym = true;
        if (a.upper && a.coef_mode == FEI_COEF_PER_ELEMENT) {
          const int c = lane - 18;
          const int partner = c == 1 ? 21 : c == 3 ? 19 : c == 2 ? 24 : c == 6 ? 20 : c == 5 ? 25 : c == 7 ? 23 : lane;
          const unsigned long long xb = (unsigned long long)__double_as_longlong(x);
          const unsigned long long pb = __shfl_sync(0xffffffffu, xb, partner);
          sym = __all_sync(0xffffffffu, (c >= 9 && c <= 11) ? (xb << 1) == 0ull : (xb == pb || ((xb | pb) << 1) == 0ull));
        }
        if (lane >= 18 && a.coef_mode == FEI_COEF_PER_ELEMENT) E.cf[lane - 18] = f64_to_f32_bits(x);
        if (lane == 0) {
          E.e = e;
          E.aoff = out_a(a, kn0 + i, e, NSH);
          E.boff = out_b(a, kn0 + i, e, NSH);
          E.qoff = a.q_off ? a.q_off[e] : e * (int64_t)NQ;
          E.status = ok ? (sym ? 0 : FEI_ERR_INVALID_ARG) : FEI_ERR_NONFINITE;
          E.mbits = 0;
        }
        // Element vectors A1, B1, A2, B2, C, D1, D2: lane j < 21 forms
        // component k = j % 3 of vector j / 3 as (X_a - X_b) +- (X_c - X_d)
        // over vertices a, b, c, d, halved, from the lanes holding them.
        // Vertical nodes (lanes 3 iz + k): c1, c2, n3 = c1 x c2 and w_z (n3.C,
        // n3.D1, n3.D2), from which w det J = w_t (..) follows at every point.
        // The vertex differences in FP64 (two independent subtractions, exact
        // to 2^-53 of the difference however far the element is from the
        // origin), split from their bit fields into FP32 pairs; the rest in
        // double-FP32 arithmetic (two-sum and FMA products, about 2^-46
        // relative): a dependent FP64 instruction takes hundreds of cycles on
        // this part, an FP32 one a few.  Differences outside 2^-60 <= |d| <
        // 2^60 (other than 0) take the same steps in FP64.  (The differences
        // by 64-bit integer arithmetic on the bit fields took longer than the
        // one FP64 latency.)
        const int v = lane < 21 ? lane / 3 : 0, kv = lane < 21 ? lane % 3 : 0;
        // vertices (a, b, c, d) of vector v, 3 bits each, 12 bits per
        // vector, in an immediate (a table in memory would be a local load)
        //   A1 (1,0,4,3)  B1 (4,3,1,0)  A2 (2,0,5,3)  B2 (5,3,2,0)
        //   C  (3,0,0,0)  D1 (4,1,3,0)  D2 (5,2,3,0)
        constexpr unsigned long long kTab =
            (0x223ull << 0) | (0x8C8ull << 12) | (0x42Bull << 24) | (0xAD0ull << 36) | (0x600ull << 48);
        constexpr unsigned long long kTab2 = (0x858ull << 0) | (0xA98ull << 12);  // D1, D2
        constexpr unsigned kNeg = 0x6Au;  // B1, B2, D1, D2 subtract
        const unsigned tv = (unsigned)((v < 5 ? kTab >> (12 * v) : kTab2 >> (12 * (v - 5))) & 0xFFFu);
        const int la = 3 * ((tv >> 9) & 7u) + kv, lb = 3 * ((tv >> 6) & 7u) + kv;
        const int lc = 3 * ((tv >> 3) & 7u) + kv, ld = 3 * (tv & 7u) + kv;
        const bool subtract = (kNeg >> v) & 1u;
        const bool act = lane < 3 * NZ;
        const int iz = act ? lane / 3 : 0, k = act ? lane % 3 : 0;
        const int g0 = lane - k, l1 = g0 + (k + 1) % 3, l2 = g0 + (k + 2) % 3;
        const double xa = __shfl_sync(0xffffffffu, x, la), xb = __shfl_sync(0xffffffffu, x, lb);
        const double xc = __shfl_sync(0xffffffffu, x, lc), xd = __shfl_sync(0xffffffffu, x, ld);
        const double t1 = xa - xb, t2 = xc - xd;
        bool r1 = true, r2 = true;
        const float2 t1s = split_f64_bits(t1, &r1), t2s = split_f64_bits(t2, &r2);
        float evf;  // the element vector value of this lane in FP32
        if (__all_sync(0xffffffffu, lane >= 21 || (r1 && r2))) {
          auto shfl2 = [](float2 q, int src) {
            return make_float2(__shfl_sync(0xffffffffu, q.x, src), __shfl_sync(0xffffffffu, q.y, src));
          };
          float2 ev = norm_ff(add_ff(t1s, subtract ? neg_ff(t2s) : t2s));
          ev = make_float2(0.5f * ev.x, 0.5f * ev.y);
          evf = ev.x;
          const float2 z2 = ax.ztab2[iz][0], wz2 = ax.ztab2[iz][1];
          const float2 c1 = norm_ff(add_ff(shfl2(ev, k), mul_ff(z2, shfl2(ev, 3 + k))));
          const float2 c2 = norm_ff(add_ff(shfl2(ev, 6 + k), mul_ff(z2, shfl2(ev, 9 + k))));
          const float2 c1a = shfl2(c1, l1), c1b = shfl2(c1, l2), c2a = shfl2(c2, l1), c2b = shfl2(c2, l2);
          const float2 n3 = norm_ff(add_ff(mul_ff(c1a, c2b), neg_ff(mul_ff(c1b, c2a))));  // (c1 x c2)_k
          float2 ab = mul_ff(n3, shfl2(ev, 12 + k));
          float2 bb = mul_ff(n3, shfl2(ev, 15 + k));
          float2 gb = mul_ff(n3, shfl2(ev, 18 + k));
          ab = norm_ff(add_ff(ab, add_ff(shfl2(ab, l1), shfl2(ab, l2))));
          bb = norm_ff(add_ff(bb, add_ff(shfl2(bb, l1), shfl2(bb, l2))));
          gb = norm_ff(add_ff(gb, add_ff(shfl2(gb, l1), shfl2(gb, l2))));
          // lane k of the node stores value k
          if (act) E.zabg[iz][k] = norm_ff(mul_ff(wz2, k == 0 ? ab : k == 1 ? bb : gb));
        } else {
          const double ev = 0.5 * (subtract ? t1 - t2 : t1 + t2);
          evf = (float)ev;
          const double z = a.znode[2 * iz], wz = a.znode[2 * iz + 1];
          const double c1 = fma(z, __shfl_sync(0xffffffffu, ev, 3 + k), __shfl_sync(0xffffffffu, ev, k));
          const double c2 = fma(z, __shfl_sync(0xffffffffu, ev, 9 + k), __shfl_sync(0xffffffffu, ev, 6 + k));
          const double c1a = __shfl_sync(0xffffffffu, c1, l1), c1b = __shfl_sync(0xffffffffu, c1, l2);
          const double c2a = __shfl_sync(0xffffffffu, c2, l1), c2b = __shfl_sync(0xffffffffu, c2, l2);
          const double n3 = c1a * c2b - c1b * c2a;  // (c1 x c2)_k
          double ab = n3 * __shfl_sync(0xffffffffu, ev, 12 + k);
          double bb = n3 * __shfl_sync(0xffffffffu, ev, 15 + k);
          double gb = n3 * __shfl_sync(0xffffffffu, ev, 18 + k);
          ab += __shfl_sync(0xffffffffu, ab, l1) + __shfl_sync(0xffffffffu, ab, l2);
          bb += __shfl_sync(0xffffffffu, bb, l1) + __shfl_sync(0xffffffffu, bb, l2);
          gb += __shfl_sync(0xffffffffu, gb, l1) + __shfl_sync(0xffffffffu, gb, l2);
          if (act) E.zabg[iz][k] = split_f64(wz * (k == 0 ? ab : k == 1 ? bb : gb));
        }
        if (lane < 21) E.evf[lane] = evf;
        // the FP32 node columns and their norms from the FP32 element vectors
        {
          const float zf = ax.ztabf[iz][0];
          const float f1 = fmaf(zf, __shfl_sync(0xffffffffu, evf, 3 + k), __shfl_sync(0xffffffffu, evf, k));
          const float f2 = fmaf(zf, __shfl_sync(0xffffffffu, evf, 9 + k), __shfl_sync(0xffffffffu, evf, 6 + k));
          const float f1a = __shfl_sync(0xffffffffu, f1, l1), f1b = __shfl_sync(0xffffffffu, f1, l2);
          const float f2a = __shfl_sync(0xffffffffu, f2, l1), f2b = __shfl_sync(0xffffffffu, f2, l2);
          const float fn = f1a * f2b - f1b * f2a;
          float s1 = f1 * f1, s2 = f2 * f2, s3 = fn * fn;
          s1 += __shfl_sync(0xffffffffu, s1, l1) + __shfl_sync(0xffffffffu, s1, l2);
          s2 += __shfl_sync(0xffffffffu, s2, l1) + __shfl_sync(0xffffffffu, s2, l2);
          s3 += __shfl_sync(0xffffffffu, s3, l1) + __shfl_sync(0xffffffffu, s3, l2);
          if (act) {
            E.zc1f[iz][k] = f1;
            E.zc2f[iz][k] = f2;
            E.zn3f[iz][k] = fn;
            if (k == 0) {
              E.zn[iz][0] = sqrtf(s1);
              E.zn[iz][1] = sqrtf(s2);
              E.zn[iz][2] = sqrtf(s3);
            }
          }
        }
        __syncwarp();
        if (lane == 0 && a.coef_mode == FEI_COEF_PER_ELEMENT) coef_norms(E.cf, E.cn);
        // triangle nodes: c3 = C + xi1 D1 + xi2 D2 (FP32) and |c3|
        for (int t = lane; t < NT; t += 32) {
          const float x1 = ax.ttabf[t][1], x2 = ax.ttabf[t][2];
          float c3[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            c3[k] = fmaf(x2, E.evf[18 + k], fmaf(x1, E.evf[15 + k], E.evf[12 + k]));
            E.tc3f[t][k] = c3[k];
          }
          E.tn[t] = norm3f(c3);
        }
        __syncwarp();
      }
      named_bar(2, ND);
      // every point of the new elements, spread over all point-operator
      // threads (one warp's serial pass over an element's points took ten
      // times longer): w det J = w_t (a + xi1 b + xi2 g) from the FP64 node
      // sums in double-FP32 arithmetic (each factor an FP32 hi + lo pair,
      // products and sum error-free to about 2^-44), rounded once -- no FP64
      // instruction per point; the status; and the bound of
      // max_{q,b} sum_a |Dt[a][b]| that sets the element's scale
      for (int base = 0; base < nnew * NQ; base += ND) {
        const int idx = base + td;
        int i = -1;
        float m = 0.f;
        if (idx < nnew * NQ) {
          i = idx / NQ;
          const int q = idx - i * NQ;
          const int sl = slot_of(kn0 + i);
          TcElem<P> &E = ax.el[sl];
          const int iz = q / NT, t = q - iz * NT;
          const float2 sd = add_ff(add_ff(mul_ff(ax.ttab[t][0], E.zabg[iz][0]), mul_ff(ax.ttab[t][1], E.zabg[iz][1])),
                                   mul_ff(ax.ttab[t][2], E.zabg[iz][2]));
          const float sf = sd.x + sd.y;
          int st = !(fabsf(sf) <= 3.402823466e38f) ? FEI_ERR_NONFINITE : (!(sf > 0.f) ? FEI_ERR_NEGATIVE_JACOBIAN : 0);
          // the bound reads the coefficient norms after the 16 values
          float cq[19];
          if (a.coef_mode == FEI_COEF_PER_POINT) {
            bool sym = true;
            if (!load_coef_tc(a, E.qoff + q, cq, &sym)) st = FEI_ERR_NONFINITE;
            else if (a.upper && !sym && st == 0) st = FEI_ERR_INVALID_ARG;
            coef_norms(cq, cq + 16);
          } else {
#pragma unroll
            for (int k = 0; k < 3; ++k) cq[16 + k] = E.cn[k];
          }
          ax.sp[sl][q] = sf;
          if (st) {
            atomicMax(&E.status, st);
          } else {
            m = tc_bound<P>(E, ax, cq + 16, iz, t, sf);
            if (!(m <= 3.0e38f)) {
              atomicMax(&E.status, FEI_ERR_NONFINITE);
              m = 0.f;
            }
          }
        }
        // one atomic per element per warp (the bound is a max of
        // non-negative floats, so their bit patterns order as integers);
        // lanes past the last point hold i = -1, lane 0 the smallest i
        const int i0 = __shfl_sync(0xffffffffu, i, 0), i1 = __reduce_max_sync(0xffffffffu, i);
        for (int i2 = i0 < 0 ? 0 : i0; i2 <= i1 && i2 < nnew; ++i2) {
          const unsigned mb = __reduce_max_sync(0xffffffffu, i == i2 ? __float_as_uint(m) : 0u);
          if (lane == 0 && mb) atomicMax(&ax.el[slot_of(kn0 + i2)].mbits, (int)mb);
        }
      }
      named_bar(2, ND);
      if (td < nnew && KD == 1) {  // TF32 operands have the FP32 range: no scale
        TcElem<P> &E = ax.el[slot_of(kn0 + td)];
        E.up = 1.f;
        E.down = 1.f;
      } else if (td < nnew) {
        TcElem<P> &E = ax.el[slot_of(kn0 + td)];
        // The A operand is H' 2^sigma and max|G| <= 2^(14 - tau), so
        // |A| <= M 2^sigma 2^(14 - tau): sigma = tau - ex with M <= 2^ex
        // keeps it within 2^14.  The B operand is G 2^tau, so the
        // accumulator holds A_e 2^(sigma + tau).
        const float M = __int_as_float(E.mbits);
        int ex = 0;
        if (M > 0.f) (void)frexpf(M, &ex);  // M <= 2^ex
        int sigma = tau - ex;
        sigma = sigma > 100 ? 100 : (sigma < -100 ? -100 : sigma);
        E.up = exp2i(sigma);
        const int dn = -(sigma + tau);
        E.down = dn >= -126 && dn <= 126 ? exp2i(dn) : ldexpf(1.0f, dn);
      }
      named_bar(2, ND);
      // prefetch for the next tile: its new elements start after k1
      pf_k = -1;
      if (tile + 1 < t_end) {
        const int64_t r0n = r0 + 128;
        int64_t k1n = (r0n + 127) / NSH;
        if (k1n > items - 1) k1n = items - 1;
        const int64_t kf = k1 + 1 + (warp - C::W_DW);
        if (kf <= k1n) {
          // an asynchronous copy: a plain load into a register that lives on
          // held the warp at the next use of that register
          pf_k = kf;
          const double *src = input_ptr(kf);
          if (src) cp_async8(pf_slot, src);
          else *pf_slot = 0.0;
          cp_async_commit();
        }
      }
      // row data of this tile (double-buffered by tile parity)
      const int slot = it & 1;
      const bool mok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&ax.meta_empty[slot]), ((uint32_t)(it >> 1) & 1u) ^ 1u, abort_flag));
      if (mok) {
        TcMeta &M = ax.meta[slot];
        for (int r = td; r < 128; r += ND) {
          const int64_t grow = r0 + r;
          if (grow < rows_total) {
            const int64_t k = grow / NSH;
            const int ri = (int)(grow - k * NSH);
            const TcElem<P> &E = ax.el[slot_of(k)];
            M.row_off[r] = E.aoff + a_pos(ri, 0, NSH, a.upper);
            M.row_lo[r] = (int16_t)(a.upper ? ri : 0);
            M.row_boff[r] = E.boff + ri;
            M.row_eid[r] = ri == 0 ? (int32_t)E.e : -1;
            M.row_down[r] = E.down;
            M.row_status[r] = E.status;
          } else {
            M.row_off[r] = -1;
            M.row_lo[r] = 0;
            M.row_boff[r] = -1;
            M.row_eid[r] = -1;
            M.row_down[r] = 0.f;
            M.row_status[r] = 0;
          }
        }
      }
      named_bar(2, ND);
      if (td == 0 && mok) mbar_arrive(smem_u32(&ax.meta_full[slot]));
      // point operators into the ring, DB chunks per round (one wait and
      // one pass over the threads for several chunks)
      for (int c0 = 0; c0 < NCH; c0 += C::DB) {
        const int cn = NCH - c0 < C::DB ? NCH - c0 : C::DB;
        bool ok = true;
        for (int j = 0; j < cn; ++j) {
          const int g = it * NCH + c0 + j;
          ok = ok && mbar_wait(smem_u32(&ax.dempty[g % DR]), ((uint32_t)(g / DR) & 1u) ^ 1u, abort_flag);
        }
        ok = __all_sync(0xffffffffu, ok);
        if (ok) {
          for (int idx = td; idx < cn * nel * PPC; idx += ND) {
            const int j = idx / (nel * PPC), rem = idx - j * (nel * PPC);
            const int el = rem / PPC, qq = rem - el * PPC, q = (c0 + j) * PPC + qq;
            const int dr = (it * NCH + c0 + j) % DR;
            const int sl = slot_of(k0 + el);
            const TcElem<P> &E = ax.el[sl];
            // value k of this point: float4 k/2 of its pair, component
            // 2 (k % 2) + (the point's position in the pair)
            float *D1 = reinterpret_cast<float *>(&ax.Dc[dr][el][qq >> 1]) + (qq & 1);
            float cv[14];
            if (q < NQ && E.status == 0) {
              float cq[16];
              if (a.coef_mode == FEI_COEF_PER_POINT) {
                (void)load_coef_tc(a, E.qoff + q, cq);  // finiteness was tested in the pre-pass
              } else {
                // four 16-byte loads (the values are the same for the points of an element)
                const float4 *c4 = reinterpret_cast<const float4 *>(E.cf);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                  const float4 v = c4[k];
                  cq[4 * k] = v.x;
                  cq[4 * k + 1] = v.y;
                  cq[4 * k + 2] = v.z;
                  cq[4 * k + 3] = v.w;
                }
              }
              float Dt[16];
              tc_point<P>(E, ax, cq, q, ax.sp[sl][q], Dt);
              const float up = E.up;
#pragma unroll
              for (int k = 0; k < 13; ++k) cv[k] = Dt[k] * up;
              cv[13] = Dt[13];
            } else {
#pragma unroll
              for (int k = 0; k < 14; ++k) cv[k] = 0.f;
            }
#pragma unroll
            for (int k = 0; k < 14; ++k) D1[(k >> 1) * 4 * C::PP + (k & 1) * 2] = cv[k];
          }
        }
        named_bar(2, ND);
        if (td < cn && ok) mbar_arrive(smem_u32(&ax.dfull[(it * NCH + c0 + td) % DR]));
      }
    }
    cp_async_wait_all();  // a prefetch not consumed (an aborted block) has landed
  } else if (warp >= C::W_PW && warp < C::W_EW && C::TS) {
    // ========================================================= producers (TS)
    // A thread owns one row of the tile (its tensor-memory lane: warp w
    // reaches lanes 32 (w % 4) ..) and PPW consecutive point pairs of every
    // chunk; it forms H' for both points of a pair with packed FP32 FMAs,
    // splits into fp16 hi/lo and writes its pairs' hi and lo values into the
    // stage's A columns with one tcgen05.st each.  The point operators of a
    // pair are broadcast loads (the warp's rows belong to one or two
    // elements).
    const int tp = tid - C::W_PW * 32;  // 0 .. NP-1
    const int pw = warp - C::W_PW;
    const int quarter = warp & 3;
    const int part = pw >> 2;  // the PQ warps of a lane quarter split the pairs
    const int pp0 = part * C::PPW;
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    const int row = quarter * 32 + lane;
    constexpr int GST = C::GST, PPW = C::PPW;
    int it = 0;
    int64_t tile = t_begin;
    for (; tile < t_end; ++tile, ++it) {
      if (*abort_flag) break;
      const int64_t r0 = tile * 128;
      const int64_t k0 = r0 / NSH;
      // a row past the end computes finite values from element 0 of the
      // tile; the epilogue drops it
      int rel = 0, ri = 0;
      {
        const int64_t grow = r0 + row;
        if (grow < rows_total) {
          const int64_t kk = grow / NSH;
          ri = (int)(grow - kk * NSH);
          rel = (int)(kk - k0);
        }
      }
      float2 bp = make_float2(0.f, 0.f);
      for (int c = 0; c < NCH; ++c) {
        const int g = it * NCH + c, s = g % S, dr = g % DR;
        const uint32_t u = (uint32_t)(g / S), ud = (uint32_t)(g / DR);
        float4 ga[PPW], gb[PPW];
        // from L2 (the table is not in the stage): the first two pairs are
        // fetched before the waits, so that their latency overlaps them
        constexpr int PRE = 0;
        if constexpr (!C::GS) {
#pragma unroll
          for (int j = 0; j < PRE; ++j) {
            ga[j] = __ldg(gp + (size_t)((c * 2 + 0) * C::PP + pp0 + j) * GST + ri);
            gb[j] = __ldg(gp + (size_t)((c * 2 + 1) * C::PP + pp0 + j) * GST + ri);
          }
        }
        // point operators ready, the A columns free (the MMAs of the chunk S
        // before completed) and, with GS, the table rows landed
        bool ok = mbar_wait(smem_u32(&ax.dfull[dr]), ud & 1u, abort_flag);
        if constexpr (C::GS) ok = ok && mbar_wait(smem_u32(&ax.gfull[s]), u & 1u, abort_flag);
        else ok = ok && mbar_wait(smem_u32(&ax.empty[s]), (u & 1u) ^ 1u, abort_flag);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) break;
        tc_fence_after();
        const float4 *Gs = reinterpret_cast<const float4 *>(dsm_raw + (stageG(s) - smem_u32(dsm_raw)));
        // a point pair is 8 K values: 4 columns of fp16 pairs, or 8 of TF32
        const uint32_t acol = tmem + lane_base + (uint32_t)(C::ABASE + s * C::ACOLS + pp0 * 8 / C::VPC);
        const float4 *D4 = &ax.Dc[dr][rel][pp0];
        // two pairs at a time: 8 columns of hi and 8 of lo per tcgen05.st
        // (holding all pairs' values until one wider store raised the
        // register peak above the budget)
        // (with the table prefetched from L2 into registers the loop is
        // unrolled, so that the prefetched values stay in registers)
#pragma unroll(PRE == 0 ? 1 : PPW / 2)
        for (int j2 = 0; j2 < PPW; j2 += 2) {
        uint32_t hv[8], lv[8];
#pragma unroll
        for (int j1 = 0; j1 < 2; ++j1) {
          const int j = j2 + j1;
          if constexpr (C::GS) {  // the table chunk in the stage, read pair by pair
            ga[j] = Gs[(pp0 + j) * GST + ri];
            gb[j] = Gs[(C::PP + pp0 + j) * GST + ri];
          } else if (j >= PRE) {
            ga[j] = __ldg(gp + (size_t)((c * 2 + 0) * C::PP + pp0 + j) * GST + ri);
            gb[j] = __ldg(gp + (size_t)((c * 2 + 1) * C::PP + pp0 + j) * GST + ri);
          }
          float2 pd[14];
#pragma unroll
          for (int k = 0; k < 7; ++k) {
            const float4 d = D4[k * C::PP + j];
            pd[2 * k] = make_float2(d.x, d.y);
            pd[2 * k + 1] = make_float2(d.z, d.w);
          }
          const float2 g0 = make_float2(ga[j].x, ga[j].y), g1 = make_float2(ga[j].z, ga[j].w);
          const float2 g2 = make_float2(gb[j].x, gb[j].y), g3 = make_float2(gb[j].z, gb[j].w);
          // H' 2^sigma = Dt 2^sigma G at both points; (w det J f) phi
          const float2 h0 = __fmul2_rn(pd[0], g0);
          const float2 h1 = __ffma2_rn(pd[10], g3, __ffma2_rn(pd[7], g2, __ffma2_rn(pd[4], g1, __fmul2_rn(pd[1], g0))));
          const float2 h2 = __ffma2_rn(pd[11], g3, __ffma2_rn(pd[8], g2, __ffma2_rn(pd[5], g1, __fmul2_rn(pd[2], g0))));
          const float2 h3 = __ffma2_rn(pd[12], g3, __ffma2_rn(pd[9], g2, __ffma2_rn(pd[6], g1, __fmul2_rn(pd[3], g0))));
          bp = __ffma2_rn(pd[13], g0, bp);
          if constexpr (KD == 1) {
            // one K value per column: 4 values of the first point, then 4 of
            // the second, as TF32 hi = rn(x) and lo = rn(x - hi) (x - hi is
            // exact in FP32)
            const float xv[8] = {h0.x, h1.x, h2.x, h3.x, h0.y, h1.y, h2.y, h3.y};
            uint32_t th[8], tl[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) {
              th[m] = tf32_rna(xv[m]);
              tl[m] = tf32_rna(xv[m] - __uint_as_float(th[m]));
            }
            tmem_st8u(acol + 8 * j, th);
            tmem_st8u(acol + C::AHALF + 8 * j, tl);
            continue;
          }
          // two consecutive K values per column: 4 values of the first
          // point, then 4 of the second, as fp16 hi and lo = rn(x - hi)
          const __half2 w0 = __floats2half2_rn(h0.x, h1.x), w1 = __floats2half2_rn(h2.x, h3.x);
          const __half2 w2 = __floats2half2_rn(h0.y, h1.y), w3 = __floats2half2_rn(h2.y, h3.y);
          const float2 e0 = split_residual(w0, h0.x, h1.x), e1 = split_residual(w1, h2.x, h3.x);
          const float2 e2 = split_residual(w2, h0.y, h1.y), e3 = split_residual(w3, h2.y, h3.y);
          const __half2 l0 = __floats2half2_rn(e0.x, e0.y), l1 = __floats2half2_rn(e1.x, e1.y);
          const __half2 l2 = __floats2half2_rn(e2.x, e2.y), l3 = __floats2half2_rn(e3.x, e3.y);
          const int h4 = 4 * j1;
          memcpy(&hv[h4 + 0], &w0, 4);
          memcpy(&hv[h4 + 1], &w1, 4);
          memcpy(&hv[h4 + 2], &w2, 4);
          memcpy(&hv[h4 + 3], &w3, 4);
          memcpy(&lv[h4 + 0], &l0, 4);
          memcpy(&lv[h4 + 1], &l1, 4);
          memcpy(&lv[h4 + 2], &l2, 4);
          memcpy(&lv[h4 + 3], &l3, 4);
        }
        if constexpr (KD == 0) {
          tmem_st8u(acol + 4 * j2, hv);
          tmem_st8u(acol + C::AHALF + 4 * j2, lv);
        }
        }
        // the point operators of this chunk are consumed and the A columns
        // written (visible to the tensor core after the wait and the fence)
        tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(smem_u32(&ax.dempty[dr]));
          if (C::GS) mbar_arrive(smem_u32(&ax.gempty[s]));
          mbar_arrive(smem_u32(&ax.full[s]));
        }
      }
      if (*abort_flag) break;
      // load-vector partial of this thread's row (the slot is free once the
      // epilogue finished the tile two before)
      const int slot = it & 1;
      const bool mok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&ax.meta_empty[slot]),
                                                         ((uint32_t)(it >> 1) & 1u) ^ 1u, abort_flag));
      if (!mok) break;
      ax.bsum[slot][part][row] = bp.x + bp.y;
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&ax.bsum_full[slot]));
    }
    // an aborted block marks every element of its remaining tiles
    if (*abort_flag) {
      for (int64_t t2 = tile; t2 < t_end; ++t2)
        for (int rr = tp; rr < 128; rr += NP) {
          const int64_t grow = t2 * 128 + rr;
          if (grow >= rows_total) continue;
          const int64_t k = grow / NSH;
          if (grow - k * NSH != 0 && rr != 0) continue;
          const int64_t e = a.list ? (int64_t)a.list[k] : k;
          a.status[e] = FEI_ERR_TIMEOUT;
        }
    }
  } else if (warp >= C::W_PW && warp < C::W_EW) {
    // ================================================================ producers
    // The thread forms H' of one point pair pp of every chunk for its RPT
    // rows rb + rs k, both points at once with packed FP32 instructions on
    // (first point, second point) pairs.  The point operators of the pair
    // stay in registers while consecutive rows belong to the same element.
    const int tp = tid - C::W_PW * 32;  // 0 .. NP-1
    const int pw = warp - C::W_PW;
    const int pp = C::GS ? lane % C::PP : pw / C::WPP;
    const int rb = C::GS ? pw * C::RW + lane / C::PP : (pw % C::WPP) * C::RWP + lane;
    constexpr int RT = C::RPT, rs = C::GS ? C::RG : 32, GST = C::GST;
    int it = 0;
    int64_t tile = t_begin;
    for (; tile < t_end; ++tile, ++it) {
      if (*abort_flag) break;
      const int64_t r0 = tile * 128;
      const int64_t k0 = r0 / NSH;
      // rows past the end compute finite values from element 0 of the
      // tile; the epilogue drops them
      int rowr[RT], rel[RT], ri[RT];
#pragma unroll
      for (int k = 0; k < RT; ++k) {
        rowr[k] = rb + rs * k;
        const int64_t grow = r0 + rowr[k];
        rel[k] = 0;
        ri[k] = 0;
        if (grow < rows_total) {
          const int64_t kk = grow / NSH;
          ri[k] = (int)(grow - kk * NSH);
          rel[k] = (int)(kk - k0);
        }
      }
      float2 bp[RT];
#pragma unroll
      for (int k = 0; k < RT; ++k) bp[k] = make_float2(0.f, 0.f);
      for (int c = 0; c < NCH; ++c) {
        const int g = it * NCH + c, s = g % S, dr = g % DR;
        const uint32_t u = (uint32_t)(g / S), ud = (uint32_t)(g / DR);
        // the paired FP32 table of this point pair at this thread's rows:
        // from the stage (copied there with the B operand), or from L2,
        // fetched before the waits so that their latency overlaps them
        // (at p = 5, 6 only the first half of the rows is fetched early:
        // holding all of them across the waits exceeded the register budget
        // and was slower; p = 7 has the registers)
        constexpr int RPRE = P == 7 ? RT : RT / 2;
        float4 ga[RT], gb[RT];
        if constexpr (!C::GS) {
#pragma unroll
          for (int k = 0; k < RPRE; ++k) {
            ga[k] = __ldg(gp + (size_t)((c * 2 + 0) * C::PP + pp) * GST + ri[k]);
            gb[k] = __ldg(gp + (size_t)((c * 2 + 1) * C::PP + pp) * GST + ri[k]);
          }
        }
        // point operators ready, the A slot free (the MMAs of the chunk S
        // before completed) and, with GS, the table chunk landed
        bool ok = mbar_wait(smem_u32(&ax.dfull[dr]), ud & 1u, abort_flag);
        if constexpr (C::GS) ok = ok && mbar_wait(smem_u32(&ax.gfull[s]), u & 1u, abort_flag);
        else ok = ok && mbar_wait(smem_u32(&ax.empty[s]), (u & 1u) ^ 1u, abort_flag);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) break;
        if constexpr (!C::GS) {
#pragma unroll
          for (int k = RPRE; k < RT; ++k) {
            ga[k] = __ldg(gp + (size_t)((c * 2 + 0) * C::PP + pp) * GST + ri[k]);
            gb[k] = __ldg(gp + (size_t)((c * 2 + 1) * C::PP + pp) * GST + ri[k]);
          }
        }
        if constexpr (C::GS) {
          const float4 *Gs = reinterpret_cast<const float4 *>(dsm_raw + (stageG(s) - smem_u32(dsm_raw)));
#pragma unroll
          for (int k = 0; k < RT; ++k) {
            ga[k] = Gs[pp * GST + ri[k]];
            gb[k] = Gs[(C::PP + pp) * GST + ri[k]];
          }
        }
        // generic pointers to the stage's hi and lo operand tiles
        unsigned char *const ahp = dsm_raw + (stageA(s, 0) - smem_u32(dsm_raw));
        unsigned char *const alp = ahp + C::A_BYTES;
        float2 pd[14];
        int cur = -1;
#pragma unroll
        for (int k = 0; k < RT; ++k) {
          if (rel[k] != cur) {
            cur = rel[k];
            const float4 *D4 = &ax.Dc[dr][cur][pp];
#pragma unroll
            for (int j = 0; j < 7; ++j) {
              const float4 d = D4[j * C::PP];
              pd[2 * j] = make_float2(d.x, d.y);
              pd[2 * j + 1] = make_float2(d.z, d.w);
            }
          }
          const float2 g0 = make_float2(ga[k].x, ga[k].y), g1 = make_float2(ga[k].z, ga[k].w);
          const float2 g2 = make_float2(gb[k].x, gb[k].y), g3 = make_float2(gb[k].z, gb[k].w);
          // H' 2^sigma = Dt 2^sigma G at both points; (w det J f) phi
          const float2 h0 = __fmul2_rn(pd[0], g0);
          const float2 h1 = __ffma2_rn(pd[10], g3, __ffma2_rn(pd[7], g2, __ffma2_rn(pd[4], g1, __fmul2_rn(pd[1], g0))));
          const float2 h2 = __ffma2_rn(pd[11], g3, __ffma2_rn(pd[8], g2, __ffma2_rn(pd[5], g1, __fmul2_rn(pd[2], g0))));
          const float2 h3 = __ffma2_rn(pd[12], g3, __ffma2_rn(pd[9], g2, __ffma2_rn(pd[6], g1, __fmul2_rn(pd[3], g0))));
          bp[k] = __ffma2_rn(pd[13], g0, bp[k]);
          if constexpr (KD == 1) {
            // two 16-byte operand chunks: the 4 values of the first point,
            // then the 4 of the second, as TF32 hi = rn(x), lo = rn(x - hi)
            const float xv[8] = {h0.x, h1.x, h2.x, h3.x, h0.y, h1.y, h2.y, h3.y};
            uint32_t th[8], tl[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) {
              th[m] = tf32_rna(xv[m]);
              tl[m] = tf32_rna(xv[m] - __uint_as_float(th[m]));
            }
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
              const uint32_t aoff = sw_off<ROWB>(rowr[k], 2 * pp + hh);
              *reinterpret_cast<uint4 *>(ahp + aoff) = make_uint4(th[4 * hh], th[4 * hh + 1], th[4 * hh + 2], th[4 * hh + 3]);
              *reinterpret_cast<uint4 *>(alp + aoff) = make_uint4(tl[4 * hh], tl[4 * hh + 1], tl[4 * hh + 2], tl[4 * hh + 3]);
            }
            continue;
          }
          // the 16-byte operand chunk: 4 values of the first point, then 4
          // of the second, as fp16 hi and lo = rn(x - hi)
          const __half2 w0 = __floats2half2_rn(h0.x, h1.x), w1 = __floats2half2_rn(h2.x, h3.x);
          const __half2 w2 = __floats2half2_rn(h0.y, h1.y), w3 = __floats2half2_rn(h2.y, h3.y);
          const float2 e0 = split_residual(w0, h0.x, h1.x), e1 = split_residual(w1, h2.x, h3.x);
          const float2 e2 = split_residual(w2, h0.y, h1.y), e3 = split_residual(w3, h2.y, h3.y);
          const __half2 l0 = __floats2half2_rn(e0.x, e0.y), l1 = __floats2half2_rn(e1.x, e1.y);
          const __half2 l2 = __floats2half2_rn(e2.x, e2.y), l3 = __floats2half2_rn(e3.x, e3.y);
          uint4 hw, lw;
          memcpy(&hw.x, &w0, 4);
          memcpy(&hw.y, &w1, 4);
          memcpy(&hw.z, &w2, 4);
          memcpy(&hw.w, &w3, 4);
          memcpy(&lw.x, &l0, 4);
          memcpy(&lw.y, &l1, 4);
          memcpy(&lw.z, &l2, 4);
          memcpy(&lw.w, &l3, 4);
          const uint32_t aoff = sw_off<ROWB>(rowr[k], pp);
          *reinterpret_cast<uint4 *>(ahp + aoff) = hw;
          *reinterpret_cast<uint4 *>(alp + aoff) = lw;
        }
        // the point operators of this chunk are consumed and the A slot is
        // written (made visible to the tensor core's proxy)
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(smem_u32(&ax.dempty[dr]));
          if (C::GS) mbar_arrive(smem_u32(&ax.gempty[s]));
          mbar_arrive(smem_u32(&ax.full[s]));
        }
      }
      if (*abort_flag) break;
      // load-vector partials of the tile's rows for this point pair (the
      // slot is free once the epilogue finished the tile two before)
      const int slot = it & 1;
      const bool mok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&ax.meta_empty[slot]),
                                                         ((uint32_t)(it >> 1) & 1u) ^ 1u, abort_flag));
      if (!mok) break;
#pragma unroll
      for (int k = 0; k < RT; ++k) ax.bsum[slot][pp][rowr[k]] = bp[k].x + bp[k].y;
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&ax.bsum_full[slot]));
    }
    // an aborted block marks every element of its remaining tiles
    if (*abort_flag) {
      for (int64_t t2 = tile; t2 < t_end; ++t2)
        for (int rr = tp; rr < 128; rr += NP) {
          const int64_t grow = t2 * 128 + rr;
          if (grow >= rows_total) continue;
          const int64_t k = grow / NSH;
          if (grow - k * NSH != 0 && rr != 0) continue;
          const int64_t e = a.list ? (int64_t)a.list[k] : k;
          a.status[e] = FEI_ERR_TIMEOUT;
        }
    }
  } else if (warp >= C::W_EW) {
    // ================================================================ epilogue
    const int ew = warp - C::W_EW;    // 0..3
    const int quarter = warp & 3;     // TMEM lanes 32*quarter ..
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    const int myrow = quarter * 32 + lane;
    // a contiguous output (uniform degree, no element list, 16-byte aligned):
    // the tile's rows of A_e are one range of A
    const bool contiguous = a.A_off == nullptr && (a.list == nullptr || a.out_by_item) && !a.upper &&
                            (reinterpret_cast<uintptr_t>(a.A) & 15u) == 0u;
    float rreg[C::RREG > 0 ? C::RREG : 1];
    int it = 0;
    uint32_t unit = 0;
    bool dead = false;
    for (int64_t tile = t_begin; tile < t_end && !dead; ++tile, ++it) {
      for (int c = 0; c < NCH && !dead; c += C::UC) {
#pragma unroll
        for (int nh = 0; nh < C::NHALF; ++nh) {
          const uint32_t pb = unit % C::NPART, k = unit / C::NPART;
          ++unit;
          const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&ax.part_full[pb]), k & 1u, abort_flag));
          if (!ok) {
            dead = true;
            break;
          }
          tc_fence_after();
          // one 16-column block at a time: load the partial (and the running
          // sum), wait, add, store.  Loading two blocks before one wait
          // raised the register peak of the whole kernel above its budget
          // (spills at every degree) and was slower.
#pragma unroll
          for (int b0 = 0; b0 < C::NMMA / 16; b0 += 1) {
            uint32_t pv[1][16], rv[1][16];
#pragma unroll
            for (int j = 0; j < 1; ++j) {
              const int b = b0 + j;
              if (b < C::NMMA / 16) {
                const int ncol = nh * C::NMMA + b * 16;
                tmem_ld16_nw(tmem + lane_base + pb * C::NMMA + b * 16, pv[j]);
                if (ncol < C::RT && c > 0) tmem_ld16_nw(tmem + lane_base + C::RSUM + ncol, rv[j]);
              }
            }
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 1; ++j) {
              const int b = b0 + j;
              if (b < C::NMMA / 16) {
                const int ncol = nh * C::NMMA + b * 16;
                float v[16];
#pragma unroll
                for (int k2 = 0; k2 < 16; ++k2) v[k2] = __uint_as_float(pv[j][k2]);
                if (ncol < C::RT) {
                  if (c > 0) {
#pragma unroll
                    for (int k2 = 0; k2 < 16; k2 += 2) {
                      const float2 t = __fadd2_rn(make_float2(v[k2], v[k2 + 1]),
                                                  make_float2(__uint_as_float(rv[j][k2]), __uint_as_float(rv[j][k2 + 1])));
                      v[k2] = t.x;
                      v[k2 + 1] = t.y;
                    }
                  }
                  tmem_st16(tmem + lane_base + C::RSUM + ncol, v);
                } else if constexpr (C::RREG > 0) {
                  const int ro = ncol - C::RT;
#pragma unroll
                  for (int k2 = 0; k2 < 16; ++k2) rreg[ro + k2] = (c > 0 ? rreg[ro + k2] : 0.f) + v[k2];
                }
              }
            }
          }
          tmem_wait_st();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&ax.promo_done[pb]));
        }
      }
      if (dead) break;
      // final: scale the running sum and store the tile's rows of A_e
      const int slot = it & 1;
      const uint32_t km = (uint32_t)(it >> 1);
      bool mok = mbar_wait(smem_u32(&ax.meta_full[slot]), km & 1u, abort_flag);
      mok = mok && mbar_wait(smem_u32(&ax.bsum_full[slot]), km & 1u, abort_flag);
      if (!__all_sync(0xffffffffu, mok)) break;
      const TcMeta &M = ax.meta[slot];
      const float dn = M.row_status[myrow] ? 0.f : M.row_down[myrow];
      // load vector and status of this lane's row
      if (M.row_boff[myrow] >= 0) {
        float bsum = 0.f;
#pragma unroll
        for (int j = 0; j < C::BSN; ++j) bsum += ax.bsum[slot][j][myrow];
        const int st = M.row_status[myrow];
        reinterpret_cast<float *>(a.bv)[M.row_boff[myrow]] = st ? 0.f : bsum;
        if (M.row_eid[myrow] >= 0) a.status[M.row_eid[myrow]] = st;
      }
      // rows of this warp: 32 * quarter + [0, 32) of the tile
      const int64_t wrow0 = tile * 128 + quarter * 32;
      const int nvalid = rows_total - wrow0 >= 32 ? 32 : (rows_total - wrow0 > 0 ? (int)(rows_total - wrow0) : 0);
      if (C::BS && contiguous) {
        // two halves of 16 rows: lanes 16h .. 16h+15 stage their rows, one
        // lane stores the half with a bulk copy (A_e rows of consecutive
        // elements are consecutive in a contiguous layout)
        float *buf = ax.rows16[ew];
        for (int h = 0; h < 2; ++h) {
          const int nh = nvalid - 16 * h >= 16 ? 16 : (nvalid - 16 * h > 0 ? nvalid - 16 * h : 0);
          if (lane == 0) bulk_wait_read();  // the previous copy has read the buffer
          __syncwarp();
          const bool mine = (lane >> 4) == h;
#pragma unroll
          for (int b = 0; b < C::NPAD / 16; ++b) {
            const int ncol = b * 16;
            if (ncol < NSH) {
              float v[16];
              if (ncol < C::RT) {
                tmem_ld16(tmem + lane_base + C::RSUM + ncol, v);
              } else if constexpr (C::RREG > 0) {
#pragma unroll
                for (int k2 = 0; k2 < 16; ++k2) v[k2] = rreg[ncol - C::RT + k2];
              }
              if (mine) {
                float *dst = buf + (lane & 15) * NSH + ncol;
#pragma unroll
                for (int k2 = 0; k2 < 16; ++k2)
                  if (ncol + k2 < NSH) dst[k2] = v[k2] * dn;
              }
            }
          }
          fence_proxy_async();
          __syncwarp();
          if (lane == 0 && nh > 0) {
            const uint32_t bytes = (uint32_t)(nh * NSH * 4);
            float *gdst = reinterpret_cast<float *>(a.A) + (wrow0 + 16 * h) * NSH;
            if ((bytes & 15u) == 0u) {
              bulk_s2g(gdst, smem_u32(buf), bytes);
            } else {
              // a ragged tail whose size is not a multiple of 16 bytes
              for (int k = 0; k < nh * NSH; ++k) gdst[k] = buf[k];
            }
          }
        }
      } else {
        float(*stg)[17] = ax.stg[ew];
  #pragma unroll
        for (int b = 0; b < C::NPAD / 16; ++b) {
          const int ncol = b * 16;
          if (ncol < NSH) {
            float v[16];
            if (ncol < C::RT) {
              tmem_ld16(tmem + lane_base + C::RSUM + ncol, v);
            } else if constexpr (C::RREG > 0) {
  #pragma unroll
              for (int k2 = 0; k2 < 16; ++k2) v[k2] = rreg[ncol - C::RT + k2];
            }
  #pragma unroll
            for (int k2 = 0; k2 < 16; ++k2) stg[lane][k2] = v[k2] * dn;
            __syncwarp();
            // two rows per store instruction: lanes 0-15 row rr, 16-31 row rr+1;
            // eight rows' values and offsets are read before their stores (a
            // global store could alias the staging buffer as far as the
            // compiler knows, so interleaving would serialise every load
            // behind the previous store)
            const int half = lane >> 4, col = ncol + (lane & 15);
            float *const Aout = reinterpret_cast<float *>(a.A);
  #pragma unroll
            for (int r16 = 0; r16 < 32; r16 += 16) {
              float vv[8];
              int64_t oo[8];
              int lo[8];
  #pragma unroll
              for (int j = 0; j < 8; ++j) {
                const int rr = r16 + 2 * j;
                oo[j] = M.row_off[quarter * 32 + rr + half];
                lo[j] = M.row_lo[quarter * 32 + rr + half];
                vv[j] = stg[rr + half][lane & 15];
              }
  #pragma unroll
              for (int j = 0; j < 8; ++j)
                if (oo[j] >= 0 && col < NSH && col >= lo[j]) Aout[oo[j] + col] = vv[j];
            }
            __syncwarp();
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&ax.meta_empty[slot]));
    }
    if (C::BS && lane == 0) bulk_wait_all();  // this warp's bulk stores have landed
  } else if (warp == 0) {
    // ================================================================ B stream
    if (lane == 0) {
      int it = 0;
      for (int64_t tile = t_begin; tile < t_end; ++tile, ++it) {
        bool ok = true;
        for (int c = 0; c < NCH; ++c) {
          const int g = it * NCH + c, s = g % S;
          const uint32_t u = (uint32_t)(g / S);
          // the table rows once the producers have read the chunk S before
          // (they are needed first, and that happens before its MMAs end)
          if (C::GS) {
            if (!mbar_wait(smem_u32(&ax.gempty[s]), (u & 1u) ^ 1u, abort_flag)) {
              ok = false;
              break;
            }
            const uint32_t gbar = smem_u32(&ax.gfull[s]);
            if (g < S) mbar_arrive(gbar);  // no MMAs before the first use
            mbar_expect_tx(gbar, (uint32_t)C::G_BYTES);
            bulk_g2s(stageG(s), gp + (size_t)c * 2 * C::PP * C::GST, (uint32_t)C::G_BYTES, gbar);
          }
          // the B operand once the MMAs of the chunk S before completed
          if (!mbar_wait(smem_u32(&ax.empty[s]), (u & 1u) ^ 1u, abort_flag)) {
            ok = false;
            break;
          }
          const uint32_t bar = smem_u32(&ax.bfull[s]);
          mbar_expect_tx(bar, 2u * C::B_BYTES);
          bulk_g2s(stageB(s), img + (size_t)c * 2 * C::B_BYTES, 2u * C::B_BYTES, bar);
        }
        if (!ok) break;
      }
    }
  } else {
    // ================================================================ MMA issue
    // The whole warp runs the loop and its waits; one elected lane issues
    // the MMAs and the commits (tc_mma_ts_w, tc_commit_w).
    {
      constexpr uint32_t IDESC = idesc_mma(128, C::NMMA, KD);
      bool ok = true;
      uint32_t unit = 0;
      int it = 0;
      for (int64_t tile = t_begin; tile < t_end && ok; ++tile, ++it) {
        for (int c0 = 0; c0 < NCH && ok; c0 += C::UC) {
          const int cn = NCH - c0 < C::UC ? NCH - c0 : C::UC;
          int st[C::UC];
          for (int j = 0; j < cn; ++j) {
            const int g = it * NCH + c0 + j;
            st[j] = g % S;
            const uint32_t u = (uint32_t)(g / S);
            ok = ok && mbar_wait(smem_u32(&ax.bfull[st[j]]), u & 1u, abort_flag) &&
                 mbar_wait(smem_u32(&ax.full[st[j]]), u & 1u, abort_flag);
          }
          ok = __all_sync(0xffffffffu, ok);
          if (!ok) break;
          tc_fence_after();
#pragma unroll
          for (int nh = 0; nh < C::NHALF; ++nh) {
            const uint32_t pb = unit % C::NPART, k = unit / C::NPART;
            ++unit;
            ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&ax.promo_done[pb]), (k & 1u) ^ 1u, abort_flag));
            if (!ok) break;
            tc_fence_after();
            const uint32_t d = tmem + pb * C::NMMA;
            for (int j = 0; j < cn; ++j) {
              const uint32_t bh = stageB(st[j]), bl = bh + C::B_BYTES;
              if constexpr (C::TS) {
                // A hi / lo from the stage's tensor-memory columns
                // one K slice (32 bytes of a row) is 8 columns in both kinds
                const uint32_t ah = tmem + (uint32_t)(C::ABASE + st[j] * C::ACOLS), alo = ah + C::AHALF;
#pragma unroll
                for (int kk = 0; kk < C::KSL; ++kk) {
                  const uint32_t boff = (uint32_t)(nh * C::NMMA * ROWB + kk * 32);
                  const uint64_t Bh = sw_desc<ROWB>(bh + boff), Bl = sw_desc<ROWB>(bl + boff);
                  tc_mma_ts_w<KD>(d, ah + kk * 8, Bh, IDESC, (j | kk) != 0);
                  tc_mma_ts_w<KD>(d, ah + kk * 8, Bl, IDESC, 1u);
                  tc_mma_ts_w<KD>(d, alo + kk * 8, Bh, IDESC, 1u);
                }
              } else {
                const uint32_t ah = stageA(st[j], 0), alo = stageA(st[j], 1);
#pragma unroll
                for (int kk = 0; kk < C::KSL; ++kk) {
                  const uint32_t boff = (uint32_t)(nh * C::NMMA * ROWB + kk * 32);
                  const uint64_t Ah = sw_desc<ROWB>(ah + kk * 32), Al = sw_desc<ROWB>(alo + kk * 32);
                  const uint64_t Bh = sw_desc<ROWB>(bh + boff), Bl = sw_desc<ROWB>(bl + boff);
                  tc_mma_ss_w<KD>(d, Ah, Bh, IDESC, (j | kk) != 0);
                  tc_mma_ss_w<KD>(d, Ah, Bl, IDESC, 1u);
                  tc_mma_ss_w<KD>(d, Al, Bh, IDESC, 1u);
                }
              }
            }
            tc_commit_w(smem_u32(&ax.part_full[pb]));
          }
          if (ok)
            for (int j = 0; j < cn; ++j) {
              tc_commit_w(smem_u32(&ax.empty[st[j]]));
              if (C::GS) tc_commit_w(smem_u32(&ax.gfull[st[j]]));
            }
        }
      }
      if (!ok) {
        // make sure no MMA is in flight before the block leaves
        tc_commit_w(smem_u32(&ax.drain));
        const uint64_t t0 = global_ns();
        while (!mbar_try_wait(smem_u32(&ax.drain), 0) && global_ns() - t0 < kWaitLimitNs) {
        }
        __syncwarp();
      }
    }
  }
  // in-flight bulk copies of an aborted block land within microseconds
  if (*abort_flag) {
    const uint64_t t0 = global_ns();
    while (global_ns() - t0 < 200000ull) {
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS) : "memory");
  }
}

// ---------------------------------------------------------------------------
// Tensor-core adjoint: dL/dDt from W^T = G gA^T, element by element
// ---------------------------------------------------------------------------
// For one element, W^T[(q,b)][i] = sum_j G[q][b][j] gA[i][j] (the transpose
// of W = gA G^T of the reverse pass, Sec. 2 with the weak form of Eq. (2)) is
// a product with M = 4 N_q rows (q, b) of the table (A operand: the same for
// every element, split G 2^tau streamed by the copy lane), N = N_sh rows of
// gA (B operand: each row split into fp16 hi/lo with its own power-of-two
// scale by the producer warps) and K = N_sh (j).  Three products per K slice
// (hi hi + hi lo + lo hi) into partial accumulators of at most four K slices,
// as in the forward.  The epilogue thread of TMEM lane (q, b) adds the
// partials and forms dL/dDt_q[a][b] = sum_i G[q][a][i] W^T[(q,b)][i] from its
// own columns, so no reduction crosses lanes; the result goes to a scratch
// array [element][N_q][16] that the chain of the FP32 adjoint reads.
template <int P>
struct TaCfg {
  static constexpr int NSH = nsh_of(P), NQ = nq_of(P);
  static constexpr int K = (NSH + 31) / 32 * 32;     // K padded to whole 64-byte rows
  static constexpr int NKC = K / 32;                 // K chunks, one 64-byte row each
  static constexpr int KS = K / 16;                  // MMA K slices
  static constexpr int NPAD = (NSH + 15) / 16 * 16;  // MMA N
  static constexpr int NMT = (4 * NQ + 127) / 128;   // M tiles of 128 rows (q, b)
  static constexpr int SPP = 4;                      // K slices per partial accumulator
  static constexpr int NPK = (KS + SPP - 1) / SPP;   // partials per M tile
  static constexpr int NBUF = 2;                     // accumulator buffers (M tiles in flight)
  static constexpr int ACC_COLS = NPK * NPAD;
  static constexpr int TMEM_COLS = NBUF * ACC_COLS <= 32 ? 32 : NBUF * ACC_COLS <= 64 ? 64
                                   : NBUF * ACC_COLS <= 128 ? 128 : NBUF * ACC_COLS <= 256 ? 256 : 512;
  static constexpr int A_TILE = 128 * 64;            // hi or lo of one K chunk of an M tile
  static constexpr int A_STAGE = 2 * A_TILE;
  static constexpr int NSTG = 4;                     // A stages
  static constexpr int B_TILE = NPAD * 64;
  static constexpr int B_BUF = NKC * 2 * B_TILE;     // [K chunk][hi, lo][NPAD rows][64 bytes]
  static constexpr int NB = 2;                       // B buffers (elements in flight)
  static constexpr int NRS = 4;                      // row-scale sets (producers run <= 2 elements ahead)
  static constexpr int DYN_SMEM = NSTG * A_STAGE + NB * B_BUF + 1024;
  // producer warps; epilogue warps, two per tensor-memory lane quarter,
  // each pair splitting the columns
  static constexpr int NPW = 4, NEW = 8;
  static constexpr int W_PW = 2, W_EW = W_PW + NPW;
  static constexpr int NTHREADS = (2 + NPW + NEW) * 32;
  static constexpr int NCB = NPAD / 16, NCB0 = (NCB + 1) / 2;  // column blocks; the first half's share
  static_assert(NBUF * ACC_COLS <= 512, "tensor memory");
  static_assert(NPAD <= 256 && NPAD % 16 == 0, "MMA N");
  static_assert(NPAD % 8 == 0 && B_TILE % 1024 == 0, "swizzle atoms of the B tiles");
  static_assert(K / 8 <= 16, "a row's 16-byte chunks fit in 16 lanes");
  static_assert(NEW == 8, "two groups of four consecutive epilogue warps cover the TMEM lane quarters");
};

template <int P>
struct TaAux {
  using C = TaCfg<P>;
  uint64_t afull[C::NSTG], aempty[C::NSTG];
  uint64_t bfull[C::NB], bempty[C::NB];
  uint64_t accfull[C::NBUF], accempty[C::NBUF];
  // the row scales of an element written (the epilogue reads them; a slot
  // is rewritten four elements later, when the epilogue is past it)
  uint64_t rsfull[C::NRS];
  uint64_t drain;
  uint32_t tmem_base;
  int abort_flag;
  float rs[C::NRS][C::NPAD];  // 2^-s of each gA row (its split scale)
  float4 comb[2][4][32];      // second-half epilogue sums, by tile parity, quarter and lane
};

// gD [count][N_q][16] (FP32, dL/dDt_q[a][b] at 4 a + b) for the elements
// e0 .. e0 + count - 1 of the batch (no list: uniform degree).
template <int P>
__global__ void __launch_bounds__(TaCfg<P>::NTHREADS, 1)
    tc_adjoint_kernel(const float *gA, const int64_t *A_off, int64_t e0, int64_t count, const unsigned char *aimg,
                      const float4 *gq4, int tau, float *gD) {
  using C = TaCfg<P>;
  constexpr int NSH = C::NSH, NQ = C::NQ, NPAD = C::NPAD, NKC = C::NKC, NMT = C::NMT, S = C::NSTG;
  extern __shared__ __align__(1024) unsigned char dsm_raw[];
  __shared__ TaAux<P> ax;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t dbase = (smem_u32(dsm_raw) + 1023u) & ~1023u;
  auto stageA = [&](int s) { return dbase + (uint32_t)(s * C::A_STAGE); };
  auto bufB = [&](int bb) { return dbase + (uint32_t)(S * C::A_STAGE + bb * C::B_BUF); };
  volatile int *abort_flag = &ax.abort_flag;
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&ax.afull[s]), 1);
      mbar_init(smem_u32(&ax.aempty[s]), 1);
    }
    for (int k = 0; k < C::NB; ++k) {
      mbar_init(smem_u32(&ax.bfull[k]), C::NPW);
      mbar_init(smem_u32(&ax.bempty[k]), 1);
    }
    for (int k = 0; k < C::NBUF; ++k) {
      mbar_init(smem_u32(&ax.accfull[k]), 1);
      mbar_init(smem_u32(&ax.accempty[k]), C::NEW);
    }
    for (int k = 0; k < C::NRS; ++k) mbar_init(smem_u32(&ax.rsfull[k]), C::NPW);
    mbar_init(smem_u32(&ax.drain), 1);
    ax.abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ax.tmem_base)),
                 "r"(C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ax.tmem_base;
  // this block's elements: b, b + grid, ... (local index k, element e0 + k)
  const int64_t kfirst = blockIdx.x, kstep = gridDim.x;

  if (warp == 0) {
    // ============================================================ A stream
    if (lane == 0) {
      uint32_t g = 0;
      bool ok = true;
      for (int64_t k = kfirst; k < count && ok; k += kstep)
        for (int m = 0; m < NMT && ok; ++m)
          for (int kc = 0; kc < NKC; ++kc, ++g) {
            const int s = (int)(g % S);
            const uint32_t u = g / S;
            if (!mbar_wait(smem_u32(&ax.aempty[s]), (u & 1u) ^ 1u, abort_flag)) {
              ok = false;
              break;
            }
            const uint32_t bar = smem_u32(&ax.afull[s]);
            mbar_expect_tx(bar, (uint32_t)C::A_STAGE);
            bulk_g2s(stageA(s), aimg + (size_t)(m * NKC + kc) * C::A_STAGE, (uint32_t)C::A_STAGE, bar);
          }
    }
  } else if (warp == 1) {
    // ================================================================ MMA
    constexpr uint32_t IDESC = idesc_mma(128, NPAD, 0);
    bool ok = true;
    uint32_t g = 0, tile = 0;
    int it = 0;
    for (int64_t k = kfirst; k < count && ok; k += kstep, ++it) {
      const int bb = it % C::NB;
      ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&ax.bfull[bb]), (uint32_t)(it / C::NB) & 1u, abort_flag));
      if (!ok) break;
      tc_fence_after();
      const uint32_t bh0 = bufB(bb);
      for (int m = 0; m < NMT && ok; ++m, ++tile) {
        const int buf = (int)(tile % C::NBUF);
        ok = __all_sync(0xffffffffu,
                        mbar_wait(smem_u32(&ax.accempty[buf]), ((tile / C::NBUF) & 1u) ^ 1u, abort_flag));
        if (!ok) break;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * C::ACC_COLS);
        for (int kc = 0; kc < NKC; ++kc, ++g) {
          const int s = (int)(g % S);
          ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&ax.afull[s]), (g / S) & 1u, abort_flag));
          if (!ok) break;
          tc_fence_after();
#pragma unroll
          for (int kk = 0; kk < 2; ++kk) {
            const int ks = kc * 2 + kk;
            const uint32_t dp = d + (uint32_t)((ks / C::SPP) * NPAD);
            const uint32_t first = (ks % C::SPP) == 0 ? 0u : 1u;
            const uint64_t Ah = sw_desc<64>(stageA(s) + kk * 32), Al = sw_desc<64>(stageA(s) + C::A_TILE + kk * 32);
            const uint64_t Bh = sw_desc<64>(bh0 + (uint32_t)((kc * 2) * C::B_TILE + kk * 32));
            const uint64_t Bl = sw_desc<64>(bh0 + (uint32_t)((kc * 2 + 1) * C::B_TILE + kk * 32));
            tc_mma_ss_w<0>(dp, Ah, Bh, IDESC, first);
            tc_mma_ss_w<0>(dp, Ah, Bl, IDESC, 1u);
            tc_mma_ss_w<0>(dp, Al, Bh, IDESC, 1u);
          }
          tc_commit_w(smem_u32(&ax.aempty[s]));
        }
        if (ok) tc_commit_w(smem_u32(&ax.accfull[buf]));
      }
      if (ok) tc_commit_w(smem_u32(&ax.bempty[bb]));
    }
    if (!ok) {
      // no MMA in flight when the block leaves
      tc_commit_w(smem_u32(&ax.drain));
      const uint64_t t0 = global_ns();
      while (!mbar_try_wait(smem_u32(&ax.drain), 0) && global_ns() - t0 < kWaitLimitNs) {
      }
      __syncwarp();
    }
  } else if (warp < C::W_EW) {
    // ========================================================== producers
    // 16 lanes per row, lane c the row's K values 8 c .. 8 c + 7; a warp two
    // rows at a time.  Each row is scaled by 2^s (s from its largest
    // magnitude, so that it is at most 2^14) and split into fp16 hi + lo.
    const int pw = warp - C::W_PW, half = lane >> 4, c8 = lane & 15;
    const int64_t cw = (int64_t)NSH * NSH;
    int it = 0;
    for (int64_t k = kfirst; k < count; k += kstep, ++it) {
      const int bb = it % C::NB;
      const bool ok =
          __all_sync(0xffffffffu, mbar_wait(smem_u32(&ax.bempty[bb]), ((uint32_t)(it / C::NB) & 1u) ^ 1u, abort_flag));
      if (!ok) break;
      const int64_t e = e0 + k;
      const float *row0 = gA + (A_off ? A_off[e] : e * cw);
      float *rs = ax.rs[it % C::NRS];
      const uint32_t b0 = bufB(bb);
#pragma unroll 4
      for (int r = 2 * pw + half; r < NPAD; r += 2 * C::NPW) {
        float v[8];
        float mx = 0.f;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int j = 8 * c8 + t;
          v[t] = (r < NSH && j < NSH) ? __ldg(row0 + (int64_t)r * NSH + j) : 0.f;
          mx = fmaxf(mx, fabsf(v[t]));
        }
#pragma unroll
        for (int o = 1; o < 16; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        int ex = 0;
        if (mx > 0.f && mx <= 3.402823466e38f) (void)frexpf(mx, &ex);  // mx <= 2^ex
        int sc = 14 - ex;
        sc = sc > 100 ? 100 : (sc < -100 ? -100 : sc);
        const float up = exp2i(sc / 2) * exp2i(sc - sc / 2);
        if (c8 == 0) rs[r] = exp2i(-(sc / 2)) * exp2i(-(sc - sc / 2));
        uint32_t hv[4], lv[4];
#pragma unroll
        for (int t = 0; t < 8; t += 2) {
          const float x0 = v[t] * up, x1 = v[t + 1] * up;
          const __half2 h = __floats2half2_rn(x0, x1);
          const float2 rr = split_residual(h, x0, x1);
          const __half2 l = __floats2half2_rn(rr.x, rr.y);
          memcpy(&hv[t / 2], &h, 4);
          memcpy(&lv[t / 2], &l, 4);
        }
        if (8 * c8 < C::K) {
          const int kc = c8 >> 2, un = c8 & 3;
          const uint32_t off = sw_off<64>(r, un);
          st_shared_v4(b0 + (uint32_t)((kc * 2) * C::B_TILE) + off, hv);
          st_shared_v4(b0 + (uint32_t)((kc * 2 + 1) * C::B_TILE) + off, lv);
        }
      }
      // the B operand is read by the tensor core (async proxy)
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(smem_u32(&ax.bfull[bb]));
        mbar_arrive(smem_u32(&ax.rsfull[it % C::NRS]));
      }
    }
  } else {
    // =========================================================== epilogue
    // Warp w of the group: lane quarter w & 3, column half (w - W_EW) / 4.
    // The second half leaves its sums in shared memory (by tile parity)
    // and the first half, after a named barrier of the pair, stores.
    const int quarter = warp & 3, ch = (warp - C::W_EW) >> 2;
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    const int r = quarter * 32 + lane;
    const int cb0 = ch == 0 ? 0 : C::NCB0, cb1 = ch == 0 ? C::NCB0 : C::NCB;
    const float down = exp2i(-tau);
    uint32_t tile = 0;
    int it = 0;
    bool ok = true;
    for (int64_t k = kfirst; k < count && ok; k += kstep, ++it) {
      const float *rs = ax.rs[it % C::NRS];
      ok = __all_sync(0xffffffffu,
                      mbar_wait(smem_u32(&ax.rsfull[it % C::NRS]), (uint32_t)(it / C::NRS) & 1u, abort_flag));
      if (!ok) break;
      for (int m = 0; m < NMT; ++m, ++tile) {
        const int buf = (int)(tile % C::NBUF);
        ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&ax.accfull[buf]), (tile / C::NBUF) & 1u, abort_flag));
        if (!ok) break;
        tc_fence_after();
        const int qb = 128 * m + r, q = qb >> 2, b = qb & 3;
        const bool valid = q < NQ;
        const float4 *g4 = gq4 + (size_t)(valid ? q : 0) * NPAD;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
        for (int cb = cb0; cb < cb1; ++cb) {
          // the table values first (no condition: the table is padded), so
          // that their latency overlaps the tensor-memory loads
          float4 gv[16];
#pragma unroll
          for (int k2 = 0; k2 < 16; ++k2) gv[k2] = __ldg(g4 + 16 * cb + k2);
          uint32_t pv[C::NPK][16];
#pragma unroll
          for (int pk = 0; pk < C::NPK; ++pk)
            tmem_ld16_nw(tmem + lane_base + (uint32_t)(buf * C::ACC_COLS + pk * NPAD + 16 * cb), pv[pk]);
          tmem_wait_ld();
#pragma unroll
          for (int k2 = 0; k2 < 16; ++k2) {
            float w = __uint_as_float(pv[0][k2]);
#pragma unroll
            for (int pk = 1; pk < C::NPK; ++pk) w += __uint_as_float(pv[pk][k2]);
            w *= rs[16 * cb + k2];
            acc[0] = fmaf(gv[k2].x, w, acc[0]);
            acc[1] = fmaf(gv[k2].y, w, acc[1]);
            acc[2] = fmaf(gv[k2].z, w, acc[2]);
            acc[3] = fmaf(gv[k2].w, w, acc[3]);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&ax.accempty[buf]));
        if (ch == 1) ax.comb[tile & 1][quarter][lane] = make_float4(acc[0], acc[1], acc[2], acc[3]);
        named_bar(1 + quarter, 64);
        if (ch == 0 && valid) {
          const float4 o2 = ax.comb[tile & 1][quarter][lane];
          float *o = gD + ((size_t)k * NQ + q) * 16 + b;
          o[0] = (acc[0] + o2.x) * down;
          o[4] = (acc[1] + o2.y) * down;
          o[8] = (acc[2] + o2.z) * down;
          o[12] = (acc[3] + o2.w) * down;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  // an aborted block marks its elements with NaN, which the chain carries
  // into their gradients
  if (*abort_flag) {
    const float nan = __int_as_float(0x7fc00000);
    for (int64_t k = kfirst; k < count; k += kstep)
      for (int t = tid; t < NQ * 16; t += blockDim.x) gD[(size_t)k * NQ * 16 + t] = nan;
    const uint64_t t0 = global_ns();  // in-flight bulk copies land within microseconds
    while (global_ns() - t0 < 200000ull) {
    }
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS) : "memory");
  }
}

// Adjoint epilogue table: out[q][i] = (G[q][0][i], .., G[q][3][i]) in FP32,
// zero for i >= nsh (i < npad).
__global__ void adj_table_kernel(const double *G, int nsh, int nq, int npad, float4 *out) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nq * npad; idx += gridDim.x * blockDim.x) {
    const int q = idx / npad, i = idx - q * npad;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (i < nsh)
      for (int a = 0; a < 4; ++a) v[a] = (float)G[(size_t)(4 * q + a) * nsh + i];
    out[idx] = make_float4(v[0], v[1], v[2], v[3]);
  }
}

// Adjoint A image: x = G[q][b][j] 2^tau at row (q, b) = 128 m + r, K value
// j = 32 kc + t, split into fp16 hi + lo at its swizzled position.
__global__ void adj_image_kernel(const double *G, int nsh, int nq, int nmt, int nkc, double scale,
                                 unsigned char *img) {
  const int64_t total = (int64_t)nmt * nkc * 128 * 32;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(idx % 32);
    const int r = (int)((idx / 32) % 128);
    const int kc = (int)((idx / (32 * 128)) % nkc);
    const int m = (int)(idx / (32 * 128 * (int64_t)nkc));
    const int qb = 128 * m + r, q = qb >> 2, b = qb & 3, j = 32 * kc + t;
    const double x = (q < nq && j < nsh) ? G[(size_t)(4 * q + b) * nsh + j] * scale : 0.0;
    const uint32_t byte = sw_off<64>(r, (2 * t) >> 4) + ((2 * t) & 15);
    unsigned char *base = img + (size_t)(m * nkc + kc) * 2 * (128 * 64);
    const __half h = __double2half(x);
    const __half l = __double2half(x - (double)__half2float(h));
    *reinterpret_cast<__half *>(base + byte) = h;
    *reinterpret_cast<__half *>(base + 128 * 64 + byte) = l;
  }
}

// ---------------------------------------------------------------------------
// B operand image: G * 2^tau split into fp16 hi/lo, K-major swizzled rows
// ---------------------------------------------------------------------------
__global__ void gmax_kernel(const double *G, int n, unsigned long long *out) {
  double m = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) m = fmax(m, fabs(G[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// B image of a split kind: x = G 2^tau (FP64) as hi + lo, fp16 (KD = 0) or
// TF32 (KD = 1, tau = 0), at the K-major swizzled position of K value k
// (point q = chunk * PPC + k / 4, component k % 4) in row n.
template <int KD>
__global__ void image_kernel(const double *G, int nsh, int nq, int npad, int nchunk, int rowb, double scale,
                             unsigned char *img) {
  constexpr int EB = KD ? 4 : 2;
  const int kch = rowb / EB, ppc = kch / 4;
  const int64_t total = (int64_t)nchunk * npad * kch;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(idx % kch);
    const int n = (int)((idx / kch) % npad);
    const int c = (int)(idx / (kch * (int64_t)npad));
    const int q = c * ppc + k / 4, b = k % 4;
    const double x = (q < nq && n < nsh) ? G[(size_t)(4 * q + b) * nsh + n] * scale : 0.0;
    // 16-byte chunk k * EB / 16 of the row, byte (k * EB) % 16 in it
    const uint32_t byte = (rowb == 128 ? sw_off<128>(n, (k * EB) >> 4) : sw_off<64>(n, (k * EB) >> 4)) + ((k * EB) & 15);
    unsigned char *hi = img + (size_t)(c * 2 + 0) * npad * rowb + byte;
    unsigned char *lo = img + (size_t)(c * 2 + 1) * npad * rowb + byte;
    if constexpr (KD == 0) {
      const __half h = __double2half(x);
      const __half l = __double2half(x - (double)__half2float(h));
      *reinterpret_cast<__half *>(hi) = h;
      *reinterpret_cast<__half *>(lo) = l;
    } else {
      const uint32_t h = tf32_rna((float)x);
      const uint32_t l = tf32_rna((float)(x - (double)__uint_as_float(h)));
      *reinterpret_cast<uint32_t *>(hi) = h;
      *reinterpret_cast<uint32_t *>(lo) = l;
    }
  }
}

__global__ void pair_table_kernel(const double *G, int nsh, int nq, int gst, int nchunk, int pp, float *out) {
  const int64_t total = (int64_t)nchunk * 2 * pp * gst * 4;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int m = (int)(idx % 4);
    const int i = (int)((idx / 4) % gst);
    const int64_t rest = idx / (4 * (int64_t)gst);
    const int pr = (int)(rest % pp), h = (int)((rest / pp) % 2), c = (int)(rest / (2 * pp));
    const int b = 2 * h + (m >> 1), q = c * 2 * pp + 2 * pr + (m & 1);
    out[idx] = q < nq && i < nsh ? (float)G[(size_t)(4 * q + b) * nsh + i] : 0.f;
  }
}

template <int P, int V, int KD>
fei_status launch_tc(const fei_reference *ref, const FwdArgs &a, int64_t grid_work, cudaStream_t s) {
  using C = TcCfg<P, V, KD>;
  static_assert(sizeof(TcAux<P, V, KD>) + C::DYN_SMEM <= 232448, "shared memory of one block (227 KB)");
  const TcImage *im = ref->tc;
  if (!im) return set_error(FEI_ERR_UNSUPPORTED, "no tensor-core image for degree %d", P);
  FEI_CUDA_TRY(cudaFuncSetAttribute(tc_forward_kernel<P, V, KD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    C::DYN_SMEM),
               "cudaFuncSetAttribute(tc_forward)");
  int dev, sms;
  FEI_CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
  FEI_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");
  const int64_t tiles = (grid_work * C::NSH + 127) / 128;
  int64_t blocks = tiles < sms ? tiles : sms;
  if (blocks < 1) blocks = 1;
  tc_forward_kernel<P, V, KD><<<(unsigned)blocks, C::NTHREADS, C::DYN_SMEM, s>>>(
      a, im->k[KD].img, reinterpret_cast<const float4 *>(im->k[KD].gp), KD ? 0 : im->tau);
  FEI_CUDA_TRY(cudaGetLastError(), "tc_forward_kernel launch");
  return FEI_OK;
}

template <int P>
fei_status launch_ta(const fei_reference *ref, const float *gA, const int64_t *A_off, int64_t e0, int64_t count,
                     float *gD, cudaStream_t s) {
  using C = TaCfg<P>;
  static_assert(sizeof(TaAux<P>) + C::DYN_SMEM <= 232448, "shared memory of one block (227 KB)");
  const TcImage *im = ref->tc;
  if (!im || !im->aimg || !im->gq4p)
    return set_error(FEI_ERR_UNSUPPORTED, "no tensor-core adjoint image for degree %d", P);
  FEI_CUDA_TRY(cudaFuncSetAttribute(tc_adjoint_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::DYN_SMEM),
               "cudaFuncSetAttribute(tc_adjoint)");
  int dev, sms;
  FEI_CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
  FEI_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");
  const int64_t blocks = count < sms ? count : sms;
  tc_adjoint_kernel<P><<<(unsigned)blocks, C::NTHREADS, C::DYN_SMEM, s>>>(
      gA, A_off, e0, count, im->aimg, im->gq4p, im->tau, gD);
  FEI_CUDA_TRY(cudaGetLastError(), "tc_adjoint_kernel launch");
  return FEI_OK;
}

template <int P, int KD>
void tc_dims(int &npad, int &nchunk, int &rowb, int &gst, int &pp) {
  npad = TcCfg<P, 0, KD>::NPAD;
  nchunk = TcCfg<P, 0, KD>::NCHUNK;
  rowb = TcCfg<P, 0, KD>::ROWB;
  gst = TcCfg<P, 0, KD>::GST;
  pp = TcCfg<P, 0, KD>::PP;
}

void ta_dims_of(int p, int &nmt, int &nkc) {
  switch (p) {
    case 3: nmt = TaCfg<3>::NMT, nkc = TaCfg<3>::NKC; break;
    case 4: nmt = TaCfg<4>::NMT, nkc = TaCfg<4>::NKC; break;
    default: nmt = TaCfg<5>::NMT, nkc = TaCfg<5>::NKC; break;
  }
}

template <int KD>
void tc_dims_of(int p, int &npad, int &nchunk, int &rowb, int &gst, int &pp) {
  switch (p) {
    case 3: tc_dims<3, KD>(npad, nchunk, rowb, gst, pp); break;
    case 4: tc_dims<4, KD>(npad, nchunk, rowb, gst, pp); break;
    case 5: tc_dims<5, KD>(npad, nchunk, rowb, gst, pp); break;
    case 6: tc_dims<6, KD>(npad, nchunk, rowb, gst, pp); break;
    default: tc_dims<7, KD>(npad, nchunk, rowb, gst, pp); break;
  }
}

}  // namespace

fei_status build_tc_image(fei_reference *ref) {
  ref->tc = nullptr;
  if (ref->p < 3) return FEI_OK;
  TcImage *im = new TcImage();
  memset(im, 0, sizeof(*im));
  unsigned long long *dmax = nullptr;
  cudaError_t e = cudaMalloc(&dmax, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(dmax, 0, sizeof(unsigned long long));
  if (e == cudaSuccess) {
    const int n = 4 * ref->nq * ref->nsh;
    gmax_kernel<<<64, 256>>>(ref->G64, n, dmax);
    e = cudaGetLastError();
  }
  unsigned long long bits = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&bits, dmax, sizeof(bits), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) {
    double gmax;
    memcpy(&gmax, &bits, sizeof(gmax));
    int ex = 0;
    frexp(gmax, &ex);  // gmax <= 2^ex
    im->tau = 14 - ex;
  }
  for (int kd = 0; kd < 2 && e == cudaSuccess; ++kd) {
    int npad = 0, nchunk = 0, rowb = 0, gst = 0, pp = 0;
    if (kd == 0) tc_dims_of<0>(ref->p, npad, nchunk, rowb, gst, pp);
    else tc_dims_of<1>(ref->p, npad, nchunk, rowb, gst, pp);
    im->npad = npad;
    im->rowb = rowb;
    TcOperands &o = im->k[kd];
    o.nchunk = nchunk;
    const size_t ibytes = (size_t)nchunk * 2 * npad * rowb;
    const size_t gfloats = (size_t)nchunk * 2 * pp * gst * 4;
    e = cudaMalloc(&o.img, ibytes);
    if (e == cudaSuccess) e = cudaMalloc(&o.gp, sizeof(float) * gfloats);
    if (e == cudaSuccess) {
      if (kd == 0)
        image_kernel<0><<<256, 256>>>(ref->G64, ref->nsh, ref->nq, npad, nchunk, rowb, ldexp(1.0, im->tau), o.img);
      else
        image_kernel<1><<<256, 256>>>(ref->G64, ref->nsh, ref->nq, npad, nchunk, rowb, 1.0, o.img);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      pair_table_kernel<<<256, 256>>>(ref->G64, ref->nsh, ref->nq, gst, nchunk, pp, o.gp);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess && ref->p <= 5) {
    int nmt = 0, nkc = 0;
    ta_dims_of(ref->p, nmt, nkc);
    const int npad = (ref->nsh + 15) / 16 * 16;
    e = cudaMalloc(&im->aimg, (size_t)nmt * nkc * 2 * 128 * 64);
    if (e == cudaSuccess) e = cudaMalloc(&im->gq4p, sizeof(float4) * (size_t)ref->nq * npad);
    if (e == cudaSuccess) {
      adj_image_kernel<<<256, 256>>>(ref->G64, ref->nsh, ref->nq, nmt, nkc, ldexp(1.0, im->tau), im->aimg);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      adj_table_kernel<<<256, 256>>>(ref->G64, ref->nsh, ref->nq, npad, im->gq4p);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (dmax) cudaFree(dmax);
  if (e != cudaSuccess) {
    for (int kd = 0; kd < 2; ++kd) {
      if (im->k[kd].img) cudaFree(im->k[kd].img);
      if (im->k[kd].gp) cudaFree(im->k[kd].gp);
    }
    if (im->aimg) cudaFree(im->aimg);
    if (im->gq4p) cudaFree(im->gq4p);
    delete im;
    return cuda_error(e, "tensor-core image");
  }
  ref->tc = im;
  return FEI_OK;
}

void free_tc_image(fei_reference *ref) {
  if (ref->tc) {
    for (int kd = 0; kd < 2; ++kd) {
      cudaFree(ref->tc->k[kd].img);
      cudaFree(ref->tc->k[kd].gp);
    }
    if (ref->tc->aimg) cudaFree(ref->tc->aimg);
    if (ref->tc->gq4p) cudaFree(ref->tc->gq4p);
    delete ref->tc;
    ref->tc = nullptr;
  }
}

bool tc_adjoint_ready(const fei_reference *ref) {
  return ref->p >= 3 && ref->p <= 5 && ref->tc && ref->tc->aimg && ref->tc->gq4p;
}

fei_status launch_tc_adjoint(int p, const fei_reference *ref, const float *gA, const int64_t *A_off, int64_t e0,
                             int64_t count, float *gD, cudaStream_t s) {
  if (count <= 0) return FEI_OK;
  switch (p) {
    case 3: return launch_ta<3>(ref, gA, A_off, e0, count, gD, s);
    case 4: return launch_ta<4>(ref, gA, A_off, e0, count, gD, s);
    case 5: return launch_ta<5>(ref, gA, A_off, e0, count, gD, s);
  }
  return set_error(FEI_ERR_UNSUPPORTED, "tensor-core adjoint for degree %d", p);
}

int tc_variant_count(int p, fei_precision prec) {
  if (prec == FEI_TC_3XTF32) return p >= 3 && p <= 7 ? 1 : 0;
  return p >= 3 && p <= 5 ? 2 : p >= 6 && p <= 7 ? 1 : 0;
}

fei_status launch_tc_forward(int p, const fei_reference *ref, const FwdArgs &a, int64_t grid_work, cudaStream_t s,
                             int variant, fei_precision prec) {
  if (grid_work <= 0) return FEI_OK;
  if (variant < 0 || variant >= tc_variant_count(p, prec))
    return set_error(FEI_ERR_UNSUPPORTED, "tensor-core variant %d for degree %d", variant, p);
  if (prec == FEI_TC_3XTF32) {
    switch (p) {
      case 3: return launch_tc<3, 0, 1>(ref, a, grid_work, s);
      case 4: return launch_tc<4, 0, 1>(ref, a, grid_work, s);
      case 5: return launch_tc<5, 0, 1>(ref, a, grid_work, s);
      case 6: return launch_tc<6, 0, 1>(ref, a, grid_work, s);
      case 7: return launch_tc<7, 0, 1>(ref, a, grid_work, s);
    }
    return set_error(FEI_ERR_UNSUPPORTED, "tensor-core path for degree %d", p);
  }
  switch (p * 2 + variant) {
    case 6: return launch_tc<3, 0, 0>(ref, a, grid_work, s);
    case 7: return launch_tc<3, 1, 0>(ref, a, grid_work, s);
    case 8: return launch_tc<4, 0, 0>(ref, a, grid_work, s);
    case 9: return launch_tc<4, 1, 0>(ref, a, grid_work, s);
    case 10: return launch_tc<5, 0, 0>(ref, a, grid_work, s);
    case 11: return launch_tc<5, 1, 0>(ref, a, grid_work, s);
    case 12: return launch_tc<6, 0, 0>(ref, a, grid_work, s);
    case 14: return launch_tc<7, 0, 0>(ref, a, grid_work, s);
  }
  return set_error(FEI_ERR_UNSUPPORTED, "tensor-core path for degree %d", p);
}

}  // namespace fei

extern "C" fei_status fei_debug_set_wait_limit(uint64_t ns) {
  const uint64_t v = ns ? ns : fei::kWaitLimitNs;
  FEI_CUDA_TRY(cudaMemcpyToSymbol(fei::g_wait_limit_ns, &v, sizeof(v)), "cudaMemcpyToSymbol(wait limit)");
  return FEI_OK;
}
