// Tensor-core fused operator for non-tensor elements (the dense element operator of the paper's
// Section 3, MAGMA backend: y^e = G^T D G u^e), written for the 5th-generation tensor cores of
// sm_103a with tcgen05 instructions in inline PTX.
//
// One thread block processes a tile of 128 elements; element m of the tile is row m of every
// matrix product, i.e. lane m of tensor memory (TMEM):
//   GEMM1  S_d = U G_d^T          [128 x 16] per direction d and chunk of 16 quadrature points
//                                  (A = U [128 x P] element inputs, B = the chunk's rows of G_d)
//   pointwise (CUDA cores): thread of element m reads its row of S from TMEM, applies the 3x3
//          (or 1x1) quadrature operator with the element's quadrature data, writes V
//   GEMM2  Y += V_d G_d            [128 x P] accumulated in TMEM over directions and chunks
// and the block finally stores Y as element vectors [P][E] (the transposed restriction that
// follows is the same deterministic kernel as for the other algorithms).
//
// Precision: FP32 operands with FP32-level accuracy from TF32 tensor cores by the three-product
// split a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi with a_hi = tf32(a), a_lo = a - a_hi (the
// "3xTF32" scheme; the dropped a_lo b_lo term is ~2^-22 of a b), accumulated in FP32 in TMEM.
//
// Operands live in shared memory in the canonical no-swizzle K-major layout: 8-row x 16-byte core
// matrices stored contiguously (128 bytes), core matrices adjacent along K at 128 bytes (LBO),
// 8-row groups at K/4 * 128 bytes (SBO).  The basis matrices are constant: at setup they are
// split, padded and written in that layout chunk by chunk, so one bulk TMA copy per chunk
// (cp.async.bulk, completion on an mbarrier) brings a chunk's operands into shared memory,
// double-buffered so the next chunk streams in while the current one is computed.
// Every wait (bulk copy, MMA completion) is bounded; on expiry the kernel records
// CEED_ERR_TIMEOUT, waits (bounded) for its own operations in flight, frees TMEM and returns.
#include <algorithm>
#include <cstring>
#include <vector>

#include "convert.cuh"
#include "nontensor.h"

namespace ceedgb {
namespace {

constexpr int TC_M = 128;      // elements per tile (MMA M, TMEM lanes)
constexpr int TC_QC = 16;      // quadrature points per chunk (GEMM1 N, GEMM2 K)

__host__ __device__ constexpr int kpad(int P) { return (P + 7) / 8 * 8; }     // K of GEMM1: multiple of 8
__host__ __device__ constexpr int npad(int P) { return (P + 15) / 16 * 16; }  // N of GEMM2: multiple of 16

// Offset (in 4-byte words) of element (r, k) in the canonical K-major no-swizzle layout of a
// matrix with K columns (K a multiple of 4).
__host__ __device__ constexpr int canon(int r, int k, int K) {
  return ((r >> 3) * (K >> 2) + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3);
}

// Words of one chunk of split tables for D directions: GT_hi, GT_lo [D][16 x KP], G_hi, G_lo [D][NP x 16].
__host__ __device__ constexpr int gt_words(int D, int KP) { return 2 * D * TC_QC * KP; }   // GEMM1 operand, hi + lo
__host__ __device__ constexpr int g_words(int D, int NP) { return 2 * D * NP * TC_QC; }    // GEMM2 operand, hi + lo
__host__ __device__ constexpr int chunk_words(int D, int KP, int NP) { return gt_words(D, KP) + g_words(D, NP); }

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of tcgen05.mma: start address, leading (K-direction core matrix)
// byte offset, stride (8-row group) byte offset, each >> 4; bits 46-48 = 0b001; no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor for kind::tf32: D F32 (bits 4-5 = 1), A and B TF32 (bits 7-9, 10-12 = 2),
// both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
template <int M, int N>
struct IDescTF32 {
  static_assert(M == 128, "one CTA, M = 128");
  static_assert(N % 16 == 0 && N >= 16 && N <= 256, "M = 128 needs N a multiple of 16 in [16, 256]");
  static constexpr uint32_t value = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
                                    ((uint32_t)(M >> 4) << 24);
};

// The issuing warps run their loops with all 32 lanes (so descriptors stay warp-uniform); only the
// lane with `leader` set issues the tensor-core instruction, the commit or the copy.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum,
                                         uint32_t leader) {
  asm volatile(
      "{\n .reg .pred p, l;\n setp.ne.b32 p, %4, 0;\n setp.ne.b32 l, %5, 0;\n"
      " @l tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum), "r"(leader)
      : "memory");
}

// Same with the A operand in tensor memory (row m of A in lane m, one TF32 value per column).
__device__ __forceinline__ void mma_tf32_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                            uint32_t accum, uint32_t leader) {
  asm volatile(
      "{\n .reg .pred p, l;\n setp.ne.b32 p, %4, 0;\n setp.ne.b32 l, %5, 0;\n"
      " @l tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(accum), "r"(leader)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar, uint32_t leader) {
  asm volatile(
      "{\n .reg .pred l;\n setp.ne.b32 l, %1, 0;\n"
      " @l tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n" ::"r"(su32(bar)),
      "r"(leader)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 4 consecutive 32-bit TMEM columns of this thread's lane (warp w reads lanes 32 (w % 4) ...),
// waiting for the load in the same statement so no use of the registers can precede it.
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float (&v)[4]) {
  uint32_t r0, r1, r2, r3;
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
      : "r"(taddr)
      : "memory");
  v[0] = __uint_as_float(r0);
  v[1] = __uint_as_float(r1);
  v[2] = __uint_as_float(r2);
  v[3] = __uint_as_float(r3);
}

// 4 consecutive 32-bit TMEM columns of this thread's lane from registers; waits for the store.
__device__ __forceinline__ void tmem_st4(uint32_t taddr, const float (&v)[4]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};\n"
      "tcgen05.wait::st.sync.aligned;\n" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3]))
      : "memory");
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   su32(dst)),
               "l"(src), "r"(bytes), "r"(su32(bar))
               : "memory");
}

// Bounded wait for phase `parity` of an mbarrier.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
  const uint32_t a = su32(bar);
  for (int it = 0; it < (1 << 22); ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// TF32 split: hi = x rounded to TF32 (10-bit mantissa), lo = x - hi (exact in FP32).
__device__ __forceinline__ void split_tf32(float x, float &hi, float &lo) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  hi = __uint_as_float(h);
  lo = x - hi;
}

__device__ __forceinline__ void st_shared4(float *p, float a, float b, float c, float d) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(su32(p)), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

// mbarrier slots
enum : int { B_T1 = 0, B_T2 = 2, B_SFULL = 4, B_SFREE = 6, B_VFULL = 8, B_VFREE = 10, B_UFULL = 12, B_YFULL = 13,
             B_YFREE = 15, B_T2FREE = 17, B_DRAIN1 = 19, B_DRAIN2 = 20, B_QFULL = 21 };
constexpr int TC_NBAR = 24;
constexpr int TC_CW = 16;                       // compute warps (0-15); warps 16, 17 issue the MMAs
constexpr int TC_COMPUTE = 32 * TC_CW;
constexpr int TC_BLOCK = TC_COMPUTE + 64;
constexpr int TC_GROUPS = TC_CW / 4;            // warps per TMEM lane quadrant
constexpr int TC_PPT = TC_QC / TC_GROUPS;       // points of a chunk per compute thread
static_assert(TC_PPT == 4, "one float4 of points per thread and direction");
// TMEM columns: S buffer s at 64 s (16 D used); V buffer v at 128 + 96 v (hi: 16 d + point, lo: 48 +
// 16 d + point); Y buffer y at 320 + 96 y (NP <= 96 used).
constexpr uint32_t TC_TMEM_ALLOC = 512;
constexpr uint32_t TC_SCOL = 64;
constexpr uint32_t TC_VCOL0 = 128, TC_VSTRIDE = 96, TC_VLO = 48;
constexpr uint32_t TC_YCOL0 = 320, TC_YSTRIDE = 96;

// Shared-memory map of one block.  U: the tile's element inputs (hi, lo); T1[TBUF], T2[TBUF]: the
// GEMM1 and GEMM2 operands of a table chunk; QS: the tile's quadrature data of the next chunk
// ([value][point][element], when QPRE); then the mbarriers, the TMEM address and an abort flag.
// (The pointwise results V, the A operand of GEMM2, live in tensor memory.)
template <int D, int KP, int NP, int TBUF, int QPRE>
struct TcLayout {
  static constexpr int U_WORDS = TC_M * KP;                // per hi/lo
  static constexpr int T1_WORDS = gt_words(D, KP);         // one GEMM1 table buffer
  static constexpr int T2_WORDS = g_words(D, NP);          // one GEMM2 table buffer
  static constexpr int TB_WORDS = T1_WORDS + T2_WORDS;     // one chunk of the global table image
  static constexpr int QS_WORDS = QPRE * (D == 3 ? 6 : 1) * TC_QC * TC_M;   // [value][point][element]
  static constexpr size_t U_HI = 0;
  static constexpr size_t U_LO = U_HI + 4 * (size_t)U_WORDS;
  static constexpr size_t T1 = U_LO + 4 * (size_t)U_WORDS;
  static constexpr size_t T2 = T1 + 4 * (size_t)T1_WORDS * TBUF;
  static constexpr size_t QS = T2 + 4 * (size_t)T2_WORDS * TBUF;
  static constexpr size_t BARS = QS + 4 * (size_t)QS_WORDS;
  static constexpr size_t BYTES = BARS + TC_NBAR * 8 + 16;
  static_assert(BYTES <= 227 * 1024, "shared memory");
};

__device__ __forceinline__ void mbar_init_n(uint64_t *bar, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait that also gives up when another thread of the block has raised the abort flag.
__device__ __forceinline__ bool mbar_wait_abortable(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
  for (int it = 0; it < (1 << 22); ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 63) == 63 && *abort_flag) return false;
  }
  *abort_flag = 1;
  return false;
}

// 16-byte asynchronous copy global -> shared; src_bytes = 0 writes zeros without reading.
__device__ __forceinline__ void cp_async16(float *dst, const float *src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(su32(dst)), "l"(src), "r"(src_bytes) : "memory");
}
// The mbarrier receives this thread's arrival once all its earlier cp.async copies have landed.
__device__ __forceinline__ void cp_async_arrive(uint64_t *bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(su32(bar)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Barrier among the compute warps only (id 1) that also ANDs a flag over them: every compute
// thread executes the same sequence of these, so the block leaves its loops together.
__device__ __forceinline__ bool compute_all(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(TC_COMPUTE)
      : "memory");
  return r != 0;
}

// Bounded wait by a whole warp, with a warp-uniform result.
__device__ __forceinline__ bool wait_warp(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
  return __all_sync(0xffffffffu, mbar_wait_abortable(bar, parity, abort_flag));
}

// The tile's element inputs, split into TF32 hi/lo, written to the canonical layout (row m,
// columns 4 k4 .. 4 k4 + 3 for this thread's share k4 = grp, grp + 4, ... of the column groups).
// Loads go out in rounds of up to two column groups (restriction entries first, then the L-vector
// values) so their latencies overlap; the FP64 -> FP32 conversion uses integer instructions only.
template <int KP>
__device__ __forceinline__ void gather_tile(int64_t E, int P, int64_t e, bool valid, int grp, int m, int masked,
                                            const uint32_t *__restrict__ rmap, const double *__restrict__ x,
                                            float *u_hi, float *u_lo) {
  constexpr int NG = KP / 4;   // column groups
  constexpr int R = 2;         // groups per round
#pragma unroll
  for (int r0 = 0; r0 < (NG + TC_GROUPS - 1) / TC_GROUPS; r0 += R) {
    uint32_t mm[R][4];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int k4 = grp + TC_GROUPS * (r0 + r), n = 4 * k4 + j;
        mm[r][j] = (valid && k4 < NG && n < P) ? __ldg(rmap + (int64_t)n * E + e) : 0xFFFFFFFFu;
      }
    double v[R][4];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t q = mm[r][j];
        v[r][j] = (q == 0xFFFFFFFFu || (masked && (q & FLAG_DIR))) ? 0.0 : __ldg(x + (q & DOF_MASK));
      }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int k4 = grp + TC_GROUPS * (r0 + r);
      if (k4 < NG) {
        float h4[4], l4[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) split_tf32(d2f_fast(v[r][j]), h4[j], l4[j]);
        const int o = canon(m, 4 * k4, KP);
        st_shared4(u_hi + o, h4[0], h4[1], h4[2], h4[3]);
        st_shared4(u_lo + o, l4[0], l4[1], l4[2], l4[3]);
      }
    }
  }
}

// Quadrature data of one thread's TC_PPT points of chunk c of a tile, into registers (zero outside
// the rule; rows are padded to whole tiles, so every element of a tile can be read).
template <int D>
__device__ __forceinline__ void load_qdata(const float *__restrict__ qd, int64_t Es, int Q, int64_t e, int c, int grp,
                                           float (&qv)[TC_PPT][D == 3 ? 6 : 1]) {
  const int64_t cs = (int64_t)Q * Es;
  const int q0 = c * TC_QC + TC_PPT * grp;
  const float *base = qd + (int64_t)q0 * Es + e;
#pragma unroll
  for (int j = 0; j < TC_PPT; ++j) {
    const bool in = q0 + j < Q;
#pragma unroll
    for (int k = 0; k < (D == 3 ? 6 : 1); ++k) qv[j][k] = in ? __ldg(base + k * cs + (int64_t)j * Es) : 0.f;
  }
}
// The tile's quadrature data of chunk c into the block's buffer qbuf [value k][point qq][element]
// with 16-byte copies: compute warp w copies rows (k, qq) = w, w + 16, ... (128 consecutive
// elements each, lane l elements 4 l .. 4 l + 3); points beyond the rule are zero-filled.  The
// thread's arrival on q_full follows the completion of its copies.
template <int D>
__device__ __forceinline__ void tile_qdata_async(const float *__restrict__ qd, int64_t Es, int Q, int64_t tile, int c,
                                                 int warp, int lane, float *qbuf, uint64_t *q_full) {
  constexpr int NQ = D == 3 ? 6 : 1;
#pragma unroll
  for (int r = warp; r < NQ * TC_QC; r += TC_CW) {
    const int k = r / TC_QC, qq = r - k * TC_QC, q = c * TC_QC + qq;
    const bool in = q < Q;
    const float *src = qd + ((int64_t)k * Q + (in ? q : 0)) * Es + tile * TC_M + 4 * lane;
    cp_async16(qbuf + r * TC_M + 4 * lane, src, in ? 16u : 0u);
  }
  cp_async_arrive(q_full);
}

// The fused kernel, persistent (block b takes tiles b, b + gridDim.x, ...) and warp-specialized.
//   warp 16: streams the GEMM1 operand of each table chunk in (bulk copies), issues GEMM1
//   warp 17: the same for GEMM2
// (the issuing warps run with all lanes; one lane issues each tensor-core instruction and copy)
//   warps 0-15: gather inputs, apply the pointwise operator, write the element vectors
// They hand buffers to each other through mbarriers (the tensor core signals completion through
// tcgen05.commit).  S (TMEM) and Y (TMEM) are double-buffered, V and the tables when shared memory
// allows, so the tensor core works on one chunk while the CUDA cores process another.  Warp w < 16
// serves TMEM lane quadrant w % 4 (elements 32 (w % 4) ... of the tile) and group grp = w / 4:
// points 4 grp .. 4 grp + 3 of each chunk, every fourth input column group and a quarter of the
// output nodes.  With QPRE, every compute thread copies its quadrature data for the next chunk into
// its own shared-memory slots with cp.async while it works on the current one.
template <int D, int KP, int NP, int TBUF, int QPRE>
__global__ void __launch_bounds__(TC_BLOCK, 1)
    nt_tc_kernel(int64_t E, int64_t Es, int P, int Q, int nch, const uint32_t *__restrict__ rmap,
                 const double *__restrict__ x, const float *__restrict__ tabs, const float *__restrict__ qd,
                 float *__restrict__ Ye, int masked, int *err) {
  using L = TcLayout<D, KP, NP, TBUF, QPRE>;
  constexpr int NQ = D == 3 ? 6 : 1;
  static_assert(NP <= (int)TC_YSTRIDE && 16 * D <= (int)TC_VLO, "tensor memory map");
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  float *u_hi = reinterpret_cast<float *>(tc_smem + L::U_HI);
  float *u_lo = reinterpret_cast<float *>(tc_smem + L::U_LO);
  float *t1 = reinterpret_cast<float *>(tc_smem + L::T1);
  float *t2 = reinterpret_cast<float *>(tc_smem + L::T2);
  float *qslots = reinterpret_cast<float *>(tc_smem + L::QS);
  uint64_t *bar = reinterpret_cast<uint64_t *>(tc_smem + L::BARS);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tc_smem + L::BARS + TC_NBAR * 8);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tc_smem + L::BARS + TC_NBAR * 8 + 4);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t ntiles = (E + TC_M - 1) / TC_M;
  const int64_t my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t G = my_tiles * nch;  // chunks this block processes
  constexpr uint32_t T1_BYTES = 4u * (uint32_t)L::T1_WORDS, T2_BYTES = 4u * (uint32_t)L::T2_WORDS;

  if (warp == TC_CW) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(TC_TMEM_ALLOC)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < TC_NBAR; ++i) {
      const bool by_threads = i == B_SFREE || i == B_SFREE + 1 || i == B_VFULL || i == B_VFULL + 1 || i == B_UFULL ||
                              i == B_YFREE || i == B_YFREE + 1 || i == B_QFULL;
      mbar_init_n(&bar[i], by_threads ? TC_COMPUTE : 1);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;

  if (warp == TC_CW) {
    // ------------------------------------------------------------------ GEMM1 tables + GEMM1 issuer
    {
      const uint32_t leader = lane == 0 ? 1u : 0u;
      constexpr uint32_t ID1 = IDescTF32<TC_M, 16 * D>::value;
      constexpr uint32_t SBO1 = (KP / 4) * 128;
      const uint64_t du_hi = sdesc(su32(u_hi), 128, SBO1), du_lo = sdesc(su32(u_lo), 128, SBO1);
      uint32_t filled[2] = {0u, 0u}, consumed[2] = {0u, 0u};   // T1 fills per buffer
      bool issued_any = false;
      for (int f = 0; f < TBUF && f < G; ++f) {
        if (leader) bulk_load(t1 + f * L::T1_WORDS, tabs + (size_t)(f % nch) * L::TB_WORDS, T1_BYTES, &bar[B_T1 + f]);
        filled[f]++;
      }
      int64_t g = 0;
      for (int64_t t = 0; t < my_tiles && ok; ++t) {
        for (int c = 0; c < nch && ok; ++c, ++g) {
          const int tbi = (int)(g % TBUF), sb = (int)(g & 1);
          const uint32_t sk = (uint32_t)(g >> 1);
          if (TBUF == 1 && g >= 1) {
            // single buffer: refill it with chunk g once GEMM1 of chunk g - 1 has completed
            if (!wait_warp(&bar[B_SFULL + (int)((g - 1) & 1)], (uint32_t)(((g - 1) >> 1) & 1), abort_flag)) {
              ok = false;
              break;
            }
            if (leader) bulk_load(t1, tabs + (size_t)(g % nch) * L::TB_WORDS, T1_BYTES, &bar[B_T1]);
            filled[0]++;
          }
          if (!wait_warp(&bar[B_T1 + tbi], consumed[tbi] & 1u, abort_flag)) { ok = false; break; }
          consumed[tbi]++;
          if (c == 0 && !wait_warp(&bar[B_UFULL], (uint32_t)(t & 1), abort_flag)) { ok = false; break; }
          if (g >= 2 && !wait_warp(&bar[B_SFREE + sb], (sk - 1) & 1u, abort_flag)) { ok = false; break; }
          tc_fence_after();
          // GEMM1: S [128 x 16 D] = U [128 x KP] * GT^T (all directions in one N = 16 D product)
          const uint32_t tbs = su32(t1 + tbi * L::T1_WORDS);
          const uint64_t dg_hi = sdesc(tbs, 128, SBO1), dg_lo = sdesc(tbs + 4u * D * TC_QC * KP, 128, SBO1);
          const uint32_t dcol = tmem + TC_SCOL * sb;
#pragma unroll
          for (int ks = 0; ks < KP / 8; ++ks) {
            const uint64_t o = (uint64_t)(ks * 256) >> 4;
            mma_tf32(dcol, du_hi + o, dg_hi + o, ID1, ks > 0, leader);
            mma_tf32(dcol, du_hi + o, dg_lo + o, ID1, 1, leader);
            mma_tf32(dcol, du_lo + o, dg_hi + o, ID1, 1, leader);
          }
          mma_commit(&bar[B_SFULL + sb], leader);
          issued_any = true;
          if (TBUF == 2 && g >= 1 && g + 1 < G) {
            // the buffer of chunk g - 1 is free once its GEMM1 has completed: load chunk g + 1 into it
            if (!wait_warp(&bar[B_SFULL + (int)((g - 1) & 1)], (uint32_t)(((g - 1) >> 1) & 1), abort_flag)) {
              ok = false;
              break;
            }
            const int ob = (int)((g + 1) & 1);
            if (leader) bulk_load(t1 + ob * L::T1_WORDS, tabs + (size_t)((g + 1) % nch) * L::TB_WORDS, T1_BYTES, &bar[B_T1 + ob]);
            filled[ob]++;
          }
        }
      }
      if (!ok) {
        if (leader) {
          *abort_flag = 1;
          atomicExch(err, (int)CEED_ERR_TIMEOUT);
        }
        // let this thread's operations in flight finish before TMEM and shared memory are released
        if (issued_any) {
          mma_commit(&bar[B_DRAIN1], leader);
          mbar_wait_bounded(&bar[B_DRAIN1], 0u);
        }
        for (int bb = 0; bb < TBUF; ++bb)
          if (filled[bb] > consumed[bb]) mbar_wait_bounded(&bar[B_T1 + bb], consumed[bb] & 1u);
      }
    }
    __syncwarp();
  } else if (warp == TC_CW + 1) {
    // ------------------------------------------------------------------ GEMM2 tables + GEMM2 issuer
    {
      const uint32_t leader = lane == 0 ? 1u : 0u;
      constexpr uint32_t ID2 = IDescTF32<TC_M, NP>::value;
      uint32_t filled[2] = {0u, 0u}, consumed[2] = {0u, 0u};   // T2 fills per buffer
      bool issued_any = false;
      for (int f = 0; f < TBUF && f < G; ++f) {
        if (leader) bulk_load(t2 + f * L::T2_WORDS, tabs + (size_t)(f % nch) * L::TB_WORDS + L::T1_WORDS, T2_BYTES, &bar[B_T2 + f]);
        filled[f]++;
      }
      int64_t g = 0;
      for (int64_t t = 0; t < my_tiles && ok; ++t) {
        const int yb = (int)(t & 1);
        for (int c = 0; c < nch && ok; ++c, ++g) {
          const int tbi = (int)(g % TBUF), vb = (int)(g & 1);
          const uint32_t vk = (uint32_t)(g >> 1);
          if (TBUF == 1 && g >= 1) {
            // single buffer: refill it with chunk g once GEMM2 of chunk g - 1 has completed
            if (!wait_warp(&bar[B_T2FREE], (uint32_t)((g - 1) & 1), abort_flag)) { ok = false; break; }
            if (leader) bulk_load(t2, tabs + (size_t)(g % nch) * L::TB_WORDS + L::T1_WORDS, T2_BYTES, &bar[B_T2]);
            filled[0]++;
          }
          if (!wait_warp(&bar[B_VFULL + vb], vk & 1u, abort_flag)) { ok = false; break; }
          if (c == 0 && t >= 2 &&
              !wait_warp(&bar[B_YFREE + yb], (uint32_t)(((t >> 1) - 1) & 1), abort_flag)) {
            ok = false;
            break;
          }
          if (!wait_warp(&bar[B_T2 + tbi], consumed[tbi] & 1u, abort_flag)) { ok = false; break; }
          consumed[tbi]++;
          tc_fence_after();
          // GEMM2: Y [128 x NP] += V_d [128 x 16] * G_d [16 x NP], V_d read from tensor memory
          const uint32_t va = tmem + TC_VCOL0 + TC_VSTRIDE * vb;
          const uint32_t gs = su32(t2 + tbi * L::T2_WORDS);
          const uint64_t dG_hi = sdesc(gs, 128, 512), dG_lo = sdesc(gs + 4u * D * NP * TC_QC, 128, 512);
          const uint32_t ycol = tmem + TC_YCOL0 + TC_YSTRIDE * yb;
#pragma unroll
          for (int d = 0; d < D; ++d) {
#pragma unroll
            for (int ks = 0; ks < TC_QC / 8; ++ks) {
              const uint32_t ao = 16u * d + 8u * ks;
              const uint64_t ob = (uint64_t)(d * NP * TC_QC * 4 + ks * 256) >> 4;
              mma_tf32_ts(ycol, va + ao, dG_hi + ob, ID2, (c > 0 || d > 0 || ks > 0) ? 1u : 0u, leader);
              mma_tf32_ts(ycol, va + ao, dG_lo + ob, ID2, 1, leader);
              mma_tf32_ts(ycol, va + TC_VLO + ao, dG_hi + ob, ID2, 1, leader);
            }
          }
          mma_commit(&bar[B_VFREE + vb], leader);
          mma_commit(&bar[B_T2FREE + tbi], leader);
          if (c == nch - 1) mma_commit(&bar[B_YFULL + yb], leader);
          issued_any = true;
          if (TBUF == 2 && g >= 1 && g + 1 < G) {
            // the buffer of chunk g - 1 is free once its GEMM2 has completed: load chunk g + 1 into it
            const int ob = (int)((g + 1) & 1);
            if (!wait_warp(&bar[B_T2FREE + ob], (consumed[ob] - 1) & 1u, abort_flag)) { ok = false; break; }
            if (leader) bulk_load(t2 + ob * L::T2_WORDS, tabs + (size_t)((g + 1) % nch) * L::TB_WORDS + L::T1_WORDS, T2_BYTES,
                      &bar[B_T2 + ob]);
            filled[ob]++;
          }
        }
      }
      if (!ok) {
        if (leader) {
          *abort_flag = 1;
          atomicExch(err, (int)CEED_ERR_TIMEOUT);
        }
        if (issued_any) {
          mma_commit(&bar[B_DRAIN2], leader);
          mbar_wait_bounded(&bar[B_DRAIN2], 0u);
        }
        for (int bb = 0; bb < TBUF; ++bb)
          if (filled[bb] > consumed[bb]) mbar_wait_bounded(&bar[B_T2 + bb], consumed[bb] & 1u);
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------------ compute warps
    // Waits record failure in `ok` (made warp-uniform before the warp-collective TMEM loads) and
    // dependent work is skipped; loops are left only right after compute_all, so every compute
    // thread passes the same barriers.
    const int quad = warp & 3, grp = warp >> 2;
    const int m = quad * 32 + lane;
    const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
    if (my_tiles > 0) {
      const int64_t e0 = (int64_t)blockIdx.x * TC_M + m;
      if (QPRE) tile_qdata_async<D>(qd, Es, Q, blockIdx.x, 0, warp, lane, qslots, &bar[B_QFULL]);
      gather_tile<KP>(E, P, e0, e0 < E, grp, m, masked, rmap, x, u_hi, u_lo);
      fence_proxy_async();
      mbar_arrive(&bar[B_UFULL]);
    }
    int64_t g = 0;
    for (int64_t t = 0; t < my_tiles; ++t) {
      const int64_t tile = (int64_t)blockIdx.x + t * gridDim.x;
      const int64_t e = tile * TC_M + m;
      const bool valid = e < E;
      const int yb = (int)(t & 1);
      for (int c = 0; c < nch; ++c, ++g) {
        const int sb = (int)(g & 1), vb = (int)(g & 1);
        const uint32_t sk = (uint32_t)(g >> 1), vk = (uint32_t)(g >> 1);
        if (ok) ok = mbar_wait_abortable(&bar[B_SFULL + sb], sk & 1u, abort_flag);
        ok = __all_sync(0xffffffffu, ok);
        float s[D][TC_PPT];
        if (ok) {
          tc_fence_after();
#pragma unroll
          for (int d = 0; d < D; ++d) tmem_ld4(tmem + lane_base + TC_SCOL * sb + 16u * d + TC_PPT * grp, s[d]);
          tc_fence_before();
          mbar_arrive(&bar[B_SFREE + sb]);
        }
        float qv[TC_PPT][NQ];
        if (QPRE) {
          if (ok) ok = mbar_wait_abortable(&bar[B_QFULL], (uint32_t)(g & 1), abort_flag);   // all copies of chunk g
          if (ok) {
#pragma unroll
            for (int j = 0; j < TC_PPT; ++j)
#pragma unroll
              for (int k = 0; k < NQ; ++k) qv[j][k] = qslots[(k * TC_QC + TC_PPT * grp + j) * TC_M + m];
          }
        } else {
          load_qdata<D>(qd, Es, Q, e, c, grp, qv);
        }
        // every compute thread has read the buffer (and agrees whether to go on)
        if (!compute_all(ok)) {
          ok = false;
          break;
        }
        if (QPRE) {
          if (c + 1 < nch) tile_qdata_async<D>(qd, Es, Q, tile, c + 1, warp, lane, qslots, &bar[B_QFULL]);
          else if (t + 1 < my_tiles)
            tile_qdata_async<D>(qd, Es, Q, tile + gridDim.x, 0, warp, lane, qslots, &bar[B_QFULL]);
        }
#pragma unroll
        for (int j = 0; j < TC_PPT; ++j) {
          if (D == 3) {
            const float g0 = s[0][j], g1 = s[1][j], g2 = s[2][j];
            s[0][j] = qv[j][0] * g0 + qv[j][1] * g1 + qv[j][2] * g2;
            s[1][j] = qv[j][1] * g0 + qv[j][3] * g1 + qv[j][4] * g2;
            s[2][j] = qv[j][2] * g0 + qv[j][4] * g1 + qv[j][5] * g2;
          } else {
            s[0][j] *= qv[j][0];
          }
        }
        // V buffer vb is free once the product of chunk g - 2 that read it has completed
        if (g >= 2 && ok) ok = mbar_wait_abortable(&bar[B_VFREE + vb], (vk - 1) & 1u, abort_flag);
        ok = __all_sync(0xffffffffu, ok);
        if (ok) {
          tc_fence_after();
          const uint32_t vcol = tmem + lane_base + TC_VCOL0 + TC_VSTRIDE * vb + TC_PPT * grp;
#pragma unroll
          for (int d = 0; d < D; ++d) {
            float h4[4], l4[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) split_tf32(s[d][j], h4[j], l4[j]);
            tmem_st4(vcol + 16u * d, h4);
            tmem_st4(vcol + TC_VLO + 16u * d, l4);
          }
          tc_fence_before();
          mbar_arrive(&bar[B_VFULL + vb]);
          if (c == nch - 1 && t + 1 < my_tiles) {
            // the next tile's inputs: U is free (this chunk's S landed, so every product reading U is done)
            const int64_t e1 = (tile + gridDim.x) * TC_M + m;
            gather_tile<KP>(E, P, e1, e1 < E, grp, m, masked, rmap, x, u_hi, u_lo);
            fence_proxy_async();
            mbar_arrive(&bar[B_UFULL]);
          }
        }
      }
      // epilogue of tile t: this thread's quarter of the element's output nodes, TMEM -> element vectors
      if (ok) ok = mbar_wait_abortable(&bar[B_YFULL + yb], (uint32_t)((t >> 1) & 1), abort_flag);
      ok = __all_sync(0xffffffffu, ok);
      if (ok) {
        tc_fence_after();
#pragma unroll
        for (int j0 = 0; j0 < NP / TC_GROUPS; j0 += 4) {
          const int n0 = grp * (NP / TC_GROUPS) + j0;
          float y4[4];
          tmem_ld4(tmem + lane_base + TC_YCOL0 + TC_YSTRIDE * yb + (uint32_t)n0, y4);
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (valid && n0 + j < P) Ye[(int64_t)(n0 + j) * E + e] = y4[j];
        }
        tc_fence_before();
        mbar_arrive(&bar[B_YFREE + yb]);
      }
      if (!compute_all(ok)) {
        ok = false;
        break;
      }
    }
    if (QPRE) cp_async_wait_all();   // no copy into shared memory may outlive the block
    if (!ok) {
      *abort_flag = 1;
      atomicExch(err, (int)CEED_ERR_TIMEOUT);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == TC_CW) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_ALLOC) : "memory");
  }
}

// Host: chunked, split, padded tables of one operator (D = 1 interp, 3 grad) in the shared-memory
// image order of the kernel.
static void build_tables(const std::vector<double> &tab, int D, int P, int Q, int KP, int NP, int nch,
                         std::vector<float> &out) {
  const int W = chunk_words(D, KP, NP);
  out.assign((size_t)W * nch, 0.f);
  auto split = [](double v, float &hi, float &lo) {
    const float f = (float)v;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    // round to nearest, ties away from zero, keeping 10 mantissa bits (the cvt.rna.tf32 rounding)
    u = (u + 0x1000u) & 0xFFFFE000u;
    std::memcpy(&hi, &u, 4);
    lo = (float)(v - (double)hi);
  };
  for (int c = 0; c < nch; ++c) {
    float *o = out.data() + (size_t)c * W;
    float *gt_hi = o, *gt_lo = o + D * TC_QC * KP;
    float *g_hi = o + 2 * D * TC_QC * KP, *g_lo = g_hi + D * NP * TC_QC;
    for (int d = 0; d < D; ++d)
      for (int r = 0; r < TC_QC; ++r) {
        const int q = c * TC_QC + r;
        if (q >= Q) continue;
        for (int n = 0; n < P; ++n) {
          float hi, lo;
          split(tab[((size_t)d * Q + q) * P + n], hi, lo);
          gt_hi[d * TC_QC * KP + canon(r, n, KP)] = hi;   // GEMM1 B: row = point, K = node
          gt_lo[d * TC_QC * KP + canon(r, n, KP)] = lo;
          g_hi[d * NP * TC_QC + canon(n, r, TC_QC)] = hi;  // GEMM2 B: row = node, K = point
          g_lo[d * NP * TC_QC + canon(n, r, TC_QC)] = lo;
        }
      }
  }
}

template <int D, int KP, int NP, int TBUF, int QPRE>
static int launch_tc(ceed_nt_t h, const float *tabs, const float *qd, const double *x, float *Ye, int masked,
                     cudaStream_t s) {
  using L = TcLayout<D, KP, NP, TBUF, QPRE>;
  // one block per SM: the block holds 512 TMEM columns (S and Y double-buffered)
  constexpr size_t SMEM = L::BYTES > 116 * 1024 ? L::BYTES : 116 * 1024;
  if (int st = ensure_dynamic_smem((const void *)nt_tc_kernel<D, KP, NP, TBUF, QPRE>, SMEM)) return st;
  int sms = 0;
  CEED_CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
  const int64_t ntiles = (h->E + TC_M - 1) / TC_M;
  const unsigned grid = (unsigned)std::min<int64_t>(ntiles, (int64_t)sms);
  nt_tc_kernel<D, KP, NP, TBUF, QPRE><<<grid, TC_BLOCK, SMEM, s>>>(h->E, h->Es, h->P, h->Q, h->tc_nchunk,
                                                                        h->d_rmap, x, tabs, qd, Ye, masked, h->d_err);
  CEED_CUDA_CHECK(cudaGetLastError());
  return CEED_OK;
}

// Buffering that fits in shared memory, in order of benefit: the quadrature-data prefetch buffer,
// then a second table buffer (the tables of the next chunk stream in during the current one).
template <int D, int KP, int NP>
struct TcBufs {
  static constexpr size_t lim = 227 * 1024;
  static constexpr size_t base = 8ull * TC_M * KP + TC_NBAR * 8 + 16;
  static constexpr size_t tbw = 4ull * chunk_words(D, KP, NP);
  static constexpr size_t qw = 4ull * (D == 3 ? 6 : 1) * TC_QC * TC_M;
  static constexpr int QPRE = base + tbw + qw <= lim ? 1 : 0;
  static constexpr int TBUF = base + 2 * tbw + QPRE * qw <= lim ? 2 : 1;
};

template <int PP>
static int dispatch_p(ceed_nt_t h, int op, const float *qd, const double *x, float *Ye, int masked, cudaStream_t s) {
  constexpr int KP = kpad(PP), NP = npad(PP);
  const float *tabs = h->d_tc_tab[op == CEED_OP_MASS ? 0 : 1];
  using B1 = TcBufs<1, KP, NP>;
  using B3 = TcBufs<3, KP, NP>;
  return op == CEED_OP_MASS ? launch_tc<1, KP, NP, B1::TBUF, B1::QPRE>(h, tabs, qd, x, Ye, masked, s)
                            : launch_tc<3, KP, NP, B3::TBUF, B3::QPRE>(h, tabs, qd, x, Ye, masked, s);
}

}  // namespace

// The kernel is instantiated for the node counts of the degree-1..6 tetrahedra (P = 4, 10, 20, 35,
// 56, 84); other bases run on the CUDA-core algorithms.
bool nt_tc_supported(int P) { return P == 4 || P == 10 || P == 20 || P == 35 || P == 56 || P == 84; }

int nt_tc_prepare(ceed_nt_t h) {
  if (h->d_tc_tab[0]) return CEED_OK;
  if (!nt_tc_supported(h->P)) return fail(CEED_ERR_UNSUPPORTED, "tensor-core operator: P must be 4, 10, 20, 35, 56 or 84");
  const int P = h->P, Q = h->Q, KP = kpad(P), NP = npad(P);
  const int nch = (Q + TC_QC - 1) / TC_QC;
  std::vector<double> tab;
  try {
    tab.resize((size_t)4 * Q * P);
  } catch (...) {
    return fail(CEED_ERR_OOM, "host allocation");
  }
  CEED_CUDA_CHECK(cudaMemcpy(tab.data(), h->d_tab64, tab.size() * 8, cudaMemcpyDeviceToHost));
  for (int op = 0; op < 2; ++op) {
    const int D = op == 0 ? 1 : 3;
    std::vector<double> t(tab.begin() + (op == 0 ? 0 : (size_t)Q * P), tab.begin() + (op == 0 ? (size_t)Q * P : tab.size()));
    std::vector<float> img;
    build_tables(t, D, P, Q, KP, NP, nch, img);
    float *d = nullptr;
    CEED_CUDA_CHECK(cudaMalloc(&d, img.size() * 4));
    h->d_tc_tab[op] = d;
    CEED_CUDA_CHECK(cudaMemcpy(d, img.data(), img.size() * 4, cudaMemcpyHostToDevice));
  }
  h->tc_nchunk = nch;
  return CEED_OK;
}

int nt_tc_apply(ceed_nt_t h, int op, const float *qd, const double *x, float *Ye, int masked, cudaStream_t s) {
  switch (h->P) {
    case 4: return dispatch_p<4>(h, op, qd, x, Ye, masked, s);
    case 10: return dispatch_p<10>(h, op, qd, x, Ye, masked, s);
    case 20: return dispatch_p<20>(h, op, qd, x, Ye, masked, s);
    case 35: return dispatch_p<35>(h, op, qd, x, Ye, masked, s);
    case 56: return dispatch_p<56>(h, op, qd, x, Ye, masked, s);
    case 84: return dispatch_p<84>(h, op, qd, x, Ye, masked, s);
    default: return fail(CEED_ERR_UNSUPPORTED, "tensor-core operator: unsupported P");
  }
}

}  // namespace ceedgb
