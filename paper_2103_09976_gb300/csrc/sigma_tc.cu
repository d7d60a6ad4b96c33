// Mixed-precision sigma = H_eff . psi on the 5th-generation tensor cores.
//
// Same decomposition as the FP64 path (Sec. II.D-E: a flat list of
// (term, sector) products summed per output tile, partial tiles reduced in a
// fixed order), reorganized for tcgen05.mma. Every FP64 operand is split
// x = hi + mid + lo (three bf16 numbers, 24 significant bits) and a product
// a*b is the sum of the slice products with i + j <= 2 (6 MMAs, BF16X3) or
// i + j <= 1 (3 MMAs, BF16X2), accumulated in FP32 in tensor memory.
//
// Work unit: up to 16 terms of one class (same output tile, same psi block,
// same transposition flags). Their left operators' rows are stacked into one
// 128-row A operand, so one MMA chain gives the intermediates
// X_t = L_t[rows, :] psi_b of all of them at once (stage 1); X leaves the
// tensor memory only to be scaled by c_t and re-split into bf16 slices in
// shared memory, where it is the A operand of each term's
// sigma[tile] += X_t R_t[cols, :]^T (stage 2). Stage 1 runs over 128-column
// chunks of psi, stage 2 over 64-column halves of each chunk.
//
// Accuracy: within a chain the correction products are issued before the
// main (hi x hi) ones, while the accumulator is still small. The FP32 tile
// accumulator is added into a per-thread FP32 running sum after every flush
// group: the terms of one half whose main MMA steps fit the launch's chain
// limit (at least one term), or both halves of a chunk of a one-term unit
// when they fit together. The sum is written to the item's FP64 partial tile
// at the end of the item. This bounds the length of every FP32 accumulation
// chain of stage 2 in the tensor memory; the running sum adds one rounding
// per flush group. (A compensated running sum cost about a fifth of the
// kernel's time for a few percent of its error.)
//
// Warp roles (384 threads): warps 0, 10 and 11 stream operator and psi tiles
// with cp.async.bulk into a 3-stage ring, warp w filling slot w (a warp
// issues its copies one lane after another, and preparing a stage costs
// about as much as the copies: three warps prepare three stages at once);
// warp 0 also fetches the unit records.
// Warp 1 issues the MMAs (one elected lane of a warp that runs the control
// flow uniformly); warps 2-9 are the epilogue (two warps per TMEM lane
// quarter, 64 columns each). Tensor memory: two 128-column X buffers, two
// 128-column tile accumulators.
// Operands are stored in 8x8 core-matrix tiles, so one stored block serves as
// a K-major operand (S) or an MN-major one (S^T) with no copy: transposed
// terms only change the shared-memory descriptors.
//
// Every wait on an mbarrier is bounded (about one second of clock); on a
// timeout the kernel raises a flag in *err, stops issuing work, waits (again
// bounded) for its own copies, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstddef>

#include "kernels.h"

namespace dmrg {

namespace {

constexpr int NEPI = 8;                         // epilogue warps
constexpr int NPW = 3;                          // producer warps (warp 0, then warps 2 + NEPI ..), one per ring slot
constexpr int NTHR = 32 * (NPW + 1 + NEPI);     // producers + MMA + epilogue
constexpr int A2_SLICE = 16 * 1024;             // X half: 16 row groups x 8 K groups x 128 B
constexpr int A2_OFF = 0;                       // A2 first: reads past its last slice land in stage 0
constexpr int NMETA = 8;                        // unit records in the shared-memory ring
constexpr int PREFETCH = 4;                     // records fetched ahead of the producer
constexpr long long WAIT_CYCLES = 2000000000ll; // ~1 s at 2 GHz

// Shared-memory layout of one precision. Operator and psi tiles are stored
// slice-interleaved: tile position k holds its NSL 8x8 slices (bf16 hi, mid,
// lo; or fp16 hi, lo) at bytes TILE*k + 128*s, in global memory and in the
// stages alike. The second-product operand (A2) holds NSL slices of X.
// Stage geometry: STAGE_TILES tile positions per stage; a stage-1 stage
// holds KG1 K groups of the stacked left operators (16 M groups) and of psi
// (16 N groups, from PSI_TILE on). NA2 second-product operands (A2) let the
// epilogue convert the next 64-column half while the MMAs read the last.
template <bool F16>
struct Lay {
  static constexpr int NSL = F16 ? 2 : 3;
  static constexpr int TILE = 128 * NSL;
  static constexpr int STAGES = 3;
  static constexpr int STAGE_TILES = F16 ? 192 : 128;
  static constexpr int KG1 = F16 ? 6 : 4;
  static constexpr int PSI_TILE = 16 * KG1;
  static constexpr int NA2 = F16 ? 2 : 1;
  static constexpr int A2_BYTES = NSL * A2_SLICE;  // one A2 buffer
  static constexpr int STAGE_BYTES = STAGE_TILES * TILE;
  static constexpr int STAGE_OFF = NA2 * A2_BYTES;
  static constexpr int META_OFF = STAGE_OFF + STAGES * STAGE_BYTES;
  static constexpr int BAR_OFF = META_OFF + NMETA * (int)sizeof(TcUnitRec);
  static constexpr int SMEM_BYTES = BAR_OFF + 512;
  // barrier slots (8 bytes each)
  static constexpr int B_FULL = 0, B_EMPTY = STAGES, B_XFULL = 2 * STAGES, B_XEMPTY = 2 * STAGES + 2,
                       B_A2FULL = 2 * STAGES + 4, B_A2EMPTY = B_A2FULL + NA2, B_SFULL = B_A2EMPTY + NA2,
                       B_SEMPTY = B_SFULL + 2, B_MFULL = B_SEMPTY + 2, B_MEMPTY = B_MFULL + NMETA,
                       B_TMEM = B_MEMPTY + NMETA, B_ABORT = B_TMEM + 1;
  static_assert(8 * (B_ABORT + 1) <= 512, "barrier region");
  static_assert(SMEM_BYTES <= 227 * 1024, "shared memory");
  static_assert(META_OFF % 16 == 0, "records are bulk-copied");
  static_assert(KG1 % 2 == 0 && 2 * PSI_TILE <= STAGE_TILES, "stage-1 stage");
  static_assert(STAGES == NPW, "one producer warp per ring slot");
};
static_assert(sizeof(TcUnitRec) == 464 && offsetof(TcUnitRec, t) == 80, "record layout");
static_assert(sizeof(TcUnitRec) % 16 == 0, "records are bulk-copied");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16, M = 128, FP32 accumulator: A and B
// both bf16 (F16 = false) or both fp16.
template <bool F16>
__device__ __forceinline__ uint32_t idesc_of(int n, int a_mn, int b_mn) {
  const uint32_t fmt = F16 ? 0u : 1u;
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n"
               ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
  return ok != 0;
}

// Per-CTA wait-time accounting (profiling only): cycles spent blocked on
// each kind of barrier, summed in shared memory, flushed to global memory.
__shared__ unsigned long long s_wait[16];

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
  return ok != 0;
}

// Bounded wait; returns false (and raises the abort flag) on timeout or if
// another role already aborted. `code` names the barrier kind (wait
// accounting and the error report). With wait accounting (PROF) the first
// probe does not block (test_wait), so every cycle spent waiting is counted.
template <bool PROF>
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          int* err, int code) {
  if (PROF ? mbar_test(bar, parity) : mbar_try(bar, parity)) return true;
  long long t0 = clock64();
  for (;;) {
    if (mbar_try(bar, parity)) {
      if (PROF) atomicAdd(&s_wait[code & 15], (unsigned long long)(clock64() - t0));
      return true;
    }
    if (*abort_flag) return false;
    if (clock64() - t0 > WAIT_CYCLES) {
      *abort_flag = 1;
      atomicExch(err, code);
      return false;
    }
  }
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

// Bits of two floats rounded to bf16 (round to nearest even), lo in bits 0-15.
__device__ __forceinline__ uint32_t bf16x2_bits(float lo, float hi) {
  const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&p);
}

__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
               ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
               "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                 "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                 "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
                 "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
                 "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------ unit geometry
// (host and device: the host counts ring stages with the same formulas)
__host__ __device__ __forceinline__ int n_chunks(const TcUnitRec& r) { return (r.n + 127) >> 7; }
__host__ __device__ __forceinline__ int chunk_cols(const TcUnitRec& r, int j) { return min(128, r.n - 128 * j); }
__host__ __device__ __forceinline__ int n_halves(const TcUnitRec& r, int j) { return (chunk_cols(r, j) + 63) >> 6; }
__host__ __device__ __forceinline__ int half_cols(const TcUnitRec& r, int j, int h) { return min(64, chunk_cols(r, j) - 64 * h); }
template <int KG1>
__host__ __device__ __forceinline__ int k1_stages(const TcUnitRec& r) { return (r.pR8 + KG1 - 1) / KG1; }
__host__ __device__ __forceinline__ int tn8e(const TcUnitRec& r) { return 2 * ((r.tn + 15) >> 4); }  // N groups read by the MMA
__host__ __device__ __forceinline__ int kg2_of(int kw) { return 2 * ((kw + 15) >> 4); }               // K groups of a half
// Shared-memory stride (tile positions) of the right operator of a stage-2
// stage. With runs (one producer warp), copies_s2 moves a term's tiles as
// one run where the stored block allows, keeping the block's stride: the
// N-group stride when not transposed (bC8 when the half holds all K groups
// of the block), the K-group stride when transposed (tn8 when the tile spans
// all stored columns); otherwise kg2 / te. Runs measured 4% faster with one
// producer (small blocks) and 3.5% slower with three (large blocks).
__host__ __device__ __forceinline__ int b_stride(const TcUnitRec& r, int j, int h, bool runs) {
  const int kg2 = kg2_of(half_cols(r, j, h)), kgx = 16 * j + 8 * h, tn8 = (r.tn + 7) >> 3;
  if (r.flags & TC_TB) return runs && tn8 == r.bC8 ? tn8 : tn8e(r);
  return runs && min(kg2, r.bC8 - kgx) == r.bC8 ? r.bC8 : kg2;
}
// Terms per flush group: the most whose main K steps in one half stay within
// max_chain (at least one); max_chain <= 0: the whole unit.
__device__ __forceinline__ int flush_terms(const TcUnitRec& r, int max_chain) {
  const int steps = (min(64, r.n) + 15) >> 4;
  return max_chain > 0 ? max(1, min(r.nterm, max_chain / steps)) : r.nterm;
}
// A unit of one term whose chunk fits the chain limit accumulates both
// halves of chunk j in one group (one flush per chunk instead of per half).
__device__ __forceinline__ bool whole_chunk_group(const TcUnitRec& r, int j, int max_chain) {
  return r.nterm == 1 && (max_chain <= 0 || ((chunk_cols(r, j) + 15) >> 4) <= max_chain);
}

// A unit's geometry, read once from its record in shared memory (the
// barrier waits clobber memory, so fields read in loops would be re-read).
struct UnitGeo {
  int flags, G, tm8, tn, tn8, te, r0g, c0g, n, aR8, aC8, bR8, bC8, pR8, pC8;
  long long p_tile;
};
__device__ __forceinline__ UnitGeo geo_of(const TcUnitRec& r) {
  UnitGeo g;
  g.flags = r.flags;
  g.G = r.nterm;
  g.tm8 = r.tm8;
  g.tn = r.tn;
  g.tn8 = (r.tn + 7) >> 3;
  g.te = 2 * ((r.tn + 15) >> 4);
  g.r0g = r.r0g;
  g.c0g = r.c0g;
  g.n = r.n;
  g.aR8 = r.aR8;
  g.aC8 = r.aC8;
  g.bR8 = r.bR8;
  g.bC8 = r.bC8;
  g.pR8 = r.pR8;
  g.pC8 = r.pC8;
  g.p_tile = r.p_tile;
  return g;
}

// Copies of one stage-1 stage (psi columns of chunk j, K groups KG1*k ..):
// the stacked left-operator rows of every term ([M group][K group], or
// [K group][M group] when the left operator is used transposed) and the psi
// tiles ([K group][N group] from PSI_TILE on); the list holds the operator
// copies, then one psi copy per K group. (Moving the stage's tiles of a term
// or of psi as one run where the stored block allows, with the run's stride
// in shared memory, measured slower on large blocks and no faster on small
// ones: only stage 2 does it.) f(src_tile, operand (0 operators, 1 psi),
// dst_tile, n_tiles) moves n_tiles tile positions; lane l issues copies l,
// l + 32, ... count_only: issue nothing, return the stage's tile positions
// (the same on every lane).
template <int KG1, class F>
__device__ __forceinline__ uint32_t copies_s1(const TcUnitRec& r, const UnitGeo& g, int j, int k, int lane,
                                              bool count_only, F&& f) {
  constexpr int PSI_TILE = 16 * KG1;
  const int kg0 = KG1 * k;
  const bool tA = g.flags & TC_TA;
  const int nkA = tA ? min(KG1, g.aR8 - kg0) : min(KG1, g.aC8 - kg0);  // K groups of A in this stage
  const int nA = nkA > 0 ? (tA ? g.G * nkA : g.G * g.tm8) : 0;         // A copies
  const int perA = tA ? g.tm8 : nkA;                                    // tiles per A copy
  const int nkP = max(0, min(KG1, g.pR8 - kg0)), nn = min(16, g.pC8 - 16 * j);
  const int ntot = nA + nkP;
  if (count_only) return (uint32_t)(nA * perA + nkP * nn);
  for (int c = lane; c < ntot; c += 32) {
    if (c >= nA) {
      const int kg = c - nA;
      f(g.p_tile + (long long)(kg0 + kg) * g.pC8 + 16 * j, 1, PSI_TILE + kg * 16, nn);
    } else if (!tA) {
      const int q = c / g.tm8, rg = c - q * g.tm8;
      f(r.t[q].a_tile + (long long)(g.r0g + rg) * g.aC8 + kg0, 0, (q * g.tm8 + rg) * KG1, perA);
    } else {
      const int q = c / nkA, kg = c - q * nkA;
      f(r.t[q].a_tile + (long long)(kg0 + kg) * g.aC8 + g.r0g, 0, kg * 16 + q * g.tm8, perA);
    }
  }
  return 0;
}

// Copies of one stage-2 stage: the right-operator tiles (output columns of
// the tile, K groups of half h of chunk j) of terms q0..q1-1, each term in a
// region of te x kg2 tile positions ([N group][K group], or [K group][N
// group] when the right operator is used transposed; with runs one copy per
// term where the block allows, strides as b_stride). As copies_s1.
template <class F>
__device__ __forceinline__ uint32_t copies_s2(const TcUnitRec& r, const UnitGeo& g, int j, int h, int q0, int q1,
                                              bool runs, int lane, bool count_only, F&& f) {
  const int kw = min(64, min(128, g.n - 128 * j) - 64 * h), kg2 = kg2_of(kw), kgx = 16 * j + 8 * h;
  const bool tB = g.flags & TC_TB;
  const int nkB = tB ? min(kg2, g.bR8 - kgx) : min(kg2, g.bC8 - kgx);  // K groups of B present
  const bool b_run = runs && (tB ? g.tn8 == g.bC8 : nkB == g.bC8);    // one run per term
  const int per = b_run ? nkB * g.tn8 : (tB ? g.tn8 : nkB);
  const int span = b_run ? 1 : (tB ? nkB : g.tn8);                    // copies per term
  const int ncopy = (q1 - q0) * span;
  if (count_only) return (uint32_t)(ncopy * per);
  for (int c = lane; c < ncopy; c += 32) {
    const int qq = c / span, x = c - qq * span, reg = qq * g.te * kg2;
    if (b_run)
      f(r.t[q0 + qq].b_tile + (long long)(tB ? kgx : g.c0g) * g.bC8, 0, reg, per);
    else if (!tB)
      f(r.t[q0 + qq].b_tile + (long long)(g.c0g + x) * g.bC8 + kgx, 0, reg + x * kg2, per);
    else
      f(r.t[q0 + qq].b_tile + (long long)(kgx + x) * g.bC8 + g.c0g, 0, reg + x * g.te, per);
  }
  return 0;
}

}  // namespace

// Slice pair of product p (hh, hm, mh, hl, mm, lh): i indexes the A slices,
// j the B slices.
__device__ __forceinline__ constexpr int prod_i(int p) { return (p == 2 || p == 4) ? 1 : (p == 5 ? 2 : 0); }
__device__ __forceinline__ constexpr int prod_j(int p) { return (p == 1 || p == 4) ? 1 : (p == 3 ? 2 : 0); }

// One K chain of slice products into tmem_d: the correction products of all
// K steps first, then the main (hi x hi) ones. Descriptors differ only in
// the start-address field, so each MMA adds its byte offset >> 4 to a base.
// `first`: the next MMA overwrites the accumulator (cleared after it).
// One MMA from descriptors given as 32-bit halves (the start-address field
// is in the low half: offsets are added there, without a 64-bit add).
__device__ __forceinline__ void mma_lohi(uint32_t tmem, uint32_t alo, uint32_t ahi, uint32_t blo, uint32_t bhi,
                                         uint32_t idesc, uint32_t acc) {
  asm volatile("{\n.reg .b64 ad, bd;\n.reg .pred p;\nmov.b64 ad, {%1, %2};\nmov.b64 bd, {%3, %4};\n"
               "setp.ne.b32 p, %6, 0;\n"
               "tcgen05.mma.cta_group::1.kind::f16 [%0], ad, bd, %5, p;\n}\n"
               ::"r"(tmem), "r"(alo), "r"(ahi), "r"(blo), "r"(bhi), "r"(idesc), "r"(acc));
}

// One lane of a converged warp (elect.sync over the full warp: the same
// lane every time). The MMA warp issues its MMAs and their commits through it,
// so each commit tracks the MMAs before it.
__device__ __forceinline__ bool elect_one() {
  uint32_t p = 0;
  asm volatile("{\n.reg .b32 rx;\n.reg .pred px;\nelect.sync rx|px, %1;\nselp.u32 %0, 1, 0, px;\n}\n"
               : "=r"(p) : "r"(0xffffffffu));
  return p != 0;
}

// One K chain of slice products into tmem_d: the correction products of all
// NKS K steps first, then the main (hi x hi) ones. a / b: descriptors;
// a_slice, b_slice: byte offsets of the mid slice; a_kstep, b_kstep: byte
// offsets of one K step. All offsets are compile-time multiples after
// unrolling, so the issuing loop is a run of MMAs on precomputed operands.
// The whole warp evaluates the (uniform) descriptors; the elected lane issues.
// `first`: the next MMA overwrites the accumulator (cleared after it).
template <int NPROD, int NKS>
__device__ __forceinline__ void mma_chain_k(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t a_slice,
                                            uint32_t b_slice, uint32_t a_kstep, uint32_t b_kstep, uint32_t idesc,
                                            bool& first) {
  const uint32_t alo = (uint32_t)a, ahi = (uint32_t)(a >> 32), blo = (uint32_t)b, bhi = (uint32_t)(b >> 32);
  const uint32_t as16 = a_slice >> 4, bs16 = b_slice >> 4, ak16 = a_kstep >> 4, bk16 = b_kstep >> 4;
  uint32_t acc = first ? 0u : 1u;
  if (elect_one()) {
#pragma unroll
    for (int ks = 0; ks < NKS; ++ks)
#pragma unroll
      for (int p = 1; p < NPROD; ++p) {
        mma_lohi(tmem_d, alo + prod_i(p) * as16 + ks * ak16, ahi, blo + prod_j(p) * bs16 + ks * bk16, bhi, idesc,
                 acc);
        acc = 1u;
      }
#pragma unroll
    for (int ks = 0; ks < NKS; ++ks) {
      mma_lohi(tmem_d, alo + ks * ak16, ahi, blo + ks * bk16, bhi, idesc, acc);
      acc = 1u;
    }
  }
  first = false;
}

template <int NPROD>
__device__ __forceinline__ void mma_chain(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t a_slice,
                                          uint32_t b_slice, uint32_t a_kstep, uint32_t b_kstep, int nks,
                                          uint32_t idesc, bool& first) {
  switch (nks) {
    case 1: mma_chain_k<NPROD, 1>(tmem_d, a, b, a_slice, b_slice, a_kstep, b_kstep, idesc, first); break;
    case 2: mma_chain_k<NPROD, 2>(tmem_d, a, b, a_slice, b_slice, a_kstep, b_kstep, idesc, first); break;
    case 3: mma_chain_k<NPROD, 3>(tmem_d, a, b, a_slice, b_slice, a_kstep, b_kstep, idesc, first); break;
    default: mma_chain_k<NPROD, 4>(tmem_d, a, b, a_slice, b_slice, a_kstep, b_kstep, idesc, first); break;
  }
}

// PROF: record wait accounting and MMA-thread cycles into a.wait_prof.
// F16: FP16X2 (two fp16 slices of scaled operands; see split_f16.cu).
// NP: producer warps (TcDev::producers, 1 or NPW), a template parameter so
// that each setting compiles only its own copy code.
template <int NPROD, bool F16, bool PROF, int NP>
__global__ void __launch_bounds__(NTHR, 1) sigma_tc_kernel(TcDev a) {
  static_assert(NP == 1 || NP == NPW, "producer warps");
  using L = Lay<F16>;
  constexpr int TILE = L::TILE, STAGES = L::STAGES, STAGE_BYTES = L::STAGE_BYTES, STAGE_OFF = L::STAGE_OFF;
  constexpr int META_OFF = L::META_OFF, BAR_OFF = L::BAR_OFF, STAGE_TILES = L::STAGE_TILES, KG1 = L::KG1,
                PSI_TILE = L::PSI_TILE, NA2 = L::NA2, A2_BYTES = L::A2_BYTES;
  constexpr int B_FULL = L::B_FULL, B_EMPTY = L::B_EMPTY, B_XFULL = L::B_XFULL, B_XEMPTY = L::B_XEMPTY,
                B_A2FULL = L::B_A2FULL, B_A2EMPTY = L::B_A2EMPTY, B_SFULL = L::B_SFULL, B_SEMPTY = L::B_SEMPTY,
                B_MFULL = L::B_MFULL, B_MEMPTY = L::B_MEMPTY, B_TMEM = L::B_TMEM, B_ABORT = L::B_ABORT;
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t sbase = smem_u32(sm);
  const uint32_t bars = sbase + BAR_OFF;
  auto bar = [&](int k) { return bars + 8u * (uint32_t)k; };
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + BAR_OFF + 8 * B_ABORT);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + BAR_OFF + 8 * B_TMEM);
  TcUnitRec* ring = reinterpret_cast<TcUnitRec*>(sm + META_OFF);

  const long long t_start = clock64();
  if (tid < 16) s_wait[tid] = 0ull;
  // zero all operand buffers once: afterwards shared memory only ever holds
  // finite operand data or zeros, so padded K positions multiply to 0 and
  // padded rows stay finite.
  for (int i = tid; i < META_OFF / 16; i += NTHR) reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(bar(B_FULL + s), 1);
      mbar_init(bar(B_EMPTY + s), 1);
    }
    for (int x = 0; x < 2; ++x) {
      mbar_init(bar(B_XFULL + x), 1);
      mbar_init(bar(B_XEMPTY + x), NEPI);
      mbar_init(bar(B_SFULL + x), 1);
      mbar_init(bar(B_SEMPTY + x), NEPI);
    }
    for (int b = 0; b < NA2; ++b) {
      mbar_init(bar(B_A2FULL + b), NEPI);
      mbar_init(bar(B_A2EMPTY + b), 1);
    }
    for (int m = 0; m < NMETA; ++m) {
      mbar_init(bar(B_MFULL + m), 1);
      mbar_init(bar(B_MEMPTY + m), NP + 1 + NEPI);  // producer, MMA and epilogue warps
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;\n" ::"r"(smem_u32(tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 || (warp >= 2 + NEPI && NP != 1)) {
    // ------------------------------------------------------------ producers
    // With NP == NPW every producer warp walks the same units and
    // stages and warp pw fills ring slot pw (NPW = STAGES), so each slot has
    // one producer and the stages of a unit are filled by three warps at
    // once; with NP == 1 warp 0 fills every slot and the others
    // stay idle. Warp 0 (pw 0) also fetches the unit records into the ring;
    // the others read them there.
    const int pw = warp == 0 ? 0 : warp - 1 - NEPI;  // 0 .. NPW-1
    constexpr bool all_slots = NP == 1;
    uint32_t stage = 0, phase = 1;  // empty barriers: first wait passes
    bool ok = true;
    const char* const ops = (const char*)a.op;
    const char* const ps = (const char*)a.psi;
    // one stage: wait for it to be free, announce its bytes, issue the copies
    // one stage: if it is this warp's ring slot, wait for the slot to be
    // free, announce its bytes, issue the copies; every warp counts it
    auto produce = [&](auto&& copies) {
      if (!ok) return;
      if (all_slots || stage == (uint32_t)pw) {
        if (!mbar_wait<PROF>(bar(B_EMPTY + stage), phase, abort_flag, a.err, 1)) { ok = false; return; }
        const uint32_t sdst = sbase + STAGE_OFF + stage * STAGE_BYTES;
        const uint32_t fb = bar(B_FULL + stage);
        // the byte count is announced before any copy can complete: lane 0
        // arrives with the expected bytes first, then all lanes issue copies
        const uint32_t tiles = copies([&](long long, int, int, int) {}, true);
        if (lane == 0) mbar_expect_tx(fb, (uint32_t)TILE * tiles);
        __syncwarp();
        copies([&](long long src, int which, int dst, int n) {
          bulk_g2s(sdst + (uint32_t)dst * TILE, (which ? ps : ops) + src * TILE, (uint32_t)TILE * (uint32_t)n, fb);
        }, false);
      }
      if (++stage == STAGES) { stage = 0; phase ^= 1; }
    };
    auto produce_s1 = [&](const TcUnitRec& u, int j) {
      const UnitGeo g = geo_of(u);
      const int nk1 = (g.pR8 + KG1 - 1) / KG1;
      for (int k = 0; k < nk1; ++k)
        produce([&](auto&& f, bool count_only) -> uint32_t {
          return copies_s1<KG1>(u, g, j, k, lane, count_only, f);
        });
    };
    auto produce_s2 = [&](const TcUnitRec& u, int j) {
      const UnitGeo g = geo_of(u);
      const int ccols = min(128, g.n - 128 * j);
      for (int h = 0; h < (ccols + 63) >> 6; ++h) {
        const int kw = min(64, ccols - 64 * h);
        const int P = max(1, min(g.G, STAGE_TILES / (g.te * kg2_of(kw))));
        for (int q0 = 0; q0 < g.G; q0 += P)
          produce([&](auto&& f, bool count_only) -> uint32_t {
            return copies_s2(u, g, j, h, q0, min(g.G, q0 + P), all_slots, lane, count_only, f);
          });
      }
    };
    bool no_more = false;
    int pf_r = 0, pf_end = 0;  // prefetch cursor: next record and end of its item
    long long pf_s = 0;        // records pushed into the ring
    auto prefetch_one = [&]() -> bool {
      if (pf_r == pf_end) {    // take the next item
        if (no_more) return false;
        int q = 0;
        if (lane == 0) q = (int)atomicAdd(a.counter, 1u);
        q = __shfl_sync(0xffffffffu, q, 0);
        if (q >= a.n_items) { no_more = true; return false; }
        const int it = a.schedule[q];
        pf_r = a.items[it].r_begin;
        pf_end = a.items[it].r_end;
      }
      const int slot = (int)(pf_s % NMETA);
      const uint32_t par = (uint32_t)(((pf_s / NMETA) & 1) ^ 1);
      if (!mbar_wait<PROF>(bar(B_MEMPTY + slot), par, abort_flag, a.err, 9)) { ok = false; return false; }
      if (lane == 0) {
        mbar_expect_tx(bar(B_MFULL + slot), (uint32_t)sizeof(TcUnitRec));
        bulk_g2s(smem_u32(ring + slot), a.recs + pf_r, (uint32_t)sizeof(TcUnitRec), bar(B_MFULL + slot));
      }
      __syncwarp();
      ++pf_r;
      ++pf_s;
      return true;
    };
    long long s = 0;
    int prev_slot = -1, prev_j = 0;  // sub-unit whose stage 2 is still to be produced
    auto finish_prev = [&]() {
      if (prev_slot < 0) return;
      const TcUnitRec& pu = ring[prev_slot];
      produce_s2(pu, prev_j);
      if (prev_j == n_chunks(pu) - 1) {
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(B_MEMPTY + prev_slot));
      }
      prev_slot = -1;
    };
    auto unit = [&](int slot) {  // the stages of one record (its slot's full barrier passed)
      const TcUnitRec& u = ring[slot];
      if (u.flags & TC_ZERO) {
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(B_MEMPTY + slot));
      } else {
        for (int j = 0; j < n_chunks(u) && ok; ++j) {
          produce_s1(u, j);
          finish_prev();
          prev_slot = slot;
          prev_j = j;
        }
      }
    };
    if (pw == 0) {
      for (;;) {
        while (ok && pf_s < s + PREFETCH && prefetch_one()) {
        }
        if (!ok) break;
        if (s == pf_s) break;  // nothing left
        const int slot = (int)(s % NMETA);
        if (!mbar_wait<PROF>(bar(B_MFULL + slot), (uint32_t)((s / NMETA) & 1), abort_flag, a.err, 10)) { ok = false; break; }
        unit(slot);
        ++s;
      }
      // terminator record, pushed before the last sub-unit's stage-2
      // operands: the MMA issuer and the other producers read it before they
      // reach those stages, and they can be more than the ring holds
      if (ok) {
        const int slot = (int)(s % NMETA);
        const uint32_t par = (uint32_t)(((s / NMETA) & 1) ^ 1);
        if (mbar_wait<PROF>(bar(B_MEMPTY + slot), par, abort_flag, a.err, 11)) {
          if (lane == 0) {
            ring[slot].flags = TC_DONE;
            mbar_arrive(bar(B_MFULL + slot));
          }
        } else {
          ok = false;
        }
        __syncwarp();
      }
      if (ok) finish_prev();
      __syncwarp();
      // drain: wait (bounded) until the MMA side released every stage (the
      // copies of all producer warps have landed once a stage is released)
      for (int k = 0; k < STAGES; ++k) {
        mbar_wait<PROF>(bar(B_EMPTY + stage), phase, abort_flag, a.err, 0);
        if (++stage == STAGES) { stage = 0; phase ^= 1; }
      }
    } else {
      // records in ring order until the terminator
      while (ok) {
        const int slot = (int)(s % NMETA);
        if (!mbar_wait<PROF>(bar(B_MFULL + slot), (uint32_t)((s / NMETA) & 1), abort_flag, a.err, 10)) { ok = false; break; }
        if (ring[slot].flags & TC_DONE) break;
        unit(slot);
        ++s;
      }
      if (ok) finish_prev();
      __syncwarp();
    }
  } else if (warp == 1) {
    // --------------------------------------------------------------- MMA
    // The whole warp runs this role's control flow, so descriptors and
    // counters stay warp-uniform; one elected lane issues the MMAs and their
    // commits, lane 0 the plain arrivals.
    {
      const bool leader = lane == 0;
      // with profiling on, slots 14 / 15 of the wait accounting receive the
      // cycles this warp spends issuing MMAs / committing them
      constexpr bool prof = PROF;
      auto tick = [&]() -> long long { return prof ? clock64() : 0ll; };
      auto tock = [&](int slot, long long t0) {
        if (prof && leader) s_wait[slot] += (unsigned long long)(clock64() - t0);
      };
      uint32_t stage = 0, phase = 0;
      uint32_t xcnt = 0, xph_empty = 3u;   // bit b: expected parity of X-empty[b]
      uint32_t h2 = 0;                     // halves consumed: A2 buffer h2 % NA2, parity (h2 / NA2) & 1
      uint32_t sb = 0, sph_empty = 3u;     // bit b: expected parity of S-empty[b]
      bool ok = true;
      auto acquire = [&]() -> uint32_t {
        if (!mbar_wait<PROF>(bar(B_FULL + stage), phase, abort_flag, a.err, 4)) { ok = false; return 0; }
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        return sbase + STAGE_OFF + stage * STAGE_BYTES;
      };
      auto release = [&]() {
        const long long t0 = tick();
        if (elect_one()) commit(bar(B_EMPTY + stage));
        tock(15, t0);
        if (++stage == STAGES) { stage = 0; phase ^= 1; }
      };
      // stage 1 of sub-unit (u, j): X = stacked left rows x psi chunk j
      auto mma_s1 = [&](const TcUnitRec& u, int j) {
        const uint32_t xb = xcnt & 1;
        if (!mbar_wait<PROF>(bar(B_XEMPTY + xb), (xph_empty >> xb) & 1u, abort_flag, a.err, 3)) { ok = false; return; }
        xph_empty ^= 1u << xb;
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        const uint32_t tmem_x = tmem + xb * 128;
        const int tA = (u.flags & TC_TA) ? 1 : 0;
        const uint32_t id1 = idesc_of<F16>(16 * ((chunk_cols(u, j) + 15) / 16), tA, 1);
        const uint32_t a_lbo = tA ? 16u * TILE : TILE, a_sbo = tA ? TILE : (uint32_t)KG1 * TILE;
        const int pR8 = u.pR8, nk1 = k1_stages<KG1>(u);  // read once: the waits below clobber memory
        bool first = true;
        for (int k = 0; k < nk1 && ok; ++k) {
          const uint32_t sst = acquire();
          if (!ok) return;
          const long long t0 = tick();
          mma_chain<NPROD>(tmem_x, sdesc(sst, a_lbo, a_sbo), sdesc(sst + PSI_TILE * TILE, 16u * TILE, TILE),
                           128u, 128u, 2 * a_lbo, 2 * 16u * TILE, min(KG1, pR8 - KG1 * k) / 2, id1, first);
          tock(14, t0);
          release();
        }
        {
          const long long t0 = tick();
          if (elect_one()) commit(bar(B_XFULL + xb));
          tock(15, t0);
        }
        ++xcnt;
      };
      // stage 2 of sub-unit (u, j): per half, per term, sigma += X_t R_t^T,
      // the tile accumulator switching buffers after every flush group
      auto mma_s2 = [&](const TcUnitRec& u, int j) {
        const int tB = (u.flags & TC_TB) ? 1 : 0, te = tn8e(u), G = u.nterm, F = flush_terms(u, a.max_chain);
        const uint32_t id2 = idesc_of<F16>(16 * ((u.tn + 15) / 16), 0, tB);
        const int nh = n_halves(u, j), tm8 = u.tm8, ccols = chunk_cols(u, j);
        const bool whole = whole_chunk_group(u, j, a.max_chain);
        constexpr bool runs = NP == 1;
        const int bst0 = b_stride(u, j, 0, runs), bst1 = nh > 1 ? b_stride(u, j, 1, runs) : 0;
        bool first = true;
        for (int h = 0; h < nh && ok; ++h) {
          const uint32_t hb = h2 % NA2;
          if (!mbar_wait<PROF>(bar(B_A2FULL + hb), (h2 / NA2) & 1u, abort_flag, a.err, 5)) { ok = false; return; }
          ++h2;
          const uint32_t a2 = sbase + A2_OFF + hb * A2_BYTES;
          const int kw = min(64, ccols - 64 * h), kg2 = kg2_of(kw), P = max(1, min(G, STAGE_TILES / (te * kg2)));
          const uint32_t bs = (uint32_t)(h == 0 ? bst0 : bst1) * TILE;
          const uint32_t b_lbo = tB ? bs : TILE;
          const uint32_t b_sbo = tB ? TILE : bs;
          int qf = 0;  // position of term q in its flush group (q % F)
          for (int q0 = 0; q0 < G && ok; q0 += P) {
            const uint32_t sst = acquire();
            if (!ok) return;
            for (int q = q0; q < min(G, q0 + P); ++q, qf = qf + 1 == F ? 0 : qf + 1) {
              const bool gstart = whole ? h == 0 : qf == 0;
              const bool gend = whole ? h == nh - 1 : (qf == F - 1 || q == G - 1);
              if (gstart) {  // a flush group starts: its tile accumulator must be free
                if (!mbar_wait<PROF>(bar(B_SEMPTY + sb), (sph_empty >> sb) & 1u, abort_flag, a.err, 2)) {
                  ok = false;
                  return;
                }
                sph_empty ^= 1u << sb;
                asm volatile("tcgen05.fence::after_thread_sync;\n");
                first = true;
              }
              const long long t0 = tick();
              mma_chain<NPROD>(tmem + 256 + sb * 128, sdesc(a2 + (uint32_t)(q * tm8) * 1024u, 128u, 1024u),
                               sdesc(sst + (uint32_t)((q - q0) * te * kg2) * TILE, b_lbo, b_sbo), A2_SLICE, 128u,
                               2 * 128u, 2 * b_lbo, kg2 / 2, id2, first);
              tock(14, t0);
              if (gend) {  // the group ends: hand the accumulator to the epilogue
                const long long t1 = tick();
                if (elect_one()) commit(bar(B_SFULL + sb));
                tock(15, t1);
                sb ^= 1;
              }
            }
            release();
          }
          const long long t1 = tick();
          if (elect_one()) commit(bar(B_A2EMPTY + hb));
          tock(15, t1);
        }
      };
      long long s = 0;
      int prev_slot = -1, prev_j = 0;
      auto finish_prev = [&]() {
        if (prev_slot < 0 || !ok) return;
        const TcUnitRec& pu = ring[prev_slot];
        mma_s2(pu, prev_j);
        if (prev_j == n_chunks(pu) - 1 && leader) mbar_arrive(bar(B_MEMPTY + prev_slot));
        prev_slot = -1;
      };
      while (ok) {
        const int slot = (int)(s % NMETA);
        if (!mbar_wait<PROF>(bar(B_MFULL + slot), (uint32_t)((s / NMETA) & 1), abort_flag, a.err, 12)) { ok = false; break; }
        const TcUnitRec& u = ring[slot];
        const int fl = u.flags;
        if (fl & TC_DONE) break;
        if (fl & TC_ZERO) {
          if (leader) mbar_arrive(bar(B_MEMPTY + slot));
        } else {
          for (int j = 0; j < n_chunks(u) && ok; ++j) {
            mma_s1(u, j);
            finish_prev();
            prev_slot = slot;
            prev_j = j;
          }
        }
        ++s;
      }
      finish_prev();
    }
    __syncwarp();
  } else if (warp < 2 + NEPI) {
    // ---------------------------------------------------------- epilogue
    const int e = warp - 2;                    // 0 .. NEPI-1
    const int quarter = warp & 3;              // TMEM lanes 32*quarter .. +31
    const int half = e >> 2;                   // columns 64*half .. +63 of a tile, 32*half .. +31 of an X half
    const int row = quarter * 32 + lane;       // TMEM lane owned by this thread
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    uint32_t xcnt = 0, xph_full = 0;           // bit b: expected parity of X-full[b]
    uint32_t h2 = 0;                           // halves converted: A2 buffer h2 % NA2, parity (h2 / NA2) & 1
    uint32_t sb = 0, sph_full = 0;             // bit b: expected parity of S-full[b]
    bool ok = true;
    uint16_t* a2 = reinterpret_cast<uint16_t*>(sm + A2_OFF);  // the A2 buffer of the current half
    // FP16X2: the flush undoes the unit's tile scale 2^(E - e_psi)
    const int e_psi = F16 ? psi_exponent(*a.psi_exp) : 0;
    // FP32 running sum of this thread's 64 tile columns
    float ahi[2][32];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int i = 0; i < 32; ++i) ahi[c][i] = 0.f;
    // write 32 K-columns (half of a 64-column X half) of A2 for this row
    auto write_a2 = [&](const float* v) {
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        uint32_t hw[4], mw[4], lw[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float x0 = v[g * 8 + 2 * q], x1 = v[g * 8 + 2 * q + 1];
          if (!F16) {
            // two columns at a time: one paired round-to-nearest conversion
            // per slice; a bf16 value is the upper half of its float, so the
            // residuals need only a mask or a shift and a subtraction
            const uint32_t hp = bf16x2_bits(x0, x1);
            const float r0 = x0 - __uint_as_float(hp << 16), r1 = x1 - __uint_as_float(hp & 0xFFFF0000u);
            const uint32_t mp = bf16x2_bits(r0, r1);
            const float s0 = r0 - __uint_as_float(mp << 16), s1 = r1 - __uint_as_float(mp & 0xFFFF0000u);
            hw[q] = hp;
            mw[q] = mp;
            lw[q] = bf16x2_bits(s0, s1);
          } else {  // fp16 hi and lo (the scaled X is below 2^14: no overflow)
            const __half2 hp = __floats2half2_rn(x0, x1);
            const float2 hf = __half22float2(hp);
            const __half2 lp = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
            hw[q] = *reinterpret_cast<const uint32_t*>(&hp);
            mw[q] = *reinterpret_cast<const uint32_t*>(&lp);
          }
        }
        const int off = (((row >> 3) * 8 + half * 4 + g) * 64 + (row & 7) * 8);  // 2-byte elements
        *reinterpret_cast<uint4*>(a2 + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4*>(a2 + A2_SLICE / 2 + off) = make_uint4(mw[0], mw[1], mw[2], mw[3]);
        if (!F16) *reinterpret_cast<uint4*>(a2 + A2_SLICE + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
      }
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_A2FULL + (h2 - 1) % NA2));
    };
    // add the tile accumulator of the next flush group into the running sum
    auto flush = [&](int tm, int tn, float fs) -> bool {
      if (!mbar_wait<PROF>(bar(B_SFULL + sb), (sph_full >> sb) & 1u, abort_flag, a.err, 8)) return false;
      sph_full ^= 1u << sb;
      asm volatile("tcgen05.fence::after_thread_sync;\n");
      if (quarter * 32 < tm) {  // warp-uniform: this warp owns tile rows
        const bool rv = row < tm;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int col0 = half * 64 + c * 32;
          if (col0 < tn) {  // warp-uniform
            float w[32];
            tmem_ld32(tmem + lane_off + 256 + sb * 128 + col0, w);
            const int nc = tn - col0;
            if (rv) {
#pragma unroll
              for (int g8 = 0; g8 < 4; ++g8) {
                if (g8 * 8 < nc) {  // warp-uniform: skip column groups past the tile
#pragma unroll
                  for (int i = 8 * g8; i < 8 * g8 + 8; ++i)
                    if (i < nc) ahi[c][i] = F16 ? fmaf(w[i], fs, ahi[c][i]) : ahi[c][i] + w[i];
                }
              }
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;\n");
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_SEMPTY + sb));
      sb ^= 1;
      return true;
    };
    long long s = 0;
    int pend = 0, pend_tm = 0, pend_tn = 0;  // flush groups deferred past the next conversion
    float pend_fs = 1.0f;
    while (ok) {
      const int slot = (int)(s % NMETA);
      if (!mbar_wait<PROF>(bar(B_MFULL + slot), (uint32_t)((s / NMETA) & 1), abort_flag, a.err, 13)) { ok = false; break; }
      const TcUnitRec& u = ring[slot];
      const int fl = u.flags;
      if (fl & TC_DONE) break;
      double* out = a.scratch + u.slot;
      if (fl & TC_ZERO) {
        if (row < u.tm)
          for (int c = half * 64; c < min(u.tn, half * 64 + 64); ++c) out[(long long)row * u.tn + c] = 0.0;
      } else {
        if (fl & TC_ITEM_FIRST) {
#pragma unroll
          for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int i = 0; i < 32; ++i) ahi[c][i] = 0.f;
        }
        // the term (and its scale) of this row of the stacked X
        const int q = row / (u.tm8 * 8), rr = row - q * (u.tm8 * 8);
        const float sc = (q < u.nterm && rr < u.tm) ? u.t[q].scale : 0.0f;
        const float fs = F16 ? ldexpf(1.0f, e_psi - u.pad[0]) : 1.0f;
        for (int j = 0; j < n_chunks(u) && ok; ++j) {
          const uint32_t xb = xcnt & 1;
          if (!mbar_wait<PROF>(bar(B_XFULL + xb), (xph_full >> xb) & 1u, abort_flag, a.err, 6)) { ok = false; break; }
          xph_full ^= 1u << xb;
          asm volatile("tcgen05.fence::after_thread_sync;\n");
          const int nh = n_halves(u, j);
          const bool whole = whole_chunk_group(u, j, a.max_chain);
          const bool wrows = quarter * 32 < u.nterm * u.tm8 * 8;  // warp-uniform: stacked rows here
          for (int h = 0; h < nh && ok; ++h) {
            const uint32_t hb = h2 % NA2;
            if (!mbar_wait<PROF>(bar(B_A2EMPTY + hb), ((h2 / NA2) & 1u) ^ 1u, abort_flag, a.err, 7)) {
              ok = false;
              break;
            }
            ++h2;
            a2 = reinterpret_cast<uint16_t*>(sm + A2_OFF + hb * A2_BYTES);
            // this warp's 32 K-columns are read by the MMA only below 16 * ceil(kw / 16)
            const int kw = half_cols(u, j, h);
            const bool wvalid = wrows && half * 32 < 16 * ((kw + 15) >> 4);
            float v[32];
            if (wvalid) tmem_ld32(tmem + lane_off + xb * 128 + h * 64 + half * 32, v);
            if (h == nh - 1) {
              asm volatile("tcgen05.fence::before_thread_sync;\n");
              __syncwarp();
              if (lane == 0) mbar_arrive(bar(B_XEMPTY + xb));
            }
            if (wvalid) {
              // scale valid columns, zero the rest (K padding of stage 2)
              const int valid = kw - half * 32;
#pragma unroll
              for (int i = 0; i < 32; ++i) v[i] = i < valid ? v[i] * sc : 0.0f;
              write_a2(v);
            } else {  // no stacked rows here (A2 rows that feed only unread D rows) or K columns never read
              __syncwarp();
              if (lane == 0) mbar_arrive(bar(B_A2FULL + hb));
            }
            // flush groups in the order the MMA issues them. The groups of a
            // half are flushed after the next half has been converted (off
            // the MMA's critical path), unless the half has more than two
            // (with two tile accumulators the MMA would then wait for them)
            // or ends its item. One call site keeps the (unrolled) flush code
            // once in the kernel.
            const int F = flush_terms(u, a.max_chain);
            const int ng = whole ? (h == nh - 1 ? 1 : 0) : (u.nterm + F - 1) / F;
            const bool item_end = (fl & TC_ITEM_LAST) && j == n_chunks(u) - 1 && h == nh - 1;
            const bool defer = ng <= 2 && !item_end;
            const int nf = pend + (defer ? 0 : ng);
            for (int g = 0; g < nf && ok; ++g) {
              const bool old = g < pend;
              ok = flush(old ? pend_tm : u.tm, old ? pend_tn : u.tn, old ? pend_fs : fs);
            }
            pend = defer ? ng : 0;
            pend_tm = u.tm;
            pend_tn = u.tn;
            pend_fs = fs;
          }
          ++xcnt;
        }
        if (ok && (fl & TC_ITEM_LAST) && row < u.tm) {  // the item's partial tile
          // fields copied out first: stores through `out` could alias the
          // record as far as the compiler knows
          const int tn = u.tn, nvalid = tn - half * 64;
          double* const orow = out + (long long)row * tn + half * 64;
#pragma unroll
          for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int i = 0; i < 32; ++i)
              if (c * 32 + i < nvalid) orow[c * 32 + i] = (double)ahi[c][i];
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_MEMPTY + slot));
      ++s;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" ::"r"(tmem));
  }
  if (PROF && a.wait_prof && tid < 16) {
    atomicAdd(a.wait_prof + tid, s_wait[tid]);
    if (tid == 0) atomicAdd(a.wait_prof + 16, (unsigned long long)(clock64() - t_start));
  }
}

// ----------------------------------------------------------------- splits
__device__ __forceinline__ void split3(double x, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
  h = __double2bfloat16(x);
  double r1 = x - (double)__bfloat162float(h);
  m = __double2bfloat16(r1);
  double r2 = r1 - (double)__bfloat162float(m);
  l = __double2bfloat16(r2);
}

__global__ void split_ops_kernel(const double* __restrict__ store, const SplitJob* __restrict__ jobs,
                                 long long njobs, __nv_bfloat16* __restrict__ out) {
  for (long long b = blockIdx.x; b < njobs; b += gridDim.x) {
    const SplitJob j = jobs[b];
    const long long n = (long long)j.R8 * j.C8 * 64;
    for (long long e = threadIdx.x; e < n; e += blockDim.x) {
      const long long t = e >> 6;
      const int w = (int)(e & 63);
      const int i = (int)(t / j.C8) * 8 + (w >> 3), c = (int)(t % j.C8) * 8 + (w & 7);
      double x = 0.0;
      if (i < j.rows && c < j.cols) x = (j.src < 0) ? (i == c ? 1.0 : 0.0) : store[j.src + (long long)i * j.cols + c];
      __nv_bfloat16 h, m, l;
      split3(x, h, m, l);
      const long long d = (j.tile + t) * 192 + w;
      out[d] = h;
      out[d + 64] = m;
      out[d + 128] = l;
    }
  }
}

__global__ void split_psi_kernel(const double* __restrict__ psi, const PsiBlock* __restrict__ blocks,
                                 const TcPsiBlock* __restrict__ pb, int nblk, __nv_bfloat16* __restrict__ out) {
  for (int b = blockIdx.x; b < nblk; b += gridDim.x) {
    const TcPsiBlock p = pb[b];
    const long long off = blocks[b].off;
    const long long n = (long long)p.R8 * p.C8 * 64;
    for (long long e = threadIdx.x; e < n; e += blockDim.x) {
      const long long t = e >> 6;
      const int w = (int)(e & 63);
      const int i = (int)(t / p.C8) * 8 + (w >> 3), c = (int)(t % p.C8) * 8 + (w & 7);
      const double x = (i < p.m && c < p.n) ? psi[off + (long long)i * p.n + c] : 0.0;
      __nv_bfloat16 h, m, l;
      split3(x, h, m, l);
      const long long d = (p.tile + t) * 192 + w;
      out[d] = h;
      out[d + 64] = m;
      out[d + 128] = l;
    }
  }
}

void launch_split_ops(const double* store, const SplitJob* jobs, long long njobs, void* out, cudaStream_t st) {
  if (njobs <= 0) return;
  long long grid = njobs < (1ll << 20) ? njobs : (1ll << 20);
  split_ops_kernel<<<(unsigned)grid, 256, 0, st>>>(store, jobs, njobs, (__nv_bfloat16*)out);
}

void launch_split_psi(const double* psi, const PsiBlock* blocks, const TcPsiBlock* pb, int nblk, void* out,
                      cudaStream_t st) {
  if (nblk <= 0) return;
  split_psi_kernel<<<nblk, 256, 0, st>>>(psi, blocks, pb, nblk, (__nv_bfloat16*)out);
}

template <int NPROD, bool F16, int NP>
static void launch_tc_np(const TcDev& a, int grid, cudaStream_t st) {
  constexpr int SMEM = Lay<F16>::SMEM_BYTES;
  set_max_dynamic_smem((const void*)sigma_tc_kernel<NPROD, F16, false, NP>, SMEM);
  set_max_dynamic_smem((const void*)sigma_tc_kernel<NPROD, F16, true, NP>, SMEM);
  if (a.wait_prof)
    sigma_tc_kernel<NPROD, F16, true, NP><<<grid, NTHR, SMEM, st>>>(a);
  else
    sigma_tc_kernel<NPROD, F16, false, NP><<<grid, NTHR, SMEM, st>>>(a);
}

template <int NPROD, bool F16>
static void launch_tc(const TcDev& a, int grid, cudaStream_t st) {
  if (a.producers == NPW)
    launch_tc_np<NPROD, F16, NPW>(a, grid, st);
  else
    launch_tc_np<NPROD, F16, 1>(a, grid, st);
}

void launch_sigma_tc(const TcDev& a, int n_sm, cudaStream_t st) {
  if (a.n_items <= 0) return;
  int grid = n_sm < a.n_items ? n_sm : a.n_items;
  if (grid < 1) grid = 1;
  if (a.f16)
    launch_tc<3, true>(a, grid, st);
  else if (a.nprod == 6)
    launch_tc<6, false>(a, grid, st);
  else
    launch_tc<3, false>(a, grid, st);
}

// Ring stages per unit, counted as the producers fill them. Large blocks
// give units of many K stages, each a long list of copies: the kernel is then
// bound by preparing and issuing stages, and three producer warps fill the
// ring faster; with few stages per unit one producer keeps the stages in
// the order the MMA issuer takes them, which is faster there.
template <bool F16>
static int default_producers(const TcPlan& plan) {
  using L = Lay<F16>;
  long long units = 0, stages = 0;
  for (const TcUnitRec& r : plan.recs) {
    if (r.flags & TC_ZERO) continue;
    ++units;
    for (int j = 0; j < n_chunks(r); ++j) {
      stages += k1_stages<L::KG1>(r);
      for (int h = 0; h < n_halves(r, j); ++h) {
        const int P = max(1, min(r.nterm, L::STAGE_TILES / (tn8e(r) * kg2_of(half_cols(r, j, h)))));
        stages += (r.nterm + P - 1) / P;
      }
    }
  }
  return units > 0 && stages >= 5 * units ? NPW : 1;
}

int tc_default_producers(const TcPlan& plan, bool f16) {
  return f16 ? default_producers<true>(plan) : default_producers<false>(plan);
}

}  // namespace dmrg
