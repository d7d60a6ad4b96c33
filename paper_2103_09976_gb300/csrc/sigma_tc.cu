// Mixed-precision sigma = H_eff . psi on the 5th-generation tensor cores.
//
// Same decomposition as the FP64 path (Sec. II.D-E: a flat list of
// (term, sector) products, summed per output tile, partials reduced in a
// fixed order), with every product
//     S[r0:r0+128, c0:c0+128] += scale * (X_L psi_b) X_R^T
// computed by tcgen05.mma kind::f16 on bf16 slices: each FP64 operand is
// split x = hi + mid + lo (three bf16 numbers, 24 significant bits) and a
// product a*b is taken as the sum of the slice products with i + j <= 2
// (6 MMAs, BF16X3) or i + j <= 1 (3 MMAs, BF16X2), accumulated in FP32 in
// tensor memory. The intermediate X = X_L psi_b never leaves the SM: it is
// read from TMEM, scaled, re-split into bf16 slices and written to shared
// memory as the A operand of the second product.
//
// Warp roles (320 threads): warp 0 streams operator and psi tiles with
// cp.async.bulk into a 3-stage ring; warp 1 issues the MMAs; warps 2-9 are
// the epilogue (two warps per TMEM lane quarter, 32 columns each). Operands are stored in 8x8 core-matrix tiles, so one stored
// block serves as a K-major operand (S) or an MN-major one (S^T) with no
// copy: transposed terms only change the shared-memory descriptors.
//
// Every wait on an mbarrier is bounded (about one second of clock); on a
// timeout the kernel raises a flag in *err, stops issuing work, waits (again
// bounded) for its own copies, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include "kernels.h"

namespace dmrg {

namespace {

constexpr int NEPI = 8;                         // epilogue warps
constexpr int NTHR = 64 + 32 * NEPI;            // producer + MMA + epilogue
constexpr int STAGES = 3;
// Operator and psi tiles are stored slice-interleaved: tile position k holds
// its hi, mid and lo 8x8 bf16 tiles at bytes 384k, 384k+128, 384k+256, in
// global memory and in the stages alike.
constexpr int TILE3 = 384;                      // bytes per tile position (3 slices)
constexpr int STAGE_TILES = 128;                // tile positions per stage
constexpr int STAGE_BYTES = STAGE_TILES * TILE3;  // 48 KB
constexpr int PSI_TILE = 64;                    // psi tiles of a large task's K1 stage start here
constexpr int A2_SLICE = 16 * 1024;             // X chunk: 16 row groups x 8 K groups
constexpr int A2_OFF = STAGES * STAGE_BYTES;
constexpr int NMETA = 16;                       // unit records in the shared-memory ring
constexpr int PREFETCH = 8;                     // records fetched ahead of the producer
constexpr int META_OFF = A2_OFF + 3 * A2_SLICE;
constexpr int BAR_OFF = META_OFF + NMETA * (int)sizeof(TcRec);
constexpr int SLACK_OFF = BAR_OFF + 512;
constexpr int SLACK = 8192;                     // descriptor reads past packed regions stay inside
constexpr int SMEM_BYTES = SLACK_OFF + SLACK;
constexpr long long WAIT_CYCLES = 2000000000ll; // ~1 s at 2 GHz

// barrier slots (8 bytes each)
enum { B_FULL = 0, B_EMPTY = STAGES, B_XFULL = 2 * STAGES, B_XEMPTY = 2 * STAGES + 2,
       B_A2FULL = 2 * STAGES + 4, B_A2EMPTY = 2 * STAGES + 5, B_SFULL = 2 * STAGES + 6,
       B_SEMPTY = 2 * STAGES + 8, B_MFULL = 2 * STAGES + 10, B_MEMPTY = B_MFULL + NMETA,
       B_TMEM = B_MEMPTY + NMETA, B_ABORT = B_TMEM + 1 };
static_assert(8 * (B_ABORT + 1) <= 512, "barrier region");
static_assert(SMEM_BYTES <= 227 * 1024, "shared memory");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ uint32_t idesc_bf16(int n, int a_mn, int b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
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

__device__ __forceinline__ void mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
               "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
               ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
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

// slice products (i, j): i indexes the A slices, j the B slices

__device__ __forceinline__ int rec_k1(const TcRec& r) {
  return (r.flags & UNIT_PACKED) ? 1 : (r.t[0].pR8 + 3) / 4;
}
__device__ __forceinline__ int rec_k2(const TcRec& r) {
  return (r.flags & UNIT_PACKED) ? 1 : (r.width + 63) / 64;
}

// The copies of one stage, distributed over the producer warp: lane `lane`
// calls f(src_tile, operand (0 operator, 1 psi), dst_tile, n_tiles) for its
// own copies only. Every copy moves n_tiles tile positions (all 3 slices).
template <class F>
__device__ __forceinline__ void lane_copies(const TcRec& u, int k1_stage, int k2_stage, int lane, F&& f) {
  const int rg0 = u.r0 / 8, cg0 = u.c0 / 8;
  if (u.flags & UNIT_PACKED) {
    if (k1_stage >= 0) {
      if (lane >= u.ntask) return;
      const TcTaskRec& tk = u.t[lane];
      const int aR8 = tk.aR8, aC8 = tk.aC8;
      if (!(tk.flags & 1)) {
        f(tk.a_tile + (long long)rg0 * aC8, 0, tk.k1a, min(16, aR8 - rg0) * aC8);
      } else {
        const int nmg = min(16, aC8 - rg0);
        if (nmg == aC8) f(tk.a_tile, 0, tk.k1a, aR8 * aC8);
        else
          for (int kg = 0; kg < aR8; ++kg) f(tk.a_tile + (long long)kg * aC8 + rg0, 0, tk.k1a + kg * nmg, nmg);
      }
      if (!(tk.flags & 4)) f(tk.p_tile, 1, tk.k1b, (int)tk.pR8 * tk.pC8);
    } else {
      // unit-wide layout of the K-concatenated right operand: the K groups
      // of task t start at xcol/8
      const int kgu = u.pad[0];
      const bool tB = u.t[0].flags & 2;
      if (!tB) {
        const int nng = min(16, u.t[0].bR8 - cg0);
        for (int j = lane; j < u.ntask * nng; j += 32) {
          const TcTaskRec& tk = u.t[j / nng];
          const int ng = j % nng;
          f(tk.b_tile + (long long)(cg0 + ng) * tk.bC8, 0, ng * kgu + tk.xcol / 8, tk.bC8);
        }
      } else {
        if (lane >= u.ntask) return;
        const TcTaskRec& tk = u.t[lane];
        const int bR8 = tk.bR8, bC8 = tk.bC8, nng = min(16, bC8 - cg0), kx = tk.xcol / 8;
        if (nng == bC8) f(tk.b_tile, 0, kx * nng, bR8 * bC8);
        else
          for (int kg = 0; kg < bR8; ++kg) f(tk.b_tile + (long long)kg * bC8 + cg0, 0, (kx + kg) * nng, nng);
      }
    }
    return;
  }
  const TcTaskRec& tk = u.t[0];
  const int aR8 = tk.aR8, aC8 = tk.aC8, bR8 = tk.bR8, bC8 = tk.bC8, pR8 = tk.pR8, pC8 = tk.pC8;
  const bool tA = tk.flags & 1, tB = tk.flags & 2;
  if (k1_stage >= 0) {  // one K chunk (4 K groups) of a large task
    const int kg0 = 4 * k1_stage;
    const int nA = !tA ? min(16, aR8 - rg0) : min(4, aR8 - kg0);
    const int nB = min(4, pR8 - kg0);
    if (lane < nA) {
      if (!tA) f(tk.a_tile + (long long)(rg0 + lane) * aC8 + kg0, 0, lane * 4, min(4, aC8 - kg0));
      else f(tk.a_tile + (long long)(kg0 + lane) * aC8 + rg0, 0, lane * 16, min(16, aC8 - rg0));
    } else if (lane < nA + nB) {
      const int r = lane - nA;
      f(tk.p_tile + (long long)(kg0 + r) * pC8 + u.pass * 16, 1, PSI_TILE + r * 16, min(16, pC8 - u.pass * 16));
    }
  } else {  // one 64-column K chunk of the second product of a large task
    const int kgx = u.pass * 16 + k2_stage * 8;
    if (!tB) {
      if (lane < min(16, bR8 - cg0)) f(tk.b_tile + (long long)(cg0 + lane) * bC8 + kgx, 0, lane * 8, min(8, bC8 - kgx));
    } else {
      if (lane < min(8, bR8 - kgx)) f(tk.b_tile + (long long)(kgx + lane) * bC8 + cg0, 0, lane * 16, min(16, bC8 - cg0));
    }
  }
}

}  // namespace

// Slice pair of product p (i + j <= 2 ordering: hh, hm, mh, hl, mm, lh).
__device__ __forceinline__ constexpr int prod_i(int p) { return (p == 2 || p == 4) ? 1 : (p == 5 ? 2 : 0); }
__device__ __forceinline__ constexpr int prod_j(int p) { return (p == 1 || p == 4) ? 1 : (p == 3 ? 2 : 0); }

// One K chain of slice products into tmem_d. Descriptors differ only in the
// start-address field, so each MMA adds its byte offset >> 4 to a base.
template <int NPROD>
__device__ __forceinline__ void mma_chain(uint32_t tmem_d, uint64_t ad0, uint64_t bd0, uint32_t a_slice,
                                          uint32_t b_slice, uint32_t a_kstep, uint32_t b_kstep, int nks,
                                          uint32_t idesc, bool acc_first) {
  for (int ks = 0; ks < nks; ++ks) {
#pragma unroll
    for (int p = 0; p < NPROD; ++p) {
      const uint64_t ad = ad0 + ((prod_i(p) * a_slice + (uint32_t)ks * a_kstep) >> 4);
      const uint64_t bd = bd0 + ((prod_j(p) * b_slice + (uint32_t)ks * b_kstep) >> 4);
      mma(tmem_d, ad, bd, idesc, (acc_first || ks > 0 || p > 0) ? 1u : 0u);
    }
  }
}

// PROF: record wait accounting and MMA-thread cycles into a.wait_prof.
template <int NPROD, bool PROF>
__global__ void __launch_bounds__(NTHR, 1) sigma_tc_kernel(TcDev a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t sbase = smem_u32(sm);
  const uint32_t bars = sbase + BAR_OFF;
  auto bar = [&](int k) { return bars + 8u * (uint32_t)k; };
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + BAR_OFF + 8 * B_ABORT);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + BAR_OFF + 8 * B_TMEM);
  TcRec* ring = reinterpret_cast<TcRec*>(sm + META_OFF);

  const long long t_start = clock64();
  if (tid < 16) s_wait[tid] = 0ull;
  // zero all operand buffers once: afterwards shared memory only ever holds
  // finite operand data or zeros, so padded K positions multiply to 0 and
  // padded rows stay finite.
  for (int i = tid; i < META_OFF / 16; i += NTHR) reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
  for (int i = tid; i < SLACK / 16; i += NTHR) reinterpret_cast<uint4*>(sm + SLACK_OFF)[i] = make_uint4(0, 0, 0, 0);
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
    mbar_init(bar(B_A2FULL), NEPI);
    mbar_init(bar(B_A2EMPTY), 1);
    for (int m = 0; m < NMETA; ++m) {
      mbar_init(bar(B_MFULL + m), 1);
      mbar_init(bar(B_MEMPTY + m), 2 + NEPI);  // producer + MMA + epilogue warps
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

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    uint32_t stage = 0, phase = 1;  // empty barriers: first wait passes
    bool ok = true;
    const char* const ops = (const char*)a.op;
    const char* const ps = (const char*)a.psi;
    auto produce = [&](const TcRec& u, int k1, int k2) {
      if (!ok) return;
      if (!mbar_wait<PROF>(bar(B_EMPTY + stage), phase, abort_flag, a.err, 1)) { ok = false; return; }
      uint32_t tiles = 0;
      lane_copies(u, k1, k2, lane, [&](long long, int, int, int n) { tiles += (uint32_t)n; });
      tiles = __reduce_add_sync(0xffffffffu, tiles);
      if (lane == 0) mbar_expect_tx(bar(B_FULL + stage), (uint32_t)TILE3 * tiles);
      __syncwarp();
      const uint32_t sdst = sbase + stage * STAGE_BYTES;
      lane_copies(u, k1, k2, lane, [&](long long src, int which, int dst, int n) {
        bulk_g2s(sdst + (uint32_t)dst * TILE3, (which ? ps : ops) + src * TILE3, (uint32_t)TILE3 * (uint32_t)n,
                 bar(B_FULL + stage));
      });
      if (++stage == STAGES) { stage = 0; phase ^= 1; }
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
        pf_r = a.item_rec[it];
        pf_end = a.item_rec[it + 1];
      }
      const int slot = (int)(pf_s % NMETA);
      const uint32_t par = (uint32_t)(((pf_s / NMETA) & 1) ^ 1);
      if (!mbar_wait<PROF>(bar(B_MEMPTY + slot), par, abort_flag, a.err, 9)) { ok = false; return false; }
      if (lane == 0) {
        mbar_expect_tx(bar(B_MFULL + slot), (uint32_t)sizeof(TcRec));
        bulk_g2s(smem_u32(ring + slot), a.recs + pf_r, (uint32_t)sizeof(TcRec), bar(B_MFULL + slot));
      }
      __syncwarp();
      ++pf_r;
      ++pf_s;
      return true;
    };
    long long s = 0;
    int prev_slot = -1;
    for (;;) {
      while (ok && pf_s < s + PREFETCH && prefetch_one()) {
      }
      if (!ok) break;
      if (s == pf_s) break;  // nothing left
      const int slot = (int)(s % NMETA);
      if (!mbar_wait<PROF>(bar(B_MFULL + slot), (uint32_t)((s / NMETA) & 1), abort_flag, a.err, 10)) { ok = false; break; }
      const TcRec& u = ring[slot];
      if (!(u.flags & REC_ZERO))
        for (int k = 0; k < rec_k1(u); ++k) produce(u, k, -1);
      if (prev_slot >= 0) {
        const TcRec& pu = ring[prev_slot];
        for (int h = 0; h < rec_k2(pu); ++h) produce(pu, -1, h);
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(B_MEMPTY + prev_slot));
      }
      if (u.flags & REC_ZERO) {
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(B_MEMPTY + slot));
        prev_slot = -1;
      } else {
        prev_slot = slot;
      }
      ++s;
    }
    if (ok && prev_slot >= 0) {
      const TcRec& pu = ring[prev_slot];
      for (int h = 0; h < rec_k2(pu); ++h) produce(pu, -1, h);
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_MEMPTY + prev_slot));
    }
    // terminator record
    if (ok) {
      const int slot = (int)(s % NMETA);
      const uint32_t par = (uint32_t)(((s / NMETA) & 1) ^ 1);
      if (mbar_wait<PROF>(bar(B_MEMPTY + slot), par, abort_flag, a.err, 11)) {
        if (lane == 0) {
          ring[slot].flags = REC_DONE;
          mbar_arrive(bar(B_MFULL + slot));
        }
      }
    }
    __syncwarp();
    // drain: wait (bounded) until the MMA side released every stage we filled
    for (int k = 0; k < STAGES; ++k) {
      mbar_wait<PROF>(bar(B_EMPTY + stage), phase, abort_flag, a.err, 0);
      if (++stage == STAGES) { stage = 0; phase ^= 1; }
    }
  } else if (warp == 1) {
    // --------------------------------------------------------------- MMA
    if (lane == 0) {
      // with profiling on, slots 14 / 15 of the wait accounting receive the
      // cycles this thread spends issuing MMAs / committing them
      constexpr bool prof = PROF;
      auto tick = [&]() -> long long { return prof ? clock64() : 0ll; };
      auto tock = [&](int slot, long long t0) {
        if (prof) s_wait[slot] += (unsigned long long)(clock64() - t0);
      };
      uint32_t stage = 0, phase = 0;
      uint32_t xcnt = 0, xph_empty = 3u;   // bit b: expected parity of X-empty[b]
      uint32_t a2_full_ph = 0;
      uint32_t sb = 0, sph_empty = 3u;     // bit b: expected parity of S-empty[b]
      bool seg_open = false, ok = true;
      auto acquire = [&]() -> uint32_t {
        if (!mbar_wait<PROF>(bar(B_FULL + stage), phase, abort_flag, a.err, 4)) { ok = false; return 0; }
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        return sbase + stage * STAGE_BYTES;
      };
      auto release = [&]() {
        const long long t0 = tick();
        commit(bar(B_EMPTY + stage));
        tock(15, t0);
        if (++stage == STAGES) { stage = 0; phase ^= 1; }
      };
      auto mma_k1 = [&](const TcRec& u) {
        const uint32_t xb = xcnt & 1;
        if (!mbar_wait<PROF>(bar(B_XEMPTY + xb), (xph_empty >> xb) & 1u, abort_flag, a.err, 3)) { ok = false; return; }
        xph_empty ^= 1u << xb;
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        const uint32_t tmem_x = tmem + xb * 128;
        if (u.flags & UNIT_PACKED) {
          const uint32_t sst = acquire();
          if (!ok) return;
          const int rg0 = u.r0 / 8;
          for (int t = 0; t < u.ntask; ++t) {
            const TcTaskRec& tk = u.t[t];
            const int tA = tk.flags & 1;
            const int aC8 = tk.aC8, pC8 = tk.pC8;
            const int n16 = 16 * ((tk.pn + 15) / 16);
            const uint32_t a_lbo = tA ? (uint32_t)min(16, aC8 - rg0) * TILE3 : TILE3;
            const uint32_t a_sbo = tA ? TILE3 : (uint32_t)aC8 * TILE3;
            const uint32_t b_lbo = (uint32_t)pC8 * TILE3;
            const long long t0 = tick();
            mma_chain<NPROD>(tmem_x + tk.xcol, sdesc(sst + tk.k1a * TILE3, a_lbo, a_sbo),
                             sdesc(sst + tk.k1b * TILE3, b_lbo, TILE3), 128u, 128u, 2 * a_lbo, 2 * b_lbo,
                             tk.pR8 / 2, idesc_bf16(n16, tA, 1), false);
            tock(14, t0);
          }
          release();
        } else {
          const TcTaskRec& tk = u.t[0];
          const int tA = tk.flags & 1;
          const uint32_t id1 = idesc_bf16(16 * ((u.width + 15) / 16), tA, 1);
          const uint32_t a_lbo = tA ? 16u * TILE3 : TILE3, a_sbo = tA ? TILE3 : 4u * TILE3;
          const int pR8 = tk.pR8, nk = (pR8 + 3) / 4;
          for (int k = 0; k < nk && ok; ++k) {
            const uint32_t sst = acquire();
            if (!ok) return;
            const long long t0 = tick();
            mma_chain<NPROD>(tmem_x, sdesc(sst, a_lbo, a_sbo), sdesc(sst + PSI_TILE * TILE3, 16u * TILE3, TILE3),
                             128u, 128u, 2 * a_lbo, 2 * 16u * TILE3, min(4, pR8 - 4 * k) / 2, id1, k > 0);
            tock(14, t0);
            release();
          }
        }
        {
          const long long t0 = tick();
          commit(bar(B_XFULL + xb));
          tock(15, t0);
        }
        ++xcnt;
      };
      auto mma_k2 = [&](const TcRec& u) {
        const uint32_t id_n = (uint32_t)(16 * ((u.ncols + 15) / 16));
        const uint32_t a2 = sbase + A2_OFF;
        const int nk2 = rec_k2(u);
        for (int h = 0; h < nk2 && ok; ++h) {
          if (!mbar_wait<PROF>(bar(B_A2FULL), a2_full_ph, abort_flag, a.err, 5)) { ok = false; return; }
          a2_full_ph ^= 1;
          if (!seg_open) {
            if (!mbar_wait<PROF>(bar(B_SEMPTY + sb), (sph_empty >> sb) & 1u, abort_flag, a.err, 2)) { ok = false; return; }
            sph_empty ^= 1u << sb;
          }
          const uint32_t sst = acquire();
          if (!ok) return;
          const uint32_t tmem_s = tmem + 256 + sb * 128;
          const int tB = (u.t[0].flags >> 1) & 1;
          const uint32_t id2 = idesc_bf16((int)id_n, 0, tB);
          uint32_t b_lbo, b_sbo;
          int nks;
          if (u.flags & UNIT_PACKED) {  // one K-concatenated chain for all tasks of the unit
            const int nng = min(16, u.t[0].bC8 - u.c0 / 8);
            b_lbo = tB ? (uint32_t)nng * TILE3 : TILE3;
            b_sbo = tB ? TILE3 : (uint32_t)u.pad[0] * TILE3;
            nks = u.width / 16;
          } else {
            b_lbo = tB ? 16u * TILE3 : TILE3;
            b_sbo = tB ? TILE3 : 8u * TILE3;
            nks = (min(64, u.width - h * 64) + 15) / 16;
          }
          const long long t0 = tick();
          mma_chain<NPROD>(tmem_s, sdesc(a2, 128u, 1024u), sdesc(sst, b_lbo, b_sbo), A2_SLICE, 128u, 2 * 128u,
                           2 * b_lbo, nks, id2, seg_open);
          tock(14, t0);
          seg_open = true;
          release();
          const long long t1 = tick();
          commit(bar(B_A2EMPTY));
          tock(15, t1);
        }
        if (ok && (u.flags & UNIT_ENDS_SEGMENT)) {
          commit(bar(B_SFULL + sb));
          sb ^= 1;
          seg_open = false;
        }
      };
      long long s = 0;
      int prev_slot = -1;
      while (ok) {
        const int slot = (int)(s % NMETA);
        if (!mbar_wait<PROF>(bar(B_MFULL + slot), (uint32_t)((s / NMETA) & 1), abort_flag, a.err, 12)) { ok = false; break; }
        const TcRec& u = ring[slot];
        const int fl = u.flags;
        if (fl & REC_DONE) break;
        if (!(fl & REC_ZERO)) mma_k1(u);
        if (prev_slot >= 0 && ok) {
          mma_k2(ring[prev_slot]);
          mbar_arrive(bar(B_MEMPTY + prev_slot));
        }
        if (fl & REC_ZERO) {
          mbar_arrive(bar(B_MEMPTY + slot));
          prev_slot = -1;
        } else {
          prev_slot = slot;
        }
        ++s;
      }
      if (ok && prev_slot >= 0) {
        mma_k2(ring[prev_slot]);
        mbar_arrive(bar(B_MEMPTY + prev_slot));
      }
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------- epilogue
    const int e = warp - 2;                    // 0 .. NEPI-1
    const int quarter = warp & 3;              // TMEM lanes 32*quarter .. +31
    const int half = e >> 2;                   // columns 32*half of each 64-column chunk
    const int row = quarter * 32 + lane;       // output / X row owned by this thread
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    uint32_t xcnt = 0, xph_full = 0;    // bit b: expected parity of X-full[b]
    uint32_t a2_empty_ph = 1;
    uint32_t sb = 0, sph_full = 0;      // bit b: expected parity of S-full[b]
    bool ok = true;
    __nv_bfloat16* a2 = reinterpret_cast<__nv_bfloat16*>(sm + A2_OFF);
    // write 32 K-columns (half of a 64-column chunk) of A2 for this row
    auto write_a2 = [&](const float* v) {
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        uint32_t hw[4], mw[4], lw[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          // two columns at a time: one paired round-to-nearest conversion per
          // slice; a bf16 value is the upper half of its float, so the
          // residuals need only a mask or a shift and a subtraction
          const float x0 = v[g * 8 + 2 * q], x1 = v[g * 8 + 2 * q + 1];
          const uint32_t hp = bf16x2_bits(x0, x1);
          const float r0 = x0 - __uint_as_float(hp << 16), r1 = x1 - __uint_as_float(hp & 0xFFFF0000u);
          const uint32_t mp = bf16x2_bits(r0, r1);
          const float s0 = r0 - __uint_as_float(mp << 16), s1 = r1 - __uint_as_float(mp & 0xFFFF0000u);
          hw[q] = hp;
          mw[q] = mp;
          lw[q] = bf16x2_bits(s0, s1);
        }
        const int off = (((row >> 3) * 8 + half * 4 + g) * 64 + (row & 7) * 8);
        *reinterpret_cast<uint4*>(a2 + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4*>(a2 + A2_SLICE / 2 + off) = make_uint4(mw[0], mw[1], mw[2], mw[3]);
        *reinterpret_cast<uint4*>(a2 + A2_SLICE + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
      }
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_A2FULL));
    };
    long long s = 0;
    while (ok) {
      const int slot = (int)(s % NMETA);
      if (!mbar_wait<PROF>(bar(B_MFULL + slot), (uint32_t)((s / NMETA) & 1), abort_flag, a.err, 13)) { ok = false; break; }
      const TcRec& u = ring[slot];
      const int fl = u.flags;
      if (fl & REC_DONE) break;
      double* out = a.scratch + u.slot;
      if (fl & REC_ZERO) {
        if (row < u.nrows)
          for (int c = half * 64; c < min(u.ncols, half * 64 + 64); ++c) out[(long long)row * u.ncols + c] = 0.0;
      } else {
        const uint32_t xb = xcnt & 1;
        if (!mbar_wait<PROF>(bar(B_XFULL + xb), (xph_full >> xb) & 1u, abort_flag, a.err, 6)) { ok = false; break; }
        xph_full ^= 1u << xb;
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        const uint32_t xaddr = tmem + lane_off + xb * 128;
        float v[32];
        const int nh = (fl & UNIT_PACKED) ? 1 : (u.width + 63) / 64;
        for (int h = 0; h < nh; ++h) {
          tmem_ld32(xaddr + h * 64 + half * 32, v);
          if (h == nh - 1) {
            asm volatile("tcgen05.fence::before_thread_sync;\n");
            __syncwarp();
            if (lane == 0) mbar_arrive(bar(B_XEMPTY + xb));
          }
          // scale valid columns, zero the rest (K padding of the second product)
          const int c0 = h * 64 + half * 32;
          if (fl & UNIT_PACKED) {
            float cs[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) cs[j] = 0.0f;
            for (int t = 0; t < u.ntask; ++t) {
              const int x0 = u.t[t].xcol - c0, x1 = x0 + u.t[t].pn;
              const float sc = u.t[t].scale;
#pragma unroll
              for (int j = 0; j < 32; ++j)
                if (j >= x0 && j < x1) cs[j] = sc;
            }
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = cs[j] != 0.0f ? v[j] * cs[j] : 0.0f;
          } else {
            const float sc = u.t[0].scale;
            const int valid = u.width - c0;
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = j < valid ? v[j] * sc : 0.0f;
          }
          if (!mbar_wait<PROF>(bar(B_A2EMPTY), a2_empty_ph, abort_flag, a.err, 7)) { ok = false; break; }
          a2_empty_ph ^= 1;
          write_a2(v);
        }
        ++xcnt;
        if (!ok) break;
        if (fl & UNIT_ENDS_SEGMENT) {
          // segment's FP32 sigma tile -> FP64 slot (store on the first segment, add after)
          if (!mbar_wait<PROF>(bar(B_SFULL + sb), (sph_full >> sb) & 1u, abort_flag, a.err, 8)) { ok = false; break; }
          sph_full ^= 1u << sb;
          asm volatile("tcgen05.fence::after_thread_sync;\n");
          const bool first = fl & UNIT_FIRST_SEGMENT;
          for (int c0 = half * 64; c0 < min(u.ncols, half * 64 + 64); c0 += 32) {
            float w[32];
            tmem_ld32(tmem + lane_off + 256 + sb * 128 + c0, w);
            if (row < u.nrows) {
              const int nc = min(32, u.ncols - c0);
              double* o = out + (long long)row * u.ncols + c0;
#pragma unroll
              for (int c = 0; c < 32; ++c)
                if (c < nc) o[c] = first ? (double)w[c] : o[c] + (double)w[c];
            }
          }
          asm volatile("tcgen05.fence::before_thread_sync;\n");
          __syncwarp();
          if (lane == 0) mbar_arrive(bar(B_SEMPTY + sb));
          sb ^= 1;
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

void launch_sigma_tc(const TcDev& a, int n_sm, cudaStream_t st) {
  set_max_dynamic_smem((const void*)sigma_tc_kernel<6, false>, SMEM_BYTES);
  set_max_dynamic_smem((const void*)sigma_tc_kernel<3, false>, SMEM_BYTES);
  set_max_dynamic_smem((const void*)sigma_tc_kernel<6, true>, SMEM_BYTES);
  set_max_dynamic_smem((const void*)sigma_tc_kernel<3, true>, SMEM_BYTES);
  int grid = n_sm < a.n_items ? n_sm : a.n_items;
  if (grid < 1) grid = 1;
  const bool prof = a.wait_prof != nullptr;
  if (a.nprod == 6) {
    if (prof)
      sigma_tc_kernel<6, true><<<grid, NTHR, SMEM_BYTES, st>>>(a);
    else
      sigma_tc_kernel<6, false><<<grid, NTHR, SMEM_BYTES, st>>>(a);
  } else {
    if (prof)
      sigma_tc_kernel<3, true><<<grid, NTHR, SMEM_BYTES, st>>>(a);
    else
      sigma_tc_kernel<3, false><<<grid, NTHR, SMEM_BYTES, st>>>(a);
  }
}

}  // namespace dmrg
