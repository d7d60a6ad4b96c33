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
// Warp roles (192 threads): warp 0 streams operator and psi tiles with
// cp.async.bulk into a 3-stage ring; warp 1 issues the MMAs; warps 2-5 are
// the epilogue. Operands are stored in 8x8 core-matrix tiles, so one stored
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

constexpr int NTHR = 192;
constexpr int STAGES = 3;
constexpr int SLICE_BYTES = 16 * 1024;          // one slice of a stage
constexpr int STAGE_BYTES = 3 * SLICE_BYTES;    // 48 KB
constexpr int PSI_OFF = 8 * 1024;               // psi tile inside a K1 stage slice
constexpr int A2_SLICE = 16 * 1024;             // X chunk: 16 row groups x 8 K groups
constexpr int A2_BYTES = 3 * A2_SLICE;
constexpr int BAR_OFF = STAGES * STAGE_BYTES + A2_BYTES;
constexpr int SMEM_BYTES = BAR_OFF + 256;
constexpr long long WAIT_CYCLES = 2000000000ll;  // ~1 s at 2 GHz

// barrier slots (8 bytes each) after the operand buffers
enum { B_FULL = 0, B_EMPTY = STAGES, B_XFULL = 2 * STAGES, B_XEMPTY = 2 * STAGES + 2,
       B_A2FULL = 2 * STAGES + 4, B_A2EMPTY = 2 * STAGES + 5, B_SFULL = 2 * STAGES + 6,
       B_SEMPTY = 2 * STAGES + 8, B_TMEM = 2 * STAGES + 10, B_ABORT = 2 * STAGES + 11 };

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

// Bounded wait; returns false (and raises the abort flag) on timeout or if
// another role already aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          int* err, int code) {
  if (mbar_try(bar, parity)) return true;
  long long t0 = clock64();
  for (;;) {
    if (mbar_try(bar, parity)) return true;
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
__constant__ int c_prod_i[6] = {0, 0, 1, 0, 1, 2};
__constant__ int c_prod_j[6] = {0, 1, 0, 2, 1, 0};

// Geometry of the stages of one task pass, shared by all roles.
struct Pass {
  int n1;       // valid X columns in this pass (<= 128)
  int nk1;      // K1 stages
  int nh;       // K2 stages (64-column sub-chunks)
};

__device__ __forceinline__ Pass pass_geom(const TcPsiBlock& ib, int pass) {
  Pass p;
  p.n1 = min(128, ib.n - pass * 128);
  p.nk1 = (ib.R8 + 3) / 4;
  p.nh = (p.n1 + 63) / 64;
  return p;
}

}  // namespace

__global__ void __launch_bounds__(NTHR, 1) sigma_tc_kernel(TcDev a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t sbase = smem_u32(sm);
  const uint32_t bars = sbase + BAR_OFF;
  auto bar = [&](int k) { return bars + 8u * (uint32_t)k; };
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + BAR_OFF + 8 * B_ABORT);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + BAR_OFF + 8 * B_TMEM);

  // zero all operand buffers once: afterwards shared memory only ever holds
  // finite operand data or zeros, so padded K positions multiply to 0.
  for (int i = tid; i < BAR_OFF / 16; i += NTHR) reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(bar(B_FULL + s), 1);
      mbar_init(bar(B_EMPTY + s), 1);
    }
    for (int x = 0; x < 2; ++x) {
      mbar_init(bar(B_XFULL + x), 1);
      mbar_init(bar(B_XEMPTY + x), 4);
      mbar_init(bar(B_SFULL + x), 1);
      mbar_init(bar(B_SEMPTY + x), 4);
    }
    mbar_init(bar(B_A2FULL), 4);
    mbar_init(bar(B_A2EMPTY), 1);
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
  const int nprod = a.nprod;
  const int nsl = nprod == 6 ? 3 : 2;  // slices read per operand

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    uint32_t stage = 0, phase = 1;  // empty barriers: first wait passes
    const char* ops[3] = {(const char*)a.op[0], (const char*)a.op[1], (const char*)a.op[2]};
    const char* ps[3] = {(const char*)a.psi[0], (const char*)a.psi[1], (const char*)a.psi[2]};
    bool ok = true;
    for (int q = blockIdx.x; q < a.n_items && ok; q += gridDim.x) {
      const TcItem it = a.items[a.schedule[q]];
      for (int t = it.t_begin; t < it.t_end && ok; ++t) {
        const TcTask tk = a.tasks[t];
        const TcPsiBlock ib = a.pblk[tk.in_blk];
        const bool tA = tk.flags & 1, tB = tk.flags & 2;
        const int npass = (ib.n + 127) / 128;
        for (int pass = 0; pass < npass && ok; ++pass) {
          const Pass pg = pass_geom(ib, pass);
          for (int k = 0; k < pg.nk1 + pg.nh && ok; ++k) {
            if (!mbar_wait(bar(B_EMPTY + stage), phase, abort_flag, a.err, 1)) { ok = false; break; }
            const uint32_t sdst = sbase + stage * STAGE_BYTES;
            int nA, tilesA, nB, tilesB;
            if (k < pg.nk1) {  // K1: left operator rows x K chunk, psi K chunk x pass columns
              const int kg0 = 4 * k;
              const int rg0 = it.r0 / 8;
              if (!tA) { nA = min(16, tk.aR8 - rg0); tilesA = min(4, tk.aC8 - kg0); }
              else     { nA = min(4, tk.aR8 - kg0);  tilesA = min(16, tk.aC8 - rg0); }
              nB = min(4, ib.R8 - kg0);
              tilesB = min(16, ib.C8 - pass * 16);
            } else {           // K2: right operator K chunk x output columns
              const int h = k - pg.nk1;
              const int kgx = pass * 16 + h * 8;
              const int cg0 = it.c0 / 8;
              if (!tB) { nA = min(16, tk.bR8 - cg0); tilesA = min(8, tk.bC8 - kgx); }
              else     { nA = min(8, tk.bR8 - kgx);  tilesA = min(16, tk.bC8 - cg0); }
              nB = 0;
              tilesB = 0;
            }
            const uint32_t bytes = (uint32_t)nsl * 128u * (uint32_t)(nA * tilesA + nB * tilesB);
            if (lane == 0) mbar_expect_tx(bar(B_FULL + stage), bytes);
            __syncwarp();
            const int per_slice = nA + nB;
            for (int j = lane; j < nsl * per_slice; j += 32) {
              const int s = j / per_slice, r = j % per_slice;
              const uint32_t slice_dst = sdst + s * SLICE_BYTES;
              if (k < pg.nk1) {
                const int kg0 = 4 * k, rg0 = it.r0 / 8;
                if (r < nA) {
                  long long src_tile;
                  uint32_t dst;
                  if (!tA) { src_tile = tk.a_tile + (long long)(rg0 + r) * tk.aC8 + kg0; dst = slice_dst + (r * 4) * 128; }
                  else     { src_tile = tk.a_tile + (long long)(kg0 + r) * tk.aC8 + rg0; dst = slice_dst + (r * 16) * 128; }
                  bulk_g2s(dst, ops[s] + src_tile * 128, 128u * tilesA, bar(B_FULL + stage));
                } else {
                  const int rr = r - nA;
                  long long src_tile = ib.tile + (long long)(kg0 + rr) * ib.C8 + pass * 16;
                  bulk_g2s(slice_dst + PSI_OFF + (rr * 16) * 128, ps[s] + src_tile * 128, 128u * tilesB,
                           bar(B_FULL + stage));
                }
              } else {
                const int h = k - pg.nk1;
                const int kgx = pass * 16 + h * 8, cg0 = it.c0 / 8;
                long long src_tile;
                uint32_t dst;
                if (!tB) { src_tile = tk.b_tile + (long long)(cg0 + r) * tk.bC8 + kgx; dst = slice_dst + (r * 8) * 128; }
                else     { src_tile = tk.b_tile + (long long)(kgx + r) * tk.bC8 + cg0; dst = slice_dst + (r * 16) * 128; }
                bulk_g2s(dst, ops[s] + src_tile * 128, 128u * tilesA, bar(B_FULL + stage));
              }
            }
            if (++stage == STAGES) { stage = 0; phase ^= 1; }
          }
        }
      }
    }
    // drain: wait (bounded) until the MMA side released every stage we filled
    for (int s = 0; s < STAGES; ++s) {
      mbar_wait(bar(B_EMPTY + stage), phase, abort_flag, a.err, 0);
      if (++stage == STAGES) { stage = 0; phase ^= 1; }
    }
  } else if (warp == 1) {
    // --------------------------------------------------------------- MMA
    if (lane == 0) {
      uint32_t stage = 0, phase = 0;
      uint32_t xb = 0, xph_empty[2] = {1, 1};
      uint32_t a2_full_ph = 0;
      uint32_t sb = 0, sph_empty[2] = {1, 1};
      bool ok = true;
      for (int q = blockIdx.x; q < a.n_items && ok; q += gridDim.x) {
        const TcItem it = a.items[a.schedule[q]];
        if (it.t_begin == it.t_end) continue;
        bool first_s = true;
        const uint32_t tmem_s = tmem + 256 + sb * 128;
        if (!mbar_wait(bar(B_SEMPTY + sb), sph_empty[sb], abort_flag, a.err, 2)) { ok = false; break; }
        sph_empty[sb] ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        const int n2 = 16 * ((it.ncols + 15) / 16);
        for (int t = it.t_begin; t < it.t_end && ok; ++t) {
          const TcTask tk = a.tasks[t];
          const TcPsiBlock ib = a.pblk[tk.in_blk];
          const int tA = tk.flags & 1, tB = (tk.flags >> 1) & 1;
          const int npass = (ib.n + 127) / 128;
          for (int pass = 0; pass < npass && ok; ++pass) {
            const Pass pg = pass_geom(ib, pass);
            const uint32_t tmem_x = tmem + xb * 128;
            if (!mbar_wait(bar(B_XEMPTY + xb), xph_empty[xb], abort_flag, a.err, 3)) { ok = false; break; }
            xph_empty[xb] ^= 1;
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            const int n1 = 16 * ((pg.n1 + 15) / 16);
            const uint32_t id1 = idesc_bf16(n1, tA, 1);
            const uint32_t a_lbo = tA ? 2048u : 128u, a_sbo = tA ? 128u : 512u;
            for (int k = 0; k < pg.nk1 + pg.nh; ++k) {
              if (!mbar_wait(bar(B_FULL + stage), phase, abort_flag, a.err, 4)) { ok = false; break; }
              asm volatile("tcgen05.fence::after_thread_sync;\n");
              const uint32_t sst = sbase + stage * STAGE_BYTES;
              if (k < pg.nk1) {
                const int nks = min(4, ib.R8 - 4 * k) / 2;
                for (int ks = 0; ks < nks; ++ks)
                  for (int p = 0; p < nprod; ++p) {
                    const uint32_t aa = sst + c_prod_i[p] * SLICE_BYTES + ks * 2 * a_lbo;
                    const uint32_t bb = sst + c_prod_j[p] * SLICE_BYTES + PSI_OFF + ks * 2 * 2048u;
                    mma(tmem_x, sdesc(aa, a_lbo, a_sbo), sdesc(bb, 2048u, 128u), id1,
                        (k > 0 || ks > 0 || p > 0) ? 1u : 0u);
                  }
                commit(bar(B_EMPTY + stage));
                if (k == pg.nk1 - 1) commit(bar(B_XFULL + xb));
              } else {
                const int h = k - pg.nk1;
                const int valid = min(64, pg.n1 - h * 64);
                const int nks = (valid + 15) / 16;
                if (!mbar_wait(bar(B_A2FULL), a2_full_ph, abort_flag, a.err, 5)) { ok = false; break; }
                a2_full_ph ^= 1;
                asm volatile("tcgen05.fence::after_thread_sync;\n");
                const uint32_t id2 = idesc_bf16(n2, 0, tB);
                const uint32_t b_lbo = tB ? 2048u : 128u, b_sbo = tB ? 128u : 1024u;
                const uint32_t a2 = sbase + STAGES * STAGE_BYTES;
                for (int ks = 0; ks < nks; ++ks)
                  for (int p = 0; p < nprod; ++p) {
                    const uint32_t aa = a2 + c_prod_i[p] * A2_SLICE + ks * 2 * 128u;
                    const uint32_t bb = sst + c_prod_j[p] * SLICE_BYTES + ks * 2 * b_lbo;
                    mma(tmem_s, sdesc(aa, 128u, 1024u), sdesc(bb, b_lbo, b_sbo), id2,
                        (!first_s || ks > 0 || p > 0) ? 1u : 0u);
                  }
                first_s = false;
                commit(bar(B_EMPTY + stage));
                commit(bar(B_A2EMPTY));
              }
              if (++stage == STAGES) { stage = 0; phase ^= 1; }
            }
            xb ^= 1;
          }
        }
        if (!ok) break;
        commit(bar(B_SFULL + sb));
        sb ^= 1;
      }
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------- epilogue
    const int quarter = warp & 3;              // TMEM lanes 32*quarter .. +31
    const int row = quarter * 32 + lane;       // output / X row owned by this thread
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    uint32_t xb = 0, xph_full[2] = {0, 0};
    uint32_t a2_empty_ph = 1;
    uint32_t sb = 0, sph_full[2] = {0, 0};
    bool ok = true;
    __nv_bfloat16* a2 = reinterpret_cast<__nv_bfloat16*>(sm + STAGES * STAGE_BYTES);
    for (int q = blockIdx.x; q < a.n_items && ok; q += gridDim.x) {
      const TcItem it = a.items[a.schedule[q]];
      double* out = a.scratch + it.slot;
      if (it.t_begin == it.t_end) {
        if (row < it.nrows)
          for (int c = 0; c < it.ncols; ++c) out[(long long)row * it.ncols + c] = 0.0;
        continue;
      }
      for (int t = it.t_begin; t < it.t_end && ok; ++t) {
        const TcTask tk = a.tasks[t];
        const TcPsiBlock ib = a.pblk[tk.in_blk];
        const int npass = (ib.n + 127) / 128;
        for (int pass = 0; pass < npass && ok; ++pass) {
          const Pass pg = pass_geom(ib, pass);
          if (!mbar_wait(bar(B_XFULL + xb), xph_full[xb], abort_flag, a.err, 6)) { ok = false; break; }
          xph_full[xb] ^= 1;
          asm volatile("tcgen05.fence::after_thread_sync;\n");
          for (int h = 0; h < pg.nh; ++h) {
            float v[64];
            tmem_ld32(tmem + lane_off + xb * 128 + h * 64, v);
            tmem_ld32(tmem + lane_off + xb * 128 + h * 64 + 32, v + 32);
            if (h == pg.nh - 1) {
              asm volatile("tcgen05.fence::before_thread_sync;\n");
              __syncwarp();
              if (lane == 0) mbar_arrive(bar(B_XEMPTY + xb));
            }
            const int valid = min(64, pg.n1 - h * 64);
            if (!mbar_wait(bar(B_A2EMPTY), a2_empty_ph, abort_flag, a.err, 7)) { ok = false; break; }
            a2_empty_ph ^= 1;
            // split scale*X into three bf16 slices, K-major 8x8 tiles
#pragma unroll
            for (int g = 0; g < 8; ++g) {
              __align__(16) __nv_bfloat16 hv[8], mv[8], lv[8];
#pragma unroll
              for (int e = 0; e < 8; ++e) {
                const int j = g * 8 + e;
                float x = (j < valid) ? v[j] * tk.scale : 0.0f;
                __nv_bfloat16 h0 = __float2bfloat16_rn(x);
                float r1 = x - __bfloat162float(h0);
                __nv_bfloat16 m0 = __float2bfloat16_rn(r1);
                float r2 = r1 - __bfloat162float(m0);
                hv[e] = h0;
                mv[e] = m0;
                lv[e] = __float2bfloat16_rn(r2);
              }
              const int off = (((row >> 3) * 8 + g) * 64 + (row & 7) * 8);
              *reinterpret_cast<uint4*>(a2 + off) = *reinterpret_cast<uint4*>(hv);
              *reinterpret_cast<uint4*>(a2 + A2_SLICE / 2 + off) = *reinterpret_cast<uint4*>(mv);
              *reinterpret_cast<uint4*>(a2 + A2_SLICE + off) = *reinterpret_cast<uint4*>(lv);
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(bar(B_A2FULL));
          }
          xb ^= 1;
        }
      }
      if (!ok) break;
      // sigma tile -> FP64 partial slot
      if (!mbar_wait(bar(B_SFULL + sb), sph_full[sb], abort_flag, a.err, 8)) { ok = false; break; }
      sph_full[sb] ^= 1;
      asm volatile("tcgen05.fence::after_thread_sync;\n");
      for (int c0 = 0; c0 < it.ncols; c0 += 32) {
        float v[32];
        tmem_ld32(tmem + lane_off + 256 + sb * 128 + c0, v);
        if (row < it.nrows) {
          const int nc = min(32, it.ncols - c0);
          for (int c = 0; c < nc; ++c) out[(long long)row * it.ncols + c0 + c] = (double)v[c];
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;\n");
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_SEMPTY + sb));
      sb ^= 1;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" ::"r"(tmem));
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
                                 long long njobs, __nv_bfloat16* __restrict__ s0,
                                 __nv_bfloat16* __restrict__ s1, __nv_bfloat16* __restrict__ s2) {
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
      const long long d = j.tile * 64 + e;
      s0[d] = h;
      s1[d] = m;
      s2[d] = l;
    }
  }
}

__global__ void split_psi_kernel(const double* __restrict__ psi, const PsiBlock* __restrict__ blocks,
                                 const TcPsiBlock* __restrict__ pb, int nblk, __nv_bfloat16* __restrict__ s0,
                                 __nv_bfloat16* __restrict__ s1, __nv_bfloat16* __restrict__ s2) {
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
      const long long d = p.tile * 64 + e;
      s0[d] = h;
      s1[d] = m;
      s2[d] = l;
    }
  }
}

void launch_split_ops(const double* store, const SplitJob* jobs, long long njobs, void* const slices[3],
                      cudaStream_t st) {
  if (njobs <= 0) return;
  long long grid = njobs < (1ll << 20) ? njobs : (1ll << 20);
  split_ops_kernel<<<(unsigned)grid, 256, 0, st>>>(store, jobs, njobs, (__nv_bfloat16*)slices[0],
                                                   (__nv_bfloat16*)slices[1], (__nv_bfloat16*)slices[2]);
}

void launch_split_psi(const double* psi, const PsiBlock* blocks, const TcPsiBlock* pb, int nblk,
                      void* const slices[3], cudaStream_t st) {
  if (nblk <= 0) return;
  split_psi_kernel<<<nblk, 256, 0, st>>>(psi, blocks, pb, nblk, (__nv_bfloat16*)slices[0],
                                         (__nv_bfloat16*)slices[1], (__nv_bfloat16*)slices[2]);
}

void launch_sigma_tc(const TcDev& a, int n_sm, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(sigma_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    attr = true;
  }
  int grid = n_sm < a.n_items ? n_sm : a.n_items;
  if (grid < 1) grid = 1;
  sigma_tc_kernel<<<grid, NTHR, SMEM_BYTES, st>>>(a);
}

}  // namespace dmrg
