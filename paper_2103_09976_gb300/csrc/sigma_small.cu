// Products of small classes on the CUDA cores (part of the mixed-precision
// sigma, Sec. II.D-E: the same (term, sector) products as the tensor-core
// kernel, for the classes whose output tile and psi block are all at most
// TC_SMALL_MAX wide).
//
// A tcgen05 instruction is at least 128 x 16 x 16, so a product of 8x8 or
// 16x16 blocks would use it by a few percent, and such products are most of
// the (term, block) pairs of a middle bond while carrying about 1% of the
// flops. Here one warp computes one term at a time,
//     sigma[tile] += c * (L psi_b) R^T,
// from the operators and psi in FP32 (products of at most 32 along K,
// accumulated in FP32: a few 2^-24 relative), summing the terms of an item
// in FP64 (in FP32 over groups of 8 terms of a warp first). The warps of a CTA take every NW-th term of the item and their
// sums are added in warp order, so the result does not depend on scheduling.
//
// A term of 16 x 16 blocks is ~16k flops against three block loads, so the
// kernel keeps many terms in flight (two size classes: all blocks <= 16 with
// 8 warps per CTA and several CTAs per SM, the rest with 4 warps), reads
// the operands from their bf16 split (no FP64 -> FP32 conversion, which
// runs on the narrow FP64 pipe), issues all loads of a block before storing
// any, and computes register-blocked products from shared memory.
#include <cuda_fp16.h>

#include "kernels.h"

namespace dmrg {

namespace {

template <int D>
struct SmallCfg;
template <>
struct SmallCfg<16> {
  static constexpr int NW = 8, MINB = 3;
};
template <>
struct SmallCfg<32> {
  static constexpr int NW = 4, MINB = 2;
};

template <int D>
struct Tile;

template <int D>
constexpr int small_smem();

// Load a stored block from its split tiles (8 x 8 tiles, row-major by tile,
// slices hi / mid / lo at bytes 0 / 128 / 256 of each 384-byte tile
// position) into a padded FP32 tile: T[r * LD + c] = stored(r, c), or
// T[c * LD + r] when `trans`. Each value is hi + mid + lo in FP32 (the
// slices hold 24 significant bits, so this is the FP64 value rounded to
// FP32 within an ulp); the bf16 -> FP32 widening is a shift on the integer
// pipe. Lane q takes tile row q (of 8 per tile) and reads its three 16-byte
// slice rows, all loads of the block first; tile padding holds zeros.
template <int D, int LD, bool F16>
__device__ __forceinline__ void load_tiles(float* T, const unsigned char* __restrict__ op, long long tile, int R8,
                                           int C8, bool trans, int lane) {
  constexpr int TILE = F16 ? 256 : 384;  // bytes per tile position
  // tile rows per lane, taken PASS at a time (registers of the <= 32 class)
  constexpr int PER = (D / 8) * (D / 8) * 8 / 32, PASS = PER < 2 ? PER : 2;
  const int nrow = R8 * C8 * 8;
#pragma unroll 1
  for (int k0 = 0; k0 < PER && 32 * k0 < nrow; k0 += PASS) {
    uint4 h[PASS], m[PASS], l[PASS];
#pragma unroll
    for (int k = 0; k < PASS; ++k) {
      const int q = lane + 32 * (k0 + k);
      if (q < nrow) {
        const uint4* p = reinterpret_cast<const uint4*>(op + (tile + (q >> 3)) * TILE + (q & 7) * 16);
        h[k] = __ldg(p);
        m[k] = __ldg(p + 8);
        if (!F16) l[k] = __ldg(p + 16);
      }
    }
#pragma unroll
    for (int k = 0; k < PASS; ++k) {
      const int q = lane + 32 * (k0 + k);
      if (q < nrow) {
        const int t = q >> 3, tr = t / C8, tc = t - tr * C8, r = 8 * tr + (q & 7), c0 = 8 * tc;
        const uint32_t hw[4] = {h[k].x, h[k].y, h[k].z, h[k].w}, mw[4] = {m[k].x, m[k].y, m[k].z, m[k].w};
        uint32_t lw[4] = {0u, 0u, 0u, 0u};
        if (!F16) {
          lw[0] = l[k].x;
          lw[1] = l[k].y;
          lw[2] = l[k].z;
          lw[3] = l[k].w;
        }
        float v[8];
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          if (!F16) {
            v[2 * w] = (__uint_as_float(hw[w] << 16) + __uint_as_float(mw[w] << 16)) + __uint_as_float(lw[w] << 16);
            v[2 * w + 1] = (__uint_as_float(hw[w] & 0xFFFF0000u) + __uint_as_float(mw[w] & 0xFFFF0000u)) +
                           __uint_as_float(lw[w] & 0xFFFF0000u);
          } else {  // fp16 hi + lo (scaled values; the coefficients undo the scales)
            const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&hw[w]));
            const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&mw[w]));
            v[2 * w] = a.x + b.x;
            v[2 * w + 1] = a.y + b.y;
          }
        }
        if (!trans) {
          *reinterpret_cast<float4*>(T + r * LD + c0) = make_float4(v[0], v[1], v[2], v[3]);
          *reinterpret_cast<float4*>(T + r * LD + c0 + 4) = make_float4(v[4], v[5], v[6], v[7]);
        } else {
#pragma unroll
          for (int c = 0; c < 8; ++c) T[(c0 + c) * LD + r] = v[c];
        }
      }
    }
  }
}

// Register-blocked products of one term whose operands are in shared
// memory: lane (rp, cg) = (lane / 4, lane % 4) owns rows rp + 8i (i < D/8)
// and columns D/4 * cg .. + D/4 - 1 of X = L psi and of the tile, so one
// step along K reads D/8 values of a column of L (or X) and D/4 consecutive
// values of a row of psi (or R^T) as 16-byte loads, for D*D/32 FMAs. Rows
// and columns past the blocks are computed from stale shared memory and
// never read: the K loops stay inside the blocks. LD (a multiple of 4 for
// the 16-byte loads) spreads the D/8 column reads of L over distinct banks.
template <>
struct Tile<16> {
  static constexpr int LD = 20, RI = 2, CJ = 4;
};
template <>
struct Tile<32> {
  static constexpr int LD = 36, RI = 4, CJ = 8;
};

template <int D>
__device__ __forceinline__ void term_product(float (&y)[Tile<D>::RI][Tile<D>::CJ], const float* sPsi,
                                             const float* sL, const float* sRt, float* sX, int m, int n, bool idL,
                                             bool idR, int lane) {
  constexpr int LD = Tile<D>::LD, RI = Tile<D>::RI, CJ = Tile<D>::CJ;
  const int rp = lane >> 2, c0 = CJ * (lane & 3);
  if (!idL) {  // X = L psi (tm x n)
    float x[RI][CJ];
#pragma unroll
    for (int i = 0; i < RI; ++i)
#pragma unroll
      for (int j = 0; j < CJ; ++j) x[i][j] = 0.0f;
    for (int kk = 0; kk < m; ++kk) {
      float b[CJ];
#pragma unroll
      for (int j = 0; j < CJ; j += 4) *reinterpret_cast<float4*>(b + j) = *reinterpret_cast<const float4*>(sPsi + kk * LD + c0 + j);
#pragma unroll
      for (int i = 0; i < RI; ++i) {
        const float a = sL[(rp + 8 * i) * LD + kk];
#pragma unroll
        for (int j = 0; j < CJ; ++j) x[i][j] = fmaf(a, b[j], x[i][j]);
      }
    }
#pragma unroll
    for (int i = 0; i < RI; ++i)
#pragma unroll
      for (int j = 0; j < CJ; j += 4)
        *reinterpret_cast<float4*>(sX + (rp + 8 * i) * LD + c0 + j) = make_float4(x[i][j], x[i][j + 1], x[i][j + 2], x[i][j + 3]);
    __syncwarp();
  }
  const float* X = idL ? sPsi : sX;
  if (idR) {  // tile = X
#pragma unroll
    for (int i = 0; i < RI; ++i)
#pragma unroll
      for (int j = 0; j < CJ; j += 4) *reinterpret_cast<float4*>(&y[i][j]) = *reinterpret_cast<const float4*>(X + (rp + 8 * i) * LD + c0 + j);
    return;
  }
#pragma unroll
  for (int i = 0; i < RI; ++i)
#pragma unroll
    for (int j = 0; j < CJ; ++j) y[i][j] = 0.0f;
  for (int kk = 0; kk < n; ++kk) {  // tile = X R^T
    float b[CJ];
#pragma unroll
    for (int j = 0; j < CJ; j += 4) *reinterpret_cast<float4*>(b + j) = *reinterpret_cast<const float4*>(sRt + kk * LD + c0 + j);
#pragma unroll
    for (int i = 0; i < RI; ++i) {
      const float a = X[(rp + 8 * i) * LD + kk];
#pragma unroll
      for (int j = 0; j < CJ; ++j) y[i][j] = fmaf(a, b[j], y[i][j]);
    }
  }
}

template <int D, bool F16>
__global__ void __launch_bounds__(32 * SmallCfg<D>::NW, SmallCfg<D>::MINB) sigma_small_kernel(SmallDev a) {
  constexpr int NW = SmallCfg<D>::NW, LD = Tile<D>::LD, BLK = D * LD, RI = Tile<D>::RI, CJ = Tile<D>::CJ;
  // terms summed in FP32 (scaled products) before each FP64 addition
  constexpr int GROUP = 8;
  extern __shared__ __align__(16) float smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rp = lane >> 2, c0 = CJ * (lane & 3);
  float* sPsi = smem + warp * 4 * BLK;
  float* sL = sPsi + BLK;
  float* sRt = sL + BLK;
  float* sX = sRt + BLK;
  for (int qi = blockIdx.x; qi < a.n_items; qi += gridDim.x) {
    const TcItem it = a.items[a.schedule[qi]];
    const int tm = it.nrows, tn = it.ncols;
    double acc[RI][CJ];
    float grp[RI][CJ];
#pragma unroll
    for (int i = 0; i < RI; ++i)
#pragma unroll
      for (int j = 0; j < CJ; ++j) {
        acc[i][j] = 0.0;
        grp[i][j] = 0.0f;
      }
    int cur = -1, ng = 0;
    for (int t = it.r_begin + warp; t < it.r_end; t += NW) {
      const SmallTerm tk = a.terms[t];
      const TcPsiBlock pb = a.pblk[tk.in_blk];
      const int m = pb.m, n = pb.n;
      const bool idL = tk.a_tile < 0, idR = tk.b_tile < 0;
      // the operands of this term; psi only when the block changes (the
      // terms of a class share it). L is tm x m (stored m x tm when used
      // transposed); R is kept transposed in shared memory (n x tn), from
      // its stored tn x n (or n x tn when used transposed).
      const unsigned char* op = reinterpret_cast<const unsigned char*>(a.op);
      if (tk.in_blk != cur)
        load_tiles<D, LD, F16>(sPsi, reinterpret_cast<const unsigned char*>(a.psi), pb.tile, pb.R8, pb.C8, false, lane);
      if (!idL) {
        const bool tA = tk.flags & 1;
        load_tiles<D, LD, F16>(sL, op, tk.a_tile, tA ? (m + 7) / 8 : (tm + 7) / 8, tA ? (tm + 7) / 8 : (m + 7) / 8, tA, lane);
      }
      if (!idR) {
        const bool tB = tk.flags & 2;
        load_tiles<D, LD, F16>(sRt, op, tk.b_tile, tB ? (n + 7) / 8 : (tn + 7) / 8, tB ? (tn + 7) / 8 : (n + 7) / 8, !tB, lane);
      }
      cur = tk.in_blk;
      __syncwarp();
      float y[RI][CJ];
      term_product<D>(y, sPsi, sL, sRt, sX, m, n, idL, idR, lane);
      if (GROUP == 1) {
#pragma unroll
        for (int i = 0; i < RI; ++i)
#pragma unroll
          for (int j = 0; j < CJ; ++j) acc[i][j] += tk.scale * (double)y[i][j];
      } else {
        const float sc = (float)tk.scale;
#pragma unroll
        for (int i = 0; i < RI; ++i)
#pragma unroll
          for (int j = 0; j < CJ; ++j) grp[i][j] = fmaf(sc, y[i][j], grp[i][j]);
        if (++ng == GROUP) {
#pragma unroll
          for (int i = 0; i < RI; ++i)
#pragma unroll
            for (int j = 0; j < CJ; ++j) {
              acc[i][j] += (double)grp[i][j];
              grp[i][j] = 0.0f;
            }
          ng = 0;
        }
      }
      __syncwarp();
    }
#pragma unroll
    for (int i = 0; i < RI; ++i)
#pragma unroll
      for (int j = 0; j < CJ; ++j) acc[i][j] += (double)grp[i][j];
    // add the warps' sums in warp order
    __syncthreads();
    double* sum = reinterpret_cast<double*>(smem);
#pragma unroll
    for (int i = 0; i < RI; ++i)
#pragma unroll
      for (int j = 0; j < CJ; ++j) {
        const int r = rp + 8 * i, c = c0 + j;
        if (r < tm && c < tn) sum[warp * D * D + r * tn + c] = acc[i][j];
      }
    __syncthreads();
    double* out = a.scratch + it.slot;
    const double ps = F16 ? ldexp(1.0, psi_exponent(*a.psi_exp) - 14) : 1.0;  // undo psi's split scale
    for (int e = threadIdx.x; e < tm * tn; e += blockDim.x) {
      double v = sum[e];
      for (int w = 1; w < NW; ++w) v += sum[w * D * D + e];
      out[e] = F16 ? v * ps : v;
    }
    __syncthreads();
  }
}

template <int D>
constexpr int small_smem() {
  return SmallCfg<D>::NW * 4 * D * Tile<D>::LD * (int)sizeof(float);
}
static_assert(SmallCfg<16>::NW * 16 * 16 * (int)sizeof(double) <= small_smem<16>(), "final sums fit");
static_assert(SmallCfg<32>::NW * 32 * 32 * (int)sizeof(double) <= small_smem<32>(), "final sums fit");
static_assert(TC_SMALL_MAX == 32 && TC_SMALL_MID == 16, "size classes");

template <int D>
void launch_class(const SmallDev& a, int n_items, const int* schedule, int n_sm, cudaStream_t st) {
  if (n_items <= 0) return;
  const void* fn = a.f16 ? (const void*)sigma_small_kernel<D, true> : (const void*)sigma_small_kernel<D, false>;
  set_max_dynamic_smem(fn, small_smem<D>());
  SmallDev b = a;
  b.schedule = schedule;
  b.n_items = n_items;
  int grid = SmallCfg<D>::MINB * n_sm;
  if (grid > n_items) grid = n_items;
  if (a.f16)
    sigma_small_kernel<D, true><<<grid, 32 * SmallCfg<D>::NW, small_smem<D>(), st>>>(b);
  else
    sigma_small_kernel<D, false><<<grid, 32 * SmallCfg<D>::NW, small_smem<D>(), st>>>(b);
}

}  // namespace

void launch_sigma_small(const SmallDev& a, int n_sm, cudaStream_t st) {
  // the schedule lists the <= 16 class first
  launch_class<16>(a, a.n_mid, a.schedule, n_sm, st);
  launch_class<32>(a, a.n_items - a.n_mid, a.schedule + a.n_mid, n_sm, st);
}

}  // namespace dmrg
