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
// from the FP64 operator store read as FP32 (products of at most 32 along K,
// accumulated in FP32: a few 2^-24 relative), summing the terms of an item
// in FP64. The four warps of a CTA take every fourth term of the item and
// their sums are added in warp order, so the result does not depend on
// scheduling.
#include "kernels.h"

namespace dmrg {

namespace {

constexpr int SW = 4;                    // warps per CTA
constexpr int LD = TC_SMALL_MAX + 1;     // padded row of the shared-memory blocks
constexpr int BLK = TC_SMALL_MAX * LD;   // floats per block
constexpr int SMALL_SMEM = SW * 4 * BLK * (int)sizeof(float);
static_assert(SW * TC_SMALL_MAX * TC_SMALL_MAX * (int)sizeof(double) <= SMALL_SMEM, "final sums fit");

__global__ void __launch_bounds__(32 * SW) sigma_small_kernel(SmallDev a) {
  extern __shared__ float smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* sPsi = smem + warp * 4 * BLK;
  float* sL = sPsi + BLK;
  float* sR = sL + BLK;
  float* sX = sR + BLK;
  for (int qi = blockIdx.x; qi < a.n_items; qi += gridDim.x) {
    const TcItem it = a.items[a.schedule[qi]];
    const int tm = it.nrows, tn = it.ncols, nout = tm * tn;
    double acc[TC_SMALL_MAX];
#pragma unroll
    for (int k = 0; k < TC_SMALL_MAX; ++k) acc[k] = 0.0;
    int cur = -1;
    for (int t = it.r_begin + warp; t < it.r_end; t += SW) {
      const SmallTerm tk = a.terms[t];
      const PsiBlock ib = a.blocks[tk.in_blk];
      const int m = ib.mL, n = ib.mR;
      if (tk.in_blk != cur) {  // psi block of this term (m x n)
        for (int e = lane; e < m * n; e += 32) sPsi[(e / n) * LD + e % n] = (float)a.psi[ib.off + e];
        cur = tk.in_blk;
      }
      const bool idL = tk.a_off < 0, idR = tk.b_off < 0;
      if (!idL) {  // L: tm x m (stored tm x m, or m x tm when used transposed)
        const double* S = a.store + tk.a_off;
        if (!(tk.flags & 1))
          for (int e = lane; e < tm * m; e += 32) sL[(e / m) * LD + e % m] = (float)S[e];
        else
          for (int e = lane; e < tm * m; e += 32) sL[(e % tm) * LD + e / tm] = (float)S[e];
      }
      if (!idR) {  // R: tn x n (stored tn x n, or n x tn when used transposed)
        const double* S = a.store + tk.b_off;
        if (!(tk.flags & 2))
          for (int e = lane; e < tn * n; e += 32) sR[(e / n) * LD + e % n] = (float)S[e];
        else
          for (int e = lane; e < tn * n; e += 32) sR[(e % tn) * LD + e / tn] = (float)S[e];
      }
      __syncwarp();
      // X = L psi (tm x n)
      for (int e = lane; e < tm * n; e += 32) {
        const int i = e / n, j = e % n;
        float x;
        if (idL) {
          x = sPsi[i * LD + j];
        } else {
          x = 0.0f;
          for (int k = 0; k < m; ++k) x = fmaf(sL[i * LD + k], sPsi[k * LD + j], x);
        }
        sX[i * LD + j] = x;
      }
      __syncwarp();
      // sigma[tile] += scale * X R^T (tm x tn), element e = i * tn + c
#pragma unroll
      for (int k = 0; k < TC_SMALL_MAX; ++k) {
        const int e = lane + 32 * k;
        if (e < nout) {
          const int i = e / tn, c = e % tn;
          float s;
          if (idR) {
            s = sX[i * LD + c];
          } else {
            s = 0.0f;
            for (int j = 0; j < n; ++j) s = fmaf(sX[i * LD + j], sR[c * LD + j], s);
          }
          acc[k] += tk.scale * (double)s;
        }
      }
      __syncwarp();
    }
    // add the warps' sums in warp order
    __syncthreads();
    double* sum = reinterpret_cast<double*>(smem);
#pragma unroll
    for (int k = 0; k < TC_SMALL_MAX; ++k) {
      const int e = lane + 32 * k;
      if (e < nout) sum[warp * TC_SMALL_MAX * TC_SMALL_MAX + e] = acc[k];
    }
    __syncthreads();
    double* out = a.scratch + it.slot;
    for (int e = threadIdx.x; e < nout; e += blockDim.x) {
      double v = sum[e];
      for (int w = 1; w < SW; ++w) v += sum[w * TC_SMALL_MAX * TC_SMALL_MAX + e];
      out[e] = v;
    }
    __syncthreads();
  }
}

}  // namespace

void launch_sigma_small(const SmallDev& a, int n_sm, cudaStream_t st) {
  if (a.n_items <= 0) return;
  set_max_dynamic_smem((const void*)sigma_small_kernel, SMALL_SMEM);
  int grid = 3 * n_sm;
  if (grid > a.n_items) grid = a.n_items;
  sigma_small_kernel<<<grid, 32 * SW, SMALL_SMEM, st>>>(a);
}

}  // namespace dmrg
