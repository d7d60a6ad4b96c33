// The FP16 hi + lo split of the FP16X2 sigma (the mixed-precision variant
// with two fp16 slices per operand, three slice products; Sec. II.D-E's
// products are unchanged, only their arithmetic).
//
// fp16 has 11 significant bits and a narrow exponent range (normal numbers
// from 2^-14), so every operand is scaled by a power of two before it is
// split: a stored operator block by 2^(14 - e) with 2^e <= max |x| < 2^(e+1)
// (so its largest element lies in [2^14, 2^15)), psi by 2^(14 - e_psi) with
// e_psi from max |psi| over the whole vector. Then hi = fp16(x), lo =
// fp16(x - hi), and x - hi - lo is below 2^-22 |x| for every element whose lo
// part is a normal fp16 number (|x| >= 2^-3 after scaling); smaller
// elements keep an absolute error below 2^-25, i.e. 2^-39 of the block's
// largest element. Powers of two are exact, so the scales are undone exactly:
// the tensor-core kernel folds the operator scales of a term into its
// coefficient (fix_recs16_kernel) and psi's into the flush of its FP32
// accumulators.
#include <cuda_fp16.h>

#include <climits>

#include "context.h"
#include "kernels.h"

namespace dmrg {

namespace {

constexpr int TILE_HALVES = 128;  // one tile position: hi (64 halves) then lo (64 halves)

__device__ __forceinline__ double block_max(double m) {
#pragma unroll
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double red[32];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = m;
  __syncthreads();
  if (w == 0) {
    m = l < (int)(blockDim.x >> 5) ? red[l] : 0.0;
#pragma unroll
    for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  }
  return m;  // valid in thread 0
}

// e with 2^e <= m < 2^(e+1); 0 for m = 0
__device__ __forceinline__ int exp2_of(double m) { return m > 0.0 ? ilogb(m) : 0; }

__global__ void block_exp_kernel(const double* __restrict__ store, const SplitJob* __restrict__ jobs, long long njobs,
                                 int* __restrict__ exps) {
  for (long long b = blockIdx.x; b < njobs; b += gridDim.x) {
    const SplitJob j = jobs[b];
    double m = 0.0;
    if (j.src < 0) {
      m = 1.0;
    } else {
      const long long n = (long long)j.rows * j.cols;
      for (long long e = threadIdx.x; e < n; e += blockDim.x) m = fmax(m, fabs(store[j.src + e]));
    }
    m = block_max(m);
    if (threadIdx.x == 0) exps[b] = exp2_of(m);
  }
}

__device__ __forceinline__ void split2(double x, __half& h, __half& l) {
  h = __double2half(x);
  l = __double2half(x - (double)__half2float(h));
}

__global__ void split_ops16_kernel(const double* __restrict__ store, const SplitJob* __restrict__ jobs, long long njobs,
                                   const int* __restrict__ exps, __half* __restrict__ out) {
  for (long long b = blockIdx.x; b < njobs; b += gridDim.x) {
    const SplitJob j = jobs[b];
    const double s = ldexp(1.0, 14 - exps[b]);
    const long long n = (long long)j.R8 * j.C8 * 64;
    for (long long e = threadIdx.x; e < n; e += blockDim.x) {
      const long long t = e >> 6;
      const int w = (int)(e & 63);
      const int i = (int)(t / j.C8) * 8 + (w >> 3), c = (int)(t % j.C8) * 8 + (w & 7);
      double x = 0.0;
      if (i < j.rows && c < j.cols) x = (j.src < 0) ? (i == c ? 1.0 : 0.0) : store[j.src + (long long)i * j.cols + c];
      __half h, l;
      split2(x * s, h, l);
      const long long d = (j.tile + t) * TILE_HALVES + w;
      out[d] = h;
      out[d + 64] = l;
    }
  }
}

__global__ void psi_exp_kernel(const double* __restrict__ psi, long long n, int* __restrict__ e_psi) {
  double m = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    m = fmax(m, fabs(psi[e]));
  m = block_max(m);
  if (threadIdx.x == 0 && m > 0.0) atomicMax(e_psi, ilogb(m));
}

__global__ void split_psi16_kernel(const double* __restrict__ psi, const PsiBlock* __restrict__ blocks,
                                   const TcPsiBlock* __restrict__ pb, int nblk, const int* __restrict__ e_psi,
                                   __half* __restrict__ out) {
  const double s = ldexp(1.0, 14 - psi_exponent(*e_psi));
  for (int b = blockIdx.x; b < nblk; b += gridDim.x) {
    const TcPsiBlock p = pb[b];
    const long long off = blocks[b].off;
    const long long n = (long long)p.R8 * p.C8 * 64;
    for (long long e = threadIdx.x; e < n; e += blockDim.x) {
      const long long t = e >> 6;
      const int w = (int)(e & 63);
      const int i = (int)(t / p.C8) * 8 + (w >> 3), c = (int)(t % p.C8) * 8 + (w & 7);
      const double x = (i < p.m && c < p.n) ? psi[off + (long long)i * p.n + c] : 0.0;
      __half h, l;
      split2(x * s, h, l);
      const long long d = (p.tile + t) * TILE_HALVES + w;
      out[d] = h;
      out[d + 64] = l;
    }
  }
}

// smallest k with |v| <= 2^k (v != 0)
__device__ __forceinline__ int ceil_log2(double v) {
  const int k = ilogb(v);
  return ldexp(1.0, k) == v ? k : k + 1;
}

// Coefficients of the FP16X2 records. A unit's terms t (left / right block
// exponents eL, eR, coefficient c, psi block of K rows) accumulate in one
// FP32 tile scaled by S = 2^(E - e_psi) with
//     E = min_t (26 - eL - eR - ceil(log2(|c| K))),
// which keeps every element of the re-split intermediate Y_t = c X_t S /
// s_R below 2^14 (|X_t| <= K max|L| max|psi| < K 2^(eL+1) 2^(e_psi+1)). The
// epilogue multiplies the scaled intermediate by f_t = c 2^(E + eL + eR - 42)
// (e_psi cancels), and the flush multiplies the tile by 2^(e_psi - E).
__global__ void fix_recs16_kernel(const TcUnitRec* __restrict__ in, long long n, const int* __restrict__ term_blk,
                                  const int* __restrict__ exps, TcUnitRec* __restrict__ out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    TcUnitRec r = in[i];
    if (!(r.flags & (TC_ZERO | TC_DONE))) {
      int E = INT_MAX;
      for (int q = 0; q < r.nterm; ++q) {
        const double c = fabs((double)r.t[q].scale) * (double)r.m;
        if (c == 0.0) continue;
        const int eL = exps[term_blk[(i * TC_MAX_G + q) * 2]], eR = exps[term_blk[(i * TC_MAX_G + q) * 2 + 1]];
        E = min(E, 26 - eL - eR - ceil_log2(c));
      }
      if (E == INT_MAX) E = 0;
      for (int q = 0; q < r.nterm; ++q) {
        const int eL = exps[term_blk[(i * TC_MAX_G + q) * 2]], eR = exps[term_blk[(i * TC_MAX_G + q) * 2 + 1]];
        r.t[q].scale = (float)ldexp((double)r.t[q].scale, E + eL + eR - 42);
      }
      r.pad[0] = E;
    }
    out[i] = r;
  }
}

// Small-class terms read the scaled fp16 split: their coefficients undo the
// operator scales (identity blocks are not read and not scaled); psi's scale
// is undone when the item's sum is written.
__global__ void fix_small16_kernel(const SmallTerm* __restrict__ in, long long n, const int* __restrict__ small_blk,
                                   const int* __restrict__ exps, SmallTerm* __restrict__ out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    SmallTerm t = in[i];
    int sh = 0;
    if (t.a_tile >= 0) sh += exps[small_blk[2 * i]] - 14;
    if (t.b_tile >= 0) sh += exps[small_blk[2 * i + 1]] - 14;
    t.scale = ldexp(t.scale, sh);
    out[i] = t;
  }
}

}  // namespace

void launch_block_exp(const double* store, const SplitJob* jobs, long long njobs, int* exps, cudaStream_t st) {
  if (njobs <= 0) return;
  const long long grid = njobs < (1ll << 20) ? njobs : (1ll << 20);
  block_exp_kernel<<<(unsigned)grid, 256, 0, st>>>(store, jobs, njobs, exps);
}

void launch_split_ops16(const double* store, const SplitJob* jobs, long long njobs, const int* exps, void* out,
                        cudaStream_t st) {
  if (njobs <= 0) return;
  const long long grid = njobs < (1ll << 20) ? njobs : (1ll << 20);
  split_ops16_kernel<<<(unsigned)grid, 256, 0, st>>>(store, jobs, njobs, exps, (__half*)out);
}

void launch_split_psi16(const double* psi, long long n, const PsiBlock* blocks, const TcPsiBlock* pb, int nblk,
                        int* e_psi, void* out, cudaStream_t st) {
  if (nblk <= 0) return;
  DMRG_CUDA(cudaMemsetAsync(e_psi, 0x80, sizeof(int), st));  // below any exponent: an all-zero psi keeps it
  psi_exp_kernel<<<256, 256, 0, st>>>(psi, n, e_psi);
  split_psi16_kernel<<<nblk, 256, 0, st>>>(psi, blocks, pb, nblk, e_psi, (__half*)out);
}

void launch_fix_recs16(const TcUnitRec* in, long long n, const int* term_blk, const int* exps, TcUnitRec* out,
                       cudaStream_t st) {
  if (n <= 0) return;
  fix_recs16_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(in, n, term_blk, exps, out);
}

void launch_fix_small16(const SmallTerm* in, long long n, const int* small_blk, const int* exps, SmallTerm* out,
                        cudaStream_t st) {
  if (n <= 0) return;
  fix_small16_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, n, small_blk, exps, out);
}

}  // namespace dmrg
