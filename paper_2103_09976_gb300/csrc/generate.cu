// Counter-based N(0,1) generator for synthetic operator blocks and vectors.
//
// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014; finalizer constants of
// Vigna's public-domain splitmix64.c) used as a counter-based generator: the
// c-th output from state `key` is mix(key + (c+1) * 0x9E3779B97F4A7C15).
// u = ((x >> 11) + 1) * 2^-53 lies in (0, 1]; a normal number for counter g
// is Box-Muller's sqrt(-2 ln u(2g)) * cos(2 pi u(2g+1)).
#include "kernels.h"

namespace dmrg {

__device__ __forceinline__ uint64_t sm_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double sm_uniform(uint64_t key, uint64_t c) {
  uint64_t x = sm_mix(key + (c + 1ull) * 0x9E3779B97F4A7C15ull);
  return (double)((x >> 11) + 1ull) * 0x1.0p-53;
}

__device__ __forceinline__ double sm_normal(uint64_t key, uint64_t g) {
  double u1 = sm_uniform(key, 2ull * g);
  double u2 = sm_uniform(key, 2ull * g + 1ull);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

__global__ void gen_blocks_kernel(double* __restrict__ store, const GenBlock* __restrict__ blocks,
                                  long long nblk, uint64_t key) {
  for (long long b = blockIdx.x; b < nblk; b += gridDim.x) {
    const GenBlock gb = blocks[b];
    const long long n = (long long)gb.rows * gb.cols;
    for (long long e = threadIdx.x; e < n; e += blockDim.x) {
      int i = (int)(e / gb.cols), j = (int)(e - (long long)i * gb.cols);
      long long idx = (gb.sym && i > j) ? (long long)j * gb.cols + i : e;
      store[gb.off + e] = sm_normal(key, (uint64_t)(gb.ctr + idx));
    }
  }
}

__global__ void gen_vector_kernel(double* __restrict__ x, long long n, uint64_t key,
                                  unsigned long long base) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] = sm_normal(key, base + (uint64_t)i);
}

void launch_gen_blocks(double* store, const GenBlock* blocks, long long nblk, uint64_t key,
                       cudaStream_t st) {
  if (nblk <= 0) return;
  long long grid = nblk < 65535 * 16 ? nblk : 65535 * 16;
  gen_blocks_kernel<<<(unsigned)grid, 128, 0, st>>>(store, blocks, nblk, key);
}

void launch_gen_vector(double* x, long long n, uint64_t key, unsigned long long base,
                       cudaStream_t st) {
  if (n <= 0) return;
  long long grid = (n + 255) / 256;
  if (grid > 152 * 64) grid = 152 * 64;
  gen_vector_kernel<<<(unsigned)grid, 256, 0, st>>>(x, n, key, base);
}

}  // namespace dmrg
