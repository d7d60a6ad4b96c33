// Launch interfaces of the CUDA kernels (host-callable, stream-ordered).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "model.h"

namespace dmrg {

// ---------------------------------------------------------------- generator
// One block of a synthetic operator: entries N(0,1) from counter off + i*cols + j
// (symmetric blocks use the counter of (min(i,j), max(i,j))).
struct GenBlock {
  long long off;
  int rows, cols;
  int sym, pad;
};
void launch_gen_blocks(double* store, const GenBlock* blocks, long long nblk, uint64_t key,
                       cudaStream_t st);
// x[i] = N(0,1) of counter base + i.
void launch_gen_vector(double* x, long long n, uint64_t key, unsigned long long base,
                       cudaStream_t st);

// ---------------------------------------------------------------- FP64 sigma
constexpr int F64_TM = 32;    // output rows per tile
constexpr int F64_TN = 320;   // output columns per tile (10 warp-wide groups)

struct SigmaDev {
  const double* store;        // operator store (FP64)
  const double* psi;
  double* sigma;
  const Task* tasks;
  const Item* items;
  const int* schedule;
  int n_items;
  const Group* groups;
  int n_groups;
  const PsiBlock* blocks;
  double* scratch;
  unsigned int* counter;      // must be zero at launch (the caller clears it)
};
void launch_sigma_f64(const SigmaDev& a, int n_sm, cudaStream_t st);
void launch_reduce(const SigmaDev& a, cudaStream_t st);

}  // namespace dmrg
