// Launch interfaces of the CUDA kernels (host-callable, stream-ordered).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "model.h"

namespace dmrg {

// Raise the dynamic shared-memory limit of kernel `fn` to `bytes` on the
// current device. The limit is a per-device attribute, so it is set once for
// every (kernel, device) pair; safe to call from several host threads.
// Throws dmrg::Error (DMRG_ECUDA) when the runtime refuses it.
void set_max_dynamic_smem(const void* fn, int bytes);

// ---------------------------------------------------------------- generator
// One block of a synthetic operator, written at element offset `off`: entries
// N(0,1) from counter ctr + i*cols + j (symmetric blocks use the counter of
// (min(i,j), max(i,j))); ctr is the block's offset in the full canonical store.
struct GenBlock {
  long long off, ctr;
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
constexpr int F64_TN = 256;   // output columns per tile (32 groups of 8)

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

// ------------------------------------------------------------ tensor cores
// One stored block (or identity, src < 0) to split into three bf16 slices.
struct SplitJob {
  long long src;     // element offset in the FP64 store, -1 = identity
  int rows, cols;
  long long tile;    // first 128-byte tile in the slice arrays
  int R8, C8;
};

struct TcDev {
  const void* op;             // operator tiles, slice-interleaved (3 bf16 or 2 fp16 slices of 128 B per tile position)
  const void* psi;            // psi tiles, same layout
  const int* psi_exp;         // FP16X2: exponent of max |psi| (psi_exponent), else unused
  const TcUnitRec* recs;      // unit records, grouped by item
  const TcItem* items;        // records of item i: [items[i].r_begin, items[i].r_end)
  const int* schedule;        // item order, most expensive first
  int n_items;
  unsigned int* counter;      // next item to take; zero at launch
  double* scratch;
  int* err;                   // nonzero after a bounded wait gave up
  int nprod;                  // 6 (three bf16 slices) or 3 (two slices)
  int f16;                    // 1: FP16X2 (fp16 slices, 256-byte tile positions, scaled operands)
  int max_chain;              // main MMA steps per FP32 accumulation (flush group); <= 0: one group per half
  int producers;              // 1: warp 0 fills every ring slot; 3: producer warp w fills slot w
  unsigned long long* wait_prof;  // optional [17]: wait cycles per barrier kind, total cycles
};

// Small classes of the mixed-precision sigma on the CUDA cores (see TC_SMALL_MAX).
struct SmallDev {
  const void* op;             // operator split (the tensor-core kernel's tiles)
  const void* psi;            // psi split
  const int* psi_exp;         // FP16X2 split: exponent of max |psi|, else unused
  int f16;                    // 1: the split is FP16X2's (2 fp16 slices, scaled operands)
  const TcPsiBlock* pblk;     // psi blocks: split tiles and dimensions
  const SmallTerm* terms;
  const TcItem* items;        // kind-1/2 items index terms
  const int* schedule;        // kind-2 items, then kind-1 items, each most expensive first
  int n_items;
  int n_mid;                  // kind-2 items (all blocks <= TC_SMALL_MID) at the head of the schedule
  double* scratch;            // partial tiles (item slots)
};
void launch_sigma_small(const SmallDev& a, int n_sm, cudaStream_t st);

void launch_split_ops(const double* store, const SplitJob* jobs, long long njobs, void* out, cudaStream_t st);
void launch_split_psi(const double* psi, const PsiBlock* blocks, const TcPsiBlock* pb, int nblk, void* out,
                      cudaStream_t st);
void launch_sigma_tc(const TcDev& a, int n_sm, cudaStream_t st);
// Default producer setting of the tensor-core kernel for a plan (TcDev::producers):
// 3 when its units average 5 or more ring stages of the kernel's geometry
// (bf16 or fp16 tiles), else 1.
int tc_default_producers(const TcPlan& plan, bool f16);

// FP16X2 split (split_f16.cu). Operator blocks and psi are scaled by powers
// of two before the split: block b by 2^(14 - exps[b]), psi by
// 2^(14 - psi_exponent(*e_psi)), where 2^e <= max |x| < 2^(e+1).
void launch_block_exp(const double* store, const SplitJob* jobs, long long njobs, int* exps, cudaStream_t st);
void launch_split_ops16(const double* store, const SplitJob* jobs, long long njobs, const int* exps, void* out,
                        cudaStream_t st);
void launch_split_psi16(const double* psi, long long n, const PsiBlock* blocks, const TcPsiBlock* pb, int nblk,
                        int* e_psi, void* out, cudaStream_t st);
// Records and small terms with coefficients for the scaled fp16 operands
// (term_blk / small_blk: split-job indices of each term's left and right
// blocks).
void launch_fix_recs16(const TcUnitRec* in, long long n, const int* term_blk, const int* exps, TcUnitRec* out,
                       cudaStream_t st);
void launch_fix_small16(const SmallTerm* in, long long n, const int* small_blk, const int* exps, SmallTerm* out,
                        cudaStream_t st);
// The exponent written by launch_split_psi16 (an all-zero psi leaves the
// initial value, far below any exponent: taken as 0).
__host__ __device__ inline int psi_exponent(int e) { return e < -100000 ? 0 : e; }

// ------------------------------------------------------------------- sweep
// One term of an enlarged operator: coef * (source op `src`, transposed when
// trans; -1 = identity) (x) |nout><nin| on the site.
struct BTerm {
  int src, trans, nout, nin;
  double coef;
};
// One destination block of the enlarged operator set: op k, sectors Qin -> Qout.
struct BDst {
  long long off;
  int k, Qin, Qout, rows, cols, pad;
};
// Everything the blocking kernel needs to expand terms into sector blocks.
struct BlockingDev {
  double* dst_store;
  const double* src_store;      // source ops [0, nsrc1)
  const double* src_store2;     // source ops [nsrc1, ...): complementary sums of the block
  int nsrc1;
  const BDst* dsts;
  int ndst;
  const int* term_start;        // per destination op, CSR into terms
  const BTerm* terms;
  const int* bq;                // block basis: (N, 2Sz) per sector, ascending
  const int* bdim;
  int nb;
  const int* eq;                // enlarged basis (N, 2Sz) per sector
  const int* chunk_off;         // [enlarged sector][block sector]: row offset of the chunk, or -1
  const long long* srcblk;      // [source op][input sector]: offset of its block, or -1
  const int* src_dq;            // (dN, d2Sz) per source op
  const int* src_par;           // fermion parity per source op
  int left;                     // 1: block x site, 0: site x block
  int* err;                     // set to 1 on an inconsistent term
};
struct GramBlock {      // one psi block for decimation / one block to orthonormalise
  long long psi_off, g_off, w_off;
  int d, m;             // Gram dimension and contracted dimension (or d x m columns)
};
struct TakeBlock {      // dst (d x k) = first k columns of Q (d x d)
  long long q_off, dst_off;
  int d, k;
};
void launch_blocking(const BlockingDev& d, cudaStream_t st);
// Linear combinations of a block's stored operators (the normal-to-
// complementary transformation, Sec. III.A): for every class g (operators
// sharing one shift, hence one block structure of E elements),
//   Y_o = sum_i C[o][i] X_i,   o < n_out, i < n_in,
// X_i the class's i-th source operator (E contiguous elements at
// src + xoff[x_start + i]), Y_o at dst + y_off + o * E, C row-major at
// coef + c_off. One 64 x 128 tile of (o, element) per CTA, FP64 tensor
// instructions, k in steps of 16 sources.
// (CombClass, COMB_TM and COMB_TN are in model.h.)
// Small strided GEMMs C = A B (one job per CTA, FP64, fixed summation
// order): A(i, k) = A[a + (ta ? k * lda + i : i * lda + k)], B(k, j) =
// B[b + (tb ? j * ldb + k : k * ldb + j)], C[c + i * ldc + j], i < m, j < n,
// k < kk. Used to carry a wavefunction from one bond to the next.
// (GJob is in model.h.)
void launch_bgemm(const double* A, const double* B, double* C, const GJob* jobs, int njobs, cudaStream_t st);
void launch_opcomb(const double* src, const long long* xoff, const double* coef, const CombClass* cls, int ncls,
                   int ntiles, double* dst, cudaStream_t st);
// Per psi block: singular vectors of its d-dimensional side (rows when left,
// columns otherwise) and squared singular values, by one-sided Jacobi over
// the whole GPU (one cooperative launch for all blocks): Q (d x d row-major,
// columns = vectors) and w (d values), by descending singular value. Work
// space: 64 doubles, then A (d x m) and V (d x d) of every block at a_off /
// v_off. max_d_hint >= every d (shared memory of the final sort).
struct SvdBlock {
  long long psi_off, q_off, w_off, a_off, v_off;
  int d, m, pair0, npairs, rounds, pad;
};
void launch_svd_blocks(const double* psi, const SvdBlock* sb, int nb, int total_pairs, int max_rounds, int max_d_hint,
                       double* Q, double* w, double* work, bool left, int n_sm, cudaStream_t st);
void launch_orthonormalize(double* store, const GramBlock* gb, int nb, cudaStream_t st);
void launch_take_columns(const double* Q, const TakeBlock* tb, int nb, double* dst, cudaStream_t st);

// ---------------------------------------------------------------- Davidson
// out[i*out_stride] = V[i] . w for i < k (V rows of length n, leading dim ld);
// partial: k * 256 doubles of workspace. Fixed-order two-stage reduction.
void dav_dots(const double* V, long long ld, int k, const double* w, long long n, double* partial, double* out,
              int out_stride, cudaStream_t st);
// out = sign * sum_i c[i*cs] V[i]  (or out += ... when add)
void dav_lincomb(const double* V, long long ld, int k, const double* c, int cs, double sign, double* out,
                 long long n, bool add, cudaStream_t st);
// r = ax - theta x; t = r / (theta - diag) with |denominator| clamped at 1e-8
void dav_residual(const double* x, const double* ax, const double* diag, const double* theta, double* r,
                  double* t, long long n, cudaStream_t st);
// x /= sqrt(*nrm2)
void dav_scale(double* x, const double* nrm2, long long n, cudaStream_t st);
// eigenpairs (ascending) of the symmetric part of a k x k matrix, k <= 32
void dav_eigh(const double* H, int k, int ldh, double* w, double* Y, int k0, cudaStream_t st);
// x <- sign(x . z) x + a z / sqrt(z . z), with xz_zz = {x . z, z . z} on the device
void dav_axpy_unit(double* x, const double* z, const double* xz_zz, double a, long long n, cudaStream_t st);
// diagonal of H_eff from the diagonal tasks (output block = input block)
void launch_heff_diag(const double* store, const Task* tasks, const int* dstart, const int* dtask,
                      const PsiBlock* blocks, int nblk, double* diag, cudaStream_t st);

}  // namespace dmrg
