// FP64 sigma = H_eff . psi as fused back-to-back GEMMs per (term, sector).
//
// Sec. II.D-E: sigma is a sum over NC operator pairs (Eq. hpsi-thread),
// each split into dense products over symmetry sectors, with the two
// parallel levels (terms, sectors) collapsed into one flat task list. Here a
// persistent CTA takes one work item = (output block tile, run of tasks) and
// accumulates, for every task,
//     S[r0:r0+32, c0:c0+nc] += scale * (X_L[r0:, :] psi_b) X_R[c0:, :]^T
// chunk by chunk (64 columns of the intermediate at a time, the intermediate
// never leaves shared memory), then writes its partial tile to a private
// scratch slot. A second kernel sums each output tile's slots in fixed order
// (Sec. II.D's final reduction), so sigma is bitwise deterministic whatever
// the schedule of the items.
//
// The FP64 path is bound by the FP64 FMA rate, so the kernel keeps the
// operands in shared memory and uses register micro-tiles (2x4 for the first
// product, 4x10 for the second).
#include "kernels.h"

namespace dmrg {

namespace {

constexpr int TM = F64_TM;    // 32 output rows
constexpr int TN = F64_TN;    // up to 320 output columns
constexpr int NCH = 64;       // intermediate columns per chunk
constexpr int KC = 16;        // k staging depth
constexpr int NT = 256;       // threads

struct Smem {
  double A[TM][KC + 1];       // left operator tile (rows x k)
  double B[KC][NCH + 1];      // psi tile (k x chunk)
  double X[TM][NCH + 1];      // intermediate chunk
  double C[KC][TN + 1];       // right operator tile, k-major: C[k][j] = X_R(c0 + j, k)
  int item;
};

__device__ __forceinline__ double ld_op(const double* __restrict__ base, long long aoff, bool trans,
                                        int rows, int cols, int i, int k) {
  // element (i, k) of the used matrix (rows x cols); stored transposed when trans
  return trans ? base[aoff + (long long)k * rows + i] : base[aoff + (long long)i * cols + k];
}

__global__ void __launch_bounds__(NT, 1)
sigma_f64_kernel(SigmaDev a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  // step-1 micro-tile: rows 2*rp, 2*rp+1; cols cg + 16*j (j < 4)
  const int rp = tid >> 4, cg = tid & 15;

  for (;;) {
    if (tid == 0) {
      unsigned k = atomicAdd(a.counter, 1u);
      sm.item = (k < (unsigned)a.n_items) ? a.schedule[k] : -1;
    }
    __syncthreads();
    const int it_idx = sm.item;
    __syncthreads();
    if (it_idx < 0) return;
    const Item it = a.items[it_idx];
    const PsiBlock ob = a.blocks[it.out];
    const int nr = it.nrows, ncol = it.ncols;
    const int nj = (ncol + 31) >> 5;

    double s[4][10];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 10; ++j) s[i][j] = 0.0;

    for (int t = it.t_begin; t < it.t_end; ++t) {
      const Task tk = a.tasks[t];
      const PsiBlock ib = a.blocks[tk.in_blk];
      const int m = ib.mL, n = ib.mR;        // input block
      const int mo = ob.mL, no = ob.mR;      // output block
      const bool tA = tk.flags & 1, tB = tk.flags & 2;
      const double* __restrict__ psib = a.psi + ib.off;

      for (int nc0 = 0; nc0 < n; nc0 += NCH) {
        // ---- step 1: X = scale * X_L[r0:r0+nr, :] * psi_b[:, nc0:nc0+NCH]
        if (tk.aoff < 0) {
          for (int e = tid; e < TM * NCH; e += NT) {
            int i = e / NCH, j = e % NCH;
            double v = 0.0;
            if (i < nr && nc0 + j < n) v = psib[(long long)(it.r0 + i) * n + nc0 + j];
            sm.X[i][j] = tk.scale * v;
          }
        } else {
          double x[2][4];
#pragma unroll
          for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) x[i][j] = 0.0;
          for (int k0 = 0; k0 < m; k0 += KC) {
            if (!tA) {
              for (int e = tid; e < TM * KC; e += NT) {
                int i = e / KC, kk = e % KC;
                sm.A[i][kk] = (i < nr && k0 + kk < m)
                                  ? ld_op(a.store, tk.aoff, false, mo, m, it.r0 + i, k0 + kk) : 0.0;
              }
            } else {
              for (int e = tid; e < TM * KC; e += NT) {
                int kk = e / TM, i = e % TM;
                sm.A[i][kk] = (i < nr && k0 + kk < m)
                                  ? ld_op(a.store, tk.aoff, true, mo, m, it.r0 + i, k0 + kk) : 0.0;
              }
            }
            for (int e = tid; e < KC * NCH; e += NT) {
              int kk = e / NCH, j = e % NCH;
              sm.B[kk][j] = (k0 + kk < m && nc0 + j < n) ? psib[(long long)(k0 + kk) * n + nc0 + j] : 0.0;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < KC; ++kk) {
              double a0 = sm.A[2 * rp][kk], a1 = sm.A[2 * rp + 1][kk];
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                double b = sm.B[kk][cg + 16 * j];
                x[0][j] = fma(a0, b, x[0][j]);
                x[1][j] = fma(a1, b, x[1][j]);
              }
            }
            __syncthreads();
          }
#pragma unroll
          for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) sm.X[2 * rp + i][cg + 16 * j] = tk.scale * x[i][j];
        }
        __syncthreads();

        // ---- step 2: S += X * X_R[c0:c0+ncol, nc0:nc0+NCH]^T
        if (tk.boff < 0) {
          // identity on the right: output columns = input columns
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 10; ++j) {
              int col = it.c0 + lane + 32 * j - nc0;
              if (j < nj && col >= 0 && col < NCH) s[i][j] += sm.X[4 * warp + i][col];
            }
        } else {
          const int kend = min(NCH, n - nc0);
          for (int kk0 = 0; kk0 < kend; kk0 += KC) {
            if (!tB) {
              for (int e = tid; e < TN * KC; e += NT) {
                int j = e / KC, kk = e % KC;
                int k = nc0 + kk0 + kk;
                sm.C[kk][j] = (j < ncol && kk0 + kk < kend)
                                  ? ld_op(a.store, tk.boff, false, no, n, it.c0 + j, k) : 0.0;
              }
            } else {
              for (int e = tid; e < TN * KC; e += NT) {
                int kk = e / TN, j = e % TN;
                int k = nc0 + kk0 + kk;
                sm.C[kk][j] = (j < ncol && kk0 + kk < kend)
                                  ? ld_op(a.store, tk.boff, true, no, n, it.c0 + j, k) : 0.0;
              }
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < KC; ++kk) {
              double xa[4];
#pragma unroll
              for (int i = 0; i < 4; ++i) xa[i] = sm.X[4 * warp + i][kk0 + kk];
#pragma unroll
              for (int j = 0; j < 10; ++j) {
                if (j < nj) {
                  double c = sm.C[kk][lane + 32 * j];
#pragma unroll
                  for (int i = 0; i < 4; ++i) s[i][j] = fma(xa[i], c, s[i][j]);
                }
              }
            }
            __syncthreads();
          }
        }
        __syncthreads();
      }
    }
    // partial tile -> private scratch slot
    double* out = a.scratch + it.slot;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 10; ++j) {
        int r = 4 * warp + i, c = lane + 32 * j;
        if (r < nr && c < ncol) out[(long long)r * ncol + c] = s[i][j];
      }
  }
}

__global__ void reduce_kernel(SigmaDev a) {
  for (int gi = blockIdx.x; gi < a.n_groups; gi += gridDim.x) {
    const Group g = a.groups[gi];
    const PsiBlock ob = a.blocks[g.out];
    const int n = g.nrows * g.ncols;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      double acc = 0.0;
      for (int i = g.i_begin; i < g.i_end; ++i) acc += a.scratch[a.items[i].slot + e];
      int r = e / g.ncols, c = e % g.ncols;
      a.sigma[ob.off + (long long)(g.r0 + r) * ob.mR + g.c0 + c] = acc;
    }
  }
}

}  // namespace

void launch_sigma_f64(const SigmaDev& a, int n_sm, cudaStream_t st) {
  static bool attr = false;
  const int smem = (int)sizeof(Smem);
  if (!attr) {
    cudaFuncSetAttribute(sigma_f64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr = true;
  }
  int grid = n_sm;
  if (grid > a.n_items) grid = a.n_items;
  if (grid < 1) grid = 1;
  sigma_f64_kernel<<<grid, NT, smem, st>>>(a);
}

void launch_reduce(const SigmaDev& a, cudaStream_t st) {
  int grid = a.n_groups < 152 * 8 ? a.n_groups : 152 * 8;
  if (grid < 1) grid = 1;
  reduce_kernel<<<grid, 256, 0, st>>>(a);
}

}  // namespace dmrg
