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
// The FP64 path is bound by the FP64 multiply-add rate, which on this GPU
// is the same for the FP64 tensor instruction (mma.sync m8n8k4 .f64: 256
// multiply-adds per warp instruction) and for scalar FMAs. The tensor form
// is used because its 8x8x4 granularity keeps padding small: every output
// tile, intermediate chunk and contraction is padded only to multiples of 8
// (rows, columns) and 4 (k), instead of to whole register micro-tiles.
// Each warp owns a set of 8x8 sub-tiles of the output tile and of the
// intermediate chunk; fragments come from shared memory.
#include <mutex>
#include <set>
#include <string>
#include <tuple>

#include "../../include/dmrg.h"
#include "kernels.h"

namespace dmrg {

namespace {

constexpr int TM = F64_TM;    // 32 output rows (4 row groups of 8)
constexpr int TN = F64_TN;    // up to 256 output columns (32 column groups)
constexpr int NCH = 64;       // intermediate columns per chunk
constexpr int KC = 32;        // k staging depth of the first product
constexpr int KC2 = 16;       // k staging depth of the second product
constexpr int NT = 256;       // threads (8 warps)
constexpr int NW = NT / 32;
constexpr int XS = (TM / 8) * (NCH / 8) / NW;  // intermediate sub-tiles per warp (4)
constexpr int SS = (TM / 8) * (TN / 8) / NW;   // output sub-tiles per warp (16)

// Row strides = 4 (mod 16) doubles: a fragment load (8 rows x 4 k, or 4 k x
// 8 columns) then touches every bank pair exactly twice.
struct Smem {
  double A[TM][KC + 4];       // left operator rows x k
  double B[KC][NCH + 4];      // psi k x chunk columns
  double X[TM][NCH + 4];      // intermediate rows x chunk columns
  double C[KC2][TN + 4];      // right operator, k-major: C[k][j] = X_R(c0 + j, k)
  int item;
};

__device__ __forceinline__ double ld_op(const double* __restrict__ base, long long aoff, bool trans,
                                        int rows, int cols, int i, int k) {
  // element (i, k) of the used matrix (rows x cols); stored transposed when trans
  return trans ? base[aoff + (long long)k * rows + i] : base[aoff + (long long)i * cols + k];
}

// D = A(8x4) B(4x8) + D; lane (g = lane/4, c = lane%4) holds A[g][c],
// B[c][g] and D[g][2c], D[g][2c+1].
__device__ __forceinline__ void dmma(double (&d)[2], double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d[0]), "+d"(d[1])
               : "d"(a), "d"(b));
}

__device__ __forceinline__ int up8(int x) { return (x + 7) & ~7; }
__device__ __forceinline__ int up4(int x) { return (x + 3) & ~3; }

__global__ void __launch_bounds__(NT, 2)
sigma_f64_kernel(SigmaDev a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, c = lane & 3;

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
    const int nr8 = up8(nr), nrg = nr8 >> 3, ncg = up8(ncol) >> 3;
    const int n_s = nrg * ncg;  // output sub-tiles of this item

    double s[SS][2];
#pragma unroll
    for (int q = 0; q < SS; ++q) s[q][0] = s[q][1] = 0.0;

    for (int t = it.t_begin; t < it.t_end; ++t) {
      const Task tk = a.tasks[t];
      const PsiBlock ib = a.blocks[tk.in_blk];
      const int m = ib.mL, n = ib.mR;        // input block
      const int mo = ob.mL, no = ob.mR;      // output block
      const bool tA = tk.flags & 1, tB = tk.flags & 2;
      const double* __restrict__ psib = a.psi + ib.off;

      for (int nc0 = 0; nc0 < n; nc0 += NCH) {
        const int nch = min(NCH, n - nc0), nch8 = up8(nch), nch4 = up4(nch);
        const int xcg = nch8 >> 3, n_x = nrg * xcg;
        // ---- step 1: X = scale * X_L[r0:r0+nr, :] psi_b[:, nc0:nc0+nch]
        if (tk.aoff < 0) {
          for (int e = tid; e < nr8 * nch8; e += NT) {
            const int i = e / nch8, j = e % nch8;
            double v = 0.0;
            if (i < nr && j < nch) v = psib[(long long)(it.r0 + i) * n + nc0 + j];
            sm.X[i][j] = tk.scale * v;
          }
        } else {
          double x[XS][2];
#pragma unroll
          for (int p = 0; p < XS; ++p) x[p][0] = x[p][1] = 0.0;
          for (int k0 = 0; k0 < m; k0 += KC) {
            const int kc = min(KC, m - k0), kc4 = up4(kc);
            if (!tA) {
              for (int e = tid; e < nr8 * kc4; e += NT) {
                const int i = e / kc4, kk = e % kc4;
                sm.A[i][kk] = (i < nr && kk < kc) ? ld_op(a.store, tk.aoff, false, mo, m, it.r0 + i, k0 + kk) : 0.0;
              }
            } else {
              for (int e = tid; e < nr8 * kc4; e += NT) {
                const int kk = e / nr8, i = e % nr8;
                sm.A[i][kk] = (i < nr && kk < kc) ? ld_op(a.store, tk.aoff, true, mo, m, it.r0 + i, k0 + kk) : 0.0;
              }
            }
            for (int e = tid; e < kc4 * nch8; e += NT) {
              const int kk = e / nch8, j = e % nch8;
              sm.B[kk][j] = (kk < kc && j < nch) ? psib[(long long)(k0 + kk) * n + nc0 + j] : 0.0;
            }
            __syncthreads();
            for (int kk = 0; kk < kc4; kk += 4) {
#pragma unroll
              for (int p = 0; p < XS; ++p) {
                const int sx = warp + NW * p;
                if (sx < n_x) {
                  const int rg = sx / xcg, cg = sx - rg * xcg;
                  dmma(x[p], sm.A[rg * 8 + g][kk + c], sm.B[kk + c][cg * 8 + g]);
                }
              }
            }
            __syncthreads();
          }
#pragma unroll
          for (int p = 0; p < XS; ++p) {
            const int sx = warp + NW * p;
            if (sx < n_x) {
              const int rg = sx / xcg, cg = sx - rg * xcg;
              sm.X[rg * 8 + g][cg * 8 + 2 * c] = tk.scale * x[p][0];
              sm.X[rg * 8 + g][cg * 8 + 2 * c + 1] = tk.scale * x[p][1];
            }
          }
        }
        __syncthreads();

        // ---- step 2: S += X X_R[c0:c0+ncol, nc0:nc0+nch]^T
        if (tk.boff < 0) {
          // identity on the right: output column j reads intermediate column j
#pragma unroll
          for (int q = 0; q < SS; ++q) {
            const int ss = warp + NW * q;
            if (ss < n_s) {
              const int rg = ss / ncg, cg = ss - rg * ncg;
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const int col = it.c0 + cg * 8 + 2 * c + h - nc0;
                if (col >= 0 && col < nch) s[q][h] += sm.X[rg * 8 + g][col];
              }
            }
          }
        } else {
          const int nc8 = ncg * 8;
          for (int k0 = 0; k0 < nch4; k0 += KC2) {
            const int kc4 = min(KC2, nch4 - k0);
            if (!tB) {
              for (int e = tid; e < nc8 * kc4; e += NT) {
                const int j = e / kc4, kk = e % kc4;
                const int k = nc0 + k0 + kk;
                sm.C[kk][j] = (j < ncol && k0 + kk < nch) ? ld_op(a.store, tk.boff, false, no, n, it.c0 + j, k) : 0.0;
              }
            } else {
              for (int e = tid; e < nc8 * kc4; e += NT) {
                const int kk = e / nc8, j = e % nc8;
                const int k = nc0 + k0 + kk;
                sm.C[kk][j] = (j < ncol && k0 + kk < nch) ? ld_op(a.store, tk.boff, true, no, n, it.c0 + j, k) : 0.0;
              }
            }
            __syncthreads();
            for (int kk = 0; kk < kc4; kk += 4) {
#pragma unroll
              for (int q = 0; q < SS; ++q) {
                const int ss = warp + NW * q;
                if (ss < n_s) {
                  const int rg = ss / ncg, cg = ss - rg * ncg;
                  dmma(s[q], sm.X[rg * 8 + g][k0 + kk + c], sm.C[kk + c][cg * 8 + g]);
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
    for (int q = 0; q < SS; ++q) {
      const int ss = warp + NW * q;
      if (ss < n_s) {
        const int rg = ss / ncg, cg = ss - rg * ncg;
        const int r = rg * 8 + g;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int col = cg * 8 + 2 * c + h;
          if (r < nr && col < ncol) out[(long long)r * ncol + col] = s[q][h];
        }
      }
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

void set_max_dynamic_smem(const void* fn, int bytes) {
  static std::mutex mu;
  static std::set<std::tuple<const void*, int, int>> done;  // (kernel, device, bytes)
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) throw Error(DMRG_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  std::lock_guard<std::mutex> lk(mu);
  if (done.count({fn, dev, bytes})) return;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess)
    throw Error(DMRG_ECUDA, std::string("cudaFuncSetAttribute(max dynamic shared memory): ") + cudaGetErrorString(e));
  done.insert({fn, dev, bytes});
}

void launch_sigma_f64(const SigmaDev& a, int n_sm, cudaStream_t st) {
  const int smem = (int)sizeof(Smem);
  set_max_dynamic_smem((const void*)sigma_f64_kernel, smem);
  int grid = 2 * n_sm;  // two resident CTAs per SM overlap one's loads with the other's products
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
