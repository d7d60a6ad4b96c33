// Davidson eigensolver on the device (FP64 control path).
//
// Appendix A (solving step, Eq. eff-eigsh) names the Davidson method. The
// steps here: projected matrix V^T H V, its eigenpairs (one-warp cyclic
// Jacobi), Ritz vector and residual, diagonal preconditioner clamped at
// 1e-8, classical Gram-Schmidt twice, thick restart from the two lowest Ritz
// vectors. Only two scalars per iteration (Ritz value, squared residual
// norm) and the new direction's norm cross to the host. All reductions are
// two-stage with a fixed order, so results are deterministic.
#include "kernels.h"

namespace dmrg {

namespace {

constexpr int RED_BLOCKS = 256;   // partial sums per dot product
constexpr int RED_THREADS = 256;

constexpr int KMAX = 32;           // vectors per dot-product call (subspace size limit)

// partial[i * RED_BLOCKS + b] = sum over block b's elements of V[i][e] * w[e],
// for all i < k in one pass: each thread keeps k running sums, then the block
// reduces them (warp shuffles, then across warps) in a fixed order.
__global__ void dots_partial(const double* __restrict__ V, long long ld, int k, const double* __restrict__ w,
                             long long n, double* __restrict__ partial) {
  __shared__ double red[RED_THREADS / 32][KMAX];
  double s[KMAX];
#pragma unroll
  for (int i = 0; i < KMAX; ++i) s[i] = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const double we = w[e];
#pragma unroll
    for (int i = 0; i < KMAX; ++i)
      if (i < k) s[i] = fma(V[i * ld + e], we, s[i]);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < KMAX; ++i) {
    if (i < k) {
      double v = s[i];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[wid][i] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < k) {
    double v = 0.0;
    for (int j = 0; j < RED_THREADS / 32; ++j) v += red[j][threadIdx.x];
    partial[threadIdx.x * RED_BLOCKS + blockIdx.x] = v;
  }
}

// out[i * out_stride] = sum_b partial[i * RED_BLOCKS + b] (fixed order); one block per i
__global__ void dots_final(const double* __restrict__ partial, int k, double* __restrict__ out, int out_stride) {
  __shared__ double red[RED_BLOCKS];
  const int i = blockIdx.x;
  red[threadIdx.x] = partial[i * RED_BLOCKS + threadIdx.x];
  __syncthreads();
  for (int h = RED_BLOCKS / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[(long long)i * out_stride] = red[0];
}

// out = sum_i c[i*cs] V[i] (+ beta * out when add)
__global__ void lincomb_kernel(const double* __restrict__ V, long long ld, int k, const double* __restrict__ c,
                               int cs, double sign, double* __restrict__ out, long long n, int add) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < k; ++i) s = fma(c[i * cs], V[i * ld + e], s);
    out[e] = add ? out[e] + sign * s : sign * s;
  }
}

// r = ax - theta x; t = r / clamp(theta - diag)
__global__ void residual_precond(const double* __restrict__ x, const double* __restrict__ ax,
                                 const double* __restrict__ diag, const double* __restrict__ theta,
                                 double* __restrict__ r, double* __restrict__ t, long long n) {
  const double th = *theta;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const double re = ax[e] - th * x[e];
    r[e] = re;
    double den = th - diag[e];
    if (fabs(den) < 1e-8) den = den < 0.0 ? -1e-8 : 1e-8;
    t[e] = re / den;
  }
}

// x <- sign(x . z) x + a z / sqrt(z . z); xz_zz = {x . z, z . z}
__global__ void axpy_unit_kernel(double* __restrict__ x, const double* __restrict__ z,
                                 const double* __restrict__ xz_zz, double a, long long n) {
  const double sg = xz_zz[0] < 0.0 ? -1.0 : 1.0;
  const double s = a / sqrt(xz_zz[1]);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    x[e] = fma(s, z[e], sg * x[e]);
}

__global__ void scale_kernel(double* __restrict__ x, const double* __restrict__ nrm2, long long n) {
  const double s = 1.0 / sqrt(*nrm2);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    x[e] *= s;
}

// Eigenpairs of the symmetric part of the k x k matrix H (row-major, leading
// dimension ldh) by cyclic Jacobi in round-robin order (Brent-Luk): each
// round rotates up to 16 disjoint index pairs at once. Four warps share the
// work (the FP64 rate of one SM sub-partition would otherwise bound it):
// pair i's rotation is computed by warp i % 4, and every thread applies the
// rotations of its warp's pairs to its row (and its column). w ascending,
// Y columns = vectors (Y row-major k x ldh). k <= 32; 128 threads.
//
// Warm start (k0 > 0): the leading k0 x k0 block of H is the previous
// projected matrix and Y holds its eigenvectors, so Q starts as
// diag(Y[:k0, :k0], 1) and A as Q^T H Q, which is diagonal except for the
// rows and columns added since; Jacobi then needs fewer sweeps.
constexpr int EIGH_WARPS = 4;
__global__ void jacobi_eigh(const double* __restrict__ H, int k, int ldh, double* __restrict__ w,
                            double* __restrict__ Y, int k0) {
  __shared__ double A[32][33];
  __shared__ double Q[32][33];
  __shared__ double T[32][33];
  __shared__ double cs[16], sn[16];
  __shared__ int pp[16], qq[16];
  __shared__ double red[2][EIGH_WARPS];
  __shared__ int stop;
  const int tid = threadIdx.x, r = tid & 31, wid = tid >> 5;
  for (int e = tid; e < k * k; e += blockDim.x) {
    const int i = e / k, c = e % k;
    A[i][c] = 0.5 * (H[i * ldh + c] + H[c * ldh + i]);
    Q[i][c] = (i < k0 && c < k0) ? Y[i * ldh + c] : (i == c ? 1.0 : 0.0);
  }
  __syncthreads();
  if (k0 > 0) {
    for (int e = tid; e < k * k; e += blockDim.x) {  // T = A Q
      const int i = e / k, c = e % k;
      double s = 0.0;
      for (int j = 0; j < k; ++j) s = fma(A[i][j], Q[j][c], s);
      T[i][c] = s;
    }
    __syncthreads();
    for (int e = tid; e < k * k; e += blockDim.x) {  // A = Q^T T, symmetrized below
      const int i = e / k, c = e % k;
      double s = 0.0;
      for (int j = 0; j < k; ++j) s = fma(Q[j][i], T[j][c], s);
      A[i][c] = s;
    }
    __syncthreads();
    for (int e = tid; e < k * k; e += blockDim.x) {
      const int i = e / k, c = e % k;
      if (c < i) T[i][c] = 0.5 * (A[i][c] + A[c][i]);
    }
    __syncthreads();
    for (int e = tid; e < k * k; e += blockDim.x) {
      const int i = e / k, c = e % k;
      if (c < i) A[i][c] = T[i][c];
      else if (c > i) A[i][c] = T[c][i];
    }
    __syncthreads();
  }
  const int kp = k + (k & 1);            // players, one dummy when k is odd
  const int npairs = kp / 2;
  for (int sweep = 0; sweep < 60 && k > 1; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int e = tid; e < k * k; e += blockDim.x) {
      const int i = e / k, c = e % k;
      const double a = A[i][c];
      tot += a * a;
      if (c != i) off += a * a;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    if (r == 0) {
      red[0][wid] = off;
      red[1][wid] = tot;
    }
    __syncthreads();
    if (tid == 0) {
      double o2 = 0.0, t2 = 0.0;
      for (int j = 0; j < EIGH_WARPS; ++j) {
        o2 += red[0][j];
        t2 += red[1][j];
      }
      stop = (o2 <= 1e-30 * t2 || o2 == 0.0) ? 1 : 0;
    }
    __syncthreads();
    if (stop) break;
    for (int round = 0; round < kp - 1; ++round) {
      // pair i = r * EIGH_WARPS + wid: lane r of warp wid
      const int i = r * EIGH_WARPS + wid;
      if (r < 4 && i < npairs) {
        auto player = [&](int x) { return x == 0 ? 0 : 1 + (x - 1 + round) % (kp - 1); };
        int p = player(i), q = player(kp - 1 - i);
        if (p > q) { const int t = p; p = q; q = t; }
        double c = 1.0, sv = 0.0;
        if (q < k) {
          const double apq = A[p][q];
          if (apq != 0.0) {
            const double th = (A[q][q] - A[p][p]) / (2.0 * apq);
            const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            sv = t * c;
          }
        }
        cs[i] = c;
        sn[i] = sv;
        pp[i] = p;
        qq[i] = q < k ? q : -1;
      }
      __syncthreads();
      // columns: A <- A J, Q <- Q J (thread (r, wid): row r, pairs wid, wid + 4, ...)
      if (r < k)
        for (int j = wid; j < npairs; j += EIGH_WARPS) {
          const int q = qq[j];
          if (q < 0 || sn[j] == 0.0) continue;
          const int p = pp[j];
          const double c = cs[j], sv = sn[j];
          const double arp = A[r][p], arq = A[r][q];
          A[r][p] = c * arp - sv * arq;
          A[r][q] = sv * arp + c * arq;
          const double qp = Q[r][p], qv = Q[r][q];
          Q[r][p] = c * qp - sv * qv;
          Q[r][q] = sv * qp + c * qv;
        }
      __syncthreads();
      // rows: A <- J^T A (thread (r, wid): column r, pairs wid, wid + 4, ...)
      if (r < k)
        for (int j = wid; j < npairs; j += EIGH_WARPS) {
          const int q = qq[j];
          if (q < 0 || sn[j] == 0.0) continue;
          const int p = pp[j];
          const double c = cs[j], sv = sn[j];
          const double apc = A[p][r], aqc = A[q][r];
          A[p][r] = c * apc - sv * aqc;
          A[q][r] = sv * apc + c * aqc;
        }
      __syncthreads();
    }
  }
  // sort ascending: rank of each eigenvalue (ties by index), then scatter
  if (tid < k) {
    const double v = A[tid][tid];
    int rank = 0;
    for (int j = 0; j < k; ++j) {
      const double u = A[j][j];
      rank += (u < v) || (u == v && j < tid);
    }
    w[rank] = v;
    for (int rr = 0; rr < k; ++rr) Y[rr * ldh + rank] = Q[rr][tid];
  }
}

}  // namespace

void dav_dots(const double* V, long long ld, int k, const double* w, long long n, double* partial, double* out,
              int out_stride, cudaStream_t st) {
  if (k <= 0) return;
  if (k > KMAX) k = KMAX;  // the subspace size is checked against this limit on the host
  dots_partial<<<RED_BLOCKS, RED_THREADS, 0, st>>>(V, ld, k, w, n, partial);
  dots_final<<<k, RED_BLOCKS, 0, st>>>(partial, k, out, out_stride);
}

void dav_lincomb(const double* V, long long ld, int k, const double* c, int cs, double sign, double* out,
                 long long n, bool add, cudaStream_t st) {
  long long grid = (n + 255) / 256;
  if (grid > 152 * 8) grid = 152 * 8;
  if (grid < 1) grid = 1;
  lincomb_kernel<<<(unsigned)grid, 256, 0, st>>>(V, ld, k, c, cs, sign, out, n, add ? 1 : 0);
}

void dav_residual(const double* x, const double* ax, const double* diag, const double* theta, double* r,
                  double* t, long long n, cudaStream_t st) {
  long long grid = (n + 255) / 256;
  if (grid > 152 * 8) grid = 152 * 8;
  if (grid < 1) grid = 1;
  residual_precond<<<(unsigned)grid, 256, 0, st>>>(x, ax, diag, theta, r, t, n);
}

void dav_scale(double* x, const double* nrm2, long long n, cudaStream_t st) {
  long long grid = (n + 255) / 256;
  if (grid > 152 * 8) grid = 152 * 8;
  if (grid < 1) grid = 1;
  scale_kernel<<<(unsigned)grid, 256, 0, st>>>(x, nrm2, n);
}

void dav_axpy_unit(double* x, const double* z, const double* xz_zz, double a, long long n, cudaStream_t st) {
  long long grid = (n + 255) / 256;
  if (grid > 152 * 8) grid = 152 * 8;
  if (grid < 1) grid = 1;
  axpy_unit_kernel<<<(unsigned)grid, 256, 0, st>>>(x, z, xz_zz, a, n);
}

void dav_eigh(const double* H, int k, int ldh, double* w, double* Y, int k0, cudaStream_t st) {
  jacobi_eigh<<<1, 32 * EIGH_WARPS, 0, st>>>(H, k, ldh, w, Y, k0 < k ? k0 : 0);
}

}  // namespace dmrg

namespace dmrg {

namespace {

// diag[b][i, j] = sum over the diagonal tasks of block b of
// scale * X_L[i, i] * X_R[j, j] (identity factors contribute 1)
__global__ void heff_diag_kernel(const double* __restrict__ store, const Task* __restrict__ tasks,
                                 const int* __restrict__ dstart, const int* __restrict__ dtask,
                                 const PsiBlock* __restrict__ blocks, int nblk, double* __restrict__ diag) {
  for (int b = blockIdx.y; b < nblk; b += gridDim.y) {
    const PsiBlock pb = blocks[b];
    const long long ne = (long long)pb.mL * pb.mR;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne; e += (long long)gridDim.x * blockDim.x) {
      const int i = (int)(e / pb.mR), j = (int)(e % pb.mR);
      double s = 0.0;
      for (int q = dstart[b]; q < dstart[b + 1]; ++q) {
        const Task t = tasks[dtask[q]];
        const double dl = t.aoff < 0 ? 1.0 : store[t.aoff + (long long)i * (pb.mL + 1)];
        const double dr = t.boff < 0 ? 1.0 : store[t.boff + (long long)j * (pb.mR + 1)];
        s = fma(t.scale * dl, dr, s);
      }
      diag[pb.off + e] = s;
    }
  }
}

}  // namespace

void launch_heff_diag(const double* store, const Task* tasks, const int* dstart, const int* dtask,
                      const PsiBlock* blocks, int nblk, double* diag, cudaStream_t st) {
  if (nblk <= 0) return;
  dim3 grid(64, nblk < 65535 ? nblk : 65535);
  heff_diag_kernel<<<grid, 256, 0, st>>>(store, tasks, dstart, dtask, blocks, nblk, diag);
}

}  // namespace dmrg
