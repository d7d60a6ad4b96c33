// Sweep kernels: blocking (Eq. blocked-ops), decimation (per-sector Gram
// matrix and Jacobi eigensolver), orthonormal bases for the initial MPS.
// The transformation of Eq. op-trans runs on the FP64 sigma kernel with a
// dedicated work list (see sweep.cpp).
#include "kernels.h"

namespace dmrg {

namespace {

__constant__ int c_site_n[4] = {0, 1, 1, 2};
__constant__ int c_site_s[4] = {0, 1, -1, 0};

// index of sector (n, s) in a basis sorted by (n, s), or -1
__device__ __forceinline__ int find_sector(const int* q, int nq, int n, int s) {
  int lo = 0, hi = nq - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int mn = q[2 * mid], ms = q[2 * mid + 1];
    if (mn == n && ms == s) return mid;
    if (mn < n || (mn == n && ms < s)) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

// One destination block per CTA (grid-stride): for every term of its
// operator, in order, find the block sector ib the term reads (enlarged
// input sector minus the site state's quantum numbers), the source block
// and its output sector ob, and add coef * sign * source into the chunk
// (rows of ob within Qout, columns of ib within Qin). Each destination
// element is owned by one thread (index mod blockDim) for the zeroing and
// every update, so terms are applied in order without barriers and the
// sums are deterministic. Signs: block x site takes (-1)^{N(block in)} when
// the site part is odd; site x block takes (-1)^{N(site in)} when the block
// operator is odd.
__global__ void blocking_kernel(BlockingDev d) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int bi = blockIdx.x; bi < d.ndst; bi += gridDim.x) {
    const BDst db = d.dsts[bi];
    double* dst = d.dst_store + db.off;
    const long long ne = (long long)db.rows * db.cols;
    for (long long e = tid; e < ne; e += nt) dst[e] = 0.0;
    const int qin_n = d.eq[2 * db.Qin], qin_s = d.eq[2 * db.Qin + 1];
    const int qout_n = d.eq[2 * db.Qout], qout_s = d.eq[2 * db.Qout + 1];
    for (int t = d.term_start[db.k]; t < d.term_start[db.k + 1]; ++t) {
      const BTerm tm = d.terms[t];
      const int ib = find_sector(d.bq, d.nb, qin_n - c_site_n[tm.nin], qin_s - c_site_s[tm.nin]);
      if (ib < 0) continue;
      const int c0 = d.chunk_off[db.Qin * d.nb + ib];
      if (c0 < 0) continue;
      int ob = ib, par = 0;
      long long soff = -1;
      if (tm.src >= 0) {
        const int dn = d.src_dq[2 * tm.src], ds = d.src_dq[2 * tm.src + 1];
        par = d.src_par[tm.src];
        if (!tm.trans) {
          soff = d.srcblk[(long long)tm.src * d.nb + ib];
          if (soff < 0) continue;
          ob = find_sector(d.bq, d.nb, d.bq[2 * ib] + dn, d.bq[2 * ib + 1] + ds);
        } else {
          ob = find_sector(d.bq, d.nb, d.bq[2 * ib] - dn, d.bq[2 * ib + 1] - ds);
          if (ob >= 0) soff = d.srcblk[(long long)tm.src * d.nb + ob];
          if (soff < 0) continue;
        }
        if (ob < 0) continue;
      }
      if (d.bq[2 * ob] + c_site_n[tm.nout] != qout_n || d.bq[2 * ob + 1] + c_site_s[tm.nout] != qout_s) {
        if (tid == 0) atomicExch(d.err, 1);
        continue;
      }
      const int r0 = d.chunk_off[db.Qout * d.nb + ob];
      if (r0 < 0) continue;
      const int rows = d.bdim[ob], cols = d.bdim[ib];
      bool neg;
      if (d.left) neg = ((c_site_n[tm.nout] - c_site_n[tm.nin]) & 1) && (d.bq[2 * ib] & 1);
      else neg = par && (c_site_n[tm.nin] & 1);
      const double w = neg ? -tm.coef : tm.coef;
      for (int i = 0; i < rows; ++i) {
        const long long base = (long long)(r0 + i) * db.cols + c0;
        int j = (int)(((long long)tid - base % nt + nt) % nt);  // first column this thread owns
        for (; j < cols; j += nt) {
          double v;
          if (tm.src < 0) v = (i == j) ? 1.0 : 0.0;
          else if (!tm.trans) v = d.src_store[soff + (long long)i * cols + j];
          else v = d.src_store[soff + (long long)j * rows + i];
          dst[base + j] += w * v;
        }
      }
    }
  }
}

// G[b] = X_b X_b^T (rows) or X_b^T X_b (cols) for every block b of psi.
__global__ void gram_kernel(const double* __restrict__ psi, const GramBlock* __restrict__ gb, int nb,
                            double* __restrict__ G, int left) {
  for (int b = blockIdx.y; b < nb; b += gridDim.y) {
    const GramBlock g = gb[b];
    const long long ne = (long long)g.d * g.d;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne; e += (long long)gridDim.x * blockDim.x) {
      const int i = (int)(e / g.d), j = (int)(e % g.d);
      double s = 0.0;
      if (left)
        for (int k = 0; k < g.m; ++k) s = fma(psi[g.psi_off + (long long)i * g.m + k], psi[g.psi_off + (long long)j * g.m + k], s);
      else
        for (int k = 0; k < g.m; ++k) s = fma(psi[g.psi_off + (long long)k * g.d + i], psi[g.psi_off + (long long)k * g.d + j], s);
      G[g.g_off + e] = s;
    }
  }
}

// Symmetric eigenproblem of each d x d matrix A (row-major, in place) by
// cyclic Jacobi in round-robin order: each round rotates d/2 disjoint index
// pairs at once. Q receives the eigenvectors (columns), w the eigenvalues,
// both sorted by descending eigenvalue (ties by index).
__global__ void jacobi_blocks_kernel(double* __restrict__ Aall, double* __restrict__ Qall, double* __restrict__ wall,
                                     const GramBlock* __restrict__ gb, int nb, int max_sweeps) {
  __shared__ double cs[512], sn[512];
  __shared__ int pp[512], qq[512];
  __shared__ double red[2][256];
  __shared__ int stop;
  for (int b = blockIdx.x; b < nb; b += gridDim.x) {
    const GramBlock g = gb[b];
    const int d = g.d;
    double* A = Aall + g.g_off;
    double* Q = Qall + g.g_off;
    double* w = wall + g.w_off;
    for (long long e = threadIdx.x; e < (long long)d * d; e += blockDim.x) Q[e] = (e / d == e % d) ? 1.0 : 0.0;
    __syncthreads();
    const int dp = d + (d & 1);  // players (one dummy when d is odd)
    for (int sweep = 0; sweep < max_sweeps && d > 1; ++sweep) {
      double off = 0.0, tot = 0.0;
      for (long long e = threadIdx.x; e < (long long)d * d; e += blockDim.x) {
        const double a = A[e];
        tot += a * a;
        if (e / d != e % d) off += a * a;
      }
      red[0][threadIdx.x] = off;
      red[1][threadIdx.x] = tot;
      __syncthreads();
      for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
          red[0][threadIdx.x] += red[0][threadIdx.x + h];
          red[1][threadIdx.x] += red[1][threadIdx.x + h];
        }
        __syncthreads();
      }
      if (threadIdx.x == 0) stop = (red[0][0] <= 1e-30 * red[1][0]) ? 1 : 0;
      __syncthreads();
      if (stop) break;
      for (int round = 0; round < dp - 1; ++round) {
        for (int k = threadIdx.x; k < dp / 2; k += blockDim.x) {
          auto player = [&](int i) { return i == 0 ? 0 : 1 + (i - 1 + round) % (dp - 1); };
          int p = player(k), q = player(dp - 1 - k);
          if (p > q) { const int t = p; p = q; q = t; }
          double c = 1.0, s = 0.0;
          if (q < d) {
            const double apq = A[(long long)p * d + q];
            if (apq != 0.0) {
              const double th = (A[(long long)q * d + q] - A[(long long)p * d + p]) / (2.0 * apq);
              const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
              c = 1.0 / sqrt(t * t + 1.0);
              s = t * c;
            }
          }
          cs[k] = c;
          sn[k] = s;
          pp[k] = p;
          qq[k] = q < d ? q : -1;
        }
        __syncthreads();
        // columns: A <- A J, Q <- Q J
        for (long long e = threadIdx.x; e < (long long)d * (dp / 2); e += blockDim.x) {
          const int k = (int)(e / d), r = (int)(e % d);
          if (qq[k] < 0 || sn[k] == 0.0) continue;
          const int p = pp[k], q = qq[k];
          const double c = cs[k], s = sn[k];
          const double arp = A[(long long)r * d + p], arq = A[(long long)r * d + q];
          A[(long long)r * d + p] = c * arp - s * arq;
          A[(long long)r * d + q] = s * arp + c * arq;
          const double qrp = Q[(long long)r * d + p], qrq = Q[(long long)r * d + q];
          Q[(long long)r * d + p] = c * qrp - s * qrq;
          Q[(long long)r * d + q] = s * qrp + c * qrq;
        }
        __syncthreads();
        // rows: A <- J^T A
        for (long long e = threadIdx.x; e < (long long)d * (dp / 2); e += blockDim.x) {
          const int k = (int)(e / d), col = (int)(e % d);
          if (qq[k] < 0 || sn[k] == 0.0) continue;
          const int p = pp[k], q = qq[k];
          const double c = cs[k], s = sn[k];
          const double apc = A[(long long)p * d + col], aqc = A[(long long)q * d + col];
          A[(long long)p * d + col] = c * apc - s * aqc;
          A[(long long)q * d + col] = s * apc + c * aqc;
        }
        __syncthreads();
      }
    }
    // eigenvalues = diagonal; sort descending with columns of Q (selection on thread 0)
    if (threadIdx.x == 0) {
      for (int i = 0; i < d; ++i) w[i] = A[(long long)i * d + i];
    }
    __syncthreads();
    for (int i = 0; i < d - 1; ++i) {
      __shared__ int best;
      if (threadIdx.x == 0) {
        int m = i;
        for (int j = i + 1; j < d; ++j)
          if (w[j] > w[m]) m = j;
        best = m;
        const double t = w[i];
        w[i] = w[m];
        w[m] = t;
      }
      __syncthreads();
      const int m = best;
      if (m != i)
        for (int r = threadIdx.x; r < d; r += blockDim.x) {
          const double t = Q[(long long)r * d + i];
          Q[(long long)r * d + i] = Q[(long long)r * d + m];
          Q[(long long)r * d + m] = t;
        }
      __syncthreads();
    }
    __syncthreads();
  }
}

// Orthonormalise the columns of each d x m block (row-major, in place) by
// classical Gram-Schmidt applied twice per column.
__global__ void orthonormalize_kernel(double* __restrict__ store, const GramBlock* __restrict__ gb, int nb) {
  __shared__ double coef[1024];
  __shared__ double red[256];
  for (int b = blockIdx.x; b < nb; b += gridDim.x) {
    const GramBlock g = gb[b];
    double* G = store + g.g_off;
    const int d = g.d, m = g.m;
    for (int j = 0; j < m; ++j) {
      for (int pass = 0; pass < 2; ++pass) {
        for (int i = threadIdx.x; i < j; i += blockDim.x) {
          double s = 0.0;
          for (int r = 0; r < d; ++r) s = fma(G[(long long)r * m + i], G[(long long)r * m + j], s);
          coef[i] = s;
        }
        __syncthreads();
        for (int r = threadIdx.x; r < d; r += blockDim.x) {
          double s = 0.0;
          for (int i = 0; i < j; ++i) s = fma(coef[i], G[(long long)r * m + i], s);
          G[(long long)r * m + j] -= s;
        }
        __syncthreads();
      }
      double s = 0.0;
      for (int r = threadIdx.x; r < d; r += blockDim.x) s = fma(G[(long long)r * m + j], G[(long long)r * m + j], s);
      red[threadIdx.x] = s;
      __syncthreads();
      for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
      }
      const double inv = red[0] > 0.0 ? 1.0 / sqrt(red[0]) : 0.0;
      __syncthreads();
      for (int r = threadIdx.x; r < d; r += blockDim.x) G[(long long)r * m + j] *= inv;
      __syncthreads();
    }
  }
}

// dst[b] (d x k, row-major) = first k columns of Q[b] (d x d), each column
// with the sign that makes its entry of largest magnitude positive (first
// such entry on ties). Eigenvectors carry an arbitrary sign; this fixes the
// gauge of the kept states, so a basis is a function of the wavefunction
// alone. One warp per column.
__global__ void take_columns_kernel(const double* __restrict__ Qall, const TakeBlock* __restrict__ tb, int nb,
                                    double* __restrict__ dst) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int b = blockIdx.y; b < nb; b += gridDim.y) {
    const TakeBlock t = tb[b];
    for (int c = blockIdx.x * nw + wid; c < t.k; c += gridDim.x * nw) {
      double best = -1.0, val = 0.0;
      int bi = 0x7fffffff;
      for (int r = lane; r < t.d; r += 32) {
        const double v = Qall[t.q_off + (long long)r * t.d + c];
        if (fabs(v) > best) {  // r ascends per lane, so ties keep the first
          best = fabs(v);
          bi = r;
          val = v;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        const double ov = __shfl_xor_sync(0xffffffffu, val, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
          val = ov;
        }
      }
      const double sg = val < 0.0 ? -1.0 : 1.0;
      for (int r = lane; r < t.d; r += 32)
        dst[t.dst_off + (long long)r * t.k + c] = sg * Qall[t.q_off + (long long)r * t.d + c];
    }
  }
}

}  // namespace

void launch_blocking(const BlockingDev& d, cudaStream_t st) {
  if (d.ndst <= 0) return;
  const int grid = d.ndst < 152 * 64 ? d.ndst : 152 * 64;
  blocking_kernel<<<grid, 256, 0, st>>>(d);
}

void launch_gram(const double* psi, const GramBlock* gb, int nb, double* G, bool left, cudaStream_t st) {
  if (nb <= 0) return;
  dim3 grid(32, nb < 65535 ? nb : 65535);
  gram_kernel<<<grid, 256, 0, st>>>(psi, gb, nb, G, left ? 1 : 0);
}

void launch_jacobi_blocks(double* A, double* Q, double* w, const GramBlock* gb, int nb, cudaStream_t st) {
  if (nb <= 0) return;
  jacobi_blocks_kernel<<<nb < 65535 ? nb : 65535, 256, 0, st>>>(A, Q, w, gb, nb, 40);
}

void launch_orthonormalize(double* store, const GramBlock* gb, int nb, cudaStream_t st) {
  if (nb <= 0) return;
  orthonormalize_kernel<<<nb < 65535 ? nb : 65535, 256, 0, st>>>(store, gb, nb);
}

void launch_take_columns(const double* Q, const TakeBlock* tb, int nb, double* dst, cudaStream_t st) {
  if (nb <= 0) return;
  dim3 grid(8, nb < 65535 ? nb : 65535);
  take_columns_kernel<<<grid, 256, 0, st>>>(Q, tb, nb, dst);
}

}  // namespace dmrg
