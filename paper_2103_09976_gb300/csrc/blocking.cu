// Sweep kernels: blocking (Eq. blocked-ops), the normal-to-complementary
// sums of the mixed NC/CN scheme (Sec. III.A), decimation (one-sided Jacobi
// SVD of the psi blocks), orthonormal bases for the initial MPS, and the
// small GEMMs that carry a wavefunction to the next bond. The
// transformation of Eq. op-trans runs on the FP64 sigma kernel with a
// dedicated work list (see sweep.cpp).
#include <cooperative_groups.h>

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
// (rows of ob within Qout, columns of ib within Qin). Terms are resolved 256
// at a time, one per thread, into shared memory (the lookups are dependent
// global loads, so doing them in parallel hides their latency), then applied
// in term order. Each destination element (row R, column C) is owned by one
// thread - warp R mod 8, lane C mod 32 - for every update, so terms are
// applied in order without atomics and the sums are deterministic; a warp
// walks its rows of a chunk and its lanes read consecutive columns. Signs:
// block x site takes (-1)^{N(block in)} when the site part is odd; site x
// block takes (-1)^{N(site in)} when the block operator is odd.
struct RTerm {        // one resolved term
  long long soff;     // source block offset
  double w;           // coefficient times sign
  int r0, c0, rows, cols;
  int kind;           // 0 skip, 1 identity, 2 source, 3 source transposed
  int store2;         // source in the second store
};
constexpr int BLK_THREADS = 256;
static_assert(BLK_THREADS == 256, "the update ownership assumes 8 warps");

__global__ void __launch_bounds__(BLK_THREADS) blocking_kernel(BlockingDev d) {
  __shared__ RTerm rt[BLK_THREADS];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31;  // 8 warps (BLK_THREADS = 256)
  for (int bi = blockIdx.x; bi < d.ndst; bi += gridDim.x) {
    const BDst db = d.dsts[bi];
    double* dst = d.dst_store + db.off;
    const long long ne = (long long)db.rows * db.cols;
    for (long long e = tid; e < ne; e += nt) dst[e] = 0.0;
    __syncthreads();  // zeroing and the updates below own elements differently
    const int qin_n = d.eq[2 * db.Qin], qin_s = d.eq[2 * db.Qin + 1];
    const int qout_n = d.eq[2 * db.Qout], qout_s = d.eq[2 * db.Qout + 1];
    const int t_end = d.term_start[db.k + 1];
    for (int t0 = d.term_start[db.k]; t0 < t_end; t0 += nt) {
      const int nhere = min(nt, t_end - t0);
      if (tid < nhere) {
        RTerm& r = rt[tid];
        r.kind = 0;
        const BTerm tm = d.terms[t0 + tid];
        const int ib = find_sector(d.bq, d.nb, qin_n - c_site_n[tm.nin], qin_s - c_site_s[tm.nin]);
        const int c0 = ib >= 0 ? d.chunk_off[db.Qin * d.nb + ib] : -1;
        int ob = ib, par = 0;
        long long soff = -1;
        bool ok = c0 >= 0;
        if (ok && tm.src >= 0) {
          const int dn = d.src_dq[2 * tm.src], ds = d.src_dq[2 * tm.src + 1];
          par = d.src_par[tm.src];
          if (!tm.trans) {
            soff = d.srcblk[(long long)tm.src * d.nb + ib];
            ob = soff < 0 ? -1 : find_sector(d.bq, d.nb, d.bq[2 * ib] + dn, d.bq[2 * ib + 1] + ds);
          } else {
            ob = find_sector(d.bq, d.nb, d.bq[2 * ib] - dn, d.bq[2 * ib + 1] - ds);
            if (ob >= 0) soff = d.srcblk[(long long)tm.src * d.nb + ob];
          }
          ok = soff >= 0 && ob >= 0;
        }
        if (ok && (d.bq[2 * ob] + c_site_n[tm.nout] != qout_n || d.bq[2 * ob + 1] + c_site_s[tm.nout] != qout_s)) {
          atomicExch(d.err, 1);
          ok = false;
        }
        const int r0 = ok ? d.chunk_off[db.Qout * d.nb + ob] : -1;
        if (ok && r0 >= 0) {
          bool neg;
          if (d.left) neg = ((c_site_n[tm.nout] - c_site_n[tm.nin]) & 1) && (d.bq[2 * ib] & 1);
          else neg = par && (c_site_n[tm.nin] & 1);
          r.soff = soff;
          r.w = neg ? -tm.coef : tm.coef;
          r.r0 = r0;
          r.c0 = c0;
          r.rows = d.bdim[ob];
          r.cols = d.bdim[ib];
          r.kind = tm.src < 0 ? 1 : (tm.trans ? 3 : 2);
          r.store2 = tm.src >= d.nsrc1;
        }
      }
      __syncthreads();
      for (int q = 0; q < nhere; ++q) {
        const RTerm r = rt[q];
        if (r.kind == 0) continue;
        const double* __restrict__ S = r.store2 ? d.src_store2 : d.src_store;
        // rows of the destination with (row mod 8) = warp, columns with (col mod 32) = lane
        for (int i = (warp - r.r0) & 7; i < r.rows; i += 8) {
          double* drow = dst + (long long)(r.r0 + i) * db.cols + r.c0;
          for (int j = (lane - r.c0) & 31; j < r.cols; j += 32) {
            double v;
            if (r.kind == 1) v = (i == j) ? 1.0 : 0.0;
            else if (r.kind == 2) v = S[r.soff + (long long)i * r.cols + j];
            else v = S[r.soff + (long long)j * r.rows + i];
            drow[j] += r.w * v;
          }
        }
      }
      __syncthreads();
    }
  }
}

// Y_o = sum_i C[o][i] X_i for one 64 x 128 (operator, element) tile per
// iteration: the coefficient tile (64 x 16) and 16 source rows of 128
// elements are staged in shared memory, each warp owns 8 output operators x
// 128 elements (16 sub-tiles of 8 x 8) and accumulates them with the FP64
// m8n8k4 tensor instruction (lane g = lane/4, c = lane%4 holds A[g][c],
// B[c][g], D[g][2c..2c+1]). Each output element is written once.
constexpr int CB_K = 16;
struct CombSmem {
  double C[COMB_TM][CB_K + 4];
  double X[CB_K][COMB_TN + 4];
};

__device__ __forceinline__ void dmma8(double (&d)[2], double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d[0]), "+d"(d[1])
               : "d"(a), "d"(b));
}

__global__ void __launch_bounds__(256, 2)
opcomb_kernel(const double* __restrict__ src, const long long* __restrict__ xoff, const double* __restrict__ coef,
              const CombClass* __restrict__ cls, int ncls, int ntiles, double* __restrict__ dst) {
  __shared__ __align__(16) CombSmem sm;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, c = lane & 3;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int k = 0;
    while (k + 1 < ncls && cls[k + 1].tile_start <= t) ++k;
    const CombClass cc = cls[k];
    const int local = t - cc.tile_start;
    const int to = local / cc.tiles_e, te = local - to * cc.tiles_e;
    const int o0 = to * COMB_TM;
    const long long e0 = (long long)te * COMB_TN;
    double acc[COMB_TN / 8][2];
#pragma unroll
    for (int q = 0; q < COMB_TN / 8; ++q) acc[q][0] = acc[q][1] = 0.0;
    for (int i0 = 0; i0 < cc.n_in; i0 += CB_K) {
      for (int x = tid; x < COMB_TM * CB_K; x += blockDim.x) {
        const int r = x / CB_K, kk = x - r * CB_K;
        const int o = o0 + r, i = i0 + kk;
        sm.C[r][kk] = (o < cc.n_out && i < cc.n_in) ? coef[cc.c_off + (long long)o * cc.n_in + i] : 0.0;
      }
      for (int x = tid; x < CB_K * COMB_TN; x += blockDim.x) {
        const int kk = x / COMB_TN, j = x - kk * COMB_TN;
        const int i = i0 + kk;
        const long long e = e0 + j;
        sm.X[kk][j] = (i < cc.n_in && e < cc.E) ? src[xoff[cc.x_start + i] + e] : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < CB_K; kk += 4) {
        const double a = sm.C[warp * 8 + g][kk + c];
#pragma unroll
        for (int q = 0; q < COMB_TN / 8; ++q) dmma8(acc[q], a, sm.X[kk + c][q * 8 + g]);
      }
      __syncthreads();
    }
    const int o = o0 + warp * 8 + g;
    if (o < cc.n_out) {
      double* y = dst + cc.y_off + (long long)o * cc.E;
#pragma unroll
      for (int q = 0; q < COMB_TN / 8; ++q)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const long long e = e0 + q * 8 + 2 * c + h;
          if (e < cc.E) y[e] = acc[q][h];
        }
    }
  }
}

// One strided GEMM job per CTA (grid-stride): 16 x 16 output tiles, one
// element per thread, k staged in shared memory 16 at a time.
__global__ void bgemm_kernel(const double* __restrict__ A, const double* __restrict__ B, double* __restrict__ C,
                             const GJob* __restrict__ jobs, int njobs) {
  __shared__ double sa[16][17], sb[16][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int jb = blockIdx.x; jb < njobs; jb += gridDim.x) {
    const GJob g = jobs[jb];
    for (int i0 = 0; i0 < g.m; i0 += 16)
      for (int j0 = 0; j0 < g.n; j0 += 16) {
        double acc = 0.0;
        for (int k0 = 0; k0 < g.kk; k0 += 16) {
          {
            const int i = i0 + ty, k = k0 + tx;
            sa[ty][tx] = (i < g.m && k < g.kk)
                             ? A[g.a + (g.ta ? (long long)k * g.lda + i : (long long)i * g.lda + k)] : 0.0;
            const int kb = k0 + ty, j = j0 + tx;
            sb[ty][tx] = (kb < g.kk && j < g.n)
                             ? B[g.b + (g.tb ? (long long)j * g.ldb + kb : (long long)kb * g.ldb + j)] : 0.0;
          }
          __syncthreads();
#pragma unroll
          for (int q = 0; q < 16; ++q) acc = fma(sa[ty][q], sb[q][tx], acc);
          __syncthreads();
        }
        const int i = i0 + ty, j = j0 + tx;
        if (i < g.m && j < g.n) C[g.c + (long long)i * g.ldc + j] = acc;
      }
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

// ---------------------------------------------------------------- SVD
// One-sided (Hestenes) Jacobi: the d columns of A (d x m data, each column a
// contiguous vector of length m) are rotated in pairs until mutually
// orthogonal; the rotations, accumulated in V (d x d), are the singular
// vectors of the psi block's d-dimensional side, and the final column norms
// are the singular values. Pairs of one round are disjoint (round-robin
// order), so every warp of the grid takes pairs of any block, and the grid
// synchronizes between rounds.
__global__ void svd_setup_kernel(const double* __restrict__ psi, const SvdBlock* __restrict__ sb, int nb,
                                 double* __restrict__ work, int left) {
  for (int b = blockIdx.y; b < nb; b += gridDim.y) {
    const SvdBlock s = sb[b];
    const long long na = (long long)s.d * s.m;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < na; e += (long long)gridDim.x * blockDim.x) {
      const int c = (int)(e / s.m), i = (int)(e % s.m);
      // left: column c = row c of X (d = rows, m = cols); right: column c = column c of X (d = cols, m = rows)
      work[s.a_off + e] = left ? psi[s.psi_off + (long long)c * s.m + i] : psi[s.psi_off + (long long)i * s.d + c];
    }
    const long long nv = (long long)s.d * s.d;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nv; e += (long long)gridDim.x * blockDim.x)
      work[s.v_off + e] = (e / s.d == e % s.d) ? 1.0 : 0.0;
  }
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// |A|_F^2 of every block's work matrix into w[w_off] (scratch until the
// singular values are written there).
__global__ void svd_norm_kernel(const SvdBlock* __restrict__ sb, int nb, const double* __restrict__ work,
                                double* __restrict__ w) {
  __shared__ double red[32];
  for (int b = blockIdx.x; b < nb; b += gridDim.x) {
    const SvdBlock s = sb[b];
    const long long na = (long long)s.d * s.m;
    double v = 0.0;
    for (long long e = threadIdx.x; e < na; e += blockDim.x) v = fma(work[s.a_off + e], work[s.a_off + e], v);
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
      double x = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
      x = warp_sum(x);
      if (threadIdx.x == 0) w[s.w_off] = x;
    }
    __syncthreads();
  }
}

// A pair is rotated while its cosine |a_p . a_q| / (|a_p| |a_q|) exceeds
// tol = max(1e-15, eps sqrt(m)) (the rounding floor of an m-term dot
// product), and only if both vectors exceed 1e-15 |A|_F: vectors below that
// are numerical zeros (a block with more rows than columns has them), whose
// mutual cosines are rounding noise and would never settle. Sweeps stop when
// no pair of any block is above its tolerance (at most 30).
__global__ void svd_jacobi_kernel(const SvdBlock* __restrict__ sb, int nb, int total_pairs, int max_rounds,
                                  double* __restrict__ work, const double* __restrict__ fro,
                                  unsigned long long* __restrict__ off_max) {
  namespace cgp = cooperative_groups;
  cgp::grid_group grid = cgp::this_grid();
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (int sweep = 0; sweep < 30; ++sweep) {
    const int slot = sweep & 1;
    double local = 0.0;
    for (int round = 0; round < max_rounds; ++round) {
      for (long long pid = warp; pid < total_pairs; pid += nwarps) {
        int lo = 0, hi = nb - 1;  // block of pair pid: last b with pair0 <= pid
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (sb[mid].pair0 <= pid) lo = mid;
          else hi = mid - 1;
        }
        const SvdBlock s = sb[lo];
        const int i = (int)(pid - s.pair0);
        if (i >= s.npairs || s.rounds <= 0) continue;
        const int dp = s.d + (s.d & 1), r = round % s.rounds;
        auto player = [&](int x) { return x == 0 ? 0 : 1 + (x - 1 + r) % (dp - 1); };
        int p = player(i), q = player(dp - 1 - i);
        if (p > q) { const int t = p; p = q; q = t; }
        if (q >= s.d) continue;
        double* ap = work + s.a_off + (long long)p * s.m;
        double* aq = work + s.a_off + (long long)q * s.m;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int e = lane; e < s.m; e += 32) {
          const double x = ap[e], y = aq[e];
          al = fma(x, x, al);
          be = fma(y, y, be);
          ga = fma(x, y, ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        const double floor2 = 1e-30 * fro[s.w_off];
        if (ga == 0.0 || al <= floor2 || be <= floor2) continue;
        const double tol = fmax(1e-15, 2.220446049250313e-16 * sqrt((double)s.m));
        const double cosv = fabs(ga) / sqrt(al * be);
        local = fmax(local, cosv / tol);
        if (cosv < tol) continue;
        const double zeta = (be - al) / (2.0 * ga);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
        for (int e = lane; e < s.m; e += 32) {
          const double x = ap[e], y = aq[e];
          ap[e] = c * x - sn * y;
          aq[e] = sn * x + c * y;
        }
        double* vp = work + s.v_off + (long long)p * s.d;
        double* vq = work + s.v_off + (long long)q * s.d;
        for (int e = lane; e < s.d; e += 32) {
          const double x = vp[e], y = vq[e];
          vp[e] = c * x - sn * y;
          vq[e] = sn * x + c * y;
        }
      }
      grid.sync();
    }
    if (lane == 0 && local > 0.0) atomicMax(off_max + slot, (unsigned long long)__double_as_longlong(local));
    grid.sync();
    const double worst = __longlong_as_double((long long)off_max[slot]);
    if (blockIdx.x == 0 && threadIdx.x == 0) off_max[slot ^ 1] = 0ull;
    grid.sync();
    if (worst < 1.0) break;
  }
}

// singular values (column norms) sorted descending (ties by index); Q row r,
// column rank(c) = V[c][r]
__global__ void svd_finish_kernel(const SvdBlock* __restrict__ sb, int nb, const double* __restrict__ work,
                                  double* __restrict__ Q, double* __restrict__ w) {
  extern __shared__ double sig[];
  for (int b = blockIdx.x; b < nb; b += gridDim.x) {
    const SvdBlock s = sb[b];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = wid; c < s.d; c += nw) {
      const double* a = work + s.a_off + (long long)c * s.m;
      double v = 0.0;
      for (int e = lane; e < s.m; e += 32) v = fma(a[e], a[e], v);
      v = warp_sum(v);
      if (lane == 0) sig[c] = v;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < s.d; c += blockDim.x) {
      const double v = sig[c];
      int rank = 0;
      for (int j = 0; j < s.d; ++j) rank += (sig[j] > v) || (sig[j] == v && j < c);
      w[s.w_off + rank] = v;
      for (int r = 0; r < s.d; ++r) Q[s.q_off + (long long)r * s.d + rank] = work[s.v_off + (long long)c * s.d + r];
    }
    __syncthreads();
  }
}

}  // namespace

void launch_blocking(const BlockingDev& d, cudaStream_t st) {
  if (d.ndst <= 0) return;
  const int grid = d.ndst < 152 * 64 ? d.ndst : 152 * 64;
  blocking_kernel<<<grid, BLK_THREADS, 0, st>>>(d);
}

void launch_opcomb(const double* src, const long long* xoff, const double* coef, const CombClass* cls, int ncls,
                   int ntiles, double* dst, cudaStream_t st) {
  if (ntiles <= 0) return;
  const int grid = ntiles < 152 * 2 * 8 ? ntiles : 152 * 2 * 8;
  opcomb_kernel<<<grid, 256, 0, st>>>(src, xoff, coef, cls, ncls, ntiles, dst);
}

void launch_bgemm(const double* A, const double* B, double* C, const GJob* jobs, int njobs, cudaStream_t st) {
  if (njobs <= 0) return;
  bgemm_kernel<<<njobs < 152 * 16 ? njobs : 152 * 16, 256, 0, st>>>(A, B, C, jobs, njobs);
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

namespace dmrg {

void launch_svd_blocks(const double* psi, const SvdBlock* sb, int nb, int total_pairs, int max_rounds, int max_d_hint,
                       double* Q, double* w, double* work, bool left, int n_sm, cudaStream_t st) {
  if (nb <= 0) return;
  if ((size_t)max_d_hint * sizeof(double) > 48 * 1024)
    set_max_dynamic_smem((const void*)svd_finish_kernel, (int)((size_t)max_d_hint * sizeof(double)));
  {
    dim3 grid(32, nb < 65535 ? nb : 65535);
    svd_setup_kernel<<<grid, 256, 0, st>>>(psi, sb, nb, work, left ? 1 : 0);
  }
  if (total_pairs > 0 && max_rounds > 0) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, svd_jacobi_kernel, 256, 0);
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 4) per_sm = 4;
    int grid = n_sm * per_sm;
    unsigned long long* off_max = reinterpret_cast<unsigned long long*>(work);  // first 2 words of work
    cudaMemsetAsync(off_max, 0, 2 * sizeof(unsigned long long), st);
    svd_norm_kernel<<<nb < 65535 ? nb : 65535, 256, 0, st>>>(sb, nb, work, w);
    const double* fro = w;
    void* args[] = {(void*)&sb,   (void*)&nb,  (void*)&total_pairs, (void*)&max_rounds,
                    (void*)&work, (void*)&fro, (void*)&off_max};
    const cudaError_t e = cudaLaunchCooperativeKernel((void*)svd_jacobi_kernel, dim3(grid), dim3(256), args, 0, st);
    if (e != cudaSuccess) return;  // the caller's cudaGetLastError reports it
  }
  svd_finish_kernel<<<nb < 65535 ? nb : 65535, 256, (size_t)max_d_hint * sizeof(double), st>>>(sb, nb, work, Q, w);
}

}  // namespace dmrg
