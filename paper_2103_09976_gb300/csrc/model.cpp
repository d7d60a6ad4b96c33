// Host-side model: bases, NC operator tables, terms, sigma work lists.
#include "model.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <numeric>
#include <thread>

namespace dmrg {

void Basis::finish() {
  for (size_t i = 1; i < q.size(); ++i)
    if (!(q[i - 1] < q[i])) throw Error(1, "sectors must be strictly ascending in (N, 2Sz)");
  off.assign(q.size() + 1, 0);
  for (size_t i = 0; i < q.size(); ++i) {
    if (dim[i] <= 0) throw Error(1, "sector dimensions must be positive");
    off[i + 1] = off[i] + dim[i];
  }
  total = off.back();
}

int Basis::find(QN x) const {
  auto it = std::lower_bound(q.begin(), q.end(), x);
  if (it == q.end() || !(*it == x)) return -1;
  return (int)(it - q.begin());
}

void add_op(OpSet& set, QN dq, int parity, bool sym, long long& cursor) {
  OpDesc d;
  d.dq = dq;
  d.parity = parity;
  d.sym = sym;
  const Basis& b = set.basis;
  d.by_qin.assign(b.size(), -1);
  for (int i = 0; i < b.size(); ++i) {
    int o = b.find(b.q[i] + dq);
    if (o < 0) continue;
    OpBlock blk{i, o, b.dim[o], b.dim[i], cursor};
    cursor += (long long)blk.rows * blk.cols;
    d.by_qin[i] = (int)d.blocks.size();
    d.blocks.push_back(blk);
  }
  set.ops.push_back(std::move(d));
}

void build_nc_opset(OpSet& out, const Basis& basis, int nL, int n, bool left, long long base, bool cn) {
  out.basis = basis;
  out.ops.clear();
  long long cur = base;
  NCIndex ix{nL, n, cn};
  add_op(out, {0, 0}, 0, true, cur);  // H
  if (left) {
    for (int p = 0; p < nL; ++p) add_op(out, {1, spin_of(p)}, 1, false, cur);        // a+_p
    for (int p = nL; p < n; ++p) add_op(out, {-1, -spin_of(p)}, 1, false, cur);      // R^L_p
  } else {
    for (int p = nL; p < n; ++p) add_op(out, {-1, -spin_of(p)}, 1, false, cur);      // a_p
    for (int p = 0; p < nL; ++p) add_op(out, {-1, -spin_of(p)}, 1, false, cur);      // R^R_p
  }
  // normal pairs (A, B: creation shift) on the NC left and CN right, complementary
  // pairs (P, Q: the adjoint shift) on the NC right and CN left
  const int sgn = left != cn ? 1 : -1;
  const int p0 = ix.pb(), p1 = ix.pb() + ix.np();
  for (int p = p0; p < p1; ++p)
    for (int r = p + 1; r < p1; ++r)  // A_pr / P_pr
      add_op(out, {2 * sgn, sgn * (spin_of(p) + spin_of(r))}, 0, false, cur);
  for (int p = p0; p < p1; ++p)
    for (int q = p; q < p1; ++q)  // B_pq / Q_pq
      add_op(out, {0, sgn * (spin_of(p) - spin_of(q))}, 0, p == q, cur);
  if ((int)out.ops.size() != ix.count()) throw Error(1, "internal: NC operator count");
  out.elements = cur - base;
}

std::vector<Term> nc_terms(int nL, int n) {
  NCIndex ix{nL, n};
  std::vector<Term> T;
  T.push_back({ix.H(), -1, false, false, 1.0, 0});
  T.push_back({-1, ix.H(), false, false, 1.0, 0});
  for (int p = 0; p < nL; ++p) {
    T.push_back({ix.cd(p), ix.RR(p), false, false, 1.0, 1});
    T.push_back({ix.cd(p), ix.RR(p), true, true, -1.0, 1});
  }
  for (int p = nL; p < n; ++p) {
    T.push_back({ix.RL(p), ix.d(p), true, false, 1.0, 1});
    T.push_back({ix.RL(p), ix.d(p), false, true, -1.0, 1});
  }
  for (int p = 0; p < nL; ++p)
    for (int r = p + 1; r < nL; ++r) {
      T.push_back({ix.A(p, r), ix.A(p, r), false, false, 1.0, 0});
      T.push_back({ix.A(p, r), ix.A(p, r), true, true, 1.0, 0});
    }
  for (int p = 0; p < nL; ++p)
    for (int q = 0; q < nL; ++q) {
      if (p <= q)
        T.push_back({ix.B(p, q), ix.B(p, q), false, false, 1.0, 0});
      else
        T.push_back({ix.B(q, p), ix.B(q, p), true, true, 1.0, 0});
    }
  return T;
}

std::vector<Term> cn_terms(int nL, int n) {
  NCIndex ix{nL, n, true};
  std::vector<Term> T;
  T.push_back({ix.H(), -1, false, false, 1.0, 0});
  T.push_back({-1, ix.H(), false, false, 1.0, 0});
  for (int p = 0; p < nL; ++p) {
    T.push_back({ix.cd(p), ix.RR(p), false, false, 1.0, 1});
    T.push_back({ix.cd(p), ix.RR(p), true, true, -1.0, 1});
  }
  for (int p = nL; p < n; ++p) {
    T.push_back({ix.RL(p), ix.d(p), true, false, 1.0, 1});
    T.push_back({ix.RL(p), ix.d(p), false, true, -1.0, 1});
  }
  for (int p = nL; p < n; ++p)
    for (int r = p + 1; r < n; ++r) {
      T.push_back({ix.A(p, r), ix.A(p, r), false, false, 1.0, 0});
      T.push_back({ix.A(p, r), ix.A(p, r), true, true, 1.0, 0});
    }
  for (int p = nL; p < n; ++p)
    for (int q = nL; q < n; ++q) {
      if (p <= q)
        T.push_back({ix.B(p, q), ix.B(p, q), false, false, 1.0, 0});
      else
        T.push_back({ix.B(q, p), ix.B(q, p), true, true, 1.0, 0});
    }
  return T;
}

std::vector<int> nc_term_ranks(int nL, int n, int n_ranks) {
  // same enumeration order as nc_terms
  std::vector<int> r;
  auto one = [&](int p) { return p % n_ranks; };
  auto two = [&](int p, int q) {
    const int i = std::min(p, q), j = std::max(p, q);
    return (int)(((long long)j * (j + 1) / 2 + i) % n_ranks);
  };
  r.push_back(0);
  r.push_back(0);
  for (int p = 0; p < nL; ++p) r.insert(r.end(), 2, one(p));
  for (int p = nL; p < n; ++p) r.insert(r.end(), 2, one(p));
  for (int p = 0; p < nL; ++p)
    for (int q = p + 1; q < nL; ++q) r.insert(r.end(), 2, two(p, q));
  for (int p = 0; p < nL; ++p)
    for (int q = 0; q < nL; ++q) r.push_back(two(p, q));
  return r;
}

std::vector<int> cn_term_ranks(int nL, int n, int n_ranks) {
  // same enumeration order as cn_terms
  std::vector<int> r;
  auto one = [&](int p) { return p % n_ranks; };
  auto two = [&](int p, int q) {
    const int i = std::min(p, q), j = std::max(p, q);
    return (int)(((long long)j * (j + 1) / 2 + i) % n_ranks);
  };
  r.push_back(0);
  r.push_back(0);
  for (int p = 0; p < nL; ++p) r.insert(r.end(), 2, one(p));
  for (int p = nL; p < n; ++p) r.insert(r.end(), 2, one(p));
  for (int p = nL; p < n; ++p)
    for (int q = p + 1; q < n; ++q) r.insert(r.end(), 2, two(p, q));
  for (int p = nL; p < n; ++p)
    for (int q = nL; q < n; ++q) r.push_back(two(p, q));
  return r;
}

void partition_nc(OpSet& L, OpSet& R, int nL, int n, int rank, int n_ranks, Partition& out) {
  if (n_ranks < 1 || rank < 0 || rank >= n_ranks) throw Error(1, "need 0 <= rank < n_ranks");
  const std::vector<Term> all = nc_terms(nL, n);
  const std::vector<int> rk = nc_term_ranks(nL, n, n_ranks);
  if (rk.size() != all.size()) throw Error(1, "internal: term rank count");
  out = Partition();
  std::vector<char> useL(L.ops.size(), 0), useR(R.ops.size(), 0);
  for (size_t t = 0; t < all.size(); ++t) {
    if (rk[t] != rank) continue;
    out.terms.push_back(all[t]);
    out.term_ids.push_back((int)t);
    if (all[t].opL >= 0) useL.at(all[t].opL) = 1;
    if (all[t].opR >= 0) useR.at(all[t].opR) = 1;
  }
  long long cur = 0;
  auto relayout = [&](OpSet& S, const std::vector<char>& use) {
    const long long start = cur;
    for (size_t k = 0; k < S.ops.size(); ++k) {
      OpDesc& o = S.ops[k];
      if (!use[k]) {
        o.blocks.clear();
        std::fill(o.by_qin.begin(), o.by_qin.end(), -1);
        continue;
      }
      for (OpBlock& b : o.blocks) {
        out.canon_off.push_back(b.off);
        b.off = cur;
        cur += (long long)b.rows * b.cols;
      }
    }
    S.elements = cur - start;
  };
  relayout(L, useL);
  relayout(R, useR);
  out.elements = cur;
}

std::vector<PsiBlock> psi_layout(const Basis& L, const Basis& R, QN Qtot, long long* size) {
  std::vector<PsiBlock> out;
  long long off = 0;
  for (int i = 0; i < L.size(); ++i) {
    int j = R.find(Qtot - L.q[i]);
    if (j < 0) continue;
    out.push_back({i, j, L.dim[i], R.dim[j], off});
    off += (long long)L.dim[i] * R.dim[j];
  }
  if (size) *size = off;
  return out;
}

// Resolve the block of `op` (optionally transposed) acting on input sector
// qin; returns the output sector (or -1) and the stored block.
static int resolve(const OpDesc& op, const Basis& b, int qin, bool trans, const OpBlock** blk) {
  if (!trans) {
    int k = op.by_qin[qin];
    if (k < 0) return -1;
    *blk = &op.blocks[k];
    return op.blocks[k].qout;
  }
  // (S^T)[qout <- qin] = S[qin <- qout]^T: the stored block whose input is qout
  int qout = b.find(b.q[qin] - op.dq);
  if (qout < 0) return -1;
  int k = op.by_qin[qout];
  if (k < 0) return -1;
  *blk = &op.blocks[k];
  return qout;
}

void build_tasks(const std::vector<PsiBlock>& blocks, const OpSet& L, const OpSet& R,
                 const std::vector<Term>& terms, WorkList& wl) {
  // output block index by left sector
  std::vector<int> blk_of_qL(L.basis.size(), -1);
  for (size_t b = 0; b < blocks.size(); ++b) blk_of_qL[blocks[b].qL] = (int)b;
  // first stored-block index of every operator (left operators, then right)
  std::vector<int> first_L(L.ops.size()), first_R(R.ops.size());
  int nblk = 0;
  for (size_t k = 0; k < L.ops.size(); ++k) {
    first_L[k] = nblk;
    nblk += (int)L.ops[k].blocks.size();
  }
  for (size_t k = 0; k < R.ops.size(); ++k) {
    first_R[k] = nblk;
    nblk += (int)R.ops[k].blocks.size();
  }
  struct TaskB {
    Task k;
    int a, b;
  };
  // terms are split into contiguous ranges handled by up to 8 threads; each
  // range keeps its tasks per output block, and the ranges are joined in
  // term order, so the list is the same as a sequential pass over the terms
  const size_t nterm = terms.size();
  const int nth = (int)std::min<size_t>(8, std::max<size_t>(1, std::min<size_t>(std::thread::hardware_concurrency(),
                                                                                  nterm * blocks.size() / 200000)));
  std::vector<std::vector<std::vector<TaskB>>> per_out(nth, std::vector<std::vector<TaskB>>(blocks.size()));
  std::vector<double> th_flops(nth, 0.0), th_bytes(nth, 0.0);
  auto work = [&](int th) {
    const size_t t_lo = nterm * th / nth, t_hi = nterm * (th + 1) / nth;
    double flops = 0, bytes = 0;
    for (size_t ti = t_lo; ti < t_hi; ++ti) {
      const Term& t = terms[ti];
      for (size_t b = 0; b < blocks.size(); ++b) {
        const PsiBlock& in = blocks[b];
        int qLo = in.qL, qRo = in.qR;
        const OpBlock* bl = nullptr;
        const OpBlock* br = nullptr;
        if (t.opL >= 0) {
          qLo = resolve(L.ops[t.opL], L.basis, in.qL, t.tL, &bl);
          if (qLo < 0) continue;
        }
        if (t.opR >= 0) {
          qRo = resolve(R.ops[t.opR], R.basis, in.qR, t.tR, &br);
          if (qRo < 0) continue;
        }
        int ob = blk_of_qL[qLo];
        if (ob < 0 || blocks[ob].qR != qRo) continue;
        double sign = (t.parR && (L.basis.q[in.qL].n & 1)) ? -1.0 : 1.0;
        Task k;
        k.aoff = bl ? bl->off : -1;
        k.boff = br ? br->off : -1;
        k.in_blk = (int)b;
        k.flags = (t.tL ? 1 : 0) | (t.tR ? 2 : 0);
        k.scale = t.coef * sign;
        const int ia = bl ? first_L[t.opL] + (int)(bl - L.ops[t.opL].blocks.data()) : -1;
        const int ib = br ? first_R[t.opR] + (int)(br - R.ops[t.opR].blocks.data()) : -1;
        per_out[th][ob].push_back({k, ia, ib});
        double m = in.mL, nn = in.mR, mo = blocks[ob].mL, no = blocks[ob].mR;
        if (!bl)
          flops += 2 * m * nn * no;
        else if (!br)
          flops += 2 * mo * m * nn;
        else
          flops += std::min(2 * mo * m * nn + 2 * mo * nn * no, 2 * m * nn * no + 2 * mo * m * no);
        if (bl) bytes += 8.0 * mo * m;
        if (br) bytes += 8.0 * no * nn;
      }
    }
    th_flops[th] = flops;
    th_bytes[th] = bytes;
  };
  if (nth == 1) {
    work(0);
  } else {
    std::vector<std::thread> pool;
    for (int th = 0; th < nth; ++th) pool.emplace_back(work, th);
    for (auto& x : pool) x.join();
  }
  double flops = 0, bytes = 0;
  for (int th = 0; th < nth; ++th) {
    flops += th_flops[th];
    bytes += th_bytes[th];
  }
  wl.tasks.clear();
  wl.flops = flops;
  wl.bytes_ops = bytes;
  wl.out_start.assign(blocks.size() + 1, 0);
  for (size_t b = 0; b < blocks.size(); ++b) {
    size_t nb = 0;
    for (int th = 0; th < nth; ++th) nb += per_out[th][b].size();
    wl.out_start[b + 1] = wl.out_start[b] + (int)nb;
  }
  wl.tasks.reserve(wl.out_start.back());
  wl.task_ablk.clear();
  wl.task_bblk.clear();
  wl.task_ablk.reserve(wl.out_start.back());
  wl.task_bblk.reserve(wl.out_start.back());
  for (size_t b = 0; b < blocks.size(); ++b)
    for (int th = 0; th < nth; ++th)
      for (const TaskB& x : per_out[th][b]) {
        wl.tasks.push_back(x.k);
        wl.task_ablk.push_back(x.a);
        wl.task_bblk.push_back(x.b);
      }
  wl.items.clear();
  wl.groups.clear();
  wl.schedule.clear();
}

// Cost of one task on one output tile as the FP64 kernel executes it: the
// multiply-adds of its 8x8x4 tensor instructions (rows and columns padded to
// 8, contractions to 4, the intermediate in 64-column chunks) plus a fixed
// per-task latency term. Items are split and ordered (largest first) by it.
static double tile_cost(const Task& k, const PsiBlock& in, int nr, int nc, double per_task) {
  auto up8 = [](int x) { return (double)((x + 7) & ~7); };
  auto up4 = [](int x) { return (double)((x + 3) & ~3); };
  double c = per_task;
  for (int nc0 = 0; nc0 < in.mR; nc0 += 64) {
    const int nch = std::min(64, in.mR - nc0);
    if (k.aoff >= 0) c += 2.0 * up8(nr) * up4(in.mL) * up8(nch);
    if (k.boff >= 0) c += 2.0 * up8(nr) * up4(nch) * up8(nc);
  }
  return c;
}

void build_items(const std::vector<PsiBlock>& blocks, WorkList& wl, const TileShape& ts,
                 int want_items, int n_out) {
  // output blocks are blocks[0, n_out); inputs may follow them
  const size_t nb = n_out < 0 ? blocks.size() : (size_t)n_out;
  wl.items.clear();
  wl.groups.clear();
  wl.scratch_elems = 0;
  double total = 0;
  for (size_t b = 0; b < nb; ++b)
    for (int t = wl.out_start[b]; t < wl.out_start[b + 1]; ++t)
      total += tile_cost(wl.tasks[t], blocks[wl.tasks[t].in_blk], blocks[b].mL, blocks[b].mR, ts.per_task);
  double target = std::max(ts.target, total / std::max(1, want_items));
  std::vector<double> cost;
  for (size_t b = 0; b < nb; ++b) {
    const PsiBlock& ob = blocks[b];
    int t0 = wl.out_start[b], t1 = wl.out_start[b + 1];
    if (t0 == t1) {
      // no contribution: one empty item writes zeros
      for (int r0 = 0; r0 < ob.mL; r0 += ts.tm)
        for (int c0 = 0; c0 < ob.mR; c0 += ts.tn) {
          Group g{(int)b, r0, std::min(ts.tm, ob.mL - r0), c0, std::min(ts.tn, ob.mR - c0),
                  (int)wl.items.size(), (int)wl.items.size() + 1, 0};
          Item it{(int)b, g.r0, g.nrows, g.c0, g.ncols, t0, t0, 0, wl.scratch_elems};
          wl.scratch_elems += (long long)g.nrows * g.ncols;
          wl.items.push_back(it);
          cost.push_back(0);
          wl.groups.push_back(g);
        }
      continue;
    }
    for (int r0 = 0; r0 < ob.mL; r0 += ts.tm) {
      int nr = std::min(ts.tm, ob.mL - r0);
      for (int c0 = 0; c0 < ob.mR; c0 += ts.tn) {
        int nc = std::min(ts.tn, ob.mR - c0);
        Group g{(int)b, r0, nr, c0, nc, (int)wl.items.size(), 0, 0};
        int start = t0;
        double acc = 0;
        for (int t = t0; t < t1; ++t) {
          double c = tile_cost(wl.tasks[t], blocks[wl.tasks[t].in_blk], nr, nc, ts.per_task);
          if (acc > 0 && acc + c > target) {
            wl.items.push_back({(int)b, r0, nr, c0, nc, start, t, 0, wl.scratch_elems});
            wl.scratch_elems += (long long)nr * nc;
            cost.push_back(acc);
            start = t;
            acc = 0;
          }
          acc += c;
        }
        wl.items.push_back({(int)b, r0, nr, c0, nc, start, t1, 0, wl.scratch_elems});
        wl.scratch_elems += (long long)nr * nc;
        cost.push_back(acc);
        g.i_end = (int)wl.items.size();
        wl.groups.push_back(g);
      }
    }
  }
  wl.schedule.resize(wl.items.size());
  std::iota(wl.schedule.begin(), wl.schedule.end(), 0);
  std::stable_sort(wl.schedule.begin(), wl.schedule.end(),
                   [&](int a, int b) { return cost[a] > cost[b]; });
}

}  // namespace dmrg

namespace dmrg {

static inline int ceil8(int x) { return (x + 7) / 8; }
static inline int up16(int x) { return (x + 15) & ~15; }

void build_tc_plan(const std::vector<PsiBlock>& blocks, const OpSet& L, const OpSet& R,
                   const WorkList& wl, TcPlan& plan, const TcShape& shape) {
  plan = TcPlan();
  // tiles of every stored block, in store order, then identity blocks
  std::vector<long long> offs;
  long long tile = 0;
  for (const OpSet* s : {&L, &R})
    for (const OpDesc& o : s->ops)
      for (const OpBlock& b : o.blocks) {
        TcBlock t{tile, ceil8(b.rows), ceil8(b.cols)};
        tile += (long long)t.R8 * t.C8;
        plan.opblocks.push_back(t);
        offs.push_back(b.off);
      }
  if (!std::is_sorted(offs.begin(), offs.end())) throw Error(1, "internal: operator blocks out of store order");
  auto find_off = [&](long long off) {  // index of the stored block at element offset off, or -1
    const auto it = std::lower_bound(offs.begin(), offs.end(), off);
    return (it == offs.end() || *it != off) ? -1 : (int)(it - offs.begin());
  };
  for (int i = 0; i < L.basis.size(); ++i) {
    TcBlock t{tile, ceil8(L.basis.dim[i]), ceil8(L.basis.dim[i])};
    tile += (long long)t.R8 * t.C8;
    plan.identL.push_back(t);
  }
  for (int i = 0; i < R.basis.size(); ++i) {
    TcBlock t{tile, ceil8(R.basis.dim[i]), ceil8(R.basis.dim[i])};
    tile += (long long)t.R8 * t.C8;
    plan.identR.push_back(t);
  }
  plan.n_tiles = tile + 64;  // slack: operand reads past the last tile stay in bounds
  long long pt = 0;
  for (const PsiBlock& b : blocks) {
    TcPsiBlock p{pt, 2 * ((b.mL + 15) / 16), ceil8(b.mR), b.mL, b.mR};
    pt += (long long)p.R8 * p.C8;
    plan.psi.push_back(p);
  }
  plan.psi_tiles = pt + 64;

  // one record per task: its stored blocks (identity factors made explicit)
  struct Base {
    long long a_tile, b_tile;
    int aR8, aC8, bR8, bC8;
    int in_blk, flags;
    float scale;
    int task;
    int a_blk, b_blk;  // split-block indices: stored blocks, then identities of the left and right sectors
  };
  const bool have_idx = wl.task_ablk.size() == wl.tasks.size() && wl.task_bblk.size() == wl.tasks.size();
  const size_t nblk = blocks.size();
  // output blocks are independent: contiguous block ranges of about equal
  // task counts are planned by up to 8 threads and joined in block order,
  // so the plan is the same as one pass over the blocks
  const int nparts = (int)std::min<size_t>(8, std::max<size_t>(1, std::min<size_t>(std::thread::hardware_concurrency(),
                                                                                     wl.tasks.size() / 100000)));
  std::vector<size_t> bstart(nparts + 1, nblk);
  bstart[0] = 0;
  for (int j = 1; j < nparts; ++j) {
    const long long goal = (long long)wl.tasks.size() * j / nparts;
    bstart[j] = (size_t)(std::lower_bound(wl.out_start.begin(), wl.out_start.begin() + nblk, (int)goal) -
                         wl.out_start.begin());
    bstart[j] = std::max(bstart[j], bstart[j - 1]);
  }
  auto in_parallel = [&](const std::function<void(int)>& fn) {
    if (nparts == 1) {
      fn(0);
      return;
    }
    std::vector<std::thread> pool;
    for (int j = 0; j < nparts; ++j) pool.emplace_back(fn, j);
    for (auto& x : pool) x.join();
  };
  std::vector<Base> base(wl.tasks.size());
  std::vector<char> bad(nparts, 0);
  in_parallel([&](int j) {
    for (int t = wl.out_start[bstart[j]]; t < wl.out_start[bstart[j + 1]]; ++t) {
      const Task& k = wl.tasks[t];
      const PsiBlock& in = blocks[k.in_blk];
      TcBlock a = plan.identL[in.qL], b = plan.identR[in.qR];
      int ab = (int)offs.size() + in.qL, bb = (int)offs.size() + L.basis.size() + in.qR;
      if (k.aoff >= 0) {
        const int f = have_idx ? wl.task_ablk[t] : find_off(k.aoff);
        if (f < 0 || f >= (int)offs.size() || offs[f] != k.aoff) bad[j] = 1;
        else {
          a = plan.opblocks[f];
          ab = f;
        }
      }
      if (k.boff >= 0) {
        const int f = have_idx ? wl.task_bblk[t] : find_off(k.boff);
        if (f < 0 || f >= (int)offs.size() || offs[f] != k.boff) bad[j] = 1;
        else {
          b = plan.opblocks[f];
          bb = f;
        }
      }
      Base x;
      x.a_blk = ab;
      x.b_blk = bb;
      x.a_tile = a.tile;
      x.aR8 = a.R8;
      x.aC8 = a.C8;
      x.b_tile = b.tile;
      x.bR8 = b.R8;
      x.bC8 = b.C8;
      x.in_blk = k.in_blk;
      x.flags = (k.aoff >= 0 ? (k.flags & 1) : 0) | (k.boff >= 0 ? (k.flags & 2) : 0);
      x.scale = (float)k.scale;
      x.task = t;
      base[t] = x;
    }
  });
  for (char x : bad)
    if (x) throw Error(1, "internal: a task names no stored block");

  // MMA multiply-adds of one slice product (rows padded to 128, N and K to 16)
  auto unit_macs = [&](int G, int tn, int m, int n) {
    double s1 = 0, s2 = 0;
    for (int c = 0; c < n; c += 128) s1 += 128.0 * up16(std::min(128, n - c)) * up16(m);
    for (int c = 0; c < n; c += 64) s2 += 128.0 * up16(tn) * up16(std::min(64, n - c));
    return s1 + G * s2;
  };
  const double unit_overhead = shape.unit_cost;  // fixed cost of a unit in the item split
  double total = 0;
  for (size_t b = 0; b < nblk; ++b) {
    const PsiBlock& ob = blocks[b];
    for (int r0 = 0; r0 < ob.mL; r0 += 128)
      for (int c0 = 0; c0 < ob.mR; c0 += 128) {
        const int tm = std::min(128, ob.mL - r0), tn = std::min(128, ob.mR - c0);
        const int G = std::max(1, 16 / ceil8(tm));
        for (int t = wl.out_start[b]; t < wl.out_start[b + 1]; ++t) {
          const TcPsiBlock& ib = plan.psi[base[t].in_blk];
          total += unit_macs(1, tn, ib.m, ib.n) / G + unit_overhead / G;
        }
      }
  }
  const double target = total / std::max(1, shape.want_items);

  struct Unit {  // one unit: positions [t0, t1) of its part's sorted task order
    int t0, t1;
  };
  struct Part {
    std::vector<TcItem> items;           // kind 0: r_begin/r_end index units; kind 1/2: small terms
    std::vector<Group> groups;
    std::vector<std::pair<int, Unit>> units;  // (output block, unit)
    std::vector<SmallTerm> small;
    std::vector<int> small_blk;          // per small term: split-block indices of its left and right blocks
    std::vector<double> icost;
    std::vector<int> order;              // sorted task indices, per block contiguous
    long long scratch = 0;
    long long n_terms = 0;
    double macs = 0;
  };
  constexpr int SMALL_ITEM = 512;        // small terms per CUDA-core item
  std::vector<Part> parts(nparts);
  in_parallel([&](int j) {
    Part& P = parts[j];
    for (size_t b = bstart[j]; b < bstart[j + 1]; ++b) {
      const PsiBlock& ob = blocks[b];
      const int t0 = wl.out_start[b], t1 = wl.out_start[b + 1];
      // classes: tasks of the block ordered by (input block, left transposed,
      // right transposed); equal keys are contiguous
      const int obase = (int)P.order.size();
      for (int t = t0; t < t1; ++t) P.order.push_back(t);
      std::stable_sort(P.order.begin() + obase, P.order.end(), [&](int x, int y) {
        if (base[x].in_blk != base[y].in_blk) return base[x].in_blk < base[y].in_blk;
        return (base[x].flags & 3) < (base[y].flags & 3);
      });
      for (int r0 = 0; r0 < ob.mL; r0 += 128)
        for (int c0 = 0; c0 < ob.mR; c0 += 128) {
          const int tm = std::min(128, ob.mL - r0), tn = std::min(128, ob.mR - c0);
          const int G = std::max(1, 16 / ceil8(tm));
          Group g{(int)b, r0, tm, c0, tn, (int)P.items.size(), 0, 0};
          if (t0 == t1) {  // no contribution: one empty item writes zeros
            P.items.push_back({(int)b, r0, tm, c0, tn, (int)P.units.size(), (int)P.units.size(), 0, P.scratch});
            P.scratch += (long long)tm * tn;
            P.icost.push_back(0);
            g.i_end = (int)P.items.size();
            P.groups.push_back(g);
            continue;
          }
          TcItem it{(int)b, r0, tm, c0, tn, (int)P.units.size(), 0, 0, P.scratch};
          double acc = 0;
          std::vector<SmallTerm> sm[2];  // CUDA-core terms: all blocks <= TC_SMALL_MID, the rest
          std::vector<int> smb[2];       // their split-block indices (left, right)
          int k = obase;
          const int kend = obase + (t1 - t0);
          while (k < kend) {
            // the class of order[k]: same input block and flags
            const Base& h = base[P.order[k]];
            int e = k;
            while (e < kend && base[P.order[e]].in_blk == h.in_blk && (base[P.order[e]].flags & 3) == (h.flags & 3)) ++e;
            const TcPsiBlock& ib = plan.psi[h.in_blk];
            // CUDA-core class: the whole output block (one tile) and the psi block are small
            const int wmax = std::max(std::max(ob.mL, ob.mR), std::max(ib.m, ib.n));
            if (wmax <= TC_SMALL_MAX) {
              const int cls = wmax <= TC_SMALL_MID ? 0 : 1;
              for (int q = k; q < e; ++q) {
                const Base& x = base[P.order[q]];
                const Task& tk = wl.tasks[x.task];
                sm[cls].push_back({tk.aoff < 0 ? -1 : x.a_tile, tk.boff < 0 ? -1 : x.b_tile, tk.in_blk, tk.flags & 3,
                                   tk.scale});
                smb[cls].push_back(x.a_blk);
                smb[cls].push_back(x.b_blk);
              }
              P.n_terms += e - k;
              k = e;
              continue;
            }
            for (int u0 = k; u0 < e; u0 += G) {
              const int u1 = std::min(e, u0 + G);
              const double c = unit_macs(u1 - u0, tn, ib.m, ib.n) + unit_overhead;
              if (acc > 0 && acc + c > target) {  // close the item
                it.r_end = (int)P.units.size();
                P.items.push_back(it);
                P.icost.push_back(acc);
                P.scratch += (long long)tm * tn;
                it = TcItem{(int)b, r0, tm, c0, tn, (int)P.units.size(), 0, 0, P.scratch};
                acc = 0;
              }
              P.units.push_back({(int)b, Unit{u0, u1}});  // positions in P.order
              acc += c;
              P.macs += unit_macs(u1 - u0, tn, ib.m, ib.n);
              P.n_terms += u1 - u0;
            }
            k = e;
          }
          if (acc > 0) {
            it.r_end = (int)P.units.size();
            P.items.push_back(it);
            P.icost.push_back(acc);
            P.scratch += (long long)tm * tn;
          }
          for (int cls = 0; cls < 2; ++cls) {  // CUDA-core items: kind 2 (<= TC_SMALL_MID), kind 1
            const size_t base0 = P.small.size();
            P.small.insert(P.small.end(), sm[cls].begin(), sm[cls].end());
            P.small_blk.insert(P.small_blk.end(), smb[cls].begin(), smb[cls].end());
            for (size_t s0 = base0; s0 < P.small.size(); s0 += SMALL_ITEM) {
              const size_t s1 = std::min(P.small.size(), s0 + SMALL_ITEM);
              double c = 0;
              for (size_t q = s0; q < s1; ++q) {
                const PsiBlock& ib = blocks[P.small[q].in_blk];
                c += 2.0 * ((double)tm * ib.mL * ib.mR + (double)tm * ib.mR * tn);
              }
              P.items.push_back({(int)b, r0, tm, c0, tn, (int)s0, (int)s1, cls == 0 ? 2 : 1, P.scratch});
              P.icost.push_back(c);
              P.scratch += (long long)tm * tn;
            }
          }
          g.i_end = (int)P.items.size();
          P.groups.push_back(g);
        }
    }
  });
  // join the parts: kind-0 items index records (one per unit, one TC_ZERO
  // record per item without units), kind-1/2 items index small terms
  std::vector<size_t> I(nparts + 1, 0), G(nparts + 1, 0), U(nparts + 1, 0), SM(nparts + 1, 0);
  std::vector<long long> S(nparts + 1, 0);
  for (int j = 0; j < nparts; ++j) {
    const Part& P = parts[j];
    I[j + 1] = I[j] + P.items.size();
    G[j + 1] = G[j] + P.groups.size();
    size_t nrec = 0;
    for (const TcItem& it : P.items)
      if (it.kind == 0) nrec += std::max(1, it.r_end - it.r_begin);
    U[j + 1] = U[j] + nrec;
    SM[j + 1] = SM[j] + P.small.size();
    S[j + 1] = S[j] + P.scratch;
    plan.n_terms += P.n_terms;
    plan.mma_macs += P.macs;
  }
  plan.items.resize(I[nparts]);
  plan.groups.resize(G[nparts]);
  plan.scratch_elems = S[nparts];
  plan.recs.resize(U[nparts]);  // uninitialized: every record is written below
  plan.term_blk.assign((size_t)U[nparts] * TC_MAX_G * 2, -1);
  plan.small.resize(SM[nparts]);
  plan.small_blk.resize(2 * SM[nparts]);
  plan.n_units = 0;
  std::vector<double> icost(I[nparts]);
  in_parallel([&](int j) {
    const Part& P = parts[j];
    std::copy(P.small.begin(), P.small.end(), plan.small.begin() + SM[j]);
    std::copy(P.small_blk.begin(), P.small_blk.end(), plan.small_blk.begin() + 2 * SM[j]);
    size_t rec = U[j];
    for (size_t i = 0; i < P.items.size(); ++i) {
      TcItem it = P.items[i];
      it.slot += S[j];
      icost[I[j] + i] = P.icost[i];
      if (it.kind != 0) {
        it.r_begin += (int)SM[j];
        it.r_end += (int)SM[j];
        plan.items[I[j] + i] = it;
        continue;
      }
      const int ub = it.r_begin, ue = it.r_end;
      it.r_begin = (int)rec;
      const int tm = it.nrows, tn = it.ncols, tm8 = ceil8(tm);
      auto header = [&](TcUnitRec& r) {
        r.tm = tm;
        r.tn = tn;
        r.tm8 = tm8;
        r.r0g = it.r0 / 8;
        r.c0g = it.c0 / 8;
        r.slot = it.slot;
        r.pad[0] = r.pad[1] = 0;
      };
      if (ub == ue) {
        TcUnitRec& r = plan.recs[rec++];
        std::memset(&r, 0, sizeof(r));
        header(r);
        r.flags = TC_ZERO | TC_ITEM_FIRST | TC_ITEM_LAST;
      } else {
        for (int u = ub; u < ue; ++u) {
          const Unit& un = P.units[u].second;
          TcUnitRec& r = plan.recs[rec++];
          std::memset(&r, 0, sizeof(r));
          header(r);
          const Base& h = base[P.order[un.t0]];
          const TcPsiBlock& ib = plan.psi[h.in_blk];
          r.flags = (h.flags & 1 ? TC_TA : 0) | (h.flags & 2 ? TC_TB : 0) | (u == ub ? TC_ITEM_FIRST : 0) |
                    (u == ue - 1 ? TC_ITEM_LAST : 0);
          r.nterm = un.t1 - un.t0;
          r.m = ib.m;
          r.n = ib.n;
          r.aR8 = (short)h.aR8;
          r.aC8 = (short)h.aC8;
          r.bR8 = (short)h.bR8;
          r.bC8 = (short)h.bC8;
          r.pR8 = (short)ib.R8;
          r.pC8 = (short)ib.C8;
          r.p_tile = ib.tile;
          r.pblk = h.in_blk;
          const size_t ri = (size_t)(&r - plan.recs.data());
          for (int q = 0; q < r.nterm; ++q) {
            const Base& x = base[P.order[un.t0 + q]];
            r.t[q].a_tile = x.a_tile;
            r.t[q].b_tile = x.b_tile;
            r.t[q].scale = x.scale;
            r.t[q].pad = 0;
            plan.term_blk[(ri * TC_MAX_G + q) * 2] = x.a_blk;
            plan.term_blk[(ri * TC_MAX_G + q) * 2 + 1] = x.b_blk;
          }
        }
      }
      it.r_end = (int)rec;
      plan.items[I[j] + i] = it;
    }
    for (size_t k = 0; k < P.groups.size(); ++k) {
      Group g = P.groups[k];
      g.i_begin += (int)I[j];
      g.i_end += (int)I[j];
      plan.groups[G[j] + k] = g;
    }
  });
  for (const Part& P : parts) plan.n_units += (long long)P.units.size();
  std::vector<int> small1;
  for (size_t i = 0; i < plan.items.size(); ++i) {
    const int kd = plan.items[i].kind;
    (kd == 0 ? plan.schedule : kd == 2 ? plan.small_schedule : small1).push_back((int)i);
  }
  auto by_cost = [&](int a, int b) { return icost[a] > icost[b]; };
  std::stable_sort(plan.schedule.begin(), plan.schedule.end(), by_cost);
  std::stable_sort(plan.small_schedule.begin(), plan.small_schedule.end(), by_cost);
  std::stable_sort(small1.begin(), small1.end(), by_cost);
  plan.n_small_mid = (int)plan.small_schedule.size();
  plan.small_schedule.insert(plan.small_schedule.end(), small1.begin(), small1.end());
}

}  // namespace dmrg
