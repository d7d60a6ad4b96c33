// Host-side model: bases, NC operator tables, terms, sigma work lists.
#include "model.h"

#include <algorithm>
#include <cmath>
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

int tc_k1_tiles(const TcTask& t, const TcPsiBlock& ib, int r0) {
  if (ib.R8 > 4 || ib.C8 > 8) return 0;               // m <= 32, n <= 64
  const bool tA = t.flags & 1;
  const int rg0 = r0 / 8;
  int ol = tA ? t.aR8 * std::min(16, t.aC8 - rg0)      // K groups x M groups
              : std::min(16, t.aR8 - rg0) * t.aC8;     // M groups x K groups
  return ol + ib.R8 * ib.C8;
}

int tc_k2_tiles(const TcTask& t, int c0) {  // tiles of the right operand for one task
  const bool tB = t.flags & 2;
  const int cg0 = c0 / 8;
  return tB ? t.bR8 * std::min(16, t.bC8 - cg0) : std::min(16, t.bR8 - cg0) * t.bC8;
}

void build_tc_plan(const std::vector<PsiBlock>& blocks, const OpSet& L, const OpSet& R,
                   const WorkList& wl, TcPlan& plan, int want_items, int seg_tasks) {
  plan = TcPlan();
  // element offset -> tiled block: offsets grow in store order, so a sorted
  // array and binary search map them
  std::vector<long long> offs;
  long long tile = 0;
  for (const OpSet* s : {&L, &R})
    for (const OpDesc& o : s->ops) {
      plan.op_first.push_back((long long)plan.opblocks.size());
      for (const OpBlock& b : o.blocks) {
        TcBlock t{tile, ceil8(b.rows), ceil8(b.cols)};
        tile += (long long)t.R8 * t.C8;
        plan.opblocks.push_back(t);
        offs.push_back(b.off);
      }
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
  plan.n_tiles = tile + 64;  // slack: descriptor reads past the last tile stay in bounds
  long long pt = 0;
  for (const PsiBlock& b : blocks) {
    TcPsiBlock p{pt, 2 * ((b.mL + 15) / 16), ceil8(b.mR), b.mL, b.mR};
    pt += (long long)p.R8 * p.C8;
    plan.psi.push_back(p);
  }
  plan.psi_tiles = pt + 64;
  // base task records (identity factors made explicit); build_tasks names
  // each task's stored blocks by index, else they are looked up by offset
  const bool have_idx = wl.task_ablk.size() == wl.tasks.size() && wl.task_bblk.size() == wl.tasks.size();
  // Output blocks are independent: contiguous block ranges of about equal
  // task counts are handled by up to 8 threads (base records, per-block task
  // order, items and units into parts with local indices); the parts are
  // joined in block order with their task / unit / item / scratch offsets,
  // so the plan is the same as one pass over the blocks.
  const size_t nblk = blocks.size();
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
  std::vector<TcTask> base(wl.tasks.size());
  std::vector<char> bad(nparts, 0);
  in_parallel([&](int j) {
    for (int t = wl.out_start[bstart[j]]; t < wl.out_start[bstart[j + 1]]; ++t) {
      const Task& k = wl.tasks[t];
      const PsiBlock& in = blocks[k.in_blk];
      TcBlock a = plan.identL[in.qL], b = plan.identR[in.qR];
      if (k.aoff >= 0) {
        const int i = have_idx ? wl.task_ablk[t] : -1;
        const int f = have_idx ? i : find_off(k.aoff);
        if (f < 0 || f >= (int)offs.size() || offs[f] != k.aoff) bad[j] = 1;
        else a = plan.opblocks[f];
      }
      if (k.boff >= 0) {
        const int i = have_idx ? wl.task_bblk[t] : -1;
        const int f = have_idx ? i : find_off(k.boff);
        if (f < 0 || f >= (int)offs.size() || offs[f] != k.boff) bad[j] = 1;
        else b = plan.opblocks[f];
      }
      TcTask x{};
      x.a_tile = a.tile;
      x.aR8 = a.R8;
      x.aC8 = a.C8;
      x.b_tile = b.tile;
      x.bR8 = b.R8;
      x.bC8 = b.C8;
      x.in_blk = k.in_blk;
      x.flags = (k.aoff >= 0 ? (k.flags & 1) : 0) | (k.boff >= 0 ? (k.flags & 2) : 0);
      x.scale = (float)k.scale;
      base[t] = x;
    }
    // order tasks of each output block by (right transposed, input block, left
    // transposed): packed units then share the layout of their second product
    // and consecutive tasks share psi tiles
    std::vector<int> idx;
    std::vector<TcTask> tmp;
    for (size_t ob = bstart[j]; ob < bstart[j + 1]; ++ob) {
      const int t0 = wl.out_start[ob], t1 = wl.out_start[ob + 1];
      idx.resize(t1 - t0);
      std::iota(idx.begin(), idx.end(), t0);
      std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
        const int kx = ((base[x].flags >> 1) & 1), ky = ((base[y].flags >> 1) & 1);
        if (kx != ky) return kx < ky;
        if (base[x].in_blk != base[y].in_blk) return base[x].in_blk < base[y].in_blk;
        return (base[x].flags & 1) < (base[y].flags & 1);
      });
      tmp.clear();
      for (int i : idx) tmp.push_back(base[i]);
      std::copy(tmp.begin(), tmp.end(), base.begin() + t0);
    }
  });
  for (char x : bad)
    if (x) throw Error(1, "internal: a task names no stored block");
  // MMA work of a task on one 128 x 128 tile (rows padded to 128)
  auto cost = [&](const TcTask& k) {
    const TcPsiBlock& in = plan.psi[k.in_blk];
    double n16 = 16.0 * ((in.n + 15) / 16), m16 = 8.0 * in.R8;
    return 128.0 * n16 * m16 + 128.0 * n16 * 128.0 + 4096.0;  // + fixed per-task overhead
  };
  double total = 0;
  for (size_t b = 0; b < blocks.size(); ++b) {
    int ntile = ((blocks[b].mL + 127) / 128) * ((blocks[b].mR + 127) / 128);
    for (int t = wl.out_start[b]; t < wl.out_start[b + 1]; ++t) total += ntile * cost(base[t]);
  }
  const double target = total / std::max(1, want_items);
  struct Part {
    std::vector<TcTask> tasks;
    std::vector<TcUnit> units;
    std::vector<TcItem> items;
    std::vector<Group> groups;
    std::vector<double> icost;
    long long scratch = 0;
  };
  auto plan_block = [&](size_t b, Part& P) {
    const PsiBlock& ob = blocks[b];
    const int t0 = wl.out_start[b], t1 = wl.out_start[b + 1];
    for (int r0 = 0; r0 < ob.mL; r0 += 128)
      for (int c0 = 0; c0 < ob.mR; c0 += 128) {
        const int nr = std::min(128, ob.mL - r0), nc = std::min(128, ob.mR - c0);
        Group g{(int)b, r0, nr, c0, nc, (int)P.items.size(), 0, 0};
        int t = t0;
        do {  // one item per iteration (at least one, even with no tasks)
          TcItem it{(int)b, r0, nr, c0, nc, (int)P.units.size(), 0, 0, P.scratch};
          const int item_idx = (int)P.items.size();
          double acc = 0;
          int seg = 0, seg_first_unit = (int)P.units.size();
          bool first_seg = true;
          auto end_segment = [&]() {
            if (P.units.size() > (size_t)seg_first_unit) {
              P.units.back().flags |= UNIT_ENDS_SEGMENT | (first_seg ? UNIT_FIRST_SEGMENT : 0);
              first_seg = false;
            }
            seg = 0;
            seg_first_unit = (int)P.units.size();
          };
          while (t < t1 && (acc == 0 || acc + cost(base[t]) <= target)) {
            TcTask k = base[t];
            const TcPsiBlock& ib = plan.psi[k.in_blk];
            int k1 = tc_k1_tiles(k, ib, r0), k2 = tc_k2_tiles(k, c0);
            if (k1 > 0 && k1 <= 128 && k2 <= 128) {
              // packed unit: greedily add following small tasks with the same
              // right-operand orientation; tasks on the same psi block share its tiles
              TcUnit u{item_idx, (int)P.tasks.size(), 0, 0, UNIT_PACKED, 0, {0, 0}};
              int w = 0, s1 = 0, last_in = -1, last_k1b = 0;
              const int tB0 = (k.flags >> 1) & 1;
              while (t < t1 && seg < seg_tasks && (acc == 0 || acc + cost(base[t]) <= target)) {
                TcTask x = base[t];
                const TcPsiBlock& xb = plan.psi[x.in_blk];
                int a1 = tc_k1_tiles(x, xb, r0);
                const bool share = x.in_blk == last_in;
                if (share) a1 -= xb.R8 * xb.C8;
                int n16 = 16 * ((xb.n + 15) / 16);
                if (tc_k1_tiles(x, xb, r0) == 0 || ((x.flags >> 1) & 1) != tB0 || w + n16 > 64 || s1 + a1 > 128) break;
                x.xcol = w;
                x.k1a = s1;
                const bool tA = x.flags & 1;
                const int rg0 = r0 / 8;
                const int ol = tA ? x.aR8 * std::min(16, x.aC8 - rg0) : std::min(16, x.aR8 - rg0) * x.aC8;
                if (share) {
                  x.k1b = last_k1b;
                  x.flags |= 4;  // psi tiles already in the stage
                } else {
                  x.k1b = s1 + ol;
                  last_k1b = x.k1b;
                }
                x.k2 = 0;
                last_in = x.in_blk;
                w += n16;
                s1 += a1;
                P.tasks.push_back(x);
                acc += cost(x);
                ++t;
                ++seg;
              }
              u.t_end = (int)P.tasks.size();
              u.width = w;
              P.units.push_back(u);
            } else {
              P.tasks.push_back(k);
              const int npass = (ib.n + 127) / 128;
              for (int p = 0; p < npass; ++p)
                P.units.push_back({item_idx, (int)P.tasks.size() - 1, (int)P.tasks.size(), p, 0,
                                   std::min(128, ib.n - 128 * p), {0, 0}});
              acc += cost(k);
              ++t;
              ++seg;
            }
            if (seg >= seg_tasks) end_segment();
          }
          end_segment();
          it.u_end = (int)P.units.size();
          P.items.push_back(it);
          P.scratch += (long long)nr * nc;
          P.icost.push_back(acc);
        } while (t < t1);
        g.i_end = (int)P.items.size();
        P.groups.push_back(g);
      }
  };
  std::vector<Part> parts(nparts);
  in_parallel([&](int j) {
    parts[j].tasks.reserve(wl.out_start[bstart[j + 1]] - wl.out_start[bstart[j]]);
    for (size_t b = bstart[j]; b < bstart[j + 1]; ++b) plan_block(b, parts[j]);
  });
  std::vector<double> icost;
  {
    std::vector<size_t> T(nparts + 1, 0), U(nparts + 1, 0), I(nparts + 1, 0), G(nparts + 1, 0);
    std::vector<long long> S(nparts + 1, 0);
    for (int j = 0; j < nparts; ++j) {
      T[j + 1] = T[j] + parts[j].tasks.size();
      U[j + 1] = U[j] + parts[j].units.size();
      I[j + 1] = I[j] + parts[j].items.size();
      G[j + 1] = G[j] + parts[j].groups.size();
      S[j + 1] = S[j] + parts[j].scratch;
    }
    plan.tasks.resize(T[nparts]);
    plan.units.resize(U[nparts]);
    plan.items.resize(I[nparts]);
    plan.groups.resize(G[nparts]);
    icost.resize(I[nparts]);
    plan.scratch_elems = S[nparts];
    in_parallel([&](int j) {
      const Part& P = parts[j];
      std::copy(P.tasks.begin(), P.tasks.end(), plan.tasks.begin() + T[j]);
      for (size_t k = 0; k < P.units.size(); ++k) {
        TcUnit u = P.units[k];
        u.item += (int)I[j];
        u.t_begin += (int)T[j];
        u.t_end += (int)T[j];
        plan.units[U[j] + k] = u;
      }
      for (size_t k = 0; k < P.items.size(); ++k) {
        TcItem it = P.items[k];
        it.u_begin += (int)U[j];
        it.u_end += (int)U[j];
        it.slot += S[j];
        plan.items[I[j] + k] = it;
      }
      for (size_t k = 0; k < P.groups.size(); ++k) {
        Group g = P.groups[k];
        g.i_begin += (int)I[j];
        g.i_end += (int)I[j];
        plan.groups[G[j] + k] = g;
      }
      std::copy(P.icost.begin(), P.icost.end(), icost.begin() + I[j]);
    });
  }
  plan.schedule.resize(plan.items.size());
  std::iota(plan.schedule.begin(), plan.schedule.end(), 0);
  std::stable_sort(plan.schedule.begin(), plan.schedule.end(),
                   [&](int a, int b) { return icost[a] > icost[b]; });
  // records: one per unit (one REC_ZERO per item without units), written in
  // item order; items are independent, so ranges of them fill in parallel
  static_assert(sizeof(TcTaskRec) == 64 && sizeof(TcRec) == 304, "record layout");
  plan.item_rec.assign(plan.items.size() + 1, 0);
  for (size_t i = 0; i < plan.items.size(); ++i)
    plan.item_rec[i + 1] = plan.item_rec[i] + std::max(1, plan.items[i].u_end - plan.items[i].u_begin);
  plan.recs.clear();
  plan.recs.resize((size_t)plan.item_rec.back());  // uninitialized: every record is written below
  auto fill = [&](size_t i0, size_t i1) {
    for (size_t i = i0; i < i1; ++i) {
      const TcItem& it = plan.items[i];
      TcRec* out = plan.recs.data() + plan.item_rec[i];
      auto header = [&](TcRec& r) {
        r.r0 = it.r0;
        r.nrows = it.nrows;
        r.c0 = it.c0;
        r.ncols = it.ncols;
        r.slot = it.slot;
      };
      if (it.u_begin == it.u_end) {
        *out = TcRec{};
        out->flags = REC_ZERO;
        header(*out);
        continue;
      }
      for (int u = it.u_begin; u < it.u_end; ++u, ++out) {
        const TcUnit& un = plan.units[u];
        TcRec& r = *out;
        r = TcRec{};
        r.flags = un.flags;
        r.ntask = un.t_end - un.t_begin;
        r.pass = un.pass;
        r.width = un.width;
        r.pad[0] = un.width / 8;  // K groups of the packed second product
        header(r);
        for (int k = 0; k < r.ntask; ++k) {
          const TcTask& t = plan.tasks[un.t_begin + k];
          const TcPsiBlock& p = plan.psi[t.in_blk];
          TcTaskRec& x = r.t[k];
          x.a_tile = t.a_tile;
          x.b_tile = t.b_tile;
          x.p_tile = p.tile;
          x.aR8 = (short)t.aR8;
          x.aC8 = (short)t.aC8;
          x.bR8 = (short)t.bR8;
          x.bC8 = (short)t.bC8;
          x.pR8 = (short)p.R8;
          x.pC8 = (short)p.C8;
          x.xcol = (short)t.xcol;
          x.k1a = (short)t.k1a;
          x.k1b = (short)t.k1b;
          x.k2 = (short)t.k2;
          x.pn = p.n;
          x.flags = t.flags;
          x.scale = t.scale;
        }
      }
    }
  };
  const size_t nit = plan.items.size();
  const int nth = (int)std::min<size_t>(8, std::max<size_t>(1, std::min<size_t>(std::thread::hardware_concurrency(),
                                                                                  plan.recs.size() / 65536)));
  if (nth <= 1) {
    fill(0, nit);
  } else {  // item ranges of about equal record counts
    std::vector<std::thread> pool;
    size_t i0 = 0;
    for (int th = 0; th < nth; ++th) {
      const long long goal = (long long)plan.recs.size() * (th + 1) / nth;
      size_t i1 = th == nth - 1 ? nit : (size_t)(std::lower_bound(plan.item_rec.begin(), plan.item_rec.end() - 1,
                                                                  (int)goal) - plan.item_rec.begin());
      i1 = std::max(i1, i0);
      pool.emplace_back(fill, i0, i1);
      i0 = i1;
    }
    for (auto& t : pool) t.join();
  }
}

}  // namespace dmrg
