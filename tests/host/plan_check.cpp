// Host-logic check of the sigma work lists (CPU only, no CUDA calls): reads
// two sector lists, builds the operator tables, the NC or CN term list, the
// psi layout, the FP64 task list and the tensor-core plan with the
// library's own host code, checks the plan's structural invariants, and
// prints a JSON summary (task count, algorithmic flops, violations) that
// the Python test compares with the oracle's independent count.
//
//   plan_check <sectors file> <nL modes> <n modes> <N> <2Sz> <nc|cn>
//   sectors file: "nl nr" then nl + nr lines "N 2Sz dim"
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <string>
#include <tuple>
#include <vector>

#include "model.h"

using namespace dmrg;

static std::vector<std::string> errors;
static void fail(const std::string& m) {
  if (errors.size() < 20) errors.push_back(m);
}

int main(int argc, char** argv) {
  if (argc < 7) return 2;
  std::ifstream f(argv[1]);
  const int nL = std::atoi(argv[2]), n = std::atoi(argv[3]);
  const QN Q{std::atoi(argv[4]), std::atoi(argv[5])};
  const bool cn = std::string(argv[6]) == "cn";
  int nl = 0, nr = 0;
  f >> nl >> nr;
  Basis L, R;
  for (int i = 0; i < nl + nr; ++i) {
    int a, b, d;
    f >> a >> b >> d;
    Basis& B = i < nl ? L : R;
    B.q.push_back({a, b});
    B.dim.push_back(d);
  }
  L.finish();
  R.finish();
  OpSet oL, oR;
  build_nc_opset(oL, L, nL, n, true, 0, cn);
  build_nc_opset(oR, R, nL, n, false, oL.elements, cn);
  const std::vector<Term> terms = cn ? cn_terms(nL, n) : nc_terms(nL, n);
  long long size = 0;
  const std::vector<PsiBlock> blocks = psi_layout(L, R, Q, &size);
  WorkList wl;
  build_tasks(blocks, oL, oR, terms, wl);
  build_items(blocks, wl, TileShape{32, 256, 2e6, 16384.0}, 152 * 8);
  TcPlan plan;
  build_tc_plan(blocks, oL, oR, wl, plan, 152 * 4, 32);

  // (0) FP64 work list: groups tile every output block into 32 x 256 tiles;
  //     the items of a group split the block's task range in order; slots
  //     are consecutive; the schedule is a permutation
  {
    size_t g = 0;
    long long sl = 0;
    int ni = 0;
    for (size_t b = 0; b < blocks.size(); ++b)
      for (int r0 = 0; r0 < blocks[b].mL; r0 += 32)
        for (int c0 = 0; c0 < blocks[b].mR; c0 += 256, ++g) {
          if (g >= wl.groups.size()) {
            fail("fp64: missing group");
            continue;
          }
          const Group& gr = wl.groups[g];
          if (gr.out != (int)b || gr.r0 != r0 || gr.c0 != c0 || gr.nrows != std::min(32, blocks[b].mL - r0) ||
              gr.ncols != std::min(256, blocks[b].mR - c0) || gr.i_begin != ni || gr.i_end <= gr.i_begin)
            fail("fp64: group");
          int t = wl.out_start[b];
          for (int i = gr.i_begin; i < gr.i_end && i < (int)wl.items.size(); ++i) {
            const Item& it = wl.items[i];
            if (it.out != gr.out || it.r0 != gr.r0 || it.c0 != gr.c0 || it.nrows != gr.nrows || it.ncols != gr.ncols)
              fail("fp64: item tile");
            if (it.t_begin != t || it.t_end < it.t_begin) fail("fp64: item task range");
            if (it.slot != sl) fail("fp64: slot");
            sl += (long long)it.nrows * it.ncols;
            t = it.t_end;
          }
          if (t != wl.out_start[b + 1]) fail("fp64: items do not cover the block's tasks");
          ni = gr.i_end;
        }
    if (g != wl.groups.size() || ni != (int)wl.items.size()) fail("fp64: extra groups or items");
    if (sl != wl.scratch_elems) fail("fp64: scratch size");
    std::vector<int> sch = wl.schedule;
    std::sort(sch.begin(), sch.end());
    for (size_t i = 0; i < sch.size(); ++i)
      if (sch[i] != (int)i) {
        fail("fp64: schedule");
        break;
      }
  }

  // (1) every task of the list, with its operator tiles, appears in the plan
  //     once per 128 x 128 tile of its output block
  std::vector<long long> offs;
  for (const OpSet* s : {&oL, &oR})
    for (const OpDesc& o : s->ops)
      for (const OpBlock& b : o.blocks) offs.push_back(b.off);
  using Key = std::tuple<int, int, long long, long long, unsigned>;
  std::vector<Key> want, got;
  std::vector<int> out_of(wl.tasks.size(), -1);
  for (size_t b = 0; b < blocks.size(); ++b)
    for (int t = wl.out_start[b]; t < wl.out_start[b + 1]; ++t) out_of[t] = (int)b;
  for (size_t t = 0; t < wl.tasks.size(); ++t) {
    const Task& k = wl.tasks[t];
    const PsiBlock& in = blocks[k.in_blk];
    long long at = plan.identL[in.qL].tile, bt = plan.identR[in.qR].tile;
    if (k.aoff >= 0) {
      const int i = wl.task_ablk[t];
      if (i < 0 || offs[i] != k.aoff) fail("task left block index");
      else at = plan.opblocks[i].tile;
    }
    if (k.boff >= 0) {
      const int i = wl.task_bblk[t];
      if (i < 0 || offs[i] != k.boff) fail("task right block index");
      else bt = plan.opblocks[i].tile;
    }
    const float sc = (float)k.scale;
    unsigned bits;
    std::memcpy(&bits, &sc, 4);
    const int fl = (k.aoff >= 0 ? (k.flags & 1) : 0) | (k.boff >= 0 ? (k.flags & 2) : 0);
    const PsiBlock& ob = blocks[out_of[t]];
    const int ntile = ((ob.mL + 127) / 128) * ((ob.mR + 127) / 128);
    for (int r = 0; r < ntile; ++r) want.emplace_back(k.in_blk, fl, at, bt, bits);
  }
  for (const TcTask& x : plan.tasks) {
    unsigned bits;
    std::memcpy(&bits, &x.scale, 4);
    got.emplace_back(x.in_blk, x.flags & 3, x.a_tile, x.b_tile, bits);
  }
  std::sort(want.begin(), want.end());
  std::sort(got.begin(), got.end());
  if (want != got) fail("plan tasks differ from the task list");

  // (2) units of each item point back to it; task ranges tile the task list in order
  int next_task = 0;
  for (size_t i = 0; i < plan.items.size(); ++i) {
    const TcItem& it = plan.items[i];
    for (int u = it.u_begin; u < it.u_end; ++u) {
      const TcUnit& un = plan.units[u];
      if (un.item != (int)i) fail("unit item");
      if (un.t_begin >= un.t_end) fail("empty unit");
      if (un.flags & UNIT_PACKED) {
        if (un.t_begin != next_task) fail("packed unit out of order");
        if (un.width > 64) fail("packed width");
        next_task = un.t_end;
      } else {
        if (un.t_end != un.t_begin + 1) fail("pass unit of more than one task");
        if (un.pass == 0) {
          if (un.t_begin != next_task) fail("pass unit out of order");
          next_task = un.t_end;
        }
      }
      const TcTask& t = plan.tasks[un.t_begin];
      if (plan.items[i].out < 0 || t.in_blk < 0 || t.in_blk >= (int)blocks.size()) fail("task input block");
    }
    if (i + 1 < plan.items.size() && plan.items[i + 1].u_begin != it.u_end) fail("item unit ranges");
  }
  if (next_task != (int)plan.tasks.size()) fail("units do not cover the tasks");

  // (3) groups tile every output block into 128 x 128 tiles; items of a group share its tile
  size_t gi = 0;
  long long slot = 0;
  int expect_item = 0;
  for (size_t b = 0; b < blocks.size(); ++b)
    for (int r0 = 0; r0 < blocks[b].mL; r0 += 128)
      for (int c0 = 0; c0 < blocks[b].mR; c0 += 128, ++gi) {
        if (gi >= plan.groups.size()) {
          fail("missing group");
          continue;
        }
        const Group& g = plan.groups[gi];
        if (g.out != (int)b || g.r0 != r0 || g.c0 != c0 || g.nrows != std::min(128, blocks[b].mL - r0) ||
            g.ncols != std::min(128, blocks[b].mR - c0))
          fail("group tile");
        if (g.i_begin != expect_item || g.i_end <= g.i_begin) fail("group item range");
        for (int i = g.i_begin; i < g.i_end && i < (int)plan.items.size(); ++i) {
          const TcItem& it = plan.items[i];
          if (it.out != g.out || it.r0 != g.r0 || it.c0 != g.c0 || it.nrows != g.nrows || it.ncols != g.ncols)
            fail("item tile");
          if (it.slot != slot) fail("scratch slot");
          slot += (long long)it.nrows * it.ncols;
        }
        expect_item = g.i_end;
      }
  if (gi != plan.groups.size()) fail("extra groups");
  if (slot != plan.scratch_elems) fail("scratch size");

  // (4) the schedule is a permutation of the items
  std::vector<int> sch = plan.schedule;
  std::sort(sch.begin(), sch.end());
  for (size_t i = 0; i < sch.size(); ++i)
    if (sch[i] != (int)i) {
      fail("schedule");
      break;
    }
  if (sch.size() != plan.items.size()) fail("schedule size");

  // (5) records: one per unit (one REC_ZERO per item without units), copies of the tasks
  for (size_t i = 0; i < plan.items.size(); ++i) {
    const TcItem& it = plan.items[i];
    const int nrec = plan.item_rec[i + 1] - plan.item_rec[i];
    if (nrec != std::max(1, it.u_end - it.u_begin)) fail("record count");
    if (it.u_begin == it.u_end) {
      if (!(plan.recs[plan.item_rec[i]].flags & REC_ZERO)) fail("empty item record");
      continue;
    }
    for (int u = it.u_begin; u < it.u_end; ++u) {
      const TcRec& r = plan.recs[plan.item_rec[i] + (u - it.u_begin)];
      const TcUnit& un = plan.units[u];
      if (r.ntask != un.t_end - un.t_begin || r.ntask > 4 || r.pass != un.pass || r.slot != it.slot) fail("record");
      for (int k = 0; k < r.ntask && k < 4; ++k) {
        const TcTask& t = plan.tasks[un.t_begin + k];
        if (r.t[k].a_tile != t.a_tile || r.t[k].b_tile != t.b_tile || r.t[k].p_tile != plan.psi[t.in_blk].tile ||
            r.t[k].scale != t.scale || r.t[k].flags != t.flags)
          fail("record task");
      }
    }
  }

  std::printf("{\"psi_size\": %lld, \"blocks\": %zu, \"terms\": %zu, \"tasks\": %zu, \"flops\": %.17g, "
              "\"plan_tasks\": %zu, \"units\": %zu, \"items\": %zu, \"layout\": [",
              size, blocks.size(), terms.size(), wl.tasks.size(), wl.flops, plan.tasks.size(), plan.units.size(),
              plan.items.size());
  for (size_t b = 0; b < blocks.size(); ++b) {
    const PsiBlock& pb = blocks[b];
    std::printf("%s[%d, %d, %d, %d, %d, %d, %lld]", b ? ", " : "", L.q[pb.qL].n, L.q[pb.qL].s, R.q[pb.qR].n,
                R.q[pb.qR].s, pb.mL, pb.mR, pb.off);
  }
  std::printf("], \"ranks3\": [");
  const std::vector<int> rk = cn ? cn_term_ranks(nL, n, 3) : nc_term_ranks(nL, n, 3);
  if (rk.size() != terms.size()) fail("rank count");
  for (size_t t = 0; t < rk.size(); ++t) std::printf("%s%d", t ? ", " : "", rk[t]);
  std::printf("], \"errors\": [");
  for (size_t i = 0; i < errors.size(); ++i) std::printf("%s\"%s\"", i ? ", " : "", errors[i].c_str());
  std::printf("]}\n");
  return 0;
}
