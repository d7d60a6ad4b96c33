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
#include <map>
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
  build_tc_plan(blocks, oL, oR, wl, plan, TcShape{152 * 4});

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

  // (1) every task of the list appears once per 128 x 128 tile of its output
  //     block: in a tensor-core unit record (by its operator tiles) or in a
  //     small-class term (by its operator tiles), never in both
  std::vector<long long> offs;
  for (const OpSet* s : {&oL, &oR})
    for (const OpDesc& o : s->ops)
      for (const OpBlock& b : o.blocks) offs.push_back(b.off);
  std::map<long long, long long> off_of_tile;  // operator tile -> store offset (identity tiles absent)
  for (size_t i = 0; i < plan.opblocks.size(); ++i) off_of_tile[plan.opblocks[i].tile] = offs[i];
  std::map<long long, int> blk_of_ptile;
  for (size_t i = 0; i < plan.psi.size(); ++i) blk_of_ptile[plan.psi[i].tile] = (int)i;
  using Key = std::tuple<int, unsigned, long long, long long, unsigned>;
  std::vector<Key> want, got;
  std::vector<int> out_of(wl.tasks.size(), -1);
  for (size_t b = 0; b < blocks.size(); ++b)
    for (int t = wl.out_start[b]; t < wl.out_start[b + 1]; ++t) out_of[t] = (int)b;
  for (size_t t = 0; t < wl.tasks.size(); ++t) {
    const Task& k = wl.tasks[t];
    if (k.aoff >= 0 && (wl.task_ablk[t] < 0 || offs[wl.task_ablk[t]] != k.aoff)) fail("task left block index");
    if (k.boff >= 0 && (wl.task_bblk[t] < 0 || offs[wl.task_bblk[t]] != k.boff)) fail("task right block index");
    const float sc = (float)k.scale;
    unsigned bits;
    std::memcpy(&bits, &sc, 4);
    const unsigned fl = (k.aoff >= 0 ? (k.flags & 1) : 0) | (k.boff >= 0 ? (k.flags & 2) : 0);
    const PsiBlock& ob = blocks[out_of[t]];
    const int ntile = ((ob.mL + 127) / 128) * ((ob.mR + 127) / 128);
    for (int r = 0; r < ntile; ++r) want.emplace_back(k.in_blk, fl, k.aoff, k.boff, bits);
  }
  long long nterms = 0;
  for (const TcUnitRec& r : plan.recs) {
    if (r.flags & TC_ZERO) continue;
    const unsigned fl = ((r.flags & TC_TA) ? 1u : 0u) | ((r.flags & TC_TB) ? 2u : 0u);
    const auto pb = blk_of_ptile.find(r.p_tile);
    if (pb == blk_of_ptile.end()) fail("record psi tile");
    for (int q = 0; q < r.nterm && q < TC_MAX_G; ++q) {
      unsigned bits;
      std::memcpy(&bits, &r.t[q].scale, 4);
      const auto ia = off_of_tile.find(r.t[q].a_tile), ib = off_of_tile.find(r.t[q].b_tile);
      const long long ao = ia == off_of_tile.end() ? -1 : ia->second, bo = ib == off_of_tile.end() ? -1 : ib->second;
      got.emplace_back(pb == blk_of_ptile.end() ? -1 : pb->second, fl, ao, bo, bits);
    }
    nterms += r.nterm;
  }
  for (const SmallTerm& x : plan.small) {
    const float sc = (float)x.scale;
    unsigned bits;
    std::memcpy(&bits, &sc, 4);
    const unsigned fl = (x.a_tile >= 0 ? (x.flags & 1) : 0) | (x.b_tile >= 0 ? (x.flags & 2) : 0);
    const auto ia = off_of_tile.find(x.a_tile), ib = off_of_tile.find(x.b_tile);
    if ((x.a_tile >= 0 && ia == off_of_tile.end()) || (x.b_tile >= 0 && ib == off_of_tile.end()))
      fail("small term tile");
    const long long ao = ia == off_of_tile.end() ? -1 : ia->second, bo = ib == off_of_tile.end() ? -1 : ib->second;
    got.emplace_back(x.in_blk, fl, ao, bo, bits);
    ++nterms;
  }
  std::sort(want.begin(), want.end());
  std::sort(got.begin(), got.end());
  if (want != got) fail("plan terms differ from the task list");
  if (nterms != plan.n_terms) fail("term count");

  // (2) records of every tensor-core item: first / last flags, the item's
  //     tile, unit geometry consistent with the blocks it reads; terms of
  //     every small item: contiguous ranges, small blocks only
  long long nunit = 0;
  int next_rec = 0, next_small = 0;
  for (size_t i = 0; i < plan.items.size(); ++i) {
    const TcItem& it = plan.items[i];
    if (it.r_end <= it.r_begin) fail("item without records or terms");
    if (it.kind == 1 || it.kind == 2) {
      // kind 2: every block at most TC_SMALL_MID wide; kind 1: at most
      // TC_SMALL_MAX, and some block of every term wider than TC_SMALL_MID
      const int lim = it.kind == 2 ? TC_SMALL_MID : TC_SMALL_MAX;
      if (it.r_begin != next_small) fail("small term ranges");
      next_small = it.r_end;
      if (it.nrows > lim || it.ncols > lim || it.r0 != 0 || it.c0 != 0) fail("small item tile");
      for (int k = it.r_begin; k < it.r_end && k < (int)plan.small.size(); ++k) {
        const PsiBlock& ib = blocks[plan.small[k].in_blk];
        if (ib.mL > lim || ib.mR > lim) fail("small term with a large psi block");
        if (it.kind == 1 && std::max(std::max(it.nrows, it.ncols), std::max(ib.mL, ib.mR)) <= TC_SMALL_MID)
          fail("size class of a small term");
      }
      continue;
    }
    if (it.kind != 0) fail("item kind");
    if (it.r_begin != next_rec) fail("item record ranges");
    next_rec = it.r_end;
    for (int k = it.r_begin; k < it.r_end && k < (int)plan.recs.size(); ++k) {
      const TcUnitRec& r = plan.recs[k];
      const bool first = k == it.r_begin, last = k == it.r_end - 1;
      if (((r.flags & TC_ITEM_FIRST) != 0) != first || ((r.flags & TC_ITEM_LAST) != 0) != last) fail("item flags");
      if (r.tm != it.nrows || r.tn != it.ncols || r.r0g * 8 != it.r0 || r.c0g * 8 != it.c0 || r.slot != it.slot)
        fail("record tile");
      if (r.tm8 != (r.tm + 7) / 8) fail("record tm8");
      if (r.flags & TC_ZERO) {
        if (it.r_end - it.r_begin != 1) fail("zero record in a non-empty item");
        continue;
      }
      ++nunit;
      if (r.nterm < 1 || (r.nterm * r.tm8 > 16 && r.nterm > 1)) fail("stacked rows exceed 128");
      if (std::max(std::max(blocks[it.out].mL, blocks[it.out].mR), std::max(r.m, r.n)) <= TC_SMALL_MAX)
        fail("small class in a unit");
      const TcPsiBlock* pb = nullptr;
      for (const TcPsiBlock& x : plan.psi)
        if (x.tile == r.p_tile) pb = &x;
      if (!pb || pb->m != r.m || pb->n != r.n || pb->R8 != r.pR8 || pb->C8 != r.pC8) fail("record psi block");
      // the left block covers the tile rows (M) and psi rows (K); the right
      // block covers the tile columns (N) and psi columns (K)
      const bool tA = r.flags & TC_TA, tB = r.flags & TC_TB;
      const int aM8 = tA ? r.aC8 : r.aR8, aK8 = tA ? r.aR8 : r.aC8;
      const int bN8 = tB ? r.bC8 : r.bR8, bK8 = tB ? r.bR8 : r.bC8;
      if (aK8 != (r.m + 7) / 8 || bK8 != (r.n + 7) / 8) fail("operand K extent");
      if (r.r0g + r.tm8 > aM8 || r.c0g + (r.tn + 7) / 8 > bN8) fail("operand M / N extent");
    }
  }
  if (next_rec != (int)plan.recs.size() || next_small != (int)plan.small.size()) fail("records or small terms unused");
  if (nunit != plan.n_units) fail("unit count");

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

  // (3b) split-block indices (the FP16X2 coefficients read the block
  //      exponents through them): every record term and small term names the
  //      split job whose tiles it reads (stored blocks, then the identities of
  //      the left and of the right sectors)
  {
    std::vector<long long> job_tile;
    for (const TcBlock& b : plan.opblocks) job_tile.push_back(b.tile);
    for (const TcBlock& b : plan.identL) job_tile.push_back(b.tile);
    for (const TcBlock& b : plan.identR) job_tile.push_back(b.tile);
    const long long nj = (long long)job_tile.size();
    auto names = [&](int j, long long tile) { return j >= 0 && j < nj && job_tile[j] == tile; };
    if (plan.term_blk.size() != plan.recs.size() * TC_MAX_G * 2) fail("term_blk size");
    else
      for (size_t i = 0; i < plan.recs.size(); ++i) {
        const TcUnitRec& r = plan.recs[i];
        if (r.flags & TC_ZERO) continue;
        for (int q = 0; q < r.nterm && q < TC_MAX_G; ++q)
          if (!names(plan.term_blk[(i * TC_MAX_G + q) * 2], r.t[q].a_tile) ||
              !names(plan.term_blk[(i * TC_MAX_G + q) * 2 + 1], r.t[q].b_tile))
            fail("record term split-block index");
      }
    if (plan.small_blk.size() != 2 * plan.small.size()) fail("small_blk size");
    else
      for (size_t k = 0; k < plan.small.size(); ++k) {
        const SmallTerm& x = plan.small[k];
        if ((x.a_tile >= 0 && !names(plan.small_blk[2 * k], x.a_tile)) ||
            (x.b_tile >= 0 && !names(plan.small_blk[2 * k + 1], x.b_tile)))
          fail("small term split-block index");
      }
  }

  // (4) the two schedules together are a permutation of the items, each
  //     holding the items of its kind
  std::vector<int> sch = plan.schedule;
  for (int i : plan.schedule)
    if (plan.items[i].kind != 0) fail("tensor-core schedule holds a small item");
  for (size_t k = 0; k < plan.small_schedule.size(); ++k)  // kind 2 first, then kind 1
    if (plan.items[plan.small_schedule[k]].kind != ((int)k < plan.n_small_mid ? 2 : 1))
      fail("small schedule: kinds or their order");
  sch.insert(sch.end(), plan.small_schedule.begin(), plan.small_schedule.end());
  std::sort(sch.begin(), sch.end());
  for (size_t i = 0; i < sch.size(); ++i)
    if (sch[i] != (int)i) {
      fail("schedule");
      break;
    }
  if (sch.size() != plan.items.size()) fail("schedule size");

  // MMA instructions per slice product (stage 1 per K step of 16, stage 2 per
  // term and K step) and stages, as the kernel issues them
  long long mma_s1 = 0, mma_s2 = 0, stages = 0;
  for (const TcUnitRec& r : plan.recs) {
    if (r.flags & TC_ZERO) continue;
    for (int j = 0; j < (r.n + 127) / 128; ++j) {
      mma_s1 += r.pR8 / 2;
      stages += (r.pR8 + 3) / 4;
      const int ncols = std::min(128, r.n - 128 * j);
      for (int h = 0; h < (ncols + 63) / 64; ++h) {
        const int kw = std::min(64, ncols - 64 * h), kg2 = 2 * ((kw + 15) / 16);
        const int te = 2 * ((r.tn + 15) / 16), P = std::max(1, std::min(r.nterm, 128 / (te * kg2)));
        mma_s2 += (long long)r.nterm * (kg2 / 2);
        stages += (r.nterm + P - 1) / P;
      }
    }
  }

  // (6) the kernel's copies, enumerated with its own formulas: every copy
  //     lands inside its stage (stage 1: operator rows below position 16 KG1,
  //     psi from there on) and reads inside the split arrays; where a term's
  //     stage-2 tiles form one run in the stored block they move as one copy
  //     and keep its stride, and every MMA operand read (K steps of 16, N
  //     rounded up to 16) stays inside the stage, or the term's stage-2
  //     region
  // (ST tile positions per stage, KG1 K groups per stage-1 stage: 128 / 4 for
  //     the bf16 kernels, 192 / 6 for FP16X2). The tile positions copied per
  //     sigma (operators and psi) give the bytes each kernel requests from
  //     L2 / HBM (384 B per position for bf16, 256 for fp16).
  long long copy_tiles[2] = {0, 0};
  for (const auto& geo : {std::pair<int, int>{128, 4}, std::pair<int, int>{192, 6}}) {
    const int ST = geo.first, KG1 = geo.second, PT = 16 * KG1;
    long long& ctiles = copy_tiles[ST == 128 ? 0 : 1];
    const long long op_tiles = plan.n_tiles, psi_tiles = plan.psi_tiles;
    auto src_ok = [&](long long src, int n, bool psi) {
      return src >= 0 && n > 0 && src + n <= (psi ? psi_tiles : op_tiles);
    };
    for (const TcUnitRec& r : plan.recs) {
      if (r.flags & TC_ZERO) continue;
      const int G = r.nterm, tm8 = r.tm8;
      const int nchunk = (r.n + 127) / 128;
      for (int j = 0; j < nchunk; ++j) {
        const int nk1 = (r.pR8 + KG1 - 1) / KG1;
        for (int k = 0; k < nk1; ++k) {
          const int kg0 = KG1 * k;
          const int nks = std::min(KG1, (int)r.pR8 - kg0) / 2;  // MMA K steps of the stage
          if (!(r.flags & TC_TA)) {
            const int nk = std::min(KG1, (int)r.aC8 - kg0);
            if (2 * nks > KG1) fail("stage-1 left operand read beyond its row group");
            if (nk > 0)
              for (int q = 0; q < G; ++q) {
                for (int rg = 0; rg < tm8; ++rg) {
                  const int dst = (q * tm8 + rg) * KG1;
                  ctiles += nk;
                  if (dst + nk > PT || !src_ok(r.t[q].a_tile + (long long)(r.r0g + rg) * r.aC8 + kg0, nk, false))
                    fail("stage-1 operator copy out of bounds");
                }
              }
          } else {
            for (int q = 0; q < G; ++q)
              for (int kg = 0; kg < KG1 && kg0 + kg < r.aR8; ++kg) {
                const int dst = kg * 16 + q * tm8;
                ctiles += tm8;
                if (q * tm8 + tm8 > 16 || dst + tm8 > PT ||
                    !src_ok(r.t[q].a_tile + (long long)(kg0 + kg) * r.aC8 + r.r0g, tm8, false))
                  fail("stage-1 transposed operator copy out of bounds");
              }
          }
          const int nn = std::min(16, (int)r.pC8 - 16 * j);
          const int nkP = std::min(KG1, (int)r.pR8 - kg0);
          const int cc = std::min(128, r.n - 128 * j), nN = 2 * ((cc + 15) / 16);
          if (PT + (2 * nks - 1) * 16 + nN > ST) fail("stage-1 psi operand read beyond the stage");
          for (int kg = 0; kg < nkP; ++kg)
            if ((ctiles += nn), PT + kg * 16 + nn > ST || !src_ok(r.p_tile + (long long)(kg0 + kg) * r.pC8 + 16 * j, nn, true))
              fail("stage-1 psi copy out of bounds");
        }
        const int ncols = std::min(128, r.n - 128 * j);
        for (int h = 0; h < (ncols + 63) / 64; ++h) {
          const int kw = std::min(64, ncols - 64 * h), kg2 = 2 * ((kw + 15) / 16), kgx = 16 * j + 8 * h;
          const int te = 2 * ((r.tn + 15) / 16), tn8 = (r.tn + 7) / 8;
          const int P = std::max(1, std::min(G, ST / (te * kg2)));
          for (int q0 = 0; q0 < G; q0 += P)
            for (int q = q0; q < std::min(G, q0 + P); ++q) {
              const int reg = (q - q0) * te * kg2;
              if (reg + te * kg2 > ST) fail("stage-2 region beyond the stage");
              if (!(r.flags & TC_TB)) {
                const int nk = std::min(kg2, (int)r.bC8 - kgx);
                // one producer: a single run (N-group stride bC8) when the
                // half holds all K groups; three: one copy per N group
                const bool run = nk == r.bC8;
                if (run && ((te - 1) * r.bC8 + kg2 > te * kg2 || reg + tn8 * nk > ST ||
                            !src_ok(r.t[q].b_tile + (long long)r.c0g * r.bC8, tn8 * nk, false)))
                  fail("stage-2 operator run out of bounds");
                for (int ng = 0; ng < tn8; ++ng)
                  if ((ctiles += std::max(nk, 0)), reg + ng * kg2 + nk > ST ||
                      !src_ok(r.t[q].b_tile + (long long)(r.c0g + ng) * r.bC8 + kgx, nk, false))
                    fail("stage-2 operator copy out of bounds");
              } else {
                const int nk = std::min(kg2, (int)r.bR8 - kgx);
                // one producer: a single run (K-group stride tn8) when the
                // tile spans the stored columns; three: one copy per K group
                const bool run = tn8 == r.bC8;
                if (run && ((kg2 - 1) * tn8 + te > te * kg2 || reg + nk * tn8 > ST ||
                            !src_ok(r.t[q].b_tile + (long long)kgx * r.bC8, nk * tn8, false)))
                  fail("stage-2 transposed operator run out of bounds");
                for (int kg = 0; kg < nk; ++kg)
                  if ((ctiles += tn8), reg + kg * te + tn8 > ST ||
                      !src_ok(r.t[q].b_tile + (long long)(kgx + kg) * r.bC8 + r.c0g, tn8, false))
                    fail("stage-2 transposed operator copy out of bounds");
              }
            }
        }
      }
    }
  }

  // bytes the FP64 kernel requests per sigma: for every (item, task) the
  // output tile's rows of the left block, the psi block and the tile's
  // columns of the right block (identities are not read)
  double f64_req = 0.0;
  for (const Item& it : wl.items)
    for (int t = it.t_begin; t < it.t_end; ++t) {
      const Task& k = wl.tasks[t];
      const PsiBlock& ib = blocks[k.in_blk];
      f64_req += 8.0 * ((k.aoff >= 0 ? (double)it.nrows * ib.mL : 0.0) + (double)ib.mL * ib.mR +
                        (k.boff >= 0 ? (double)it.ncols * ib.mR : 0.0));
    }
  // tile positions the small-class kernels read per sigma: each term's left
  // and right blocks, and its psi block once per warp and run of terms of
  // one psi block (warps take every 8th (<= 16 class) or 4th term)
  long long small_tiles = 0;
  for (const TcItem& it : plan.items) {
    if (it.kind != 1 && it.kind != 2) continue;
    const int nw = it.kind == 2 ? 8 : 4;
    for (int w = 0; w < nw; ++w) {
      int cur = -1;
      for (int k = it.r_begin + w; k < it.r_end; k += nw) {
        const SmallTerm& x = plan.small[k];
        const TcPsiBlock& pb = plan.psi[x.in_blk];
        const int m = pb.m, n = pb.n, tm = it.nrows, tn = it.ncols;
        if (x.in_blk != cur) small_tiles += (long long)pb.R8 * pb.C8;
        cur = x.in_blk;
        if (x.a_tile >= 0) small_tiles += (long long)((tm + 7) / 8) * ((m + 7) / 8);
        if (x.b_tile >= 0) small_tiles += (long long)((tn + 7) / 8) * ((n + 7) / 8);
      }
    }
  }
  std::printf("{\"psi_size\": %lld, \"blocks\": %zu, \"terms\": %zu, \"tasks\": %zu, \"flops\": %.17g, "
              "\"plan_tasks\": %lld, \"units\": %lld, \"items\": %zu, \"mma_s1\": %lld, \"mma_s2\": %lld, "
              "\"stages\": %lld, \"op_elements\": %lld, \"f64_request_bytes\": %.17g, "
              "\"tc_copy_bytes_bf16\": %lld, \"tc_copy_bytes_fp16\": %lld, \"small_read_bytes_bf16\": %lld, "
              "\"small_read_bytes_fp16\": %lld, \"layout\": [",
              size, blocks.size(), terms.size(), wl.tasks.size(), wl.flops, plan.n_terms, plan.n_units,
              plan.items.size(), mma_s1, mma_s2, stages, (long long)(oL.elements + oR.elements), f64_req,
              copy_tiles[0] * 384, copy_tiles[1] * 256, small_tiles * 384, small_tiles * 256);
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
