// Host-logic check of the blocking formulas (CPU only, no CUDA calls): reads
// the integrals, a block's basis and its operator store, builds the term
// lists of the enlarged block with the library's own host code (terms.h:
// NC, CN and the normal-to-complementary transformation), applies them with
// a plain CPU loop that follows the blocking kernel's rules (sector lookup,
// chunk offsets, fermion signs, transposed sources; complementary sums as
// a plain matrix product), and writes the enlarged operator store.
//
//   blocking_check <in file> <out file>
//   in: int32 K, side (0 left, 1 right), site, src_cn, dst_cn, nsec;
//       nsec x (N, 2Sz, dim); float64 t (K*K), v (K^4), store (its length)
//   out: int64 count, then that many float64 (the enlarged store)
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "model.h"
#include "terms.h"

using namespace dmrg;
using namespace dmrg::terms;

int main(int argc, char** argv) {
  if (argc < 3) return 2;
  FILE* f = std::fopen(argv[1], "rb");
  if (!f) return 3;
  int hdr[6];
  if (std::fread(hdr, sizeof(int), 6, f) != 6) return 4;
  const int K = hdr[0], side = hdr[1], s = hdr[2], src_cn = hdr[3], dst_cn = hdr[4], nsec = hdr[5];
  const bool left = side == 0;
  Basis bb;
  for (int i = 0; i < nsec; ++i) {
    int q[3];
    if (std::fread(q, sizeof(int), 3, f) != 3) return 4;
    bb.q.push_back({q[0], q[1]});
    bb.dim.push_back(q[2]);
  }
  bb.finish();
  Ints I;
  I.K = K;
  I.t.resize((size_t)K * K);
  I.v.resize((size_t)K * K * K * K);
  if (std::fread(I.t.data(), sizeof(double), I.t.size(), f) != I.t.size()) return 4;
  if (std::fread(I.v.data(), sizeof(double), I.v.size(), f) != I.v.size()) return 4;
  const int n = 2 * K;
  const int nLb = left ? 2 * s : 2 * s + 2, nE = left ? 2 * s + 2 : 2 * s;
  OpSet B;
  build_nc_opset(B, bb, nLb, n, left, 0, src_cn != 0);
  std::vector<double> src((size_t)B.elements);
  if (std::fread(src.data(), sizeof(double), src.size(), f) != src.size()) return 4;
  std::fclose(f);

  const Enlarged E = enlarge(bb);
  OpSet EO;
  build_nc_opset(EO, E.basis, nE, n, left, 0, dst_cn != 0);
  // complementary sums (the transformation): Y_o = sum_i C[o][i] X_i per class
  CompSet cs;
  std::vector<double> comp;
  const int nsrc1 = (int)B.ops.size();
  const bool transform = src_cn != dst_cn;
  if (transform) {
    const NCIndex bx = left ? NCIndex{2 * s, n, false} : NCIndex{2 * s + 2, n, true};
    if (left) make_comp(I, bx, B, 2 * s + 2, n, cs);
    else make_comp(I, bx, B, 0, 2 * s, cs);
    comp.assign((size_t)cs.set.elements, 0.0);
    for (const CombClass& c : cs.cls)
      for (int o = 0; o < c.n_out; ++o)
        for (long long e = 0; e < c.E; ++e) {
          double acc = 0.0;
          for (int i = 0; i < c.n_in; ++i) acc += cs.coef[c.c_off + (long long)o * c.n_in + i] * src[cs.xoff[c.x_start + i] + e];
          comp[c.y_off + (long long)o * c.E + e] = acc;
        }
  }
  std::vector<ETerms> T;
  if (left) T = dst_cn ? left_terms_cn(I, s, !src_cn, &cs, nsrc1) : left_terms(I, s);
  else T = src_cn ? right_terms_cn(I, s, !dst_cn, &cs, nsrc1) : right_terms(I, s);
  if (T.size() != EO.ops.size()) return 5;

  auto op_of = [&](int k) -> const OpDesc& { return k < nsrc1 ? B.ops[k] : cs.set.ops[k - nsrc1]; };
  auto store_of = [&](int k) -> const double* { return k < nsrc1 ? src.data() : comp.data(); };
  std::vector<double> out((size_t)EO.elements, 0.0);
  int bad = 0;
  for (size_t k = 0; k < EO.ops.size(); ++k)
    for (const OpBlock& db : EO.ops[k].blocks) {
      double* dst = out.data() + db.off;
      const QN Qin = E.basis.q[db.qin], Qout = E.basis.q[db.qout];
      for (const ETerm& tm : T[k]) {
        const int ib = bb.find(Qin - SITE_Q[tm.nin]);
        if (ib < 0) continue;
        const int c0 = E.chunk_off[db.qin][ib];
        if (c0 < 0) continue;
        int ob = ib, par = 0;
        long long soff = -1;
        const double* S = nullptr;
        if (tm.src >= 0) {
          const OpDesc& o = op_of(tm.src);
          par = o.parity;
          S = store_of(tm.src);
          if (!tm.trans) {
            const int kb = o.by_qin[ib];
            if (kb < 0) continue;
            soff = o.blocks[kb].off;
            ob = o.blocks[kb].qout;
          } else {
            ob = bb.find(bb.q[ib] - o.dq);
            if (ob < 0 || o.by_qin[ob] < 0) continue;
            soff = o.blocks[o.by_qin[ob]].off;
          }
        }
        if (!(bb.q[ob] + SITE_Q[tm.nout] == Qout)) {
          ++bad;
          continue;
        }
        const int r0 = E.chunk_off[db.qout][ob];
        if (r0 < 0) continue;
        const int rows = bb.dim[ob], cols = bb.dim[ib];
        bool neg;
        if (left) neg = ((SITE_N[tm.nout] - SITE_N[tm.nin]) & 1) && (bb.q[ib].n & 1);
        else neg = par && (SITE_N[tm.nin] & 1);
        const double w = neg ? -tm.coef : tm.coef;
        for (int i = 0; i < rows; ++i)
          for (int j = 0; j < cols; ++j) {
            double v;
            if (tm.src < 0) v = i == j ? 1.0 : 0.0;
            else if (!tm.trans) v = S[soff + (long long)i * cols + j];
            else v = S[soff + (long long)j * rows + i];
            dst[(long long)(r0 + i) * db.cols + c0 + j] += w * v;
          }
      }
    }
  if (bad) return 6;
  FILE* g = std::fopen(argv[2], "wb");
  const long long cnt = (long long)out.size();
  std::fwrite(&cnt, sizeof(cnt), 1, g);
  std::fwrite(out.data(), sizeof(double), out.size(), g);
  std::fclose(g);
  return 0;
}
