// Host-side blocking formulas of the sweeps (definitions; see terms.h).
#include "terms.h"

#include <algorithm>
#include <cmath>

namespace dmrg {
namespace terms {

void add(ETerms& e, int src, bool trans, double c, const Mat4& m) {
  if (c == 0.0) return;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j)
      if (m[i][j] != 0.0) e.push_back({src, trans, c * m[i][j], i, j});
}

Enlarged enlarge(const Basis& b) {
  std::map<std::pair<int, int>, int> dims;
  for (int i = 0; i < b.size(); ++i)
    for (int n = 0; n < 4; ++n) {
      QN Q = b.q[i] + SITE_Q[n];
      dims[{Q.n, Q.s}] += b.dim[i];
    }
  Enlarged E;
  for (auto& kv : dims) {
    E.basis.q.push_back({kv.first.first, kv.first.second});
    E.basis.dim.push_back(kv.second);
  }
  E.basis.finish();
  E.chunk_off.assign(E.basis.size(), std::vector<int>(b.size(), -1));
  std::vector<int> fill(E.basis.size(), 0);
  for (int i = 0; i < b.size(); ++i)  // ascending block sector
    for (int n = 0; n < 4; ++n) {
      const int Qi = E.basis.find(b.q[i] + SITE_Q[n]);
      E.chunk_off[Qi][i] = fill[Qi];
      fill[Qi] += b.dim[i];
    }
  return E;
}

// ----------------------------------------------------- blocking formulas
// Left: block L holds modes [0, 2s); site s; enlarged NC set nL' = 2s + 2.
std::vector<ETerms> left_terms(const Ints& I, int s) {
  const int n = 2 * I.K, nL = 2 * s, nE = 2 * s + 2;
  NCIndex bx{nL, n}, ex{nE, n};
  Site st{I, s};
  std::vector<ETerms> T(ex.count());
  const int S0 = 2 * s, S1 = 2 * s + 1;
  auto B = [&](int p, int q, bool& t) {  // B_pq = B_pq or B_qp^T
    t = p > q;
    return p <= q ? bx.B(p, q) : bx.B(q, p);
  };
  // H
  {
    ETerms& e = T[ex.H()];
    add(e, bx.H(), false, 1.0, eye4());
    add(e, -1, false, 1.0, st.H());
    for (int p = 0; p < nL; ++p) {
      const Mat4 Rs = st.R(p, true);
      add(e, bx.cd(p), false, 1.0, Rs);
      add(e, bx.cd(p), true, -1.0, tr(Rs));
    }
    for (int p = S0; p <= S1; ++p) {
      add(e, bx.RL(p), true, 1.0, st.ann(p));
      add(e, bx.RL(p), false, -1.0, st.cre(p));
    }
    for (int p = 0; p < nL; ++p)
      for (int r = p + 1; r < nL; ++r) {
        const Mat4 Ps = st.P(p, r);
        add(e, bx.A(p, r), false, 1.0, Ps);
        add(e, bx.A(p, r), true, 1.0, tr(Ps));
      }
    for (int p = 0; p < nL; ++p)
      for (int q = 0; q < nL; ++q) {
        bool t;
        const int k = B(p, q, t);
        add(e, k, t, 1.0, st.Q(p, q));
      }
  }
  // a+_p
  for (int p = 0; p < nL; ++p) add(T[ex.cd(p)], bx.cd(p), false, 1.0, eye4());
  for (int p = S0; p <= S1; ++p) add(T[ex.cd(p)], -1, false, 1.0, st.cre(p));
  // A_pr, B_pq
  for (int p = 0; p < nE; ++p)
    for (int r = p; r < nE; ++r) {
      if (p < r) {
        ETerms& e = T[ex.A(p, r)];
        if (r < nL) add(e, bx.A(p, r), false, 1.0, eye4());
        else if (p < nL) add(e, bx.cd(p), false, 1.0, st.cre(r));
        else add(e, -1, false, 1.0, mul(st.cre(p), st.cre(r)));
      }
      ETerms& e = T[ex.B(p, r)];
      if (r < nL) add(e, bx.B(p, r), false, 1.0, eye4());
      else if (p < nL) add(e, bx.cd(p), false, 1.0, st.ann(r));
      else add(e, -1, false, 1.0, mul(st.cre(p), st.ann(r)));
    }
  // R^L_p for p right of the enlarged block
  for (int p = nE; p < n; ++p) {
    ETerms& e = T[ex.RL(p)];
    add(e, bx.RL(p), false, 1.0, eye4());
    add(e, -1, false, 1.0, st.R(p, false));
    for (int x = S0; x <= S1; ++x)  // (sum_{r,y} (v_pxry - v_pyrx) B_ry) (x) a_x
      for (int r = 0; r < nL; ++r)
        for (int y = 0; y < nL; ++y) {
          const double c = I.vso(p, x, r, y) - I.vso(p, y, r, x);
          if (c == 0.0) continue;
          bool t;
          const int k = B(r, y, t);
          add(e, k, t, c, st.ann(x));
        }
    for (int r = S0; r <= S1; ++r)  // (sum_{q,w} v_pqrw a_w a_q) (x) a+_r
      for (int q = 0; q < nL; ++q)
        for (int w = 0; w < nL; ++w) {
          const double c = I.vso(p, q, r, w);
          if (c == 0.0 || q == w) continue;
          if (q < w) add(e, bx.A(q, w), true, c, st.cre(r));   // a_w a_q = A_qw^T
          else add(e, bx.A(w, q), true, -c, st.cre(r));        // = -A_wq^T
        }
    for (int w = 0; w < nL; ++w) {  // -a_w (x) sum v_pqrw a+_r a_q  (q, r on the site)
      Mat4 m = zero4();
      for (int q = S0; q <= S1; ++q)
        for (int r = S0; r <= S1; ++r) axpy(m, I.vso(p, q, r, w), mul(st.cre(r), st.ann(q)));
      add(e, bx.cd(w), true, -1.0, m);
    }
    for (int r = 0; r < nL; ++r) {  // a+_r (x) sum v_pqrw a_w a_q  (q, w on the site)
      Mat4 m = zero4();
      for (int q = S0; q <= S1; ++q)
        for (int w = S0; w <= S1; ++w) axpy(m, I.vso(p, q, r, w), mul(st.ann(w), st.ann(q)));
      add(e, bx.cd(r), false, 1.0, m);
    }
    for (int q = 0; q < nL; ++q) {  // a_q (x) sum v_pqrw a+_r a_w  (r, w on the site)
      Mat4 m = zero4();
      for (int r = S0; r <= S1; ++r)
        for (int w = S0; w <= S1; ++w) axpy(m, I.vso(p, q, r, w), mul(st.cre(r), st.ann(w)));
      add(e, bx.cd(q), true, 1.0, m);
    }
  }
  return T;
}

// Right: block R holds modes [2s+2, n) (complementary indices p < 2s+2);
// site s; enlarged NC set (right kind) nL' = 2s. Terms read site (x) block.
std::vector<ETerms> right_terms(const Ints& I, int s) {
  const int n = 2 * I.K, nLb = 2 * s + 2, nE = 2 * s;
  NCIndex bx{nLb, n}, ex{nE, n};
  Site st{I, s};
  std::vector<ETerms> T(ex.count());
  const int S0 = 2 * s, S1 = 2 * s + 1;
  auto Qk = [&](int p, int q, bool& t) {
    t = p > q;
    return p <= q ? bx.B(p, q) : bx.B(q, p);
  };
  for (int p = S0; p <= S1; ++p) add(T[ex.d(p)], -1, false, 1.0, st.ann(p));
  for (int p = nLb; p < n; ++p) add(T[ex.d(p)], bx.d(p), false, 1.0, eye4());
  {  // H of site x R: NC decomposition over (site | R)
    ETerms& e = T[ex.H()];
    add(e, -1, false, 1.0, st.H());
    add(e, bx.H(), false, 1.0, eye4());
    for (int p = S0; p <= S1; ++p) {
      add(e, bx.RR(p), false, 1.0, st.cre(p));
      add(e, bx.RR(p), true, -1.0, st.ann(p));
    }
    for (int p = nLb; p < n; ++p) {
      const Mat4 Rs = st.R(p, false);
      add(e, bx.d(p), false, 1.0, tr(Rs));
      add(e, bx.d(p), true, -1.0, Rs);
    }
    const Mat4 A = mul(st.cre(S0), st.cre(S1));
    add(e, bx.A(S0, S1), false, 1.0, A);
    add(e, bx.A(S0, S1), true, 1.0, tr(A));
    for (int p = S0; p <= S1; ++p)
      for (int q = S0; q <= S1; ++q) {
        bool t;
        const int k = Qk(p, q, t);
        add(e, k, t, 1.0, mul(st.cre(p), st.ann(q)));
      }
  }
  for (int p = 0; p < nE; ++p) {  // R^R_p
    ETerms& e = T[ex.RR(p)];
    add(e, bx.RR(p), false, 1.0, eye4());
    add(e, -1, false, 1.0, st.R(p, true));
    for (int x = S0; x <= S1; ++x) {
      add(e, bx.B(p, x), false, 1.0, st.ann(x));  // a_x (x) Q_px
      add(e, bx.A(p, x), false, 1.0, st.cre(x));  // a+_x (x) P_px
    }
    for (int y = nLb; y < n; ++y) {
      Mat4 m1 = zero4(), m2 = zero4(), m3 = zero4();
      for (int u = S0; u <= S1; ++u)
        for (int w = S0; w <= S1; ++w) {
          axpy(m1, I.vso(p, u, w, y), mul(st.cre(w), st.ann(u)));
          axpy(m2, I.vso(p, u, y, w), mul(st.ann(w), st.ann(u)));
          axpy(m3, I.vso(p, y, u, w), mul(st.cre(u), st.ann(w)));
        }
      add(e, bx.d(y), false, -1.0, m1);
      add(e, bx.d(y), true, 1.0, m2);
      add(e, bx.d(y), false, 1.0, m3);
    }
  }
  for (int p = 0; p < nE; ++p)
    for (int r = p; r < nE; ++r) {
      if (p < r) {  // P_pr
        ETerms& e = T[ex.A(p, r)];
        add(e, bx.A(p, r), false, 1.0, eye4());
        add(e, -1, false, 1.0, st.P(p, r));
        for (int x = S0; x <= S1; ++x)
          for (int y = nLb; y < n; ++y) add(e, bx.d(y), false, I.vso(p, y, r, x) - I.vso(p, x, r, y), st.ann(x));
      }
      {  // Q_pr
        ETerms& e = T[ex.B(p, r)];
        const int q = r;
        add(e, bx.B(p, q), false, 1.0, eye4());
        add(e, -1, false, 1.0, st.Q(p, q));
        for (int x = S0; x <= S1; ++x)
          for (int y = nLb; y < n; ++y) {
            add(e, bx.d(y), false, I.vso(p, q, x, y) - I.vso(p, y, x, q), st.cre(x));
            add(e, bx.d(y), true, -(I.vso(p, q, y, x) - I.vso(p, x, y, q)), st.ann(x));
          }
      }
    }
  return T;
}

void make_comp(const Ints& I, const NCIndex& bx, const OpSet& bset, int o0, int o1, CompSet& cs) {
  const int s0 = bx.pb(), s1 = bx.pb() + bx.np();
  struct Src {
    int op, a, b;
    bool isB;
  };
  struct Out {
    char kind;  // 'T', 'U', 'V'
    int p, q;
  };
  std::map<std::pair<int, int>, std::pair<std::vector<Src>, std::vector<Out>>> cl;  // by (dN, d2Sz)
  for (int q = s0; q < s1; ++q)
    for (int w = q + 1; w < s1; ++w) cl[{2, spin_of(q) + spin_of(w)}].first.push_back({bx.A(q, w), q, w, false});
  for (int r = s0; r < s1; ++r)
    for (int w = r; w < s1; ++w) cl[{0, spin_of(r) - spin_of(w)}].first.push_back({bx.B(r, w), r, w, true});
  for (int p = o0; p < o1; ++p)
    for (int r = p + 1; r < o1; ++r) cl[{2, spin_of(p) + spin_of(r)}].second.push_back({'T', p, r});
  for (int p = o0; p < o1; ++p)
    for (int q = p; q < o1; ++q) {
      cl[{0, spin_of(q) - spin_of(p)}].second.push_back({'U', p, q});
      cl[{0, spin_of(p) - spin_of(q)}].second.push_back({'V', p, q});
    }
  cs.set = OpSet();
  cs.set.basis = bset.basis;
  long long cur = 0;
  for (auto& kv : cl) {
    const QN dq{kv.first.first, kv.first.second};
    const auto& src = kv.second.first;
    const auto& out = kv.second.second;
    if (out.empty()) continue;
    CombClass cc{};
    const int first = (int)cs.set.ops.size();
    for (const Out& o : out) {
      const int idx = (int)cs.set.ops.size();
      add_op(cs.set, dq, 0, false, cur);
      (o.kind == 'T' ? cs.T : o.kind == 'U' ? cs.U : cs.V)[{o.p, o.q}] = idx;
    }
    const OpDesc& f = cs.set.ops[first];
    long long E = 0;
    for (const OpBlock& b : f.blocks) E += (long long)b.rows * b.cols;
    cc.y_off = f.blocks.empty() ? 0 : f.blocks[0].off;
    cc.E = E;
    cc.n_out = (int)out.size();
    cc.n_in = (int)src.size();
    cc.x_start = (int)cs.xoff.size();
    cc.c_off = (long long)cs.coef.size();
    for (const Src& x : src) {
      const OpDesc& so = bset.ops[x.op];
      cs.xoff.push_back(so.blocks.empty() ? 0 : so.blocks[0].off);
    }
    for (const Out& o : out)
      for (const Src& x : src) {
        double c = 0.0;
        if (o.kind == 'T') {
          if (!x.isB) c = I.vso(o.p, x.a, o.q, x.b) - I.vso(o.p, x.b, o.q, x.a);
        } else if (x.isB) {
          if (o.kind == 'U') c = I.vso(o.p, o.q, x.a, x.b) - I.vso(o.p, x.b, x.a, o.q);
          else if (x.a < x.b) c = I.vso(o.p, o.q, x.b, x.a) - I.vso(o.p, x.a, x.b, o.q);
        }
        cs.coef.push_back(c);
      }
    cc.tiles_e = (int)((E + COMB_TN - 1) / COMB_TN);
    cc.tile_start = cs.ntiles;
    cs.ntiles += cc.tiles_e * ((cc.n_out + COMB_TM - 1) / COMB_TM);
    cs.flops += 2.0 * cc.n_out * cc.n_in * (double)E;
    cs.cls.push_back(cc);
  }
  cs.set.elements = cur;
}

// Left: block L holds modes [0, 2s) (NC form when src_nc, else CN form); the
// enlarged block (modes [0, 2s+2)) is in CN form: H, a+_p, R^L_p (p >= 2s+2),
// P^L_pr, Q^L_pq (2s+2 <= p, q, r). Comp ops (src_nc) are source indices
// nsrc1 + comp index.
std::vector<ETerms> left_terms_cn(const Ints& I, int s, bool src_nc, const CompSet* cs, int nsrc1) {
  const int n = 2 * I.K, nL = 2 * s, nE = 2 * s + 2;
  NCIndex bx{nL, n, !src_nc}, ex{nE, n, true};
  Site st{I, s};
  std::vector<ETerms> T(ex.count());
  const int S0 = 2 * s, S1 = 2 * s + 1;
  auto herm = [](const NCIndex& x, int p, int q, bool& t) {  // O_pq = O_pq or O_qp^T
    t = p > q;
    return p <= q ? x.B(p, q) : x.B(q, p);
  };
  {  // H of L x s
    ETerms& e = T[ex.H()];
    add(e, bx.H(), false, 1.0, eye4());
    add(e, -1, false, 1.0, st.H());
    for (int p = 0; p < nL; ++p) {
      const Mat4 Rs = st.R(p, true);
      add(e, bx.cd(p), false, 1.0, Rs);
      add(e, bx.cd(p), true, -1.0, tr(Rs));
    }
    for (int p = S0; p <= S1; ++p) {
      add(e, bx.RL(p), true, 1.0, st.ann(p));
      add(e, bx.RL(p), false, -1.0, st.cre(p));
    }
    if (src_nc) {  // NC form at the cut (L | s)
      for (int p = 0; p < nL; ++p)
        for (int r = p + 1; r < nL; ++r) {
          const Mat4 Ps = st.P(p, r);
          add(e, bx.A(p, r), false, 1.0, Ps);
          add(e, bx.A(p, r), true, 1.0, tr(Ps));
        }
      for (int p = 0; p < nL; ++p)
        for (int q = 0; q < nL; ++q) {
          bool t;
          const int k = herm(bx, p, q, t);
          add(e, k, t, 1.0, st.Q(p, q));
        }
    } else {  // CN form: P^L / Q^L of the site's modes with the site's normal pairs
      const Mat4 A = mul(st.cre(S0), st.cre(S1));
      add(e, bx.A(S0, S1), false, 1.0, A);
      add(e, bx.A(S0, S1), true, 1.0, tr(A));
      for (int p = S0; p <= S1; ++p)
        for (int q = S0; q <= S1; ++q) {
          bool t;
          const int k = herm(bx, p, q, t);
          add(e, k, t, 1.0, mul(st.cre(p), st.ann(q)));
        }
    }
  }
  for (int p = 0; p < nL; ++p) add(T[ex.cd(p)], bx.cd(p), false, 1.0, eye4());
  for (int p = S0; p <= S1; ++p) add(T[ex.cd(p)], -1, false, 1.0, st.cre(p));
  for (int p = nE; p < n; ++p) {  // R^L_p
    ETerms& e = T[ex.RL(p)];
    add(e, bx.RL(p), false, 1.0, eye4());
    add(e, -1, false, 1.0, st.R(p, false));
    if (src_nc) {  // Q^L_px and P^L_pr of L written out over its B and A
      for (int x = S0; x <= S1; ++x)
        for (int r = 0; r < nL; ++r)
          for (int y = 0; y < nL; ++y) {
            const double c = I.vso(p, x, r, y) - I.vso(p, y, r, x);
            if (c == 0.0) continue;
            bool t;
            const int k = herm(bx, r, y, t);
            add(e, k, t, c, st.ann(x));
          }
      for (int r = S0; r <= S1; ++r)
        for (int q = 0; q < nL; ++q)
          for (int w = 0; w < nL; ++w) {
            const double c = I.vso(p, q, r, w);
            if (c == 0.0 || q == w) continue;
            if (q < w) add(e, bx.A(q, w), true, c, st.cre(r));
            else add(e, bx.A(w, q), true, -c, st.cre(r));
          }
    } else {  // stored: Q^L_px = (Q^L_xp)^T, P^L_pr = -P^L_rp (x, r < p)
      for (int x = S0; x <= S1; ++x) add(e, bx.B(x, p), true, 1.0, st.ann(x));
      for (int r = S0; r <= S1; ++r) add(e, bx.A(r, p), false, -1.0, st.cre(r));
    }
    for (int w = 0; w < nL; ++w) {  // -a_w (x) sum v_pqrw a+_r a_q  (q, r on the site)
      Mat4 m = zero4();
      for (int q = S0; q <= S1; ++q)
        for (int r = S0; r <= S1; ++r) axpy(m, I.vso(p, q, r, w), mul(st.cre(r), st.ann(q)));
      add(e, bx.cd(w), true, -1.0, m);
    }
    for (int r = 0; r < nL; ++r) {  // a+_r (x) sum v_pqrw a_w a_q  (q, w on the site)
      Mat4 m = zero4();
      for (int q = S0; q <= S1; ++q)
        for (int w = S0; w <= S1; ++w) axpy(m, I.vso(p, q, r, w), mul(st.ann(w), st.ann(q)));
      add(e, bx.cd(r), false, 1.0, m);
    }
    for (int q = 0; q < nL; ++q) {  // a_q (x) sum v_pqrw a+_r a_w  (r, w on the site)
      Mat4 m = zero4();
      for (int r = S0; r <= S1; ++r)
        for (int w = S0; w <= S1; ++w) axpy(m, I.vso(p, q, r, w), mul(st.cre(r), st.ann(w)));
      add(e, bx.cd(q), true, 1.0, m);
    }
  }
  for (int p = nE; p < n; ++p)
    for (int r = p; r < n; ++r) {
      if (p < r) {  // P^L_pr = sum_{q,w in L+s} v_pqrw a_w a_q
        ETerms& e = T[ex.A(p, r)];
        if (src_nc) add(e, nsrc1 + cs->T.at({p, r}), true, 1.0, eye4());
        else add(e, bx.A(p, r), false, 1.0, eye4());
        add(e, -1, false, 1.0, st.P(p, r));
        for (int x = S0; x <= S1; ++x)  // one of q, w on the site (x), the other in L (y)
          for (int y = 0; y < nL; ++y) add(e, bx.cd(y), true, I.vso(p, x, r, y) - I.vso(p, y, r, x), st.ann(x));
      }
      {  // Q^L_pq = sum_{r',w in L+s} (v_pqr'w - v_pwr'q) a+_r' a_w
        ETerms& e = T[ex.B(p, r)];
        const int q = r;
        if (src_nc) {
          add(e, nsrc1 + cs->U.at({p, q}), false, 1.0, eye4());
          add(e, nsrc1 + cs->V.at({p, q}), true, 1.0, eye4());
        } else {
          add(e, bx.B(p, q), false, 1.0, eye4());
        }
        add(e, -1, false, 1.0, st.Q(p, q));
        for (int x = S0; x <= S1; ++x)
          for (int y = 0; y < nL; ++y) {
            add(e, bx.cd(y), false, I.vso(p, q, y, x) - I.vso(p, x, y, q), st.ann(x));    // a+_y (x) a_x
            add(e, bx.cd(y), true, -(I.vso(p, q, x, y) - I.vso(p, y, x, q)), st.cre(x));  // -a_y (x) a+_x
          }
      }
    }
  return T;
}

// Right: block R holds modes [2s+2, n) in CN form (normal A, B over its
// modes); the enlarged block (modes [2s, n)) is in NC form when dst_nc (P, Q
// over [0, 2s) from the comp ops: the transformation), else in CN form.
std::vector<ETerms> right_terms_cn(const Ints& I, int s, bool dst_nc, const CompSet* cs, int nsrc1) {
  const int n = 2 * I.K, nLb = 2 * s + 2, nE = 2 * s;
  NCIndex bx{nLb, n, true}, ex{nE, n, !dst_nc};
  Site st{I, s};
  std::vector<ETerms> T(ex.count());
  const int S0 = 2 * s, S1 = 2 * s + 1;
  auto herm = [&](int p, int q, bool& t) {
    t = p > q;
    return p <= q ? bx.B(p, q) : bx.B(q, p);
  };
  for (int p = S0; p <= S1; ++p) add(T[ex.d(p)], -1, false, 1.0, st.ann(p));
  for (int p = nLb; p < n; ++p) add(T[ex.d(p)], bx.d(p), false, 1.0, eye4());
  {  // H of site x R, CN form at the cut (s | R)
    ETerms& e = T[ex.H()];
    add(e, -1, false, 1.0, st.H());
    add(e, bx.H(), false, 1.0, eye4());
    for (int p = S0; p <= S1; ++p) {
      add(e, bx.RR(p), false, 1.0, st.cre(p));
      add(e, bx.RR(p), true, -1.0, st.ann(p));
    }
    for (int p = nLb; p < n; ++p) {
      const Mat4 Rs = st.R(p, false);
      add(e, bx.d(p), false, 1.0, tr(Rs));
      add(e, bx.d(p), true, -1.0, Rs);
    }
    for (int p = nLb; p < n; ++p)
      for (int r = p + 1; r < n; ++r) {
        const Mat4 Ps = st.P(p, r);
        add(e, bx.A(p, r), false, 1.0, Ps);
        add(e, bx.A(p, r), true, 1.0, tr(Ps));
      }
    for (int p = nLb; p < n; ++p)
      for (int q = nLb; q < n; ++q) {
        bool t;
        const int k = herm(p, q, t);
        add(e, k, t, 1.0, st.Q(p, q));
      }
  }
  for (int p = 0; p < nE; ++p) {  // R^R_p
    ETerms& e = T[ex.RR(p)];
    add(e, bx.RR(p), false, 1.0, eye4());
    add(e, -1, false, 1.0, st.R(p, true));
    for (int x = S0; x <= S1; ++x) {
      // a_x (x) Q^R_px: sum_{r,y in R} (v_pxry - v_pyrx) a+_r a_y
      for (int r = nLb; r < n; ++r)
        for (int y = nLb; y < n; ++y) {
          const double c = I.vso(p, x, r, y) - I.vso(p, y, r, x);
          if (c == 0.0) continue;
          bool t;
          const int k = herm(r, y, t);
          add(e, k, t, c, st.ann(x));
        }
      // a+_x (x) P^R_px: sum_{q,w in R} v_pqxw a_w a_q
      for (int q = nLb; q < n; ++q)
        for (int w = nLb; w < n; ++w) {
          const double c = I.vso(p, q, x, w);
          if (c == 0.0 || q == w) continue;
          if (q < w) add(e, bx.A(q, w), true, c, st.cre(x));
          else add(e, bx.A(w, q), true, -c, st.cre(x));
        }
    }
    for (int y = nLb; y < n; ++y) {
      Mat4 m1 = zero4(), m2 = zero4(), m3 = zero4();
      for (int u = S0; u <= S1; ++u)
        for (int w = S0; w <= S1; ++w) {
          axpy(m1, I.vso(p, u, w, y), mul(st.cre(w), st.ann(u)));
          axpy(m2, I.vso(p, u, y, w), mul(st.ann(w), st.ann(u)));
          axpy(m3, I.vso(p, y, u, w), mul(st.cre(u), st.ann(w)));
        }
      add(e, bx.d(y), false, -1.0, m1);
      add(e, bx.d(y), true, 1.0, m2);
      add(e, bx.d(y), false, 1.0, m3);
    }
  }
  if (!dst_nc) {
    for (int p = nE; p < n; ++p)
      for (int r = p; r < n; ++r) {
        if (p < r) {  // A_pr
          ETerms& e = T[ex.A(p, r)];
          if (p >= nLb) add(e, bx.A(p, r), false, 1.0, eye4());
          else if (r >= nLb) add(e, bx.d(r), true, 1.0, st.cre(p));  // a+_p (site) a+_r (block)
          else add(e, -1, false, 1.0, mul(st.cre(p), st.cre(r)));
        }
        ETerms& e = T[ex.B(p, r)];  // B_pq, q = r
        if (p >= nLb) add(e, bx.B(p, r), false, 1.0, eye4());
        else if (r >= nLb) add(e, bx.d(r), false, 1.0, st.cre(p));  // a+_p (site) a_q (block)
        else add(e, -1, false, 1.0, mul(st.cre(p), st.ann(r)));
      }
    return T;
  }
  for (int p = 0; p < nE; ++p)
    for (int r = p; r < nE; ++r) {
      if (p < r) {  // P_pr
        ETerms& e = T[ex.A(p, r)];
        add(e, nsrc1 + cs->T.at({p, r}), true, 1.0, eye4());
        add(e, -1, false, 1.0, st.P(p, r));
        for (int x = S0; x <= S1; ++x)
          for (int y = nLb; y < n; ++y) add(e, bx.d(y), false, I.vso(p, y, r, x) - I.vso(p, x, r, y), st.ann(x));
      }
      {  // Q_pq
        ETerms& e = T[ex.B(p, r)];
        const int q = r;
        add(e, nsrc1 + cs->U.at({p, q}), false, 1.0, eye4());
        add(e, nsrc1 + cs->V.at({p, q}), true, 1.0, eye4());
        add(e, -1, false, 1.0, st.Q(p, q));
        for (int x = S0; x <= S1; ++x)
          for (int y = nLb; y < n; ++y) {
            add(e, bx.d(y), false, I.vso(p, q, x, y) - I.vso(p, y, x, q), st.cre(x));
            add(e, bx.d(y), true, -(I.vso(p, q, y, x) - I.vso(p, x, y, q)), st.ann(x));
          }
      }
    }
  return T;
}

void carry_jobs(bool forward, const std::vector<PsiBlock>& prev_blocks, const Enlarged& prev_EL,
                const Enlarged& prev_ER, const Enlarged& EL, const Enlarged& ER, const std::vector<PsiBlock>& blocks,
                const BlockBasis& Lb, const BlockBasis& Rb, std::vector<GJob>& j1, std::vector<GJob>& j2,
                long long& phi_size) {
  std::vector<int> blk_of_qL(EL.basis.size(), -1);
  for (size_t b = 0; b < blocks.size(); ++b) blk_of_qL[blocks[b].qL] = (int)b;
  auto site_state = [](QN d) {
    for (int n = 0; n < 4; ++n)
      if (SITE_Q[n] == d) return n;
    return -1;
  };
  const Basis& lb = *Lb.basis;
  const Basis& rb = *Rb.basis;
  const std::vector<long long>& luoff = *Lb.uoff;
  const std::vector<long long>& ruoff = *Rb.uoff;
  const std::vector<int>& lesec = *Lb.esec;
  const std::vector<int>& resec = *Rb.esec;
  j1.clear();
  j2.clear();
  phi_size = 0;
  if (forward) {  // Lb: kept states of the previous left enlarged block; Rb: basis over the new ER
    std::vector<int> kept_of(prev_EL.basis.size(), -1);
    for (size_t s = 0; s < lesec.size(); ++s) kept_of[lesec[s]] = (int)s;
    for (const PsiBlock& pb : prev_blocks) {
      const int s = kept_of[pb.qL];
      if (s < 0) continue;
      const int k = lb.dim[s];
      const long long phi_off = phi_size;
      phi_size += (long long)k * pb.mR;
      j1.push_back({luoff[s], pb.off, phi_off, k, pb.mR, pb.mL, k, pb.mR, pb.mR, 1, 0});  // U^T psi
      const QN qR = prev_ER.basis.q[pb.qR];
      for (int jb = 0; jb < rb.size(); ++jb) {
        const int offc = prev_ER.chunk_off[pb.qR][jb];
        if (offc < 0) continue;
        const int n = site_state(qR - rb.q[jb]);
        if (n < 0) continue;
        const int QLn = EL.basis.find(lb.q[s] + SITE_Q[n]);
        if (QLn < 0) continue;
        const int b = blk_of_qL[QLn];
        if (b < 0 || blocks[b].qR != resec[jb]) continue;
        const PsiBlock& nb = blocks[b];
        const int r0 = EL.chunk_off[QLn][s], kr = rb.dim[jb];
        j2.push_back({phi_off + offc, ruoff[jb], nb.off + (long long)r0 * nb.mR, k, nb.mR, kr, pb.mR, kr, nb.mR,
                      0, 1});  // phi[:, chunk] V^T
      }
    }
  } else {  // Rb: kept states of the previous right enlarged block; Lb: basis over the new EL
    std::vector<int> kept_of(prev_ER.basis.size(), -1);
    for (size_t s = 0; s < resec.size(); ++s) kept_of[resec[s]] = (int)s;
    for (const PsiBlock& pb : prev_blocks) {
      const int s = kept_of[pb.qR];
      if (s < 0) continue;
      const int k = rb.dim[s];
      const long long phi_off = phi_size;
      phi_size += (long long)pb.mL * k;
      j1.push_back({pb.off, ruoff[s], phi_off, pb.mL, k, pb.mR, pb.mR, k, k, 0, 0});  // psi V
      const QN qL = prev_EL.basis.q[pb.qL];
      for (int ja = 0; ja < lb.size(); ++ja) {
        const int offc = prev_EL.chunk_off[pb.qL][ja];
        if (offc < 0) continue;
        const int n = site_state(qL - lb.q[ja]);
        if (n < 0) continue;
        const int QRn = ER.basis.find(rb.q[s] + SITE_Q[n]);
        if (QRn < 0) continue;
        const int b = blk_of_qL[lesec[ja]];
        if (b < 0 || blocks[b].qR != QRn) continue;
        const PsiBlock& nb = blocks[b];
        const int c0 = ER.chunk_off[QRn][s], kl = lb.dim[ja];
        j2.push_back({luoff[ja], phi_off + (long long)offc * k, nb.off + c0, nb.mL, k, kl, kl, k, nb.mR, 0,
                      0});  // U phi[chunk, :]
      }
    }
  }
}

std::vector<int> select_kept(const std::vector<std::vector<double>>& sv, const std::vector<QN>& qL, int M,
                             bool keep_one_per_q, double* discarded) {
  struct Cand {
    double s;
    QN qL;
    int idx, b;
  };
  const int nb = (int)sv.size();
  std::vector<Cand> cand;
  for (int b = 0; b < nb; ++b)
    for (int i = 0; i < (int)sv[b].size(); ++i) cand.push_back({sv[b][i], qL[b], i, b});
  std::stable_sort(cand.begin(), cand.end(), [](const Cand& a, const Cand& b) {
    if (a.s != b.s) return a.s > b.s;
    if (!(a.qL == b.qL)) return a.qL < b.qL;
    return a.idx < b.idx;
  });
  const size_t keep = std::min<size_t>((size_t)std::max(0, M), cand.size());
  std::vector<int> kept(nb, 0);
  double disc = 0.0;
  for (size_t i = 0; i < cand.size(); ++i) {
    if (i < keep) kept[cand[i].b]++;
    else disc += cand[i].s * cand[i].s;
  }
  if (keep_one_per_q)  // every quantum number of psi keeps its largest state
    for (int b = 0; b < nb; ++b)
      if (kept[b] == 0 && !sv[b].empty()) {
        kept[b] = 1;
        disc -= sv[b][0] * sv[b][0];
      }
  if (discarded) *discarded = disc;
  return kept;
}

}  // namespace terms
}  // namespace dmrg
