// Host-side blocking formulas of the sweeps (Appendix A, Eq. blocked-ops;
// App. B, Eqs. h-nc and h-cn): site operators built from the integrals,
// the enlarged basis of block x site, and for every operator of an
// enlarged block its terms (block operator or identity, transposed or not,
// coefficient, site matrix element), which the blocking kernel expands over
// the sectors; the complementary sums of the normal-to-complementary
// transformation at the mixed NC/CN cut. Plain C++, no CUDA.
#pragma once

#include <array>
#include <map>
#include <vector>

#include "model.h"

namespace dmrg {
namespace terms {

inline constexpr QN SITE_Q[4] = {{0, 0}, {1, 1}, {1, -1}, {2, 0}};  // |0>, |a>, |b>, |ab>
inline constexpr int SITE_N[4] = {0, 1, 1, 2};

using Mat4 = std::array<std::array<double, 4>, 4>;

inline Mat4 zero4() {
  Mat4 m{};
  return m;
}
inline Mat4 eye4() {
  Mat4 m{};
  for (int i = 0; i < 4; ++i) m[i][i] = 1.0;
  return m;
}
inline Mat4 mul(const Mat4& a, const Mat4& b) {
  Mat4 c{};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j)
      for (int k = 0; k < 4; ++k) c[i][j] += a[i][k] * b[k][j];
  return c;
}
inline Mat4 tr(const Mat4& a) {
  Mat4 c{};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) c[i][j] = a[j][i];
  return c;
}
inline void axpy(Mat4& y, double c, const Mat4& x) {
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) y[i][j] += c * x[i][j];
}
// a+ of spin sigma on one spatial orbital; local states: bit0 = alpha, bit1 = beta
inline Mat4 site_cre(int sigma) {
  Mat4 m{};
  for (int s = 0; s < 4; ++s)
    if (!((s >> sigma) & 1)) m[s | (1 << sigma)][s] = (sigma == 1 && (s & 1)) ? -1.0 : 1.0;
  return m;
}
inline const Mat4 SC[2] = {site_cre(0), site_cre(1)};
inline const Mat4 SA[2] = {tr(SC[0]), tr(SC[1])};

struct Ints {
  int K = 0;
  std::vector<double> t, v;
  double tso(int p, int q) const { return (p & 1) == (q & 1) ? t[(p / 2) * K + q / 2] : 0.0; }
  double vso(int p, int q, int r, int s) const {
    if ((p & 1) != (q & 1) || (r & 1) != (s & 1)) return 0.0;
    return v[(((size_t)(p / 2) * K + q / 2) * K + r / 2) * K + s / 2];
  }
};

// site operators built from the integrals; x(p) = local a+ / a of mode p of the site
struct Site {
  const Ints& I;
  int s;  // spatial orbital
  int m0() const { return 2 * s; }
  const Mat4& cre(int p) const { return SC[p - 2 * s]; }
  const Mat4& ann(int p) const { return SA[p - 2 * s]; }
  Mat4 R(int p, bool one_body) const {  // [sum t_pq a_q] + sum v_pqrs a+_r a_s a_q over site modes
    Mat4 m = zero4();
    const int a = 2 * s, b = 2 * s + 1;
    if (one_body)
      for (int q = a; q <= b; ++q) axpy(m, I.tso(p, q), ann(q));
    for (int q = a; q <= b; ++q)
      for (int r = a; r <= b; ++r)
        for (int w = a; w <= b; ++w) {
          const double x = I.vso(p, q, r, w);
          if (x != 0.0) axpy(m, x, mul(mul(cre(r), ann(w)), ann(q)));
        }
    return m;
  }
  Mat4 P(int p, int r) const {  // sum v_pqrs a_s a_q
    Mat4 m = zero4();
    for (int q = 2 * s; q <= 2 * s + 1; ++q)
      for (int w = 2 * s; w <= 2 * s + 1; ++w) {
        const double x = I.vso(p, q, r, w);
        if (x != 0.0) axpy(m, x, mul(ann(w), ann(q)));
      }
    return m;
  }
  Mat4 Q(int p, int q) const {  // sum (v_pqrs - v_psrq) a+_r a_s
    Mat4 m = zero4();
    for (int r = 2 * s; r <= 2 * s + 1; ++r)
      for (int w = 2 * s; w <= 2 * s + 1; ++w) {
        const double x = I.vso(p, q, r, w) - I.vso(p, w, r, q);
        if (x != 0.0) axpy(m, x, mul(cre(r), ann(w)));
      }
    return m;
  }
  Mat4 H() const {
    Mat4 m = zero4();
    const int a = 2 * s, b = 2 * s + 1;
    for (int p = a; p <= b; ++p)
      for (int q = a; q <= b; ++q) axpy(m, I.tso(p, q), mul(cre(p), ann(q)));
    for (int p = a; p <= b; ++p)
      for (int q = a; q <= b; ++q)
        for (int r = a; r <= b; ++r)
          for (int w = a; w <= b; ++w) {
            const double x = I.vso(p, q, r, w);
            if (x != 0.0) axpy(m, 0.5 * x, mul(mul(mul(cre(p), cre(r)), ann(w)), ann(q)));
          }
    return m;
  }
};

// One term of an enlarged operator: (block op src, maybe transposed) (x) E_{nout,nin}
struct ETerm {
  int src;  // op index in the block's NC set, -1 = identity
  bool trans;
  double coef;
  int nout, nin;
};
using ETerms = std::vector<ETerm>;

void add(ETerms& e, int src, bool trans, double c, const Mat4& m);

// Enlarged basis: sector Q = q_block + q_site; chunks in ascending block sector.
struct Enlarged {
  Basis basis;
  std::vector<std::vector<int>> chunk_off;  // [Q index][block sector index] -> offset in Q, or -1
};
Enlarged enlarge(const Basis& b);

// Left: block L holds modes [0, 2s); site s; enlarged NC set nL' = 2s + 2.
std::vector<ETerms> left_terms(const Ints& I, int s);
// Right: block R holds modes [2s+2, n) (complementary indices p < 2s+2);
// site s; enlarged NC set (right kind) nL' = 2s. Terms read site (x) block.
std::vector<ETerms> right_terms(const Ints& I, int s);
// ------------------------------------------- CN form and the transformation
// Complementary sums of one block whose two-index operators are normal (an
// NC left block, or a CN right block), for the pairs (p, r) of `out` modes:
//   T_pr = sum_{q<s} (v_pqrs - v_psrq) A_qs          (P~_pr = T_pr^T)
//   U_pq = sum_{r<=s} c_pq,rs B_rs,  V_pq = sum_{r<s} c_pq,sr B_rs
//   (Q~_pq = U_pq + V_pq^T,  c_pq,rs = v_pqrs - v_psrq)
// with q, r, s over the block's modes: P~_pr = sum_{q,s} v_pqrs a_s a_q and
// Q~_pq = sum_{r,s} c_pq,rs a+_r a_s written with the stored A_qs = a+_q a+_s
// (q < s) and B_rs = a+_r a_s (r <= s). Every output is a linear combination
// of source operators of one shift, so the sums are one GEMM per shift class
// (launch_opcomb); the comp ops are stored class by class.
struct CompSet {
  std::map<std::pair<int, int>, int> T, U, V;  // output pair -> comp op index
  OpSet set;                                   // over the block's basis
  std::vector<CombClass> cls;
  std::vector<long long> xoff;
  std::vector<double> coef;
  int ntiles = 0;
  double flops = 0.0;
};


void make_comp(const Ints& I, const NCIndex& bx, const OpSet& bset, int o0, int o1, CompSet& cs);
// Left: block L holds modes [0, 2s) (NC form when src_nc, else CN form); the
// enlarged block (modes [0, 2s+2)) is in CN form. Comp ops (src_nc) are
// source indices nsrc1 + comp index.
std::vector<ETerms> left_terms_cn(const Ints& I, int s, bool src_nc, const CompSet* cs, int nsrc1);
// Right: block R holds modes [2s+2, n) in CN form; the enlarged block (modes
// [2s, n)) is in NC form when dst_nc (the transformation), else in CN form.
std::vector<ETerms> right_terms_cn(const Ints& I, int s, bool dst_nc, const CompSet* cs, int nsrc1);

// Kept states of a block over the enlarged basis it was made from: sector s
// of `basis` is enlarged sector esec[s], its d x k basis matrix (row-major,
// columns = states) at element uoff[s] of the block's basis store.
struct BlockBasis {
  const Basis* basis;
  const std::vector<long long>* uoff;
  const std::vector<int>* esec;
};
// The two GEMM passes that carry the previous step's psi (blocks
// prev_blocks over prev_EL x prev_ER) to the next bond (blocks over EL x ER).
// Moving right (forward): Lb holds the kept states of prev_EL, Rb the basis
// of the block the sweep enters over ER; pass 1 phi = U^T psi per block,
// pass 2 psi'[(l, n), :] = phi[l, (n, r)] V^T per chunk. Moving left: Rb
// holds the kept states of prev_ER, Lb the basis over EL; phi = psi V, then
// psi'[:, (n, r)] = U phi[(l, n), r]. Pass 1 reads (basis store, psi) or
// (psi, basis store) and writes phi (phi_size elements); pass 2 reads
// (phi, basis store) or (basis store, phi) and writes psi'; every element of
// psi' is written by at most one job.
void carry_jobs(bool forward, const std::vector<PsiBlock>& prev_blocks, const Enlarged& prev_EL,
                const Enlarged& prev_ER, const Enlarged& EL, const Enlarged& ER, const std::vector<PsiBlock>& blocks,
                const BlockBasis& Lb, const BlockBasis& Rb, std::vector<GJob>& j1, std::vector<GJob>& j2,
                long long& phi_size);

// Global truncation (Appendix A, decimation): the singular values of all psi
// blocks (sv[b] in descending order, min(mL, mR) of them; qL[b] the block's
// left quantum number) sorted by (value descending, q_L ascending, index
// ascending), the first min(M, count) kept, zero values included; with
// keep_one_per_q a block none of whose values made the cut keeps its
// largest (Sec. III keeps a state per quantum number). Returns the kept
// count per block; *discarded = sum of the squares not kept.
std::vector<int> select_kept(const std::vector<std::vector<double>>& sv, const std::vector<QN>& qL, int M,
                             bool keep_one_per_q, double* discarded);

}  // namespace terms
}  // namespace dmrg
