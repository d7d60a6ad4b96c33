// Two-site DMRG sweeps on the device (Appendix A): blocking (Eq.
// blocked-ops), solving (Eq. eff-eigsh, device Davidson over the NC or CN
// sigma, started from the previous step's wavefunction), decimation
// (one-sided Jacobi SVD of every psi block, global truncation) and
// transformation (Eq. op-trans). The host decides which blocks to add and
// which states to keep; every floating-point step runs in CUDA kernels.
//
// Operators of a block are a set in canonical order (model.h NCIndex). NC
// form: a left block holding modes [0, nL) keeps H, a+_p (p < nL), R^L_p
// (p >= nL), A_pr and B_pq (p, q, r < nL); a right block holding modes
// [nL, n) keeps H, a_p (p >= nL), R^R_p, P_pr, Q_pq (p, q, r < nL). CN form
// (App. B, Eq. h-cn) moves the two-index pairs to the modes right of the
// cut: P^L_pr, Q^L_pq on a left block, A_pr, B_pq on a right block. With the
// mixed NC/CN scheme (Sec. III.A) blocks left of the cut are in NC form and
// blocks right of it in CN form; the block that crosses the cut is built by
// the normal-to-complementary transformation. The enlarged blocks L x site
// and site x R of one bond share a form, so the sigma work list (NC or CN
// terms) applies to them directly.
//
// Blocking: each enlarged operator is a sum of terms (block operator or 1)
// (x) (4x4 site matrix) derived by splitting every second-quantized string
// into its block part and its site part (the formulas are in terms.cpp).
// Every nonzero site-matrix element of a term becomes a scaled copy of one
// block-operator block into one chunk of one enlarged block; a kernel
// applies the copies of each destination block in a fixed order.
#include <algorithm>
#include <chrono>
#include <array>
#include <cmath>
#include <cstring>
#include <numeric>

#include "context.h"
#include "terms.h"

namespace dmrg {

namespace {

using namespace terms;

constexpr uint64_t KEY_MPS = 0x4D50535F494E4954ull;    // "MPS_INIT"
constexpr uint64_t KEY_NOISE = 0x4E4F495345505349ull;  // "NOISEPSI"
bool can_hold(int n_modes, QN q) {
  return q.n >= 0 && q.n <= n_modes && ((q.s - q.n) % 2 == 0) && std::abs(q.s) <= std::min(q.n, n_modes - q.n);
}

}  // namespace

// ------------------------------------------------------------------ state
struct DevBlock {
  OpSet set;
  int nL = 0;
  bool left = true;
  bool cn = false;  // CN form (two-index pairs over the modes right of the cut)
  DevBuf store;
  // the block's states over the enlarged basis it was made from: sector s is
  // enlarged sector esec[s], basis u + uoff[s] (d x k row-major, columns = states)
  DevBuf u;
  std::vector<long long> uoff;
  std::vector<int> esec;
};

struct SweepState {
  Ints I;
  QN Q;
  int K = 0;
  std::vector<std::unique_ptr<DevBlock>> L, R;  // L[i]: modes [0, 2i); R[j]: modes [2j, 2K)
  int prob_site = -1;
  int cut = 0;            // mixed NC/CN cut (orbitals); K = NC everywhere
  bool prob_cn = false;   // partition of the current problem
  Enlarged EL, ER;
  // previous step of the sweep (wavefunction prediction)
  bool has_prev = false;
  int prev_site = -1;
  bool prev_fwd = true;
  long long prev_size = 0;
  DevBuf prev_x;
  std::vector<PsiBlock> prev_blocks;
  Enlarged prev_EL, prev_ER;
  std::vector<dmrg_step_log> log;
};

void sweep_block_info(const Context& c, int side, int j, int* n_sectors, int* q, int* dims, int* n_ops) {
  if (!c.sweep) throw Error(DMRG_ESTATE, "call dmrg_build_blocks first");
  const SweepState& S = *c.sweep;
  if (side != 0 && side != 1) throw Error(DMRG_EINVAL, "side must be 0 (left) or 1 (right)");
  if (j < 0 || j > S.K) throw Error(DMRG_EINVAL, "block index out of range (0 .. K)");
  const auto& blk = side == 0 ? S.L[j] : S.R[j];
  if (!blk) throw Error(DMRG_ESTATE, "this block is not built");
  const Basis& b = blk->set.basis;
  *n_sectors = b.size();
  for (int i = 0; i < b.size(); ++i) {
    if (q) {
      q[2 * i] = b.q[i].n;
      q[2 * i + 1] = b.q[i].s;
    }
    if (dims) dims[i] = b.dim[i];
  }
  if (n_ops) *n_ops = (int)blk->set.ops.size();
}

void sweep_block_read(Context& c, int side, int j, int op, double* dense) {
  int ns = 0, nops = 0;
  sweep_block_info(c, side, j, &ns, nullptr, nullptr, &nops);
  if (op < 0 || op >= nops) throw Error(DMRG_EINVAL, "operator index out of range");
  const DevBlock& B = side == 0 ? *c.sweep->L[j] : *c.sweep->R[j];
  const Basis& b = B.set.basis;
  const long long tot = b.total;
  std::fill(dense, dense + tot * tot, 0.0);
  std::vector<double> tmp;
  for (const OpBlock& ob : B.set.ops[op].blocks) {
    tmp.resize((size_t)ob.rows * ob.cols);
    if (tmp.empty()) continue;
    DMRG_CUDA(cudaMemcpyAsync(tmp.data(), B.store.as<double>() + ob.off, tmp.size() * sizeof(double),
                              cudaMemcpyDeviceToHost, c.stream));
    DMRG_CUDA(cudaStreamSynchronize(c.stream));
    const long long r0 = b.off[ob.qout], c0 = b.off[ob.qin];
    for (int r = 0; r < ob.rows; ++r)
      for (int k = 0; k < ob.cols; ++k) dense[(r0 + r) * tot + c0 + k] = tmp[(size_t)r * ob.cols + k];
  }
}

const std::vector<dmrg_step_log>& sweep_log(const Context& c) {
  static const std::vector<dmrg_step_log> none;
  return c.sweep ? c.sweep->log : none;
}

namespace {

std::unique_ptr<DevBlock> vacuum(const Ints& I, bool left, cudaStream_t st, bool cn = false) {
  auto b = std::make_unique<DevBlock>();
  Basis v;
  v.q.push_back({0, 0});
  v.dim.push_back(1);
  v.finish();
  b->left = left;
  b->nL = left ? 0 : 2 * I.K;
  b->cn = cn;
  build_nc_opset(b->set, v, b->nL, 2 * I.K, left, 0, cn);
  b->store.alloc(std::max<long long>(1, b->set.elements) * sizeof(double));
  DMRG_CUDA(cudaMemsetAsync(b->store.p, 0, std::max<long long>(1, b->set.elements) * sizeof(double), st));
  return b;
}

// Enlarged operators of one side into `store` (NC form, or CN form when
// e_cn): the host lists each enlarged operator's terms (block op or
// identity, transposed or not, coefficient, site matrix element); the
// blocking kernel expands them over the sectors. When the block and the
// enlarged block differ in form (the normal-to-complementary transformation
// at the mixed NC/CN cut), the block's complementary sums are first formed
// by one GEMM per shift class and serve as further source operators.
void build_enlarged(Context& c, const Ints& I, const DevBlock& B, int site, bool left, const Enlarged& E,
                    OpSet& EO, double* store, bool e_cn) {
  const int n = 2 * I.K;
  const bool transform_step = B.cn != e_cn;
  if (transform_step && (left ? B.cn : !B.cn)) throw Error(DMRG_EINVAL, "internal: blocks change form only at the cut");
  CompSet cs;
  DevBuf d_comp, d_cls, d_xoff, d_coef;
  const int nsrc1 = (int)B.set.ops.size();
  cudaStream_t st = c.stream;
  if (transform_step) {
    const NCIndex bx = left ? NCIndex{2 * site, n, false} : NCIndex{2 * site + 2, n, true};
    if (left) make_comp(I, bx, B.set, 2 * site + 2, n, cs);
    else make_comp(I, bx, B.set, 0, 2 * site, cs);
    d_comp.alloc(std::max<long long>(1, cs.set.elements) * sizeof(double));
    d_cls.upload(cs.cls, st);
    d_xoff.upload(cs.xoff, st);
    d_coef.upload(cs.coef, st);
    ProfScope ps(c.prof, 3, st);
    launch_opcomb(B.store.as<double>(), d_xoff.as<long long>(), d_coef.as<double>(), d_cls.as<CombClass>(),
                  (int)cs.cls.size(), cs.ntiles, d_comp.as<double>(), st);
    DMRG_CUDA(cudaGetLastError());
  }
  std::vector<ETerms> terms;
  if (left) terms = e_cn ? left_terms_cn(I, site, !B.cn, &cs, nsrc1) : left_terms(I, site);
  else terms = B.cn ? right_terms_cn(I, site, !e_cn, &cs, nsrc1) : right_terms(I, site);
  std::vector<int> term_start(EO.ops.size() + 1, 0);
  std::vector<BTerm> flat;
  size_t total = 0;
  for (const ETerms& t : terms) total += t.size();
  flat.reserve(total);
  for (size_t k = 0; k < EO.ops.size(); ++k) {
    for (const ETerm& e : terms[k]) flat.push_back({e.src, e.trans ? 1 : 0, e.nout, e.nin, e.coef});
    term_start[k + 1] = (int)flat.size();
  }
  const Basis& bb = B.set.basis;
  const int nb = bb.size(), ne = E.basis.size();
  std::vector<int> bq(2 * nb), eq(2 * ne), chunk((size_t)ne * nb, -1);
  for (int i = 0; i < nb; ++i) {
    bq[2 * i] = bb.q[i].n;
    bq[2 * i + 1] = bb.q[i].s;
  }
  for (int i = 0; i < ne; ++i) {
    eq[2 * i] = E.basis.q[i].n;
    eq[2 * i + 1] = E.basis.q[i].s;
    for (int j = 0; j < nb; ++j) chunk[(size_t)i * nb + j] = E.chunk_off[i][j];
  }
  const size_t nsrc = B.set.ops.size() + cs.set.ops.size();
  std::vector<long long> srcblk(std::max<size_t>(1, nsrc * nb), -1);
  std::vector<int> src_dq(std::max<size_t>(2, 2 * nsrc)), src_par(std::max<size_t>(1, nsrc));
  for (size_t j = 0; j < nsrc; ++j) {
    const OpDesc& o = j < (size_t)nsrc1 ? B.set.ops[j] : cs.set.ops[j - nsrc1];
    for (const OpBlock& ob : o.blocks) srcblk[j * nb + ob.qin] = ob.off;
    src_dq[2 * j] = o.dq.n;
    src_dq[2 * j + 1] = o.dq.s;
    src_par[j] = o.parity;
  }
  std::vector<BDst> dsts;
  for (size_t k = 0; k < EO.ops.size(); ++k)
    for (const OpBlock& ob : EO.ops[k].blocks)
      dsts.push_back({ob.off, (int)k, ob.qin, ob.qout, ob.rows, ob.cols, 0});
  DevBuf d_ts, d_terms, d_bq, d_bdim, d_eq, d_chunk, d_srcblk, d_dq, d_par, d_dsts, d_err;
  d_ts.upload(term_start, st);
  d_terms.upload(flat, st);
  d_bq.upload(bq, st);
  d_bdim.upload(bb.dim, st);
  d_eq.upload(eq, st);
  d_chunk.upload(chunk, st);
  d_srcblk.upload(srcblk, st);
  d_dq.upload(src_dq, st);
  d_par.upload(src_par, st);
  d_dsts.upload(dsts, st);
  d_err.alloc(sizeof(int));
  DMRG_CUDA(cudaMemsetAsync(d_err.p, 0, sizeof(int), st));
  BlockingDev d;
  d.dst_store = store;
  d.src_store = B.store.as<double>();
  d.src_store2 = d_comp.as<double>();
  d.nsrc1 = nsrc1;
  d.dsts = d_dsts.as<BDst>();
  d.ndst = (int)dsts.size();
  d.term_start = d_ts.as<int>();
  d.terms = d_terms.as<BTerm>();
  d.bq = d_bq.as<int>();
  d.bdim = d_bdim.as<int>();
  d.nb = nb;
  d.eq = d_eq.as<int>();
  d.chunk_off = d_chunk.as<int>();
  d.srcblk = d_srcblk.as<long long>();
  d.src_dq = d_dq.as<int>();
  d.src_par = d_par.as<int>();
  d.left = left ? 1 : 0;
  d.err = d_err.as<int>();
  {
    ProfScope ps(c.prof, 3, st);
    launch_blocking(d, st);
  }
  DMRG_CUDA(cudaGetLastError());
  int herr = 0;
  DMRG_CUDA(cudaMemcpyAsync(&herr, d_err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  DMRG_CUDA(cudaStreamSynchronize(st));  // tables are freed on return
  if (herr) throw Error(DMRG_EINVAL, "internal: blocking term shifts a sector inconsistently");
}

// Transformation O_new[Q' <- Q] = U_Q'^T O[Q' <- Q] U_Q of every operator of
// the enlarged set EO (values at `enl_store`) onto the kept basis `nb`
// (U blocks per enlarged sector in `u_store`, d x k row-major, offsets uoff).
void transform(Context& c, const OpSet& EO, const double* enl_store, const Basis& nb,
               const std::vector<int>& esec_of_new, const std::vector<long long>& uoff, const double* u_store,
               DevBlock& out, int nL, int n, bool left, bool cn) {
  build_nc_opset(out.set, nb, nL, n, left, 0, cn);
  out.nL = nL;
  out.left = left;
  out.cn = cn;
  out.store.alloc(std::max<long long>(1, out.set.elements) * sizeof(double));
  if ((int)out.set.ops.size() != (int)EO.ops.size()) throw Error(DMRG_EINVAL, "internal: transform op count");
  std::vector<PsiBlock> blocks;
  std::vector<std::pair<int, int>> in_ref;  // (op, enlarged block) per output block
  WorkList wl;
  std::vector<Task> tasks;
  for (size_t k = 0; k < out.set.ops.size(); ++k)
    for (const OpBlock& ob : out.set.ops[k].blocks) {
      const int eq_in = esec_of_new[ob.qin], eq_out = esec_of_new[ob.qout];
      const int kb = EO.ops[k].by_qin[eq_in];
      if (kb < 0 || EO.ops[k].blocks[kb].qout != eq_out) throw Error(DMRG_EINVAL, "internal: transform block");
      blocks.push_back({0, 0, ob.rows, ob.cols, ob.off});
      in_ref.push_back({(int)k, kb});
    }
  const int nout = (int)blocks.size();
  wl.out_start.assign(nout + 1, 0);
  {
    // one task per output block: rows side U_Q'^T, columns side U_Q^T (both
    // stored d x k row-major, used transposed), input = the enlarged block
    int b = 0;
    for (size_t k = 0; k < out.set.ops.size(); ++k)
      for (const OpBlock& ob : out.set.ops[k].blocks) {
        const OpBlock& eb = EO.ops[in_ref[b].first].blocks[in_ref[b].second];
        Task t;
        t.aoff = uoff[ob.qout];
        t.boff = uoff[ob.qin];
        t.in_blk = (int)blocks.size();
        t.flags = 3;
        t.scale = 1.0;
        blocks.push_back({0, 0, eb.rows, eb.cols, eb.off});
        tasks.push_back(t);
        wl.out_start[b + 1] = b + 1;
        ++b;
      }
  }
  wl.tasks = tasks;
  build_items(blocks, wl, TileShape{F64_TM, F64_TN, 2e6}, c.n_sm * 8, nout);
  DevBuf d_tasks, d_items, d_groups, d_sched, d_blocks, d_scratch, d_counter;
  cudaStream_t st = c.stream;
  d_tasks.upload(wl.tasks, st);
  d_items.upload(wl.items, st);
  d_groups.upload(wl.groups, st);
  d_sched.upload(wl.schedule, st);
  d_blocks.upload(blocks, st);
  d_scratch.alloc(std::max<long long>(1, wl.scratch_elems) * sizeof(double));
  d_counter.alloc(16);
  DMRG_CUDA(cudaMemsetAsync(d_counter.p, 0, sizeof(unsigned int), st));
  SigmaDev a;
  a.store = u_store;
  a.psi = enl_store;
  a.sigma = out.store.as<double>();
  a.tasks = d_tasks.as<Task>();
  a.items = d_items.as<Item>();
  a.schedule = d_sched.as<int>();
  a.n_items = (int)wl.items.size();
  a.groups = d_groups.as<Group>();
  a.n_groups = (int)wl.groups.size();
  a.blocks = d_blocks.as<PsiBlock>();
  a.scratch = d_scratch.as<double>();
  a.counter = d_counter.as<unsigned int>();
  if (a.n_items > 0) {
    ProfScope ps(c.prof, 3, st);
    launch_sigma_f64(a, c.n_sm, st);
    launch_reduce(a, st);
  }
  DMRG_CUDA(cudaGetLastError());
  DMRG_CUDA(cudaStreamSynchronize(st));
}

}  // namespace

// Build (if needed) the two-site problem at bond `site`: enlarged blocks
// L[site] x s_site and s_{site+1} x R[site+2], NC terms, sigma work list.
bool sweep_problem_ready(const Context& c, int site) {
  return c.sweep && c.prob && c.sweep->prob_site == site;
}

void sweep_problem(Context& c, int site) {
  SweepState& S = *c.sweep;
  if (site < 0 || site > S.K - 2) throw Error(DMRG_EINVAL, "site out of range (0 .. K-2)");
  if (S.prob_site == site && c.prob) return;
  if (!S.L[site] || !S.R[site + 2]) throw Error(DMRG_ESTATE, "blocks for this bond are not built");
  const DevBlock& Lb = *S.L[site];
  const DevBlock& Rb = *S.R[site + 2];
  auto p = std::make_unique<Problem>();
  p->nL = 2 * (site + 1);
  p->n = 2 * S.K;
  p->Q = S.Q;
  S.EL = enlarge(Lb.set.basis);
  S.ER = enlarge(Rb.set.basis);
  const bool cn = site + 1 > S.cut;  // mixed NC/CN: partition of this bond
  build_nc_opset(p->L, S.EL.basis, p->nL, p->n, true, 0, cn);
  build_nc_opset(p->R, S.ER.basis, p->nL, p->n, false, p->L.elements, cn);
  p->terms = cn ? cn_terms(p->nL, p->n) : nc_terms(p->nL, p->n);
  p->cn = cn;
  p->blocks = psi_layout(S.EL.basis, S.ER.basis, p->Q, &p->psi_size);
  if (p->blocks.empty()) throw Error(DMRG_EINVAL, "no psi block at this bond");
  const long long elems = p->L.elements + p->R.elements;
  c.prob.reset();
  p->store.alloc(std::max<long long>(1, elems) * sizeof(double));
  build_enlarged(c, S.I, Lb, site, true, S.EL, p->L, p->store.as<double>(), cn);
  build_enlarged(c, S.I, Rb, site + 1, false, S.ER, p->R, p->store.as<double>(), cn);
  prepare_worklist(c, *p);
  c.prob = std::move(p);
  S.prob_site = site;
  S.prob_cn = cn;
}

namespace {

struct Decim {
  Basis nb;                      // kept sectors (of the growing side's enlarged basis)
  std::vector<int> esec_of_new;  // new sector -> enlarged sector index
  std::vector<long long> uoff;   // new sector -> offset of its U block
  DevBuf u;                      // U blocks (d x k row-major)
  double discarded = 0.0;
};

// Decimation of psi (device, problem layout) keeping at most M states
// (Appendix A step iii): singular vectors and values of every psi block by
// one-sided Jacobi on the device, global sort by (s desc, q_L asc, index
// asc), kept count min(M, sum min(mL, mR)) (plus one state per quantum
// number with keep_one_per_q).
void decimate(Context& c, Problem& p, const Enlarged& E, const double* psi, int M, bool forward, Decim& D) {
  cudaStream_t st = c.stream;
  const int nb = (int)p.blocks.size();
  std::vector<GramBlock> gb(nb);   // Q / w offsets and the two dimensions of every block
  std::vector<SvdBlock> sb(nb);
  long long goff = 0, woff = 0, aoff = 64;
  int pairs = 0, max_rounds = 0, max_d = 1;
  for (int b = 0; b < nb; ++b) {
    const PsiBlock& pb = p.blocks[b];
    const int d = forward ? pb.mL : pb.mR, m = forward ? pb.mR : pb.mL;
    gb[b] = {pb.off, goff, woff, d, m};
    const int dp = d + (d & 1);
    sb[b] = {pb.off, goff, woff, aoff, aoff + (long long)d * m, d, m, pairs, dp / 2, dp - 1, 0};
    pairs += dp / 2;
    max_rounds = std::max(max_rounds, dp - 1);
    max_d = std::max(max_d, d);
    aoff += (long long)d * m + (long long)d * d;
    goff += (long long)d * d;
    woff += d;
  }
  DevBuf dsb, Q, W, work;
  dsb.upload(sb, st);
  Q.alloc(std::max<long long>(1, goff) * sizeof(double));
  W.alloc(std::max<long long>(1, woff) * sizeof(double));
  work.alloc((size_t)aoff * sizeof(double));
  {
    ProfScope ps(c.prof, 3, st);
    launch_svd_blocks(psi, dsb.as<SvdBlock>(), nb, pairs, max_rounds, max_d, Q.as<double>(), W.as<double>(),
                      work.as<double>(), forward, c.n_sm, st);
  }
  DMRG_CUDA(cudaGetLastError());
  std::vector<double> w(woff);
  DMRG_CUDA(cudaMemcpyAsync(w.data(), W.p, woff * sizeof(double), cudaMemcpyDeviceToHost, st));
  DMRG_CUDA(cudaStreamSynchronize(st));
  std::vector<std::vector<double>> sv(nb);  // singular values per block, descending
  std::vector<QN> qLs(nb);
  for (int b = 0; b < nb; ++b) {
    const PsiBlock& pb = p.blocks[b];
    const int r = std::min(pb.mL, pb.mR);
    for (int i = 0; i < r; ++i) sv[b].push_back(std::sqrt(std::max(0.0, w[gb[b].w_off + i])));
    qLs[b] = p.L.basis.q[pb.qL];
  }
  const std::vector<int> kept = select_kept(sv, qLs, M, c.opts.keep_one_per_q != 0, &D.discarded);
  // new basis: sectors of the growing side in ascending order
  std::vector<std::pair<QN, int>> secs;  // (q, block)
  for (int b = 0; b < nb; ++b)
    if (kept[b] > 0) secs.push_back({forward ? p.L.basis.q[p.blocks[b].qL] : p.R.basis.q[p.blocks[b].qR], b});
  std::sort(secs.begin(), secs.end(), [](const std::pair<QN, int>& a, const std::pair<QN, int>& b) {
    return a.first < b.first;
  });
  D.nb = Basis();
  D.esec_of_new.clear();
  D.uoff.clear();
  std::vector<TakeBlock> tb;
  long long uo = 0;
  for (auto& sb : secs) {
    const int b = sb.second;
    D.nb.q.push_back(sb.first);
    D.nb.dim.push_back(kept[b]);
    D.esec_of_new.push_back(forward ? p.blocks[b].qL : p.blocks[b].qR);
    D.uoff.push_back(uo);
    tb.push_back({gb[b].g_off, uo, gb[b].d, kept[b]});
    uo += (long long)gb[b].d * kept[b];
  }
  D.nb.finish();
  (void)E;
  D.u.alloc(std::max<long long>(1, uo) * sizeof(double));
  DevBuf dtb;
  dtb.upload(tb, st);
  launch_take_columns(Q.as<double>(), dtb.as<TakeBlock>(), (int)tb.size(), D.u.as<double>(), st);
  DMRG_CUDA(cudaGetLastError());
  DMRG_CUDA(cudaStreamSynchronize(st));
}

// Davidson guess for the step at bond i: the previous step's psi carried to
// this bond, into g (p.psi_size doubles). Moving right (previous step at
// bond i-1), psi over (L_{i-1} x s_{i-1}) x (s_i x R_{i+1}) is projected on
// the kept states of L_i (phi = U^T psi), which leaves (L_i x s_i) x R_{i+1}
// with no fermion sign (the product state is c_l c_n c_r |0> in either
// grouping), and every state of R_{i+1} is expanded in s_{i+1} x R_{i+2}
// through its stored basis V: psi'[(l, n), :] = phi[l, (n, r)] V^T. Moving
// left is the mirror image (phi = psi V, psi'[:, (n, r)] = U phi[(l, n), r]
// with the stored basis U of L_{i+1}). At the turn of a sweep the bond and
// its blocks are unchanged and the previous psi is the guess. Returns false
// (random guess) without a usable previous step or if the carried vector
// vanishes.
bool predict_guess(Context& c, int i, bool forward, const Problem& p, double* g) {
  SweepState& S = *c.sweep;
  if (!S.has_prev) return false;
  cudaStream_t st = c.stream;
  if (S.prev_site == i) {
    if (S.prev_size != p.psi_size) return false;
    DMRG_CUDA(cudaMemcpyAsync(g, S.prev_x.as<double>(), p.psi_size * sizeof(double), cudaMemcpyDeviceToDevice, st));
    return true;
  }
  const bool fw = forward && S.prev_fwd && S.prev_site == i - 1;
  const bool bw = !forward && !S.prev_fwd && S.prev_site == i + 1;
  if (!fw && !bw) return false;
  std::vector<GJob> j1, j2;
  long long phi_size = 0;
  const DevBlock& Lb = fw ? *S.L[i] : *S.L[i + 1];
  const DevBlock& Rb = fw ? *S.R[i + 1] : *S.R[i + 2];
  carry_jobs(fw, S.prev_blocks, S.prev_EL, S.prev_ER, S.EL, S.ER, p.blocks, {&Lb.set.basis, &Lb.uoff, &Lb.esec},
             {&Rb.set.basis, &Rb.uoff, &Rb.esec}, j1, j2, phi_size);
  if (j2.empty()) return false;
  DevBuf phi, d1, d2;
  phi.alloc(std::max<long long>(1, phi_size) * sizeof(double));
  d1.upload(j1, st);
  d2.upload(j2, st);
  DMRG_CUDA(cudaMemsetAsync(g, 0, p.psi_size * sizeof(double), st));
  if (fw) {
    launch_bgemm(Lb.u.as<double>(), S.prev_x.as<double>(), phi.as<double>(), d1.as<GJob>(), (int)j1.size(), st);
    launch_bgemm(phi.as<double>(), Rb.u.as<double>(), g, d2.as<GJob>(), (int)j2.size(), st);
  } else {
    launch_bgemm(S.prev_x.as<double>(), Rb.u.as<double>(), phi.as<double>(), d1.as<GJob>(), (int)j1.size(), st);
    launch_bgemm(Lb.u.as<double>(), phi.as<double>(), g, d2.as<GJob>(), (int)j2.size(), st);
  }
  DMRG_CUDA(cudaGetLastError());
  // |g|^2 (the oracle falls back to a random guess below norm 1e-12)
  double* sc = p.dav_s.as<double>() + 60;  // scratch scalar of the Davidson workspace
  dav_dots(g, p.psi_size, 1, g, p.psi_size, p.dav_partial.as<double>(), sc, 1, st);
  double nrm2 = 0.0;
  DMRG_CUDA(cudaMemcpyAsync(&nrm2, sc, sizeof(double), cudaMemcpyDeviceToHost, st));
  DMRG_CUDA(cudaStreamSynchronize(st));
  return std::sqrt(nrm2) > 1e-12;
}

}  // namespace

void sweep_build_blocks(Context& c, const double* t, const double* v, int K, int N, int two_sz, int M_init) {
  if (K < 2 || K > 256) throw Error(DMRG_EINVAL, "K must be in [2, 256]");
  if (M_init < 1) throw Error(DMRG_EINVAL, "M_init must be >= 1");
  if (!can_hold(2 * K, {N, two_sz})) throw Error(DMRG_EINVAL, "N, 2Sz not reachable with K orbitals");
  auto S = std::make_unique<SweepState>();
  S->K = K;
  S->Q = {N, two_sz};
  S->I.K = K;
  S->I.t.assign(t, t + (size_t)K * K);
  S->I.v.assign(v, v + (size_t)K * K * K * K);
  for (double x : S->I.t)
    if (!std::isfinite(x)) throw Error(DMRG_EINVAL, "non-finite one-electron integral");
  for (double x : S->I.v)
    if (!std::isfinite(x)) throw Error(DMRG_EINVAL, "non-finite two-electron integral");
  c.prob.reset();
  cudaStream_t st = c.stream;
  S->cut = c.opts.mixed_cut < 0 ? K : std::min(c.opts.mixed_cut, K);
  S->L.resize(K + 1);
  S->R.resize(K + 1);
  S->R[K] = vacuum(S->I, false, st, K > S->cut);
  S->L[0] = vacuum(S->I, true, st);
  const uint64_t key = c.opts.seed ^ KEY_MPS;
  unsigned long long counter = 0;
  for (int j = K - 1; j >= 1; --j) {
    const DevBlock& Rb = *S->R[j + 1];
    Enlarged E = enlarge(Rb.set.basis);
    OpSet EO;
    const bool cn = j > S->cut;  // right block starting at orbital j
    build_nc_opset(EO, E.basis, 2 * j, 2 * K, false, 0, cn);
    DevBuf est;
    est.alloc(std::max<long long>(1, EO.elements) * sizeof(double));
    build_enlarged(c, S->I, Rb, j, false, E, EO, est.as<double>(), cn);
    // kept sectors: those the left part (2j modes) can complement to the target
    std::vector<int> comp;
    long long D = 0;
    for (int i = 0; i < E.basis.size(); ++i)
      if (can_hold(2 * j, S->Q - E.basis.q[i])) {
        comp.push_back(i);
        D += E.basis.dim[i];
      }
    std::vector<int> m(comp.size());
    if (D <= M_init) {
      for (size_t a = 0; a < comp.size(); ++a) m[a] = E.basis.dim[comp[a]];
    } else {
      std::vector<double> exact(comp.size());
      std::vector<long long> base(comp.size());
      long long sum = 0;
      for (size_t a = 0; a < comp.size(); ++a) {
        exact[a] = (double)M_init * (double)E.basis.dim[comp[a]] / (double)D;
        base[a] = (long long)std::floor(exact[a]);
        sum += base[a];
      }
      std::vector<int> order(comp.size());
      std::iota(order.begin(), order.end(), 0);
      std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const double rx = exact[x] - (double)base[x], ry = exact[y] - (double)base[y];
        if (rx != ry) return rx > ry;
        return x < y;
      });
      for (long long a = 0; a < M_init - sum; ++a) base[order[a]] += 1;
      for (size_t a = 0; a < comp.size(); ++a) m[a] = (int)base[a];
    }
    // random bases: counter-based normals, orthonormalised per sector
    Decim Dm;
    std::vector<GramBlock> gb;
    long long uo = 0;
    for (size_t a = 0; a < comp.size(); ++a) {
      if (m[a] <= 0) continue;
      const int d = E.basis.dim[comp[a]];
      if (m[a] > 1024) throw Error(DMRG_EINVAL, "sector dimension above 1024 in the initial MPS");
      Dm.nb.q.push_back(E.basis.q[comp[a]]);
      Dm.nb.dim.push_back(m[a]);
      Dm.esec_of_new.push_back(comp[a]);
      Dm.uoff.push_back(uo);
      gb.push_back({0, uo, 0, d, m[a]});
      uo += (long long)d * m[a];
    }
    Dm.nb.finish();
    Dm.u.alloc(std::max<long long>(1, uo) * sizeof(double));
    launch_gen_vector(Dm.u.as<double>(), uo, key, counter, st);
    counter += (unsigned long long)uo;
    DevBuf dgb;
    dgb.upload(gb, st);
    {
      ProfScope ps(c.prof, 3, st);
      launch_orthonormalize(Dm.u.as<double>(), dgb.as<GramBlock>(), (int)gb.size(), st);
    }
    DMRG_CUDA(cudaGetLastError());
    auto nbk = std::make_unique<DevBlock>();
    transform(c, EO, est.as<double>(), Dm.nb, Dm.esec_of_new, Dm.uoff, Dm.u.as<double>(), *nbk, 2 * j, 2 * K, false,
              cn);
    nbk->u.take(Dm.u);
    nbk->uoff = Dm.uoff;
    nbk->esec = Dm.esec_of_new;
    S->R[j] = std::move(nbk);
  }
  c.sweep = std::move(S);
}

void sweep_run(Context& c, const int* Ms, int n_sweeps, double tol, double* energies, double* max_discard) {
  if (!c.sweep) throw Error(DMRG_ESTATE, "call dmrg_build_blocks first");
  SweepState& S = *c.sweep;
  const int K = S.K;
  S.log.clear();
  for (int s = 0; s < n_sweeps; ++s) {
    if (Ms[s] < 1) throw Error(DMRG_EINVAL, "bond dimension must be >= 1");
    const bool fwd = (s % 2) == 0;
    double emin = 1e300, dmax = 0.0;
    for (int k = 0; k < K - 1; ++k) {
      const int i = fwd ? k : K - 2 - k;
      auto clk = [] { return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count(); };
      const double t0 = clk();
      S.prob_site = -1;
      sweep_problem(c, i);
      Problem& p = *c.prob;
      const double t1 = clk();
      DevBuf x, guess;
      x.alloc(p.psi_size * sizeof(double));
      guess.alloc(p.psi_size * sizeof(double));
      double e = 0.0;
      int it = 0;
      const unsigned long long step_id = (unsigned long long)s * K + i;
      ensure_davidson_workspace(c, p);
      const bool have_guess = predict_guess(c, i, fwd, p, guess.as<double>());
      const bool conv = run_davidson(c, p, have_guess ? guess.as<double>() : nullptr, tol, &e, x.as<double>(), &it,
                                     step_id << 32);
      // the solver's psi (before any noise) seeds the next step's guess
      S.prev_x.alloc(p.psi_size * sizeof(double));
      DMRG_CUDA(cudaMemcpyAsync(S.prev_x.as<double>(), x.as<double>(), p.psi_size * sizeof(double),
                                cudaMemcpyDeviceToDevice, c.stream));
      S.prev_blocks = p.blocks;
      S.prev_EL = S.EL;
      S.prev_ER = S.ER;
      S.prev_site = i;
      S.prev_fwd = fwd;
      S.prev_size = p.psi_size;
      S.has_prev = true;
      if (c.opts.noise > 0.0) {
        // perturbative noise: decimate s x + noise z / |z|, renormalized, with
        // z seeded N(0,1) numbers of the noise stream and s = sign(x . z)
        // (the solver's sign of x is arbitrary)
        DevBuf z;
        z.alloc(p.psi_size * sizeof(double));
        launch_gen_vector(z.as<double>(), p.psi_size, (uint64_t)(c.opts.seed ^ KEY_NOISE), step_id << 32, c.stream);
        double* sc = p.dav_s.as<double>() + 50;
        double* part = p.dav_partial.as<double>();
        dav_dots(x.as<double>(), p.psi_size, 1, z.as<double>(), p.psi_size, part, sc, 1, c.stream);
        dav_dots(z.as<double>(), p.psi_size, 1, z.as<double>(), p.psi_size, part, sc + 1, 1, c.stream);
        dav_axpy_unit(x.as<double>(), z.as<double>(), sc, c.opts.noise, p.psi_size, c.stream);
        dav_dots(x.as<double>(), p.psi_size, 1, x.as<double>(), p.psi_size, part, sc + 2, 1, c.stream);
        dav_scale(x.as<double>(), sc + 2, p.psi_size, c.stream);
        DMRG_CUDA(cudaGetLastError());
      }
      emin = std::min(emin, e);
      const double t2 = clk();
      Decim D;
      decimate(c, p, fwd ? S.EL : S.ER, x.as<double>(), Ms[s], fwd, D);
      dmax = std::max(dmax, D.discarded);
      int kept = 0;
      for (int d : D.nb.dim) kept += d;
      const double t3 = clk();
      auto nbk = std::make_unique<DevBlock>();
      if (fwd) {
        transform(c, p.L, p.store.as<double>(), D.nb, D.esec_of_new, D.uoff, D.u.as<double>(), *nbk, 2 * (i + 1),
                  2 * K, true, S.prob_cn);
        nbk->u.take(D.u);
        nbk->uoff = D.uoff;
        nbk->esec = D.esec_of_new;
        S.L[i + 1] = std::move(nbk);
      } else {
        transform(c, p.R, p.store.as<double>(), D.nb, D.esec_of_new, D.uoff, D.u.as<double>(), *nbk, 2 * (i + 1),
                  2 * K, false, S.prob_cn);
        nbk->u.take(D.u);
        nbk->uoff = D.uoff;
        nbk->esec = D.esec_of_new;
        S.R[i + 1] = std::move(nbk);
      }
      const double t4 = clk();
      S.log.push_back({s, i, fwd ? 1 : 0, it, conv ? 1 : 0, kept, p.psi_size, e, D.discarded, t1 - t0, t2 - t1,
                       t3 - t2, t4 - t3});
      c.prob.reset();
      S.prob_site = -1;
    }
    if (energies) energies[s] = emin;
    if (max_discard) max_discard[s] = dmax;
  }
}

}  // namespace dmrg
